/*
 * Seeded synthetic inputs for block-sparse coupled-cluster-shaped tensors.
 *
 * This module is shared by the FP64 CPU oracle and by the GPU library's tests
 * and benchmark.  It holds no contraction arithmetic: it only draws numbers.
 *
 *   - Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11), written from the
 *     published round function: two 32x32->64 multiplies per round with the
 *     constants 0xD2511F53 / 0xCD9E8D57 and a Weyl key schedule with
 *     0x9E3779B9 / 0xBB67AE85, ten rounds.
 *   - Box-Muller transform of two 53-bit uniforms to one N(0,1) draw.
 *   - Antisymmetrisation of same-space mode pairs, defined per dense element
 *     so that any block can be regenerated on its own:
 *       both pairs:  ((X[pqrs] - X[qprs]) - (X[pqsr] - X[qpsr])) / 2
 *       one pair:    (X[pq..] - X[qp..]) / sqrt(2)
 *     which keeps the off-diagonal standard deviation at sigma and makes the
 *     diagonal (p == q) exactly zero.
 *   - Symmetrisation of the first two modes of a 3-mode tensor (pair code 2,
 *     for Cholesky vectors X[p,r,L] = X[r,p,L]):
 *       (X[prL] + X[rpL]) / sqrt(2)
 *     (off-diagonal standard deviation sigma, diagonal sqrt(2) sigma).
 *
 * Pair codes for modes (0,1): 0 plain, 1 antisymmetrised, 2 symmetrised.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static inline void philox_round(uint32_t c[4], const uint32_t k[2]) {
  uint64_t p0 = (uint64_t)PHILOX_M0 * c[0];
  uint64_t p1 = (uint64_t)PHILOX_M1 * c[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k[0];
  uint32_t n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

void tamm_synth_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k[0] += PHILOX_W0;
      k[1] += PHILOX_W1;
    }
    philox_round(c, k);
  }
  out[0] = c[0];
  out[1] = c[1];
  out[2] = c[2];
  out[3] = c[3];
}

/* One N(0,1) draw for element `index` of stream `stream` under `seed`. */
double tamm_synth_normal(uint64_t seed, uint32_t stream, uint64_t index) {
  uint32_t ctr[4] = {(uint32_t)index, (uint32_t)(index >> 32), stream, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t x[4];
  tamm_synth_philox4x32_10(ctr, key, x);
  const double two53 = 9007199254740992.0;
  double u1 = ((double)(((uint64_t)(x[0] >> 5) << 26) | (x[1] >> 6)) + 0.5) / two53;
  double u2 = ((double)(((uint64_t)(x[2] >> 5) << 26) | (x[3] >> 6)) + 0.5) / two53;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);
}

static inline uint64_t lin4(const int64_t* d, int64_t p, int64_t q, int64_t r, int64_t s) {
  return (uint64_t)(((p * d[1] + q) * d[2] + r) * d[3] + s);
}

/* Value of one element of a conceptually dense tensor with `ndim` <= 4 modes. */
double tamm_synth_value(uint64_t seed, uint32_t stream, double sigma, int ndim, const int64_t* dims,
                        int anti01, int anti23, const int64_t* idx) {
  int64_t d[4] = {1, 1, 1, 1};
  int64_t i[4] = {0, 0, 0, 0};
  /* Right-align so that lin4 covers 1..4 modes with the same formula. */
  for (int m = 0; m < ndim; ++m) {
    d[4 - ndim + m] = dims[m];
    i[4 - ndim + m] = idx[m];
  }
  int64_t p = i[0], q = i[1], r = i[2], s = i[3];
  double v;
  if (ndim == 4 && anti01 && anti23) {
    /* grouped so that swapping p<->q or r<->s flips the sign exactly in floating point */
    double d1 = tamm_synth_normal(seed, stream, lin4(d, p, q, r, s)) -
                tamm_synth_normal(seed, stream, lin4(d, q, p, r, s));
    double d2 = tamm_synth_normal(seed, stream, lin4(d, p, q, s, r)) -
                tamm_synth_normal(seed, stream, lin4(d, q, p, s, r));
    v = (d1 - d2) * 0.5;
  } else if (ndim == 4 && anti01) {
    v = (tamm_synth_normal(seed, stream, lin4(d, p, q, r, s)) -
         tamm_synth_normal(seed, stream, lin4(d, q, p, r, s))) * 0.70710678118654752440;
  } else if (ndim == 4 && anti23) {
    v = (tamm_synth_normal(seed, stream, lin4(d, p, q, r, s)) -
         tamm_synth_normal(seed, stream, lin4(d, p, q, s, r))) * 0.70710678118654752440;
  } else if (ndim == 3 && anti01 == 2) {
    v = (tamm_synth_normal(seed, stream, lin4(d, 0, q, r, s)) +
         tamm_synth_normal(seed, stream, lin4(d, 0, r, q, s))) * 0.70710678118654752440;
  } else if (ndim == 2 && anti01) {
    v = (tamm_synth_normal(seed, stream, lin4(d, 0, 0, r, s)) -
         tamm_synth_normal(seed, stream, lin4(d, 0, 0, s, r))) * 0.70710678118654752440;
  } else {
    v = tamm_synth_normal(seed, stream, lin4(d, p, q, r, s));
  }
  return sigma * v;
}

/*
 * Fill many boxes (blocks) of a dense tensor.  Box b has its lower corner at
 * lo[b*ndim ...], extents ext[b*ndim ...], and is written row-major (last mode
 * fastest) to out + off[b].
 */
void tamm_synth_fill_boxes(uint64_t seed, uint32_t stream, double sigma, int ndim, const int64_t* dims,
                           int anti01, int anti23, int64_t nbox, const int64_t* lo, const int64_t* ext,
                           const int64_t* off, double* out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t b = 0; b < nbox; ++b) {
    const int64_t* L = lo + b * ndim;
    const int64_t* E = ext + b * ndim;
    int64_t n = 1;
    for (int m = 0; m < ndim; ++m) n *= E[m];
    double* o = out + off[b];
    for (int64_t e = 0; e < n; ++e) {
      int64_t idx[4];
      int64_t rem = e;
      for (int m = ndim - 1; m >= 0; --m) {
        idx[m] = L[m] + rem % E[m];
        rem /= E[m];
      }
      o[e] = tamm_synth_value(seed, stream, sigma, ndim, dims, anti01, anti23, idx);
    }
  }
}
