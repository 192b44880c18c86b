/*
 * FP64 CPU oracle for block-sparse tensor contractions (TAMM, arXiv:2201.01257).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code with the GPU library: index spaces, tiling, the nonzero-block rule and
 * the contraction loops are written here from the paper's definitions, in the
 * plainest form that can be checked by eye.
 *
 *   - Index spaces and tilings (Sec. III.A, Fig. "tensor_const"): a space is a
 *     range of orbitals made of contiguous groups; a tiled space cuts every
 *     group into tiles of a fixed size (last tile of a group takes the
 *     remainder) or into an explicit list of sizes covering every group.
 *   - Block sparsity (Sec. III.A, spin attributes; Sec. III.B, sparsity-aware
 *     allocation): a block, i.e. a tuple of tiles one per mode, is stored only
 *     when the sum of the spins of the upper modes equals that of the lower
 *     modes, and, for the irrep rule, when the product (XOR in D2h) of the tile
 *     irreps is the totally symmetric irrep 0.  Stored blocks are laid out one
 *     after another in lexicographic tile order, each row-major over the
 *     tensor's modes in declared order.
 *   - Operations (Sec. III.A, grammar figure "tensor_ops"):
 *       C(lc) = beta*C + alpha * A(la) * B(lb)   (MultOp, Einstein summation
 *                                                over labels in A and B only)
 *       C(lc) = beta*C + alpha * A(la)           (AddOp with label permutation)
 *       E     = alpha * sum A(la) * B(lb)        (full contraction to a scalar)
 *       ||T||  Frobenius norm over stored entries (utility norm)
 *   - Cholesky-built two-electron tensor (Eq. cc12): V[p,q,r,s] from the
 *     Cholesky vectors X[p,r,L], for the on-the-fly ("lambda") tensor.
 *     beta is 0 for "=" and 1 for "+=" ("-=" is a negative alpha).
 *
 * Summation order is fixed: contracted tile tuples in lexicographic order
 * (first contracted label slowest), then contracted elements in row-major
 * order, so every result is deterministic.  OpenMP runs over output blocks.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_MAX_MODES 8
#define OR_MAX_LABELS 16

enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOMEM = -2 };
enum { OR_SYM_DENSE = 0, OR_SYM_SPIN = 1, OR_SYM_SPIN_IRREP = 2 };

typedef struct {
  int n_tiles;
  int64_t n;
  int64_t* off;
  int64_t* size;
  int* spin;
  int* irrep;
} ospace;

typedef struct {
  int nm, n_upper, sym;
  const ospace* sp[OR_MAX_MODES];
  int64_t n_blocks;
  int64_t* tiles;  /* n_blocks * nm tile indices */
  int64_t* off;    /* n_blocks element offsets */
  int64_t* lookup; /* dense tile-tuple index -> block index or -1 */
  int64_t n_tuples;
  int64_t n_elems;
} otensor;

/* ------------------------------------------------------------------ spaces */

ospace* oracle_space_create(int n_groups, const int64_t* gsize, const int* gspin, const int* girrep,
                            int64_t fixed_tile, int n_tiles_in, const int64_t* tile_sizes) {
  if (n_groups <= 0) return NULL;
  int cap = 0;
  if (fixed_tile > 0) {
    for (int g = 0; g < n_groups; ++g) {
      if (gsize[g] < 0) return NULL;
      cap += (int)((gsize[g] + fixed_tile - 1) / fixed_tile);
    }
  } else {
    if (n_tiles_in <= 0 || !tile_sizes) return NULL;
    cap = n_tiles_in;
  }
  ospace* s = (ospace*)calloc(1, sizeof(ospace));
  s->off = (int64_t*)calloc(cap > 0 ? cap : 1, sizeof(int64_t));
  s->size = (int64_t*)calloc(cap > 0 ? cap : 1, sizeof(int64_t));
  s->spin = (int*)calloc(cap > 0 ? cap : 1, sizeof(int));
  s->irrep = (int*)calloc(cap > 0 ? cap : 1, sizeof(int));
  int t = 0;
  int64_t pos = 0;
  for (int g = 0; g < n_groups; ++g) {
    int64_t left = gsize[g];
    while (left > 0) {
      int64_t ts;
      if (fixed_tile > 0) {
        ts = left < fixed_tile ? left : fixed_tile;
      } else {
        if (t >= n_tiles_in || tile_sizes[t] <= 0 || tile_sizes[t] > left) goto bad; /* straddles a group */
        ts = tile_sizes[t];
      }
      s->off[t] = pos;
      s->size[t] = ts;
      s->spin[t] = gspin[g];
      s->irrep[t] = girrep ? girrep[g] : 0;
      pos += ts;
      left -= ts;
      ++t;
    }
  }
  if (fixed_tile <= 0 && t != n_tiles_in) goto bad;
  s->n_tiles = t;
  s->n = pos;
  return s;
bad:
  free(s->off);
  free(s->size);
  free(s->spin);
  free(s->irrep);
  free(s);
  return NULL;
}

void oracle_space_destroy(ospace* s) {
  if (!s) return;
  free(s->off);
  free(s->size);
  free(s->spin);
  free(s->irrep);
  free(s);
}

int oracle_space_ntiles(const ospace* s) { return s->n_tiles; }
int64_t oracle_space_size(const ospace* s) { return s->n; }

void oracle_space_tile(const ospace* s, int t, int64_t* off, int64_t* size, int* spin, int* irrep) {
  *off = s->off[t];
  *size = s->size[t];
  *spin = s->spin[t];
  *irrep = s->irrep[t];
}

/* ----------------------------------------------------------------- tensors */

static int block_allowed(const otensor* T, const int64_t* tt) {
  if (T->sym == OR_SYM_DENSE) return 1;
  int up = 0, lo = 0, x = 0;
  for (int m = 0; m < T->nm; ++m) {
    int sp = T->sp[m]->spin[tt[m]];
    if (m < T->n_upper) up += sp; else lo += sp;
    x ^= T->sp[m]->irrep[tt[m]];
  }
  if (up != lo) return 0;
  if (T->sym == OR_SYM_SPIN_IRREP && x != 0) return 0;
  return 1;
}

otensor* oracle_tensor_create(int nm, const ospace* const* sp, int n_upper, int sym) {
  if (nm <= 0 || nm > OR_MAX_MODES || n_upper < 0 || n_upper > nm) return NULL;
  if (sym < OR_SYM_DENSE || sym > OR_SYM_SPIN_IRREP) return NULL;
  otensor* T = (otensor*)calloc(1, sizeof(otensor));
  T->nm = nm;
  T->n_upper = n_upper;
  T->sym = sym;
  int64_t nt = 1;
  for (int m = 0; m < nm; ++m) {
    T->sp[m] = sp[m];
    nt *= sp[m]->n_tiles;
  }
  T->n_tuples = nt;
  T->lookup = (int64_t*)malloc(sizeof(int64_t) * (size_t)nt);
  int64_t nb = 0;
  int64_t tt[OR_MAX_MODES];
  for (int64_t lin = 0; lin < nt; ++lin) {
    int64_t r = lin;
    for (int m = nm - 1; m >= 0; --m) {
      tt[m] = r % sp[m]->n_tiles;
      r /= sp[m]->n_tiles;
    }
    T->lookup[lin] = block_allowed(T, tt) ? nb++ : -1;
  }
  T->n_blocks = nb;
  T->tiles = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nb * nm + 1));
  T->off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nb + 1));
  int64_t pos = 0;
  for (int64_t lin = 0; lin < nt; ++lin) {
    int64_t b = T->lookup[lin];
    if (b < 0) continue;
    int64_t r = lin, sz = 1;
    for (int m = nm - 1; m >= 0; --m) {
      tt[m] = r % sp[m]->n_tiles;
      r /= sp[m]->n_tiles;
    }
    for (int m = 0; m < nm; ++m) {
      T->tiles[b * nm + m] = tt[m];
      sz *= sp[m]->size[tt[m]];
    }
    T->off[b] = pos;
    pos += sz;
  }
  T->off[nb] = pos;
  T->n_elems = pos;
  return T;
}

void oracle_tensor_destroy(otensor* T) {
  if (!T) return;
  free(T->lookup);
  free(T->tiles);
  free(T->off);
  free(T);
}

int64_t oracle_tensor_nblocks(const otensor* T) { return T->n_blocks; }
int64_t oracle_tensor_nelems(const otensor* T) { return T->n_elems; }

void oracle_tensor_blocks(const otensor* T, int64_t* tiles, int64_t* off) {
  memcpy(tiles, T->tiles, sizeof(int64_t) * (size_t)(T->n_blocks * T->nm));
  memcpy(off, T->off, sizeof(int64_t) * (size_t)T->n_blocks);
}

/* Block index for a tile tuple, or -1 when the block is not stored. */
static int64_t find_block(const otensor* T, const int64_t* tt) {
  int64_t lin = 0;
  for (int m = 0; m < T->nm; ++m) lin = lin * T->sp[m]->n_tiles + tt[m];
  return T->lookup[lin];
}

int64_t oracle_tensor_find_block(const otensor* T, const int64_t* tt) { return find_block(T, tt); }

/* ------------------------------------------------------------------ labels */

typedef struct {
  int n;                      /* distinct labels */
  char name[OR_MAX_LABELS];
  const ospace* sp[OR_MAX_LABELS];
  int posC[OR_MAX_LABELS], posA[OR_MAX_LABELS], posB[OR_MAX_LABELS]; /* mode position or -1 */
} labelset;

static int label_id(labelset* L, char c) {
  for (int i = 0; i < L->n; ++i)
    if (L->name[i] == c) return i;
  if (L->n >= OR_MAX_LABELS) return -1;
  L->name[L->n] = c;
  L->sp[L->n] = NULL;
  L->posC[L->n] = L->posA[L->n] = L->posB[L->n] = -1;
  return L->n++;
}

/* Register the labels of one tensor; `which` selects the position array. */
static int add_labels(labelset* L, const otensor* T, const char* l, int which) {
  if (!T || !l || (int)strlen(l) != T->nm) return OR_EINVAL;
  for (int m = 0; m < T->nm; ++m) {
    int id = label_id(L, l[m]);
    if (id < 0) return OR_EINVAL;
    int* pos = which == 0 ? L->posC : (which == 1 ? L->posA : L->posB);
    if (pos[id] >= 0) return OR_EINVAL; /* a label twice in one tensor */
    pos[id] = m;
    if (L->sp[id] && L->sp[id] != T->sp[m]) return OR_EINVAL; /* label bound to two spaces */
    L->sp[id] = T->sp[m];
  }
  return OR_OK;
}

/* ---------------------------------------------------------------- contract */

static void strides_of(const otensor* T, const int64_t* tt, int64_t* st) {
  int64_t s = 1;
  for (int m = T->nm - 1; m >= 0; --m) {
    st[m] = s;
    s *= T->sp[m]->size[tt[m]];
  }
}

typedef struct {
  labelset L;
  int nk;               /* contracted labels, in order of appearance in A */
  int k_ids[OR_MAX_LABELS];
} cplan;

static int contract_plan(cplan* P, const otensor* C, const char* lc, const otensor* A, const char* la,
                         const otensor* B, const char* lb) {
  memset(P, 0, sizeof(*P));
  if (add_labels(&P->L, C, lc, 0) || add_labels(&P->L, A, la, 1) || add_labels(&P->L, B, lb, 2))
    return OR_EINVAL;
  for (int i = 0; i < P->L.n; ++i) {
    int c = P->L.posC[i] >= 0, a = P->L.posA[i] >= 0, b = P->L.posB[i] >= 0;
    if (c && (a == b)) return OR_EINVAL;   /* output label in both inputs or in none */
    if (!c && !(a && b)) return OR_EINVAL; /* summed label must be in both inputs */
  }
  for (int m = 0; m < A->nm; ++m) {
    int id = label_id(&P->L, la[m]);
    if (P->L.posC[id] < 0) P->k_ids[P->nk++] = id;
  }
  return OR_OK;
}

/* Compute the box [lo, lo+ext) of stored C block `cb` into out (row-major over the box). */
static int contract_box(const cplan* P, double alpha, const otensor* C, double beta, const otensor* A,
                        const otensor* B, const double* a, const double* b, int64_t cb, const int64_t* lo,
                        const int64_t* ext, const double* c_in, double* out) {
  const labelset* L = &P->L;
  int64_t tile[OR_MAX_LABELS];
  const int64_t* ct = C->tiles + cb * C->nm;
  int64_t box_n = 1;
  for (int m = 0; m < C->nm; ++m) {
    if (lo[m] < 0 || ext[m] < 0 || lo[m] + ext[m] > C->sp[m]->size[ct[m]]) return OR_EINVAL;
    box_n *= ext[m];
  }
  int cid[OR_MAX_MODES]; /* label id of each C mode */
  for (int i = 0; i < L->n; ++i) tile[i] = -1;
  for (int i = 0; i < L->n; ++i)
    if (L->posC[i] >= 0) {
      tile[i] = ct[L->posC[i]];
      cid[L->posC[i]] = i;
    }

  double* acc = (double*)calloc((size_t)(box_n > 0 ? box_n : 1), sizeof(double));
  if (!acc) return OR_ENOMEM;

  int64_t nkt = 1;
  for (int k = 0; k < P->nk; ++k) nkt *= L->sp[P->k_ids[k]]->n_tiles;

  for (int64_t kt = 0; kt < nkt; ++kt) {
    int64_t r = kt;
    for (int k = P->nk - 1; k >= 0; --k) {
      int id = P->k_ids[k];
      tile[id] = r % L->sp[id]->n_tiles;
      r /= L->sp[id]->n_tiles;
    }
    int64_t at[OR_MAX_MODES], bt[OR_MAX_MODES];
    for (int i = 0; i < L->n; ++i) {
      if (L->posA[i] >= 0) at[L->posA[i]] = tile[i];
      if (L->posB[i] >= 0) bt[L->posB[i]] = tile[i];
    }
    int64_t ab = find_block(A, at), bb = find_block(B, bt);
    if (ab < 0 || bb < 0) continue;
    int64_t sa[OR_MAX_MODES], sb[OR_MAX_MODES];
    strides_of(A, at, sa);
    strides_of(B, bt, sb);
    /* per-label strides into A and B, and contracted extents */
    int64_t strA[OR_MAX_LABELS], strB[OR_MAX_LABELS];
    for (int i = 0; i < L->n; ++i) {
      strA[i] = L->posA[i] >= 0 ? sa[L->posA[i]] : 0;
      strB[i] = L->posB[i] >= 0 ? sb[L->posB[i]] : 0;
    }
    int64_t kext[OR_MAX_LABELS];
    int64_t kn = 1;
    for (int k = 0; k < P->nk; ++k) {
      kext[k] = L->sp[P->k_ids[k]]->size[tile[P->k_ids[k]]];
      kn *= kext[k];
    }
    /* offsets of every contracted element (row-major over the contracted labels) in A and B */
    int64_t* kofs = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * kn + 2));
    if (!kofs) {
      free(acc);
      return OR_ENOMEM;
    }
    for (int64_t k = 0; k < kn; ++k) {
      int64_t rk = k, ka = 0, kb = 0;
      for (int q = P->nk - 1; q >= 0; --q) {
        int64_t x = rk % kext[q];
        rk /= kext[q];
        ka += x * strA[P->k_ids[q]];
        kb += x * strB[P->k_ids[q]];
      }
      kofs[2 * k] = ka;
      kofs[2 * k + 1] = kb;
    }
    const double* ablk = a + A->off[ab];
    const double* bblk = b + B->off[bb];
    int64_t cidx[OR_MAX_MODES];
    for (int64_t e = 0; e < box_n; ++e) {
      int64_t rr = e;
      for (int m = C->nm - 1; m >= 0; --m) {
        cidx[m] = lo[m] + rr % ext[m];
        rr /= ext[m];
      }
      int64_t abase = 0, bbase = 0;
      for (int m = 0; m < C->nm; ++m) {
        abase += cidx[m] * strA[cid[m]];
        bbase += cidx[m] * strB[cid[m]];
      }
      double s = acc[e];
      for (int64_t k = 0; k < kn; ++k) s += ablk[abase + kofs[2 * k]] * bblk[bbase + kofs[2 * k + 1]];
      acc[e] = s;
    }
    free(kofs);
  }
  for (int64_t e = 0; e < box_n; ++e) {
    double prev = (beta != 0.0 && c_in) ? beta * c_in[e] : 0.0;
    out[e] = prev + alpha * acc[e];
  }
  free(acc);
  return OR_OK;
}

/* Full contraction over every stored block of C (in place on c). */
int oracle_contract(double alpha, const otensor* C, const char* lc, double beta, const otensor* A,
                    const char* la, const otensor* B, const char* lb, double* c, const double* a,
                    const double* b) {
  cplan P;
  if (contract_plan(&P, C, lc, A, la, B, lb)) return OR_EINVAL;
  int err = OR_OK;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t cb = 0; cb < C->n_blocks; ++cb) {
    int64_t lo[OR_MAX_MODES], ext[OR_MAX_MODES];
    const int64_t* ct = C->tiles + cb * C->nm;
    for (int m = 0; m < C->nm; ++m) {
      lo[m] = 0;
      ext[m] = C->sp[m]->size[ct[m]];
    }
    double* cblk = c + C->off[cb];
    int e = contract_box(&P, alpha, C, beta, A, B, a, b, cb, lo, ext, cblk, cblk);
    if (e) {
#pragma omp atomic write
      err = e;
    }
  }
  return err;
}

/* Like oracle_contract, restricted to the listed stored C blocks (others untouched). */
int oracle_contract_blocks(double alpha, const otensor* C, const char* lc, double beta, const otensor* A,
                           const char* la, const otensor* B, const char* lb, double* c, const double* a,
                           const double* b, const int64_t* blocks, int64_t n_blocks) {
  cplan P;
  if (contract_plan(&P, C, lc, A, la, B, lb)) return OR_EINVAL;
  for (int64_t i = 0; i < n_blocks; ++i)
    if (blocks[i] < 0 || blocks[i] >= C->n_blocks) return OR_EINVAL;
  int err = OR_OK;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n_blocks; ++i) {
    const int64_t cb = blocks[i];
    int64_t lo[OR_MAX_MODES], ext[OR_MAX_MODES];
    const int64_t* ct = C->tiles + cb * C->nm;
    for (int m = 0; m < C->nm; ++m) {
      lo[m] = 0;
      ext[m] = C->sp[m]->size[ct[m]];
    }
    double* cblk = c + C->off[cb];
    int e = contract_box(&P, alpha, C, beta, A, B, a, b, cb, lo, ext, cblk, cblk);
    if (e) {
#pragma omp atomic write
      err = e;
    }
  }
  return err;
}

/* One box of one C block; c_box_in holds the box's current C values (ignored when beta == 0). */
int oracle_contract_box(double alpha, const otensor* C, const char* lc, double beta, const otensor* A,
                        const char* la, const otensor* B, const char* lb, const double* a, const double* b,
                        int64_t cb, const int64_t* lo, const int64_t* ext, const double* c_box_in,
                        double* out) {
  cplan P;
  if (contract_plan(&P, C, lc, A, la, B, lb)) return OR_EINVAL;
  if (cb < 0 || cb >= C->n_blocks) return OR_EINVAL;
  return contract_box(&P, alpha, C, beta, A, B, a, b, cb, lo, ext, c_box_in, out);
}

/* Many boxes at once (OpenMP over boxes): box i is [lo[i], lo[i]+ext[i]) of C
 * block cblocks[i], written row-major at out + out_off[i] (beta taken as 0). */
int oracle_contract_boxes(double alpha, const otensor* C, const char* lc, const otensor* A, const char* la,
                          const otensor* B, const char* lb, const double* a, const double* b, int64_t n_boxes,
                          const int64_t* cblocks, const int64_t* lo, const int64_t* ext, const int64_t* out_off,
                          double* out) {
  cplan P;
  if (contract_plan(&P, C, lc, A, la, B, lb)) return OR_EINVAL;
  int err = OR_OK;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n_boxes; ++i) {
    int e = OR_EINVAL;
    if (cblocks[i] >= 0 && cblocks[i] < C->n_blocks)
      e = contract_box(&P, alpha, C, 0.0, A, B, a, b, cblocks[i], lo + i * C->nm, ext + i * C->nm, NULL,
                       out + out_off[i]);
    if (e) {
#pragma omp atomic write
      err = e;
    }
  }
  return err;
}

/* --------------------------------------------------------------------- add */

int oracle_add(double alpha, const otensor* C, const char* lc, double beta, const otensor* A, const char* la,
               double* c, const double* a) {
  labelset L;
  memset(&L, 0, sizeof(L));
  if (add_labels(&L, C, lc, 0) || add_labels(&L, A, la, 1)) return OR_EINVAL;
  for (int i = 0; i < L.n; ++i)
    if ((L.posC[i] >= 0) != (L.posA[i] >= 0)) return OR_EINVAL;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t cb = 0; cb < C->n_blocks; ++cb) {
    const int64_t* ct = C->tiles + cb * C->nm;
    int64_t at[OR_MAX_MODES], sa[OR_MAX_MODES], perm[OR_MAX_MODES];
    for (int m = 0; m < C->nm; ++m) {
      int id = -1;
      for (int i = 0; i < L.n; ++i)
        if (L.posC[i] == m) id = i;
      perm[m] = L.posA[id]; /* A mode holding C mode m's label */
      at[L.posA[id]] = ct[m];
    }
    int64_t ab = find_block(A, at);
    double* cblk = c + C->off[cb];
    int64_t n = C->off[cb + 1] - C->off[cb];
    if (ab < 0) {
      for (int64_t e = 0; e < n; ++e) cblk[e] = beta != 0.0 ? beta * cblk[e] : 0.0;
      continue;
    }
    strides_of(A, at, sa);
    const double* ablk = a + A->off[ab];
    for (int64_t e = 0; e < n; ++e) {
      int64_t r = e, ai = 0;
      for (int m = C->nm - 1; m >= 0; --m) {
        int64_t x = r % C->sp[m]->size[ct[m]];
        r /= C->sp[m]->size[ct[m]];
        ai += x * sa[perm[m]];
      }
      double prev = beta != 0.0 ? beta * cblk[e] : 0.0;
      cblk[e] = prev + alpha * ablk[ai];
    }
  }
  return OR_OK;
}

/* ------------------------------------------------------------------ energy */

int oracle_energy(double alpha, const otensor* A, const char* la, const otensor* B, const char* lb,
                  const double* a, const double* b, double* result) {
  labelset L;
  memset(&L, 0, sizeof(L));
  if (add_labels(&L, A, la, 1) || add_labels(&L, B, lb, 2)) return OR_EINVAL;
  for (int i = 0; i < L.n; ++i)
    if ((L.posA[i] >= 0) != (L.posB[i] >= 0)) return OR_EINVAL;
  double* part = (double*)calloc((size_t)(A->n_blocks + 1), sizeof(double));
  if (!part) return OR_ENOMEM;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t ab = 0; ab < A->n_blocks; ++ab) {
    const int64_t* at = A->tiles + ab * A->nm;
    int64_t bt[OR_MAX_MODES], sb[OR_MAX_MODES], perm[OR_MAX_MODES];
    for (int m = 0; m < A->nm; ++m) {
      int id = -1;
      for (int i = 0; i < L.n; ++i)
        if (L.posA[i] == m) id = i;
      perm[m] = L.posB[id];
      bt[L.posB[id]] = at[m];
    }
    int64_t bb = find_block(B, bt);
    if (bb < 0) continue;
    strides_of(B, bt, sb);
    const double* ablk = a + A->off[ab];
    const double* bblk = b + B->off[bb];
    int64_t n = A->off[ab + 1] - A->off[ab];
    double s = 0.0;
    for (int64_t e = 0; e < n; ++e) {
      int64_t r = e, bi = 0;
      for (int m = A->nm - 1; m >= 0; --m) {
        int64_t x = r % A->sp[m]->size[at[m]];
        r /= A->sp[m]->size[at[m]];
        bi += x * sb[perm[m]];
      }
      s += ablk[e] * bblk[bi];
    }
    part[ab] = s;
  }
  double s = 0.0;
  for (int64_t ab = 0; ab < A->n_blocks; ++ab) s += part[ab];
  free(part);
  *result = alpha * s;
  return OR_OK;
}

/* -------------------------------------------------------------------- norm */

double oracle_norm(const otensor* T, const double* x) {
  double s = 0.0;
  for (int64_t e = 0; e < T->n_elems; ++e) s += x[e] * x[e];
  return sqrt(s);
}

/* ---------------------------------------------------- Cholesky-built tensor */

/*
 * Two-electron tensor from Cholesky vectors (Eq. cc12; the "lambda tensor" of
 * Sec. III.A is a tensor whose blocks are computed on demand like this):
 *
 *   V[p,q,r,s] = sum_L ( X[p,r,L] * X[q,s,L] - X[p,s,L] * X[q,r,L] )
 *
 * X has modes (P, R, aux) and V modes (P, P, R, R).  An entry of X in a block
 * that X does not store is zero.  Fills the listed stored blocks of V (every
 * block when `blocks` is NULL).  Summation order: aux tiles in order, then L
 * inside the tile; each L contributes one product difference.
 */
int oracle_cholesky_v(const otensor* V, const otensor* X, const double* x, double* v, const int64_t* blocks,
                      int64_t n_list) {
  if (!V || !X || V->nm != 4 || X->nm != 3) return OR_EINVAL;
  if (V->sp[0] != X->sp[0] || V->sp[1] != X->sp[0] || V->sp[2] != X->sp[1] || V->sp[3] != X->sp[1])
    return OR_EINVAL;
  const ospace* aux = X->sp[2];
  const int64_t n = blocks ? n_list : V->n_blocks;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n; ++i) {
    const int64_t b = blocks ? blocks[i] : i;
    if (b < 0 || b >= V->n_blocks) continue;
    const int64_t* t = V->tiles + b * 4;
    const int64_t tp = t[0], tq = t[1], tr = t[2], ts = t[3];
    const int64_t np = V->sp[0]->size[tp], nq = V->sp[1]->size[tq];
    const int64_t nr = V->sp[2]->size[tr], ns = V->sp[3]->size[ts];
    double* out = v + V->off[b];
    for (int64_t ip = 0; ip < np; ++ip)
      for (int64_t iq = 0; iq < nq; ++iq)
        for (int64_t ir = 0; ir < nr; ++ir)
          for (int64_t is = 0; is < ns; ++is) {
            double acc = 0.0;
            for (int tl = 0; tl < aux->n_tiles; ++tl) {
              const int64_t nl = aux->size[tl];
              int64_t k_pr[3] = {tp, tr, tl}, k_qs[3] = {tq, ts, tl};
              int64_t k_ps[3] = {tp, ts, tl}, k_qr[3] = {tq, tr, tl};
              const int64_t b_pr = find_block(X, k_pr), b_qs = find_block(X, k_qs);
              const int64_t b_ps = find_block(X, k_ps), b_qr = find_block(X, k_qr);
              for (int64_t l = 0; l < nl; ++l) {
                /* X block (tile a, tile c, tl) is row-major: element (ia, ic, l) at (ia*nc + ic)*nl + l */
                const double x_pr = b_pr >= 0 ? x[X->off[b_pr] + (ip * nr + ir) * nl + l] : 0.0;
                const double x_qs = b_qs >= 0 ? x[X->off[b_qs] + (iq * ns + is) * nl + l] : 0.0;
                const double x_ps = b_ps >= 0 ? x[X->off[b_ps] + (ip * ns + is) * nl + l] : 0.0;
                const double x_qr = b_qr >= 0 ? x[X->off[b_qr] + (iq * nr + ir) * nl + l] : 0.0;
                acc += x_pr * x_qs - x_ps * x_qr;
              }
            }
            out[((ip * nq + iq) * nr + ir) * ns + is] = acc;
          }
  }
  return OR_OK;
}

/* --------------------------------------------------- (T) triples correction */

/*
 * Perturbative triples correction of CCSD(T) (Sec. IV.B, Eqs. cc14, tensort,
 * tensort2), for real amplitudes:
 *
 *   E(T) = sum_{i<j<k} sum_{a<b<c} (W + Y) * W / D,
 *   D    = e_i + e_j + e_k - e_a - e_b - e_c,
 *
 * where W = <Phi_ijk^abc| V_N T2 |Phi> is the eighteen-term sum of Eq. tensort
 * (nine terms summed over an occupied m, nine over a virtual e) and
 * Y = <Phi_ijk^abc| V_N T1 |Phi> the nine products of Eq. tensort2.  For real
 * amplitudes the bra factors <Phi|T2^+ V_N|Phi_ijk^abc> and <Phi|T1^+ V_N|...>
 * equal W and Y.  Tensor conventions (upper indices first, as in the paper's
 * v^{pq}_{rs} and t^{ij}_{ab}):
 *   v^{ij}_{ma} = Vooov[i,j,m,a]   v^{ei}_{ab} = Vvovv[e,i,a,b]
 *   v^{ij}_{ab} = Voovv[i,j,a,b]   t^{ij}_{ab} = T2[a,b,i,j]   t^i_a = T1[a,i]
 * An entry of a block the tensor does not store is zero.
 *
 * Reading: the sixth term of Eq. tensort is printed as +v^{ik}_{mc} t^{mj}_{ab};
 * W must change sign under the exchange of j and k (it is an amplitude of the
 * antisymmetric determinant Phi_ijk^abc), which the other seventeen terms
 * respect and which fixes that term's sign to minus.  It is taken with a minus.
 */

/* Dense copy of a block-sparse tensor (zeros where no block is stored). */
static double* dense_copy(const otensor* X, const double* x) {
  int64_t n = 1, dims[OR_MAX_MODES];
  for (int m = 0; m < X->nm; ++m) {
    dims[m] = X->sp[m]->n;
    n *= dims[m];
  }
  double* d = (double*)calloc((size_t)n, sizeof(double));
  if (!d) return NULL;
  for (int64_t b = 0; b < X->n_blocks; ++b) {
    const int64_t* tt = X->tiles + b * X->nm;
    int64_t ext[OR_MAX_MODES], lo[OR_MAX_MODES], bn = 1;
    for (int m = 0; m < X->nm; ++m) {
      ext[m] = X->sp[m]->size[tt[m]];
      lo[m] = X->sp[m]->off[tt[m]];
      bn *= ext[m];
    }
    for (int64_t e = 0; e < bn; ++e) {
      int64_t r = e, di = 0, idx[OR_MAX_MODES];
      for (int m = X->nm - 1; m >= 0; --m) {
        idx[m] = r % ext[m];
        r /= ext[m];
      }
      for (int m = 0; m < X->nm; ++m) di = di * dims[m] + lo[m] + idx[m];
      d[di] = x[X->off[b] + e];
    }
  }
  return d;
}

typedef struct {
  int64_t no, nv;
  double *t2, *t1, *vo, *vv, *voo; /* dense T2[v,v,o,o], T1[v,o], Vooov, Vvovv, Voovv */
} triples_in;

#define T2_(a, b, i, j) in->t2[(((a) * nv + (b)) * no + (i)) * no + (j)]
#define T1_(a, i) in->t1[(a) * no + (i)]
#define VO_(i, j, m, a) in->vo[(((i) * no + (j)) * no + (m)) * nv + (a)]
#define VV_(e, i, a, b) in->vv[(((e) * no + (i)) * nv + (a)) * nv + (b)]
#define VOO_(i, j, a, b) in->voo[(((i) * no + (j)) * nv + (a)) * nv + (b)]

/* W of Eq. tensort for one (i,j,k,a,b,c), any index order. */
static double triples_w(const triples_in* in, int64_t i, int64_t j, int64_t k, int64_t a, int64_t b, int64_t c) {
  const int64_t no = in->no, nv = in->nv;
  double s = 0.0;
  for (int64_t m = 0; m < no; ++m) { /* A: contractions over the occupied index m */
    s += VO_(i, j, m, a) * T2_(b, c, m, k);
    s -= VO_(i, j, m, b) * T2_(a, c, m, k);
    s += VO_(i, j, m, c) * T2_(a, b, m, k);
    s -= VO_(i, k, m, a) * T2_(b, c, m, j);
    s += VO_(i, k, m, b) * T2_(a, c, m, j);
    s -= VO_(i, k, m, c) * T2_(a, b, m, j);
    s += VO_(j, k, m, a) * T2_(b, c, m, i);
    s -= VO_(j, k, m, b) * T2_(a, c, m, i);
    s += VO_(j, k, m, c) * T2_(a, b, m, i);
  }
  for (int64_t e = 0; e < nv; ++e) { /* B: contractions over the virtual index e */
    s -= VV_(e, i, a, b) * T2_(e, c, j, k);
    s += VV_(e, i, a, c) * T2_(e, b, j, k);
    s -= VV_(e, i, b, c) * T2_(e, a, j, k);
    s += VV_(e, j, a, b) * T2_(e, c, i, k);
    s -= VV_(e, j, a, c) * T2_(e, b, i, k);
    s += VV_(e, j, b, c) * T2_(e, a, i, k);
    s -= VV_(e, k, a, b) * T2_(e, c, i, j);
    s += VV_(e, k, a, c) * T2_(e, b, i, j);
    s -= VV_(e, k, b, c) * T2_(e, a, i, j);
  }
  return s;
}

/* Y of Eq. tensort2 for one (i,j,k,a,b,c). */
static double triples_y(const triples_in* in, int64_t i, int64_t j, int64_t k, int64_t a, int64_t b, int64_t c) {
  const int64_t no = in->no, nv = in->nv;
  return VOO_(i, j, a, b) * T1_(c, k) - VOO_(i, j, a, c) * T1_(b, k) + VOO_(i, j, b, c) * T1_(a, k) -
         VOO_(i, k, a, b) * T1_(c, j) + VOO_(i, k, a, c) * T1_(b, j) - VOO_(i, k, b, c) * T1_(a, j) +
         VOO_(j, k, a, b) * T1_(c, i) - VOO_(j, k, a, c) * T1_(b, i) + VOO_(j, k, b, c) * T1_(a, i);
}

#undef T2_
#undef T1_
#undef VO_
#undef VV_
#undef VOO_

static int triples_load(triples_in* in, const otensor* T2, const double* t2, const otensor* T1, const double* t1,
                        const otensor* Vo, const double* vo, const otensor* Vv, const double* vv, const otensor* Voo,
                        const double* voo) {
  memset(in, 0, sizeof(*in));
  if (!T2 || !T1 || !Vo || !Vv || !Voo || T2->nm != 4 || T1->nm != 2 || Vo->nm != 4 || Vv->nm != 4 || Voo->nm != 4)
    return OR_EINVAL;
  const ospace* O = T2->sp[2];
  const ospace* V = T2->sp[0];
  if (T2->sp[1] != V || T2->sp[3] != O || T1->sp[0] != V || T1->sp[1] != O) return OR_EINVAL;
  if (Vo->sp[0] != O || Vo->sp[1] != O || Vo->sp[2] != O || Vo->sp[3] != V) return OR_EINVAL;
  if (Vv->sp[0] != V || Vv->sp[1] != O || Vv->sp[2] != V || Vv->sp[3] != V) return OR_EINVAL;
  if (Voo->sp[0] != O || Voo->sp[1] != O || Voo->sp[2] != V || Voo->sp[3] != V) return OR_EINVAL;
  in->no = O->n;
  in->nv = V->n;
  in->t2 = dense_copy(T2, t2);
  in->t1 = dense_copy(T1, t1);
  in->vo = dense_copy(Vo, vo);
  in->vv = dense_copy(Vv, vv);
  in->voo = dense_copy(Voo, voo);
  if (!in->t2 || !in->t1 || !in->vo || !in->vv || !in->voo) return OR_ENOMEM;
  return OR_OK;
}

static void triples_free(triples_in* in) {
  free(in->t2);
  free(in->t1);
  free(in->vo);
  free(in->vv);
  free(in->voo);
}

/* E(T) of Eq. cc14 with the restricted sums i<j<k, a<b<c.  Deterministic: one
 * partial sum per occupied triple (abc in lexicographic order), the partials
 * then added in triple order.  `eps_o`, `eps_v`: orbital energies. */
int oracle_triples_energy(const otensor* T2, const double* t2, const otensor* T1, const double* t1,
                          const otensor* Vo, const double* vo, const otensor* Vv, const double* vv,
                          const otensor* Voo, const double* voo, const double* eps_o, const double* eps_v,
                          double* energy) {
  triples_in in;
  int st = triples_load(&in, T2, t2, T1, t1, Vo, vo, Vv, vv, Voo, voo);
  if (st) {
    triples_free(&in);
    return st;
  }
  const int64_t no = in.no, nv = in.nv;
  const int64_t n_trip = no * no * no;
  double* part = (double*)calloc((size_t)(n_trip > 0 ? n_trip : 1), sizeof(double));
  if (!part) {
    triples_free(&in);
    return OR_ENOMEM;
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < n_trip; ++q) {
    const int64_t i = q / (no * no), j = (q / no) % no, k = q % no;
    if (!(i < j && j < k)) continue;
    double s = 0.0;
    for (int64_t a = 0; a < nv; ++a)
      for (int64_t b = a + 1; b < nv; ++b)
        for (int64_t c = b + 1; c < nv; ++c) {
          const double w = triples_w(&in, i, j, k, a, b, c);
          const double y = triples_y(&in, i, j, k, a, b, c);
          const double d = eps_o[i] + eps_o[j] + eps_o[k] - eps_v[a] - eps_v[b] - eps_v[c];
          s += (w + y) * w / d;
        }
    part[q] = s;
  }
  double e = 0.0;
  for (int64_t q = 0; q < n_trip; ++q) e += part[q];
  free(part);
  triples_free(&in);
  *energy = e;
  return OR_OK;
}

/* W and Y of one occupied triple (i,j,k), any order, over every (a,b,c):
 * dense n_v^3 arrays, row-major over (a,b,c). */
int oracle_triples_wy(const otensor* T2, const double* t2, const otensor* T1, const double* t1, const otensor* Vo,
                      const double* vo, const otensor* Vv, const double* vv, const otensor* Voo, const double* voo,
                      int64_t i, int64_t j, int64_t k, double* w, double* y) {
  triples_in in;
  int st = triples_load(&in, T2, t2, T1, t1, Vo, vo, Vv, vv, Voo, voo);
  if (!st && (i < 0 || j < 0 || k < 0 || i >= in.no || j >= in.no || k >= in.no)) st = OR_EINVAL;
  if (st) {
    triples_free(&in);
    return st;
  }
  const int64_t nv = in.nv;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t a = 0; a < nv; ++a)
    for (int64_t b = 0; b < nv; ++b)
      for (int64_t c = 0; c < nv; ++c) {
        w[(a * nv + b) * nv + c] = triples_w(&in, i, j, k, a, b, c);
        y[(a * nv + b) * nv + c] = triples_y(&in, i, j, k, a, b, c);
      }
  triples_free(&in);
  return OR_OK;
}
