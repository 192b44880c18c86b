// FP64 kernels: permuted add (AddOp), block-sparse FP64 GEMM (MultOp, plain
// precision), and deterministic reductions (energy, norm).
//
// GB300 has a small FP64 pipe, so the FP64 GEMM is arithmetic-bound at any
// reasonable tile; it is a register-tiled DFMA kernel (64x64 CTA tile, 4x4 per
// thread, K step 16) over a device task list grouped by output block.  Each CTA
// owns one output tile and sums every block pair of its group in a fixed order,
// so results are deterministic and need no atomics.
#include "tamm_internal.h"

namespace tamm {
namespace {

struct Alpha4 {
  double v[kMaxAddTerms];
};

// Mixed-radix digits (row-major over dim[0..nm)) of the element index x and
// of the thread stride q; the loops below then step the digits by q with one
// carry pass per element instead of dividing.  Blocks hold < 2^31 elements.
struct Digits {
  int32_t idx[kMaxKernelModes], stp[kMaxKernelModes];
};

__device__ __forceinline__ void digits_init(const AddBlock& B, int32_t x, int32_t q, Digits& d) {
  for (int m = B.nm - 1; m >= 0; --m) {
    d.idx[m] = x % B.dim[m];
    x /= B.dim[m];
    d.stp[m] = q % B.dim[m];
    q /= B.dim[m];
  }
}

// The same with the mode count known at compile time (a permuted add's blocks all have the destination's
// NM modes): the loops unroll and the digits stay in registers instead of local memory.
template <int NM>
__device__ __forceinline__ void digits_init_n(const AddBlock& B, int32_t x, int32_t q, Digits& d) {
#pragma unroll
  for (int m = NM - 1; m >= 0; --m) {
    d.idx[m] = x % B.dim[m];
    x /= B.dim[m];
    d.stp[m] = q % B.dim[m];
    q /= B.dim[m];
  }
}

template <int NM>
__device__ __forceinline__ void digits_step_n(const AddBlock& B, Digits& d) {
  int32_t carry = 0;
#pragma unroll
  for (int m = NM - 1; m >= 0; --m) {
    int32_t v = d.idx[m] + d.stp[m] + carry;
    carry = v >= B.dim[m] ? 1 : 0;
    d.idx[m] = carry ? v - B.dim[m] : v;
  }
}

__device__ __forceinline__ void digits_step(const AddBlock& B, Digits& d) {
  int32_t carry = 0;
  for (int m = B.nm - 1; m >= 0; --m) {
    int32_t v = d.idx[m] + d.stp[m] + carry;
    carry = v >= B.dim[m] ? 1 : 0;
    d.idx[m] = carry ? v - B.dim[m] : v;
  }
}

// GB300's FP64 pipe is narrow (about two operations per clock per SM), so the adds keep FP64 arithmetic
// off the per-element path where they can: each term's factor is classified once per thread (bit t of
// `plus` / `minus`: alpha_t is +1 / -1), a first term with alpha = +-1 is a move of bits (the sign by an
// integer XOR) and a copy does no FP64 operation at all.
__device__ __forceinline__ double neg(double v) {
  return __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ull);
}
__device__ __forceinline__ double term0(unsigned plus, unsigned minus, int t, double alpha, double v) {
  return ((plus >> t) & 1u) ? v : (((minus >> t) & 1u) ? neg(v) : alpha * v);
}
__device__ __forceinline__ double term_n(unsigned plus, unsigned minus, int t, double alpha, double v, double acc) {
  return ((plus >> t) & 1u) ? acc + v : (((minus >> t) & 1u) ? acc - v : fma(alpha, v, acc));
}
__device__ __forceinline__ void classify(const Alpha4& alpha, int n_terms, unsigned& plus, unsigned& minus) {
  plus = minus = 0u;
#pragma unroll
  for (int t = 0; t < kMaxAddTerms; ++t) {
    if (t < n_terms && alpha.v[t] == 1.0) plus |= 1u << t;
    if (t < n_terms && alpha.v[t] == -1.0) minus |= 1u << t;
  }
}

// dst = beta*dst + sum_t alpha_t * src(perm_t), one chunk of one block per CTA (any layout: each source
// term is read through its strides).  NM: modes of the block.
template <int NM>
__global__ void __launch_bounds__(256) add_kernel(double* __restrict__ dst, const double* __restrict__ src,
                                                  const AddBlock* __restrict__ blocks,
                                                  const ChunkItem* __restrict__ items, int n_terms, double beta,
                                                  Alpha4 alpha, const double* __restrict__ scale) {
  const ChunkItem it = items[blockIdx.x];
  if (scale) {  // alpha_t * (*scale), read once per thread
    const double sc = *scale;
#pragma unroll
    for (int t = 0; t < kMaxAddTerms; ++t)
      if (t < n_terms) alpha.v[t] *= sc;
  }
  const AddBlock& B = blocks[it.block];
  const int64_t end = min(B.n, it.start + (int64_t)kChunk);
  unsigned plus, minus;
  classify(alpha, n_terms, plus, minus);
  const bool accumulate = beta != 0.0;  // beta is 0 or 1
  Digits dg;
  digits_init_n<NM>(B, (int32_t)(it.start + threadIdx.x), (int32_t)blockDim.x, dg);
  for (int64_t e = it.start + threadIdx.x; e < end; e += blockDim.x, digits_step_n<NM>(B, dg)) {
    double acc = 0.0;
    bool any = false;
#pragma unroll
    for (int t = 0; t < kMaxAddTerms; ++t) {
      if (t >= n_terms || B.src_off[t] < 0) continue;
      int64_t s = B.src_off[t];
#pragma unroll
      for (int m = 0; m < NM; ++m) s += (int64_t)dg.idx[m] * B.sstride[t][m];
      const double v = src[s];
      acc = any ? term_n(plus, minus, t, alpha.v[t], v, acc) : term0(plus, minus, t, alpha.v[t], v);
      any = true;
    }
    double* d = dst + B.dst_off + e;
    *d = accumulate ? *d + acc : acc;
  }
}

// x / d for 0 <= x < 2^16 and 1 <= d <= 2^16 by a multiply-high with m = floor((2^32 - 1) / d) + 1: the
// product overshoots x / d by less than x / 2^32 < 1 / d, so the floor is exact (d = 1 is taken apart: its
// m does not fit 32 bits).
__device__ __forceinline__ uint32_t div_magic(int d) { return d == 1 ? 0u : 0xFFFFFFFFu / (uint32_t)d + 1u; }
__device__ __forceinline__ int div_small(int x, uint32_t m, int d) { return d == 1 ? x : (int)__umulhi((uint32_t)x, m); }

// The same sum for a block whose source terms read the destination's last mode q with a stride (a
// transposition): the work item is a TP x TQ tile of the plane of q and the block's "row" mode p (the
// mode every transposed term reads contiguously) for n_o indices of the other modes.  All n_o planes of
// the transposed terms are staged through shared memory at once with reads that run along p
// (coalesced); the destination and the untransposed terms are then read and written along q.  The
// per-plane base offsets sit in shared memory, computed once per item.
__global__ void __launch_bounds__(256) add_tiled_kernel(double* __restrict__ dst, const double* __restrict__ src,
                                                        const AddBlock* __restrict__ blocks,
                                                        const TileItem* __restrict__ items, int n_terms, double beta,
                                                        Alpha4 alpha, const double* __restrict__ scale) {
  __shared__ double tile[kAddTileSmem];
  __shared__ int64_t sb[kMaxAddTerms][kAddMaxOuter];
  __shared__ int64_t db[kAddMaxOuter];
  const TileItem it = items[blockIdx.x];
  const AddBlock& B = blocks[it.block];
  const int nm = B.nm, p = B.tmode, q = nm - 1, n_o = it.n_o;
  const int TP = min(kAddTile, B.dim[p] - it.p0), TQ = min(kAddTile, B.dim[q] - it.q0), TQ1 = TQ + 1;
  const int plane = TP * TQ;
  if (scale) {
    const double sc = *scale;
#pragma unroll
    for (int t = 0; t < kMaxAddTerms; ++t)
      if (t < n_terms) alpha.v[t] *= sc;
  }
  unsigned plus, minus;
  classify(alpha, n_terms, plus, minus);
  const bool accumulate = beta != 0.0;
  unsigned trans = 0u, live = 0u;  // bit t: term t reads q with a stride / has a source block
#pragma unroll
  for (int t = 0; t < kMaxAddTerms; ++t) {
    if (t < n_terms && B.src_off[t] >= 0) {
      live |= 1u << t;
      if (B.sstride[t][q] != 1) trans |= 1u << t;
    }
  }
  int64_t dstr_p = 1;
  for (int m = nm - 1; m > p; --m) dstr_p *= B.dim[m];
  if (threadIdx.x < n_o) {  // base offsets of the item's planes
    int r = it.o0 + threadIdx.x;
    int64_t d = B.dst_off + (int64_t)it.p0 * dstr_p + it.q0, st = 1;
    int64_t s[kMaxAddTerms];
#pragma unroll
    for (int t = 0; t < kMaxAddTerms; ++t)
      s[t] = t < n_terms ? B.src_off[t] + (int64_t)it.p0 * B.sstride[t][p] + (int64_t)it.q0 * B.sstride[t][q] : 0;
    for (int m = nm - 1; m >= 0; --m) {
      if (m != p && m != q) {
        const int x = r % B.dim[m];
        r /= B.dim[m];
        d += x * st;
#pragma unroll
        for (int t = 0; t < kMaxAddTerms; ++t)
          if (t < n_terms) s[t] += (int64_t)x * B.sstride[t][m];
      }
      st *= B.dim[m];
    }
    db[threadIdx.x] = d;
#pragma unroll
    for (int t = 0; t < kMaxAddTerms; ++t) sb[t][threadIdx.x] = s[t];
  }
  __syncthreads();
  // stage the transposed terms: slot k holds term t's n_o planes, [plane][pl][ql] with row pitch TQ + 1.
  // Both loops run over all n_o planes at once (no thread idles at a plane's end); the indices come
  // from multiply-high divisions, exact for n_o * plane < 2^16 (at most kAddTileSmem elements).
  const int total = n_o * plane;
  const uint32_t m_plane = div_magic(plane), m_tp = div_magic(TP), m_tq = div_magic(TQ);
  int k = 0;
  for (int t = 0; t < n_terms; ++t) {
    if (!((trans >> t) & 1u)) continue;
    const int64_t sq = B.sstride[t][q];
    double* tk = tile + (size_t)k * n_o * TP * TQ1;
    for (int x = threadIdx.x; x < total; x += blockDim.x) {
      const int o = div_small(x, m_plane, plane), u = x - o * plane;
      const int ql = div_small(u, m_tp, TP), pl = u - ql * TP;  // along p: consecutive source addresses
      tk[(o * TP + pl) * TQ1 + ql] = src[sb[t][o] + pl + (int64_t)ql * sq];
    }
    ++k;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < total; x += blockDim.x) {
    const int o = div_small(x, m_plane, plane), u = x - o * plane;
    {
      const int pl = div_small(u, m_tq, TQ), ql = u - pl * TQ;  // along q: consecutive destination addresses
      double acc = 0.0;
      bool any = false;
      int kk = 0;
#pragma unroll
      for (int t = 0; t < kMaxAddTerms; ++t) {
        if (t >= n_terms || !((live >> t) & 1u)) continue;
        double v;
        if ((trans >> t) & 1u) {
          v = tile[((size_t)kk * n_o * TP + o * TP + pl) * TQ1 + ql];
          ++kk;
        } else {
          v = src[sb[t][o] + (int64_t)pl * B.sstride[t][p] + ql];
        }
        acc = any ? term_n(plus, minus, t, alpha.v[t], v, acc) : term0(plus, minus, t, alpha.v[t], v);
        any = true;
      }
      double* d = dst + db[o] + (int64_t)pl * dstr_p + ql;
      *d = accumulate ? *d + acc : acc;
    }
  }
}

// Cholesky pair difference for row p of one V block: for each q, the second product's (s, r) plane
// X1[p, :, q, :] of block (tp,ts,tq,tr) is staged in shared memory (row pitch nr + 1 against bank
// conflicts), so that the reads of both X1 blocks and the write of V all run along the contiguous last
// index; then V[p,q,r,s] = X1[p,r,q,s] - plane[s][r].
__global__ void __launch_bounds__(256) cholesky_pair_kernel(double* __restrict__ v, const double* __restrict__ x1,
                                                            const PairBlock* __restrict__ blocks,
                                                            const PairItem* __restrict__ items) {
  extern __shared__ double plane[];
  const PairItem it = items[blockIdx.x];
  const PairBlock B = blocks[it.block];
  const int p = it.p, nq = B.nq, nr = B.nr, ns = B.ns;
  const int n = nr * ns;
  for (int q = 0; q < nq; ++q) {
    if (B.b_off >= 0) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int s = i / nr, r = i - s * nr;
        plane[s * (nr + 1) + r] = x1[B.b_off + ((int64_t)(p * ns + s) * nq + q) * nr + r];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int r = i / ns, s = i - r * ns;
      double val = B.a_off >= 0 ? x1[B.a_off + ((int64_t)(p * nr + r) * nq + q) * ns + s] : 0.0;
      if (B.b_off >= 0) val -= plane[s * (nr + 1) + r];
      v[B.v_off + ((int64_t)(p * nq + q) * nr + r) * ns + s] = val;
    }
    __syncthreads();
  }
}

template <int NT>
__device__ double block_sum(double v) {
  __shared__ double red[NT / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// partials[item] = sum over the chunk of a[x] * b[perm(x)]
__global__ void __launch_bounds__(256) energy_partials_kernel(const double* __restrict__ a,
                                                              const double* __restrict__ b,
                                                              const AddBlock* __restrict__ blocks,
                                                              const ChunkItem* __restrict__ items,
                                                              double* __restrict__ partials) {
  const ChunkItem it = items[blockIdx.x];
  const AddBlock& B = blocks[it.block];
  const int64_t end = min(B.n, it.start + (int64_t)kChunk);
  const int nm = B.nm;
  double acc = 0.0;
  if (B.src_off[0] >= 0) {
    Digits dg;
    digits_init(B, (int32_t)(it.start + threadIdx.x), (int32_t)blockDim.x, dg);
    for (int64_t e = it.start + threadIdx.x; e < end; e += blockDim.x, digits_step(B, dg)) {
      int64_t s = B.src_off[0];
      for (int m = 0; m < nm; ++m) s += (int64_t)dg.idx[m] * B.sstride[0][m];
      acc = fma(a[B.dst_off + e], b[s], acc);
    }
  }
  double s = block_sum<256>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) sumsq_partials_kernel(const double* __restrict__ x, int64_t n,
                                                             int64_t per, double* __restrict__ partials) {
  const int64_t lo = (int64_t)blockIdx.x * per;
  const int64_t hi = min(n, lo + per);
  double acc = 0.0;
  for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) acc = fma(x[e], x[e], acc);
  double s = block_sum<256>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) diff_sumsq_partials_kernel(const double* __restrict__ x,
                                                                  const double* __restrict__ y, int64_t n,
                                                                  int64_t per, double* __restrict__ partials) {
  const int64_t lo = (int64_t)blockIdx.x * per;
  const int64_t hi = min(n, lo + per);
  double acc = 0.0;
  for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    const double d = x[e] - y[e];
    acc = fma(d, d, acc);
  }
  double s = block_sum<256>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) reduce_final_kernel(const double* __restrict__ p, int64_t n, double alpha,
                                                            int take_sqrt, double* __restrict__ out) {
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += p[i];
  double s = block_sum<1024>(acc);
  if (threadIdx.x == 0) *out = take_sqrt ? sqrt(s) : alpha * s;
}

// ------------------------------------------------------------------ FP64 GEMM

constexpr int BM = kGemmTileM, BN = kGemmTileN, BK = 16;

__global__ void __launch_bounds__(256) gemm_f64_kernel(const double* __restrict__ A, const double* __restrict__ Bm,
                                                       double* __restrict__ C, const GemmGroup* __restrict__ groups,
                                                       const GemmTask* __restrict__ tasks,
                                                       const GemmItem* __restrict__ items, double alpha,
                                                       double beta) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN];
  const GemmItem it = items[blockIdx.x];
  const GemmGroup g = groups[it.group];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  // loader coordinates: A tile 64 x 16 (4 consecutive k per thread), B tile 16 x 64 (4 consecutive n)
  const int ar = tid / 4, ac = (tid % 4) * 4;
  const int bk = tid / 16, bn = (tid % 16) * 4;
  const int M = g.M, N = g.N;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int t = g.task_begin; t < g.task_end; ++t) {
    const GemmTask tk = tasks[t];
    const int K = tk.K;
    const double* a = A + tk.a_off;
    const double* b = Bm + tk.b_off;
    double ra[4], rb[4];
    auto load = [&](int k0) {
      const int row = it.m0 + ar;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + ac + q;
        ra[q] = (row < M && k < K) ? __ldg(a + (int64_t)row * K + k) : 0.0;
      }
      const int kk = k0 + bk;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int col = it.n0 + bn + q;
        rb[q] = (kk < K && col < N) ? __ldg(b + (int64_t)kk * N + col) : 0.0;
      }
    };
    load(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        As[ac + q][ar] = ra[q];
        Bs[bk][bn + q] = rb[q];
      }
      __syncthreads();
      if (k0 + BK < K) load(k0 + BK);
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        double av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = As[k][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bv[j] = Bs[k][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = it.m0 + ty + 16 * i;
    if (row >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = it.n0 + tx + 16 * j;
      if (col >= N) continue;
      double* c = C + g.c_off + (int64_t)row * N + col;
      *c = beta != 0.0 ? fma(beta, *c, alpha * acc[i][j]) : alpha * acc[i][j];
    }
  }
}

}  // namespace

cudaError_t launch_add(tamm_ctx* ctx, double* dst, const double* src, const AddBlock* blocks,
                       const ChunkItem* items, int64_t n_items, int n_terms, double beta, const double* alpha_host,
                       const double* scale_device, int nm, const TileItem* tiles, int64_t n_tiles) {
  if (n_items == 0 && n_tiles == 0) return cudaSuccess;
  Alpha4 al{};
  for (int t = 0; t < n_terms; ++t) al.v[t] = alpha_host[t];
  if (n_items > 0) {
    kernel_begin(ctx, TAMM_KERNEL_ADD);
    switch (nm) {
      case 1: add_kernel<1><<<(unsigned)n_items, 256, 0, ctx->stream>>>(dst, src, blocks, items, n_terms, beta, al,
                                                                        scale_device); break;
      case 2: add_kernel<2><<<(unsigned)n_items, 256, 0, ctx->stream>>>(dst, src, blocks, items, n_terms, beta, al,
                                                                        scale_device); break;
      case 3: add_kernel<3><<<(unsigned)n_items, 256, 0, ctx->stream>>>(dst, src, blocks, items, n_terms, beta, al,
                                                                        scale_device); break;
      default: add_kernel<4><<<(unsigned)n_items, 256, 0, ctx->stream>>>(dst, src, blocks, items, n_terms, beta, al,
                                                                         scale_device); break;
    }
    kernel_end(ctx, TAMM_KERNEL_ADD);
  }
  if (n_tiles > 0) {
    kernel_begin(ctx, TAMM_KERNEL_ADD);
    add_tiled_kernel<<<(unsigned)n_tiles, 256, 0, ctx->stream>>>(dst, src, blocks, tiles, n_terms, beta, al,
                                                                  scale_device);
    kernel_end(ctx, TAMM_KERNEL_ADD);
  }
  return cudaGetLastError();
}

cudaError_t launch_cholesky_pair(tamm_ctx* ctx, double* v, const double* x1, const PairBlock* blocks,
                                 const PairItem* items, int64_t n_items, size_t smem_bytes) {
  if (n_items == 0) return cudaSuccess;
  if (smem_bytes > kPairSmemMax) return cudaErrorInvalidValue;  // the caller uses the permuted add instead
  kernel_begin(ctx, TAMM_KERNEL_ADD);
  cholesky_pair_kernel<<<(unsigned)n_items, 256, smem_bytes, ctx->stream>>>(v, x1, blocks, items);
  kernel_end(ctx, TAMM_KERNEL_ADD);
  return cudaGetLastError();
}

cudaError_t launch_energy_partials(tamm_ctx* ctx, const double* a, const double* b, const AddBlock* blocks,
                                   const ChunkItem* items, int64_t n_items, double* partials) {
  if (n_items == 0) return cudaSuccess;
  kernel_begin(ctx, TAMM_KERNEL_REDUCE);
  energy_partials_kernel<<<(unsigned)n_items, 256, 0, ctx->stream>>>(a, b, blocks, items, partials);
  kernel_end(ctx, TAMM_KERNEL_REDUCE);
  return cudaGetLastError();
}

cudaError_t launch_sumsq_partials(tamm_ctx* ctx, const double* x, int64_t n, double* partials, int64_t n_parts) {
  if (n_parts == 0) return cudaSuccess;
  const int64_t per = (n + n_parts - 1) / n_parts;
  kernel_begin(ctx, TAMM_KERNEL_REDUCE);
  sumsq_partials_kernel<<<(unsigned)n_parts, 256, 0, ctx->stream>>>(x, n, per, partials);
  kernel_end(ctx, TAMM_KERNEL_REDUCE);
  return cudaGetLastError();
}

cudaError_t launch_diff_sumsq_partials(tamm_ctx* ctx, const double* x, const double* y, int64_t n,
                                       double* partials, int64_t n_parts) {
  if (n_parts == 0) return cudaSuccess;
  const int64_t per = (n + n_parts - 1) / n_parts;
  kernel_begin(ctx, TAMM_KERNEL_REDUCE);
  diff_sumsq_partials_kernel<<<(unsigned)n_parts, 256, 0, ctx->stream>>>(x, y, n, per, partials);
  kernel_end(ctx, TAMM_KERNEL_REDUCE);
  return cudaGetLastError();
}

cudaError_t launch_reduce_final(tamm_ctx* ctx, const double* partials, int64_t n, double alpha, int take_sqrt,
                                double* out_device) {
  kernel_begin(ctx, TAMM_KERNEL_REDUCE);
  reduce_final_kernel<<<1, 1024, 0, ctx->stream>>>(partials, n, alpha, take_sqrt, out_device);
  kernel_end(ctx, TAMM_KERNEL_REDUCE);
  return cudaGetLastError();
}

cudaError_t launch_gemm_f64(tamm_ctx* ctx, const double* a, const double* b, double* c, const GemmGroup* groups,
                            const GemmTask* tasks, const GemmItem* items, int64_t n_items, double alpha,
                            double beta) {
  if (n_items == 0) return cudaSuccess;
  kernel_begin(ctx, TAMM_KERNEL_GEMM_F64);
  gemm_f64_kernel<<<(unsigned)n_items, 256, 0, ctx->stream>>>(a, b, c, groups, tasks, items, alpha, beta);
  kernel_end(ctx, TAMM_KERNEL_GEMM_F64);
  return cudaGetLastError();
}

}  // namespace tamm
