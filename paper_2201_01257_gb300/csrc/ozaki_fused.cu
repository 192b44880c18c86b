// Split-precision block GEMM that slices its A operand itself (short summed ranges, narrow outputs).
//
// Warp roles (384 threads, as the pre-sliced GEMM): warp 0 copies the pre-sliced B tiles into the
// stages with 1-D bulk copies; warp 1 issues the tcgen05 MMAs and owns TMEM; warps 2 and 3 idle;
// warps 4..11 are workers.  For every block pair (a "chunk": the exact accumulation unit) a worker
// thread loads its 24 of its row's FP64 values (row = TMEM lane, 32 rows per warp quadrant; the two
// warps of a quadrant take alternate 8-index halves of each 16-index K tile), the two threads of a row
// exchange their maxima through shared memory, and each turns its values into S BF16 digit slices
// written in the 32-byte-swizzled K-major layout the MMA descriptors expect.  After producing chunk
// c the workers drain chunk c - 1 (one chunk behind, so the MMAs of chunk c overlap the drain), fold
// it into the (hi, lo) pair of its output tile, and after an item's last chunk write C through the
// output block's strides.  All waits are bounded; a timeout records TAMM_ETIMEOUT and every role
// still passes the same named barriers.
#include <algorithm>
#include <mutex>

#include "ozaki.h"
#include "ozaki_device.cuh"
#include "sm100.cuh"

namespace tamm {
namespace {

constexpr int kFaWorkers = 8;
static_assert(kThreads == 128 + 32 * kFaWorkers, "the register split assumes the pre-sliced GEMM's warp count");
constexpr int kFaMaxStages = 4;

__device__ __forceinline__ void fa_barrier() { asm volatile("bar.sync 2, %0;" ::"n"(32 * kFaWorkers) : "memory"); }

// Generic-proxy shared-memory writes made visible to the tensor core's (async proxy) reads.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// The two worker warps of one TMEM lane quadrant (the two halves of every row) synchronise on their own
// named barrier (ids 3..6), so the four quadrants do not wait for each other.
__device__ __forceinline__ void pair_barrier(int q) { asm volatile("bar.sync %0, 64;" ::"r"(3 + q) : "memory"); }

// Dependency wait without back-off: the chunks here are short, so a sleeping waiter would add its sleep
// to every hand-off between the workers, the copy warp and the MMA issuer.  Bounded like wait_bounded.
__device__ __forceinline__ bool wait_hot(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* status,
                                         long long limit) {
  const long long t0 = clock64();
  while (!sm100::mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
      *abort_flag = 1;
      atomicExch(status, TAMM_ETIMEOUT);
      return false;
    }
  }
  return true;
}

// This thread's FP64 values of block pair t for item i: K tiles kt, summed indices 16 kt + 8 h + u (zero past
// the block's rows and summed range).
__device__ __forceinline__ void fa_load(const FaParams& p, int64_t i, int t, int row, int h, double (&x)[3][8]) {
  const FaItem it = p.items[i];
  const FaTask tk = p.tasks[t];
  const SliceBlock& A = p.a_recs[tk.a_rec];
  const int32_t grow = it.mt * kOzTileM + row;
  const int64_t roff = grow < A.rows ? A.src_off + mixed_offset(grow, A.nr, A.rdim, A.rstride) : -1;
  const int32_t K = A.K, nk = A.nk;
  const int64_t ks0 = A.kstride[0];
#pragma unroll
  for (int kt = 0; kt < 3; ++kt)
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int32_t k = 16 * kt + 8 * h + u;
      x[kt][u] = (roff >= 0 && kt < tk.k_tiles && k < K)
                     ? __ldg(p.a_src + roff + (nk == 1 ? (int64_t)k * ks0 : mixed_offset(k, nk, A.kdim, A.kstride)))
                     : 0.0;
    }
}

template <int S>
__global__ void __launch_bounds__(kThreads, 1) ozaki_gemm_fused_a_kernel(const __grid_constant__ FaParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int stages = p.stages;
  constexpr uint32_t half_bytes = (uint32_t)S * kOzTileBytesPerSlice;  // A part of a stage; the B part as large
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)stages * 2 * half_bytes);
  uint64_t* full = bars;                      // [stages]: B copy (arrival + bytes) and the worker warps
  uint64_t* empty = bars + kFaMaxStages;      // [stages]: MMA commit
  uint64_t* acc_full = empty + kFaMaxStages;  // [kAccBufs]
  uint64_t* acc_empty = acc_full + kAccBufs;  // [kAccBufs]: worker warps
  uint64_t* drain = acc_empty + kAccBufs;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  unsigned long long* rmax = reinterpret_cast<unsigned long long*>(tmem_holder + 4);  // [2 chunks][2 halves][128]
  int* fref = reinterpret_cast<int*>(rmax + 2 * 2 * 128);                              // [2 items][kOzFaMaxN]
  int64_t* coff = reinterpret_cast<int64_t*>(fref + 2 * kOzFaMaxN);                    // [2 items][kOzFaMaxN]

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      sm100::mbar_init(&full[s], 1 + kFaWorkers);
      sm100::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < kAccBufs; ++b) {
      sm100::mbar_init(&acc_full[b], 1);
      sm100::mbar_init(&acc_empty[b], kFaWorkers);
    }
    sm100::mbar_init(drain, 1);
    *abort_flag = 0;
    sm100::fence_mbar_init();
  }
  if (warp == 1) {
    sm100::tmem_alloc(tmem_holder, 512);
    sm100::tmem_relinquish();
  }
  sm100::tc_fence_before();
  __syncthreads();
  sm100::tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsLow));
  }
  if (warp == 0) {
    // ------------------------------------------------------------ B producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, issued_mask = 0, issued_parity = 0;
      for (int64_t i = blockIdx.x; i < p.n_items && !*abort_flag; i += gridDim.x) {
        const FaGroup& g = p.groups[p.items[i].group];
        const uint32_t b_bytes = (uint32_t)S * 32u * (uint32_t)g.n_tile;
        for (int t = g.task_begin; t < g.task_end && !*abort_flag; ++t) {
          const FaTask tk = p.tasks[t];
          for (int kt = 0; kt < tk.k_tiles; ++kt) {
            if (!wait_hot(&empty[stage], phase ^ 1u, abort_flag, p.status, p.wait_cycles)) break;
            uint8_t* sb = smem + (size_t)stage * 2 * half_bytes + half_bytes;
            sm100::mbar_arrive_expect_tx(&full[stage], b_bytes);
            sm100::bulk_g2s(sb, p.b_tiles + tk.b_off + (size_t)kt * b_bytes, b_bytes, &full[stage]);
            issued_mask |= 1u << stage;
            issued_parity = (issued_parity & ~(1u << stage)) | (phase << stage);
            if (++stage == stages) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
      // every issued copy must land before the CTA may exit
      for (int s = 0; s < stages; ++s) {
        if (!(issued_mask >> s & 1u)) continue;
        const long long t0 = clock64();
        while (!sm100::mbar_try_wait(&full[s], (issued_parity >> s) & 1u) && clock64() - t0 < kDrainWaitCycles) {
        }
      }
    }
  } else if (warp == 1) {
    // --------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint64_t desc_stage0 = sm100::desc_kmajor_sw32(sm100::smem_u32(smem));
      int stage = 0;
      uint32_t phase = 0, acc_parity = 0, acc_used = 0, buf = 0, cur_H = 0;
      bool ok = true;
      for (int64_t i = blockIdx.x; i < p.n_items && ok; i += gridDim.x) {
        const FaGroup& g = p.groups[p.items[i].group];
        if (g.task_begin == g.task_end) continue;  // no chunk: the workers write such an item alone
        const uint32_t H = (uint32_t)g.n_tile;
        const uint32_t nbuf = acc_buffers(H);
        if (H != cur_H) {
          // another buffer layout: every buffer still being drained must be free first
          for (int b = 0; b < kAccBufs && ok; ++b)
            if ((acc_used >> b) & 1u)
              ok = wait_hot(&acc_empty[b], ((acc_parity >> b) & 1u) ^ 1u, abort_flag, p.status, p.wait_cycles);
          if (!ok) break;
          buf = 0;
          cur_H = H;
        }
        // B images are H rows with zero rows past N, so every tile runs the fused N = 2H schedule
        const uint32_t idesc1 = sm100::idesc_bf16_f32(128, H);
        const uint32_t idesc2 = sm100::idesc_bf16_f32(128, 2u * H);
        for (int t = g.task_begin; t < g.task_end && ok; ++t) {
          const int k_tiles = p.tasks[t].k_tiles;
          for (int kt = 0; kt < k_tiles; ++kt) {
            const bool first = kt == 0, last = kt + 1 == k_tiles;
            if (first) {
              if (!wait_hot(&acc_empty[buf], ((acc_parity >> buf) & 1u) ^ 1u, abort_flag, p.status,
                            p.wait_cycles)) {
                ok = false;
                break;
              }
              sm100::tc_fence_after();
            }
            if (!wait_hot(&full[stage], phase, abort_flag, p.status, p.wait_cycles)) {
              ok = false;
              break;
            }
            sm100::tc_fence_after();
            const uint64_t a0 = desc_stage0 + (uint64_t)((uint32_t)stage * (2u * half_bytes >> 4));
            const uint64_t b0 = a0 + (half_bytes >> 4);
            issue_ops<S, true, 0>(tmem + buf * 4u * H, a0, b0, H, idesc1, idesc2, first);
            sm100::mma_commit(&empty[stage]);
            if (last) {
              sm100::mma_commit(&acc_full[buf]);
              acc_parity ^= 1u << buf;
              acc_used |= 1u << buf;
              buf = buf + 1 == nbuf ? 0u : buf + 1;
            }
            if (++stage == stages) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
      // all issued MMAs must finish before TMEM is released
      sm100::mma_commit(drain);
      const long long t0 = clock64();
      while (!sm100::mbar_try_wait(drain, 0) && clock64() - t0 < kDrainWaitCycles) {
      }
    }
    __syncwarp();
  } else if (warp >= 4) {
    // ------------------------------------------------------------- workers
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsHigh));
    const int q = warp & 3;              // TMEM lane quadrant
    const int h = (warp - 4) >> 2;       // K half of every K tile; column half of the output tile
    const int wid = threadIdx.x - 128;   // 0..255
    const int row = q * 32 + lane;
    const int swz = (row >> 2) & 1;
    const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
    const int ae = p.alpha_exp;
    const bool a_p2 = p.alpha_pow2 != 0, a_neg = p.alpha < 0.0;
    int stage = 0;
    uint32_t phase = 0;
    uint32_t acc_parity = 0, dbuf = 0;
    int drain_H = 0;
    bool ok = true;
    float hi[32], lo[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0.0f;
    // the chunk waiting for its drain, and the item it belongs to
    bool pend = false;
    int pend_ea = kOzExpZero, pend_task = 0, pend_ip = 0, pend_H = 16, pend_N = 0;
    bool pend_last = false;
    int pend_Eref = kOzExpZero;
    int64_t pend_rowoff = -1;

    // fold the pending chunk into (hi, lo); after an item's last chunk, write its outputs
    auto drain_pending = [&]() {
      const int H = pend_H;
      const uint32_t nbuf = acc_buffers((uint32_t)H);
      if (H != drain_H) {  // mirrors the MMA issuer's buffer sequence
        dbuf = 0;
        drain_H = H;
      }
      if (ok && !wait_hot(&acc_full[dbuf], (acc_parity >> dbuf) & 1u, abort_flag, p.status, p.wait_cycles))
        ok = false;
      const int hc = H >> 1;  // columns per worker: [h hc, h hc + hc)
      const int c0 = h * hc;
      if (ok) {
        sm100::tc_fence_after();
        const float sA = (pend_ea == kOzExpZero || pend_Eref == kOzExpZero) ? 0.0f : pow2f(pend_ea - pend_Eref);
        const int32_t* eb = p.b_exp + p.tasks[pend_task].b_exp;
        const int* fr = fref + pend_ip * kOzFaMaxN;
        const uint32_t tb = trow + dbuf * 4u * (uint32_t)H;
#pragma unroll
        for (int g8 = 0; g8 < 4; ++g8) {
          if (8 * g8 >= hc) break;
          const int col = c0 + 8 * g8;
          float r0[8], r1[8], r2[8], r3[8];
          sm100::tmem_ld8(tb + 0 * H + col, r0);
          sm100::tmem_ld8(tb + 1 * H + col, r1);
          sm100::tmem_ld8(tb + 2 * H + col, r2);
          if constexpr (S >= 4) {
            sm100::tmem_ld8(tb + 3 * H + col, r3);
          } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) r3[j] = 0.0f;
          }
          sm100::tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int c = col + j;
            const int e = c < pend_N ? eb[c] : kOzExpZero;
            const float sB = (e == kOzExpZero || fr[c] == kOzExpZero) ? 0.0f : pow2f(e - fr[c]);
            fold(hi[8 * g8 + j], lo[8 * g8 + j], r0[j], r1[j], r2[j], r3[j], sA * sB);
          }
        }
        sm100::tc_fence_before();
        __syncwarp();
        if (lane == 0) sm100::mbar_arrive(&acc_empty[dbuf]);
      }
      acc_parity ^= 1u << dbuf;
      dbuf = dbuf + 1 == nbuf ? 0u : dbuf + 1;
      if (pend_last) {
        if (ok && pend_rowoff >= 0) {
          const int* fr = fref + pend_ip * kOzFaMaxN;
          const int64_t* co = coff + pend_ip * kOzFaMaxN;
          const double alpha = p.alpha, beta = p.beta;
#pragma unroll
          for (int g8 = 0; g8 < 4; ++g8) {
            if (8 * g8 >= hc) break;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int c = c0 + 8 * g8 + j;
              if (c < pend_N) {
                double av = 0.0;  // alpha * (product)
                if (pend_Eref != kOzExpZero && fr[c] != kOzExpZero) {
                  const int sc = pend_Eref + fr[c] - 12;
                  double dh, dl;
                  if (a_p2 && f2d_scaled(hi[8 * g8 + j], sc + ae, a_neg, dh) &&
                      f2d_scaled(lo[8 * g8 + j], sc + ae, a_neg, dl))
                    av = dh + dl;
                  else
                    av = alpha * (((double)hi[8 * g8 + j] + (double)lo[8 * g8 + j]) * pow2d(sc));
                } else {
                  av = alpha * 0.0;
                }
                double* cp = p.c + pend_rowoff + co[c];
                *cp = beta != 0.0 ? fma(beta, *cp, av) : av;
              }
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0.0f;
      }
    };

    int item_count = 0, chunk = 0;
    // The values of the next block pair are loaded as soon as the current pair is converted, before the
    // previous pair's drain, so HBM latency overlaps the drain and the next row-maximum exchange.
    double x[3][8];
    bool have = false;  // x holds the values of (have_i, have_t)
    int64_t have_i = -1;
    int have_t = -1;
    for (int64_t i = blockIdx.x; i < p.n_items; i += gridDim.x, ++item_count) {
      const int ip = item_count & 1;
      const FaItem it = p.items[i];
      const FaGroup& g = p.groups[it.group];
      const int H = g.n_tile, N = g.N;
      // the item's column data: reference exponents (maxima over its block pairs) and C offsets.  The
      // slot was last read by the drain of item i - 2's last chunk, which every worker has finished
      // before this barrier.
      fa_barrier();
      if (wid < H) {
        int F = kOzExpZero;
        int64_t co = 0;
        if (wid < N) {
          for (int t = g.task_begin; t < g.task_end; ++t) F = max(F, p.b_exp[p.tasks[t].b_exp + wid]);
          co = mixed_offset(wid, g.nc, g.cdim, g.cstride);
        }
        fref[ip * kOzFaMaxN + wid] = F;
        coff[ip * kOzFaMaxN + wid] = co;
      }
      const int32_t grow = it.mt * kOzTileM + row;
      const bool live = grow < g.M;
      const int64_t rowoff = live ? g.c_off + mixed_offset(grow, g.nr, g.rdim, g.rstride) : -1;
      if (g.task_begin == g.task_end) {
        // no block pair feeds this output block: C = beta C + alpha * 0
        if (ok && live && p.beta == 0.0) {
          const int hc = H >> 1;
          for (int c = h * hc; c < h * hc + hc && c < N; ++c) p.c[rowoff + mixed_offset(c, g.nc, g.cdim, g.cstride)] = p.alpha * 0.0;
        }
        continue;
      }
      int Eref = kOzExpZero;  // the row's first nonzero block exponent: the item's reference
      for (int t = g.task_begin; t < g.task_end; ++t, ++chunk) {
        const int k_tiles = p.tasks[t].k_tiles;
        const int cp = chunk & 1;
        if (!(have && have_i == i && have_t == t)) fa_load(p, i, t, row, h, x);
        unsigned long long m = 0ull;
#pragma unroll
        for (int kt = 0; kt < 3; ++kt)
#pragma unroll
          for (int u = 0; u < 8; ++u)
            m = max(m, (unsigned long long)__double_as_longlong(x[kt][u]) & 0x7FFFFFFFFFFFFFFFull);
        // the row maximum over both halves
        rmax[(cp * 2 + h) * 128 + row] = m;
        pair_barrier(q);
        m = max(m, rmax[(cp * 2 + (h ^ 1)) * 128 + row]);
        int e = kOzExpZero;
        if (m != 0ull) (void)frexp(__longlong_as_double((long long)m), &e);
        if (Eref == kOzExpZero) Eref = e;
        // digits into the stages
#pragma unroll
        for (int kt = 0; kt < 3; ++kt) {
          if (kt >= k_tiles) break;
          if (ok && !wait_hot(&empty[stage], phase ^ 1u, abort_flag, p.status, p.wait_cycles)) ok = false;
          if (ok) {
            uint32_t w[4][S];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              if (e != kOzExpZero) {
                pack_digits<S>(x[kt][2 * j], x[kt][2 * j + 1], e, w[j]);
              } else {
#pragma unroll
                for (int s = 0; s < S; ++s) w[j][s] = 0u;
              }
            }
            uint8_t* sa = smem + (size_t)stage * 2 * half_bytes + row * 32 + ((h ^ swz) * 16);
#pragma unroll
            for (int s = 0; s < S; ++s)
              *reinterpret_cast<uint4*>(sa + (size_t)s * kOzTileBytesPerSlice) = make_uint4(w[0][s], w[1][s], w[2][s], w[3][s]);
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) sm100::mbar_arrive(&full[stage]);
          }
          if (++stage == stages) {
            stage = 0;
            phase ^= 1u;
          }
        }
        // the next block pair's values: the next pair of this item, else the first of the next item
        have = false;
        if (t + 1 < g.task_end) {
          have_i = i;
          have_t = t + 1;
          have = true;
        } else if (i + gridDim.x < p.n_items) {
          const FaGroup& gn = p.groups[p.items[i + gridDim.x].group];
          if (gn.task_begin < gn.task_end) {
            have_i = i + gridDim.x;
            have_t = gn.task_begin;
            have = true;
          }
        }
        if (have) fa_load(p, have_i, have_t, row, h, x);
        // the previous chunk's drain overlaps this chunk's MMAs and the loads just issued
        if (pend) drain_pending();
        pend = true;
        pend_ea = e;
        pend_task = t;
        pend_ip = ip;
        pend_H = H;
        pend_N = N;
        pend_last = t + 1 == g.task_end;
        pend_Eref = Eref;
        pend_rowoff = rowoff;
      }
    }
    if (pend) drain_pending();
  }
  __syncthreads();
  if (warp == 1) {
    sm100::tc_fence_after();
    sm100::tmem_dealloc(tmem, 512);
  }
}

}  // namespace

static std::mutex g_fa_mutex;

static int fa_stages(int S) { return std::min(kFaMaxStages, (192 * 1024) / (2 * S * kOzTileBytesPerSlice)); }

static size_t fa_smem_bytes(int S) { return (size_t)fa_stages(S) * 2 * S * kOzTileBytesPerSlice + 1024 + 8192; }

template <int S>
static cudaError_t fa_dispatch(tamm_ctx* ctx, const FaParams& p, int grid) {
  static bool ready[64] = {};
  if (ctx->device < 0 || ctx->device >= 64) return cudaErrorInvalidDevice;
  const size_t smem = fa_smem_bytes(S);
  {
    std::lock_guard<std::mutex> lock(g_fa_mutex);
    if (!ready[ctx->device]) {
      cudaFuncAttributes fa;
      cudaError_t e = cudaFuncGetAttributes(&fa, ozaki_gemm_fused_a_kernel<S>);
      if (e != cudaSuccess) return e;
      if (fa.numRegs < kRegsLaunchNeeded) return cudaErrorLaunchOutOfResources;  // setmaxnreg pool
      e = cudaFuncSetAttribute(ozaki_gemm_fused_a_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      ready[ctx->device] = true;
    }
  }
  ozaki_gemm_fused_a_kernel<S><<<(unsigned)grid, kThreads, smem, ctx->stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_ozaki_fused(tamm_ctx* ctx, FaParams& p, int S) {
  if (p.n_items == 0) return cudaSuccess;
  p.status = ctx->d_status;
  p.wait_cycles = ctx->oz_wait_cycles;
  p.stages = fa_stages(S);
  const int grid = (int)std::min<int64_t>(p.n_items, std::max(1, ctx->sm_count));
  kernel_begin(ctx, TAMM_KERNEL_GEMM_OZ);
  cudaError_t e = cudaErrorInvalidValue;
  switch (S) {
    case 3: e = fa_dispatch<3>(ctx, p, grid); break;
    case 4: e = fa_dispatch<4>(ctx, p, grid); break;
    case 5: e = fa_dispatch<5>(ctx, p, grid); break;
    case 6: e = fa_dispatch<6>(ctx, p, grid); break;
    case 7: e = fa_dispatch<7>(ctx, p, grid); break;
    case 8: e = fa_dispatch<8>(ctx, p, grid); break;
  }
  kernel_end(ctx, TAMM_KERNEL_GEMM_OZ);
  return e;
}

}  // namespace tamm
