// Split-precision block-sparse contraction: slicing kernel, tcgen05 GEMM
// kernel and the host plan that drives them.  The arithmetic scheme is
// described in ozaki.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>

#include "ozaki.h"
#include "ozaki_device.cuh"
#include "sm100.cuh"

namespace tamm {

// ======================================================================
// Device: slicing
// ======================================================================
namespace {

// One CTA (W = blockDim.x / 32 warps) slices rows [r0, r0+nr) of one block.
// Dense summed range (every row one contiguous run): one warp per row, nr <=
// W.  The row comes into the warp's shared buffer through one 1-D bulk copy
// of its 16-byte-aligned span (the start rounded down, so element k sits at
// k + shift; the at most one element past the rounded-down end by a plain
// load), so HBM is read once.  The row maximum comes from conflict-free
// strided reads and a warp reduction; then each lane turns two adjacent
// elements into one 32-bit word per slice, a warp's stores filling whole
// 32-byte sectors of four tiles.
// Other layouts: 8-wide units read straight from global memory twice, lanes
// walking rows fastest so that the contiguous direction is coalesced.
// `kbuf`: doubles per warp buffer (>= K + 2 of every dense block, even);
// `bulk`: the source base is 16-byte aligned, so that rounding a row's start
// down stays inside the tensor.
template <int S, bool kFloat>
__global__ void __launch_bounds__(256) ozaki_slice_kernel(const double* __restrict__ src,
                                                          const SliceBlock* __restrict__ blocks,
                                                          const SliceItem* __restrict__ items,
                                                          uint8_t* __restrict__ tiles, int32_t* __restrict__ exps,
                                                          int kbuf, int bulk, int* __restrict__ status,
                                                          long long wait_cycles, int mode,
                                                          unsigned long long* __restrict__ smax) {
  extern __shared__ __align__(16) double rowbuf[];
  __shared__ unsigned long long rmax[kOzSliceMaxRows];
  __shared__ int rexp[kOzSliceMaxRows];
  __shared__ int64_t roff[kOzSliceMaxRows];
  __shared__ __align__(8) uint64_t wbar[8];
  const SliceItem it = items[blockIdx.x];
  const SliceBlock& B = blocks[it.block];
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  const int nr = it.nr;
  const int K = B.K;
  const int H = B.tile_rows;
  const size_t slice_bytes = (size_t)H * 32;  // one slice of one tile: H rows x 16 bf16
  const size_t tile_bytes = (size_t)S * slice_bytes;

  if (B.k_dense) {
    if (warp >= nr) return;  // no block-wide barrier on this path
    const int32_t grow = it.r0 + warp;
    const bool live = grow < B.rows;
    double* buf = rowbuf + (size_t)warp * kbuf;
    int shift = 0;
    if (live) {
      const double* xr = src + B.src_off + mixed_offset(grow, B.nr, B.rdim, B.rstride);
      int copied = 0;  // elements of the row now in buf
      if (bulk) {
        const uintptr_t s0 = reinterpret_cast<uintptr_t>(xr);
        const uintptr_t a0 = s0 & ~uintptr_t(15), a1 = (s0 + (uintptr_t)K * 8) & ~uintptr_t(15);
        shift = (int)((s0 - a0) >> 3);
        if (a1 > a0) {
          const uint32_t nbytes = (uint32_t)(a1 - a0);
          copied = (int)(nbytes >> 3) - shift;
          if (lane == 0) {
            sm100::mbar_init(&wbar[warp], 1);
            sm100::fence_mbar_init();
            sm100::mbar_arrive_expect_tx(&wbar[warp], nbytes);
            sm100::bulk_g2s(buf, reinterpret_cast<const void*>(a0), nbytes, &wbar[warp]);
          }
          __syncwarp();
          const long long t0 = clock64();
          bool ok = true;
          while (!sm100::mbar_try_wait(&wbar[warp], 0)) {
            if (clock64() - t0 > wait_cycles) {
              ok = false;
              break;
            }
          }
          if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) atomicExch(status, TAMM_ETIMEOUT);
            const long long t1 = clock64();  // the copy must land before the CTA may exit
            while (!sm100::mbar_try_wait(&wbar[warp], 0) && clock64() - t1 < kDrainWaitCycles) {
            }
            return;
          }
        }
      }
      for (int k = copied + lane; k < K; k += 32) buf[shift + k] = __ldg(xr + k);
      __syncwarp();
    }
    unsigned long long m = 0ull;
    if (live)
      for (int k = lane; k < K; k += 32)
        m = max(m, (unsigned long long)__double_as_longlong(buf[shift + k]) & 0x7FFFFFFFFFFFFFFFull);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (mode == kOzSliceSharedMax) {  // fold the row maximum into its shared slot, write nothing else
      if (lane == 0 && live && m != 0ull) atomicMax(&smax[B.shared_off + grow], m);
      return;
    }
    if (mode == kOzSliceSharedPack) m = live ? smax[B.shared_off + grow] : 0ull;
    int e = kOzExpZero;
    if (m != 0ull) (void)frexp(__longlong_as_double((long long)m), &e);
    if (kFloat && m != 0ull) e = 6;  // floating pieces: unit scale
    const int32_t vrow = B.dst_row0 + grow;  // row of the (possibly concatenated) sliced image
    if (lane == 0) exps[B.exp_off + vrow] = e;
    const int32_t rr = vrow % H;
    uint8_t* rbase = tiles + B.tile_off + (size_t)(vrow / H) * B.k_tiles * tile_bytes + rr * 32;
    const int swz_row = (rr >> 2) & 1;
    const int npairs = B.k_tiles * 8;  // 32-bit words (element pairs) per row of the padded K range
    for (int pw = lane; pw < npairs; pw += 32) {
      uint32_t wd[S];
#pragma unroll
      for (int q = 0; q < S; ++q) wd[q] = 0u;
      const int k = 2 * pw;
      if (e != kOzExpZero && k < K) {
        const double x0 = buf[shift + k];
        const double x1 = k + 1 < K ? buf[shift + k + 1] : 0.0;
        if constexpr (kFloat) pack_float3(x0, x1, wd);
        else pack_digits<S>(x0, x1, e, wd);
      }
      const int wt = pw & 7;
      uint8_t* base = rbase + (size_t)(pw >> 3) * tile_bytes + (((wt >> 2) ^ swz_row) * 16) + (wt & 3) * 4;
#pragma unroll
      for (int q = 0; q < S; ++q) *reinterpret_cast<uint32_t*>(base + (size_t)q * slice_bytes) = wd[q];
    }
    return;
  }

  for (int r = tid; r < nr; r += blockDim.x) {
    const int32_t grow = it.r0 + r;
    rmax[r] = 0ull;
    roff[r] = grow < B.rows ? B.src_off + mixed_offset(grow, B.nr, B.rdim, B.rstride) : -1;
  }
  __syncthreads();

  // ---- general layouts: two passes over global memory (the maximum pass is skipped when the
  // exponents come from the shared slots)
  const int nch = mode == kOzSliceSharedPack ? 0 : (K + 7) / 8;
  for (int u = tid; u < nr * nch; u += blockDim.x) {
    const int r = B.k_contig ? u / nch : u % nr;
    const int ch = B.k_contig ? u % nch : u / nr;
    if (roff[r] < 0) continue;
    int64_t off[8];
    k_offsets8(B, ch * 8, off);
    unsigned long long m = 0ull;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (ch * 8 + j < K) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(__ldg(src + roff[r] + off[j]));
        m = max(m, b & 0x7FFFFFFFFFFFFFFFull);
      }
    }
    if (m) atomicMax(&rmax[r], m);
  }
  __syncthreads();
  if (mode == kOzSliceSharedMax) {
    for (int r = tid; r < nr; r += blockDim.x)
      if (roff[r] >= 0 && rmax[r] != 0ull) atomicMax(&smax[B.shared_off + it.r0 + r], rmax[r]);
    return;
  }
  if (mode == kOzSliceSharedPack) {
    for (int r = tid; r < nr; r += blockDim.x) rmax[r] = roff[r] >= 0 ? smax[B.shared_off + it.r0 + r] : 0ull;
    __syncthreads();
  }
  for (int r = tid; r < nr; r += blockDim.x) {
    int e = kOzExpZero;
    if (rmax[r] != 0ull) (void)frexp(__longlong_as_double((long long)rmax[r]), &e);
    if (kFloat && rmax[r] != 0ull) e = 6;
    rexp[r] = e;
    exps[B.exp_off + B.dst_row0 + it.r0 + r] = e;
  }
  __syncthreads();
  const int nch2 = B.k_tiles * 2;
  for (int u = tid; u < nr * nch2; u += blockDim.x) {
    const int r = u % nr, ch = u / nr;
    uint32_t packed[S][4];
#pragma unroll
    for (int q = 0; q < S; ++q)
#pragma unroll
      for (int w = 0; w < 4; ++w) packed[q][w] = 0u;
    const int e = rexp[r];
    if (roff[r] >= 0 && e != kOzExpZero) {
      int64_t off[8];
      k_offsets8(B, ch * 8, off);
      double xs[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) xs[j] = ch * 8 + j < K ? __ldg(src + roff[r] + off[j]) : 0.0;
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        uint32_t wd[S];
        if constexpr (kFloat) pack_float3(xs[j], xs[j + 1], wd);
        else pack_digits<S>(xs[j], xs[j + 1], e, wd);
#pragma unroll
        for (int q = 0; q < S; ++q) packed[q][j >> 1] = wd[q];
      }
    }
    const int32_t vrow = B.dst_row0 + it.r0 + r;
    const int32_t rr = vrow % H;
    const int64_t tile = (int64_t)(vrow / H) * B.k_tiles + ch / 2;
    const int swz = (ch & 1) ^ ((rr >> 2) & 1);
    uint8_t* base = tiles + B.tile_off + (size_t)tile * tile_bytes + rr * 32 + swz * 16;
#pragma unroll
    for (int q = 0; q < S; ++q)
      *reinterpret_cast<uint4*>(base + (size_t)q * slice_bytes) =
          make_uint4(packed[q][0], packed[q][1], packed[q][2], packed[q][3]);
  }
}

// ======================================================================
// Device: tcgen05 GEMM
// ======================================================================

struct OzParams {
  int64_t n_items;
  int* status;
  long long wait_cycles;  // limit of every dependency wait (the drains before exit keep kDrainWaitCycles)
  int withhold;           // failure-path test hook: CTA 0 skips its first operand copy
  int stages;
  int chunk_tiles;  // K tiles per exact accumulation chunk (<= kOzChunkTiles)
  int n_problems;
  OzProblem problems[kOzMaxProblems];
};

// Problem and work item of global item i (problems hold consecutive item ranges).
__device__ __forceinline__ int problem_of(const OzParams& p, int64_t i) {
  int q = 0;
  while (q + 1 < p.n_problems && i >= p.problems[q + 1].item_begin) ++q;
  return q;
}

template <int S>
__global__ void __launch_bounds__(kThreads, 1) ozaki_gemm_kernel(const __grid_constant__ OzParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int stages = p.stages;
  constexpr uint32_t half_bytes = (uint32_t)S * kOzTileBytesPerSlice;  // A part of a stage (B part: at most this)
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)stages * 2 * half_bytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + stages;
  uint64_t* acc_full = bars + 2 * stages;  // [kAccBufs]
  uint64_t* acc_empty = acc_full + kAccBufs;  // [kAccBufs]
  uint64_t* drain = acc_empty + kAccBufs;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  float* sB = reinterpret_cast<float*>(tmem_holder + 4);  // [2][128] per-task column scales
  int* fref = reinterpret_cast<int*>(sB + 256);            // [128] reference column exponents
  int64_t* col_base = reinterpret_cast<int64_t*>(fref + 128);        // [128] column map of a panel item
  int32_t* col_stride = reinterpret_cast<int32_t*>(col_base + 128);  // [128]

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      sm100::mbar_init(&full[s], 1);
      sm100::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < kAccBufs; ++b) {
      sm100::mbar_init(&acc_full[b], 1);
      sm100::mbar_init(&acc_empty[b], kEpiWarps);
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
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, issued_mask = 0, issued_parity = 0;
      bool withhold = p.withhold != 0 && blockIdx.x == 0;  // test hook: leave the first stage unfilled
      for (int64_t i = blockIdx.x; i < p.n_items && !*abort_flag; i += gridDim.x) {
        const int q = problem_of(p, i);
        const OzItem it = p.problems[q].items[i - p.problems[q].item_begin];
        const OzTask* tasks = p.problems[q].tasks;
        const uint8_t* a_tiles = p.problems[q].a_tiles;
        const uint8_t* b_tiles = p.problems[q].b_tiles;
        const OzGroup g = p.problems[q].groups[it.group];
        const uint32_t b_bytes = (uint32_t)S * 32u * (uint32_t)g.n_tile;
        OzTask tk_next{};
        if (it.t0 < it.t1) tk_next = tasks[it.t0];
        for (int t = it.t0; t < it.t1 && !*abort_flag; ++t) {
          const OzTask tk = tk_next;
          if (t + 1 < it.t1) tk_next = tasks[t + 1];  // loaded while this task's copies issue
          const uint8_t* a = a_tiles + tk.a_off + (size_t)((int64_t)it.mt * tk.k_tiles) * half_bytes;
          const uint8_t* b = b_tiles + tk.b_off + (size_t)((int64_t)it.nt * tk.k_tiles) * b_bytes;
          for (int kt = 0; kt < tk.k_tiles; ++kt) {
            if (!wait_bounded(&empty[stage], phase ^ 1u, abort_flag, p.status, p.wait_cycles)) break;
            if (withhold) {
              // no copy and no arrival: the MMA issuer's wait on this stage cannot end
              withhold = false;
            } else {
              uint8_t* sa = smem + (size_t)stage * 2 * half_bytes;
              sm100::mbar_arrive_expect_tx(&full[stage], half_bytes + b_bytes);
              sm100::bulk_g2s(sa, a + (size_t)kt * half_bytes, half_bytes, &full[stage]);
              sm100::bulk_g2s(sa + half_bytes, b + (size_t)kt * b_bytes, b_bytes, &full[stage]);
              issued_mask |= 1u << stage;
              issued_parity = (issued_parity & ~(1u << stage)) | (phase << stage);
            }
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
      uint32_t phase = 0;
      // accumulator buffers: parity bit and "ever used" bit per buffer, the buffer of the next chunk
      uint32_t acc_parity = 0, acc_used = 0, buf = 0, cur_H = 0;
      bool ok = true;
      for (int64_t i = blockIdx.x; i < p.n_items && ok; i += gridDim.x) {
        const int q = problem_of(p, i);
        const OzItem it = p.problems[q].items[i - p.problems[q].item_begin];
        const OzTask* tasks = p.problems[q].tasks;
        const OzGroup g = p.problems[q].groups[it.group];
        const uint32_t H = (uint32_t)g.n_tile;
        const uint32_t nbuf = acc_buffers(H);
        if (H != cur_H) {
          // another buffer layout: every buffer still being drained must be free first
          for (int b = 0; b < kAccBufs && ok; ++b)
            if ((acc_used >> b) & 1u)
              ok = wait_bounded(&acc_empty[b], ((acc_parity >> b) & 1u) ^ 1u, abort_flag, p.status, p.wait_cycles);
          if (!ok) break;
          buf = 0;
          cur_H = H;
        }
        const int n_valid = min((int)H, g.N - it.nt * (int)H);
        const bool full_tile = n_valid == (int)H;
        // a ragged tile runs unfused with N rounded up to 16 columns
        const uint32_t idesc1 = sm100::idesc_bf16_f32(128, full_tile ? H : (uint32_t)((n_valid + 15) & ~15));
        const uint32_t idesc2 = sm100::idesc_bf16_f32(128, 2u * H);
        int kt_next = it.t0 < it.t1 ? tasks[it.t0].k_tiles : 0;
        int in_chunk = 0;  // position inside the current chunk (no division on the issue path)
        for (int t = it.t0; t < it.t1 && ok; ++t) {
          const int k_tiles = kt_next;
          if (t + 1 < it.t1) kt_next = tasks[t + 1].k_tiles;  // loaded while this task issues
          // a chunk ends with its task, unless the group's tasks share their scaling (then only with the
          // item's last task)
          const bool chunk_ends_with_task = !g.shared || t + 1 == it.t1;
          if (!g.shared) in_chunk = 0;
          for (int kt = 0; kt < k_tiles; ++kt) {
            const bool first = in_chunk == 0;
            const bool last = ++in_chunk == p.chunk_tiles || (kt + 1 == k_tiles && chunk_ends_with_task);
            if (last) in_chunk = 0;
            if (first) {
              if (!wait_bounded(&acc_empty[buf], ((acc_parity >> buf) & 1u) ^ 1u, abort_flag, p.status,
                                p.wait_cycles)) {
                ok = false;
                break;
              }
              sm100::tc_fence_after();
            }
            if (!wait_bounded(&full[stage], phase, abort_flag, p.status, p.wait_cycles)) {
              ok = false;
              break;
            }
            sm100::tc_fence_after();
            // descriptor start addresses count 16-byte units and stay below 2^14, so stage and
            // operand offsets add straight onto the stage-0 descriptor
            const uint64_t a0 = desc_stage0 + (uint64_t)((uint32_t)stage * (2u * half_bytes >> 4));
            const uint64_t b0 = a0 + (half_bytes >> 4);
            const uint32_t tacc = tmem + buf * 4u * H;
            if (full_tile) issue_ops<S, true, 0>(tacc, a0, b0, H, idesc1, idesc2, first);
            else issue_ops<S, false, 0>(tacc, a0, b0, H, idesc1, idesc2, first);
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
    // ----------------------------------------------------------- epilogue
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsHigh));
    const int q = warp & 3;                 // TMEM lane quadrant of this warp
    const int h = (warp - 4) >> 2;          // column half of the item's tile
    const int etid = threadIdx.x - 128;     // 0..255
    const int row = q * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
    uint32_t task_count = 0;
    uint32_t acc_parity = 0, buf = 0;  // same buffer sequence as the MMA issuer
    int cur_H = 0;
    bool ok = true;
    // Every epilogue warp passes the same named barriers on every path (also after a timeout).
    for (int64_t i = blockIdx.x; i < p.n_items; i += gridDim.x) {
      const int q = problem_of(p, i);
      const OzItem it = p.problems[q].items[i - p.problems[q].item_begin];
      const OzTask* tasks = p.problems[q].tasks;
      const int32_t* a_exp = p.problems[q].a_exp;
      const int32_t* b_exp = p.problems[q].b_exp;
      const OzGroup g = p.problems[q].groups[it.group];
      const int H = g.n_tile;
      const int n_valid = min(H, g.N - it.nt * H);
      // the two column halves split the tile's H columns evenly (H is a multiple of 16), so a narrow tile
      // (H = 80: 40 + 40) does not leave one half of the epilogue with most of the drain
      const int c0 = h * (H >> 1), c_end = min(c0 + (H >> 1), n_valid);
      const uint32_t nbuf = acc_buffers((uint32_t)H);
      if (H != cur_H) {
        buf = 0;
        cur_H = H;
      }
      const int64_t arow = (int64_t)it.mt * kOzTileM + row, bcol = (int64_t)it.nt * H + etid;
      const bool has_col = etid < H;
      // reference exponents: the maxima over the group's tasks (loads unrolled so that several
      // are in flight at once)
      int Eref = kOzExpZero, F = kOzExpZero;
      {
        int t = it.t0;
        for (; t + 4 <= it.t1; t += 4) {
          int ea4[4], eb4[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            ea4[u] = a_exp[tasks[t + u].a_exp + arow];
            eb4[u] = has_col ? b_exp[tasks[t + u].b_exp + bcol] : kOzExpZero;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            Eref = max(Eref, ea4[u]);
            F = max(F, eb4[u]);
          }
        }
        for (; t < it.t1; ++t) {
          Eref = max(Eref, a_exp[tasks[t].a_exp + arow]);
          if (has_col) F = max(F, b_exp[tasks[t].b_exp + bcol]);
        }
      }
      epi_barrier();  // the previous item's output writes (which read fref and the column map) are done
      if (has_col) fref[etid] = F;
      if (g.colmap >= 0 && has_col && bcol < g.N) {
        col_base[etid] = p.problems[q].col_base[g.colmap + bcol];
        col_stride[etid] = p.problems[q].col_stride[g.colmap + bcol];
      }
      float hi[64], lo[64];
#pragma unroll
      for (int j = 0; j < 64; ++j) hi[j] = lo[j] = 0.0f;
      // exponents of the next task are loaded one task ahead, while this task's chunks drain
      int ea_next = kOzExpZero, eb_next = kOzExpZero, kt_next = 0;
      if (it.t0 < it.t1) {
        const OzTask t0 = tasks[it.t0];
        ea_next = a_exp[t0.a_exp + arow];
        if (has_col) eb_next = b_exp[t0.b_exp + bcol];
        kt_next = t0.k_tiles;
      }
      // shared scaling: the item's tasks are one sequence of chunks with the first task's scales (every
      // task has the same exponents), as the MMA issuer chunks them
      int shared_tiles = 0;
      if (g.shared)
        for (int t = it.t0; t < it.t1; ++t) shared_tiles += tasks[t].k_tiles;
      const int t_end = g.shared ? min(it.t1, it.t0 + 1) : it.t1;
      for (int t = it.t0; t < t_end; ++t, ++task_count) {
        const int ea = ea_next, eb = eb_next, k_tiles = g.shared ? shared_tiles : kt_next;
        if (t + 1 < t_end) {
          const OzTask tn = tasks[t + 1];
          ea_next = a_exp[tn.a_exp + arow];
          if (has_col) eb_next = b_exp[tn.b_exp + bcol];
          kt_next = tn.k_tiles;
        }
        float* sbuf = sB + (task_count & 1u) * 128;
        epi_barrier();  // fref is set, and sbuf's previous readers (two tasks ago) are done
        if (has_col) sbuf[etid] = (eb == kOzExpZero) ? 0.0f : pow2f(eb - fref[etid]);
        epi_barrier();
        const float sA = (ea == kOzExpZero) ? 0.0f : pow2f(ea - Eref);
        const int n_chunks = ok ? (k_tiles + p.chunk_tiles - 1) / p.chunk_tiles : 0;
        for (int ck = 0; ck < n_chunks; ++ck) {
          if (!wait_bounded(&acc_full[buf], (acc_parity >> buf) & 1u, abort_flag, p.status, p.wait_cycles)) {
            ok = false;
            break;
          }
          sm100::tc_fence_after();
          const uint32_t tb = trow + buf * 4u * (uint32_t)H;
#pragma unroll
          for (int g8 = 0; g8 < 8; ++g8) {
            const int col = c0 + 8 * g8;
            if (col >= c_end) break;  // this half's end; columns past a ragged tile's width were not computed
            float r0[8], r1[8], r2[8], r3[8];
            sm100::tmem_ld8(tb + 0 * H + col, r0);
            sm100::tmem_ld8(tb + 1 * H + col, r1);
            sm100::tmem_ld8(tb + 2 * H + col, r2);
            // with S < 4 no product has k + l >= 5: region 3 is never written and holds stale
            // TMEM contents of an earlier kernel, so it must not be read
            if constexpr (S >= 4) {
              sm100::tmem_ld8(tb + 3 * H + col, r3);
            } else {
#pragma unroll
              for (int j = 0; j < 8; ++j) r3[j] = 0.0f;
            }
            sm100::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 8; ++j)
              fold(hi[8 * g8 + j], lo[8 * g8 + j], r0[j], r1[j], r2[j], r3[j], sA * sbuf[col + j]);
          }
          sm100::tc_fence_before();
          __syncwarp();
          if (lane == 0) sm100::mbar_arrive(&acc_empty[buf]);
          acc_parity ^= 1u << buf;
          buf = buf + 1 == nbuf ? 0u : buf + 1;
        }
      }
      if (it.t0 == it.t1) epi_barrier();  // keep the fref barrier count uniform
      if (ok) {
        const int grow = it.mt * kOzTileM + row;
        if (grow < g.M && it.split >= 0) {
          // a partial over one summed range of a split group: its FP64 value, dense [split][M][N]
          double* wrow = p.problems[q].ws + g.ws_off + ((int64_t)it.split * g.M + grow) * g.N + (int64_t)it.nt * H;
#pragma unroll
          for (int j = 0; j < 64; ++j) {
            const int col = c0 + j;
            if (col < c_end) {
              double v = 0.0;
              if (Eref != kOzExpZero && fref[col] != kOzExpZero) {
                const int sc = Eref + fref[col] - 12;
                double dh, dl;
                if (f2d_scaled(hi[j], sc, false, dh) && f2d_scaled(lo[j], sc, false, dl)) v = dh + dl;
                else v = ((double)hi[j] + (double)lo[j]) * pow2d(sc);
              }
              wrow[col] = v;
            }
          }
        } else if (grow < g.M) {
          // one output block: row-major M x N at c_off; a column panel: column c of block m at
          // col_base[c] + row * col_stride[c]
          double* c = p.problems[q].c;
          double* crow = c + g.c_off + (int64_t)grow * g.N + (int64_t)it.nt * H;
          const double alpha = p.problems[q].alpha, beta = p.problems[q].beta;
          const bool panel = g.colmap >= 0;
          // alpha = +-2^ae folds into the exponent: alpha 2^sc (hi + lo) costs one FP64 add, and
          // C + that one more; the result is the same rounding as the FP64 route below
          const int ae = p.problems[q].alpha_exp;
          const bool a_p2 = p.problems[q].alpha_pow2 != 0, a_neg = alpha < 0.0;
#pragma unroll
          for (int j = 0; j < 64; ++j) {
            const int col = c0 + j;
            if (col < c_end) {
              double av = 0.0;  // alpha * (product)
              if (Eref != kOzExpZero && fref[col] != kOzExpZero) {
                const int sc = Eref + fref[col] - 12;
                double dh, dl;
                if (a_p2 && f2d_scaled(hi[j], sc + ae, a_neg, dh) && f2d_scaled(lo[j], sc + ae, a_neg, dl))
                  av = dh + dl;
                else
                  av = alpha * (((double)hi[j] + (double)lo[j]) * pow2d(sc));
              } else {
                av = alpha * 0.0;
              }
              double* cp = panel ? c + col_base[col] + (int64_t)grow * col_stride[col] : crow + col;
              *cp = beta != 0.0 ? fma(beta, *cp, av) : av;
            }
          }
        }
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    sm100::tc_fence_after();
    sm100::tmem_dealloc(tmem, 512);
  }
}

// Sum of a split group's partials in range order, then C = beta C + alpha sum.
__global__ void __launch_bounds__(256) ozaki_reduce_kernel(const OzReduceItem* __restrict__ items,
                                                           const OzGroup* __restrict__ groups,
                                                           const double* __restrict__ ws, double* __restrict__ c,
                                                           const int64_t* __restrict__ col_base,
                                                           const int32_t* __restrict__ col_stride, double alpha,
                                                           double beta) {
  const OzReduceItem it = items[blockIdx.x];
  const OzGroup g = groups[it.group];
  const int64_t MN = (int64_t)g.M * g.N;
  for (int64_t e = it.e0 + threadIdx.x; e < it.e1; e += blockDim.x) {
    double v = 0.0;
    for (int sp = 0; sp < g.nsplit; ++sp) v += ws[g.ws_off + sp * MN + e];
    const int64_t row = e / g.N, col = e - row * g.N;
    double* cp = g.colmap >= 0 ? c + col_base[g.colmap + col] + row * col_stride[g.colmap + col] : c + g.c_off + e;
    *cp = beta != 0.0 ? fma(beta, *cp, alpha * v) : alpha * v;
  }
}

}  // namespace

// ======================================================================
// Launchers
// ======================================================================

// Kernel attributes are per device: the one-time setup is tracked per device ordinal.
constexpr int kMaxDevices = 64;
static std::mutex g_attr_mutex;

template <int S, bool kFloat = false>
static cudaError_t slice_dispatch(tamm_ctx* ctx, const double* src, const SliceBlock* blocks, const SliceItem* items,
                                  int64_t n_items, uint8_t* tiles, int32_t* exps, int warps, int kbuf, int mode,
                                  unsigned long long* smax) {
  static size_t attr_bytes[kMaxDevices] = {};  // dynamic shared memory opted in so far, per device
  const size_t smem = (size_t)warps * kbuf * sizeof(double);
  if (ctx->device < 0 || ctx->device >= kMaxDevices) return cudaErrorInvalidDevice;
  {
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    if (smem > attr_bytes[ctx->device]) {
      cudaError_t e = cudaFuncSetAttribute(ozaki_slice_kernel<S, kFloat>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr_bytes[ctx->device] = smem;
    }
  }
  const int bulk = (reinterpret_cast<uintptr_t>(src) & 15) == 0 ? 1 : 0;
  ozaki_slice_kernel<S, kFloat><<<(unsigned)n_items, 32 * warps, smem, ctx->stream>>>(
      src, blocks, items, tiles, exps, kbuf, bulk, ctx->d_status, ctx->oz_wait_cycles, mode, smax);
  return cudaGetLastError();
}

cudaError_t launch_ozaki_slice(tamm_ctx* ctx, const double* src, const SliceBlock* blocks, const SliceItem* items,
                               int64_t n_items, int S, bool float_split, uint8_t* tiles, int32_t* exps, int warps,
                               int kbuf, int mode, unsigned long long* smax) {
  if (n_items == 0) return cudaSuccess;
  if (warps < 1 || warps > 8 || kbuf < 2 || (size_t)warps * kbuf * sizeof(double) > kOzSliceSmemMax)
    return cudaErrorInvalidValue;
  if (mode != kOzSliceOwn && (!smax || float_split)) return cudaErrorInvalidValue;
  kernel_begin(ctx, TAMM_KERNEL_SLICE);
  cudaError_t e = cudaErrorInvalidValue;
  if (float_split) {
    if (S == 3) e = slice_dispatch<3, true>(ctx, src, blocks, items, n_items, tiles, exps, warps, kbuf, mode, smax);
    kernel_end(ctx, TAMM_KERNEL_SLICE);
    return e;
  }
  switch (S) {
    case 3: e = slice_dispatch<3>(ctx, src, blocks, items, n_items, tiles, exps, warps, kbuf, mode, smax); break;
    case 4: e = slice_dispatch<4>(ctx, src, blocks, items, n_items, tiles, exps, warps, kbuf, mode, smax); break;
    case 5: e = slice_dispatch<5>(ctx, src, blocks, items, n_items, tiles, exps, warps, kbuf, mode, smax); break;
    case 6: e = slice_dispatch<6>(ctx, src, blocks, items, n_items, tiles, exps, warps, kbuf, mode, smax); break;
    case 7: e = slice_dispatch<7>(ctx, src, blocks, items, n_items, tiles, exps, warps, kbuf, mode, smax); break;
    case 8: e = slice_dispatch<8>(ctx, src, blocks, items, n_items, tiles, exps, warps, kbuf, mode, smax); break;
  }
  kernel_end(ctx, TAMM_KERNEL_SLICE);
  return e;
}

static int oz_stages(int S) { return std::min(6, (192 * 1024) / (2 * S * kOzTileBytesPerSlice)); }

static size_t oz_smem_bytes(int S) {
  return (size_t)oz_stages(S) * 2 * S * kOzTileBytesPerSlice + 1024 + 4096;
}

template <int S>
static cudaError_t gemm_dispatch(tamm_ctx* ctx, const OzParams& p, int grid) {
  static bool ready[kMaxDevices] = {};
  const size_t smem = oz_smem_bytes(S);
  if (ctx->device < 0 || ctx->device >= kMaxDevices) return cudaErrorInvalidDevice;
  {
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    if (!ready[ctx->device]) {
      cudaFuncAttributes fa;
      cudaError_t e = cudaFuncGetAttributes(&fa, ozaki_gemm_kernel<S>);
      if (e != cudaSuccess) return e;
      // setmaxnreg.inc would wait forever if the launch pool were too small
      if (fa.numRegs < kRegsLaunchNeeded) return cudaErrorLaunchOutOfResources;
      e = cudaFuncSetAttribute(ozaki_gemm_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      ready[ctx->device] = true;
    }
  }
  ozaki_gemm_kernel<S><<<(unsigned)grid, kThreads, smem, ctx->stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_ozaki_reduce(tamm_ctx* ctx, const OzReduceItem* items, int64_t n_items, const OzGroup* groups,
                                const double* ws, double* c, const int64_t* col_base, const int32_t* col_stride,
                                double alpha, double beta) {
  if (n_items == 0) return cudaSuccess;
  kernel_begin(ctx, TAMM_KERNEL_SPLIT_REDUCE);
  ozaki_reduce_kernel<<<(unsigned)n_items, 256, 0, ctx->stream>>>(items, groups, ws, c, col_base, col_stride, alpha,
                                                                   beta);
  kernel_end(ctx, TAMM_KERNEL_SPLIT_REDUCE);
  return cudaGetLastError();
}

cudaError_t launch_ozaki_gemm(tamm_ctx* ctx, OzProblem* problems, const int64_t* n_items_per_problem,
                              int n_problems, int S, int chunk_tiles, bool persistent) {
  if (chunk_tiles < 1 || chunk_tiles > kOzChunkTiles) return cudaErrorInvalidValue;
  if (n_problems < 1 || n_problems > kOzMaxProblems) return cudaErrorInvalidValue;
  int64_t n_items = 0;
  for (int i = 0; i < n_problems; ++i) {
    problems[i].item_begin = n_items;
    n_items += n_items_per_problem[i];
  }
  if (n_items == 0) return cudaSuccess;
  OzParams p{};  // the whole problem table travels as the kernel's parameter block
  p.n_items = n_items;
  p.status = ctx->d_status;
  p.wait_cycles = ctx->oz_wait_cycles;
  p.withhold = ctx->oz_test_withhold;
  ctx->oz_test_withhold = 0;  // the hook applies to one launch
  p.stages = oz_stages(S);
  p.chunk_tiles = chunk_tiles;
  p.n_problems = n_problems;
  for (int i = 0; i < n_problems; ++i) p.problems[i] = problems[i];
  // persistent: one CTA per SM walks items round-robin; otherwise one CTA per item
  const int grid = persistent ? (int)std::min<int64_t>(n_items, std::max(1, ctx->sm_count))
                                      : (int)std::min<int64_t>(n_items, 0x7FFFFFFF);
  kernel_begin(ctx, TAMM_KERNEL_GEMM_OZ);
  cudaError_t e = cudaErrorInvalidValue;
  switch (S) {
    case 3: e = gemm_dispatch<3>(ctx, p, grid); break;
    case 4: e = gemm_dispatch<4>(ctx, p, grid); break;
    case 5: e = gemm_dispatch<5>(ctx, p, grid); break;
    case 6: e = gemm_dispatch<6>(ctx, p, grid); break;
    case 7: e = gemm_dispatch<7>(ctx, p, grid); break;
    case 8: e = gemm_dispatch<8>(ctx, p, grid); break;
  }
  kernel_end(ctx, TAMM_KERNEL_GEMM_OZ);
  return e;
}

// ======================================================================
// Host plan
// ======================================================================

// Slicing launch shape and items for an operand's records; record i covers
// image rows [dst_row0, dst_row0 + extent[i]) (rows past its own are zero).
// Warp row buffers hold K + 2 doubles (room for the aligned-down start) of
// the longest dense row; as many warps (<= 8) as fit the shared-memory
// budget.  Rows too long for one warp buffer go through the general path.
void oz_slicing_items(std::vector<SliceBlock>& recs, const std::vector<int32_t>& extent,
                      std::vector<SliceItem>& items, int& warps, int& kbuf) {
  int64_t kmax = 0;
  for (const SliceBlock& B : recs)
    if (B.k_dense) kmax = std::max<int64_t>(kmax, B.K);
  kbuf = (int)((kmax + 2 + 1) & ~int64_t(1));
  warps = (int)std::min<int64_t>(8, (int64_t)kOzSliceSmemBudget / ((int64_t)kbuf * 8));
  if (warps < 1) {
    for (SliceBlock& B : recs) B.k_dense = 0;
    warps = 8;
    kbuf = 2;
  }
  for (size_t i = 0; i < recs.size(); ++i) {
    const SliceBlock& B = recs[i];
    // rows per slicing CTA: one per warp for a dense summed range, else enough rows for every
    // thread to have work, at least 32 for coalescing along rows
    int R;
    if (B.k_dense) {
      R = warps;
    } else {
      R = 32;
      while (R < kOzSliceMaxRows && (int64_t)R * ((B.K + 7) / 8) < 32 * warps * 4) R *= 2;
    }
    for (int32_t r = 0; r < extent[i]; r += R)
      items.push_back({(int32_t)i, r, std::min<int32_t>(R, extent[i] - r), 0});
  }
}

// Every block pair sums at most kOzFaMaxK indices and every output block has at most kOzFaMaxN columns.
bool oz_fused_eligible(const ContractLayout& lay) {
  if (lay.free_left.size() > 4 || lay.free_right.size() > 4 || lay.summed.size() > 4) return false;
  if (lay.groups.empty()) return false;
  for (const auto& g : lay.groups)
    if (g.N < 1 || g.N > kOzFaMaxN || g.M < 1 || g.M > (int64_t(1) << 30)) return false;
  for (const auto& t : lay.tasks)
    if (t.K < 1 || t.K > kOzFaMaxK) return false;
  return true;
}

struct OzakiPlan : Plan {
  ContractLayout lay;
  int S;
  SliceBlock* d_sa = nullptr;
  SliceItem* d_ia = nullptr;
  int64_t n_ia = 0;
  SliceBlock* d_sb = nullptr;
  SliceItem* d_ib = nullptr;
  int64_t n_ib = 0;
  OzGroup* d_groups = nullptr;
  OzTask* d_tasks = nullptr;
  OzItem* d_items = nullptr;
  int64_t* d_col_base = nullptr;
  int32_t* d_col_stride = nullptr;
  int64_t n_items = 0;
  OzReduceItem* d_red = nullptr;  // reduction chunks of the split groups
  int64_t n_red = 0;
  std::unique_ptr<AddPlan> perm_out;
  size_t off_ta = 0, off_tb = 0, off_ea = 0, off_eb = 0, off_x = 0, off_ws = 0, scratch_bytes = 0;
  // shared scaling: one exponent per output row (A operand rows with the same free-left tiles) and per
  // output column (B operand rows with the same free-right tiles), over every block that feeds it
  bool shared = false;
  int64_t slots_a = 0, slots_b = 0;
  size_t off_sa = 0, off_sb = 0;
  int warps_a = 8, kbuf_a = 2, warps_b = 8, kbuf_b = 2;  // slicing launch shapes
  // the A-slicing GEMM (short summed ranges, narrow outputs): A stays FP64 (d_sa holds its block
  // geometry only), B is sliced into one image per block, C is written through its own strides
  bool fused = false;
  FaGroup* d_fg = nullptr;
  FaTask* d_ft = nullptr;
  FaItem* d_fi = nullptr;
  int64_t n_fi = 0;

  // Geometry of block b of the GEMM-order operand `gemm` (blocks of `native`
  // permuted by perm); row modes are [r0, r0+nr), summed modes [k0, k0+nk).
  // The image layout fields (tile_rows, row_tiles, tile_off, exp_off,
  // dst_row0) are filled by the caller.
  static SliceBlock block_geometry(const tamm_tensor& native, const tamm_tensor& gemm, const std::vector<int>& perm,
                                   int r0, int nr, int k0, int nk, int64_t b) {
    const int64_t* gt = &gemm.tiles[(size_t)(b * gemm.nm)];
    int64_t nt[kMaxModes];
    for (int m = 0; m < gemm.nm; ++m) nt[perm[m]] = gt[m];
    const int64_t nb = native.find(nt);
    if (nb < 0) throw Error(TAMM_EINVAL, "ozaki: operand block lookup failed");
    int64_t stride[kMaxModes], s = 1;
    for (int q = native.nm - 1; q >= 0; --q) {
      stride[q] = s;
      s *= native.sp[q]->size[(size_t)nt[q]];
    }
    SliceBlock B;
    memset(&B, 0, sizeof(B));
    B.src_off = native.off[(size_t)nb];
    if (nr > 4 || nk > 4) throw Error(TAMM_EUNSUPPORTED, "ozaki: at most 4 free and 4 summed modes per operand");
    B.nr = nr;
    B.nk = nk;
    int64_t rows = 1, K = 1;
    for (int m = 0; m < nr; ++m) {
      B.rdim[m] = (int32_t)gemm.sp[r0 + m]->size[(size_t)gt[r0 + m]];
      B.rstride[m] = (int32_t)stride[perm[r0 + m]];
      rows *= B.rdim[m];
    }
    for (int m = 0; m < nk; ++m) {
      B.kdim[m] = (int32_t)gemm.sp[k0 + m]->size[(size_t)gt[k0 + m]];
      B.kstride[m] = (int32_t)stride[perm[k0 + m]];
      K *= B.kdim[m];
    }
    if (rows > (1 << 30) || K > (1 << 30)) throw Error(TAMM_EUNSUPPORTED, "ozaki: block too large");
    B.rows = (int32_t)rows;
    B.K = (int32_t)K;
    B.k_tiles = (int32_t)((K + kOzTileK - 1) / kOzTileK);
    B.k_contig = (nk > 0 && B.kstride[nk - 1] == 1) ? 1 : 0;
    if (nk == 0) B.k_contig = 1;
    int64_t st = 1;
    B.k_dense = 1;
    for (int m = nk - 1; m >= 0; --m) {
      if (B.kstride[m] != st) B.k_dense = 0;
      st *= B.kdim[m];
    }
    return B;
  }

  bool fused_eligible() const { return oz_fused_eligible(lay); }

  void build_fused(const tamm_tensor& Lg, const tamm_tensor& Rg, const std::vector<int>& perm_l,
                   const std::vector<int>& perm_r, const std::vector<int>& perm_c) {
    fused = true;
    const int nfl = (int)lay.free_left.size(), nfr = (int)lay.free_right.size(), nk = (int)lay.summed.size();
    std::vector<SliceBlock> sa;  // FP64 geometry of every A block (no image)
    for (int64_t b = 0; b < Lg.n_blocks; ++b) sa.push_back(block_geometry(*lay.left, Lg, perm_l, 0, nfl, nfl, nk, b));
    std::vector<SliceBlock> sb;
    std::vector<int32_t> ext_b;
    std::map<int64_t, size_t> image_of;  // right block -> its record in sb
    int64_t tb = 0, eb = 0;
    const tamm_tensor& O = lay.out_gemm_tensor();
    std::vector<FaGroup> fg;
    std::vector<FaTask> ft;
    std::vector<FaItem> fi;
    for (size_t gi = 0; gi < lay.groups.size(); ++gi) {
      const auto& g = lay.groups[gi];
      const int H = (int)((g.N + 15) / 16 * 16);
      const SliceBlock Cg = block_geometry(*lay.c, O, perm_c, 0, nfl, nfl, nfr, g.out_block);
      FaGroup G;
      memset(&G, 0, sizeof(G));
      G.c_off = Cg.src_off;
      G.M = (int32_t)g.M;
      G.N = (int32_t)g.N;
      G.n_tile = H;
      G.nr = Cg.nr;
      G.nc = Cg.nk;
      for (int m = 0; m < 4; ++m) {
        G.rdim[m] = Cg.rdim[m];
        G.rstride[m] = Cg.rstride[m];
        G.cdim[m] = Cg.kdim[m];
        G.cstride[m] = Cg.kstride[m];
      }
      G.task_begin = (int32_t)ft.size();
      for (int64_t t = g.task_begin; t < g.task_end; ++t) {
        const auto& tk = lay.tasks[(size_t)t];
        auto it = image_of.find(tk.right_block);
        if (it == image_of.end()) {
          SliceBlock R = block_geometry(*lay.right, Rg, perm_r, nk, nfr, 0, nk, tk.right_block);
          if (R.rows != g.N) throw Error(TAMM_EINVAL, "ozaki: B block rows differ from the output columns");
          R.tile_rows = H;
          R.row_tiles = 1;
          R.tile_off = tb;
          R.exp_off = eb;
          R.dst_row0 = 0;
          R.shared_off = 0;
          tb += (int64_t)R.k_tiles * S * H * 32;
          eb += H;
          it = image_of.emplace(tk.right_block, sb.size()).first;
          sb.push_back(R);
          ext_b.push_back(H);
        }
        const SliceBlock& R = sb[it->second];
        const SliceBlock& A_ = sa[(size_t)tk.left_block];
        if (A_.k_tiles != R.k_tiles || R.tile_rows != H || A_.rows != g.M)
          throw Error(TAMM_EINVAL, "ozaki: block pair shapes disagree");
        ft.push_back({R.tile_off, R.exp_off, (int32_t)tk.left_block, A_.k_tiles});
      }
      G.task_end = (int32_t)ft.size();
      fg.push_back(G);
      for (int32_t mt = 0; mt < (G.M + kOzTileM - 1) / kOzTileM; ++mt) fi.push_back({(int32_t)gi, mt});
    }
    std::vector<SliceItem> ib;
    oz_slicing_items(sb, ext_b, ib, warps_b, kbuf_b);
    auto align = [](size_t x) { return (x + 1023) & ~size_t(1023); };
    off_tb = 0;
    scratch_bytes = align((size_t)tb);
    off_eb = scratch_bytes;
    scratch_bytes += align((size_t)std::max<int64_t>(eb, 1) * 4);
    n_ib = (int64_t)ib.size();
    n_fi = (int64_t)fi.size();
    d_sa = upload(sa);
    d_sb = upload(sb);
    d_ib = upload(ib);
    d_fg = upload(fg);
    d_ft = upload(ft);
    d_fi = upload(fi);
  }

  OzakiPlan(tamm_ctx* c, const tamm_tensor* C, const char* lc, const tamm_tensor* A, const char* la,
            const tamm_tensor* B, const char* lb, int slices, int tile_policy, bool panels, bool allow_split,
            bool shared_scale, bool fused_ok)
      : Plan(c), lay(c, C, lc, A, la, B, lb), S(slices), shared(shared_scale) {
    std::map<std::vector<int64_t>, int64_t> slot_a, slot_b;  // free tile tuple -> first slot
    auto slot_of = [](std::map<std::vector<int64_t>, int64_t>& m, int64_t& n, std::vector<int64_t> key,
                      int64_t rows) {
      auto it = m.find(key);
      if (it != m.end()) return it->second;
      const int64_t base = n;
      m[key] = base;
      n += rows;
      return base;
    };
    const int nfl = (int)lay.free_left.size(), nfr = (int)lay.free_right.size(), nk = (int)lay.summed.size();
    auto perm_of = [](const std::string& need, const std::string& have) {
      std::vector<int> p(need.size());
      for (size_t m = 0; m < need.size(); ++m) p[m] = (int)have.find(need[m]);
      return p;
    };
    const tamm_tensor& Lg = lay.left_gemm();
    const tamm_tensor& Rg = lay.right_gemm();
    const std::vector<int> perm_l = perm_of(lay.need_left, lay.label_left);
    const std::vector<int> perm_r = perm_of(lay.need_right, lay.label_right);
    if (fused_ok && !shared && fused_eligible()) {
      build_fused(Lg, Rg, perm_l, perm_r, perm_of(lay.out_gemm, lay.label_c));
      return;
    }

    // A operand: one image per block, 128-row tiles
    std::vector<SliceBlock> sa;
    std::vector<int32_t> ext_a;
    int64_t ta = 0, ea = 0;
    for (int64_t b = 0; b < Lg.n_blocks; ++b) {
      SliceBlock R = block_geometry(*lay.left, Lg, perm_l, 0, nfl, nfl, nk, b);
      R.tile_rows = kOzTileM;
      R.row_tiles = (R.rows + kOzTileM - 1) / kOzTileM;
      R.tile_off = ta;
      R.exp_off = ea;
      R.dst_row0 = 0;
      {
        const int64_t* gt = &Lg.tiles[(size_t)(b * Lg.nm)];
        R.shared_off = slot_of(slot_a, slots_a, std::vector<int64_t>(gt, gt + nfl), R.rows);
      }
      ta += (int64_t)R.row_tiles * R.k_tiles * S * kOzTileM * 32;
      ea += (int64_t)R.row_tiles * kOzTileM;
      sa.push_back(R);
      ext_a.push_back(R.row_tiles * kOzTileM);
    }

    // Column panels: output blocks with the same rows and the same A block in every task (the
    // same summed tiles) share every A tile, so their columns are concatenated into one wider
    // output; each task's B blocks become one image with the members' rows stacked.
    std::vector<std::vector<int>> members;
    {
      std::map<std::vector<int64_t>, int> panel_of;
      for (size_t gi = 0; gi < lay.groups.size(); ++gi) {
        const auto& g = lay.groups[gi];
        std::vector<int64_t> key{g.M};
        for (int64_t t = g.task_begin; t < g.task_end; ++t) key.push_back(lay.tasks[(size_t)t].left_block);
        if (!panels) key.push_back(-1 - (int64_t)gi);  // every group alone
        auto it = panel_of.find(key);
        if (it == panel_of.end()) {
          panel_of[key] = (int)members.size();
          members.push_back({(int)gi});
        } else {
          members[(size_t)it->second].push_back((int)gi);
        }
      }
    }
    // B images: one per distinct (task, member B blocks) list
    std::vector<SliceBlock> sb;
    std::vector<int32_t> ext_b;
    struct Image {
      int64_t tile_off, exp_off;
      int32_t k_tiles;
    };
    std::vector<Image> images;
    std::map<std::vector<int64_t>, int> image_of;
    int64_t tb = 0, eb = 0;
    const tamm_tensor& O = lay.out_gemm_tensor();
    std::vector<OzGroup> groups;
    std::vector<OzTask> tasks;
    std::vector<int64_t> col_base;
    std::vector<int32_t> col_stride;
    std::vector<int64_t> group_k;  // summed extent per output group
    for (const auto& mem : members) {
      const auto& g0 = lay.groups[(size_t)mem[0]];
      int64_t Np = 0;
      for (int gi : mem) Np += lay.groups[(size_t)gi].N;
      if (Np > (int64_t(1) << 30)) throw Error(TAMM_EUNSUPPORTED, "ozaki: output panel too wide");
      const int H = oz_tile_rows(Np, tile_policy);
      const int32_t row_tiles = (int32_t)((Np + H - 1) / H);
      OzGroup gg;
      gg.M = (int32_t)g0.M;
      gg.N = (int32_t)Np;
      gg.n_tile = H;
      gg.nsplit = 1;
      gg.shared = shared ? 1 : 0;
      gg.pad = 0;
      gg.ws_off = 0;
      if (mem.size() == 1) {
        gg.c_off = O.off[(size_t)g0.out_block];
        gg.colmap = -1;
      } else {
        gg.c_off = 0;
        gg.colmap = (int64_t)col_base.size();
        for (int gi : mem) {
          const auto& g = lay.groups[(size_t)gi];
          for (int64_t cc = 0; cc < g.N; ++cc) {
            col_base.push_back(O.off[(size_t)g.out_block] + cc);
            col_stride.push_back((int32_t)g.N);
          }
        }
      }
      gg.task_begin = (int32_t)tasks.size();
      const int64_t ntask = g0.task_end - g0.task_begin;
      int64_t Ksum = 0;
      for (int64_t t = 0; t < ntask; ++t) {
        const auto& tk0 = lay.tasks[(size_t)(g0.task_begin + t)];
        std::vector<int64_t> key{(int64_t)H};
        for (int gi : mem) key.push_back(lay.tasks[(size_t)(lay.groups[(size_t)gi].task_begin + t)].right_block);
        auto it = image_of.find(key);
        int img;
        if (it != image_of.end()) {
          img = it->second;
        } else {
          img = (int)images.size();
          image_of[key] = img;
          Image im{tb, eb, 0};
          int32_t row0 = 0;
          for (size_t m = 0; m < mem.size(); ++m) {
            SliceBlock R = block_geometry(*lay.right, Rg, perm_r, nk, nfr, 0, nk, key[m + 1]);
            if (m == 0) im.k_tiles = R.k_tiles;
            if (R.k_tiles != im.k_tiles) throw Error(TAMM_EINVAL, "ozaki: K mismatch in a panel");
            R.tile_rows = H;
            R.row_tiles = row_tiles;
            R.tile_off = im.tile_off;
            R.exp_off = im.exp_off;
            R.dst_row0 = row0;
            {
              const int64_t* gt = &Rg.tiles[(size_t)(key[m + 1] * Rg.nm)];
              R.shared_off = slot_of(slot_b, slots_b, std::vector<int64_t>(gt + nk, gt + nk + nfr), R.rows);
            }
            const bool last = m + 1 == mem.size();
            ext_b.push_back(last ? row_tiles * H - row0 : R.rows);
            row0 += R.rows;
            sb.push_back(R);
          }
          if (row0 != Np) throw Error(TAMM_EINVAL, "ozaki: B block rows differ from the output columns");
          tb += (int64_t)row_tiles * im.k_tiles * S * H * 32;
          eb += (int64_t)row_tiles * H;
          images.push_back(im);
        }
        const SliceBlock& A_ = sa[(size_t)tk0.left_block];
        const Image& im = images[(size_t)img];
        if (A_.k_tiles != im.k_tiles) throw Error(TAMM_EINVAL, "ozaki: K mismatch");
        tasks.push_back({A_.tile_off, im.tile_off, A_.exp_off, im.exp_off, A_.k_tiles, 0});
        Ksum += (int64_t)A_.k_tiles * kOzTileK;
      }
      // the double-float accumulator holds sums of |G0| <= Ksum * 64 * 64 far below 2^40
      if (Ksum > (int64_t(1) << 26)) throw Error(TAMM_EUNSUPPORTED, "ozaki: summed extent too large");
      gg.task_end = (int32_t)tasks.size();
      groups.push_back(gg);
      group_k.push_back(Ksum);
    }
    std::vector<SliceItem> ia, ib;
    oz_slicing_items(sa, ext_a, ia, warps_a, kbuf_a);
    oz_slicing_items(sb, ext_b, ib, warps_b, kbuf_b);

    auto align = [](size_t x) { return (x + 1023) & ~size_t(1023); };
    off_ta = 0;
    scratch_bytes = align((size_t)ta);
    off_tb = scratch_bytes;
    scratch_bytes += align((size_t)tb);
    off_ea = scratch_bytes;
    scratch_bytes += align((size_t)ea * 4);
    off_eb = scratch_bytes;
    scratch_bytes += align((size_t)eb * 4);
    if (lay.out_perm) {
      const char* ls[1] = {lay.out_gemm.c_str()};
      perm_out.reset(new AddPlan(c, *C, lay.label_c.c_str(), *lay.out_perm, 1, ls));
      off_x = scratch_bytes;
      scratch_bytes += align((size_t)lay.out_perm->n_elems * 8);
    }
    // Split summed ranges when the contraction has too few output tiles to fill the GPU (two
    // 128 x 128 tiles per SM): every group's tasks are cut into the same number of consecutive
    // ranges (at most 8, at most one per task).  The count depends only on the block structure,
    // so it is the same whatever the tile policy, grid kind or panel setting.
    int64_t base_tiles = 0;
    for (const auto& g : lay.groups) base_tiles += ((g.M + 127) / 128) * ((g.N + 127) / 128);
    const int64_t target = 2 * std::max(1, c->sm_count);
    const int split = !allow_split || base_tiles >= target || base_tiles == 0
                          ? 1
                          : (int)std::min<int64_t>(8, (target + base_tiles - 1) / base_tiles);
    int64_t ws_doubles = 0;
    std::vector<OzReduceItem> red;
    for (size_t gi = 0; gi < groups.size(); ++gi) {
      OzGroup& gg = groups[gi];
      const int32_t T = gg.task_end - gg.task_begin;
      gg.nsplit = std::max(1, std::min(split, T));
      if (gg.nsplit > 1) {
        gg.ws_off = ws_doubles;
        const int64_t MN = (int64_t)gg.M * gg.N;
        ws_doubles += gg.nsplit * MN;
        for (int64_t e = 0; e < MN; e += 4096) red.push_back({(int32_t)gi, 0, e, std::min<int64_t>(MN, e + 4096)});
      }
    }
    // work items, the groups with the longest summed range first (the grid then ends on short
    // items); inside a group, the items sharing an A row tile are adjacent (L2 reuse)
    std::vector<OzItem> items;
    std::vector<int32_t> order(groups.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int32_t)i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
      return group_k[(size_t)x] / groups[(size_t)x].nsplit > group_k[(size_t)y] / groups[(size_t)y].nsplit;
    });
    for (int32_t gi : order) {
      const OzGroup& gg = groups[(size_t)gi];
      const int32_t mts = (gg.M + kOzTileM - 1) / kOzTileM, nts = (gg.N + gg.n_tile - 1) / gg.n_tile;
      const int32_t T = gg.task_end - gg.task_begin;
      for (int32_t sp = 0; sp < gg.nsplit; ++sp) {
        const int32_t t0 = gg.task_begin + (int32_t)((int64_t)sp * T / gg.nsplit);
        const int32_t t1 = gg.task_begin + (int32_t)((int64_t)(sp + 1) * T / gg.nsplit);
        for (int32_t mt = 0; mt < mts; ++mt)
          for (int32_t nt = 0; nt < nts; ++nt) items.push_back({gi, mt, nt, gg.nsplit > 1 ? sp : -1, t0, t1});
      }
    }
    if (shared) {
      off_sa = scratch_bytes;
      scratch_bytes += align((size_t)std::max<int64_t>(slots_a, 1) * 8);
      off_sb = scratch_bytes;
      scratch_bytes += align((size_t)std::max<int64_t>(slots_b, 1) * 8);
    }
    if (ws_doubles) {
      off_ws = scratch_bytes;
      scratch_bytes += align((size_t)ws_doubles * 8);
    }
    n_ia = (int64_t)ia.size();
    n_ib = (int64_t)ib.size();
    n_items = (int64_t)items.size();
    d_sa = upload(sa);
    d_ia = upload(ia);
    d_sb = upload(sb);
    d_ib = upload(ib);
    d_groups = upload(groups);
    d_tasks = upload(tasks);
    d_items = upload(items);
    if (!col_base.empty()) {
      d_col_base = upload(col_base);
      d_col_stride = upload(col_stride);
    }
    n_red = (int64_t)red.size();
    if (n_red) d_red = upload(red);
  }
};

void run_contract_ozaki(tamm_ctx* ctx, double alpha, tamm_tensor* C, const char* lc, double beta,
                        const tamm_tensor* A, const char* la, const tamm_tensor* B, const char* lb, int slices,
                        bool float_split) {
  int chunk_k = ctx->oz_chunk_k;
  int tile_policy = ctx->oz_tile_policy;
  bool persistent = ctx->oz_persistent;
  const bool panels = ctx->oz_panels;
  const bool allow_split = ctx->oz_split;
  bool shared = ctx->oz_shared;
  bool fused_opt = ctx->oz_fused_a;
  if (slices == 0) {
    slices = kOzDefaultSlices;
    if (!float_split) {
      auto t = ctx->tuned.find(tune_key(C, lc, A, la, B, lb));
      if (t != ctx->tuned.end()) {
        slices = t->second.slices;
        chunk_k = t->second.chunk_k;
        tile_policy = t->second.tile_policy;
        persistent = t->second.persistent;
        shared = t->second.shared;
        fused_opt = t->second.fused;
      }
    }
  }
  if (slices < kOzMinSlices || slices > kOzMaxSlices)
    throw Error(TAMM_EINVAL, "ozaki: slices must be %d..%d (0 = %d)", kOzMinSlices, kOzMaxSlices, kOzDefaultSlices);
  const bool fused_a = fused_opt && !float_split && !(shared && !float_split);
  const std::string key = "oz" + std::to_string(slices) + "|" + std::to_string(tile_policy) +
                          (panels ? "p" : "") + (allow_split ? "s" : "") + (shared && !float_split ? "h" : "") +
                          (fused_a ? "f|" : "|") +
                          std::to_string(C->id) + "|" + lc + "|" + std::to_string(A->id) + "|" + la + "|" +
                          std::to_string(B->id) + "|" + lb;
  OzakiPlan* p;
  auto itp = ctx->plans.find(key);
  if (itp != ctx->plans.end()) {
    p = static_cast<OzakiPlan*>(itp->second.get());
  } else {
    if (ctx->capturing) throw Error(TAMM_EINVAL, "a new contraction plan cannot be built during graph capture");
    p = new OzakiPlan(ctx, C, lc, A, la, B, lb, slices, tile_policy, panels, allow_split, shared && !float_split,
                      fused_a);
    ctx->plans[key].reset(p);
  }
  OzOpRecord op;
  op.plan = p;
  op.slices = slices;
  op.float_split = float_split;
  op.alpha = alpha;
  op.beta = beta;
  op.c = C->data;
  const tamm_tensor* L = p->lay.swap ? B : A;
  const tamm_tensor* R = p->lay.swap ? A : B;
  op.left = L->data;
  op.right = R->data;
  op.c_bytes = (size_t)C->n_elems * 8;
  op.left_bytes = (size_t)L->n_elems * 8;
  op.right_bytes = (size_t)R->n_elems * 8;
  op.chunk_k = chunk_k;
  op.persistent = persistent;
  if (ctx->group_active) {
    ctx->group_ops.push_back(op);
    return;
  }
  execute_ozaki(ctx, {op});
}

void execute_ozaki(tamm_ctx* ctx, const std::vector<OzOpRecord>& ops) {
  if (ops.empty()) return;
  auto align = [](size_t x) { return (x + 1023) & ~size_t(1023); };
  std::vector<size_t> base(ops.size());
  size_t total = 0;
  for (size_t i = 0; i < ops.size(); ++i) {
    base[i] = total;
    total += align(static_cast<OzakiPlan*>(ops[i].plan)->scratch_bytes);
  }
  char* scratch = (char*)ctx_scratch(ctx, total);
  std::vector<OzProblem> probs(ops.size());
  std::vector<int64_t> counts(ops.size());
  for (size_t i = 0; i < ops.size(); ++i) {
    const OzakiPlan* p = static_cast<const OzakiPlan*>(ops[i].plan);
    char* s = scratch + base[i];
    uint8_t* ta = (uint8_t*)(s + p->off_ta);
    uint8_t* tb = (uint8_t*)(s + p->off_tb);
    int32_t* ea = (int32_t*)(s + p->off_ea);
    int32_t* eb = (int32_t*)(s + p->off_eb);
    if (p->fused) {
      // B sliced into its images, then the GEMM that slices A from FP64 and writes C itself
      cuda_check(launch_ozaki_slice(ctx, ops[i].right, p->d_sb, p->d_ib, p->n_ib, ops[i].slices, false, tb, eb,
                                    p->warps_b, p->kbuf_b),
                 "ozaki slice (right)");
      FaParams fp{};
      fp.n_items = p->n_fi;
      fp.items = p->d_fi;
      fp.groups = p->d_fg;
      fp.tasks = p->d_ft;
      fp.a_recs = p->d_sa;
      fp.a_src = ops[i].left;
      fp.b_tiles = tb;
      fp.b_exp = eb;
      fp.c = ops[i].c;
      fp.alpha = ops[i].alpha;
      fp.beta = ops[i].beta;
      {
        int e = 0;
        const double m = std::frexp(ops[i].alpha, &e);
        fp.alpha_pow2 = (m == 0.5 || m == -0.5) ? 1 : 0;
        fp.alpha_exp = fp.alpha_pow2 ? e - 1 : 0;
      }
      cuda_check(launch_ozaki_fused(ctx, fp, ops[i].slices), "ozaki gemm (A sliced in the kernel)");
      counts[i] = -1;  // not part of the pre-sliced GEMM launches
      continue;
    }
    if (p->shared) {
      // shared scaling: every row maximum into its slot, then every row sliced with its slot's exponent
      unsigned long long* sma = (unsigned long long*)(s + p->off_sa);
      unsigned long long* smb = (unsigned long long*)(s + p->off_sb);
      cuda_check(cudaMemsetAsync(sma, 0, (size_t)p->slots_a * 8, ctx->stream), "shared maxima clear");
      cuda_check(cudaMemsetAsync(smb, 0, (size_t)p->slots_b * 8, ctx->stream), "shared maxima clear");
      for (int mode : {kOzSliceSharedMax, kOzSliceSharedPack}) {
        cuda_check(launch_ozaki_slice(ctx, ops[i].left, p->d_sa, p->d_ia, p->n_ia, ops[i].slices, false, ta, ea,
                                      p->warps_a, p->kbuf_a, mode, sma),
                   "ozaki slice (left)");
        cuda_check(launch_ozaki_slice(ctx, ops[i].right, p->d_sb, p->d_ib, p->n_ib, ops[i].slices, false, tb, eb,
                                      p->warps_b, p->kbuf_b, mode, smb),
                   "ozaki slice (right)");
      }
    } else {
      cuda_check(launch_ozaki_slice(ctx, ops[i].left, p->d_sa, p->d_ia, p->n_ia, ops[i].slices, ops[i].float_split,
                                    ta, ea, p->warps_a, p->kbuf_a),
                 "ozaki slice (left)");
      cuda_check(launch_ozaki_slice(ctx, ops[i].right, p->d_sb, p->d_ib, p->n_ib, ops[i].slices,
                                    ops[i].float_split, tb, eb, p->warps_b, p->kbuf_b),
                 "ozaki slice (right)");
    }
    OzProblem& pr = probs[i];
    pr.a_tiles = ta;
    pr.b_tiles = tb;
    pr.a_exp = ea;
    pr.b_exp = eb;
    pr.groups = p->d_groups;
    pr.tasks = p->d_tasks;
    pr.items = p->d_items;
    pr.col_base = p->d_col_base;
    pr.col_stride = p->d_col_stride;
    pr.ws = (double*)(s + p->off_ws);
    pr.c = p->perm_out ? (double*)(s + p->off_x) : ops[i].c;
    pr.alpha = ops[i].alpha;
    {
      int e = 0;
      const double m = std::frexp(ops[i].alpha, &e);
      pr.alpha_pow2 = (m == 0.5 || m == -0.5) ? 1 : 0;  // alpha = +-2^(e-1)
      pr.alpha_exp = pr.alpha_pow2 ? e - 1 : 0;
    }
    pr.beta = p->perm_out ? 0.0 : ops[i].beta;
    counts[i] = p->n_items;
  }
  // one GEMM launch per (slice count, chunk length, grid kind), at most kOzMaxProblems problems each
  std::vector<bool> done(ops.size(), false);
  for (size_t i = 0; i < ops.size(); ++i) done[i] = counts[i] < 0;
  for (size_t i = 0; i < ops.size(); ++i) {
    if (done[i]) continue;
    std::vector<OzProblem> batch;
    std::vector<int64_t> n;
    for (size_t j = i; j < ops.size() && (int)batch.size() < kOzMaxProblems; ++j) {
      if (done[j] || ops[j].slices != ops[i].slices || ops[j].chunk_k != ops[i].chunk_k ||
          ops[j].persistent != ops[i].persistent)
        continue;
      batch.push_back(probs[j]);
      n.push_back(counts[j]);
      done[j] = true;
    }
    cuda_check(launch_ozaki_gemm(ctx, batch.data(), n.data(), (int)batch.size(), ops[i].slices,
                                 ops[i].chunk_k / kOzTileK, ops[i].persistent),
               "ozaki gemm");
  }
  for (size_t i = 0; i < ops.size(); ++i) {
    const OzakiPlan* p = static_cast<const OzakiPlan*>(ops[i].plan);
    if (p->n_red)
      cuda_check(launch_ozaki_reduce(ctx, p->d_red, p->n_red, p->d_groups, probs[i].ws, probs[i].c, p->d_col_base,
                                     p->d_col_stride, probs[i].alpha, probs[i].beta),
                 "ozaki split reduction");
  }
  const double one = 1.0;
  for (size_t i = 0; i < ops.size(); ++i) {
    const OzakiPlan* p = static_cast<const OzakiPlan*>(ops[i].plan);
    if (p->perm_out) p->perm_out->run(ops[i].c, (double*)(scratch + base[i] + p->off_x), ops[i].beta, &one);
  }
}

}  // namespace tamm
