// Split-precision (Ozaki-style) block GEMMs on the tcgen05 tensor cores.
//
// Every FP64 operand row (A) / column (B) of a block is scaled by a power of
// two 2^e with |x| < 2^e and cut into S balanced base-2^7 integer digits
//     x = 2^(e-6) * sum_k d_k 2^(-7(k-1)),   |d_k| <= 64,
// stored as BF16 values v_k = d_k 2^(-7(k-1)) (exact: at most 7 significant
// bits).  Products of slices k,l (k+l <= S+1) run as BF16 MMAs with FP32
// accumulation in TMEM, in four accumulator regions:
//     G0: k+l=2, G1: k+l=3, G2: k+l=4 (each sums integer multiples of 2^-7G),
//     G3: every k+l >= 5 (weighted tail, rounding allowed there).
// A chunk of at most kOzChunkK summed indices keeps |G0|, |G1| 2^7, |G2| 2^14
// below 3 * 1280 * 64 * 64 < 2^24, so G0..G2 are exact in FP32.  The tail G3
// is summed by the tensor core with FP32 rounding that is not unbiased, so its
// error grows with the chunk length; the default chunk is 640.  After each
// chunk the epilogue scales the four partial sums by the chunk's power-of-two
// row/column factors and folds them into a (hi, lo) FP32 pair, G0..G2 through
// error-free TwoSum steps and G3 by a rounded add into lo; FP64 is used only
// for the final reconstruction
//     C = beta*C + alpha * 2^(Eref+Fref-12) * (hi + lo).
#pragma once

#include <algorithm>
#include <vector>

#include "tamm_contract.h"

namespace tamm {

constexpr int kOzTileM = 128;     // A-tile rows (MMA M)
constexpr int kOzTileN = 128;     // B-tile rows = output columns per CTA
constexpr int kOzTileK = 16;      // summed indices per tile (32 bytes of bf16)
constexpr int kOzChunkK = 1280;   // summed indices per exact FP32 chunk
constexpr int kOzChunkTiles = kOzChunkK / kOzTileK;
constexpr int kOzMinSlices = 3;
constexpr int kOzMaxSlices = 8;
constexpr int kOzDefaultSlices = 6;
constexpr int kOzTileBytesPerSlice = 128 * 32;  // 128 rows x 16 bf16
constexpr int kOzExpZero = -30000;              // exponent of an all-zero (or padding) row
constexpr int kOzMaxOps = 40;

// One GEMM-order operand block to slice.  Rows are the output-side index
// (M for A, N for B), K the summed index; native element (r, k) sits at
//   src_off + sum_m r_m*rstride[m] + sum_m k_m*kstride[m]
// with r, k decomposed row-major over rdim / kdim.
struct SliceBlock {
  int64_t src_off;
  int64_t tile_off;  // byte offset of this block's first tile in the sliced buffer (tiles ordered [row tile][k tile])
  int64_t exp_off;   // exponent of row 0
  int64_t shared_off;  // shared scaling: slot of row 0 in the shared row-maximum array (see kOzSliceShared*)
  int32_t rows, K;
  int32_t row_tiles, k_tiles;
  int32_t nr, nk;
  int32_t rdim[4], rstride[4];
  int32_t kdim[4], kstride[4];
  int32_t k_contig;  // consecutive k are adjacent in memory (else consecutive rows are)
  int32_t k_dense;   // the whole summed range is one contiguous run: offset of k is k
  int32_t tile_rows; // rows per tile H (a multiple of 16, <= 128): a tile is S slices of H x 16 bf16
  int32_t dst_row0;  // image row of this block's row 0 (blocks concatenated along rows share an image)
};

// Slicing modes.  Own: each row's exponent comes from the row's maximum over this block.  Shared
// scaling takes two launches: kOzSliceSharedMax folds every row's maximum into its slot of a shared
// array (all blocks whose rows meet the same output rows or columns share slots) and writes no
// tiles; kOzSliceSharedPack then slices every row with the exponent of its slot, so that all block
// pairs of an output tile are scaled alike and their products may share one exact accumulation chunk.
constexpr int kOzSliceOwn = 0;
constexpr int kOzSliceSharedMax = 1;
constexpr int kOzSliceSharedPack = 2;

constexpr int kOzSliceMaxRows = 128;  // rows per slicing CTA
constexpr size_t kOzSliceSmemBudget = 104 * 1024;  // warp row buffers of one slicing CTA (two CTAs per SM)
constexpr size_t kOzSliceSmemMax = 200 * 1024;     // launch check

struct SliceItem {
  int32_t block;
  int32_t r0;  // first row (padding rows up to row_tiles * tile_rows are written as zeros)
  int32_t nr;
  int32_t pad;
};

// An output group: one output block (row-major M x N at c_off), or a column
// panel -- output blocks that share M and every A block, concatenated along
// N (colmap >= 0: column c lives at col_base[colmap + c] + row * col_stride[colmap + c]).
// A group's tasks may be split into nsplit summed ranges (few output tiles,
// long summed extent): each range's work items write their FP64 partials to
// the workspace, dense [split][M][N] at ws_off, and a reduction adds them in
// range order into C.
struct OzGroup {
  int64_t c_off;
  int64_t colmap;
  int64_t ws_off;
  int32_t M, N;
  int32_t task_begin, task_end;
  int32_t n_tile;  // output columns per work item = rows per B tile (a multiple of 16, <= 128)
  int32_t nsplit;
  int32_t shared;  // every task of the group has the same row and column exponents (shared scaling): the
                   // exact accumulation chunks run across task boundaries
  int32_t pad;
};

struct OzTask {
  int64_t a_off, b_off;    // byte offsets of the A / B block's first tile
  int64_t a_exp, b_exp;    // exponent offsets of the A / B block
  int32_t k_tiles;
  int32_t pad;
};

// One contraction inside a (possibly grouped) persistent GEMM launch.  Its
// work items are global items [item_begin, item_begin + n_items) of the launch.
struct OzProblem {
  const uint8_t* a_tiles;
  const uint8_t* b_tiles;
  const int32_t* a_exp;
  const int32_t* b_exp;
  const OzGroup* groups;
  const OzTask* tasks;
  const struct OzItem* items;
  const int64_t* col_base;    // column maps of the panels
  const int32_t* col_stride;
  double* ws;                 // partials of split groups
  int64_t item_begin;
  double* c;
  double alpha, beta;
  int32_t alpha_pow2;  // alpha = +-2^alpha_exp (then folded into the output scaling)
  int32_t alpha_exp;
};
constexpr int kOzMaxProblems = 64;  // problems per launch (kernel-parameter table)

struct OzItem {
  int32_t group, mt, nt;
  int32_t split;   // summed range of a split group (-1: the group is not split)
  int32_t t0, t1;  // tasks [t0, t1) of this item
};

// One chunk of the reduction of a split group's partials.
struct OzReduceItem {
  int32_t group;
  int32_t pad;
  int64_t e0, e1;  // elements [e0, e1) of the group's M x N output
};

// MMA schedule for one K step: A slice, first B slice, number of adjacent B
// slices fused along N (1 or 2), accumulator region, and whether it is the
// first write of its region(s) in a chunk.  Products (k, l) with k + l <= S + 1
// (1-based) go to region min(k + l - 2, 3); products of adjacent B slices that
// land in adjacent regions are fused into one N = 2H MMA when `fuse` is set
// (full tiles).
struct OzOp {
  int a, b, nb, region, first;
};
struct OzSched {
  int n;
  OzOp op[kOzMaxOps];
};

__host__ __device__ constexpr OzSched oz_schedule(int S, bool fuse) {
  OzSched s{};
  bool written[4] = {false, false, false, false};
  for (int k = 1; k <= S; ++k) {
    int l = 1;
    while (l <= S + 1 - k) {
      const int region = k + l - 2 < 3 ? k + l - 2 : 3;
      // (k, l) and (k, l + 1) share one MMA when they land in two adjacent regions (region <= 2)
      // that are both written for the first time in the chunk, or both accumulated
      const bool pair = fuse && region < 3 && l + 1 <= S + 1 - k && written[region] == written[region + 1];
      OzOp& o = s.op[s.n++];
      o.a = k - 1;
      o.b = l - 1;
      o.nb = pair ? 2 : 1;
      o.region = region;
      o.first = written[region] ? 0 : 1;
      written[region] = true;
      if (pair) written[region + 1] = true;
      l += pair ? 2 : 1;
    }
  }
  return s;
}


// Rows per B tile (= output columns per work item) for a B block of `rows`
// rows, a multiple of 16 in [16, 128].
//   policy 0: always 128 (a block's last tile is ragged; its MMAs run with N
//             rounded up to 16, but its image is padded to 128 rows);
//   policy 1: 128, or rows rounded up to 16 when the block has fewer rows
//             (same tiles, smaller images and copies for narrow blocks);
//   policy 2: the fewest tiles of 128 at most, of equal width rounded up to
//             16 (no ragged tile, so every tile runs the fused N = 2H MMAs);
//   policy 3: as 2 with tiles of 64 at most, so that two accumulator buffers
//             fit in TMEM and the MMAs never wait for an accumulator drain.
inline int oz_tile_rows(int64_t rows, int policy) {
  if (rows <= 0) return 128;
  const auto up16 = [](int64_t x) { return (int)std::max<int64_t>(16, (x + 15) / 16 * 16); };
  if (policy == 1) return rows >= 128 ? 128 : up16(rows);
  if (policy == 2 || policy == 3) {
    const int64_t cap = policy == 2 ? 128 : 64;
    const int64_t n = (rows + cap - 1) / cap;
    return (int)std::min<int64_t>(cap, up16((rows + n - 1) / n));
  }
  return 128;
}

// Short-K, narrow-N contractions (every block pair sums at most kOzFaMaxK indices, every output block
// has at most kOzFaMaxN columns; e.g. a singles amplitude against a 4-index integral block) run through
// a second GEMM kernel that slices its A operand itself: worker warps read the FP64 block straight
// from the tensor, take each row's exponent over the block pair's summed range and write the digits
// into the shared-memory stages the MMAs read, so A is read once from HBM and never stored as an
// image.  B is pre-sliced as usual.  The same warps drain the accumulators, one exact chunk per block
// pair, and write C through its own strides (the output permutation is fused).
constexpr int kOzFaMaxK = 48;  // summed indices per block pair (three K tiles)
constexpr int kOzFaMaxN = 64;  // output columns per output block

struct FaGroup {
  int64_t c_off;     // output block in C
  int32_t M, N;
  int32_t task_begin, task_end;
  int32_t n_tile;    // H: N rounded up to 16
  int32_t nr, nc;    // output row / column modes
  int32_t rdim[4], rstride[4];  // GEMM output row -> C offset (mixed radix over C's strides)
  int32_t cdim[4], cstride[4];  // GEMM output column -> C offset
};

struct FaTask {
  int64_t b_off, b_exp;  // pre-sliced B image of the block pair and its exponents
  int32_t a_rec;         // FP64 geometry of the A block (a SliceBlock record)
  int32_t k_tiles;
};

struct FaItem {
  int32_t group, mt;  // output block and 128-row tile
};

struct FaParams {
  int64_t n_items;
  int* status;
  long long wait_cycles;
  int stages;
  const FaItem* items;
  const FaGroup* groups;
  const FaTask* tasks;
  const SliceBlock* a_recs;
  const double* a_src;
  const uint8_t* b_tiles;
  const int32_t* b_exp;
  double* c;
  double alpha, beta;
  int32_t alpha_pow2, alpha_exp;
};

// Persistent launch of the A-slicing GEMM (one CTA per SM).
cudaError_t launch_ozaki_fused(tamm_ctx* ctx, FaParams& p, int S);

// Slicing launch shape and items for an operand's records: record i covers image rows
// [dst_row0, dst_row0 + extent[i]); sets the warps per CTA and the warp row buffer length.
void oz_slicing_items(std::vector<SliceBlock>& recs, const std::vector<int32_t>& extent,
                      std::vector<SliceItem>& items, int& warps, int& kbuf);

// float_split (S = 3 only): BF16x3 floating pieces instead of integer digits.
// mode: kOzSliceOwn / kOzSliceSharedMax / kOzSliceSharedPack; smax: the shared row-maximum array (|x| bit
// patterns, zeroed before the kOzSliceSharedMax launches), unused in kOzSliceOwn.
cudaError_t launch_ozaki_slice(tamm_ctx* ctx, const double* src, const SliceBlock* blocks, const SliceItem* items,
                               int64_t n_items, int S, bool float_split, uint8_t* tiles, int32_t* exps, int warps,
                               int kbuf, int mode = kOzSliceOwn, unsigned long long* smax = nullptr);
// Reduction of split groups' partials into C (after the GEMM launch).
cudaError_t launch_ozaki_reduce(tamm_ctx* ctx, const OzReduceItem* items, int64_t n_items, const OzGroup* groups,
                                const double* ws, double* c, const int64_t* col_base, const int32_t* col_stride,
                                double alpha, double beta);
// One launch over the work items of up to kOzMaxProblems problems (item_begin
// of each problem is filled in here); `n_items` is the total.
cudaError_t launch_ozaki_gemm(tamm_ctx* ctx, OzProblem* problems, const int64_t* n_items_per_problem,
                              int n_problems, int S, int chunk_tiles, bool persistent);

}  // namespace tamm
