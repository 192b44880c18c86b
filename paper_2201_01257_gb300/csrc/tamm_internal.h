// Internal structures of the GB300 block-sparse contraction library.
// Host side: index spaces, block-sparse tensors, contraction plans.
// Device side: plain-old-data task records consumed by the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <functional>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tamm_gb300.h"

namespace tamm {

constexpr int kMaxModes = 8;
constexpr int kMaxKernelModes = 4;  // add/energy kernels handle tensors of up to 4 modes
constexpr int kMaxAddTerms = 4;

// ------------------------------------------------------------ device records

// One output block of a permuted add (and of the energy's pairing).
// Element e of the destination block (row-major over dim[0..nm)) reads term t's
// source at src_off[t] + sum_m idx_m * sstride[t][m]  (src_off < 0: no source block).
struct AddBlock {
  int64_t dst_off;
  int64_t n;
  int32_t nm;
  int32_t dim[kMaxKernelModes];
  int64_t src_off[kMaxAddTerms];
  int32_t sstride[kMaxAddTerms][kMaxKernelModes];
  int32_t tmode;  // mode that every term reading the last mode with a stride reads contiguously (tiled
                  // transposition path), or -1
};

// A tile of a transposed permuted add: rows [p0, p0 + kAddTile) of the block's mode tmode, columns
// [q0, q0 + kAddTile) of its last mode, for the indices o0 .. o0 + n_o - 1 of its other modes (row-major).
constexpr int kAddTile = 32;
constexpr int kAddTileSmem = 5120;  // doubles of staged planes per CTA (40 KB)
constexpr int kAddMaxOuter = 32;    // planes per item
struct TileItem {
  int32_t block;
  int32_t p0, q0;
  int32_t o0, n_o;
  int32_t pad;
};

// One block of the Cholesky pair difference V[p,q,r,s] = X1[p,r,q,s] - X1[p,s,q,r]: V's block (tiles
// tp,tq,tr,ts; extents np,nq,nr,ns) and the X1 blocks (tp,tr,tq,ts) and (tp,ts,tq,tr), -1 when not stored.
struct PairBlock {
  int64_t v_off, a_off, b_off;
  int32_t np, nq, nr, ns;
};

// Row p of one PairBlock processed by one CTA.
struct PairItem {
  int32_t block;
  int32_t p;
};

// A chunk of one AddBlock processed by one CTA.
struct ChunkItem {
  int32_t block;
  int32_t pad;
  int64_t start;
};

// FP64 block GEMM records.  One group per output block (in GEMM layout);
// tasks of a group are the block pairs summed into it, in fixed order.
struct GemmGroup {
  int64_t c_off;
  int32_t M, N;
  int32_t task_begin, task_end;
};
struct GemmTask {
  int64_t a_off;  // A block, row-major M x K
  int64_t b_off;  // B block, row-major K x N
  int32_t K;
  int32_t pad;
};
struct GemmItem {
  int32_t group;
  int32_t m0, n0;
  int32_t pad;
};

// ------------------------------------------------------------- host objects

struct Allocator {
  tamm_alloc_fn alloc = nullptr;
  tamm_free_fn release = nullptr;
  void* user = nullptr;
};

// Device buffer obtained from the context allocator, released stream-ordered.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct Plan;  // contraction / add / energy plans, cached per context

// A split-precision contraction ready to run (recorded inside a group).
struct OzOpRecord {
  Plan* plan;  // the contraction's cached split-precision plan
  int slices;
  bool float_split;
  double alpha, beta;
  double* c;
  const double* left;   // GEMM-left operand data
  const double* right;  // GEMM-right operand data
  size_t c_bytes, left_bytes, right_bytes;
  int chunk_k;      // summed indices per exact FP32 chunk
  bool persistent;  // GEMM grid: one CTA per SM walking the work items
};

// Split-precision configuration picked by the autotuner for one contraction.
struct TunedConfig {
  int slices;
  int chunk_k;
  int tile_policy;
  bool persistent;
  bool shared;  // shared row/column scaling (TAMM_OPT_OZAKI_SHARED_SCALE)
  bool fused;   // A sliced inside the GEMM (TAMM_OPT_OZAKI_FUSED_A)
};

}  // namespace tamm

namespace tamm {
struct CholeskyLambda;  // tamm_lambda.h
}  // namespace tamm

struct tamm_space {
  tamm_ctx* ctx = nullptr;
  uint64_t id = 0;
  int n_tiles = 0;
  int64_t n = 0;
  std::vector<int64_t> off, size;
  std::vector<int> spin, irrep;
};

struct tamm_tensor {
  tamm_ctx* ctx = nullptr;
  uint64_t id = 0;
  int nm = 0, n_upper = 0, sym = 0;
  const tamm_space* sp[tamm::kMaxModes] = {};
  int64_t n_blocks = 0, n_elems = 0;
  std::vector<int64_t> tiles;   // n_blocks * nm
  std::vector<int64_t> off;     // n_blocks + 1
  std::vector<int64_t> lookup;  // dense tile tuple -> block index, -1 if not stored
  double* data = nullptr;
  bool owned = false;
  size_t owned_bytes = 0;
  std::shared_ptr<tamm::CholeskyLambda> lambda;  // set for a Cholesky lambda tensor (never stored)

  int64_t find(const int64_t* tt) const {
    int64_t lin = 0;
    for (int m = 0; m < nm; ++m) lin = lin * sp[m]->n_tiles + tt[m];
    return lookup[(size_t)lin];
  }
  int64_t block_size(int64_t b) const { return off[(size_t)b + 1] - off[(size_t)b]; }
};

struct tamm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  tamm::Allocator allocator;
  std::string last_error;
  uint64_t next_id = 1;
  int* d_status = nullptr;    // device status word (TAMM_ETIMEOUT)
  double* d_reduce = nullptr; // partial sums of reductions
  size_t reduce_cap = 0;
  double* h_result = nullptr; // pinned host double for synchronous results
  tamm::DevBuf scratch;       // grows on demand, stream-ordered reuse
  std::map<std::string, std::unique_ptr<tamm::Plan>> plans;
  int sm_count = 0;
  bool host_only = false;  // device -1: metadata and planning only
  int oz_chunk_k = 640;    // split precision: summed indices per exact FP32 chunk
  bool oz_persistent = false;  // split precision: persistent GEMM grid (one CTA per SM)
  int oz_tile_policy = 1;      // split precision: output columns per work item (TAMM_OPT_OZAKI_TILE_POLICY)
  bool oz_panels = true;       // split precision: concatenate output blocks sharing their A blocks
  bool oz_split = true;        // split precision: split long summed ranges of small contractions
  bool oz_shared = false;      // split precision: shared row/column scaling (TAMM_OPT_OZAKI_SHARED_SCALE)
  bool oz_fused_a = false;     // split precision: short-K narrow-N contractions slice A in the GEMM (TAMM_OPT_OZAKI_FUSED_A)
  long long oz_wait_cycles = 4000000000ll;  // limit of a kernel's dependency waits (TAMM_OPT_WAIT_CYCLES)
  int oz_test_withhold = 0;    // failure-path test hook (TAMM_OPT_TEST_WITHHOLD_COPY), one launch
  int64_t launches = 0;    // kernels launched by this context
  bool profiling = false;  // bracket launches with CUDA events
  struct TimedLaunch {
    int kind;
    cudaEvent_t start, stop;
  };
  std::vector<TimedLaunch> timed;
  std::vector<cudaEvent_t> event_pool;
  bool group_active = false;                  // between tamm_group_begin and tamm_group_end
  std::vector<tamm::OzOpRecord> group_ops;    // recorded split-precision contractions
  std::map<std::string, tamm::TunedConfig> tuned;  // autotuned contractions (used when slices = 0)
  bool capturing = false;                     // between tamm_graph_begin and tamm_graph_end
  bool capture_failed = false;                // an operation failed while capturing
  int64_t capture_launch0 = 0;
  // graphs destroyed while this context was capturing: freed after the capture ends (destroying a
  // graph inside an open capture would invalidate it)
  std::vector<std::pair<cudaGraph_t, cudaGraphExec_t>> deferred_graphs;
};

namespace tamm {

// Launch bookkeeping: call around every kernel launch (counts, optional event timing).
void kernel_begin(tamm_ctx* ctx, int kind);
void kernel_end(tamm_ctx* ctx, int kind);

// Fill a tensor's block table (lookup, tiles, offsets) with the tile tuples `keep` accepts, in
// lexicographic order; the spaces (nm, sp) must be set.
void build_blocks_where(tamm_tensor& T, const std::function<bool(const int64_t*)>& keep);
void require_device(tamm_ctx* ctx);

// allocation through the context allocator (stream-ordered)
void* ctx_alloc(tamm_ctx* ctx, size_t bytes);
void ctx_free(tamm_ctx* ctx, void* p, size_t bytes);
void* ctx_scratch(tamm_ctx* ctx, size_t bytes);  // valid until the next ctx_scratch call

// ------------------------------------------------------------ kernel launch
// Implemented in kernels_f64.cu.  All launch on ctx->stream; return cudaError_t.
// Chunked items (any layout; nm = the blocks' mode count) and tiled items (blocks with tmode >= 0).
cudaError_t launch_add(tamm_ctx* ctx, double* dst, const double* src, const AddBlock* blocks,
                       const ChunkItem* items, int64_t n_items, int n_terms, double beta, const double* alpha_host,
                       const double* scale_device = nullptr, int nm = kMaxKernelModes,
                       const TileItem* tiles = nullptr, int64_t n_tiles = 0);
// V = X1(p,r,q,s) - X1(p,s,q,r) over the listed blocks; `smem_bytes` = 8 * max ns * (nr + 1), at most
// kPairSmemMax (the default dynamic shared memory limit, so no attribute call is needed).
constexpr size_t kPairSmemMax = 48 * 1024;
cudaError_t launch_cholesky_pair(tamm_ctx* ctx, double* v, const double* x1, const PairBlock* blocks,
                                 const PairItem* items, int64_t n_items, size_t smem_bytes);
cudaError_t launch_energy_partials(tamm_ctx* ctx, const double* a, const double* b, const AddBlock* blocks,
                                   const ChunkItem* items, int64_t n_items, double* partials);
cudaError_t launch_sumsq_partials(tamm_ctx* ctx, const double* x, int64_t n, double* partials, int64_t n_parts);
// partial sums of (x - y)^2
cudaError_t launch_diff_sumsq_partials(tamm_ctx* ctx, const double* x, const double* y, int64_t n,
                                       double* partials, int64_t n_parts);
cudaError_t launch_reduce_final(tamm_ctx* ctx, const double* partials, int64_t n, double alpha, int take_sqrt,
                                double* out_device);
cudaError_t launch_gemm_f64(tamm_ctx* ctx, const double* a, const double* b, double* c, const GemmGroup* groups,
                            const GemmTask* tasks, const GemmItem* items, int64_t n_items, double alpha,
                            double beta);

constexpr int kChunk = 4096;         // elements per add/energy chunk
constexpr int kGemmTileM = 64;       // FP64 GEMM CTA tile
constexpr int kGemmTileN = 64;

}  // namespace tamm
