// Autotuner of the split-precision contraction: picks the number of BF16
// slices per operand and the length of the exact FP32 accumulation chunk for
// one contraction, given a normwise relative error target, and the tile
// policy (output columns per work item) and GEMM grid kind (one CTA per work
// item, or one per SM walking the items) that run that configuration fastest.
//
// Both knobs trade accuracy for speed.  Fewer slices mean fewer slice
// products (S(S+1)/2 of them) but a coarser representation of the operands
// (about 7 bits per slice); a longer chunk means fewer FP32-to-double folds
// but a larger rounding error in the inexact tail products, which grows with
// the chunk length.  The tuner measures, on the caller's own operands:
//   * the FP64 contraction (the reference), once;
//   * for each chunk length, the split-precision contraction with 3, 4, ...
//     slices until its error against the reference is at most
//     kSafety * target (the first passing count is the fastest one for that
//     chunk, since time grows with the slice count);
//   * the run time of every passing candidate under each tile policy and
//     grid kind (CUDA events, after one untimed run); both split the same
//     arithmetic into different work items, so they change time, not results;
//   * all of the above once with each block's own row/column scaling and once
//     with shared scaling (one exponent per output row and column, so that
//     short block pairs share accumulation chunks), whose error differs;
//   * where the contraction qualifies (block pairs of at most 48 summed
//     indices, output blocks of at most 64 columns), once more with the A
//     operand sliced inside the GEMM: one chunk per block pair and the
//     persistent grid, so one timing;
// and keeps the fastest.  The result is remembered per (tensors, labels) and
// used by tamm_contract whenever slices = 0.
#include <algorithm>
#include <cmath>

#include "ozaki.h"
#include "tamm_plan.h"

namespace tamm {

std::string tune_key(const tamm_tensor* C, const char* lc, const tamm_tensor* A, const char* la,
                     const tamm_tensor* B, const char* lb) {
  return "tune|" + std::to_string(C->id) + "|" + lc + "|" + std::to_string(A->id) + "|" + la + "|" +
         std::to_string(B->id) + "|" + lb;
}

}  // namespace tamm

using namespace tamm;

namespace {

constexpr double kSafety = 0.5;  // margin for other data of the same contraction
constexpr int kChunks[] = {1280, 800, 640, 320};  // 800: half of a 40 x 40 block pair's summed range
constexpr int kPolicies[] = {0, 1, 2, 3};  // tile policies (TAMM_OPT_OZAKI_TILE_POLICY)
constexpr int kTimedRuns = 3;

// A view of C's block structure on another buffer (same id: the same cached plans).
struct Shadow {
  tamm_tensor t;
  Shadow(const tamm_tensor& C, double* data) : t(C) {
    t.data = data;
    t.owned = false;
    t.owned_bytes = 0;
  }
};

double host_scalar(tamm_ctx* ctx, const double* dev) {
  cuda_check(cudaMemcpyAsync(ctx->h_result, dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "D2H");
  sync_and_check(ctx);
  return ctx->h_result[0];
}

double diff_norm(tamm_ctx* ctx, const double* x, const double* y, int64_t n) {
  const int64_t parts = std::max<int64_t>(1, std::min<int64_t>((n + 8191) / 8192, 4L * ctx->sm_count * 8));
  double* partials = ctx_reduce_buffer(ctx, (size_t)parts);
  double* out = result_slot(ctx, 2);
  if (n == 0) cuda_check(cudaMemsetAsync(partials, 0, sizeof(double), ctx->stream), "memset");
  else cuda_check(launch_diff_sumsq_partials(ctx, x, y, n, partials, parts), "diff kernel");
  cuda_check(launch_reduce_final(ctx, partials, parts, 1.0, 1, out), "reduce kernel");
  return host_scalar(ctx, out);
}

}  // namespace

extern "C" tamm_status tamm_autotune(tamm_ctx* ctx, const tamm_tensor* C, const char* lc, const tamm_tensor* A,
                                     const char* la, const tamm_tensor* B, const char* lb, double target_rel_err,
                                     int* slices, int* chunk_k, int* tile_policy, int* persistent,
                                     int* shared_scale, double* rel_err, double* ms) {
  if (!ctx) return TAMM_EINVAL;
  void* ref = nullptr;
  void* trial = nullptr;
  size_t bytes = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const int saved_chunk = ctx->oz_chunk_k;
  const int saved_policy = ctx->oz_tile_policy;
  const bool saved_persistent = ctx->oz_persistent;
  const bool saved_shared = ctx->oz_shared;
  const bool saved_fused = ctx->oz_fused_a;
  tamm_status st = TAMM_OK;
  try {
    if (ctx->host_only) throw Error(TAMM_ECUDA, "host-only context (device -1) cannot run device work");
    if (!C || !A || !B || !lc || !la || !lb) throw Error(TAMM_EINVAL, "autotune: null argument");
    if (!(target_rel_err > 0.0)) throw Error(TAMM_EINVAL, "autotune: target error must be positive");
    if (ctx->group_active || ctx->capturing) throw Error(TAMM_EINVAL, "autotune inside a group or capture");
    if (A->lambda || B->lambda || C->lambda) throw Error(TAMM_EUNSUPPORTED, "autotune: lambda tensor operand");
    if (!A->data || !B->data) throw Error(TAMM_EINVAL, "autotune: operand without data");
    bytes = (size_t)std::max<int64_t>(C->n_elems, 1) * sizeof(double);
    ref = ctx_alloc(ctx, bytes);
    trial = ctx_alloc(ctx, bytes);
    Shadow R(*C, (double*)ref), X(*C, (double*)trial);
    run_contract(ctx, 1.0, &R.t, lc, 0.0, A, la, B, lb, TAMM_PREC_F64, 0);
    run_norm(ctx, &R.t, result_slot(ctx, 3));
    const double ref_norm = host_scalar(ctx, result_slot(ctx, 3));
    // a zero product says nothing about the error of other operands: refuse rather than pick 3 slices
    if (!(ref_norm > 0.0)) throw Error(TAMM_EINVAL, "autotune: the FP64 product of these operands is zero");
    const double denom = ref_norm;
    cuda_check(cudaEventCreate(&e0), "cudaEventCreate");
    cuda_check(cudaEventCreate(&e1), "cudaEventCreate");
    int best_s = 0, best_chunk = 0, best_policy = 0, best_mode = 0;
    bool best_persistent = false;
    double best_ms = 0.0, best_err = 0.0;
    // scaling modes: 0 = each block's own row/column scaling, 1 = shared scaling, 2 = own scaling with
    // the A operand sliced inside the GEMM (only for contractions that path takes; its chunk is one block
    // pair and its grid persistent, so one chunk length and one timing)
    const bool fused_ok = oz_fused_eligible(ContractLayout(ctx, C, lc, A, la, B, lb));
    for (int sh = 0; sh < 3; ++sh)
    for (int chunk : kChunks) {
      if (sh == 2 && (!fused_ok || chunk != kChunks[0])) continue;
      ctx->oz_shared = sh == 1;
      ctx->oz_fused_a = sh == 2;
      ctx->oz_chunk_k = chunk;
      ctx->oz_tile_policy = saved_policy;
      ctx->oz_persistent = saved_persistent;
      int s_ok = 0;
      double err_ok = 0.0;
      for (int s = kOzMinSlices; s <= kOzMaxSlices && !s_ok; ++s) {
        run_contract(ctx, 1.0, &X.t, lc, 0.0, A, la, B, lb, TAMM_PREC_OZAKI_BF16, s);
        const double err = diff_norm(ctx, (const double*)trial, (const double*)ref, C->n_elems) / denom;
        if (err <= kSafety * target_rel_err) {
          s_ok = s;  // more slices only cost more time at this chunk length
          err_ok = err;
        }
      }
      if (!s_ok) continue;
      // the tile policy and the grid kind change the work split, not the arithmetic of an output
      // element: time each combination
      const int n_combos = sh == 2 ? 1 : 2 * (int)(sizeof(kPolicies) / sizeof(kPolicies[0]));
      for (int combo = 0; combo < n_combos; ++combo) {
        const int policy = kPolicies[combo / 2];
        const bool persistent = sh == 2 || combo % 2 == 1;  // the A-slicing GEMM always walks its items
        ctx->oz_tile_policy = policy;
        ctx->oz_persistent = persistent;
        run_contract(ctx, 1.0, &X.t, lc, 0.0, A, la, B, lb, TAMM_PREC_OZAKI_BF16, s_ok);  // builds the plan
        cuda_check(cudaEventRecord(e0, ctx->stream), "cudaEventRecord");
        for (int r = 0; r < kTimedRuns; ++r)
          run_contract(ctx, 1.0, &X.t, lc, 0.0, A, la, B, lb, TAMM_PREC_OZAKI_BF16, s_ok);
        cuda_check(cudaEventRecord(e1, ctx->stream), "cudaEventRecord");
        sync_and_check(ctx);
        float f = 0.0f;
        cuda_check(cudaEventElapsedTime(&f, e0, e1), "cudaEventElapsedTime");
        const double t = f / kTimedRuns;
        if (best_s == 0 || t < best_ms) {
          best_s = s_ok;
          best_chunk = chunk;
          best_policy = policy;
          best_persistent = persistent;
          best_mode = sh;
          best_ms = t;
          best_err = err_ok;
        }
      }
    }
    if (best_s == 0)
      throw Error(TAMM_EUNSUPPORTED, "autotune: no slice count (<= %d) reaches %.3g on these operands", kOzMaxSlices,
                  target_rel_err);
    ctx->tuned[tune_key(C, lc, A, la, B, lb)] = {best_s, best_chunk, best_policy, best_persistent, best_mode == 1,
                                                  best_mode == 2};
    if (slices) *slices = best_s;
    if (shared_scale) *shared_scale = best_mode;
    if (chunk_k) *chunk_k = best_chunk;
    if (tile_policy) *tile_policy = best_policy;
    if (persistent) *persistent = best_persistent ? 1 : 0;
    if (rel_err) *rel_err = best_err;
    if (ms) *ms = best_ms;
    ctx->last_error.clear();
  } catch (const Error& e) {
    ctx->last_error = e.msg;
    st = e.status;
  } catch (const std::exception& e) {
    ctx->last_error = e.what();
    st = TAMM_EINVAL;
  }
  ctx->oz_chunk_k = saved_chunk;
  ctx->oz_tile_policy = saved_policy;
  ctx->oz_persistent = saved_persistent;
  ctx->oz_shared = saved_shared;
  ctx->oz_fused_a = saved_fused;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (ref) ctx_free(ctx, ref, bytes);
  if (trial) ctx_free(ctx, trial, bytes);
  return st;
}
