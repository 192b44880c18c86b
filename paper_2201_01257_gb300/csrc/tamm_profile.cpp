// Launch counting and optional CUDA-event timing per kernel class.
#include "tamm_plan.h"

namespace tamm {

static cudaEvent_t take_event(tamm_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cuda_check(cudaEventCreate(&e), "cudaEventCreate");
  return e;
}

void kernel_begin(tamm_ctx* ctx, int kind) {
  ++ctx->launches;
  if (!ctx->profiling) return;
  tamm_ctx::TimedLaunch t{kind, take_event(ctx), take_event(ctx)};
  cuda_check(cudaEventRecord(t.start, ctx->stream), "cudaEventRecord");
  ctx->timed.push_back(t);
}

void kernel_end(tamm_ctx* ctx, int kind) {
  if (!ctx->profiling || ctx->timed.empty() || ctx->timed.back().kind != kind) return;
  cuda_check(cudaEventRecord(ctx->timed.back().stop, ctx->stream), "cudaEventRecord");
}

}  // namespace tamm

using namespace tamm;

extern "C" tamm_status tamm_ctx_launch_count(const tamm_ctx* ctx, int64_t* launches) {
  if (!ctx || !launches) return TAMM_EINVAL;
  *launches = ctx->launches;
  return TAMM_OK;
}

extern "C" tamm_status tamm_ctx_profile(tamm_ctx* ctx, int enable) {
  if (!ctx) return TAMM_EINVAL;
  if (ctx->host_only) return TAMM_ECUDA;
  ctx->profiling = enable != 0;
  return TAMM_OK;
}

extern "C" tamm_status tamm_ctx_profile_read(tamm_ctx* ctx, double* ms, int64_t* launches) {
  if (!ctx) return TAMM_EINVAL;
  if (ctx->host_only) return TAMM_ECUDA;
  try {
    cuda_check(cudaStreamSynchronize(ctx->stream), "stream synchronize");
    double acc[TAMM_KERNEL_CLASSES] = {};
    int64_t cnt[TAMM_KERNEL_CLASSES] = {};
    for (auto& t : ctx->timed) {
      float f = 0.0f;
      cuda_check(cudaEventElapsedTime(&f, t.start, t.stop), "cudaEventElapsedTime");
      if (t.kind >= 0 && t.kind < TAMM_KERNEL_CLASSES) {
        acc[t.kind] += f;
        cnt[t.kind] += 1;
      }
      ctx->event_pool.push_back(t.start);
      ctx->event_pool.push_back(t.stop);
    }
    ctx->timed.clear();
    for (int k = 0; k < TAMM_KERNEL_CLASSES; ++k) {
      if (ms) ms[k] = acc[k];
      if (launches) launches[k] = cnt[k];
    }
    return TAMM_OK;
  } catch (const Error& e) {
    ctx->last_error = e.msg;
    return e.status;
  }
}
