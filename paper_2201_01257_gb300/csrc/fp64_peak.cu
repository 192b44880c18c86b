// FP64 throughput probe: the measured denominator of the FP64 path's roofline.  Two arithmetic forms
// run back to back on every SM, each thread or warp carrying independent accumulator chains so that
// latency is hidden: scalar fused multiply-adds (DFMA) and the warp-wide FP64 tensor-core MMA
// (mma.sync m8n8k4 f64).  The result is the flop rate of the timed launch (CUDA events on the
// context's stream, after one untimed launch).
#include <algorithm>

#include "tamm_plan.h"

namespace tamm {
namespace {

constexpr int kProbeIters = 4096;
constexpr int kChains = 8;

// Each thread: kChains independent chains x = x * a + b, kProbeIters steps (2 flops each).
__global__ void __launch_bounds__(256) probe_dfma_kernel(double a, double b, double* __restrict__ sink) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c);
  for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678) sink[0] = s;  // keeps the chains live (one in-bounds slot either way)
}

// Each warp: kChains independent 8x8 accumulators, D = A(8x4) B(4x8) + D per step (512 flops per MMA).
__global__ void __launch_bounds__(256) probe_dmma_kernel(double a, double b, double* __restrict__ sink) {
  double d[kChains][2];
#pragma unroll
  for (int c = 0; c < kChains; ++c) d[c][0] = d[c][1] = 0.0;
  const double av = a * (double)(threadIdx.x % 3), bv = b;
  for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(d[c][0]), "+d"(d[c][1])
                   : "d"(av), "d"(bv));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += d[c][0] + d[c][1];
  if (s == 12345.678) sink[0] = s;
}

}  // namespace
}  // namespace tamm

using namespace tamm;

extern "C" tamm_status tamm_fp64_peak(tamm_ctx* ctx, int kind, double* tflops) {
  if (!ctx || !tflops || (kind != 0 && kind != 1)) return TAMM_EINVAL;
  try {
    require_device(ctx);
    if (ctx->capturing || ctx->group_active) throw Error(TAMM_EINVAL, "fp64 probe inside a group or capture");
    double* sink = result_slot(ctx, 2);  // never written in practice
    const int blocks = std::max(1, ctx->sm_count) * 8;
    const double a = 0.999999, b = 1e-9;
    auto launch = [&] {
      if (kind == 0) probe_dfma_kernel<<<blocks, 256, 0, ctx->stream>>>(a, b, sink);
      else probe_dmma_kernel<<<blocks, 256, 0, ctx->stream>>>(a, b, sink);
      cuda_check(cudaGetLastError(), "fp64 probe launch");
    };
    launch();
    cudaEvent_t e0, e1;
    cuda_check(cudaEventCreate(&e0), "event");
    cuda_check(cudaEventCreate(&e1), "event");
    cudaEventRecord(e0, ctx->stream);
    launch();
    cudaEventRecord(e1, ctx->stream);
    cudaError_t st = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (st == cudaSuccess) st = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cuda_check(st, "fp64 probe timing");
    const double per_thread = kind == 0 ? 2.0 * kChains * kProbeIters : 512.0 * kChains * kProbeIters / 32.0;
    *tflops = per_thread * blocks * 256.0 / (ms * 1e-3) / 1e12;
    ctx->launches += 2;
    ctx->last_error.clear();
    return TAMM_OK;
  } catch (const Error& e) {
    ctx->last_error = e.msg;
    return e.status;
  }
}
