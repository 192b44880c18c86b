// Perturbative triples correction E(T) (Sec. IV.B): host plan and launchers (tamm_triples.cu).
#pragma once

#include "tamm_internal.h"

namespace tamm {

// E(T) into energy (one device double) and, if not null, each occupied triple's contribution.
void run_triples(tamm_ctx* ctx, const tamm_tensor* T2, const tamm_tensor* T1, const tamm_tensor* Vooov,
                 const tamm_tensor* Vvovv, const tamm_tensor* Voovv, const double* eps_o, const double* eps_v,
                 int precision, int slices, int64_t workspace_bytes, double* energy, double* triple_energies);
// Host-only counts: occupied triples, block-GEMM flops per evaluation, batches.
void triples_info(tamm_ctx* ctx, const tamm_tensor* T2, const tamm_tensor* T1, const tamm_tensor* Vooov,
                  const tamm_tensor* Vvovv, const tamm_tensor* Voovv, int64_t workspace_bytes, int64_t* n_triples,
                  double* gemm_flops, int* n_batches);

// Double-float (two FP32) copies of FP64 arrays for the fused energy kernel.
cudaError_t launch_to_df(tamm_ctx* ctx, const double* x, int64_t n, float2* out);
cudaError_t launch_triples_energy(tamm_ctx* ctx, const double* U, const void* items, int64_t n_items,
                                  const float2* voo, const float2* t1, const float2* eps_o, const float2* eps_v,
                                  double* partials);
cudaError_t launch_triples_segments(tamm_ctx* ctx, const double* partials, const int64_t* seg, int64_t n,
                                    double* out);

}  // namespace tamm
