// Cholesky lambda tensor: the two-electron tensor of Eq. cc12,
//     V[p,q,r,s] = sum_L X[p,r,L] X[q,s,L] - X[p,s,L] X[q,r,L],
// never stored whole but formed slab by slab (consecutive tiles of V's first
// mode) when a contraction reads it (Sec. III.A, lambda tensors: blocks
// computed on demand and consumed by tensor operations).
#pragma once

#include <memory>
#include <vector>

#include "tamm_internal.h"
#include "tamm_plan.h"

namespace tamm {

struct CholeskySlab {
  int64_t tile_lo = 0, tile_hi = 0;  // V's first-mode tiles [tile_lo, tile_hi)
  int64_t v_begin = 0;               // element offset of the slab's first block in V's packed layout
  int64_t x_begin = 0;               // element offset in X of its first block with first tile >= tile_lo
  std::unique_ptr<tamm_tensor> v;    // V's blocks of the slab
  std::unique_ptr<tamm_tensor> x1;   // X1[p,r,q,s] = sum_L X[p,r,L] X[q,s,L] for p in the slab
  std::unique_ptr<tamm_tensor> xs;   // X's blocks with p in the slab (a view of X's storage)
  // device lists of the pair-difference kernel (pair_smem = 0: the two-term permuted add serves the slab)
  std::unique_ptr<Plan> pair_plan;
  const PairBlock* d_pair_blocks = nullptr;
  const PairItem* d_pair_items = nullptr;
  int64_t n_pair_items = 0;
  size_t pair_smem = 0;
};

struct CholeskyLambda {
  tamm_ctx* ctx = nullptr;
  const tamm_tensor* X = nullptr;
  std::vector<CholeskySlab> slabs;
  double* v_buf = nullptr;   // one slab of V
  double* x1_buf = nullptr;  // one slab of X1
  size_t v_bytes = 0, x1_bytes = 0;
  double form_flops = 0.0;  // FP64-equivalent flops of forming every slab once
  ~CholeskyLambda();
};

std::unique_ptr<tamm_tensor> make_cholesky_tensor(tamm_ctx* ctx, const tamm_tensor* X, int64_t slab_bytes);
// Form all of V (a lambda tensor) into `out`, a stored tensor with V's block table.
void cholesky_form(tamm_ctx* ctx, const tamm_tensor* V, tamm_tensor* out, int precision, int slices);
// C(lc) = beta*C + alpha*A(la)*B(lb) where A or B is a lambda tensor: one contraction per slab.
void run_contract_lambda(tamm_ctx* ctx, double alpha, tamm_tensor* C, const char* lc, double beta,
                         const tamm_tensor* A, const char* la, const tamm_tensor* B, const char* lb, int precision,
                         int slices);

}  // namespace tamm
