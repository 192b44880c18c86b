// Host planner: label analysis, operand layouts, device task lists.
#pragma once

#include <string>
#include <vector>

#include "tamm_internal.h"

namespace tamm {

struct Error {
  tamm_status status;
  std::string msg;
  Error(tamm_status s, const char* fmt, ...);
};

void cuda_check(cudaError_t e, const char* what);
void sync_and_check(tamm_ctx* ctx);
double* ctx_reduce_buffer(tamm_ctx* ctx, size_t n);
std::unique_ptr<tamm_tensor> make_permuted_tensor(const tamm_tensor& S, const int* perm);

// Device scalar result slots (8 doubles after the status word, same allocation).
inline double* result_slot(tamm_ctx* ctx, int i) { return (double*)((char*)ctx->d_status + 64) + i; }

// A cached plan owns its device task arrays.
struct Plan {
  tamm_ctx* ctx = nullptr;
  std::vector<DevBuf> bufs;
  explicit Plan(tamm_ctx* c) : ctx(c) {}
  virtual ~Plan();
  void* upload_bytes(const void* host, size_t bytes);
  template <class T>
  T* upload(const std::vector<T>& v) {
    return (T*)upload_bytes(v.data(), v.size() * sizeof(T));
  }
};

void run_contract(tamm_ctx* ctx, double alpha, tamm_tensor* C, const char* lc, double beta, const tamm_tensor* A,
                  const char* la, const tamm_tensor* B, const char* lb, int precision, int slices);
double contract_flops(tamm_ctx* ctx, const tamm_tensor* C, const char* lc, const tamm_tensor* A, const char* la,
                      const tamm_tensor* B, const char* lb);
void run_add(tamm_ctx* ctx, tamm_tensor* C, const char* lc, double beta, const tamm_tensor* A, int n_terms,
             const char* const* la, const double* alpha, const double* scale_device = nullptr);
void run_energy(tamm_ctx* ctx, double alpha, const tamm_tensor* A, const char* la, const tamm_tensor* B,
                const char* lb, double* out_device);
void run_norm(tamm_ctx* ctx, const tamm_tensor* t, double* out_device);

}  // namespace tamm
