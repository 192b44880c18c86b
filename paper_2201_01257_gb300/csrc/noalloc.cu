// Allocation-free Frobenius norm: the one entry point of this library that
// never allocates device memory, for callers that must not (or cannot) call
// cudaMalloc or any allocator while they run.
//
// Its scratch -- one partial sum per block of kNoallocChunk input elements --
// lives in a file-scope __device__ array of fixed size.  Every GPU that loads
// the library holds that array until the process exits, and every call on a
// device shares it, so calls whose kernels overlap on the GPU race on it.
#include <mutex>

#include "tamm_internal.h"

namespace {

constexpr int64_t kNoallocMaxPartials = 32768;  // 256 KB of partial sums
constexpr int64_t kNoallocChunk = 16384;        // input elements per partial sum
constexpr int64_t kNoallocMaxElems = kNoallocMaxPartials * kNoallocChunk;  // 2^29 doubles
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoallocMaxPartials];

// Device addresses of g_noalloc_partials, looked up once per device with that device current.
std::mutex g_noalloc_mutex;
double* g_noalloc_addr[kNoallocMaxDevices] = {};

__global__ void __launch_bounds__(256) noalloc_sumsq_kernel(const double* __restrict__ x, int64_t n,
                                                            double* __restrict__ partials) {
  __shared__ double red[8];
  const int64_t lo = (int64_t)blockIdx.x * kNoallocChunk;
  const int64_t hi = lo + kNoallocChunk < n ? lo + kNoallocChunk : n;
  double acc = 0.0;
  for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) acc = fma(x[e], x[e], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    partials[blockIdx.x] = s;  // every slot this call reads is written first: nothing needs zeroing
  }
}

__global__ void __launch_bounds__(1024) noalloc_final_kernel(const double* __restrict__ partials, int64_t n_parts,
                                                             double* __restrict__ out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n_parts; i += blockDim.x) acc += partials[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 32; ++w) s += red[w];
    *out = sqrt(s);
  }
}

}  // namespace

extern "C" tamm_status tamm_norm_noalloc(const double* x_device, int64_t n, double* result_device, void* stream) {
  if (n < 0 || !result_device || (n > 0 && !x_device)) return TAMM_EINVAL;
  // a double load or store through a pointer that is not 8-byte aligned would fault on the GPU
  if ((reinterpret_cast<uintptr_t>(x_device) | reinterpret_cast<uintptr_t>(result_device)) % 8) return TAMM_EINVAL;
  if (n > kNoallocMaxElems) return TAMM_ELIMIT;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) {
    (void)cudaGetLastError();
    return TAMM_ECUDA;
  }
  double* partials;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
      // first call on this device: the host-side name of the array is not a device address
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return TAMM_ECUDA;
      }
      g_noalloc_addr[dev] = static_cast<double*>(p);
    }
    partials = g_noalloc_addr[dev];
  }
  const int64_t n_parts = (n + kNoallocChunk - 1) / kNoallocChunk;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n_parts > 0) noalloc_sumsq_kernel<<<(unsigned)n_parts, 256, 0, s>>>(x_device, n, partials);
  noalloc_final_kernel<<<1, 1024, 0, s>>>(partials, n_parts, result_device);
  if (cudaGetLastError() != cudaSuccess) return TAMM_ECUDA;
  return TAMM_OK;
}
