// Device helpers of the split-precision kernels (the tcgen05 block GEMM with pre-sliced operands, the
// GEMM that slices its A operand itself, and the slicing kernel): the digit split of FP64 values, the
// warp roles and register split of the warp-specialised GEMMs, bounded mbarrier waits, the exact
// (hi, lo) fold of the accumulator groups, the FP64 reconstruction and the MMA schedule issue.  The
// arithmetic scheme is described in ozaki.h.
#pragma once

#include <cstdint>

#include "ozaki.h"
#include "sm100.cuh"

namespace tamm {
namespace {

__host__ __device__ constexpr unsigned long long digit_bias(int S) {
  unsigned long long b = 0;
  for (int j = 0; j + 1 < S; ++j) b |= 64ull << (7 * j);
  return b;
}

// 2^(23-7k) + (k > 0 ? 64 : 0) 2^(-7k), exact in FP32
__host__ __device__ constexpr float slice_offset(int k) {
  float f = k == 0 ? 8388608.0f : 8388672.0f;
  for (int i = 0; i < 7 * k; ++i) f *= 0.5f;
  return f;
}

// Slice values of |x| for row exponent e, as float bit patterns: |x| carries
// v_k = d_k 2^(-7k), k = 0..S-1, where d_0 (6 bits) and the balanced base-2^7
// digits d_1..d_{S-1} (|d| <= 64) represent F = round(|x| 2^(7S-1-e)).  F
// comes from the FP64 bit pattern; adding 64 to every lower digit position,
// G = F + 64 (1 + 2^7 + ... + 2^(7(S-2))), turns the balanced digits into
// plain 7-bit fields, d_k = field_k(G) - 64 (k >= 1), d_0 = G >> 7(S-1).  A
// field placed in the mantissa of 2^(23-7k) gives 2^(23-7k) + field 2^(-7k)
// exactly; one float subtraction of 2^(23-7k) + 64 2^(-7k) leaves v_k, an
// exact BF16 (at most 7 significant bits).  The sign of x is applied by the
// caller to the packed BF16 pairs.
template <int S>
__device__ __forceinline__ void slice_magnitudes(double x, int e, uint32_t (&v)[S]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int Eb = (int)((bits >> 52) & 0x7FF);
  const unsigned long long M = (bits & ((1ull << 52) - 1)) | ((unsigned long long)(Eb != 0) << 52);
  const int shift = max(Eb, 1) - 1075 + 7 * S - 1 - e;
  unsigned long long F = 0;
  // a left shift only for S = 8 or subnormal x (a normal |x| <= 2^e gives shift <= 7S - 54)
  if (shift >= 0) F = M << shift;
  if (shift < 0 && shift > -63) {
    const int rs = -shift;
    F = (M + (1ull << (rs - 1))) >> rs;  // round half up
  }
  constexpr unsigned long long kBias = digit_bias(S);
  const unsigned long long G = F + kBias;
#pragma unroll
  for (int k = 0; k < S; ++k) {
    const int sh = 7 * (S - 1 - k);
    const uint32_t field = k == 0 ? (uint32_t)(G >> sh) : (uint32_t)(G >> sh) & 127u;
    const float top = __uint_as_float((uint32_t)(150 - 7 * k) << 23 | field);
    v[k] = __float_as_uint(__fsub_rn(top, slice_offset(k)));
  }
}

// BF16 pairs of the slice values of two adjacent elements: x0 in the low half of each word.
template <int S>
__device__ __forceinline__ void pack_digits(const double x0, const double x1, int e, uint32_t (&w)[S]) {
  uint32_t v0[S], v1[S];
  slice_magnitudes<S>(x0, e, v0);
  slice_magnitudes<S>(x1, e, v1);
  const uint32_t sign = (uint32_t)((unsigned long long)__double_as_longlong(x0) >> 63) << 15 |
                        (uint32_t)((unsigned long long)__double_as_longlong(x1) >> 63) << 31;
#pragma unroll
  for (int k = 0; k < S; ++k) w[k] = __byte_perm(v0[k], v1[k], 0x7632) ^ sign;
}

__device__ __forceinline__ int64_t mixed_offset(int32_t idx, int n, const int32_t* dim, const int32_t* stride) {
  int64_t off = 0;
  for (int m = n - 1; m >= 0; --m) {
    const int32_t x = idx % dim[m];
    idx /= dim[m];
    off += (int64_t)x * stride[m];
  }
  return off;
}

// Offsets of the 8 consecutive summed indices k0..k0+7 (entries past K are unused).
__device__ __forceinline__ void k_offsets8(const SliceBlock& B, int32_t k0, int64_t (&off)[8]) {
  if (B.nk == 1) {  // one summed mode: a plain stride, no mixed-radix decomposition
#pragma unroll
    for (int j = 0; j < 8; ++j) off[j] = (int64_t)(k0 + j) * B.kstride[0];
    return;
  }
  int32_t kk[4] = {0, 0, 0, 0};
  int32_t r = k0;
  int64_t o = 0;
  for (int m = B.nk - 1; m >= 0; --m) {
    kk[m] = r % B.kdim[m];
    r /= B.kdim[m];
    o += (int64_t)kk[m] * B.kstride[m];
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    off[j] = o;
    int m = B.nk - 1;
    if (m < 0) continue;
    ++kk[m];
    o += B.kstride[m];
    while (m > 0 && kk[m] == B.kdim[m]) {
      o -= (int64_t)kk[m] * B.kstride[m];
      kk[m] = 0;
      --m;
      ++kk[m];
      o += B.kstride[m];
    }
  }
}

// bf16 bits of a float, round to nearest even (finite inputs).
__device__ __forceinline__ uint32_t bf16_rne(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}

// Floating three-piece split (BF16x3): x ~ a1 + a2 + a3 with each a_i the BF16
// rounding of what the previous pieces left of fl32(x); the pieces carry about
// 24 bits relative to x itself.  Products a_k b_l of different k + l land in
// the same accumulator regions as the integer digits.
__device__ __forceinline__ void pack_float3(const double x0, const double x1, uint32_t (&w)[3]) {
  float r[2] = {__double2float_rn(x0), __double2float_rn(x1)};
  uint32_t b[3][2];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      b[k][j] = bf16_rne(r[j]);
      r[j] = __fsub_rn(r[j], __uint_as_float(b[k][j] << 16));  // exact: r and the piece share the leading bits
    }
#pragma unroll
  for (int k = 0; k < 3; ++k) w[k] = b[k][0] | (b[k][1] << 16);
}

// ~2 s at 2 GHz: how long a kernel waits for copies already in flight to land before it exits (the
// dependency waits take their limit from the launch, TAMM_OPT_WAIT_CYCLES)
constexpr long long kDrainWaitCycles = 4000000000ll;

// Warp roles: warpgroup 0 = producer (warp 0), MMA issuer + TMEM owner (warp 1),
// two idle warps; warpgroups 1 and 2 = eight epilogue warps, two per TMEM lane
// quadrant.  Registers move from warpgroup 0 to the epilogue with setmaxnreg:
// 128 * kRegsLow + 256 * kRegsHigh must not exceed 384 * (registers at launch).
constexpr int kEpiWarps = 8;
constexpr int kThreads = 128 + 32 * kEpiWarps;
constexpr int kRegsLow = 40;
constexpr int kRegsHigh = 232;
constexpr int kRegsLaunchNeeded = (128 * kRegsLow + 256 * kRegsHigh + kThreads - 1) / kThreads;

// Accumulator buffers in the 512 TMEM columns: each holds four regions of H
// columns, so items with H <= 64 keep two (H <= 32: four) chunks in flight
// and the MMAs of one chunk overlap the draining of the previous one.
constexpr int kAccBufs = 4;
__device__ __forceinline__ uint32_t acc_buffers(uint32_t H) {
  const uint32_t n = 128u / H;
  return n < (uint32_t)kAccBufs ? n : (uint32_t)kAccBufs;
}

__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                             int* status, long long limit) {
  const long long t0 = clock64();
  uint32_t ns = 16;
  while (!sm100::mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
      *abort_flag = 1;
      atomicExch(status, TAMM_ETIMEOUT);
      return false;
    }
    __nanosleep(ns);
    if (ns < 512) ns <<= 1;
  }
  return true;
}

__device__ __forceinline__ float pow2f(int d) {
  return d < -126 ? 0.0f : __int_as_float((127 + d) << 23);
}

// x * 2^s as a double, exactly, built from the bits of the float x with integer operations (GB300's
// FP64 pipe is narrow, and the output stage would otherwise spend most of its time there); `neg`
// flips the sign.  False when x is subnormal, infinite or NaN, or the result leaves the normal
// range: the caller then takes the FP64 route.
__device__ __forceinline__ bool f2d_scaled(float x, int s, bool neg, double& out) {
  const uint32_t u = __float_as_uint(x);
  const unsigned long long sign = ((unsigned long long)(u >> 31) ^ (neg ? 1ull : 0ull)) << 63;
  const uint32_t a = u & 0x7FFFFFFFu;
  if (a == 0u) {
    out = __longlong_as_double((long long)sign);
    return true;
  }
  const int e = (int)(a >> 23);
  const int de = e - 127 + 1023 + s;
  if (e == 0 || e == 255 || de <= 0 || de >= 2047) return false;
  out = __longlong_as_double(
      (long long)(sign | ((unsigned long long)de << 52) | ((unsigned long long)(a & 0x7FFFFFu) << 29)));
  return true;
}

__device__ __forceinline__ double pow2d(int d) {
  if (d < -1022) return 0.0;
  if (d > 1023) return __longlong_as_double(0x7FF0000000000000ll);
  return __longlong_as_double((long long)(1023 + d) << 52);
}

__device__ __forceinline__ void two_sum(float& hi, float x, float& err) {
  const float s = __fadd_rn(hi, x);
  const float bb = __fsub_rn(s, hi);
  err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  hi = s;
}

// (hi, lo) += (s0 + s1 + s2 + s3) * sc.  The exact groups s0..s2 enter through
// error-free TwoSum steps; only the weighted tail s3 is rounded.
__device__ __forceinline__ void fold(float& hi, float& lo, float s0, float s1, float s2, float s3, float sc) {
  float e0, e1, e2;
  two_sum(hi, __fmul_rn(s0, sc), e0);
  two_sum(hi, __fmul_rn(s1, sc), e1);
  two_sum(hi, __fmul_rn(s2, sc), e2);
  lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(e0, e1), __fadd_rn(e2, __fmul_rn(s3, sc))));
}

__device__ __forceinline__ void epi_barrier() { asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory"); }

// Issue the MMAs of one K step for schedule (S, fuse), op I onwards; every
// operand offset, shape and flag is a compile-time constant.
// B slices are H rows apart (2H descriptor units of 16 bytes) and accumulator
// regions H TMEM columns apart; idesc1 / idesc2 are the instruction
// descriptors of one B slice and of two adjacent fused ones.
template <int S, bool kFuse, int I>
__device__ __forceinline__ void issue_ops(uint32_t tmem, uint64_t a0, uint64_t b0, uint32_t H, uint32_t idesc1,
                                          uint32_t idesc2, bool first) {
  constexpr OzSched sch = oz_schedule(S, kFuse);
  if constexpr (I < sch.n) {
    constexpr OzOp op = sch.op[I];
    // descriptor start address counts 16-byte units: one 4096-byte A slice is +256
    sm100::mma_bf16(tmem + H * (uint32_t)op.region, a0 + (uint64_t)(256 * op.a), b0 + (uint64_t)(2u * H * op.b),
                    op.nb == 2 ? idesc2 : idesc1, (op.first && first) ? 0u : 1u);
    issue_ops<S, kFuse, I + 1>(tmem, a0, b0, H, idesc1, idesc2, first);
  }
}

}  // namespace
}  // namespace tamm
