// Device-side FP64 <-> FP32 conversions and FP32 complex arithmetic for the
// mixed path (included by .cu files only).
//
// GB300's FP64 pipe executes two operations per clock per SM, and the hardware
// conversions F2F.F32.F64 / F2F.F64.F32 issue to it; the FP32 parts of the mixed
// path convert with integer operations instead, so that reading FP64 data into
// FP32 arithmetic costs no FP64-pipe time.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace hz {

// FP64 -> FP32, round to nearest (ties away); |x| below the FP32 normal range -> signed 0,
// above it -> signed infinity.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int e32 = (int)((b >> 52) & 0x7ff) - 896;              // FP32 biased exponent
  if (e32 <= 0) return __uint_as_float(sign);
  if (e32 >= 255) return __uint_as_float(sign | 0x7f800000u);
  const unsigned long long full = ((unsigned long long)e32 << 52) + (b & 0x000fffffffffffffULL) + (1ULL << 28);
  return __uint_as_float(sign | (uint32_t)(full >> 29));       // a rounding carry moves into the exponent
}

// FP64 -> FP32 by truncation, with fewer operations, for splitting data into TF32 hi / lo
// parts: the sign, the exponent rebiased (for exponents 897..1150 the low 8 bits of the FP64
// exponent with the top bit flipped are the FP32 exponent) and the top 23 mantissa bits
// (a funnel shift).  |x| below the FP32 normal range -> signed 0; |x| must stay below
// 2^128 (non-finite or larger inputs give finite garbage; the refinement's FP64 residual,
// computed from the FP64 data, still reports a non-finite input).
__device__ __forceinline__ float f64_to_f32_trunc(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  uint32_t u = (__funnelshift_l(lo, hi, 3) & 0x7fffffffu) ^ 0x40000000u;
  u = ((hi & 0x7ff00000u) < 0x38100000u) ? 0u : u;
  return __uint_as_float(u | (hi & 0x80000000u));
}

// complex FP64 -> FP32 by the truncating conversion (the FP32 kernels of the mixed path are
// bound by instruction issue; the refinement absorbs the last bit)
__device__ __forceinline__ float2 to_c64t(double2 v) {
  return make_float2(f64_to_f32_trunc(v.x), f64_to_f32_trunc(v.y));
}

// FP32 -> FP64 (exact for normal numbers; FP32 denormals -> signed 0).
__device__ __forceinline__ double f32_to_f64(float v) {
  const uint32_t u = __float_as_uint(v);
  const uint32_t sign = u & 0x80000000u;
  const uint32_t e = (u >> 23) & 0xffu;
  if (e == 0) return __hiloint2double((int)sign, 0);
  const uint32_t e64 = (e == 255u) ? 2047u : e + 896u;
  return __hiloint2double((int)(sign | (e64 << 20) | ((u & 0x7fffffu) >> 3)), (int)((u & 7u) << 29));
}

__device__ __forceinline__ double2 to_c128(float2 v) { return make_double2(f32_to_f64(v.x), f32_to_f64(v.y)); }

// Identity forms, so that kernels templated on the storage type (the mixed path keeps its
// mode-space volumes as complex64, the FP64 path as complex128) read either through one
// call: to_c64t gives FP32 operands, to_c128 FP64 operands.
__device__ __forceinline__ float2 to_c64t(float2 v) { return v; }
__device__ __forceinline__ double2 to_c128(double2 v) { return v; }
// Store a value computed in FP64 into either storage type (complex64: truncated).
__device__ __forceinline__ void store_c(double2* p, double2 v) { *p = v; }
__device__ __forceinline__ void store_c(float2* p, double2 v) { *p = to_c64t(v); }
// an FP32 value into a complex64 or complex128 element
__device__ __forceinline__ void store_f32(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void store_f32(double2* p, float2 v) { *p = to_c128(v); }

// acc + c * y in FP32
__device__ __forceinline__ float2 cfma32(float2 c, float2 y, float2 acc) {
  return make_float2(fmaf(c.x, y.x, fmaf(-c.y, y.y, acc.x)), fmaf(c.x, y.y, fmaf(c.y, y.x, acc.y)));
}

}  // namespace hz
