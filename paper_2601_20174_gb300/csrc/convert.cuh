#pragma once

#include <cuda_runtime.h>

// FP64 <-> FP32 conversions on the integer pipe.  GB300 executes F2F
// conversions on its FP64 unit (~2 lanes/clk/SM), so the PCG solver's
// per-node conversions (the FP32 copy of the updated residual, also on the
// halo nodes of the persistent solver's staged restriction, and the FP64 copy
// of the preconditioned residual z) are done with bit operations on the
// IEEE-754 encodings instead: exact for FP32 -> FP64, round-to-nearest-even
// for FP64 -> FP32, so both give the hardware conversion's result bit for
// bit.  Inputs whose result is zero, subnormal, infinite or NaN (exponent
// outside the normal range) take the hardware conversion.
__device__ __forceinline__ float f64_to_f32_rn(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const int e32 = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  if (e32 <= 0 || e32 >= 255) return (float)d;
  const unsigned m23 = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1FFFFFFFu;  // the 29 dropped bits; half = 2^28
  unsigned bits = (hi & 0x80000000u) | ((unsigned)e32 << 23) | m23;
  if (rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) ++bits;  // a carry moves into the exponent
  return __uint_as_float(bits);
}

__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xFFu;
  if (ex == 0u || ex == 0xFFu) return (double)f;
  const unsigned hi = (u & 0x80000000u) | ((ex + (1023u - 127u)) << 20) | ((u & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// The solver's element type T from / to FP64 with the conversions above.
template <typename T>
__device__ __forceinline__ T from_f64(double v) {
  if constexpr (sizeof(T) == 4) return f64_to_f32_rn(v);
  else return (T)v;
}
template <typename T>
__device__ __forceinline__ double to_f64(T v) {
  if constexpr (sizeof(T) == 4) return f32_to_f64(v);
  else return (double)v;
}
