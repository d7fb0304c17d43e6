// Base-2 exponentials of the fused products' epilogues, on two pipes: the
// MUFU ex2.approx, and a polynomial on the FMA pipe.  The throughput probe in
// krr_bench.cu runs the same two routines, so the roofline it reports is the
// one these epilogues can reach.
#pragma once

namespace krr {

__device__ __forceinline__ float ex2_mufu(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 2^x on the FMA pipe: x = n + f with n = rint(x) (through the 1.5 * 2^23
// rounding constant), f in [-1/2, 1/2], p(f) ~ 2^f (a degree-5 polynomial
// fitted for this project: near-minimax in relative error, 7.5e-8 in exact
// arithmetic), n added to the exponent bits.
__device__ __forceinline__ float ex2_fma(float x) {
  x = fmaxf(x, -125.f);
  const float t = x + 12582912.f;
  const float f = x - (t - 12582912.f);
  float p = fmaf(0.0013278163969516754f, f, 0.009675555862486362f);
  p = fmaf(p, f, 0.055507078766822815f);
  p = fmaf(p, f, 0.24022118747234344f);
  p = fmaf(p, f, 0.6931469440460205f);
  p = fmaf(p, f, 1.0000001192092896f);
  const int n = __float_as_int(t) - 0x4B400000;
  return __int_as_float(__float_as_int(p) + (n << 23));
}

}  // namespace krr
