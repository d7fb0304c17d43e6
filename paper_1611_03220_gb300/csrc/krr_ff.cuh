// Float-float (double-word FP32) arithmetic shared by the high-precision
// kernel products: exact two-sum, and 2^x for x given as a float pair.
//
// 2^x: x = k/256 + r with k = rint(256 x); 2^(k/256) from a 256-entry table
// of (hi, lo) pairs (after P. T. P. Tang's table method, 1989); e^(r ln 2) by
// a degree-4 Taylor polynomial on |r ln 2| <= ln 2 / 512, with the low word
// of x folded into r by an exact two-sum so that y = r ln 2 keeps a tiny low
// part.  About 1e-13 relative for x >= -125 (smaller x is clamped there).
#pragma once

#include <cstdint>

namespace krr {
namespace ff {

constexpr int NTAB = 256;

// s + e = a + b exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (kh, kl) ~= 2^(xh + xl); tab holds 2^(j/256) as (hi, lo) pairs, j < 256.
__device__ __forceinline__ void exp2_ff(float xh, float xl, const float* tab, float& kh,
                                        float& kl) {
  if (xh < -125.f) {
    xh = -125.f;
    xl = 0.f;
  }
  const float kf = rintf(xh * 256.f);
  float rh, rl;
  two_sum(fmaf(kf, -0.00390625f, xh), xl, rh, rl);
  const float yh = rh * 0.693147182464599609375f;
  float yl = fmaf(rh, 0.693147182464599609375f, -yh);
  yl = fmaf(rh, -1.904654299957768e-09f, yl);  // ln 2 - float(ln 2)
  yl = fmaf(rl, 0.693147182464599609375f, yl);
  // e^yh = 1 + yh + pp (degree-4 Taylor), then times (1 + yl)
  float pp = fmaf(yh, 0.041666666666666667f, 0.16666666666666667f);
  pp = fmaf(yh, pp, 0.5f);
  pp = pp * yh * yh;
  const float eh = 1.f + yh;
  const float e0 = ((1.f - eh) + yh) + pp;
  const float el = fmaf(yl, eh + e0, e0);
  const int k = (int)kf;
  const float2 tv = *reinterpret_cast<const float2*>(tab + 2 * (k & (NTAB - 1)));
  const float kh0 = eh * tv.x;
  float kl0 = fmaf(eh, tv.x, -kh0);
  kl0 = fmaf(eh, tv.y, kl0);
  kl0 = fmaf(el, tv.x, kl0);
  const float s2 = __int_as_float((127 + (k >> 8)) << 23);
  kh = kh0 * s2;
  kl = kl0 * s2;
}

}  // namespace ff
}  // namespace krr
