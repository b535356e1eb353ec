// Double-float accumulation of exact FP32 products, shared by the QRP kernels.
//
// s += a * (bh + bl), where bh + bl is an FP64 value split into two floats.  a * bh is
// formed exactly as p + e (FMA residual), p is added to the running high part with
// TwoSum (Knuth), and every rounding error goes into the low part.  With a flush of
// (hi + lo) into an FP64 sum every few hundred terms the relative error of a dot
// product stays near 2^-46, while every operation runs on the FP32 pipe.
#pragma once

namespace tk {

struct DF {
  float hi = 0.f, lo = 0.f;
};

__device__ __forceinline__ void df_fma(DF &s, float a, float bh, float bl) {
  const float p = a * bh;
  const float e = fmaf(a, bh, -p);
  const float q = a * bl;
  const float t = s.hi + p;
  const float bp = t - s.hi;
  const float err = (s.hi - (t - bp)) + (p - bp);
  s.hi = t;
  s.lo += err + (e + q);
}

}  // namespace tk
