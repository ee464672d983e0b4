// Double-float arithmetic: a value held as the unevaluated sum s + c of two
// FP32 numbers (48 significant bits), products made exact with an FMA
// (Dekker's product) and running sums kept with their rounding errors
// (Knuth's TwoSum) -- the compensated dot product of Ogita, Rump and Oishi,
// as accurate as an evaluation in twice the float precision.  On this part
// FP64 issues at 1/64 of the FP32 rate, so a multiply-add in about eleven
// FP32 operations is several times faster than one in FP64.
#pragma once
#include <cuda_runtime.h>

namespace css {

struct DF {
  float s, c;
};

// v = hi + lo to 48 bits (v must lie in FP32's range; callers scale first)
__device__ __forceinline__ void df_split(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}
// acc += x * (yh + yl): exact product of x and yh (FMA), the x*yl term in the
// compensation, Knuth's TwoSum for the running sum.
__device__ __forceinline__ void df_fma(DF& a, float x, float yh, float yl) {
  const float p = x * yh;
  float e = fmaf(x, yh, -p);
  e = fmaf(x, yl, e);
  const float s = a.s + p;
  const float bb = s - a.s;
  const float t = (a.s - (s - bb)) + (p - bb);
  a.s = s;
  a.c += t + e;
}
// acc += (xh + xl) * (yh + yl)
__device__ __forceinline__ void df_fma2(DF& a, float xh, float xl, float yh, float yl) {
  const float p = xh * yh;
  float e = fmaf(xh, yh, -p);
  e = fmaf(xh, yl, e);
  e = fmaf(xl, yh, e);
  const float s = a.s + p;
  const float bb = s - a.s;
  const float t = (a.s - (s - bb)) + (p - bb);
  a.s = s;
  a.c += t + e;
}

}  // namespace css
