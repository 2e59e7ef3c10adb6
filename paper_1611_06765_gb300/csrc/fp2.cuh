// fp2.cuh -- element arithmetic shared by the contraction kernels: FP64, FP32, and FP32 pairs.
//
// An FP32 pair carries a value as the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, i.e. 48 significant bits (relative precision 2^-48, against FP64's
// 2^-53).  A multiply-add acc += a b is done on the FP32 pipe, which a GB300 runs at 64 times
// its FP64 rate:
//   p = a.hi b.hi rounded, and its rounding error fma(a.hi, b.hi, -p), exact (Dekker's
//   product through the fused multiply-add), plus the cross terms a.hi b.lo + a.lo b.hi
//   (a.lo b.lo, below 2^-48 |ab|, is dropped);
//   acc.hi + p by Knuth's two-sum (the rounded sum and its exact error), the errors of both
//   steps collected in acc.lo, which is not folded back into acc.hi until the value is read.
// Twelve FP32 instructions per multiply-add.  The error-free steps use __fmul_rn / __fadd_rn /
// __fsub_rn, which the compiler never contracts into a fused multiply-add (a contraction of
// acc.hi + a.hi b.hi would break the two-sum).  For sums of K products the result stays within
// a few K 2^-48 of the sum of absolute values; the contractions of the ph term (K <= 66, two
// chained products) come out within about 1e-13 of their largest element.
#pragma once
#include <cuda_runtime.h>

struct f2 {
  float hi, lo;
};

template <typename T_>
struct Arith;

// Out: the type a kernel stores its results in (FP32 pairs keep the pair, so that a consumer
// summing several results does so on the FP32 pipe and converts once); to_double converts.
template <>
struct Arith<double> {
  using Out = double;
  __device__ __forceinline__ static double zero() { return 0.0; }
  __device__ __forceinline__ static double from_double(double x) { return x; }
  __device__ __forceinline__ static Out out(double x) { return x; }
  __device__ __forceinline__ static double to_double(double x) { return x; }
  __device__ __forceinline__ static double add(double a, double b) { return a + b; }
  __device__ __forceinline__ static double sub(double a, double b) { return a - b; }
  __device__ __forceinline__ static double neg(double a) { return -a; }
  __device__ __forceinline__ static double half(double a) { return 0.5 * a; }
  __device__ __forceinline__ static void mac(double& acc, double a, double b) { acc = fma(a, b, acc); }
};

template <>
struct Arith<float> {
  using Out = float;
  __device__ __forceinline__ static float zero() { return 0.0f; }
  __device__ __forceinline__ static float from_double(double x) { return (float)x; }
  __device__ __forceinline__ static Out out(float x) { return x; }
  __device__ __forceinline__ static double to_double(float x) { return (double)x; }
  __device__ __forceinline__ static float add(float a, float b) { return a + b; }
  __device__ __forceinline__ static float sub(float a, float b) { return a - b; }
  __device__ __forceinline__ static float neg(float a) { return -a; }
  __device__ __forceinline__ static float half(float a) { return 0.5f * a; }
  __device__ __forceinline__ static void mac(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
};

template <>
struct Arith<f2> {
  using Out = f2;
  __device__ __forceinline__ static f2 zero() { return f2{0.0f, 0.0f}; }
  // x = hi + lo with hi = x rounded to FP32 and lo = (x - hi) rounded (x - hi is exact in FP64)
  __device__ __forceinline__ static f2 from_double(double x) {
    const float h = (float)x;
    return f2{h, (float)(x - (double)h)};
  }
  __device__ __forceinline__ static Out out(f2 a) { return a; }
  __device__ __forceinline__ static double to_double(f2 a) { return (double)a.hi + (double)a.lo; }
  // two-sum of the high parts, the error and the low parts folded and renormalised
  __device__ __forceinline__ static f2 add(f2 a, f2 b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, e);
    return f2{h, __fsub_rn(e, __fsub_rn(h, s))};
  }
  __device__ __forceinline__ static f2 neg(f2 a) { return f2{-a.hi, -a.lo}; }
  __device__ __forceinline__ static f2 sub(f2 a, f2 b) { return add(a, neg(b)); }
  __device__ __forceinline__ static f2 half(f2 a) { return f2{0.5f * a.hi, 0.5f * a.lo}; }
  __device__ __forceinline__ static void mac(f2& acc, f2 a, f2 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float s = __fadd_rn(acc.hi, p);
    const float bb = __fsub_rn(s, acc.hi);
    const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
  }
};
