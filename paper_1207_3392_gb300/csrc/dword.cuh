// dword.cuh -- double-word arithmetic: a value is the unevaluated sum hi + lo
// of two FP32 numbers (|lo| <= ulp(hi)/2), about 48 significant bits.  It runs
// the FP64 update on the FP32 pipes, whose rate on this GPU is many times the
// FP64 rate.  Building blocks:
//   TwoSum (Knuth, TAOCP vol. 2), FastTwoSum (Dekker 1971) and TwoProd by FMA
//   are error-free; addition is the short double-word sum (TwoSum of the
//   high parts, the low parts added in, one FastTwoSum): its error is at most
//   ~2u^2 |x| + 2u^2 |y| (u = 2^-24), relative to the operands like an FP64
//   sum, though not relative to a cancelled result; the product is Joldes,
//   Muller and Popescu's FMA-based double-word product (ACM TOMS 44(2), 2017,
//   relative error <= 5u^2);
//   division is Dekker's: an approximate float quotient q1 = x.hi / y.hi, the
//   exact residual x - q1 y in double-word (x.hi - q1 y.hi is exact because
//   q1 y.hi lies within a factor 2 of x.hi), and a second quotient of that
//   residual; the approximate reciprocal of the hardware suffices because the
//   residual corrects q1;
//   square root is one Newton correction of an approximate float root s from
//   the exact residual x - s^2.
// The operations are hidden friends (found by argument-dependent lookup), so
// they add to, rather than hide, the float and double overloads of fma,
// fmax, fmin, fabs and __ldg.  Every float operation is an explicitly rounded
// intrinsic, so the compiler cannot contract or reassociate the
// error-free transformations.
#pragma once

#include <cuda_runtime.h>

namespace gh {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

struct __align__(8) dw {
  float hi, lo;

  dw() = default;
  __host__ __device__ constexpr dw(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ dw(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ dw(int x) : dw((double)x) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ explicit operator float() const { return (float)((double)hi + (double)lo); }

  friend __device__ __forceinline__ dw operator-(dw x) { return dw(-x.hi, -x.lo); }

  friend __device__ __forceinline__ dw operator+(dw x, dw y) {
    float sh, sl, zh, zl;
    two_sum(x.hi, y.hi, sh, sl);
    fast_two_sum(sh, __fadd_rn(sl, __fadd_rn(x.lo, y.lo)), zh, zl);
    return dw(zh, zl);
  }
  friend __device__ __forceinline__ dw operator-(dw x, dw y) { return x + (-y); }

  friend __device__ __forceinline__ dw operator*(dw x, dw y) {
    float ch, cl1, zh, zl;
    two_prod(x.hi, y.hi, ch, cl1);
    const float tl0 = __fmul_rn(x.lo, y.lo);
    const float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
    const float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
    fast_two_sum(ch, __fadd_rn(cl1, cl2), zh, zl);
    return dw(zh, zl);
  }

  friend __device__ __forceinline__ dw operator/(dw x, dw y) {
    const float r0 = __fdividef(1.0f, y.hi);  // hardware reciprocal, a few ulp
    const float q1 = __fmul_rn(x.hi, r0);
    float ph, pl, zh, zl;
    two_prod(q1, y.hi, ph, pl);
    const float rh = __fsub_rn(x.hi, ph);  // exact: q1 y.hi is within a factor 2 of x.hi
    const float r = __fadd_rn(__fsub_rn(rh, pl), __fmaf_rn(-q1, y.lo, x.lo));
    fast_two_sum(q1, __fmul_rn(r, r0), zh, zl);
    return dw(zh, zl);
  }

  friend __device__ __forceinline__ dw& operator+=(dw& x, dw y) { return x = x + y; }
  friend __device__ __forceinline__ dw& operator-=(dw& x, dw y) { return x = x - y; }

  // ordering of normalised pairs: by hi, then by lo
  friend __device__ __forceinline__ bool operator<(dw x, dw y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }
  friend __device__ __forceinline__ bool operator>(dw x, dw y) { return y < x; }
  friend __device__ __forceinline__ bool operator<=(dw x, dw y) { return x.hi < y.hi || (x.hi == y.hi && x.lo <= y.lo); }
  friend __device__ __forceinline__ bool operator>=(dw x, dw y) { return y <= x; }
  friend __device__ __forceinline__ bool operator==(dw x, dw y) { return x.hi == y.hi && x.lo == y.lo; }
  friend __device__ __forceinline__ bool operator!=(dw x, dw y) { return !(x == y); }

  friend __device__ __forceinline__ dw fma(dw a, dw b, dw c) { return a * b + c; }
  friend __device__ __forceinline__ dw fabs(dw x) { return x.hi < 0.0f ? -x : x; }
  friend __device__ __forceinline__ dw fmax(dw x, dw y) { return x < y ? y : x; }
  friend __device__ __forceinline__ dw fmin(dw x, dw y) { return y < x ? y : x; }

  friend __device__ __forceinline__ dw sqrt(dw x) {
    if (!(x.hi > 0.0f)) return dw(sqrtf(x.hi), 0.0f);  // 0, or NaN for a negative argument
    const float rs = rsqrtf(x.hi);  // hardware reciprocal square root, a few ulp
    const float s = __fmul_rn(x.hi, rs);
    float ph, pl, zh, zl;
    two_prod(s, s, ph, pl);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, ph), pl), x.lo);  // x.hi - ph exact
    fast_two_sum(s, __fmul_rn(r, __fmul_rn(0.5f, rs)), zh, zl);
    return dw(zh, zl);
  }

  friend __device__ __forceinline__ dw __ldg(const dw* p) {
    const float2 v = ::__ldg(reinterpret_cast<const float2*>(p));
    return dw(v.x, v.y);
  }
};

}  // namespace gh
