// hydro_device.cuh -- device-side arithmetic of the finite-volume hydro update
// (GenASiS, Cardall et al., arXiv:1207.3392, Secs. 3.1-3.5) for sm_103a.
//
// Variables: conserved U = (D, S_1..S_ndim, G), primitive W = (n, v_1..v_ndim, e),
// auxiliary p = (gamma-1) e, m = 1 (Sec. 3.5).  NV = ndim + 2 per cell.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dword.cuh"

namespace gh {

enum : int { BC_PERIODIC = 0, BC_REFLECT = 1, BC_OUTFLOW = 2 };
// SOLVER_HLLC_SW: HLLC, with HLL on faces transverse to a shock (Sec. 3.2)
enum : int { SOLVER_HLL = 0, SOLVER_HLLC = 1, SOLVER_HLLC_SW = 2 };
enum : unsigned { STATUS_NONPHYS = 1u, STATUS_TIMEOUT = 2u };

// Per-cell reconstruction geometry along one axis (Eq. MinMod with
// non-uniform centre distances): theta / (q_c - q_-), 1 / (q_+ - q_-),
// theta / (q_+ - q_c), and the half width (face offset from the geometric
// centre).  The limiter parameter theta is folded into the one-sided terms.
template <class T>
struct __align__(sizeof(T) * 4) Geo {
  T ticm, ipm, tipc, h;
};

// Ghost-cell source along one axis: periodic wrap, reflecting mirror (normal
// momentum negated), or outflow copy of the edge cell.  Indices beyond the two
// ghost layers are clamped onto the outermost ghost so every load stays in
// bounds (such cells only ever feed discarded results).
__device__ __forceinline__ int bc_map(int c, int n, int bc_lo, int bc_hi, bool& flip) {
  flip = false;
  if (c >= 0 && c < n) return c;
  if (c < 0) {
    c = c < -2 ? -2 : c;
    if (bc_lo == BC_PERIODIC) return c + n;
    if (bc_lo == BC_REFLECT) { flip = true; return -1 - c; }
    return 0;
  }
  c = c > n + 1 ? n + 1 : c;
  if (bc_hi == BC_PERIODIC) return c - n;
  if (bc_hi == BC_REFLECT) { flip = true; return 2 * n - 1 - c; }
  return n - 1;
}

// Three-argument minmod: zero unless all arguments share a strict sign, else
// the one of smallest magnitude (Eq. MinMod).
template <class T>
__device__ __forceinline__ T minmod3(T a, T b, T c) {
  T lo = fmin(a, fmin(b, c));
  T hi = fmax(a, fmax(b, c));
  return lo > T(0) ? lo : (hi < T(0) ? hi : T(0));
}

// FP32: the extremes from the three-input min/max of sm_100+, and the case
// split as max(lo, 0) + min(hi, 0) (one of the two terms is zero): the same
// value as the template above in five instructions instead of eight.
__device__ __forceinline__ float minmod3(float a, float b, float c) {
  float lo, hi;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(lo) : "f"(a), "f"(b), "f"(c));
  asm("max.f32 %0, %1, %2, %3;" : "=f"(hi) : "f"(a), "f"(b), "f"(c));
  return fmaxf(lo, 0.0f) + fminf(hi, 0.0f);
}

// FP64: the extremes and sign tests on the integer pipe.  GB300's FP64 pipe
// is the bound of the FP64 path (~2 operations per clock per SM), its integer
// ALU far from it.  A double's bits, with the magnitude bits flipped when the
// sign is set, order as signed integers like the doubles (NaN aside); -0.0
// maps to -1 and +0.0 to 0.  The values returned are the operands themselves.
__device__ __forceinline__ long long okey(double x) {
  const long long i = __double_as_longlong(x);
  return i ^ ((i >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double minmod3(double a, double b, double c) {
  const long long ka = okey(a), kb = okey(b), kc = okey(c);
  long long klo = ka, khi = ka;
  double lo = a, hi = a;
  if (kb < klo) { klo = kb; lo = b; }
  if (kb > khi) { khi = kb; hi = b; }
  if (kc < klo) { klo = kc; lo = c; }
  if (kc > khi) { khi = kc; hi = c; }
  return klo > 0 ? lo : (khi < -1 ? hi : 0.0);  // strictly positive / strictly negative
}

// max(0, a, b), x == 0 and x >= 0 for the wave speeds and the HLLC branch:
// plain for float and double word, on the integer pipe for double.
template <class T>
__device__ __forceinline__ T max0(T a, T b) { return fmax(T(0), fmax(a, b)); }
__device__ __forceinline__ double max0(double a, double b) {
  const long long ka = okey(a), kb = okey(b);
  const double m = ka < kb ? b : a;
  return (ka < kb ? kb : ka) > 0 ? m : 0.0;
}
template <class T>
__device__ __forceinline__ bool is_zero(T x) { return x == T(0); }
__device__ __forceinline__ bool is_zero(double x) { return ((unsigned long long)__double_as_longlong(x) << 1) == 0; }
template <class T>
__device__ __forceinline__ bool nonneg(T x) { return x >= T(0); }
__device__ __forceinline__ bool nonneg(double x) { return okey(x) >= -1; }

// Limited slope of cell c from its neighbours (Eq. MinMod; theta is in g).
template <class T>
__device__ __forceinline__ T limited_slope(T wm, T wc, T wp, const Geo<T>& g) {
  return minmod3((wc - wm) * g.ticm, (wp - wm) * g.ipm, (wp - wc) * g.tipc);
}

// Division, reciprocal and square root used by the flux arithmetic.  FP64
// takes Newton reciprocals from an FP32 seed (a few ulp, far inside its 1e-10
// parity bar); FP32 uses the hardware approximations (a few ulp, far inside
// its 1e-5 bar).
// FP64 reciprocal by Newton's method for 1/x: the FP32 hardware approximation
// as the seed (relative error ~2^-22), then two steps r <- r + r (1 - x r),
// each of which squares the relative error (~2^-44, then the FP64 rounding
// level): four FP64 FMAs in place of an IEEE division on GB300's slow FP64
// pipe, within a few ulp.  Arguments whose exponent lies outside the normal
// FP32 range (and 0, infinities, NaN) take the IEEE division; the test is on
// the exponent bits, on the integer pipe.
__device__ __forceinline__ double frcp(double x) {
  const unsigned ex = (unsigned)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ffu;
  if (ex - 900u > 246u) return 1.0 / x;  // biased exponent outside [900, 1146] (|x| ~ 1e-37 .. 1e37)
  double r = (double)__fdividef(1.0f, (float)x);
  r = fma(r, fma(-x, r, 1.0), r);
  r = fma(r, fma(-x, r, 1.0), r);
  return r;
}
// a / b from the reciprocal and one residual correction q + r (a - b q).
__device__ __forceinline__ double fdiv(double a, double b) {
  const double r = frcp(b);
  const double q = a * r;
  return fma(r, fma(-b, q, a), q);
}
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float frcp(float x) { return __fdividef(1.0f, x); }
// Correctly rounded sum that the compiler may not fuse with a product feeding
// it: keeps the stage combine bitwise the same in every kernel that inlines it,
// whatever the surrounding code lets the compiler contract.
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
// sqrt of a positive argument
__device__ __forceinline__ double fsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float fsqrt(float x) { return x * rsqrtf(x); }
// double-word: the operations of dword.cuh
__device__ __forceinline__ dw fdiv(dw a, dw b) { return a / b; }
__device__ __forceinline__ dw frcp(dw x) { return dw(1.0f, 0.0f) / x; }
__device__ __forceinline__ dw fsqrt(dw x) { return sqrt(x); }
__device__ __forceinline__ dw add_rn(dw a, dw b) { return a + b; }

// Sound speed c = sqrt(gamma p / n) (Sec. 3.5).  FP64: gamma p rsqrt(gamma p n),
// one reciprocal square root (CUDA's rsqrt, 1 ulp) in place of an IEEE division
// and an IEEE square root on the slow FP64 pipe; 0 where gamma p is not
// positive.  FP32: the same form with the hardware approximation (one
// multi-function-unit operation instead of two).  Double word: the quotient
// and square root of dword.cuh.
template <class T>
__device__ __forceinline__ T sound_speed(T gamma, T p, T n) { return fsqrt(gamma * fdiv(p, n)); }
__device__ __forceinline__ float sound_speed(float gamma, float p, float n) {
  const float gp = gamma * p;
  return gp * rsqrtf(gp * n);
}
__device__ __forceinline__ double sound_speed(double gamma, double p, double n) {
  const double gp = gamma * p;
  return okey(gp) > 0 ? gp * rsqrt(gp * n) : 0.0;
}

// ---------------------------------------------------------------------------
// Conserved -> primitive recovery.
//
// FP64 path: plain double arithmetic.
// Mixed path (FP32 storage): e = G - |S|^2 / (2 D) cancels when the kinetic
// energy density is a large part of G.  Where the kinetic part is at most
// half of G the FP32 difference loses at most one bit and is used as is;
// elsewhere the difference is formed in FP64 as e D = G D - |S|^2 / 2, where
// every product of two FP32 values is exact, so the cancellation loses
// nothing, and the well-conditioned division by D runs in FP32.
// ---------------------------------------------------------------------------
template <int NDIM>
__device__ __forceinline__ void recover(const double (&u)[NDIM + 2], double (&w)[NDIM + 2]) {
  constexpr int NV = NDIM + 2;
  const double rn = frcp(u[0]);
  double v2 = 0.0;
  w[0] = u[0];
#pragma unroll
  for (int q = 0; q < NDIM; ++q) {
    w[1 + q] = u[1 + q] * rn;
    v2 += w[1 + q] * w[1 + q];
  }
  w[NV - 1] = u[NV - 1] - 0.5 * u[0] * v2;
}

// e D = G D - |S|^2 / 2 in FP64 (products of FP32 values are exact in FP64).
// Kept out of line so that only lanes that need it execute FP64 instructions.
static __device__ __noinline__ float energy_density_times_n_fp64(float n, float s1, float s2, float s3, float G) {
  const double s2d = fma((double)s1, (double)s1, fma((double)s2, (double)s2, (double)s3 * (double)s3));
  return (float)fma(-0.5, s2d, (double)G * (double)n);
}

// Double-word path: the FP64 formulas in double-word arithmetic.
template <int NDIM>
__device__ __forceinline__ void recover(const dw (&u)[NDIM + 2], dw (&w)[NDIM + 2]) {
  constexpr int NV = NDIM + 2;
  const dw rn = frcp(u[0]);
  dw v2 = dw(0.0f, 0.0f);
  w[0] = u[0];
#pragma unroll
  for (int q = 0; q < NDIM; ++q) {
    w[1 + q] = u[1 + q] * rn;
    v2 = fma(w[1 + q], w[1 + q], v2);
  }
  w[NV - 1] = u[NV - 1] - dw(0.5f, 0.0f) * u[0] * v2;
}

template <int NDIM>
__device__ __forceinline__ void recover(const float (&u)[NDIM + 2], float (&w)[NDIM + 2]) {
  constexpr int NV = NDIM + 2;
  const float rn = frcp(u[0]);
  float s2 = 0.0f;
#pragma unroll
  for (int q = 0; q < NDIM; ++q) s2 = fmaf(u[1 + q], u[1 + q], s2);
  const float ke = 0.5f * s2 * rn;
  float e = u[NV - 1] - ke;
  if (__builtin_expect(!(ke <= 0.5f * u[NV - 1]), 0)) {
    const float eD = energy_density_times_n_fp64(u[0], u[1], NDIM > 1 ? u[2] : 0.0f, NDIM > 2 ? u[3] : 0.0f,
                                                 u[NV - 1]);
    e = eD * rn;
  }
  w[0] = u[0];
#pragma unroll
  for (int q = 0; q < NDIM; ++q) w[1 + q] = u[1 + q] * rn;
  w[NV - 1] = e;
}

// ---------------------------------------------------------------------------
// Face flux along axis Q from reconstructed primitive states on the left (wl)
// and right (wr) of the face (Eqs. conservedLeft..conservedRight).
//   wave speeds  alpha_+ = max(0, v_L + c_L, v_R + c_R),
//                alpha_- = max(0, c_L - v_L, c_R - v_R)         (Sec. 3.2, 3.5)
//   HLL          Eq. FluxHLL
//   HLLC         Eq. MiddleWaveSpeed for alpha_m, then one middle state on the
//                side selected by the sign of alpha_m (Eq. FluxHLLC), written
//                with the signed outer wave speed S_K (S_L = -alpha_-,
//                S_R = alpha_+):
//                  D*  = D_K (S_K - v_K) / (S_K - alpha_m)
//                  p*  = p_K + D_K (S_K - v_K)(alpha_m - v_K)
//                  G*  = [(S_K - v_K) G_K - p_K v_K + p* alpha_m] / (S_K - alpha_m)
//                  S*  = D* (alpha_m e_Q + transverse v_K)
//                  F*  = F_K + S_K (U* - U_K)
//                which are the outer jump conditions of Sec. 3.2 solved for the
//                middle state (this form satisfies p*_L = p*_R).
//                alpha_- = 0 gives F_L, alpha_+ = 0 gives F_R (upwind): those
//                cases select that side, where S_K = 0, so F* = F_K exactly
//                once the factor 1 / (S_K - alpha_m) of the (unused) middle
//                state is replaced by 0 to keep it finite.
// ---------------------------------------------------------------------------
// Conserved state U(W) and physical flux F^Q(U) of one side of a face
// (Sec. 3.5): p is its pressure, w[1 + Q] its normal velocity.
template <class T, int NDIM, int Q>
__device__ __forceinline__ void side_state(const T (&w)[NDIM + 2], T p, T (&u)[NDIM + 2], T (&f)[NDIM + 2]) {
  constexpr int NV = NDIM + 2;
  const T n = w[0], vq = w[1 + Q];
  T v2 = T(0);
#pragma unroll
  for (int q = 0; q < NDIM; ++q) v2 += w[1 + q] * w[1 + q];
  u[0] = n;
#pragma unroll
  for (int q = 0; q < NDIM; ++q) u[1 + q] = n * w[1 + q];
  u[NV - 1] = w[NV - 1] + T(0.5) * n * v2;
#pragma unroll
  for (int v = 0; v < NV - 1; ++v) f[v] = u[v] * vq;
  f[1 + Q] += p;
  f[NV - 1] = (u[NV - 1] + p) * vq;
}

template <class T, int NDIM, int Q, int SOLVER>
__device__ __forceinline__ void face_flux(const T (&wl)[NDIM + 2], const T (&wr)[NDIM + 2],
                                          T gamma, T gm1, T (&F)[NDIM + 2]) {
  constexpr int NV = NDIM + 2;
  const T nl = wl[0], nr = wr[0];
  const T pl = gm1 * wl[NV - 1], pr = gm1 * wr[NV - 1];
  const T vl = wl[1 + Q], vr = wr[1 + Q];
  const T cl = sound_speed(gamma, pl, nl);
  const T cr = sound_speed(gamma, pr, nr);
  const T ap = max0(vl + cl, vr + cr);
  const T am = max0(cl - vl, cr - vr);

  if constexpr (SOLVER == SOLVER_HLL) {
    T ul[NV], ur[NV], fl[NV], fr[NV];
    side_state<T, NDIM, Q>(wl, pl, ul, fl);
    side_state<T, NDIM, Q>(wr, pr, ur, fr);
    const T inv = frcp(ap + am);
    const T apam = ap * am;
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = (ap * fl[v] + am * fr[v] - apam * (ur[v] - ul[v])) * inv;
  } else {
    // HLLC.  Only the selected side K enters F* = F_K + S_K (U* - U_K), so
    // its primitives are selected first and U_K, F_K formed once.
    const T sl = am + vl;  // = -(S_L - v_L) > 0
    const T sr = ap - vr;  // =   S_R - v_R  > 0
    const T ml = nl * vl, mr = nr * vr;  // normal momenta
    const T alpha_m = fdiv(mr * sr + ml * sl - (pr - pl), nr * sr + nl * sl);
    const bool left = is_zero(am) || (!is_zero(ap) && nonneg(alpha_m));
    const T SK = left ? -am : ap;
    const T pK = left ? pl : pr;
    T wK[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) wK[v] = left ? wl[v] : wr[v];
    const T nK = wK[0], vK = wK[1 + Q];
    T uK[NV], fK[NV];
    side_state<T, NDIM, Q>(wK, pK, uK, fK);
    const T dK = SK - vK;  // S_K - v_K
    const T rden = is_zero(SK) ? T(0) : frcp(SK - alpha_m);
    const T Ds = nK * dK * rden;
    const T ps = pK + nK * dK * (alpha_m - vK);
    T us[NV];
    us[0] = Ds;
#pragma unroll
    for (int q = 0; q < NDIM; ++q) us[1 + q] = Ds * (q == Q ? alpha_m : wK[1 + q]);
    us[NV - 1] = (dK * uK[NV - 1] - pK * vK + ps * alpha_m) * rden;
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = fK[v] + SK * (us[v] - uK[v]);
  }
}

// Column sums of the conserved totals.  FP64 state: plain FP64 FMA.  FP32
// state: a compensated pair of floats (Knuth's TwoSum plus the exact rounding
// error of each product from an FMA), about 48 significant bits, so no FP64
// instruction runs per cell; the pair is folded into FP64 once per column.
template <class T>
struct ColumnSum;

template <>
struct ColumnSum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add_product(double u, double dz_hi, double) { s = fma(u, dz_hi, s); }
  __device__ __forceinline__ double value() const { return s; }
};

template <>
struct ColumnSum<float> {
  float hi = 0.0f, lo = 0.0f;
  // add u * (dz_hi + dz_lo)
  __device__ __forceinline__ void add_product(float u, float dz_hi, float dz_lo) {
    const float p = u * dz_hi;
    const float pe = fmaf(u, dz_hi, -p) + u * dz_lo;
    const float t = hi + p;
    const float bp = t - hi;
    const float err = (hi - (t - bp)) + (p - bp);
    hi = t;
    lo += err + pe;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Double-word state: the column sum in double-word arithmetic (dz as a pair).
template <>
struct ColumnSum<dw> {
  dw s = dw(0.0f, 0.0f);
  __device__ __forceinline__ void add_product(dw u, dw dz, dw) { s = fma(u, dz, s); }
  __device__ __forceinline__ double value() const { return (double)s; }
};

// Deterministic block reductions (fixed shuffle tree, then warps in order).
template <class T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
template <class T>
__device__ __forceinline__ T warp_max(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

}  // namespace gh
