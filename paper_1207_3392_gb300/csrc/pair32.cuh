// pair32.cuh -- two FP32 values per register pair, computed with the packed
// FP32 instructions of sm_100+ ({add,sub,mul,fma}.rn.f32x2: two results per
// issue slot), and the parts of the hydro update (Secs. 3.1-3.5) that the
// z-paired 3D stage kernel (stage_pair.cuh) runs on such pairs: the two lanes
// hold the same cell of two consecutive march planes.
//
// Every rounding is written out (no product is left for the compiler to fuse
// or not), so a value comes out the same whichever lane computes it: a face
// flux computed by the CTAs on both sides of a chunk boundary, in either
// lane, has the same bits, and the update stays conservative.  Operations
// without a packed form (min/max, compare and select, the multi-function
// unit's reciprocal and reciprocal square root) run per lane.
#pragma once

#include <cuda_runtime.h>

#include "hydro_device.cuh"

namespace gh {

using f2 = float2;

__device__ __forceinline__ f2 mk2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ f2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 r;
  asm("{.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ f2 neg2(f2 a) { return mk2(-a.x, -a.y); }
__device__ __forceinline__ f2 abs2(f2 a) { return mk2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ f2 max2(f2 a, f2 b) { return mk2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
// lane-wise: c ? a : b
__device__ __forceinline__ f2 sel2(bool cx, bool cy, f2 a, f2 b) { return mk2(cx ? a.x : b.x, cy ? a.y : b.y); }
// the reciprocal and quotient of the scalar FP32 path, per lane
__device__ __forceinline__ f2 frcp2(f2 a) { return mk2(frcp(a.x), frcp(a.y)); }
__device__ __forceinline__ f2 fdiv2(f2 a, f2 b) { return mk2(fdiv(a.x, b.x), fdiv(a.y, b.y)); }

// Reconstruction geometry of one axis as pairs (Geo of hydro_device.cuh), with
// the negated half width for the lower-face value W - s h.
struct Geo2 {
  f2 ticm, ipm, tipc, h, nh;
};
__device__ __forceinline__ Geo2 geo2(const Geo<float>& a, const Geo<float>& b) {
  Geo2 g;
  g.ticm = mk2(a.ticm, b.ticm);
  g.ipm = mk2(a.ipm, b.ipm);
  g.tipc = mk2(a.tipc, b.tipc);
  g.h = mk2(a.h, b.h);
  g.nh = mk2(-a.h, -b.h);
  return g;
}

// Eq. MinMod per lane: the three-input extremes, then max(lo, 0) + min(hi, 0)
// (one term is zero, so the sum is exact), the sum as one packed add.
__device__ __forceinline__ f2 minmod3_2(f2 a, f2 b, f2 c) {
  float lx, hx, ly, hy;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(lx) : "f"(a.x), "f"(b.x), "f"(c.x));
  asm("max.f32 %0, %1, %2, %3;" : "=f"(hx) : "f"(a.x), "f"(b.x), "f"(c.x));
  asm("min.f32 %0, %1, %2, %3;" : "=f"(ly) : "f"(a.y), "f"(b.y), "f"(c.y));
  asm("max.f32 %0, %1, %2, %3;" : "=f"(hy) : "f"(a.y), "f"(b.y), "f"(c.y));
  return add2(mk2(fmaxf(lx, 0.0f), fmaxf(ly, 0.0f)), mk2(fminf(hx, 0.0f), fminf(hy, 0.0f)));
}

__device__ __forceinline__ f2 limited_slope2(f2 wm, f2 wc, f2 wp, const Geo2& g) {
  return minmod3_2(mul2(sub2(wc, wm), g.ticm), mul2(sub2(wp, wm), g.ipm), mul2(sub2(wp, wc), g.tipc));
}

// c = gamma p rsqrt(gamma p n) (Sec. 3.5), the form of the scalar FP32 path.
__device__ __forceinline__ f2 sound_speed2(f2 gamma, f2 p, f2 n) {
  const f2 gp = mul2(gamma, p);
  const f2 q = mul2(gp, n);
  return mul2(gp, mk2(rsqrtf(q.x), rsqrtf(q.y)));
}

// Conserved -> primitive (3D): n = D, v = S / D, e = G - |S|^2 / (2D); a lane
// whose kinetic energy exceeds half of G recomputes e in FP64, as the scalar
// FP32 path does.
__device__ __forceinline__ void recover2(const f2 (&u)[5], f2 (&w)[5]) {
  const f2 rn = frcp2(u[0]);
  f2 s2 = mul2(u[1], u[1]);
  s2 = fma2(u[2], u[2], s2);
  s2 = fma2(u[3], u[3], s2);
  const f2 ke = mul2(mul2(bc2(0.5f), s2), rn);
  f2 e = sub2(u[4], ke);
  if (__builtin_expect(!(ke.x <= 0.5f * u[4].x), 0))
    e.x = energy_density_times_n_fp64(u[0].x, u[1].x, u[2].x, u[3].x, u[4].x) * rn.x;
  if (__builtin_expect(!(ke.y <= 0.5f * u[4].y), 0))
    e.y = energy_density_times_n_fp64(u[0].y, u[1].y, u[2].y, u[3].y, u[4].y) * rn.y;
  w[0] = u[0];
  w[1] = mul2(u[1], rn);
  w[2] = mul2(u[2], rn);
  w[3] = mul2(u[3], rn);
  w[4] = e;
}

// U(W) and F^Q(U) of one face side (Sec. 3.5), p its pressure.
template <int Q>
__device__ __forceinline__ void side_state2(const f2 (&w)[5], f2 p, f2 (&u)[5], f2 (&f)[5]) {
  const f2 n = w[0], vq = w[1 + Q];
  f2 v2 = mul2(w[1], w[1]);
  v2 = fma2(w[2], w[2], v2);
  v2 = fma2(w[3], w[3], v2);
  u[0] = n;
  u[1] = mul2(n, w[1]);
  u[2] = mul2(n, w[2]);
  u[3] = mul2(n, w[3]);
  u[4] = fma2(mul2(bc2(0.5f), n), v2, w[4]);
#pragma unroll
  for (int v = 0; v < 4; ++v) f[v] = mul2(u[v], vq);
  f[1 + Q] = add2(f[1 + Q], p);
  f[4] = mul2(add2(u[4], p), vq);
}

// Face flux along axis Q (0, 1, 2) of a pair of faces: the HLL and HLLC fluxes
// of face_flux in hydro_device.cuh (Sec. 3.2, Eqs. FluxHLL, MiddleWaveSpeed,
// FluxHLLC), term for term, with the roundings written out.
template <int Q, int SOLVER>
__device__ __forceinline__ void face_flux2(const f2 (&wl)[5], const f2 (&wr)[5], f2 gamma, f2 gm1, f2 (&F)[5]) {
  const f2 nl = wl[0], nr = wr[0];
  const f2 pl = mul2(gm1, wl[4]), pr = mul2(gm1, wr[4]);
  const f2 vl = wl[1 + Q], vr = wr[1 + Q];
  const f2 cl = sound_speed2(gamma, pl, nl);
  const f2 cr = sound_speed2(gamma, pr, nr);
  const f2 ap = max2(bc2(0.0f), max2(add2(vl, cl), add2(vr, cr)));
  const f2 am = max2(bc2(0.0f), max2(sub2(cl, vl), sub2(cr, vr)));
  if constexpr (SOLVER == SOLVER_HLL) {
    f2 ul[5], ur[5], fl[5], fr[5];
    side_state2<Q>(wl, pl, ul, fl);
    side_state2<Q>(wr, pr, ur, fr);
    const f2 inv = frcp2(add2(ap, am));
    const f2 napam = mul2(neg2(ap), am);
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] = mul2(fma2(napam, sub2(ur[v], ul[v]), fma2(am, fr[v], mul2(ap, fl[v]))), inv);
  } else {
    const f2 sl = add2(am, vl);  // = -(S_L - v_L)
    const f2 sr = sub2(ap, vr);  // =   S_R - v_R
    const f2 ml = mul2(nl, vl), mr = mul2(nr, vr);
    const f2 alpha_m = fdiv2(fma2(mr, sr, fma2(ml, sl, sub2(pl, pr))), fma2(nr, sr, mul2(nl, sl)));
    const bool lx = am.x == 0.0f || (ap.x != 0.0f && alpha_m.x >= 0.0f);
    const bool ly = am.y == 0.0f || (ap.y != 0.0f && alpha_m.y >= 0.0f);
    const f2 SK = sel2(lx, ly, neg2(am), ap);
    const f2 pK = sel2(lx, ly, pl, pr);
    f2 wK[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) wK[v] = sel2(lx, ly, wl[v], wr[v]);
    const f2 nK = wK[0], vK = wK[1 + Q];
    f2 uK[5], fK[5];
    side_state2<Q>(wK, pK, uK, fK);
    const f2 dK = sub2(SK, vK);
    const f2 rc = frcp2(sub2(SK, alpha_m));
    const f2 rden = mk2(SK.x == 0.0f ? 0.0f : rc.x, SK.y == 0.0f ? 0.0f : rc.y);
    const f2 ndk = mul2(nK, dK);
    const f2 Ds = mul2(ndk, rden);
    const f2 ps = fma2(ndk, sub2(alpha_m, vK), pK);
    f2 us[5];
    us[0] = Ds;
#pragma unroll
    for (int q = 0; q < 3; ++q) us[1 + q] = mul2(Ds, q == Q ? alpha_m : wK[1 + q]);
    us[4] = mul2(fma2(ps, alpha_m, fma2(dK, uK[4], mul2(neg2(pK), vK))), rden);
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] = fma2(SK, sub2(us[v], uK[v]), fK[v]);
  }
}

// Compensated column sum of u dz per lane (ColumnSum<float> of
// hydro_device.cuh: TwoSum plus the product's rounding error).
struct ColumnSum2 {
  f2 hi = {0.0f, 0.0f}, lo = {0.0f, 0.0f};
  __device__ __forceinline__ void add_product(f2 u, f2 dz_hi, f2 dz_lo) {
    const f2 p = mul2(u, dz_hi);
    const f2 pe = fma2(u, dz_lo, fma2(u, dz_hi, neg2(p)));
    const f2 t = add2(hi, p);
    const f2 bp = sub2(t, hi);
    const f2 err = add2(sub2(hi, sub2(t, bp)), sub2(p, bp));
    hi = t;
    lo = add2(lo, add2(err, pe));
  }
  __device__ __forceinline__ double value() const {
    return ((double)hi.x + (double)lo.x) + ((double)hi.y + (double)lo.y);
  }
};

}  // namespace gh
