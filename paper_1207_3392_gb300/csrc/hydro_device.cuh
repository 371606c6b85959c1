// hydro_device.cuh -- device-side arithmetic of the finite-volume hydro update
// (GenASiS, Cardall et al., arXiv:1207.3392, Secs. 3.1-3.5) for sm_103a.
//
// Variables: conserved U = (D, S_1..S_ndim, G), primitive W = (n, v_1..v_ndim, e),
// auxiliary p = (gamma-1) e, m = 1 (Sec. 3.5).  NV = ndim + 2 per cell.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gh {

enum : int { BC_PERIODIC = 0, BC_REFLECT = 1, BC_OUTFLOW = 2 };
enum : int { SOLVER_HLL = 0, SOLVER_HLLC = 1 };
enum : unsigned { STATUS_NONPHYS = 1u, STATUS_TIMEOUT = 2u };

// Per-cell reconstruction geometry along one axis (Eq. MinMod with
// non-uniform centre distances): inverse distances centre-to-left-centre,
// left-to-right centre, centre-to-right-centre, and the half width (face
// offset from the geometric centre).
template <class T>
struct __align__(sizeof(T) * 4) Geo {
  T icm, ipm, ipc, h;
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

// Limited slope of cell c from its neighbours (Eq. MinMod).
template <class T>
__device__ __forceinline__ T limited_slope(T wm, T wc, T wp, const Geo<T>& g, T theta) {
  return minmod3(theta * ((wc - wm) * g.icm), (wp - wm) * g.ipm, theta * ((wp - wc) * g.ipc));
}

// ---------------------------------------------------------------------------
// Conserved -> primitive recovery.
//
// FP64 path: plain double arithmetic.
// Mixed path (FP32 storage): the cancelling difference G - |S|^2 / (2 D) is
// formed in FP64 as e D = G D - |S|^2 / 2, where every product of two FP32
// values is exact in FP64, so the cancellation loses nothing; the
// well-conditioned divisions v = S / D and e = (e D) / D then run in FP32.
// ---------------------------------------------------------------------------
template <int NDIM>
__device__ __forceinline__ void recover(const double (&u)[NDIM + 2], double (&w)[NDIM + 2]) {
  constexpr int NV = NDIM + 2;
  const double rn = 1.0 / u[0];
  double v2 = 0.0;
  w[0] = u[0];
#pragma unroll
  for (int q = 0; q < NDIM; ++q) {
    w[1 + q] = u[1 + q] * rn;
    v2 += w[1 + q] * w[1 + q];
  }
  w[NV - 1] = u[NV - 1] - 0.5 * u[0] * v2;
}

template <int NDIM>
__device__ __forceinline__ void recover(const float (&u)[NDIM + 2], float (&w)[NDIM + 2]) {
  constexpr int NV = NDIM + 2;
  double s2 = 0.0;
#pragma unroll
  for (int q = 0; q < NDIM; ++q) s2 = fma((double)u[1 + q], (double)u[1 + q], s2);
  const double eD = fma(-0.5, s2, (double)u[NV - 1] * (double)u[0]);
  const float rn = 1.0f / u[0];
  w[0] = u[0];
#pragma unroll
  for (int q = 0; q < NDIM; ++q) w[1 + q] = u[1 + q] * rn;
  w[NV - 1] = (float)eD * rn;
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
//                alpha_- = 0 gives F_L, alpha_+ = 0 gives F_R (upwind).
// ---------------------------------------------------------------------------
template <class T, int NDIM, int Q, int SOLVER>
__device__ __forceinline__ void face_flux(const T (&wl)[NDIM + 2], const T (&wr)[NDIM + 2],
                                          T gamma, T gm1, T (&F)[NDIM + 2]) {
  constexpr int NV = NDIM + 2;
  const T nl = wl[0], nr = wr[0];
  const T pl = gm1 * wl[NV - 1], pr = gm1 * wr[NV - 1];
  T v2l = T(0), v2r = T(0);
#pragma unroll
  for (int q = 0; q < NDIM; ++q) {
    v2l += wl[1 + q] * wl[1 + q];
    v2r += wr[1 + q] * wr[1 + q];
  }
  T ul[NV], ur[NV];
  ul[0] = nl;
  ur[0] = nr;
#pragma unroll
  for (int q = 0; q < NDIM; ++q) {
    ul[1 + q] = nl * wl[1 + q];
    ur[1 + q] = nr * wr[1 + q];
  }
  ul[NV - 1] = wl[NV - 1] + T(0.5) * nl * v2l;
  ur[NV - 1] = wr[NV - 1] + T(0.5) * nr * v2r;

  const T vl = wl[1 + Q], vr = wr[1 + Q];
  T fl[NV], fr[NV];
#pragma unroll
  for (int v = 0; v < NV - 1; ++v) {
    fl[v] = ul[v] * vl;
    fr[v] = ur[v] * vr;
  }
  fl[1 + Q] += pl;
  fr[1 + Q] += pr;
  fl[NV - 1] = (ul[NV - 1] + pl) * vl;
  fr[NV - 1] = (ur[NV - 1] + pr) * vr;

  const T cl = sqrt(gamma * pl / nl);
  const T cr = sqrt(gamma * pr / nr);
  const T ap = fmax(T(0), fmax(vl + cl, vr + cr));
  const T am = fmax(T(0), fmax(cl - vl, cr - vr));

  if (SOLVER == SOLVER_HLL) {
    const T inv = T(1) / (ap + am);
    const T apam = ap * am;
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = (ap * fl[v] + am * fr[v] - apam * (ur[v] - ul[v])) * inv;
    return;
  }

  // HLLC
  const T sl = am + vl;  // = -(S_L - v_L) > 0
  const T sr = ap - vr;  // =   S_R - v_R  > 0
  const T alpha_m = (ur[1 + Q] * sr + ul[1 + Q] * sl - (pr - pl)) / (nr * sr + nl * sl);
  const bool left = alpha_m >= T(0);
  const T SK = left ? -am : ap;
  const T nK = left ? nl : nr;
  const T vK = left ? vl : vr;
  const T pK = left ? pl : pr;
  const T dK = SK - vK;                       // S_K - v_K
  const T rden = T(1) / (SK - alpha_m);
  const T Ds = nK * dK * rden;
  const T ps = pK + nK * dK * (alpha_m - vK);
  T us[NV];
  us[0] = Ds;
#pragma unroll
  for (int q = 0; q < NDIM; ++q) us[1 + q] = Ds * (q == Q ? alpha_m : (left ? wl[1 + q] : wr[1 + q]));
  const T GK = left ? ul[NV - 1] : ur[NV - 1];
  us[NV - 1] = (dK * GK - pK * vK + ps * alpha_m) * rden;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const T fK = left ? fl[v] : fr[v];
    const T uK = left ? ul[v] : ur[v];
    T f = fK + SK * (us[v] - uK);
    f = (am == T(0)) ? fl[v] : f;
    f = (ap == T(0)) ? fr[v] : f;
    F[v] = f;
  }
}

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
