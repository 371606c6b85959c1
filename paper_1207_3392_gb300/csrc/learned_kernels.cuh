// learned_kernels.cuh -- device code of the learned flux correction for 2D
// runs: per-face features and plain fluxes, MLP inference and training on
// BF16 tensor cores, the corrected update with its positivity fallback, and
// the face-flux accumulation and restriction that build training targets
// from fine runs.  (The correction is the benchmark's addition to Sec. 3.2's
// HLLC flux; the paper has no counterpart.)
#pragma once

#include "hydro_device.cuh"
#include "mlp.cuh"

namespace gh {

// Cell index along an axis of n cells with up to n ghost cells on each side:
// periodic wrap, reflecting mirror (flip = normal momentum negated), outflow
// clamp.  Used where stencils reach three cells out.
__device__ __forceinline__ int wrap_cell(int c, int n, int bc_lo, int bc_hi, bool& flip) {
  flip = false;
  if (c >= 0 && c < n) return c;
  if (c < 0) {
    if (bc_lo == BC_PERIODIC) return ((c % n) + n) % n;
    if (bc_lo == BC_REFLECT) { flip = true; c = -1 - c; return c < n ? c : n - 1; }
    return 0;
  }
  if (bc_hi == BC_PERIODIC) return c % n;
  if (bc_hi == BC_REFLECT) { flip = true; c = 2 * n - 1 - c; return c >= 0 ? c : 0; }
  return n - 1;
}

// A 2D mesh for the learned path (FP32 state).
struct Mesh2 {
  int nx, ny;
  int bc_lo[2], bc_hi[2];
  float gamma, gm1;
  const Geo<float>* geo[2];   // index c + 2, c in [-2, n + 2)
  const float* iw[2];
};

// Load through L2 only (ld.global.cg) when COH, for arrays written earlier in
// the same launch; a plain load otherwise.
template <bool COH, class V>
__device__ __forceinline__ V lf_ld(const V* p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}

// Conserved state of cell (i, j) (any integer indices), as U = un + dt * k when
// k is non-null, with boundary mapping; returns primitives (n, vx, vy, e).
template <bool COH = false>
__device__ __forceinline__ void cell_prim(const Mesh2& M, const float* __restrict__ un, const float* __restrict__ k,
                                          float dt, int i, int j, float (&w)[4]) {
  bool fx, fy;
  const int si = wrap_cell(i, M.nx, M.bc_lo[0], M.bc_hi[0], fx);
  const int sj = wrap_cell(j, M.ny, M.bc_lo[1], M.bc_hi[1], fy);
  const size_t vs = (size_t)M.nx * M.ny, c = (size_t)sj * M.nx + si;
  float u[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    float x = lf_ld<COH>(un + v * vs + c);
    if (k) x = fmaf(dt, lf_ld<COH>(k + v * vs + c), x);
    u[v] = x;
  }
  if (fx) u[1] = -u[1];
  if (fy) u[2] = -u[2];
  recover<2>(u, w);
}

__device__ __forceinline__ Geo<float> geo_at(const Mesh2& M, int q, int c) {
  const int n = q == 0 ? M.nx : M.ny;
  c = c < -2 ? -2 : (c > n + 1 ? n + 1 : c);
  return M.geo[q][c + 2];
}

// Plain face flux (Sec. 3.1 reconstruction + Sec. 3.2 Riemann solver) through
// the face between cells (i-1, j) and (i, j) (axis 0) or (i, j-1) and (i, j)
// (axis 1), from primitive stencils w[0..3] = cells -2, -1, 0, +1 along the axis.
template <int Q, int SOLVER>
__device__ __forceinline__ void plain_face_flux(const Mesh2& M, const float (&w)[4][4], int cl, float (&F)[4]) {
  const Geo<float> gl = geo_at(M, Q, cl), gr = geo_at(M, Q, cl + 1);
  float wl[4], wr[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    wl[v] = fmaf(limited_slope(w[0][v], w[1][v], w[2][v], gl), gl.h, w[1][v]);
    wr[v] = fmaf(-limited_slope(w[1][v], w[2][v], w[3][v], gr), gr.h, w[2][v]);
  }
  face_flux<float, 2, Q, SOLVER>(wl, wr, M.gamma, M.gm1, F);
}

// Features (24) and flux scales (4) of a face from its six-cell primitive
// stencil s[0..5] (cells -3 .. +2 along the normal Q): per cell
// rho/rho_bar - 1, v_n/c_bar, v_t/c_bar, p/p_bar - 1 with rho_bar, p_bar the
// stencil means and c_bar = sqrt(gamma p_bar / rho_bar); scales
// (rho_bar c_bar, rho_bar c_bar^2, rho_bar c_bar^2, rho_bar c_bar^3).
// x receives the four 16-byte chunks of the row xstride uint4 apart (1: a
// plain row; 8: a row of the tensor cores' core-matrix layout).
template <int Q>
__device__ __forceinline__ void face_features(const Mesh2& M, const float (&s)[6][4], __nv_bfloat16* __restrict__ x,
                                              float* __restrict__ scale, int xstride = 1) {
  // Every rounding is spelt out (the pressures as separate products, the
  // ratios minus one as fused multiply-adds), so that each kernel that inlines
  // this computes bitwise the same features.
  float pk[6], rs = 0.f, ps = 0.f;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    pk[k] = __fmul_rn(M.gm1, s[k][3]);
    rs += s[k][0];
    ps += pk[k];
  }
  const float rbar = rs * (1.0f / 6.0f), pbar = ps * (1.0f / 6.0f);
  const float cbar = sqrtf(M.gamma * pbar / rbar);
  const float ir = 1.0f / rbar, ip = 1.0f / pbar, ic = 1.0f / cbar;
  uint32_t packed[16];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float vn = s[k][1 + Q], vt = s[k][2 - Q];
    packed[2 * k] = mlp::pack2(fmaf(s[k][0], ir, -1.0f), vn * ic);
    packed[2 * k + 1] = mlp::pack2(vt * ic, fmaf(pk[k], ip, -1.0f));
  }
#pragma unroll
  for (int k = 12; k < 16; ++k) packed[k] = 0u;
  uint4* dst = reinterpret_cast<uint4*>(x);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    dst[k * xstride] = make_uint4(packed[4 * k], packed[4 * k + 1], packed[4 * k + 2], packed[4 * k + 3]);
  const float rc = rbar * cbar;
  scale[0] = rc;
  scale[1] = rc * cbar;
  scale[2] = rc * cbar;
  scale[3] = rc * cbar * cbar;
}

}  // namespace gh
