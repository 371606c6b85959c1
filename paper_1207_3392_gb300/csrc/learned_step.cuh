// learned_step.cuh -- the per-face and per-cell work of one RK stage of the
// corrected 2D scheme: the plain face flux (Sec. 3.1 reconstruction, Sec. 3.2
// Riemann solver) with the network features, the flux-corrected-transport
// ratios, and the corrected update with its positivity fallback.  The
// per-phase kernels of learned.cu and the one-launch advance of
// learned_advance.cu both call these, so the two paths do the same arithmetic
// on every face and cell.
//
// COH = true reads every array that a launch may itself have written (states,
// K, fluxes, network outputs, scales, ratios, flags) through L2
// (ld.global.cg): the phases of the one-launch advance see one another's
// writes across its grid barriers.  The geometry tables are read-only.
#pragma once

#include "learned_kernels.cuh"

namespace gh {

struct UpdateArgs {
  Mesh2 M;
  const float* un;
  const float* k1;      // stage 2: K of stage 1
  const double* dtp;
  const float* F;       // plain face fluxes [nf][4]
  const float* dY;      // network outputs [nf][4], or null (no correction)
  const float* scale;   // [nf][4]
  float* out;                   // stage 1: K; stage 2: U^{n+1}
  const unsigned char* flag;    // per cell: keeps the plain flux on all its faces (read)
  unsigned char* flag_out;      // flags for the next pass (written)
  unsigned long long* nfallback;
  unsigned* status;
  int stage;
  int fixup;                    // 0: corrected pass; k > 0: k-th widening pass; -1: all-plain pass
  int last;                     // last widening pass: remaining failures request the all-plain pass
  unsigned* all_plain;          // device flags: [0] redo the whole stage with plain fluxes,
                                // [1] some cell failed in the corrected pass of this stage
  float ylim;                   // network outputs are clamped to [-ylim, ylim]
  const float* R;               // FCT ratios [ncell][8] (R+ then R- per variable), or null
};

// The per-face arrays (fluxes, network outputs, flux scales) hold 4 floats
// per face and the FCT ratios 8 per cell, so that each is read with 16-byte
// loads.
template <bool COH>
__device__ __forceinline__ float4 lf_ld4(const float* p) {
  return lf_ld<COH>(reinterpret_cast<const float4*>(p));
}

// Plain flux of face f (x faces (nx+1) x ny first, then y faces nx x (ny+1))
// of the state un (+ dt k) into F [nf][4]; with x non-null also the face's 32
// BF16 features at x (16-byte chunks xstride uint4 apart) and its 4 flux
// scales at scale + 4 f.
template <int SOLVER, bool COH>
__device__ __forceinline__ void lf_face(const Mesh2& M, const float* un, const float* k, float dt, long long f,
                                        long long nxf, long long nf, float* F, __nv_bfloat16* x, float* scale,
                                        int xstride = 1) {
  float s[6][4], Fl[4];
  if (f < nxf) {
    const int i = (int)(f % (M.nx + 1)), j = (int)(f / (M.nx + 1));
#pragma unroll
    for (int c = 0; c < 6; ++c) cell_prim<COH>(M, un, k, dt, i - 3 + c, j, s[c]);
    const float(&w)[4][4] = *reinterpret_cast<const float(*)[4][4]>(&s[1][0]);
    plain_face_flux<0, SOLVER>(M, w, i - 1, Fl);
    if (x) face_features<0>(M, s, x, scale + f * 4, xstride);
  } else {
    const long long gidx = f - nxf;
    const int i = (int)(gidx % M.nx), j = (int)(gidx / M.nx);
#pragma unroll
    for (int c = 0; c < 6; ++c) cell_prim<COH>(M, un, k, dt, i, j - 3 + c, s[c]);
    const float(&w)[4][4] = *reinterpret_cast<const float(*)[4][4]>(&s[1][0]);
    plain_face_flux<1, SOLVER>(M, w, j - 1, Fl);
    if (x) face_features<1>(M, s, x, scale + f * 4, xstride);
  }
  reinterpret_cast<float4*>(F)[f] = make_float4(Fl[0], Fl[1], Fl[2], Fl[3]);
}

template <bool COH>
__device__ __forceinline__ bool cell_flagged(const UpdateArgs& A, int i, int j) {
  const Mesh2& M = A.M;
  if (i < 0 || i >= M.nx) {
    if (M.bc_lo[0] != BC_PERIODIC) return false;
    i = ((i % M.nx) + M.nx) % M.nx;
  }
  if (j < 0 || j >= M.ny) {
    if (M.bc_lo[1] != BC_PERIODIC) return false;
    j = ((j % M.ny) + M.ny) % M.ny;
  }
  return lf_ld<COH>(A.flag + (size_t)j * M.nx + i) != 0;
}

// Learned correction of face f in conserved order (network output clamped to
// [-ylim, ylim], times the face's flux scale, rotated from the face frame).
template <bool COH>
__device__ __forceinline__ void face_correction(const float* dY, const float* scale, float ylim, long long f, int axis,
                                                float (&d)[4]) {
  const float4 yr = lf_ld4<COH>(dY + f * 4), s = lf_ld4<COH>(scale + f * 4);
  const float y[4] = {fminf(fmaxf(yr.x, -ylim), ylim), fminf(fmaxf(yr.y, -ylim), ylim),
                      fminf(fmaxf(yr.z, -ylim), ylim), fminf(fmaxf(yr.w, -ylim), ylim)};
  d[0] = s.x * y[0];
  d[1 + axis] = s.y * y[1];
  d[2 - axis] = s.z * y[2];
  d[3] = s.w * y[3];
}

// Flux-corrected-transport factor of a face with correction d between cells
// l and r (linear indices, -1 outside the mesh): the correction may raise a
// cell by at most its R+ and lower it by at most its R-, for every variable.
template <bool COH>
__device__ __forceinline__ float fct_factor(const float* R, long long l, long long r, const float (&d)[4]) {
  const float4 one = make_float4(1.f, 1.f, 1.f, 1.f);
  const float4 rp4 = r >= 0 ? lf_ld4<COH>(R + 8 * r) : one, rm4 = r >= 0 ? lf_ld4<COH>(R + 8 * r + 4) : one;
  const float4 lp4 = l >= 0 ? lf_ld4<COH>(R + 8 * l) : one, lm4 = l >= 0 ? lf_ld4<COH>(R + 8 * l + 4) : one;
  const float rpr[4] = {rp4.x, rp4.y, rp4.z, rp4.w}, rmr[4] = {rm4.x, rm4.y, rm4.z, rm4.w};
  const float rpl[4] = {lp4.x, lp4.y, lp4.z, lp4.w}, rml[4] = {lm4.x, lm4.y, lm4.z, lm4.w};
  float C = 1.0f;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    if (d[v] > 0.f) C = fminf(C, fminf(rpr[v], rml[v]));
    else if (d[v] < 0.f) C = fminf(C, fminf(rmr[v], rpl[v]));
  }
  return C;
}

// Face flux: plain flux plus the (FCT-limited) learned correction, unless the
// correction is off or, in a widening pass, either neighbour is flagged.
template <bool COH>
__device__ __forceinline__ void face_total(const UpdateArgs& A, long long f, int axis, bool corr, long long nf,
                                           long long lcell, long long rcell, float (&Fo)[4]) {
  const float4 f4 = lf_ld4<COH>(A.F + 4 * f);
  Fo[0] = f4.x;
  Fo[1] = f4.y;
  Fo[2] = f4.z;
  Fo[3] = f4.w;
  if (!corr || !A.dY) return;
  float d[4];
  face_correction<COH>(A.dY, A.scale, A.ylim, f, axis, d);
  const float C = A.R ? fct_factor<COH>(A.R, lcell, rcell, d) : 1.0f;
#pragma unroll
  for (int v = 0; v < 4; ++v) Fo[v] = fmaf(C, d[v], Fo[v]);
}

// Neighbour cell index with periodic wrap, or -1 across a non-periodic wall.
__device__ __forceinline__ long long neighbour(const Mesh2& M, int i, int j) {
  if (i < 0 || i >= M.nx) {
    if (M.bc_lo[0] != BC_PERIODIC) return -1;
    i = ((i % M.nx) + M.nx) % M.nx;
  }
  if (j < 0 || j >= M.ny) {
    if (M.bc_lo[1] != BC_PERIODIC) return -1;
    j = ((j % M.ny) + M.ny) % M.ny;
  }
  return (long long)j * M.nx + i;
}

// Zalesak's ratios of cell c for the stage U_new = U_b - c dt div(F): with
// the low-order update U_L = U_b - c dt div(F_plain), bounds over the cell and
// its face neighbours of U_L and of the stage input, and P+/P- the sums of
// the positive/negative correction contributions of the cell's faces,
// R+ = min(1, (U_max - U_L)/P+), R- = min(1, (U_L - U_min)/P-), into
// R [ncell][8].  dt is the step's dt in FP32.
template <bool COH>
__device__ __forceinline__ void lf_fct_cell(const UpdateArgs& A, long long c, float dt, float* R) {
  const Mesh2& M = A.M;
  const long long ncell = (long long)M.nx * M.ny;
  const long long nxf = (long long)(M.nx + 1) * M.ny;
  const float cdt = A.stage == 1 ? dt : 0.5f * dt;
  const int i = (int)(c % M.nx), j = (int)(c / M.nx);
  float umax[4], umin[4], UL[4];
  const int di[5] = {0, -1, 1, 0, 0}, dj[5] = {0, 0, 0, -1, 1};
  // the cell and its face neighbours; across a wall (index -1) the cell's own
  // values are loaded and not used, so that every load can be issued at once
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const long long nk = k == 0 ? c : neighbour(M, i + di[k], j + dj[k]);
    const bool valid = nk >= 0;
    const long long n = valid ? nk : c;
    const int ni = (int)(n % M.nx), nj = (int)(n / M.nx);
    const long long xl = (long long)nj * (M.nx + 1) + ni, yb = nxf + (long long)nj * M.nx + ni;
    const float iwx = M.iw[0][ni + 2], iwy = M.iw[1][nj + 2];
    const float4 fw = lf_ld4<COH>(A.F + 4 * xl), fe = lf_ld4<COH>(A.F + 4 * (xl + 1));
    const float4 fs = lf_ld4<COH>(A.F + 4 * yb), fn = lf_ld4<COH>(A.F + 4 * (yb + M.nx));
    const float Fw[4] = {fw.x, fw.y, fw.z, fw.w}, Fe[4] = {fe.x, fe.y, fe.z, fe.w};
    const float Fs[4] = {fs.x, fs.y, fs.z, fs.w}, Fn[4] = {fn.x, fn.y, fn.z, fn.w};
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const float u0 = lf_ld<COH>(A.un + v * ncell + n);
      const float kk = A.stage == 2 ? lf_ld<COH>(A.k1 + v * ncell + n) : 0.f;
      const float ub = fmaf(A.stage == 2 ? 0.5f * dt : 0.f, kk, u0);
      const float uin = fmaf(A.stage == 2 ? dt : 0.f, kk, u0);
      // the fused multiply-add is written out, so that every kernel that
      // inlines this rounds it alike
      const float div = fmaf(Fe[v] - Fw[v], iwx, (Fn[v] - Fs[v]) * iwy);
      const float ul = fmaf(-cdt, div, ub);
      if (k == 0) {
        UL[v] = ul;
        umax[v] = fmaxf(ul, uin);
        umin[v] = fminf(ul, uin);
      } else if (valid) {
        umax[v] = fmaxf(umax[v], fmaxf(ul, uin));
        umin[v] = fminf(umin[v], fminf(ul, uin));
      }
    }
  }
  const long long xl = (long long)j * (M.nx + 1) + i, yb = nxf + (long long)j * M.nx + i;
  const float iwx = M.iw[0][i + 2], iwy = M.iw[1][j + 2];
  float dl[4], dr[4], db[4], dt4[4];
  face_correction<COH>(A.dY, A.scale, A.ylim, xl, 0, dl);
  face_correction<COH>(A.dY, A.scale, A.ylim, xl + 1, 0, dr);
  face_correction<COH>(A.dY, A.scale, A.ylim, yb, 1, db);
  face_correction<COH>(A.dY, A.scale, A.ylim, yb + M.nx, 1, dt4);
  float rp[4], rm[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const float q[4] = {cdt * dl[v] * iwx, -cdt * dr[v] * iwx, cdt * db[v] * iwy, -cdt * dt4[v] * iwy};
    float pp = 0.f, pm = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      pp += fmaxf(q[k], 0.f);
      pm += fmaxf(-q[k], 0.f);
    }
    rp[v] = pp > 0.f ? fminf(1.f, (umax[v] - UL[v]) / pp) : 1.f;
    rm[v] = pm > 0.f ? fminf(1.f, (UL[v] - umin[v]) / pm) : 1.f;
  }
  reinterpret_cast<float4*>(R)[2 * c] = make_float4(rp[0], rp[1], rp[2], rp[3]);
  reinterpret_cast<float4*>(R)[2 * c + 1] = make_float4(rm[0], rm[1], rm[2], rm[3]);
}

// The update of cell c in pass A.fixup of a stage (dt the step's dt in FP32):
//   0   corrected fluxes on every face; a cell left with rho <= 0 or p <= 0 is
//       flagged and counted, and requests the widening passes;
//   k>0 cells at or next to a flagged cell take the plain flux on the faces
//       they share with flagged cells (flags only grow); failures left after
//       the last pass request the all-plain pass;
//   -1  the plain flux on every face.
template <bool COH>
__device__ __forceinline__ void lf_update_cell(const UpdateArgs& A, long long c, float dt) {
  const Mesh2& M = A.M;
  const long long ncell = (long long)M.nx * M.ny;
  const long long nxf = (long long)(M.nx + 1) * M.ny, nf = nxf + (long long)M.nx * (M.ny + 1);
  const int i = (int)(c % M.nx), j = (int)(c / M.nx);
  bool cl = true, cr = true, cb = true, ct = true, me = false;
  if (A.fixup < 0) {
    cl = cr = cb = ct = false;
  } else if (A.fixup) {
    me = lf_ld<COH>(A.flag + c) != 0;
    const bool fl = cell_flagged<COH>(A, i - 1, j), fr = cell_flagged<COH>(A, i + 1, j);
    const bool fb = cell_flagged<COH>(A, i, j - 1), ft = cell_flagged<COH>(A, i, j + 1);
    if (!(me || fl || fr || fb || ft)) {
      A.flag_out[c] = 0;
      return;
    }
    cl = !(me || fl);
    cr = !(me || fr);
    cb = !(me || fb);
    ct = !(me || ft);
  }
  const long long xl = (long long)j * (M.nx + 1) + i, yb = nxf + (long long)j * M.nx + i;
  float FL[4], FR[4], FB[4], FT[4];
  face_total<COH>(A, xl, 0, cl, nf, neighbour(M, i - 1, j), c, FL);
  face_total<COH>(A, xl + 1, 0, cr, nf, c, neighbour(M, i + 1, j), FR);
  face_total<COH>(A, yb, 1, cb, nf, neighbour(M, i, j - 1), c, FB);
  face_total<COH>(A, yb + M.nx, 1, ct, nf, c, neighbour(M, i, j + 1), FT);
  const float iwx = M.iw[0][i + 2], iwy = M.iw[1][j + 2];
  float u[4], w[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const float L = -fmaf(FR[v] - FL[v], iwx, (FT[v] - FB[v]) * iwy);  // explicit, as in lf_fct_cell
    const float u0 = lf_ld<COH>(A.un + v * ncell + c);
    if (A.stage == 1) {
      A.out[v * ncell + c] = L;
      u[v] = fmaf(dt, L, u0);
    } else {
      u[v] = fmaf(0.5f * dt, lf_ld<COH>(A.k1 + v * ncell + c) + L, u0);
      A.out[v * ncell + c] = u[v];
    }
  }
  recover<2>(u, w);
  const bool ok = w[0] > 0.f && M.gm1 * w[3] > 0.f && fabsf(w[1]) < INFINITY && fabsf(w[2]) < INFINITY;
  if (A.fixup == 0) {
    A.flag_out[c] = ok ? 0 : 1;
    if (!ok) {
      atomicAdd(A.nfallback, 1ull);
      atomicOr(A.all_plain + 1, 1u);
    }
  } else if (A.fixup > 0) {
    // flags only grow: a flagged cell stays plain, a newly failing one joins
    A.flag_out[c] = (me || !ok) ? 1 : 0;
    if (!ok && me) atomicOr(A.status, STATUS_NONPHYS);  // all its faces are plain already
    if (!ok && A.last) atomicOr(A.all_plain, 1u);  // flag [0]
  } else if (!ok) {
    atomicOr(A.status, STATUS_NONPHYS);  // the plain scheme itself fails
  }
}

}  // namespace gh
