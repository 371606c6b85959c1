// stage_kernel.cuh -- one Runge-Kutta stage of the single-level update
// (Algorithm 1 of arXiv:1207.3392 fused into one pass per stage).
//
// Time stepping (Sec. 3.4, Eqs. Update, RungeKutta1-3):
//   stage 1 : K = L[U^n]                      (written to `out`)
//   stage 2 : U1 = U^n + dt K  (formed on the fly while loading),
//             U^{n+1} = U^n + dt (K + L[U1]) / 2  (written to `out`)
// so that the CFL reduction (Eq. courantTimeStep) and the conserved totals can
// be taken from the primitive recovery stage 1 already does on U^n.
//
// Tiling: a CTA owns a TX x TY tile of the "plane" axes (1D/2D: one row of
// TX - 1 cells, see OWN) and marches along the last axis (z in 3D, y in 2D;
// 1D has one plane).  Per plane it
//   1. loads + recovers the plane two ahead for its own columns (register ring
//      of W along the march axis; limited slopes and the march-axis face flux
//      are computed once per cell per stage),
//   2. loads + recovers the cross-shaped in-plane halo (2 cells each side),
//   3. (PRE) limits the in-plane slopes of each cell once and stores the
//      reconstructed values at both of its in-plane faces in shared memory,
//   4. computes every in-plane face flux exactly once into shared memory
//      (PRE: while loading the next plane, steps 1-2, into a second buffer,
//      so that a plane takes two barriers),
//   5. forms the flux divergence (Eq. BalanceEquationAverage, A_q/V = 1/dq)
//      and the stage combine for its own cells.
// Without PRE each in-plane face limits the slopes of its two cells itself,
// so every in-plane slope is formed twice (one barrier per plane fewer).
// Boundary conditions are applied by index mapping on load (bc_map).
#pragma once

#include <type_traits>

#include "hydro_device.cuh"

namespace gh {

template <class T>
struct StageArgs {
  int n[3];               // cells per axis; 1 on inactive axes
  int bc_lo[3], bc_hi[3];
  T gamma, gm1;
  const Geo<T>* geo[3];   // per axis, index c + 2 for c in [-2, n + 2)
  const T* iw[3];         // inverse widths, index c + 2
  const double* wd[3];    // widths in FP64, index c (totals)
  const T* wdh[3];        // widths split as wdh + wdl (FP32 state: both floats; FP64 state: wdh = wd)
  const T* wdl[3];
  const T* __restrict__ un;   // U^n      [NV][n2][n1][n0]
  const T* __restrict__ k1;   // K of stage 1 (stage 2 only)
  T* __restrict__ out;        // stage 1: K; stage 2: U^{n+1}
  const double* dt;           // device scalar (stage 2)
  int kchunk;                 // planes per CTA along the march axis
  double* part_speed;         // stage 1: per-CTA max over cells of max_q (|v_q| + c_s) / dq
  double* part_tot;           // stage 1: per-CTA sums of U dV, [nblocks][NV]
  unsigned* status;
  int want_totals;
  int has_source;             // external-force source on (Sec. 4.3.2)
  const unsigned char* flags; // SOLVER_HLLC_SW: per-cell shock bits (bit r: shock moving along r)
  T grad_phi[3];              // gradient of the linear external potential
};

// PRE pays in 3D, where both in-plane axes would form every slope twice; in
// 1D/2D one axis gains less than the extra barrier costs.
// COH: the state arrays may have been written earlier in the same launch (the
// one-launch advance of small 1D meshes), so they are read through L2 (__ldcg), which
// is coherent, instead of the read-only cache (__ldg).  Same values either way.
template <int NDIM, class T, int SOLVER, int STAGE, int TX, int TY, bool PRE = (NDIM == 3), bool COH = false>
struct StageKernel {
  static __device__ __forceinline__ T ld(const T* p) {
    if constexpr (COH) return __ldcg(p);
    else return __ldg(p);
  }
  static constexpr int NV = NDIM + 2;
  static constexpr bool SW = SOLVER == SOLVER_HLLC_SW;  // per-face HLLC/HLL choice from shock bits
  static constexpr bool MARCH = NDIM >= 2;
  static constexpr bool HAS_Y = NDIM == 3;
  static constexpr int AM = NDIM - 1;  // march axis (2D: y, 3D: z)
  static constexpr int NT = TX * TY;
  static constexpr int SX = TX + 4;
  static constexpr int SY = HAS_Y ? TY + 4 : 1;
  static constexpr int NHALO = HAS_Y ? 4 * TX + 4 * TY : 4;
  static_assert(HAS_Y || TY == 1, "tiles of 1D/2D runs are one row high");
  static_assert(NT % 32 == 0, "whole warps");
  static constexpr int HSLOTS = (NHALO + NT - 1) / NT;  // halo slots per thread
  // PRE: one-sided face states of the halo cells next to the tile (columns
  // -1 and TX of every row; rows -1 and TY of every column in 3D), formed by
  // the last NJ threads, which load no halo cells when NT >= NHALO + NJ.
  static constexpr int NJ = HAS_Y ? 2 * TY + 2 * TX : 2;
  static_assert(!PRE || NJ <= NT, "one halo face state per thread at most");
  // PRE double-buffers the shared plane: the next plane is loaded while the
  // faces of this one are computed.
  static constexpr int NB = PRE ? 2 : 1;
  // 1D/2D tiles are one row of many warps: in the partial last tile of a
  // small problem whole warps lie past the domain.  Their columns, beyond the
  // two ghost cells the last cell's slopes read, skip the loads, slopes and
  // march-axis faces, and x faces past the last cell are skipped, so that such
  // warps only take the barriers.  (Nothing skipped is ever read.)
  static constexpr bool SKIP = !HAS_Y;
  // Columns of cells a tile owns.  A 1D/2D tile is one row of TX threads; it
  // would have TX + 1 x faces, and one warp would run a second flux round for
  // a single face every plane.  Owning TX - 1 cells instead (the last
  // thread's cell is the next tile's first, loaded only as a neighbour) gives
  // exactly TX faces, one per thread.
  static constexpr int OWN = HAS_Y ? TX : TX - 1;
  static constexpr int NXR = OWN + 1;  // x faces per tile row
  // VEC (3D FP32 with face states): each shared slot holds its 5 values as
  // one float4 (variables 0..3) and one float (variable 4), so a slot is read
  // or written with two accesses instead of five.  Otherwise each variable
  // has its own plane.  The values are the same either way.
  // In 3D, stage 2 only: stage 1 also carries the column totals through the
  // march, and holding whole slots there spilled (measured: stage 1 slower,
  // stage 2 4% faster).  1D and 2D FP32 (3 or 4 values per slot): one float4
  // per slot (in 1D its last lane is unused).
  static constexpr bool VEC5 = NDIM == 3 && PRE && STAGE == 2 && std::is_same<T, float>::value;
  static constexpr bool VEC4 = NDIM <= 2 && std::is_same<T, float>::value;
  static constexpr bool VEC = VEC5 || VEC4;
  static constexpr bool VECF = VEC;
  static constexpr int P = VEC ? 1 : 0;  // plane arrays collapse to one element under VEC
  static constexpr int Q = VEC ? 0 : 1;  // and the float4 arrays otherwise
  static constexpr int Q5 = VEC5 ? 0 : 1;  // the float arrays of the fifth value
  static constexpr int PF = VECF ? 1 : 0;
  static constexpr int QF = VECF ? 0 : 1;

  struct Smem {
    Geo<T> gx[TX + 4];                 // geometry of cells a0 - 2 .. a0 + TX + 1
    Geo<T> gy[HAS_Y ? TY + 4 : 1];     // geometry of cells b0 - 2 .. b0 + TY + 1
    T w[NB][P ? 1 : NV][P ? 1 : SY][P ? 1 : SX];
    T fx[PF ? 1 : NV][PF ? 1 : TY][PF ? 1 : TX + 1];
    T fy[HAS_Y && !PF ? NV : 1][HAS_Y && !PF ? TY + 1 : 1][PF ? 1 : TX];
    double red[NT / 32][NV + 1];
    unsigned char fl[NB][SW ? SY : 1][SW ? SX : 1];  // shock bits of the plane (own cells and halo)
    // PRE: reconstructed primitives at the lower [0] and upper [1] x face of
    // the cells of column slot j (cell a0 + j - 1) and at the lower/upper y
    // face of the cells of row slot i (cell b0 + i - 1)
    T xs[PRE && !P ? 2 : 1][PRE && !P ? NV : 1][PRE && !P ? TY : 1][PRE && !P ? TX + 2 : 1];
    T ys[PRE && HAS_Y && !P ? 2 : 1][PRE && HAS_Y && !P ? NV : 1][PRE && HAS_Y && !P ? TY + 2 : 1]
        [PRE && HAS_Y && !P ? TX : 1];
    // VEC: the same arrays as float4 (+ float in 3D) slots
    float4 w4[Q ? 1 : NB][Q ? 1 : SY][Q ? 1 : SX];
    float w1[Q5 ? 1 : NB][Q5 ? 1 : SY][Q5 ? 1 : SX];
    float4 fx4[QF ? 1 : TY][QF ? 1 : TX + 1];
    float fx1[Q5 ? 1 : TY][Q5 ? 1 : TX + 1];
    float4 fy4[Q5 ? 1 : TY + 1][Q5 ? 1 : TX];
    float fy1[Q5 ? 1 : TY + 1][Q5 ? 1 : TX];
    float4 xs4[Q5 ? 1 : 2][Q5 ? 1 : TY][Q5 ? 1 : TX + 2];
    float xs1[Q5 ? 1 : 2][Q5 ? 1 : TY][Q5 ? 1 : TX + 2];
    float4 ys4[Q5 ? 1 : 2][Q5 ? 1 : TY + 2][Q5 ? 1 : TX];
    float ys1[Q5 ? 1 : 2][Q5 ? 1 : TY + 2][Q5 ? 1 : TX];
  };

  // Slot accessors of the shared arrays (all NV values of one slot).
  static __device__ __forceinline__ void unpack(const float4& q, float s, T (&o)[NV]) {
    o[0] = q.x;
    o[1] = q.y;
    o[2] = q.z;
    if constexpr (NV >= 4) o[3] = q.w;
    if constexpr (NV == 5) o[4] = s;
  }
  static __device__ __forceinline__ void pack(const T (&i)[NV], float4& q, float& s) {
    if constexpr (NV >= 4) q = make_float4(i[0], i[1], i[2], i[3]);
    else q = make_float4(i[0], i[1], i[2], 0.0f);
    if constexpr (NV == 5) s = i[4];
  }
  static __device__ __forceinline__ void get_w(const Smem& S, int b, int r, int c, T (&o)[NV]) {
    if constexpr (VEC) {
      unpack(S.w4[b][r][c], S.w1[VEC5 ? b : 0][VEC5 ? r : 0][VEC5 ? c : 0], o);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) o[v] = S.w[b][v][r][c];
    }
  }
  static __device__ __forceinline__ void put_w(Smem& S, int b, int r, int c, const T (&i)[NV]) {
    if constexpr (VEC) {
      pack(i, S.w4[b][r][c], S.w1[VEC5 ? b : 0][VEC5 ? r : 0][VEC5 ? c : 0]);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) S.w[b][v][r][c] = i[v];
    }
  }
  static __device__ __forceinline__ void get_xs(const Smem& S, int side, int r, int c, T (&o)[NV]) {
    if constexpr (VEC) {
      unpack(S.xs4[side][r][c], S.xs1[side][r][c], o);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) o[v] = S.xs[side][v][r][c];
    }
  }
  static __device__ __forceinline__ void put_xs(Smem& S, int side, int r, int c, const T (&i)[NV]) {
    if constexpr (VEC) {
      pack(i, S.xs4[side][r][c], S.xs1[side][r][c]);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) S.xs[side][v][r][c] = i[v];
    }
  }
  static __device__ __forceinline__ void get_ys(const Smem& S, int side, int r, int c, T (&o)[NV]) {
    if constexpr (VEC) {
      unpack(S.ys4[side][r][c], S.ys1[side][r][c], o);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) o[v] = S.ys[side][v][r][c];
    }
  }
  static __device__ __forceinline__ void put_ys(Smem& S, int side, int r, int c, const T (&i)[NV]) {
    if constexpr (VEC) {
      pack(i, S.ys4[side][r][c], S.ys1[side][r][c]);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) S.ys[side][v][r][c] = i[v];
    }
  }
  static __device__ __forceinline__ void get_fx(const Smem& S, int r, int c, T (&o)[NV]) {
    if constexpr (VECF) {
      unpack(S.fx4[r][c], S.fx1[VEC5 ? r : 0][VEC5 ? c : 0], o);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) o[v] = S.fx[v][r][c];
    }
  }
  static __device__ __forceinline__ void put_fx(Smem& S, int r, int c, const T (&i)[NV]) {
    if constexpr (VECF) {
      pack(i, S.fx4[r][c], S.fx1[VEC5 ? r : 0][VEC5 ? c : 0]);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) S.fx[v][r][c] = i[v];
    }
  }
  static __device__ __forceinline__ void get_fy(const Smem& S, int r, int c, T (&o)[NV]) {
    if constexpr (VECF) {
      unpack(S.fy4[r][c], S.fy1[r][c], o);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) o[v] = S.fy[v][r][c];
    }
  }
  static __device__ __forceinline__ void put_fy(Smem& S, int r, int c, const T (&i)[NV]) {
    if constexpr (VECF) {
      pack(i, S.fy4[r][c], S.fy1[r][c]);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) S.fy[v][r][c] = i[v];
    }
  }

  // Linear index of cell (a, b, m): a = x, b = in-plane y (3D), m = march
  // coordinate; all three already inside the domain.
  static __device__ __forceinline__ size_t cell(const StageArgs<T>& A, int a, int b, int m) {
    if (NDIM == 3) return ((size_t)m * A.n[1] + b) * A.n[0] + a;
    if (NDIM == 2) return (size_t)m * A.n[0] + a;
    return (size_t)a;
  }

  // Boundary-mapped in-plane part of a cell address (fixed for a tile): the
  // march coordinate is mapped per plane by load_col.
  struct ColRef {
    unsigned off;  // in-plane offset: below n0 n1 (< 2^32 for any plane held in memory)
    bool fa, fb;
  };

  static __device__ __forceinline__ ColRef col_ref(const StageArgs<T>& A, int a, int b) {
    ColRef r;
    bool fb = false;
    const int sa = bc_map(a, A.n[0], A.bc_lo[0], A.bc_hi[0], r.fa);
    int sb = 0;
    if constexpr (HAS_Y) sb = bc_map(b, A.n[1], A.bc_lo[1], A.bc_hi[1], fb);
    r.fb = fb;
    r.off = HAS_Y ? (unsigned)sb * (unsigned)A.n[0] + (unsigned)sa : (unsigned)sa;
    return r;
  }

  // Primitives of the (possibly ghost) cell (ref, m) and, for the shock
  // switch, the shock bits of the interior cell it maps to.
  static __device__ __forceinline__ void load_col(const StageArgs<T>& A, const ColRef& r, int m, T dt, size_t vs,
                                                  T (&w)[NV], unsigned char& fl) {
    bool fm = false;
    size_t c = r.off;
    if constexpr (MARCH) {
      const int sm = bc_map(m, A.n[AM], A.bc_lo[AM], A.bc_hi[AM], fm);
      c += (size_t)sm * (HAS_Y ? (size_t)A.n[0] * A.n[1] : (size_t)A.n[0]);
    }
    T u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T x = ld(A.un + v * vs + c);
      if (STAGE == 2) x = fma(dt, ld(A.k1 + v * vs + c), x);
      u[v] = x;
    }
    if (r.fa) u[1] = -u[1];
    if constexpr (HAS_Y) { if (r.fb) u[2] = -u[2]; }
    if constexpr (MARCH) { if (fm) u[1 + AM] = -u[1 + AM]; }
    recover<NDIM>(u, w);
    if constexpr (SW) fl = A.flags[c];
  }

  // L2 prefetch of the cell (ref, m) that load_col will read PFD - 2 march
  // iterations later (the same boundary-mapped address, so always inside the
  // arrays): the load then meets L2 latency instead of DRAM latency.  Only
  // the 2D march (rows of one CTA) gains; in 3D the extra instructions cost
  // more than the latency they hide.
  static constexpr int PFD = NDIM == 2 ? 3 : 0;
  static __device__ __forceinline__ void prefetch_col(const StageArgs<T>& A, const ColRef& r, int m, size_t vs) {
    bool fm = false;
    const int sm = bc_map(m, A.n[AM], A.bc_lo[AM], A.bc_hi[AM], fm);
    const size_t c = r.off + (size_t)sm * (HAS_Y ? (size_t)A.n[0] * A.n[1] : (size_t)A.n[0]);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      asm volatile("prefetch.global.L2 [%0];" ::"l"(A.un + v * vs + c));
      if (STAGE == 2) asm volatile("prefetch.global.L2 [%0];" ::"l"(A.k1 + v * vs + c));
    }
  }

  // Face flux along axis Q; with the switch, HLL when either cell's shock
  // bits name an axis other than Q (a shock moving transverse to the face).
  template <int Q>
  static __device__ __forceinline__ void flux(const StageArgs<T>& A, const T (&wl)[NV], const T (&wr)[NV],
                                              unsigned bits, T (&f)[NV]) {
    if constexpr (SW) {
      if (bits & ~(1u << Q)) face_flux<T, NDIM, Q, SOLVER_HLL>(wl, wr, A.gamma, A.gm1, f);
      else face_flux<T, NDIM, Q, SOLVER_HLLC>(wl, wr, A.gamma, A.gm1, f);
    } else {
      face_flux<T, NDIM, Q, SOLVER>(wl, wr, A.gamma, A.gm1, f);
    }
  }

  static __device__ __forceinline__ Geo<T> geo(const StageArgs<T>& A, int q, int c) {
    c = c < -2 ? -2 : (c > A.n[q] + 1 ? A.n[q] + 1 : c);
    return A.geo[q][c + 2];
  }

  // Flux through the face between slot positions (s - 1, s) along x of shared
  // row `row`; slot s holds cell a0 + s - 2.
  static __device__ __forceinline__ void x_face(const StageArgs<T>& A, Smem& S, int b, int face, int srow,
                                                int frow) {
    const int sl = face + 1;  // slot of the left cell
    T wl[NV], wr[NV], f[NV];
    if constexpr (PRE) {
      get_xs(S, 1, frow, face, wl);
      get_xs(S, 0, frow, face + 1, wr);
    } else {
      const Geo<T> gl = S.gx[face + 1], gr = S.gx[face + 2];
      T w0[NV], w1[NV], w2[NV], w3[NV];
      get_w(S, b, srow, sl - 1, w0);
      get_w(S, b, srow, sl, w1);
      get_w(S, b, srow, sl + 1, w2);
      get_w(S, b, srow, sl + 2, w3);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        wl[v] = fma(limited_slope(w0[v], w1[v], w2[v], gl), gl.h, w1[v]);
        wr[v] = fma(-limited_slope(w1[v], w2[v], w3[v], gr), gr.h, w2[v]);
      }
    }
    flux<0>(A, wl, wr, SW ? (unsigned)(S.fl[b][SW ? srow : 0][SW ? sl : 0] | S.fl[b][SW ? srow : 0][SW ? sl + 1 : 0]) : 0u,
            f);
    put_fx(S, frow, face, f);
  }

  static __device__ __forceinline__ void y_face(const StageArgs<T>& A, Smem& S, int b, int face, int scol) {
    const int sl = face + 1;
    T wl[NV], wr[NV], f[NV];
    if constexpr (PRE) {
      get_ys(S, 1, face, scol - 2, wl);
      get_ys(S, 0, face + 1, scol - 2, wr);
    } else {
      const Geo<T> gl = S.gy[face + 1], gr = S.gy[face + 2];
      T w0[NV], w1[NV], w2[NV], w3[NV];
      get_w(S, b, sl - 1, scol, w0);
      get_w(S, b, sl, scol, w1);
      get_w(S, b, sl + 1, scol, w2);
      get_w(S, b, sl + 2, scol, w3);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        wl[v] = fma(limited_slope(w0[v], w1[v], w2[v], gl), gl.h, w1[v]);
        wr[v] = fma(-limited_slope(w1[v], w2[v], w3[v], gr), gr.h, w2[v]);
      }
    }
    flux<1>(A, wl, wr, SW ? (unsigned)(S.fl[b][SW ? sl : 0][SW ? scol : 0] | S.fl[b][SW ? sl + 1 : 0][SW ? scol : 0]) : 0u,
            f);
    put_fy(S, face, scol - 2, f);
  }

  // Flux through the march-axis face between cells with primitives wa (below,
  // slope sa, geometry ga) and wb (above, slope sb, geometry gb).
  static __device__ __forceinline__ void m_face(const StageArgs<T>& A, const T (&wa)[NV], const T (&sa)[NV],
                                                T ha, const T (&wb)[NV], const T (&sb)[NV], T hb,
                                                unsigned bits, T (&f)[NV]) {
    T wl[NV], wr[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      wl[v] = fma(sa[v], ha, wa[v]);
      wr[v] = fma(-sb[v], hb, wb[v]);
    }
    flux<AM>(A, wl, wr, bits, f);
  }

  static __device__ __forceinline__ void slopes(const StageArgs<T>& A, const T (&wm)[NV], const T (&wc)[NV],
                                                const T (&wp)[NV], const Geo<T>& g, T (&s)[NV]) {
#pragma unroll
    for (int v = 0; v < NV; ++v) s[v] = limited_slope(wm[v], wc[v], wp[v], g);
  }

  // PRE: the reconstructed values at the in-plane faces of the own cell (W in
  // registers, neighbours from the shared plane), and the one-sided value of
  // the halo cell that job tid - (NT - NJ) names.  The formulas are those of
  // the face routines without PRE, so that both forms give the same bits.
  static __device__ __forceinline__ void face_states(Smem& S, int b, int tid, int tx, int ty, const T (&wc)[NV]) {
    const int sy = HAS_Y ? ty + 2 : 0;
    {
      const Geo<T> g = S.gx[tx + 2];
      T wm[NV], wp[NV], lo[NV], hi[NV];
      get_w(S, b, sy, tx + 1, wm);
      get_w(S, b, sy, tx + 3, wp);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T sv = limited_slope(wm[v], wc[v], wp[v], g);
        lo[v] = fma(-sv, g.h, wc[v]);
        hi[v] = fma(sv, g.h, wc[v]);
      }
      put_xs(S, 0, ty, tx + 1, lo);
      put_xs(S, 1, ty, tx + 1, hi);
    }
    if constexpr (HAS_Y) {
      const Geo<T> g = S.gy[ty + 2];
      T wm[NV], wp[NV], lo[NV], hi[NV];
      get_w(S, b, ty + 1, tx + 2, wm);
      get_w(S, b, ty + 3, tx + 2, wp);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T sv = limited_slope(wm[v], wc[v], wp[v], g);
        lo[v] = fma(-sv, g.h, wc[v]);
        hi[v] = fma(sv, g.h, wc[v]);
      }
      put_ys(S, 0, ty + 1, tx, lo);
      put_ys(S, 1, ty + 1, tx, hi);
    }
    const int j = tid - (NT - NJ);
    if (j < 0) return;
    if (j < 2 * (HAS_Y ? TY : 1)) {
      // x: column -1 (upper face value) or column TX (lower face value) of row j / 2
      const int r = j >> 1;
      const bool up = j & 1;
      const int srow = HAS_Y ? r + 2 : 0;
      const int slot = up ? TX + 2 : 1;
      const Geo<T> g = S.gx[slot];
      T wm[NV], w1[NV], wp[NV], o[NV];
      get_w(S, b, srow, slot - 1, wm);
      get_w(S, b, srow, slot, w1);
      get_w(S, b, srow, slot + 1, wp);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T sv = limited_slope(wm[v], w1[v], wp[v], g);
        o[v] = up ? fma(-sv, g.h, w1[v]) : fma(sv, g.h, w1[v]);
      }
      if (up) put_xs(S, 0, r, TX + 1, o);
      else put_xs(S, 1, r, 0, o);
    } else if constexpr (HAS_Y) {
      // y: row -1 (upper face value) or row TY (lower face value) of column c
      const int jj = j - 2 * TY;
      const bool up = jj >= TX;
      const int c = up ? jj - TX : jj;
      const int slot = up ? TY + 2 : 1;
      const Geo<T> g = S.gy[slot];
      T wm[NV], w1[NV], wp[NV], o[NV];
      get_w(S, b, slot - 1, c + 2, wm);
      get_w(S, b, slot, c + 2, w1);
      get_w(S, b, slot + 1, c + 2, wp);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T sv = limited_slope(wm[v], w1[v], wp[v], g);
        o[v] = up ? fma(-sv, g.h, w1[v]) : fma(sv, g.h, w1[v]);
      }
      if (up) put_ys(S, 0, TY + 1, c, o);
      else put_ys(S, 1, 0, c, o);
    }
  }

  // The own cell (primitives wo, shock bits fo) and this thread's halo cells
  // of plane m into buffer b of the shared plane.
  static __device__ __forceinline__ void put_plane(const StageArgs<T>& A, Smem& S, int b, int m, int tid, int tx,
                                                   int ty, const T (&wo)[NV], unsigned char fo,
                                                   const ColRef (&halo)[HSLOTS], const int (&hsx)[HSLOTS],
                                                   const int (&hsy)[HSLOTS], T dt, size_t vs) {
    put_w(S, b, HAS_Y ? ty + 2 : 0, tx + 2, wo);
    if constexpr (SW) S.fl[b][HAS_Y ? ty + 2 : 0][tx + 2] = fo;
#pragma unroll
    for (int k = 0; k < HSLOTS; ++k) {
      if (tid + k * NT < NHALO) {
        T wh[NV];
        unsigned char fh = 0;
        load_col(A, halo[k], m, dt, vs, wh, fh);
        put_w(S, b, hsy[k], hsx[k], wh);
        if constexpr (SW) S.fl[b][hsy[k]][hsx[k]] = fh;
      }
    }
  }

  // In-plane faces, each computed once, one call site per axis.  Whole
  // rounds of NT faces go to all threads; the REM faces left over go to the
  // last threads, which load no halo cells, so that no warp does both a halo
  // load and an extra face.
  static __device__ __forceinline__ void faces(const StageArgs<T>& A, Smem& S, int b, int tid, int tx, int ty,
                                               int xlast) {
    if constexpr (PRE && HAS_Y && TX % 32 == 0 && !std::is_same<T, dw>::value) {
      // Cell-aligned: thread (tx, ty) takes the lower x face of its cell, then
      // its lower y face; the TY upper x faces of the last column and the TX
      // upper y faces of the last row go to the last TX + TY threads.  A warp
      // lies in one row, so every warp runs one flux routine per round.  (The
      // double-word flux is large enough that its four inlined copies cost
      // more than the straddling warp saves: it keeps the numbered loop.)
      x_face(A, S, b, tx, ty + 2, ty);
      y_face(A, S, b, ty, tx + 2);
      const int j = tid - (NT - (TX + TY));
      if (j >= 0) {
        if (j < TY) x_face(A, S, b, TX, j + 2, j);
        else y_face(A, S, b, TY, j - TY + 2);
      }
      return;
    }
    constexpr int NXF = NXR * TY;
    constexpr int NYF = HAS_Y ? TX * (TY + 1) : 0;
    constexpr int NF = NXF + NYF, ROUNDS = NF / NT, REM = NF - ROUNDS * NT;
    for (int k = 0; k <= ROUNDS; ++k) {
      int f = tid + k * NT;
      if (k == ROUNDS) {
        if (REM == 0 || tid < NT - REM) break;
        f = ROUNDS * NT + (tid - (NT - REM));
      }
      if (f < NXF) {
        const int row = f / NXR;
        const int face = f - row * NXR;
        if (SKIP && face > xlast) continue;
        x_face(A, S, b, face, HAS_Y ? row + 2 : 0, row);
      } else {
        if constexpr (HAS_Y) {
          const int g = f - NXF;
          const int face = g / TX;
          const int col = g - face * TX;
          y_face(A, S, b, face, col + 2);
        }
      }
    }
  }

  static __device__ __forceinline__ bool nonphysical(const T (&w)[NV], T gm1) {
    bool bad = !(w[0] > T(0)) || !(gm1 * w[NV - 1] > T(0));
#pragma unroll
    for (int v = 1; v < NV - 1; ++v) bad |= !(fabs(w[v]) < T(INFINITY));
    return bad;
  }

  // One tile (bx, by) and march chunk bz of the stage.  Accumulates the
  // thread's CFL speed (stage 1), its share of the totals (stage 1) and the
  // non-physical flag; the caller reduces them.  All threads of the block must
  // call it together (it synchronises).
  static __device__ void tile(const StageArgs<T>& A, Smem& S, int bx, int by, int bz, double& speed_out,
                              double (&tot)[NV], bool& bad) {
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int nx = A.n[0];
    const int ny = HAS_Y ? A.n[1] : 1;
    const int nm = MARCH ? A.n[AM] : 1;
    const size_t vs = (size_t)A.n[0] * A.n[1] * A.n[2];
    const int a0 = bx * OWN;
    const int b0 = HAS_Y ? by * TY : 0;
    const int ca = a0 + tx, cb = b0 + ty;
    const bool own_valid = ca < nx && cb < ny && (HAS_Y || tx < OWN);
    const bool live = !SKIP || ca < nx + 2;
    const int m0 = MARCH ? bz * A.kchunk : 0;
    const int m1 = MARCH ? min(nm, m0 + A.kchunk) : 1;
    const T dt = STAGE == 2 ? (T)(*A.dt) : T(0);

    const T iwx = A.iw[0][min(ca, nx + 1) + 2];
    const T iwy = HAS_Y ? A.iw[1][min(cb, ny + 1) + 2] : T(0);

    // per-tile tables: in-plane geometry in shared memory (made visible by the
    // first barrier of the plane loop), boundary-mapped column addresses
    for (int k = tid; k < TX + 4; k += NT) S.gx[k] = geo(A, 0, a0 + k - 2);
    if constexpr (HAS_Y)
      for (int k = tid; k < TY + 4; k += NT) S.gy[k] = geo(A, 1, b0 + k - 2);
    const ColRef own = col_ref(A, ca, cb);
    // this thread's halo slots h = tid + k NT: rows -2, -1, TY, TY+1 of the
    // tile (3D), then columns -2, -1, TX, TX+1 of every row
    int hsx[HSLOTS], hsy[HSLOTS];
    ColRef halo[HSLOTS];
#pragma unroll
    for (int k = 0; k < HSLOTS; ++k) {
      const int h = tid + k * NT;
      int sx = 0, sy = 0;
      if (h < NHALO) {
        if (HAS_Y && h < 4 * TX) {
          const int r = h / TX;
          sx = h % TX + 2;
          sy = r < 2 ? r : TY + r;
        } else {
          const int hh = HAS_Y ? h - 4 * TX : h;
          const int c = hh & 3;
          sy = HAS_Y ? (hh >> 2) + 2 : 0;
          sx = c < 2 ? c : TX + c;
        }
      }
      hsx[k] = sx;
      hsy[k] = sy;
      halo[k] = col_ref(A, a0 + sx - 2, HAS_Y ? b0 + sy - 2 : 0);
    }

    ColumnSum<T> tcol[NV];  // this column's sum of U dq along the march axis
    T speed_max = T(0);

    // March-axis register ring.  At the top of iteration m: wk = W(m),
    // wk1 = W(m+1), sk = slope(m), flo = flux(m-1/2).  The loop starts two
    // planes early so that every march-axis slope and face flux of the chunk
    // comes from the same code (bitwise the same values as the neighbouring
    // chunk computes for the shared face).
    T wk[NV], wk1[NV], sk[NV], flo[NV];
    unsigned char fk = 0, fk1 = 0;  // shock bits of the own column at m, m + 1 (switch only)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      sk[v] = T(0);
      flo[v] = T(0);
    }
    int mstart = m0;
    if constexpr (MARCH) {
      if (live) {
        load_col(A, own, m0 - 2, dt, vs, wk, fk);
        load_col(A, own, m0 - 1, dt, vs, wk1, fk1);
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) wk[v] = wk1[v] = T(0);
      }
      mstart = m0 - 2;
    }

    for (int m = mstart; m < m1; ++m) {
      T fhi[NV], wk2[NV], sk1[NV];
      T wown[NV];
      unsigned char fk2 = 0, fown = 0;
      if constexpr (MARCH) {
        if (live) {
          if (PFD > 0 && m + PFD < m1 + 2) prefetch_col(A, own, m + PFD, vs);
          load_col(A, own, m + 2, dt, vs, wk2, fk2);
          const Geo<T> g0 = geo(A, AM, m), g1 = geo(A, AM, m + 1);
          slopes(A, wk, wk1, wk2, g1, sk1);
          // the face m0 - 3/2 of the first warm-up plane is never used
          if (m > m0 - 2) {
            m_face(A, wk, sk, g0.h, wk1, sk1, g1.h, (unsigned)(fk | fk1), fhi);
          } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) fhi[v] = T(0);
          }
        } else {
#pragma unroll
          for (int v = 0; v < NV; ++v) wk2[v] = sk1[v] = fhi[v] = T(0);
        }
        if (m < m0) {  // warm-up planes: advance the ring only
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            flo[v] = fhi[v];
            wk[v] = wk1[v];
            wk1[v] = wk2[v];
            sk[v] = sk1[v];
          }
          fk = fk1;
          fk1 = fk2;
          continue;
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) wown[v] = wk[v];
        fown = fk;
      } else if (live) {
        load_col(A, own, 0, dt, vs, wown, fown);
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) wown[v] = T(0);
      }
      // Without PRE: plane m into the shared plane; barrier; faces; barrier.
      // With PRE the plane was put into buffer `buf` during the faces of the
      // previous plane (the first plane of the chunk here): face states;
      // barrier; faces, and plane m + 1 into the other buffer; barrier.
      const int buf = PRE ? ((m - m0) & 1) : 0;
      if (!PRE || m == m0) {
        put_plane(A, S, buf, m, tid, tx, ty, wown, fown, halo, hsx, hsy, dt, vs);
        __syncthreads();
      }
      if constexpr (PRE) {
        face_states(S, buf, tid, tx, ty, wown);
        __syncthreads();
      }
      faces(A, S, buf, tid, tx, ty, nx - a0);
      if constexpr (PRE) {
        if (m + 1 < m1) put_plane(A, S, buf ^ 1, m + 1, tid, tx, ty, wk1, fk1, halo, hsx, hsy, dt, vs);
      }
      __syncthreads();

      if (own_valid) {
        const T iwm = MARCH ? A.iw[AM][m + 2] : T(0);
        T L[NV], fxr[NV], fxl[NV], fyt[NV], fyb[NV];
        get_fx(S, ty, tx + 1, fxr);
        get_fx(S, ty, tx, fxl);
        if constexpr (HAS_Y) {
          get_fy(S, ty + 1, tx, fyt);
          get_fy(S, ty, tx, fyb);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T d = (fxr[v] - fxl[v]) * iwx;
          if constexpr (HAS_Y) d += (fyt[v] - fyb[v]) * iwy;
          if constexpr (MARCH) d += (fhi[v] - flo[v]) * iwm;
          L[v] = -d;
        }
        if (A.has_source) {
          // external force and power (Sec. 4.3.2): S_q -= D dPhi/dq,
          // G -= sum_q S_q dPhi/dq, from this cell's stage-input state
          T power = T(0);
#pragma unroll
          for (int q = 0; q < NDIM; ++q) {
            L[1 + q] -= wown[0] * A.grad_phi[q];
            power = fma(wown[0] * wown[1 + q], A.grad_phi[q], power);
          }
          L[NV - 1] -= power;
        }
        const size_t c = cell(A, ca, cb, m);
        bad |= nonphysical(wown, A.gm1);
        if (STAGE == 1) {
#pragma unroll
          for (int v = 0; v < NV; ++v) A.out[v * vs + c] = L[v];
          // CFL speed (Eq. courantTimeStep) on U^n at the cell centre
          const T cs = sound_speed(A.gamma, A.gm1 * wown[NV - 1], wown[0]);
          T s = (fabs(wown[1]) + cs) * iwx;
          if constexpr (HAS_Y) s = fmax(s, (fabs(wown[2]) + cs) * iwy);
          if constexpr (MARCH) s = fmax(s, (fabs(wown[1 + AM]) + cs) * iwm);
          speed_max = fmax(speed_max, s);
          if (A.want_totals) {
            const T dm_hi = MARCH ? A.wdh[AM][m] : T(1), dm_lo = MARCH ? A.wdl[AM][m] : T(0);
#pragma unroll
            for (int v = 0; v < NV; ++v) tcol[v].add_product(ld(A.un + v * vs + c), dm_hi, dm_lo);
          }
        } else {
          const T hdt = T(0.5) * dt;
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const T u0 = ld(A.un + v * vs + c), k = ld(A.k1 + v * vs + c);
            A.out[v * vs + c] = fma(hdt, add_rn(k, L[v]), u0);
          }
        }
      }
      if constexpr (MARCH) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          flo[v] = fhi[v];
          wk[v] = wk1[v];
          wk1[v] = wk2[v];
          sk[v] = sk1[v];
        }
        fk = fk1;
        fk1 = fk2;
      }
    }

    if (STAGE == 1 && own_valid && A.want_totals) {
      double area = A.wd[0][ca];
      if constexpr (HAS_Y) area *= A.wd[1][cb];
#pragma unroll
      for (int v = 0; v < NV; ++v) tot[v] = fma(tcol[v].value(), area, tot[v]);
    }
    speed_out = fmax(speed_out, (double)speed_max);
  }

  // Fixed-order block reduction of (max speed, totals) into per-CTA partials.
  static __device__ void write_partials(const StageArgs<T>& A, Smem& S, size_t blk, double speed_max,
                                        const double (&tot)[NV]) {
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    double r[NV + 1];
    r[0] = warp_max(speed_max);
#pragma unroll
    for (int v = 0; v < NV; ++v) r[1 + v] = warp_sum(tot[v]);
    if (lane == 0) {
#pragma unroll
      for (int v = 0; v <= NV; ++v) S.red[warp][v] = r[v];
    }
    __syncthreads();
    if (tid <= NV) {
      double acc = S.red[0][tid];
      for (int wi = 1; wi < NT / 32; ++wi) acc = tid == 0 ? fmax(acc, S.red[wi][0]) : acc + S.red[wi][tid];
      if (tid == 0) A.part_speed[blk] = acc;
      else A.part_tot[blk * NV + (tid - 1)] = acc;
    }
  }

  static __device__ void run(const StageArgs<T>& A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& S = *reinterpret_cast<Smem*>(smem_raw);
    double speed_max = 0.0;
    double tot[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) tot[v] = 0.0;
    bool bad = false;
    tile(A, S, blockIdx.x, blockIdx.y, blockIdx.z, speed_max, tot, bad);
    if (bad) atomicOr(A.status, STATUS_NONPHYS);
    if (STAGE == 1) {
      const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      write_partials(A, S, blk, speed_max, tot);
    }
  }
};

// MINB: CTAs per SM the register allocation must allow (__launch_bounds__).
template <int NDIM, class T, int SOLVER, int STAGE, int TX, int TY, int MINB, bool PRE>
__global__ void __launch_bounds__(TX * TY, MINB) hydro_stage_kernel(const StageArgs<T> A) {
  StageKernel<NDIM, T, SOLVER, STAGE, TX, TY, PRE>::run(A);
}

}  // namespace gh
