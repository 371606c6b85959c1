// stage_pair.cuh -- one Runge-Kutta stage of the 3D FP32 update (Algorithm 1,
// Secs. 3.1-3.4) with each thread holding a cell of two consecutive march
// planes, computed with the packed FP32 instructions (pair32.cuh).
//
// The scalar stage kernel (stage_kernel.cuh) is bound by instruction issue:
// ~1,100 instructions per cell and stage, about half of them FP32
// arithmetic.  Here a march step takes the planes m and m + 1 together: lane x
// of every pair is plane m, lane y plane m + 1.  In the plane every neighbour
// of a pair is again a pair of the same two planes, so the in-plane
// reconstruction, the x and y face fluxes and the flux divergence run once for
// both planes, at two results per issue slot, and shared memory moves 8 bytes
// per access.  The plane loop runs half as many times (half the barriers,
// addressing and control per cell).
//
// Along the march axis the stencil straddles pairs.  At the step of the pair
// P = (m, m+1) the thread has W(m-1) (from the previous pair), P and the next
// pair N = (m+2, m+3), and forms the shifted pair S = (m+1, m+2):
//   slopes  s(P) from (W(m-1), W(m)), P, S;   s(S) from P, S, N
//   faces   F(m+1/2), F(m+3/2) as one pair: left W(P) + s(P) h(P),
//           right W(S) - s(S) h(S)
//   divergence of P: upper faces (F(m+1/2), F(m+3/2)), lower faces
//           (F(m-1/2) from the previous pair, F(m+1/2)).
// (s(m+1) is formed in both lanes, from the same values, so both uses agree.)
// A chunk starts with one warm-up pair (m0 - 2, m0 - 1) that only provides
// W(m0 - 1) and F(m0 - 1/2); its other lane values are never used.
// Chunks hold an even number of planes; a last chunk of odd length computes
// one plane past its end in lane y and stores nothing of it.
//
// The arithmetic is written with explicit roundings, the same code for every
// face in either lane, so the flux of a chunk-boundary face is bitwise the
// same from both sides (the update stays conservative) and tile shapes and
// chunk lengths give bitwise the same states.  The scalar kernels let the
// compiler fuse products, so the two families agree to FP32 rounding, not
// bitwise.  HLL and HLLC only (the shock switch keeps the scalar kernels).
#pragma once

#include "pair32.cuh"
#include "stage_kernel.cuh"

namespace gh {

template <int SOLVER, int STAGE, int TX, int TY>
struct StagePair {
  static constexpr int NV = 5;
  static constexpr int NT = TX * TY;
  static constexpr int SX = TX + 4;
  static constexpr int SY = TY + 4;
  static constexpr int NHALO = 4 * TX + 4 * TY;
  static constexpr int HSLOTS = (NHALO + NT - 1) / NT;
  static constexpr int NJ = 2 * TY + 2 * TX;  // one-sided face states of the halo cells next to the tile
  static_assert(TX % 32 == 0 && NT % 32 == 0, "whole warps along x");
  static_assert(NJ <= NT, "one halo face state per thread at most");
  static_assert(SOLVER == SOLVER_HLL || SOLVER == SOLVER_HLLC, "HLL or HLLC");

  struct Smem {
    Geo2 gx[TX + 4];  // in-plane geometry of cells a0 - 2 .. a0 + TX + 1 (both lanes alike)
    Geo2 gy[TY + 4];
    f2 w[2][NV][SY][SX];  // primitives of the plane pair (own cells and halo), double-buffered
    f2 fx[NV][TY][TX + 1];
    f2 fy[NV][TY + 1][TX];
    // reconstructed values at the lower [0] / upper [1] x face of column slot
    // j (cell a0 + j - 1) and y face of row slot i (cell b0 + i - 1)
    f2 xs[2][NV][TY][TX + 2];
    f2 ys[2][NV][TY + 2][TX];
    double red[NT / 32][NV + 1];
  };

  using K = StageKernel<3, float, SOLVER, STAGE, TX, TY, true>;  // addressing helpers

  static __device__ __forceinline__ Geo2 geo_b(const StageArgs<float>& A, int q, int c) {
    const Geo<float> g = K::geo(A, q, c);
    return geo2(g, g);
  }

  // Primitives of the (possibly ghost) cell `r` in the planes m and m + 1.
  static __device__ __forceinline__ void load_pair(const StageArgs<float>& A, const typename K::ColRef& r, int m,
                                                   f2 dt, size_t vs, f2 (&w)[NV]) {
    bool f0 = false, f1 = false;
    const size_t plane = (size_t)A.n[0] * A.n[1];
    const size_t c0 = r.off + (size_t)bc_map(m, A.n[2], A.bc_lo[2], A.bc_hi[2], f0) * plane;
    const size_t c1 = r.off + (size_t)bc_map(m + 1, A.n[2], A.bc_lo[2], A.bc_hi[2], f1) * plane;
    f2 u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      u[v] = mk2(__ldg(A.un + v * vs + c0), __ldg(A.un + v * vs + c1));
      if (STAGE == 2) u[v] = fma2(dt, mk2(__ldg(A.k1 + v * vs + c0), __ldg(A.k1 + v * vs + c1)), u[v]);
    }
    if (r.fa) u[1] = neg2(u[1]);
    if (r.fb) u[2] = neg2(u[2]);
    if (f0) u[3].x = -u[3].x;
    if (f1) u[3].y = -u[3].y;
    recover2(u, w);
  }

  template <int Q>
  static __device__ __forceinline__ void flux(const StageArgs<float>& A, const f2 (&wl)[NV], const f2 (&wr)[NV],
                                              f2 (&f)[NV]) {
    face_flux2<Q, SOLVER>(wl, wr, bc2(A.gamma), bc2(A.gm1), f);
  }

  static __device__ __forceinline__ void x_face(const StageArgs<float>& A, Smem& S, int face, int row) {
    f2 wl[NV], wr[NV], f[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      wl[v] = S.xs[1][v][row][face];
      wr[v] = S.xs[0][v][row][face + 1];
    }
    flux<0>(A, wl, wr, f);
#pragma unroll
    for (int v = 0; v < NV; ++v) S.fx[v][row][face] = f[v];
  }

  static __device__ __forceinline__ void y_face(const StageArgs<float>& A, Smem& S, int face, int col) {
    f2 wl[NV], wr[NV], f[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      wl[v] = S.ys[1][v][face][col];
      wr[v] = S.ys[0][v][face + 1][col];
    }
    flux<1>(A, wl, wr, f);
#pragma unroll
    for (int v = 0; v < NV; ++v) S.fy[v][face][col] = f[v];
  }

  // Reconstructed values at the in-plane faces of the own cell and the
  // one-sided value of the halo cell that job tid - (NT - NJ) names.
  static __device__ __forceinline__ void face_states(Smem& S, int b, int tid, int tx, int ty, const f2 (&wc)[NV]) {
    {
      const Geo2& g = S.gx[tx + 2];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const f2 sv = limited_slope2(S.w[b][v][ty + 2][tx + 1], wc[v], S.w[b][v][ty + 2][tx + 3], g);
        S.xs[0][v][ty][tx + 1] = fma2(sv, g.nh, wc[v]);
        S.xs[1][v][ty][tx + 1] = fma2(sv, g.h, wc[v]);
      }
    }
    {
      const Geo2& g = S.gy[ty + 2];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const f2 sv = limited_slope2(S.w[b][v][ty + 1][tx + 2], wc[v], S.w[b][v][ty + 3][tx + 2], g);
        S.ys[0][v][ty + 1][tx] = fma2(sv, g.nh, wc[v]);
        S.ys[1][v][ty + 1][tx] = fma2(sv, g.h, wc[v]);
      }
    }
    const int j = tid - (NT - NJ);
    if (j < 0) return;
    if (j < 2 * TY) {
      // x: column -1 (upper face value) or column TX (lower face value) of row j / 2
      const int r = j >> 1;
      const bool up = j & 1;
      const int slot = up ? TX + 2 : 1;
      const Geo2& g = S.gx[slot];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const f2 w1 = S.w[b][v][r + 2][slot];
        const f2 sv = limited_slope2(S.w[b][v][r + 2][slot - 1], w1, S.w[b][v][r + 2][slot + 1], g);
        if (up) S.xs[0][v][r][TX + 1] = fma2(sv, g.nh, w1);
        else S.xs[1][v][r][0] = fma2(sv, g.h, w1);
      }
    } else {
      // y: row -1 (upper face value) or row TY (lower face value) of column c
      const int jj = j - 2 * TY;
      const bool up = jj >= TX;
      const int c = up ? jj - TX : jj;
      const int slot = up ? TY + 2 : 1;
      const Geo2& g = S.gy[slot];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const f2 w1 = S.w[b][v][slot][c + 2];
        const f2 sv = limited_slope2(S.w[b][v][slot - 1][c + 2], w1, S.w[b][v][slot + 1][c + 2], g);
        if (up) S.ys[0][v][TY + 1][c] = fma2(sv, g.nh, w1);
        else S.ys[1][v][0][c] = fma2(sv, g.h, w1);
      }
    }
  }

  // The own cell pair and this thread's halo cells of planes (m, m + 1) into
  // buffer b of the shared plane pair.
  static __device__ __forceinline__ void put_plane(const StageArgs<float>& A, Smem& S, int b, int m, int tid, int tx,
                                                   int ty, const f2 (&wo)[NV],
                                                   const typename K::ColRef (&halo)[HSLOTS], const int (&hsx)[HSLOTS],
                                                   const int (&hsy)[HSLOTS], f2 dt, size_t vs) {
#pragma unroll
    for (int v = 0; v < NV; ++v) S.w[b][v][ty + 2][tx + 2] = wo[v];
#pragma unroll
    for (int k = 0; k < HSLOTS; ++k) {
      if (tid + k * NT < NHALO) {
        f2 wh[NV];
        load_pair(A, halo[k], m, dt, vs, wh);
#pragma unroll
        for (int v = 0; v < NV; ++v) S.w[b][v][hsy[k]][hsx[k]] = wh[v];
      }
    }
  }

  // In-plane faces, cell-aligned: thread (tx, ty) takes the lower x and lower
  // y face of its cell; the TY upper x faces of the last column and the TX
  // upper y faces of the last row go to the last TX + TY threads.
  static __device__ __forceinline__ void faces(const StageArgs<float>& A, Smem& S, int tid, int tx, int ty) {
    x_face(A, S, tx, ty);
    y_face(A, S, ty, tx);
    const int j = tid - (NT - (TX + TY));
    if (j >= 0) {
      if (j < TY) x_face(A, S, TX, j);
      else y_face(A, S, TY, j - TY);
    }
  }

  static __device__ __forceinline__ bool nonphysical(const f2 (&w)[NV], bool lane_y, float gm1) {
    const auto bad1 = [&](float n, float v1, float v2, float v3, float e) {
      return !(n > 0.0f) || !(gm1 * e > 0.0f) || !(fabsf(v1) < INFINITY) || !(fabsf(v2) < INFINITY) ||
             !(fabsf(v3) < INFINITY);
    };
    return lane_y ? bad1(w[0].y, w[1].y, w[2].y, w[3].y, w[4].y) : bad1(w[0].x, w[1].x, w[2].x, w[3].x, w[4].x);
  }

  static __device__ void tile(const StageArgs<float>& A, Smem& S, int bx, int by, int bz, double& speed_out,
                              double (&tot)[NV], bool& bad) {
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int nx = A.n[0], ny = A.n[1], nm = A.n[2];
    const size_t plane = (size_t)nx * ny;
    const size_t vs = plane * nm;
    const int a0 = bx * TX, b0 = by * TY;
    const int ca = a0 + tx, cb = b0 + ty;
    const bool own_valid = ca < nx && cb < ny;
    const int m0 = bz * A.kchunk;
    const int m1 = min(nm, m0 + A.kchunk);
    const f2 dt = bc2(STAGE == 2 ? (float)(*A.dt) : 0.0f);
    const f2 iwx = bc2(A.iw[0][min(ca, nx + 1) + 2]);
    const f2 iwy = bc2(A.iw[1][min(cb, ny + 1) + 2]);

    for (int k = tid; k < TX + 4; k += NT) S.gx[k] = geo_b(A, 0, a0 + k - 2);
    for (int k = tid; k < TY + 4; k += NT) S.gy[k] = geo_b(A, 1, b0 + k - 2);
    const typename K::ColRef own = K::col_ref(A, ca, cb);
    int hsx[HSLOTS], hsy[HSLOTS];
    typename K::ColRef halo[HSLOTS];
#pragma unroll
    for (int k = 0; k < HSLOTS; ++k) {
      const int h = tid + k * NT;
      int sx = 0, sy = 0;
      if (h < NHALO) {
        if (h < 4 * TX) {
          const int r = h / TX;
          sx = h % TX + 2;
          sy = r < 2 ? r : TY + r;
        } else {
          const int hh = h - 4 * TX;
          const int c = hh & 3;
          sy = (hh >> 2) + 2;
          sx = c < 2 ? c : TX + c;
        }
      }
      hsx[k] = sx;
      hsy[k] = sy;
      halo[k] = K::col_ref(A, a0 + sx - 2, b0 + sy - 2);
    }

    ColumnSum2 tcol[NV];
    f2 speed_max = bc2(0.0f);
    // ring: wp = W(m, m+1) of the pair being processed, wlo = W(m - 1) and
    // flo = F(m - 1/2) from the previous pair
    f2 wp[NV];
    float wlo[NV], flo[NV];
    load_pair(A, own, m0 - 2, dt, vs, wp);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      wlo[v] = wp[v].x;  // stands in for W(m0 - 3), which only feeds unused values
      flo[v] = 0.0f;
    }

    for (int m = m0 - 2; m < m1; m += 2) {
      f2 wn[NV], fu[NV];
      load_pair(A, own, m + 2, dt, vs, wn);
      {
        // march-axis slopes of P = (m, m+1) and S = (m+1, m+2), faces m+1/2, m+3/2
        const Geo2 gp = geo2(K::geo(A, 2, m), K::geo(A, 2, m + 1));
        const Geo2 gs = geo2(K::geo(A, 2, m + 1), K::geo(A, 2, m + 2));
        f2 wl[NV], wr[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const f2 ws = mk2(wp[v].y, wn[v].x);
          const f2 sp = limited_slope2(mk2(wlo[v], wp[v].x), wp[v], ws, gp);
          const f2 ss = limited_slope2(wp[v], ws, wn[v], gs);
          wl[v] = fma2(sp, gp.h, wp[v]);
          wr[v] = fma2(ss, gs.nh, ws);
        }
        flux<2>(A, wl, wr, fu);
      }
      if (m < m0) {  // warm-up pair: advance the ring only
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          flo[v] = fu[v].y;
          wlo[v] = wp[v].y;
          wp[v] = wn[v];
        }
        continue;
      }
      // With the pair in buffer `buf` (put during the previous pair, or here
      // for the first): face states; barrier; faces, and the next pair into
      // the other buffer; barrier.
      const int buf = ((m - m0) >> 1) & 1;
      if (m == m0) {
        put_plane(A, S, buf, m, tid, tx, ty, wp, halo, hsx, hsy, dt, vs);
        __syncthreads();
      }
      face_states(S, buf, tid, tx, ty, wp);
      __syncthreads();
      faces(A, S, tid, tx, ty);
      if (m + 2 < m1) put_plane(A, S, buf ^ 1, m + 2, tid, tx, ty, wn, halo, hsx, hsy, dt, vs);
      __syncthreads();

      if (own_valid) {
        const bool has_y = m + 1 < m1;  // lane y lies in the chunk
        const f2 iwm = mk2(A.iw[2][m + 2], A.iw[2][m + 3]);
        f2 L[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          f2 d = mul2(sub2(S.fx[v][ty][tx + 1], S.fx[v][ty][tx]), iwx);
          d = fma2(sub2(S.fy[v][ty + 1][tx], S.fy[v][ty][tx]), iwy, d);
          d = fma2(sub2(fu[v], mk2(flo[v], fu[v].x)), iwm, d);
          L[v] = neg2(d);
        }
        if (A.has_source) {
          // external force and power (Sec. 4.3.2), from the stage-input state
          f2 power = bc2(0.0f);
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const f2 g = bc2(A.grad_phi[q]);
            L[1 + q] = sub2(L[1 + q], mul2(wp[0], g));
            power = fma2(mul2(wp[0], wp[1 + q]), g, power);
          }
          L[NV - 1] = sub2(L[NV - 1], power);
        }
        const size_t c0 = ((size_t)m * ny + cb) * nx + ca;
        const size_t c1 = c0 + plane;
        bad |= nonphysical(wp, false, A.gm1);
        if (has_y) bad |= nonphysical(wp, true, A.gm1);
        if (STAGE == 1) {
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            A.out[v * vs + c0] = L[v].x;
            if (has_y) A.out[v * vs + c1] = L[v].y;
          }
          // CFL speed (Eq. courantTimeStep) on U^n at the cell centres
          const f2 cs = sound_speed2(bc2(A.gamma), mul2(bc2(A.gm1), wp[4]), wp[0]);
          f2 s = max2(mul2(add2(abs2(wp[1]), cs), iwx), mul2(add2(abs2(wp[2]), cs), iwy));
          s = max2(s, mul2(add2(abs2(wp[3]), cs), iwm));
          speed_max = max2(speed_max, mk2(s.x, has_y ? s.y : 0.0f));
          if (A.want_totals) {
            const f2 dh = mk2(A.wdh[2][m], has_y ? A.wdh[2][m + 1] : 0.0f);
            const f2 dl = mk2(A.wdl[2][m], has_y ? A.wdl[2][m + 1] : 0.0f);
#pragma unroll
            for (int v = 0; v < NV; ++v)
              tcol[v].add_product(mk2(__ldg(A.un + v * vs + c0), has_y ? __ldg(A.un + v * vs + c1) : 0.0f), dh, dl);
          }
        } else {
          const f2 hdt = mul2(bc2(0.5f), dt);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const f2 u0 = mk2(__ldg(A.un + v * vs + c0), has_y ? __ldg(A.un + v * vs + c1) : 0.0f);
            const f2 k = mk2(__ldg(A.k1 + v * vs + c0), has_y ? __ldg(A.k1 + v * vs + c1) : 0.0f);
            const f2 o = fma2(hdt, add2(k, L[v]), u0);
            A.out[v * vs + c0] = o.x;
            if (has_y) A.out[v * vs + c1] = o.y;
          }
        }
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        flo[v] = fu[v].y;
        wlo[v] = wp[v].y;
        wp[v] = wn[v];
      }
    }

    if (STAGE == 1 && own_valid && A.want_totals) {
      const double area = A.wd[0][ca] * A.wd[1][cb];
#pragma unroll
      for (int v = 0; v < NV; ++v) tot[v] = fma(tcol[v].value(), area, tot[v]);
    }
    speed_out = fmax(speed_out, (double)fmaxf(speed_max.x, speed_max.y));
  }

  static __device__ void run(const StageArgs<float>& A) {
    extern __shared__ __align__(16) unsigned char smem_pair[];
    Smem& S = *reinterpret_cast<Smem*>(smem_pair);
    double speed_max = 0.0;
    double tot[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) tot[v] = 0.0;
    bool bad = false;
    tile(A, S, blockIdx.x, blockIdx.y, blockIdx.z, speed_max, tot, bad);
    if (bad) atomicOr(A.status, STATUS_NONPHYS);
    if (STAGE == 1) {
      // the fixed-order block reduction of the scalar kernel
      const int warp = tid_warp(), lane = threadIdx.x & 31;
      double r[NV + 1];
      r[0] = warp_max(speed_max);
#pragma unroll
      for (int v = 0; v < NV; ++v) r[1 + v] = warp_sum(tot[v]);
      if (lane == 0) {
#pragma unroll
        for (int v = 0; v <= NV; ++v) S.red[warp][v] = r[v];
      }
      __syncthreads();
      const int tid = threadIdx.x;
      if (tid <= NV) {
        const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        double acc = S.red[0][tid];
        for (int wi = 1; wi < NT / 32; ++wi) acc = tid == 0 ? fmax(acc, S.red[wi][0]) : acc + S.red[wi][tid];
        if (tid == 0) A.part_speed[blk] = acc;
        else A.part_tot[blk * NV + (tid - 1)] = acc;
      }
    }
  }

  static __device__ __forceinline__ int tid_warp() { return threadIdx.x >> 5; }
};

// MINB: CTAs per SM the register allocation must allow.
template <int SOLVER, int STAGE, int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX * TY, MINB) hydro_stage_pair_kernel(const StageArgs<float> A) {
  StagePair<SOLVER, STAGE, TX, TY>::run(A);
}

}  // namespace gh
