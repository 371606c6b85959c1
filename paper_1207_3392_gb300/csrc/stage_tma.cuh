// stage_tma.cuh -- one Runge-Kutta stage of the 3D FP32 update with the state
// planes staged in shared memory by the tensor memory accelerator (TMA).
//
// The arithmetic is that of stage_kernel.cuh (Algorithm 1 of arXiv:1207.3392
// fused into one pass per stage; same functions, same order of operations,
// so the results are bitwise those of every other tile shape).  What differs
// is how the state reaches the compute threads:
//
//   * One producer warp (the CTA's last) walks the CTA's planes along the
//     march axis (z) and, per plane, issues one 4D cp.async.bulk.tensor load
//     of the box x in [a0 - 4, a0 + TX + 4), y in [b0 - 2, b0 + TY + 2), all
//     five conserved variables (stage 2: also the stage buffer K) into a ring
//     of NS shared-memory slots, completing on the slot's `full` mbarrier.
//     Planes outside the domain along z are loaded from the plane the
//     boundary rule maps them to (the reflecting flip of S_z is applied on
//     read).  x starts on a 16-byte boundary (a0 is a multiple of 32).
//   * The TX x TY compute threads read the raw state of their cells from the
//     slot (no global loads, no address arithmetic), recover the primitives
//     and write them back into the same slot positions (in place), which is
//     then the shared plane the slopes and face states read.  Cells outside
//     the domain in x or y (ghost cells and the columns past a ragged edge)
//     are read from global memory through the boundary map instead, so no
//     thread reads another's raw value in shared memory.
//   * A slot is released to the producer (its `empty` mbarrier, one arrival
//     per compute warp after a proxy fence) when the plane's faces are done.
//
// Iteration m (planes m0 .. m1-1 of the chunk):
//   A  face states of plane m from its slot            (compute barrier)
//   B  in-plane fluxes of plane m; plane m+1 recovered in place (barrier)
//   C  own column of plane m+2 read from its slot; march-axis slope at m+1
//      and face flux at m + 1/2
//   D  divergence and stage combine of plane m
// so the load of plane m+2 into the slot plane m-1 left has a whole
// iteration to land: NS = 3 slots suffice.
//
// Every mbarrier wait is bounded (about one second of %globaltimer).  A wait
// that gives up sets STATUS_TIMEOUT in the device status word; a compute
// thread also keeps a flag that the next compute barrier ORs over all compute
// threads (bar.red.or), so they all leave the plane loop at the same barrier.
// A producer that gives up stops issuing (the compute threads then give up
// on the missing plane) and waits, bounded, for its loads still in flight
// before returning.
#pragma once

#include <cuda.h>

#include "mbarrier.cuh"
#include "stage_kernel.cuh"

namespace gh {

// Kernel parameters of the TMA stage kernel: the plain stage arguments plus
// the tensor maps of U^n and K (4D: x, y, z, variable; FP32).
struct TmaStageArgs {
  StageArgs<float> A;
  CUtensorMap map_u;
  CUtensorMap map_k;
};

template <int SOLVER, int STAGE, int TX, int TY, int NS>
struct StageTma {
  using T = float;
  using Base = StageKernel<3, float, SOLVER, STAGE, TX, TY, true>;
  using ColRef = typename Base::ColRef;
  static constexpr int NV = 5;
  static constexpr int NT = TX * TY;  // compute threads
  static constexpr int NW = NT / 32;  // compute warps
  static constexpr int NTHR = NT + 32;
  static constexpr int XB = TX + 8;  // box columns: cells a0 - 4 .. a0 + TX + 3
  static constexpr int YB = TY + 4;  // box rows: cells b0 - 2 .. b0 + TY + 1
  static constexpr int PL = NV * YB * XB;
  static constexpr int NARR = STAGE == 2 ? 2 : 1;
  static constexpr unsigned BOX_BYTES = (unsigned)(PL * sizeof(T));
  // each box array starts on a 128-byte boundary (TMA destination)
  static constexpr int ARR = ((PL * (int)sizeof(T) + 127) / 128) * 128 / (int)sizeof(T);
  static constexpr int SLOT = NARR * ARR;
  static constexpr int NHALO = 4 * TX + 4 * TY;
  static constexpr int HSLOTS = (NHALO + NT - 1) / NT;
  static constexpr int NJ = 2 * TY + 2 * TX;
  static_assert(TX == 32 && NT % 32 == 0, "rows of one warp");
  static_assert(NJ <= NT && TX + TY <= NT, "halo face states and edge faces: one job per thread at most");
  static_assert(NS >= 3, "the ring needs the plane being faced, the next one and the one after");

  struct Smem {
    alignas(128) T ring[NS][SLOT];
    unsigned long long full[NS];
    unsigned long long empty[NS];
    Geo<T> gx[TX + 4];
    Geo<T> gy[TY + 4];
    T fx[NV][TY][TX + 1];
    T fy[NV][TY + 1][TX];
    T xs[2][NV][TY][TX + 2];
    T ys[2][NV][TY + 2][TX];
    double red[NW][NV + 1];
  };

  // Value of variable v at box row r, column c of slot s (raw U, or W once
  // recovered in place); stage 2: the stage buffer K behind it.
  static __device__ __forceinline__ T& box(Smem& S, int s, int v, int r, int c) {
    return S.ring[s][(v * YB + r) * XB + c];
  }
  static __device__ __forceinline__ T kbox(Smem& S, int s, int v, int r, int c) {
    return S.ring[s][ARR + (v * YB + r) * XB + c];
  }

  // Primitives of the cell at box (r, c) of slot s, plane index p mapped to
  // pm (flip fz of S_z).  Inside the domain in x and y: from the slot; else
  // (ghost cell or a column past a ragged edge) from global memory through
  // the boundary map `ref`, exactly as the kernel without TMA loads it.
  static __device__ __forceinline__ void read_cell(const StageArgs<T>& A, Smem& S, int s, int r, int c, bool inside,
                                                   const ColRef& ref, int pm, bool fz, T dt, size_t vs, T (&w)[NV]) {
    T u[NV];
    if (inside) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T x = box(S, s, v, r, c);
        if (STAGE == 2) x = fma(dt, kbox(S, s, v, r, c), x);
        u[v] = x;
      }
    } else {
      const size_t cg = (size_t)ref.off + (size_t)pm * ((size_t)A.n[0] * A.n[1]);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T x = __ldg(A.un + v * vs + cg);
        if (STAGE == 2) x = fma(dt, __ldg(A.k1 + v * vs + cg), x);
        u[v] = x;
      }
      if (ref.fa) u[1] = -u[1];
      if (ref.fb) u[2] = -u[2];
    }
    if (fz) u[3] = -u[3];
    recover<3>(u, w);
  }

  // Face states of the own cell and the one-sided halo states (the formulas
  // of StageKernel::face_states on the slot's in-place primitives).
  static __device__ __forceinline__ void face_states(Smem& S, int s, int tid, int tx, int ty, const T (&wc)[NV]) {
    const int r = ty + 2, c = tx + 4;
    {
      const Geo<T> g = S.gx[tx + 2];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T sv = limited_slope(box(S, s, v, r, c - 1), wc[v], box(S, s, v, r, c + 1), g);
        S.xs[0][v][ty][tx + 1] = fma(-sv, g.h, wc[v]);
        S.xs[1][v][ty][tx + 1] = fma(sv, g.h, wc[v]);
      }
    }
    {
      const Geo<T> g = S.gy[ty + 2];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T sv = limited_slope(box(S, s, v, r - 1, c), wc[v], box(S, s, v, r + 1, c), g);
        S.ys[0][v][ty + 1][tx] = fma(-sv, g.h, wc[v]);
        S.ys[1][v][ty + 1][tx] = fma(sv, g.h, wc[v]);
      }
    }
    const int j = tid - (NT - NJ);
    if (j < 0) return;
    if (j < 2 * TY) {
      // x: column -1 (upper face value) or column TX (lower face value) of row j / 2
      const int rr = j >> 1;
      const bool up = j & 1;
      const int slot = up ? TX + 2 : 1;  // slot column of the halo cell (cell a0 + slot - 2)
      const Geo<T> g = S.gx[slot];
      const int cc = slot + 2;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T w1 = box(S, s, v, rr + 2, cc);
        const T sv = limited_slope(box(S, s, v, rr + 2, cc - 1), w1, box(S, s, v, rr + 2, cc + 1), g);
        if (up) S.xs[0][v][rr][TX + 1] = fma(-sv, g.h, w1);
        else S.xs[1][v][rr][0] = fma(sv, g.h, w1);
      }
    } else {
      // y: row -1 (upper face value) or row TY (lower face value) of column cl
      const int jj = j - 2 * TY;
      const bool up = jj >= TX;
      const int cl = up ? jj - TX : jj;
      const int slot = up ? TY + 2 : 1;
      const Geo<T> g = S.gy[slot];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T w1 = box(S, s, v, slot, cl + 4);
        const T sv = limited_slope(box(S, s, v, slot - 1, cl + 4), w1, box(S, s, v, slot + 1, cl + 4), g);
        if (up) S.ys[0][v][TY + 1][cl] = fma(-sv, g.h, w1);
        else S.ys[1][v][0][cl] = fma(sv, g.h, w1);
      }
    }
  }

  static __device__ __forceinline__ void x_face(const StageArgs<T>& A, Smem& S, int face, int frow) {
    T wl[NV], wr[NV], f[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      wl[v] = S.xs[1][v][frow][face];
      wr[v] = S.xs[0][v][frow][face + 1];
    }
    face_flux<T, 3, 0, SOLVER>(wl, wr, A.gamma, A.gm1, f);
#pragma unroll
    for (int v = 0; v < NV; ++v) S.fx[v][frow][face] = f[v];
  }

  static __device__ __forceinline__ void y_face(const StageArgs<T>& A, Smem& S, int face, int col) {
    T wl[NV], wr[NV], f[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      wl[v] = S.ys[1][v][face][col];
      wr[v] = S.ys[0][v][face + 1][col];
    }
    face_flux<T, 3, 1, SOLVER>(wl, wr, A.gamma, A.gm1, f);
#pragma unroll
    for (int v = 0; v < NV; ++v) S.fy[v][face][col] = f[v];
  }

  // Cell-aligned in-plane faces (as the PRE path of StageKernel::faces).
  static __device__ __forceinline__ void faces(const StageArgs<T>& A, Smem& S, int tid, int tx, int ty) {
    x_face(A, S, tx, ty);
    y_face(A, S, ty, tx);
    const int j = tid - (NT - (TX + TY));
    if (j >= 0) {
      if (j < TY) x_face(A, S, TX, j);
      else y_face(A, S, TY, j - TY);
    }
  }

  static __device__ void run(const TmaStageArgs& P) {
    extern __shared__ __align__(128) unsigned char tma_smem_raw[];
    Smem& S = *reinterpret_cast<Smem*>(tma_smem_raw);
    const StageArgs<T>& A = P.A;
    const int tid = threadIdx.x;
    const int nx = A.n[0], ny = A.n[1], nm = A.n[2];
    const size_t vs = (size_t)nx * ny * nm;
    const int a0 = blockIdx.x * TX, b0 = blockIdx.y * TY;
    const int m0 = blockIdx.z * A.kchunk;
    const int m1 = min(nm, m0 + A.kchunk);
    const int nplanes = (m1 - m0) + 4;  // m0 - 2 .. m1 + 1

    if (tid == 0) {
      for (int s = 0; s < NS; ++s) {
        tma::mbar_init(&S.full[s], 1u);
        tma::mbar_init(&S.empty[s], (unsigned)NW);
      }
      tma::fence_mbar_init();
    }
    for (int k = tid; k < TX + 4; k += NTHR) S.gx[k] = Base::geo(A, 0, a0 + k - 2);
    for (int k = tid; k < TY + 4; k += NTHR) S.gy[k] = Base::geo(A, 1, b0 + k - 2);
    __syncthreads();

    if (tid >= NT) {
      // producer warp: lane 0 issues the plane loads
      if (tid != NT) return;
      int issued = 0;
      for (int i = 0; i < nplanes; ++i) {
        const int s = i % NS;
        if (i >= NS && !tma::mbar_wait(&S.empty[s], (unsigned)(((i / NS) - 1) & 1))) {
          atomicOr(A.status, STATUS_TIMEOUT);
          break;
        }
        bool fz;
        const int pm = bc_map(m0 - 2 + i, nm, A.bc_lo[2], A.bc_hi[2], fz);
        tma::mbar_expect_tx(&S.full[s], BOX_BYTES * NARR);
        tma::load_4d(&S.ring[s][0], &P.map_u, a0 - 4, b0 - 2, pm, 0, &S.full[s]);
        if (STAGE == 2) tma::load_4d(&S.ring[s][ARR], &P.map_k, a0 - 4, b0 - 2, pm, 0, &S.full[s]);
        ++issued;
      }
      // do not leave while a load of this CTA may still write its shared memory
      for (int i = issued > NS ? issued - NS : 0; i < issued; ++i)
        if (!tma::mbar_wait(&S.full[i % NS], (unsigned)((i / NS) & 1))) atomicOr(A.status, STATUS_TIMEOUT);
      return;
    }

    // compute threads
    const int tx = tid % TX, ty = tid / TX, lane = tid & 31;
    const int ca = a0 + tx, cb = b0 + ty;
    const bool own_valid = ca < nx && cb < ny;
    const ColRef own_ref = Base::col_ref(A, ca, cb);
    const T dt = STAGE == 2 ? (T)(*A.dt) : T(0);
    const T iwx = A.iw[0][min(ca, nx + 1) + 2];
    const T iwy = A.iw[1][min(cb, ny + 1) + 2];
    // halo slots h = tid + k NT: rows -2, -1, TY, TY+1 of the tile, then
    // columns -2, -1, TX, TX+1 of every row (box row r, column c)
    int hr[HSLOTS], hc[HSLOTS];
    bool hin[HSLOTS];
    ColRef halo[HSLOTS];
#pragma unroll
    for (int k = 0; k < HSLOTS; ++k) {
      const int h = tid + k * NT;
      int sx = 0, sy = 0;
      if (h < NHALO) {
        if (h < 4 * TX) {
          const int rr = h / TX;
          sx = h % TX + 2;
          sy = rr < 2 ? rr : TY + rr;
        } else {
          const int hh = h - 4 * TX;
          const int cc = hh & 3;
          sy = (hh >> 2) + 2;
          sx = cc < 2 ? cc : TX + cc;
        }
      }
      const int gxh = a0 + sx - 2, gyh = b0 + sy - 2;
      hr[k] = sy;
      hc[k] = sx + 2;
      hin[k] = gxh >= 0 && gxh < nx && gyh >= 0 && gyh < ny;
      halo[k] = Base::col_ref(A, gxh, gyh);
    }

    double speed_out = 0.0;
    double tot[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) tot[v] = 0.0;
    bool bad = false;
    ColumnSum<T> tcol[NV];
    T speed_max = T(0);

    auto slot_of = [&](int p) { return (p - (m0 - 2)) % NS; };
    auto parity_of = [&](int p) { return (unsigned)(((p - (m0 - 2)) / NS) & 1); };
    bool timed_out = false;  // this thread gave up waiting for a plane
    // primitives of the own cell at plane p (waits for the plane)
    auto own = [&](int p, T (&w)[NV]) {
      const int s = slot_of(p);
      if (timed_out || !tma::mbar_wait(&S.full[s], parity_of(p))) {
        if (!timed_out) atomicOr(A.status, STATUS_TIMEOUT);
        timed_out = true;
#pragma unroll
        for (int v = 0; v < NV; ++v) w[v] = T(1);
        return;
      }
      bool fz;
      const int pm = bc_map(p, nm, A.bc_lo[2], A.bc_hi[2], fz);
      read_cell(A, S, s, ty + 2, tx + 4, own_valid, own_ref, pm, fz, dt, vs, w);
    };
    // the warp is done with plane p
    auto release = [&](int p) {
      tma::fence_proxy_async();
      __syncwarp();
      if (lane == 0) tma::mbar_arrive(&S.empty[slot_of(p)]);
    };
    // own primitives wo and the halo of plane p into its slot, in place
    auto put_plane = [&](int p, const T (&wo)[NV]) {
      const int s = slot_of(p);
      bool fz;
      const int pm = bc_map(p, nm, A.bc_lo[2], A.bc_hi[2], fz);
#pragma unroll
      for (int k = 0; k < HSLOTS; ++k) {
        if (tid + k * NT < NHALO) {
          T wh[NV];
          read_cell(A, S, s, hr[k], hc[k], hin[k], halo[k], pm, fz, dt, vs, wh);
#pragma unroll
          for (int v = 0; v < NV; ++v) box(S, s, v, hr[k], hc[k]) = wh[v];
        }
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) box(S, s, v, ty + 2, tx + 4) = wo[v];
    };

    // ring warm-up: W at m0-2 .. m0+1, slopes at m0-1 and m0, the face m0 - 1/2
    T wk[NV], wk1[NV], sk[NV], flo[NV];
    {
      T wa[NV], wb[NV], sa[NV];
      own(m0 - 2, wa);
      release(m0 - 2);
      own(m0 - 1, wb);
      release(m0 - 1);
      own(m0, wk);
      own(m0 + 1, wk1);
      if (m0 + 1 >= m1) release(m0 + 1);
      const Geo<T> gm = Base::geo(A, 2, m0 - 1), g0 = Base::geo(A, 2, m0);
      Base::slopes(A, wa, wb, wk, gm, sa);
      Base::slopes(A, wb, wk, wk1, g0, sk);
      Base::m_face(A, wb, sa, gm.h, wk, sk, g0.h, 0u, flo);
    }
    put_plane(m0, wk);
    bool abort = tma::sync_compute_or<NT>(timed_out);

    for (int m = m0; m < m1 && !abort; ++m) {
      // A: face states of plane m; a thread that gave up on a plane (phase C
      // of the previous iteration) makes the whole CTA stop at this barrier
      face_states(S, slot_of(m), tid, tx, ty, wk);
      abort = tma::sync_compute_or<NT>(timed_out);
      if (abort) break;
      // B: in-plane fluxes of plane m; plane m + 1 recovered in place
      faces(A, S, tid, tx, ty);
      if (m + 1 < m1) put_plane(m + 1, wk1);
      tma::sync_compute_or<NT>(false);
      release(m);
      // C: own column at m + 2; slope at m + 1; face m + 1/2
      T wk2[NV], sk1[NV], fhi[NV];
      own(m + 2, wk2);
      if (m + 2 >= m1) release(m + 2);
      const Geo<T> g0 = Base::geo(A, 2, m), g1 = Base::geo(A, 2, m + 1);
      Base::slopes(A, wk, wk1, wk2, g1, sk1);
      Base::m_face(A, wk, sk, g0.h, wk1, sk1, g1.h, 0u, fhi);
      // D: divergence and stage combine of plane m
      if (own_valid) {
        const T iwm = A.iw[2][m + 2];
        T L[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T d = (S.fx[v][ty][tx + 1] - S.fx[v][ty][tx]) * iwx;
          d += (S.fy[v][ty + 1][tx] - S.fy[v][ty][tx]) * iwy;
          d += (fhi[v] - flo[v]) * iwm;
          L[v] = -d;
        }
        if (A.has_source) {
          T power = T(0);
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            L[1 + q] -= wk[0] * A.grad_phi[q];
            power = fma(wk[0] * wk[1 + q], A.grad_phi[q], power);
          }
          L[NV - 1] -= power;
        }
        const size_t c = ((size_t)m * ny + cb) * nx + ca;
        bad |= Base::nonphysical(wk, A.gm1);
        if (STAGE == 1) {
#pragma unroll
          for (int v = 0; v < NV; ++v) A.out[v * vs + c] = L[v];
          const T cs = sound_speed(A.gamma, A.gm1 * wk[NV - 1], wk[0]);
          T sp = (fabs(wk[1]) + cs) * iwx;
          sp = fmax(sp, (fabs(wk[2]) + cs) * iwy);
          sp = fmax(sp, (fabs(wk[3]) + cs) * iwm);
          speed_max = fmax(speed_max, sp);
          if (A.want_totals) {
            const T dm_hi = A.wdh[2][m], dm_lo = A.wdl[2][m];
#pragma unroll
            for (int v = 0; v < NV; ++v) tcol[v].add_product(__ldg(A.un + v * vs + c), dm_hi, dm_lo);
          }
        } else {
          const T hdt = T(0.5) * dt;
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const T u0 = __ldg(A.un + v * vs + c), k = __ldg(A.k1 + v * vs + c);
            A.out[v * vs + c] = fma(hdt, add_rn(k, L[v]), u0);
          }
        }
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        flo[v] = fhi[v];
        wk[v] = wk1[v];
        wk1[v] = wk2[v];
        sk[v] = sk1[v];
      }
    }

    if (STAGE == 1 && own_valid && A.want_totals) {
      double area = A.wd[0][ca] * A.wd[1][cb];
#pragma unroll
      for (int v = 0; v < NV; ++v) tot[v] = fma(tcol[v].value(), area, tot[v]);
    }
    speed_out = fmax(speed_out, (double)speed_max);
    if (bad) atomicOr(A.status, STATUS_NONPHYS);
    if (STAGE == 1) {
      // fixed-order block reduction of (max speed, totals) into the CTA's partials
      const int warp = tid >> 5;
      double rr[NV + 1];
      rr[0] = warp_max(speed_out);
#pragma unroll
      for (int v = 0; v < NV; ++v) rr[1 + v] = warp_sum(tot[v]);
      if (lane == 0) {
#pragma unroll
        for (int v = 0; v <= NV; ++v) S.red[warp][v] = rr[v];
      }
      tma::sync_compute_or<NT>(false);
      if (tid <= NV) {
        double acc = S.red[0][tid];
        for (int wi = 1; wi < NW; ++wi) acc = tid == 0 ? fmax(acc, S.red[wi][0]) : acc + S.red[wi][tid];
        const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        if (tid == 0) A.part_speed[blk] = acc;
        else A.part_tot[blk * NV + (tid - 1)] = acc;
      }
    }
  }
};

template <int SOLVER, int STAGE, int TX, int TY, int NS, int MINB>
__global__ void __launch_bounds__(TX * TY + 32, MINB) hydro_stage_tma_kernel(const __grid_constant__ TmaStageArgs P) {
  StageTma<SOLVER, STAGE, TX, TY, NS>::run(P);
}

}  // namespace gh
