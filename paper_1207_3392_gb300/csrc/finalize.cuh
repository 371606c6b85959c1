// finalize.cuh -- the per-cell CFL speed, the fixed-order fold of the per-CTA
// reduction partials and the time-step update (Eq. courantTimeStep x C_CFL),
// shared by the speed and finalize kernels and the one-launch advances, so
// that all give bitwise the same dt, time and totals.
#pragma once

#include "aux_kernels.h"
#include "hydro_device.cuh"

namespace gh {
namespace fin {

// Inverse CFL time of cell c, max_q (|v_q| + c_s) / dq (Eq. courantTimeStep),
// from the state A.U (read through L2 when COH: the one-launch advances read
// states written earlier in the same launch); bad is set for rho <= 0 or
// p <= 0.
template <class T, int NDIM, bool COH>
__device__ __forceinline__ T cell_speed(const ReduceArgs<T>& A, size_t c, bool& bad) {
  constexpr int NV = NDIM + 2;
  const T gm1 = (T)(A.gamma - 1.0), gamma = (T)A.gamma;
  T u[NV], w[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    if constexpr (COH) u[v] = __ldcg(A.U + v * A.ncell + c);
    else u[v] = A.U[v * A.ncell + c];
  }
  recover<NDIM>(u, w);
  const T p = gm1 * w[NV - 1];
  bad |= !(w[0] > T(0)) || !(p > T(0));
  const T cs = sqrt(gamma * p / w[0]);
  size_t r = c;
  T s = T(0);
#pragma unroll
  for (int q = 0; q < NDIM; ++q) {
    const size_t i = r % A.n[q];
    r /= A.n[q];
    s = fmax(s, (fabs(w[1 + q]) + cs) * A.iw[q][i + 2]);
  }
  return s;
}

// Fixed butterfly over the warp: every lane ends with the same sum / max.
__device__ __forceinline__ void fold_warp(double (&s)[5], unsigned long long& m) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int v = 0; v < 5; ++v) s[v] += __shfl_xor_sync(0xffffffffu, s[v], o);
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, m, o);
    m = b > m ? b : m;
  }
}

// Partials [lo, hi) folded by one warp: lane j takes the partials j, j + 32,
// ... in order (the totals of every variable, and the largest speed compared
// as bit patterns, which order like positive doubles), then the butterfly.
__device__ __forceinline__ void fold_slice(const FinalizeArgs& A, long long lo, long long hi, int lane, double (&s)[5],
                                           unsigned long long& mb) {
  constexpr unsigned long long SIGNLESS = 0x7fffffffffffffffull;  // a -0.0 compares as +0.0
  const bool tot = A.part_tot != nullptr, spd = A.part_speed != nullptr;
#pragma unroll
  for (int v = 0; v < 5; ++v) s[v] = 0.0;
  mb = 0;
#pragma unroll 8
  for (long long i = lo + lane; i < hi; i += 32) {
    if (tot) {
#pragma unroll
      for (int v = 0; v < 5; ++v)
        if (v < A.nv) s[v] += __ldcg(A.part_tot + i * A.nv + v);
    }
    if (spd) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(__ldcg(A.part_speed + i)) & SIGNLESS;
      mb = b > mb ? b : mb;
    }
  }
  fold_warp(s, mb);
}

// The step dt at time t from the folded maximum speed (bit pattern mb), for
// modes FIN_FIXED and FIN_CFL; an invalid dt sets STATUS_NONPHYS and gives 0.
__device__ __forceinline__ double step_dt(const FinalizeArgs& A, unsigned long long mb, double t) {
  const double m = __longlong_as_double((long long)mb);
  double dt = A.mode == FIN_CFL ? A.cfl * (1.0 / m) : A.fixed_dt;
  if (A.t_end > 0.0) {
    if (t + dt > A.t_end) dt = A.t_end - t;
    if (!(dt > 0.0)) dt = 0.0;
  }
  if (!(dt >= 0.0) || !(dt < INFINITY)) {
    atomicOr(A.status, STATUS_NONPHYS);
    dt = 0.0;
  }
  return dt;
}

// The folded totals and speed into the scalar block; dt and t:
//   mode FIN_FIXED : dt = fixed_dt
//   mode FIN_CFL   : dt = cfl / max speed            (Eq. courantTimeStep x C_CFL)
//   mode FIN_REDUCE: only store dt_CFL and totals
// With t_end > 0 the step is clamped so that t never passes t_end.
__device__ __forceinline__ void finish(const FinalizeArgs& A, const double (&s)[5], unsigned long long mb, int lane) {
  unsigned* ticket = reinterpret_cast<unsigned*>(A.scal + SCAL_COUNT + FIN_CTAS * 6);
  if (A.part_tot != nullptr && lane < A.nv) {
    double tv = s[0];
#pragma unroll
    for (int v = 1; v < 5; ++v) tv = lane == v ? s[v] : tv;
    A.scal[SCAL_TOT + lane] = tv;
  }
  const double mx = __longlong_as_double((long long)mb);
  if (lane == 0) {
    const double m = mx;
    *ticket = 0;  // for the next launch on this scalar block
    if (A.part_speed) A.scal[SCAL_DTCFL] = 1.0 / m;
    if (A.mode != FIN_REDUCE) {
      const double t = A.scal[SCAL_T];
      const double dt = step_dt(A, mb, t);
      A.scal[SCAL_DT] = dt;
      A.scal[SCAL_T] = t + dt;
    }
  }
}

}  // namespace fin
}  // namespace gh
