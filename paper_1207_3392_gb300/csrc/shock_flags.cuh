// shock_flags.cuh -- the shock detector of the HLLC -> HLL switch, shared by
// the plain pass (aux_kernels.cu) and the TMA-staged pass (flags_tma.cu).
//
// Sec. 3.2 describes the switch but not its detector.  The detector here:
// cell c lies on a shock moving along axis r when, across its two neighbours
// along r (boundary-mapped like the stage kernel's ghosts), the flow is
// compressive, v_r(+) - v_r(-) < 0, and the pressure jumps by more than half
// the smaller pressure.  Bit r of flags[c] records it.
#pragma once

#include "aux_kernels.h"
#include "hydro_device.cuh"

namespace gh {
namespace shock {

// The test across one axis: (pm, vm) of the lower neighbour, (pp, vp) of the
// upper one (both comparisons evaluated, no branch).
template <class T>
__device__ __forceinline__ bool jump(T pm, T vm, T pp, T vp) {
  return (vp - vm < T(0)) & (fabs(pp - pm) > T(0.5) * fmin(pm, pp));
}

// Pressure and velocity of the cell (i, j, k) of the stage's state (U^n, or
// U^n + dt K in stage 2), each index in [-1, n] so that bc_map returns a cell
// of the mesh.  A mirrored ghost negates the normal momentum, which negates
// that velocity component and leaves p unchanged.
template <class T, int NDIM>
__device__ __forceinline__ void cell_pv(const FlagArgs<T>& A, T gm1, T dt, int i, int j, int k, T& p, T (&v)[NDIM]) {
  constexpr int NV = NDIM + 2;
  bool f0 = false, f1 = false, f2 = false;
  const int ii = bc_map(i, A.n[0], A.bc_lo[0], A.bc_hi[0], f0);
  const int jj = bc_map(j, A.n[1], A.bc_lo[1], A.bc_hi[1], f1);
  const int kk = NDIM > 2 ? bc_map(k, A.n[2], A.bc_lo[2], A.bc_hi[2], f2) : 0;
  const size_t cc = ((size_t)kk * A.n[1] + jj) * A.n[0] + ii;
  T u[NV], w[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    T x = A.un[q * A.ncell + cc];
    if (A.stage == 2) x = fma(dt, A.k1[q * A.ncell + cc], x);
    u[q] = x;
  }
  if (f0) u[1] = -u[1];
  if (f1) u[2] = -u[2];
  if (NDIM > 2 && f2) u[NV - 2] = -u[NV - 2];
  recover<NDIM>(u, w);
  p = gm1 * w[NV - 1];
#pragma unroll
  for (int q = 0; q < NDIM; ++q) v[q] = w[1 + q];
}

// Flag bits of the mesh cell (x, y, z) from its neighbours read one by one
// through the boundary map.
template <class T, int NDIM>
__device__ __forceinline__ unsigned bits_direct(const FlagArgs<T>& A, T gm1, T dt, int x, int y, int z) {
  unsigned bits = 0;
#pragma unroll
  for (int r = 0; r < NDIM; ++r) {
    T p[2], v[2];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      int c[3] = {x, y, z};
      c[r] += side ? 1 : -1;
      T vv[NDIM];
      cell_pv<T, NDIM>(A, gm1, dt, c[0], c[1], c[2], p[side], vv);
      v[side] = vv[r];
    }
    if (jump(p[0], v[0], p[1], v[1])) bits |= 1u << r;
  }
  return bits;
}

}  // namespace shock
}  // namespace gh
