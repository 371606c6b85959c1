// aux_kernels.cu -- small kernels around the stage kernels: initial state
// from primitives, precision conversion, the standalone CFL and totals
// reductions, and the single-CTA finalisation of dt and totals.
#include "aux_kernels.h"
#include "finalize.cuh"
#include "hydro_device.cuh"
#include "shock_flags.cuh"

namespace gh {

// U = (D, S, G) from (rho, v, p): D = rho, S = rho v, G = p/(gamma-1) + rho |v|^2 / 2
// (Sec. 3.5, m = 1), evaluated in FP64 and rounded once to the storage type.
template <class T>
__global__ void init_from_primitive_kernel(int ndim, size_t ncell, double gamma, const double* __restrict__ rho,
                                           const double* __restrict__ vel, const double* __restrict__ p,
                                           T* __restrict__ U) {
  const int nv = ndim + 2;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < ncell; c += (size_t)gridDim.x * blockDim.x) {
    const double n = rho[c];
    double v2 = 0.0;
    for (int q = 0; q < ndim; ++q) {
      const double v = vel[q * ncell + c];
      v2 += v * v;
      U[(1 + q) * ncell + c] = (T)(n * v);
    }
    U[c] = (T)n;
    U[(nv - 1) * ncell + c] = (T)(p[c] / (gamma - 1.0) + 0.5 * n * v2);
  }
}

template <class Tin, class Tout>
__global__ void convert_kernel(size_t count, const Tin* __restrict__ in, Tout* __restrict__ out) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < count; c += (size_t)gridDim.x * blockDim.x)
    out[c] = (Tout)in[c];
}

// Per-block max over cells of max_q (|v_q| + c_s) / dq, i.e. the inverse of the
// cell's CFL time (Eq. courantTimeStep).
template <class T, int NDIM>
__global__ void speed_kernel(ReduceArgs<T> A) {
  __shared__ double red[32];
  double best = 0.0;
  bool bad = false;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < A.ncell; c += (size_t)gridDim.x * blockDim.x)
    best = fmax(best, (double)fin::cell_speed<T, NDIM, false>(A, c, bad));
  if (bad) atomicOr(A.status, STATUS_NONPHYS);
  best = warp_max(best);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = red[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) acc = fmax(acc, red[i]);
    A.part_speed[blockIdx.x] = acc;
  }
}

// Per-block sums of U dV (FP64, fixed order).
template <class T, int NDIM>
__global__ void totals_kernel(ReduceArgs<T> A) {
  constexpr int NV = NDIM + 2;
  __shared__ double red[32][NV];
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < A.ncell; c += (size_t)gridDim.x * blockDim.x) {
    size_t r = c;
    double dV = 1.0;
#pragma unroll
    for (int q = 0; q < NDIM; ++q) {
      const size_t i = r % A.n[q];
      r /= A.n[q];
      dV *= A.wd[q][i];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = fma((double)A.U[v * A.ncell + c], dV, acc[v]);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = warp_sum(acc[v]);
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) red[threadIdx.x >> 5][v] = acc[v];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = red[0][threadIdx.x];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) s += red[i][threadIdx.x];
    A.part_tot[blockIdx.x * NV + threadIdx.x] = s;
  }
}

// Fold the per-CTA partials in a fixed order, spread over G <= FIN_CTAS CTAs
// of one warp (FP64 arithmetic is slow on this GPU: a single 256-thread CTA
// spent ~17 us on 1.5k partials; with few partials one CTA, G = 1, is fastest).
// CTA g takes slice g of the partials: lane j the partials j, j + 32, ... of
// the slice in order (the totals of every variable, and the largest speed,
// compared as bit patterns, which order like positive doubles), then a fixed
// butterfly across the lanes.  The last CTA to finish folds the FIN_CTAS slice
// results the same way (one per lane; G = 1 skips this), then sets dt and t:
//   mode FIN_FIXED : dt = fixed_dt
//   mode FIN_CFL   : dt = cfl / max speed            (Eq. courantTimeStep x C_CFL)
//   mode FIN_REDUCE: only store dt_CFL and totals
// With t_end > 0 the step is clamped so that t never passes t_end.  No CTA
// waits for another: the last one to take a ticket does the fold.
__global__ void __launch_bounds__(32) finalize_kernel(FinalizeArgs A) {
  static_assert(FIN_CTAS <= 32, "one slice result per lane in the last fold");
  const int lane = threadIdx.x, g = blockIdx.x;
  double* work = A.scal + SCAL_COUNT;  // [FIN_CTAS][6]: totals 0..4, speed bits 5
  unsigned* ticket = reinterpret_cast<unsigned*>(A.scal + SCAL_COUNT + FIN_CTAS * 6);
  const int G = gridDim.x;
  const long long lo = (long long)A.nblk * g / G, hi = (long long)A.nblk * (g + 1) / G;
  double s[5];
  unsigned long long mb;
  fin::fold_slice(A, lo, hi, lane, s, mb);
  if (G > 1) {
    // lane 0 publishes the slice, then takes a ticket
    unsigned t = 0;
    if (lane == 0) {
#pragma unroll
      for (int v = 0; v < 5; ++v) work[g * 6 + v] = s[v];
      work[g * 6 + 5] = __longlong_as_double((long long)mb);
      __threadfence();
      t = atomicAdd(ticket, 1u);
    }
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t != (unsigned)G - 1) return;
    __threadfence();
#pragma unroll
    for (int v = 0; v < 5; ++v) s[v] = lane < G ? __ldcg(work + lane * 6 + v) : 0.0;
    mb = lane < G ? (unsigned long long)__double_as_longlong(__ldcg(work + lane * 6 + 5)) : 0ull;
    fin::fold_warp(s, mb);
  }
  fin::finish(A, s, mb, lane);
}

// Shock detector of the HLLC -> HLL switch (the test: shock_flags.cuh): the
// pass of Runge-Kutta stage 2 everywhere, and of stage 1 on the meshes the
// TMA pass of flags_tma.cu does not take (2D, FP64, rows that are not
// 16-byte multiples, an n below 3).  One CTA covers a TX x TY tile of the (x, y) plane
// and marches along z over a chunk of planes.  Every cell's pressure and
// velocity is recovered once per CTA: the tile's cells of the next plane in
// registers, the current plane with a one-cell ring of x and y neighbours in
// shared memory, the previous plane's (p, v_z) in registers.  Only the ring
// and the two planes that bound a chunk are recovered by more than one CTA.
template <class T, int NDIM, int TX, int TY>
__global__ void __launch_bounds__(TX * TY) shock_flags_kernel(FlagArgs<T> A, int kz) {
  static_assert(NDIM == 2 || NDIM == 3, "the switch runs in 2D and 3D");
  static_assert(2 * (TX + TY) <= TX * TY, "one ring cell per thread at most");
  __shared__ T sp[TY + 2][TX + 2], svx[TY + 2][TX + 2], svy[TY + 2][TX + 2];
  const T gm1 = (T)(A.gamma - 1.0);
  const T dt = A.stage == 2 ? (T)(*A.dt) : T(0);
  const int nx = A.n[0], ny = A.n[1], nz = A.n[2];
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int x = x0 + tx, y = y0 + ty;
  const int z0 = NDIM > 2 ? blockIdx.z * kz : 0;
  const int z1 = NDIM > 2 ? min(z0 + kz, nz) : 1;
  // own column: a mesh cell, or the ghost just past the high x or y edge
  const bool own = x <= nx && y <= ny;
  // ring cell of this thread: left/right columns, then bottom/top rows
  int ri = -2, rj = -2, rs = -1, rx = 0, ry = 0;
  if (threadIdx.x < 2 * TY) {
    const int side = threadIdx.x / TY, row = threadIdx.x % TY;
    ri = side ? x0 + TX : x0 - 1;
    rj = y0 + row;
    rs = 0;
    rx = side ? TX + 1 : 0;
    ry = row + 1;
  } else if (threadIdx.x < 2 * (TX + TY)) {
    const int t = threadIdx.x - 2 * TY, side = t / TX, col = t % TX;
    ri = x0 + col;
    rj = side ? y0 + TY : y0 - 1;
    rs = 1;
    rx = col + 1;
    ry = side ? TY + 1 : 0;
  }
  const bool ring = rs >= 0 && ri <= nx && rj <= ny;
  T pm = T(0), vzm = T(0), pc = T(0), vc[NDIM];
#pragma unroll
  for (int q = 0; q < NDIM; ++q) vc[q] = T(0);
  if (own) {
    if constexpr (NDIM > 2) {
      T vv[NDIM];
      shock::cell_pv<T, NDIM>(A, gm1, dt, x, y, z0 - 1, pm, vv);
      vzm = vv[2];
    }
    shock::cell_pv<T, NDIM>(A, gm1, dt, x, y, z0, pc, vc);
  }
  for (int z = z0; z < z1; ++z) {
    T pn = T(0), vn[NDIM];
#pragma unroll
    for (int q = 0; q < NDIM; ++q) vn[q] = T(0);
    if constexpr (NDIM > 2)
      if (own) shock::cell_pv<T, NDIM>(A, gm1, dt, x, y, z + 1, pn, vn);
    if (ring) {
      T pr, vr[NDIM];
      shock::cell_pv<T, NDIM>(A, gm1, dt, ri, rj, z, pr, vr);
      sp[ry][rx] = pr;
      if (rs == 0) svx[ry][rx] = vr[0];
      else svy[ry][rx] = vr[1];
    }
    sp[ty + 1][tx + 1] = pc;
    svx[ty + 1][tx + 1] = vc[0];
    svy[ty + 1][tx + 1] = vc[1];
    __syncthreads();
    if (x < nx && y < ny) {
      unsigned bits = 0;
      if (shock::jump(sp[ty + 1][tx], svx[ty + 1][tx], sp[ty + 1][tx + 2], svx[ty + 1][tx + 2])) bits |= 1u;
      if (shock::jump(sp[ty][tx + 1], svy[ty][tx + 1], sp[ty + 2][tx + 1], svy[ty + 2][tx + 1])) bits |= 2u;
      if constexpr (NDIM > 2)
        if (shock::jump(pm, vzm, pn, vn[2])) bits |= 4u;
      A.flags[((size_t)z * ny + y) * nx + x] = (unsigned char)bits;
    }
    __syncthreads();
    if constexpr (NDIM > 2) {
      pm = pc;
      vzm = vc[2];
      pc = pn;
#pragma unroll
      for (int q = 0; q < NDIM; ++q) vc[q] = vn[q];
    }
  }
}

// ------------------------------------------------------------------ launchers

static int grid_for(size_t count, int block, int max_blocks) {
  size_t g = (count + block - 1) / block;
  if (g < 1) g = 1;
  return (int)(g > (size_t)max_blocks ? max_blocks : g);
}

template <class T>
cudaError_t launch_init_from_primitive(int ndim, size_t ncell, double gamma, const double* rho, const double* vel,
                                       const double* p, T* U, cudaStream_t s) {
  init_from_primitive_kernel<T><<<grid_for(ncell, 256, 4096), 256, 0, s>>>(ndim, ncell, gamma, rho, vel, p, U);
  return cudaGetLastError();
}

template <class Tin, class Tout>
cudaError_t launch_convert(size_t count, const Tin* in, Tout* out, cudaStream_t s) {
  convert_kernel<Tin, Tout><<<grid_for(count, 256, 4096), 256, 0, s>>>(count, in, out);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_speed(int ndim, const ReduceArgs<T>& A, cudaStream_t s) {
  switch (ndim) {
    case 1: speed_kernel<T, 1><<<A.nblk, 256, 0, s>>>(A); break;
    case 2: speed_kernel<T, 2><<<A.nblk, 256, 0, s>>>(A); break;
    default: speed_kernel<T, 3><<<A.nblk, 256, 0, s>>>(A); break;
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_totals(int ndim, const ReduceArgs<T>& A, cudaStream_t s) {
  switch (ndim) {
    case 1: totals_kernel<T, 1><<<A.nblk, 256, 0, s>>>(A); break;
    case 2: totals_kernel<T, 2><<<A.nblk, 256, 0, s>>>(A); break;
    default: totals_kernel<T, 3><<<A.nblk, 256, 0, s>>>(A); break;
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_shock_flags(int ndim, const FlagArgs<T>& A, cudaStream_t s) {
  if (ndim == 2) {
    constexpr int TX = 32, TY = 8;
    const long long bx = (A.n[0] + TX - 1) / TX, by = (A.n[1] + TY - 1) / TY;
    if (by > 65535) return cudaErrorInvalidConfiguration;
    shock_flags_kernel<T, 2, TX, TY><<<dim3((unsigned)bx, (unsigned)by, 1), TX * TY, 0, s>>>(A, 1);
    return cudaGetLastError();
  }
  if (ndim != 3) return cudaErrorInvalidValue;  // 1D runs plain HLLC
  // 32 x 4 tiles (many small CTAs keep the most loads in flight); z chunks
  // for about 32 CTAs per SM
  constexpr int TX = 32, TY = 4;
  const long long bx = (A.n[0] + TX - 1) / TX, by = (A.n[1] + TY - 1) / TY;
  if (by > 65535) return cudaErrorInvalidConfiguration;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long target = 32LL * (sms > 0 ? sms : 1);
  const int nz = A.n[2];
  long long chunks = (target + bx * by - 1) / (bx * by);
  chunks = chunks < 1 ? 1 : (chunks > nz ? nz : (chunks > 65535 ? 65535 : chunks));
  const int kz = (int)((nz + chunks - 1) / chunks);
  chunks = (nz + kz - 1) / kz;
  shock_flags_kernel<T, 3, TX, TY><<<dim3((unsigned)bx, (unsigned)by, (unsigned)chunks), TX * TY, 0, s>>>(A, kz);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeArgs& A, cudaStream_t s) {
  finalize_kernel<<<A.nblk <= 512 ? 1 : FIN_CTAS, 32, 0, s>>>(A);
  return cudaGetLastError();
}

template cudaError_t launch_init_from_primitive<float>(int, size_t, double, const double*, const double*,
                                                       const double*, float*, cudaStream_t);
template cudaError_t launch_init_from_primitive<double>(int, size_t, double, const double*, const double*,
                                                        const double*, double*, cudaStream_t);
template cudaError_t launch_convert<float, double>(size_t, const float*, double*, cudaStream_t);
template cudaError_t launch_convert<double, float>(size_t, const double*, float*, cudaStream_t);
template cudaError_t launch_speed<float>(int, const ReduceArgs<float>&, cudaStream_t);
template cudaError_t launch_speed<double>(int, const ReduceArgs<double>&, cudaStream_t);
template cudaError_t launch_totals<float>(int, const ReduceArgs<float>&, cudaStream_t);
template cudaError_t launch_totals<double>(int, const ReduceArgs<double>&, cudaStream_t);
template cudaError_t launch_init_from_primitive<dw>(int, size_t, double, const double*, const double*, const double*,
                                                    dw*, cudaStream_t);
template cudaError_t launch_convert<double, dw>(size_t, const double*, dw*, cudaStream_t);
template cudaError_t launch_convert<float, dw>(size_t, const float*, dw*, cudaStream_t);
template cudaError_t launch_convert<dw, double>(size_t, const dw*, double*, cudaStream_t);
template cudaError_t launch_convert<dw, float>(size_t, const dw*, float*, cudaStream_t);
template cudaError_t launch_speed<dw>(int, const ReduceArgs<dw>&, cudaStream_t);
template cudaError_t launch_totals<dw>(int, const ReduceArgs<dw>&, cudaStream_t);
template cudaError_t launch_shock_flags<float>(int, const FlagArgs<float>&, cudaStream_t);
template cudaError_t launch_shock_flags<double>(int, const FlagArgs<double>&, cudaStream_t);

}  // namespace gh
