// aux_kernels.cu -- small kernels around the stage kernels: initial state
// from primitives, precision conversion, the standalone CFL and totals
// reductions, and the single-CTA finalisation of dt and totals.
#include "aux_kernels.h"
#include "finalize.cuh"
#include "hydro_device.cuh"

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

// Shock detector of the HLLC -> HLL switch (Sec. 3.2 describes the switch, not
// the detector): cell c lies on a shock moving along axis r when, across its
// two neighbours along r (boundary-mapped like the stage kernel's ghosts), the
// flow is compressive, v_r(+) - v_r(-) < 0, and the pressure jumps by more
// than half the smaller pressure.  Bit r of flags[c] records it.
template <class T, int NDIM>
__global__ void shock_flags_kernel(FlagArgs<T> A) {
  constexpr int NV = NDIM + 2;
  const T gm1 = (T)(A.gamma - 1.0);
  const T dt = A.stage == 2 ? (T)(*A.dt) : T(0);
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < A.ncell; c += (size_t)gridDim.x * blockDim.x) {
    int idx[3] = {0, 0, 0};
    size_t r_ = c;
#pragma unroll
    for (int q = 0; q < NDIM; ++q) {
      idx[q] = (int)(r_ % A.n[q]);
      r_ /= A.n[q];
    }
    unsigned bits = 0;
#pragma unroll
    for (int r = 0; r < NDIM; ++r) {
      T p[2], v[2];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        int j[3] = {idx[0], idx[1], idx[2]};
        bool flip = false;
        j[r] = bc_map(idx[r] + (side ? 1 : -1), A.n[r], A.bc_lo[r], A.bc_hi[r], flip);
        const size_t cc = ((size_t)j[2] * A.n[1] + j[1]) * A.n[0] + j[0];
        T u[NV], w[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          T x = A.un[k * A.ncell + cc];
          if (A.stage == 2) x = fma(dt, A.k1[k * A.ncell + cc], x);
          u[k] = x;
        }
        if (flip) u[1 + r] = -u[1 + r];
        recover<NDIM>(u, w);
        p[side] = gm1 * w[NV - 1];
        v[side] = w[1 + r];
      }
      if (v[1] - v[0] < T(0) && fabs(p[1] - p[0]) > T(0.5) * fmin(p[0], p[1])) bits |= 1u << r;
    }
    A.flags[c] = (unsigned char)bits;
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
  const int nb = grid_for(A.ncell, 256, 4096);
  switch (ndim) {
    case 1: shock_flags_kernel<T, 1><<<nb, 256, 0, s>>>(A); break;
    case 2: shock_flags_kernel<T, 2><<<nb, 256, 0, s>>>(A); break;
    default: shock_flags_kernel<T, 3><<<nb, 256, 0, s>>>(A); break;
  }
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
