// kern_1d_advance.cu -- a whole multi-step advance of a small 1D mesh in one
// kernel launch.
//
// A 1D mesh of a few hundred cells fills a handful of CTAs, so the three
// launches of an RK2 step (stage 1, finalize, stage 2) cost more than their
// work.  Here one cooperative launch of one CTA per tile runs every step of
// the call:
//   stage 1 of the CTA's tile, its reduction partial written as in the
//   multi-launch path                                          grid barrier
//   every CTA folds all partials in the fixed order of the finalize kernel
//   (so every CTA computes bitwise the same dt); CTA 0 stores dt, t and the
//   totals; stage 2 of the tile with that dt                   grid barrier
//   the buffers swap.
// The tile arithmetic and the fold are those of the multi-launch path, so the
// states, dt and time are bitwise the same (the totals are summed over tiles
// of another width, so they agree to rounding).  The state arrays are
// written and read within the launch, so the tiles read them through L2
// (StageKernel<..., COH = true>).  Spreading the tiles over SMs matters on
// this GPU even for 256 cells: an SM retires about two FP64 operations per
// clock.
//
// The CTAs are co-resident (cooperative launch) and meet at the bounded grid
// barrier of grid_sync.cuh: a CTA that gives up waiting sets STATUS_TIMEOUT,
// and every CTA leaves at its next barrier.
#include "finalize.cuh"
#include "grid_sync.cuh"
#include "registry.h"
#include "stage_kernel.cuh"

namespace gh {

template <class T, int SOLVER, int TX>
__global__ void __launch_bounds__(TX)
    hydro_1d_advance_kernel(StageArgs<T> A, FinalizeArgs F, int nsteps, T* ua, T* ub, unsigned* bar, double* dts) {
  using K1 = StageKernel<1, T, SOLVER, 1, TX, 1, false, true>;
  using K2 = StageKernel<1, T, SOLVER, 2, TX, 1, false, true>;
  static_assert(sizeof(typename K1::Smem) == sizeof(typename K2::Smem), "one shared layout for both stages");
  extern __shared__ __align__(16) unsigned char smem_1d[];
  auto& S1 = *reinterpret_cast<typename K1::Smem*>(smem_1d);
  auto& S2 = *reinterpret_cast<typename K2::Smem*>(smem_1d);
  constexpr int NV = 3;
  const int bx = blockIdx.x;
  const unsigned nb = gridDim.x;
  unsigned my_gen = 0;
  bool failed = false;
  if (threadIdx.x == 0) my_gen = atomicAdd(bar + 1, 0u);  // the generation at launch (no CTA can move it yet)
  // the time, kept by every CTA (CTA 0 also stores it): read before any CTA
  // of this launch writes it
  double t = __ldcg(F.scal + SCAL_T);
  T* cur = ua;
  T* nxt = ub;
  for (int s = 0; s < nsteps; ++s) {
    StageArgs<T> a1 = A;
    a1.un = cur;
    a1.out = const_cast<T*>(A.k1);
    {
      double speed = 0.0, tot[NV] = {0.0, 0.0, 0.0};
      bool bad = false;
      K1::tile(a1, S1, bx, 0, 0, speed, tot, bad);
      if (bad) atomicOr(A.status, STATUS_NONPHYS);
      K1::write_partials(a1, S1, bx, speed, tot);
    }
    if (!grid_barrier(bar, bar + 1, nb, my_gen, A.status, failed)) return;
    // every CTA folds the partials the same way and takes the same dt; CTA 0
    // also stores dt, t and the totals in the scalar block
    if (threadIdx.x < 32) {
      double sums[5];
      unsigned long long mb;
      fin::fold_slice(F, 0, nb, threadIdx.x, sums, mb);
      if (bx == 0) fin::finish(F, sums, mb, threadIdx.x);
      if (threadIdx.x == 0) dts[bx] = fin::step_dt(F, mb, t);
    }
    __syncthreads();
    t += dts[bx];
    StageArgs<T> a2 = A;
    a2.un = cur;
    a2.out = nxt;
    a2.dt = dts + bx;
    {
      double speed = 0.0, tot[NV] = {0.0, 0.0, 0.0};
      bool bad = false;
      K2::tile(a2, S2, bx, 0, 0, speed, tot, bad);
      if (bad) atomicOr(A.status, STATUS_NONPHYS);
    }
    if (!grid_barrier(bar, bar + 1, nb, my_gen, A.status, failed)) return;
    T* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
}

namespace {

template <class T, int TX>
const void* pick_1d_advance(int solver) {
  if (solver == SOLVER_HLL) return reinterpret_cast<const void*>(&hydro_1d_advance_kernel<T, SOLVER_HLL, TX>);
  if (solver == SOLVER_HLLC) return reinterpret_cast<const void*>(&hydro_1d_advance_kernel<T, SOLVER_HLLC, TX>);
  return nullptr;
}

}  // namespace

// The one-launch 1D advance for (precision, solver) with tx threads per CTA
// (one tile of tx - 1 cells each); smem receives the dynamic shared memory
// per CTA.  nullptr if not compiled.
const void* advance_1d_kernel(bool fp64, int solver, int tx, size_t* smem) {
  if (tx == 32) {
    *smem = fp64 ? sizeof(StageKernel<1, double, SOLVER_HLLC, 1, 32, 1, false, true>::Smem)
                 : sizeof(StageKernel<1, float, SOLVER_HLLC, 1, 32, 1, false, true>::Smem);
    return fp64 ? pick_1d_advance<double, 32>(solver) : pick_1d_advance<float, 32>(solver);
  }
  if (tx == 256) {
    *smem = fp64 ? sizeof(StageKernel<1, double, SOLVER_HLLC, 1, 256, 1, false, true>::Smem)
                 : sizeof(StageKernel<1, float, SOLVER_HLLC, 1, 256, 1, false, true>::Smem);
    return fp64 ? pick_1d_advance<double, 256>(solver) : pick_1d_advance<float, 256>(solver);
  }
  return nullptr;
}

}  // namespace gh
