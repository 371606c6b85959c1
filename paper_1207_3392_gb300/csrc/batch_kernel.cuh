// batch_kernel.cuh -- persistent stage kernel over many independent 1D and 2D
// problems of uneven size.  Each CTA repeatedly takes the next (problem, tile,
// chunk) item from a global counter (items are sorted largest first) and runs
// the same tile body as the single-grid stage kernel on it, with that
// problem's mesh, boundaries, gamma and time step.
#pragma once

#include "stage_kernel.cuh"

namespace gh {

// One problem of the batch (device copy).
template <class T>
struct BatchProblem {
  int ndim;
  int n[2];
  int bc_lo[2], bc_hi[2];
  T gamma, gm1;
  size_t off;       // element offset of the problem's U in the state arenas
  size_t goff[2];   // offset of its axis-q tables in the geometry arenas (n[q] + 4 entries)
  size_t woff[2];   // offset of its axis-q widths in the FP64 width arena (n[q] entries)
};

struct BatchItem {
  int prob, tx, chunk, pad;
};

template <class T>
struct BatchArgs {
  const BatchProblem<T>* probs;
  const BatchItem* items;
  int nitems;
  unsigned* counter;        // this launch's work counter (zeroed before the launch)
  const Geo<T>* geo;        // geometry arena
  const T* iw;              // inverse-width arena
  const double* wd;         // width arena
  const T* un;              // U^n arena
  const T* k1;              // stage-1 K arena
  T* out;                   // stage 1: K arena; stage 2: U^{n+1} arena
  const double* dt;         // per-problem dt
  unsigned long long* speed;  // per-problem max CFL speed (FP64 bit pattern; stage 1)
  unsigned* status;         // per-problem status
  int kchunk;               // planes (rows) per 2D item
};

template <class T, int SOLVER, int STAGE, int TX>
struct BatchKernel {
  using K1 = StageKernel<1, T, SOLVER, STAGE, TX, 1>;
  using K2 = StageKernel<2, T, SOLVER, STAGE, TX, 1>;
  static_assert(K1::OWN == K2::OWN, "1D and 2D items share the x tiling");
  static constexpr size_t SMEM = sizeof(typename K1::Smem) > sizeof(typename K2::Smem) ? sizeof(typename K1::Smem)
                                                                                          : sizeof(typename K2::Smem);

  template <int NDIM>
  static __device__ __forceinline__ StageArgs<T> args_for(const BatchArgs<T>& B, const BatchProblem<T>& P, int p) {
    StageArgs<T> A;
    A.n[0] = P.n[0];
    A.n[1] = NDIM == 2 ? P.n[1] : 1;
    A.n[2] = 1;
    for (int q = 0; q < 2; ++q) {
      A.bc_lo[q] = P.bc_lo[q];
      A.bc_hi[q] = P.bc_hi[q];
      A.geo[q] = B.geo + P.goff[q];
      A.iw[q] = B.iw + P.goff[q];
      A.wd[q] = B.wd + P.woff[q];
    }
    A.bc_lo[2] = A.bc_hi[2] = BC_OUTFLOW;
    A.geo[2] = nullptr;
    A.iw[2] = nullptr;
    A.wd[2] = nullptr;
    for (int q = 0; q < 3; ++q) {
      A.wdh[q] = nullptr;
      A.wdl[q] = nullptr;
    }
    A.gamma = P.gamma;
    A.gm1 = P.gm1;
    A.un = B.un + P.off;
    A.k1 = B.k1 + P.off;
    A.out = B.out + P.off;
    A.dt = B.dt + p;
    A.kchunk = B.kchunk;
    A.part_speed = nullptr;
    A.part_tot = nullptr;
    A.status = B.status + p;
    A.want_totals = 0;
    A.has_source = 0;
    A.flags = nullptr;
    A.grad_phi[0] = A.grad_phi[1] = A.grad_phi[2] = T(0);
    return A;
  }

  static __device__ void run(const BatchArgs<T>& B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    __shared__ double s_red[TX / 32];
    const int tid = threadIdx.x;
    for (;;) {
      if (tid == 0) s_item = (int)atomicAdd(B.counter, 1u);
      __syncthreads();
      const int it = s_item;
      __syncthreads();  // everyone has read s_item before thread 0 may overwrite it
      if (it >= B.nitems) break;
      const BatchItem w = B.items[it];
      const BatchProblem<T> P = B.probs[w.prob];
      double speed_max = 0.0;
      bool bad = false;
      if (P.ndim == 1) {
        double tot[3] = {0, 0, 0};
        const StageArgs<T> A = args_for<1>(B, P, w.prob);
        K1::tile(A, *reinterpret_cast<typename K1::Smem*>(smem_raw), w.tx, 0, 0, speed_max, tot, bad);
      } else {
        double tot[4] = {0, 0, 0, 0};
        const StageArgs<T> A = args_for<2>(B, P, w.prob);
        K2::tile(A, *reinterpret_cast<typename K2::Smem*>(smem_raw), w.tx, 0, w.chunk, speed_max, tot, bad);
      }
      if (bad) atomicOr(B.status + w.prob, STATUS_NONPHYS);
      if (STAGE == 1) {
        const double m = warp_max(speed_max);
        if ((tid & 31) == 0) s_red[tid >> 5] = m;
        __syncthreads();
        if (tid == 0) {
          double acc = s_red[0];
          for (int i = 1; i < TX / 32; ++i) acc = fmax(acc, s_red[i]);
          // positive doubles order like their bit patterns
          atomicMax(B.speed + w.prob, (unsigned long long)__double_as_longlong(acc));
        }
      }
      __syncthreads();  // shared memory is reused by the next item
    }
  }
};

// FP32: 64 registers, so that 2,048 threads (8 CTAs of 128) stay resident;
// the FP64 and double-word bodies would spill at that limit.
template <class T, int TX>
constexpr int batch_min_blocks() { return std::is_same<T, float>::value ? 1024 / TX : 1; }

template <class T, int SOLVER, int STAGE, int TX>
__global__ void __launch_bounds__(TX, (batch_min_blocks<T, TX>())) hydro_batch_kernel(const BatchArgs<T> B) {
  BatchKernel<T, SOLVER, STAGE, TX>::run(B);
}

// Per problem: dt = cfl / speed (or fixed), clamp at t_end, advance t, reset
// the speed slot for the next stage 1.
__global__ void batch_finalize_kernel(int nprob, int mode, double cfl, double fixed_dt, double t_end,
                                      unsigned long long* speed, double* dt, double* t, unsigned* status);

}  // namespace gh
