// learned_advance.cu -- every step of a corrected 2D advance in one kernel
// launch.
//
// A 256^2 mesh holds 1 MB of state, so the per-phase path (CFL speed,
// finalize, and per stage the faces, the network, the FCT ratios, the
// corrected update and four fallback passes: 18 launches a step) spends most
// of its time launching and draining kernels.  Here one cooperative launch of
// a persistent grid runs all phases, with a bounded grid barrier
// (grid_sync.cuh) wherever a phase reads what another CTA wrote:
//   CFL speed of U^n, one partial per CTA                        barrier
//   every CTA reads the largest speed (one atomic maximum per CTA; a
//   maximum does not depend on the order) and takes the same dt; CTA 0
//   stores dt and t
//   per stage:
//     plain flux and features of a tile of 256 faces; each warp runs the
//     network on its own 32 faces (BF16 weights in shared memory, loaded
//     once per launch)                                           barrier
//     FCT ratios of every cell (when limiting)                   barrier
//     corrected update of every cell                             barrier
//     only if a cell failed: the three widening passes and, if failures
//     remain, the all-plain pass                                 barrier each
// The per-face and per-cell arithmetic is that of the per-phase kernels
// (learned_step.cuh, the same network code), so states, dt, time and
// fallback counts are bitwise those of the per-phase path.  Arrays written
// inside the launch are read through L2 (COH = true).
//
// The sync words: [0..1] the grid barrier, [2..5] the all-plain flags, [8..11]
// two 64-bit speed slots (used by alternate steps).  The all-plain flags come
// as one pair per stage: a stage clears the other
// stage's pair after its faces barrier, when every CTA has read that pair and
// before any CTA can write it again.
#include "finalize.cuh"
#include "grid_sync.cuh"
#include "learned_internal.h"
#include "learned_step.cuh"

namespace gh {

namespace {

constexpr int LFA_WARPS = LF_ADVANCE_THREADS / 32;
constexpr int LFA_PASSES = 3;  // widening passes, as in the per-phase path

template <int SOLVER>
__global__ void __launch_bounds__(LF_ADVANCE_THREADS, 2) lf_advance_kernel(LfAdvanceArgs P) {
  __shared__ mlp::InferWeights W;
  __shared__ __align__(16) __nv_bfloat16 xs[LF_ADVANCE_THREADS][mlp::KIN];  // features of the tile's faces
  __shared__ double red[LFA_WARPS];
  const Mesh2& M = P.M;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, bx = blockIdx.x;
  const unsigned nb = gridDim.x;
  const long long ncell = (long long)M.nx * M.ny;
  const long long nxf = (long long)(M.nx + 1) * M.ny, nf = nxf + (long long)M.nx * (M.ny + 1);
  const long long first = (long long)bx * LF_ADVANCE_THREADS, stride = (long long)nb * LF_ADVANCE_THREADS;
  const bool corr = P.W != nullptr;
  unsigned* bar = P.sync;
  unsigned long long* speed_slot = reinterpret_cast<unsigned long long*>(P.sync + 8);  // one per step parity
  if (corr) mlp::copy_weights(W, P.W);
  unsigned my_gen = 0;
  bool failed = false;
  if (tid == 0) my_gen = atomicAdd(bar + 1, 0u);  // the generation at launch (no CTA can move it yet)
  // the time, kept by every CTA (CTA 0 also stores it): read before any CTA
  // of this launch writes it
  double t = __ldcg(P.Fa.scal + SCAL_T);
  int cur = 0;
  for (int s = 0; s < P.nsteps; ++s) {
    const float* un = P.U[cur];
    {  // this CTA's partial of the CFL speed of U^n, as the speed kernel's
      ReduceArgs<float> R = P.R;
      R.U = un;
      double best = 0.0;
      bool bad = false;
      for (long long c = first + tid; c < ncell; c += stride)
        best = fmax(best, (double)fin::cell_speed<float, 2, true>(R, (size_t)c, bad));
      if (bad) atomicOr(P.status, STATUS_NONPHYS);
      best = warp_max(best);
      if (lane == 0) red[warp] = best;
      __syncthreads();
      if (tid == 0) {
        double acc = red[0];
        for (int i = 1; i < LFA_WARPS; ++i) acc = fmax(acc, red[i]);
        // speeds are >= 0, so their bit patterns order like the values
        atomicMax(speed_slot + (s & 1), (unsigned long long)__double_as_longlong(acc));
      }
    }
    if (!grid_barrier(bar, bar + 1, nb, my_gen, P.status, failed)) return;
    if (warp == 0) {
      // the largest speed of the step; the other slot is free again (its
      // last reads were before this barrier, its next writes come after the
      // stage barriers)
      const unsigned long long mb = __ldcg(speed_slot + (s & 1));
      if (bx == 0) {
        const double zeros[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        fin::finish(P.Fa, zeros, mb, lane);
        if (lane == 0) speed_slot[(s + 1) & 1] = 0ull;
      }
      if (lane == 0) P.dts[bx] = fin::step_dt(P.Fa, mb, t);
    }
    __syncthreads();
    const double dtd = __ldcg(P.dts + bx);
    t += dtd;
    const float dt = (float)dtd;
#pragma unroll 1
    for (int stage = 1; stage <= 2; ++stage) {
      const float* kin = stage == 2 ? P.K : nullptr;
      // plain fluxes, and features and network outputs, of every face
      for (long long base = first; base < nf; base += stride) {
        const long long f = base + tid;
        if (f < nf) lf_face<SOLVER, true>(M, un, kin, dt, f, nxf, nf, P.F, corr ? xs[tid] : nullptr, P.scale);
        if (corr) {
          __syncwarp();
#pragma unroll 1
          for (int h = 0; h < 2; ++h) {
            const long long s0 = base + 32 * warp + 16 * h, left = nf - s0;
            if (left <= 0) break;
            const int rows = left < 16 ? (int)left : 16;
            mlp::Forward Fw;
            mlp::load_x(Fw, &xs[32 * warp + 16 * h][0], rows);
            mlp::forward(Fw, W);
            const int g = lane >> 2, q = lane & 3;
            if (q < 2) {
              if (g < rows) {
                P.dY[(s0 + g) * 4 + 2 * q] = Fw.y[0];
                P.dY[(s0 + g) * 4 + 2 * q + 1] = Fw.y[1];
              }
              if (g + 8 < rows) {
                P.dY[(s0 + g + 8) * 4 + 2 * q] = Fw.y[2];
                P.dY[(s0 + g + 8) * 4 + 2 * q + 1] = Fw.y[3];
              }
            }
          }
          __syncwarp();  // the rows are read before the next tile's features
        }
      }
      if (!grid_barrier(bar, bar + 1, nb, my_gen, P.status, failed)) return;
      unsigned* ap = P.sync + 2 * stage;  // this stage's all-plain flags
      if (bx == 0 && tid == 0) {
        unsigned* other = P.sync + 2 * (3 - stage);
        other[0] = 0u;
        other[1] = 0u;
      }
      UpdateArgs A;
      A.M = M;
      A.un = un;
      A.k1 = P.K;
      A.dtp = nullptr;
      A.F = P.F;
      A.dY = corr ? P.dY : nullptr;
      A.scale = P.scale;
      A.out = stage == 1 ? P.K : P.U[cur ^ 1];
      A.flag = P.flag[1];
      A.flag_out = P.flag[0];
      A.nfallback = P.nfallback;
      A.status = P.status;
      A.stage = stage;
      A.fixup = 0;
      A.last = 0;
      A.all_plain = ap;
      A.ylim = P.ylim;
      A.R = nullptr;
      if (corr && P.fct) {
        for (long long c = first + tid; c < ncell; c += stride) lf_fct_cell<true>(A, c, dt, P.Rfct);
        if (!grid_barrier(bar, bar + 1, nb, my_gen, P.status, failed)) return;
        A.R = P.Rfct;
      }
      // the corrected pass, then only when some cell failed the widening
      // passes and, if failures remain, the all-plain pass (one decision per
      // CTA, the same in every CTA: the flags are final once the barrier is
      // passed); one call site, so the update is inlined once
#pragma unroll 1
      for (int pass = 0;;) {
        for (long long c = first + tid; c < ncell; c += stride) lf_update_cell<true>(A, c, dt);
        if (!grid_barrier(bar, bar + 1, nb, my_gen, P.status, failed)) return;
        if (!corr || pass < 0) break;
        if (pass == 0 && !__syncthreads_or(tid == 0 && __ldcg(ap + 1) != 0u)) break;
        if (pass == LFA_PASSES) {
          if (!__syncthreads_or(tid == 0 && __ldcg(ap) != 0u)) break;
          pass = -1;
        } else {
          ++pass;
          A.flag = P.flag[(pass + 1) & 1];
          A.flag_out = P.flag[pass & 1];
          A.last = pass == LFA_PASSES;
        }
        A.fixup = pass;
      }
    }
    cur ^= 1;
  }
}

const void* advance_fn(int solver) {
  return solver == SOLVER_HLL ? reinterpret_cast<const void*>(&lf_advance_kernel<SOLVER_HLL>)
                              : reinterpret_cast<const void*>(&lf_advance_kernel<SOLVER_HLLC>);
}

}  // namespace

int learned_advance_max_grid(int solver) {
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, advance_fn(solver), LF_ADVANCE_THREADS, 0) != cudaSuccess)
    return 0;
  return per_sm * sms;
}

cudaError_t launch_learned_advance(const LfAdvanceArgs& P, int solver, int grid, cudaStream_t st) {
  LfAdvanceArgs a = P;
  void* args[] = {&a};
  // cooperative: the CTAs wait on one another, so all must be resident
  return cudaLaunchCooperativeKernel(advance_fn(solver), dim3(grid), dim3(LF_ADVANCE_THREADS), args, 0, st);
}

}  // namespace gh
