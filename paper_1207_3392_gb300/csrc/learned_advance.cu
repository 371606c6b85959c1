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
//     plain flux and features of a tile of one face per thread, and the
//     network on them (BF16 weights in shared memory, loaded once per
//     launch): each warp on its own 32 faces with mma.sync (CTAs of 128
//     threads, 4 per SM), or, with the tcgen05 engine, each group of four
//     warps on its 128 faces (accumulators in TMEM, mlp_tc.cuh; CTAs of 512
//     threads, 1 per SM)                                        barrier
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
#include "mlp_tc.cuh"

namespace gh {

namespace {

constexpr int LFA_PASSES = 3;  // widening passes, as in the per-phase path

// The CTA shape and shared memory per network engine.  tcgen05: one group of
// four warps per 128 faces of a tile (the network's MMA tile).  Dynamic
// shared memory: mma.sync: the BF16 weight image and one feature row per
// thread; tcgen05: the weights as B operands and each group's operand tile.
// It is sized so that at most CTAS CTAs fit on an SM (with tcgen05 their TMEM
// columns then fill at most the SM's 512: another CTA could not allocate
// while the others wait for it at a grid barrier).
template <bool TC>
struct Lfa {
  static constexpr int CTAS = lf_advance_ctas_per_sm(TC);
  static constexpr int THREADS = lf_advance_threads(TC);
  static constexpr int WARPS = THREADS / 32;
  static constexpr int GROUPS = THREADS / mlptc::M;
  static_assert(GROUPS * mlptc::M == THREADS, "a tile is whole network tiles");
  struct SmemSync {
    mlp::InferWeights W;
    __align__(16) __nv_bfloat16 xs[THREADS][mlp::KIN];
  };
  static constexpr size_t SMEM_MIN = 228 * 1024 / (CTAS + 1) + 1024;
  static constexpr size_t NEED = TC ? sizeof(mlptc::Weights) + GROUPS * sizeof(mlptc::Tile) : sizeof(SmemSync);
  static constexpr size_t SMEM = ((NEED > SMEM_MIN ? NEED : SMEM_MIN) + 1023) / 1024 * 1024;
  static_assert((CTAS + 1) * SMEM > 228 * 1024, "at most CTAS CTAs per SM");
  static_assert(SMEM <= 227 * 1024, "fits one CTA's shared memory");
  static constexpr uint32_t TMEM_COLS = GROUPS * mlptc::TMEM_COLS;
  static_assert(!TC || TMEM_COLS * CTAS <= 512, "the resident CTAs' TMEM fits the SM");
};

// Every step of the launch; returns early (on every thread of the CTA
// together) when a grid barrier gives up.  TC: the network on tcgen05 (W,
// tiles, mbar, tmem), else on mma.sync (S).
template <int SOLVER, bool TC>
__device__ __forceinline__ void lf_advance_body(const LfAdvanceArgs& P, typename Lfa<TC>::SmemSync& S,
                                                const mlptc::Weights& W, mlptc::Tile* tiles,
                                                unsigned long long* mbar, uint32_t tmem, double* red) {
  constexpr int LF_ADVANCE_THREADS = Lfa<TC>::THREADS;
  constexpr int LFA_WARPS = Lfa<TC>::WARPS;
  const Mesh2& M = P.M;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, bx = blockIdx.x;
  const int grp = tid / mlptc::M, row = tid % mlptc::M;  // network group and sample row
  const unsigned nb = gridDim.x;
  const long long ncell = (long long)M.nx * M.ny;
  const long long nxf = (long long)(M.nx + 1) * M.ny, nf = nxf + (long long)M.nx * (M.ny + 1);
  const long long first = (long long)bx * LF_ADVANCE_THREADS, stride = (long long)nb * LF_ADVANCE_THREADS;
  const bool corr = P.W != nullptr;
  unsigned* bar = P.sync;
  unsigned long long* speed_slot = reinterpret_cast<unsigned long long*>(P.sync + 8);  // one per step parity
  // this thread's feature row: in its group's operand tile (tcgen05,
  // core-matrix layout: 16-byte chunks 8 uint4 apart), or a plain row
  __nv_bfloat16* xrow = TC ? tiles[grp].x + mlptc::core_idx(row, 0, mlp::KIN) : S.xs[tid];
  constexpr int XSTRIDE = TC ? 8 : 1;
  unsigned phase = 0;    // of the group's mbarrier
  bool mlp_ok = true;    // the group's tensor-core waits have all completed
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
        if (f < nf) {
          lf_face<SOLVER, true>(M, un, kin, dt, f, nxf, nf, P.F, corr ? xrow : nullptr, P.scale, XSTRIDE);
        } else if (corr && TC) {
#pragma unroll
          for (int c = 0; c < mlp::KIN / 8; ++c)
            *reinterpret_cast<uint4*>(xrow + 8 * XSTRIDE * c) = make_uint4(0, 0, 0, 0);
        }
        if (corr && TC) {
          // the group's 128 faces through the network on the tensor cores
          float y[4] = {NAN, NAN, NAN, NAN};
          if (mlp_ok) {
            mlp_ok = mlptc::forward_tile(W, tiles[grp], mbar + grp, phase, tmem + (uint32_t)(grp * mlptc::TMEM_COLS),
                                         1 + grp, row, y);
            if (!mlp_ok) {
              y[0] = y[1] = y[2] = y[3] = NAN;
              if (row == 0) atomicOr(P.status, STATUS_TIMEOUT);
            }
          }
          if (f < nf) *reinterpret_cast<float4*>(P.dY + 4 * f) = make_float4(y[0], y[1], y[2], y[3]);
        } else if (corr) {
          // each warp runs the network on its own 32 faces (rows past nf
          // read as zero), in two mma.sync tiles of 16
          __syncwarp();
#pragma unroll 1
          for (int h = 0; h < 2; ++h) {
            const long long s0 = base + 32 * warp + 16 * h, left = nf - s0;
            if (left <= 0) break;
            const int rows = left < 16 ? (int)left : 16;
            mlp::Forward Fw;
            mlp::load_x(Fw, &S.xs[32 * warp + 16 * h][0], rows);
            mlp::forward(Fw, S.W);
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

template <int SOLVER, bool TC>
__global__ void __launch_bounds__(Lfa<TC>::THREADS, Lfa<TC>::CTAS) lf_advance_kernel(LfAdvanceArgs P) {
  using L = Lfa<TC>;
  extern __shared__ __align__(128) unsigned char lfa_smem[];
  auto& S = *reinterpret_cast<typename L::SmemSync*>(lfa_smem);
  auto& W = *reinterpret_cast<mlptc::Weights*>(lfa_smem);
  auto* tiles = reinterpret_cast<mlptc::Tile*>(lfa_smem + sizeof(mlptc::Weights));
  __shared__ unsigned long long mbar[L::GROUPS];
  __shared__ uint32_t tmem_slot;
  __shared__ double red[L::WARPS];
  const bool corr = P.W != nullptr;
  if (corr && TC) {
    mlptc::load_weights(W, P.W);
    if (threadIdx.x < L::GROUPS) tma::mbar_init(mbar + threadIdx.x, 1);
    tma::fence_mbar_init();
    if (threadIdx.x < 32) mlptc::tmem_alloc(&tmem_slot, L::TMEM_COLS);
    mlptc::fence_before();
  } else if (corr) {
    mlp::copy_weights(S.W, P.W);
  }
  __syncthreads();
  if (TC) mlptc::fence_after();
  lf_advance_body<SOLVER, TC>(P, S, W, tiles, mbar, corr && TC ? tmem_slot : 0u, red);
  if (corr && TC) {  // no MMA is in flight here: every network tile waited for its own
    mlptc::fence_before();
    __syncthreads();
    mlptc::fence_after();
    if (threadIdx.x < 32) mlptc::tmem_dealloc(tmem_slot, L::TMEM_COLS);
  }
}

template <bool TC>
const void* advance_fn_t(int solver) {
  return solver == SOLVER_HLL ? reinterpret_cast<const void*>(&lf_advance_kernel<SOLVER_HLL, TC>)
                              : reinterpret_cast<const void*>(&lf_advance_kernel<SOLVER_HLLC, TC>);
}
const void* advance_fn(int solver, bool tc) { return tc ? advance_fn_t<true>(solver) : advance_fn_t<false>(solver); }

}  // namespace

int learned_advance_max_grid(int solver, bool mlp_tc) {
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
  const void* fn = advance_fn(solver, mlp_tc);
  const size_t smem = mlp_tc ? Lfa<true>::SMEM : Lfa<false>::SMEM;
  const int threads = lf_advance_threads(mlp_tc), cap = lf_advance_ctas_per_sm(mlp_tc);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess) return 0;
  if (per_sm > cap) per_sm = cap;  // the shared-memory size already ensures it
  return per_sm * sms;
}

cudaError_t launch_learned_advance(const LfAdvanceArgs& P, int solver, int grid, cudaStream_t st) {
  LfAdvanceArgs a = P;
  void* args[] = {&a};
  // cooperative: the CTAs wait on one another, so all must be resident
  const bool tc = P.mlp_tc != 0;
  return cudaLaunchCooperativeKernel(advance_fn(solver, tc), dim3(grid), dim3(lf_advance_threads(tc)), args,
                                     tc ? Lfa<true>::SMEM : Lfa<false>::SMEM, st);
}

}  // namespace gh
