// fmr.cu -- multilevel evolution with subcycling on a fixed mesh of nested
// boxes (GenASiS I, Sec. 3.7: Algorithms Evolve, EvolveLevel, StepLevel).
//
// Level 0 is an N^d single-level handle over the domain with the problem's
// walls; level l >= 1 is an N^d mesh over the central half of level l-1 at
// twice the resolution, stored with a two-cell exterior ring ((N+4)^d, a
// handle whose own walls are never read by its interior cells).  Per level
// step (StepLevel):
//   deeper level first (EvolveLevel, two steps with a provisional forward-
//   Euler coarse substep between them), prolongation of the ring, the time
//   step (deepest level: C min_l dt_CFL(l) / 2^(L-1-l); others: the time the
//   child advanced), the two RK stages with the ring held (its K zeroed after
//   stage 1), flux replacement on the uncovered coarse cells next to the
//   child's box, restriction of the child onto the covered cells, and the
//   accumulation of this level's boundary fluxes for its parent.
// All scalars (level times and steps) live on the device; the recursion only
// enqueues work on the stream.
#include <cuda_runtime.h>

#include <math.h>
#include <string.h>

#include <vector>

#include "common.h"
#include "genasis_hydro.h"
#include "hydro_handle.h"

namespace gh {
namespace {

constexpr int FNG = 2;  // exterior ring width

// Stored-array geometry of a level.
struct LevelGeo {
  int npad;  // cells per axis as stored
  int off;   // offset of the interior (0 or FNG)
  int N;
};

__device__ __forceinline__ size_t lin(int nd, int n, int i, int j, int k) {
  return nd == 1 ? (size_t)i : nd == 2 ? (size_t)j * n + i : ((size_t)k * n + j) * n + i;
}

// ---------------------------------------------------------------- transfers

// Exterior ring of fine level from the coarse level: child = coarse value +
// minmod-limited conserved slopes x (-+ h_c / 4) per axis (added in axis order).
template <class T, int NDIM>
__global__ void fmr_prolong_kernel(const T* __restrict__ Uc, LevelGeo gc, T* __restrict__ Uf, LevelGeo gf) {
  constexpr int NV = NDIM + 2;
  const unsigned np = gf.npad;
  const int N = gf.N;
  const unsigned nf = np * (NDIM > 1 ? np : 1) * (NDIM > 2 ? np : 1);  // < 2^31 (n <= 1024)
  const size_t vsc = (size_t)gc.npad * (NDIM > 1 ? gc.npad : 1) * (NDIM > 2 ? gc.npad : 1);
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < nf; t += gridDim.x * blockDim.x) {
    const unsigned t1 = t / np;
    int p[3] = {(int)(t - t1 * np), NDIM > 1 ? (int)(t1 % np) : FNG, NDIM > 2 ? (int)(t1 / np) : FNG};
    bool ring = false;
    for (int q = 0; q < NDIM; ++q) ring |= p[q] < FNG || p[q] >= FNG + N;
    if (!ring) continue;
    int c[3] = {0, 0, 0};
    for (int q = 0; q < NDIM; ++q) c[q] = N / 4 + p[q] / 2 - 1 + gc.off;  // coarse stored index
    const size_t cc = lin(NDIM, gc.npad, c[0], c[1], c[2]);
    for (int v = 0; v < NV; ++v) {
      const T u = Uc[v * vsc + cc];
      T out = u;
      for (int q = 0; q < NDIM; ++q) {
        int cm[3] = {c[0], c[1], c[2]}, cp[3] = {c[0], c[1], c[2]};
        cm[q] -= 1;
        cp[q] += 1;
        const T um = Uc[v * vsc + lin(NDIM, gc.npad, cm[0], cm[1], cm[2])];
        const T up = Uc[v * vsc + lin(NDIM, gc.npad, cp[0], cp[1], cp[2])];
        // minmod of the one-sided differences times the child offset (-+1/4 of a coarse cell)
        const T dm = u - um, dp = up - u;
        const T s = dm * dp > T(0) ? (fabs(dm) < fabs(dp) ? dm : dp) : T(0);
        out = out + s * (p[q] % 2 == 0 ? T(-0.25) : T(0.25));
      }
      Uf[v * nf + t] = out;
    }
  }
}

// Covered coarse cells = mean of their 2^d children (pairs along the slowest
// axis first, as the reference averages).
template <class T, int NDIM>
__global__ void fmr_restrict_kernel(const T* __restrict__ Uf, LevelGeo gf, T* __restrict__ Uc, LevelGeo gc) {
  constexpr int NV = NDIM + 2;
  const unsigned M = gc.N / 2;  // covered cells per axis
  const unsigned ncov = M * (NDIM > 1 ? M : 1) * (NDIM > 2 ? M : 1);
  const size_t vsf = (size_t)gf.npad * (NDIM > 1 ? gf.npad : 1) * (NDIM > 2 ? gf.npad : 1);
  const size_t vsc = (size_t)gc.npad * (NDIM > 1 ? gc.npad : 1) * (NDIM > 2 ? gc.npad : 1);
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < ncov; t += gridDim.x * blockDim.x) {
    const unsigned t1 = t / M;
    const int a[3] = {(int)(t - t1 * M), NDIM > 1 ? (int)(t1 % M) : 0, NDIM > 2 ? (int)(t1 / M) : 0};
    int f0[3] = {0, 0, 0};
    for (int q = 0; q < NDIM; ++q) f0[q] = gf.off + 2 * a[q];
    for (int v = 0; v < NV; ++v) {
      const T* U = Uf + v * vsf;
      const T half = T(0.5);  // (a + b) / 2, exactly as the mean of two
      T m;
      if (NDIM == 1) {
        m = (U[f0[0]] + U[f0[0] + 1]) * half;
      } else if (NDIM == 2) {
        T bx[2];
        for (int dx = 0; dx < 2; ++dx)
          bx[dx] = (U[lin(2, gf.npad, f0[0] + dx, f0[1], 0)] + U[lin(2, gf.npad, f0[0] + dx, f0[1] + 1, 0)]) * half;
        m = (bx[0] + bx[1]) * half;
      } else {
        T byx[2][2];
        for (int dy = 0; dy < 2; ++dy)
          for (int dx = 0; dx < 2; ++dx)
            byx[dy][dx] = (U[lin(3, gf.npad, f0[0] + dx, f0[1] + dy, f0[2])] +
                           U[lin(3, gf.npad, f0[0] + dx, f0[1] + dy, f0[2] + 1)]) * half;
        T bx[2];
        for (int dx = 0; dx < 2; ++dx) bx[dx] = (byx[0][dx] + byx[1][dx]) * half;
        m = (bx[0] + bx[1]) * half;
      }
      int c[3] = {0, 0, 0};
      for (int q = 0; q < NDIM; ++q) c[q] = gc.off + gc.N / 4 + a[q];
      Uc[v * vsc + lin(NDIM, gc.npad, c[0], c[1], c[2])] = m;
    }
  }
}

// K = 0 on the exterior ring (the ring is held through both RK stages).
template <class T, int NDIM>
__global__ void fmr_ring_zero_kernel(T* __restrict__ K, LevelGeo g) {
  constexpr int NV = NDIM + 2;
  const unsigned np = g.npad;
  const unsigned nf = np * (NDIM > 1 ? np : 1) * (NDIM > 2 ? np : 1);
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < nf; t += gridDim.x * blockDim.x) {
    const unsigned t1 = t / np;
    const int p[3] = {(int)(t - t1 * np), NDIM > 1 ? (int)(t1 % np) : FNG, NDIM > 2 ? (int)(t1 / np) : FNG};
    bool ring = false;
    for (int q = 0; q < NDIM; ++q) ring |= p[q] < FNG || p[q] >= FNG + g.N;
    if (ring)
      for (int v = 0; v < NV; ++v) K[v * nf + t] = T(0);
  }
}

// Provisional coarse substep: U += (t_child - t_coarse) K (forward Euler).
template <class T>
__global__ void fmr_euler_kernel(T* __restrict__ U, const T* __restrict__ K, size_t count, const double* ltime,
                                 int child, int coarse) {
  const T dt = (T)(ltime[child] - ltime[coarse]);
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x)
    U[t] = U[t] + dt * K[t];
}

// Per-block max over the interior of max_q (|v_q| + c_s).
template <class T, int NDIM>
__global__ void fmr_speed_kernel(const T* __restrict__ U, LevelGeo g, double gamma, double* __restrict__ part) {
  constexpr int NV = NDIM + 2;
  __shared__ double red[32];
  const unsigned N = g.N, np = g.npad;
  const unsigned ni = N * (NDIM > 1 ? N : 1) * (NDIM > 2 ? N : 1);
  const size_t vs = (size_t)np * (NDIM > 1 ? np : 1) * (NDIM > 2 ? np : 1);
  T best = T(0);  // a max is exact in the state precision; widened once below
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < ni; t += gridDim.x * blockDim.x) {
    const unsigned t1 = t / N;
    const int i = (int)(t - t1 * N) + g.off, j = NDIM > 1 ? (int)(t1 % N) + g.off : 0,
              k = NDIM > 2 ? (int)(t1 / N) + g.off : 0;
    const size_t c = lin(NDIM, np, i, j, k);
    T u[NV], w[NV];
    for (int v = 0; v < NV; ++v) u[v] = U[v * vs + c];
    recover<NDIM>(u, w);
    const T cs = sound_speed((T)gamma, (T)(gamma - 1.0) * w[NV - 1], w[0]);
    for (int q = 0; q < NDIM; ++q) best = fmax(best, fabs(w[1 + q]) + cs);
  }
  const double bw = warp_max((double)best);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = bw;
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = red[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) acc = fmax(acc, red[i]);
    part[blockIdx.x] = acc;
  }
}

struct DtArgs {
  int L, level, nblk;
  double cfl;
  const double* part;  // [L][nblk] speed partials
  const double* hcell; // [L]
  double* ltime;
  double* ldt;
  double* scal_dt;     // the level handle's dt slot
};

// The level's step: deepest level C min_l (h_l / s_l) / 2^(L-1-l); else the
// time its child has advanced beyond it.  One CTA: warp w folds level w's
// speed partials (max, order-free), thread 0 combines.
__global__ void __launch_bounds__(512) fmr_dt_kernel(DtArgs A) {
  __shared__ double smax[16];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (A.level == A.L - 1 && warp < A.L) {
    double s = 0.0;
    for (int b = lane; b < A.nblk; b += 32) s = fmax(s, A.part[warp * A.nblk + b]);
    s = warp_max(s);
    if (lane == 0) smax[warp] = s;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double dt;
  if (A.level == A.L - 1) {
    double m = INFINITY;
    for (int l = 0; l < A.L; ++l) m = fmin(m, A.hcell[l] / smax[l] / (double)(1 << (A.L - 1 - l)));
    dt = A.cfl * m;
  } else {
    dt = A.ltime[A.level + 1] - A.ltime[A.level];
  }
  A.ldt[A.level] = dt;
  *A.scal_dt = dt;
}

__global__ void fmr_advance_time_kernel(double* ltime, const double* ldt, int level) {
  if (threadIdx.x == 0 && blockIdx.x == 0) ltime[level] += ldt[level];
}

__global__ void fmr_sync_times_kernel(double* ltime, int L) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    for (int l = 1; l < L; ++l) ltime[l] = ltime[0];
}

// Heun-effective face flux (F(U^n) + F(U^n + dt K)) / 2 through the face of
// axis Q between stored cells c - e_Q and c (same reconstruction and Riemann
// solver as the stage kernels, with the handle's geometry tables).
template <class T, int NDIM, int Q, int SOLVER>
__device__ void face_eff(const StageArgs<T>& A, const T* U0, const T* K, T dt, int i, int j, int k, size_t vs,
                         double (&Fe)[NDIM + 2]) {
  constexpr int NV = NDIM + 2;
  T w[4][NV];
  for (int s = 0; s < 2; ++s) {
    for (int a = 0; a < 4; ++a) {
      int c[3] = {i, j, k};
      c[Q] += a - 2;
      const size_t cc = lin(NDIM, A.n[0], c[0], c[1], c[2]);
      T u[NV];
      for (int v = 0; v < NV; ++v) {
        T x = U0[v * vs + cc];
        if (s) x = fma(dt, K[v * vs + cc], x);
        u[v] = x;
      }
      recover<NDIM>(u, w[a]);
    }
    const int cq = (Q == 0 ? i : Q == 1 ? j : k);
    const Geo<T> gl = A.geo[Q][cq - 1 + 2], gr = A.geo[Q][cq + 2];
    T wl[NV], wr[NV], f[NV];
    for (int v = 0; v < NV; ++v) {
      wl[v] = fma(limited_slope(w[0][v], w[1][v], w[2][v], gl), gl.h, w[1][v]);
      wr[v] = fma(-limited_slope(w[1][v], w[2][v], w[3][v], gr), gr.h, w[2][v]);
    }
    face_flux<T, NDIM, Q, SOLVER>(wl, wr, A.gamma, A.gm1, f);
    for (int v = 0; v < NV; ++v) Fe[v] = s ? 0.5 * (Fe[v] + (double)f[v]) : (double)f[v];
  }
}

template <class T, int NDIM, int SOLVER>
__device__ void face_eff_q(int q, const StageArgs<T>& A, const T* U0, const T* K, T dt, int i, int j, int k, size_t vs,
                           double (&Fe)[NDIM + 2]) {
  if (q == 0) face_eff<T, NDIM, 0, SOLVER>(A, U0, K, dt, i, j, k, vs, Fe);
  else if constexpr (NDIM > 1) {
    if (q == 1) face_eff<T, NDIM, 1, SOLVER>(A, U0, K, dt, i, j, k, vs, Fe);
    else if constexpr (NDIM > 2) face_eff<T, NDIM, 2, SOLVER>(A, U0, K, dt, i, j, k, vs, Fe);
  }
}

// Face-array layout of a coarse/fine boundary: [q][side][v][M^(d-1)] with M =
// N/2 coarse faces per transverse axis, transverse indices x-fastest over the
// axes other than q.
__host__ __device__ inline size_t cf_index(int nd, int M, int q, int side, int v, int tr) {
  const size_t per = nd == 1 ? 1 : nd == 2 ? (size_t)M : (size_t)M * M;
  return (((size_t)q * 2 + side) * (nd + 2) + v) * per + tr;
}

// This level as parent: Heun-effective fluxes through the faces of its child's
// box, one thread per coarse face -> fc.
template <class T, int NDIM, int SOLVER>
__global__ void fmr_parent_faces_kernel(StageArgs<T> A, const T* __restrict__ U0, const T* __restrict__ K,
                                        LevelGeo g, double* __restrict__ fc) {
  constexpr int NV = NDIM + 2;
  const int M = g.N / 2;
  const int per = NDIM == 1 ? 1 : NDIM == 2 ? M : M * M;
  const size_t vs = (size_t)A.n[0] * A.n[1] * A.n[2];
  const T dt = (T)(*A.dt);
  const int total = NDIM * 2 * per;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int tr = t % per, side = (t / per) % 2, q = t / (2 * per);
    int c[3] = {0, 0, 0};
    int r0 = tr;
    for (int r = 0; r < NDIM; ++r) {
      if (r == q) continue;
      c[r] = g.off + g.N / 4 + r0 % M;
      r0 /= M;
    }
    c[q] = g.off + (side == 0 ? g.N / 4 : 3 * g.N / 4);  // face between cells c - e_q and c
    double Fe[NV];
    face_eff_q<T, NDIM, SOLVER>(q, A, U0, K, dt, c[0], c[1], c[2], vs, Fe);
    for (int v = 0; v < NV; ++v) fc[cf_index(NDIM, M, q, side, v, tr)] = Fe[v];
  }
}

// This level as child: acc += dt x the mean over the 2^(d-1) fine faces of
// each parent face of the Heun-effective fluxes through the level's own box
// boundary (pairs along the slowest transverse axis first).  One thread per
// fine face; the 2^(d-1) threads of a parent face are adjacent lanes of one
// warp and combine their fluxes by shuffles in that pairing order.  Launched
// with exactly ceil(total / 128) blocks of 128 threads and no early return,
// so every lane of a warp reaches the shuffles.
template <class T, int NDIM, int SOLVER>
__global__ void __launch_bounds__(128) fmr_child_faces_kernel(StageArgs<T> A, const T* __restrict__ U0,
                                                              const T* __restrict__ K, LevelGeo g,
                                                              double* __restrict__ acc) {
  constexpr int NV = NDIM + 2;
  constexpr int G = 1 << (NDIM - 1);  // fine faces per parent face
  const int M = g.N / 2;
  const int per = NDIM == 1 ? 1 : NDIM == 2 ? M : M * M;
  const size_t vs = (size_t)A.n[0] * A.n[1] * A.n[2];
  const double dtd = *A.dt;
  const T dt = (T)dtd;
  const int total = NDIM * 2 * per;
  const int tt = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = tt / G, sub = tt % G;  // parent face, fine face within it
  const bool act = t < total;
  double m[NV];
  for (int v = 0; v < NV; ++v) m[v] = 0.0;
  int tr = 0, side = 0, q = 0;
  if (act) {
    tr = t % per;
    side = (t / per) % 2;
    q = t / (2 * per);
    int c[3] = {0, 0, 0}, na = 0;
    int r0 = tr;
    for (int r = 0; r < NDIM; ++r) {
      if (r == q) continue;
      // transverse axes, fastest first: sub bit 0 along the faster, bit 1 along the slower
      c[r] = g.off + 2 * (r0 % M) + ((sub >> na) & 1);
      r0 /= M;
      ++na;
    }
    c[q] = side == 0 ? g.off : g.off + g.N;
    face_eff_q<T, NDIM, SOLVER>(q, A, U0, K, dt, c[0], c[1], c[2], vs, m);
  }
  if constexpr (NDIM == 3) {
    for (int v = 0; v < NV; ++v) m[v] = (m[v] + __shfl_xor_sync(0xffffffffu, m[v], 2)) / 2.0;  // slower axis
  }
  if constexpr (NDIM >= 2) {
    for (int v = 0; v < NV; ++v) m[v] = (m[v] + __shfl_xor_sync(0xffffffffu, m[v], 1)) / 2.0;  // faster axis
  }
  if (act && sub == 0) {
    for (int v = 0; v < NV; ++v) {
      const size_t o = cf_index(NDIM, M, q, side, v, tr);
      acc[o] = acc[o] + dtd * m[v];
    }
  }
}

// Flux replacement on the uncovered coarse cells next to the child's box:
// U += sign (dt F_coarse - Phi) / h, sign +1 below the box, -1 above.
template <class T, int NDIM>
__global__ void fmr_replace_kernel(T* __restrict__ U, LevelGeo g, const double* __restrict__ fc,
                                   const double* __restrict__ phi, const double* __restrict__ dtp, double h) {
  constexpr int NV = NDIM + 2;
  const int M = g.N / 2;
  const int per = NDIM == 1 ? 1 : NDIM == 2 ? M : M * M;
  const size_t vs = (size_t)g.npad * (NDIM > 1 ? g.npad : 1) * (NDIM > 2 ? g.npad : 1);
  const double dt = *dtp;
  const int total = NDIM * 2 * per;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int tr = t % per, side = (t / per) % 2, q = t / (2 * per);
    int c[3] = {0, 0, 0};
    int r0 = tr;
    for (int r = 0; r < NDIM; ++r) {
      if (r == q) continue;
      c[r] = g.off + g.N / 4 + r0 % M;
      r0 /= M;
    }
    c[q] = g.off + (side == 0 ? g.N / 4 - 1 : 3 * g.N / 4);
    const double sign = side == 0 ? 1.0 : -1.0;
    const size_t cc = lin(NDIM, g.npad, c[0], c[1], c[2]);
    for (int v = 0; v < NV; ++v) {
      const size_t o = cf_index(NDIM, M, q, side, v, tr);
      U[v * vs + cc] = (T)((double)U[v * vs + cc] + sign * (dt * fc[o] - phi[o]) / h);
    }
  }
}

int grid_of(size_t n) {
  size_t g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

}  // namespace
}  // namespace gh

using namespace gh;

struct genasis_fmr {
  int ndim = 2, N = 16, L = 1, prec = GENASIS_FP64, solver = GENASIS_HLLC;
  double gamma = 1.4;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<genasis_hydro_t> lev;
  std::vector<LevelGeo> geo;
  std::vector<double> hcell;
  std::vector<void*> save;
  std::vector<double*> acc;  // acc[l]: Phi accumulated by level l (>= 1) for its parent
  std::vector<double*> fc;   // fc[l]: level l's fluxes through its child's box
  size_t cf_count = 0;       // doubles per face array
  int nblk = 0;
  double* part = nullptr;    // [L][nblk]
  double* d_hcell = nullptr;
  double* ltime = nullptr;
  double* ldt = nullptr;
  std::vector<char> dirty;   // level interior changed since its speed partials were taken
  long long steps_done = 0;
  cudaGraphExec_t graph = nullptr;  // two global steps, captured after the first
  double graph_cfl = 0.0;
  int graph_cur0 = 0;               // level 0's state buffer when the capture started
};

namespace gh {
namespace {

template <class T, int NDIM, int SOLVER>
struct FmrRun {
  static int launch_stage(genasis_hydro* h, int stage, cudaStream_t st) { return gh::launch_stage<T>(h, stage, st); }

  static int ring_zero(genasis_fmr* f, int l) {
    genasis_hydro* h = f->lev[l];
    fmr_ring_zero_kernel<T, NDIM><<<grid_of(h->ncell), 256, 0, f->stream>>>((T*)h->K, f->geo[l]);
    GH_CK(cudaGetLastError());
    return GENASIS_OK;
  }

  static int evolve_level(genasis_fmr* f, int i, double* acc, double cfl) {
    int rc = step_level(f, i, acc, cfl);
    if (rc || i == 0) return rc;
    genasis_hydro* c = f->lev[i - 1];
    cudaStream_t st = f->stream;
    const size_t bytes = c->ncell * c->nv * c->esize;
    GH_CK(cudaMemcpyAsync(f->save[i - 1], c->U[c->cur], bytes, cudaMemcpyDeviceToDevice, st));
    // provisional coarse substep (forward Euler by the child's first step), ring held
    rc = launch_stage(c, 1, st);
    if (rc) return rc;
    if (i - 1 >= 1 && (rc = ring_zero(f, i - 1))) return rc;
    fmr_euler_kernel<T><<<grid_of(c->ncell * c->nv), 256, 0, st>>>((T*)c->U[c->cur], (const T*)c->K, c->ncell * c->nv,
                                                                    f->ltime, i, i - 1);
    GH_CK(cudaGetLastError());
    f->dirty[i - 1] = 1;
    rc = step_level(f, i, acc, cfl);
    if (rc) return rc;
    GH_CK(cudaMemcpyAsync(c->U[c->cur], f->save[i - 1], bytes, cudaMemcpyDeviceToDevice, st));
    f->dirty[i - 1] = 1;
    return GENASIS_OK;
  }

  static int step_level(genasis_fmr* f, int i, double* acc, double cfl) {
    genasis_hydro* h = f->lev[i];
    cudaStream_t st = f->stream;
    const int L = f->L;
    int rc;
    if (i + 1 < L) {
      GH_CK(cudaMemsetAsync(f->acc[i + 1], 0, f->cf_count * sizeof(double), st));
      if ((rc = evolve_level(f, i + 1, f->acc[i + 1], cfl))) return rc;
    }
    if (i > 0) {
      genasis_hydro* c = f->lev[i - 1];
      fmr_prolong_kernel<T, NDIM><<<grid_of(h->ncell), 256, 0, st>>>((const T*)c->U[c->cur], f->geo[i - 1],
                                                                     (T*)h->U[h->cur], f->geo[i]);
      GH_CK(cudaGetLastError());
    }
    if (i == L - 1) {
      // speed partials of every level whose interior changed since they were taken
      for (int l = 0; l < L; ++l) {
        if (!f->dirty[l]) continue;
        genasis_hydro* g = f->lev[l];
        fmr_speed_kernel<T, NDIM><<<f->nblk, 256, 0, st>>>((const T*)g->U[g->cur], f->geo[l], f->gamma,
                                                            f->part + (size_t)l * f->nblk);
        GH_CK(cudaGetLastError());
        f->dirty[l] = 0;
      }
    }
    DtArgs D;
    D.L = L;
    D.level = i;
    D.nblk = f->nblk;
    D.cfl = cfl;
    D.part = f->part;
    D.hcell = f->d_hcell;
    D.ltime = f->ltime;
    D.ldt = f->ldt;
    D.scal_dt = h->scal + SCAL_DT;
    fmr_dt_kernel<<<1, 32 * L, 0, st>>>(D);
    GH_CK(cudaGetLastError());
    // the two RK stages with the exterior ring held
    if ((rc = launch_stage(h, 1, st))) return rc;
    if (i >= 1 && (rc = ring_zero(f, i))) return rc;
    if ((rc = launch_stage(h, 2, st))) return rc;
    h->cur = 1 - h->cur;
    f->dirty[i] = 1;
    StageArgs<T> A = stage_args<T>(h, 1);  // geometry, gamma and the dt slot of this level
    const T* U0 = (const T*)h->U[1 - h->cur];
    const int nfc = grid_of(f->cf_count / (NDIM + 2));
    if (i + 1 < L) {
      fmr_parent_faces_kernel<T, NDIM, SOLVER><<<nfc, 128, 0, st>>>(A, U0, (const T*)h->K, f->geo[i], f->fc[i]);
      GH_CK(cudaGetLastError());
      fmr_replace_kernel<T, NDIM><<<nfc, 128, 0, st>>>((T*)h->U[h->cur], f->geo[i], f->fc[i], f->acc[i + 1],
                                                        f->ldt + i, f->hcell[i]);
      GH_CK(cudaGetLastError());
      genasis_hydro* c = f->lev[i + 1];
      fmr_restrict_kernel<T, NDIM><<<grid_of(h->ncell), 256, 0, st>>>((const T*)c->U[c->cur], f->geo[i + 1],
                                                                      (T*)h->U[h->cur], f->geo[i]);
      GH_CK(cudaGetLastError());
    }
    fmr_advance_time_kernel<<<1, 32, 0, st>>>(f->ltime, f->ldt, i);
    GH_CK(cudaGetLastError());
    if (acc) {
      const size_t nfine = (f->cf_count / (NDIM + 2)) << (NDIM - 1);  // fine faces on the box boundary
      fmr_child_faces_kernel<T, NDIM, SOLVER>
          <<<(unsigned)((nfine + 127) / 128), 128, 0, st>>>(A, U0, (const T*)h->K, f->geo[i], acc);
      GH_CK(cudaGetLastError());
    }
    return GENASIS_OK;
  }

  static int global_step(genasis_fmr* f, double cfl) {
    fmr_sync_times_kernel<<<1, 32, 0, f->stream>>>(f->ltime, f->L);
    GH_CK(cudaGetLastError());
    return evolve_level(f, 0, nullptr, cfl);
  }
};

template <class T, int NDIM>
int fmr_step_t(genasis_fmr* f, double cfl) {
  return f->solver == GENASIS_HLL ? FmrRun<T, NDIM, SOLVER_HLL>::global_step(f, cfl)
                                  : FmrRun<T, NDIM, SOLVER_HLLC>::global_step(f, cfl);
}

int fmr_step(genasis_fmr* f, double cfl) {
  if (f->prec == GENASIS_FP64) return f->ndim == 2 ? fmr_step_t<double, 2>(f, cfl) : fmr_step_t<double, 3>(f, cfl);
  return f->ndim == 2 ? fmr_step_t<float, 2>(f, cfl) : fmr_step_t<float, 3>(f, cfl);
}

void fmr_free(genasis_fmr* f) {
  if (f->stream) cudaStreamSynchronize(f->stream);
  if (f->graph) cudaGraphExecDestroy(f->graph);
  for (auto h : f->lev) genasis_hydro_destroy(h);
  for (auto p : f->save) cudaFree(p);
  for (auto p : f->acc) cudaFree(p);
  for (auto p : f->fc) cudaFree(p);
  cudaFree(f->part);
  cudaFree(f->d_hcell);
  cudaFree(f->ltime);
  cudaFree(f->ldt);
  if (f->own_stream && f->stream) cudaStreamDestroy(f->stream);
  delete f;
}

}  // namespace
}  // namespace gh

extern "C" {

int genasis_fmr_create(const genasis_fmr_desc* d, genasis_fmr_t* out) {
  if (!d || !out) return fail(GENASIS_EINVAL, "fmr_create: NULL argument");
  *out = nullptr;
  if (d->ndim != 2 && d->ndim != 3) return fail(GENASIS_EINVAL, "fmr_create: ndim must be 2 or 3");
  if (d->n % 4 || d->n < 16 || d->n > 1024)
    return fail(GENASIS_EINVAL, "fmr_create: n must be a multiple of 4 in [16, 1024]");
  if (d->nlevels < 1 || d->nlevels > 12) return fail(GENASIS_EINVAL, "fmr_create: nlevels must be in [1, 12]");
  // (the dt kernel folds each level's speed partials in one warp: 12 levels, 384 threads)
  if (!(d->size > 0.0)) return fail(GENASIS_EINVAL, "fmr_create: size must be > 0");
  if (d->precision != GENASIS_FP64 && d->precision != GENASIS_FP32_MIXED)
    return fail(GENASIS_EINVAL, "fmr_create: precision must be GENASIS_FP64 or GENASIS_FP32_MIXED");
  if (d->solver != GENASIS_HLL && d->solver != GENASIS_HLLC) return fail(GENASIS_EINVAL, "fmr_create: bad solver");
  if (d->bc < 0 || d->bc > 2) return fail(GENASIS_EINVAL, "fmr_create: bad boundary rule");
  genasis_fmr* f = new genasis_fmr();
  f->ndim = d->ndim;
  f->N = d->n;
  f->L = d->nlevels;
  f->prec = d->precision;
  f->solver = d->solver;
  f->gamma = d->gamma;
  if (d->stream) {
    f->stream = (cudaStream_t)d->stream;
  } else {
    if (cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete f;
      return fail(GENASIS_ECUDA, "fmr_create: stream creation failed");
    }
    f->own_stream = true;
  }
  const int N = f->N, nd = f->ndim;
  for (int l = 0; l < f->L; ++l) {
    const int npad = N + (l ? 2 * FNG : 0);
    const double hl = d->size / N / (double)(1 << l);
    std::vector<double> w(npad, hl);
    genasis_hydro_desc hd;
    memset(&hd, 0, sizeof(hd));
    hd.ndim = nd;
    for (int q = 0; q < 3; ++q) {
      hd.n[q] = q < nd ? npad : 1;
      hd.widths[q] = q < nd ? w.data() : nullptr;
      hd.bc_lo[q] = hd.bc_hi[q] = l == 0 ? d->bc : GENASIS_BC_OUTFLOW;
    }
    hd.gamma = d->gamma;
    hd.solver = d->solver;
    hd.theta = d->theta;
    hd.precision = d->precision;
    hd.stream = f->stream;
    genasis_hydro_t h = nullptr;
    int rc = genasis_hydro_create(&hd, &h);
    if (rc) {
      fmr_free(f);
      return rc;
    }
    h->want_totals = 0;
    f->lev.push_back(h);
    f->geo.push_back(LevelGeo{npad, l ? FNG : 0, N});
    f->hcell.push_back(hl);
  }
  const int M = N / 2;
  const size_t per = nd == 2 ? (size_t)M : (size_t)M * M;
  f->cf_count = (size_t)nd * 2 * (nd + 2) * per;
  f->nblk = 1024;
  bool ok = true;
  for (int l = 0; l < f->L && ok; ++l) {
    void* s = nullptr;
    double* a = nullptr;
    double* c = nullptr;
    ok &= cudaMalloc(&s, f->lev[l]->ncell * f->lev[l]->nv * f->lev[l]->esize) == cudaSuccess;
    ok &= cudaMalloc((void**)&a, f->cf_count * sizeof(double)) == cudaSuccess;
    ok &= cudaMalloc((void**)&c, f->cf_count * sizeof(double)) == cudaSuccess;
    f->save.push_back(s);
    f->acc.push_back(a);
    f->fc.push_back(c);
  }
  ok &= cudaMalloc((void**)&f->part, (size_t)f->L * f->nblk * sizeof(double)) == cudaSuccess;
  ok &= cudaMalloc((void**)&f->d_hcell, f->L * sizeof(double)) == cudaSuccess;
  ok &= cudaMalloc((void**)&f->ltime, f->L * sizeof(double)) == cudaSuccess;
  ok &= cudaMalloc((void**)&f->ldt, f->L * sizeof(double)) == cudaSuccess;
  if (!ok) {
    fmr_free(f);
    return fail(GENASIS_ENOMEM, "fmr_create: device allocation failed");
  }
  cudaMemcpy(f->d_hcell, f->hcell.data(), f->L * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemset(f->ltime, 0, f->L * sizeof(double));
  f->dirty.assign(f->L, 1);
  *out = f;
  return GENASIS_OK;
}

int genasis_fmr_destroy(genasis_fmr_t f) {
  if (f) fmr_free(f);
  return GENASIS_OK;
}

int genasis_fmr_set_level(genasis_fmr_t f, int level, const double* U) {
  if (!f || !U) return fail(GENASIS_EINVAL, "NULL argument");
  if (level < 0 || level >= f->L) return fail(GENASIS_EINVAL, "fmr: level out of range");
  f->dirty[level] = 1;
  if (f->graph) {  // the captured step assumed the previous speed bookkeeping
    cudaGraphExecDestroy(f->graph);
    f->graph = nullptr;
  }
  f->steps_done = 0;
  return genasis_hydro_set_conserved(f->lev[level], U, GENASIS_FP64);
}

int genasis_fmr_get_level(genasis_fmr_t f, int level, double* U) {
  if (!f || !U) return fail(GENASIS_EINVAL, "NULL argument");
  if (level < 0 || level >= f->L) return fail(GENASIS_EINVAL, "fmr: level out of range");
  return genasis_hydro_get_conserved(f->lev[level], U, GENASIS_FP64);
}

int genasis_fmr_autotune(genasis_fmr_t f, int trial_steps) {
  if (!f) return fail(GENASIS_EINVAL, "NULL handle");
  if (trial_steps < 1) return fail(GENASIS_EINVAL, "fmr_autotune: trial_steps must be >= 1");
  // each level's tile and plane count, timed on its own mesh and state (which
  // the level's autotune restores); the captured steps hold the old launches
  for (genasis_hydro* h : f->lev) {
    const int rc = genasis_hydro_autotune(h, trial_steps, nullptr);
    if (rc) return rc;
  }
  if (f->graph) {
    cudaGraphExecDestroy(f->graph);
    f->graph = nullptr;
  }
  return GENASIS_OK;
}

int genasis_fmr_step(genasis_fmr_t f, int nsteps, double cfl, double* t_out) {
  if (!f) return fail(GENASIS_EINVAL, "NULL handle");
  if (nsteps < 0 || !(cfl > 0.0)) return fail(GENASIS_EINVAL, "fmr_step: bad nsteps or cfl");
  // From the second global step on, the launch sequence of two global steps
  // (level 0 steps once per global step, so its buffers alternate; every
  // deeper level steps an even number of times) repeats, including which
  // levels' speeds are retaken: it is captured once as a CUDA graph and
  // replayed while level 0 starts from the same buffer.
  int s = 0;
  while (s < nsteps) {
    if (f->graph && f->graph_cfl != cfl) {
      cudaGraphExecDestroy(f->graph);
      f->graph = nullptr;
    }
    if (!f->graph && f->steps_done >= 1 && nsteps - s >= 2) {
      cudaGraph_t g;
      const std::vector<char> dirty0 = f->dirty;
      std::vector<int> cur_before(f->L);
      for (int l = 0; l < f->L; ++l) cur_before[l] = f->lev[l]->cur;
      const int cur0 = cur_before[0];
      GH_CK(cudaStreamBeginCapture(f->stream, cudaStreamCaptureModeThreadLocal));
      int rc = fmr_step(f, cfl);
      if (!rc) rc = fmr_step(f, cfl);
      cudaError_t e = cudaStreamEndCapture(f->stream, &g);
      // nothing ran during the capture: every level has stepped an even number
      // of times in it, so its buffer index is back where it started
      bool even = true;
      for (int l = 0; l < f->L; ++l) {
        even &= f->lev[l]->cur == cur_before[l];
        f->lev[l]->cur = cur_before[l];
      }
      if (rc) {
        if (e == cudaSuccess) cudaGraphDestroy(g);
        return rc;
      }
      GH_CK(e);
      const bool periodic = f->dirty == dirty0 && even;
      f->dirty = dirty0;
      if (!periodic) {
        cudaGraphDestroy(g);
      } else {
        e = cudaGraphInstantiate(&f->graph, g, 0);
        cudaGraphDestroy(g);
        GH_CK(e);
        f->graph_cfl = cfl;
        f->graph_cur0 = cur0;
      }
    }
    if (f->graph && nsteps - s >= 2 && f->lev[0]->cur == f->graph_cur0) {
      GH_CK(cudaGraphLaunch(f->graph, f->stream));
      s += 2;
      f->steps_done += 2;
    } else {
      int rc = fmr_step(f, cfl);
      if (rc) return rc;
      ++s;
      ++f->steps_done;
    }
  }
  if (t_out) {
    GH_CK(cudaMemcpyAsync(t_out, f->ltime, sizeof(double), cudaMemcpyDeviceToHost, f->stream));
    for (auto h : f->lev) {
      int rc = genasis_hydro_sync(h);
      if (rc) return rc;
    }
  }
  return GENASIS_OK;
}

}  // extern "C"
