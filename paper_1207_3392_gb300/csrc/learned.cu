// learned.cu -- the learned flux correction (2D, FP32 state): the corrected
// solver handle genasis_learned_*, the BF16 tensor-core MLP kernels
// (inference, gradients, Adam) behind genasis_mlp_*, and the kernels that turn
// fine runs into training targets.  The correction is the benchmark's
// addition to the HLLC flux of Sec. 3.2; the paper has no counterpart.
#include <cuda_runtime.h>

#include <math.h>
#include <string.h>

#include <vector>

#include "aux_kernels.h"
#include "common.h"
#include "genasis_hydro.h"
#include "geometry.h"
#include "learned_internal.h"
#include "learned_kernels.cuh"
#include "learned_step.cuh"
#include "mlp_tc.cuh"

namespace gh {

// ============================================================== MLP kernels

// BF16 image of the forward-pass weights (one CTA).
__global__ void __launch_bounds__(256) mlp_pack_kernel(const float* __restrict__ P, mlp::InferWeights* __restrict__ out) {
  mlp::fill_layers(*out, P);
}

// Y[n][4] = net(X[n][32]); one warp per 16 samples, weights (a prepared
// image) in shared memory; a persistent grid loops over the 16-sample tiles.
__global__ void __launch_bounds__(256) mlp_infer_kernel(const mlp::InferWeights* __restrict__ Wg,
                                                        const __nv_bfloat16* __restrict__ X, long long n,
                                                        float* __restrict__ Y) {
  __shared__ mlp::InferWeights W;
  mlp::copy_weights(W, Wg);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long ntile = (n + 15) / 16;
  for (long long tile = (long long)blockIdx.x * 8 + warp; tile < ntile; tile += (long long)gridDim.x * 8) {
    const long long s0 = tile * 16;
    const int rows = (int)(n - s0 < 16 ? n - s0 : 16);
    mlp::Forward F;
    mlp::load_x(F, X + s0 * mlp::KIN, rows);
    mlp::forward(F, W);
    if (t < 2) {
      if (g < rows) {
        Y[(s0 + g) * 4 + 2 * t] = F.y[0];
        Y[(s0 + g) * 4 + 2 * t + 1] = F.y[1];
      }
      if (g + 8 < rows) {
        Y[(s0 + g + 8) * 4 + 2 * t] = F.y[2];
        Y[(s0 + g + 8) * 4 + 2 * t + 1] = F.y[3];
      }
    }
  }
}

// Y[n][4] = net(X[n][32]) on the tensor cores (mlp_tc.cuh): a persistent
// grid over tiles of MLP_TC_GROUPS x 128 samples, one sample per thread; each
// group of four warps runs its 128 samples with its own mbarrier, operand tile
// and 128 TMEM columns.  The weights sit in shared memory once per CTA.  One
// CTA per SM, which takes all 512 TMEM columns: the shared-memory request
// keeps a second CTA off the SM.  If a wait for the tensor cores runs out,
// *status (if non-null) gets STATUS_TIMEOUT and the rows of the group's
// remaining tiles are NaN.
constexpr int MLP_TC_GROUPS = 4;
constexpr int MLP_TC_THREADS = MLP_TC_GROUPS * mlptc::M;
constexpr size_t MLP_TC_SMEM = 120 * 1024;  // > 228 KB / 2: one CTA per SM
static_assert(sizeof(mlptc::Weights) + MLP_TC_GROUPS * sizeof(mlptc::Tile) <= MLP_TC_SMEM, "operand images fit");
static_assert(MLP_TC_GROUPS * mlptc::TMEM_COLS <= 512, "the CTA's TMEM fits the SM");

__global__ void __launch_bounds__(MLP_TC_THREADS, 1) mlp_infer_tc_kernel(const mlp::InferWeights* __restrict__ Wg,
                                                                       const __nv_bfloat16* __restrict__ X,
                                                                       long long n, float* __restrict__ Y,
                                                                       unsigned* status) {
  extern __shared__ __align__(128) unsigned char smem_mlptc[];
  auto& W = *reinterpret_cast<mlptc::Weights*>(smem_mlptc);
  auto* tiles = reinterpret_cast<mlptc::Tile*>(smem_mlptc + sizeof(mlptc::Weights));
  __shared__ unsigned long long mbar[MLP_TC_GROUPS];
  __shared__ uint32_t tmem_slot;
  const int grp = threadIdx.x / mlptc::M, t = threadIdx.x % mlptc::M;
  mlptc::load_weights(W, Wg);
  if (threadIdx.x < MLP_TC_GROUPS) tma::mbar_init(mbar + threadIdx.x, 1);
  tma::fence_mbar_init();
  if (threadIdx.x < 32) mlptc::tmem_alloc(&tmem_slot, MLP_TC_GROUPS * mlptc::TMEM_COLS);
  mlptc::fence_before();
  __syncthreads();
  mlptc::fence_after();
  const uint32_t tmem = tmem_slot + (uint32_t)(grp * mlptc::TMEM_COLS);
  mlptc::Tile& T = tiles[grp];
  unsigned phase = 0;
  const long long ntile = (n + mlptc::M - 1) / mlptc::M;  // 128-sample tiles, group-strided
  long long tile = (long long)blockIdx.x * MLP_TC_GROUPS + grp;
  const long long step = (long long)gridDim.x * MLP_TC_GROUPS;
  bool ok = true;
  for (; tile < ntile; tile += step) {
    const long long r = tile * mlptc::M + t;
    const uint4* src = reinterpret_cast<const uint4*>(X + r * mlp::KIN);
#pragma unroll
    for (int c = 0; c < mlp::KIN / 8; ++c)
      *reinterpret_cast<uint4*>(T.x + mlptc::core_idx(t, 8 * c, mlp::KIN)) = r < n ? __ldg(src + c) : make_uint4(0, 0, 0, 0);
    float y[4];
    ok = mlptc::forward_tile(W, T, mbar + grp, phase, tmem, 1 + grp, t, y);
    if (!ok) break;
    if (r < n) *reinterpret_cast<float4*>(Y + r * 4) = make_float4(y[0], y[1], y[2], y[3]);
  }
  if (!ok) {  // poison what this group did not compute
    if (t == 0 && status) atomicOr(status, STATUS_TIMEOUT);
    for (; tile < ntile; tile += step) {
      const long long r = tile * mlptc::M + t;
      if (r < n) *reinterpret_cast<float4*>(Y + r * 4) = make_float4(NAN, NAN, NAN, NAN);
    }
  }
  mlptc::fence_before();
  __syncthreads();
  mlptc::fence_after();
  if (threadIdx.x < 32) mlptc::tmem_dealloc(tmem_slot, MLP_TC_GROUPS * mlptc::TMEM_COLS);
}

// Inference over n samples with a persistent grid: on mma.sync fragments in
// registers (tc = false, the default engine, up to 4 CTAs per SM), or on
// tcgen05 (tc = true, one CTA per SM).
cudaError_t launch_mlp_infer(const mlp::InferWeights* W, const __nv_bfloat16* X, long long n, float* Y,
                             unsigned* status, bool tc, cudaStream_t st) {
  static bool attr_set = false;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long cap = 4LL * sms;
  if (!tc) {
    const long long tiles = (n + 15) / 16, want = (tiles + 7) / 8;
    mlp_infer_kernel<<<(int)(want < cap ? want : cap), 256, 0, st>>>(W, X, n, Y);
    return cudaGetLastError();
  }
  if (!attr_set) {
    e = cudaFuncSetAttribute(mlp_infer_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_TC_SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const long long tiles = (n + MLP_TC_THREADS - 1) / MLP_TC_THREADS, one_per_sm = sms;
  mlp_infer_tc_kernel<<<(int)(tiles < one_per_sm ? tiles : one_per_sm), MLP_TC_THREADS, MLP_TC_SMEM, st>>>(W, X, n, Y,
                                                                                                         status);
  return cudaGetLastError();
}

constexpr int TS = 128;            // samples per CTA iteration in training (8 warps x 16)
constexpr int TSP = TS + mlp::PAD;

struct TrainSmem {
  mlp::Weights W;
  __nv_bfloat16 xt[mlp::KIN][TSP];   // X^T
  __nv_bfloat16 h1t[mlp::NH][TSP];   // h1^T
  __nv_bfloat16 h2t[mlp::NH][TSP];   // h2^T
  __nv_bfloat16 d1t[mlp::NH][TSP];   // (dL/dz1)^T
  __nv_bfloat16 d2t[mlp::NH][TSP];   // (dL/dz2)^T
  __nv_bfloat16 dyt[16][TSP];        // (dL/dy)^T, rows >= 4 zero
  float red[256];
};

// Scatter a 16 x 16 A fragment (rows = samples s0 + g / + 8, columns c0 + ...)
// into a transposed [column][sample] array.
__device__ __forceinline__ void store_afrag_t(__nv_bfloat16 (*dst)[TSP], const uint32_t (&a)[4], int c0, int s0) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const __nv_bfloat162* v = reinterpret_cast<const __nv_bfloat162*>(a);
  dst[c0 + 2 * t][s0 + g] = v[0].x;
  dst[c0 + 2 * t + 1][s0 + g] = v[0].y;
  dst[c0 + 2 * t][s0 + g + 8] = v[1].x;
  dst[c0 + 2 * t + 1][s0 + g + 8] = v[1].y;
  dst[c0 + 2 * t + 8][s0 + g] = v[2].x;
  dst[c0 + 2 * t + 9][s0 + g] = v[2].y;
  dst[c0 + 2 * t + 8][s0 + g + 8] = v[3].x;
  dst[c0 + 2 * t + 9][s0 + g + 8] = v[3].y;
}

// One accumulator tile (16 x 8) of A^T B where A^T rows come from `a` ([row][sample])
// and B columns from `b` ([col][sample]), K = TS samples.
__device__ __forceinline__ void grad_tile(float (&acc)[4], const __nv_bfloat16 (*a)[TSP], int r0,
                                          const __nv_bfloat16 (*b)[TSP], int c0) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll 4
  for (int kk = 0; kk < TS / 16; ++kk) {
    const int k = 16 * kk + 2 * t;
    uint32_t af[4] = {mlp::ld32(&a[r0 + g][k]), mlp::ld32(&a[r0 + g + 8][k]), mlp::ld32(&a[r0 + g][k + 8]),
                      mlp::ld32(&a[r0 + g + 8][k + 8])};
    mlp::mma16816(acc, af, mlp::ld32(&b[c0 + g][k]), mlp::ld32(&b[c0 + g][k + 8]));
  }
}

// Gradient of mean((y - T)^2) (over n samples x 4 outputs) with respect to the
// parameters, summed per CTA into part[blockIdx.x][NPARAM]; loss sums into
// part_loss[blockIdx.x].  Deterministic: fixed sample-to-CTA assignment.
__global__ void __launch_bounds__(256) mlp_train_kernel(const float* __restrict__ P, const __nv_bfloat16* __restrict__ X,
                                                        const float* __restrict__ T, long long n, float inv_count,
                                                        float* __restrict__ part, float* __restrict__ part_loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
  mlp::load_weights(S.W, P);
  for (int i = threadIdx.x; i < 16 * TSP; i += blockDim.x) (&S.dyt[0][0])[i] = __float2bfloat16(0.0f);
  __syncthreads();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  float gw1[2][4] = {}, gw2[4][4] = {}, gw3[4] = {};
  float gb = 0.0f, loss = 0.0f;
  for (long long base = (long long)blockIdx.x * TS; base < n; base += (long long)gridDim.x * TS) {
    const long long s0 = base + 16 * warp;
    const int rows = (int)(n - s0 <= 0 ? 0 : (n - s0 < 16 ? n - s0 : 16));
    mlp::Forward F;
    mlp::load_x(F, X + s0 * mlp::KIN, rows);
    mlp::forward(F, S.W);
    // dL/dy
    float dy[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = g + (e >= 2 ? 8 : 0), c = 2 * t + (e & 1);
      float d = 0.0f;
      if (c < mlp::NOUT && r < rows) {
        const float diff = F.y[e] - T[(s0 + r) * 4 + c];
        loss += diff * diff;
        d = 2.0f * diff * inv_count;
      }
      dy[e] = d;
    }
    uint32_t dya[4] = {mlp::pack2(dy[0], dy[1]), mlp::pack2(dy[2], dy[3]), 0u, 0u};
    // dL/dz2 = (dy W3) * silu'(z2)
    float d2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      mlp::mma16816(acc, dya, mlp::ld32(&S.W.w3t[8 * nt + g][2 * t]), mlp::ld32(&S.W.w3t[8 * nt + g][2 * t + 8]));
#pragma unroll
      for (int e = 0; e < 4; ++e) d2[nt][e] = acc[e] * mlp::dsilu(F.z2[nt][e]);
    }
    uint32_t d2a[4][4];
    mlp::to_afrag(d2, d2a, false);
    // dL/dz1 = (dz2 W2) * silu'(z1)
    float d1[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kc = 0; kc < 4; ++kc)
        mlp::mma16816(acc, d2a[kc], mlp::ld32(&S.W.w2t[8 * nt + g][16 * kc + 2 * t]),
                      mlp::ld32(&S.W.w2t[8 * nt + g][16 * kc + 2 * t + 8]));
#pragma unroll
      for (int e = 0; e < 4; ++e) d1[nt][e] = acc[e] * mlp::dsilu(F.z1[nt][e]);
    }
    uint32_t d1a[4][4];
    mlp::to_afrag(d1, d1a, false);
    // transposed copies for the weight-gradient products
    const int sl = 16 * warp;
    store_afrag_t(S.xt, F.xa[0], 0, sl);
    store_afrag_t(S.xt, F.xa[1], 16, sl);
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      store_afrag_t(S.h1t, F.h1a[kc], 16 * kc, sl);
      store_afrag_t(S.h2t, F.h2a[kc], 16 * kc, sl);
      store_afrag_t(S.d1t, d1a[kc], 16 * kc, sl);
      store_afrag_t(S.d2t, d2a[kc], 16 * kc, sl);
    }
    {
      const __nv_bfloat162* v = reinterpret_cast<const __nv_bfloat162*>(dya);
      S.dyt[2 * t][sl + g] = v[0].x;
      S.dyt[2 * t + 1][sl + g] = v[0].y;
      S.dyt[2 * t][sl + g + 8] = v[1].x;
      S.dyt[2 * t + 1][sl + g + 8] = v[1].y;
    }
    __syncthreads();
    // weight gradients, K = TS samples: dW1 (4 x 4 tiles), dW2 (4 x 8), dW3 (1 x 8)
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int tile = warp + 8 * i;
      grad_tile(gw1[i], S.d1t, 16 * (tile / 4), S.xt, 8 * (tile % 4));
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int tile = 4 * warp + i;
      grad_tile(gw2[i], S.d2t, 16 * (tile / 8), S.h1t, 8 * (tile % 8));
    }
    grad_tile(gw3, S.dyt, 0, S.h2t, 8 * warp);
    // bias gradients: row sums of the transposed derivative tables
    {
      const __nv_bfloat16* row = tid < 64 ? S.d1t[tid] : tid < 128 ? S.d2t[tid - 64] : S.dyt[(tid - 128) & 15];
      if (tid < 132) {
        float s = 0.f;
        for (int k = 0; k < TS; k += 2) {
          const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(row + k);
          s += __bfloat162float(v.x) + __bfloat162float(v.y);
        }
        gb += s;
      }
    }
    __syncthreads();
  }
  // write this CTA's partial gradient
  float* G = part + (size_t)blockIdx.x * mlp::NPARAM;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int tile = warp + 8 * i, r0 = 16 * (tile / 4), c0 = 8 * (tile % 4);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = r0 + g + (e >= 2 ? 8 : 0), c = c0 + 2 * t + (e & 1);
      if (c < mlp::NIN) G[mlp::OW1 + r * mlp::NIN + c] = gw1[i][e];
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int tile = 4 * warp + i, r0 = 16 * (tile / 8), c0 = 8 * (tile % 8);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = r0 + g + (e >= 2 ? 8 : 0), c = c0 + 2 * t + (e & 1);
      G[mlp::OW2 + r * mlp::NH + c] = gw2[i][e];
    }
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int r = g + (e >= 2 ? 8 : 0), c = 8 * warp + 2 * t + (e & 1);
    if (r < mlp::NOUT) G[mlp::OW3 + r * mlp::NH + c] = gw3[e];
  }
  if (tid < 64) G[mlp::OB1 + tid] = gb;
  else if (tid < 128) G[mlp::OB2 + tid - 64] = gb;
  else if (tid < 132) G[mlp::OB3 + tid - 128] = gb;
  // loss: fixed-order block sum
  S.red[tid] = loss;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w) S.red[tid] += S.red[tid + w];
    __syncthreads();
  }
  if (tid == 0) part_loss[blockIdx.x] = S.red[0];
}

// Sum the per-CTA partials in order (gradient, loss); optionally one Adam step
// on the FP32 parameters (Kingma & Ba, bias-corrected).
__global__ void mlp_reduce_adam_kernel(const float* __restrict__ part, const float* __restrict__ part_loss, int nblk,
                                       float* __restrict__ grad_out, float* __restrict__ loss_out, float* P, float* m,
                                       float* v, int step, float lr, float b1, float b2, float eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0 && loss_out) {
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += part_loss[b];
    *loss_out = s;
  }
  if (p >= mlp::NPARAM) return;
  float g = 0.f;
  for (int b = 0; b < nblk; ++b) g += part[(size_t)b * mlp::NPARAM + p];
  if (grad_out) grad_out[p] = g;
  if (step > 0) {
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float mh = mm / (1.f - powf(b1, (float)step));
    const float vh = vv / (1.f - powf(b2, (float)step));
    P[p] -= lr * mh / (sqrtf(vh) + eps);
  }
}

// ====================================================== learned-solver kernels

// Plain flux of every face (x faces (nx+1) x ny, then y faces nx x (ny+1)) of
// the state un (+ dt k), and, if X is non-null, the MLP features and scales.
template <int SOLVER>
__global__ void lf_faces_kernel(Mesh2 M, const float* __restrict__ un, const float* __restrict__ k,
                                const double* __restrict__ dtp, float* __restrict__ F, __nv_bfloat16* __restrict__ X,
                                float* __restrict__ scale) {
  const long long nxf = (long long)(M.nx + 1) * M.ny, nf = nxf + (long long)M.nx * (M.ny + 1);
  const float dt = k ? (float)*dtp : 0.f;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x)
    lf_face<SOLVER, false>(M, un, k, dt, f, nxf, nf, F, X ? X + f * mlp::KIN : nullptr, scale);
}

// FCT ratios of every cell (lf_fct_cell).
__global__ void lf_fct_kernel(UpdateArgs A, float* __restrict__ R) {
  const long long ncell = (long long)A.M.nx * A.M.ny;
  const float dt = (float)*A.dtp;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x)
    lf_fct_cell<false>(A, c, dt, R);
}

// One pass of the corrected update over every cell (lf_update_cell); the
// widening and all-plain passes return at once unless requested.
__global__ void lf_update_kernel(UpdateArgs A) {
  const long long ncell = (long long)A.M.nx * A.M.ny;
  const float dt = (float)*A.dtp;
  if (A.fixup < 0 && A.all_plain[0] == 0u) return;
  if (A.fixup > 0 && A.all_plain[1] == 0u) return;  // nothing to widen
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x)
    lf_update_cell<false>(A, c, dt);
}

// Training targets: add weight * (F(U) + F(U + dt K)) / 2, averaged over the
// `s` fine faces that make up each coarse face, to acc[axis][v][J][I] (double).
// Coarse x face (I, J) is the face between coarse cells (I - 1, J) and (I, J).
template <int SOLVER>
__global__ void face_flux_accumulate_kernel(Mesh2 M, const float* __restrict__ un, const float* __restrict__ k,
                                            const double* __restrict__ dtp, int s, double weight,
                                            double* __restrict__ acc) {
  const int ncx = M.nx / s, ncy = M.ny / s;
  const long long nc = (long long)ncx * ncy;
  const float dt = (float)*dtp;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < 2 * nc; f += (long long)gridDim.x * blockDim.x) {
    const int axis = (int)(f / nc);
    const long long r = f - axis * nc;
    const int I = (int)(r % ncx), J = (int)(r / ncx);
    double sum[4] = {0, 0, 0, 0};
    for (int q = 0; q < s; ++q) {
      for (int st = 0; st < 2; ++st) {
        const float* kk = st ? k : nullptr;
        float w[4][4], Fl[4];
        if (axis == 0) {
          const int i = s * I, j = s * J + q;
#pragma unroll
          for (int c = 0; c < 4; ++c) cell_prim(M, un, kk, dt, i - 2 + c, j, w[c]);
          plain_face_flux<0, SOLVER>(M, w, i - 1, Fl);
        } else {
          const int i = s * I + q, j = s * J;
#pragma unroll
          for (int c = 0; c < 4; ++c) cell_prim(M, un, kk, dt, i, j - 2 + c, w[c]);
          plain_face_flux<1, SOLVER>(M, w, j - 1, Fl);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) sum[v] += (double)Fl[v];
      }
    }
    const double scale = weight * 0.5 / s;
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[((size_t)axis * 4 + v) * nc + r] += scale * sum[v];
  }
}

// Conservative restriction of a 2D FP32 state by an integer factor on a
// uniform mesh: each coarse cell holds the mean of its factor^2 fine cells.
__global__ void restrict_kernel(int nx, int ny, int s, const float* __restrict__ uf, float* __restrict__ uc) {
  const int ncx = nx / s, ncy = ny / s;
  const long long nc = (long long)ncx * ncy, nfc = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < 4 * nc; c += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(c / nc);
    const long long r = c - v * nc;
    const int I = (int)(r % ncx), J = (int)(r / ncx);
    double sum = 0.0;
    for (int b = 0; b < s; ++b)
      for (int a = 0; a < s; ++a) sum += (double)uf[v * nfc + (long long)(s * J + b) * nx + s * I + a];
    uc[c] = (float)(sum / ((double)s * s));
  }
}

// Features of the distinct faces of a periodic 2D state in compact order
// (axis, j, i): face (i, j) of axis 0 lies between cells (i-1, j) and (i, j).
__global__ void train_features_kernel(Mesh2 M, const float* __restrict__ un, __nv_bfloat16* __restrict__ X,
                                      float* __restrict__ scale) {
  const long long nc = (long long)M.nx * M.ny;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < 2 * nc; f += (long long)gridDim.x * blockDim.x) {
    const int axis = (int)(f / nc);
    const long long r = f - axis * nc;
    const int i = (int)(r % M.nx), j = (int)(r / M.nx);
    float s[6][4];
    if (axis == 0) {
#pragma unroll
      for (int c = 0; c < 6; ++c) cell_prim(M, un, nullptr, 0.f, i - 3 + c, j, s[c]);
      face_features<0>(M, s, X + f * mlp::KIN, scale + f * 4);
    } else {
#pragma unroll
      for (int c = 0; c < 6; ++c) cell_prim(M, un, nullptr, 0.f, i, j - 3 + c, s[c]);
      face_features<1>(M, s, X + f * mlp::KIN, scale + f * 4);
    }
  }
}

// Targets in the face frame: T = rot^-1(F_target - F_plain) / scale, in the
// compact face order of train_features_kernel.
__global__ void train_targets_kernel(long long nc, const double* __restrict__ ft, const double* __restrict__ fp,
                                     const float* __restrict__ scale, float* __restrict__ T) {
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < 2 * nc; f += (long long)gridDim.x * blockDim.x) {
    const int axis = (int)(f / nc);
    const long long r = f - axis * nc;
    double d[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const size_t idx = ((size_t)axis * 4 + v) * nc + r;
      d[v] = ft[idx] - fp[idx];
    }
    const double dn = axis == 0 ? d[1] : d[2], dtv = axis == 0 ? d[2] : d[1];
    const float* s = scale + f * 4;
    T[f * 4 + 0] = (float)(d[0] / s[0]);
    T[f * 4 + 1] = (float)(dn / s[1]);
    T[f * 4 + 2] = (float)(dtv / s[2]);
    T[f * 4 + 3] = (float)(d[3] / s[3]);
  }
}

// ----------------------------------------------------------------- launchers

static int blocks_for(long long n, int block = 256, int cap = 8192) {
  long long b = (n + block - 1) / block;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

cudaError_t launch_face_flux_accumulate(const Mesh2& M, int solver, const float* un, const float* k, const double* dtp,
                                        int s, double weight, double* acc, cudaStream_t st) {
  const long long n = 2LL * (M.nx / s) * (M.ny / s);
  if (solver == SOLVER_HLL) face_flux_accumulate_kernel<SOLVER_HLL><<<blocks_for(n), 256, 0, st>>>(M, un, k, dtp, s, weight, acc);
  else face_flux_accumulate_kernel<SOLVER_HLLC><<<blocks_for(n), 256, 0, st>>>(M, un, k, dtp, s, weight, acc);
  return cudaGetLastError();
}

cudaError_t launch_restrict(int nx, int ny, int s, const float* uf, float* uc, cudaStream_t st) {
  restrict_kernel<<<blocks_for(4LL * (nx / s) * (ny / s)), 256, 0, st>>>(nx, ny, s, uf, uc);
  return cudaGetLastError();
}

}  // namespace gh

using namespace gh;

// ================================================================ MLP C API

namespace {

int mlp_grad_impl(const float* P, const void* X, const float* T, long long n, float* grad, float* loss, float* Pupd,
                  float* m, float* v, int step, float lr, cudaStream_t st) {
  if (n < 1) return fail(GENASIS_EINVAL, "mlp: n must be >= 1");
  static bool attr_set = false;
  if (!attr_set) {
    GH_CK(cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem)));
    attr_set = true;
  }
  int dev = 0, sms = 0;
  GH_CK(cudaGetDevice(&dev));
  GH_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  long long iters = (n + TS - 1) / TS;
  int nblk = (int)(iters < (long long)sms ? iters : (long long)sms);
  float* part = nullptr;
  float* part_loss = nullptr;
  GH_CK(cudaMallocAsync((void**)&part, (size_t)nblk * mlp::NPARAM * sizeof(float), st));
  GH_CK(cudaMallocAsync((void**)&part_loss, (size_t)nblk * sizeof(float), st));
  const float inv = 1.0f / (float)(4.0 * (double)n);
  mlp_train_kernel<<<nblk, 256, sizeof(TrainSmem), st>>>(P, (const __nv_bfloat16*)X, T, n, inv, part, part_loss);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    mlp_reduce_adam_kernel<<<(mlp::NPARAM + 255) / 256, 256, 0, st>>>(part, part_loss, nblk, grad, loss, Pupd, m, v, step,
                                                                       lr, 0.9f, 0.999f, 1e-8f);
    e = cudaGetLastError();
  }
  cudaFreeAsync(part, st);
  cudaFreeAsync(part_loss, st);
  GH_CK(e);
  return GENASIS_OK;
}

}  // namespace

struct genasis_mlp_opt {
  float* P = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* loss = nullptr;
  int step = 0;
  cudaStream_t stream = nullptr;
};

extern "C" {

int genasis_mlp_param_count(void) { return mlp::NPARAM; }

int genasis_mlp_forward(const float* params, const void* X, long long n, float* Y, void* stream) {
  if (!params || !X || !Y || n < 0) return fail(GENASIS_EINVAL, "mlp_forward: bad argument");
  if (!is_device_ptr(params) || !is_device_ptr(X) || !is_device_ptr(Y))
    return fail(GENASIS_EINVAL, "mlp_forward: params, X and Y must be device pointers");
  if (((uintptr_t)X & 15u) || ((uintptr_t)Y & 15u))
    return fail(GENASIS_EINVAL, "mlp_forward: X and Y must be 16-byte aligned (rows are moved as 16-byte vectors)");
  if (n == 0) return GENASIS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  mlp::InferWeights* W = nullptr;
  GH_CK(cudaMallocAsync((void**)&W, sizeof(mlp::InferWeights), st));
  mlp_pack_kernel<<<1, 256, 0, st>>>(params, W);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_mlp_infer(W, (const __nv_bfloat16*)X, n, Y, nullptr, false, st);
  cudaFreeAsync(W, st);
  GH_CK(e);
  return GENASIS_OK;
}

int genasis_mlp_gradient(const float* params, const void* X, const float* T, long long n, float* grad, float* loss,
                         void* stream) {
  if (!params || !X || !T || !grad) return fail(GENASIS_EINVAL, "mlp_gradient: NULL argument");
  if (!is_device_ptr(params) || !is_device_ptr(X) || !is_device_ptr(T) || !is_device_ptr(grad) ||
      (loss && !is_device_ptr(loss)))
    return fail(GENASIS_EINVAL, "mlp_gradient: all pointers must be device pointers");
  return mlp_grad_impl(params, X, T, n, grad, loss, nullptr, nullptr, nullptr, 0, 0.f, (cudaStream_t)stream);
}

int genasis_mlp_opt_create(const float* params, void* stream, genasis_mlp_opt_t* out) {
  if (!params || !out) return fail(GENASIS_EINVAL, "mlp_opt_create: NULL argument");
  genasis_mlp_opt* o = new genasis_mlp_opt();
  o->stream = (cudaStream_t)stream;
  const size_t bytes = mlp::NPARAM * sizeof(float);
  cudaError_t e = cudaMalloc(&o->P, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&o->m, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&o->v, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&o->loss, sizeof(float));
  if (e == cudaSuccess) e = cudaMemsetAsync(o->m, 0, bytes, o->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(o->v, 0, bytes, o->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(o->P, params, bytes, is_device_ptr(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        o->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(o->stream);
  if (e != cudaSuccess) {
    cudaFree(o->P);
    cudaFree(o->m);
    cudaFree(o->v);
    cudaFree(o->loss);
    delete o;
    return fail(e == cudaErrorMemoryAllocation ? GENASIS_ENOMEM : GENASIS_ECUDA, "mlp_opt_create: %s",
                cudaGetErrorString(e));
  }
  *out = o;
  return GENASIS_OK;
}

int genasis_mlp_opt_destroy(genasis_mlp_opt_t o) {
  if (!o) return GENASIS_OK;
  if (o->stream) cudaStreamSynchronize(o->stream);
  cudaFree(o->P);
  cudaFree(o->m);
  cudaFree(o->v);
  cudaFree(o->loss);
  delete o;
  return GENASIS_OK;
}

int genasis_mlp_opt_step(genasis_mlp_opt_t o, const void* X, const float* T, long long n, float lr, float* loss_out) {
  if (!o || !X || !T) return fail(GENASIS_EINVAL, "mlp_opt_step: NULL argument");
  if (!is_device_ptr(X) || !is_device_ptr(T)) return fail(GENASIS_EINVAL, "mlp_opt_step: X and T must be device pointers");
  if (!(lr > 0.f)) return fail(GENASIS_EINVAL, "mlp_opt_step: lr must be > 0");
  o->step += 1;
  int rc = mlp_grad_impl(o->P, X, T, n, nullptr, o->loss, o->P, o->m, o->v, o->step, lr, o->stream);
  if (rc) return rc;
  if (loss_out) {
    float l = 0.f;
    GH_CK(cudaMemcpyAsync(&l, o->loss, sizeof(float), cudaMemcpyDeviceToHost, o->stream));
    GH_CK(cudaStreamSynchronize(o->stream));
    *loss_out = l / (float)(4.0 * (double)n);
  }
  return GENASIS_OK;
}

int genasis_mlp_opt_get_params(genasis_mlp_opt_t o, float* params) {
  if (!o || !params) return fail(GENASIS_EINVAL, "mlp_opt_get_params: NULL argument");
  GH_CK(cudaMemcpyAsync(params, o->P, mlp::NPARAM * sizeof(float),
                        is_device_ptr(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, o->stream));
  GH_CK(cudaStreamSynchronize(o->stream));
  return GENASIS_OK;
}

}  // extern "C"

// ===================================================== learned solver handle

struct genasis_learned {
  Mesh2 M{};
  int solver = 1;
  size_t ncell = 0;
  long long nf = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* U[2] = {nullptr, nullptr};
  int cur = 0;
  float* K = nullptr;
  Geo<float>* geo[2] = {nullptr, nullptr};
  float* iw[2] = {nullptr, nullptr};
  double* wd[2] = {nullptr, nullptr};
  float* F = nullptr;
  __nv_bfloat16* X = nullptr;
  float* scale = nullptr;
  float* dY = nullptr;
  unsigned char* flag[2] = {nullptr, nullptr};
  float* params = nullptr;
  mlp::InferWeights* wimg = nullptr;  // BF16 image of params for inference
  bool corrected = false;
  float ylim = INFINITY;
  bool fct = true;
  float* R = nullptr;
  double* scal = nullptr;
  double* part_speed = nullptr;
  unsigned* status = nullptr;
  unsigned long long* nfallback = nullptr;
  unsigned* all_plain = nullptr;
  int one_launch = 1;           // GENASIS_OPT_ONE_LAUNCH
  int mlp_tc = 0;               // GENASIS_OPT_MLP_TCGEN05
  int adv_grid[2] = {-1, -1};   // CTAs of the one-launch advance per MLP engine (0: not available; -1: not yet asked)
  unsigned* adv = nullptr;      // its barrier and all-plain words, then (at 256 B) one double per CTA
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int g_nsteps = -1;
  double g_cfl = 0, g_tend = 0;
  bool g_corr = false;
};

namespace {

constexpr int kFallbackPasses = 3;

int learned_free(genasis_learned* l) {
  if (l->stream) cudaStreamSynchronize(l->stream);
  for (int b = 0; b < 2; ++b) {
    if (l->graph[b]) cudaGraphExecDestroy(l->graph[b]);
    cudaFree(l->U[b]);
    cudaFree(l->geo[b]);
    cudaFree(l->iw[b]);
    cudaFree(l->wd[b]);
  }
  for (void* p : {(void*)l->K, (void*)l->F, (void*)l->X, (void*)l->scale, (void*)l->dY, (void*)l->flag[0],
                  (void*)l->flag[1], (void*)l->params, (void*)l->scal, (void*)l->part_speed, (void*)l->status,
                  (void*)l->nfallback, (void*)l->all_plain, (void*)l->R, (void*)l->wimg, (void*)l->adv})
    cudaFree(p);
  if (l->own_stream && l->stream) cudaStreamDestroy(l->stream);
  delete l;
  return GENASIS_OK;
}

void drop_graphs(genasis_learned* l) {
  for (int b = 0; b < 2; ++b)
    if (l->graph[b]) {
      cudaGraphExecDestroy(l->graph[b]);
      l->graph[b] = nullptr;
    }
}

constexpr int kAdvanceMaxGrid = 1024;  // part_speed holds 1024 partials
constexpr size_t kAdvanceBytes = 256 + kAdvanceMaxGrid * sizeof(double);

bool one_launch_usable(genasis_learned* l) {
  if (!l->one_launch) return false;
  int& grid = l->adv_grid[l->mlp_tc];
  if (grid < 0) grid = learned_advance_max_grid(l->solver, l->mlp_tc != 0);
  return grid > 0;
}

// nsteps corrected RK2 steps in one cooperative launch (learned_advance.cu),
// dt by the finalize rule `mode` (FIN_CFL: cfl * dt_CFL clamped at t_end > 0;
// FIN_FIXED: fixed_dt).  Needs one_launch_usable(l).
int enqueue_one_launch(genasis_learned* l, int nsteps, int mode, double cfl, double fixed_dt, double t_end) {
  const long long threads = lf_advance_threads(l->mlp_tc != 0);
  const long long tiles = (l->nf + threads - 1) / threads;
  const int max_grid = l->adv_grid[l->mlp_tc];
  long long grid = max_grid < tiles ? max_grid : tiles;
  if (grid > kAdvanceMaxGrid) grid = kAdvanceMaxGrid;
  if (!l->adv) GH_CK(cudaMalloc((void**)&l->adv, kAdvanceBytes));
  // barrier, all-plain and speed words start at zero in every launch (even after one that gave up)
  GH_CK(cudaMemsetAsync(l->adv, 0, 12 * sizeof(unsigned), l->stream));
  LfAdvanceArgs P;
  memset(&P, 0, sizeof(P));
  P.M = l->M;
  P.R.ncell = l->ncell;
  P.R.n[0] = l->M.nx;
  P.R.n[1] = l->M.ny;
  P.R.n[2] = 1;
  P.R.gamma = l->M.gamma;
  P.R.iw[0] = l->iw[0];
  P.R.iw[1] = l->iw[1];
  P.R.wd[0] = l->wd[0];
  P.R.wd[1] = l->wd[1];
  P.R.part_speed = l->part_speed;
  P.R.status = l->status;
  P.R.nblk = (int)grid;
  P.Fa.part_speed = l->part_speed;
  P.Fa.nblk = (int)grid;
  P.Fa.nv = 4;
  P.Fa.mode = mode;
  P.Fa.cfl = cfl;
  P.Fa.fixed_dt = fixed_dt;
  P.Fa.t_end = t_end;
  P.Fa.scal = l->scal;
  P.Fa.status = l->status;
  P.U[0] = (float*)l->U[l->cur];
  P.U[1] = (float*)l->U[1 - l->cur];
  P.K = l->K;
  P.F = l->F;
  P.dY = l->dY;
  P.scale = l->scale;
  P.Rfct = l->R;
  P.flag[0] = l->flag[0];
  P.flag[1] = l->flag[1];
  P.W = l->corrected ? l->wimg : nullptr;
  P.mlp_tc = l->mlp_tc;
  P.fct = l->fct ? 1 : 0;
  P.ylim = l->ylim;
  P.nfallback = l->nfallback;
  P.status = l->status;
  P.sync = l->adv;
  P.dts = (double*)((char*)l->adv + 256);
  P.nsteps = nsteps;
  GH_CK(launch_learned_advance(P, l->solver, (int)grid, l->stream));
  l->cur ^= nsteps & 1;
  return GENASIS_OK;
}

// One corrected RK2 step: dt = cfl * dt_CFL (clamped at t_end > 0), or the
// given dt when fixed_dt > 0.
int learned_enqueue_step(genasis_learned* l, double cfl, double t_end, double fixed_dt = 0.0) {
  cudaStream_t st = l->stream;
  // CFL time step from U^n (Eq. courantTimeStep)
  ReduceArgs<float> R;
  memset(&R, 0, sizeof(R));
  R.ncell = l->ncell;
  R.n[0] = l->M.nx;
  R.n[1] = l->M.ny;
  R.n[2] = 1;
  R.iw[0] = l->iw[0];
  R.iw[1] = l->iw[1];
  R.wd[0] = l->wd[0];
  R.wd[1] = l->wd[1];
  R.gamma = l->M.gamma;
  R.U = (const float*)l->U[l->cur];
  R.part_speed = l->part_speed;
  R.status = l->status;
  R.nblk = blocks_for((long long)l->ncell, 256, 1024);
  GH_CK(launch_speed<float>(2, R, st));
  FinalizeArgs Fa;
  memset(&Fa, 0, sizeof(Fa));
  Fa.part_speed = l->part_speed;
  Fa.nblk = R.nblk;
  Fa.nv = 4;
  Fa.mode = fixed_dt > 0.0 ? FIN_FIXED : FIN_CFL;
  Fa.cfl = cfl;
  Fa.fixed_dt = fixed_dt;
  Fa.t_end = t_end;
  Fa.scal = l->scal;
  Fa.status = l->status;
  GH_CK(launch_finalize(Fa, st));
  const float* un = (const float*)l->U[l->cur];
  for (int stage = 1; stage <= 2; ++stage) {
    const float* kin = stage == 2 ? l->K : nullptr;
    const int nb = blocks_for(l->nf);
    if (l->solver == SOLVER_HLL)
      lf_faces_kernel<SOLVER_HLL><<<nb, 256, 0, st>>>(l->M, un, kin, l->scal + SCAL_DT, l->F, l->corrected ? l->X : nullptr, l->scale);
    else
      lf_faces_kernel<SOLVER_HLLC><<<nb, 256, 0, st>>>(l->M, un, kin, l->scal + SCAL_DT, l->F, l->corrected ? l->X : nullptr, l->scale);
    GH_CK(cudaGetLastError());
    if (l->corrected) {
      GH_CK(launch_mlp_infer(l->wimg, l->X, l->nf, l->dY, l->status, l->mlp_tc != 0, st));
    }
    UpdateArgs A;
    A.M = l->M;
    A.un = un;
    A.k1 = l->K;
    A.dtp = l->scal + SCAL_DT;
    A.F = l->F;
    A.dY = l->corrected ? l->dY : nullptr;
    A.scale = l->scale;
    A.out = stage == 1 ? l->K : (float*)l->U[1 - l->cur];
    A.flag = l->flag[1];
    A.flag_out = l->flag[0];
    A.nfallback = l->nfallback;
    A.status = l->status;
    A.stage = stage;
    A.fixup = 0;
    A.last = 0;
    A.all_plain = l->all_plain;
    A.ylim = l->ylim;
    A.R = nullptr;
    const int nc = blocks_for((long long)l->ncell);
    if (l->corrected && l->fct) {
      lf_fct_kernel<<<nc, 256, 0, st>>>(A, l->R);
      GH_CK(cudaGetLastError());
      A.R = l->R;
    }
    lf_update_kernel<<<nc, 256, 0, st>>>(A);
    GH_CK(cudaGetLastError());
    if (l->corrected) {
      // widening passes: cells touching flagged cells use the plain flux on
      // those faces (both sides of a face decide alike, so the update stays
      // conservative); flags only grow
      for (int pass = 1; pass <= kFallbackPasses; ++pass) {
        A.flag = l->flag[(pass + 1) & 1];
        A.flag_out = l->flag[pass & 1];
        A.fixup = pass;
        A.last = pass == kFallbackPasses;
        lf_update_kernel<<<nc, 256, 0, st>>>(A);
        GH_CK(cudaGetLastError());
      }
      // if widening did not clear every failure, the whole stage takes the plain flux
      A.fixup = -1;
      lf_update_kernel<<<nc, 256, 0, st>>>(A);
      GH_CK(cudaGetLastError());
      GH_CK(cudaMemsetAsync(l->all_plain, 0, 2 * sizeof(unsigned), st));
    }
  }
  l->cur = 1 - l->cur;
  return GENASIS_OK;
}

}  // namespace

namespace gh {

__global__ void or_status_kernel(unsigned* dst, const unsigned* src) { *dst |= *src; }

int learned_run_on(genasis_learned_t l, void* U, double* t, unsigned* status, int nsteps, double cfl, double t_end,
                   double dt_fixed) {
  const size_t bytes = l->ncell * 4 * sizeof(float);
  GH_CK(cudaMemcpyAsync(l->U[l->cur], U, bytes, cudaMemcpyDeviceToDevice, l->stream));
  GH_CK(cudaMemcpyAsync(l->scal + SCAL_T, t, sizeof(double), cudaMemcpyDeviceToDevice, l->stream));
  const int rc = nsteps > 0 ? genasis_learned_advance(l, nsteps, cfl, t_end, nullptr) : genasis_learned_step(l, dt_fixed);
  if (rc) return rc;
  GH_CK(cudaMemcpyAsync(U, l->U[l->cur], bytes, cudaMemcpyDeviceToDevice, l->stream));
  GH_CK(cudaMemcpyAsync(t, l->scal + SCAL_T, sizeof(double), cudaMemcpyDeviceToDevice, l->stream));
  or_status_kernel<<<1, 1, 0, l->stream>>>(status, l->status);
  GH_CK(cudaGetLastError());
  return GENASIS_OK;
}

}  // namespace gh

extern "C" {

int genasis_learned_create(const genasis_hydro_desc* d, genasis_learned_t* out) {
  if (!d || !out) return fail(GENASIS_EINVAL, "learned_create: NULL argument");
  *out = nullptr;
  if (d->ndim != 2) return fail(GENASIS_EINVAL, "learned_create: the learned correction is 2D (ndim = 2)");
  if (d->precision != GENASIS_FP32_MIXED) return fail(GENASIS_EINVAL, "learned_create: precision must be GENASIS_FP32_MIXED");
  if (d->solver != GENASIS_HLL && d->solver != GENASIS_HLLC) return fail(GENASIS_EINVAL, "learned_create: bad solver");
  if (!(d->gamma > 1.0) || !(d->theta >= 1.0 && d->theta <= 2.0)) return fail(GENASIS_EINVAL, "learned_create: bad gamma or theta");
  for (int q = 0; q < 2; ++q) {
    if (d->n[q] < 6) return fail(GENASIS_EINVAL, "learned_create: n[%d] must be >= 6", q);
    if (!d->widths[q]) return fail(GENASIS_EINVAL, "learned_create: widths[%d] is NULL", q);
    for (int i = 0; i < d->n[q]; ++i)
      if (!(d->widths[q][i] > 0.0) || !isfinite(d->widths[q][i])) return fail(GENASIS_EINVAL, "learned_create: bad width");
    if (d->bc_lo[q] < 0 || d->bc_lo[q] > 2 || d->bc_hi[q] < 0 || d->bc_hi[q] > 2) return fail(GENASIS_EINVAL, "learned_create: bad boundary code");
    if ((d->bc_lo[q] == GENASIS_BC_PERIODIC) != (d->bc_hi[q] == GENASIS_BC_PERIODIC))
      return fail(GENASIS_EINVAL, "learned_create: periodic must be set on both ends");
  }
  genasis_learned* l = new genasis_learned();
  l->solver = d->solver;
  l->M.nx = d->n[0];
  l->M.ny = d->n[1];
  for (int q = 0; q < 2; ++q) {
    l->M.bc_lo[q] = d->bc_lo[q];
    l->M.bc_hi[q] = d->bc_hi[q];
  }
  l->M.gamma = (float)d->gamma;
  l->M.gm1 = (float)(d->gamma - 1.0);
  l->ncell = (size_t)l->M.nx * l->M.ny;
  l->nf = (long long)(l->M.nx + 1) * l->M.ny + (long long)l->M.nx * (l->M.ny + 1);
#define LCK(call)                                                                                   \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      int code_ = fail(e_ == cudaErrorMemoryAllocation ? GENASIS_ENOMEM : GENASIS_ECUDA, "%s: %s", #call, \
                       cudaGetErrorString(e_));                                                     \
      learned_free(l);                                                                              \
      return code_;                                                                                 \
    }                                                                                               \
  } while (0)
  if (d->stream) {
    l->stream = (cudaStream_t)d->stream;
  } else {
    LCK(cudaStreamCreateWithFlags(&l->stream, cudaStreamNonBlocking));
    l->own_stream = true;
  }
  const size_t sbytes = l->ncell * 4 * sizeof(float);
  for (int b = 0; b < 2; ++b) {
    LCK(cudaMalloc(&l->U[b], sbytes));
    LCK(cudaMemsetAsync(l->U[b], 0, sbytes, l->stream));
  }
  LCK(cudaMalloc((void**)&l->K, sbytes));
  LCK(cudaMalloc((void**)&l->F, (size_t)l->nf * 4 * sizeof(float)));
  LCK(cudaMalloc((void**)&l->X, (size_t)l->nf * mlp::KIN * sizeof(__nv_bfloat16)));
  LCK(cudaMalloc((void**)&l->scale, (size_t)l->nf * 4 * sizeof(float)));
  LCK(cudaMalloc((void**)&l->dY, (size_t)l->nf * 4 * sizeof(float)));
  for (int b = 0; b < 2; ++b) {
    LCK(cudaMalloc((void**)&l->flag[b], l->ncell));
    LCK(cudaMemsetAsync(l->flag[b], 0, l->ncell, l->stream));
  }
  LCK(cudaMalloc((void**)&l->params, mlp::NPARAM * sizeof(float)));
  LCK(cudaMalloc((void**)&l->scal, SCAL_ALLOC * sizeof(double)));
  LCK(cudaMemsetAsync(l->scal, 0, SCAL_ALLOC * sizeof(double), l->stream));
  LCK(cudaMalloc((void**)&l->part_speed, 1024 * sizeof(double)));
  LCK(cudaMalloc((void**)&l->status, sizeof(unsigned)));
  LCK(cudaMemsetAsync(l->status, 0, sizeof(unsigned), l->stream));
  LCK(cudaMalloc((void**)&l->R, l->ncell * 8 * sizeof(float)));
  LCK(cudaMalloc((void**)&l->wimg, sizeof(mlp::InferWeights)));
  LCK(cudaMalloc((void**)&l->all_plain, 2 * sizeof(unsigned)));
  LCK(cudaMemsetAsync(l->all_plain, 0, 2 * sizeof(unsigned), l->stream));
  LCK(cudaMalloc((void**)&l->nfallback, sizeof(unsigned long long)));
  LCK(cudaMemsetAsync(l->nfallback, 0, sizeof(unsigned long long), l->stream));
  for (int q = 0; q < 2; ++q) {
    std::vector<Geo<float>> geo;
    std::vector<float> iw;
    append_geometry<float>(extended_widths(d->widths[q], d->n[q], d->bc_lo[q], d->bc_hi[q]), d->theta, geo, iw);
    LCK(cudaMalloc((void**)&l->geo[q], geo.size() * sizeof(Geo<float>)));
    LCK(cudaMalloc((void**)&l->iw[q], iw.size() * sizeof(float)));
    LCK(cudaMalloc((void**)&l->wd[q], d->n[q] * sizeof(double)));
    LCK(cudaMemcpy(l->geo[q], geo.data(), geo.size() * sizeof(Geo<float>), cudaMemcpyHostToDevice));
    LCK(cudaMemcpy(l->iw[q], iw.data(), iw.size() * sizeof(float), cudaMemcpyHostToDevice));
    LCK(cudaMemcpy(l->wd[q], d->widths[q], d->n[q] * sizeof(double), cudaMemcpyHostToDevice));
    l->M.geo[q] = l->geo[q];
    l->M.iw[q] = l->iw[q];
  }
  LCK(cudaStreamSynchronize(l->stream));
#undef LCK
  *out = l;
  return GENASIS_OK;
}

int genasis_learned_destroy(genasis_learned_t l) {
  if (!l) return GENASIS_OK;
  return learned_free(l);
}

int genasis_learned_set_params(genasis_learned_t l, const float* params) {
  if (!l) return fail(GENASIS_EINVAL, "NULL handle");
  drop_graphs(l);
  if (!params) {
    l->corrected = false;
    return GENASIS_OK;
  }
  GH_CK(cudaMemcpyAsync(l->params, params, mlp::NPARAM * sizeof(float),
                        is_device_ptr(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, l->stream));
  mlp_pack_kernel<<<1, 256, 0, l->stream>>>(l->params, l->wimg);
  GH_CK(cudaGetLastError());
  GH_CK(cudaStreamSynchronize(l->stream));
  l->corrected = true;
  return GENASIS_OK;
}

int genasis_learned_set_fct(genasis_learned_t l, int enabled) {
  if (!l || (enabled != 0 && enabled != 1)) return fail(GENASIS_EINVAL, "learned_set_fct: bad argument");
  l->fct = enabled == 1;
  drop_graphs(l);
  return GENASIS_OK;
}

int genasis_learned_set_limit(genasis_learned_t l, float ylim) {
  if (!l) return fail(GENASIS_EINVAL, "NULL handle");
  if (!(ylim >= 0.0f)) return fail(GENASIS_EINVAL, "learned_set_limit: limit must be >= 0 (INFINITY: none)");
  l->ylim = ylim;
  drop_graphs(l);
  return GENASIS_OK;
}

int genasis_learned_set_primitive(genasis_learned_t l, const double* rho, const double* vel, const double* p) {
  if (!l || !rho || !vel || !p) return fail(GENASIS_EINVAL, "NULL argument");
  const double* src[3] = {rho, vel, p};
  const size_t cnt[3] = {l->ncell, 2 * l->ncell, l->ncell};
  double* tmp[3] = {nullptr, nullptr, nullptr};
  const double* use[3];
  int rc = GENASIS_OK;
  for (int a = 0; a < 3; ++a) {
    use[a] = src[a];
    if (is_device_ptr(src[a])) continue;
    cudaError_t e = cudaMallocAsync((void**)&tmp[a], cnt[a] * sizeof(double), l->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp[a], src[a], cnt[a] * sizeof(double), cudaMemcpyHostToDevice, l->stream);
    if (e != cudaSuccess) rc = fail(GENASIS_ECUDA, "staging primitives: %s", cudaGetErrorString(e));
    use[a] = tmp[a];
  }
  if (!rc) {
    cudaError_t e = launch_init_from_primitive<float>(2, l->ncell, (double)l->M.gamma, use[0], use[1], use[2],
                                                      (float*)l->U[l->cur], l->stream);
    if (e != cudaSuccess) rc = fail(GENASIS_ECUDA, "init kernel: %s", cudaGetErrorString(e));
  }
  for (int a = 0; a < 3; ++a)
    if (tmp[a]) cudaFreeAsync(tmp[a], l->stream);
  if (rc) return rc;
  GH_CK(cudaMemsetAsync(l->scal + SCAL_T, 0, sizeof(double), l->stream));
  GH_CK(cudaStreamSynchronize(l->stream));
  return GENASIS_OK;
}

int genasis_learned_set_conserved(genasis_learned_t l, const float* U) {
  if (!l || !U) return fail(GENASIS_EINVAL, "NULL argument");
  GH_CK(cudaMemcpyAsync(l->U[l->cur], U, l->ncell * 4 * sizeof(float),
                        is_device_ptr(U) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, l->stream));
  GH_CK(cudaStreamSynchronize(l->stream));
  return GENASIS_OK;
}

int genasis_learned_get_conserved(genasis_learned_t l, float* U) {
  if (!l || !U) return fail(GENASIS_EINVAL, "NULL argument");
  GH_CK(cudaMemcpyAsync(U, l->U[l->cur], l->ncell * 4 * sizeof(float),
                        is_device_ptr(U) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, l->stream));
  unsigned st = 0;
  GH_CK(cudaMemcpyAsync(&st, l->status, sizeof(unsigned), cudaMemcpyDeviceToHost, l->stream));
  GH_CK(cudaStreamSynchronize(l->stream));
  if (st & STATUS_TIMEOUT) return fail(GENASIS_ETIMEOUT, "a bounded device wait gave up");
  if (st & STATUS_NONPHYS) return fail(GENASIS_ENONPHYS, "non-physical state (rho <= 0, p <= 0 or NaN) on the device");
  return GENASIS_OK;
}

int genasis_learned_advance(genasis_learned_t l, int nsteps, double cfl, double t_end, double* t_out) {
  if (!l) return fail(GENASIS_EINVAL, "NULL handle");
  if (nsteps < 0 || !(cfl > 0.0)) return fail(GENASIS_EINVAL, "learned_advance: bad nsteps or cfl");
  if (nsteps > 0 && one_launch_usable(l)) {
    const int rc = enqueue_one_launch(l, nsteps, FIN_CFL, cfl, 0.0, t_end);
    if (rc) return rc;
  } else if (nsteps > 0) {
    if (l->g_nsteps != nsteps || l->g_cfl != cfl || l->g_tend != t_end || l->g_corr != l->corrected) {
      drop_graphs(l);
      l->g_nsteps = nsteps;
      l->g_cfl = cfl;
      l->g_tend = t_end;
      l->g_corr = l->corrected;
    }
    const int cur0 = l->cur;
    if (!l->graph[cur0]) {
      cudaGraph_t g;
      GH_CK(cudaStreamBeginCapture(l->stream, cudaStreamCaptureModeThreadLocal));
      int rc = GENASIS_OK;
      for (int s = 0; s < nsteps && !rc; ++s) rc = learned_enqueue_step(l, cfl, t_end);
      cudaError_t e = cudaStreamEndCapture(l->stream, &g);
      l->cur = cur0;
      if (rc) {
        if (e == cudaSuccess) cudaGraphDestroy(g);
        return rc;
      }
      GH_CK(e);
      e = cudaGraphInstantiate(&l->graph[cur0], g, 0);
      cudaGraphDestroy(g);
      GH_CK(e);
    }
    GH_CK(cudaGraphLaunch(l->graph[cur0], l->stream));
    l->cur = cur0 ^ (nsteps & 1);
  }
  if (t_out) {
    GH_CK(cudaMemcpyAsync(t_out, l->scal + SCAL_T, sizeof(double), cudaMemcpyDeviceToHost, l->stream));
    unsigned st = 0;
    GH_CK(cudaMemcpyAsync(&st, l->status, sizeof(unsigned), cudaMemcpyDeviceToHost, l->stream));
    GH_CK(cudaStreamSynchronize(l->stream));
    if (st & STATUS_TIMEOUT) return fail(GENASIS_ETIMEOUT, "a bounded device wait gave up");
    if (st & STATUS_NONPHYS) return fail(GENASIS_ENONPHYS, "non-physical state even with the plain flux");
  }
  return GENASIS_OK;
}

int genasis_learned_step(genasis_learned_t l, double dt) {
  if (!l) return fail(GENASIS_EINVAL, "NULL handle");
  if (!(dt > 0.0) || !(dt < INFINITY)) return fail(GENASIS_EINVAL, "learned_step: dt must be finite and > 0");
  if (one_launch_usable(l)) return enqueue_one_launch(l, 1, FIN_FIXED, 1.0, dt, 0.0);
  return learned_enqueue_step(l, 1.0, 0.0, dt);
}

int genasis_learned_set_option(genasis_learned_t l, int option, int value) {
  if (!l) return fail(GENASIS_EINVAL, "NULL handle");
  if (option != GENASIS_OPT_ONE_LAUNCH && option != GENASIS_OPT_MLP_TCGEN05)
    return fail(GENASIS_EINVAL, "learned_set_option: unknown option %d", option);
  if (value != 0 && value != 1) return fail(GENASIS_EINVAL, "learned_set_option: option %d takes 0 or 1", option);
  if (option == GENASIS_OPT_ONE_LAUNCH) {
    l->one_launch = value;
  } else if (l->mlp_tc != value) {
    l->mlp_tc = value;
    drop_graphs(l);
  }
  return GENASIS_OK;
}

int genasis_learned_launches_per_step(genasis_learned_t l) {
  if (!l) return fail(GENASIS_EINVAL, "NULL handle");
  if (one_launch_usable(l)) return 1;  // one launch covers all the steps of a call
  // CFL speed and finalize; per stage the faces and the update, with a
  // network also the inference, the 3 widening passes, the all-plain pass
  // and (limiting) the FCT ratios
  const int per_stage = l->corrected ? (l->fct ? 8 : 7) : 2;
  return 2 + 2 * per_stage;
}

int genasis_learned_fallbacks(genasis_learned_t l, long long* cells) {
  if (!l || !cells) return fail(GENASIS_EINVAL, "NULL argument");
  unsigned long long v = 0;
  GH_CK(cudaMemcpyAsync(&v, l->nfallback, sizeof(v), cudaMemcpyDeviceToHost, l->stream));
  GH_CK(cudaStreamSynchronize(l->stream));
  *cells = (long long)v;
  return GENASIS_OK;
}

int genasis_learned_features(genasis_learned_t l, void* X, float* scale) {
  if (!l || !X || !scale) return fail(GENASIS_EINVAL, "NULL argument");
  if (!is_device_ptr(X) || !is_device_ptr(scale)) return fail(GENASIS_EINVAL, "learned_features: device pointers required");
  if (l->M.bc_lo[0] != GENASIS_BC_PERIODIC || l->M.bc_lo[1] != GENASIS_BC_PERIODIC)
    return fail(GENASIS_EINVAL, "learned_features: training features need a periodic mesh");
  train_features_kernel<<<blocks_for(2LL * l->ncell), 256, 0, l->stream>>>(l->M, (const float*)l->U[l->cur],
                                                                           (__nv_bfloat16*)X, scale);
  GH_CK(cudaGetLastError());
  GH_CK(cudaStreamSynchronize(l->stream));
  return GENASIS_OK;
}

int genasis_learned_targets(genasis_learned_t l, const double* f_target, const double* f_plain, const float* scale,
                            float* T) {
  if (!l || !f_target || !f_plain || !scale || !T) return fail(GENASIS_EINVAL, "NULL argument");
  if (!is_device_ptr(f_target) || !is_device_ptr(f_plain) || !is_device_ptr(scale) || !is_device_ptr(T))
    return fail(GENASIS_EINVAL, "learned_targets: device pointers required");
  const long long nc = (long long)l->ncell;
  train_targets_kernel<<<blocks_for(2 * nc), 256, 0, l->stream>>>(nc, f_target, f_plain, scale, T);
  GH_CK(cudaGetLastError());
  GH_CK(cudaStreamSynchronize(l->stream));
  return GENASIS_OK;
}

}  // extern "C"
