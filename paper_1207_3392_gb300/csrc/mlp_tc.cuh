// mlp_tc.cuh -- forward pass of the flux-correction network (24 -> 64 -> 64
// -> 4, SiLU, BF16 weights and activations, FP32 accumulation) on the
// 5th-generation tensor cores: tcgen05.mma with both operands in shared
// memory and the accumulator in tensor memory (TMEM).  The correction is the
// benchmark's addition to the HLLC flux of Sec. 3.2; the paper has no
// counterpart.
//
// A tile is 128 samples, one per thread of a group of four warps: the MMA
// shape is M = 128 (a TMEM lane per sample), N = 64 for the hidden layers and
// N = 16 (the output layer's 4 rows padded) for the last, K = 16 per
// instruction.  One elected thread issues the MMAs of a layer and commits them
// to an mbarrier; the group waits on it (bounded), reads its rows of the
// accumulator with tcgen05.ld, adds the bias, applies SiLU and writes the BF16
// activations back to shared memory as the next layer's A operand.
//
// Operands use the canonical no-swizzle K-major layout: 8 x 8 core matrices
// of 8 rows x 16 bytes; the core matrix next along K is 128 bytes on (the
// descriptor's leading byte offset), the next 8 rows K x 16 bytes on (its
// stride byte offset).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "mbarrier.cuh"
#include "mlp.cuh"

namespace gh {
namespace mlptc {

constexpr int M = 128;  // samples per tile
constexpr int N3 = 16;  // output layer padded to the smallest N of an M = 128 MMA
constexpr int TMEM_COLS = 128;  // per group: layers 1 and 2 in columns 0..63, layer 3 in 64..79

// Element index of (row r, column k) of a K-column operand in the core-matrix layout.
__host__ __device__ constexpr int core_idx(int r, int k, int K) {
  return (r >> 3) * (K * 8) + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

// The weights as B operands ([N][K], K-major) and the biases.  W3 comes
// first: every operand's footprint, under either reading of the two
// descriptor offsets, then stays inside this struct and the tile after it.
struct __align__(128) Weights {
  __nv_bfloat16 w3[N3 * mlp::NH];
  __nv_bfloat16 w1[mlp::NH * mlp::KIN];
  __nv_bfloat16 w2[mlp::NH * mlp::NH];
  float b1[mlp::NH], b2[mlp::NH], b3[4];
};

// The A operands of one tile.
struct __align__(128) Tile {
  __nv_bfloat16 x[M * mlp::KIN];  // features of the 128 samples
  __nv_bfloat16 h[M * mlp::NH];   // hidden activations
};

// Fill W from a prepared BF16 image (all threads of the block).
__device__ __forceinline__ void load_weights(Weights& W, const mlp::InferWeights* __restrict__ G) {
  for (int i = threadIdx.x; i < mlp::NH * mlp::KIN; i += blockDim.x) {
    const int o = i / mlp::KIN, k = i % mlp::KIN;
    W.w1[core_idx(o, k, mlp::KIN)] = G->w1[o][k];
  }
  for (int i = threadIdx.x; i < mlp::NH * mlp::NH; i += blockDim.x) {
    const int o = i / mlp::NH, k = i % mlp::NH;
    W.w2[core_idx(o, k, mlp::NH)] = G->w2[o][k];
  }
  for (int i = threadIdx.x; i < N3 * mlp::NH; i += blockDim.x) {
    const int o = i / mlp::NH, k = i % mlp::NH;
    W.w3[core_idx(o, k, mlp::NH)] = o < mlp::NOUTP ? G->w3[o][k] : __float2bfloat16(0.0f);
  }
  for (int i = threadIdx.x; i < mlp::NH; i += blockDim.x) {
    W.b1[i] = G->b1[i];
    W.b2[i] = G->b2[i];
  }
  for (int i = threadIdx.x; i < 4; i += blockDim.x) W.b3[i] = G->b3[i];
}

// Shared-memory matrix descriptor (tcgen05): start address, leading byte
// offset 128 (K direction), stride byte offset K x 16 (M/N direction),
// descriptor version 1, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t sdesc(const void* p, int K) {
  const uint32_t a = tma::smem_u32(p);
  return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)((K * 16) >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t idesc(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(accumulate)
      : "memory");
}
// Arrive on the mbarrier once the MMAs this thread issued have completed.
__device__ __forceinline__ void commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tma::smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void ld4(uint32_t taddr, float (&v)[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
// TMEM allocation by one whole warp: the address lands in *slot (shared).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tma::smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Barrier of the NTHR threads of group barrier `id` (1..15) that ORs a flag
// over them: every thread leaves with the same answer.
template <int NTHR>
__device__ __forceinline__ bool group_or(int id, bool flag) {
  unsigned out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(out)
      : "r"((unsigned)flag), "r"(id), "n"(NTHR)
      : "memory");
  return out != 0u;
}

// One layer's activations: the 64 accumulator columns of this thread's lane
// (base column col0) plus the bias, SiLU, rounded to BF16 into row t of h.
__device__ __forceinline__ void hidden_out(uint32_t taddr, const float* __restrict__ b, __nv_bfloat16* h, int t) {
#pragma unroll 1
  for (int c0 = 0; c0 < mlp::NH; c0 += 16) {
    float z[16];
    ld16(taddr + (uint32_t)c0, z);
    wait_ld();
    uint32_t p[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) p[i] = mlp::pack2(mlp::silu(z[2 * i] + b[c0 + 2 * i]), mlp::silu(z[2 * i + 1] + b[c0 + 2 * i + 1]));
    *reinterpret_cast<uint4*>(h + core_idx(t, c0, mlp::NH)) = make_uint4(p[0], p[1], p[2], p[3]);
    *reinterpret_cast<uint4*>(h + core_idx(t, c0 + 8, mlp::NH)) = make_uint4(p[4], p[5], p[6], p[7]);
  }
}

// Forward pass of the 128 samples in T.x by the 128 threads of group barrier
// `bar_id` (thread t, 0..127, owns sample row t; its warp index within the CTA
// is t / 32 modulo 4, which is the TMEM lane quarter it may read).  tmem: the
// group's TMEM_COLS columns.  y receives the row's 4 outputs.  False (on
// every thread of the group) if a wait for the tensor cores ran out; the
// group's MMAs are then no longer waited for.
__device__ __forceinline__ bool forward_tile(const Weights& W, Tile& T, unsigned long long* mbar, unsigned& phase,
                                             uint32_t tmem, int bar_id, int t, float (&y)[4]) {
  const uint32_t lane = tmem + ((uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16);
  // layer 1: D[., 0..63] = X W1^T (K = 32: two MMAs)
  tma::fence_proxy_async();
  fence_before();
  if (group_or<M>(bar_id, false)) return false;
  if (t == 0) {
    fence_after();
#pragma unroll
    for (int ks = 0; ks < mlp::KIN / 16; ++ks)
      mma(tmem, sdesc(T.x + ks * 128, mlp::KIN), sdesc(W.w1 + ks * 128, mlp::KIN), idesc(mlp::NH), ks > 0);
    commit(mbar);
  }
  bool ok = tma::mbar_wait(mbar, phase);
  phase ^= 1u;
  if (group_or<M>(bar_id, !ok)) return false;
  fence_after();
  hidden_out(lane, W.b1, T.h, t);
  // layer 2: D[., 0..63] = H1 W2^T (K = 64: four MMAs); H1 is read before
  // the next activations overwrite it (the commit's arrival covers the reads)
  tma::fence_proxy_async();
  fence_before();
  group_or<M>(bar_id, false);
  if (t == 0) {
    fence_after();
#pragma unroll
    for (int ks = 0; ks < mlp::NH / 16; ++ks)
      mma(tmem, sdesc(T.h + ks * 128, mlp::NH), sdesc(W.w2 + ks * 128, mlp::NH), idesc(mlp::NH), ks > 0);
    commit(mbar);
  }
  ok = tma::mbar_wait(mbar, phase);
  phase ^= 1u;
  if (group_or<M>(bar_id, !ok)) return false;
  fence_after();
  hidden_out(lane, W.b2, T.h, t);
  // layer 3: D[., 64..79] = H2 W3^T (N = 16, K = 64)
  tma::fence_proxy_async();
  fence_before();
  group_or<M>(bar_id, false);
  if (t == 0) {
    fence_after();
#pragma unroll
    for (int ks = 0; ks < mlp::NH / 16; ++ks)
      mma(tmem + 64u, sdesc(T.h + ks * 128, mlp::NH), sdesc(W.w3 + ks * 128, mlp::NH), idesc(N3), ks > 0);
    commit(mbar);
  }
  ok = tma::mbar_wait(mbar, phase);
  phase ^= 1u;
  if (group_or<M>(bar_id, !ok)) return false;
  fence_after();
  float o[4];
  ld4(lane + 64u, o);
  wait_ld();
#pragma unroll
  for (int i = 0; i < 4; ++i) y[i] = o[i] + W.b3[i];
  return true;
}

}  // namespace mlptc
}  // namespace gh
