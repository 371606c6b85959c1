// mlp.cuh -- the learned flux-correction network on BF16 tensor cores
// (mma.sync m16n8k16, FP32 accumulation).  The correction is not in the paper:
// it is the benchmark's addition to the HLLC flux of Sec. 3.2.
//
// Network: x (24) -> z1 = W1 x + b1 (64) -> h1 = silu(z1) -> z2 = W2 h1 + b2
// (64) -> h2 = silu(z2) -> y = W3 h2 + b3 (4).  Parameters are one FP32
// vector (W1 [64][24], b1, W2 [64][64], b2, W3 [4][64], b3; 6020 values);
// kernels stage BF16 copies (K padded 24 -> 32, outputs 4 -> 8) in shared
// memory.  Samples are BF16 rows of 32 (24 features + zeros).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gh {
namespace mlp {

constexpr int NIN = 24, KIN = 32, NH = 64, NOUT = 4, NOUTP = 8;
constexpr int OW1 = 0, OB1 = OW1 + NH * NIN, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NOUT * NH, NPARAM = OB3 + NOUT;
constexpr int PAD = 8;  // row padding (bf16) that keeps fragment loads free of bank conflicts

struct __align__(16) Weights {
  __nv_bfloat16 w1[NH][KIN + PAD];     // [out][in]
  __nv_bfloat16 w2[NH][NH + PAD];      // [out][in]
  __nv_bfloat16 w3[NOUTP][NH + PAD];   // [out][in], rows >= NOUT zero
  __nv_bfloat16 w2t[NH][NH + PAD];     // [in][out]
  __nv_bfloat16 w3t[NH][16 + PAD];     // [in][out], out >= NOUT zero
  float b1[NH], b2[NH], b3[NOUTP];
};

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// D += A (16x16, row) * B (16x8, col), BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// SiLU z sigma(z) and its derivative, with the hardware exponential and
// reciprocal (z -> -inf gives 1 + e^{-z} = inf and sigma = 0, the limit).
__device__ __forceinline__ float sigmoid(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }
__device__ __forceinline__ float silu(float z) { return z * sigmoid(z); }
__device__ __forceinline__ float dsilu(float z) {
  const float s = sigmoid(z);
  return s * (1.0f + z * (1.0f - s));
}

// The layers the forward pass reads; a BF16 image of this struct is built once
// per parameter set and copied to shared memory by each inference CTA.
struct __align__(16) InferWeights {
  __nv_bfloat16 w1[NH][KIN + PAD];
  __nv_bfloat16 w2[NH][NH + PAD];
  __nv_bfloat16 w3[NOUTP][NH + PAD];
  float b1[NH], b2[NH], b3[NOUTP];
};
static_assert(sizeof(InferWeights) % 16 == 0, "copied as 16-byte vectors");

// Fill the forward-pass layers of W (Weights or InferWeights) from the FP32
// parameter vector (all threads of the block).
template <class WT>
__device__ __forceinline__ void fill_layers(WT& W, const float* __restrict__ P) {
  for (int i = threadIdx.x; i < NH * (KIN + PAD); i += blockDim.x) {
    const int o = i / (KIN + PAD), k = i % (KIN + PAD);
    W.w1[o][k] = __float2bfloat16(k < NIN ? P[OW1 + o * NIN + k] : 0.0f);
  }
  for (int i = threadIdx.x; i < NH * (NH + PAD); i += blockDim.x) {
    const int o = i / (NH + PAD), k = i % (NH + PAD);
    W.w2[o][k] = __float2bfloat16(k < NH ? P[OW2 + o * NH + k] : 0.0f);
  }
  for (int i = threadIdx.x; i < NOUTP * (NH + PAD); i += blockDim.x) {
    const int o = i / (NH + PAD), k = i % (NH + PAD);
    W.w3[o][k] = __float2bfloat16(o < NOUT && k < NH ? P[OW3 + o * NH + k] : 0.0f);
  }
  for (int i = threadIdx.x; i < NH; i += blockDim.x) {
    W.b1[i] = P[OB1 + i];
    W.b2[i] = P[OB2 + i];
  }
  for (int i = threadIdx.x; i < NOUTP; i += blockDim.x) W.b3[i] = i < NOUT ? P[OB3 + i] : 0.0f;
}

// Stage all BF16 weights, with the transposed copies the backward pass needs.
__device__ __forceinline__ void load_weights(Weights& W, const float* __restrict__ P) {
  fill_layers(W, P);
  for (int i = threadIdx.x; i < NH * (NH + PAD); i += blockDim.x) {
    const int o = i / (NH + PAD), k = i % (NH + PAD);
    W.w2t[o][k] = __float2bfloat16(k < NH ? P[OW2 + k * NH + o] : 0.0f);
  }
  for (int i = threadIdx.x; i < NH * (16 + PAD); i += blockDim.x) {
    const int j = i / (16 + PAD), o = i % (16 + PAD);
    W.w3t[j][o] = __float2bfloat16(o < NOUT ? P[OW3 + o * NH + j] : 0.0f);
  }
}

// Copy a prepared InferWeights image into shared memory (all threads).
__device__ __forceinline__ void copy_weights(InferWeights& W, const InferWeights* __restrict__ G) {
  const uint4* src = reinterpret_cast<const uint4*>(G);
  uint4* dst = reinterpret_cast<uint4*>(&W);
  for (int i = threadIdx.x; i < (int)(sizeof(InferWeights) / 16); i += blockDim.x) dst[i] = __ldg(src + i);
}

// Forward pass of one warp over 16 samples whose rows start at X (row stride
// 32, rows beyond `rows` read as zero).  Fragment conventions of
// m16n8k16: g = lane / 4, t = lane % 4; accumulator tile n holds rows g, g+8
// and columns 8n + 2t, 8n + 2t + 1.
struct Forward {
  uint32_t xa[2][4];   // X as A fragments (two k-steps of 16)
  float z1[8][4], z2[8][4];
  uint32_t h1a[4][4], h2a[4][4];  // silu outputs as A fragments of the next layer
  float y[4];          // output tile (columns 2t, 2t+1 valid for t < 2)
};

__device__ __forceinline__ void load_x(Forward& F, const __nv_bfloat16* __restrict__ X, int rows) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int ks = 0; ks < 2; ++ks) {
    const int c = 16 * ks + 2 * t;
    F.xa[ks][0] = g < rows ? ld32(X + g * KIN + c) : 0u;
    F.xa[ks][1] = g + 8 < rows ? ld32(X + (g + 8) * KIN + c) : 0u;
    F.xa[ks][2] = g < rows ? ld32(X + g * KIN + c + 8) : 0u;
    F.xa[ks][3] = g + 8 < rows ? ld32(X + (g + 8) * KIN + c + 8) : 0u;
  }
}

__device__ __forceinline__ void to_afrag(const float (&z)[8][4], uint32_t (&a)[4][4], bool act) {
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    const float* p = z[2 * kc];
    const float* q = z[2 * kc + 1];
    if (act) {
      a[kc][0] = pack2(silu(p[0]), silu(p[1]));
      a[kc][1] = pack2(silu(p[2]), silu(p[3]));
      a[kc][2] = pack2(silu(q[0]), silu(q[1]));
      a[kc][3] = pack2(silu(q[2]), silu(q[3]));
    } else {
      a[kc][0] = pack2(p[0], p[1]);
      a[kc][1] = pack2(p[2], p[3]);
      a[kc][2] = pack2(q[0], q[1]);
      a[kc][3] = pack2(q[2], q[3]);
    }
  }
}

template <class WT>
__device__ __forceinline__ void forward(Forward& F, const WT& W) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float b0 = W.b1[8 * nt + 2 * t], b1 = W.b1[8 * nt + 2 * t + 1];
    F.z1[nt][0] = b0;
    F.z1[nt][1] = b1;
    F.z1[nt][2] = b0;
    F.z1[nt][3] = b1;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
      mma16816(F.z1[nt], F.xa[ks], ld32(&W.w1[8 * nt + g][16 * ks + 2 * t]), ld32(&W.w1[8 * nt + g][16 * ks + 2 * t + 8]));
  }
  to_afrag(F.z1, F.h1a, true);
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float b0 = W.b2[8 * nt + 2 * t], b1 = W.b2[8 * nt + 2 * t + 1];
    F.z2[nt][0] = b0;
    F.z2[nt][1] = b1;
    F.z2[nt][2] = b0;
    F.z2[nt][3] = b1;
#pragma unroll
    for (int kc = 0; kc < 4; ++kc)
      mma16816(F.z2[nt], F.h1a[kc], ld32(&W.w2[8 * nt + g][16 * kc + 2 * t]), ld32(&W.w2[8 * nt + g][16 * kc + 2 * t + 8]));
  }
  to_afrag(F.z2, F.h2a, true);
  F.y[0] = W.b3[2 * t];
  F.y[1] = W.b3[2 * t + 1];
  F.y[2] = W.b3[2 * t];
  F.y[3] = W.b3[2 * t + 1];
#pragma unroll
  for (int kc = 0; kc < 4; ++kc)
    mma16816(F.y, F.h2a[kc], ld32(&W.w3[g][16 * kc + 2 * t]), ld32(&W.w3[g][16 * kc + 2 * t + 8]));
}

}  // namespace mlp
}  // namespace gh
