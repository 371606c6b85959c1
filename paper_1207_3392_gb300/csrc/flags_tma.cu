// flags_tma.cu -- the shock detector of the HLLC -> HLL switch (the test:
// shock_flags.cuh) for Runge-Kutta stage 1 (state U^n) on 3D FP32 meshes,
// with the state planes staged in shared memory by the tensor memory
// accelerator (TMA).  Stage 2 (U^n + dt K, twice the bytes per cell) runs the
// register-tile pass of aux_kernels.cu, which measured faster there: its
// small CTAs keep more loads in flight than slots of both arrays allow.
//
// The detector needs, per cell, the pressure and velocity of its six
// neighbours.  One launch has two kinds of CTA:
//
//   * Tile CTAs flag the cells whose six neighbours all lie in the mesh.  A
//     tile is TX x TY cells of the (x, y) plane over a chunk of planes along
//     z.  One producer warp issues, per plane z0 - 1 .. z1 of the chunk, one
//     4D cp.async.bulk.tensor load of the box x in [a0 - 4, a0 + TX + 4),
//     y in [b0 - 1, b0 + TY + 1), all five conserved variables, into a ring
//     of NS slots, completing on the slot's `full` mbarrier.  x starts on a
//     16-byte boundary (a0 is a multiple of 32).
//     The TX x TY compute threads turn the tile's cells and its one-cell
//     ring (no corners) into (p, v) once, into a ring of three planes.
//     After one compute barrier, one thread releases the slot (its `empty`
//     mbarrier) and each flags its own cell of the plane before, whose
//     neighbours are then all converted.  Box cells outside the mesh arrive
//     as the TMA fill value and are never converted or read.
//   * Shell CTAs (the launch's first) flag the cells of the boundary shell,
//     one cell deep on every face, whose neighbours include ghost cells:
//     cell by cell through the boundary map.  They share no data with the
//     tiles.
//
// The (p, v_x, v_y) of three planes in shared memory let one barrier per
// plane separate the conversion of plane c + 1 from the reads of plane c - 1
// by its flags; the own column's (p, v_z) of the planes below and above stay
// in registers.  Every mbarrier wait is bounded (about one second); a wait that
// gives up sets STATUS_TIMEOUT, the compute threads agree on leaving through
// the compute barrier (bar.red.or), and the producer waits, bounded, for its
// loads still in flight before returning.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>

#include "aux_kernels.h"
#include "hydro_device.cuh"
#include "mbarrier.cuh"
#include "shock_flags.cuh"

namespace gh {
namespace {

// Tile shape of the pass: TX x TY compute threads (one cell each), NS staged
// planes.  The box holds the tile and its ring: x in [a0 - 4, a0 + TX + 4)
// (x on a 16-byte boundary), y in [b0 - 1, b0 + TY + 1).
template <int TX_, int TY_, int NS_>
struct Shape {
  static constexpr int TX = TX_, TY = TY_, NS = NS_, NT = TX * TY, NTHR = NT + 32;
  static constexpr int XB = TX + 8, YB = TY + 2, NV = 5;
  static constexpr int PL = NV * YB * XB;                     // floats of one staged box
  static constexpr unsigned BOX_BYTES = PL * 4u;
  static constexpr int ARR = (PL * 4 + 127) / 128 * 128 / 4;  // box arrays on 128-byte boundaries
  static constexpr int SX = TX + 2, SXY = SX * YB;            // (p, v) plane: columns a0 - 1 .. a0 + TX
  static constexpr int NRING = 2 * (TX + TY);
  static_assert(TX % 32 == 0 && NRING <= NT, "rows of whole warps; one ring cell per thread at most");
  static_assert(NS >= 2, "at least one plane in flight");
  struct Smem {
    alignas(128) float box[NS][ARR];
    float pv[3][3][SXY];  // [plane ring][p, v_x, v_y][box row * SX + column]
    unsigned long long full[NS];
    unsigned long long empty[NS];
  };
};

struct FlagTmaArgs {
  FlagArgs<float> A;
  CUtensorMap map_u;
  int gx, gy, kz;      // tiles along x and y, planes per chunk
  int nshell;          // shell CTAs, ahead of the tile CTAs
  long long shell;     // cells of the boundary shell
};

// Shell cell s: the z = 0 and z = n2 - 1 planes, then the y = 0 and
// y = n1 - 1 rows of the planes between, then the x = 0 and x = n0 - 1
// columns of what is left (every n >= 3; the shell count fits 32 bits).
__device__ __forceinline__ void shell_cell(unsigned s, unsigned nx, unsigned ny, unsigned nz, int& x, int& y, int& z) {
  const unsigned a = nx * ny, b = nx * (nz - 2), c = (ny - 2) * (nz - 2);
  if (s < 2 * a) {
    z = s < a ? 0 : (int)nz - 1;
    const unsigned r = s < a ? s : s - a;
    y = (int)(r / nx);
    x = (int)(r - (unsigned)y * nx);
    return;
  }
  s -= 2 * a;
  if (s < 2 * b) {
    y = s < b ? 0 : (int)ny - 1;
    const unsigned r = s < b ? s : s - b;
    const unsigned zz = r / nx;
    z = 1 + (int)zz;
    x = (int)(r - zz * nx);
    return;
  }
  s -= 2 * b;
  x = s < c ? 0 : (int)nx - 1;
  const unsigned r = s < c ? s : s - c;
  const unsigned zz = r / (ny - 2);
  z = 1 + (int)zz;
  y = 1 + (int)(r - zz * (ny - 2));
}

// (p, v) of the staged cell at u0 (variable stride YB * XB); (p, v_x, v_y)
// also into position q of a plane.
template <class SH>
__device__ __forceinline__ void convert(const float* u0, float gm1, float* dst, int q, float& p, float& vz) {
  float u[SH::NV], w[SH::NV];
#pragma unroll
  for (int v = 0; v < SH::NV; ++v) u[v] = u0[v * SH::YB * SH::XB];
  recover<3>(u, w);
  p = gm1 * w[SH::NV - 1];
  vz = w[3];
  dst[q] = p;
  dst[SH::SXY + q] = w[1];
  dst[2 * SH::SXY + q] = w[2];
}

template <int TX, int TY, int NS>
__global__ void __launch_bounds__(TX * TY + 32) shock_flags_tma_kernel(const __grid_constant__ FlagTmaArgs P) {
  using SH = Shape<TX, TY, NS>;
  constexpr int NT = SH::NT, NTHR = SH::NTHR, XB = SH::XB, SX = SH::SX, SXY = SH::SXY;
  const FlagArgs<float>& A = P.A;
  const int nx = A.n[0], ny = A.n[1], nz = A.n[2];
  const float gm1 = (float)(A.gamma - 1.0);
  const int tid = threadIdx.x;

  if ((int)blockIdx.x < P.nshell) {  // one shell cell per thread
    const unsigned s = blockIdx.x * (unsigned)NTHR + tid;
    if (s < P.shell) {
      int x, y, z;
      shell_cell(s, nx, ny, nz, x, y, z);
      A.flags[((size_t)z * ny + y) * nx + x] = (unsigned char)shock::bits_direct<float, 3>(A, gm1, 0.0f, x, y, z);
    }
    return;
  }

  extern __shared__ __align__(128) unsigned char flags_smem[];
  typename SH::Smem& S = *reinterpret_cast<typename SH::Smem*>(flags_smem);
  const int b = blockIdx.x - P.nshell;
  const int a0 = (b % P.gx) * TX, b0 = ((b / P.gx) % P.gy) * TY;
  const int z0 = (b / (P.gx * P.gy)) * P.kz, z1 = min(z0 + P.kz, nz);
  const int nl = z1 - z0 + 2;  // planes z0 - 1 .. z1

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      tma::mbar_init(&S.full[s], 1u);
      tma::mbar_init(&S.empty[s], 1u);
    }
    tma::fence_mbar_init();
  }
  __syncthreads();

  if (tid >= NT) {
    // producer warp: lane 0 issues the plane loads
    if (tid != NT) return;
    int issued = 0;
    for (int l = 0; l < nl; ++l) {
      const int s = l % NS;
      if (l >= NS && !tma::mbar_wait_spin(&S.empty[s], (unsigned)(((l / NS) - 1) & 1))) {
        atomicOr(A.status, STATUS_TIMEOUT);
        break;
      }
      tma::mbar_expect_tx(&S.full[s], SH::BOX_BYTES);
      tma::load_4d(&S.box[s][0], &P.map_u, a0 - 4, b0 - 1, z0 - 1 + l, 0, &S.full[s]);
      ++issued;
    }
    // do not leave while a load of this CTA may still write its shared memory
    for (int l = issued > NS ? issued - NS : 0; l < issued; ++l)
      if (!tma::mbar_wait(&S.full[l % NS], (unsigned)((l / NS) & 1))) atomicOr(A.status, STATUS_TIMEOUT);
    return;
  }

  // compute threads: the own cell, and for tid < NRING one ring cell
  const int tx = tid % TX, ty = tid / TX;
  const int x = a0 + tx, y = b0 + ty;
  const bool own_in = x < nx && y < ny;
  const bool own_inner = x >= 1 && x <= nx - 2 && y >= 1 && y <= ny - 2;
  int rr = 0, rc = 0;  // ring cell's box row and column
  if (tid < 2 * TY) {
    rr = tid % TY + 1;
    rc = tid < TY ? 3 : TX + 4;
  } else if (tid < SH::NRING) {
    const int t = tid - 2 * TY;
    rr = t < TX ? 0 : TY + 1;
    rc = t % TX + 4;
  }
  const int ri = a0 - 4 + rc, rj = b0 - 1 + rr;
  const bool ring_in = tid < SH::NRING && ri >= 0 && ri < nx && rj >= 0 && rj < ny;
  const int qo = (ty + 1) * SX + tx + 1, qr = rr * SX + rc - 3;  // (p, v) positions
  const int uo = (ty + 1) * XB + tx + 4, ur = rr * XB + rc;        // box positions
  const size_t plane = (size_t)nx * ny;
  unsigned char* fcol = A.flags + (own_inner ? (size_t)y * nx + x : 0);  // own column of flags
  bool failed = false;
  float p1 = 0.0f, vz1 = 0.0f, p2 = 0.0f, vz2 = 0.0f;  // own column at planes c - 1, c - 2
  int s = 0, pc = 0;                                   // slot and (p, v) plane of plane c
  unsigned phase = 0;                                  // parity of the slot's fill
  for (int c = 0; c < nl; ++c) {
    const int z = z0 - 1 + c;
    if (!failed && !tma::mbar_wait_spin(&S.full[s], phase)) {
      atomicOr(A.status, STATUS_TIMEOUT);
      failed = true;
    }
    float p0 = 0.0f, vz0 = 0.0f;  // own column at plane c
    if (!failed && z >= 0 && z < nz) {
      float* dst = &S.pv[pc][0][0];
      const float* slot = &S.box[s][0];
      if (own_in) convert<SH>(slot + uo, gm1, dst, qo, p0, vz0);
      float pr, vr;
      if (ring_in) convert<SH>(slot + ur, gm1, dst, qr, pr, vr);
    }
    if (tma::sync_compute_or<NT>(failed)) break;
    if (tid == 0) {  // every compute thread is done with the slot
      tma::fence_proxy_async();
      tma::mbar_arrive(&S.empty[s]);
    }
    const int zf = z - 1;  // the plane flagged now
    if (c >= 2 && own_inner && zf >= 1 && zf <= nz - 2) {
      const float* mid = &S.pv[pc == 0 ? 2 : pc - 1][0][0];
      unsigned bits = 0;
      bits |= shock::jump(mid[qo - 1], mid[SXY + qo - 1], mid[qo + 1], mid[SXY + qo + 1]) ? 1u : 0u;
      bits |= shock::jump(mid[qo - SX], mid[2 * SXY + qo - SX], mid[qo + SX], mid[2 * SXY + qo + SX]) ? 2u : 0u;
      bits |= shock::jump(p2, vz2, p0, vz0) ? 4u : 0u;
      fcol[(size_t)zf * plane] = (unsigned char)bits;
    }
    p2 = p1;
    vz2 = vz1;
    p1 = p0;
    vz1 = vz0;
    pc = pc == 2 ? 0 : pc + 1;
    if (++s == NS) {
      s = 0;
      phase ^= 1u;
    }
  }
}

// Grid and launch of one shape: shell CTAs first, then the tiles with z
// chunks sized for about `waves` waves of resident tile CTAs.  The shared-
// memory opt-in and the residency are found once per device.
template <int TX, int TY, int NS>
cudaError_t launch_shape(const FlagTmaArgs& P0, cudaStream_t s, int waves = 4) {
  using SH = Shape<TX, TY, NS>;
  constexpr size_t SMEM = sizeof(typename SH::Smem);
  auto* kern = shock_flags_tma_kernel<TX, TY, NS>;
  constexpr int MAXDEV = 64;
  static int resident[MAXDEV] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAXDEV) return cudaErrorInvalidDevice;
  if (!resident[dev]) {
    int per_sm = 0, sms = 0;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM)) != cudaSuccess)
      return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SH::NTHR, SMEM)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    resident[dev] = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  }
  FlagTmaArgs P = P0;
  const int nx = P.A.n[0], ny = P.A.n[1], nz = P.A.n[2];
  P.gx = (nx + TX - 1) / TX;
  P.gy = (ny + TY - 1) / TY;
  const long long gxy = (long long)P.gx * P.gy;
  long long chunks = ((long long)waves * resident[dev] + gxy - 1) / gxy;
  chunks = chunks < 1 ? 1 : (chunks > nz ? nz : chunks);
  P.kz = (int)((nz + chunks - 1) / chunks);
  chunks = (nz + P.kz - 1) / P.kz;
  P.shell = 2LL * nx * ny + 2LL * nx * (nz - 2) + 2LL * (ny - 2) * (nz - 2);
  if (P.shell > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  P.nshell = (int)((P.shell + SH::NTHR - 1) / SH::NTHR);
  const long long grid = P.nshell + gxy * chunks;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  kern<<<(unsigned)grid, SH::NTHR, SMEM, s>>>(P);
  return cudaGetLastError();
}

// The shape the library launches (its box is the maps' box): 32 x 8 cells,
// two slots (one plane in flight while one is converted), the fastest of
// the shapes and depths measured on the 256^3 point blast.
constexpr int FTX = 32, FTY = 8, FNS = 2;
static_assert(FTX + 8 == FLAGS_TMA_BOX_X && FTY + 2 == FLAGS_TMA_BOX_Y, "the maps' box is the tile's box");

}  // namespace

bool flags_tma_usable(int ndim, bool fp32, const int* n) {
  return ndim == 3 && fp32 && n[0] % 4 == 0 && n[0] >= 3 && n[1] >= 3 && n[2] >= 3;
}

cudaError_t launch_shock_flags_tma(const FlagArgs<float>& A, const CUtensorMap& map_u, cudaStream_t s) {
  if (A.stage != 1 || !flags_tma_usable(3, true, A.n)) return cudaErrorInvalidValue;
  FlagTmaArgs P;
  memset(&P, 0, sizeof(P));
  P.A = A;
  P.map_u = map_u;
  return launch_shape<FTX, FTY, FNS>(P, s);
}

}  // namespace gh
