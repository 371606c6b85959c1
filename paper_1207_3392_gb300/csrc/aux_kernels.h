// aux_kernels.h -- launchers of the small kernels around the stage kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>

namespace gh {

// Slots of the per-handle device scalar block.
enum { SCAL_DT = 0, SCAL_T = 1, SCAL_DTCFL = 2, SCAL_TOT = 3, SCAL_COUNT = 8 };
enum { FIN_FIXED = 0, FIN_CFL = 1, FIN_REDUCE = 2 };
// The finalize kernel folds the per-CTA partials over FIN_CTAS CTAs.  Its
// workspace follows the scalar block: FIN_CTAS x 6 doubles (slice results),
// then a ticket counter (zero between launches).  A scalar block that a
// finalize launch uses holds SCAL_ALLOC doubles, zeroed at allocation.
constexpr int FIN_CTAS = 32;
constexpr int SCAL_ALLOC = SCAL_COUNT + FIN_CTAS * 6 + 1;

template <class T>
struct ReduceArgs {
  size_t ncell;
  int n[3];
  double gamma;
  const T* U;
  const T* iw[3];        // inverse widths, index c + 2
  const double* wd[3];   // widths, index c
  double* part_speed;
  double* part_tot;
  unsigned* status;
  int nblk;
};

struct FinalizeArgs {
  const double* part_speed;  // may be null
  const double* part_tot;    // may be null
  int nblk;
  int nv;
  int mode;
  double cfl, fixed_dt, t_end;
  double* scal;
  unsigned* status;
};

// Shock bits of every cell for the HLLC -> HLL switch, from a stage's input
// state (stage 1: U^n; stage 2: U^n + dt K).
template <class T>
struct FlagArgs {
  int n[3];
  int bc_lo[3], bc_hi[3];
  double gamma;
  const T* un;
  const T* k1;        // stage 2 only
  const double* dt;   // stage 2 only
  unsigned char* flags;
  size_t ncell;
  int stage;
  unsigned* status;   // STATUS_TIMEOUT when a bounded wait of the TMA pass gives up
};

template <class T>
cudaError_t launch_shock_flags(int ndim, const FlagArgs<T>& A, cudaStream_t s);

// The detector of Runge-Kutta stage 1 on 3D FP32 meshes with the state
// planes staged by TMA (flags_tma.cu).  Usable when n[0] is a multiple of 4
// (16-byte rows) and every n >= 3.  map_u is a 4D map (x, y, z, variable) of
// U^n with the box FLAGS_TMA_BOX_X x FLAGS_TMA_BOX_Y x 1 x 5.
constexpr int FLAGS_TMA_BOX_X = 40, FLAGS_TMA_BOX_Y = 10;
bool flags_tma_usable(int ndim, bool fp32, const int* n);
cudaError_t launch_shock_flags_tma(const FlagArgs<float>& A, const CUtensorMap& map_u, cudaStream_t s);

template <class T>
cudaError_t launch_init_from_primitive(int ndim, size_t ncell, double gamma, const double* rho, const double* vel,
                                       const double* p, T* U, cudaStream_t s);
template <class Tin, class Tout>
cudaError_t launch_convert(size_t count, const Tin* in, Tout* out, cudaStream_t s);
template <class T>
cudaError_t launch_speed(int ndim, const ReduceArgs<T>& A, cudaStream_t s);
template <class T>
cudaError_t launch_totals(int ndim, const ReduceArgs<T>& A, cudaStream_t s);
cudaError_t launch_finalize(const FinalizeArgs& A, cudaStream_t s);

}  // namespace gh
