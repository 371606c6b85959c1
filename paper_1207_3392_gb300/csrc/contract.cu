// contract.cu -- the batched and learned workloads behind genasis_hydro_t:
// genasis_hydro_batch_* (many independent problems, each described by a
// genasis_hydro_desc, on the engine of genasis_batch_*), the flux-correction
// network attached to a single-mesh handle (genasis_hydro_set_flux_mlp, on the
// solver of genasis_learned_*), and the cell centres of a handle.
#include <cuda_runtime.h>

#include <math.h>
#include <string.h>

#include <vector>

#include "common.h"
#include "genasis_hydro.h"
#include "hydro_handle.h"

using namespace gh;

namespace {

genasis_batch_t batch_of(genasis_hydro_t h) { return h ? h->batch : nullptr; }

}  // namespace

extern "C" {

int genasis_hydro_get_centers(genasis_hydro_t h, int axis, double* x) {
  GH_SINGLE_MESH(h);
  if (!h || !x) return fail(GENASIS_EINVAL, "get_centers: NULL argument");
  if (axis < 0 || axis >= h->ndim) return fail(GENASIS_EINVAL, "get_centers: axis %d outside [0, %d)", axis, h->ndim);
  // running low-face coordinate plus half the width (geometric centre, Sec. 3.1)
  double lo = h->origin[axis];
  const std::vector<double>& w = h->hw[axis];
  for (size_t i = 0; i < w.size(); ++i) {
    x[i] = lo + 0.5 * w[i];
    lo += w[i];
  }
  return GENASIS_OK;
}

int genasis_hydro_batch_create(int nprob, const genasis_hydro_desc* descs, genasis_hydro_t* out) {
  if (!out) return fail(GENASIS_EINVAL, "batch_create: out is NULL");
  *out = nullptr;
  if (nprob < 1 || !descs) return fail(GENASIS_EINVAL, "batch_create: need nprob >= 1 descriptions");
  const genasis_hydro_desc& d0 = descs[0];
  std::vector<genasis_batch_problem> probs((size_t)nprob);
  for (int i = 0; i < nprob; ++i) {
    const genasis_hydro_desc& d = descs[i];
    if (d.ndim != 1 && d.ndim != 2)
      return fail(GENASIS_EINVAL, "batch_create: problem %d has ndim %d; a batch takes 1D and 2D problems", i, d.ndim);
    if (d.solver != d0.solver || d.theta != d0.theta || d.precision != d0.precision || d.stream != d0.stream)
      return fail(GENASIS_EINVAL, "batch_create: problem %d: solver, theta, precision and stream must match problem 0", i);
    genasis_batch_problem& p = probs[(size_t)i];
    memset(&p, 0, sizeof(p));
    p.ndim = d.ndim;
    p.gamma = d.gamma;
    for (int q = 0; q < d.ndim; ++q) {
      p.n[q] = d.n[q];
      p.widths[q] = d.widths[q];
      p.bc_lo[q] = d.bc_lo[q];
      p.bc_hi[q] = d.bc_hi[q];
    }
  }
  genasis_batch_t b = nullptr;
  const int rc = genasis_batch_create(nprob, probs.data(), d0.solver, d0.theta, d0.precision, d0.stream, &b);
  if (rc) return rc;
  genasis_hydro* h = new genasis_hydro();
  h->batch = b;
  h->prec = d0.precision;
  h->solver = d0.solver;
  h->theta = d0.theta;
  *out = h;
  return GENASIS_OK;
}

int genasis_hydro_batch_set_primitive(genasis_hydro_t h, int iprob, const double* rho, const double* vel,
                                      const double* p) {
  genasis_batch_t b = batch_of(h);
  if (!b) return fail(GENASIS_EINVAL, "batch_set_primitive: not a batch handle");
  return genasis_batch_set_primitive(b, iprob, rho, vel, p);
}

int genasis_hydro_batch_run(genasis_hydro_t h, int nsteps, double cfl, double t_end) {
  genasis_batch_t b = batch_of(h);
  if (!b) return fail(GENASIS_EINVAL, "batch_run: not a batch handle");
  return genasis_batch_run(b, nsteps, cfl, t_end);
}

int genasis_hydro_batch_get_conserved(genasis_hydro_t h, int iprob, void* U, int precision) {
  genasis_batch_t b = batch_of(h);
  if (!b) return fail(GENASIS_EINVAL, "batch_get_conserved: not a batch handle");
  return genasis_batch_get_conserved(b, iprob, U, precision);
}

int genasis_hydro_batch_get_times(genasis_hydro_t h, double* t) {
  genasis_batch_t b = batch_of(h);
  if (!b) return fail(GENASIS_EINVAL, "batch_get_times: not a batch handle");
  return genasis_batch_get_times(b, t);
}

int genasis_hydro_set_flux_mlp(genasis_hydro_t h, const void* bf16_weights, size_t bytes) {
  GH_SINGLE_MESH(h);
  if (!h) return fail(GENASIS_EINVAL, "set_flux_mlp: NULL handle");
  if (!bf16_weights) {
    if (bytes != 0) return fail(GENASIS_EINVAL, "set_flux_mlp: NULL weights with a nonzero size");
    if (h->lf) {
      GH_CK(cudaStreamSynchronize(h->stream));
      genasis_learned_destroy(h->lf);
      h->lf = nullptr;
    }
    return GENASIS_OK;
  }
  const int np = genasis_mlp_param_count();
  if (bytes != (size_t)np * 2)
    return fail(GENASIS_EINVAL, "set_flux_mlp: %zu bytes given, the network has %d BF16 parameters (%d bytes)", bytes,
                np, 2 * np);
  if (h->ndim != 2 || h->prec != GENASIS_FP32_MIXED)
    return fail(GENASIS_EINVAL, "set_flux_mlp: the flux correction is for 2D GENASIS_FP32_MIXED handles");
  if (h->solver != GENASIS_HLL && h->solver != GENASIS_HLLC)
    return fail(GENASIS_EINVAL, "set_flux_mlp: the flux correction is for the HLL and HLLC solvers");
  // BF16 -> FP32 is exact: the BF16 bits are the upper half of the float
  std::vector<unsigned short> w16((size_t)np);
  if (is_device_ptr(bf16_weights)) {
    GH_CK(cudaMemcpyAsync(w16.data(), bf16_weights, bytes, cudaMemcpyDeviceToHost, h->stream));
    GH_CK(cudaStreamSynchronize(h->stream));
  } else {
    memcpy(w16.data(), bf16_weights, bytes);
  }
  std::vector<float> params((size_t)np);
  for (int i = 0; i < np; ++i) {
    const unsigned bits = (unsigned)w16[(size_t)i] << 16;
    memcpy(&params[(size_t)i], &bits, sizeof(float));
    if (!isfinite(params[(size_t)i])) return fail(GENASIS_EINVAL, "set_flux_mlp: parameter %d is not finite", i);
  }
  if (!h->lf) {
    genasis_hydro_desc d;
    memset(&d, 0, sizeof(d));
    d.ndim = 2;
    for (int q = 0; q < 2; ++q) {
      d.n[q] = h->n[q];
      d.widths[q] = h->hw[q].data();
      d.origin[q] = h->origin[q];
      d.bc_lo[q] = h->bc_lo[q];
      d.bc_hi[q] = h->bc_hi[q];
    }
    d.n[2] = 1;
    d.gamma = h->gamma;
    d.solver = h->solver;
    d.theta = h->theta;
    d.precision = GENASIS_FP32_MIXED;
    d.stream = (void*)h->stream;
    genasis_learned_t l = nullptr;
    const int rc = genasis_learned_create(&d, &l);
    if (rc) return rc;
    genasis_learned_set_option(l, GENASIS_OPT_ONE_LAUNCH, h->one_launch);
    genasis_learned_set_option(l, GENASIS_OPT_MLP_TCGEN05, h->mlp_tc);
    h->lf = l;
  }
  return genasis_learned_set_params(h->lf, params.data());
}

}  // extern "C"
