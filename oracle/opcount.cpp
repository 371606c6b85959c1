/*
 * opcount.cpp -- floating-point operation counts of the oracle's update
 * (hydro_oracle.c, Secs. 3.1-3.6 of arXiv:1207.3392), for the arithmetic
 * roofline of the measured kernels.
 *
 * TEST INFRASTRUCTURE ONLY, like the oracle it counts: only tests/ and
 * bench.py's reporting may load it.
 *
 * How: hydro_oracle.c is compiled a second time, here, as C++ with the token
 * `double` replaced by og_count_t, a scalar that carries an FP64 value and
 * counts every arithmetic operation applied to it.  The oracle's code runs
 * unchanged; only the type of its floating-point variables differs, so the
 * counts are those of the formulas exactly as the oracle evaluates them.
 *
 * Counting rule (the usual one for flop counts): +, -, * and / count 1 each
 * (a product feeding a sum counts 2, fused or not); sqrt, min, max and fabs
 * count 1; comparisons, negation, selection and copies count 0.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>

struct og_counts {
  long long add, mul, div, sqrt, minmax, abs;
};
static og_counts g_ops;

struct og_count_t {
  double v;
  og_count_t() = default;
  og_count_t(double x) : v(x) {}
  explicit operator double() const { return v; }
  explicit operator int() const { return (int)v; }
  og_count_t& operator+=(og_count_t o) { ++g_ops.add; v += o.v; return *this; }
  og_count_t& operator-=(og_count_t o) { ++g_ops.add; v -= o.v; return *this; }
  og_count_t& operator*=(og_count_t o) { ++g_ops.mul; v *= o.v; return *this; }
  og_count_t& operator/=(og_count_t o) { ++g_ops.div; v /= o.v; return *this; }
  friend og_count_t operator+(og_count_t a, og_count_t b) { ++g_ops.add; return a.v + b.v; }
  friend og_count_t operator-(og_count_t a, og_count_t b) { ++g_ops.add; return a.v - b.v; }
  friend og_count_t operator*(og_count_t a, og_count_t b) { ++g_ops.mul; return a.v * b.v; }
  friend og_count_t operator/(og_count_t a, og_count_t b) { ++g_ops.div; return a.v / b.v; }
  friend og_count_t operator-(og_count_t a) { return -a.v; }
  friend bool operator<(og_count_t a, og_count_t b) { return a.v < b.v; }
  friend bool operator>(og_count_t a, og_count_t b) { return a.v > b.v; }
  friend bool operator<=(og_count_t a, og_count_t b) { return a.v <= b.v; }
  friend bool operator>=(og_count_t a, og_count_t b) { return a.v >= b.v; }
  friend bool operator==(og_count_t a, og_count_t b) { return a.v == b.v; }
  friend bool operator!=(og_count_t a, og_count_t b) { return a.v != b.v; }
  friend og_count_t sqrt(og_count_t a) { ++g_ops.sqrt; return std::sqrt(a.v); }
  friend og_count_t fabs(og_count_t a) { ++g_ops.abs; return std::fabs(a.v); }
  friend og_count_t fmin(og_count_t a, og_count_t b) { ++g_ops.minmax; return std::fmin(a.v, b.v); }
  friend og_count_t fmax(og_count_t a, og_count_t b) { ++g_ops.minmax; return std::fmax(a.v, b.v); }
  friend bool isfinite(og_count_t a) { return std::isfinite(a.v); }
};

#define double og_count_t
#include "hydro_oracle.c"
#undef double

namespace {

void build_desc(og_desc* d, int ndim, const int* n, const double* const* widths, const int* bc_lo, const int* bc_hi,
                double gamma, double theta, int solver, og_count_t* const* w) {
  memset(d, 0, sizeof(*d));
  d->ndim = ndim;
  for (int q = 0; q < 3; ++q) {
    d->n[q] = q < ndim ? n[q] : 1;
    d->bc_lo[q] = q < ndim ? bc_lo[q] : 0;
    d->bc_hi[q] = q < ndim ? bc_hi[q] : 0;
    d->width[q] = q < ndim ? w[q] : NULL;
    if (q < ndim)
      for (int i = 0; i < n[q]; ++i) w[q][i] = widths[q][i];
    d->grad_phi[q] = 0.0;
  }
  d->gamma = gamma;
  d->theta = theta;
  d->solver = solver;
}

}  // namespace

/* Count the operations of one oracle call on the conserved state U (ndim + 2
 * planes of the mesh, FP64):
 *   what 0  og_rhs (one evaluation of L[U])
 *        1  og_step (one TVD RK2 step with dt = param)
 *        2  og_cfl_dt
 *        3  og_totals
 *        4  og_riemann_flux on one face: U = (W_L, W_R) primitives, axis = n[0]
 * counts[0..6] receive add/sub, mul, div, sqrt, min/max, abs and their sum.
 * Returns the oracle's status (0 on success). */
extern "C" int og_count_ops(int what, int ndim, const int* n, const double* const* widths, const int* bc_lo,
                            const int* bc_hi, double gamma, double theta, int solver, const double* U, double param,
                            long long* counts) {
  memset(&g_ops, 0, sizeof(g_ops));
  int rc = 0;
  if (what == 4) {
    og_count_t wl[5], wr[5], f[5];
    const int nv = ndim + 2;
    for (int v = 0; v < nv; ++v) {
      wl[v] = U[v];
      wr[v] = U[nv + v];
    }
    memset(&g_ops, 0, sizeof(g_ops));
    rc = og_riemann_flux(solver, gamma, ndim, n[0], wl, wr, f, NULL);
  } else {
    size_t ncell = 1;
    for (int q = 0; q < ndim; ++q) ncell *= (size_t)n[q];
    const size_t nvc = (size_t)(ndim + 2) * ncell;
    og_count_t* u = (og_count_t*)malloc(sizeof(og_count_t) * nvc);
    og_count_t* l = (og_count_t*)malloc(sizeof(og_count_t) * nvc);
    og_count_t* w[3] = {NULL, NULL, NULL};
    for (int q = 0; q < ndim; ++q) w[q] = (og_count_t*)malloc(sizeof(og_count_t) * (size_t)n[q]);
    for (size_t i = 0; i < nvc; ++i) u[i] = U[i];
    og_desc d;
    build_desc(&d, ndim, n, widths, bc_lo, bc_hi, gamma, theta, solver, w);
    og_count_t out = 0.0;
    og_count_t tot[5];
    memset(&g_ops, 0, sizeof(g_ops));
    if (what == 0) rc = og_rhs(&d, u, l);
    else if (what == 1) rc = og_step(&d, u, param);
    else if (what == 2) rc = og_cfl_dt(&d, u, &out);
    else if (what == 3) rc = og_totals(&d, u, tot);
    else rc = -1;
    free(u);
    free(l);
    for (int q = 0; q < ndim; ++q) free(w[q]);
  }
  counts[0] = g_ops.add;
  counts[1] = g_ops.mul;
  counts[2] = g_ops.div;
  counts[3] = g_ops.sqrt;
  counts[4] = g_ops.minmax;
  counts[5] = g_ops.abs;
  counts[6] = g_ops.add + g_ops.mul + g_ops.div + g_ops.sqrt + g_ops.minmax + g_ops.abs;
  return rc;
}
