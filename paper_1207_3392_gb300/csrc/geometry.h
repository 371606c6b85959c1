// geometry.h -- host construction of the per-axis reconstruction tables.
#pragma once

#include <vector>

#include "genasis_hydro.h"
#include "hydro_device.cuh"

namespace gh {

// Widths of cells -2 .. n+1 along an axis: the interior widths with two ghost
// widths on each side by the boundary rule (periodic wrap, reflecting mirror,
// outflow copy).
inline std::vector<double> extended_widths(const double* w, int n, int lo, int hi) {
  std::vector<double> e(n + 4);
  for (int c = -2; c < n + 2; ++c) {
    int s = c;
    if (c < 0) s = lo == GENASIS_BC_PERIODIC ? c + n : lo == GENASIS_BC_REFLECT ? -1 - c : 0;
    else if (c >= n) s = hi == GENASIS_BC_PERIODIC ? c - n : hi == GENASIS_BC_REFLECT ? 2 * n - 1 - c : n - 1;
    e[c + 2] = w[s];
  }
  return e;
}

// Reconstruction geometry (Eq. MinMod with centre distances of a non-uniform
// Cartesian mesh): q_c - q_- = (d_{c-1} + d_c)/2, q_+ - q_- = d_{c-1}/2 + d_c +
// d_{c+1}/2, q_+ - q_c = (d_c + d_{c+1})/2, face offset d_c / 2, with the
// limiter parameter theta folded into the one-sided inverse distances; plus
// inverse widths.  Appends one entry per extended cell.
template <class T>
inline void append_geometry(const std::vector<double>& e, double theta, std::vector<Geo<T>>& geo,
                            std::vector<T>& iw) {
  const int m = (int)e.size();
  for (int k = 0; k < m; ++k) {
    const double dc = e[k];
    const double dm = e[k > 0 ? k - 1 : 0], dp = e[k + 1 < m ? k + 1 : m - 1];
    Geo<T> g;
    g.ticm = (T)(theta / (0.5 * (dm + dc)));
    g.ipm = (T)(1.0 / (0.5 * dm + dc + 0.5 * dp));
    g.tipc = (T)(theta / (0.5 * (dc + dp)));
    g.h = (T)(0.5 * dc);
    geo.push_back(g);
    iw.push_back((T)(1.0 / dc));
  }
}

}  // namespace gh
