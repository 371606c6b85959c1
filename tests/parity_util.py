"""Helpers shared by the GPU parity tests: run a problem through the CUDA
library and through the oracle, and compare them element by element."""
from __future__ import annotations

import json
import os

import numpy as np

import oracle as O
from paper_1207_3392_gb300 import hydro as H

# Tolerances (relative L1 per conserved variable against the FP64 oracle).
TOL_FP64 = 1e-10
TOL_FP32 = 1e-5
# L-infinity bars (largest cell difference over the largest magnitude of the
# variable): ten times the L1 bar.  Rounding differences spread over the whole
# field keep L-infinity near L1 (a relative rounding error is at most a few
# units in the last place in any cell); one wrong cell, as a halo or tile-seam
# fault makes, shows as an O(1e-2 .. 1) L-infinity while moving L1 by only
# its share of the cells, so it fails this bar at any mesh size.
LINF_FACTOR = 10.0


def rel_l1(gpu, ref, ndim):
    """Relative L1 difference per conserved variable.  Momentum components are
    normalised by the L1 norm of the whole momentum vector field (one component
    can vanish identically); Eq. L1ErrorNorm otherwise."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    nv = ndim + 2
    out = np.zeros(nv)
    mom = np.sum(np.abs(ref[1:1 + ndim]))
    dens = np.sum(np.abs(ref[0]))
    for v in range(nv):
        den = mom if 1 <= v <= ndim else np.sum(np.abs(ref[v]))
        if den == 0.0:
            den = dens
        out[v] = np.sum(np.abs(gpu[v] - ref[v])) / den
    return out


def linf_rel_per_var(gpu, ref, ndim):
    """Largest cell difference per conserved variable over the largest
    magnitude of that variable (momenta: over the whole momentum field)."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    nv = ndim + 2
    out = np.zeros(nv)
    mom = np.max(np.abs(ref[1:1 + ndim])) if ndim > 0 else 0.0
    dens = np.max(np.abs(ref[0]))
    for v in range(nv):
        den = mom if 1 <= v <= ndim else np.max(np.abs(ref[v]))
        if den == 0.0:
            den = dens
        out[v] = np.max(np.abs(gpu[v] - ref[v])) / den
    return out


def check(gpu, ref, ndim, tol, what="", tol_linf=None):
    """Assert the relative L1 bar and the L-infinity bar per conserved variable.
    tol and tol_linf are scalars or per-variable arrays; tol_linf defaults to
    LINF_FACTOR x tol.  With PARITY_LOG set, every comparison is appended to
    that file as one JSON line (test, what, L1, L-infinity, bars)."""
    e = rel_l1(gpu, ref, ndim)
    li = linf_rel_per_var(gpu, ref, ndim)
    tol = np.broadcast_to(np.asarray(tol, dtype=np.float64), e.shape)
    tol_linf = LINF_FACTOR * tol if tol_linf is None else np.broadcast_to(np.asarray(tol_linf, dtype=np.float64),
                                                                          e.shape)
    log = os.environ.get("PARITY_LOG")
    if log:
        with open(log, "a") as f:
            f.write(json.dumps({"test": os.environ.get("PYTEST_CURRENT_TEST", ""), "what": what,
                                "l1": e.tolist(), "linf": li.tolist(), "tol": tol.tolist(),
                                "tol_linf": tol_linf.tolist()}) + "\n")
    assert np.all(e <= tol), f"{what}: rel L1 {e} above {tol}; rel Linf {li}"
    assert np.all(li <= tol_linf), f"{what}: rel Linf {li} above {tol_linf}; rel L1 {e}"
    return e, li


def linf_rel(gpu, ref):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(gpu - ref)) / np.max(np.abs(ref)))


def gpu_run(prob, precision, solver=None, steps=None, t_end=None, tile=None, kchunk=0):
    """Evolve prob on the GPU with device-side CFL steps; returns (U, t)."""
    h = H.Hydro.from_problem(prob, precision=precision, solver=solver)
    try:
        if tile is not None:
            h.set_tile(tile, kchunk)
        if t_end:
            t = h.evolve(prob.cfl, t_end)
        else:
            t = h.advance(steps, prob.cfl)
        U = h.get_conserved(precision=H.FP64)
        return U, t
    finally:
        h.close()


def oracle_run(prob, solver=None, steps=None, t_end=None):
    g = O.Grid(prob, solver=solver)
    U0 = O.initial_state(prob, g)
    if t_end:
        U, t, _ = O.evolve(g, U0, prob.cfl, t_end)
    else:
        U, t, _ = O.evolve(g, U0, prob.cfl, max_steps=steps)
    return U, t
