"""Helpers shared by the GPU parity tests: run a problem through the CUDA
library and through the oracle, and compare them element by element."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_1207_3392_gb300 import hydro as H

# Tolerances (relative L1 per conserved variable against the FP64 oracle).
TOL_FP64 = 1e-10
TOL_FP32 = 1e-5


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
