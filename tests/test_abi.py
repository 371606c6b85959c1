"""CPU checks of the boundary: the CUDA library builds, loads without a GPU and
exports every entry point include/*.h declares; descriptors are validated on
the host before any CUDA call."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from conftest import ROOT


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        with open(hdr) as f:
            text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
        names |= set(re.findall(r"\b(genasis_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1207_3392_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for must in ("genasis_hydro_create", "genasis_hydro_compute_dt", "genasis_hydro_step",
                 "genasis_hydro_get_conserved"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi():
    from paper_1207_3392_gb300 import hydro as H
    for name in _declared():
        if name.startswith("genasis_hydro_") and name != "genasis_hydro_last_error":
            assert name in H.SIGNATURES or name.startswith("genasis_batch"), name


def test_invalid_descriptors_rejected_on_host(lib):
    """Validation happens before any CUDA call, so it runs without a GPU."""
    from paper_1207_3392_gb300 import hydro as H
    H.load()
    w = np.full(8, 0.125)
    bad = []
    for field, value in (("ndim", 4), ("gamma", 1.0), ("theta", 2.5), ("solver", 7), ("precision", 3)):
        d = H.Desc()
        d.ndim = 1
        d.n[0], d.n[1], d.n[2] = 8, 1, 1
        d.widths[0] = w.ctypes.data
        d.gamma, d.solver, d.theta, d.precision = 1.4, 1, 1.4, 0
        d.bc_lo[0] = d.bc_hi[0] = 2
        setattr(d, field, value)
        out = ctypes.c_void_p()
        rc = H.load().genasis_hydro_create(ctypes.byref(d), ctypes.byref(out))
        bad.append((field, rc))
        assert rc == H.EINVAL, (field, rc)
    # a zero width and a one-sided periodic axis
    w0 = w.copy()
    w0[3] = 0.0
    d = H.Desc()
    d.ndim, d.n[0], d.gamma, d.solver, d.theta = 1, 8, 1.4, 1, 1.4
    d.widths[0] = w0.ctypes.data
    out = ctypes.c_void_p()
    assert H.load().genasis_hydro_create(ctypes.byref(d), ctypes.byref(out)) == H.EINVAL
    assert b"width" in H.load().genasis_hydro_last_error()
    d.widths[0] = w.ctypes.data
    d.bc_lo[0], d.bc_hi[0] = 0, 1
    assert H.load().genasis_hydro_create(ctypes.byref(d), ctypes.byref(out)) == H.EINVAL


def test_null_handle_calls_fail_cleanly(lib):
    from paper_1207_3392_gb300 import hydro as H
    L = H.load()
    assert L.genasis_hydro_step(None, 0.1) == H.EINVAL
    assert L.genasis_hydro_destroy(None) == H.OK
