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
    """Every call on a NULL handle returns GENASIS_EINVAL before touching a
    device (destroy accepts NULL); the calls run here without a GPU."""
    import ctypes
    from paper_1207_3392_gb300 import hydro as H
    L = H.load()
    d = ctypes.c_double()
    buf = (ctypes.c_double * 16)()
    fbuf = (ctypes.c_float * 16)()
    ibuf = (ctypes.c_int * 8)()
    calls = {
        "genasis_hydro_step": (0.1,), "genasis_hydro_sync": (), "genasis_hydro_status": (),
        "genasis_hydro_clear_status": (), "genasis_hydro_compute_dt": (0.5, ctypes.byref(d)),
        "genasis_hydro_advance": (1, 0.5, 0.0, None), "genasis_hydro_get_time": (ctypes.byref(d),),
        "genasis_hydro_set_time": (0.0,), "genasis_hydro_get_totals": (buf,),
        "genasis_hydro_set_tile": (0, 0), "genasis_hydro_get_tile": (ibuf,),
        "genasis_hydro_autotune": (1, None), "genasis_hydro_set_potential_gradient": (buf,),
        "genasis_hydro_get_step_totals": (buf,), "genasis_hydro_profile_step": (0.5, fbuf),
        "genasis_hydro_get_conserved": (buf, H.FP64), "genasis_hydro_set_conserved": (buf, H.FP64),
        "genasis_learned_step": (0.1,), "genasis_learned_set_fct": (1,), "genasis_learned_get_conserved": (fbuf,),
        "genasis_learned_advance": (1, 0.5, 0.0, None),
        "genasis_batch_run": (1, 0.5, 0.0), "genasis_batch_get_times": (buf,), "genasis_batch_get_tile": (ibuf,),
        "genasis_batch_set_tile": (0, 32), "genasis_batch_autotune": (1, None),
        "genasis_fmr_step": (1, 0.3, None), "genasis_fmr_autotune": (1,), "genasis_fmr_get_level": (0, buf),
        "genasis_fmr_set_level": (0, buf),
        "genasis_hydro_get_centers": (0, buf), "genasis_hydro_batch_run": (1, 0.5, 0.0),
        "genasis_hydro_batch_get_times": (buf,), "genasis_hydro_batch_get_conserved": (0, buf, H.FP64),
        "genasis_hydro_batch_set_primitive": (0, buf, buf, buf), "genasis_hydro_set_flux_mlp": (buf, 16),
    }
    for name, args in calls.items():
        assert getattr(L, name)(None, *args) == H.EINVAL, name
    for name in ("genasis_hydro_destroy", "genasis_learned_destroy", "genasis_batch_destroy", "genasis_fmr_destroy"):
        assert getattr(L, name)(None) == H.OK, name


def test_batch_descriptions_validated_on_host(lib):
    """genasis_hydro_batch_create refuses 3D problems and descriptions whose
    solver, theta or precision differ, before any CUDA call."""
    from paper_1207_3392_gb300 import hydro as H
    L = H.load()
    w = np.full(8, 0.125)
    arr = (H.Desc * 2)()
    for d in arr:
        d.ndim, d.n[0], d.n[1], d.n[2] = 1, 8, 1, 1
        d.widths[0] = w.ctypes.data
        d.gamma, d.solver, d.theta, d.precision = 1.4, 1, 1.4, 0
        d.bc_lo[0] = d.bc_hi[0] = 2
    out = ctypes.c_void_p()
    arr[1].theta = 1.5
    assert L.genasis_hydro_batch_create(2, ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(out)) == H.EINVAL
    assert b"theta" in L.genasis_hydro_last_error()
    arr[1].theta = 1.4
    arr[1].ndim = 3
    assert L.genasis_hydro_batch_create(2, ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(out)) == H.EINVAL
    assert L.genasis_hydro_batch_create(0, None, ctypes.byref(out)) == H.EINVAL


def test_descriptor_layout_matches_the_header():
    """The binding's genasis_hydro_desc has the header's fields in order."""
    from paper_1207_3392_gb300 import hydro as H
    with open(os.path.join(ROOT, "include", "genasis_hydro.h")) as f:
        text = f.read()
    body = text[text.index("typedef struct {\n  int ndim;"):]
    body = body[: body.index("} genasis_hydro_desc;")]
    fields = re.findall(r"\*?(\w+)(?:\[\d\])?;", body)
    assert fields == [name for name, _ in H.Desc._fields_], fields
