"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element
by element on the same seeded inputs: FP64 within 1e-10 relative L1 per
conserved variable, FP32-mixed within 1e-5, and L-infinity (largest cell
difference over the variable's largest magnitude) within ten times those bars.
Sizes span several tiles and ragged tails; every boundary rule, both solvers,
non-uniform widths, the near-vacuum double rarefaction and the interacting
blast waves in every precision, and the full-size workloads (one step)."""
import numpy as np
import pytest

import oracle as O
from paper_1207_3392_gb300 import hydro as H
from paper_1207_3392_gb300 import problems as P
from parity_util import TOL_FP32, TOL_FP64, check, gpu_run, oracle_run, rel_l1

pytestmark = pytest.mark.gpu

PRECISIONS = ((H.FP64, TOL_FP64), (H.FP32_MIXED, TOL_FP32))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1207_3392_gb300 import build
    build.build()
    yield


def _check(gpu, ref, ndim, tol, what):
    check(gpu, ref, ndim, tol, what)


@pytest.mark.parametrize("solver", [H.HLL, H.HLLC])
def test_sod_1d_full_run(solver):
    """The 1D benchmark case in full: Sod, 256 cells, C_CFL 0.8, to t = 0.2."""
    pr = P.sod(256, solver=solver)
    Uo, to = oracle_run(pr, t_end=pr.t_end)
    for precision, tol in PRECISIONS:
        Ug, tg = gpu_run(pr, precision, t_end=pr.t_end)
        assert tg == pytest.approx(to, rel=1e-12)
        _check(Ug, Uo, 1, tol, f"sod prec={precision}")


@pytest.mark.parametrize("n", [256, 1500])
@pytest.mark.parametrize("precision", [H.FP64, H.FP32_MIXED])
def test_one_launch_1d_advance_is_the_multi_launch_advance(n, precision):
    """Small 1D meshes run every step of an advance (and a fixed-dt step) in
    one cooperative launch: bitwise the states and time of the three launches
    per step, on one tile (256 cells) and on three (1500), in a run clamped
    to its end time.  The step totals sum the same cells in tiles of another
    width, so they agree to rounding."""
    pr = P.sod(n, t_end=0.1)
    out = []
    for one in (True, False):
        h = H.Hydro.from_problem(pr, precision=precision)
        h.set_one_launch(one)
        assert h.launches_per_step() == (1 if one else 3)
        t = h.evolve(pr.cfl, pr.t_end, chunk=17)
        h.step(1e-4)
        out.append((h.get_conserved(), t, h.time, h.step_totals()))
        h.close()
    (ua, ta, t2a, sa), (ub, tb, t2b, sb) = out
    np.testing.assert_array_equal(ua, ub)
    assert ta == tb == pytest.approx(0.1, rel=1e-14) and t2a == t2b
    np.testing.assert_allclose(sa, sb, rtol=1e-12)


@pytest.mark.parametrize("solver", [H.HLL, H.HLLC])
@pytest.mark.parametrize("bc", [P.PERIODIC, P.REFLECT, P.OUTFLOW])
def test_random_blocks_2d(solver, bc):
    """Discontinuous 2D state, non-uniform widths, ragged tile tails (197 x 75)."""
    pr = P.random_blocks(2, (197, 75), seed=20 + bc, bc=bc)
    Uo, _ = oracle_run(pr, solver=solver, steps=12)
    for precision, tol in PRECISIONS:
        Ug, _ = gpu_run(pr, precision, solver=solver, steps=12)
        _check(Ug, Uo, 2, tol, f"2d bc={bc} prec={precision}")


@pytest.mark.parametrize("solver", [H.HLL, H.HLLC])
@pytest.mark.parametrize("bc", [P.PERIODIC, P.REFLECT, P.OUTFLOW])
def test_random_blocks_3d(solver, bc):
    """Discontinuous 3D state, non-uniform widths, ragged tiles (45 x 21 x 38)."""
    pr = P.random_blocks(3, (45, 21, 38), seed=40 + bc, bc=bc)
    Uo, _ = oracle_run(pr, solver=solver, steps=6)
    for precision, tol in PRECISIONS:
        Ug, _ = gpu_run(pr, precision, solver=solver, steps=6)
        _check(Ug, Uo, 3, tol, f"3d bc={bc} prec={precision}")


def test_mixed_boundaries_3d():
    """Different rules on each face of the box."""
    pr = P.random_blocks(3, (36, 40, 20), seed=77, bc=P.REFLECT)
    pr = pr.with_(bc_lo=(P.REFLECT, P.OUTFLOW, P.PERIODIC), bc_hi=(P.OUTFLOW, P.REFLECT, P.PERIODIC))
    Ug, _ = gpu_run(pr, H.FP64, steps=8)
    Uo, _ = oracle_run(pr, steps=8)
    _check(Ug, Uo, 3, TOL_FP64, "mixed bc")


@pytest.mark.parametrize("solver", [H.HLL, H.HLLC])
def test_sedov_3d_reduced(solver):
    """Point blast (benchmark setup) at 64^3 for 50 steps."""
    pr = P.sedov_3d(64, solver=solver)
    Uo, to = oracle_run(pr, steps=50)
    for precision, tol in PRECISIONS:
        Ug, tg = gpu_run(pr, precision, steps=50)
        assert tg == pytest.approx(to, rel=1e-9 if precision == H.FP64 else 1e-5)
        _check(Ug, Uo, 3, tol, f"sedov 64^3 prec={precision}")


def test_stretched_pulse_reduced():
    """Centrally refined mesh (ratio 1.01 widths), Gaussian pulse, FP32-mixed
    HLLC, 80^3 for 20 steps."""
    pr = P.stretched_pulse_3d(80, steps=20)
    Ug, _ = gpu_run(pr, H.FP32_MIXED, steps=20)
    Uo, _ = oracle_run(pr, steps=20)
    _check(Ug, Uo, 3, TOL_FP32, "stretched 80^3")


@pytest.mark.parametrize("solver", [H.HLL, H.HLLC])
def test_rayleigh_taylor_reduced(solver):
    """Rayleigh-Taylor set-up of Sec. 4.3.2 (uniform external force, periodic
    x, reflecting y) at 32 x 96 for 60 steps."""
    pr = P.rayleigh_taylor(32, 96, solver=solver)
    Uo, to = oracle_run(pr, steps=60)
    # FP32 momenta: in hydrostatic balance the momentum tendency is the
    # difference of the pressure-flux difference (p ~ 2.5, formed in FP32) and
    # the source rho g, each ~ rho g; the FP32 rounding of p, 2.5 x 6e-8,
    # against rho g dy ~ 1.6e-3 is a relative error of ~1e-4 on a tendency
    # that the small perturbation velocities only barely exceed.  Density and
    # energy keep the 1e-5 bar.
    tol32 = np.array([TOL_FP32, 3e-4, 3e-4, TOL_FP32])
    for precision, tol in ((H.FP64, TOL_FP64), (H.FP32_MIXED, tol32)):
        Ug, tg = gpu_run(pr, precision, steps=60)
        assert tg == pytest.approx(to, rel=1e-9 if precision == H.FP64 else 1e-5)
        _check(Ug, Uo, 2, tol, f"rayleigh-taylor prec={precision}")


def test_potential_gradient_on_every_axis_3d():
    """A force with components on all three axes (x and y in the tile plane,
    z along the march) on random blocks with reflecting walls."""
    pr = P.random_blocks(3, (30, 26, 22), seed=21, bc=P.REFLECT).with_(grad_phi=(0.3, -0.2, 0.5))
    Uo, _ = oracle_run(pr, steps=8)
    for precision, tol in PRECISIONS:
        Ug, _ = gpu_run(pr, precision, steps=8)
        _check(Ug, Uo, 3, tol, f"3d source prec={precision}")


def test_free_fall_closed_form_gpu():
    """Uniform gas in a periodic box: S(t) = -rho grad_phi t and
    G(t) = G(0) + rho |grad_phi|^2 t^2 / 2 exactly; switching the source off
    again gives the plain step bitwise."""
    grad = (0.2, -0.5, 0.35)
    pr = P.free_fall(3, 16, grad, rho=1.3, p=0.9)
    h = H.Hydro.from_problem(pr, precision=H.FP64)
    G0 = h.get_conserved()[-1].copy()
    t = 0.0
    for dt in (0.02, 0.013, 0.031):
        h.step(dt)
        t += dt
    U = h.get_conserved()
    for q in range(3):
        np.testing.assert_allclose(U[1 + q], -1.3 * grad[q] * t, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(U[-1], G0 + 0.5 * 1.3 * sum(x * x for x in grad) * t * t, rtol=1e-13)
    h.set_potential_gradient((0.0, 0.0, 0.0))
    h2 = H.Hydro.from_problem(pr.with_(grad_phi=(0.0, 0.0, 0.0)), precision=H.FP64)
    h2.set_conserved(U)
    h.step(0.01)
    h2.step(0.01)
    np.testing.assert_array_equal(h.get_conserved(), h2.get_conserved())
    with pytest.raises(H.HydroError):
        h.set_potential_gradient((0.0, float("nan"), 0.0))
    h.close()
    h2.close()


def test_kelvin_helmholtz_reduced():
    """Periodic shear layer at 64^2, HLLC, FP32-mixed and FP64, 40 steps."""
    pr = P.kelvin_helmholtz(64, seed=5)
    Uo, _ = oracle_run(pr, steps=40)
    for precision, tol in ((H.FP64, TOL_FP64), (H.FP32_MIXED, TOL_FP32)):
        Ug, _ = gpu_run(pr, precision, steps=40)
        _check(Ug, Uo, 2, tol, f"kh prec={precision}")


@pytest.mark.parametrize("ndim,precision,shape", [(3, H.FP32_MIXED, (70, 34, 41)), (3, H.FP32_MIXED, (72, 34, 41)),
                                                  (3, H.FP64, (70, 34, 41)), (2, H.FP32_MIXED, (150, 97)),
                                                  (1, H.FP32_MIXED, (700,)), (3, H.FP64_DW, (70, 34, 41))])
def test_every_tile_shape_identical(ndim, precision, shape):
    """Each compiled tile shape and plane count gives bitwise the same state.
    Tiles that stage the state with TMA need n[0] a multiple of 4: on other
    meshes they are refused (EINVAL), on (72, 34, 41) they run."""
    pr = P.random_blocks(ndim, shape, seed=3, bc=P.REFLECT)
    ref, _ = gpu_run(pr, precision, steps=4, tile=0, kchunk=0)
    h = H.Hydro.from_problem(pr, precision=precision)
    count = h.tile_info()["tile_count"]
    h.close()
    ran = 0
    pair_ref = None
    for tile in range(count):
        paired = ndim == 3 and precision == H.FP32_MIXED and tile in PAIR_TILES
        for kc in ((0, 7, shape[-1]) if ndim > 1 else (0,)):
            try:
                U, _ = gpu_run(pr, precision, steps=4, tile=tile, kchunk=kc)
            except H.HydroError as e:
                assert e.code == H.EINVAL and "TMA" in str(e) and shape[0] % 4 != 0, (tile, str(e))
                continue
            if paired:
                # the paired family: bitwise among themselves, within the
                # FP32 bar of the scalar tiles
                if pair_ref is None:
                    pair_ref = U
                    _check(U, ref, 3, TOL_FP32, f"paired tile {tile} against tile 0")
                np.testing.assert_array_equal(U, pair_ref, err_msg=f"tile {tile} kchunk {kc}")
            else:
                np.testing.assert_array_equal(U, ref, err_msg=f"tile {tile} kchunk {kc}")
            ran += 1
    assert ran >= 1
    if ndim == 3 and precision == H.FP32_MIXED:
        assert pair_ref is not None


PAIR_TILES = (11, 12, 13)  # 3D FP32 tiles taking two march planes per thread (packed FP32)


@pytest.mark.parametrize("bc", ["periodic", "reflect", "outflow", "mixed"])
def test_pair_tiles_match_the_oracle_and_each_other(bc):
    """The z-paired tiles under every boundary rule, HLL and HLLC, on a mesh
    ragged in x, y and z (72 x 29 x 23: an odd plane count, so a last chunk
    computes one plane past its end): within the FP32 bar of the oracle and of
    the scalar tiles, and bitwise the same state for every paired tile and
    chunk length (2 planes per chunk: a warm-up pair per pair; odd requests
    round up to whole plane pairs)."""
    codes = {"periodic": P.PERIODIC, "reflect": P.REFLECT, "outflow": P.OUTFLOW, "mixed": P.REFLECT}
    pr = P.random_blocks(3, (72, 29, 23), seed=19, bc=codes[bc])
    if bc == "mixed":
        pr = pr.with_(bc_lo=(P.REFLECT, P.OUTFLOW, P.PERIODIC), bc_hi=(P.OUTFLOW, P.REFLECT, P.PERIODIC))
    for solver in (H.HLL, H.HLLC):
        Uo, to = oracle_run(pr, solver=solver, steps=3)
        ref, t = gpu_run(pr, H.FP32_MIXED, solver=solver, steps=3, tile=PAIR_TILES[0], kchunk=0)
        assert t == pytest.approx(to, rel=1e-5)
        _check(ref, Uo, 3, TOL_FP32, f"paired tiles bc={bc} solver={solver}")
        scalar, _ = gpu_run(pr, H.FP32_MIXED, solver=solver, steps=3, tile=0, kchunk=0)
        _check(ref, scalar, 3, TOL_FP32, f"paired against scalar bc={bc} solver={solver}")
        for tile in PAIR_TILES:
            for kc in (0, 2, 5, 23):
                U, _ = gpu_run(pr, H.FP32_MIXED, solver=solver, steps=3, tile=tile, kchunk=kc)
                np.testing.assert_array_equal(U, ref, err_msg=f"solver {solver} tile {tile} kchunk {kc}")


def test_pair_tiles_sedov_source_and_totals():
    """The paired tiles on the point blast (50 steps at 64^3) and with an
    external force on all three axes: within the FP32 bar of the oracle; the
    step totals (each column's two lanes summed apart) within rounding of the
    scalar tiles' totals."""
    pr = P.sedov_3d(64)
    Uo, to = oracle_run(pr, steps=50)
    for tile in PAIR_TILES:
        Ug, tg = gpu_run(pr, H.FP32_MIXED, steps=50, tile=tile, kchunk=0)
        assert tg == pytest.approx(to, rel=1e-5)
        _check(Ug, Uo, 3, TOL_FP32, f"sedov 64^3 paired tile {tile}")
    pf = P.random_blocks(3, (30, 26, 22), seed=21, bc=P.REFLECT).with_(grad_phi=(0.3, -0.2, 0.5))
    Uo, _ = oracle_run(pf, steps=8)
    Ug, _ = gpu_run(pf, H.FP32_MIXED, steps=8, tile=PAIR_TILES[1], kchunk=0)
    _check(Ug, Uo, 3, TOL_FP32, "3d source, paired tile")
    tots = []
    for tile in (0, PAIR_TILES[2]):
        h = H.Hydro.from_problem(pf, precision=H.FP32_MIXED)
        h.set_tile(tile, 0)
        h.advance(2, pf.cfl)
        tots.append(np.asarray(h.step_totals()))
        h.close()
    np.testing.assert_allclose(tots[1], tots[0], rtol=1e-6, atol=1e-9 * np.max(np.abs(tots[0])))


TMA_TILES = (9, 10)  # 3D FP32 tiles whose stage 1 stages the state planes with TMA


@pytest.mark.parametrize("bc", ["periodic", "reflect", "outflow", "mixed"])
def test_tma_tile_identical_under_every_boundary(bc):
    """The tiles that stage the state planes with TMA (3D FP32) give
    bitwise the state of tile 0 under every boundary rule, on a mesh ragged
    in x (72 = 2 x 32 + 8 columns) and in y (29 rows), with several plane
    counts per CTA; its ghost cells come from global memory through the
    boundary map, its planes along z from the mapped plane."""
    codes = {"periodic": P.PERIODIC, "reflect": P.REFLECT, "outflow": P.OUTFLOW, "mixed": P.REFLECT}
    pr = P.random_blocks(3, (72, 29, 23), seed=17, bc=codes[bc])
    if bc == "mixed":
        pr = pr.with_(bc_lo=(P.REFLECT, P.OUTFLOW, P.PERIODIC), bc_hi=(P.OUTFLOW, P.REFLECT, P.PERIODIC))
    for solver in (H.HLL, H.HLLC):
        ref, _ = gpu_run(pr, H.FP32_MIXED, solver=solver, steps=3, tile=0, kchunk=0)
        for tile in TMA_TILES:
            for kc in (0, 5, 23):
                U, _ = gpu_run(pr, H.FP32_MIXED, solver=solver, steps=3, tile=tile, kchunk=kc)
                np.testing.assert_array_equal(U, ref, err_msg=f"solver {solver} tile {tile} kchunk {kc}")


DW_CASES = {
    "sod_1d": lambda: (P.sod(256), 200),
    "blocks_2d_reflect": lambda: (P.random_blocks(2, (70, 45), seed=4, bc=P.REFLECT), 20),
    "blocks_3d_periodic": lambda: (P.random_blocks(3, (36, 28, 22), seed=6, bc=P.PERIODIC), 8),
    "blocks_3d_outflow": lambda: (P.random_blocks(3, (30, 34, 26), seed=8, bc=P.OUTFLOW), 8),
    "sedov_48": lambda: (P.sedov_3d(48), 40),
    "stretched_40": lambda: (P.stretched_pulse_3d(40, steps=10), 10),
    "kelvin_helmholtz_64": lambda: (P.kelvin_helmholtz(64, seed=5), 40),
    "rayleigh_taylor_32x96": lambda: (P.rayleigh_taylor(32, 96), 40),
}


@pytest.mark.parametrize("case", sorted(DW_CASES))
def test_double_word_matches_oracle(case):
    """Double-word FP32 pairs (GENASIS_FP64_DW) hold the FP64 parity bar."""
    pr, steps = DW_CASES[case]()
    Uo, to = oracle_run(pr, steps=steps)
    Ug, tg = gpu_run(pr, H.FP64_DW, steps=steps)
    assert tg == pytest.approx(to, rel=1e-10)
    _check(Ug, Uo, pr.ndim, TOL_FP64, f"double-word {case}")


def _tube_3d(tube, axis, n_cross=6):
    """The 1D problem `tube` as a 3D box with the tube along `axis` (0 = x, an
    in-plane axis of the tiles; 2 = z, the march axis), periodic and uniform
    across it: every row along `axis` evolves like the 1D problem."""
    n = tube.n[0]
    nn = [n_cross, n_cross + 1, n_cross + 2]
    nn[axis] = n
    shape = tuple(reversed(nn))
    ax = 2 - axis  # numpy axis of `axis`
    bshape = [1, 1, 1]
    bshape[ax] = n
    rho = np.broadcast_to(tube.rho.reshape(bshape), shape).copy()
    p = np.broadcast_to(tube.p.reshape(bshape), shape).copy()
    vel = np.zeros((3,) + shape)
    vel[axis] = np.broadcast_to(tube.vel[0].reshape(bshape), shape)
    widths = [P.uniform_widths(nn[q], 0.0, nn[q] / n) for q in range(3)]
    widths[axis] = tube.widths[0]
    lo = [P.PERIODIC] * 3
    hi = [P.PERIODIC] * 3
    lo[axis], hi[axis] = tube.bc_lo[0], tube.bc_hi[0]
    return tube.with_(name=f"{tube.name}_3d_axis{axis}", ndim=3, n=tuple(nn), widths=widths, bc_lo=tuple(lo),
                      bc_hi=tuple(hi), rho=rho, vel=vel, p=p, origin=(0.0, 0.0, 0.0))


ALL_PRECISIONS = ((H.FP64, TOL_FP64), (H.FP32_MIXED, TOL_FP32), (H.FP64_DW, TOL_FP64))
NEAR_VACUUM = {
    # Einfeldt 1-2-0-3 (Sec. 4.2.1): the two rarefactions leave a near-vacuum
    # in the middle, where the kinetic energy is most of G and e = G - S^2/(2D)
    # cancels; the FP32-mixed recovery takes its FP64 branch there
    "double_rarefaction_1d": lambda: P.double_rarefaction(128),
    "double_rarefaction_3d_x": lambda: _tube_3d(P.double_rarefaction(128), 0),
    "double_rarefaction_3d_z": lambda: _tube_3d(P.double_rarefaction(128), 2),
    # Woodward-Colella interacting blast waves (Sec. 4.2.2): pressure ratios of
    # 1e5, reflecting walls, to t = 0.038
    "blast_waves_1d": lambda: P.blast_waves(400),
    "blast_waves_3d_z": lambda: _tube_3d(P.blast_waves(400), 2, n_cross=4),
}


@pytest.mark.parametrize("case", sorted(NEAR_VACUUM))
def test_near_vacuum_and_blast_waves_every_precision(case):
    """The cases that stress the FP32 cancellation branch and the largest
    pressure ratios, run to their end times in FP64, FP32-mixed and double
    word against the oracle."""
    pr = NEAR_VACUUM[case]()
    Uo, to = oracle_run(pr, t_end=pr.t_end)
    if pr.ndim == 1 and pr.name == "double_rarefaction":
        # the cancellation branch is exercised: somewhere the kinetic energy
        # density exceeds half of G
        ke = 0.5 * Uo[1] ** 2 / Uo[0]
        assert np.any(ke > 0.5 * Uo[2])
    for precision, tol in ALL_PRECISIONS:
        Ug, tg = gpu_run(pr, precision, t_end=pr.t_end)
        assert tg == pytest.approx(to, rel=1e-12 if precision != H.FP32_MIXED else 1e-6)
        _check(Ug, Uo, pr.ndim, tol, f"{case} prec={precision}")


@pytest.mark.parametrize("shape", [(200, 20), (20, 200)])
def test_shock_switch_matches_oracle_2d(shape):
    """HLLC with the HLL switch (GENASIS_HLLC_SWITCH) on the odd-even planar
    shock, moving along x (in-plane faces switch) or along y (the march axis)."""
    nx, ny = shape
    pr = P.planar_shock(nx=max(shape), ny=min(shape), solver=P.HLLC_SWITCH)
    if nx < ny:  # the same shock moving along y
        pr = pr.with_(n=(ny // 10, ny, 1)[:2] + (1,), widths=[pr.widths[1], pr.widths[0]],
                      bc_lo=(P.PERIODIC, P.OUTFLOW, P.PERIODIC), bc_hi=(P.PERIODIC, P.OUTFLOW, P.PERIODIC),
                      rho=np.ascontiguousarray(pr.rho.T), p=np.ascontiguousarray(pr.p.T),
                      vel=np.ascontiguousarray(np.stack([pr.vel[1].T, pr.vel[0].T])))
    Uo, _ = oracle_run(pr, steps=60)
    for precision, tol in PRECISIONS:
        Ug, _ = gpu_run(pr, precision, steps=60)
        _check(Ug, Uo, 2, tol, f"shock switch {shape} prec={precision}")


@pytest.mark.parametrize("axis", [0, 2])
def test_shock_switch_matches_oracle_3d(axis):
    pr = P.planar_shock_3d(n_long=64, n_cross=10, axis=axis, solver=P.HLLC_SWITCH)
    Uo, _ = oracle_run(pr, steps=25)
    for precision, tol in PRECISIONS:
        Ug, _ = gpu_run(pr, precision, steps=25)
        _check(Ug, Uo, 3, tol, f"shock switch 3d axis {axis} prec={precision}")


@pytest.mark.parametrize("bc", [P.PERIODIC, P.REFLECT, P.OUTFLOW])
@pytest.mark.parametrize("shape", [(4, 3, 5), (36, 9, 3), (100, 17, 70), (8, 2, 3), (2, 5, 4)])
def test_shock_switch_edge_meshes_3d(shape, bc):
    """The switch on piecewise-constant random blocks at the edges of the
    detector's passes (in FP32 the stage-1 detector stages planes by TMA):
    rows of 4 cells, axes of 3 cells (almost every cell in the boundary
    shell that is flagged cell by cell), tiles ragged in x and y, a z march
    in chunks; axes of 2 cells (the register-tile pass in both stages); every
    boundary kind, both precisions."""
    pr = P.random_blocks(3, shape, seed=sum(shape), bc=bc)
    Uo, _ = oracle_run(pr, solver=P.HLLC_SWITCH, steps=4)
    for precision, tol in PRECISIONS:
        Ug, _ = gpu_run(pr, precision, solver=P.HLLC_SWITCH, steps=4)
        _check(Ug, Uo, 3, tol, f"switch blocks {shape} bc={bc} prec={precision}")


def _step_from_evolved(prob, precisions, what, steps=20, tile=None):
    """`steps` GPU steps, so that a moving front exists, then one GPU step from
    that state against one oracle step from the same state widened to FP64,
    with the oracle's dt.  Returns {precision: (GPU state, start state, dt,
    rel L1)} for further checks."""
    g = O.Grid(prob)
    out = {}
    for precision, tol in precisions:
        h = H.Hydro.from_problem(prob, precision=precision)
        if tile is not None and precision == H.FP32_MIXED:
            h.set_tile(*tile)
        t0 = h.advance(steps, prob.cfl)
        U0 = h.get_conserved(precision=H.FP64)
        t1 = h.advance(1, prob.cfl)
        Ug = h.get_conserved(precision=H.FP64)
        h.close()
        dt = prob.cfl * O.cfl_dt(g, U0)
        assert t1 - t0 == pytest.approx(dt, rel=1e-5 if precision == H.FP32_MIXED else 1e-9)
        Uo = O.step(g, U0, dt)
        e, _ = check(Ug, Uo, prob.ndim, tol, f"{what} step {steps + 1} prec={precision}")
        out[precision] = (Ug, U0, dt, e)
    return out


def test_shock_switch_full_size_step_from_an_evolved_state():
    """The switch at the bench's size (256^3 blast) and, in FP32, its launch
    configuration (tile 8, 40 planes per CTA): a moving shock front sets flags
    in both detector passes.  Plain HLLC from the same state is at least 10x
    farther from the GPU result than the switched oracle step, so the switch
    acted in that step."""
    prob = P.sedov_3d(256, solver=P.HLLC_SWITCH)
    res = _step_from_evolved(prob, PRECISIONS, "switch 256^3", tile=(8, 40))
    gh = O.Grid(prob, solver=P.HLLC)
    for precision, (Ug, U0, dt, e) in res.items():
        Uh = O.step(gh, U0, dt)
        assert rel_l1(Ug, Uh, 3).max() > 10.0 * e.max(), (precision, rel_l1(Ug, Uh, 3), e)


def test_full_size_hll_and_double_word_steps_from_an_evolved_state():
    """The other blast variants of the bench at 256^3: HLL in FP64 and FP32
    (tile 8, 40 planes per CTA) and HLLC in double word, one step from a state
    20 steps in."""
    _step_from_evolved(P.sedov_3d(256, solver=P.HLL), PRECISIONS, "hll 256^3", tile=(8, 40))
    _step_from_evolved(P.sedov_3d(256), ((H.FP64_DW, TOL_FP64),), "double word 256^3")


def test_shock_switch_tiles_identical():
    """Every tile compiled with the switch (3D FP32) gives bitwise the same state."""
    pr = P.planar_shock_3d(n_long=64, n_cross=10, axis=0, solver=P.HLLC_SWITCH)
    ref, _ = gpu_run(pr, H.FP32_MIXED, steps=10, tile=0, kchunk=0)
    h = H.Hydro.from_problem(pr, precision=H.FP32_MIXED)
    count = h.tile_info()["tile_count"]
    h.close()
    done = 0
    for tile in range(1, count):
        try:
            U, _ = gpu_run(pr, H.FP32_MIXED, steps=10, tile=tile, kchunk=7)
        except H.HydroError as e:
            if e.code != H.EINVAL:
                raise
            continue  # not compiled with the switch
        np.testing.assert_array_equal(U, ref, err_msg=f"tile {tile}")
        done += 1
    assert done >= 1


def test_shock_switch_suppresses_odd_even_gpu():
    """The odd-even decoupling of HLLC behind a Mach 20 shock (from 1e-6
    noise) on the GPU, and its absence with the switch; shock-free flows are
    plain HLLC bitwise."""
    dev = {}
    for solver in (P.HLLC, P.HLLC_SWITCH):
        pr = P.planar_shock(solver=solver)
        U, _ = gpu_run(pr, H.FP32_MIXED, steps=600)
        dev[solver] = np.abs(U[0] - U[0].mean(axis=0, keepdims=True)).max()
    assert dev[P.HLLC] > 0.1 and dev[P.HLLC_SWITCH] < 1e-4, dev
    pr = P.kelvin_helmholtz(64, seed=2)
    a, _ = gpu_run(pr, H.FP32_MIXED, solver=P.HLLC, steps=20)
    b, _ = gpu_run(pr, H.FP32_MIXED, solver=P.HLLC_SWITCH, steps=20)
    np.testing.assert_array_equal(a, b)


def test_fixed_dt_step_matches_oracle():
    """genasis_hydro_step with a caller-given dt."""
    pr = P.random_blocks(2, (64, 50), seed=9, bc=P.OUTFLOW)
    g = O.Grid(pr)
    Uo = O.initial_state(pr, g)
    h = H.Hydro.from_problem(pr, precision=H.FP64)
    for dt in (1e-3, 2e-3, 5e-4):
        h.step(dt)
        Uo = O.step(g, Uo, dt)
    _check(h.get_conserved(), Uo, 2, TOL_FP64, "fixed dt")
    h.close()


def test_compute_dt_and_totals_match_oracle():
    pr = P.random_blocks(3, (33, 29, 17), seed=12, bc=P.PERIODIC)
    g = O.Grid(pr)
    U0 = O.initial_state(pr, g)
    for precision, tol in ((H.FP64, 1e-14), (H.FP32_MIXED, 1e-6)):
        h = H.Hydro.from_problem(pr, precision=precision)
        assert h.compute_dt(0.4) == pytest.approx(0.4 * O.cfl_dt(g, U0), rel=tol)
        np.testing.assert_allclose(h.totals(), O.totals(g, U0), rtol=tol, atol=tol * np.abs(O.totals(g, U0)).max())
        h.close()


def test_conservation_periodic_gpu():
    """Totals stay constant to roundoff on a periodic box (FP64 and FP32)."""
    pr = P.smooth_periodic(3, 48, seed=4, nonuniform=True)
    for precision, tol in ((H.FP64, 1e-13), (H.FP32_MIXED, 2e-6)):
        h = H.Hydro.from_problem(pr, precision=precision)
        t0 = h.totals()
        h.advance(30, 0.4)
        t1 = h.totals()
        np.testing.assert_allclose(t1, t0, rtol=0, atol=tol * np.abs(t0).max())
        h.close()


def test_device_and_host_pointers_agree():
    """set/get through torch CUDA tensors equals the host-pointer path."""
    import torch
    pr = P.random_blocks(2, (40, 30), seed=1)
    a = H.Hydro.from_problem(pr, precision=H.FP32_MIXED)
    b = H.Hydro(pr.ndim, pr.n, pr.widths, pr.bc_lo, pr.bc_hi, pr.gamma, pr.solver, pr.theta, H.FP32_MIXED)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    b.set_primitive(dev(pr.rho), dev(pr.vel), dev(pr.p))
    for h in (a, b):
        h.advance(5, 0.4)
    Ua = a.get_conserved()
    Ub = torch.empty((4, 30, 40), dtype=torch.float32, device="cuda")
    b.get_conserved(Ub)
    np.testing.assert_array_equal(Ua, Ub.cpu().numpy())
    # resume: set_conserved of a saved state continues bitwise identically
    c = H.Hydro(pr.ndim, pr.n, pr.widths, pr.bc_lo, pr.bc_hi, pr.gamma, pr.solver, pr.theta, H.FP32_MIXED)
    c.set_conserved(Ua)
    a.advance(3, 0.4)
    c.advance(3, 0.4)
    np.testing.assert_array_equal(a.get_conserved(), c.get_conserved())
    for h in (a, b, c):
        h.close()


def test_async_copies_pipelined_over_handles():
    """Three handles on three streams, each step's state copied in from
    page-locked host memory and back without waiting in between, give the
    same states as the synchronous path."""
    import torch
    pr = P.random_blocks(3, (24, 20, 18), seed=12, bc=P.REFLECT)
    ref = H.Hydro.from_problem(pr, precision=H.FP32_MIXED)
    U0 = ref.get_conserved()
    ref.advance(1, 0.3)
    want = ref.get_conserved()
    ref.close()
    streams = [torch.cuda.Stream() for _ in range(3)]
    hs = [H.Hydro.from_problem(pr, precision=H.FP32_MIXED, stream=s.cuda_stream, set_state=False) for s in streams]
    ins = [torch.from_numpy(U0.copy()).pin_memory() for _ in range(3)]
    outs = [torch.empty(U0.shape, dtype=torch.float32).pin_memory() for _ in range(6)]
    for k in range(6):
        h = hs[k % 3]
        if k >= 3:
            h.sync()
        h.set_conserved_async(ins[k % 3])
        h.advance(1, 0.3, sync=False)
        h.get_conserved_async(outs[k])
    for h in hs:
        h.sync()
    for k in range(6):
        np.testing.assert_array_equal(outs[k].numpy(), want, err_msg=f"step {k}")
    with pytest.raises(ValueError):
        hs[0].set_conserved_async(U0.astype(np.float64))  # would copy into a temporary
    for h in hs:
        h.close()


def test_nonphysical_state_sets_status():
    pr = P.sod(64)
    pr.p[10] = -1.0
    h = H.Hydro.from_problem(pr, precision=H.FP64)
    with pytest.raises(H.NonPhysicalState):
        h.advance(1, 0.5, sync=True)
    h.clear_status()
    h.close()


# ----------------------------------------------------------- full-size workloads

def _one_step_full(prob, precisions, pair_tile=None):
    """One device-CFL step at full size, in the benchmark's launch
    configuration, against one oracle step with the oracle's dt."""
    g = O.Grid(prob)
    U0 = O.initial_state(prob, g)
    dt = prob.cfl * O.cfl_dt(g, U0)
    Uo = O.step(g, U0, dt)
    del U0
    runs = [(precision, tol, None) for precision, tol in precisions]
    if pair_tile is not None:
        runs.append((H.FP32_MIXED, TOL_FP32, pair_tile))
    for precision, tol, tile in runs:
        h = H.Hydro.from_problem(prob, precision=precision)
        if tile is not None:
            h.set_tile(tile, 40)
        t = h.advance(1, prob.cfl)
        assert t == pytest.approx(dt, rel=1e-12 if precision == H.FP64 else 1e-6)
        Ug = h.get_conserved(precision=H.FP64)
        h.close()
        _check(Ug, Uo, prob.ndim, tol, f"{prob.name} prec={precision} tile={tile}")


def test_sedov_full_size_one_step():
    """256^3 point blast, one step, in FP64, FP32-mixed and double word; FP32
    also on the paired tile that the bench offers, at 40 planes per CTA."""
    _one_step_full(P.sedov_3d(256), ALL_PRECISIONS, pair_tile=PAIR_TILES[2])


def test_stretched_pulse_full_size_one_step():
    """320^3 centrally refined mesh, one FP32-mixed step."""
    _one_step_full(P.stretched_pulse_3d(320), ((H.FP32_MIXED, TOL_FP32),))


def test_sedov_full_size_symmetry_and_mass():
    """256^3, 20 FP64 steps: octant mirror symmetry and mass/energy totals."""
    pr = P.sedov_3d(256)
    h = H.Hydro.from_problem(pr, precision=H.FP64)
    t0 = h.totals()
    h.advance(20, pr.cfl)
    t1 = h.totals()
    U = h.get_conserved()
    h.close()
    assert t1[0] == pytest.approx(t0[0], rel=1e-12)
    assert t1[4] == pytest.approx(t0[4], rel=1e-12)
    np.testing.assert_allclose(U[0], U[0][::-1, ::-1, ::-1], rtol=1e-12)
    np.testing.assert_allclose(U[0], np.transpose(U[0], (2, 1, 0)), rtol=1e-12)


def test_largest_mesh_rows_match_the_1d_oracle():
    """A mesh whose arrays hold more than 2^32 values per state (1100^3
    cells x 5 variables, 80 GB of FP32 state): a Sod tube along x, uniform in
    y and z, one CFL step.  Every (y, z) row must equal the 1D oracle's step
    of the same tube (fluxes along y and z cancel exactly); rows are sampled
    across the mesh, including the last planes, whose offsets need 64 bits."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    if free < 200e9:
        pytest.skip(f"needs ~150 GB of free device memory, {free / 1e9:.0f} GB free")
    n = 1100
    tube = P.sod(n)
    U1, t1 = oracle_run(tube, steps=1)   # 1D oracle, same CFL rule (1D speeds only)
    shape = (n, n, n)
    rho = torch.from_numpy(tube.rho).cuda().reshape(1, 1, n).expand(shape).contiguous()
    vel = torch.zeros((3,) + shape, dtype=torch.float64, device="cuda")
    p = torch.from_numpy(tube.p).cuda().reshape(1, 1, n).expand(shape).contiguous()
    w = tube.widths[0]
    pr3 = P.Problem(name="sod_tube_3d", ndim=3, n=(n, n, n), widths=[w, w, w],
                    bc_lo=(P.OUTFLOW, P.PERIODIC, P.PERIODIC), bc_hi=(P.OUTFLOW, P.PERIODIC, P.PERIODIC),
                    gamma=tube.gamma, rho=np.zeros(1), vel=np.zeros(1), p=np.zeros(1), solver=tube.solver,
                    theta=tube.theta, cfl=tube.cfl)
    h = H.Hydro.from_problem(pr3, precision=H.FP32_MIXED, set_state=False)
    torch.cuda.synchronize()  # the library's stream does not wait for torch's
    h.set_primitive(rho, vel, p)
    del rho, vel, p
    torch.cuda.empty_cache()
    tg = h.advance(1, tube.cfl)
    out = torch.empty((5,) + shape, dtype=torch.float32, device="cuda")
    h.get_conserved(out)
    h.close()
    assert tg == pytest.approx(t1, rel=1e-6)
    want = np.stack([U1[0], U1[1], np.zeros(n), np.zeros(n), U1[2]])
    for (k, j) in ((0, 0), (n // 2, 7), (n - 1, n - 1), (n - 2, 3), (517, n - 5)):
        row = out[:, k, j, :].double().cpu().numpy()
        err = rel_l1(row[[0, 1, 4]], want[[0, 1, 4]], 1)
        assert np.all(err <= TOL_FP32), (k, j, err)
        assert np.abs(row[2:4]).max() == 0.0
    del out
    torch.cuda.empty_cache()


def test_cell_centers_from_origin():
    """genasis_hydro_get_centers: origin plus the running widths (the
    geometric centres of Sec. 3.1), on a stretched mesh with an offset origin."""
    pr = P.random_blocks(3, (12, 9, 7), seed=5, bc=P.OUTFLOW).with_(origin=(-0.3, 1.25, 7.0))
    h = H.Hydro.from_problem(pr, precision=H.FP64)
    for q in range(3):
        np.testing.assert_allclose(h.centers(q), pr.centers(q), rtol=1e-15, atol=1e-15)
    with pytest.raises(H.HydroError):
        h.centers(3)
    h.close()
