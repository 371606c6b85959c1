"""Training and evaluation of the learned flux correction on the periodic
shear layer (2D Kelvin-Helmholtz set-up of problems.kelvin_helmholtz).

Every step runs in the CUDA library; PyTorch only holds device buffers and
gathers random mini-batches.

Targets.  Over one coarse step dt_c, a fine run at `factor` times the
resolution takes `factor` steps of dt_c / factor.  The time integral of its
face fluxes through the fine faces that make up a coarse face, divided by
dt_c and the coarse face area, is the flux that would move the restricted
fine state exactly.  The target of a coarse face is that flux minus the plain
coarse scheme's own effective RK2 flux from the restricted state, in the face
frame and divided by the face's flux scale.  The network sees the features
of the restricted state.

Evaluation.  Truth is the plain fine run restricted to the coarse mesh.  The
plain runs at 1x, 2x and 3x the coarse resolution (restricted to the coarse
mesh) give the error-vs-GPU-time frontier; the learned coarse run is one
more point.  All errors are the relative L1 norm of Eq. L1ErrorNorm on the
density.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np

from . import hydro as H
from . import problems as P


def _torch():
    import torch
    return torch


_STREAM = None


def _stream():
    """One dedicated CUDA stream, made current, shared by torch and every
    library handle here so that their work is ordered."""
    global _STREAM
    torch = _torch()
    if _STREAM is None:
        _STREAM = torch.cuda.Stream()
    torch.cuda.set_stream(_STREAM)
    return _STREAM


def _restricted(h, factor):
    torch = _torch()
    ny, nx = h.shape
    out = torch.empty((4, ny // factor, nx // factor), dtype=torch.float32, device="cuda")
    if factor == 1:
        h.get_conserved(out)
        return out
    return h.restrict(out, factor)


def generate(seeds, n_coarse=256, factor=4, t_end=1.0, snap_every=16, keep_fraction=1.0 / 16, cfl=0.5,
             solver=P.HLLC, rng_seed=0, log=None):
    """Training pairs (X [N, 32] bf16, T [N, 4] f32, CUDA) from fine runs."""
    torch = _torch()
    st = _stream()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(rng_seed)
    nc = n_coarse * n_coarse
    Xs, Ts = [], []
    for seed in seeds:
        pf = P.kelvin_helmholtz(n_coarse * factor, seed=seed, solver=solver)
        pc = P.kelvin_helmholtz(n_coarse, seed=seed, solver=solver)
        fine = H.Hydro.from_problem(pf, precision=H.FP32_MIXED, stream=st.cuda_stream)
        coarse = H.Hydro.from_problem(pc, precision=H.FP32_MIXED, set_state=False, stream=st.cuda_stream)
        feat = H.Learned(pc, stream=st.cuda_stream)
        Ft = torch.zeros((2, 4, n_coarse, n_coarse), dtype=torch.float64, device="cuda")
        Fp = torch.zeros_like(Ft)
        X = torch.empty((2 * nc, 32), dtype=torch.bfloat16, device="cuda")
        sc = torch.empty((2 * nc, 4), dtype=torch.float32, device="cuda")
        T = torch.empty((2 * nc, 4), dtype=torch.float32, device="cuda")
        t, k = 0.0, 0
        while t < t_end:
            Uc = _restricted(fine, factor)
            if k % snap_every == 0:
                coarse.set_conserved(Uc)
                feat.set_conserved(Uc)
                dt_c = min(coarse.compute_dt(cfl), factor * fine.compute_dt(cfl))
                Fp.zero_()
                coarse.step(dt_c)
                coarse.accumulate_face_flux(Fp, 1, 1.0)
                Ft.zero_()
                for _ in range(factor):
                    fine.step(dt_c / factor)
                    fine.accumulate_face_flux(Ft, factor, 1.0 / factor)
                feat.features(X, sc)
                feat.targets(Ft, Fp, sc, T)
                keep = torch.rand(2 * nc, generator=gen, device="cuda") < keep_fraction
                Xs.append(X[keep].clone())
                Ts.append(T[keep].clone())
                t = fine.time
            else:
                t = fine.advance(factor, cfl)
            k += 1
        fine.close()
        coarse.close()
        feat.close()
        if log:
            log(f"seed {seed}: {sum(x.shape[0] for x in Xs)} samples so far")
    return torch.cat(Xs), torch.cat(Ts)


def _init_params(seed=0):
    """He-style uniform initial weights with a zero last layer (the corrected
    scheme starts as the plain one); layout of genasis_mlp_param_count()."""
    rng = np.random.default_rng(seed)
    nin, nh, nout = 24, 64, 4
    parts = [rng.uniform(-1, 1, nh * nin) * math.sqrt(3.0 / nin), np.zeros(nh),
             rng.uniform(-1, 1, nh * nh) * math.sqrt(3.0 / nh), np.zeros(nh), np.zeros(nout * nh), np.zeros(nout)]
    return np.concatenate(parts).astype(np.float32)


def train(X, T, epochs=4, batch=32768, lr=2e-3, init_seed=0, log=None):
    """Adam with cosine decay over random mini-batches; returns FP32 params."""
    torch = _torch()
    st = _stream()
    n = X.shape[0]
    opt = H.MlpOptimizer(_init_params(init_seed), stream=st)
    steps = max(1, epochs * (n // batch))
    s = 0
    history = []
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda")
        for b in range(n // batch):
            idx = perm[b * batch:(b + 1) * batch]
            rate = lr * 0.5 * (1.0 + math.cos(math.pi * s / steps))
            loss = opt.step(X[idx].contiguous(), T[idx].contiguous(), rate, want_loss=(b % 50 == 0))
            if b % 50 == 0:
                history.append((ep, b, loss))
                if log:
                    log(f"epoch {ep} batch {b} loss {loss:.4e}")
            s += 1
    params = opt.params()
    opt.close()
    return params, history


def _l1(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def _timed(run, stream):
    """(result, device seconds between events on `stream`, wall seconds)."""
    torch = _torch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    out = run()
    e1.record(stream)
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1) * 1e-3, time.perf_counter() - t0


def output_limit(T, quantile=0.999, factor=2.0):
    """Bound for the network outputs: `factor` times the `quantile` of |T|."""
    torch = _torch()
    a = T.abs().flatten()
    k = max(1, int(quantile * a.numel()))
    return float(factor * torch.kthvalue(a.float().cpu(), k).values)


def evaluate(params, seeds=range(64, 72), n_coarse=256, t_evals=(0.6, 1.0), cfl=0.5, solver=P.HLLC, log=None,
             variants=(("learned", True, math.inf),)):
    """L1(rho) against the restricted 4x run and GPU time, for plain runs at
    1x, 2x, 3x and the learned coarse run in each variant (name, FCT limiter
    on, output bound), per seed and evaluation time."""
    st = _stream()
    rows = []
    for seed in seeds:
        for t_eval in t_evals:
            res = {"seed": int(seed), "t": t_eval}
            fine_n = 4 * n_coarse
            pf = P.kelvin_helmholtz(fine_n, seed=seed, solver=solver)
            h = H.Hydro.from_problem(pf, precision=H.FP32_MIXED, stream=st.cuda_stream)
            _, gpu_s, _ = _timed(lambda: h.evolve(cfl, t_eval), st)
            truth = _restricted(h, 4).cpu().numpy()
            res["time_4x"] = gpu_s
            h.close()
            for m in (1, 2, 3):
                pr = P.kelvin_helmholtz(m * n_coarse, seed=seed, solver=solver)
                h = H.Hydro.from_problem(pr, precision=H.FP32_MIXED, stream=st.cuda_stream)
                _, gpu_s, _ = _timed(lambda: h.evolve(cfl, t_eval), st)
                res[f"l1_{m}x"] = _l1(_restricted(h, m).cpu().numpy()[0], truth[0])
                res[f"time_{m}x"] = gpu_s
                h.close()
            pc = P.kelvin_helmholtz(n_coarse, seed=seed, solver=solver)
            for name, fct, limit in variants:
                L = H.Learned(pc, params=params, stream=st.cuda_stream)
                L.set_fct(fct)
                L.set_limit(limit)
                L.set_primitive(pc.rho, pc.vel, pc.p)
                try:
                    t_got, gpu_s, _ = _timed(lambda: L.evolve(cfl, t_eval, max_chunks=400), st)
                    if t_got < t_eval:
                        raise H.HydroError(0, f"time step collapsed: t = {t_got:.4g} after 400 chunks")
                    res[f"l1_{name}"] = _l1(L.get_conserved()[0], truth[0])
                except H.HydroError as e:   # the run left the physical states
                    res[f"l1_{name}"], gpu_s = math.inf, math.inf
                    res[f"error_{name}"] = str(e)
                res[f"time_{name}"] = gpu_s
                res[f"fallback_cells_{name}"] = L.fallbacks()
                L.close()
            rows.append(res)
            if log:
                log(json.dumps(res))
    return rows


def short_horizon(params, seeds=range(64, 72), n_coarse=256, factor=4, t_starts=(0.2, 0.6), horizons=(1, 4, 16, 64),
                  cfl=0.5, solver=P.HLLC, log=None):
    """Error of the coarse schemes over a few coarse steps from the restricted
    fine state, against the fine run over the same steps (the quantity the
    network is trained on, at horizon 1, and how it carries over as the
    coarse run drifts).  Plain, learned with FCT and learned unlimited take
    the same dt sequence (from the plain coarse state and the fine CFL)."""
    torch = _torch()
    st = _stream()
    rows = []
    for seed in seeds:
        pf = P.kelvin_helmholtz(n_coarse * factor, seed=seed, solver=solver)
        pc = P.kelvin_helmholtz(n_coarse, seed=seed, solver=solver)
        fine = H.Hydro.from_problem(pf, precision=H.FP32_MIXED, stream=st.cuda_stream)
        for t0 in t_starts:
            fine.evolve(cfl, t0)
            Uc = _restricted(fine, factor).clone()
            plain = H.Hydro.from_problem(pc, precision=H.FP32_MIXED, set_state=False, stream=st.cuda_stream)
            plain.set_conserved(Uc)
            runs = {}
            for name, fct in (("learned_fct", True), ("learned_unlimited", False)):
                L = H.Learned(pc, params=params, stream=st.cuda_stream)
                L.set_fct(fct)
                L.set_conserved(Uc)
                runs[name] = L
            out = torch.empty_like(Uc)
            alive = {k: True for k in runs}
            for m in range(1, max(horizons) + 1):
                dt = min(plain.compute_dt(cfl), factor * fine.compute_dt(cfl))
                plain.step(dt)
                for k, L in runs.items():
                    if alive[k]:
                        L.step(dt)
                for _ in range(factor):
                    fine.step(dt / factor)
                if m in horizons:
                    truth = _restricted(fine, factor).cpu().numpy()[0]
                    res = {"seed": int(seed), "t0": t0, "steps": m,
                           "l1_change": _l1(Uc[0].cpu().numpy(), truth),
                           "l1_plain": _l1(plain.get_conserved()[0], truth)}
                    for k, L in runs.items():
                        if alive[k]:
                            try:
                                L.get_conserved(out)
                                U = out.cpu().numpy()
                                ok = bool(np.isfinite(U).all() and U[0].min() > 0)
                            except H.HydroError:   # left the physical states
                                ok = False
                            alive[k] = ok
                            res[f"l1_{k}"] = _l1(U[0], truth) if ok else math.inf
                        else:
                            res[f"l1_{k}"] = math.inf
                    rows.append(res)
                    if log:
                        log(json.dumps(res))
            plain.close()
            for L in runs.values():
                L.close()
        fine.close()
    summary = []
    for t0 in t_starts:
        for m in horizons:
            sel = [r for r in rows if r["t0"] == t0 and r["steps"] == m]
            row = {"t0": t0, "steps": m, "l1_change": float(np.mean([r["l1_change"] for r in sel])),
                   "l1_plain": float(np.mean([r["l1_plain"] for r in sel]))}
            for k in ("learned_fct", "learned_unlimited"):
                v = float(np.mean([r[f"l1_{k}"] for r in sel]))
                row[f"l1_{k}"] = v
                row[f"ratio_{k}"] = v / row["l1_plain"]
            summary.append(row)
    return rows, summary


def restart_frontier(params, seeds=range(64, 72), n_coarse=256, t_starts=(0.2, 0.6), spans=(0.05, 0.2), cfl=0.5,
                     solver=P.HLLC, log=None):
    """The equal-L1 comparison from restarts: from the 4x run's state at t0,
    restricted to 1x and 2x, the plain 1x and 2x runs and the learned 1x run
    (FCT) each advance by `span` with their own CFL steps.  L1(rho) against
    the 4x run restricted to 1x at t0 + span, and each run's GPU time (the 4x
    run's own time over the span beside them).  Unlike `evaluate`, the runs do
    not inherit the coarse scheme's drift from t = 0."""
    torch = _torch()
    st = _stream()
    rows = []
    for seed in seeds:
        pf = P.kelvin_helmholtz(4 * n_coarse, seed=seed, solver=solver)
        fine = H.Hydro.from_problem(pf, precision=H.FP32_MIXED, stream=st.cuda_stream)
        for t0 in t_starts:
            fine.evolve(cfl, t0)
            Uf0 = fine.get_conserved(torch.empty((4,) + fine.shape, dtype=torch.float32, device="cuda"))
            U1 = _restricted(fine, 4).clone()
            U2 = _restricted(fine, 2).clone()
            for span in spans:
                fine.set_conserved(Uf0)
                fine.time = t0
                res = {"seed": int(seed), "t0": t0, "span": span}
                _, res["time_4x"], _ = _timed(lambda: fine.evolve(cfl, t0 + span), st)
                truth = _restricted(fine, 4).cpu().numpy()[0]
                for m, U0 in ((1, U1), (2, U2)):
                    pm = P.kelvin_helmholtz(m * n_coarse, seed=seed, solver=solver)
                    h = H.Hydro.from_problem(pm, precision=H.FP32_MIXED, set_state=False, stream=st.cuda_stream)
                    h.set_conserved(U0)
                    _, res[f"time_{m}x"], _ = _timed(lambda: h.evolve(cfl, span), st)
                    res[f"l1_{m}x"] = _l1(_restricted(h, m).cpu().numpy()[0], truth)
                    h.close()
                pc = P.kelvin_helmholtz(n_coarse, seed=seed, solver=solver)
                L = H.Learned(pc, params=params, stream=st.cuda_stream)
                L.set_fct(True)
                L.set_conserved(U1)
                try:
                    t_got, res["time_learned"], _ = _timed(lambda: L.evolve(cfl, span, max_chunks=400), st)
                    if t_got < span:
                        raise H.HydroError(0, f"time step collapsed: t = {t_got:.4g}")
                    res["l1_learned"] = _l1(L.get_conserved()[0], truth)
                except H.HydroError as e:
                    res["l1_learned"], res["time_learned"] = math.inf, math.inf
                    res["error_learned"] = str(e)
                L.close()
                rows.append(res)
                if log:
                    log(json.dumps(res))
        fine.close()
    summary = []
    for t0 in t_starts:
        for span in spans:
            sel = [r for r in rows if r["t0"] == t0 and r["span"] == span]
            mean = lambda k: float(np.mean([r[k] for r in sel]))
            pts = [(mean(f"l1_{m}x"), mean(f"time_{m}x")) for m in (1, 2)]
            row = {"t0": t0, "span": span, "l1_plain": {"1x": pts[0][0], "2x": pts[1][0]},
                   "time_plain_s": {"1x": pts[0][1], "2x": pts[1][1]}, "time_4x_s": mean("time_4x")}
            l1l, tl = mean("l1_learned"), mean("time_learned")
            if math.isfinite(l1l):
                tf = frontier_time_at(l1l, pts)
                row["learned_fct"] = {"l1": l1l, "time_s": tl, "frontier_time_at_l1_s": tf, "below_frontier": tl < tf,
                                      "error_ratio_vs_plain_1x": l1l / pts[0][0]}
            else:
                row["learned_fct"] = {"l1": l1l, "failed_runs": sum(1 for r in sel if not math.isfinite(r["l1_learned"]))}
            summary.append(row)
    return rows, summary


def frontier_time_at(l1, pts):
    """GPU time the plain frontier needs for error l1: log-log interpolation
    between the plain points (l1_m, time_m), extrapolated from the two nearest."""
    pts = sorted(pts, key=lambda p: -p[0])  # decreasing error
    ls = np.log([p[0] for p in pts])
    ts = np.log([p[1] for p in pts])
    x = math.log(l1)
    if x >= ls[0]:
        i = 0
    elif x <= ls[-1]:
        i = len(ls) - 2
    else:
        i = max(j for j in range(len(ls) - 1) if ls[j] >= x)
    slope = (ts[i + 1] - ts[i]) / (ls[i + 1] - ls[i])
    return float(math.exp(ts[i] + slope * (x - ls[i])))


def summarize(rows, names=("learned",)):
    out = []
    for t_eval in sorted({r["t"] for r in rows}):
        sel = [r for r in rows if r["t"] == t_eval]
        mean = lambda k: float(np.mean([r[k] for r in sel]))
        pts = [(mean(f"l1_{m}x"), mean(f"time_{m}x")) for m in (1, 2, 3)]
        row = {"t": t_eval, "l1_plain": {f"{m}x": p[0] for m, p in zip((1, 2, 3), pts)},
               "time_plain_s": {f"{m}x": p[1] for m, p in zip((1, 2, 3), pts)}, "time_4x_s": mean("time_4x")}
        for name in names:
            l1l, tl = mean(f"l1_{name}"), mean(f"time_{name}")
            if not math.isfinite(l1l):
                row[name] = {"l1": l1l, "failed_runs": sum(1 for r in sel if not math.isfinite(r[f"l1_{name}"]))}
                continue
            tf = frontier_time_at(l1l, pts)
            row[name] = {"l1": l1l, "time_s": tl, "frontier_time_at_l1_s": tf, "below_frontier": tl < tf,
                         "error_reduction_vs_plain_1x": pts[0][0] / l1l,
                         "fallback_cells": int(sum(r[f"fallback_cells_{name}"] for r in sel))}
        out.append(row)
    return out


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--train-seeds", type=int, default=64)
    ap.add_argument("--eval-seeds", type=int, default=8)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--t-end", type=float, default=1.0)
    ap.add_argument("--snap-every", type=int, default=16)
    ap.add_argument("--keep", type=float, default=1.0 / 16)
    ap.add_argument("--epochs", type=int, default=16)
    ap.add_argument("--batch", type=int, default=32768)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--limit", type=float, default=-1.0,
                    help="bound on network outputs (< 0: twice the 99.9th percentile of |target|)")
    ap.add_argument("--no-fct", action="store_true", help="also evaluate without the FCT limiter")
    ap.add_argument("--out", default=None, help="write params (.npy) and results (.json) with this prefix")
    ap.add_argument("--params", default=None,
                    help="evaluate these trained parameters (.npy) instead of generating data and training")
    a = ap.parse_args(argv)
    from . import build
    build.build()
    log = lambda m: print(m, flush=True)
    if a.params:
        params = np.load(a.params)
        rs_rows, rs_summ = restart_frontier(params, seeds=range(64, 64 + a.eval_seeds), n_coarse=a.n, log=log)
        print(json.dumps({"restart_frontier": rs_summ}), flush=True)
        if a.out:
            with open(a.out + "_restart.json", "w") as f:
                json.dump({"per_seed": rs_rows, "summary": rs_summ}, f, indent=1)
        return
    t0 = time.perf_counter()
    X, T = generate(range(a.train_seeds), n_coarse=a.n, t_end=a.t_end, snap_every=a.snap_every,
                    keep_fraction=a.keep, log=log)
    t_gen = time.perf_counter() - t0
    log(f"dataset {X.shape[0]} samples in {t_gen:.1f} s")
    t0 = time.perf_counter()
    params, hist = train(X, T, epochs=a.epochs, batch=a.batch, lr=a.lr, log=log)
    t_train = time.perf_counter() - t0
    log(f"trained in {t_train:.1f} s")
    limit = a.limit if a.limit >= 0 else output_limit(T)
    log(f"output limit {limit:.4e}")
    sh_rows, sh_summ = short_horizon(params, seeds=range(64, 64 + a.eval_seeds), n_coarse=a.n, log=log)
    print(json.dumps({"short_horizon": sh_summ}), flush=True)
    rs_rows, rs_summ = restart_frontier(params, seeds=range(64, 64 + a.eval_seeds), n_coarse=a.n, log=log)
    print(json.dumps({"restart_frontier": rs_summ}), flush=True)
    variants = [("learned_fct", True, math.inf), ("learned_fct_bounded", True, limit)]
    if a.no_fct:
        variants.append(("learned_bounded", False, limit))
    rows = evaluate(params, seeds=range(64, 64 + a.eval_seeds), n_coarse=a.n, log=log, variants=variants)
    summ = summarize(rows, [v[0] for v in variants])
    result = {"samples": int(X.shape[0]), "gen_s": t_gen, "train_s": t_train, "loss_history": hist,
              "output_limit": limit, "per_seed": rows, "summary": summ,
              "short_horizon_per_seed": sh_rows, "short_horizon": sh_summ,
              "restart_frontier_per_seed": rs_rows, "restart_frontier": rs_summ}
    print(json.dumps({"summary": summ}), flush=True)
    if a.out:
        np.save(a.out + "_params.npy", params)
        with open(a.out + "_results.json", "w") as f:
            json.dump(result, f, indent=1)


if __name__ == "__main__":
    main()
