"""Benchmark of the GB300 hydro update (one RK2 step = the whole hot path).

Default workload: 3D point blast, 256^3 cells on [-1, 1]^3, gamma = 1.4,
reflecting walls, HLLC, FP32 storage/fluxes with FP64 recovery and reductions,
C_CFL = 0.3, device-side CFL time step and conserved totals every step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision fp32|fp64] [--solver hllc|hll] [--n 256]

Prints one JSON line (rank 0).  Metric: cell-updates per second per RK stage
(cells x 2 stages x steps / time), whole job.  With N > 1 (torchrun) every
rank runs an independent replica of the workload ("replicas only": the
single-grid update needs no data exchange between problems) and the value is
the sum over ranks with the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per RK stage"
UNIT = "cell-updates/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp64dw"])
    ap.add_argument("--solver", default="hllc", choices=["hllc", "hll", "hllc_switch"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="sedov", choices=["sedov", "batch", "learned", "fmr"])
    ap.add_argument("--levels", type=int, default=4, help="fmr workload: nested levels")
    ap.add_argument("--problems", type=int, default=4096,
                    help="batch workload: problems per GPU (each drawn from the same size mix)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default tile instead of autotuning")
    ap.add_argument("--tile", type=int, default=-1, help="use this tile (and --kchunk) instead of autotuning")
    ap.add_argument("--kchunk", type=int, default=0)
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _workload(n, solver_name):
    from paper_1207_3392_gb300 import problems as P
    solver = {"hllc": P.HLLC, "hll": P.HLL, "hllc_switch": P.HLLC_SWITCH}[solver_name]
    return P.sedov_3d(n, solver=solver)


def _config(args, n):
    return {"workload": f"sedov3d_{n}^3_{args.solver}_{args.precision}",
            "cells": n ** 3, "domain": "[-1,1]^3", "gamma": 1.4, "bc": "reflecting",
            "solver": args.solver.upper(),
            "precision": PRECISION_LABEL[args.precision],
            "cfl": 0.3, "step": "one TVD-RK2 step: 2 stage kernels + dt/totals finalize",
            "l2": f"inputs larger than L2 (state {n**3 * 5 * (4 if args.precision == 'fp32' else 8) / 1e6:.0f} MB)",
            "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Floating-point operations per cell of the 3D update, counted by running the
# oracle's own code with an operation-counting scalar (oracle/opcount.cpp; the
# test tests/test_oracle_opcount.py fixes these numbers from the counter).
# Rule: +, -, *, / each 1 (a product feeding a sum 2), sqrt, min, max, fabs 1.
# Stage 1 (the dominant kernel) = L[U^n] + the CFL speed + the conserved
# totals; a step = the oracle's RK2 step + CFL + totals.  The oracle forms
# both sides' states and fluxes at every HLLC face and divides where the
# kernel multiplies by stored reciprocals, so these counts are the method's
# operations as the plain definition writes them.
FLOPS_STAGE1_3D = {"hllc": 744, "hll": 720}
FLOPS_STEP_3D = {"hllc": 1469, "hll": 1421}
FLOPS_STAGE1_3D["hllc_switch"] = FLOPS_STAGE1_3D["hllc"]  # away from shocks; the detector is not counted
FLOPS_STEP_3D["hllc_switch"] = FLOPS_STEP_3D["hllc"]
# DRAM bytes (read + write) per launch of the FP32 HLLC 3D stage kernels at
# 256^3, from one ncu capture of the bench's own launch configuration (tile
# 8, 40 planes per CTA; profiles/stage_fp32_hllc_sedov256_ncu.md).  Other
# configurations, precisions and sizes report no traffic.
TRAFFIC_FP32_HLLC_256 = {
    (8, 40): {"stage1": 356.859136e6 + 300.052480e6, "stage2": 732.600576e6 + 312.649472e6},
}
PRECISION_LABEL = {
    "fp32": ("FP32 storage, FP32 fluxes and FP32 per-cell CFL speeds; the internal-energy recovery "
             "e = G - |S|^2/(2D) in FP64 only where the kinetic energy exceeds half of G; per-column "
             "conserved totals as compensated FP32 pairs; the dt and totals reductions across threads "
             "and CTAs in FP64"),
    "fp64": "FP64 throughout",
    "fp64dw": ("double-word FP32 pairs (~48 significant bits) for every value and operation, on the FP32 "
               "pipes; FP64 parity"),
}


def _sample_parity(pr, U_ref, steps):
    """The GPU path on the cpu_baseline sample: the same problem for the same
    number of device-CFL RK2 steps in both precisions, against the oracle's
    result U_ref.  Relative L1 per conserved variable (Eq. L1ErrorNorm; the
    momenta against the L1 norm of the whole momentum field) and relative
    L-infinity over all variables.  Errors are reported, never raised."""
    import numpy as np
    from paper_1207_3392_gb300 import hydro as H
    out = {"sample_steps": steps}
    try:
        ref = np.asarray(U_ref, dtype=np.float64)
        nd = pr.ndim
        mom = float(np.sum(np.abs(ref[1:1 + nd])))
        for name, prec in (("fp32_mixed", H.FP32_MIXED), ("fp64", H.FP64)):
            h = H.Hydro.from_problem(pr, precision=prec)
            try:
                h.advance(steps, pr.cfl)
                Ug = h.get_conserved(precision=H.FP64)
            finally:
                h.close()
            l1 = []
            for v in range(nd + 2):
                den = mom if 1 <= v <= nd else float(np.sum(np.abs(ref[v])))
                l1.append(float(np.sum(np.abs(Ug[v] - ref[v])) / den))
            linf = float(np.max(np.abs(Ug - ref)) / np.max(np.abs(ref)))
            out[name] = {"rel_l1": l1, "linf_rel": linf}
            del Ug
    except Exception as e:  # report, do not fail the bench
        out["error"] = str(e)[:200]
    return out


def cpu_baseline(n_sample=256, steps=3):
    """The oracle, as it stands, on a bounded sample of the workload: the same
    point blast at n_sample^3 for `steps` RK2 steps, all host cores.  The
    oracle's result on that sample is also the reference of `parity`."""
    import oracle as O
    from paper_1207_3392_gb300 import problems as P
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    pr = P.sedov_3d(n_sample)
    g = O.Grid(pr)
    U = O.initial_state(pr, g)
    t0 = time.perf_counter()
    U, _, done = O.evolve(g, U, pr.cfl, max_steps=steps)
    dt = time.perf_counter() - t0
    out = {"value": pr.ncells * 2 * done / dt, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
           "kind": "oracle",
           "sample": f"FP64 oracle, same point blast at {n_sample}^3 for {done} RK2 steps ({dt:.1f} s)"}
    out["parity"] = _sample_parity(pr, U, done)
    del U
    # one host core: a smaller sample of the same blast, in a child process so
    # that the OpenMP runtime starts with one thread
    code = ("import json, time, oracle as O; from paper_1207_3392_gb300 import problems as P; "
            "pr = P.sedov_3d(128); g = O.Grid(pr); U = O.initial_state(pr, g); t0 = time.perf_counter(); "
            "U, _, d = O.evolve(g, U, pr.cfl, max_steps=2); "
            "print(json.dumps({'v': pr.ncells * 2 * d / (time.perf_counter() - t0), 'd': d}))")
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300,
                           env=dict(os.environ, OMP_NUM_THREADS="1"))
        st = json.loads(r.stdout.strip().splitlines()[-1])
        out["single_thread"] = {"value": st["v"], "unit": UNIT, "cores": 1,
                                "sample": f"FP64 oracle, the same blast at 128^3 for {st['d']} RK2 steps"}
    except Exception as e:  # report, do not fail the bench
        out["single_thread"] = {"error": str(e)[:200]}
    return out


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    import oracle as O
    from paper_1207_3392_gb300 import problems as P
    n_sample = args.n
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    pr = P.sedov_3d(n_sample, solver={"hllc": P.HLLC, "hll": P.HLL, "hllc_switch": P.HLLC_SWITCH}[args.solver])
    g = O.Grid(pr)
    U = O.initial_state(pr, g)
    U, _, _ = O.evolve(g, U, pr.cfl, max_steps=args.warmup)
    t0 = time.perf_counter()
    U, _, done = O.evolve(g, U, pr.cfl, max_steps=args.steps)
    el = time.perf_counter() - t0
    val = pr.ncells * 2 * done / el
    cfg = _config(args, args.n)
    # the same workload; the arm's own arithmetic and hardware
    cfg["precision"] = PRECISION_LABEL["fp64"] + " (the plain CPU oracle)"
    cfg["implementation"] = f"FP64 CPU oracle, OpenMP over cells on {os.environ['OMP_NUM_THREADS']} host cores"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(done, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"kind": "oracle", "cores": int(os.environ["OMP_NUM_THREADS"]), "value": val,
                             "unit": UNIT,
                             "sample": f"FP64 oracle, the same {n_sample}^3 point blast, {done} timed RK2 steps"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _fma_peaks():
    """Measured vector FMA rates of this GPU (TFLOP/s) from the library's FMA
    chain kernel: FP64, FP32 and FP32 pairs."""
    from paper_1207_3392_gb300 import hydro as H
    out = {}
    for name, kind in (("fp64", 0), ("fp32", 1), ("fp32x2", 2)):
        try:
            out[name] = H.measure_fma_rate(kind)
        except Exception as e:  # report, do not fail the bench
            out[name + "_error"] = str(e)[:200]
    return out


_PEAKS = {}


def _stage_roofline(args, prec, cells, tile, st1, fin, st2):
    """Roofline of the dominant stage kernel (the slower of the two).  The
    metric's roofline is HBM: algorithmic bytes per launch (stage 1 reads U^n
    and writes K, 2 nv b per cell; stage 2 reads U^n and K and writes
    U^{n+1}, 3 nv b) over the launch's event-timed duration, against the
    measured copy bandwidth.  Beside it, the arithmetic roofline: the
    oracle-counted operations per cell over the same duration, against the
    FMA rate measured on this GPU (FP32 pipes for FP32 and double word, FP64
    pipe for FP64)."""
    from paper_1207_3392_gb300 import hydro as H
    b = 4 if prec == H.FP32_MIXED else 8
    nv = 5
    bytes1, bytes2 = 2 * nv * b * cells, 3 * nv * b * cells
    peak, peak_kind = _peaks()
    dom = "stage2" if st2 >= st1 else "stage1"
    dom_ms, dom_bytes = (st2, bytes2) if dom == "stage2" else (st1, bytes1)
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    per_launch = TRAFFIC_FP32_HLLC_256.get((tile["tile"], tile["kchunk"]))
    traffic = (per_launch[dom] if per_launch and b == 4 and args.solver == "hllc" and cells == 256 ** 3
               else None)
    if not _PEAKS:
        _PEAKS.update(_fma_peaks())
    fkey = "fp64" if prec == H.FP64 else "fp32"
    flops_cell = FLOPS_STAGE1_3D[args.solver] if dom == "stage1" else FLOPS_STEP_3D[args.solver] - FLOPS_STAGE1_3D[
        args.solver]
    achieved_f = flops_cell * cells / (dom_ms * 1e-3) / 1e12
    peak_f = _PEAKS.get(fkey)
    tname = {H.FP32_MIXED: "float", H.FP64: "double", H.FP64_DW: "dw"}[prec]
    return {"bound": "hbm", "kernel": f"hydro_stage_kernel<3,{tname},{args.solver.upper()},{dom[-1]}>",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured"
            else "fallback 6800 GB/s",
            "algorithmic_bytes_per_cell": dom_bytes // cells, "traffic": traffic,
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of this launch configuration "
                               "at 256^3" if traffic else None),
            "step_frac": (bytes1 + bytes2) / ((st1 + fin + st2) * 1e-3) / 1e9 / peak,
            "alu": {"achieved": achieved_f, "peak": peak_f, "unit": "TFLOP/s",
                    "frac": achieved_f / peak_f if peak_f else None,
                    "peak_source": f"measured {fkey} FMA chains on this GPU (genasis_measure_fma_rate)",
                    "flops_per_cell": flops_cell,
                    "flops_source": "the oracle's own code run with an operation-counting scalar"},
            "fma_rates_tflops": dict(_PEAKS),
            "kernel_ms": {"stage1": st1, "finalize": fin, "stage2": st2}}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1207_3392_gb300 import build
    from paper_1207_3392_gb300 import hydro as H

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    n = args.n
    prob = _workload(n, args.solver)
    prec = {"fp32": H.FP32_MIXED, "fp64": H.FP64, "fp64dw": H.FP64_DW}[args.precision]
    # a dedicated (non-default) stream: the library and the timing events share it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    h = H.Hydro.from_problem(prob, precision=prec, stream=stream.cuda_stream)
    del prob
    cells = h.ncell
    cfl = 0.3
    if args.tile >= 0:
        h.set_tile(args.tile, args.kchunk)
    elif not args.no_autotune:
        h.autotune(trial_steps=3)
    tile = h.tile_info()

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up (also captures the one-step graph)
    for _ in range(max(args.warmup, 3)):
        h.advance(1, cfl, sync=False)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        h.advance(1, cfl, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    h.status()
    value = world * cells * 2 / (ms * 1e-3)

    # per-kernel durations (CUDA events between the launches on the same stream)
    ks = [h.profile_step(cfl) for _ in range(args.steps)]
    st1 = float(np.mean([k[0] for k in ks]))
    fin = float(np.mean([k[1] for k in ks]))
    st2 = float(np.mean([k[2] for k in ks]))
    roofline = _stage_roofline(args, prec, cells, tile, st1, fin, st2)
    b = 4 if prec == H.FP32_MIXED else 8

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {H.FP32_MIXED: "f32", H.FP64: "f64", H.FP64_DW: "f32x2 double-word"}[prec],
            "data": "synthetic",
            "config": dict(_config(args, n), tile=tile), "roofline": roofline, "clocks": clocks,
            "gpu_launches": args.steps * h.launches_per_step()}

    # end to end through the C ABI with page-locked host buffers: every step
    # copies its input state host -> device (set_conserved_async), steps, and
    # copies the result device -> host (get_conserved_async).  Three handles on
    # three streams let one handle's transfers overlap another's step; a
    # handle is reused only after sync() has returned its previous result.
    if not args.no_e2e:
        nh = 3
        tinfo = h.tile_info()
        e_streams = [torch.cuda.Stream() for _ in range(nh)]
        prob_e = _workload(n, args.solver)
        hs = [H.Hydro.from_problem(prob_e, precision=prec, stream=es.cuda_stream, set_state=False)
              for es in e_streams]
        del prob_e
        dt_host = torch.float32 if b == 4 else torch.float64
        first = torch.empty((h.nvar,) + h.shape, dtype=dt_host).pin_memory()
        h.get_conserved(first)
        host_in = [first] + [first.clone().pin_memory() for _ in range(nh - 1)]
        host_out = [torch.empty_like(first).pin_memory() for _ in range(nh)]
        for hh in hs:
            hh.set_tile(tinfo["tile"], tinfo["kchunk"])
            hh.set_conserved_async(host_in[0])
            hh.advance(1, cfl, sync=False)  # captures the step graphs
            hh.sync()
        # 100 steps a repetition: the pipeline's fill and drain (the first
        # copy in and the last copy out, which nothing overlaps) is a fixed
        # cost of about one step; over 30 steps it was 4% of the time
        k = max(2 * nh, min(args.steps, 100))
        reps = []
        for _ in range(5):  # five timed repetitions; the median is reported, with min and max
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            for s_ in range(k):
                hh = hs[s_ % nh]
                if s_ >= nh:
                    hh.sync()
                hh.set_conserved_async(host_in[s_ % nh])
                hh.advance(1, cfl, sync=False)
                hh.get_conserved_async(host_out[s_ % nh])
            for hh in hs:
                hh.sync()
            reps.append(time.perf_counter() - t0)
        el = statistics.median(reps)
        if world > 1:
            t = torch.tensor([el], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        nbytes = first.numel() * first.element_size()
        line["e2e"] = {"value": world * cells * 2 * k / el, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                       "d2h_bytes_per_step": nbytes, "ms_per_step": 1e3 * el / k, "steps": k,
                       "repetitions_ms_per_step": [1e3 * r / k for r in reps],
                       "min_ms_per_step": 1e3 * min(reps) / k, "max_ms_per_step": 1e3 * max(reps) / k,
                       "pipeline": f"{nh} handles on {nh} streams, page-locked host buffers"}
        for hh in hs:
            hh.close()
        # the end-to-end roofline: each step copies its state in and out over
        # the host link, whose copy rates are measured here (both directions
        # at once is the pipeline's case)
        link = {"h2d": H.measure_link_rate(0), "d2h": H.measure_link_rate(1), "both": H.measure_link_rate(2)}
        achieved = 2 * nbytes / (el / k) / 1e9
        line["e2e"]["roofline"] = {"bound": "host link", "achieved": achieved, "peak": link["both"], "unit": "GB/s",
                                   "frac": achieved / link["both"],
                                   "peak_source": "measured cudaMemcpyAsync, host to device and device to host "
                                                  "at once (genasis_measure_link_rate)",
                                   "link_gbs": link}
    h.close()

    # other precision / solver combinations of the same workload (context)
    if not args.no_variants and rank == 0:
        from paper_1207_3392_gb300 import problems as P
        variants = {}
        for pname, pc, sname, totals in (("fp32", H.FP32_MIXED, args.solver, False),
                                         ("fp32", H.FP32_MIXED, "hllc", True), ("fp32", H.FP32_MIXED, "hll", True),
                                         ("fp64", H.FP64, "hllc", True), ("fp64", H.FP64, "hll", True),
                                         ("fp64dw", H.FP64_DW, "hllc", True),
                                         ("fp32", H.FP32_MIXED, "hllc_switch", True)):
                if (pname, sname, totals) == (args.precision, args.solver, True):
                    continue
                pr = _workload(n, sname)
                hv = H.Hydro.from_problem(pr, precision=pc, stream=stream.cuda_stream)
                hv.set_step_totals(totals)
                del pr
                hv.autotune(trial_steps=2)
                kv = 3 if pc == H.FP64 else 5
                for _ in range(2):
                    hv.advance(1, cfl, sync=False)
                torch.cuda.synchronize()
                a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(kv):
                    hv.advance(1, cfl, sync=False)
                z.record(stream)
                torch.cuda.synchronize()
                mv = a.elapsed_time(z) / kv
                key = f"{sname}_{pname}" + ("" if totals else "_no_step_totals")
                bv = 4 if pc == H.FP32_MIXED else 8
                peak, _ = _peaks()
                variants[key] = {"value": cells * 2 / (mv * 1e-3), "ms_per_step": mv,
                                 "hbm_frac_step": 5 * 5 * bv * cells / (mv * 1e-3) / 1e9 / peak}
                if pname in ("fp32", "fp64"):
                    # the arithmetic roofline of the step: the oracle-counted
                    # operations against the measured FMA rate of the pipe that
                    # runs them (double word runs FP64 operations as FP32 ones,
                    # so it has no such rate)
                    if not _PEAKS:
                        _PEAKS.update(_fma_peaks())
                    fl = FLOPS_STEP_3D[sname] * cells / (mv * 1e-3) / 1e12
                    pk = _PEAKS.get(pname)
                    variants[key]["alu_step"] = {"achieved": fl, "peak": pk, "unit": "TFLOP/s",
                                                 "frac": fl / pk if pk else None,
                                                 "flops_per_cell": FLOPS_STEP_3D[sname]}
                hv.close()
        # the centrally refined 320^3 pulse (stretched widths, gamma = 5/3), FP32 HLLC
        pr = P.stretched_pulse_3d(320)
        hv = H.Hydro.from_problem(pr, precision=H.FP32_MIXED, stream=stream.cuda_stream)
        del pr
        hv.autotune(trial_steps=2)
        for _ in range(3):
            hv.advance(1, cfl, sync=False)
        torch.cuda.synchronize()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(20):
            hv.advance(1, cfl, sync=False)
        z.record(stream)
        torch.cuda.synchronize()
        mv = a.elapsed_time(z) / 20
        variants["stretched_pulse_320^3_hllc_fp32"] = {"value": hv.ncell * 2 / (mv * 1e-3), "ms_per_step": mv}
        hv.close()
        # the Rayleigh-Taylor set-up of Sec. 4.3.2 (external-force source), 256 x 768
        pr = P.rayleigh_taylor(256, 768)
        hv = H.Hydro.from_problem(pr, precision=H.FP32_MIXED, stream=stream.cuda_stream)
        del pr
        hv.autotune(trial_steps=2)
        for _ in range(3):
            hv.advance(1, 0.5, sync=False)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(50):
            hv.advance(1, 0.5, sync=False)
        z.record(stream)
        torch.cuda.synchronize()
        mv = a.elapsed_time(z) / 50
        variants["rayleigh_taylor_256x768_hllc_fp32"] = {"value": hv.ncell * 2 / (mv * 1e-3), "ms_per_step": mv}
        hv.close()
        # the other workloads of the benchmark set, each with its own line
        for name, fn in (("sod1d_256_hllc_fp64", lambda: measure_sod(stream)),
                         ("batched_riemann_4096", lambda: measure_batch(("fp32", "fp64dw", "fp64"), 5, 3, stream)),
                         ("learned_kh2d_256^2_hllc_fct", lambda: measure_learned(50, 3, stream)),
                         ("sedov3d_fmr_4x128^3_hllc_fp32", lambda: measure_fmr(128, 4, "fp32", "hllc", 10, 3, stream))):
            try:
                variants[name] = fn()
            except Exception as e:  # report, do not fail the bench
                variants[name] = {"error": str(e)[:300]}
        line["variants"] = variants

    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _batch_specs(world=1, rank=0, per_rank=4096):
    from paper_1207_3392_gb300 import shard
    all_specs = shard.weak_scaling_specs(world, per_rank=per_rank)
    return all_specs, shard.rank_specs(all_specs, rank, world)


class _Mesh:
    """Mesh-only view of a BatchSpec (the batch needs no arrays at creation)."""

    def __init__(self, sp):
        from paper_1207_3392_gb300 import problems as P
        self.ndim, self.gamma = sp.ndim, sp.gamma
        self.n = (sp.n, sp.n if sp.ndim == 2 else 1, 1)
        w = P.uniform_widths(sp.n, 0.0, 1.0)
        self.widths = [w, w][: sp.ndim]
        self.bc_lo = self.bc_hi = (P.OUTFLOW,) * 3


def measure_batch(precisions, steps, warmup, stream, specs=None, autotune=True, sampler=None, barrier=None,
                  scale_steps=True):
    """The batched Riemann set (4096 independent 1D/2D problems, 2.09e8 cells)
    in each precision: one persistent launch per RK stage, per-problem CFL dt,
    graph-captured steps.  All batches are built first from one pass over the
    problems (the initial conditions are generated once).  Returns
    {precision: record}; the record's roofline is that of the dominant stage
    kernel against the measured HBM bandwidth."""
    import torch
    from paper_1207_3392_gb300 import hydro as H
    from paper_1207_3392_gb300 import problems as P
    if specs is None:
        _, specs = _batch_specs()
    pc = {"fp32": H.FP32_MIXED, "fp64": H.FP64, "fp64dw": H.FP64_DW}
    batches = {name: H.Batch([_Mesh(sp) for sp in specs], precision=pc[name], stream=stream.cuda_stream)
               for name in precisions}
    for i, sp in enumerate(specs):
        pr = P.batch_problem(sp)
        for bb in batches.values():
            bb.set_primitive(i, pr.rho, pr.vel, pr.p)
    cells = sum(sp.n ** sp.ndim for sp in specs)
    cells_nv = sum(sp.n ** sp.ndim * (sp.ndim + 2) for sp in specs)
    peak, peak_kind = _peaks()
    out = {}
    for name in precisions:
        bb = batches[name]
        if autotune:
            bb.autotune(trial_steps=2)
        # the slower precisions take fewer steps unless the caller asked for this one alone
        k = steps if (name == "fp32" or not scale_steps) else max(2, steps // (8 if name == "fp64" else 3))
        for _ in range(max(warmup, 3)):
            bb.run(1, 0.5)
        torch.cuda.synchronize()
        if sampler is not None and name == precisions[0]:
            sampler.start()
        if barrier is not None:
            barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bb.run(k, 0.5)
        e1.record(stream)
        torch.cuda.synchronize()
        if barrier is not None:
            barrier()
        clocks = sampler.stop() if sampler is not None and name == precisions[0] else None
        ms = e0.elapsed_time(e1) / k
        bb.status()
        ks = [bb.profile_step(0.5) for _ in range(3)]
        st1 = float(np.mean([x[0] for x in ks]))
        fin = float(np.mean([x[1] for x in ks]))
        st2 = float(np.mean([x[2] for x in ks]))
        esz = 4 if name == "fp32" else 8
        dom, dom_ms, dom_bytes = (("stage2", st2, 3 * esz * cells_nv) if st2 >= st1
                                  else ("stage1", st1, 2 * esz * cells_nv))
        achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
        info = bb.tile_info()
        out[name] = {"value": cells * 2 / (ms * 1e-3), "ms_per_step": ms, "steps": k, "cells": cells,
                     "dtype": {"fp32": "f32", "fp64": "f64", "fp64dw": "f32x2 double-word"}[name],
                     "tile": info, "l2": f"inputs larger than L2 (state {cells_nv * esz / 1e9:.2f} GB)",
                     "roofline": {"bound": "hbm", "kernel": f"hydro_batch_kernel ({dom})", "achieved": achieved,
                                  "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                                  "peak_source": f"{peak_kind} hbm_gbs",
                                  "algorithmic_bytes": dom_bytes,
                                  "step_frac": 5 * esz * cells_nv / ((st1 + fin + st2) * 1e-3) / 1e9 / peak,
                                  "kernel_ms": {"stage1": st1, "finalize": fin, "stage2": st2}},
                     "clocks": clocks, "gpu_launches": 3 * k}
    for bb in batches.values():
        bb.close()
    return out


def run_batch(args):
    """Batched Riemann set on its own line (--workload batch): `world` draws of
    4096 problems LPT-sharded by cells x steps, no exchange between ranks."""
    import torch
    import torch.distributed as dist
    from paper_1207_3392_gb300 import build

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    all_specs, specs = _batch_specs(world, rank, args.problems)
    total_cells = sum(sp.n ** sp.ndim for sp in all_specs)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sampler = ClockSampler(local)
    rec = measure_batch((args.precision,), args.steps, args.warmup, stream, specs=specs,
                        autotune=not args.no_autotune, sampler=sampler,
                        barrier=(lambda: dist.barrier()) if world > 1 else None,
                        scale_steps=False)[args.precision]
    ms = rec["ms_per_step"]
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    line = {"metric": METRIC, "value": total_cells * 2 / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": rec["steps"], "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": rec["dtype"], "data": "synthetic",
            "config": {"workload": f"batched_riemann_{args.problems}_{args.precision}", "problems": len(all_specs),
                       "cells": total_cells, "rank0_problems": len(specs), "rank0_cells": rec["cells"],
                       "parallelism": f"{world} GPU(s), problems LPT-sharded by cells x steps, no exchange",
                       "tile": rec["tile"], "cfl": 0.5, "solver": "HLLC", "l2": rec["l2"]},
            "roofline": rec["roofline"], "clocks": rec["clocks"], "gpu_launches": rec["gpu_launches"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def measure_learned(steps, warmup, stream, sampler=None):
    """Learned flux correction on the 2D periodic shear layer, 256^2 FP32: one
    RK2 step = CFL reduction, and per stage the plain face fluxes and
    features, the BF16 MLP, the FCT ratios, the corrected update (plus the
    fallback passes, which run only when a cell failed).  By default a step
    (one advance call) is one cooperative launch; the per-phase launches
    (a CUDA graph of 18 kernels) are timed beside it.  The network is a seeded
    random one of the trained shape; the cost does not depend on the weights
    while no cell falls back."""
    import torch
    from paper_1207_3392_gb300 import hydro as H
    from paper_1207_3392_gb300 import learned_flux as LF
    from paper_1207_3392_gb300 import problems as P
    pr = P.kelvin_helmholtz(256, seed=64)
    params = LF._init_params(0)
    nlast = 4 * 64 + 4                      # output layer W3, b3 (zero at initialisation)
    params[-nlast:] = np.random.default_rng(0).normal(0.0, 0.02, nlast).astype(np.float32)

    def timed(one_launch, smp, tc=False):
        L = H.Learned(pr, params=params, stream=stream.cuda_stream)
        L.set_one_launch(one_launch)
        L.set_mlp_tcgen05(tc)
        L.set_primitive(pr.rho, pr.vel, pr.p)
        for _ in range(max(warmup, 3)):
            L.advance(1, 0.5, sync=False)
        torch.cuda.synchronize()
        if smp is not None:
            smp.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            L.advance(1, 0.5, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        clk = smp.stop() if smp is not None else None
        ms = e0.elapsed_time(e1) / steps
        res = (ms, L.fallbacks(), L.launches_per_step(), clk)
        L.close()
        return res

    ms_pp, _, lps_pp, _ = timed(False, None)
    ms_pp_tc, _, _, _ = timed(False, None, tc=True)
    ms_tc, _, _, _ = timed(True, None, tc=True)
    ms, fb, lps, clocks = timed(True, sampler)
    cells = 256 * 256
    return {"value": cells * 2 / (ms * 1e-3), "ms_per_step": ms, "steps": steps, "cells": cells,
            "network": "24-64-64-4 SiLU, BF16 mma.sync, FP32 accumulate", "fallback_cells": fb,
            "l2": "inputs smaller than L2 (state 1 MB): the step is launch- and latency-bound",
            "launch": ("one cooperative launch per advance call (persistent grid, 7 grid barriers a step)"
                       if lps == 1 else f"{lps} launches per step"),
            "per_phase_ms_per_step": ms_pp, "per_phase_launches_per_step": lps_pp,
            # the same one-launch step with the network on tcgen05 (accumulators
            # in tensor memory) instead of mma.sync fragments in registers
            "tcgen05_ms_per_step": ms_tc, "per_phase_tcgen05_ms_per_step": ms_pp_tc,
            # one advance call per step
            "gpu_launches": steps * lps, "clocks": clocks}


def run_learned(args):
    import torch
    from paper_1207_3392_gb300 import build
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    rec = measure_learned(args.steps, args.warmup, stream, sampler=ClockSampler(local))
    line = {"metric": METRIC, "value": world * rec["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
            "config": {"workload": "learned_kh2d_256^2_hllc_fct", "cells": rec["cells"], "faces": 2 * rec["cells"],
                       "network": rec["network"], "l2": rec["l2"], "fallback_cells": rec["fallback_cells"],
                       "launch": rec["launch"], "per_phase_ms_per_step": rec["per_phase_ms_per_step"],
                       "tcgen05_ms_per_step": rec["tcgen05_ms_per_step"],
                       "per_phase_tcgen05_ms_per_step": rec["per_phase_tcgen05_ms_per_step"]},
            "roofline": None, "clocks": rec["clocks"], "gpu_launches": rec["gpu_launches"]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_fmr(n, levels, precision, solver, steps, warmup, stream, autotune=True, sampler=None):
    """Point blast on nested levels (multilevel evolution with subcycling,
    Algorithms Evolve / EvolveLevel / StepLevel): `levels` boxes of n^3 cells,
    each covering the central half of its parent at twice its resolution, so
    the finest level has the resolution of a (n 2^(levels-1))^3 single-level
    mesh.  A step is one global step (2^l steps of level l)."""
    import torch
    from paper_1207_3392_gb300 import hydro as H
    L = levels
    prec = {"fp32": H.FP32_MIXED, "fp64": H.FP64, "fp64dw": H.FP64}[precision]
    g = H.Fmr(3, n, L, 1.0, 1, solver=H.HLLC if solver != "hll" else H.HLL, precision=prec, stream=stream)
    gamma = 1.4
    for l in range(L):
        m = n + (4 if l else 0)
        U = torch.zeros((5, m, m, m), dtype=torch.float64, device="cuda")
        U[0] = 1.0
        U[4] = 1e-5 / (gamma - 1.0)
        if l == L - 1:
            o = (2 if l else 0) + n // 2 - 1
            hh = 1.0 / n / 2 ** l
            U[4, o:o + 2, o:o + 2, o:o + 2] = 1.0 / (8 * hh ** 3)
        g.set_level(l, U)
        del U
    if autotune:
        g.autotune(2)
    # warm-up; the first global step also restricts the deposit onto the covered coarse cells
    g.step(max(warmup, 3), 0.3)  # also captures the two-step graph
    torch.cuda.synchronize()
    if sampler is not None:
        sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lib = H.load()
    H.check(lib.genasis_fmr_step(g._h, steps, 0.3, None))  # replays the captured two-step graph
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler is not None else None
    ms = e0.elapsed_time(e1) / steps
    t = g.step(0, 0.3)
    g.close()
    cells_per_step = sum(2 ** l * n ** 3 for l in range(L))
    return {"value": cells_per_step * 2 / (ms * 1e-3), "ms_per_step": ms, "steps": steps, "levels": L,
            "cells_per_level": n ** 3, "finest_equivalent": f"{n * 2 ** (L - 1)}^3",
            "cell_updates_per_global_step": cells_per_step, "time_reached": t, "clocks": clocks,
            "dtype": "f32" if prec == H.FP32_MIXED else "f64"}


def run_fmr(args):
    import torch
    from paper_1207_3392_gb300 import build
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    build.build()
    n = args.n if args.n != 256 else 128
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    rec = measure_fmr(n, args.levels, args.precision, args.solver, args.steps, args.warmup, stream,
                      autotune=not args.no_autotune, sampler=ClockSampler(local))
    line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": rec["dtype"], "data": "synthetic",
            "config": {"workload": f"sedov3d_fmr_{args.levels}x{n}^3_{args.solver}_{args.precision}",
                       "levels": args.levels, "cells_per_level": n ** 3, "finest_equivalent": rec["finest_equivalent"],
                       "cell_updates_per_global_step": rec["cell_updates_per_global_step"],
                       "step": "one global step: 2^l RK2 steps of level l, prolongation, restriction, "
                               "flux replacement, provisional coarse substeps", "time_reached": rec["time_reached"]},
            "roofline": None, "clocks": rec["clocks"], "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_sod(stream, n=256):
    """The 1D benchmark case in full: Sod, 256 cells, HLLC, FP64, C_CFL 0.8,
    from t = 0 to t = 0.2 with the device CFL step (one graph launch of all
    steps, the last clamped to t_end).  Reports the time per RK2 step and of
    the whole run."""
    import torch
    from paper_1207_3392_gb300 import hydro as H
    from paper_1207_3392_gb300 import problems as P
    pr = P.sod(n)
    h = H.Hydro.from_problem(pr, precision=H.FP64, stream=stream.cuda_stream)
    U0 = h.get_conserved()
    # the number of steps to t_end (same rule as the timed run)
    nsteps = 0
    t = 0.0
    while t < pr.t_end and nsteps < 100000:
        t = h.advance(1, pr.cfl, pr.t_end)
        nsteps += 1
    for _ in range(2):  # warm-up of the nsteps-step graph
        h.set_conserved(U0)
        h.time = 0.0
        h.advance(nsteps, pr.cfl, pr.t_end)
    h.set_conserved(U0)
    h.time = 0.0
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.advance(nsteps, pr.cfl, pr.t_end, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    t = h.time
    lps = h.launches_per_step()
    h.close()
    return {"value": n * 2 * nsteps / (ms * 1e-3), "ms_per_step": ms / nsteps, "run_ms": ms, "steps": nsteps,
            "time_reached": t, "cells": n, "dtype": "f64",
            # launches_per_step() == 1: the whole advance call is one cooperative launch
            "gpu_launches": 1 if lps == 1 else nsteps * lps,
            "launch": ("one cooperative launch for all steps (one CTA per 31-cell tile, grid barriers between "
                       "phases)") if lps == 1 else f"{lps} launches per step",
            "note": "the step is bound by latency and by each SM's FP64 rate, not by the 256 cells' bytes"}


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "fmr":
        run_fmr(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
