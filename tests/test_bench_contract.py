"""The benchmark's reference arm (the oracle timed on the host cores) prints
one JSON line with the keys its contract names; a small sample runs on CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "16", "--steps", "2",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "cell-updates/s per RK stage" and d["unit"] == "cell-updates/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["vs_baseline"] is None and d["data"] == "synthetic"
    assert d["config"]["workload"].startswith("sedov3d_")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_sample_parity_measures_a_planted_error(monkeypatch):
    """The bench's parity report on the CPU sample: a GPU result equal to the
    oracle's except for a planted relative error in the density gives that
    error as the density's relative L1 and zero for the other variables."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench
    import oracle as O
    from paper_1207_3392_gb300 import hydro as H
    from paper_1207_3392_gb300 import problems as P

    pr = P.sedov_3d(12)
    g = O.Grid(pr)
    U, _, done = O.evolve(g, O.initial_state(pr, g), pr.cfl, max_steps=2)
    planted = {H.FP32_MIXED: 3e-6, H.FP64: 2e-12}

    class FakeHydro:
        def __init__(self, precision):
            self.precision = precision

        @classmethod
        def from_problem(cls, prob, precision):
            return cls(precision)

        def advance(self, steps, cfl):
            assert steps == done and cfl == pr.cfl

        def get_conserved(self, precision):
            X = np.array(U, dtype=np.float64)
            X[0] *= 1.0 + planted[self.precision]
            return X

        def close(self):
            pass

    monkeypatch.setattr(H, "Hydro", FakeHydro)
    r = bench._sample_parity(pr, U, done)
    assert r["sample_steps"] == done and "error" not in r
    for name, prec in (("fp32_mixed", H.FP32_MIXED), ("fp64", H.FP64)):
        l1 = r[name]["rel_l1"]
        assert len(l1) == 5 and abs(l1[0] - planted[prec]) <= 1e-3 * planted[prec]
        assert l1[1:] == [0.0, 0.0, 0.0, 0.0]
        assert 0 < r[name]["linf_rel"] <= planted[prec]
