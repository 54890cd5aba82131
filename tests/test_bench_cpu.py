"""Host-side logic of bench.py, without a GPU: the reference arm's JSON line
(the oracle on a bounded sample), the silent exit of non-zero ranks, and the
map and two-sample helpers its galactic leg uses, each against a brute-force
restatement."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
        "cpu_baseline", "e2e"}


def _run(args, env_extra=None, timeout=300):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT,
                          env=env, capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    r = _run(["--impl", "reference", "--n", "32", "--steps", "2", "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert KEYS <= set(d)
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == bench.workloads.MIXED_INTERACTIONS["name"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_silently():
    r = _run(["--impl", "reference", "--n", "32", "--steps", "1", "--warmup", "0"],
             {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def _ring_tables(nside):
    """Ring number, first pixel and ring length of every RING-scheme pixel,
    by walking the 4 nside - 1 rings in order."""
    ring, first, length = [], [], []
    p0 = 0
    for i in range(1, 4 * nside):
        n = 4 * min(i, nside, 4 * nside - i)
        ring += [i] * n
        first += [p0] * n
        length += [n] * n
        p0 += n
    assert p0 == 12 * nside * nside
    return np.array(ring), np.array(first), np.array(length)


def test_coarse_ring_map_matches_ring_walk():
    rng = np.random.default_rng(3)
    for nside in (1, 2, 4, 16, 64):
        npix = 12 * nside * nside
        hist = rng.integers(0, 50, npix).astype(float)
        ring, first, length = _ring_tables(nside)
        for n_bands, n_sectors in ((16, 8), (3, 5), (1, 1)):
            want = np.zeros(n_bands * n_sectors)
            for p in range(npix):
                b = (ring[p] - 1) * n_bands // (4 * nside - 1)
                s = (p - first[p]) * n_sectors // length[p]
                want[b * n_sectors + s] += hist[p]
            got = bench.coarse_ring_map(hist, nside, n_bands, n_sectors)
            assert np.array_equal(got, want), (nside, n_bands, n_sectors)


def test_two_sample_chi2_special_cases():
    a = np.array([10.0, 0.0, 30.0, 5.0, 0.0])
    s, dof, p = bench.two_sample_chi2(a, 3.0 * a)   # same shape, other total
    assert abs(s) < 1e-12 and dof == 2 and abs(p - 1.0) < 1e-12
    # a 2 x k contingency table's Pearson statistic, from scipy
    from scipy.stats import chi2_contingency
    g = np.random.default_rng(1)
    a, b = g.integers(0, 40, 20).astype(float), g.integers(0, 90, 20).astype(float)
    a[3] = b[3] = 0.0
    s, dof, p = bench.two_sample_chi2(a, b)
    keep = (a + b) > 0
    r = chi2_contingency(np.stack([a[keep], b[keep]]), correction=False)
    assert dof == r.dof == 18
    assert abs(s - r.statistic) < 1e-9 * r.statistic and abs(p - r.pvalue) < 1e-9 * r.pvalue


def test_kick_turns_directions_by_the_requested_angle():
    g = np.random.default_rng(3)
    u = g.normal(size=(200, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    inj = dict(ux=u[:, 0].copy(), uy=u[:, 1].copy(), uz=u[:, 2].copy(), E=np.ones(200))
    delta = 10.0 ** g.uniform(-9, -4, 200)
    for axis in bench.FLOOR_AXES:
        k = bench.kicked(inj, delta, axis)
        v = np.stack([k["ux"], k["uy"], k["uz"]], 1)
        assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-15)
        ang = np.arccos(np.clip(np.sum(u * v, axis=1), -1, 1))
        # first order: the angle is delta (arccos loses digits near 1: compare the chord)
        chord = np.linalg.norm(v - u, axis=1)
        assert np.allclose(chord, delta, rtol=1e-6), np.max(np.abs(chord / delta - 1))
        assert np.all(ang < 2 * delta + 1e-7)


def test_endpoint_errors_and_agreement():
    import oracle
    n = 50
    rec = np.zeros(n, dtype=oracle.RECORD_DTYPE)
    rec["id"] = np.arange(n)
    rec["x"] = np.random.default_rng(1).normal(size=(n, 3)) * 10
    rec["u"] = [0.0, 0.0, 1.0]
    rec["E"] = 1e19
    rec["s"] = 20.0
    other = rec.copy()
    other["x"][:, 0] += 2e-4
    other["E"] *= 1 + 1e-6
    e = bench.endpoint_errors(other, rec)
    assert np.allclose(e["pos_over_s"], 1e-5)
    assert np.allclose(e["pos_over_x"], 2e-4 / np.maximum(1, np.linalg.norm(rec["x"], axis=1)))
    assert np.all(e["dir"] == 0) and np.allclose(e["E"], 1e-6)
    a = bench.agreement(rec, rec)
    assert a["n"] == n and a["status_agree"] == 1.0 and a["pos_over_s"]["max"] == 0.0
    assert a["E"]["frac_le_1e-05"] == 1.0


def test_equal_error_statement_host_logic(monkeypatch):
    """The oracle part of the mixed-vs-FP64 block on a small case, with the
    oracle's own records standing in for both paths' (so the two paths agree
    exactly and the binary64 path equals the oracle): truth, floors and the
    block's structure."""
    import oracle
    import workloads
    oracle.build()
    monkeypatch.setattr(bench, "TRUTH_SAMPLE", 24)
    monkeypatch.setattr(bench, "BALLISTIC_TRUTH_SAMPLE", 32)
    hw = dict(workloads.MIXED_INTERACTIONS, grid_n=(16, 16, 16), spacing=0.5)
    B = oracle.turbulent_field(hw["grid_n"], hw["spacing"], 1.0, 5.0, 1.0, seed=9)
    inj = workloads.mixed_interactions(n=120, seed=4)
    inj["s_max"] = np.full(120, 20.0)
    T = oracle.tables_build(n=1000)
    P = bench._oracle_params(oracle, hw, hw["tol"], hw["h_min"], T)
    rec = oracle.propagate(P, B, inj, tables=T)
    ids = np.arange(60)
    Pt = bench._oracle_params(oracle, hw, bench.TIGHT_TOL, bench.TIGHT_HMIN, T)
    rect = oracle.propagate(Pt, B, workloads.subsample(inj, ids), tables=T)
    wb = dict(workloads.PLAIN_SMALL, grid_n=(16, 16, 16), spacing=0.5)
    binj = workloads.plain_small(n=80, seed=2)
    binj["s_max"] = np.full(80, 10.0)
    ball = {"w": wb, "workload": "small", "inj": binj, "grid_host": B}
    for tol, hmin in ((1e-4, 0.01), (bench.TIGHT_TOL, bench.TIGHT_HMIN)):
        r = oracle.propagate(bench._oracle_params(oracle, wb, tol, hmin, interactions=False),
                             B, binj)
        ball[f"tol_{tol:g}"] = {"tol": tol, "h_min": hmin,
                                "steps_per_s": {"mixed": 2.0, "fp64": 1.0, "mixed_over_fp64": 2.0},
                                "records": (r, r)}
    legs = {"headline": {"w": hw, "tol": hw["tol"], "h_min": hw["h_min"],
                         "steps_per_s": {"mixed": 2.0, "fp64": 1.0, "mixed_over_fp64": 2.0},
                         "records": (rec, rec)},
            "headline_tight": {"tol": bench.TIGHT_TOL, "h_min": bench.TIGHT_HMIN,
                               "candidates": 60, "ids": ids,
                               "steps_per_s": {"mixed": 2.0, "fp64": 1.0,
                                               "mixed_over_fp64": 2.0},
                               "records": (rect, rect)},
            "ballistic": ball}
    out = bench.equal_error_statement(legs, inj, B)
    json.dumps(out)
    h = out["headline"]
    assert h["mixed_vs_fp64"]["pos_over_s"]["max"] == 0.0
    assert h["vs_truth"]["mixed"] == h["vs_truth"]["fp64"]
    assert h["vs_truth"]["mixed"]["n"] == 24
    assert 0.0 <= h["chaos_floor"]["frac_resolvable"] <= 1.0
    for key in ("tol_0.0001", "tol_1e-08"):
        b = out["ballistic"][key]
        assert b["fp64_equals_oracle"] is True
        assert b["vs_truth"]["mixed"]["n"] == 32
    # tighter tolerance, closer to the truth
    assert (out["ballistic"]["tol_1e-08"]["vs_truth"]["fp64"]["pos_over_x"]["median"]
            < out["ballistic"]["tol_0.0001"]["vs_truth"]["fp64"]["pos_over_x"]["median"])
    # without the oracle (other ranks): GPU-side agreement only
    bare = bench.equal_error_statement(legs, None, None)
    assert "vs_truth" not in bare["headline"] and "chaos_floor" not in bare["headline"]
