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
