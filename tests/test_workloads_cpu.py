"""The seeded synthetic inputs against the recipes they are stated to follow
(power law E^-2 between the bounds, isotropy, the H/He/N/Fe number fractions,
rigidity-scaled maximum energies, sources uniform in the box outside the
observer, log-uniform path budgets and rigidities), each by a statistical
test against the closed-form distribution, plus seeding and subsampling."""
import numpy as np
from scipy import stats

import workloads as W

N = 200_000
P_MIN = 1e-4


def _e2_cdf(E, lo, hi):
    return (1.0 / lo - 1.0 / E) / (1.0 / lo - 1.0 / hi)


def _isotropic_ok(ux, uy, uz):
    n = len(ux)
    assert np.allclose(ux * ux + uy * uy + uz * uz, 1.0, atol=1e-12)
    m = np.array([ux.mean(), uy.mean(), uz.mean()])
    assert np.all(np.abs(m) < 5.0 / np.sqrt(3.0 * n))
    assert stats.kstest(uz, stats.uniform(loc=-1, scale=2).cdf).pvalue > P_MIN
    phi = np.arctan2(uy, ux)
    assert stats.kstest(phi, stats.uniform(loc=-np.pi, scale=2 * np.pi).cdf).pvalue > P_MIN


def test_plain_small_recipe():
    w = W.PLAIN_SMALL
    d = W.plain_small(n=N)
    assert np.array_equal(d["id"], np.arange(N, dtype=np.uint64))
    assert np.all((d["x"] == 0) & (d["y"] == 0) & (d["z"] == 0))
    assert np.all((d["A"] == 1) & (d["Z"] == 1) & (d["q"] == 1))
    assert np.all((d["E"] >= w["e_lo"]) & (d["E"] <= w["e_hi"]))
    assert stats.kstest(d["E"], lambda e: _e2_cdf(e, w["e_lo"], w["e_hi"])).pvalue > P_MIN
    _isotropic_ok(d["ux"], d["uy"], d["uz"])
    assert np.all(d["s_max"] == w["s_max"])


def test_mixed_recipe():
    w = W.MIXED_INTERACTIONS
    d = W.mixed_interactions(n=N)
    comp = W.MIXED_COMPOSITION
    counts = np.array([np.sum((d["A"] == a) & (d["Z"] == z)) for a, z, _ in comp])
    assert counts.sum() == N
    assert stats.chisquare(counts, np.array([f for _, _, f in comp]) * N).pvalue > P_MIN
    for a, z, _ in comp:
        sel = d["Z"] == z
        hi = w["e_hi_per_z"] * z            # rigidity-scaled: iron reaches 1e21 eV
        assert np.all((d["E"][sel] >= w["e_lo"]) & (d["E"][sel] <= hi))
        assert stats.kstest(d["E"][sel], lambda e: _e2_cdf(e, w["e_lo"], hi)).pvalue > P_MIN
    assert abs(w["e_hi_per_z"] * 26 - 1e21) < 1e6
    _isotropic_ok(d["ux"], d["uy"], d["uz"])
    pos = np.stack([d["x"], d["y"], d["z"]], axis=1)
    src = np.unique(pos, axis=0)
    assert len(src) == w["n_sources"]
    assert np.all(np.abs(src) <= w["box"]) and np.all(np.linalg.norm(src, axis=1) > w["observer_r"])
    for k in range(3):    # uniform in the box (the excluded ball is 3e-5 of it)
        assert stats.kstest(src[:, k], stats.uniform(loc=-w["box"], scale=2 * w["box"]).cdf).pvalue > P_MIN
    assert np.all(d["q"] == 1) and np.array_equal(d["id"], np.arange(N, dtype=np.uint64))
    assert np.all(d["s_max"] == w["s_max"])


def test_uneven_recipe():
    w = W.UNEVEN_SECONDARIES
    d, brms = W.uneven_secondaries(n=N)
    assert w["brms_lo"] <= brms <= w["brms_hi"]
    ls = np.log(d["s_max"])
    assert np.all((d["s_max"] >= w["s_lo"]) & (d["s_max"] <= w["s_hi"]))
    lo, hi = np.log(w["s_lo"]), np.log(w["s_hi"])
    assert stats.kstest(ls, stats.uniform(loc=lo, scale=hi - lo).cdf).pvalue > P_MIN


def test_seeding_and_subsample():
    a, b = W.mixed_interactions(n=1000), W.mixed_interactions(n=1000)
    c = W.mixed_interactions(n=1000, seed=W.MIXED_INTERACTIONS["seed"] + 1)
    for k in a:
        assert np.array_equal(a[k], b[k])
    assert not np.array_equal(a["E"], c["E"])
    idx = np.array([3, 17, 999])
    s = W.subsample(a, idx)
    for k in a:
        assert np.array_equal(s[k], a[k][idx]) and s[k].flags["C_CONTIGUOUS"]


def test_lens_and_backtrack_samples():
    r_lo, r_hi, nb, per = 1e18, 1e20, 10, 5000
    dirs, E, bins = W.lens_samples(nb, per, r_lo, r_hi, seed=5)
    assert len(E) == nb * per and np.array_equal(np.bincount(bins), np.full(nb, per))
    edges = np.geomspace(r_lo, r_hi, nb + 1)
    assert np.allclose(E, np.sqrt(edges[bins] * edges[bins + 1]), rtol=1e-13)
    _isotropic_ok(dirs[:, 0], dirs[:, 1], dirs[:, 2])
    d2, R = W.backtrack_directions(N, r_lo, r_hi, seed=6)
    _isotropic_ok(d2[:, 0], d2[:, 1], d2[:, 2])
    lo, hi = np.log(r_lo), np.log(r_hi)
    assert stats.kstest(np.log(R), stats.uniform(loc=lo, scale=hi - lo).cdf).pvalue > P_MIN
