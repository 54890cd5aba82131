"""Candidate sharding (the multi-GPU partition: candidates are independent,
Sect. 3) through the library on one GPU: a batch split into two id-disjoint
shards, propagated one after the other, gives per-id records byte-identical
to the run of the whole batch, and the shards' device histograms (detected
energy spectrum and HEALPix arrival map), summed on the device, equal the
whole batch's.  This is what a multi-rank job relies on when it sums the
ranks' histograms and gathers their records."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402
from paper_1307_2643_gb300 import crp  # noqa: E402

H0_OVER_C = 67.3e3 / 299792458.0
FLAGS = crp.PAIR | crp.ADIABATIC | crp.PION | crp.PHOTODIS | crp.EMIN | crp.OBSERVER
NSIDE = 16


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_1307_2643_gb300.build import build
    build()
    n, dx = (64, 64, 64), 0.25
    field = oracle.turbulent_field(n, dx, 0.5, 8.0, 1.0, seed=17).astype(np.float32)
    inj = workloads.mixed_interactions(n=24_000, seed=23)
    inj["s_max"] = np.full(len(inj["E"]), 150.0)
    # sources near the observer, so that the shards detect enough
    inj["x"] *= 0.1
    inj["y"] *= 0.1
    inj["z"] *= 0.1
    tabs = oracle.tables_build(n=1000)
    return torch, n, dx, field, crp.host_injection(inj), tabs


def _run(setup, precision, shards):
    torch, n, dx, field, inj, tabs = setup
    m = len(inj["E"])
    ctx = crp.crp_context_create(0, 77, 40 * m)
    try:
        g = crp.crp_grid_create(ctx, crp.grid_desc(n, dx, dtype=crp.F32, data=field,
                                                   data_dtype=crp.F32))
        th = crp.crp_tables_from_host(ctx, crp.tables_desc(n=1000), tabs.beta_pair,
                                      tabs.rate_pion, tabs.rate_gdr)
        mods = crp.modules(precision=precision, flags=FLAGS, tol=1e-4, h_min=0.01, h_max=1.0,
                           beta_ad=H0_OVER_C, e_min=1e18, tables=th, observer_radius=1.0)
        hist = torch.zeros(60, dtype=torch.int64, device="cuda")
        amap = torch.zeros(12 * NSIDE * NSIDE, dtype=torch.int64, device="cuda")
        recs = []
        for k, idx in enumerate(shards):
            sub = {key: np.ascontiguousarray(v[idx]) for key, v in inj.items()}
            crp.crp_candidates_clear(ctx)
            crp.crp_candidates_inject(ctx, crp.candidate_arrays(sub), len(idx))
            status, _ = crp.crp_propagate(ctx, g, mods)
            assert status == crp.OK
            recs.append(crp.crp_collect(ctx, crp.COLLECT_ALL))
            crp.crp_histogram_energy_device(ctx, crp.COLLECT_DETECTED, 1e18, 1e21, 60, hist,
                                            accumulate=k > 0)
            crp.crp_histogram_healpix_device(ctx, crp.COLLECT_DETECTED, NSIDE, 0, amap,
                                             accumulate=k > 0)
        torch.cuda.synchronize()
        crp.crp_tables_destroy(th)
        crp.crp_grid_destroy(g)
    finally:
        crp.crp_context_destroy(ctx)
    return np.sort(np.concatenate(recs), order="id"), hist.cpu().numpy(), amap.cpu().numpy()


@pytest.mark.parametrize("precision", [crp.FP64, crp.MIXED])
def test_shards_equal_the_union(setup, precision):
    m = len(setup[4]["E"])
    whole = [np.arange(m)]
    perm = np.random.default_rng(3).permutation(m)
    split = [np.sort(perm[: m // 3]), np.sort(perm[m // 3:])]
    rec_u, hist_u, map_u = _run(setup, precision, whole)
    rec_s, hist_s, map_s = _run(setup, precision, split)
    assert len(rec_u) > m  # photodisintegration secondaries included
    assert (rec_u["generation"] > 0).sum() > 100
    assert rec_s.tobytes() == rec_u.tobytes()
    det = (rec_u["status"] == crp.DETECTED).sum()
    assert det > 50, det
    assert np.array_equal(hist_s, hist_u) and hist_u.sum() > 0
    assert np.array_equal(map_s, map_u) and map_u.sum() == det


def test_healpix_device_map_equals_host_map(setup):
    """crp_histogram_healpix_device against crp_histogram_healpix, and its
    argument checks (an unaligned device array is rejected before any
    kernel runs)."""
    torch, n, dx, field, inj, tabs = setup
    m = 4000
    sub = {key: np.ascontiguousarray(v[:m]) for key, v in inj.items()}
    ctx = crp.crp_context_create(0, 5, 40 * m)
    try:
        g = crp.crp_grid_create(ctx, crp.grid_desc(n, dx, dtype=crp.F32, data=field,
                                                   data_dtype=crp.F32))
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(sub), m)
        crp.crp_propagate(ctx, g, crp.modules(precision=crp.MIXED, h_min=0.01, h_max=1.0))
        for what in (crp.COLLECT_ALL, crp.COLLECT_FINISHED):
            host = crp.crp_histogram_healpix(ctx, what, NSIDE, 0)
            dev = torch.full((12 * NSIDE * NSIDE,), 7, dtype=torch.int64, device="cuda")
            crp.crp_histogram_healpix_device(ctx, what, NSIDE, 0, dev)
            assert np.array_equal(dev.cpu().numpy().astype(np.uint64), host)
            crp.crp_histogram_healpix_device(ctx, what, NSIDE, 0, dev, accumulate=True)
            assert np.array_equal(dev.cpu().numpy().astype(np.uint64), 2 * host)
        raw = torch.zeros(12 * NSIDE * NSIDE + 1, dtype=torch.int64, device="cuda")
        bad = raw.view(torch.uint8)[4:4 + 8 * 12 * NSIDE * NSIDE]
        with pytest.raises(crp.CrpError) as e:
            crp.crp_histogram_healpix_device(ctx, crp.COLLECT_ALL, NSIDE, 0, bad)
        assert e.value.status == crp.E_INVALID
        with pytest.raises(crp.CrpError):
            crp.crp_histogram_healpix_device(ctx, crp.COLLECT_ALL, 0, 0, raw)
        crp.crp_grid_destroy(g)
    finally:
        crp.crp_context_destroy(ctx)
