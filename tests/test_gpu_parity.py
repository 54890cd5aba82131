"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle on
the same seeded inputs.

Bars (from the method's required tolerances):
  * integer / index results (statuses, interaction counts, draw counters,
    species, lineage ids, generations) bit-exact;
  * FP64 path: positions, directions, energies, lengths within rel 1e-9;
  * mixed path: within rel 1e-5 on quasi-ballistic candidates, and by
    distribution (KS p > 0.01) where the trajectories are chaotic.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402
from gpu_util import assert_chains_equal, oracle_params, rel_err, run_gpu  # noqa: E402
from paper_1307_2643_gb300 import crp  # noqa: E402

H0_OVER_C = 67.3e3 / 299792458.0  # 1/Mpc


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1307_2643_gb300.build import build
    build()
    oracle.build()


@pytest.fixture(scope="module")
def field64():
    n, dx = (64, 64, 64), 0.25
    return n, dx, oracle.turbulent_field(n, dx, 0.5, 8.0, 1.0, seed=21)


@pytest.fixture(scope="module")
def tables():
    return oracle.tables_build(n=1000)


def _plain(n_cand, seed=31, s_max=50.0):
    inj = workloads.plain_small(n=n_cand, seed=seed)
    inj["s_max"] = np.full(n_cand, s_max)
    return inj


# ---------------------------------------------------------------------------
# setup kernels
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [(64, 64, 64), (24, 20, 18)])
def test_turbulence_generator_matches_oracle(n):
    dx, lmin, lmax, brms, seed = 0.25, 0.5, 5.0, 1.7, 4242
    ref = oracle.turbulent_field(n, dx, lmin, lmax, brms, seed=seed)
    ctx = crp.crp_context_create(0, 1, 16)
    try:
        d = crp.grid_desc(n, dx, dtype=crp.F64, source=crp.GRID_TURBULENT, lmin=lmin, lmax=lmax,
                          brms=brms, seed=seed)
        g = crp.crp_grid_create(ctx, d)
        got = crp.crp_grid_copy_out(g, n)
        crp.crp_grid_destroy(g)
    finally:
        crp.crp_context_destroy(ctx)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) < 1e-10 * brms


def test_turbulence_f32_storage_is_rounded_f64():
    n, dx = (32, 32, 32), 0.25
    ctx = crp.crp_context_create(0, 1, 16)
    try:
        out = []
        for dt in (crp.F64, crp.F32):
            d = crp.grid_desc(n, dx, dtype=dt, source=crp.GRID_TURBULENT, lmin=0.5, lmax=8.0,
                              brms=1.0, seed=3)
            g = crp.crp_grid_create(ctx, d)
            out.append(crp.crp_grid_copy_out(g, n))
            crp.crp_grid_destroy(g)
    finally:
        crp.crp_context_destroy(ctx)
    assert np.array_equal(out[0].astype(np.float32).astype(np.float64), out[1])


def test_tables_match_oracle(tables):
    ctx = crp.crp_context_create(0, 1, 16)
    try:
        t = crp.crp_tables_build(ctx, crp.tables_desc(n=1000))
        beta, pion, gdr = crp.crp_tables_copy_out(t, 1000)
        crp.crp_tables_destroy(t)
    finally:
        crp.crp_context_destroy(ctx)
    for got, ref in ((beta, tables.beta_pair), (pion, tables.rate_pion), (gdr, tables.rate_gdr)):
        live = ref > 1e-200 * ref.max()
        assert np.all((got == 0) == (ref == 0)) or np.all(np.abs(got[~live]) < 1e-150 * ref.max())
        assert np.max(rel_err(got[live], ref[live], floor=0.0)) < 1e-8


def test_tables_with_synthetic_infrared_background_match_oracle():
    """Pair table with the synthetic infrared / optical background (two dilute
    blackbodies) built on the device against the oracle's, and the
    propagation with it: FP64 path bit-exact with the oracle."""
    irb = ((35.0, 8.5e-7), (4500.0, 3.1e-15))
    ref = oracle.tables_build(n=400, irb=irb)
    ctx = crp.crp_context_create(0, 1, 16)
    try:
        t = crp.crp_tables_build(ctx, crp.tables_desc(n=400, irb=irb))
        beta, pion, gdr = crp.crp_tables_copy_out(t, 400)
        crp.crp_tables_destroy(t)
        with pytest.raises(crp.CrpError):
            crp.crp_tables_build(ctx, crp.tables_desc(n=400, irb=((0.0, 1e-6),)))
    finally:
        crp.crp_context_destroy(ctx)
    live = ref.beta_pair > 1e-200 * ref.beta_pair.max()
    assert np.max(rel_err(beta[live], ref.beta_pair[live], floor=0.0)) < 1e-8
    assert np.max(rel_err(pion, ref.rate_pion, floor=1e-300)) < 1e-8
    # propagation with the background: protons of 1e17-1e18.5 eV, where the
    # infrared light dominates the pair losses
    n, dx = (16, 16, 16), 0.5
    B = oracle.turbulent_field(n, dx, 1.0, 4.0, 1.0, seed=3)
    g = np.random.default_rng(8)
    m = 500
    v = g.normal(size=(m, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    inj = dict(id=np.arange(m, dtype=np.uint64), x=np.zeros(m), y=np.zeros(m), z=np.zeros(m),
               ux=v[:, 0].copy(), uy=v[:, 1].copy(), uz=v[:, 2].copy(),
               E=10 ** g.uniform(17, 18.5, m), A=np.ones(m, np.int32), Z=np.ones(m, np.int32),
               q=np.ones(m, np.int32), s_max=np.full(m, 30.0))
    kw = dict(tol=1e-4, h_min=0.01, h_max=1.0)
    P = oracle_params(n, dx, tables=ref, flags=oracle.PAIR, **kw)
    r_irb = oracle.propagate(P, B, inj, tables=ref)
    gpu, _, status = run_gpu(B, n, dx, inj, precision=crp.FP64, tables=ref, flags=crp.PAIR, **kw)
    assert status == crp.OK
    assert_chains_equal(gpu, r_irb)
    for f in ("x", "u", "E", "s"):
        assert np.max(rel_err(gpu[f], r_irb[f])) < 1e-9, f
    plain = oracle.tables_build(n=400)
    r_cmb = oracle.propagate(oracle_params(n, dx, tables=plain, flags=oracle.PAIR, **kw), B, inj,
                             tables=plain)
    assert np.all(r_irb["E"] <= r_cmb["E"]) and np.mean(r_irb["E"] < r_cmb["E"]) > 0.9


# ---------------------------------------------------------------------------
# FP64 path: bit-level agreement expected (same operation order, no FMA)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [crp.F64, crp.F32])
def test_fp64_plain_parity(field64, dtype):
    n, dx, B = field64
    Bin = B if dtype == crp.F64 else B.astype(np.float32).astype(np.float64)
    inj = _plain(3001)
    kw = dict(tol=1e-4, h_min=0.01, h_max=1.0)
    gpu, st, status = run_gpu(Bin, n, dx, inj, precision=crp.FP64, dtype=dtype, **kw)
    ref = oracle.propagate(oracle_params(n, dx, **kw), Bin, inj)
    assert status == crp.OK
    assert_chains_equal(gpu, ref)
    assert np.array_equal(gpu["n_acc"], ref["n_acc"]) and np.array_equal(gpu["n_rej"], ref["n_rej"])
    for f in ("x", "u", "E", "s"):
        assert np.max(rel_err(gpu[f], ref[f])) < 1e-9, f
    assert st["accepted_steps"] == int(ref["n_acc"].sum())
    assert st["rejected_trials"] == int(ref["n_rej"].sum())
    assert np.all(gpu["status"] == crp.MAX_LENGTH)


def _interaction_inputs(n_mixed=1200, n_hot=240, seed=77):
    w = workloads.MIXED_INTERACTIONS
    inj = workloads.mixed_interactions(n=n_mixed, seed=seed)
    g = np.random.default_rng(seed)
    A = np.where(g.random(n_hot) < 0.5, 56, 14).astype(np.int32)
    Z = np.where(A == 56, 26, 7).astype(np.int32)
    v = g.normal(size=(n_hot, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    hot = dict(id=np.arange(n_mixed, n_mixed + n_hot, dtype=np.uint64),
               x=g.uniform(-20, 20, n_hot), y=g.uniform(-20, 20, n_hot), z=g.uniform(-20, 20, n_hot),
               ux=v[:, 0].copy(), uy=v[:, 1].copy(), uz=v[:, 2].copy(),
               E=10 ** g.uniform(19.8, 21.0, n_hot), A=A, Z=Z, q=np.ones(n_hot, np.int32))
    out = {k: np.concatenate([inj[k], hot[k]]) for k in hot}
    out["s_max"] = np.full(len(out["E"]), 40.0)
    return out


INTERACTION_FLAGS = (crp.PAIR | crp.ADIABATIC | crp.PION | crp.PHOTODIS | crp.EMIN |
                     crp.OBSERVER)


def _interaction_kw():
    return dict(tol=1e-4, h_min=0.01, h_max=1.0, beta_ad=H0_OVER_C, e_min=1e18)


@pytest.fixture(scope="module")
def field_f32_small():
    n, dx = (64, 64, 64), 0.1
    B = oracle.turbulent_field(n, dx, 0.2, 5.0, 1.0, seed=22)
    return n, dx, B.astype(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def interaction_ref(field_f32_small, tables):
    n, dx, B = field_f32_small
    inj = _interaction_inputs()
    P = oracle_params(n, dx, tables=tables, flags=INTERACTION_FLAGS, obs_r=1.0, **_interaction_kw())
    return inj, oracle.propagate(P, B, inj, tables=tables)


def test_fp64_interactions_parity(field_f32_small, tables, interaction_ref):
    n, dx, B = field_f32_small
    inj, ref = interaction_ref
    gpu, st, status = run_gpu(B, n, dx, inj, precision=crp.FP64, dtype=crp.F32, tables=tables,
                              flags=INTERACTION_FLAGS, observer_radius=1.0, **_interaction_kw())
    assert status == crp.OK
    # the workload exercises every module
    assert ref["n_pion"].sum() > 50 and ref["n_pd"].sum() > 50
    assert (ref["generation"] > 0).sum() > 20
    assert set(np.unique(ref["status"])) >= {crp.BELOW_EMIN, crp.MAX_LENGTH}
    assert_chains_equal(gpu, ref)
    for f in ("x", "u", "E", "s", "x0", "u0", "E0"):
        assert np.max(rel_err(gpu[f], ref[f])) < 1e-9, f
    assert st["n_pion"] == int(ref["n_pion"].sum())
    assert st["n_pd"] == int(ref["n_pd"].sum())
    assert st["n_secondaries"] == int((ref["generation"] > 0).sum())


def _decay_inputs(seed=41):
    """Nuclei (some photodisintegrating into free neutrons) plus injected free
    neutrons of 10^17.5 - 10^20 eV (decay lengths 3 kpc - 0.9 Mpc)."""
    inj = _interaction_inputs(n_mixed=400, n_hot=160, seed=seed)
    g = np.random.default_rng(seed)
    m = 400
    v = g.normal(size=(m, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    neu = dict(id=np.arange(10 ** 6, 10 ** 6 + m, dtype=np.uint64), x=g.uniform(-20, 20, m),
               y=g.uniform(-20, 20, m), z=g.uniform(-20, 20, m), ux=v[:, 0].copy(),
               uy=v[:, 1].copy(), uz=v[:, 2].copy(), E=10 ** g.uniform(17.5, 20.0, m),
               A=np.ones(m, np.int32), Z=np.zeros(m, np.int32), q=np.ones(m, np.int32),
               s_max=np.full(m, 40.0))
    return {k: np.concatenate([inj[k], neu[k]]) for k in neu}


def test_neutron_decay_parity(field_f32_small, tables):
    """Neutron beta decay on top of pion production and photodisintegration:
    the FP64 path equals the oracle (chains, decays of injected and of
    secondary neutrons, every float within 1e-9); the mixed path decays the
    same neutrons wherever its stopping condition agrees."""
    n, dx, B = field_f32_small
    inj = _decay_inputs()
    flags = INTERACTION_FLAGS | crp.DECAY
    P = oracle_params(n, dx, tables=tables, flags=flags, obs_r=1.0, **_interaction_kw())
    ref = oracle.propagate(P, B, inj, tables=tables)
    gpu, st, status = run_gpu(B, n, dx, inj, precision=crp.FP64, dtype=crp.F32, tables=tables,
                              flags=flags, observer_radius=1.0, **_interaction_kw())
    assert status == crp.OK
    decayed = (ref["A0"] == 1) & (ref["Z0"] == 0) & (ref["Z"] == 1)
    assert decayed.sum() > 100
    assert ((ref["generation"] > 0) & (ref["Z0"] == 0) & (ref["Z"] == 1)).sum() > 0
    assert_chains_equal(gpu, ref)
    for f in ("x", "u", "E", "s", "x0", "u0", "E0"):
        assert np.max(rel_err(gpu[f], ref[f])) < 1e-9, f
    mx, _, status = run_gpu(B, n, dx, inj, precision=crp.MIXED, dtype=crp.F32, tables=tables,
                            flags=flags, observer_radius=1.0, **_interaction_kw())
    assert status == crp.OK
    prim_r, prim_m = ref[ref["generation"] == 0], mx[mx["generation"] == 0]
    assert np.array_equal(prim_r["id"], prim_m["id"])
    neutrons = (prim_r["A0"] == 1) & (prim_r["Z0"] == 0)
    same = neutrons & (prim_r["status"] == prim_m["status"])
    assert same.sum() > 0.9 * neutrons.sum()
    assert np.mean(prim_r["Z"][same] == prim_m["Z"][same]) > 0.99


def test_launch_configuration_does_not_change_results(field_f32_small, tables):
    n, dx, B = field_f32_small
    inj = _interaction_inputs(n_mixed=300, n_hot=100, seed=5)
    kw = dict(precision=crp.FP64, dtype=crp.F32, tables=tables, flags=INTERACTION_FLAGS,
              observer_radius=1.0, **_interaction_kw())
    a, _, _ = run_gpu(B, n, dx, inj, block_size=32, blocks_per_sm=1, **kw)
    b, _, _ = run_gpu(B, n, dx, inj, block_size=128, slice=7, **kw)
    c, _, _ = run_gpu(B, n, dx, inj, block_size=64, blocks_per_sm=3, slice=100000, **kw)
    assert a.tobytes() == b.tobytes() == c.tobytes()


def test_timeout_and_resume_is_bit_identical(field_f32_small, tables):
    n, dx, B = field_f32_small
    inj = crp.host_injection(_interaction_inputs(n_mixed=400, n_hot=80, seed=9))
    m = len(inj["E"])
    full, _, _ = run_gpu(B, n, dx, inj, precision=crp.FP64, dtype=crp.F32, tables=tables,
                         flags=INTERACTION_FLAGS, observer_radius=1.0, **_interaction_kw())
    ctx = crp.crp_context_create(0, 1234, 64 * m)
    try:
        g = crp.crp_grid_create(ctx, crp.grid_desc(n, dx, dtype=crp.F32, data=B))
        th = crp.crp_tables_from_host(ctx, crp.tables_desc(n=tables.n), tables.beta_pair,
                                      tables.rate_pion, tables.rate_gdr)
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), m)
        M = crp.modules(precision=crp.FP64, tables=th, flags=INTERACTION_FLAGS,
                        observer_radius=1.0, step_budget=20000, **_interaction_kw())
        calls = 0
        while True:
            status, st = crp.crp_propagate(ctx, g, M, raise_on_error=False)
            calls += 1
            assert status in (crp.OK, crp.E_TIMEOUT)
            if status == crp.OK:
                break
            assert st.n_active > 0
            assert calls < 10000
        resumed = np.sort(crp.crp_collect(ctx, crp.COLLECT_ALL), order="id")
        crp.crp_tables_destroy(th)
        crp.crp_grid_destroy(g)
    finally:
        crp.crp_context_destroy(ctx)
    assert calls > 3
    assert resumed.tobytes() == full.tobytes()


def test_queue_overflow_reports_and_finishes(field_f32_small, tables):
    n, dx, B = field_f32_small
    inj = _interaction_inputs(n_mixed=0, n_hot=200, seed=13)
    m = len(inj["E"])
    gpu, st, status = run_gpu(B, n, dx, inj, precision=crp.FP64, dtype=crp.F32, tables=tables,
                              capacity=m + 5, flags=INTERACTION_FLAGS, observer_radius=1.0,
                              **_interaction_kw())
    assert status == crp.E_QUEUE_FULL
    assert st["n_overflow"] > 0 and st["error_word"] & 1
    assert len(gpu) == m + 5
    assert np.all(gpu["status"] != crp.ACTIVE)


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_edge_cases(field64):
    n, dx, B = field64
    kw = dict(tol=1e-4, h_min=0.01, h_max=1.0, flags=crp.EMIN | crp.OBSERVER, e_min=2e19,
              observer_radius=1.0)
    inj = _plain(7)
    inj["E"][:] = 5e19
    inj["s_max"][0] = 0.0                      # zero budget: one zero-length step
    inj["E"][1] = 1e19                         # below e_min at injection
    inj["x"][2], inj["y"][2], inj["z"][2] = 0.3, 0.0, 0.0  # starts inside the observer
    inj["x"][3] = 5.0                          # heads for the observer
    inj["ux"][3], inj["uy"][3], inj["uz"][3] = -1.0, 0.0, 0.0
    inj["E"][3] = 1e21
    gpu, _, status = run_gpu(B, n, dx, inj, precision=crp.FP64, **kw)
    okw = dict(kw)
    flags = okw.pop("flags")
    okw.pop("observer_radius")
    ref = oracle.propagate(oracle_params(n, dx, flags=oracle.EMIN | oracle.OBSERVER, obs_r=1.0,
                                         **okw), B, inj)
    assert status == crp.OK
    assert_chains_equal(gpu, ref)
    assert gpu["status"][0] == crp.MAX_LENGTH and gpu["n_acc"][0] == 1 and gpu["s"][0] == 0.0
    assert gpu["status"][1] == crp.BELOW_EMIN and gpu["n_acc"][1] == 1
    assert gpu["status"][2] != crp.DETECTED
    assert gpu["status"][3] == crp.DETECTED
    assert np.max(rel_err(gpu["x"], ref["x"])) < 1e-9


def test_empty_and_invalid_inputs(field64):
    n, dx, B = field64
    ctx = crp.crp_context_create(0, 1, 8)
    try:
        g = crp.crp_grid_create(ctx, crp.grid_desc(n, dx, dtype=crp.F64, data=B))
        status, st = crp.crp_propagate(ctx, g, crp.modules())   # empty pool
        assert status == crp.OK and st.accepted_steps == 0
        assert len(crp.crp_collect(ctx)) == 0
        bad = crp.host_injection(_plain(3))
        bad["A"][1] = 0
        with pytest.raises(crp.CrpError) as e:
            crp.crp_candidates_inject(ctx, crp.candidate_arrays(bad), 3)
        assert e.value.status == crp.E_INVALID
        assert crp.crp_context_size(ctx) == 0
        with pytest.raises(crp.CrpError) as e:
            crp.crp_candidates_inject(ctx, crp.candidate_arrays(crp.host_injection(_plain(9))), 9)
        assert e.value.status == crp.E_QUEUE_FULL
        with pytest.raises(crp.CrpError):
            crp.crp_propagate(ctx, g, crp.modules(h_min=0.0))
        # the other calls on an empty pool: histograms of nothing, the
        # surrogate on no samples
        assert not np.any(crp.crp_histogram_energy(ctx, crp.COLLECT_ALL, 1e18, 1e21, 10))
        assert not np.any(crp.crp_histogram_healpix(ctx, crp.COLLECT_ALL, 4, 0))
        import torch
        mlp = crp.crp_mlp_create(ctx, 4, 256, 4, 7)
        try:
            crp.crp_mlp_forward(mlp, torch.zeros((0, 4), device="cuda"),
                                torch.zeros((0, 3), device="cuda"), 0)
        finally:
            crp.crp_mlp_destroy(mlp)
        crp.crp_grid_destroy(g)
    finally:
        crp.crp_context_destroy(ctx)


# ---------------------------------------------------------------------------
# mixed precision
# ---------------------------------------------------------------------------
def _pos_err(a, b):
    return np.linalg.norm(a["x"] - b["x"], axis=1) / np.maximum(1.0, np.linalg.norm(b["x"], axis=1))


FLOOR_AXES = ((0.267, 0.535, 0.802), (0.9, -0.3, 0.1), (-0.2, 0.7, -0.6))
FLOOR_GATE = 2e-6


def _kicked(inj, delta, axis):
    """Injection with each direction turned by delta[i] radians (to first
    order) about an axis perpendicular to it and to `axis`."""
    p = dict(inj)
    u = np.stack([p["ux"], p["uy"], p["uz"]], 1)
    v = np.cross(u, np.asarray(axis, dtype=np.float64))
    v /= np.linalg.norm(v, axis=1)[:, None]
    u2 = u + delta[:, None] * v
    u2 /= np.linalg.norm(u2, axis=1)[:, None]
    p["ux"], p["uy"], p["uz"] = [np.ascontiguousarray(u2[:, k]) for k in range(3)]
    return p


@pytest.fixture(scope="module")
def ballistic_refs(field64):
    """Oracle at the operating tolerance, at a resolving tolerance, and a
    tol = 1e-10 reference ("truth") for 1e19-1e20 eV protons over 50 Mpc;
    and, per tolerance, each candidate's chaos floor: the largest endpoint
    change of the oracle's own history when the initial direction is turned
    by 2^-24 sqrt(N) radians (N: the candidate's accepted steps), about
    three different axes.  2^-24 is the binary32 unit roundoff and sqrt(N)
    the random-walk growth of one rounding per step, so the floor is the
    endpoint spread the method itself shows under binary32-sized
    perturbations."""
    n, dx, B = field64
    B32 = B.astype(np.float32).astype(np.float64)
    inj = _plain(3001)
    refs, floors = {}, {}
    for tol, hmin in ((1e-4, 0.01), (1e-8, 1e-4), (1e-10, 1e-4)):
        P = oracle_params(n, dx, tol=tol, h_min=hmin, h_max=1.0)
        refs[tol] = oracle.propagate(P, B32, inj)
        if tol >= 1e-8:
            delta = 2.0 ** -24 * np.sqrt(refs[tol]["n_acc"].astype(np.float64))
            floors[tol] = np.max([_pos_err(oracle.propagate(P, B32, _kicked(inj, delta, a)),
                                           refs[tol]) for a in FLOOR_AXES], axis=0)
    return B32, inj, refs, floors


@pytest.mark.parametrize("tol,hmin", [(1e-4, 0.01), (1e-8, 1e-4)])
def test_mixed_equal_error(field64, ballistic_refs, tol, hmin):
    """Mixed precision at equal error: against a tol = 1e-10 reference the
    mixed path's endpoint errors have the same distribution as the FP64
    method's own discretization errors at the same tolerance.  Per
    candidate: wherever the chaos floor (see ballistic_refs) is at most
    2e-6, the mixed endpoint is within 1e-5 of the FP64 endpoint; where the
    floor is larger the method itself does not fix the endpoint to 1e-5
    (the step controller turns a rounding-level difference into another
    step sequence) and only the distribution is compared."""
    n, dx, _ = field64
    B32, inj, refs, floors = ballistic_refs
    gpu, st, status = run_gpu(B32, n, dx, inj, precision=crp.MIXED, dtype=crp.F32, tol=tol,
                              h_min=hmin, h_max=1.0)
    assert status == crp.OK
    ref, truth = refs[tol], refs[1e-10]
    assert_chains_equal(gpu, ref)
    assert np.array_equal(gpu["E"], ref["E"]) and np.array_equal(gpu["s"], ref["s"])
    e_mx, e_64 = _pos_err(gpu, truth), _pos_err(ref, truth)
    assert np.median(e_mx) <= 1.5 * np.median(e_64) + 1e-9, (np.median(e_mx), np.median(e_64))
    assert np.percentile(e_mx, 90) <= 2.0 * np.percentile(e_64, 90) + 1e-9
    assert abs(int(gpu["n_acc"].sum()) - int(ref["n_acc"].sum())) < 0.01 * ref["n_acc"].sum()
    # per candidate, where the chaos floor allows 1e-5
    e = _pos_err(gpu, ref)
    gated = floors[tol] <= FLOOR_GATE
    report = (f"tol {tol}: {gated.sum()} of {len(e)} candidates gated; gated max "
              f"{e[gated].max() if gated.any() else 0:.3g}; ungated median "
              f"{np.median(e[~gated]):.3g}, p90 {np.percentile(e[~gated], 90):.3g}, "
              f"within 1e-5 {np.mean(e[~gated] <= 1e-5):.3f}")
    print(report)
    assert np.all(e[gated] <= 1e-5), report
    if tol <= 1e-8:
        # where the method resolves 1e-5 the gate is not vacuous
        assert gated.sum() >= 0.1 * len(e), report


def test_mixed_interactions_statistics(field_f32_small, tables, interaction_ref):
    """Chaotic low-rigidity nuclei: per-candidate paths diverge, the physics
    must not: energies and species agree by distribution, interaction counts
    and energies of quasi-ballistic candidates per candidate."""
    from scipy.stats import ks_2samp
    n, dx, B = field_f32_small
    inj, ref = interaction_ref
    gpu, _, status = run_gpu(B, n, dx, inj, precision=crp.MIXED, dtype=crp.F32, tables=tables,
                             flags=INTERACTION_FLAGS, observer_radius=1.0, **_interaction_kw())
    assert status == crp.OK
    assert abs(len(gpu) - len(ref)) <= 0.02 * len(ref)
    for f in ("E",):
        p = ks_2samp(np.log(gpu[f]), np.log(ref[f])).pvalue
        assert p > 0.01, (f, p)
    prim_g = gpu[gpu["generation"] == 0]
    prim_r = ref[ref["generation"] == 0]
    assert np.array_equal(prim_g["id"], prim_r["id"])
    # energy losses and interactions do not depend on position: per candidate
    # they agree wherever the stopping condition did
    same = prim_g["status"] == prim_r["status"]
    assert same.mean() > 0.95
    e = rel_err(prim_g["E"][same], prim_r["E"][same], floor=0.0)
    assert np.median(e) < 1e-5
    assert np.mean(prim_g["n_pion"][same] == prim_r["n_pion"][same]) > 0.95
    # arrival maps: final directions by distribution (cos theta, phi) and a
    # HEALPix nside-4 map (two-sample chi-square)
    from scipy.stats import chi2 as chi2_dist
    for comp in (lambda u: u[:, 2], lambda u: np.arctan2(u[:, 1], u[:, 0])):
        p = ks_2samp(comp(gpu["u"]), comp(ref["u"])).pvalue
        assert p > 0.01, p
    a = np.bincount(oracle.ang2pix_vec(4, gpu["u"]), minlength=192).astype(float)
    b = np.bincount(oracle.ang2pix_vec(4, ref["u"]), minlength=192).astype(float)
    keep = (a + b) > 0
    a, b = a[keep], b[keep]
    stat = np.sum((np.sqrt(b.sum() / a.sum()) * a - np.sqrt(a.sum() / b.sum()) * b) ** 2 / (a + b))
    assert chi2_dist.sf(stat, len(a) - 1) > 0.01


@pytest.mark.parametrize("precision", [crp.FP64, crp.MIXED])
def test_checkpoint_restore_resumes_bit_identically(field_f32_small, tables, precision):
    """Interrupt by a step budget and checkpoint; finish once in the same
    context and once in a new context (other seed and capacity: the image
    carries the seed) restored from the image.  Both give the same records;
    on the binary64 path they also equal an uninterrupted run's (the mixed
    path re-derives its binary32 cell coordinates when a candidate is
    reloaded, so where it was interrupted is part of its history)."""
    n, dx, B = field_f32_small
    inj = crp.host_injection(_interaction_inputs(n_mixed=300, n_hot=60, seed=19))
    m = len(inj["E"])
    full, _, _ = run_gpu(B, n, dx, inj, precision=precision, dtype=crp.F32, tables=tables,
                         flags=INTERACTION_FLAGS, observer_radius=1.0, **_interaction_kw())

    def open_ctx(seed, cap):
        ctx = crp.crp_context_create(0, seed, cap)
        g = crp.crp_grid_create(ctx, crp.grid_desc(n, dx, dtype=crp.F32, data=B))
        th = crp.crp_tables_from_host(ctx, crp.tables_desc(n=tables.n), tables.beta_pair,
                                      tables.rate_pion, tables.rate_gdr)
        M = crp.modules(precision=precision, tables=th, flags=INTERACTION_FLAGS,
                        observer_radius=1.0, **_interaction_kw())
        return ctx, g, M

    ctx, g, M = open_ctx(1234, 64 * m)
    try:
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), m)
        M.step_budget = 30000
        status, st = crp.crp_propagate(ctx, g, M, raise_on_error=False)
        assert status == crp.E_TIMEOUT and st.n_active > 0
        image = crp.crp_checkpoint(ctx)
        M.step_budget = 0
        crp.crp_propagate(ctx, g, M)
        same_ctx = np.sort(crp.crp_collect(ctx, crp.COLLECT_ALL), order="id")
    finally:
        crp.crp_context_destroy(ctx)
    ctx, g, M = open_ctx(999, 80 * m)
    try:
        bad = image.copy()
        bad[len(bad) // 2] ^= 0x40
        for broken in (bad, image[:-4]):
            with pytest.raises(crp.CrpError) as ei:
                crp.crp_restore(ctx, broken)
            assert ei.value.status == crp.E_INVALID
        crp.crp_restore(ctx, image)
        crp.crp_propagate(ctx, g, M)
        restored = np.sort(crp.crp_collect(ctx, crp.COLLECT_ALL), order="id")
        small = crp.crp_context_create(0, 1, 4)  # capacity below the image's candidates
        try:
            with pytest.raises(crp.CrpError):
                crp.crp_restore(small, image)
        finally:
            crp.crp_context_destroy(small)
    finally:
        crp.crp_context_destroy(ctx)
    assert restored.tobytes() == same_ctx.tobytes()
    if precision == crp.FP64:
        assert restored.tobytes() == full.tobytes()


EGAL_FLAGS = crp.PAIR | crp.ADIABATIC | crp.PION | crp.EMIN | crp.OBSERVER


@pytest.mark.parametrize("flags", [INTERACTION_FLAGS, EGAL_FLAGS])
def test_mixed_launch_configuration_does_not_change_results(field_f32_small, tables, flags):
    """The mixed path's results do not depend on block size, register
    variant, queue order or slice (the library rounds slices up to multiples
    of its rebase period, so the 64-step slice here runs as 128).  Both module lists here (with and without
    photodisintegration) have kernels that fix the list at compile time: the
    256 x 2 launch runs those, the other launches the generic kernel, and
    all give the same bytes."""
    n, dx, B = field_f32_small
    inj = _interaction_inputs(n_mixed=300, n_hot=100, seed=6)
    kw = dict(precision=crp.MIXED, dtype=crp.F32, tables=tables, flags=flags,
              observer_radius=1.0, **_interaction_kw())
    a, _, _ = run_gpu(B, n, dx, inj, block_size=256, blocks_per_sm=2, slice=512, queue_order=0,
                      **kw)
    b, _, _ = run_gpu(B, n, dx, inj, block_size=128, blocks_per_sm=6, slice=64, queue_order=1,
                      **kw)
    c, _, _ = run_gpu(B, n, dx, inj, block_size=32, blocks_per_sm=3, queue_order=-1, **kw)
    assert a.tobytes() == b.tobytes() == c.tobytes()


def test_autotune_keeps_state_and_results(field_f32_small, tables):
    n, dx, B = field_f32_small
    inj = crp.host_injection(_interaction_inputs(n_mixed=3000, n_hot=300, seed=8))
    m = len(inj["E"])
    ref, _, _ = run_gpu(B, n, dx, inj, precision=crp.MIXED, dtype=crp.F32, tables=tables,
                        flags=INTERACTION_FLAGS, observer_radius=1.0, **_interaction_kw())
    ctx = crp.crp_context_create(0, 1234, 64 * m)
    try:
        g = crp.crp_grid_create(ctx, crp.grid_desc(n, dx, dtype=crp.F32, data=B))
        th = crp.crp_tables_from_host(ctx, crp.tables_desc(n=tables.n), tables.beta_pair,
                                      tables.rate_pion, tables.rate_gdr)
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), m)
        M = crp.modules(precision=crp.MIXED, tables=th, flags=INTERACTION_FLAGS,
                        observer_radius=1.0, **_interaction_kw())
        r = crp.crp_autotune(ctx, g, M, steps_per_trial=200_000)
        assert r["n_tried"] == 27 and r["steps_per_s"] > 0
        assert (M.block_size, M.blocks_per_sm, M.slice, M.queue_order) == \
            (r["block_size"], r["blocks_per_sm"], r["slice"], r["queue_order"])
        assert M.slice % 32 == 0 and M.queue_order in (-1, 0, 1)
        assert crp.crp_context_size(ctx) == m
        crp.crp_propagate(ctx, g, M)
        got = np.sort(crp.crp_collect(ctx, crp.COLLECT_ALL), order="id")
        # whole-run scoring mode
        crp.crp_candidates_clear(ctx)
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), m)
        r2 = crp.crp_autotune(ctx, g, M, steps_per_trial=2**64 - 1)
        assert r2["n_tried"] == 27
        crp.crp_tables_destroy(th)
        crp.crp_grid_destroy(g)
    finally:
        crp.crp_context_destroy(ctx)
    assert got.tobytes() == ref.tobytes()


@pytest.mark.parametrize("precision", [crp.FP64, crp.MIXED])
def test_graph_mode_equals_host_rounds(field_f32_small, tables, precision):
    """The round loop captured as one CUDA graph (device-side loop
    condition) gives the host-driven loop's records, over several rounds
    (short slices, photodisintegration secondaries), for every queue order,
    and replays its cached graph on a second call."""
    n, dx, B = field_f32_small
    inj = _interaction_inputs(n_mixed=300, n_hot=120, seed=31)
    kw = dict(precision=precision, dtype=crp.F32, tables=tables, flags=INTERACTION_FLAGS,
              observer_radius=1.0, slice=64, **_interaction_kw())
    host, st_h, _ = run_gpu(B, n, dx, inj, **kw)
    assert st_h["launches"] > 3 and st_h["n_secondaries"] > 0
    for order in (0, 1, -1):
        g, st_g, status = run_gpu(B, n, dx, inj, use_graph=1, queue_order=order, **kw)
        assert status == crp.OK
        assert g.tobytes() == host.tobytes()
        assert st_g["accepted_steps"] == st_h["accepted_steps"]
        assert st_g["launches"] == st_h["launches"]
    # replay of the cached graph within one context, and a budgeted graph run
    inj = crp.host_injection(inj)
    m = len(inj["E"])
    ctx = crp.crp_context_create(0, 1234, 64 * m)
    try:
        gr = crp.crp_grid_create(ctx, crp.grid_desc(n, dx, dtype=crp.F32, data=B))
        th = crp.crp_tables_from_host(ctx, crp.tables_desc(n=tables.n), tables.beta_pair,
                                      tables.rate_pion, tables.rate_gdr)
        M = crp.modules(precision=precision, tables=th, flags=INTERACTION_FLAGS,
                        observer_radius=1.0, slice=64, use_graph=1, **_interaction_kw())
        outs = []
        for _ in range(2):
            crp.crp_candidates_clear(ctx)
            crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), m)
            crp.crp_propagate(ctx, gr, M)
            outs.append(np.sort(crp.crp_collect(ctx, crp.COLLECT_ALL), order="id"))
        crp.crp_candidates_clear(ctx)
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), m)
        M.step_budget = 20000
        calls = 0
        while True:
            status, _ = crp.crp_propagate(ctx, gr, M, raise_on_error=False)
            calls += 1
            assert status in (crp.OK, crp.E_TIMEOUT) and calls < 10000
            if status == crp.OK:
                break
        budgeted = np.sort(crp.crp_collect(ctx, crp.COLLECT_ALL), order="id")
        crp.crp_tables_destroy(th)
        crp.crp_grid_destroy(gr)
    finally:
        crp.crp_context_destroy(ctx)
    assert outs[0].tobytes() == outs[1].tobytes() == host.tobytes()
    assert calls > 3
    if precision == crp.FP64:
        assert budgeted.tobytes() == host.tobytes()


@pytest.mark.parametrize("galactic", [False, True])
def test_field_sampling_matches_oracle(galactic):
    """The field the kernels see: binary64 sampling equals the oracle's
    trilinear (+ analytic galactic) field bit for bit; binary32 sampling, from
    the cell polynomial records or from the nodes, agrees to binary32
    rounding (1e-5 of the field scale)."""
    W = workloads.GALACTIC_LENS
    n2 = (24, 20, 18)  # ragged, not powers of two: exercises every wrap
    dx = 0.9
    B = oracle.turbulent_field(n2, dx, 2 * dx, 8.0, 3.0, seed=5)
    B32 = B.astype(np.float32).astype(np.float64)
    g = np.random.default_rng(4)
    pts = g.uniform(-25.0, 25.0, size=(4000, 3))
    pts[:8] = [[0, 0, 0], [dx, 0, 0], [23 * dx, 19 * dx, 17 * dx], [-dx, -dx, -dx],
               [24 * dx, 0, 0], [0.5 * dx, 0.5 * dx, 0.5 * dx], [-8.5, 0.0, 0.0], [3.0, 4.0, 1.0]]
    flags = crp.GALACTIC if galactic else 0
    gal = W["disk"] if galactic else None
    P = oracle.make_params(grid_n=n2, spacing=dx, origin=(-10.0, -9.0, -8.0),
                           field_unit_T=oracle.MICROGAUSS_T, length_unit_m=oracle.KPC_M,
                           flags=oracle.GALACTIC if galactic else 0, galactic=gal)
    ctx = crp.crp_context_create(0, 1, 16)
    try:
        for dtype, data, ref_field in ((crp.F64, B, B), (crp.F32, B32, B32)):
            ref = oracle.field_at(P, ref_field, pts)
            scale = np.sqrt(np.mean(np.sum(ref ** 2, axis=1)))
            for cells in ((0, -1) if dtype == crp.F32 else (0,)):
                gr = crp.crp_grid_create(ctx, crp.grid_desc(
                    n2, dx, origin=(-10.0, -9.0, -8.0), dtype=dtype, data=data,
                    data_dtype=crp.F64, cell_records=cells))
                m64 = crp.modules(precision=crp.FP64, flags=flags, galactic=gal,
                                  field_unit_T=crp.MICROGAUSS_T, length_unit_m=crp.KPC_M)
                m32 = crp.modules(precision=crp.MIXED, flags=flags, galactic=gal,
                                  field_unit_T=crp.MICROGAUSS_T, length_unit_m=crp.KPC_M)
                got64 = crp.crp_grid_sample(gr, m64, pts)
                got32 = crp.crp_grid_sample(gr, m32, pts)
                crp.crp_grid_destroy(gr)
                assert np.array_equal(got64, ref), (dtype, cells)
                err = np.max(np.abs(got32 - ref))
                assert err < 1e-5 * scale, (dtype, cells, err / scale)
    finally:
        crp.crp_context_destroy(ctx)




def test_histogram_device_matches_host():
    """crp_histogram_energy_device counts into a device array what
    crp_histogram_energy returns on the host; accumulate adds; an empty pool
    leaves the array cleared."""
    import torch
    n = 5000
    inj = crp.host_injection(workloads.plain_small(n=n, seed=23))
    inj["E"][:] = 10 ** np.random.default_rng(3).uniform(17.5, 21.5, n)
    ctx = crp.crp_context_create(0, 5, n)
    try:
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), n)
        ref = crp.crp_histogram_energy(ctx, crp.COLLECT_ALL, 1e18, 1e21, 60)
        dev = torch.full((60,), 99, dtype=torch.int64, device="cuda")
        crp.crp_histogram_energy_device(ctx, crp.COLLECT_ALL, 1e18, 1e21, 60, dev)
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy(), ref.astype(np.int64)) and 0 < ref.sum() < n
        crp.crp_histogram_energy_device(ctx, crp.COLLECT_ALL, 1e18, 1e21, 60, dev, accumulate=True)
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy(), 2 * ref.astype(np.int64))
        crp.crp_candidates_clear(ctx)
        crp.crp_histogram_energy_device(ctx, crp.COLLECT_ALL, 1e18, 1e21, 60, dev)
        torch.cuda.synchronize()
        assert not dev.cpu().numpy().any()
    finally:
        crp.crp_context_destroy(ctx)
