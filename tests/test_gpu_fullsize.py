"""Full-size parity: the 10^6-candidate mixed-composition workload (256^3
float32 field, losses, pion production, observer) in the launch
configuration the benchmark times, checked on sampled candidates that the
oracle recomputes one by one (histories are keyed by candidate id, so a
sample's histories are those of the full run)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402
from gpu_util import EXACT_FIELDS, rel_err  # noqa: E402
from paper_1307_2643_gb300 import crp  # noqa: E402

H0_OVER_C = 67.3e3 / 299792458.0
FLAGS = crp.PAIR | crp.ADIABATIC | crp.PION | crp.EMIN | crp.OBSERVER


@pytest.fixture(scope="module")
def full_run():
    from paper_1307_2643_gb300.build import build
    build()
    w = workloads.MIXED_INTERACTIONS
    field = oracle.turbulent_field(w["grid_n"], w["spacing"], w["lmin"], w["lmax"], w["brms"],
                                   seed=w["seed"]).astype(np.float32)
    inj = crp.host_injection(workloads.mixed_interactions())
    n = len(inj["E"])
    tabs = oracle.tables_build(n=1000)
    out = {}
    ctx = crp.crp_context_create(0, w["seed"], n + 1024)
    try:
        g = crp.crp_grid_create(ctx, crp.grid_desc(w["grid_n"], w["spacing"], dtype=crp.F32,
                                                   data=field, data_dtype=crp.F32))
        th = crp.crp_tables_from_host(ctx, crp.tables_desc(n=1000), tabs.beta_pair,
                                      tabs.rate_pion, tabs.rate_gdr)
        for name, prec in (("fp64", crp.FP64), ("mixed", crp.MIXED)):
            crp.crp_candidates_clear(ctx)
            crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), n)
            m = crp.modules(precision=prec, flags=FLAGS, tol=w["tol"], h_min=w["h_min"],
                            h_max=w["h_max"], beta_ad=H0_OVER_C, e_min=w["e_min"], tables=th,
                            observer_radius=w["observer_r"])
            status, st = crp.crp_propagate(ctx, g, m)
            assert status == crp.OK
            out[name] = (np.sort(crp.crp_collect(ctx, crp.COLLECT_ALL), order="id"), st)
        crp.crp_tables_destroy(th)
        crp.crp_grid_destroy(g)
    finally:
        crp.crp_context_destroy(ctx)
    return w, field.astype(np.float64), inj, tabs, out


def test_fullsize_fp64_sampled_against_oracle(full_run):
    w, field, inj, tabs, out = full_run
    rec, st = out["fp64"]
    assert len(rec) == len(inj["E"])
    idx = np.sort(np.random.default_rng(11).choice(len(rec), 48, replace=False))
    sub = workloads.subsample(inj, idx)
    P = oracle.make_params(grid_n=w["grid_n"], spacing=w["spacing"], tol=w["tol"],
                           h_min=w["h_min"], h_max=w["h_max"],
                           flags=oracle.PAIR | oracle.ADIABATIC | oracle.PION | oracle.EMIN |
                           oracle.OBSERVER, e_min=w["e_min"], beta_ad=H0_OVER_C, seed=w["seed"],
                           tables=tabs, obs_r=w["observer_r"])
    ref = oracle.propagate(P, field, sub, tables=tabs)
    got = rec[idx]
    for f in EXACT_FIELDS:
        assert np.array_equal(got[f], ref[f]), f
    assert np.array_equal(got["n_acc"], ref["n_acc"])
    for f in ("x", "u", "E", "s"):
        assert np.max(rel_err(got[f], ref[f])) < 1e-9, f
    assert st.accepted_steps == int(rec["n_acc"].sum())


def test_fullsize_mixed_against_fp64(full_run):
    """The whole batch: break statuses, interaction counts and energies of the
    mixed path against the FP64 path (energy losses and interactions do not
    depend on position, so they agree per candidate wherever the stopping
    condition does)."""
    _, _, inj, _, out = full_run
    r64, _ = out["fp64"]
    rmx, _ = out["mixed"]
    assert np.array_equal(r64["id"], rmx["id"])
    same = r64["status"] == rmx["status"]
    assert same.mean() > 0.98, same.mean()
    assert np.mean(r64["n_pion"][same] == rmx["n_pion"][same]) > 0.98
    e = rel_err(rmx["E"][same], r64["E"][same], floor=0.0)
    assert np.median(e) < 1e-6 and np.percentile(e, 99) < 1e-4, (np.median(e), np.percentile(e, 99))
    # detection counts agree statistically
    d64, dmx = (r64["status"] == crp.DETECTED).sum(), (rmx["status"] == crp.DETECTED).sum()
    assert abs(int(d64) - int(dmx)) <= 5 * np.sqrt(max(d64, 1)) + 5


def test_fullsize_mixed_spectra_and_arrival_maps(full_run):
    """Spectra and arrival maps of the mixed path against the FP64 path at
    full size: two-sample KS on log E (all records and detected ones) and on
    the arrival directions of the detected candidates."""
    from scipy.stats import ks_2samp
    _, _, _, _, out = full_run
    r64, _ = out["fp64"]
    rmx, _ = out["mixed"]
    assert ks_2samp(np.log(rmx["E"]), np.log(r64["E"])).pvalue > 0.01
    d64 = r64[r64["status"] == crp.DETECTED]
    dmx = rmx[rmx["status"] == crp.DETECTED]
    assert len(d64) > 100 and len(dmx) > 100
    assert ks_2samp(np.log(dmx["E"]), np.log(d64["E"])).pvalue > 0.01
    for comp in (lambda u: -u[:, 2], lambda u: np.arctan2(-u[:, 1], -u[:, 0])):
        assert ks_2samp(comp(dmx["u"]), comp(d64["u"])).pvalue > 0.01


def test_plain_1e4_protons_64cube_fp64_bit_exact():
    """The plain small workload at its stated size: all 10^4 protons (E^-2 on
    10^19-10^20 eV, isotropic from the origin) through the 64^3 binary64
    Kolmogorov grid (250 kpc spacing, lmin 0.5, lmax 8 Mpc, B_rms 1 nG),
    tol 1e-4, h in [10 kpc, 1 Mpc], stopped at 50 Mpc, binary64 on both
    sides: every record field equals the oracle's bit for bit."""
    from paper_1307_2643_gb300.build import build
    build()
    oracle.build()
    w = workloads.PLAIN_SMALL
    field = oracle.turbulent_field(w["grid_n"], w["spacing"], w["lmin"], w["lmax"], w["brms"],
                                   seed=w["seed"])
    inj = crp.host_injection(workloads.plain_small())
    n = len(inj["E"])
    assert n == 10_000
    ctx = crp.crp_context_create(0, w["seed"], n + 64)
    try:
        g = crp.crp_grid_create(ctx, crp.grid_desc(w["grid_n"], w["spacing"], dtype=crp.F64,
                                                   data=field))
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), n)
        m = crp.modules(precision=crp.FP64, tol=w["tol"], h_min=w["h_min"], h_max=w["h_max"])
        status, st = crp.crp_propagate(ctx, g, m)
        assert status == crp.OK
        rec = np.sort(crp.crp_collect(ctx, crp.COLLECT_ALL), order="id")
        crp.crp_grid_destroy(g)
    finally:
        crp.crp_context_destroy(ctx)
    P = oracle.make_params(grid_n=w["grid_n"], spacing=w["spacing"], tol=w["tol"],
                           h_min=w["h_min"], h_max=w["h_max"], seed=w["seed"])
    ref = oracle.propagate(P, field, inj)
    assert len(rec) == len(ref) == n
    for f in EXACT_FIELDS + ("n_acc", "n_rej"):
        assert np.array_equal(rec[f], ref[f]), f
    for f in ("x", "u", "E", "s", "x0", "u0", "E0"):
        assert np.max(rel_err(rec[f], ref[f])) < 1e-9, f
        assert np.array_equal(rec[f], ref[f]), f   # measured: bit for bit
    assert np.all(rec["status"] == crp.MAX_LENGTH)
    assert st.accepted_steps == int(ref["n_acc"].sum())
    assert st.rejected_trials == int(ref["n_rej"].sum())
