"""Decay of unstable nuclei (Sect. 2: nuclear decay among the interactions)
on the GPU against the oracle, with the synthetic nuclide table of the
workloads: the binary64 path reproduces the oracle's histories bit for bit
(chains of photodisintegration, pion production and decays, secondaries and
lineage ids, positions, energies); the mixed path reproduces the chains
wherever the stopping condition agrees, and the spectra by distribution."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402
from gpu_util import EXACT_FIELDS, rel_err  # noqa: E402
from paper_1307_2643_gb300 import crp  # noqa: E402

H0_OVER_C = 67.3e3 / 299792458.0
FLAGS = crp.PAIR | crp.ADIABATIC | crp.PION | crp.PHOTODIS | crp.DECAY | crp.EMIN
OFLAGS = (oracle.PAIR | oracle.ADIABATIC | oracle.PION | oracle.PHOTODIS | oracle.DECAY |
          oracle.EMIN)
E_MIN = 1e18


@pytest.fixture(scope="module")
def setup():
    from paper_1307_2643_gb300.build import build
    build()
    oracle.build()
    n, dx = (32, 32, 32), 0.25
    field = oracle.turbulent_field(n, dx, 0.5, 4.0, 0.3, seed=41).astype(np.float32)
    tabs = oracle.tables_build(n=1000)
    table = workloads.synthetic_decay_table()
    g = np.random.default_rng(19)
    m = 3000
    # iron and nitrogen (photodisintegration makes unstable isotopes), and
    # short-lived nuclides injected directly (decays from the start)
    species = np.array([(56, 26), (14, 7), (56, 28), (45, 26), (13, 5), (50, 26), (4, 2)])
    k = g.integers(0, len(species), m)
    A, Z = species[k, 0].astype(np.int32), species[k, 1].astype(np.int32)
    E = 10 ** g.uniform(19.5, 20.8, m) * A / 56
    u = g.normal(size=(m, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    inj = crp.host_injection(dict(id=np.arange(m, dtype=np.uint64) * 3 + 11,
                                  x=g.uniform(-4, 4, m), y=g.uniform(-4, 4, m),
                                  z=g.uniform(-4, 4, m), ux=u[:, 0], uy=u[:, 1], uz=u[:, 2],
                                  E=E, A=A, Z=Z, s_max=np.full(m, 80.0)))
    return n, dx, field, tabs, table, inj


def _gpu(setup, precision, table=True, flags=FLAGS):
    n, dx, field, tabs, table_d, inj = setup
    m = len(inj["E"])
    ctx = crp.crp_context_create(0, 606, 64 * m)
    try:
        g = crp.crp_grid_create(ctx, crp.grid_desc(n, dx, dtype=crp.F32, data=field,
                                                   data_dtype=crp.F32))
        th = crp.crp_tables_from_host(ctx, crp.tables_desc(n=1000), tabs.beta_pair,
                                      tabs.rate_pion, tabs.rate_gdr)
        if table:
            crp.crp_tables_set_decay(th, table_d)
        mods = crp.modules(precision=precision, flags=flags, tol=1e-4, h_min=1e-3, h_max=0.5,
                           beta_ad=H0_OVER_C, e_min=E_MIN, tables=th)
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), m)
        status, st = crp.crp_propagate(ctx, g, mods)
        assert status == crp.OK
        rec = np.sort(crp.crp_collect(ctx, crp.COLLECT_ALL), order="id")
        crp.crp_tables_destroy(th)
        crp.crp_grid_destroy(g)
    finally:
        crp.crp_context_destroy(ctx)
    return rec, st


@pytest.fixture(scope="module")
def ref(setup):
    n, dx, field, tabs, table, inj = setup
    P = oracle.make_params(grid_n=n, spacing=dx, tol=1e-4, h_min=1e-3, h_max=0.5, flags=OFLAGS,
                           e_min=E_MIN, beta_ad=H0_OVER_C, seed=606, tables=tabs,
                           decay_table=table)
    return oracle.propagate(P, field.astype(np.float64), inj, tables=tabs)


def test_fp64_decay_chains_bit_exact(setup, ref):
    rec, st = _gpu(setup, crp.FP64)
    assert len(rec) == len(ref)
    for f in EXACT_FIELDS + ("n_acc", "n_rej"):
        assert np.array_equal(rec[f], ref[f]), (f, np.nonzero(rec[f] != ref[f])[0][:10])
    for f in ("x", "u", "E", "s", "E0"):
        assert np.max(rel_err(rec[f], ref[f])) < 1e-9, f
        assert np.array_equal(rec[f], ref[f]), f   # measured: bit for bit
    # the histories exercise decays of primaries (species changed without
    # photodisintegration), nucleon emission by decay (secondaries of
    # primaries with n_pd = 0) and photodisintegration
    prim = ref[ref["generation"] == 0]
    decayed = (prim["n_pd"] == 0) & ((prim["A"] != prim["A0"]) | (prim["Z"] != prim["Z0"]))
    assert decayed.sum() > 200
    kids_of = set(ref["parent_id"][ref["generation"] == 1].tolist())
    emitted = [int(i) for i in prim["id"][prim["n_pd"] == 0] if int(i) in kids_of]
    assert len(emitted) > 20
    assert prim["n_pd"].sum() > 100
    assert st.accepted_steps == int(ref["n_acc"].sum())


def test_mixed_decay_chains_and_spectra(setup, ref):
    """The mixed path: the same chains wherever the stopping condition
    agrees (losses, rates, lifetimes and channel draws do not depend on
    position), the same number of secondaries, and the same spectra."""
    from scipy.stats import ks_2samp
    rec, _ = _gpu(setup, crp.MIXED)
    assert abs(len(rec) - len(ref)) <= 0.01 * len(ref)
    pg, pr = rec[rec["generation"] == 0], ref[ref["generation"] == 0]
    assert np.array_equal(pg["id"], pr["id"])
    same = pg["status"] == pr["status"]
    assert same.mean() > 0.97
    for f in ("A", "Z", "n_pd", "n_pion"):
        assert np.mean(pg[f][same] == pr[f][same]) > 0.98, f
    e = rel_err(pg["E"][same], pr["E"][same], floor=0.0)
    assert np.median(e) < 1e-5
    assert ks_2samp(np.log(rec["E"]), np.log(ref["E"])).pvalue > 0.01
    for f in ("A", "Z"):
        a = np.bincount(rec[f], minlength=60)
        b = np.bincount(ref[f], minlength=60)
        assert np.abs(a - b).sum() <= 0.02 * len(ref), f


def test_without_table_only_neutrons_decay(setup):
    """No nuclide table: the binary64 kernel without the third free path,
    and no nucleus decays; the decay module's uniform is still drawn for
    every species."""
    rec, _ = _gpu(setup, crp.FP64, table=False)
    n, dx, field, tabs, table, inj = setup
    P = oracle.make_params(grid_n=n, spacing=dx, tol=1e-4, h_min=1e-3, h_max=0.5, flags=OFLAGS,
                           e_min=E_MIN, beta_ad=H0_OVER_C, seed=606, tables=tabs)
    ref0 = oracle.propagate(P, field.astype(np.float64), inj, tables=tabs)
    assert len(rec) == len(ref0)
    for f in EXACT_FIELDS + ("n_acc", "x", "u", "E", "s"):
        assert np.array_equal(rec[f], ref0[f]), f
    prim = rec[rec["generation"] == 0]
    assert np.all((prim["n_pd"] > 0) | ((prim["A"] == prim["A0"]) & (prim["Z"] == prim["Z0"])))


def test_decay_table_arguments():
    ctx = crp.crp_context_create(0, 1, 16)
    try:
        T = oracle.tables_build(n=50)
        th = crp.crp_tables_from_host(ctx, crp.tables_desc(n=50), T.beta_pair, T.rate_pion,
                                      T.rate_gdr)
        ok = dict(A=[20], Z=[10], tau_s=[5.0], branching=[[0.25, 0.25, 0.25, 0.25]])
        crp.crp_tables_set_decay(th, ok)
        bad = [dict(ok, A=[1], Z=[0]), dict(ok, A=[65], Z=[30]), dict(ok, Z=[0]),
               dict(ok, Z=[20]), dict(ok, tau_s=[0.0]), dict(ok, tau_s=[np.nan]),
               dict(ok, branching=[[0.5, 0.5, 0.5, 0.0]]),
               dict(ok, branching=[[1.0, -0.5, 0.5, 0.0]]),
               dict(A=[20, 20], Z=[10, 10], tau_s=[1.0, 2.0], branching=[[1, 0, 0, 0]] * 2),
               # beta+ of (3, 1) would leave (3, 0)
               dict(A=[3], Z=[1], tau_s=[1.0], branching=[[0, 1, 0, 0]])]
        for b in bad:
            with pytest.raises(crp.CrpError) as e:
                crp.crp_tables_set_decay(th, b)
            assert e.value.status == crp.E_INVALID, b
        crp.crp_tables_set_decay(th, None)
        # 1D mode: neutrons only
        crp.crp_tables_set_decay(th, ok)
        with pytest.raises(crp.CrpError):
            crp.crp_propagate_1d(ctx, crp.cosmology(), crp.modules(flags=crp.DECAY, tables=th))
        crp.crp_tables_destroy(th)
    finally:
        crp.crp_context_destroy(ctx)
