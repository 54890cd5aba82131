"""Galactic lens on the GPU against the oracle: the lens built by FP64
back-tracking through the analytic disk + halo field plus a random grid
(integer structure exact), lens application (exact, Philox-driven), the
zero-field identity, and HEALPix arrival maps."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import oracle.lens as olens  # noqa: E402
import workloads  # noqa: E402
from paper_1307_2643_gb300 import crp  # noqa: E402

W = workloads.GALACTIC_LENS
NSIDE, NBINS, PER_BIN = 4, 3, 4 * 192


@pytest.fixture(scope="module")
def setup():
    from paper_1307_2643_gb300.build import build
    build()
    oracle.build()
    n = (32, 32, 32)
    dx, lmin, org = workloads.galactic_grid_geometry(32, W["box"])
    field = oracle.turbulent_field(n, dx, lmin, 4.0 * lmin, W["brms"], seed=W["seed"])
    assert np.sqrt(np.mean(np.sum(field ** 2, axis=-1))) > 0.99 * W["brms"]
    dirs, E, bins = workloads.lens_samples(NBINS, PER_BIN, W["r_lo"], W["r_hi"], seed=W["seed"])
    return n, dx, org, field, dirs, E, bins


def _mods(flags=crp.GALACTIC | crp.BORDER, precision=crp.FP64):
    return crp.modules(precision=precision, flags=flags, tol=W["tol"], h_min=W["h_min"],
                       h_max=W["h_max"], field_unit_T=crp.MICROGAUSS_T, length_unit_m=crp.KPC_M,
                       border_radius=W["border_r"], galactic=W["disk"], max_steps=2_000_000)


def _oracle_params(n, dx, org, flags):
    return oracle.make_params(grid_n=n, spacing=dx, origin=org, tol=W["tol"], h_min=W["h_min"],
                              h_max=W["h_max"], field_unit_T=oracle.MICROGAUSS_T,
                              length_unit_m=oracle.KPC_M, flags=flags, border_r=W["border_r"],
                              galactic=W["disk"], seed=7, max_steps=2_000_000)


def _gpu_lens(n, dx, org, field, dirs, E, bins, mods):
    ctx = crp.crp_context_create(0, 7, 16)
    try:
        g = crp.crp_grid_create(ctx, crp.grid_desc(n, dx, origin=org, dtype=crp.F64, data=field))
        lens, st = crp.crp_lens_build(ctx, g, mods, NSIDE, NBINS, W["r_lo"], W["r_hi"],
                                      W["earth"], dirs, E, bins)
        out = crp.crp_lens_copy_out(lens, NBINS * 12 * NSIDE * NSIDE, NBINS)
        crp.crp_lens_destroy(lens)
        crp.crp_grid_destroy(g)
    finally:
        crp.crp_context_destroy(ctx)
    return out, st


def test_lens_build_matches_oracle(setup):
    n, dx, org, field, dirs, E, bins = setup
    got, st = _gpu_lens(n, dx, org, field, dirs, E, bins, _mods())
    P = _oracle_params(n, dx, org, oracle.GALACTIC | oracle.BORDER)
    inj_E = E
    recs = oracle.propagate(P, field, dict(
        id=np.arange(len(E), dtype=np.uint64), x=np.full(len(E), W["earth"][0]),
        y=np.full(len(E), W["earth"][1]), z=np.full(len(E), W["earth"][2]),
        ux=dirs[:, 0].copy(), uy=dirs[:, 1].copy(), uz=dirs[:, 2].copy(), E=inj_E,
        A=np.ones(len(E), np.int32), Z=np.ones(len(E), np.int32), q=-np.ones(len(E), np.int32)))
    ref = olens.build(NSIDE, NBINS, bins, dirs, recs)
    assert (recs["status"] == oracle.AT_BORDER).mean() > 0.99
    assert st.accepted_steps == int(recs["n_acc"].sum())
    assert np.array_equal(got["col_start"], ref["col_start"])
    assert np.array_equal(got["entries"], ref["entries"])
    assert np.array_equal(got["max_count"], ref["max_count"])
    # the field really deflects: most samples leave through another pixel
    earth_pix = oracle.ang2pix_vec(NSIDE, dirs)
    moved = 0
    for b in range(NBINS):
        for j in range(12 * NSIDE * NSIDE):
            c = b * 12 * NSIDE * NSIDE + j
            col = ref["entries"][ref["col_start"][c]:ref["col_start"][c + 1]]
            moved += int(np.sum(col != j))
    assert moved > 0.5 * len(ref["entries"])


def test_lens_zero_field_is_identity(setup):
    n, dx, org, _, dirs, E, bins = setup
    zero = np.zeros((32, 32, 32, 3))
    got, _ = _gpu_lens(n, dx, org, zero, dirs, E, bins, _mods(flags=crp.BORDER))
    npix = 12 * NSIDE * NSIDE
    for c in range(NBINS * npix):
        col = got["entries"][got["col_start"][c]:got["col_start"][c + 1]]
        assert np.all(col == c % npix)
    assert got["col_start"][-1] == len(E)


def test_lens_apply_matches_oracle(setup):
    n, dx, org, field, dirs, E, bins = setup
    P = _oracle_params(n, dx, org, oracle.GALACTIC | oracle.BORDER)
    recs = oracle.propagate(P, field, dict(
        id=np.arange(len(E), dtype=np.uint64), x=np.full(len(E), W["earth"][0]),
        y=np.full(len(E), W["earth"][1]), z=np.full(len(E), W["earth"][2]),
        ux=dirs[:, 0].copy(), uy=dirs[:, 1].copy(), uz=dirs[:, 2].copy(), E=E,
        A=np.ones(len(E), np.int32), Z=np.ones(len(E), np.int32), q=-np.ones(len(E), np.int32)))
    ref_lens = olens.build(NSIDE, NBINS, bins, dirs, recs)
    # candidates arriving at the Galaxy: random directions, rigidities inside
    # and outside the lens range, a few neutrons
    m = 5000
    g = np.random.default_rng(3)
    u = g.normal(size=(m, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    Z = np.where(g.random(m) < 0.05, 0, np.where(g.random(m) < 0.5, 1, 26)).astype(np.int32)
    A = np.where(Z == 26, 56, 1).astype(np.int32)
    Ev = 10 ** g.uniform(17.5, 20.5, m) * np.maximum(Z, 1)
    inj = dict(id=np.arange(100, 100 + m, dtype=np.uint64), x=np.zeros(m), y=np.zeros(m),
               z=np.zeros(m), ux=u[:, 0].copy(), uy=u[:, 1].copy(), uz=u[:, 2].copy(), E=Ev,
               A=A, Z=Z)
    seed = 4242
    ctx = crp.crp_context_create(0, seed, m)
    try:
        gr = crp.crp_grid_create(ctx, crp.grid_desc(n, dx, origin=org, dtype=crp.F64, data=field))
        lens, _ = crp.crp_lens_build(ctx, gr, _mods(), NSIDE, NBINS, W["r_lo"], W["r_hi"],
                                     W["earth"], dirs, E, bins)
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(crp.host_injection(inj)), m)
        crp.crp_lens_apply(ctx, lens, crp.COLLECT_ALL)
        rec = np.sort(crp.crp_collect(ctx, crp.COLLECT_ALL), order="id")
        hist_earth = crp.crp_histogram_healpix(ctx, crp.COLLECT_ALL, NSIDE, 1)
        hist_sky = crp.crp_histogram_healpix(ctx, crp.COLLECT_ALL, NSIDE, 0)
        crp.crp_lens_destroy(lens)
        crp.crp_grid_destroy(gr)
    finally:
        crp.crp_context_destroy(ctx)
    want = olens.apply(ref_lens, NSIDE, W["r_lo"], W["r_hi"], NBINS, seed, inj["id"], u, Ev, Z)
    assert np.array_equal(rec["lens_pixel"], want)
    observed = want < 12 * NSIDE * NSIDE
    assert 0.2 < observed.mean() < 0.98
    assert np.all(want[Z == 0] == olens.NOT_APPLIED)
    npix = 12 * NSIDE * NSIDE
    assert np.array_equal(hist_earth, np.bincount(want[observed], minlength=npix))
    assert np.array_equal(hist_sky, np.bincount(oracle.ang2pix_vec(NSIDE, -u), minlength=npix))
