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
        # the status filter: every injected candidate is active, so DETECTED
        # selects none (pixels stay "not applied") and ACTIVE all of them
        crp.crp_lens_apply(ctx, lens, crp.COLLECT_DETECTED)
        rec_none = np.sort(crp.crp_collect(ctx, crp.COLLECT_ALL), order="id")
        crp.crp_lens_apply(ctx, lens, crp.COLLECT_ACTIVE)
        rec_active = np.sort(crp.crp_collect(ctx, crp.COLLECT_ALL), order="id")
        crp.crp_lens_apply(ctx, lens, crp.COLLECT_ALL)
        rec = np.sort(crp.crp_collect(ctx, crp.COLLECT_ALL), order="id")
        hist_earth = crp.crp_histogram_healpix(ctx, crp.COLLECT_ALL, NSIDE, 1)
        hist_sky = crp.crp_histogram_healpix(ctx, crp.COLLECT_ALL, NSIDE, 0)
        crp.crp_lens_destroy(lens)
        crp.crp_grid_destroy(gr)
    finally:
        crp.crp_context_destroy(ctx)
    want = olens.apply(ref_lens, NSIDE, W["r_lo"], W["r_hi"], NBINS, seed, inj["id"], u, Ev, Z)
    assert np.all(rec_none["lens_pixel"] == olens.NOT_APPLIED)
    assert np.array_equal(rec_active["lens_pixel"], want)
    assert np.array_equal(rec["lens_pixel"], want)
    observed = want < 12 * NSIDE * NSIDE
    assert 0.2 < observed.mean() < 0.98
    assert np.all(want[Z == 0] == olens.NOT_APPLIED)
    npix = 12 * NSIDE * NSIDE
    assert np.array_equal(hist_earth, np.bincount(want[observed], minlength=npix))
    assert np.array_equal(hist_sky, np.bincount(oracle.ang2pix_vec(NSIDE, -u), minlength=npix))


@pytest.fixture(scope="module")
def built():
    from paper_1307_2643_gb300.build import build
    build()
    oracle.build()


def _unit(g, m):
    u = g.normal(size=(m, 3))
    return u / np.linalg.norm(u, axis=1, keepdims=True)


def _boundary_directions(nside):
    """Pixel centres, the cap / belt border z = +-2/3, the poles and the
    azimuths 0, pi/2, pi, 3 pi/2 (where the binary32 decisions fall back)."""
    out = []
    if 12 * nside * nside <= 50_000:
        for p in range(12 * nside * nside):
            z, ph = oracle.pix2ang(nside, p)
            s = np.sqrt(1.0 - z * z)
            out.append([s * np.cos(ph), s * np.sin(ph), z])
    for z in (2 / 3, -2 / 3, np.nextafter(2 / 3, 1), np.nextafter(2 / 3, 0), 1.0, -1.0, 0.0,
              1 - 1e-12, -1 + 1e-12, 1e-300, -1e-300):
        for ph in (0.0, 1e-12, -1e-12, np.pi / 2, np.pi, -np.pi, 1.5 * np.pi, np.nextafter(np.pi, 0)):
            s = np.sqrt(max(0.0, 1 - z * z))
            out.append([s * np.cos(ph), s * np.sin(ph), z])
    return np.array(out)


@pytest.mark.parametrize("nside", [1, 4, 64, 1024])
def test_healpix_pixels_match_oracle(built, nside):
    """Arrival-direction pixels at several resolutions against the oracle's
    binary64 HEALPix, on 2^21 random and boundary directions (the histogram
    of -u over the pool)."""
    g = np.random.default_rng(nside)
    b = _boundary_directions(nside)
    u = np.concatenate([_unit(g, 1 << 21), -b])
    m = len(u)
    inj = dict(x=np.zeros(m), y=np.zeros(m), z=np.zeros(m), ux=u[:, 0].copy(), uy=u[:, 1].copy(),
               uz=u[:, 2].copy(), E=np.full(m, 1e19), A=np.ones(m, np.int32),
               Z=np.ones(m, np.int32))
    ctx = crp.crp_context_create(0, 1, m)
    try:
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(crp.host_injection(inj)), m)
        got = crp.crp_histogram_healpix(ctx, crp.COLLECT_ALL, nside, 0)
    finally:
        crp.crp_context_destroy(ctx)
    want = np.bincount(oracle.ang2pix_vec(nside, -u), minlength=12 * nside * nside)
    assert np.array_equal(got, want)


def test_lens_apply_at_scale_matches_oracle(built):
    """The lens application at the galactic workload's resolution (nside 64,
    100 rigidity bins) on 2^20 candidates: random directions, protons to
    iron, rigidities across and beyond the binned range and on the bin edges;
    every Earth pixel equals the oracle's application of the same lens."""
    nside, nb = W["nside"], W["n_bins"]
    npix = 12 * nside * nside
    dirs, E, bins = workloads.lens_samples(nb, 2 * npix // 8, W["r_lo"], W["r_hi"], W["seed"])
    g = np.random.default_rng(17)
    m = 1 << 20
    u = _unit(g, m)
    Z = g.choice(np.array([0, 1, 1, 2, 7, 26], np.int32), m)
    R = np.exp(g.uniform(np.log(W["r_lo"]) - 1.0, np.log(W["r_hi"]) + 1.0, m))
    edges = np.exp(np.linspace(np.log(W["r_lo"]), np.log(W["r_hi"]), nb + 1))
    k = 4 * len(edges)
    R[:k] = np.repeat(edges, 4) * np.tile([1.0, 1 - 1e-15, 1 + 1e-15, 1 + 1e-7], len(edges))
    Ev = R * np.maximum(Z, 1)
    A = np.select([Z == 26, Z == 7, Z == 2], [56, 14, 4], 1).astype(np.int32)
    ids = np.arange(7, 7 + m, dtype=np.uint64)
    seed = 99
    ctx = crp.crp_context_create(0, seed, max(m, len(E)) + 16)
    try:
        zn = (4, 4, 4)
        gr = crp.crp_grid_create(ctx, crp.grid_desc(zn, 20.0, origin=(-40.0, -40.0, -40.0),
                                                    dtype=crp.F32, data=np.zeros(zn + (3,))))
        mods = crp.modules(precision=crp.MIXED, flags=crp.BORDER, tol=W["tol"], h_min=W["h_min"],
                           h_max=W["h_max"], field_unit_T=crp.MICROGAUSS_T,
                           length_unit_m=crp.KPC_M, border_radius=W["border_r"],
                           max_steps=2_000_000)
        lens, _ = crp.crp_lens_build(ctx, gr, mods, nside, nb, W["r_lo"], W["r_hi"], W["earth"],
                                     dirs, E, bins)
        L = crp.crp_lens_copy_out(lens, nb * npix, nb)
        crp.crp_candidates_clear(ctx)
        inj = dict(id=ids, x=np.zeros(m), y=np.zeros(m), z=np.zeros(m), ux=u[:, 0].copy(),
                   uy=u[:, 1].copy(), uz=u[:, 2].copy(), E=Ev, A=A, Z=Z)
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(crp.host_injection(inj)), m)
        # the status filter: every injected candidate is active, so DETECTED
        # selects none (pixels stay "not applied") and ACTIVE all of them
        crp.crp_lens_apply(ctx, lens, crp.COLLECT_DETECTED)
        rec_none = np.sort(crp.crp_collect(ctx, crp.COLLECT_ALL), order="id")
        crp.crp_lens_apply(ctx, lens, crp.COLLECT_ACTIVE)
        rec_active = np.sort(crp.crp_collect(ctx, crp.COLLECT_ALL), order="id")
        crp.crp_lens_apply(ctx, lens, crp.COLLECT_ALL)
        rec = np.sort(crp.crp_collect(ctx, crp.COLLECT_ALL), order="id")
        crp.crp_lens_destroy(lens)
    finally:
        crp.crp_context_destroy(ctx)
    want = olens.apply(L, nside, W["r_lo"], W["r_hi"], nb, seed, ids, u, Ev, Z)
    assert np.array_equal(rec["lens_pixel"], want)
    seen = want < npix
    # a quarter of a sample per column on average: most columns are empty
    assert 0.01 < seen.mean() < 0.9 and np.all(want[Z == 0] == olens.NOT_APPLIED)
