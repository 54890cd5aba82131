"""The analytic multi-arm galactic field on the GPU against the oracle:
binary64 sampling and FP64 back-tracking agree bit for bit; binary32 sampling
agrees to binary32 rounding except within rounding of an arm edge; the mixed
back-tracking agrees with the FP64 one per candidate at high rigidity and in
distribution over the whole rigidity range."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402
from paper_1307_2643_gb300 import crp  # noqa: E402

W = workloads.GALACTIC_MULTIARM
GMF = workloads.multiarm_gmf_params()
N0, DX0, ORG0 = (4, 4, 4), 20.0, (-40.0, -40.0, -40.0)  # all-zero grid under the analytic field


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1307_2643_gb300.build import build
    build()
    oracle.build()


def _mods(precision, flags=crp.GMF | crp.BORDER, **kw):
    return crp.modules(precision=precision, flags=flags, tol=W["tol"], h_min=W["h_min"],
                       h_max=W["h_max"], field_unit_T=crp.MICROGAUSS_T, length_unit_m=crp.KPC_M,
                       border_radius=W["border_r"], gmf=GMF, max_steps=2_000_000, **kw)


def _oracle_params(flags):
    return oracle.make_params(grid_n=N0, spacing=DX0, origin=ORG0, tol=W["tol"], h_min=W["h_min"],
                              h_max=W["h_max"], field_unit_T=oracle.MICROGAUSS_T,
                              length_unit_m=oracle.KPC_M, flags=flags, border_r=W["border_r"],
                              gmf=oracle.make_gmf(**GMF), seed=7, max_steps=2_000_000)


def _zero_grid(ctx, dtype=crp.F64):
    return crp.crp_grid_create(ctx, crp.grid_desc(N0, DX0, origin=ORG0, dtype=dtype,
                                                  data=np.zeros(N0 + (3,)), data_dtype=crp.F64))


def _sample_points():
    g = np.random.default_rng(11)
    n = 100_000
    r = g.uniform(0.0, 22.0, n)
    phi = g.uniform(-np.pi, np.pi, n)
    pts = np.stack([r * np.cos(phi), r * np.sin(phi), g.uniform(-8.0, 8.0, n)], axis=1)
    tan_p = np.tan(GMF["pitch_rad"])
    edges = [[-rx, 0.0, 0.0] for rx in GMF["arm_rx"]]  # arm boundaries on the phi = pi ray
    special = [[0, 0, 0], [0, 0, 3.0], [0, 0, -3.0], [-8.5, 0, 0], [-8.5, 0, 1e-12],
               [-8.5, 0, -1e-12], [-8.5, -0.0, 0.0], [5.0, 0, 0], [0, 5.0, 0], [0, -5.0, 0],
               [3.0, 0, 0], [20.0, 0, 0], [1.0, 0, 0], [0, 0, 1.0], [12.0, 7.0, 0.0],
               [-GMF["arm_rx"][0] * np.exp(2 * np.pi * tan_p) * 0.999, 0.0, 0.0],
               [GMF["x_rc"] + 2.0 / np.tan(GMF["x_theta_rad"]), 0.0, 2.0]]  # on r_p = x_rc
    pts[: len(edges) + len(special)] = edges + special
    return pts


def test_gmf_sampling_matches_oracle():
    pts = _sample_points()
    ref = oracle.field_at(_oracle_params(oracle.GMF), np.zeros(N0 + (3,)), pts)
    ctx = crp.crp_context_create(0, 1, 16)
    try:
        g64 = _zero_grid(ctx, crp.F64)
        got64 = crp.crp_grid_sample(g64, _mods(crp.FP64, flags=crp.GMF), pts)
        g32 = _zero_grid(ctx, crp.F32)
        got32 = crp.crp_grid_sample(g32, _mods(crp.MIXED, flags=crp.GMF), pts)
    finally:
        crp.crp_context_destroy(ctx)
    assert np.abs(ref).max() > 1.0 and (np.abs(ref).sum(axis=1) == 0).sum() > 1000  # cuts hit
    assert np.array_equal(got64, ref)
    scale = np.abs(ref).max()
    err = np.linalg.norm(got32 - ref, axis=1)
    # binary32 arguments move the spiral phase by ~1e-6; a point that close to
    # an arm edge takes the neighbouring arm's strength
    assert np.mean(err < 2e-5 * scale) > 0.999, np.mean(err < 2e-5 * scale)
    assert np.median(err) < 1e-6 * scale


def _antiprotons(n, seed):
    dirs, R = workloads.backtrack_directions(n, W["r_lo"], W["r_hi"], seed)
    e = W["earth"]
    return dict(id=np.arange(n, dtype=np.uint64), x=np.full(n, e[0]), y=np.full(n, e[1]),
                z=np.full(n, e[2]), ux=dirs[:, 0], uy=dirs[:, 1], uz=dirs[:, 2], E=R,
                A=np.ones(n, np.int32), Z=np.ones(n, np.int32), q=-np.ones(n, np.int32))


def _gpu_backtrack(inj, precision):
    n = len(inj["E"])
    ctx = crp.crp_context_create(0, 7, n + 16)
    try:
        g = _zero_grid(ctx, crp.F64 if precision == crp.FP64 else crp.F32)
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(crp.host_injection(inj)), n)
        _, st = crp.crp_propagate(ctx, g, _mods(precision))
        rec = crp.crp_collect(ctx, crp.COLLECT_ALL)
    finally:
        crp.crp_context_destroy(ctx)
    return rec[np.argsort(rec["id"], kind="stable")], st


def test_gmf_backtracking_fp64_matches_oracle():
    inj = _antiprotons(384, W["seed"])
    gpu, st = _gpu_backtrack(inj, crp.FP64)
    ref = oracle.propagate(_oracle_params(oracle.GMF | oracle.BORDER), np.zeros(N0 + (3,)), inj)
    assert len(gpu) == len(ref) == 384
    assert np.all(ref["status"] == oracle.AT_BORDER)
    for f in ("x", "u", "E", "s", "n_acc", "n_rej", "status"):
        assert np.array_equal(gpu[f], ref[f]), f
    assert st.accepted_steps == int(ref["n_acc"].sum())


def test_gmf_backtracking_mixed_vs_fp64():
    inj = _antiprotons(20_000, W["seed"] + 1)
    r64, _ = _gpu_backtrack(inj, crp.FP64)
    r32, _ = _gpu_backtrack(inj, crp.MIXED)
    assert np.all(r64["status"] == crp.AT_BORDER) and np.all(r32["status"] == crp.AT_BORDER)
    ang = np.arccos(np.clip(np.sum(r64["u"] * r32["u"], axis=1), -1.0, 1.0))
    R = inj["E"]
    hi = R >= 1e19
    # both are tol-1e-4 integrations of the same field: at rigidities where the
    # map is smooth they agree to the integration error
    assert np.median(ang[hi]) < 1e-3, np.median(ang[hi])
    assert np.mean(ang[hi] < 1e-2) > 0.95
    # over all rigidities, in distribution: coarse border maps agree
    nside = 4
    p64 = oracle.ang2pix_vec(nside, r64["u"])
    p32 = oracle.ang2pix_vec(nside, r32["u"])
    h64 = np.bincount(p64, minlength=12 * nside * nside).astype(float)
    h32 = np.bincount(p32, minlength=12 * nside * nside).astype(float)
    live = (h64 + h32) > 0
    chi2 = np.sum((h64[live] - h32[live]) ** 2 / (h64[live] + h32[live]))
    assert chi2 < 2.0 * live.sum(), (chi2, live.sum())


def test_all_fields_together_fp64_matches_oracle():
    """Random grid (32^3 Kolmogorov, periodic) + analytic disk and halo + the
    multi-arm field, all at once: FP64 back-tracking bit for bit."""
    WL = workloads.GALACTIC_LENS
    n3 = (32, 32, 32)
    dx, lmin, org = workloads.galactic_grid_geometry(32, WL["box"])
    field = oracle.turbulent_field(n3, dx, lmin, 4.0 * lmin, 1.0, seed=WL["seed"])
    inj = _antiprotons(256, W["seed"] + 9)
    ctx = crp.crp_context_create(0, 7, 256 + 16)
    try:
        g = crp.crp_grid_create(ctx, crp.grid_desc(n3, dx, origin=org, dtype=crp.F64, data=field))
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(crp.host_injection(inj)), 256)
        _, st = crp.crp_propagate(ctx, g, _mods(crp.FP64, flags=crp.GMF | crp.GALACTIC | crp.BORDER,
                                                galactic=WL["disk"]))
        gpu = crp.crp_collect(ctx, crp.COLLECT_ALL)
        gpu = gpu[np.argsort(gpu["id"], kind="stable")]
    finally:
        crp.crp_context_destroy(ctx)
    P = oracle.make_params(grid_n=n3, spacing=dx, origin=org, tol=W["tol"], h_min=W["h_min"],
                           h_max=W["h_max"], field_unit_T=oracle.MICROGAUSS_T,
                           length_unit_m=oracle.KPC_M,
                           flags=oracle.GMF | oracle.GALACTIC | oracle.BORDER,
                           border_r=W["border_r"], galactic=WL["disk"],
                           gmf=oracle.make_gmf(**GMF), seed=7, max_steps=2_000_000)
    ref = oracle.propagate(P, field, inj)
    assert np.all(ref["status"] == oracle.AT_BORDER)
    for f in ("x", "u", "E", "s", "n_acc", "n_rej", "status"):
        assert np.array_equal(gpu[f], ref[f]), f
    assert st.accepted_steps == int(ref["n_acc"].sum())



def test_invalid_gmf_and_histogram_arguments_are_rejected():
    """Argument errors come back as CRP_E_INVALID before any kernel runs:
    CRP_GMF without parameters, arm radii out of order or beyond one spiral
    turn, a zero transition width, an X field without its geometry; and
    device-histogram calls with bad bins or ranges."""
    import torch
    ctx = crp.crp_context_create(0, 1, 64)
    try:
        g = _zero_grid(ctx)
        inj = crp.host_injection(_antiprotons(8, 1))
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), 8)
        m = crp.modules(precision=crp.FP64, flags=crp.GMF | crp.BORDER, border_radius=20.0,
                        field_unit_T=crp.MICROGAUSS_T, length_unit_m=crp.KPC_M)
        with pytest.raises(crp.CrpError, match="gmf"):
            crp.crp_propagate(ctx, g, m)
        bad = [dict(arm_rx=tuple(reversed(GMF["arm_rx"]))),
               dict(arm_rx=GMF["arm_rx"][:7] + (GMF["arm_rx"][0] * 10.0,)),
               dict(w_disk=0.0),
               dict(x_rc=0.0)]
        for over in bad:
            p = dict(GMF)
            p.update(over)
            m = crp.modules(precision=crp.FP64, flags=crp.GMF | crp.BORDER, border_radius=20.0,
                            field_unit_T=crp.MICROGAUSS_T, length_unit_m=crp.KPC_M, gmf=p)
            with pytest.raises(crp.CrpError) as e:
                crp.crp_propagate(ctx, g, m)
            assert e.value.status == crp.E_INVALID, over
        # nothing ran: the candidates are still active and at Earth
        rec = crp.crp_collect(ctx, crp.COLLECT_ALL)
        assert np.all(rec["status"] == crp.ACTIVE) and np.all(rec["s"] == 0.0)
        h = torch.zeros(8, dtype=torch.int64, device="cuda")
        for args in ((crp.COLLECT_ALL, 1e18, 1e21, 0), (crp.COLLECT_ALL, 1e21, 1e18, 8),
                     (crp.COLLECT_ALL, 0.0, 1e18, 8), (99, 1e18, 1e21, 8)):
            with pytest.raises(crp.CrpError):
                crp.crp_histogram_energy_device(ctx, *args, h)
    finally:
        crp.crp_context_destroy(ctx)
