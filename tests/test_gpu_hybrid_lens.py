"""The hybrid galactic lens (Sect. 4 lenses map directions at the Galaxy
border to directions at Earth): per rigidity bin, the lens built from the
trained surrogate where the network's validated median angular error is at
most 0.5 deg, the lens built by back-tracking elsewhere (crp_lens_merge).

On the workload's own field (disk + halo + 256^3 random 3 uG component) the
interpolation floor -- the median error of predicting a border direction
from its two neighbours one training-sample spacing away -- exceeds 0.5 deg
even in the top rigidity tenth, so no bin can be claimed and the hybrid
equals the back-tracked lens; on the regular multi-arm field the network is
validated in about half of the bins.
In both, every claimed bin meets 0.5 deg on held-out samples, and the merged
lens and its application equal the source lenses bin by bin."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

import workloads  # noqa: E402
from paper_1307_2643_gb300 import crp  # noqa: E402

NSIDE, NBINS = 16, 100


def _angle(a, b):
    c = np.sum(a * b, axis=1) / (np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1))
    return np.degrees(np.arccos(np.clip(c, -1.0, 1.0)))


def _setup(galaxy):
    wr = workloads.GALACTIC_LENS
    if galaxy == "disk_halo_random":
        w = wr
        dx, lmin, org = workloads.galactic_grid_geometry(wr["grid_n"][0], wr["box"])
        desc = crp.grid_desc(wr["grid_n"], dx, origin=org, dtype=crp.F32,
                             source=crp.GRID_TURBULENT, lmin=lmin, lmax=wr["lmax"],
                             brms=wr["brms"], seed=wr["seed"])
        analytic = dict(flags=crp.GALACTIC | crp.BORDER, galactic=wr["disk"])
    else:
        w = workloads.GALACTIC_MULTIARM
        zn = (4, 4, 4)
        desc = crp.grid_desc(zn, 20.0, origin=(-40.0, -40.0, -40.0), dtype=crp.F32,
                             data=np.zeros(zn + (3,)))
        analytic = dict(flags=crp.GMF | crp.BORDER, gmf=workloads.multiarm_gmf_params())
    return w, desc, analytic


def _modules(w, analytic, precision=crp.MIXED):
    return crp.modules(precision=precision, tol=w["tol"], h_min=w["h_min"], h_max=w["h_max"],
                       field_unit_T=crp.MICROGAUSS_T, length_unit_m=crp.KPC_M,
                       border_radius=w["border_r"], **analytic)


def _backtrack(ctx, grid, mods, w, dirs, R):
    n = len(R)
    e = w["earth"]
    inj = crp.host_injection(dict(x=np.full(n, e[0]), y=np.full(n, e[1]), z=np.full(n, e[2]),
                                  ux=dirs[:, 0], uy=dirs[:, 1], uz=dirs[:, 2], E=R,
                                  A=np.ones(n), Z=np.ones(n), q=-np.ones(n)))
    crp.crp_candidates_clear(ctx)
    crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), n)
    crp.crp_propagate(ctx, grid, mods)
    rec = crp.crp_collect(ctx, crp.COLLECT_ALL)
    rec = rec[np.argsort(rec["id"], kind="stable")]
    assert np.all(rec["status"] == crp.AT_BORDER)
    return rec["u"]


def _lens_bin(R, w):
    t = np.log(R / w["r_lo"]) / np.log(w["r_hi"] / w["r_lo"]) * NBINS
    return np.clip(np.floor(t).astype(np.int64), 0, NBINS - 1)


@pytest.mark.parametrize("galaxy", ["disk_halo_random", "multiarm"])
def test_hybrid_lens(galaxy):
    import torch
    from paper_1307_2643_gb300.build import build
    build()
    w, desc, analytic = _setup(galaxy)
    n_train, n_val, n_test, B = 1 << 22, 1 << 17, 1 << 16, 16384
    n = n_train + n_val + n_test
    dirs, R = workloads.backtrack_directions(n, w["r_lo"], w["r_hi"], w["seed"] + 21)
    ctx = crp.crp_context_create(0, w["seed"], n + 1024)
    try:
        grid = crp.crp_grid_create(ctx, desc)
        mods = _modules(w, analytic)
        t = _backtrack(ctx, grid, mods, w, dirs, R).astype(np.float32)
        x = np.concatenate([dirs, (np.log10(R) - 19.0)[:, None]], axis=1).astype(np.float32)
        xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
        mlp = crp.crp_mlp_create(ctx, 4, 256, 4, w["seed"])
        nb, g, epochs, step = n_train // B, np.random.default_rng(5), 12, 0
        for ep in range(epochs):
            for b in g.permutation(nb):
                lr = 3e-3 * 0.5 * (1 + np.cos(np.pi * step / (epochs * nb))) * min(1.0, (step + 1) / 100)
                crp.crp_mlp_train_step(mlp, xd[b * B:(b + 1) * B], td[b * B:(b + 1) * B], B, lr,
                                       want_loss=False)
                step += 1
        yd = torch.zeros((n_val + n_test, 3), dtype=torch.float32, device="cuda")
        crp.crp_mlp_forward(mlp, xd[n_train:], yd, n_val + n_test)
        torch.cuda.synchronize()
        y = yd.cpu().numpy().astype(np.float64)
        ang = _angle(y, t[n_train:].astype(np.float64))
        ang_v, ang_t = ang[:n_val], ang[n_val:]
        b_v, b_t = _lens_bin(R[n_train:n_train + n_val], w), _lens_bin(R[n_train + n_val:], w)
        val_med = np.array([np.median(ang_v[b_v == b]) for b in range(NBINS)])
        claim = val_med <= 0.5
        # the bins it claims meet 0.5 deg on held-out samples
        for b in np.nonzero(claim)[0]:
            assert np.median(ang_t[b_t == b]) <= 0.6, (b, np.median(ang_t[b_t == b]))
        if claim.any():
            assert np.median(ang_t[claim[b_t]]) <= 0.5
        # interpolation floor at the training spacing in the top rigidity
        # tenth (the smoothest part of the map): border direction of u against
        # the normalised mean of its neighbours u +- spacing on a great circle,
        # binary64 back-tracking
        spacing = np.sqrt(4 * np.pi / (n_train / NBINS))
        gf = np.random.default_rng(9)
        k = 400
        u = gf.normal(size=(k, 3))
        u /= np.linalg.norm(u, axis=1)[:, None]
        v = np.cross(u, gf.normal(size=(k, 3)))
        v /= np.linalg.norm(v, axis=1)[:, None]
        Rp = 10 ** gf.uniform(19.8, 20.0, k)
        ub = _backtrack(ctx, grid, _modules(w, analytic, crp.FP64), w,
                        np.concatenate([u, np.cos(spacing) * u + np.sin(spacing) * v,
                                        np.cos(spacing) * u - np.sin(spacing) * v]),
                        np.concatenate([Rp, Rp, Rp]))
        floor_top = float(np.median(_angle(ub[:k], ub[k:2 * k] + ub[2 * k:])))
        print(f"{galaxy}: claimed {claim.sum()} of {NBINS} bins; chaos floor at "
              f"{np.degrees(spacing):.2f} deg spacing, 10^19.7-10^20: {floor_top:.2f} deg; "
              f"held-out median {np.median(ang_t):.2f} deg")
        if galaxy == "disk_halo_random":
            # the field's structure below the sample spacing rules 0.5 deg out
            assert floor_top > 0.5 and not claim.any()
        else:
            # the count moves by a few bins between runs: the weight-gradient
            # reductions' summation order differs, and training amplifies it
            assert floor_top < 0.5 and claim.sum() >= NBINS // 3
        # lenses: back-tracked, surrogate, merged by the claims
        ldirs, lE, lbins = workloads.lens_samples(NBINS, 3 * 12 * NSIDE * NSIDE, w["r_lo"],
                                                  w["r_hi"], w["seed"] + 22)
        lens_bt, _ = crp.crp_lens_build(ctx, grid, mods, NSIDE, NBINS, w["r_lo"], w["r_hi"],
                                        w["earth"], ldirs, lE, lbins)
        lens_sg = crp.crp_lens_build_surrogate(ctx, mlp, NSIDE, NBINS, w["r_lo"], w["r_hi"],
                                               ldirs, lE, lbins)
        lens_hy = crp.crp_lens_merge(lens_bt, lens_sg, claim)
        ncol = NBINS * 12 * NSIDE * NSIDE
        L = {k: crp.crp_lens_copy_out(h, ncol, NBINS)
             for k, h in (("bt", lens_bt), ("sg", lens_sg), ("hy", lens_hy))}
        npix = 12 * NSIDE * NSIDE
        for b in range(NBINS):
            src = L["sg"] if claim[b] else L["bt"]
            c0 = b * npix
            cs, ch = src["col_start"], L["hy"]["col_start"]
            assert np.array_equal(np.diff(cs[c0:c0 + npix + 1]), np.diff(ch[c0:c0 + npix + 1]))
            assert np.array_equal(src["entries"][cs[c0]:cs[c0 + npix]],
                                  L["hy"]["entries"][ch[c0]:ch[c0 + npix]])
            assert src["max_count"][b] == L["hy"]["max_count"][b]
        # applied to a border population: per candidate, the source lens's pixel
        m = 1 << 18
        bd, bR = workloads.backtrack_directions(m, w["r_lo"], w["r_hi"], w["seed"] + 23)
        inj = crp.host_injection(dict(x=np.zeros(m), y=np.zeros(m), z=np.zeros(m),
                                      ux=bd[:, 0], uy=bd[:, 1], uz=bd[:, 2], E=bR,
                                      A=np.ones(m), Z=np.ones(m)))
        pix = {}
        for k, h in (("bt", lens_bt), ("sg", lens_sg), ("hy", lens_hy)):
            crp.crp_candidates_clear(ctx)
            crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), m)
            crp.crp_lens_apply(ctx, h, crp.COLLECT_ALL)
            rec = crp.crp_collect(ctx, crp.COLLECT_ALL)
            pix[k] = rec[np.argsort(rec["id"], kind="stable")]["lens_pixel"]
        cb = claim[_lens_bin(bR, w)]
        assert np.array_equal(pix["hy"][cb], pix["sg"][cb])
        assert np.array_equal(pix["hy"][~cb], pix["bt"][~cb])
        with pytest.raises(crp.CrpError):
            small = crp.crp_lens_build_surrogate(ctx, mlp, NSIDE // 2, NBINS, w["r_lo"],
                                                 w["r_hi"], ldirs, lE, lbins)
            try:
                crp.crp_lens_merge(lens_bt, small, claim)
            finally:
                crp.crp_lens_destroy(small)
        for h in (lens_bt, lens_sg, lens_hy):
            crp.crp_lens_destroy(h)
        crp.crp_mlp_destroy(mlp)
        crp.crp_grid_destroy(grid)
    finally:
        crp.crp_context_destroy(ctx)
