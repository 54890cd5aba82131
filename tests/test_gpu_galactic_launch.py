"""Back-tracking through the galactic fields on the mixed path (Sect. 4 lenses
are built this way), for the disk + halo + random field and the analytic
multi-arm field: the records do not depend on the launch (block size,
resident blocks, queue order), and the kernel with the module list fixed at
compile time (the field + border) gives the same bytes as the generic kernel,
which a run with one more module that never fires (E_min far below every
energy) takes."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

import workloads  # noqa: E402
from paper_1307_2643_gb300 import crp  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    from paper_1307_2643_gb300.build import build
    build()
    return crp


def _setup(galaxy):
    w = workloads.GALACTIC_LENS
    if galaxy == "disk_halo_random":
        dx, lmin, org = workloads.galactic_grid_geometry(64, w["box"])
        desc = crp.grid_desc((64,) * 3, dx, origin=org, dtype=crp.F32,
                             source=crp.GRID_TURBULENT, lmin=lmin, lmax=w["lmax"],
                             brms=w["brms"], seed=w["seed"])
        return w, desc, dict(flags=crp.GALACTIC | crp.BORDER, galactic=w["disk"])
    w = workloads.GALACTIC_MULTIARM
    zn = (4, 4, 4)
    desc = crp.grid_desc(zn, 20.0, origin=(-40.0, -40.0, -40.0), dtype=crp.F32,
                         data=np.zeros(zn + (3,)))
    return w, desc, dict(flags=crp.GMF | crp.BORDER, gmf=workloads.multiarm_gmf_params())


def _run(galaxy, inj, n, extra_flags=0, **launch):
    w, desc, analytic = _setup(galaxy)
    analytic = dict(analytic)
    analytic["flags"] |= extra_flags
    ctx = crp.crp_context_create(0, w["seed"], n + 16)
    try:
        grid = crp.crp_grid_create(ctx, desc)
        mods = crp.modules(precision=crp.MIXED, tol=w["tol"], h_min=w["h_min"], h_max=w["h_max"],
                           field_unit_T=crp.MICROGAUSS_T, length_unit_m=crp.KPC_M,
                           border_radius=w["border_r"], e_min=1.0, **analytic, **launch)
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), n)
        crp.crp_propagate(ctx, grid, mods)
        rec = crp.crp_collect(ctx, crp.COLLECT_ALL)
        crp.crp_grid_destroy(grid)
    finally:
        crp.crp_context_destroy(ctx)
    return np.sort(rec, order="id")


@pytest.mark.parametrize("galaxy", ["disk_halo_random", "multiarm"])
def test_galactic_backtracking_records_do_not_depend_on_the_launch(lib, galaxy):
    w = workloads.GALACTIC_LENS
    n = 3000
    dirs, R = workloads.backtrack_directions(n, w["r_lo"], w["r_hi"], 91)
    e = w["earth"]
    inj = crp.host_injection(dict(x=np.full(n, e[0]), y=np.full(n, e[1]), z=np.full(n, e[2]),
                                  ux=dirs[:, 0], uy=dirs[:, 1], uz=dirs[:, 2], E=R,
                                  A=np.ones(n), Z=np.ones(n), q=-np.ones(n)))
    fixed = _run(galaxy, inj, n, block_size=256, blocks_per_sm=2, queue_order=0)
    assert np.all(fixed["status"] == crp.AT_BORDER)
    others = [_run(galaxy, inj, n, block_size=128, blocks_per_sm=5, queue_order=1),
              _run(galaxy, inj, n, block_size=32, blocks_per_sm=3, queue_order=-1),
              _run(galaxy, inj, n, extra_flags=crp.EMIN, block_size=256, blocks_per_sm=2)]
    for o in others:
        assert o.tobytes() == fixed.tobytes()
