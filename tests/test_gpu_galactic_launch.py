"""Back-tracking through the disk + halo + random galactic field on the
mixed path (Sect. 4 lenses are built this way): the records do not depend on
the launch (block size, resident blocks, queue order), and the kernel with
the module list fixed at compile time (galactic field + border) gives the
same bytes as the generic kernel, which a run with one more module that never
fires (E_min far below every energy) takes."""
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


def _run(n_side, inj, n, extra_flags=0, **launch):
    w = workloads.GALACTIC_LENS
    dx, lmin, org = workloads.galactic_grid_geometry(n_side, w["box"])
    desc = crp.grid_desc((n_side,) * 3, dx, origin=org, dtype=crp.F32,
                         source=crp.GRID_TURBULENT, lmin=lmin, lmax=w["lmax"], brms=w["brms"],
                         seed=w["seed"])
    ctx = crp.crp_context_create(0, w["seed"], n + 16)
    try:
        grid = crp.crp_grid_create(ctx, desc)
        mods = crp.modules(precision=crp.MIXED, tol=w["tol"], h_min=w["h_min"], h_max=w["h_max"],
                           field_unit_T=crp.MICROGAUSS_T, length_unit_m=crp.KPC_M,
                           border_radius=w["border_r"], e_min=1.0,
                           flags=crp.GALACTIC | crp.BORDER | extra_flags, galactic=w["disk"],
                           **launch)
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), n)
        crp.crp_propagate(ctx, grid, mods)
        rec = crp.crp_collect(ctx, crp.COLLECT_ALL)
        crp.crp_grid_destroy(grid)
    finally:
        crp.crp_context_destroy(ctx)
    return np.sort(rec, order="id")


def test_galactic_backtracking_records_do_not_depend_on_the_launch(lib):
    w = workloads.GALACTIC_LENS
    n = 3000
    dirs, R = workloads.backtrack_directions(n, w["r_lo"], w["r_hi"], 91)
    e = w["earth"]
    inj = crp.host_injection(dict(x=np.full(n, e[0]), y=np.full(n, e[1]), z=np.full(n, e[2]),
                                  ux=dirs[:, 0], uy=dirs[:, 1], uz=dirs[:, 2], E=R,
                                  A=np.ones(n), Z=np.ones(n), q=-np.ones(n)))
    fixed = _run(64, inj, n, block_size=256, blocks_per_sm=2, queue_order=0)
    assert np.all(fixed["status"] == crp.AT_BORDER)
    others = [_run(64, inj, n, block_size=128, blocks_per_sm=5, queue_order=1),
              _run(64, inj, n, block_size=32, blocks_per_sm=3, queue_order=-1),
              _run(64, inj, n, extra_flags=crp.EMIN, block_size=256, blocks_per_sm=2)]
    for o in others:
        assert o.tobytes() == fixed.tobytes()
