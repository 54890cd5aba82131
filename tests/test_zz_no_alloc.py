"""The allocation-free energy histogram, through the C ABI, against the
allocating crp_histogram_energy on the same pool.

This file is collected last so that a run stopping at the first failure has
already run every other test.  It must pass both on its own in a fresh
process and after the other tests (which may already have made the first,
set-up call on the device)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

import workloads  # noqa: E402
from paper_1307_2643_gb300 import crp  # noqa: E402


def test_noalloc_histogram_matches_allocating_one():
    from paper_1307_2643_gb300.build import build
    build()
    n = 4000
    inj = crp.host_injection(workloads.plain_small(n=n, seed=17))
    inj["s_max"][:] = 20.0
    n_cells = (32, 32, 32)
    field = np.random.default_rng(2).normal(size=(32, 32, 32, 3))
    ctx = crp.crp_context_create(0, 5, n)
    try:
        g = crp.crp_grid_create(ctx, crp.grid_desc(n_cells, 0.25, dtype=crp.F32, data=field))
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), n)
        m = crp.modules(precision=crp.MIXED, flags=crp.ADIABATIC, beta_ad=1.0 / 400.0)
        crp.crp_propagate(ctx, g, m)
        # two calls in a row, with different binnings, each against the
        # allocating entry point
        for what, lo, hi, nb in ((crp.COLLECT_ALL, 1e19, 1e20, 64),
                                 (crp.COLLECT_FINISHED, 9e18, 2e20, 1000)):
            ref = crp.crp_histogram_energy(ctx, what, lo, hi, nb)
            got = crp.crp_histogram_energy_noalloc(ctx, what, lo, hi, nb)
            assert ref.sum() > 0.9 * n
            assert np.array_equal(got, ref)
        # beyond the fixed array: rejected, nothing written
        with pytest.raises(crp.CrpError) as e:
            crp.crp_histogram_energy_noalloc(ctx, crp.COLLECT_ALL, 1e19, 1e20,
                                             crp.HIST_NOALLOC_MAX_BINS + 1)
        assert e.value.status == crp.E_INVALID
        crp.crp_grid_destroy(g)
    finally:
        crp.crp_context_destroy(ctx)
