"""Helpers for the GPU tests: run the CUDA library through its C ABI and the
oracle on the same seeded inputs."""
import numpy as np

import oracle
from paper_1307_2643_gb300 import crp


def run_gpu(field, n, spacing, inj, *, precision=crp.FP64, dtype=crp.F64, origin=(0, 0, 0),
            seed=1234, capacity=None, tables=None, tables_n=None, grid_source=None,
            block_size=0, blocks_per_sm=0, collect=crp.COLLECT_ALL, **mods):
    """Propagate `inj` on the GPU; returns (records sorted by id, stats dict, status)."""
    inj = crp.host_injection(inj)
    m = len(inj["E"])
    cap = capacity or max(64, 64 * m)
    ctx = crp.crp_context_create(0, seed, cap)
    try:
        if grid_source is not None:
            g = crp.crp_grid_create(ctx, grid_source)
        else:
            f = np.ascontiguousarray(field, dtype=np.float64)
            g = crp.crp_grid_create(ctx, crp.grid_desc(n, spacing, origin=origin, dtype=dtype,
                                                       data=f, data_dtype=crp.F64))
        th = None
        if tables is not None:
            th = crp.crp_tables_from_host(ctx, crp.tables_desc(n=tables.n, gamma_lo=tables.g_lo,
                                                               gamma_hi=tables.g_hi),
                                          tables.beta_pair, tables.rate_pion, tables.rate_gdr)
        M = crp.modules(precision=precision, tables=th, block_size=block_size,
                        blocks_per_sm=blocks_per_sm, **mods)
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), m)
        status, st = crp.crp_propagate(ctx, g, M, raise_on_error=False)
        rec = np.sort(crp.crp_collect(ctx, collect), order="id")
        if th is not None:
            crp.crp_tables_destroy(th)
        crp.crp_grid_destroy(g)
    finally:
        crp.crp_context_destroy(ctx)
    return rec, st.as_dict(), status


def oracle_params(n, spacing, origin=(0, 0, 0), seed=1234, tables=None, **kw):
    return oracle.make_params(grid_n=n, spacing=spacing, origin=origin, seed=seed, tables=tables,
                              **kw)


def rel_err(a, b, floor=1.0):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


EXACT_FIELDS = ("id", "parent_id", "A", "Z", "A0", "Z0", "q", "status", "n_pion", "n_pd",
                "draws", "generation", "n_dropped")


def assert_chains_equal(gpu, ref):
    """Integer / index results must match bit for bit."""
    assert len(gpu) == len(ref), (len(gpu), len(ref))
    for f in EXACT_FIELDS:
        assert np.array_equal(gpu[f], ref[f]), (f, np.nonzero(gpu[f] != ref[f])[0][:10])
