"""The multi-rank bench path on CPU (gloo, world size 2): every rank draws its
own candidate shard (disjoint ids, distinct draws), the per-rank spectra and
arrival maps are summed over ranks, the detected records are gathered (the
data exchanges), and per-rank times and step counts become whole-job figures
(slowest rank's time, sum of steps)."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench

RECORD_DTYPE = np.dtype([
    ("id", "<u8"), ("parent_id", "<u8"), ("x", "<f8", 3), ("u", "<f8", 3), ("E", "<f8"),
    ("s", "<f8"), ("status", "<i4"), ("pad", "<i4")])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        _, inj = bench.workload_inputs(2000, rank)
        elapsed, steps = bench.aggregate_ranks(dist, 1.0 + rank, 1000 * (rank + 1))
        ids = torch.from_numpy(inj["id"].astype(np.int64))
        gathered = [torch.zeros_like(ids) for _ in range(world)]
        dist.all_gather(gathered, ids)  # test-side check only
        e = torch.from_numpy(inj["E"])
        energies = [torch.zeros_like(e) for _ in range(world)]
        dist.all_gather(energies, e)
        # the spectrum exchange: per-rank histograms summed over ranks
        edges = np.geomspace(bench.SPECTRUM["e_lo"], bench.SPECTRUM["e_hi"],
                             bench.SPECTRUM["nbins"] + 1)
        hist = torch.from_numpy(np.histogram(inj["E"], edges)[0].astype(np.int64))
        merged = bench.merge_histogram(dist, hist.clone()).numpy()
        # arrival map: HEALPix nside-8 ring pixels of the shard's directions
        import oracle
        u = np.stack([inj["ux"], inj["uy"], inj["uz"]], 1)
        amap = torch.from_numpy(np.bincount(oracle.ang2pix_vec(8, u), minlength=768)
                                .astype(np.int64))
        amap_merged = bench.merge_histogram(dist, amap.clone()).numpy()
        # detected records: a rank-dependent number of records of its own ids
        rec = np.zeros(37 + 20 * rank, dtype=RECORD_DTYPE)
        rec["id"] = inj["id"][::-1][:len(rec)]
        rec["E"] = inj["E"][::-1][:len(rec)]
        rec["x"][:, 0] = rank
        got = bench.gather_records(dist, rec)
        out[rank] = (elapsed, steps, [g.numpy() for g in gathered], [x.numpy() for x in energies],
                     merged, hist.numpy(), amap_merged, rec, got)
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_and_aggregation():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    edges = np.geomspace(bench.SPECTRUM["e_lo"], bench.SPECTRUM["e_hi"], bench.SPECTRUM["nbins"] + 1)
    import oracle
    recs = [res[r][7] for r in range(world)]
    union = np.sort(np.concatenate(recs), order="id")
    dirs = []
    for r in range(world):
        _, inj = bench.workload_inputs(2000, r)
        dirs.append(np.stack([inj["ux"], inj["uy"], inj["uz"]], 1))
    union_map = np.bincount(oracle.ang2pix_vec(8, np.concatenate(dirs)), minlength=768)
    for r in range(world):
        elapsed, steps, ids, energies, merged, own, amap, _, got = res[r]
        # the gathered records: the union of the shards' records, sorted by id
        assert got.dtype == RECORD_DTYPE and len(got) == 37 + 57
        assert got.tobytes() == union.tobytes()
        assert np.all(np.diff(got["id"].astype(np.int64)) > 0)
        # the merged arrival map equals the map of all ranks' directions
        assert np.array_equal(amap, union_map) and amap.sum() == 4000
        assert np.array_equal(merged, np.histogram(np.concatenate(energies), edges)[0])
        assert not np.array_equal(merged, own) and merged.sum() > own.sum() > 0
        assert elapsed == 2.0            # the slowest rank's time
        assert steps == 3000.0           # the sum over ranks
        assert len(np.intersect1d(ids[0], ids[1])) == 0
        assert ids[1].min() == 2000 and ids[0].max() == 1999
        assert not np.array_equal(energies[0], energies[1])


def test_single_rank_aggregation_is_identity():
    assert bench.aggregate_ranks(None, 1.5, 42) == (1.5, 42.0)
    rec = np.zeros(5, dtype=RECORD_DTYPE)
    rec["id"] = [9, 3, 7, 1, 5]
    assert list(bench.gather_records(None, rec)["id"]) == [1, 3, 5, 7, 9]
