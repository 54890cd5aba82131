#!/usr/bin/env python
"""Throughput of the candidate propagator: accepted Cash-Karp candidate-steps/s.

One bench step = one full pass of the hot path over one batch: inject the
batch of candidates into the pool, run the module list (Cash-Karp Lorentz
steps with trilinear gathers, pair / adiabatic losses, Philox-sampled pion
production, E_min / length / observer breaks) until every candidate is
inactive.  Workload: 10^6 mixed H/He/N/Fe candidates from 1000 sources in a
100 Mpc box, rigidity-scaled E^-2 spectrum, 256^3 float32 Kolmogorov grid
(100 kpc spacing, B_rms 1 nG, lmax 5 Mpc), observer sphere R = 1 Mpc, E_min
10^18 eV, 500 Mpc path budget.  Field and tables are built on the GPU before
the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank propagates its own batch (weak scaling, candidate ids
offset by rank; no data-path collective).  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "Cash-Karp candidate-steps/s on 1 GB300, mixed-precision vs FP64 at equal error"
UNIT = "candidate-steps/s"
H0_OVER_C = 67.3e3 / 299792458.0          # 1/Mpc (H0 = 67.3 km/s/Mpc)
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("mixed", "fp64"), default="mixed")
    ap.add_argument("--n", type=int, default=None, help="candidates per rank (default 10^6)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison leg")
    ap.add_argument("--no-equal-error", action="store_true",
                    help="skip the mixed-vs-FP64 error legs (tight tolerance, ballistic)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--graph", action="store_true",
                    help="run each propagation's round loop as one captured CUDA graph")
    ap.add_argument("--workload", choices=("mixed", "galactic", "uneven", "e2e", "cosmology",
                                           "train", "lens", "plain"),
                    default="mixed",
                    help="mixed: the propagation benchmark; galactic: back-tracking, MLP "
                         "surrogate training / inference and lens builds; uneven: 10^7 "
                         "candidates, 512^3 grid, photodisintegration secondaries, log-uniform "
                         "path lengths; e2e: 10^8 candidates through the mixed workload's "
                         "field, then the galactic lens and its surrogate; cosmology: 1D mode "
                         "with cosmology and the a-posteriori 3D correction (sources to "
                         "4000 Mpc, index -2.2, protons and iron); lens: lens application "
                         "(nside 64, 100 rigidity bins) to --n candidates (default 2^24); "
                         "plain: the 10^4-proton 64^3 binary64 workload, FP64 on the GPU "
                         "beside the oracle on one thread and on all host cores")
    ap.add_argument("--galaxy", choices=("disk_halo_random", "multiarm", "multiarm_random"),
                    default="disk_halo_random",
                    help="galactic workload field: the disk + halo + random grid, the analytic "
                         "multi-arm field alone, or the multi-arm field plus the random grid")
    ap.add_argument("--n-train", type=int, default=9_000_000)
    ap.add_argument("--n-test", type=int, default=1_000_000)
    ap.add_argument("--epochs", type=int, default=32)
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--lens-per-bin", type=int, default=49152)
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def setup_dist(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist
        # host scalars over gloo; the device spectra over NCCL
        backend = "cpu:gloo,cuda:nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return rank, world, local, dist


def bench_config(w, n, world):
    """The workload the metric is quoted on (the same for both arms)."""
    return {"workload": w["name"], "candidates_per_gpu": n, "grid": "256^3 f32",
            "l2": "inputs larger than L2 (268 MB grid, 245 MB candidate pool)",
            "parallelism": f"candidate shards x{world}"}


SPECTRUM = dict(e_lo=1e18, e_hi=1e21, nbins=60)  # detected-energy histogram, 20 bins/decade
ARRIVAL_NSIDE = 64                               # HEALPix map of the detected arrival directions


def merge_histogram(dist, hist):
    """The data exchange of a multi-rank step: each rank propagates its own
    candidate shard and histograms what its observer detected (spectrum and
    arrival map); the job's histogram is the sum over ranks (all-reduce, in
    place, on the histogram's device)."""
    if dist:
        dist.all_reduce(hist)
    return hist


merge_spectrum = merge_histogram


def gather_records(dist, rec):
    """The detected records of every rank, on every rank, sorted by id: the
    one gather of the multi-rank data plane (host buffers over the CPU
    group).  Candidate ids are disjoint across ranks."""
    if not dist:
        return np.sort(rec, order="id")
    import torch
    world = dist.get_world_size()
    n = torch.tensor([len(rec)], dtype=torch.int64)
    counts = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(counts, n)
    counts = [int(c[0]) for c in counts]
    item = rec.dtype.itemsize
    buf = torch.zeros(max(counts) * item, dtype=torch.uint8)
    if len(rec):
        buf[:len(rec) * item] = torch.from_numpy(np.ascontiguousarray(rec).view(np.uint8).copy())
    bufs = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(bufs, buf)
    parts = [b.numpy()[:c * item].view(rec.dtype) for b, c in zip(bufs, counts)]
    return np.sort(np.concatenate(parts), order="id")


def aggregate_ranks(dist, elapsed, steps):
    """Whole-job figures: the slowest rank's time and the steps of all ranks
    (each rank propagates its own shard)."""
    if not dist:
        return elapsed, float(steps)
    import torch
    t = torch.tensor([elapsed], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    a = torch.tensor([float(steps)], dtype=torch.float64)
    dist.all_reduce(a)
    return float(t[0]), float(a[0])


def workload_inputs(n, rank):
    w = workloads.MIXED_INTERACTIONS
    inj = workloads.mixed_interactions(n=n, seed=w["seed"] + 7919 * rank)
    inj["id"] = inj["id"] + np.uint64(rank * n)
    return w, inj


def modules_for(crp, precision, tables, use_graph=0, tol=None, h_min=None):
    w = workloads.MIXED_INTERACTIONS
    return crp.modules(precision=precision,
                       flags=crp.PAIR | crp.ADIABATIC | crp.PION | crp.EMIN | crp.OBSERVER,
                       tol=w["tol"] if tol is None else tol,
                       h_min=w["h_min"] if h_min is None else h_min, h_max=w["h_max"],
                       beta_ad=H0_OVER_C, e_min=w["e_min"], tables=tables,
                       observer_radius=w["observer_r"], use_graph=use_graph)


def flops_per_trial_mixed():
    """Algorithmic binary32 flops of one mixed-precision Cash-Karp trial, by
    count of the arithmetic the method needs:
      field gather (x6): 3 fma + 3 floor + 3 sub for the in-cell coordinates,
                         21 lerps x 3 flops                         = 75
      Lorentz force (x6): cross product 9 + scale 3                  = 12
      stage directions u_2..u_6: sum_j (2j - 1) x 3 components       = 105
      stage offsets o_2..o_6:    sum_j 2(j - 1) x 3 components       = 90
      fifth-order offset 8 x 3, direction 9 x 3, error 10 x 3        = 81
    """
    return 6 * (75 + 12) + 105 + 90 + 81


# field bytes one Cash-Karp trial needs: 6 trilinear gathers x 8 corners x 3 binary32;
# the algorithmic cost of an accepted step is one trial's gathers
GATHER_BYTES_PER_TRIAL_F32 = 6 * 8 * 3 * 4
# DRAM bytes (read + write) per Cash-Karp trial of the mixed propagate kernel this
# workload runs (its module list fixed at compile time), from one ncu capture of the
# current kernel (2e5 candidates of this workload: 154.594 GB read + 0.157 GB written
# over 1.5611e9 trials); traffic grows with the number of trials, so a launch's
# traffic is this figure times its trials
DRAM_BYTES_PER_TRIAL_MIXED = (154.594e9 + 0.157e9) / 1.5611e9

# the equal-error statement: tolerances, subsample sizes and the chaos-floor kick
TIGHT_TOL, TIGHT_HMIN = 1e-8, 1e-4          # where the method resolves 1e-5 per candidate
TRUTH_TOL, TRUTH_HMIN = 1e-10, 1e-5         # the oracle reference ("truth")
TIGHT_SUBSAMPLE = 100_000                   # ids of the batch timed at TIGHT_TOL
TRUTH_SAMPLE = 256                          # ids of that subsample the oracle recomputes
BALLISTIC_N = 1_000_000                     # protons of the plain small recipe
BALLISTIC_TRUTH_SAMPLE = 512
FLOOR_AXES = ((0.267, 0.535, 0.802), (0.9, -0.3, 0.1), (-0.2, 0.7, -0.6))
FLOOR_GATE = 2e-6


def quantiles(v, within=1e-5):
    v = np.asarray(v, dtype=np.float64)
    if len(v) == 0:
        return None
    return {"median": float(np.median(v)), "p90": float(np.percentile(v, 90)),
            "p99": float(np.percentile(v, 99)), "max": float(v.max()),
            f"frac_le_{within:g}": float(np.mean(v <= within))}


def endpoint_errors(a, b):
    """Per-candidate differences of record set `a` from `b` (same ids, both
    sorted by id): position change relative to the trajectory length and to
    max(1, |x|) (length units), direction change |u_a - u_b|, relative
    energy change."""
    assert np.array_equal(a["id"], b["id"])
    dx = np.linalg.norm(a["x"] - b["x"], axis=1)
    return {"pos_over_s": dx / np.maximum(b["s"], 1e-300),
            "pos_over_x": dx / np.maximum(1.0, np.linalg.norm(b["x"], axis=1)),
            "dir": np.linalg.norm(a["u"] - b["u"], axis=1),
            "E": np.abs(a["E"] - b["E"]) / b["E"]}


def agreement(a, b):
    """Quantiles of endpoint_errors plus agreement of the integer results."""
    e = endpoint_errors(a, b)
    out = {k: quantiles(v) for k, v in e.items()}
    out["n"] = int(len(a))
    out["status_agree"] = float(np.mean(a["status"] == b["status"]))
    out["n_pion_agree"] = float(np.mean(a["n_pion"] == b["n_pion"]))
    return out


def kicked(inj, delta, axis):
    """Injection with each direction turned by delta[i] radians (first order)
    about an axis perpendicular to it and to `axis` (chaos-floor runs)."""
    p = dict(inj)
    u = np.stack([p["ux"], p["uy"], p["uz"]], 1)
    v = np.cross(u, np.asarray(axis, dtype=np.float64))
    v /= np.linalg.norm(v, axis=1)[:, None]
    u2 = u + delta[:, None] * v
    u2 /= np.linalg.norm(u2, axis=1)[:, None]
    p["ux"], p["uy"], p["uz"] = [np.ascontiguousarray(u2[:, k]) for k in range(3)]
    return p


def ballistic_inputs(n):
    """The plain small recipe (protons E^-2 on 10^19-10^20 eV, isotropic from
    the origin, 50 Mpc) at n candidates: quasi-ballistic histories, where a
    per-candidate 1e-5 endpoint agreement is a property of the method."""
    w = workloads.PLAIN_SMALL
    return w, workloads.plain_small(n=n, seed=w["seed"])


def timed_propagate(crp, torch, ctx, grid, arrays, n, mods, stream):
    """Inject, propagate (CUDA events on the launching stream), collect."""
    crp.crp_candidates_clear(ctx)
    crp.crp_candidates_inject(ctx, arrays, n, 0, stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    _, st = crp.crp_propagate(ctx, grid, mods, stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    rec = np.sort(crp.crp_collect(ctx, crp.COLLECT_ALL), order="id")
    return rec, st, e0.elapsed_time(e1) / 1e3


def run_ours(args):
    import torch
    from paper_1307_2643_gb300 import crp
    from paper_1307_2643_gb300.build import build

    rank, world, local, dist = setup_dist(args)
    torch.cuda.set_device(local)
    build()
    crp.use_torch_allocator(local)
    n = args.n or workloads.MIXED_INTERACTIONS["n"]
    w, inj = workload_inputs(n, rank)
    inj = crp.host_injection(inj)
    cap = max(int(n * 1.02) + 1024, BALLISTIC_N + 1024)
    ctx = crp.crp_context_create(local, w["seed"], cap)
    gd = crp.grid_desc(w["grid_n"], w["spacing"], dtype=crp.F32, source=crp.GRID_TURBULENT,
                       lmin=w["lmin"], lmax=w["lmax"], brms=w["brms"], seed=w["seed"])
    grid = crp.crp_grid_create(ctx, gd)
    tables = crp.crp_tables_build(ctx, crp.tables_desc(n=1000))
    prec = crp.MIXED if args.precision == "mixed" else crp.FP64
    mods = modules_for(crp, prec, tables, use_graph=1 if args.graph else 0)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    dev = {k: torch.from_numpy(v).cuda() for k, v in inj.items()}
    arr_dev = crp.candidate_arrays(dev, on_device=True)
    pinned = {k: torch.from_numpy(v).pin_memory() for k, v in inj.items()}
    arr_host = crp.candidate_arrays(pinned, on_device=False)

    hist = torch.zeros(SPECTRUM["nbins"], dtype=torch.int64, device="cuda")
    amap = torch.zeros(12 * ARRIVAL_NSIDE ** 2, dtype=torch.int64, device="cuda")

    def one_step(arrays):
        crp.crp_candidates_clear(ctx)
        crp.crp_candidates_inject(ctx, arrays, n, 0, sh)
        _, st = crp.crp_propagate(ctx, grid, mods, sh)
        crp.crp_histogram_energy_device(ctx, crp.COLLECT_DETECTED, SPECTRUM["e_lo"],
                                        SPECTRUM["e_hi"], SPECTRUM["nbins"], hist, stream=sh)
        crp.crp_histogram_healpix_device(ctx, crp.COLLECT_DETECTED, ARRIVAL_NSIDE, 0, amap,
                                         stream=sh)
        merge_histogram(dist, hist)
        merge_histogram(dist, amap)
        return st

    for _ in range(args.warmup):
        one_step(arr_dev)

    # ---- device-resident timed region -------------------------------------
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = [one_step(arr_dev) for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    elapsed = e0.elapsed_time(e1) / 1e3
    acc = sum(s.accepted_steps for s in stats)
    rej = sum(s.rejected_trials for s in stats)
    kern_ms = sum(s.kernel_ms for s in stats)
    launches = sum(s.launches for s in stats)
    elapsed, acc_all = aggregate_ranks(dist, elapsed, acc)
    value = acc_all / elapsed
    # the last timed step's records (outside the timed region), and the job's
    # detected records gathered from every rank
    rec_main = np.sort(crp.crp_collect(ctx, crp.COLLECT_ALL), order="id")
    detected = gather_records(dist, rec_main[rec_main["status"] == crp.DETECTED])

    # ---- end to end through the public API with host buffers ---------------
    e2e = None
    if not args.no_e2e:
        rec_cap = int(n * 1.02) + 1024
        out = np.zeros(rec_cap, dtype=crp.RECORD_DTYPE)
        out_t = torch.from_numpy(out.view(np.uint8)).pin_memory()
        out_p = out_t.numpy().view(crp.RECORD_DTYPE)
        h2d = sum(v.nbytes for v in inj.values())
        d2h = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        acc_e = 0
        for _ in range(args.steps):
            st = one_step(arr_host)
            acc_e += st.accepted_steps
            nrec = crp.C.c_size_t()
            crp._check(crp.lib().crp_collect(ctx, crp.COLLECT_FINISHED, out_p.ctypes.data, rec_cap,
                                             crp.C.byref(nrec), 0, sh))
            d2h += nrec.value * crp.RECORD_DTYPE.itemsize
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        e2e = {"value": acc_e / te * world, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h // args.steps)}

    # ---- FP64 leg on the same workload, and the equal-error legs -----------
    fp64, equal_error, gpu_legs = None, None, None
    if not args.no_fp64 and prec == crp.MIXED:
        rec64, st64, ft = timed_propagate(crp, torch, ctx, grid, arr_dev, n,
                                          modules_for(crp, crp.FP64, tables), stream)
        fp64 = {"value": st64.accepted_steps / ft, "unit": UNIT,
                "kernel_ms": st64.kernel_ms, "accepted_steps": st64.accepted_steps,
                "rejected_trials": st64.rejected_trials,
                "mixed_over_fp64": value / world / (st64.accepted_steps / ft),
                "note": "the binary64 kernel is the parity path (no contraction, bit-exact "
                        "with the oracle), not a binary64 kernel tuned for speed"}
        if not args.no_equal_error:
            gpu_legs = equal_error_gpu_legs(crp, torch, ctx, grid, tables, inj, stream,
                                            rec_main, rec64, value / world, fp64["value"])

    # ---- roofline of the propagate kernel ----------------------------------
    # denominators: HBM from MEASURED_PEAKS.json; FP32 issue measured on this
    # device by the library's own probe
    probe = crp.crp_measure_peaks(local)
    peaks = json.load(open(PEAKS_PATH)) if os.path.exists(PEAKS_PATH) else {}
    sm_mhz = clk.get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median") or 1440.0
    n_sm = probe["sm_count"]
    trials = acc + rej
    kern_s = kern_ms / 1e3
    derived32 = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12   # FP32 FMA lanes x 2 flops x clock
    hbm_peak = peaks.get("hbm_gbs")
    hbm_src = "measured (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)"
    if not hbm_peak:
        hbm_peak, hbm_src = 6800.0, "fallback 6.8 TB/s (no measured peak on this host)"
    roof = None
    if prec == crp.MIXED:
        gather = acc * GATHER_BYTES_PER_TRIAL_F32 / kern_s / 1e9
        traffic = DRAM_BYTES_PER_TRIAL_MIXED * trials / max(launches, 1)
        dram = DRAM_BYTES_PER_TRIAL_MIXED * trials / kern_s / 1e9
        flops = trials * flops_per_trial_mixed() / kern_s / 1e12
        roof = {"bound": "hbm", "achieved": gather, "peak": hbm_peak, "unit": "GB/s",
                "frac": gather / hbm_peak, "traffic": traffic,
                "algorithmic": f"{GATHER_BYTES_PER_TRIAL_F32} B of field gathers per accepted "
                               "step (6 trilinear gathers x 8 corners x 3 binary32) x accepted "
                               "steps per launch / mean propagate-kernel launch time (CUDA "
                               "events on the launching stream)",
                "peak_source": hbm_src,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per trial "
                                  "(2e5-candidate capture) x trials per launch",
                "per_trial": {"achieved": trials * GATHER_BYTES_PER_TRIAL_F32 / kern_s / 1e9,
                              "frac": trials * GATHER_BYTES_PER_TRIAL_F32 / kern_s / 1e9
                              / hbm_peak,
                              "note": "the same gathers counted over every Cash-Karp trial, "
                                      "rejected ones included"},
                "dram_actual": {"achieved": dram, "frac": dram / hbm_peak,
                                "note": "DRAM bytes per launch (traffic) / launch time; most "
                                        "gathers hit L1 and the per-lane record cache"},
                "fp32_issue": {"achieved": flops, "peak": probe["fp32_tflops"],
                               "unit": "TFLOP/s", "frac": flops / probe["fp32_tflops"],
                               "flops_per_trial": flops_per_trial_mixed(),
                               "peak_source": "measured: crp_measure_peaks binary32 FMA probe "
                                              f"(derived {derived32:.1f} TFLOP/s = {n_sm} SMs x "
                                              f"128 lanes x 2 x {sm_mhz:.0f} MHz)"},
                "l2_read_peak_GBs": probe["l2_read_gbs"]}
    else:
        achieved = trials * flops_per_trial_mixed() / kern_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": probe["fp64_tflops"],
                "unit": "TFLOP/s", "frac": achieved / probe["fp64_tflops"], "traffic": None,
                "peak_source": "measured: crp_measure_peaks binary64 FMA probe",
                "flops_per_trial": flops_per_trial_mixed()}
    if fp64 is not None:
        f_ach = (fp64["accepted_steps"] + fp64["rejected_trials"]) * flops_per_trial_mixed() \
            / (fp64["kernel_ms"] / 1e3) / 1e12
        fp64["roofline"] = {"bound": "alu", "achieved": f_ach, "peak": probe["fp64_tflops"],
                            "unit": "TFLOP/s", "frac": f_ach / probe["fp64_tflops"],
                            "peak_source": "measured: crp_measure_peaks binary64 FMA probe"}

    # ---- CPU leg (rank 0): the oracle as baseline and as error reference ---
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        grid_host = crp.crp_grid_copy_out(grid, w["grid_n"])
        cpu = cpu_baseline(inj, grid_host=grid_host, seconds=args.cpu_seconds)
        if gpu_legs is not None:
            equal_error = equal_error_statement(gpu_legs, inj, grid_host)
    if equal_error is None and gpu_legs is not None:
        equal_error = equal_error_statement(gpu_legs, None, None)

    crp.crp_tables_destroy(tables)
    crp.crp_grid_destroy(grid)
    crp.crp_context_destroy(ctx)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if prec == crp.MIXED else "f64",
            "data": "synthetic (seeded injection, GPU-generated turbulent field)",
            "config": bench_config(w, n, world),
            "precision": args.precision, "round_loop": "cuda-graph" if args.graph else "host",
            "accepted_steps": acc, "rejected_trials": rej,
            "rejected_trials_per_s": rej / elapsed,
            "kernel_ms_per_step": kern_ms / args.steps,
            # per step: inject (1), queue build (2), queue sort (3), detected-
            # energy histogram (1), arrival map (1); per round: host loop =
            # reset + propagate (+ sort of requeued work), graph = 5
            "gpu_launches": int(args.steps * 8 + launches * (5 if args.graph else 2)),
            "spectrum": {"bins": SPECTRUM["nbins"], "e_lo_eV": SPECTRUM["e_lo"],
                         "e_hi_eV": SPECTRUM["e_hi"], "detected_last_step": int(hist.sum()),
                         "exchange": "sum over ranks on the device (NCCL all-reduce)"
                                     if world > 1 else "single rank: none"},
            "arrival_map": {"nside": ARRIVAL_NSIDE, "detected_last_step": int(amap.sum()),
                            "exchange": "sum over ranks on the device (NCCL all-reduce)"
                                        if world > 1 else "single rank: none"},
            "detected_records": {"gathered": int(len(detected)),
                                 "unique_ids": bool(len(np.unique(detected["id"]))
                                                    == len(detected)),
                                 "exchange": "all-gather of host records (gloo)"
                                             if world > 1 else "single rank: none"},
            "e2e": e2e, "fp64": fp64, "mixed_vs_fp64": equal_error, "roofline": roof,
            "cpu_baseline": cpu, "clocks": clk, "measured_peaks": probe,
        }
        print(json.dumps(line))


def equal_error_gpu_legs(crp, torch, ctx, grid, tables, inj, stream, rec_mx, rec64,
                         mixed_sps, fp64_sps):
    """GPU part of the equal-error statement (outside the timed region):
    the two paths' records of the headline batch at its tolerance, both paths
    timed on an id-subsample of the batch at TIGHT_TOL, and both paths timed
    on the quasi-ballistic plain recipe at both tolerances."""
    n = len(inj["E"])
    legs = {"headline": {"w": workloads.MIXED_INTERACTIONS,
                         "tol": workloads.MIXED_INTERACTIONS["tol"],
                         "h_min": workloads.MIXED_INTERACTIONS["h_min"],
                         "steps_per_s": {"mixed": mixed_sps, "fp64": fp64_sps,
                                         "mixed_over_fp64": mixed_sps / fp64_sps},
                         "records": (rec_mx, rec64)}}
    idx = np.sort(np.random.default_rng(5).permutation(n)[:min(TIGHT_SUBSAMPLE, n)])
    sub = workloads.subsample(inj, idx)
    dev = {k: torch.from_numpy(v).cuda() for k, v in sub.items()}
    arr = crp.candidate_arrays(dev, on_device=True)
    tight = {"tol": TIGHT_TOL, "h_min": TIGHT_HMIN, "candidates": int(len(idx)),
             "ids": idx}
    recs, sps = {}, {}
    for name, prec in (("mixed", crp.MIXED), ("fp64", crp.FP64)):
        m = modules_for(crp, prec, tables, tol=TIGHT_TOL, h_min=TIGHT_HMIN)
        recs[name], st, dt = timed_propagate(crp, torch, ctx, grid, arr, len(idx), m, stream)
        sps[name] = st.accepted_steps / dt
        tight[f"accepted_steps_{name}"] = int(st.accepted_steps)
    tight["steps_per_s"] = {"mixed": sps["mixed"], "fp64": sps["fp64"],
                            "mixed_over_fp64": sps["mixed"] / sps["fp64"]}
    tight["records"] = (recs["mixed"], recs["fp64"])
    legs["headline_tight"] = tight
    del dev

    # the quasi-ballistic plain recipe, 10^6 protons, its 64^3 grid in binary32
    wb, binj = ballistic_inputs(BALLISTIC_N)
    binj = crp.host_injection(binj)
    bgrid = crp.crp_grid_create(ctx, crp.grid_desc(wb["grid_n"], wb["spacing"], dtype=crp.F32,
                                                   source=crp.GRID_TURBULENT, lmin=wb["lmin"],
                                                   lmax=wb["lmax"], brms=wb["brms"],
                                                   seed=wb["seed"]))
    dev = {k: torch.from_numpy(v).cuda() for k, v in binj.items()}
    arr = crp.candidate_arrays(dev, on_device=True)
    ball = {"w": wb,
            "workload": f"{BALLISTIC_N} protons of {wb['name']}: E^-2 on 1e19-1e20 eV, "
                        "isotropic from the origin, 50 Mpc, 64^3 Kolmogorov grid stored in "
                        "binary32 for both paths", "candidates": BALLISTIC_N,
            "inj": binj, "grid_host": crp.crp_grid_copy_out(bgrid, wb["grid_n"])}
    for tol, hmin in ((wb["tol"], wb["h_min"]), (TIGHT_TOL, TIGHT_HMIN)):
        recs, sps = {}, {}
        for name, prec in (("mixed", crp.MIXED), ("fp64", crp.FP64)):
            m = crp.modules(precision=prec, tol=tol, h_min=hmin, h_max=wb["h_max"])
            recs[name], st, dt = timed_propagate(crp, torch, ctx, bgrid, arr, BALLISTIC_N, m,
                                                 stream)
            sps[name] = st.accepted_steps / dt
        ball[f"tol_{tol:g}"] = {"tol": tol, "h_min": hmin,
                                "steps_per_s": {"mixed": sps["mixed"], "fp64": sps["fp64"],
                                                "mixed_over_fp64": sps["mixed"] / sps["fp64"]},
                                "records": (recs["mixed"], recs["fp64"])}
    crp.crp_grid_destroy(bgrid)
    legs["ballistic"] = ball
    return legs


def _oracle_params(oracle, w, tol, h_min, T=None, interactions=True):
    kw = dict(grid_n=w["grid_n"], spacing=w["spacing"], tol=tol, h_min=h_min, h_max=w["h_max"],
              seed=w["seed"])
    if interactions:
        kw.update(flags=oracle.PAIR | oracle.ADIABATIC | oracle.PION | oracle.EMIN |
                  oracle.OBSERVER, e_min=w["e_min"], beta_ad=H0_OVER_C, tables=T,
                  obs_r=w["observer_r"])
    return oracle.make_params(**kw)


def _floor(oracle, P, B, sub, ref, T=None):
    """Per-candidate chaos floor: the largest endpoint change (relative to
    max(1, |x|)) of the oracle's own history when the initial direction is
    turned by 2^-24 sqrt(N) radians about each of three axes (N: the
    candidate's accepted steps; 2^-24 is the binary32 unit roundoff)."""
    delta = 2.0 ** -24 * np.sqrt(ref["n_acc"].astype(np.float64))
    errs = []
    for a in FLOOR_AXES:
        r = oracle.propagate(P, B, kicked(sub, delta, a), tables=T)
        r = r[r["generation"] == 0]
        errs.append(endpoint_errors(r, ref)["pos_over_x"])
    return np.max(errs, axis=0)


def equal_error_statement(legs, inj, grid_host):
    """The mixed-vs-FP64 error block of the bench line.  With inj / grid_host
    (rank 0, CPU leg) the oracle recomputes id-subsamples at TRUTH_TOL and
    the chaos floors; otherwise only the GPU-side agreement is reported."""
    out = {"definitions": {
        "pos_over_s": "|x_a - x_b| / trajectory length", "pos_over_x": "|x_a - x_b| / max(1, |x|)",
        "dir": "|u_a - u_b|", "E": "|E_a - E_b| / E_b",
        "truth": f"oracle (binary64 CPU) at tol {TRUTH_TOL:g}, h_min {TRUTH_HMIN:g} (headline) "
                 "or 1e-4 (ballistic), on an id-subsample",
        "chaos_floor": "largest endpoint change of the oracle's own history under a "
                       "2^-24 sqrt(N) rad kick of the initial direction about 3 axes; a "
                       f"candidate is 'resolvable' where it is <= {FLOOR_GATE:g}"}}
    oracle = None
    if inj is not None:
        import oracle as _oracle
        oracle = _oracle
        oracle.build()
    hw = legs["headline"]["w"]
    # headline batch at its tolerance and at TIGHT_TOL
    h, t = legs["headline"], legs["headline_tight"]
    head = {"tol": h["tol"], "h_min": h["h_min"], "steps_per_s": h["steps_per_s"],
            "mixed_vs_fp64": agreement(*h["records"])}
    tight = {"tol": t["tol"], "h_min": t["h_min"], "candidates": t["candidates"],
             "sample": "ids drawn from the headline batch (seed 5)",
             "steps_per_s": t["steps_per_s"], "mixed_vs_fp64": agreement(*t["records"])}
    if oracle is not None:
        T = oracle.tables_build(n=1000)
        pick = np.sort(np.random.default_rng(6).choice(len(t["ids"]), TRUTH_SAMPLE,
                                                        replace=False))
        ids = t["ids"][pick]
        sub = workloads.subsample(inj, ids)
        t0 = time.perf_counter()
        P = _oracle_params(oracle, hw, TRUTH_TOL, TRUTH_HMIN, T)
        truth = oracle.propagate(P, grid_host, sub, tables=T)
        truth = truth[truth["generation"] == 0]
        floor = _floor(oracle, P, grid_host, sub, truth, T)
        secs = time.perf_counter() - t0
        resolvable = floor <= FLOOR_GATE
        for blk, (rm, rf) in ((head, h["records"]), (tight, t["records"])):
            sm = np.isin(rm["id"], truth["id"])
            blk["vs_truth"] = {"mixed": agreement(rm[sm], truth),
                               "fp64": agreement(rf[sm], truth)}
        head["chaos_floor"] = {"candidates": TRUTH_SAMPLE, "floor": quantiles(floor),
                               "frac_resolvable": float(resolvable.mean()),
                               "oracle_seconds": secs}
    out["headline"] = head
    out["headline_tight"] = tight
    # quasi-ballistic protons
    b = legs["ballistic"]
    ball = {"workload": b["workload"]}
    wb = b["w"]
    for key in [k for k in b if k.startswith("tol_")]:
        blk = b[key]
        rm, rf = blk["records"]
        r = {"tol": blk["tol"], "h_min": blk["h_min"], "steps_per_s": blk["steps_per_s"],
             "mixed_vs_fp64": agreement(rm, rf)}
        if oracle is not None:
            pick = np.sort(np.random.default_rng(7).choice(len(rm), BALLISTIC_TRUTH_SAMPLE,
                                                            replace=False))
            sub = workloads.subsample(b["inj"], pick)
            Pt = _oracle_params(oracle, wb, TRUTH_TOL, 1e-4, interactions=False)
            truth = oracle.propagate(Pt, b["grid_host"], sub)
            Pr = _oracle_params(oracle, wb, blk["tol"], blk["h_min"], interactions=False)
            ref = oracle.propagate(Pr, b["grid_host"], sub)
            floor = _floor(oracle, Pr, b["grid_host"], sub, ref)
            gated = floor <= FLOOR_GATE
            em = endpoint_errors(rm[pick], rf[pick])["pos_over_x"]
            r["vs_truth"] = {"mixed": agreement(rm[pick], truth),
                             "fp64": agreement(rf[pick], truth)}
            r["fp64_equals_oracle"] = bool(np.array_equal(rf[pick]["x"], ref["x"]))
            r["chaos_floor"] = {"candidates": BALLISTIC_TRUTH_SAMPLE,
                                "floor": quantiles(floor),
                                "frac_resolvable": float(gated.mean()),
                                "mixed_vs_fp64_resolvable": quantiles(em[gated]),
                                "mixed_vs_fp64_rest": quantiles(em[~gated])}
        ball[key] = r
    out["ballistic"] = ball
    return out


def cpu_baseline(inj, grid_host, seconds=15.0):
    """The oracle, as it stands, on a bounded id-subsample of the workload,
    timed on this host's cores (histories are the same ids' histories)."""
    import oracle
    w = workloads.MIXED_INTERACTIONS
    oracle.build()
    T = oracle.tables_build(n=1000)
    P = _oracle_params(oracle, w, w["tol"], w["h_min"], T)
    cores = len(os.sched_getaffinity(0))
    rng = np.random.default_rng(1)
    order = rng.permutation(len(inj["E"]))

    def timed(threads, budget, limit):
        steps, done, t_used, chunk = 0, 0, 0.0, 64
        while t_used < budget and done < limit:
            idx = np.sort(order[done:min(done + chunk, limit)])
            sub = workloads.subsample(inj, idx)
            t0 = time.perf_counter()
            r = oracle.propagate(P, grid_host, sub, tables=T, nthreads=threads)
            t_used += time.perf_counter() - t0
            steps += int(r["n_acc"].sum())
            done += len(idx)
            chunk = min(4096 if threads > 1 else 256, chunk * 2)
        return steps, done, t_used

    # all host cores for two thirds of the budget; then one thread for the
    # rest, on the first of the same ids (like for like)
    steps, done, t_used = timed(cores, seconds * 2.0 / 3.0, len(order))
    s1, d1, t1 = timed(1, seconds / 3.0, done)
    single = {"value": s1 / t1, "unit": UNIT, "cores": 1,
              "sample": f"the first {d1} of the same {done} candidates, in the same order, "
                        f"{s1} accepted steps in {t1:.1f} s"} if d1 > 0 and t1 > 0 else \
        {"value": None, "unit": UNIT, "cores": 1,
         "sample": "not run: the all-cores leg processed no candidates"}
    return {"value": steps / t_used, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} candidates drawn by id from the same 10^6-candidate batch, "
                      f"{steps} accepted steps in {t_used:.1f} s",
            "single_thread": single}


def run_plain(args):
    """The plain small workload at its stated size: 10^4 protons (E^-2 on
    10^19-10^20 eV, isotropic from the origin) through the 64^3 binary64
    Kolmogorov grid, 50 Mpc, no interactions, binary64 on the GPU; the GPU
    timed with CUDA events (steps after warm-ups).  Its CPU baseline is the
    oracle on the same candidates on all host cores and on one thread."""
    import torch
    import oracle
    from paper_1307_2643_gb300 import crp
    from paper_1307_2643_gb300.build import build
    torch.cuda.set_device(0)
    build()
    crp.use_torch_allocator(0)
    w = workloads.PLAIN_SMALL
    n = args.n or w["n"]
    inj = crp.host_injection(workloads.plain_small(n=n))
    ctx = crp.crp_context_create(0, w["seed"], n + 64)
    grid = crp.crp_grid_create(ctx, crp.grid_desc(w["grid_n"], w["spacing"], dtype=crp.F64,
                                                  source=crp.GRID_TURBULENT, lmin=w["lmin"],
                                                  lmax=w["lmax"], brms=w["brms"], seed=w["seed"]))
    stream = torch.cuda.current_stream()
    dev = {k: torch.from_numpy(v).cuda() for k, v in inj.items()}
    arr = crp.candidate_arrays(dev, on_device=True)
    mods = crp.modules(precision=crp.FP64, tol=w["tol"], h_min=w["h_min"], h_max=w["h_max"])
    for _ in range(args.warmup):
        rec, st, dt = timed_propagate(crp, torch, ctx, grid, arr, n, mods, stream)
    ts = []
    for _ in range(args.steps):
        rec, st, dt = timed_propagate(crp, torch, ctx, grid, arr, n, mods, stream)
        ts.append(dt)
    t = statistics.median(ts)
    B = crp.crp_grid_copy_out(grid, w["grid_n"])
    crp.crp_grid_destroy(grid)
    crp.crp_context_destroy(ctx)
    oracle.build()
    P = oracle.make_params(grid_n=w["grid_n"], spacing=w["spacing"], tol=w["tol"],
                           h_min=w["h_min"], h_max=w["h_max"], seed=w["seed"])
    cores = len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    ref = oracle.propagate(P, B, inj, nthreads=cores)
    t_all = time.perf_counter() - t0
    n1 = min(n, 2000)
    t0 = time.perf_counter()
    ref1 = oracle.propagate(P, B, workloads.subsample(inj, np.arange(n1)), nthreads=1)
    t_one = time.perf_counter() - t0
    same = bool(len(ref) == len(rec) and np.array_equal(ref["x"], rec["x"])
                and np.array_equal(ref["n_acc"], rec["n_acc"]))
    print(json.dumps({
        "workload": w["name"], "metric": "accepted Cash-Karp candidate-steps/s (binary64)",
        "unit": UNIT, "candidates": n, "steps": args.steps, "warmup": args.warmup,
        "accepted_steps": int(st.accepted_steps), "rejected_trials": int(st.rejected_trials),
        "gpu_fp64": {"value": st.accepted_steps / t, "ms_per_step": t * 1e3,
                     "kernel_ms": st.kernel_ms,
                     "note": "10^4 candidates fill 0.2 of the GPU's resident lanes; a parity "
                             "workload, not a throughput one"},
        "cpu_baseline": {"value": int(ref["n_acc"].sum()) / t_all, "unit": UNIT,
                         "cores": cores, "kind": "oracle",
                         "sample": f"all {n} candidates, {t_all:.2f} s",
                         "single_thread": {"value": int(ref1["n_acc"].sum()) / t_one,
                                           "unit": UNIT, "cores": 1,
                                           "sample": f"the first {n1} candidates, "
                                                     f"{t_one:.2f} s"}},
        "gpu_records_equal_oracle": same,
    }))


def run_reference(args):
    """The oracle (FP64 C++ on the host cores) on bounded samples of the same
    workload; rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    w = workloads.MIXED_INTERACTIONS
    n = args.n or w["n"]
    _, inj = workload_inputs(n, 0)
    field = oracle.turbulent_field(w["grid_n"], w["spacing"], w["lmin"], w["lmax"], w["brms"],
                                   seed=w["seed"]).astype(np.float32).astype(np.float64)
    T = oracle.tables_build(n=1000)
    P = oracle.make_params(grid_n=w["grid_n"], spacing=w["spacing"], tol=w["tol"],
                           h_min=w["h_min"], h_max=w["h_max"],
                           flags=oracle.PAIR | oracle.ADIABATIC | oracle.PION | oracle.EMIN |
                           oracle.OBSERVER, e_min=w["e_min"], beta_ad=H0_OVER_C,
                           seed=w["seed"], tables=T, obs_r=w["observer_r"])
    cores = len(os.sched_getaffinity(0))
    # a bounded id-sample of the batch per step: histories are per id, so they
    # are the full run's; 4096 keeps every host core busy for the whole step
    per_step = max(16, min(n, 4096))
    rng = np.random.default_rng(2)

    def step(i):
        idx = np.sort(rng.choice(n, per_step, replace=False))
        return int(oracle.propagate(P, field, workloads.subsample(inj, idx), tables=T,
                                    nthreads=cores)["n_acc"].sum())

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    acc = sum(step(i) for i in range(args.steps))
    dt = time.perf_counter() - t0
    v = acc / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": bench_config(w, n, args.gpus), "precision": "fp64 (oracle)",
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} random candidates of the batch per step"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def coarse_ring_map(hist, nside, n_bands=16, n_sectors=8):
    """Sum a HEALPix RING map into n_bands latitude bands (by ring index) x
    n_sectors longitude sectors (by position within the ring)."""
    npix = 12 * nside * nside
    p = np.arange(npix, dtype=np.int64)
    ncap = 2 * nside * (nside - 1)
    ring = np.empty(npix, np.int64)
    first = np.empty(npix, np.int64)
    length = np.empty(npix, np.int64)
    north = p < ncap
    i = np.floor((1 + np.sqrt(1 + 2 * p[north])) / 2).astype(np.int64)
    i -= (2 * i * (i - 1) > p[north])
    i += (2 * (i + 1) * i <= p[north])
    ring[north], first[north], length[north] = i, 2 * i * (i - 1), 4 * i
    eq = (p >= ncap) & (p < npix - ncap)
    ie = (p[eq] - ncap) // (4 * nside) + nside
    ring[eq], first[eq], length[eq] = ie, ncap + 4 * nside * (ie - nside), 4 * nside
    south = p >= npix - ncap
    ps = npix - 1 - p[south]
    j = np.floor((1 + np.sqrt(1 + 2 * ps)) / 2).astype(np.int64)
    j -= (2 * j * (j - 1) > ps)
    j += (2 * (j + 1) * j <= ps)
    ring[south], length[south] = 4 * nside - j, 4 * j
    first[south] = npix - 2 * j * (j + 1)
    band = (ring - 1) * n_bands // (4 * nside - 1)
    sector = (p - first) * n_sectors // length
    return np.bincount(band * n_sectors + sector, weights=hist, minlength=n_bands * n_sectors)


def two_sample_chi2(a, b):
    """Chi-square test that two histograms come from one distribution (their
    totals may differ); cells empty in both are skipped."""
    from scipy.stats import chi2 as chi2_dist
    keep = (a + b) > 0
    a, b = a[keep], b[keep]
    na, nb = a.sum(), b.sum()
    stat = float(np.sum((np.sqrt(nb / na) * a - np.sqrt(na / nb) * b) ** 2 / (a + b)))
    dof = int(len(a) - 1)
    return stat, dof, float(chi2_dist.sf(stat, dof))


def run_uneven(args):
    """Uneven batched propagation with secondaries: 10^7 mixed nuclei through a
    512^3 binary32 grid (B_rms drawn per run), pair + adiabatic + pion +
    photodisintegration (nucleons join the device work queue), path budgets
    log-uniform in [1 Mpc, 2 Gpc]; mixed precision, host-driven and
    graph-captured round loops."""
    import torch
    from paper_1307_2643_gb300 import crp
    from paper_1307_2643_gb300.build import build

    torch.cuda.set_device(0)
    build()
    crp.use_torch_allocator(0)
    w = workloads.UNEVEN_SECONDARIES
    n = args.n or w["n"]
    inj, brms = workloads.uneven_secondaries(n=n)
    inj = crp.host_injection(inj)
    cap = int(n * 1.5) + 4096
    ctx = crp.crp_context_create(0, w["seed"], cap)
    t0 = time.perf_counter()
    grid = crp.crp_grid_create(ctx, crp.grid_desc(w["grid_n"], w["spacing"], dtype=crp.F32,
                                                  source=crp.GRID_TURBULENT, lmin=w["lmin"],
                                                  lmax=w["lmax"], brms=brms, seed=w["seed"]))
    torch.cuda.synchronize()
    t_grid = time.perf_counter() - t0
    tables = crp.crp_tables_build(ctx, crp.tables_desc(n=1000))
    dev = {k: torch.from_numpy(v).cuda() for k, v in inj.items()}
    arr = crp.candidate_arrays(dev, on_device=True)
    flags = crp.PAIR | crp.ADIABATIC | crp.PION | crp.PHOTODIS | crp.EMIN | crp.OBSERVER
    results = {}
    for loop in ("host", "graph"):
        mods = crp.modules(precision=crp.MIXED, flags=flags, tol=w["tol"], h_min=w["h_min"],
                           h_max=w["h_max"], beta_ad=H0_OVER_C, e_min=w["e_min"], tables=tables,
                           observer_radius=w["observer_r"], use_graph=1 if loop == "graph" else 0)
        runs = []
        for k in range(args.warmup + args.steps):
            crp.crp_candidates_clear(ctx)
            crp.crp_candidates_inject(ctx, arr, n)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            status, st = crp.crp_propagate(ctx, grid, mods, raise_on_error=False)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if status != crp.OK:
                raise RuntimeError(f"propagate status {status}: {crp.lib().crp_last_error()}")
            if k >= args.warmup:
                runs.append((dt, st))
        dt = sum(r[0] for r in runs) / len(runs)
        st = runs[-1][1]
        results[loop] = {"seconds": dt, "accepted_steps": st.accepted_steps,
                         "steps_per_s": st.accepted_steps / dt,
                         "rejected_trials": st.rejected_trials, "rounds": st.launches,
                         "photodisintegrations": st.n_pd, "pion_events": st.n_pion,
                         "secondaries": st.n_secondaries, "nucleons_below_emin": st.n_dropped,
                         "detected": st.n_detected, "kernel_ms": st.kernel_ms}
    rec = crp.crp_collect(ctx, crp.COLLECT_ALL)
    nacc = np.sort(rec["n_acc"])
    crp.crp_tables_destroy(tables)
    crp.crp_grid_destroy(grid)
    crp.crp_context_destroy(ctx)
    print(json.dumps({
        "workload": w["name"], "metric": METRIC, "unit": UNIT, "candidates": n,
        "brms_nG": brms, "grid": "512^3 f32 (2.1 GB nodes + 17.2 GB cell records)",
        "grid_setup_s": t_grid, "steps": args.steps, "warmup": args.warmup,
        "value": results["host"]["steps_per_s"], "loops": results,
        "records": int(len(rec)),
        "accepted_steps_per_candidate": {"median": float(np.median(nacc)),
                                         "p99": float(nacc[int(0.99 * (len(nacc) - 1))]),
                                         "max": int(nacc[-1])},
    }))


def run_cosmology(args):
    """1D mode with cosmology on the paper's comparison setup (sources uniform
    in comoving volume up to 4000 Mpc, spectral index -2.2, pure protons and
    pure iron): 1D throughput, and a 3D run without field corrected a
    posteriori against the 1D spectrum."""
    import torch
    from scipy.stats import ks_2samp
    from paper_1307_2643_gb300 import crp
    from paper_1307_2643_gb300.build import build

    torch.cuda.set_device(0)
    build()
    crp.use_torch_allocator(0)
    n = args.n or 200_000  # sources per species (iron: up to 56 nucleons each)
    g = workloads.rng(workloads.MASTER_SEED + 6)
    out = {"workload": "cosmology_1d_4000Mpc_index2.2", "metric": "1D candidate-steps/s"}
    flags = crp.PAIR | crp.ADIABATIC | crp.PION | crp.PHOTODIS | crp.DECAY | crp.EMIN
    cos = crp.cosmology()
    ctx = crp.crp_context_create(0, workloads.MASTER_SEED + 6, 64 * n)
    tables = crp.crp_tables_build(ctx, crp.tables_desc(n=1000))
    m1 = crp.modules(flags=flags, e_min=1e18, tables=tables)
    for name, A, Z in (("proton", 1, 1), ("iron", 56, 26)):
        d = 4000.0 * g.random(n) ** (1.0 / 3.0)
        u = g.random(n)
        lo, hi = 1e18, 1e21
        E = lo * (1 - u * (1 - (lo / hi) ** 1.2)) ** (-1 / 1.2)
        z = crp.crp_redshift_of_distance(cos, crp.MPC_M, d)
        inj = crp.host_injection(dict(x=z, y=np.zeros(n), z=np.zeros(n), ux=np.zeros(n),
                                      uy=np.zeros(n), uz=np.ones(n), E=E, A=np.full(n, A),
                                      Z=np.full(n, Z)))
        rates = []
        for k in range(args.warmup + args.steps):
            crp.crp_candidates_clear(ctx)
            crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), n)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st = crp.crp_propagate_1d(ctx, cos, m1)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if k >= args.warmup:
                rates.append(st.accepted_steps / dt)
        out[name] = {"sources": n, "accepted_steps": st.accepted_steps,
                     "steps_per_s": float(np.median(rates)), "detected": st.n_detected,
                     "photodisintegrations": st.n_pd, "secondaries": st.n_secondaries,
                     "rounds": st.launches}
    # 3D without field, corrected a posteriori, against 1D (a bounded sample)
    m = max(1000, n // 20)
    d = np.sort(4000.0 * g.random(m) ** (1.0 / 3.0))
    u = g.random(m)
    E = 1e18 * (1 - u * (1 - (1e-3) ** 1.2)) ** (-1 / 1.2)
    res = {}
    grid = crp.crp_grid_create(ctx, crp.grid_desc((4, 4, 4), 1.0, dtype=crp.F64,
                                                  data=np.zeros((4, 4, 4, 3))))
    for name, A, Z in (("proton", 1, 1), ("iron", 56, 26)):
        ids = np.arange(m, dtype=np.uint64)
        crp.crp_candidates_clear(ctx)
        inj = crp.host_injection(dict(id=ids, x=d + 1.0, y=np.zeros(m), z=np.zeros(m),
                                      ux=-np.ones(m), uy=np.zeros(m), uz=np.zeros(m), E=E,
                                      A=np.full(m, A), Z=np.full(m, Z)))
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), m)
        m3 = crp.modules(precision=crp.FP64, flags=crp.PAIR | crp.PION | crp.PHOTODIS |
                         crp.DECAY | crp.EMIN | crp.OBSERVER, observer_radius=1.0, h_max=10.0,
                         h_min=1e-3, e_min=1e18, tables=tables)
        t0 = time.perf_counter()
        crp.crp_propagate(ctx, grid, m3)
        rec = crp.crp_collect(ctx, crp.COLLECT_ALL)
        idx = {int(i): k for k, i in enumerate(rec["id"])}
        det = np.nonzero(rec["status"] == crp.DETECTED)[0]
        root = []
        for k in det:
            cur = k
            while rec["generation"][cur] > 0:
                cur = idx[int(rec["parent_id"][cur])]
            root.append(cur)
        src = rec[np.array(root, dtype=np.int64)]
        r3 = rec[det]
        Ec, _, _, nk = crp.crp_cosmology_correct(ctx, cos, m1, r3["id"], r3["s"] + 1.0, src["E0"],
                                                 src["A0"], src["Z0"])
        t_corr = time.perf_counter() - t0
        crp.crp_candidates_clear(ctx)
        zz = crp.crp_redshift_of_distance(cos, crp.MPC_M, d + 1.0)
        inj1 = crp.host_injection(dict(id=ids, x=zz, y=np.zeros(m), z=np.zeros(m), ux=np.zeros(m),
                                       uy=np.zeros(m), uz=np.ones(m), E=E, A=np.full(m, A),
                                       Z=np.full(m, Z)))
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj1), m)
        crp.crp_propagate_1d(ctx, cos, m1)
        r1 = crp.crp_collect(ctx, crp.COLLECT_DETECTED)
        corrected = Ec[nk > 0]
        res[name] = {"sources": m, "observed_3d": int(len(r3)), "corrected": int(len(corrected)),
                     "arrived_1d": int(len(r1)), "seconds_3d_plus_correction": t_corr,
                     "ks_distance_corrected_vs_1d":
                         float(ks_2samp(np.log(corrected), np.log(r1["E"])).statistic),
                     "ks_distance_uncorrected_vs_1d":
                         float(ks_2samp(np.log(r3["E"]), np.log(r1["E"])).statistic)}
    out["correction"] = res
    crp.crp_grid_destroy(grid)
    crp.crp_tables_destroy(tables)
    crp.crp_context_destroy(ctx)
    print(json.dumps(out))


HYBRID_MAX_DEG = 0.5   # a bin's surrogate columns are used where its validated median is at most this


def lens_bin_of(R, w):
    """Rigidity bin of the lens (log bins over [r_lo, r_hi])."""
    t = np.log(R / w["r_lo"]) / np.log(w["r_hi"] / w["r_lo"]) * w["n_bins"]
    return np.clip(np.floor(t).astype(np.int64), 0, w["n_bins"] - 1)


def chaos_floor(crp, ctx, grid, w, analytic, delta_deg, bands, triplets=500, seed=3):
    """Interpolation floor of the border-direction map at sample spacing
    delta_deg, per rigidity band: arrival directions u - delta, u, u + delta
    on a great circle (one rigidity, log-uniform in the band) are back-tracked
    by the binary64 path, and the floor is the median angle between the
    border direction of u and the normalised mean of its two neighbours'.
    A map smooth at that scale gives O(delta^2); structure below the spacing
    gives an error no fit to samples that far apart can be expected to beat."""
    mods = crp.modules(precision=crp.FP64, tol=w["tol"], h_min=w["h_min"], h_max=w["h_max"],
                       field_unit_T=crp.MICROGAUSS_T, length_unit_m=crp.KPC_M,
                       border_radius=w["border_r"], **analytic)
    g = np.random.default_rng(seed)
    out = {}
    d = np.radians(delta_deg)
    k = triplets
    for lo, hi in zip(bands[:-1], bands[1:]):
        u = g.normal(size=(k, 3))
        u /= np.linalg.norm(u, axis=1)[:, None]
        v = np.cross(u, g.normal(size=(k, 3)))
        v /= np.linalg.norm(v, axis=1)[:, None]
        R = 10 ** g.uniform(lo, hi, k)
        dd = np.concatenate([u, np.cos(d) * u + np.sin(d) * v, np.cos(d) * u - np.sin(d) * v])
        RR, m = np.concatenate([R, R, R]), 3 * k
        inj = crp.host_injection(dict(x=np.full(m, w["earth"][0]), y=np.full(m, w["earth"][1]),
                                      z=np.full(m, w["earth"][2]), ux=dd[:, 0], uy=dd[:, 1],
                                      uz=dd[:, 2], E=RR, A=np.ones(m), Z=np.ones(m),
                                      q=-np.ones(m)))
        crp.crp_candidates_clear(ctx)
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), m)
        crp.crp_propagate(ctx, grid, mods)
        rec = crp.crp_collect(ctx, crp.COLLECT_ALL)
        rec = rec[np.argsort(rec["id"], kind="stable")]
        b0, bp, bm = rec["u"][:k], rec["u"][k:2 * k], rec["u"][2 * k:]
        mid = bp + bm
        mid /= np.linalg.norm(mid, axis=1)[:, None]
        out[f"{lo:.1f}-{hi:.1f}"] = round(float(np.median(np.degrees(
            np.arccos(np.clip(np.sum(b0 * mid, axis=1), -1.0, 1.0))))), 3)
    return out


def run_galactic(args, keep=False):
    """Galactic workload: back-track antiprotons from Earth through the
    synthetic galactic field (disk + halo + 256^3 random component), train the
    BF16 MLP surrogate on the border directions, and build the nside-64,
    100-bin lens by back-tracking and by the surrogate.  With keep=True the
    lenses (and the context that owns them) are returned for further use
    instead of printed and released."""
    import torch
    from paper_1307_2643_gb300 import crp
    from paper_1307_2643_gb300.build import build

    torch.cuda.set_device(0)
    build()
    crp.use_torch_allocator(0)
    wr = workloads.GALACTIC_LENS  # the random component's grid
    galaxy = getattr(args, "galaxy", "disk_halo_random")
    w = wr if galaxy == "disk_halo_random" else workloads.GALACTIC_MULTIARM
    wname = w["name"] + ("_random256" if galaxy == "multiarm_random" else "")
    n_all = args.n_train + args.n_test
    dx, lmin, org = workloads.galactic_grid_geometry(wr["grid_n"][0], wr["box"])
    m = 2_000_000  # border candidates sent through both lenses
    ctx = crp.crp_context_create(0, w["seed"], max(n_all, m) + 1024)
    if galaxy == "multiarm":  # the analytic field over an all-zero 4^3 grid
        zn = (4, 4, 4)
        grid = crp.crp_grid_create(ctx, crp.grid_desc(zn, 20.0, origin=(-40.0, -40.0, -40.0),
                                                      dtype=crp.F32, data=np.zeros(zn + (3,))))
    else:
        grid = crp.crp_grid_create(ctx, crp.grid_desc(wr["grid_n"], dx, origin=org, dtype=crp.F32,
                                                      source=crp.GRID_TURBULENT, lmin=lmin,
                                                      lmax=wr["lmax"], brms=wr["brms"],
                                                      seed=wr["seed"]))
    if galaxy == "disk_halo_random":
        analytic = dict(flags=crp.GALACTIC | crp.BORDER, galactic=w["disk"])
    else:
        analytic = dict(flags=crp.GMF | crp.BORDER, gmf=workloads.multiarm_gmf_params())
    mods = crp.modules(precision=crp.MIXED, tol=w["tol"], h_min=w["h_min"], h_max=w["h_max"],
                       field_unit_T=crp.MICROGAUSS_T, length_unit_m=crp.KPC_M,
                       border_radius=w["border_r"], **analytic)
    dirs, R = workloads.backtrack_directions(n_all, w["r_lo"], w["r_hi"], w["seed"] + 1)
    inj = crp.host_injection(dict(x=np.full(n_all, w["earth"][0]), y=np.full(n_all, w["earth"][1]),
                                  z=np.full(n_all, w["earth"][2]), ux=dirs[:, 0], uy=dirs[:, 1],
                                  uz=dirs[:, 2], E=R, A=np.ones(n_all), Z=np.ones(n_all),
                                  q=-np.ones(n_all)))
    crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), n_all)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, st = crp.crp_propagate(ctx, grid, mods)
    torch.cuda.synchronize()
    t_bt = time.perf_counter() - t0
    rec = crp.crp_collect(ctx, crp.COLLECT_ALL)
    rec = rec[np.argsort(rec["id"], kind="stable")]
    ok = rec["status"] == crp.AT_BORDER
    # network inputs (direction at Earth, log10 R - 19), the surrogate's input convention
    x_all = np.concatenate([dirs, (np.log10(R) - 19.0)[:, None]], axis=1).astype(np.float32)
    t_all = rec["u"].astype(np.float32)
    tr = np.nonzero(ok[: args.n_train])[0]
    te = args.n_train + np.nonzero(ok[args.n_train:])[0]
    # validation samples (from the training draw, not trained on): they decide
    # which lens bins the hybrid lens takes from the surrogate
    n_val = min(200_000, len(tr) // 20) // 128 * 128
    va, tr = tr[:n_val], tr[n_val:]
    # ---- training ---------------------------------------------------------
    mlp = crp.crp_mlp_create(ctx, 4, 256, 4, w["seed"])
    B = args.batch
    g = workloads.rng(w["seed"] + 5)
    shuf = tr[g.permutation(len(tr))]
    n_batches = len(tr) // B
    xd = torch.from_numpy(x_all[shuf[: n_batches * B]]).cuda()
    td = torch.from_numpy(t_all[shuf[: n_batches * B]]).cuda()
    steps, total = 0, args.epochs * n_batches
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ep in range(args.epochs):
        for i, b in enumerate(g.permutation(n_batches)):
            # linear warm-up over 200 steps, cosine decay to zero
            lr = args.lr * 0.5 * (1 + np.cos(np.pi * steps / total)) * min(1.0, (steps + 1) / 200)
            b0 = int(b) * B
            loss = crp.crp_mlp_train_step(mlp, xd[b0:b0 + B], td[b0:b0 + B], B, lr,
                                          want_loss=(i == n_batches - 1))
            steps += 1
        losses.append(round(loss, 5))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    # ---- held-out accuracy and inference throughput -----------------------
    n_te = (len(te) // 128) * 128
    xt = torch.from_numpy(x_all[te[:n_te]]).cuda()
    yt = torch.zeros((n_te, 3), dtype=torch.float32, device="cuda")
    # inference throughput of both forward kernels (fused tensor-core, layered GEMMs)
    t_paths = {}
    for path, name in ((crp.MLP_PATH_LAYERED, "layered_mma_sync"),
                       (crp.MLP_PATH_AUTO, "fused_tcgen05")):
        crp.crp_mlp_set_forward_path(mlp, path)
        crp.crp_mlp_forward(mlp, xt, yt, n_te)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            crp.crp_mlp_forward(mlp, xt, yt, n_te)
        torch.cuda.synchronize()
        t_paths[name] = (time.perf_counter() - t0) / 5
    t_inf = t_paths["fused_tcgen05"]
    yh = yt.cpu().numpy().astype(np.float64)
    tt = t_all[te[:n_te]].astype(np.float64)
    cosang = np.sum(yh * tt, axis=1) / (np.linalg.norm(yh, axis=1) * np.linalg.norm(tt, axis=1))
    ang = np.degrees(np.arccos(np.clip(cosang, -1.0, 1.0)))
    Rt = R[te[:n_te]]
    ident = np.degrees(np.arccos(np.clip(np.sum(dirs[te[:n_te]] * tt, axis=1)
                                         / np.linalg.norm(tt, axis=1), -1.0, 1.0)))
    # per lens bin: validated median (claims) and held-out median
    crp.crp_mlp_set_forward_path(mlp, crp.MLP_PATH_AUTO)
    xv = torch.from_numpy(x_all[va]).cuda()
    yv = torch.zeros((len(va), 3), dtype=torch.float32, device="cuda")
    crp.crp_mlp_forward(mlp, xv, yv, len(va))
    tv = t_all[va].astype(np.float64)
    yvh = yv.cpu().numpy().astype(np.float64)
    ang_v = np.degrees(np.arccos(np.clip(np.sum(yvh * tv, axis=1) / (
        np.linalg.norm(yvh, axis=1) * np.linalg.norm(tv, axis=1)), -1.0, 1.0)))
    bv, bt = lens_bin_of(R[va], w), lens_bin_of(Rt, w)
    val_med = np.full(w["n_bins"], np.inf)
    test_med = np.full(w["n_bins"], np.inf)
    for b in range(w["n_bins"]):
        if (bv == b).sum() >= 100:
            val_med[b] = np.median(ang_v[bv == b])
        if (bt == b).sum() >= 100:
            test_med[b] = np.median(ang[bt == b])
    claim = val_med <= HYBRID_MAX_DEG
    # chaos floor per 0.1-decade band: at the training set's angular spacing
    # per lens bin, and at 0.2 deg
    bands = np.round(np.arange(18.0, 20.001, 0.1), 1)
    spacing = float(np.degrees(np.sqrt(4 * np.pi / (len(tr) / w["n_bins"]))))
    floor_train = chaos_floor(crp, ctx, grid, w, analytic, spacing, bands)
    floor_02 = chaos_floor(crp, ctx, grid, w, analytic, 0.2, bands)
    q_edges = 10.0 ** np.arange(18.0, 20.01, 0.25)
    by_q = {f"{np.log10(lo):.2f}-{np.log10(hi):.2f}":
            [round(float(np.median(ang[(Rt >= lo) & (Rt < hi)])), 3),
             round(float(np.median(ident[(Rt >= lo) & (Rt < hi)])), 3)]
            for lo, hi in zip(q_edges[:-1], q_edges[1:])}
    # ---- lens builds -------------------------------------------------------
    ldirs, lE, lbins = workloads.lens_samples(w["n_bins"], args.lens_per_bin, w["r_lo"], w["r_hi"],
                                              w["seed"] + 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lens_bt, lst = crp.crp_lens_build(ctx, grid, mods, w["nside"], w["n_bins"], w["r_lo"],
                                      w["r_hi"], w["earth"], ldirs, lE, lbins)
    torch.cuda.synchronize()
    t_lens_bt = time.perf_counter() - t0
    t0 = time.perf_counter()
    lens_sg = crp.crp_lens_build_surrogate(ctx, mlp, w["nside"], w["n_bins"], w["r_lo"],
                                           w["r_hi"], ldirs, lE, lbins)
    torch.cuda.synchronize()
    t_lens_sg = time.perf_counter() - t0
    # hybrid lens: back-track only the samples of the bins the surrogate does
    # not claim, take the claimed bins from the surrogate
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    keep_bt = ~claim[lbins]
    if claim.all():
        lens_hy = crp.crp_lens_merge(lens_sg, lens_sg, claim)
        torch.cuda.synchronize()
    elif claim.any():
        part_bt, _ = crp.crp_lens_build(ctx, grid, mods, w["nside"], w["n_bins"], w["r_lo"],
                                        w["r_hi"], w["earth"], ldirs[keep_bt], lE[keep_bt],
                                        lbins[keep_bt])
        part_sg = crp.crp_lens_build_surrogate(ctx, mlp, w["nside"], w["n_bins"], w["r_lo"],
                                               w["r_hi"], ldirs[~keep_bt], lE[~keep_bt],
                                               lbins[~keep_bt])
        lens_hy = crp.crp_lens_merge(part_bt, part_sg, claim)
        torch.cuda.synchronize()
        crp.crp_lens_destroy(part_bt)
        crp.crp_lens_destroy(part_sg)
    else:
        lens_hy = crp.crp_lens_merge(lens_bt, lens_sg, claim)
        torch.cuda.synchronize()
    t_lens_hy = time.perf_counter() - t0 + (0.0 if claim.any() else t_lens_bt)
    if claim.all():
        t_lens_hy += t_lens_sg
    # arrival maps of an isotropic border population through both lenses
    bd, bR = workloads.backtrack_directions(m, w["r_lo"], w["r_hi"], w["seed"] + 4)
    inj2 = crp.host_injection(dict(x=np.zeros(m), y=np.zeros(m), z=np.zeros(m), ux=bd[:, 0],
                                   uy=bd[:, 1], uz=bd[:, 2], E=bR, A=np.ones(m), Z=np.ones(m)))
    maps = {}
    for name, lens in (("backtracked", lens_bt), ("surrogate", lens_sg), ("hybrid", lens_hy)):
        crp.crp_candidates_clear(ctx)
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj2), m)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        crp.crp_lens_apply(ctx, lens, crp.COLLECT_ALL)
        torch.cuda.synchronize()
        maps[name + "_apply_s"] = time.perf_counter() - t0
        maps[name] = crp.crp_histogram_healpix(ctx, crp.COLLECT_ALL, w["nside"], 1).astype(np.float64)
    a, b = maps["backtracked"], maps["surrogate"]
    ca, cb = coarse_ring_map(a, w["nside"]), coarse_ring_map(b, w["nside"])
    chi2, dof, pval = two_sample_chi2(ca, cb)
    corr = float(np.corrcoef(ca, cb)[0, 1])
    ch = coarse_ring_map(maps["hybrid"], w["nside"])
    chi2_h, dof_h, pval_h = two_sample_chi2(ca, ch)
    summary = {
        "workload": wname, "metric": "galactic back-tracking and lens surrogate",
        "backtrack": {"candidates": n_all, "accepted_steps": st.accepted_steps,
                      "rejected_trials": st.rejected_trials, "seconds": t_bt,
                      "steps_per_s": st.accepted_steps / t_bt,
                      "at_border_fraction": float(ok.mean()), "precision": "mixed"},
        "mlp": {"train_samples": int(n_batches * B), "epochs": args.epochs, "batch": B, "steps": steps,
                "train_seconds": t_train, "train_samples_per_s": steps * B / t_train,
                "loss_per_epoch": losses, "test_samples": n_te,
                "median_angle_deg": float(np.median(ang)),
                "p90_angle_deg": float(np.percentile(ang, 90)),
                "median_angle_deg_no_lens": float(np.median(ident)),
                "median_angle_deg_by_log10R_net_vs_no_lens": by_q,
                "inference_samples_per_s": n_te / t_inf,
                "inference_samples_per_s_by_kernel": {k: n_te / v for k, v in t_paths.items()},
                "inference_tflops_by_kernel": {k: n_te * 2 * (4 * 256 + 3 * 256 * 256 + 256 * 3)
                                               / v / 1e12 for k, v in t_paths.items()}},
        "lens": {"nside": w["nside"], "n_bins": w["n_bins"], "samples": int(len(lE)),
                 "build_backtrack_s": t_lens_bt, "build_surrogate_s": t_lens_sg,
                 "backtrack_steps": lst.accepted_steps, "apply_s": {k: maps[k + "_apply_s"]
                 for k in ("backtracked", "surrogate")},
                 "map_cells": int(len(ca)), "map_chi2": chi2, "map_dof": dof, "map_p": pval,
                 "map_correlation": corr,
                 "observed_fraction": {"backtracked": float(a.sum() / m),
                                       "surrogate": float(b.sum() / m)}},
        "hybrid_lens": {
            "rule": f"surrogate columns in the lens bins whose validated median is <= "
                    f"{HYBRID_MAX_DEG} deg ({n_val} validation samples, not trained on), "
                    "back-tracked columns elsewhere",
            "claimed_bins": [int(b) for b in np.nonzero(claim)[0]],
            "lowest_claimed_rigidity_V": (float(w["r_lo"] * (w["r_hi"] / w["r_lo"]) ** (
                np.nonzero(claim)[0][0] / w["n_bins"])) if claim.any() else None),
            "held_out_median_deg_in_claimed_bins": (float(np.median(ang[claim[bt]]))
                                                    if claim.any() else None),
            "held_out_worst_bin_median_deg_in_claimed_bins": (float(test_med[claim].max())
                                                              if claim.any() else None),
            "validated_median_deg_by_bin": [round(float(v), 3) for v in val_med],
            "build_s": t_lens_hy, "build_backtrack_s": t_lens_bt,
            "observed_fraction": float(maps["hybrid"].sum() / m),
            "map_vs_backtracked": {"chi2": chi2_h, "dof": dof_h, "p": pval_h},
        },
        "chaos_floor_deg": {
            "definition": "median angle between the border direction of an arrival direction "
                          "and the normalised mean of those of its two neighbours delta away "
                          "on a great circle (same rigidity; binary64 back-tracking): the "
                          "interpolation error at sample spacing delta, per 0.1-decade "
                          "rigidity band (log10 R/V)",
            "training_spacing_deg": spacing, "at_training_spacing": floor_train,
            "at_0.2_deg": floor_02,
            "bands_where_floor_allows_0.5deg": [k for k, v in floor_train.items() if v <= 0.5],
        },
    }
    if keep:
        return dict(ctx=ctx, grid=grid, mlp=mlp, lens_bt=lens_bt, lens_sg=lens_sg,
                    lens_hy=lens_hy, summary=summary, t_lens_bt=t_lens_bt, t_lens_sg=t_lens_sg,
                    t_lens_hy=t_lens_hy)
    for lens in (lens_bt, lens_sg, lens_hy):
        crp.crp_lens_destroy(lens)
    crp.crp_mlp_destroy(mlp)
    crp.crp_grid_destroy(grid)
    crp.crp_context_destroy(ctx)
    print(json.dumps(summary))


def run_e2e(args):
    """End to end at scale: 10^8 candidates of the mixed workload's
    composition propagated through its 256^3 field to the observer sphere,
    then mapped to Earth through the galactic lens built by back-tracking and
    through the lens built from the trained surrogate; arrival maps, observed
    spectra (two-sample KS) and the throughput of each path."""
    import torch
    from scipy.stats import ks_2samp
    from paper_1307_2643_gb300 import crp

    gal = run_galactic(args, keep=True)
    w = workloads.MIXED_INTERACTIONS
    n = args.n or 100_000_000
    chunk = 10_000_000
    ctx = crp.crp_context_create(0, w["seed"], n + 4096)
    grid = crp.crp_grid_create(ctx, crp.grid_desc(w["grid_n"], w["spacing"], dtype=crp.F32,
                                                  source=crp.GRID_TURBULENT, lmin=w["lmin"],
                                                  lmax=w["lmax"], brms=w["brms"], seed=w["seed"]))
    tables = crp.crp_tables_build(ctx, crp.tables_desc(n=1000))
    t0 = time.perf_counter()
    for k in range(0, n, chunk):
        m = min(chunk, n - k)
        inj = workloads.mixed_interactions(n=m, seed=w["seed"] + 1000 + k // chunk)
        inj["id"] = inj["id"] + np.uint64(k)
        inj = crp.host_injection(inj)
        crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), m)
    torch.cuda.synchronize()
    t_inject = time.perf_counter() - t0
    mods = modules_for(crp, crp.MIXED, tables)
    t0 = time.perf_counter()
    _, st = crp.crp_propagate(ctx, grid, mods)
    torch.cuda.synchronize()
    t_prop = time.perf_counter() - t0
    nside = workloads.GALACTIC_LENS["nside"]
    sky = crp.crp_histogram_healpix(ctx, crp.COLLECT_DETECTED, nside, 0).astype(np.float64)
    paths = {}
    for name in ("backtracked", "surrogate", "hybrid"):
        lens = gal[{"backtracked": "lens_bt", "surrogate": "lens_sg", "hybrid": "lens_hy"}[name]]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        crp.crp_lens_apply(ctx, lens, crp.COLLECT_DETECTED)
        torch.cuda.synchronize()
        t_apply = time.perf_counter() - t0
        hist = crp.crp_histogram_healpix(ctx, crp.COLLECT_DETECTED, nside, 1).astype(np.float64)
        rec = crp.crp_collect(ctx, crp.COLLECT_DETECTED)
        seen = rec["lens_pixel"] < 12 * nside * nside
        paths[name] = dict(hist=hist, E=rec["E"][seen], t_apply=t_apply,
                           observed=int(seen.sum()), detected=int(len(rec)))
    a, b = paths["backtracked"], paths["surrogate"]
    ca, cb = coarse_ring_map(a["hist"], nside), coarse_ring_map(b["hist"], nside)
    chi2, dof, pval = two_sample_chi2(ca, cb)
    ks = ks_2samp(a["E"], b["E"])
    hy = paths["hybrid"]
    ks_h = ks_2samp(a["E"], hy["E"])
    chh = coarse_ring_map(hy["hist"], nside)
    chi2_h, dof_h, pval_h = two_sample_chi2(ca, chh)
    summary = {
        "workload": "e2e_1e8_mixed_256cube_then_galactic_lens",
        "metric": "end-to-end propagation + lens (plain vs surrogate)",
        "extragalactic": {"candidates": n, "inject_s": t_inject, "seconds": t_prop,
                          "accepted_steps": st.accepted_steps,
                          "steps_per_s": st.accepted_steps / t_prop,
                          "detected": int(st.n_detected), "pion_events": int(st.n_pion)},
        "lens_build_s": {"backtracked": gal["t_lens_bt"], "surrogate": gal["t_lens_sg"],
                         "hybrid": gal["t_lens_hy"]},
        "lens_apply_s": {"backtracked": a["t_apply"], "surrogate": b["t_apply"],
                         "hybrid": hy["t_apply"]},
        "observed_at_earth": {"backtracked": a["observed"], "surrogate": b["observed"],
                              "hybrid": hy["observed"]},
        "hybrid_vs_backtracked": {"spectrum_ks": {"statistic": float(ks_h.statistic),
                                                  "p": float(ks_h.pvalue)},
                                  "arrival_map": {"chi2": chi2_h, "dof": dof_h, "p": pval_h}},
        "arrival_map": {"cells": int(len(ca)), "chi2": chi2, "dof": dof, "p": pval,
                        "correlation": float(np.corrcoef(ca, cb)[0, 1]),
                        "sky_before_lens_events": float(sky.sum())},
        "spectrum_ks": {"statistic": float(ks.statistic), "p": float(ks.pvalue)},
        "galactic": gal["summary"],
    }
    crp.crp_tables_destroy(tables)
    crp.crp_grid_destroy(grid)
    crp.crp_context_destroy(ctx)
    for lens in (gal["lens_bt"], gal["lens_sg"], gal["lens_hy"]):
        crp.crp_lens_destroy(lens)
    crp.crp_mlp_destroy(gal["mlp"])
    crp.crp_grid_destroy(gal["grid"])
    crp.crp_context_destroy(gal["ctx"])
    print(json.dumps(summary))


MLP_FLOPS_PER_SAMPLE_FWD = 2 * (4 * 256 + 3 * 256 * 256 + 256 * 3)  # 4 -> 256^3 -> 3


def run_train(args):
    """MLP lens surrogate training step (4 inputs, 4 hidden layers of 256, batch
    16384, Adam) on synthetic inputs of the surrogate's shape (isotropic
    directions, log10 R - 19 in [-1, 1], smooth targets): the tensor-core path
    replayed from its CUDA graph against the layered mma.sync path.  Time per
    step by CUDA events over `steps` steps after `warmup`."""
    import torch
    from paper_1307_2643_gb300 import crp
    from paper_1307_2643_gb300.build import build

    torch.cuda.set_device(0)
    build()
    crp.use_torch_allocator(0)
    B, nb = 16384, 16
    g = workloads.rng(workloads.MASTER_SEED + 8)
    ux, uy, uz = workloads.isotropic(g, B * nb)
    lr10 = g.uniform(-1.0, 1.0, B * nb)
    x = np.stack([ux, uy, uz, lr10], axis=1).astype(np.float32)
    ang = 0.8 * (1.0 - lr10)
    t = np.stack([np.cos(ang) * ux - np.sin(ang) * uy, np.sin(ang) * ux + np.cos(ang) * uy, uz],
                 axis=1).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    ctx = crp.crp_context_create(0, workloads.MASTER_SEED + 8, 1024)
    out = {"workload": "mlp_train_4x256x4_batch16384", "metric": "training samples/s",
           "flops_per_sample": 3 * MLP_FLOPS_PER_SAMPLE_FWD}
    steps, warm = max(args.steps, 1) * 50, max(args.warmup, 1) * 10
    for path, name in ((crp.MLP_PATH_AUTO, "tcgen05_graph"), (crp.MLP_PATH_LAYERED, "mma_sync")):
        mlp = crp.crp_mlp_create(ctx, 4, 256, 4, workloads.MASTER_SEED + 8)
        crp.crp_mlp_set_forward_path(mlp, path)
        for k in range(warm):
            b = k % nb
            crp.crp_mlp_train_step(mlp, xd[b * B:(b + 1) * B], td[b * B:(b + 1) * B], B, 1e-3,
                                   want_loss=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(steps):
            b = k % nb
            crp.crp_mlp_train_step(mlp, xd[b * B:(b + 1) * B], td[b * B:(b + 1) * B], B, 1e-3,
                                   want_loss=False)
        e1.record()
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) / 1e3 / steps
        loss = crp.crp_mlp_train_step(mlp, xd[:B], td[:B], B, 0.0)
        out[name] = {"us_per_step": dt * 1e6, "samples_per_s": B / dt,
                     "tflops": B * 3 * MLP_FLOPS_PER_SAMPLE_FWD / dt / 1e12, "steps": steps,
                     "loss_after": loss}
        crp.crp_mlp_destroy(mlp)
    crp.crp_context_destroy(ctx)
    print(json.dumps(out))


LENS_HBM_BYTES_PER_CANDIDATE = 4 + 4 + 8 + 24 + 8 + 4   # status, Z, E, u, id read; pixel written


def run_lens(args):
    """Lens application alone: a lens of the galactic workload's shape (nside
    64, 100 rigidity bins, 49152 samples per bin, built by back-tracking
    through a zero field, so every column holds its own pixel), applied to
    n candidates of isotropic direction and log-uniform rigidity.  Timed with
    CUDA events on the launching stream, L2 flushed before every launch."""
    import torch
    from paper_1307_2643_gb300 import crp
    from paper_1307_2643_gb300.build import build
    build()
    crp.use_torch_allocator(0)
    W = workloads.GALACTIC_LENS
    n = args.n or (1 << 24)
    nside, nb = W["nside"], W["n_bins"]
    ctx = crp.crp_context_create(0, 7, max(n, 16))
    zn = (4, 4, 4)
    g = crp.crp_grid_create(ctx, crp.grid_desc(zn, 20.0, origin=(-40.0, -40.0, -40.0),
                                               dtype=crp.F32, data=np.zeros(zn + (3,))))
    mods = crp.modules(precision=crp.MIXED, flags=crp.BORDER, tol=W["tol"], h_min=W["h_min"],
                       h_max=W["h_max"], field_unit_T=crp.MICROGAUSS_T, length_unit_m=crp.KPC_M,
                       border_radius=W["border_r"], max_steps=2_000_000)
    dirs, E, bins = workloads.lens_samples(nb, args.lens_per_bin, W["r_lo"], W["r_hi"], W["seed"])
    lens, _ = crp.crp_lens_build(ctx, g, mods, nside, nb, W["r_lo"], W["r_hi"], W["earth"],
                                 dirs, E, bins)
    d, R = workloads.backtrack_directions(n, W["r_lo"], W["r_hi"], W["seed"] + 5)
    inj = crp.host_injection(dict(x=np.zeros(n), y=np.zeros(n), z=np.zeros(n), ux=d[:, 0],
                                  uy=d[:, 1], uz=d[:, 2], E=R, A=np.ones(n), Z=np.ones(n)))
    crp.crp_candidates_inject(ctx, crp.candidate_arrays(inj), n)
    s = torch.cuda.current_stream()
    for _ in range(args.warmup):
        crp.crp_lens_apply(ctx, lens, crp.COLLECT_ALL, s.cuda_stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    ts = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        crp.crp_lens_apply(ctx, lens, crp.COLLECT_ALL, s.cuda_stream)
        e1.record(s)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    clocks = clk.stop()
    rec = crp.crp_collect(ctx, crp.COLLECT_ALL)
    observed = float(np.mean(rec["lens_pixel"] < 12 * nside * nside))
    probe = crp.crp_measure_peaks(torch.cuda.current_device())
    crp.crp_lens_destroy(lens)
    crp.crp_grid_destroy(g)
    crp.crp_context_destroy(ctx)
    t = statistics.median(ts)
    peaks = json.load(open(PEAKS_PATH)) if os.path.exists(PEAKS_PATH) else {}
    hbm = peaks.get("hbm_gbs")
    ach = n * LENS_HBM_BYTES_PER_CANDIDATE / t / 1e9
    print(json.dumps({
        "workload": f"lens_apply_nside{nside}_{nb}bins", "metric": "lens applications/s",
        "value": n / t, "unit": "candidates/s", "candidates": n, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "observed_fraction": observed,
        "lens_samples": len(E), "l2": "256 MB buffer written before every launch",
        "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                     "frac": ach / hbm if hbm else None,
                     "bytes_per_candidate": LENS_HBM_BYTES_PER_CANDIDATE,
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if hbm else None},
        "fp64_peak_tflops_measured": probe["fp64_tflops"], "clocks": clocks,
        "gpu_launches": 2 * args.steps}))

if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "plain":
        run_plain(a)
    elif a.workload == "galactic":
        run_galactic(a)
    elif a.workload == "uneven":
        run_uneven(a)
    elif a.workload == "e2e":
        run_e2e(a)
    elif a.workload == "cosmology":
        run_cosmology(a)
    elif a.workload == "train":
        run_train(a)
    elif a.workload == "lens":
        run_lens(a)
    else:
        run_ours(a)
