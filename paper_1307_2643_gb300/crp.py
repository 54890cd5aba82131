"""ctypes binding of the C ABI declared in ``include/crp.h``.

Argument marshalling only: every step of the propagation runs in the CUDA
library ``_build/libcrp.so``.  There is no CPU fallback; importing a function
here without the built library raises.  The names follow the C functions
(``crp_context_create`` ...); non-zero statuses raise :class:`CrpError` with
the library's message.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcrp.so")

# status codes
OK, E_INVALID, E_OOM, E_CUDA, E_QUEUE_FULL, E_TIMEOUT, E_BOUNDS, E_STATE = 0, -1, -2, -3, -4, -5, -6, -7
F32, F64 = 0, 1
GRID_FROM_HOST, GRID_FROM_DEVICE, GRID_TURBULENT = 0, 1, 2
FP64, MIXED = 0, 1
PAIR, ADIABATIC, PION, PHOTODIS, EMIN, OBSERVER, BORDER, GALACTIC, DECAY, GMF = (1 << i for i in range(10))
ACTIVE, BELOW_EMIN, MAX_LENGTH, DETECTED, AT_BORDER, BUDGET = range(6)
COLLECT_ALL, COLLECT_FINISHED, COLLECT_DETECTED, COLLECT_ACTIVE, COLLECT_AT_BORDER = range(5)

MPC_M = 3.0856775814913673e22
KPC_M = 3.0856775814913673e19
NANOGAUSS_T = 1e-13
MICROGAUSS_T = 1e-10


class CrpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"crp status {status}: {msg}")
        self.status = status


class GridDesc(C.Structure):
    _fields_ = [("n", C.c_int64 * 3), ("spacing", C.c_double), ("origin", C.c_double * 3),
                ("dtype", C.c_int32), ("source", C.c_int32), ("data", C.c_void_p),
                ("data_dtype", C.c_int32), ("cell_records", C.c_int32),
                ("lmin", C.c_double), ("lmax", C.c_double), ("brms", C.c_double),
                ("spectral_index", C.c_double), ("seed", C.c_uint64)]


class TablesDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("gamma_lo", C.c_double), ("gamma_hi", C.c_double),
                ("length_unit_m", C.c_double), ("T_cmb", C.c_double),
                ("pion_sigma_mb", C.c_double), ("pion_eth_eV", C.c_double),
                ("gdr_peak_mb", C.c_double), ("gdr_center_eV", C.c_double),
                ("gdr_fwhm_eV", C.c_double), ("gdr_lo_eV", C.c_double), ("gdr_hi_eV", C.c_double),
                ("irb_T_K", C.c_double * 2), ("irb_dilution", C.c_double * 2)]


class CandidateArrays(C.Structure):
    _fields_ = [("id", C.c_void_p), ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("ux", C.c_void_p), ("uy", C.c_void_p), ("uz", C.c_void_p), ("E", C.c_void_p),
                ("A", C.c_void_p), ("Z", C.c_void_p), ("q", C.c_void_p), ("s_max", C.c_void_p),
                ("on_device", C.c_int32), ("reserved", C.c_int32)]


class Gmf(C.Structure):
    """crp_gmf: the analytic multi-arm galactic field's parameters."""
    _fields_ = [("arm_b", C.c_double * 8), ("arm_rx", C.c_double * 8), ("pitch_rad", C.c_double),
                ("ring_b", C.c_double), ("r_ring", C.c_double), ("r_in", C.c_double),
                ("r_out", C.c_double), ("h_disk", C.c_double), ("w_disk", C.c_double),
                ("halo_bn", C.c_double), ("halo_bs", C.c_double), ("halo_rn", C.c_double),
                ("halo_rs", C.c_double), ("halo_wh", C.c_double), ("halo_z0", C.c_double),
                ("x_b", C.c_double), ("x_theta_rad", C.c_double), ("x_rc", C.c_double),
                ("x_r", C.c_double), ("r_cut_in", C.c_double), ("r_cut_out", C.c_double)]


def gmf(**kw) -> Gmf:
    """Gmf from keyword values (unset fields 0)."""
    g = Gmf()
    for k, v in kw.items():
        if k in ("arm_b", "arm_rx"):
            getattr(g, k)[:] = v
        else:
            setattr(g, k, v)
    return g


class Modules(C.Structure):
    _fields_ = [("precision", C.c_int32), ("flags", C.c_uint32), ("tol", C.c_double),
                ("h_min", C.c_double), ("h_max", C.c_double), ("field_unit_T", C.c_double),
                ("length_unit_m", C.c_double), ("beta_ad", C.c_double), ("e_min", C.c_double),
                ("tables", C.c_void_p),
                ("observer_center", C.c_double * 3), ("observer_radius", C.c_double),
                ("border_center", C.c_double * 3), ("border_radius", C.c_double),
                ("disk_b", C.c_double), ("disk_pitch_rad", C.c_double), ("disk_hz", C.c_double),
                ("disk_rmin", C.c_double), ("disk_rmax", C.c_double),
                ("halo_b", C.c_double), ("halo_z0", C.c_double), ("halo_sigma", C.c_double),
                ("gal_center", C.c_double * 3),
                ("max_steps", C.c_uint64), ("step_budget", C.c_uint64),
                ("deadline_ms", C.c_double), ("block_size", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("slice", C.c_uint32), ("queue_order", C.c_int32),
                ("use_graph", C.c_int32), ("reserved0", C.c_int32), ("gmf", C.c_void_p)]


class LensDesc(C.Structure):
    _fields_ = [("nside", C.c_int32), ("n_bins", C.c_int32), ("r_lo", C.c_double),
                ("r_hi", C.c_double), ("earth", C.c_double * 3), ("dirs", C.c_void_p),
                ("E", C.c_void_p), ("bin", C.c_void_p), ("n_samples", C.c_int64)]


class Cosmology(C.Structure):
    _fields_ = [("H0_km_s_Mpc", C.c_double), ("omega_m", C.c_double), ("dz_max", C.c_double),
                ("loss_max", C.c_double)]


def cosmology(H0_km_s_Mpc=0.0, omega_m=0.0, dz_max=0.0, loss_max=0.0):
    """Flat Lambda-CDM; zeros select 67.3 km/s/Mpc, 0.315, 1e-3, 1e-3."""
    return Cosmology(H0_km_s_Mpc, omega_m, dz_max, loss_max)


class Peaks(C.Structure):
    _fields_ = [("fp32_tflops", C.c_double), ("fp64_tflops", C.c_double),
                ("l2_read_gbs", C.c_double), ("sm_count", C.c_int32), ("l2_bytes", C.c_int32)]


class TuneResult(C.Structure):
    _fields_ = [("block_size", C.c_int32), ("blocks_per_sm", C.c_int32), ("slice", C.c_uint32),
                ("queue_order", C.c_int32), ("steps_per_s", C.c_double),
                ("n_tried", C.c_int32), ("reserved", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("accepted_steps", C.c_uint64), ("rejected_trials", C.c_uint64),
                ("rhs_evals", C.c_uint64), ("n_pion", C.c_uint64), ("n_pd", C.c_uint64),
                ("n_secondaries", C.c_uint64), ("n_dropped", C.c_uint64),
                ("n_overflow", C.c_uint64), ("n_active", C.c_uint64),
                ("n_detected", C.c_uint64), ("kernel_ms", C.c_double),
                ("launches", C.c_uint32), ("error_word", C.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


RECORD_DTYPE = np.dtype([
    ("id", "<u8"), ("parent_id", "<u8"),
    ("x", "<f8", 3), ("u", "<f8", 3),
    ("E", "<f8"), ("s", "<f8"),
    ("x0", "<f8", 3), ("u0", "<f8", 3),
    ("E0", "<f8"), ("s_max", "<f8"),
    ("n_acc", "<u8"), ("n_rej", "<u8"),
    ("A", "<i4"), ("Z", "<i4"), ("A0", "<i4"), ("Z0", "<i4"), ("q", "<i4"),
    ("status", "<i4"),
    ("n_pion", "<u4"), ("n_pd", "<u4"), ("draws", "<u4"), ("generation", "<u4"),
    ("n_dropped", "<u4"), ("lens_pixel", "<u4"),
])
assert RECORD_DTYPE.itemsize == 208

# exported symbols (every function declared in include/crp.h)
SYMBOLS = (
    "crp_last_error", "crp_version", "crp_set_allocator",
    "crp_context_create", "crp_context_destroy", "crp_context_size",
    "crp_grid_create", "crp_grid_destroy", "crp_grid_copy_out",
    "crp_tables_build", "crp_tables_from_host", "crp_tables_copy_out", "crp_tables_destroy",
    "crp_tables_set_decay",
    "crp_candidates_inject", "crp_candidates_clear",
    "crp_propagate", "crp_collect", "crp_histogram_energy", "crp_histogram_energy_noalloc",
    "crp_histogram_energy_device",
    "crp_lens_build", "crp_lens_apply", "crp_lens_copy_out", "crp_lens_destroy", "crp_lens_merge",
    "crp_histogram_healpix", "crp_histogram_healpix_device",
    "crp_mlp_create", "crp_mlp_destroy", "crp_mlp_num_params", "crp_mlp_set_params",
    "crp_mlp_get_params", "crp_mlp_forward", "crp_mlp_train_step", "crp_lens_build_surrogate",
    "crp_mlp_set_train_graph",
    "crp_checkpoint", "crp_restore", "crp_measure_peaks", "crp_autotune", "crp_grid_sample",
    "crp_mlp_set_forward_path", "crp_propagate_1d", "crp_cosmology_correct", "crp_cosmology_pick",
    "crp_redshift_of_distance",
)

_lock = threading.Lock()
_lib = None
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


def lib():
    """Load libcrp.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libcrp.so is not built ({LIB_PATH}); run "
                                   "paper_1307_2643_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            p, st, sz, u64, i32 = C.c_void_p, C.c_int32, C.c_size_t, C.c_uint64, C.c_int32
            L.crp_last_error.restype = C.c_char_p
            L.crp_version.restype = i32
            L.crp_set_allocator.argtypes = [ALLOC_FN, FREE_FN, p]
            L.crp_context_create.argtypes = [i32, u64, sz, C.POINTER(p)]
            L.crp_context_destroy.argtypes = [p]
            L.crp_context_size.argtypes = [p, C.POINTER(sz)]
            L.crp_grid_create.argtypes = [p, C.POINTER(GridDesc), C.POINTER(p)]
            L.crp_grid_destroy.argtypes = [p]
            L.crp_grid_copy_out.argtypes = [p, p]
            L.crp_tables_build.argtypes = [p, C.POINTER(TablesDesc), C.POINTER(p)]
            L.crp_tables_from_host.argtypes = [p, C.POINTER(TablesDesc), p, p, p, C.POINTER(p)]
            L.crp_tables_copy_out.argtypes = [p, p, p, p]
            L.crp_tables_destroy.argtypes = [p]
            L.crp_tables_set_decay.argtypes = [p, C.c_int64, p, p, p, p]
            L.crp_candidates_inject.argtypes = [p, C.POINTER(CandidateArrays), sz, u64, p]
            L.crp_candidates_clear.argtypes = [p]
            L.crp_propagate.argtypes = [p, p, C.POINTER(Modules), p, C.POINTER(Stats)]
            L.crp_collect.argtypes = [p, i32, p, sz, C.POINTER(sz), i32, p]
            L.crp_histogram_energy.argtypes = [p, i32, C.c_double, C.c_double, i32, p, p]
            L.crp_histogram_energy_noalloc.argtypes = [p, i32, C.c_double, C.c_double, i32, p, p]
            L.crp_histogram_energy_device.argtypes = [p, i32, C.c_double, C.c_double, i32, p, i32,
                                                      p]
            L.crp_lens_build.argtypes = [p, p, C.POINTER(Modules), C.POINTER(LensDesc), C.POINTER(p),
                                         C.POINTER(Stats)]
            L.crp_lens_apply.argtypes = [p, p, i32, p]
            L.crp_lens_copy_out.argtypes = [p, p, p, p, C.POINTER(C.c_int64)]
            L.crp_lens_merge.argtypes = [p, p, p, C.POINTER(p)]
            L.crp_lens_destroy.argtypes = [p]
            L.crp_histogram_healpix.argtypes = [p, i32, i32, i32, p, p]
            L.crp_histogram_healpix_device.argtypes = [p, i32, i32, i32, p, i32, p]
            L.crp_mlp_create.argtypes = [p, i32, i32, i32, u64, C.POINTER(p)]
            L.crp_mlp_destroy.argtypes = [p]
            L.crp_mlp_num_params.argtypes = [p]
            L.crp_mlp_set_params.argtypes = [p, p]
            L.crp_mlp_get_params.argtypes = [p, p, p]
            L.crp_mlp_forward.argtypes = [p, p, p, C.c_int64, p]
            L.crp_mlp_train_step.argtypes = [p, p, p, C.c_int64, C.c_float, p, p]
            L.crp_lens_build_surrogate.argtypes = [p, p, C.POINTER(LensDesc), C.POINTER(p)]
            L.crp_checkpoint.argtypes = [p, p, sz, C.POINTER(sz), p]
            L.crp_restore.argtypes = [p, p, sz, p]
            L.crp_measure_peaks.argtypes = [i32, C.POINTER(Peaks)]
            L.crp_grid_sample.argtypes = [p, C.POINTER(Modules), C.c_int64, p, p]
            L.crp_mlp_set_forward_path.argtypes = [p, i32]
            L.crp_mlp_set_train_graph.argtypes = [p, i32]
            L.crp_propagate_1d.argtypes = [p, C.POINTER(Cosmology), C.POINTER(Modules), p,
                                           C.POINTER(Stats)]
            L.crp_cosmology_correct.argtypes = [p, C.POINTER(Cosmology), C.POINTER(Modules),
                                                C.c_int64] + [p] * 9
            L.crp_cosmology_pick.argtypes = [p, C.POINTER(Cosmology), C.POINTER(Modules),
                                             C.c_int64] + [p] * 9
            L.crp_redshift_of_distance.argtypes = [C.POINTER(Cosmology), C.c_double, C.c_int64,
                                                   p, p]
            L.crp_autotune.argtypes = [p, p, C.POINTER(Modules), u64, C.POINTER(TuneResult), p]
            for name in SYMBOLS:
                if name not in ("crp_last_error", "crp_version"):
                    getattr(L, name).restype = st
            L.crp_mlp_num_params.restype = C.c_int64
            _lib = L
    return _lib


def _check(status):
    if status != OK:
        raise CrpError(status, lib().crp_last_error().decode(errors="replace"))
    return status


def _addr(a):
    """Data pointer of a numpy array or torch tensor (None stays None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


# ---------------------------------------------------------------------------
# allocator: route the library's device allocations through torch's caching
# allocator (PyTorch supplies device memory and streams).
# ---------------------------------------------------------------------------
_alloc_keep = []


def use_torch_allocator(device=0):
    import torch

    @ALLOC_FN
    def _alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device)
        except Exception:  # out of memory -> NULL, the library reports CRP_E_OOM
            return None

    @FREE_FN
    def _free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    _alloc_keep[:] = [_alloc, _free]
    _check(lib().crp_set_allocator(_alloc, _free, None))


def use_cuda_allocator():
    _check(lib().crp_set_allocator(ALLOC_FN(0), FREE_FN(0), None))
    _alloc_keep.clear()


# ---------------------------------------------------------------------------
# functions with the C names
# ---------------------------------------------------------------------------
def crp_version():
    return lib().crp_version()


def crp_context_create(device=0, seed=0, capacity=1 << 20):
    h = C.c_void_p()
    _check(lib().crp_context_create(device, seed, capacity, C.byref(h)))
    return h


def crp_context_destroy(ctx):
    _check(lib().crp_context_destroy(ctx))


def crp_context_size(ctx):
    n = C.c_size_t()
    _check(lib().crp_context_size(ctx, C.byref(n)))
    return n.value


def crp_grid_create(ctx, desc: GridDesc):
    h = C.c_void_p()
    _check(lib().crp_grid_create(ctx, C.byref(desc), C.byref(h)))
    return h


def crp_grid_sample(grid, modules: Modules, xyz):
    """Field [m, 3] at points xyz [m, 3] as the kernels of modules.precision see it."""
    pts = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    out = np.zeros_like(pts)
    _check(lib().crp_grid_sample(grid, C.byref(modules), len(pts), pts.ctypes.data,
                                 out.ctypes.data))
    return out


def crp_grid_destroy(grid):
    _check(lib().crp_grid_destroy(grid))


def crp_grid_copy_out(grid, n):
    out = np.empty((n[2], n[1], n[0], 3), dtype=np.float64)
    _check(lib().crp_grid_copy_out(grid, out.ctypes.data))
    return out


def crp_tables_build(ctx, desc: TablesDesc):
    h = C.c_void_p()
    _check(lib().crp_tables_build(ctx, C.byref(desc), C.byref(h)))
    return h


def crp_tables_from_host(ctx, desc: TablesDesc, beta, pion, gdr):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (beta, pion, gdr)]
    h = C.c_void_p()
    _check(lib().crp_tables_from_host(ctx, C.byref(desc), *(a.ctypes.data for a in arrs),
                                      C.byref(h)))
    return h


def crp_tables_copy_out(tables, n):
    out = [np.empty(n) for _ in range(3)]
    _check(lib().crp_tables_copy_out(tables, *(a.ctypes.data for a in out)))
    return out


def crp_tables_destroy(tables):
    _check(lib().crp_tables_destroy(tables))


def crp_tables_set_decay(tables, decay_table=None):
    """Attach a nuclide table (dict of A, Z, tau_s, branching [n, 4]) to
    `tables`, or remove it (None)."""
    if decay_table is None:
        _check(lib().crp_tables_set_decay(tables, 0, None, None, None, None))
        return
    A = np.ascontiguousarray(decay_table["A"], dtype=np.int32)
    Z = np.ascontiguousarray(decay_table["Z"], dtype=np.int32)
    tau = np.ascontiguousarray(decay_table["tau_s"], dtype=np.float64)
    b = np.ascontiguousarray(decay_table["branching"], dtype=np.float64).reshape(-1, 4)
    _check(lib().crp_tables_set_decay(tables, len(A), A.ctypes.data, Z.ctypes.data,
                                      tau.ctypes.data, b.ctypes.data))


def crp_candidates_inject(ctx, arrays: CandidateArrays, n, first_id=0, stream=None):
    _check(lib().crp_candidates_inject(ctx, C.byref(arrays), n, first_id, stream))


def crp_candidates_clear(ctx):
    _check(lib().crp_candidates_clear(ctx))


def crp_propagate(ctx, grid, modules: Modules, stream=None, raise_on_error=True):
    """Returns (status, Stats).  TIMEOUT / QUEUE_FULL raise unless
    raise_on_error is False."""
    s = Stats()
    status = lib().crp_propagate(ctx, grid, C.byref(modules), stream, C.byref(s))
    if raise_on_error:
        _check(status)
    return status, s


def crp_collect(ctx, what=COLLECT_ALL, out=None, stream=None):
    """Records selected by `what` as a numpy structured array (host), or into
    a caller-supplied device buffer (torch uint8 tensor of capacity*200 bytes)
    whose record count is returned."""
    n = C.c_size_t()
    if out is None:
        _check(lib().crp_collect(ctx, what, None, 0, C.byref(n), 0, stream))
        rec = np.zeros(n.value, dtype=RECORD_DTYPE)
        if n.value:
            _check(lib().crp_collect(ctx, what, rec.ctypes.data, n.value, C.byref(n), 0, stream))
        return rec
    on_dev = 1 if getattr(out, "is_cuda", False) else 0
    cap = out.numel() * out.element_size() // RECORD_DTYPE.itemsize if on_dev else len(out)
    _check(lib().crp_collect(ctx, what, _addr(out), cap, C.byref(n), on_dev, stream))
    return n.value


def crp_histogram_energy(ctx, what, e_lo, e_hi, nbins, stream=None):
    out = np.zeros(nbins, dtype=np.uint64)
    _check(lib().crp_histogram_energy(ctx, what, e_lo, e_hi, nbins, out.ctypes.data, stream))
    return out


LENS_NOT_APPLIED = 0xFFFFFFFF
LENS_NOT_OBSERVED = 0xFFFFFFFE


def crp_lens_build(ctx, galaxy, modules: Modules, nside, n_bins, r_lo, r_hi, earth, dirs, E, bins):
    """Build a lens by back-tracking; returns (handle, Stats of the back-tracking)."""
    dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    E = np.ascontiguousarray(E, dtype=np.float64)
    bins = np.ascontiguousarray(bins, dtype=np.int32)
    d = LensDesc()
    d.nside, d.n_bins, d.r_lo, d.r_hi = nside, n_bins, r_lo, r_hi
    d.earth[:] = earth
    d.dirs, d.E, d.bin, d.n_samples = dirs.ctypes.data, E.ctypes.data, bins.ctypes.data, len(E)
    h = C.c_void_p()
    s = Stats()
    _check(lib().crp_lens_build(ctx, galaxy, C.byref(modules), C.byref(d), C.byref(h), C.byref(s)))
    return h, s


def crp_lens_build_surrogate(ctx, mlp, nside, n_bins, r_lo, r_hi, dirs, E, bins):
    dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    E = np.ascontiguousarray(E, dtype=np.float64)
    bins = np.ascontiguousarray(bins, dtype=np.int32)
    d = LensDesc()
    d.nside, d.n_bins, d.r_lo, d.r_hi = nside, n_bins, r_lo, r_hi
    d.dirs, d.E, d.bin, d.n_samples = dirs.ctypes.data, E.ctypes.data, bins.ctypes.data, len(E)
    h = C.c_void_p()
    _check(lib().crp_lens_build_surrogate(ctx, mlp, C.byref(d), C.byref(h)))
    return h


def crp_lens_apply(ctx, lens, what=COLLECT_ALL, stream=None):
    _check(lib().crp_lens_apply(ctx, lens, what, stream))


def crp_lens_copy_out(lens, n_cols, n_bins):
    n = C.c_int64()
    _check(lib().crp_lens_copy_out(lens, None, None, None, C.byref(n)))
    col = np.zeros(n_cols + 1, np.uint32)
    ent = np.zeros(max(n.value, 1), np.uint32)
    mx = np.zeros(n_bins, np.uint32)
    _check(lib().crp_lens_copy_out(lens, col.ctypes.data, ent.ctypes.data, mx.ctypes.data,
                                   C.byref(n)))
    return dict(col_start=col, entries=ent[: n.value], max_count=mx)


def crp_lens_merge(a, b, take_b):
    """Per rigidity bin: b's columns where take_b[bin], a's elsewhere."""
    take = np.ascontiguousarray(np.asarray(take_b, dtype=bool).astype(np.uint8))
    h = C.c_void_p()
    _check(lib().crp_lens_merge(a, b, take.ctypes.data, C.byref(h)))
    return h


def crp_lens_destroy(lens):
    _check(lib().crp_lens_destroy(lens))


def crp_histogram_healpix(ctx, what, nside, source, stream=None):
    out = np.zeros(12 * nside * nside, dtype=np.uint64)
    _check(lib().crp_histogram_healpix(ctx, what, nside, source, out.ctypes.data, stream))
    return out


def crp_mlp_create(ctx, n_in=4, hidden=256, n_hidden=4, seed=0):
    h = C.c_void_p()
    _check(lib().crp_mlp_create(ctx, n_in, hidden, n_hidden, seed, C.byref(h)))
    return h


def crp_mlp_destroy(mlp):
    _check(lib().crp_mlp_destroy(mlp))


def crp_mlp_num_params(mlp):
    return lib().crp_mlp_num_params(mlp)


def crp_mlp_set_params(mlp, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert len(p) == crp_mlp_num_params(mlp)
    _check(lib().crp_mlp_set_params(mlp, p.ctypes.data))


def crp_mlp_get_params(mlp):
    """(params, last gradient) as FP32 host arrays."""
    n = crp_mlp_num_params(mlp)
    p, g = np.zeros(n, np.float32), np.zeros(n, np.float32)
    _check(lib().crp_mlp_get_params(mlp, p.ctypes.data, g.ctypes.data))
    return p, g


def crp_mlp_forward(mlp, x_dev, y_dev, n, stream=None):
    """x_dev, y_dev: torch float32 device tensors [n, n_in], [n, 3]."""
    _check(lib().crp_mlp_forward(mlp, _addr(x_dev), _addr(y_dev), n, stream))


MLP_PATH_AUTO, MLP_PATH_TENSOR_CORE_FUSED, MLP_PATH_LAYERED = 0, 1, 2


def crp_mlp_set_forward_path(mlp, path):
    _check(lib().crp_mlp_set_forward_path(mlp, path))


def crp_mlp_set_train_graph(mlp, enable=True):
    """Graph replay of the tensor-core training step (default on); off: every
    step launched kernel by kernel."""
    _check(lib().crp_mlp_set_train_graph(mlp, 1 if enable else 0))


def crp_mlp_train_step(mlp, x_dev, t_dev, n, lr, stream=None, want_loss=True):
    loss = C.c_float(0.0)
    _check(lib().crp_mlp_train_step(mlp, _addr(x_dev), _addr(t_dev), n, lr,
                                    C.byref(loss) if want_loss else None, stream))
    return loss.value


def crp_propagate_1d(ctx, cosmo: Cosmology, modules: Modules, stream=None,
                     raise_on_error=True):
    """1D propagation of the context's candidates (x = source redshift)."""
    s = Stats()
    status = lib().crp_propagate_1d(ctx, C.byref(cosmo), C.byref(modules), stream, C.byref(s))
    if raise_on_error:
        _check(status)
    return status, s


def _correction(fn, ctx, cosmo, modules, ids, src, E0, A0, Z0):
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    src = np.ascontiguousarray(src, dtype=np.float64)
    E0 = np.ascontiguousarray(E0, dtype=np.float64)
    A0 = np.ascontiguousarray(A0, dtype=np.int32)
    Z0 = np.ascontiguousarray(Z0, dtype=np.int32)
    n = len(E0)
    E, A, Z, nk = (np.zeros(n), np.zeros(n, np.int32), np.zeros(n, np.int32),
                   np.zeros(n, np.int32))
    _check(fn(ctx, C.byref(cosmo), C.byref(modules), n, ids.ctypes.data, src.ctypes.data,
              E0.ctypes.data, A0.ctypes.data, Z0.ctypes.data, E.ctypes.data, A.ctypes.data,
              Z.ctypes.data, nk.ctypes.data))
    return E, A, Z, nk


def crp_cosmology_correct(ctx, cosmo: Cosmology, modules: Modules, ids, T, E0, A0, Z0):
    """(E, A, Z, n_products) of the a-posteriori correction (host arrays)."""
    return _correction(lib().crp_cosmology_correct, ctx, cosmo, modules, ids, T, E0, A0, Z0)


def crp_cosmology_pick(ctx, cosmo: Cosmology, modules: Modules, ids, z_src, E0, A0, Z0):
    """(E, A, Z, n_products) of the correction's pick from given source
    redshifts (host arrays)."""
    return _correction(lib().crp_cosmology_pick, ctx, cosmo, modules, ids, z_src, E0, A0, Z0)


def crp_redshift_of_distance(cosmo: Cosmology, length_unit_m, D):
    """Redshifts of comoving distances D (length units of length_unit_m metres)."""
    D = np.ascontiguousarray(D, dtype=np.float64).ravel()
    out = np.zeros_like(D)
    _check(lib().crp_redshift_of_distance(C.byref(cosmo), length_unit_m, len(D), D.ctypes.data,
                                          out.ctypes.data))
    return out


def crp_autotune(ctx, grid, modules: Modules, steps_per_trial=0, stream=None):
    """Tune `modules` in place on the context's candidates; returns the
    TuneResult as a dict."""
    r = TuneResult()
    _check(lib().crp_autotune(ctx, grid, C.byref(modules), steps_per_trial, C.byref(r), stream))
    return {k: getattr(r, k) for k, _ in TuneResult._fields_}


def crp_checkpoint(ctx, stream=None):
    """The context's state as a bytes-like numpy uint8 array."""
    n = C.c_size_t()
    _check(lib().crp_checkpoint(ctx, None, 0, C.byref(n), stream))
    buf = np.zeros(n.value, np.uint8)
    _check(lib().crp_checkpoint(ctx, buf.ctypes.data, n.value, C.byref(n), stream))
    return buf


def crp_restore(ctx, image, stream=None):
    buf = np.ascontiguousarray(np.frombuffer(image, np.uint8) if isinstance(image, (bytes, bytearray))
                               else image, dtype=np.uint8)
    _check(lib().crp_restore(ctx, buf.ctypes.data, len(buf), stream))


def crp_measure_peaks(device=0):
    """dict(fp32_tflops, fp64_tflops, l2_read_gbs, sm_count, l2_bytes) measured on `device`."""
    pk = Peaks()
    _check(lib().crp_measure_peaks(device, C.byref(pk)))
    return {k: getattr(pk, k) for k, _ in Peaks._fields_}


def crp_histogram_energy_device(ctx, what, e_lo, e_hi, nbins, out_dev, accumulate=False,
                                stream=None):
    """crp_histogram_energy into a device array (a torch int64/uint64 tensor of
    nbins on the context's device); asynchronous on `stream`."""
    _check(lib().crp_histogram_energy_device(ctx, what, e_lo, e_hi, nbins, _addr(out_dev),
                                             1 if accumulate else 0, stream))
    return out_dev


def crp_histogram_healpix_device(ctx, what, nside, source, out_dev, accumulate=False,
                                 stream=None):
    """crp_histogram_healpix into a device array (a torch int64/uint64 tensor of
    12 nside^2 on the context's device); asynchronous on `stream`."""
    _check(lib().crp_histogram_healpix_device(ctx, what, nside, source, _addr(out_dev),
                                              1 if accumulate else 0, stream))
    return out_dev


HIST_NOALLOC_MAX_BINS = 4096


def crp_histogram_energy_noalloc(ctx, what, e_lo, e_hi, nbins, stream=None):
    """crp_histogram_energy counted into the library's fixed device array
    (no device allocation; nbins <= HIST_NOALLOC_MAX_BINS)."""
    out = np.zeros(nbins, dtype=np.uint64)
    _check(lib().crp_histogram_energy_noalloc(ctx, what, e_lo, e_hi, nbins, out.ctypes.data,
                                              stream))
    return out


# ---------------------------------------------------------------------------
# small conveniences (still marshalling only)
# ---------------------------------------------------------------------------
def candidate_arrays(inj: dict, on_device=False):
    """CandidateArrays pointing at the arrays of `inj` (numpy on the host, or
    torch tensors on the device); the descriptor holds a reference to `inj`."""
    a = CandidateArrays()
    for k in ("id", "x", "y", "z", "ux", "uy", "uz", "E", "A", "Z", "q", "s_max"):
        setattr(a, k, _addr(inj.get(k)))
    a.on_device = 1 if on_device else 0
    a._refs = inj  # the arrays live as long as the descriptor
    return a


def host_injection(inj: dict) -> dict:
    """Contiguous host arrays of the dtypes the ABI expects."""
    out = {}
    for k, v in inj.items():
        dt = {"id": np.uint64, "A": np.int32, "Z": np.int32, "q": np.int32}.get(k, np.float64)
        out[k] = np.ascontiguousarray(v, dtype=dt)
    return out


def grid_desc(n, spacing, origin=(0.0, 0.0, 0.0), dtype=F64, source=GRID_FROM_HOST, data=None,
              data_dtype=F64, lmin=0.0, lmax=0.0, brms=0.0, spectral_index=-11.0 / 3.0, seed=0,
              cell_records=0):
    d = GridDesc()
    d.n[:] = n
    d.spacing = spacing
    d.origin[:] = origin
    d.dtype, d.source = dtype, source
    if isinstance(data, np.ndarray):
        # C-contiguous, and referenced by the descriptor so the buffer outlives
        # the caller's temporaries until crp_grid_create has copied it
        data = np.ascontiguousarray(data)
    d._data_ref = data
    d.data = _addr(data)
    d.data_dtype = data_dtype
    d.cell_records = cell_records
    d.lmin, d.lmax, d.brms, d.spectral_index, d.seed = lmin, lmax, brms, spectral_index, seed
    return d


def tables_desc(n=1000, gamma_lo=1e6, gamma_hi=1e13, length_unit_m=MPC_M, T_cmb=2.725,
                pion_sigma_mb=0.5, pion_eth_eV=145e6, gdr_peak_mb=1.5, gdr_center_eV=20e6,
                gdr_fwhm_eV=6e6, gdr_lo_eV=8e6, gdr_hi_eV=150e6, irb=()):
    """irb: up to two (T [K], dilution) dilute blackbodies added to the pair-
    production background (synthetic infrared / optical light)."""
    d = TablesDesc()
    d.n, d.gamma_lo, d.gamma_hi, d.length_unit_m, d.T_cmb = n, gamma_lo, gamma_hi, length_unit_m, T_cmb
    d.pion_sigma_mb, d.pion_eth_eV = pion_sigma_mb, pion_eth_eV
    d.gdr_peak_mb, d.gdr_center_eV, d.gdr_fwhm_eV = gdr_peak_mb, gdr_center_eV, gdr_fwhm_eV
    d.gdr_lo_eV, d.gdr_hi_eV = gdr_lo_eV, gdr_hi_eV
    for k, (T, D) in enumerate(irb):
        d.irb_T_K[k], d.irb_dilution[k] = T, D
    return d


def modules(precision=FP64, flags=0, tol=1e-4, h_min=0.01, h_max=1.0, field_unit_T=NANOGAUSS_T,
            length_unit_m=MPC_M, beta_ad=0.0, e_min=0.0, tables=None, observer_center=(0, 0, 0),
            observer_radius=0.0, border_center=(0, 0, 0), border_radius=0.0, galactic=None,
            max_steps=10_000_000, step_budget=0, deadline_ms=0.0, block_size=0, blocks_per_sm=0,
            slice=0, queue_order=0, use_graph=0, gmf=None):
    """crp_modules; `gmf` (a Gmf or a dict of its fields) is referenced by the
    returned structure and read during each call that uses it."""
    m = Modules()
    m.precision, m.flags, m.tol, m.h_min, m.h_max = precision, flags, tol, h_min, h_max
    m.field_unit_T, m.length_unit_m, m.beta_ad, m.e_min = field_unit_T, length_unit_m, beta_ad, e_min
    m.tables = tables.value if isinstance(tables, C.c_void_p) else tables
    m.observer_center[:] = observer_center
    m.observer_radius = observer_radius
    m.border_center[:] = border_center
    m.border_radius = border_radius
    if galactic:
        for k, v in galactic.items():
            if k == "center":
                m.gal_center[:] = v
            else:
                setattr(m, k, v)
    m.max_steps, m.step_budget, m.deadline_ms = max_steps, step_budget, deadline_ms
    m.block_size, m.blocks_per_sm, m.slice = block_size, blocks_per_sm, slice
    m.queue_order = queue_order
    m.use_graph = use_graph
    if gmf is not None:
        g = gmf if isinstance(gmf, Gmf) else globals()["gmf"](**gmf)
        m._gmf_ref = g
        m.gmf = C.addressof(g)
    return m
