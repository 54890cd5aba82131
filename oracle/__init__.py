"""FP64 CPU oracle for the CRPropa 3.0 candidate-propagation method.

TEST INFRASTRUCTURE ONLY.  This package is the independent reference the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import it; the product
package never does.  It shares no code, header, table or constant generator
with the CUDA path.

The compiled part (``crp_oracle.cpp``) holds the per-candidate module cycle of
the paper (Sect. 3 and Fig. 1: integration, interaction modules, boundary /
observer modules, IsActive checked after each cycle), the Philox4x32-10
generator, the Blumenthal / pion / giant-dipole rate tables and the
turbulence mode synthesis.  This Python layer adds the steps that are a plain
library primitive: the inverse FFT of the turbulence modes (numpy) and the
HEALPix, lens and MLP oracles in ``oracle.healpix``, ``oracle.lens`` and
``oracle.mlp``.

Parity status per function is listed in the module docstrings; the rate
tables for the synthetic pion and giant-dipole cross sections are pinned to
the definitions they come from, not to physical data ("parity unpinned" for
their absolute physics beyond those definitions).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "crp_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None

# Status of a finished candidate.
ACTIVE, BELOW_EMIN, MAX_LENGTH, DETECTED, AT_BORDER, BUDGET = range(6)

# Module flags.
PAIR = 1 << 0
ADIABATIC = 1 << 1
PION = 1 << 2
PHOTODIS = 1 << 3
EMIN = 1 << 4
OBSERVER = 1 << 5
BORDER = 1 << 6
GALACTIC = 1 << 7
DECAY = 1 << 8
GMF = 1 << 9


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-pthread", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Gmf(C.Structure):
    """Analytic multi-arm galactic field (orc_gmf): arm strengths at r_in,
    arm boundary radii on the phi = pi ray, pitch, ring, disk/halo transition,
    toroidal halo, X field, spherical cuts."""
    _fields_ = [
        ("arm_b", C.c_double * 8), ("arm_rx", C.c_double * 8), ("pitch_rad", C.c_double),
        ("ring_b", C.c_double), ("r_ring", C.c_double), ("r_in", C.c_double),
        ("r_out", C.c_double), ("h_disk", C.c_double), ("w_disk", C.c_double),
        ("halo_bn", C.c_double), ("halo_bs", C.c_double), ("halo_rn", C.c_double),
        ("halo_rs", C.c_double), ("halo_wh", C.c_double), ("halo_z0", C.c_double),
        ("x_b", C.c_double), ("x_theta_rad", C.c_double), ("x_rc", C.c_double),
        ("x_r", C.c_double), ("r_cut_in", C.c_double), ("r_cut_out", C.c_double),
    ]


def make_gmf(**kw) -> Gmf:
    """Gmf from keyword values (unset fields 0)."""
    g = Gmf()
    for k, v in kw.items():
        if k in ("arm_b", "arm_rx"):
            getattr(g, k)[:] = v
        else:
            setattr(g, k, v)
    return g


class Params(C.Structure):
    _fields_ = [
        ("origin", C.c_double * 3), ("spacing", C.c_double), ("n", C.c_int64 * 3),
        ("tol", C.c_double), ("h_min", C.c_double), ("h_max", C.c_double),
        ("curv_k", C.c_double),
        ("beta_ad", C.c_double), ("e_min", C.c_double),
        ("flags", C.c_uint32), ("pad0", C.c_uint32), ("seed", C.c_uint64),
        ("tab_lg0", C.c_double), ("tab_inv_dlg", C.c_double), ("tab_n", C.c_int64),
        ("obs_c", C.c_double * 3), ("obs_r", C.c_double),
        ("border_c", C.c_double * 3), ("border_r", C.c_double),
        ("gal_disk_b", C.c_double), ("gal_disk_pitch_rad", C.c_double), ("gal_disk_hz", C.c_double),
        ("gal_disk_rmin", C.c_double), ("gal_disk_rmax", C.c_double),
        ("gal_halo_b", C.c_double), ("gal_halo_z0", C.c_double), ("gal_halo_sigma", C.c_double),
        ("gal_center", C.c_double * 3),
        ("max_steps", C.c_int64),
        ("length_unit_m", C.c_double),
        ("gmf", Gmf),
        ("nuc_tab", C.c_void_p), ("nuc_amax", C.c_int64),
    ]


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
    ("n_dropped", "<u4"), ("pad", "<u4"),
])


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            d, u32, u64, i64, p = C.c_double, C.c_uint32, C.c_uint64, C.c_int64, C.c_void_p
            L.orc_philox4x32_10.argtypes = [p, p, p]
            L.orc_uniform_open.argtypes = [u32, u32]
            L.orc_uniform_open.restype = d
            L.orc_child_id.argtypes = [u64, u32]
            L.orc_child_id.restype = u64
            for name in ("orc_phi_pair", "orc_series_log", "orc_series_exp"):
                getattr(L, name).argtypes = [d]
                getattr(L, name).restype = d
            L.orc_planck_density.argtypes = [d, d]
            L.orc_planck_density.restype = d
            L.orc_beta_pair_proton.argtypes = [d, d]
            L.orc_beta_pair_proton.restype = d
            L.orc_rate_pion_nucleon.argtypes = [d, d, d, d]
            L.orc_rate_pion_nucleon.restype = d
            L.orc_rate_gdr_nucleon.argtypes = [d, d, d, d, d, d, d]
            L.orc_rate_gdr_nucleon.restype = d
            L.orc_cash_karp_tableau.argtypes = [p]
            L.orc_tables_build.argtypes = [i64, d, d, d, d, d, d, d, d, d, d, d, p, p, p, C.c_int,
                                           C.c_int, p, p]
            L.orc_turbulence_modes.argtypes = [i64, i64, i64, d, d, d, d, u64, p]
            L.orc_propagate.argtypes = [C.POINTER(Params), p, p, p, p, i64] + [p] * 12 + \
                [p, i64, C.POINTER(i64), C.c_int]
            L.orc_propagate.restype = C.c_int
            L.orc_field_at.argtypes = [C.POINTER(Params), p, i64, p, p]
            L.orc_series_atan2_vec.argtypes = [i64, p, p, p]
            L.orc_ang2pix.argtypes = [i64, d, d]
            L.orc_ang2pix.restype = i64
            L.orc_pix2ang.argtypes = [i64, i64, C.POINTER(d), C.POINTER(d)]
            L.orc_ang2pix_vec.argtypes = [i64, i64, p, p]
            L.orc_uniform_pairs.argtypes = [u64, u32, u32, i64, p, p]
            L.orc_series_log_vec.argtypes = [i64, p, p]
            L.orc_table_axis.argtypes = [i64, d, d, C.POINTER(d), C.POINTER(d)]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------------------
# Physical constants (CODATA 2018, IAU parsec), restated for the Python layer.
# ---------------------------------------------------------------------------
C_LIGHT = 299792458.0
MPC_M = 3.0856775814913673e22
KPC_M = 3.0856775814913673e19
NANOGAUSS_T = 1e-13
MICROGAUSS_T = 1e-10
MP_C2_EV = 938.27208816e6
KB_EV = 8.617333262e-5
HBARC_EVM = 1.973269804e-7


def curvature_constant(field_unit_T: float, length_unit_m: float) -> float:
    """c * B_unit * L_unit: turns q Z B / E [eV] into 1 / length unit."""
    return C_LIGHT * field_unit_T * length_unit_m


# ---------------------------------------------------------------------------
# Primitives
# ---------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform_open(lo: int, hi: int) -> float:
    return lib().orc_uniform_open(lo, hi)


def uniform_pairs(seed: int, tag: int, draw: int, ids) -> np.ndarray:
    """[n, 2] open uniforms of Philox draw `draw` / `tag` for each id."""
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    out = np.zeros((len(ids), 2))
    lib().orc_uniform_pairs(seed, tag, draw, len(ids), _ptr(ids), _ptr(out))
    return out


def child_id(parent: int, event_index: int) -> int:
    return lib().orc_child_id(parent, event_index)


def series_log(x: float) -> float:
    return lib().orc_series_log(x)


def series_log_vec(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    lib().orc_series_log_vec(len(x), _ptr(x), _ptr(out))
    return out


def series_exp(x: float) -> float:
    return lib().orc_series_exp(x)


def ang2pix(nside: int, z: float, phi: float) -> int:
    """HEALPix RING pixel of the direction (z = cos theta, phi)."""
    return lib().orc_ang2pix(nside, z, phi)


def pix2ang(nside: int, pix: int):
    """(z, phi) of the centre of HEALPix RING pixel `pix`."""
    z, phi = C.c_double(), C.c_double()
    lib().orc_pix2ang(nside, pix, C.byref(z), C.byref(phi))
    return z.value, phi.value


def ang2pix_vec(nside: int, u) -> np.ndarray:
    """HEALPix RING pixels of unit vectors u [n, 3]."""
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(len(u), dtype=np.int64)
    lib().orc_ang2pix_vec(nside, len(u), _ptr(u), _ptr(out))
    return out


def phi_pair(k: float) -> float:
    return lib().orc_phi_pair(k)


def planck_density(eps_eV: float, T: float) -> float:
    """Planck photon number density per unit energy [1/(m^3 eV)]."""
    return lib().orc_planck_density(eps_eV, KB_EV * T)


def beta_pair_proton(gamma: float, T: float = 2.725) -> float:
    """(1/E) dE/dx for pair production on a blackbody of temperature T [1/m]."""
    return lib().orc_beta_pair_proton(gamma, T)


def rate_pion_nucleon(gamma, T=2.725, sigma_mb=0.5, eth_eV=145e6):
    return lib().orc_rate_pion_nucleon(gamma, T, sigma_mb, eth_eV)


def rate_gdr_nucleon(gamma, T=2.725, peak_mb=1.5, ec_eV=20e6, fwhm_eV=6e6, lo_eV=8e6, hi_eV=150e6):
    return lib().orc_rate_gdr_nucleon(gamma, T, peak_mb, ec_eV, fwhm_eV, lo_eV, hi_eV)


def cash_karp_tableau() -> dict:
    out = np.zeros(24)
    lib().orc_cash_karp_tableau(_ptr(out))
    names = ["b21", "b31", "b32", "b41", "b42", "b43", "b51", "b52", "b53", "b54",
             "b61", "b62", "b63", "b64", "b65", "c1", "c3", "c4", "c6",
             "e1", "e3", "e4", "e5", "e6"]
    return dict(zip(names, out))


class Tables:
    """Rate tables on n nodes uniform in ln(Gamma), units of 1/length."""

    def __init__(self, n, g_lo, g_hi, beta_pair, rate_pion, rate_gdr):
        self.n, self.g_lo, self.g_hi = n, g_lo, g_hi
        self.beta_pair, self.rate_pion, self.rate_gdr = beta_pair, rate_pion, rate_gdr

    def axis(self):
        """(ln Gamma of node 0, nodes per unit ln Gamma), evaluated in C."""
        lg0, inv = C.c_double(), C.c_double()
        lib().orc_table_axis(self.n, self.g_lo, self.g_hi, C.byref(lg0), C.byref(inv))
        return lg0.value, inv.value


def tables_build(n=1000, g_lo=1e6, g_hi=1e13, length_unit_m=MPC_M, T=2.725,
                 pion_sigma_mb=0.5, pion_eth_eV=145e6, gdr_peak_mb=1.5, gdr_ec_eV=20e6,
                 gdr_fwhm_eV=6e6, gdr_lo_eV=8e6, gdr_hi_eV=150e6, nthreads=None,
                 irb=()) -> Tables:
    """irb: ((T_k [K], dilution_k), ...) dilute blackbodies added to the
    pair-production background (the synthetic infrared / optical light)."""
    nthreads = nthreads or os.cpu_count() or 1
    bp, rp, rg = np.zeros(n), np.zeros(n), np.zeros(n)
    irb_T = np.array([t for t, _ in irb] or [0.0], dtype=np.float64)
    irb_D = np.array([d for _, d in irb] or [0.0], dtype=np.float64)
    lib().orc_tables_build(n, g_lo, g_hi, length_unit_m, T, pion_sigma_mb, pion_eth_eV,
                           gdr_peak_mb, gdr_ec_eV, gdr_fwhm_eV, gdr_lo_eV, gdr_hi_eV,
                           _ptr(bp), _ptr(rp), _ptr(rg), int(nthreads), len(irb),
                           _ptr(irb_T), _ptr(irb_D))
    return Tables(n, g_lo, g_hi, bp, rp, rg)


def turbulence_modes(n, spacing, lmin, lmax, seed, index=-11.0 / 3.0):
    """Complex Fourier modes [nz, ny, nx, 3] of the turbulent field."""
    nx, ny, nz = n
    raw = np.zeros((nz, ny, nx, 3, 2), dtype=np.float64)
    lib().orc_turbulence_modes(nx, ny, nz, spacing, lmin, lmax, index, seed, _ptr(raw))
    return raw[..., 0] + 1j * raw[..., 1]


def turbulent_field(n, spacing, lmin, lmax, brms, seed, index=-11.0 / 3.0):
    """Real turbulent field [nz, ny, nx, 3] (float64): real part of the inverse
    FFT of the modes, mean removed, scaled so that <|B|^2> = brms^2."""
    modes = turbulence_modes(n, spacing, lmin, lmax, seed, index)
    B = np.empty(modes.shape, dtype=np.float64)
    for c in range(3):
        B[..., c] = np.fft.ifftn(modes[..., c], axes=(0, 1, 2)).real
    B -= B.mean(axis=(0, 1, 2), keepdims=True)
    ms = np.mean(np.sum(B * B, axis=-1))
    if ms > 0:
        B *= brms / np.sqrt(ms)
    return B


# ---------------------------------------------------------------------------
# Propagation
# ---------------------------------------------------------------------------
def make_params(*, grid_n, spacing, origin=(0.0, 0.0, 0.0), tol=1e-4, h_min=0.01, h_max=1.0,
                field_unit_T=NANOGAUSS_T, length_unit_m=MPC_M, flags=0, e_min=0.0,
                beta_ad=0.0, seed=0, tables: Tables | None = None,
                obs_c=(0.0, 0.0, 0.0), obs_r=0.0, border_c=(0.0, 0.0, 0.0), border_r=0.0,
                galactic=None, gmf: Gmf | None = None, max_steps=10_000_000,
                decay_table=None) -> Params:
    """decay_table: unstable nuclei for the DECAY module, a dict of arrays A, Z
    (A >= 2), tau_s (rest-frame mean lifetime, seconds) and branching [n, 4]
    (beta-, beta+, neutron emission, proton emission); nuclides not listed
    are stable."""
    P = Params()
    P.origin[:] = origin
    P.spacing = spacing
    P.n[:] = grid_n
    P.tol, P.h_min, P.h_max = tol, h_min, h_max
    P.curv_k = curvature_constant(field_unit_T, length_unit_m)
    P.length_unit_m = length_unit_m
    P.beta_ad, P.e_min = beta_ad, e_min
    P.flags = flags
    P.seed = seed
    if tables is not None:
        (P.tab_lg0, P.tab_inv_dlg), P.tab_n = tables.axis(), tables.n
    else:
        P.tab_n = 2
    P.obs_c[:] = obs_c
    P.obs_r = obs_r
    P.border_c[:] = border_c
    P.border_r = border_r
    if galactic is not None:
        for k, v in galactic.items():
            if k == "center":
                P.gal_center[:] = v
            else:
                setattr(P, "gal_" + k, v)
    if gmf is not None:
        P.gmf = gmf
    P.max_steps = max_steps
    if decay_table is not None:
        tab = nuclide_table(decay_table)
        P._nuc_ref = tab
        P.nuc_tab = tab.ctypes.data
        P.nuc_amax = int(round((np.sqrt(8 * len(tab) // 5 + 1) - 3) / 2))
    return P


def nuclide_table(decay_table) -> np.ndarray:
    """The oracle's dense lookup of a decay table: for 0 <= Z <= A <= A_max,
    entry A (A + 1) / 2 + Z holds [tau_s, b_beta-, b_beta+, b_n, b_p]
    (unlisted nuclides: infinite lifetime, all fractions 0)."""
    A = np.asarray(decay_table["A"], dtype=np.int64)
    Z = np.asarray(decay_table["Z"], dtype=np.int64)
    amax = int(A.max()) if len(A) else 2
    n = (amax + 1) * (amax + 2) // 2
    tab = np.zeros((n, 5))
    tab[:, 0] = np.inf
    idx = A * (A + 1) // 2 + Z
    tab[idx, 0] = np.asarray(decay_table["tau_s"], dtype=np.float64)
    tab[idx, 1:] = np.asarray(decay_table["branching"], dtype=np.float64)
    return np.ascontiguousarray(tab.reshape(-1))


def gmf_at(gmf: Gmf, pts, center=(0.0, 0.0, 0.0)):
    """The multi-arm galactic field alone at points [m, 3]."""
    P = make_params(grid_n=(2, 2, 2), spacing=1.0, flags=GMF, gmf=gmf,
                    galactic={"center": center})
    return field_at(P, np.zeros((2, 2, 2, 3)), pts)


def series_atan2(y, x):
    """The arctangent both sides steer the spiral phase with."""
    y = np.ascontiguousarray(y, dtype=np.float64).ravel()
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    out = np.empty_like(y)
    lib().orc_series_atan2_vec(len(y), _ptr(y), _ptr(x), _ptr(out))
    return out


def field_at(P: Params, field, pts):
    """Interpolated field at points [m, 3] (grid plus optional galactic part)."""
    field = np.ascontiguousarray(field, dtype=np.float64)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    out = np.zeros_like(pts)
    lib().orc_field_at(C.byref(P), _ptr(field), len(pts), _ptr(pts), _ptr(out))
    return out


def propagate(P: Params, field, inj: dict, tables: Tables | None = None, nthreads=None,
              out_cap=None):
    """Propagate injected candidates; returns a structured array of records
    (RECORD_DTYPE), primaries and all their secondaries, sorted by id."""
    field = np.ascontiguousarray(field, dtype=np.float64)
    n = len(inj["E"])
    nthreads = nthreads or os.cpu_count() or 1
    cols = {}
    for k in ("x", "y", "z", "ux", "uy", "uz", "E"):
        cols[k] = np.ascontiguousarray(inj[k], dtype=np.float64)
    ids = np.ascontiguousarray(inj["id"], dtype=np.uint64)
    s_max = np.ascontiguousarray(inj["s_max"], dtype=np.float64) if "s_max" in inj else None
    A = np.ascontiguousarray(inj["A"], dtype=np.int32)
    Z = np.ascontiguousarray(inj["Z"], dtype=np.int32)
    q = np.ascontiguousarray(inj["q"], dtype=np.int32) if "q" in inj else None
    if tables is None:
        dummy = np.zeros(2)
        tb = tp = tg = dummy
    else:
        tb, tp, tg = (np.ascontiguousarray(t, dtype=np.float64)
                      for t in (tables.beta_pair, tables.rate_pion, tables.rate_gdr))
    cap = out_cap or max(16, 4 * n)
    while True:
        out = np.zeros(cap, dtype=RECORD_DTYPE)
        n_out = C.c_int64(0)
        rc = lib().orc_propagate(C.byref(P), _ptr(field), _ptr(tb), _ptr(tp), _ptr(tg), n,
                                 _ptr(ids), _ptr(cols["x"]), _ptr(cols["y"]), _ptr(cols["z"]),
                                 _ptr(cols["ux"]), _ptr(cols["uy"]), _ptr(cols["uz"]),
                                 _ptr(cols["E"]), _ptr(s_max), _ptr(A), _ptr(Z), _ptr(q),
                                 _ptr(out), cap, C.byref(n_out), int(nthreads))
        if rc == -1:
            cap = int(n_out.value)
            continue
        if rc != 0:
            raise RuntimeError(f"oracle propagate failed: {rc}")
        out = out[: n_out.value]
        return np.sort(out, order="id")
