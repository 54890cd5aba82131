"""1D mode with cosmology and the a-posteriori 3D cosmology correction
(TEST INFRASTRUCTURE ONLY; see the package docstring).

The paper's Sect. 2 lists the 1D mode with cosmological effects (redshift
evolution of the photon backgrounds, adiabatic expansion); Sect. 4
("Cosmology in 3D") corrects a 3D run made without cosmology: each observed
particle is re-simulated in 1D from its injected energy and species with the
source at the distance of its 3D trajectory length (read as a comoving
distance), and one of the 1D
products that reach the observer, drawn at random, replaces it.  Readings
are listed in crp_oracle.cpp (flat Lambda-CDM; redshift steps with midpoint
comoving length; exact adiabatic factor; (1+z)^2 rate((1+z) Gamma) per
comoving length from the z = 0 tables; optical depths for stochastic
states; the source redshift is the one whose comoving distance equals the
trajectory length; product pick by Philox tag 5).

Pins (tests/test_oracle_pins.py): adiabatic-only propagation gives
E_obs = E_src / (1 + z) exactly; the light-travel distance agrees with a
library quadrature; the pair loss rate at redshift z equals the blackbody
loss at temperature T0 (1 + z); the fraction of protons reaching the
observer without a pion event equals exp(-optical depth) from a library
quadrature.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import RECORD_DTYPE, Tables, lib, _ptr  # noqa: F401

H0_KM_S_MPC = 67.3
OMEGA_M = 0.315
C_KM_S = 299792.458


class Params1d(C.Structure):
    _fields_ = [("flags", C.c_uint32), ("pad0", C.c_uint32), ("seed", C.c_uint64),
                ("e_min", C.c_double), ("H0", C.c_double), ("omega_m", C.c_double),
                ("omega_l", C.c_double), ("dz_max", C.c_double), ("loss_max", C.c_double),
                ("tab_lg0", C.c_double), ("tab_inv_dlg", C.c_double), ("tab_n", C.c_int64),
                ("length_unit_m", C.c_double), ("max_steps", C.c_int64)]


_declared = False


def _lib():
    global _declared
    L = lib()
    if not _declared:
        p, i64, d = C.c_void_p, C.c_int64, C.c_double
        P = C.POINTER(Params1d)
        L.orc_propagate_1d.argtypes = [P, p, p, p, i64, p, p, p, p, p, p, i64,
                                       C.POINTER(i64), C.c_int]
        L.orc_propagate_1d.restype = C.c_int
        L.orc_comoving_distance.argtypes = [P, i64, p, p]
        L.orc_redshift_of_distance.argtypes = [P, i64, p, p]
        L.orc_cosmology_pick.argtypes = [P, p, p, p, i64, p, p, p, p, p, p, p, p, p, C.c_int]
        L.orc_cosmology_pick.restype = C.c_int
        _declared = True
    return L


def make_params1d(*, tables: Tables | None = None, flags=0, seed=0, e_min=0.0,
                  H0_km_s_Mpc=H0_KM_S_MPC, omega_m=OMEGA_M, dz_max=1e-3, loss_max=1e-3,
                  length_unit_m=3.0856775814913673e22, max_steps=10_000_000) -> Params1d:
    """Lengths in Mpc by default; H0 enters as H0 / c per length unit."""
    P = Params1d()
    P.flags, P.seed, P.e_min = flags, seed, e_min
    mpc_per_unit = length_unit_m / 3.0856775814913673e22
    P.H0 = H0_km_s_Mpc / C_KM_S * mpc_per_unit
    P.omega_m, P.omega_l = omega_m, 1.0 - omega_m
    P.dz_max, P.loss_max = dz_max, loss_max
    if tables is not None:
        P.tab_lg0 = np.log(tables.g_lo)
        P.tab_inv_dlg = (tables.n - 1) / (np.log(tables.g_hi) - np.log(tables.g_lo))
        P.tab_n = tables.n
    else:
        P.tab_lg0, P.tab_inv_dlg, P.tab_n = 0.0, 1.0, 2
    P.length_unit_m, P.max_steps = length_unit_m, max_steps
    return P


def _tab(tables):
    if tables is None:
        z = np.zeros(2)
        return z, z, z
    return tables.beta_pair, tables.rate_pion, tables.rate_gdr


def propagate_1d(P: Params1d, inj: dict, tables: Tables | None = None, nthreads=None):
    """inj: id, z (source redshift), E, A, Z.  Records sorted by id."""
    n = len(inj["E"])
    nthreads = nthreads or os.cpu_count() or 1
    ids = np.ascontiguousarray(inj["id"], dtype=np.uint64)
    z = np.ascontiguousarray(inj["z"], dtype=np.float64)
    E = np.ascontiguousarray(inj["E"], dtype=np.float64)
    A = np.ascontiguousarray(inj["A"], dtype=np.int32)
    Z = np.ascontiguousarray(inj["Z"], dtype=np.int32)
    tb, tp, tg = _tab(tables)
    cap = max(16, 4 * n)
    while True:
        out = np.zeros(cap, dtype=RECORD_DTYPE)
        n_out = C.c_int64()
        rc = _lib().orc_propagate_1d(C.byref(P), _ptr(tb), _ptr(tp), _ptr(tg), n, _ptr(ids),
                                     _ptr(z), _ptr(E), _ptr(A), _ptr(Z), _ptr(out), cap,
                                     C.byref(n_out), int(nthreads))
        if rc == 0:
            return np.sort(out[: n_out.value], order="id")
        if rc != -1:
            raise RuntimeError(f"orc_propagate_1d: {rc}")
        cap = n_out.value


def comoving_distance(P: Params1d, z):
    z = np.ascontiguousarray(z, dtype=np.float64).ravel()
    out = np.zeros_like(z)
    _lib().orc_comoving_distance(C.byref(P), len(z), _ptr(z), _ptr(out))
    return out


def redshift_of_distance(P: Params1d, D):
    D = np.ascontiguousarray(D, dtype=np.float64).ravel()
    out = np.zeros_like(D)
    _lib().orc_redshift_of_distance(C.byref(P), len(D), _ptr(D), _ptr(out))
    return out


def cosmology_pick(P: Params1d, ids, z_src, E, A, Z, tables: Tables | None = None,
                   nthreads=None):
    """The correction's 1D re-simulation and product pick: (E, A, Z, n_products)."""
    n = len(E)
    nthreads = nthreads or os.cpu_count() or 1
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    z_src = np.ascontiguousarray(z_src, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    A = np.ascontiguousarray(A, dtype=np.int32)
    Z = np.ascontiguousarray(Z, dtype=np.int32)
    Eo, Ao, Zo, nk = np.zeros(n), np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.int32)
    tb, tp, tg = _tab(tables)
    rc = _lib().orc_cosmology_pick(C.byref(P), _ptr(tb), _ptr(tp), _ptr(tg), n, _ptr(ids),
                                   _ptr(z_src), _ptr(E), _ptr(A), _ptr(Z), _ptr(Eo), _ptr(Ao),
                                   _ptr(Zo), _ptr(nk), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"orc_cosmology_pick: {rc}")
    return Eo, Ao, Zo, nk
