"""Seeded synthetic workloads shaped like the paper's scenarios.

This module only draws injection arrays and holds workload sizes.  It contains
none of the propagation method's arithmetic, so the CUDA library and the CPU
oracle can both be fed from it.  Draws use numpy's Philox bit generator keyed
by the workload seed; the arrays are handed bit-identically to both sides.

Source model (the paper's Sect. 3 source class composed of position,
spectrum and composition properties):
  * spectrum: power law dN/dE ~ E^-2 between e_lo and e_hi by inverse CDF;
  * directions: isotropic, cos(theta) = 2 u1 - 1, phi = 2 pi u2;
  * composition: by number fractions over (A, Z) species;
  * positions: one point, or a set of uniform sources in a box.
"""
from __future__ import annotations

import numpy as np

MASTER_SEED = 1307264300

# (A, Z, fraction by number) of the mixed composition: H, He, N, Fe
MIXED_COMPOSITION = ((1, 1, 0.40), (4, 2, 0.25), (14, 7, 0.20), (56, 26, 0.15))


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=seed))


def power_law_e2(g, n, e_lo, e_hi):
    """E^-2 by inverse CDF; e_lo / e_hi may be arrays (per-candidate bounds)."""
    u = g.random(n)
    return 1.0 / (1.0 / e_lo - u * (1.0 / e_lo - 1.0 / e_hi))


def isotropic(g, n):
    u1, u2 = g.random(n), g.random(n)
    ct = 2.0 * u1 - 1.0
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    ph = 2.0 * np.pi * u2
    return st * np.cos(ph), st * np.sin(ph), ct


# ---------------------------------------------------------------------------
# Workload descriptions (field, integrator, modules); units Mpc / nG / eV for
# the extragalactic ones, kpc / microgauss for the galactic one.
# ---------------------------------------------------------------------------
PLAIN_SMALL = dict(          # 10^4 protons, 64^3 float64 field, no interactions
    name="plain_small_1e4p_64cube_f64",
    n=10_000, grid_n=(64, 64, 64), spacing=0.25, lmin=0.5, lmax=8.0, brms=1.0,
    field_dtype="f64", tol=1e-4, h_min=0.01, h_max=1.0, s_max=50.0,
    e_lo=1e19, e_hi=1e20, seed=MASTER_SEED + 1,
)

MIXED_INTERACTIONS = dict(   # 10^6 mixed nuclei, 256^3 float32 field, losses + pion
    name="mixed_1e6_256cube_f32_pair_adiab_pion_observer",
    n=1_000_000, grid_n=(256, 256, 256), spacing=0.1, lmin=0.2, lmax=5.0, brms=1.0,
    field_dtype="f32", tol=1e-4, h_min=0.01, h_max=1.0, s_max=500.0,
    e_lo=1e18, e_hi_per_z=1e21 / 26.0, e_min=1e18, n_sources=1000, box=50.0,
    observer_r=1.0, seed=MASTER_SEED + 2,
)

UNEVEN_SECONDARIES = dict(   # 10^7, 512^3 float32 field, photodisintegration + queue
    name="uneven_1e7_512cube_f32_photodis_queue",
    n=10_000_000, grid_n=(512, 512, 512), spacing=0.25, lmin=0.5, lmax=8.0,
    brms_lo=0.1, brms_hi=10.0, field_dtype="f32", tol=1e-4, h_min=0.01, h_max=1.0,
    s_lo=1.0, s_hi=2000.0, e_lo=1e18, e_hi_per_z=1e21 / 26.0, e_min=1e18, n_sources=1000,
    box=50.0, observer_r=1.0, seed=MASTER_SEED + 3,
)


def plain_small(n=None, seed=None):
    """Protons from the origin, E^-2 on [1e19, 1e20] eV, isotropic."""
    w = PLAIN_SMALL
    n = w["n"] if n is None else n
    g = rng(w["seed"] if seed is None else seed)
    E = power_law_e2(g, n, w["e_lo"], w["e_hi"])
    ux, uy, uz = isotropic(g, n)
    z = np.zeros(n)
    return dict(id=np.arange(n, dtype=np.uint64), x=z.copy(), y=z.copy(), z=z.copy(),
                ux=ux, uy=uy, uz=uz, E=E, A=np.ones(n, np.int32), Z=np.ones(n, np.int32),
                q=np.ones(n, np.int32), s_max=np.full(n, w["s_max"]))


def _sources(g, n_sources, box, r_excl):
    pts = np.empty((0, 3))
    while len(pts) < n_sources:
        p = g.uniform(-box, box, size=(n_sources, 3))
        p = p[np.sum(p * p, axis=1) > r_excl * r_excl]
        pts = np.concatenate([pts, p])
    return pts[:n_sources]


def _mixed(g, n, w):
    frac = np.array([c[2] for c in MIXED_COMPOSITION])
    species = np.searchsorted(np.cumsum(frac), g.random(n), side="right")
    species = np.minimum(species, len(frac) - 1)
    A = np.array([c[0] for c in MIXED_COMPOSITION], np.int32)[species]
    Z = np.array([c[1] for c in MIXED_COMPOSITION], np.int32)[species]
    E = power_law_e2(g, n, w["e_lo"], w["e_hi_per_z"] * Z)
    src = _sources(g, w["n_sources"], w["box"], w["observer_r"])
    which = g.integers(0, w["n_sources"], size=n)
    ux, uy, uz = isotropic(g, n)
    pos = src[which]
    return dict(id=np.arange(n, dtype=np.uint64), x=pos[:, 0].copy(), y=pos[:, 1].copy(),
                z=pos[:, 2].copy(), ux=ux, uy=uy, uz=uz, E=E, A=A, Z=Z,
                q=np.ones(n, np.int32))


def mixed_interactions(n=None, seed=None):
    """Mixed H/He/N/Fe from 1000 uniform sources in a 100 Mpc box."""
    w = MIXED_INTERACTIONS
    n = w["n"] if n is None else n
    g = rng(w["seed"] if seed is None else seed)
    d = _mixed(g, n, w)
    d["s_max"] = np.full(n, w["s_max"])
    return d


def uneven_secondaries(n=None, seed=None):
    """As the mixed workload, with per-candidate path budgets log-uniform in
    [1 Mpc, 2 Gpc]; also returns the run's B_rms (log-uniform in [0.1, 10] nG)."""
    w = UNEVEN_SECONDARIES
    n = w["n"] if n is None else n
    g = rng(w["seed"] if seed is None else seed)
    brms = float(np.exp(g.uniform(np.log(w["brms_lo"]), np.log(w["brms_hi"]))))
    d = _mixed(g, n, w)
    d["s_max"] = np.exp(g.uniform(np.log(w["s_lo"]), np.log(w["s_hi"]), size=n))
    return d, brms


def subsample(inj: dict, idx) -> dict:
    """Candidates with the given indices (ids are kept, so every stochastic
    history is the same as in the full run)."""
    return {k: np.ascontiguousarray(v[idx]) for k, v in inj.items()}


GALACTIC_LENS = dict(       # back-tracking through a synthetic galactic field (kpc, microgauss)
    name="galactic_backtrack_256cube_f32_disk_halo_random",
    grid_n=(256, 256, 256), box=40.0, brms=3.0, lmax=2.0, field_dtype="f32",
    disk=dict(disk_b=2.0, disk_pitch_rad=11.5 * np.pi / 180.0, disk_hz=1.0, disk_rmin=3.0,
              disk_rmax=20.0, halo_b=1.0, halo_z0=1.5, halo_sigma=1.0, center=(0.0, 0.0, 0.0)),
    earth=(-8.5, 0.0, 0.0), border_r=20.0, tol=1e-4, h_min=0.001, h_max=0.05,
    r_lo=1e18, r_hi=1e20, n_bins=100, nside=64, seed=MASTER_SEED + 4,
)


def flux_free_last_arm(arm_b7, arm_rx, pitch_rad):
    """Eighth arm strength for which the spiral disk has no net radial flux
    through a circle: at fixed r, arm j spans ln(rx[j+1] / rx[j]) / tan p in
    azimuth (rx[8] = rx[0] e^{2 pi tan p}) with B_r = b_j (r_in / r) sin p, so
    sum_j b_j ln(rx[j+1] / rx[j]) = 0 fixes b_8."""
    rx = list(arm_rx) + [arm_rx[0] * np.exp(2.0 * np.pi * np.tan(pitch_rad))]
    w = [np.log(rx[j + 1] / rx[j]) for j in range(8)]
    return -sum(b * wj for b, wj in zip(arm_b7, w[:7])) / w[7]


def multiarm_gmf_params():
    """Synthetic parameters of the analytic multi-arm galactic field (kpc, uG):
    eight logarithmic spiral arms (pitch 11.5 deg) between 5 and 20 kpc with a
    ring inside, a north/south toroidal halo and an X-shaped poloidal field;
    values chosen for this workload, not fitted to data."""
    pitch = 11.5 * np.pi / 180.0
    arm_rx = (5.0, 6.0, 7.0, 8.5, 10.0, 11.5, 13.0, 15.0)
    arm_b7 = (0.5, 2.5, -1.0, -0.5, -2.0, -3.5, 0.5)
    arm_b = arm_b7 + (flux_free_last_arm(arm_b7, arm_rx, pitch),)
    return dict(arm_b=arm_b, arm_rx=arm_rx, pitch_rad=pitch, ring_b=0.2, r_ring=3.0,
                r_in=5.0, r_out=20.0, h_disk=0.4, w_disk=0.25, halo_bn=1.2, halo_bs=-1.0,
                halo_rn=9.0, halo_rs=15.0, halo_wh=0.2, halo_z0=5.0, x_b=4.0,
                x_theta_rad=50.0 * np.pi / 180.0, x_rc=5.0, x_r=3.0, r_cut_in=1.0,
                r_cut_out=20.0)


GALACTIC_MULTIARM = dict(   # back-tracking through the analytic multi-arm field alone
    name="galactic_backtrack_multiarm_analytic",
    earth=(-8.5, 0.0, 0.0), border_r=20.0, tol=1e-4, h_min=0.001, h_max=0.05,
    r_lo=1e18, r_hi=1e20, n_bins=100, nside=64, seed=MASTER_SEED + 7,
)


def galactic_grid_geometry(n=256, box=40.0):
    """Node spacing, lmin (= 2 spacings) and origin of a periodic random-field
    grid of n^3 nodes filling a cube of side `box` centred on the Galactic centre."""
    spacing = box / n
    return spacing, 2.0 * spacing, (-0.5 * box, -0.5 * box, -0.5 * box)


def lens_samples(n_bins, per_bin, r_lo, r_hi, seed):
    """Isotropic arrival directions, per_bin per rigidity bin; each sample at
    its bin's geometric-centre rigidity (energy of a proton, eV)."""
    g = rng(seed)
    n = n_bins * per_bin
    ux, uy, uz = isotropic(g, n)
    edges = np.exp(np.linspace(np.log(r_lo), np.log(r_hi), n_bins + 1))
    centres = np.sqrt(edges[:-1] * edges[1:])
    bins = np.repeat(np.arange(n_bins, dtype=np.int32), per_bin)
    return np.stack([ux, uy, uz], axis=1), centres[bins], bins


def backtrack_directions(n, r_lo, r_hi, seed):
    """Isotropic arrival directions with rigidities log-uniform in [r_lo, r_hi]."""
    g = rng(seed)
    ux, uy, uz = isotropic(g, n)
    R = np.exp(g.uniform(np.log(r_lo), np.log(r_hi), n))
    return np.stack([ux, uy, uz], axis=1), R


def beta_stability_z(A):
    """Charge of the beta-stability line at mass number A: Green's
    approximation Z = A / (1.98 + 0.0155 A^(2/3)) (from the semi-empirical
    mass formula)."""
    A = np.asarray(A, dtype=np.float64)
    return A / (1.98 + 0.0155 * A ** (2.0 / 3.0))


def synthetic_decay_table(a_max=56, tau0_s=1.0e6, decades_per_charge=2.0, width=1.0,
                          drip=3.0):
    """Synthetic lifetimes and branchings of unstable nuclei (input data; the
    measured tables are not in the container).  For 2 <= A <= a_max and
    1 <= Z <= A - 1, with D = Z - Z_s(A) the distance from the beta-stability
    line: stable for |D| <= width; otherwise the rest-frame mean lifetime is
    tau0_s * 10^(-decades_per_charge (|D| - width)) seconds, and the nucleus
    beta decays toward the line (beta+ for D > 0, beta- for D < 0) except for
    a fraction min(0.9, 0.3 (|D| - drip)) beyond |D| > drip, which emits a
    nucleon (proton for D > 0, neutron for D < 0).  A channel whose daughter
    would have Z' = 0 or N' = 0 with A' >= 2 is left out.  Returns dict(A, Z,
    tau_s, branching [n, 4]: beta-, beta+, neutron emission, proton
    emission) of the unstable nuclides only."""
    rows = []
    for A in range(2, a_max + 1):
        zs = float(beta_stability_z(A))
        for Z in range(1, A):
            D = Z - zs
            if abs(D) <= width:
                continue
            tau = tau0_s * 10.0 ** (-decades_per_charge * (abs(D) - width))
            f_nuc = min(0.9, 0.3 * (abs(D) - drip)) if abs(D) > drip else 0.0
            b = np.zeros(4)
            if D > 0:
                b[1], b[3] = 1.0 - f_nuc, f_nuc
            else:
                b[0], b[2] = 1.0 - f_nuc, f_nuc
            # daughters: beta- (A, Z+1), beta+ (A, Z-1), n (A-1, Z), p (A-1, Z-1)
            for k, (Ad, Zd) in enumerate(((A, Z + 1), (A, Z - 1), (A - 1, Z), (A - 1, Z - 1))):
                if b[k] > 0 and Ad >= 2 and (Zd <= 0 or Zd >= Ad):
                    b[k] = 0.0
            if b.sum() == 0.0:
                continue
            b /= b.sum()
            rows.append((A, Z, tau, b))
    return dict(A=np.array([r[0] for r in rows], np.int32),
                Z=np.array([r[1] for r in rows], np.int32),
                tau_s=np.array([r[2] for r in rows]),
                branching=np.array([r[3] for r in rows]))
