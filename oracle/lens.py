"""Galactic lens oracle (TEST INFRASTRUCTURE ONLY; see the package docstring).

The lensing technique of CRPropa 3.0 (Sect. 4, "Galactic propagation"): a set
of transformation matrices, one per energy (here: rigidity) bin, maps the
directions of cosmic rays at the border of the Galaxy to the directions
observed at Earth.  Readings (the paper gives no construction):

* Build by back-tracking (Sect. 4: forward- and back-tracking through the
  galactic field): antiparticles (charge sign -1) leave Earth along sampled
  arrival directions n_i (Earth pixel i = HEALPix RING pixel of n_i) at the
  bin's centre rigidity and are propagated to the border sphere; the border
  pixel j is the pixel of the antiparticle's direction there (the sky
  direction the particle came from).  N_b[i, j] counts samples.
* Normalisation: M_b = N_b / max_j sum_i N_b[i, j], so every column sums to at
  most 1; the remainder is "not observed".
* Storage: per (bin, column j) the list of sample Earth pixels, sorted
  ascending (a column's multiset of i with multiplicities N_b[i, j]).
* Apply: a candidate of rigidity R = E / Z arriving from sky direction -u
  (u: its direction of motion) goes to the bin containing R,
  b = floor((ln R - ln r_lo) * n_bins / (ln r_hi - ln r_lo)) clamped to
  [0, n_bins - 1] (logarithms by the atanh series), and to column
  j = pixel(-u); with the two uniforms (u1, u2) of Philox draw 0, tag 3 of
  its id it is observed if u1 * max_count_b < count_j, at Earth pixel
  entries[min(floor(u2 * count_j), count_j - 1)] of the sorted column.

Pins: the build by the zero-field case (straight lines: the lens is the
identity on pixels); the application by a hand-made lens whose outcome
frequencies match the column-normalised matrix (chi-square), with rigidity
bins by E / Z, clamping and bin edges; the synthetic disk + halo field the
lens is built through by its own pins (log-spiral field lines, vertical
profiles, halo parity and divergence).  Its values are those of the
synthetic model, not of a measured galactic field.
"""
from __future__ import annotations

import numpy as np

from . import DETECTED, AT_BORDER, ang2pix_vec, propagate, series_log, series_log_vec, uniform_pairs  # noqa: F401

TAG_LENS = 3
NOT_APPLIED = 0xFFFFFFFF
NOT_OBSERVED = 0xFFFFFFFE


def rigidity_bins(n_bins, r_lo, r_hi):
    """Bin edges (log-uniform) and geometric centres [V]."""
    edges = np.exp(np.linspace(np.log(r_lo), np.log(r_hi), n_bins + 1))
    return edges, np.sqrt(edges[:-1] * edges[1:])


def backtrack_samples(P, field, earth, dirs, bin_of_sample, centres, nthreads=None):
    """Back-track antiprotons from Earth; returns the oracle records sorted by
    id (id = sample index)."""
    n = len(dirs)
    E = centres[bin_of_sample]
    inj = dict(id=np.arange(n, dtype=np.uint64), x=np.full(n, earth[0]), y=np.full(n, earth[1]),
               z=np.full(n, earth[2]), ux=dirs[:, 0].copy(), uy=dirs[:, 1].copy(),
               uz=dirs[:, 2].copy(), E=E, A=np.ones(n, np.int32), Z=np.ones(n, np.int32),
               q=-np.ones(n, np.int32))
    return propagate(P, field, inj, nthreads=nthreads)


def build(nside, n_bins, bin_of_sample, dirs, records):
    """Lens from back-tracked records.  Returns dict(col_start, entries,
    max_count) with col_start of length n_bins * npix + 1."""
    npix = 12 * nside * nside
    ok = records["status"] == AT_BORDER
    i_earth = ang2pix_vec(nside, dirs)
    j_border = ang2pix_vec(nside, records["u"])
    key = bin_of_sample.astype(np.int64) * npix + j_border
    key, i_kept = key[ok], i_earth[ok]
    order = np.lexsort((i_kept, key))
    key, entries = key[order], i_kept[order].astype(np.uint32)
    counts = np.bincount(key, minlength=n_bins * npix)
    col_start = np.zeros(n_bins * npix + 1, dtype=np.uint32)
    col_start[1:] = np.cumsum(counts)
    max_count = counts.reshape(n_bins, npix).max(axis=1).astype(np.uint32)
    return dict(col_start=col_start, entries=entries, max_count=max_count)


def apply(lens, nside, r_lo, r_hi, n_bins, seed, ids, u, E, Z):
    """Earth pixel per candidate (NOT_OBSERVED when shadowed, NOT_APPLIED for
    neutral candidates)."""
    npix = 12 * nside * nside
    out = np.full(len(ids), NOT_APPLIED, dtype=np.uint32)
    charged = Z > 0
    R = E / np.maximum(Z, 1).astype(np.float64)
    lg_lo = series_log(r_lo)
    inv = float(n_bins) / (series_log(r_hi) - lg_lo)
    t = (series_log_vec(R) - lg_lo) * inv
    b = np.clip(np.floor(t), 0, n_bins - 1).astype(np.int64)
    j = ang2pix_vec(nside, -u)
    col = b * npix + j
    start = lens["col_start"][col].astype(np.int64)
    count = lens["col_start"][col + 1].astype(np.int64) - start
    mx = lens["max_count"][b].astype(np.float64)
    uu = uniform_pairs(seed, TAG_LENS, 0, ids)
    observed = (count > 0) & (uu[:, 0] * mx < count)
    pick = np.minimum((uu[:, 1] * count).astype(np.int64), np.maximum(count - 1, 0))
    res = np.where(observed, lens["entries"][np.where(observed, start + pick, 0)], NOT_OBSERVED)
    out[charged] = res[charged].astype(np.uint32)
    return out
