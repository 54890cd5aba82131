"""Pins of the oracle's lens build and apply on a hand-made lens: columns are
the sorted Earth pixels of the samples that left through each border pixel;
applying the lens draws Earth pixel i of column j with probability
N[i, j] / max_j' sum_i N[i, j'] (the column-normalised matrix) and "not
observed" with the rest, measured here by chi-square on 2*10^5 candidates;
rigidity bins by E / Z, clamped at both ends; neutral candidates untouched.
A column taken from +u instead of -u, a normalisation by the column's own
sum, or a bin taken from E instead of E / Z each fail one of them."""
import numpy as np
from scipy.stats import chisquare

NSIDE, NB, R_LO, R_HI = 2, 2, 1e18, 1e20
# (rigidity bin, border pixel j) -> {Earth pixel i: N[i, j]}
COLS = {(0, 5): {3: 5, 10: 2, 40: 1}, (0, 17): {17: 12}, (1, 5): {0: 1, 47: 3}}


def _centre(oracle, pix):
    z, phi = oracle.pix2ang(NSIDE, pix)
    s = np.sqrt(1.0 - z * z)
    return np.array([s * np.cos(phi), s * np.sin(phi), z])


def _lens(oracle):
    import oracle.lens as L
    dirs, border, bins, status = [], [], [], []
    for (b, j), col in COLS.items():
        for i, m in col.items():
            dirs += [_centre(oracle, i)] * m
            border += [_centre(oracle, j)] * m
            bins += [b] * m
            status += [oracle.AT_BORDER] * m
    # samples that never reached the border carry no count
    for i in (3, 10, 17):
        dirs.append(_centre(oracle, i))
        border.append(_centre(oracle, 5))
        bins.append(0)
        status.append(oracle.DETECTED)
    rec = dict(status=np.array(status), u=np.array(border))
    return L, L.build(NSIDE, NB, np.array(bins), np.array(dirs), rec)


def test_build_columns_and_normalisation(oracle):
    L, lens = _lens(oracle)
    npix = 12 * NSIDE * NSIDE
    assert len(lens["col_start"]) == NB * npix + 1
    assert list(lens["max_count"]) == [12, 4]
    for c in range(NB * npix):
        col = list(lens["entries"][lens["col_start"][c]:lens["col_start"][c + 1]])
        want = sorted(i for i, m in COLS.get((c // npix, c % npix), {}).items() for _ in range(m))
        assert col == want, c


def _apply(oracle, L, lens, u, E, Z, seed=21):
    n = len(E)
    return L.apply(lens, NSIDE, R_LO, R_HI, NB, seed, np.arange(n, dtype=np.uint64),
                   np.repeat(u[None, :], n, axis=0), np.asarray(E, dtype=np.float64),
                   np.asarray(Z, dtype=np.int32))


def _check_frequencies(out, probs):
    """probs: {outcome: probability}, outcomes with probability 0 never seen."""
    keys = sorted(probs)
    assert set(np.unique(out)) <= {k for k in keys if probs[k] > 0}
    obs = np.array([np.sum(out == k) for k in keys if probs[k] > 0], dtype=float)
    exp = np.array([probs[k] for k in keys if probs[k] > 0]) * len(out)
    if len(obs) > 1:
        assert chisquare(obs, exp).pvalue > 1e-3, (obs, exp)


def test_apply_samples_the_normalised_matrix(oracle):
    L, lens = _lens(oracle)
    n = 200_000
    u = -_centre(oracle, 5)                       # moving away from border pixel 5
    # bin 0 (protons at 3 EeV): counts 5, 2, 1 of max 12
    out = _apply(oracle, L, lens, u, np.full(n, 3e18), np.ones(n))
    _check_frequencies(out, {3: 5 / 12, 10: 2 / 12, 40: 1 / 12, L.NOT_OBSERVED: 4 / 12})
    # the same rigidity as iron: E / Z picks the bin
    out_fe = _apply(oracle, L, lens, u, np.full(n, 26 * 3e18), np.full(n, 26))
    _check_frequencies(out_fe, {3: 5 / 12, 10: 2 / 12, 40: 1 / 12, L.NOT_OBSERVED: 4 / 12})
    # bin 1: the fullest column, always observed
    out = _apply(oracle, L, lens, u, np.full(n, 3e19), np.ones(n))
    _check_frequencies(out, {0: 1 / 4, 47: 3 / 4})
    # below and above the binned range: clamped to the end bins
    assert set(_apply(oracle, L, lens, u, np.full(1000, 1e16), np.ones(1000))) <= {3, 10, 40, L.NOT_OBSERVED}
    assert set(_apply(oracle, L, lens, u, np.full(1000, 1e22), np.ones(1000))) <= {0, 47}
    # a column with no samples: never observed; neutral candidates: not applied
    u17 = -_centre(oracle, 17)
    assert np.all(_apply(oracle, L, lens, u17, np.full(100, 3e19), np.ones(100)) == L.NOT_OBSERVED)
    assert np.all(_apply(oracle, L, lens, u17, np.full(100, 3e18), np.ones(100)) == 17)
    assert np.all(_apply(oracle, L, lens, u, np.full(100, 3e18), np.zeros(100)) == L.NOT_APPLIED)


def test_apply_bin_edges(oracle):
    """The bin edge between the two bins is at R = 10^19 (log-uniform): just
    below goes to bin 0 (pixel set {3, 10, 40}), just above to bin 1 ({0, 47})."""
    L, lens = _lens(oracle)
    u = -_centre(oracle, 5)
    lo = _apply(oracle, L, lens, u, np.full(2000, 1e19 * (1 - 1e-9)), np.ones(2000))
    hi = _apply(oracle, L, lens, u, np.full(2000, 1e19 * (1 + 1e-9)), np.ones(2000))
    assert set(lo) <= {3, 10, 40, L.NOT_OBSERVED} and set(hi) <= {0, 47}
