"""Pins of the CPU oracle to facts fixed outside the oracle itself: published
known-answer vectors, the order conditions of the Cash-Karp tableau, the
analytic helix in a uniform field, time reversal of the Lorentz force, the
spectral properties of the generated turbulence, closed forms of the
interaction rates, blackbody integrals and sampling statistics.

Each test states which published fact it checks; none re-types the oracle's
own formula as its expected value.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11)
# ---------------------------------------------------------------------------
def test_philox_known_answers(oracle):
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(o) for o in out] == v[6:10]


def test_uniform_open_interval(oracle):
    assert oracle.uniform_open(0, 0) == 2.0 ** -53
    assert oracle.uniform_open(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert oracle.uniform_open(0, 0x80000000) == 0.5 + 2.0 ** -53


def test_child_ids_unique(oracle):
    ids = {oracle.child_id(p, e) for p in range(2000) for e in range(40)}
    assert len(ids) == 2000 * 40
    assert not (ids & set(range(2000)))


# ---------------------------------------------------------------------------
# Cash-Karp 5(4) tableau (Cash & Karp, ACM TOMS 16, 201, 1990): the Butcher
# order conditions (rooted trees up to order 5 for the fifth-order weights,
# up to order 4 for the embedded weights) hold exactly for the rationals the
# oracle's doubles round from.
# ---------------------------------------------------------------------------
def _order_conditions(b, A, c, order):
    """Residuals of the Butcher order conditions up to `order` (Fractions)."""
    s = len(b)
    dot = lambda u, v: sum(x * y for x, y in zip(u, v))
    Av = lambda v: [sum(A[i][j] * v[j] for j in range(s)) for i in range(s)]
    mul = lambda u, v: [x * y for x, y in zip(u, v)]
    one = [Fraction(1)] * s
    Ac = Av(c)
    res = [dot(b, one) - 1]
    if order >= 2:
        res += [dot(b, c) - Fraction(1, 2)]
    if order >= 3:
        res += [dot(b, mul(c, c)) - Fraction(1, 3), dot(b, Ac) - Fraction(1, 6)]
    if order >= 4:
        c2 = mul(c, c)
        res += [dot(b, mul(c2, c)) - Fraction(1, 4), dot(b, mul(c, Ac)) - Fraction(1, 8),
                dot(b, Av(c2)) - Fraction(1, 12), dot(b, Av(Ac)) - Fraction(1, 24)]
    if order >= 5:
        c2 = mul(c, c)
        c3 = mul(c2, c)
        res += [dot(b, mul(c2, c2)) - Fraction(1, 5),
                dot(b, mul(c2, Ac)) - Fraction(1, 10),
                dot(b, mul(Ac, Ac)) - Fraction(1, 20),
                dot(b, mul(c, Av(c2))) - Fraction(1, 15),
                dot(b, Av(c3)) - Fraction(1, 20),
                dot(b, mul(c, Av(Ac))) - Fraction(1, 30),
                dot(b, Av(mul(c, Ac))) - Fraction(1, 40),
                dot(b, Av(Av(c2))) - Fraction(1, 60),
                dot(b, Av(Av(Ac))) - Fraction(1, 120)]
    return res


def test_cash_karp_order_conditions(oracle):
    T = oracle.cash_karp_tableau()
    F = {k: Fraction(v).limit_denominator(10 ** 6) for k, v in T.items()}
    for k, v in T.items():  # each double is the nearest double of its rational
        assert float(F[k]) == v, k
    A = [[Fraction(0)] * 6 for _ in range(6)]
    A[1][0] = F["b21"]
    A[2][:2] = [F["b31"], F["b32"]]
    A[3][:3] = [F["b41"], F["b42"], F["b43"]]
    A[4][:4] = [F["b51"], F["b52"], F["b53"], F["b54"]]
    A[5][:5] = [F["b61"], F["b62"], F["b63"], F["b64"], F["b65"]]
    c = [sum(row) for row in A]           # row-sum nodes
    assert c == [0, Fraction(1, 5), Fraction(3, 10), Fraction(3, 5), 1, Fraction(7, 8)]
    b5 = [F["c1"], Fraction(0), F["c3"], F["c4"], Fraction(0), F["c6"]]
    e = [F["e1"], Fraction(0), F["e3"], F["e4"], F["e5"], F["e6"]]
    b4 = [x - y for x, y in zip(b5, e)]
    assert all(r == 0 for r in _order_conditions(b5, A, c, 5))
    assert all(r == 0 for r in _order_conditions(b4, A, c, 4))
    # the embedded pair really differs at fifth order (the error estimate is live)
    assert any(r != 0 for r in _order_conditions(b4, A, c, 5))


# ---------------------------------------------------------------------------
# Uniform field: analytic helix with Larmor radius r_L = E / (Z e c B).
# ---------------------------------------------------------------------------
def _uniform_field(n=4, bz=1.0):
    B = np.zeros((n, n, n, 3))
    B[..., 2] = bz
    return B


def _one(E, ux=1.0, uy=0.0, uz=0.0, A=1, Z=1, q=1, s_max=1.0, x=(0.0, 0.0, 0.0), n=1):
    return dict(id=np.arange(n, dtype=np.uint64), x=np.full(n, x[0]), y=np.full(n, x[1]),
                z=np.full(n, x[2]), ux=np.full(n, ux), uy=np.full(n, uy), uz=np.full(n, uz),
                E=np.full(n, E), A=np.full(n, A, np.int32), Z=np.full(n, Z, np.int32),
                q=np.full(n, q, np.int32), s_max=np.full(n, s_max))


def _larmor_mpc(E_eV, Z, B_nG):
    # SI: r = p c / (Z e c B) = E[J] / (Z e c B[T]) = E[eV] / (Z c B[T]) metres
    return E_eV / (Z * 299792458.0 * B_nG * 1e-13) / 3.0856775814913673e22


def test_helix_half_turn(oracle):
    E = 1e19
    rl = _larmor_mpc(E, 1, 1.0)
    assert abs(rl - 10.810) < 1e-3  # 1.0810 Mpc per EeV per nG, times 10 EeV
    P = oracle.make_params(grid_n=(4, 4, 4), spacing=1.0, tol=1e-9, h_min=1e-6, h_max=1.0)
    r = oracle.propagate(P, _uniform_field(), _one(E, s_max=math.pi * rl))[0]
    # positive charge, u = +x, B = +z: force along -y, centre at (0, -r_L, 0)
    assert np.allclose(r["x"], [0.0, -2.0 * rl, 0.0], atol=1e-6 * rl)
    assert np.allclose(r["u"], [-1.0, 0.0, 0.0], atol=1e-7)
    assert abs(np.linalg.norm(r["u"]) - 1.0) < 1e-14
    assert r["E"] == E and r["status"] == oracle.MAX_LENGTH and r["s"] == math.pi * rl


def test_helix_pitch_and_antiparticle(oracle):
    E, rl = 3e19, _larmor_mpc(3e19, 2, 1.0)
    ct = 0.6
    P = oracle.make_params(grid_n=(4, 4, 4), spacing=1.0, tol=1e-9, h_min=1e-6, h_max=1.0)
    inj = _one(E, ux=0.8, uz=ct, A=4, Z=2, q=-1, s_max=2 * math.pi * rl)
    r = oracle.propagate(P, _uniform_field(), inj)[0]
    # u precesses about B at 1/r_L per unit path whatever the pitch: after
    # s = 2 pi r_L one full gyration, drift along B = s cos(pitch)
    assert np.allclose(r["x"], [0.0, 0.0, ct * 2 * math.pi * rl], atol=1e-6 * rl)
    # antiparticle (q = -1) gyrates the other way: after a quarter turn
    inj["s_max"] = np.full(1, 0.5 * math.pi * rl)
    r = oracle.propagate(P, _uniform_field(), inj)[0]
    assert np.allclose(r["x"][:2], [0.8 * rl, 0.8 * rl], atol=1e-6 * rl)


def test_convergence_order_five(oracle):
    """Global error of fixed-step Cash-Karp on the helix falls as h^5."""
    E = 1e19
    rl = _larmor_mpc(E, 1, 1.0)
    errs = []
    s = 4.0 * rl
    for m in (16, 32, 64):
        h = rl / m
        P = oracle.make_params(grid_n=(4, 4, 4), spacing=1.0, tol=1e30, h_min=h, h_max=h)
        r = oracle.propagate(P, _uniform_field(), _one(E, s_max=s))[0]
        assert r["n_acc"] in (4 * m, 4 * m + 1)  # last step may be a rounding sliver
        exact = np.array([rl * math.sin(s / rl), -rl * (1 - math.cos(s / rl)), 0.0])
        errs.append(np.linalg.norm(r["x"] - exact))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(4.7 < sl < 5.4 for sl in slopes), (errs, slopes)


# ---------------------------------------------------------------------------
# Time reversal: reversing the direction and the charge retraces the path.
# ---------------------------------------------------------------------------
def test_backtrack_returns_to_start(oracle):
    n, dx = (32, 32, 32), 0.25
    B = oracle.turbulent_field(n, dx, 0.5, 4.0, 1.0, seed=11)
    P = oracle.make_params(grid_n=n, spacing=dx, tol=1e-10, h_min=1e-5, h_max=0.5)
    m = 16
    g = np.random.default_rng(5)
    v = g.normal(size=(m, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    inj = _one(3e19, n=m, s_max=20.0)
    inj["ux"], inj["uy"], inj["uz"] = v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy()
    fwd = oracle.propagate(P, B, inj)
    back = _one(3e19, n=m, s_max=20.0, q=-1)
    back["x"], back["y"], back["z"] = (fwd["x"][:, i].copy() for i in range(3))
    back["ux"], back["uy"], back["uz"] = (-fwd["u"][:, i] for i in range(3))
    ret = oracle.propagate(P, B, back)
    d = np.linalg.norm(ret["x"], axis=1)
    assert np.all(d < 1e-5), d
    # and it really was deflected on the way out
    assert np.max(np.linalg.norm(fwd["u"] - v, axis=1)) > 0.05


# ---------------------------------------------------------------------------
# Trilinear interpolation on the periodic vertex-centred grid: exact for
# fields that are linear inside a cell, periodic with the tile.
# ---------------------------------------------------------------------------
def test_trilinear_exact_on_linear_and_periodic(oracle):
    n, dx, org = (5, 6, 7), 0.5, (-1.0, 2.0, 0.25)
    ii, jj, kk = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    # field [nz, ny, nx, 3]: component c = c-th affine function of the node position
    X = org[0] + ii * dx
    Y = org[1] + jj * dx
    Zc = org[2] + kk * dx
    comps = [1.0 + 2.0 * X - Y + 0.5 * Zc, -3.0 + 0.25 * X + Y, 4.0 * Zc - X]
    field = np.stack([c.transpose(2, 1, 0) for c in comps], axis=-1)
    P = oracle.make_params(grid_n=n, spacing=dx, origin=org)
    g = np.random.default_rng(0)
    # points strictly inside the last-but-one cell range (no wrap needed)
    lo = np.array(org)
    hi = lo + (np.array(n) - 1) * dx
    pts = lo + g.random((200, 3)) * (hi - lo)
    got = oracle.field_at(P, field, pts)
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    want = np.stack([1.0 + 2.0 * x - y + 0.5 * z, -3.0 + 0.25 * x + y, 4.0 * z - x], axis=1)
    assert np.allclose(got, want, rtol=0, atol=1e-12)
    # periodicity: shifting by a whole tile gives identical bits
    shift = np.array(n) * dx * np.array([2, -1, 3])
    assert np.array_equal(oracle.field_at(P, field, pts + 0 * shift), got)
    got2 = oracle.field_at(P, field, pts + shift)
    assert np.allclose(got2, got, atol=1e-12)
    # nodes give node values exactly
    node = np.array([[org[0] + 2 * dx, org[1] + 3 * dx, org[2] + 4 * dx]])
    assert np.array_equal(oracle.field_at(P, field, node)[0], field[4, 3, 2])


# ---------------------------------------------------------------------------
# Turbulence: divergence free, band limited, k^(-11/3), zero mean, exact rms.
# ---------------------------------------------------------------------------
def test_turbulence_spectrum(oracle):
    N, dx, lmin, lmax, brms = 64, 0.25, 0.5, 8.0, 1.0
    B = oracle.turbulent_field((N, N, N), dx, lmin, lmax, brms, seed=3)
    assert B.shape == (N, N, N, 3)
    assert np.max(np.abs(B.mean(axis=(0, 1, 2)))) < 1e-14
    assert abs(math.sqrt(np.mean(np.sum(B * B, axis=-1))) - brms) < 1e-13
    Bk = np.stack([np.fft.fftn(B[..., c]) for c in range(3)], axis=-1)
    f = np.fft.fftfreq(N) * N
    mz, my, mx = np.meshgrid(f, f, f, indexing="ij")
    kv = 2 * np.pi / (N * dx) * np.stack([mx, my, mz], axis=-1)
    kk = np.linalg.norm(kv, axis=-1)
    power = np.sum(np.abs(Bk) ** 2, axis=-1)
    band = (kk >= 2 * np.pi / lmax) & (kk <= 2 * np.pi / lmin)
    assert power[~band].sum() < 1e-24 * power.sum()
    live = band & (power > 1e-12 * power.max())
    div = np.abs(np.sum(kv * Bk, axis=-1))[live] / (kk[live] * np.sqrt(power[live]))
    assert div.max() < 1e-12
    # shell-averaged power per mode ~ k^(-11/3)
    edges = np.geomspace(2 * np.pi / lmax, 2 * np.pi / lmin, 9)
    kc, pc = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        m = band & (kk >= a) & (kk < b)
        if m.sum() > 20:
            kc.append(np.exp(np.mean(np.log(kk[m]))))
            pc.append(power[m].mean())
    slope = np.polyfit(np.log(kc), np.log(pc), 1)[0]
    assert abs(slope - (-11.0 / 3.0)) < 0.15, slope


def test_turbulence_correlation_length(oracle):
    """Correlation length of the generated field against the closed form of
    Harari, Mollerach & Roulet (JHEP 03 (2002) 045) for a Kolmogorov band
    [lmin, lmax]: L_c = (lmax/2) (a-1)/a (1 - r^a) / (1 - r^(a-1)), a = 5/3,
    r = lmin/lmax.  For an isotropic field L_c = pi sum |B(k)|^2/|k| /
    sum |B(k)|^2 over the modes, so this ties the generator's wavenumber
    convention (k = 2 pi / wavelength) to an external formula.  A 64^3 box
    holds few modes near 2 pi / lmax, so the agreement is approximate."""
    a = 5.0 / 3.0
    for (N, dx, lmin, lmax, seed) in ((64, 0.25, 0.5, 8.0, 3), (64, 0.25, 0.5, 4.0, 4)):
        B = oracle.turbulent_field((N, N, N), dx, lmin, lmax, 1.0, seed=seed)
        Bk = np.stack([np.fft.fftn(B[..., c]) for c in range(3)], axis=-1)
        f = np.fft.fftfreq(N) * N
        mz, my, mx = np.meshgrid(f, f, f, indexing="ij")
        kk = 2 * np.pi / (N * dx) * np.sqrt(mx * mx + my * my + mz * mz)
        P = np.sum(np.abs(Bk) ** 2, axis=-1)
        live = kk > 0
        lc = np.pi * np.sum(P[live] / kk[live]) / np.sum(P[live])
        r = lmin / lmax
        want = lmax / 2 * (a - 1) / a * (1 - r ** a) / (1 - r ** (a - 1))
        assert abs(lc / want - 1.0) < 0.12, (lc, want)


def test_turbulence_seed_dependence(oracle):
    a = oracle.turbulent_field((16, 16, 16), 0.25, 0.5, 4.0, 1.0, seed=1)
    b = oracle.turbulent_field((16, 16, 16), 0.25, 0.5, 4.0, 1.0, seed=1)
    c = oracle.turbulent_field((16, 16, 16), 0.25, 0.5, 4.0, 1.0, seed=2)
    assert np.array_equal(a, b)
    assert np.abs(a - c).max() > 0.1


# ---------------------------------------------------------------------------
# Photon field and interaction rates.
# ---------------------------------------------------------------------------
def test_blackbody_number_density(oracle):
    from scipy.integrate import quad
    T = 2.725
    kT = oracle.KB_EV * T
    n, _ = quad(lambda x: oracle.planck_density(x * kT, T) * kT, 1e-8, 200, limit=400)
    # n = 2 zeta(3) / pi^2 (kT / hbar c)^3 ; 410.5 per cm^3 at 2.725 K
    zeta3 = 1.2020569031595942
    closed = 2 * zeta3 / math.pi ** 2 * (kT / oracle.HBARC_EVM) ** 3
    assert abs(n / closed - 1) < 1e-9
    assert abs(n * 1e-6 - 410.5) < 0.5


def test_phi_pair_branches(oracle):
    # low-kappa limit (Blumenthal 1970): phi -> (pi/12) (kappa - 2)^4
    for k in (2.001, 2.01):
        assert abs(oracle.phi_pair(k) / (math.pi / 12 * (k - 2) ** 4) - 1) < 1e-2 * (k - 2) * 100
    # the two fitted branches of Chodorowski et al. (1992) meet at kappa = 25
    lo, hi = oracle.phi_pair(25 - 1e-9), oracle.phi_pair(25.0)
    assert abs(lo / hi - 1) < 2e-3
    assert oracle.phi_pair(2.0) == 0.0
    # monotone increasing above threshold
    ks = np.geomspace(2.01, 1e6, 400)
    v = np.array([oracle.phi_pair(k) for k in ks])
    assert np.all(np.diff(v) > 0)


def test_pair_loss_length_literature_shape(oracle):
    """Proton pair-production loss length on the CMB: minimum of roughly
    1-1.5 Gpc near 10^19.5 eV (Blumenthal 1970, Chodorowski et al. 1992),
    rising steeply towards 10^18 eV."""
    lE = np.linspace(18.0, 21.0, 31)
    L = np.array([1 / oracle.beta_pair_proton(10 ** e / oracle.MP_C2_EV) / oracle.MPC_M
                  for e in lE])
    i = int(np.argmin(L))
    assert 19.2 <= lE[i] <= 19.8
    assert 900 < L[i] < 1500
    assert L[0] > 10 * L[i]


def test_pair_loss_quadrature_converged(oracle):
    from scipy.integrate import quad
    g = 10 ** 19.5 / oracle.MP_C2_EV
    T = 2.725
    kT = oracle.KB_EV * T
    me = 0.51099895e6
    f = lambda k: oracle.planck_density(k * me / (2 * g), T) * oracle.phi_pair(k) / k ** 2
    kmax = 1400 * g * kT / me
    I = quad(f, 2, 25, limit=500, epsrel=1e-12)[0] + quad(f, 25, kmax, limit=500, epsrel=1e-12)[0]
    alpha, re = 7.2973525693e-3, 2.8179403262e-15
    beta = alpha * re ** 2 * me ** 2 * I / (g * oracle.MP_C2_EV)
    assert abs(beta / oracle.beta_pair_proton(g) - 1) < 1e-8


def _rate_definition(oracle, gamma, inner, eps_lo):
    """R = 1/(2 Gamma^2) int d eps n(eps)/eps^2 inner(2 Gamma eps), by quadrature."""
    from scipy.integrate import quad
    T = 2.725
    kT = oracle.KB_EV * T
    f = lambda eps: oracle.planck_density(eps, T) / eps ** 2 * inner(2 * gamma * eps)
    hi = 700 * kT
    pts = np.geomspace(max(eps_lo, 1e-12 * kT), hi, 60)
    I = sum(quad(f, a, b, epsrel=1e-11, limit=200)[0] for a, b in zip(pts[:-1], pts[1:]))
    return I / (2 * gamma ** 2)


def test_pion_rate_closed_form_vs_definition(oracle):
    s0, eth = 0.5e-31, 145e6
    inner = lambda emax: 0.0 if emax <= eth else s0 * (emax ** 2 - eth ** 2) / 2
    for lE in (19.6, 20.0, 20.5, 21.0):
        g = 10 ** lE / oracle.MP_C2_EV
        want = _rate_definition(oracle, g, inner, eth / (2 * g))
        assert abs(oracle.rate_pion_nucleon(g) / want - 1) < 1e-7, lE
    # high-Gamma limit: every photon is above threshold, R -> sigma0 n_gamma
    kT = oracle.KB_EV * 2.725
    n_gamma = 2 * 1.2020569031595942 / math.pi ** 2 * (kT / oracle.HBARC_EVM) ** 3
    assert abs(oracle.rate_pion_nucleon(1e16) / (s0 * n_gamma) - 1) < 1e-4
    assert oracle.rate_pion_nucleon(1e8) < 1e-60


def test_gdr_rate_vs_definition(oracle):
    from scipy.integrate import quad
    s_pk, ec, w, lo, hi = 1.5e-31, 20e6, 3e6, 8e6, 150e6
    sig = lambda e: s_pk * w * w / ((e - ec) ** 2 + w * w) if lo <= e <= hi else 0.0

    def inner(emax):
        if emax <= lo:
            return 0.0
        return quad(lambda e: e * sig(e), lo, min(emax, hi), points=[ec], epsrel=1e-12)[0]

    for lE in (19.5, 20.0, 20.5):
        g = 10 ** lE / (56 * oracle.MP_C2_EV)
        want = _rate_definition(oracle, g, inner, lo / (2 * g))
        assert abs(oracle.rate_gdr_nucleon(g) / want - 1) < 1e-6, lE


# ---------------------------------------------------------------------------
# Module cycle: sampling, resets, observer, losses.
# ---------------------------------------------------------------------------
def _tables(oracle):
    return oracle.tables_build(n=200, g_lo=1e6, g_hi=1e13)


def test_pion_free_paths_are_exponential(oracle):
    """P(no event within s) = exp(-R s): neutrons at constant high Gamma."""
    T = _tables(oracle)
    g = 1e12
    R = np.interp(np.log(g), np.linspace(np.log(1e6), np.log(1e13), 200), T.rate_pion)
    n = 4000
    inj = _one(g * oracle.MP_C2_EV, A=1, Z=0, n=n, s_max=1.0 / R)
    P = oracle.make_params(grid_n=(4, 4, 4), spacing=1.0, tables=T, flags=oracle.PION,
                           seed=77, h_max=1.0)
    r = oracle.propagate(P, _uniform_field(), inj, tables=T)
    none = np.mean(r["n_pion"] == 0)
    sd = math.sqrt(math.exp(-1) * (1 - math.exp(-1)) / n)
    assert abs(none - math.exp(-1)) < 4 * sd
    # one uniform per reset, reset at start and after each event
    assert np.all(r["draws"] == 1 + r["n_pion"])
    # the survival function at other lengths: the same ids draw the same first
    # free path, so these are points of one empirical distribution
    for x in (0.1, 0.5, 2.0, 3.0):
        inj_x = _one(g * oracle.MP_C2_EV, A=1, Z=0, n=n, s_max=x / R)
        rx = oracle.propagate(P, _uniform_field(), inj_x, tables=T)
        px = math.exp(-x)
        assert abs(np.mean(rx["n_pion"] == 0) - px) < 4 * math.sqrt(px * (1 - px) / n), x


def test_photodisintegration_branching_and_lineage(oracle):
    T = _tables(oracle)
    n = 3000
    E = 10 ** 20.6  # nitrogen: Gamma ~ 3e10, short GDR free path
    inj = _one(E, A=14, Z=7, n=n, s_max=0.05)
    P = oracle.make_params(grid_n=(4, 4, 4), spacing=1.0, tables=T, flags=oracle.PHOTODIS,
                           seed=5, h_max=0.1, h_min=1e-4)
    r = oracle.propagate(P, np.zeros((4, 4, 4, 3)), inj, tables=T)
    prim = r[r["generation"] == 0]
    sec = r[r["generation"] == 1]
    assert len(prim) == n and len(sec) == prim["n_pd"].sum()
    # nucleon number and charge are conserved per lineage
    by_parent = {}
    for s in sec:
        by_parent.setdefault(int(s["parent_id"]), []).append(s)
    for p in prim:
        kids = by_parent.get(int(p["id"]), [])
        assert p["A"] + len(kids) == 14
        assert p["Z"] + sum(int(k["Z"]) for k in kids) == 7
        # energy per nucleon is conserved by the emission
        for k in kids:
            assert k["A"] == 1
    # first emission from N-14: proton with probability Z/A = 1/2
    firsts = []
    for pid, kids in by_parent.items():
        k0 = [k for k in kids if int(k["id"]) == oracle.child_id(pid, 0)]
        firsts.append(int(k0[0]["Z"]))
    frac = np.mean(firsts)
    assert abs(frac - 0.5) < 4 * math.sqrt(0.25 / len(firsts))
    # draws: one per interaction per reset, plus one branching draw per event
    assert np.all(prim["draws"] == 1 + 2 * prim["n_pd"])
    # ids: lineage-derived and unique
    assert len(np.unique(r["id"])) == len(r)


def test_neutron_decay_survival_and_products(oracle):
    """Free-neutron beta decay.  The decay length is gamma c tau: the textbook
    figure is 9.2 kpc per EeV for tau = 886 s, i.e. 9.12 kpc for the
    878.4 s lifetime used here, so at that path length a fraction 1 - 1/e of
    the neutrons has decayed.  A decay product is a proton of the neutron's
    Lorentz factor; protons and nuclei never decay; each reset of the
    interaction states draws one uniform per active module."""
    n = 6000
    E = 1e18
    L = 9.2 * (878.4 / 886.0) * 1e-3  # Mpc
    inj = _one(E, A=1, Z=0, n=n, s_max=L)
    P = oracle.make_params(grid_n=(4, 4, 4), spacing=1.0, flags=oracle.DECAY, seed=12,
                           h_max=0.1 * L, h_min=1e-6)
    r = oracle.propagate(P, np.zeros((4, 4, 4, 3)), inj)
    decayed = r["Z"] == 1
    frac = decayed.mean()
    p = 1 - math.exp(-1)
    assert abs(frac - p) < 4 * math.sqrt(p * (1 - p) / n) + 0.003, frac
    m_n, m_p = 939.56542052e6, 938.27208816e6  # CODATA 2018 [eV]
    gam_before = r["E0"][decayed] / m_n
    gam_after = r["E"][decayed] / m_p
    assert np.max(np.abs(gam_after / gam_before - 1)) < 1e-15
    assert np.all(r["E"][~decayed] == E) and np.all(r["A"] == 1)
    assert np.all(r["draws"] == 1 + decayed)
    assert np.all(r["s"] == L)
    # protons and iron never decay; one uniform drawn at the start
    inj2 = _one(1e19, A=1, Z=1, n=50, s_max=1.0)
    inj3 = _one(1e20, A=56, Z=26, n=50, s_max=1.0)
    for inj_x in (inj2, inj3):
        r2 = oracle.propagate(P, np.zeros((4, 4, 4, 3)), inj_x)
        assert np.all(r2["Z"] == inj_x["Z"]) and np.all(r2["E"] == inj_x["E"])
        assert np.all(r2["draws"] == 1)


def test_observer_sphere_straight_lines(oracle):
    """Neutral particles fly straight: detection iff the line passes within R."""
    g = np.random.default_rng(9)
    m = 400
    start = np.array([5.0, 0.0, 0.0])
    tgt = g.uniform(-2, 2, size=(m, 3))
    tgt[:, 0] = 0.0
    v = tgt - start
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    inj = _one(1e20, A=1, Z=0, n=m, s_max=20.0, x=start)
    inj["ux"], inj["uy"], inj["uz"] = v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy()
    P = oracle.make_params(grid_n=(4, 4, 4), spacing=1.0, flags=oracle.OBSERVER, obs_r=1.0,
                           h_max=0.7)
    r = oracle.propagate(P, _uniform_field(), inj)
    # impact parameter of the line start + t v with respect to the origin
    b = np.linalg.norm(np.cross(start, v), axis=1)
    det = r["status"] == oracle.DETECTED
    assert np.array_equal(det, b < 1.0)
    # started inside never detects
    inj2 = _one(1e20, A=1, Z=0, n=1, s_max=5.0, x=(0.2, 0.0, 0.0))
    assert oracle.propagate(P, _uniform_field(), inj2)[0]["status"] == oracle.MAX_LENGTH


def test_losses_only_adiabatic_closed_form(oracle):
    """With only the adiabatic loss, E after n fixed steps is E0 (1 - b h)^n."""
    h, b = 0.5, 1.0 / 4454.0
    P = oracle.make_params(grid_n=(4, 4, 4), spacing=1.0, flags=oracle.ADIABATIC, beta_ad=b,
                           h_min=h, h_max=h, tol=1e30)
    r = oracle.propagate(P, _uniform_field(bz=0.0), _one(1e19, Z=0, s_max=100 * h))[0]
    assert r["n_acc"] == 100
    assert abs(r["E"] / (1e19 * (1 - b * h) ** 100) - 1) < 1e-13


def test_emin_break_and_status(oracle):
    P = oracle.make_params(grid_n=(4, 4, 4), spacing=1.0, flags=oracle.ADIABATIC | oracle.EMIN,
                           beta_ad=0.01, e_min=0.9e19, h_min=1.0, h_max=1.0, tol=1e30)
    r = oracle.propagate(P, _uniform_field(bz=0.0), _one(1e19, Z=0, s_max=1e3))[0]
    # (1 - 0.01)^k < 0.9 first at k = 11
    assert r["status"] == oracle.BELOW_EMIN and r["n_acc"] == 11


def test_step_budget_status(oracle):
    P = oracle.make_params(grid_n=(4, 4, 4), spacing=1.0, h_min=0.1, h_max=0.1, max_steps=7)
    r = oracle.propagate(P, _uniform_field(), _one(1e19, s_max=1e3))[0]
    assert r["status"] == oracle.BUDGET and r["n_acc"] == 7


def test_series_log_against_library(oracle):
    """The atanh-series logarithm steering free paths and table lookups is
    within a few ulp of the library log over the ranges it is used on
    (uniforms in (0, 1), Lorentz factors 1e5..1e14)."""
    g = np.random.default_rng(3)
    xs = np.concatenate([g.random(20000), 10 ** g.uniform(5, 14, 20000),
                         [2.0 ** -53, 1 - 2.0 ** -53, 0.5, 1.0, 2.0, math.sqrt(2.0), 1e13]])
    for x in xs:
        got, want = oracle.series_log(float(x)), math.log(float(x))
        assert abs(got - want) <= 4 * np.spacing(abs(want)) + 1e-300, (x, got, want)
    assert oracle.series_log(1.0) == 0.0


def test_series_exp_against_library(oracle):
    g = np.random.default_rng(4)
    xs = np.concatenate([g.uniform(-700, 0, 20000), g.uniform(-5, 5, 20000), [0.0, -1e-300, 1.0]])
    for x in xs:
        got, want = oracle.series_exp(float(x)), math.exp(float(x))
        assert abs(got - want) <= 4 * np.spacing(want), (x, got, want)
    assert oracle.series_exp(0.0) == 1.0
    assert oracle.series_exp(-800.0) == 0.0


# ---------------------------------------------------------------------------
# HEALPix RING (Gorski et al., ApJ 622, 759, 2005)
# ---------------------------------------------------------------------------
def test_healpix_round_trip_and_ring_structure(oracle):
    for nside in (1, 2, 4, 16, 64):
        npix = 12 * nside * nside
        zs = np.empty(npix)
        for p in range(npix):
            z, phi = oracle.pix2ang(nside, p)
            assert oracle.ang2pix(nside, z, phi) == p
            zs[p] = z
        # rings of constant z: 4 nside - 1 rings; pixel z decreasing with index
        rings = np.unique(np.round(zs, 12))
        assert len(rings) == 4 * nside - 1
        assert np.all(np.diff(zs) <= 1e-12)
    # nside = 1: 4 pixels per ring at z = 2/3, 0, -2/3
    z = [oracle.pix2ang(1, p)[0] for p in range(12)]
    assert np.allclose(z, [2 / 3] * 4 + [0.0] * 4 + [-2 / 3] * 4)


def test_healpix_equal_area(oracle):
    """Uniform directions fill the 12 nside^2 pixels equally (equal-area
    property): chi-square of the counts is consistent with uniform."""
    from scipy.stats import chisquare
    nside = 16
    g = np.random.default_rng(8)
    v = g.normal(size=(600000, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    pix = oracle.ang2pix_vec(nside, v)
    counts = np.bincount(pix, minlength=12 * nside * nside)
    assert chisquare(counts).pvalue > 1e-3
    # a direction maps to the pixel whose centre is nearest (within a pixel size)
    sub = v[:5000]
    for u, p in zip(sub, pix[:5000]):
        z, phi = oracle.pix2ang(nside, int(p))
        c = np.array([np.sqrt(1 - z * z) * np.cos(phi), np.sqrt(1 - z * z) * np.sin(phi), z])
        assert np.degrees(np.arccos(np.clip(c @ u, -1, 1))) < 2.0 * 58.6 / nside


def test_lens_zero_field_is_identity(oracle):
    """In a zero field back-tracked antiparticles fly straight: every sample
    leaves through its own arrival pixel, so the lens is the identity on
    pixels and a candidate is always observed in its own pixel or shadowed."""
    import oracle.lens as L
    import workloads as W
    nside, nb = 4, 2
    dirs, E, bins = W.lens_samples(nb, 192 * 3, 1e18, 1e20, 1)
    P = oracle.make_params(grid_n=(4, 4, 4), spacing=10.0, origin=(-20, -20, -20), tol=1e-4,
                           h_min=0.001, h_max=0.05, field_unit_T=oracle.MICROGAUSS_T,
                           length_unit_m=oracle.KPC_M, flags=oracle.BORDER, border_r=20.0)
    n = len(E)
    r = oracle.propagate(P, np.zeros((4, 4, 4, 3)), dict(
        id=np.arange(n, dtype=np.uint64), x=np.full(n, -8.5), y=np.zeros(n), z=np.zeros(n),
        ux=dirs[:, 0].copy(), uy=dirs[:, 1].copy(), uz=dirs[:, 2].copy(), E=E,
        A=np.ones(n, np.int32), Z=np.ones(n, np.int32), q=-np.ones(n, np.int32)))
    assert np.all(r["status"] == oracle.AT_BORDER)
    lens = L.build(nside, nb, bins, dirs, r)
    npix = 12 * nside * nside
    for c in range(nb * npix):
        col = lens["entries"][lens["col_start"][c]:lens["col_start"][c + 1]]
        assert np.all(col == c % npix)
    g = np.random.default_rng(0)
    u = g.normal(size=(2000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    Ev = 10 ** g.uniform(18, 20, 2000)
    out = L.apply(lens, nside, 1e18, 1e20, nb, 9, np.arange(2000, dtype=np.uint64), u, Ev,
                  np.ones(2000, np.int32))
    seen = out < npix
    assert seen.mean() > 0.3
    assert np.array_equal(out[seen], oracle.ang2pix_vec(nside, -u)[seen])


# ---------------------------------------------------------------------------
# MLP surrogate oracle
# ---------------------------------------------------------------------------
def _tiny_mlp():
    import oracle.mlp as M
    shapes = M.layer_shapes(4, 8, 2, 3)
    g = np.random.default_rng(12)
    flat = g.normal(scale=0.5, size=M.n_params(shapes))
    x = g.normal(size=(7, 4))
    t = g.normal(size=(7, 3))
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    return M, shapes, flat, x, t


def test_mlp_backward_matches_finite_differences(oracle):
    M, shapes, flat, x, t = _tiny_mlp()
    y, cache = M.forward(flat, shapes, x)
    grad = M.backward(flat, shapes, cache, t)
    eps = 1e-6
    num = np.zeros_like(flat)
    for k in range(len(flat)):
        fp, fm = flat.copy(), flat.copy()
        fp[k] += eps
        fm[k] -= eps
        num[k] = (M.loss(M.forward(fp, shapes, x)[0], t) -
                  M.loss(M.forward(fm, shapes, x)[0], t)) / (2 * eps)
    assert np.max(np.abs(grad - num)) < 1e-6 * max(1.0, np.max(np.abs(num)))


def test_mlp_forward_explicit_loops(oracle):
    M, shapes, flat, x, t = _tiny_mlp()
    y, _ = M.forward(flat, shapes, x)
    Ws, bs = M.unpack(flat, shapes)
    for r in range(len(x)):
        h = list(x[r])
        for l, (W, b) in enumerate(zip(Ws, bs)):
            out = []
            for o in range(W.shape[0]):
                acc = b[o]
                for i in range(W.shape[1]):
                    acc += W[o, i] * h[i]
                out.append(max(acc, 0.0) if l < len(Ws) - 1 else acc)
            h = out
        nrm = math.sqrt(sum(v * v for v in h))
        assert np.allclose(y[r], np.array(h) / nrm, rtol=0, atol=1e-13)


def test_adam_first_step_and_bf16_rounding(oracle):
    import oracle.mlp as M
    g = np.array([0.5, -2.0, 1e-3])
    p, m, v = M.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # bias-corrected first step is -lr * g / (|g| + eps)
    assert np.allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    vals = M.bf16_round([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -3.0e-3, 65504.0])
    assert vals[0] == 1.0 and vals[1] == 1.0 and vals[2] == 1 + 2 ** -6
    assert abs(vals[3] / -3.0e-3 - 1) < 2 ** -8


def test_pair_loss_blackbody_temperature_scaling(oracle):
    """For a Planck photon gas the Blumenthal loss depends on Gamma and T only
    through Gamma T and an overall T^3 (substitute eps = kappa m_e c^2 / 2 Gamma
    in the integral): beta(Gamma, T) = (T / T0)^3 beta(Gamma T / T0, T0)."""
    T0 = 2.725
    for T in (35.0, 4500.0):
        for g in (3e5, 2e7, 1e9):
            lhs = oracle.lib().orc_beta_pair_proton(g, T)
            rhs = (T / T0) ** 3 * oracle.lib().orc_beta_pair_proton(g * T / T0, T0)
            assert lhs > 0 and abs(lhs / rhs - 1) < 1e-8, (T, g, lhs, rhs)


def test_pair_table_with_synthetic_infrared_background(oracle):
    """The pair table with a background of dilute blackbodies equals the CMB
    table plus sum_k D_k (T_k / T0)^3 beta_CMB(Gamma T_k / T0) (linearity in the
    photon density plus the temperature scaling); the background matters only
    below the CMB threshold region."""
    irb = ((35.0, 8.5e-7), (4500.0, 3.1e-15))
    n, g_lo, g_hi = 60, 1e6, 1e13
    Tc = oracle.tables_build(n=n, g_lo=g_lo, g_hi=g_hi)
    Ti = oracle.tables_build(n=n, g_lo=g_lo, g_hi=g_hi, irb=irb)
    gam = np.exp(np.linspace(np.log(g_lo), np.log(g_hi), n))
    extra = np.zeros(n)
    for T, D in irb:
        extra += D * (T / 2.725) ** 3 * np.array(
            [oracle.lib().orc_beta_pair_proton(g * T / 2.725, 2.725) for g in gam])
    extra *= oracle.MPC_M
    assert np.allclose(Ti.beta_pair, Tc.beta_pair + extra, rtol=1e-8, atol=0)
    # the infrared light adds losses below the CMB pair threshold and is
    # negligible at the top of the range
    assert Ti.beta_pair[5] > 1.5 * Tc.beta_pair[5]
    assert Ti.beta_pair[-1] < 1.01 * Tc.beta_pair[-1]
    assert np.array_equal(Ti.rate_pion, Tc.rate_pion)


# ---------------------------------------------------------------------------
# 1D mode with cosmology (flat Lambda-CDM, H0 = 67.3, Om = 0.315)
# ---------------------------------------------------------------------------
def _cosmo(oracle):
    import oracle.cosmology as cm
    return cm


def test_1d_adiabatic_only_is_pure_redshift(oracle):
    """Adiabatic expansion alone: the observed energy is E_src / (1 + z_src)
    (photon-like redshift of an ultrarelativistic particle), and arrival is
    at z = 0 after the comoving distance to z_src."""
    cm = _cosmo(oracle)
    from scipy.integrate import quad
    P = cm.make_params1d(flags=oracle.ADIABATIC, dz_max=1e-3)
    zs = np.array([0.01, 0.3, 1.0, 2.5])
    inj = dict(id=np.arange(4, dtype=np.uint64), z=zs, E=np.full(4, 1e20),
               A=np.ones(4, np.int32), Z=np.ones(4, np.int32))
    r = cm.propagate_1d(P, inj)
    assert np.all(r["status"] == oracle.DETECTED) and np.all(r["x"][:, 0] == 0.0)
    assert np.max(np.abs(r["E"] * (1 + zs) / 1e20 - 1)) < 1e-14
    # comoving distance against a library quadrature of c / H(z)
    H0 = cm.H0_KM_S_MPC / cm.C_KM_S
    Dc = np.array([quad(lambda x: 1 / (H0 * np.sqrt(0.315 * (1 + x) ** 3 + 0.685)), 0, z,
                        epsabs=0, epsrel=1e-12)[0] for z in zs])
    assert np.max(np.abs(r["s"] / Dc - 1)) < 1e-6


def test_1d_comoving_distance(oracle):
    """Comoving distance c int dz / H against a library quadrature, and its
    inverse; 4000 Mpc comoving is z ~ 1.35 for these parameters."""
    cm = _cosmo(oracle)
    from scipy.integrate import quad
    P = cm.make_params1d()
    H0 = cm.H0_KM_S_MPC / cm.C_KM_S
    zs = np.array([1e-3, 0.1, 0.5, 1.4, 3.0])
    ref = np.array([quad(lambda x: 1 / (H0 * np.sqrt(0.315 * (1 + x) ** 3 + 0.685)),
                         0, z, epsabs=0, epsrel=1e-13)[0] for z in zs])
    got = cm.comoving_distance(P, zs)
    assert np.max(np.abs(got / ref - 1)) < 1e-11
    back = cm.redshift_of_distance(P, got)
    assert np.max(np.abs(back / zs - 1)) < 1e-12
    z4000 = cm.redshift_of_distance(P, [4000.0])[0]
    assert 1.2 < z4000 < 1.5


def test_1d_pair_loss_rate_is_hotter_cmb(oracle):
    """At redshift z the CMB is a blackbody at T0 (1 + z): over a tiny step
    the 1D relative pair loss per proper length equals the blackbody loss rate
    at that temperature (direct quadrature), to the table's interpolation."""
    cm = _cosmo(oracle)
    T = oracle.tables_build(n=2000, g_lo=1e8, g_hi=1e13)
    for z in (0.5, 2.0):
        P = cm.make_params1d(tables=T, flags=oracle.PAIR, dz_max=1e-7, loss_max=1.0,
                             max_steps=1)
        E = 3e19
        inj = dict(id=np.zeros(1, np.uint64), z=np.array([z]), E=np.array([E]),
                   A=np.ones(1, np.int32), Z=np.ones(1, np.int32))
        r = cm.propagate_1d(P, inj, tables=T)
        dz = z - r["x"][0, 0]
        h_com = r["s"][0]
        proper = h_com / (1 + z)
        loss = (1 - r["E"][0] / E) / proper                       # per proper Mpc
        g = E / oracle.MP_C2_EV
        direct = oracle.lib().orc_beta_pair_proton(g, 2.725 * (1 + z)) * oracle.MPC_M
        assert dz > 0 and abs(loss / direct - 1) < 2e-4, (z, loss, direct)


def test_1d_pion_optical_depth(oracle):
    """Protons injected at z_src reach the observer without a pion event with
    probability exp(-tau), tau = int (1+z)^2 R((1+z) Gamma(z)) dD_c (energy
    redshifting only), here from a library quadrature of the same tables."""
    cm = _cosmo(oracle)
    from scipy.integrate import quad
    T = oracle.tables_build(n=400, g_lo=1e9, g_hi=1e13)
    n = 6000
    z_src, E_src = 0.002, 1e20
    P = cm.make_params1d(tables=T, flags=oracle.PION | oracle.ADIABATIC, seed=3, dz_max=1e-5)
    inj = dict(id=np.arange(n, dtype=np.uint64), z=np.full(n, z_src), E=np.full(n, E_src),
               A=np.ones(n, np.int32), Z=np.ones(n, np.int32))
    r = cm.propagate_1d(P, inj, tables=T)
    none = np.mean(r["n_pion"] == 0)
    H0 = cm.H0_KM_S_MPC / cm.C_KM_S
    lng = np.linspace(np.log(1e9), np.log(1e13), 400)

    def integrand(z):
        E = E_src * (1 + z) / (1 + z_src)
        g = (1 + z) * E / oracle.MP_C2_EV
        R = np.interp(np.log(g), lng, T.rate_pion)
        return (1 + z) ** 2 * R / (H0 * np.sqrt(0.315 * (1 + z) ** 3 + 0.685))

    tau = quad(integrand, 0, z_src, epsrel=1e-10)[0]
    p = np.exp(-tau)
    assert 0.2 < p < 0.9
    assert abs(none - p) < 4 * np.sqrt(p * (1 - p) / n) + 2e-3, (none, p)


def test_bf16_rounding_against_torch(oracle):
    """The oracle's bfloat16 rounding against PyTorch's binary32 -> bfloat16
    conversion (round to nearest, ties to even) on values spanning the range,
    the rounding ties, and subnormals."""
    import torch
    import oracle.mlp as M
    g = np.random.default_rng(5)
    x = np.concatenate([g.normal(size=20000) * 10.0 ** g.uniform(-30, 30, 20000),
                        1 + np.arange(-512, 512) * 2.0 ** -9,            # ties and neighbours
                        np.array([0.0, -0.0, 1e-40, -1e-40, 3.0e38])]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    got = M.bf16_round(x.astype(np.float64))
    assert np.array_equal(got, want)


def test_mlp_bf16_mode_explicit_loops(oracle):
    """bf16 mode on a tiny network, restated as explicit loops: the hidden
    weights, every hidden activation and every hidden backward signal are
    rounded, the first / output layers' weights, the biases, the output and
    dy are not."""
    M, shapes, flat0, x, t = _tiny_mlp()
    flat = M.bf16_weights(flat0, shapes)
    Ws, bs = M.unpack(flat, shapes)
    W0, b0 = M.unpack(flat0, shapes)
    L = len(Ws)
    for l in range(L):
        want = M.bf16_round(W0[l]) if 0 < l < L - 1 else W0[l]
        assert np.array_equal(Ws[l], want) and np.array_equal(bs[l], b0[l])
        assert not np.array_equal(W0[l], M.bf16_round(W0[l]))   # rounding is visible
    y, cache = M.forward(flat, shapes, x, bf16=True)
    grad = M.backward(flat, shapes, cache, t, bf16=True)
    gW, gb = M.unpack(grad, shapes)
    n = len(x)
    acts_all, dzs_all = [], []
    for r in range(n):
        hs = [list(x[r])]
        for l, (W, b) in enumerate(zip(Ws, bs)):
            out = []
            for o in range(W.shape[0]):
                acc = b[o]
                for i in range(W.shape[1]):
                    acc += W[o, i] * hs[-1][i]
                if l < L - 1:
                    acc = float(M.bf16_round(max(acc, 0.0)))
                out.append(acc)
            hs.append(out)
        nrm = math.sqrt(sum(v * v for v in hs[-1]))
        yh = [v / nrm for v in hs[-1]]
        assert np.allclose(y[r], yh, rtol=0, atol=1e-13)
        d = sum(a * b for a, b in zip(yh, t[r]))
        dz = [-(t[r][k] - d * yh[k]) / nrm / n for k in range(3)]
        dzs = [None] * L
        dzs[L - 1] = dz
        for l in range(L - 1, 0, -1):
            W = Ws[l]
            prev = []
            for i in range(W.shape[1]):
                acc = sum(dzs[l][o] * W[o, i] for o in range(W.shape[0]))
                prev.append(float(M.bf16_round(acc if hs[l][i] > 0.0 else 0.0)))
            dzs[l - 1] = prev
        acts_all.append(hs)
        dzs_all.append(dzs)
    for l in range(L):
        for o in range(Ws[l].shape[0]):
            assert abs(gb[l][o] - sum(dzs_all[r][l][o] for r in range(n))) < 1e-13
            for i in range(Ws[l].shape[1]):
                want = sum(dzs_all[r][l][o] * acts_all[r][l][i] for r in range(n))
                assert abs(gW[l][o, i] - want) < 1e-13
