"""The lens kernel takes its integer decisions (HEALPix pixel, rigidity bin,
observed or not, pick within a column) in binary32 and repeats them in
binary64 only inside a guard band around each floor or comparison.  This test
models those binary32 steps with numpy float32 arithmetic (the inputs
truncated to 24 significant bits, 1 - |z| formed exactly, the same guards)
and checks, against the oracle's binary64 decisions, that (1) every decision
the guards call sure is the binary64 one and (2) the largest binary32 error
seen stays well inside the guard.  The GPU tests check the kernels
themselves pixel by pixel."""
import os
import re

import numpy as np
import pytest

f32 = np.float32
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_1307_2643_gb300", "csrc", "device_common.cuh")


def _phase_coefficients():
    """The binary32 coefficients of the kernel's phase polynomial, highest
    degree first, read from its source so that the test checks what is
    compiled."""
    src = open(HEADER).read()
    body = src[src.index("float phase_quarter_turns("):]
    body = body[:body.index("\n}\n")]
    first = re.search(r"float p = (-?[0-9.e+-]+)f;", body).group(1)
    rest = re.findall(r"p = fmaf\(p, s, (-?[0-9.e+-]+)f\);", body)
    return [f32(float(c)) for c in [first] + rest]


def _fma32(a, b, c):
    """binary32 fma: the product is exact in binary64, one rounding of the sum
    (a binary64 rounding first, harmless at the bounds tested)."""
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64)
            + np.asarray(c, np.float64)).astype(f32)


def _phase32(x, y):
    """The kernel's phase in quarter turns, t in [0, 4), in binary32 (the
    quotient correctly rounded here; __fdividef's 2 ulp are in the bound)."""
    C = _phase_coefficients()
    ax, ay = np.abs(x), np.abs(y)
    mn, mx = np.minimum(ax, ay), np.maximum(ax, ay)
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.where(mx > 0, (mn / np.where(mx > 0, mx, f32(1))).astype(f32), f32(0)).astype(f32)
    s = (r * r).astype(f32)
    p = np.full_like(s, C[0])
    for c in C[1:]:
        p = _fma32(p, s, c)
    g = (p * r).astype(f32)
    west, south = x < 0, y < 0
    base = np.where(west, f32(2), np.where(south, f32(4), f32(0))).astype(f32)
    sg = np.where(west == south, f32(1), f32(-1)).astype(f32)
    steep = ay > ax
    return _fma32(np.where(steep, -sg, sg), g, np.where(steep, (base + sg).astype(f32), base))


def _trunc32(x):
    """Significand truncated to 24 bits, as the kernel's bit-level conversion."""
    b = np.ascontiguousarray(x, dtype=np.float64).view(np.uint64) & np.uint64(0xFFFFFFFFE0000000)
    return b.view(np.float64).astype(f32)


def _one_minus_abs(z):
    b = np.abs(z).view(np.uint64)
    d = (np.uint64(1) << np.uint64(52)) - (b & np.uint64(0x000FFFFFFFFFFFFF))
    hi = (d >> np.uint64(32)).astype(np.uint32).astype(f32)
    lo = (d & np.uint64(0xFFFFFFFF)).astype(np.uint32).astype(f32)
    v = (hi * f32(4294967296.0) + lo).astype(f32) * f32(2.0 ** -53)
    return np.where(np.abs(z) >= 1.0, f32(0), v).astype(f32)


def _floor_sure(a, g):
    fl = np.floor(a).astype(f32)
    f = (a - fl).astype(f32)
    return fl.astype(np.int64), (f >= g) & (f <= f32(1) - g)


def _pixel_guarded(ns, u, guard_per_nside=4e-6):
    fx, fy, fz = _trunc32(u[:, 0]), _trunc32(u[:, 1]), _trunc32(u[:, 2])
    nsf = f32(ns)
    g = f32(guard_per_nside) * nsf
    tt = _phase32(fx, fy)
    itt, ok = _floor_sure(tt, f32(2e-5))
    za = np.abs(fz)
    ok &= np.abs((za - f32(2.0 / 3.0)).astype(f32)) > f32(1e-6)
    eq = za <= f32(2.0 / 3.0)
    vm = (nsf * _fma32(f32(-0.75), fz, f32(0.5))).astype(f32)
    vp = (nsf * _fma32(f32(0.75), fz, f32(0.5))).astype(f32)
    a1, a2 = _fma32(nsf, tt, vm), _fma32(nsf, tt, vp)
    jp, o1 = _floor_sure(a1, g)
    jm, o2 = _floor_sure(a2, g)
    ir = ns + 1 + jp - jm
    ip = np.trunc((jp + jm - ns + (1 - (ir & 1)) + 1) / 2).astype(np.int64)
    ip = ((ip % (4 * ns)) + 4 * ns) % (4 * ns)
    p_eq = 2 * ns * (ns - 1) + (ir - 1) * 4 * ns + ip
    tp = (tt - itt.astype(f32)).astype(f32)
    tmp = (nsf * np.sqrt((f32(3) * _one_minus_abs(u[:, 2])).astype(f32))).astype(f32)
    b1, b2 = (tp * tmp).astype(f32), ((f32(1) - tp).astype(f32) * tmp).astype(f32)
    jp2, o3 = _floor_sure(b1, g)
    jm2, o4 = _floor_sure(b2, g)
    ir2 = jp2 + jm2 + 1
    b3 = (tt * ir2.astype(f32)).astype(f32)
    ip2, o5 = _floor_sure(b3, g)
    irs = np.maximum(ir2, 1)
    ip2 = ((ip2 % (4 * irs)) + 4 * irs) % (4 * irs)
    p_cap = np.where(u[:, 2] > 0, 2 * ir2 * (ir2 - 1) + ip2,
                     12 * ns * ns - 2 * ir2 * (ir2 + 1) + ip2)
    pix = np.where(eq, p_eq, p_cap)
    ok &= np.where(eq, o1 & o2, o3 & o4 & o5)
    # binary32 floor arguments and their binary64 counterparts (for the error)
    phd = np.arctan2(u[:, 1], u[:, 0])
    phd = np.where(phd < 0, phd + 2 * np.pi, phd)
    ttd = phd / (np.pi / 2)
    a1d = ns * (0.5 + ttd) - ns * u[:, 2] * 0.75
    err = np.abs(a1.astype(np.float64) - a1d)
    err = np.minimum(err, np.abs(err - 4 * ns))     # the phase may wrap by 4
    return pix, ok, float(err[eq].max()) / ns


def _directions(oracle, n, seed):
    g = np.random.default_rng(seed)
    u = g.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    extra = []
    for ns in (1, 4):
        for p in range(12 * ns * ns):
            z, ph = oracle.pix2ang(ns, p)
            s = np.sqrt(1 - z * z)
            extra.append([s * np.cos(ph), s * np.sin(ph), z])
    for z in (2 / 3, -2 / 3, np.nextafter(2 / 3, 1), np.nextafter(2 / 3, 0), 1.0, -1.0, 0.0,
              1 - 1e-12, -1 + 1e-12):
        for ph in (0.0, 1e-12, -1e-12, np.pi / 2, np.pi, -np.pi, 1.5 * np.pi):
            s = np.sqrt(max(0.0, 1 - z * z))
            extra.append([s * np.cos(ph), s * np.sin(ph), z])
    return np.concatenate([u, np.array(extra)])


@pytest.mark.parametrize("nside", [1, 4, 64, 1024])
def test_guarded_pixels_agree_with_binary64(oracle, nside):
    u = _directions(oracle, 500_000, nside)
    want = oracle.ang2pix_vec(nside, u)
    pix, ok, err_over_ns = _pixel_guarded(nside, u)
    assert np.array_equal(pix[ok], want[ok])
    # the kernel's guard is nside * 4e-6, its error bound nside * 9.5e-7
    assert err_over_ns < 9.5e-7 and err_over_ns < 4e-6 / 3
    assert ok[:500_000].mean() > (0.99 if nside <= 64 else 0.9)


def test_unit_range_truncation_matches_the_general_one():
    """f32_trunc_unit's shortcut for |x| < 2 (the upper word shifted left by
    three with three bits of the lower word, rebiased by 384 << 23) gives the
    same binary32 as the general truncation, and +-0 below 2^-126."""
    g = np.random.default_rng(5)
    x = np.concatenate([g.uniform(-2, 2, 1_000_000), g.normal(size=1000) * 1e-30,
                        np.ldexp(1.0, np.arange(-130, 1)), -np.ldexp(1.0, np.arange(-130, 1)),
                        [0.0, -0.0, 1.0, -1.0, np.nextafter(2.0, 0), -np.nextafter(2.0, 0),
                         np.nextafter(1.0, 2), np.ldexp(1.0, -126), np.nextafter(np.ldexp(1.0, -126), 0)]])
    b = x.view(np.uint64)
    hi = (b >> np.uint64(32)).astype(np.uint32)
    lo = (b & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    sign = hi & np.uint32(0x80000000)
    ah = hi & np.uint32(0x7FFFFFFF)
    assert np.all(ah < np.uint32(0x40000000))
    funnel = ((hi.astype(np.uint64) << np.uint64(3)) | (lo.astype(np.uint64) >> np.uint64(29)))
    m = ((funnel & np.uint64(0xFFFFFFFF)) - np.uint64(384 << 23)) & np.uint64(0xFFFFFFFF)
    bits = np.where(ah < np.uint32(897 << 20), sign, sign | m.astype(np.uint32)).astype(np.uint32)
    got = bits.view(np.float32)
    want = np.where(np.abs(x) < np.ldexp(1.0, -126), np.copysign(0.0, x), x)
    want = _trunc32(want)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_phase_polynomial_within_its_bound():
    """(2/pi) atan(r) ~ r P(r^2) on [0, 1]: within 4.5e-8 with the binary32
    coefficients in exact (binary64) arithmetic; the whole binary32 phase
    within 3.9e-7 of the exact phase of its binary32 inputs, on directions of
    every octant, the axes and the diagonals."""
    C = [float(c) for c in _phase_coefficients()]
    assert len(C) == 8
    r = np.linspace(0.0, 1.0, 2_000_001)
    p = np.zeros_like(r)
    for c in C:
        p = p * r * r + c
    assert np.max(np.abs(r * p - (2 / np.pi) * np.arctan(r))) < 4.5e-8
    g = np.random.default_rng(11)
    ph = np.concatenate([g.uniform(-np.pi, np.pi, 2_000_000),
                         np.arange(-8, 9) * np.pi / 8,
                         np.arange(-8, 9) * np.pi / 8 + 1e-9])
    rad = np.concatenate([np.ones(2_000_000), g.uniform(1e-6, 1, 34)])
    x, y = (rad * np.cos(ph)).astype(f32), (rad * np.sin(ph)).astype(f32)
    t = _phase32(x, y).astype(np.float64)
    exact = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    exact = np.where(exact < 0, exact + 2 * np.pi, exact) / (np.pi / 2)
    err = np.abs(t - exact)
    err = np.minimum(err, np.abs(err - 4))  # 4 and 0 are the same phase
    assert err.max() < 3.9e-7
    assert np.all((t >= 0) & (t <= 4))


def test_guarded_bins_agree_with_binary64(oracle):
    g = np.random.default_rng(3)
    for r_lo, r_hi, nb in ((1e18, 1e20, 100), (1e17, 1e21, 1000), (1.0, 10.0, 7)):
        n = 400_000
        Z = g.choice([1, 2, 7, 26], n)
        R = np.exp(g.uniform(np.log(r_lo) - 1, np.log(r_hi) + 1, n))
        edges = np.exp(np.linspace(np.log(r_lo), np.log(r_hi), nb + 1))
        k = 4 * len(edges)
        R[:k] = np.repeat(edges, 4) * np.tile([1, 1 - 1e-15, 1 + 1e-15, 1 + 1e-7], len(edges))
        E = R * Z
        lg_lo = oracle.series_log(r_lo)
        inv = nb / (oracle.series_log(r_hi) - lg_lo)
        t = (oracle.series_log_vec(E / Z) - lg_lo) * inv
        want = np.clip(np.floor(t), 0, nb - 1).astype(np.int64)
        # the kernel: __fdividef and __log2f (modelled correctly rounded here;
        # their documented error is in the kernel's bound), times inv ln 2
        x = ((_trunc32(E) * f32(1.0 / r_lo)).astype(f32) / Z.astype(f32)).astype(f32)
        tf = (np.log2(x).astype(f32) * f32(inv * np.log(2.0))).astype(f32)
        gg = (f32(inv) * f32(1e-5) + np.abs(tf) * f32(1.5e-6) + f32(1e-6)).astype(f32)
        b, ok = _floor_sure(tf, gg)
        lo, hi = (tf + gg) < 0, (tf - gg) >= f32(nb - 1)
        b = np.where(lo, 0, np.where(hi, nb - 1, b))
        ok = lo | hi | ok
        assert np.array_equal(b[ok], want[ok])
        inside = np.abs(t) < nb + 5
        err = np.abs(tf.astype(np.float64) - t)[inside]
        bound = float(inv) * 6.5e-7 + np.abs(t[inside]) * 3.6e-7
        assert np.all(err <= bound)
        assert ok[k:].mean() > 0.99


def test_guarded_observe_and_pick_agree_with_binary64():
    g = np.random.default_rng(4)
    n = 2_000_000
    v = g.integers(0, 2 ** 32, (n, 4), dtype=np.uint64)
    mx = g.integers(1, 5000, n)
    cnt = np.minimum(g.integers(1, 5000, n), mx)
    def u01(lo, hi):
        return ((((hi << np.uint64(32)) | lo) >> np.uint64(12)).astype(np.float64) + 0.5) * 2.0 ** -52
    u1, u2 = u01(v[:, 0], v[:, 1]), u01(v[:, 2], v[:, 3])
    obs = u1 * mx < cnt
    p1 = ((v[:, 1] >> np.uint64(8)).astype(f32) * f32(2.0 ** -24) * mx.astype(f32)).astype(f32)
    sure = np.abs(p1 - cnt.astype(f32)) > f32(2e-6) * mx.astype(f32)
    assert np.array_equal((p1 < cnt.astype(f32))[sure], obs[sure])
    pk = np.minimum((u2 * cnt).astype(np.int64), cnt - 1)
    p2 = ((v[:, 3] >> np.uint64(8)).astype(f32) * f32(2.0 ** -24) * cnt.astype(f32)).astype(f32)
    pk32, ok = _floor_sure(p2, f32(2e-6) * cnt.astype(f32))
    assert np.array_equal(pk32[ok], pk[ok])
    assert sure.mean() > 0.9999 and ok.mean() > 0.98
