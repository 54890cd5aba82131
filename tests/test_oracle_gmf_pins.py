"""Pins of the oracle's analytic multi-arm galactic field, and of the
arctangent that steers its spiral phase, to facts fixed outside the oracle:
numpy's arctan2, the absence of magnetic monopoles (div B = 0, by finite
differences), the log-spiral field lines of the disk (integrated here by RK4),
zero net flux of the arms through a circle, straight X-field lines, and the
limits the model reduces to (midplane, scale height, north/south strengths,
cuts).  A dropped 1/r, a wrong pitch sign, a mirrored arm assignment or a wrong
power in the X field each fail one of them."""
import numpy as np
import pytest

import workloads


def _gmf(oracle, **over):
    p = workloads.multiarm_gmf_params()
    p.update(over)
    return oracle.make_gmf(**p)


DISK_ONLY = dict(halo_bn=0.0, halo_bs=0.0, x_b=0.0)
HALO_ONLY = dict(arm_b=(0.0,) * 8, ring_b=0.0, x_b=0.0)
X_ONLY = dict(arm_b=(0.0,) * 8, ring_b=0.0, halo_bn=0.0, halo_bs=0.0)


def _cyl(r, phi, z):
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def _radial_azimuthal(B, pts):
    phi = np.arctan2(pts[:, 1], pts[:, 0])
    br = B[:, 0] * np.cos(phi) + B[:, 1] * np.sin(phi)
    bp = -B[:, 0] * np.sin(phi) + B[:, 1] * np.cos(phi)
    return br, bp


def test_series_atan2_against_numpy(oracle):
    g = np.random.default_rng(3)
    n = 200_000
    y = g.normal(size=n) * 10 ** g.uniform(-6, 6, n)
    x = g.normal(size=n) * 10 ** g.uniform(-6, 6, n)
    a = oracle.series_atan2(y, x)
    ref = np.arctan2(y, x)
    assert np.max(np.abs(a - ref) / np.spacing(np.abs(ref))) <= 8
    axes_y = np.array([0.0, 1.0, -1.0, 0.0, 2.0, -2.0, 3.0, -3.0, 0.0])
    axes_x = np.array([1.0, 0.0, 0.0, -1.0, 2.0, 2.0, -3.0, -3.0, 0.0])
    exact = np.array([0.0, np.pi / 2, -np.pi / 2, np.pi, np.pi / 4, -np.pi / 4,
                      3 * np.pi / 4, -3 * np.pi / 4, 0.0])
    assert np.max(np.abs(oracle.series_atan2(axes_y, axes_x) - exact)) <= 4.5e-16


@pytest.mark.parametrize("part", ["disk", "halo", "x"])
def test_gmf_is_divergence_free(oracle, part):
    off = dict(disk=DISK_ONLY, halo=HALO_ONLY, x=X_ONLY)[part]
    g = _gmf(oracle, **off)
    rng = np.random.default_rng(5)
    n = 20_000
    pts = _cyl(rng.uniform(0.5, 19.5, n), rng.uniform(-np.pi, np.pi, n), rng.uniform(-6, 6, n))
    R = np.linalg.norm(pts, axis=1)
    pts = pts[(R > 1.01) & (R < 19.99)]
    scale = np.abs(oracle.gmf_at(g, pts)).max()
    h = 1e-4
    div = np.zeros(len(pts))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        div += (oracle.gmf_at(g, pts + e)[:, k] - oracle.gmf_at(g, pts - e)[:, k]) / (2 * h)
    # finite-difference truncation ~h^2 B''' (transition widths 0.1-0.2 kpc);
    # points within h of a tangential discontinuity (arm edges, the plane for
    # the X field's B_r) are the only ones allowed above it
    assert scale > 0.5
    assert np.mean(np.abs(div) < 1e-5 * scale) > 0.99
    assert np.median(np.abs(div)) < 1e-6 * scale


def test_gmf_arms_carry_no_net_flux(oracle):
    n = 1 << 16
    phi = (np.arange(n) + 0.5) * (2 * np.pi / n) - np.pi
    p = workloads.multiarm_gmf_params()

    def flux(g, r):
        pts = _cyl(np.full(n, r), phi, np.zeros(n))
        br, _ = _radial_azimuthal(oracle.gmf_at(g, pts), pts)
        return br.sum() * r * (2 * np.pi / n), np.abs(br).sum() * r * (2 * np.pi / n)

    g = _gmf(oracle, **DISK_ONLY)
    for r in (5.5, 7.7, 10.3, 14.0, 18.5):
        f, s = flux(g, r)
        assert s > 1.0 and abs(f) < 1e-3 * s, (r, f, s)
    b = list(p["arm_b"])
    b[7] *= 1.1  # the flux-free eighth arm, perturbed: the net flux shows
    f, s = flux(_gmf(oracle, **DISK_ONLY, arm_b=tuple(b)), 10.3)
    assert abs(f) > 2e-2 * s


def test_gmf_disk_field_lines_are_log_spirals(oracle):
    """RK4 along the midplane field: ln r - phi tan p stays constant (pitch p
    log spiral), and |B| r stays |b_j| r_in (1 - L(0)) -- the line never leaves
    the arm it starts in."""
    p = workloads.multiarm_gmf_params()
    g = _gmf(oracle, **DISK_ONLY, r_cut_out=0.0, r_out=40.0)
    tan_p = np.tan(p["pitch_rad"])
    rx = list(p["arm_rx"]) + [p["arm_rx"][0] * np.exp(2 * np.pi * tan_p)]
    r0 = np.array([np.sqrt(rx[j] * rx[j + 1]) for j in range(8)])  # middle of arm j on phi = pi
    x = _cyl(r0, np.full(8, np.pi), np.zeros(8))
    L0 = 1.0 / (1.0 + np.exp(2.0 * p["h_disk"] / p["w_disk"]))
    expect = np.abs(np.array(p["arm_b"])) * p["r_in"] * (1.0 - L0)

    def direction(x):
        B = oracle.gmf_at(g, x)
        _, bp = _radial_azimuthal(B, x)
        d = B / np.linalg.norm(B, axis=1, keepdims=True)
        return d * np.sign(bp)[:, None]  # always toward +phi

    ds = 0.02
    phi_unwrapped = np.full(8, np.pi)
    inv0 = np.log(r0) - phi_unwrapped * tan_p
    for step in range(1500):  # a quarter to a full turn, depending on r0
        k1 = direction(x)
        k2 = direction(x + 0.5 * ds * k1)
        k3 = direction(x + 0.5 * ds * k2)
        k4 = direction(x + ds * k3)
        xn = x + ds / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        dphi = np.angle(np.exp(1j * (np.arctan2(xn[:, 1], xn[:, 0]) - np.arctan2(x[:, 1], x[:, 0]))))
        phi_unwrapped += dphi
        x = xn
        r = np.hypot(x[:, 0], x[:, 1])
        if step % 100 == 99:
            assert np.max(np.abs(np.log(r) - phi_unwrapped * tan_p - inv0)) < 1e-7
            Bn = np.linalg.norm(oracle.gmf_at(g, x), axis=1)
            assert np.max(np.abs(Bn * r / expect - 1)) < 1e-9
    assert np.all(phi_unwrapped - np.pi > 1.0)


def test_gmf_reference_ray_and_ring(oracle):
    """On the phi = pi ray each arm boundary is where the definition puts it:
    between arm_rx[j] and arm_rx[j+1] the field is b_j (r_in / r)(1 - L(0)) along
    (sin p r_hat + cos p phi_hat); the ring is azimuthal with ring_b (1 - L(0))."""
    p = workloads.multiarm_gmf_params()
    g = _gmf(oracle, **DISK_ONLY)
    L0 = 1.0 / (1.0 + np.exp(2.0 * p["h_disk"] / p["w_disk"]))
    sp, cp = np.sin(p["pitch_rad"]), np.cos(p["pitch_rad"])
    rx = list(p["arm_rx"]) + [p["arm_rx"][0] * np.exp(2 * np.pi * np.tan(p["pitch_rad"]))]
    for j in range(8):
        for r in np.linspace(rx[j], rx[j + 1], 7)[1:-1]:
            B = oracle.gmf_at(g, [[-r, 0.0, 0.0]])[0]
            bd = p["arm_b"][j] * p["r_in"] / r * (1 - L0)
            # r_hat = (-1, 0, 0), phi_hat = (0, -1, 0) on this ray
            assert np.allclose(B, [-bd * sp, -bd * cp, 0.0], rtol=1e-13, atol=1e-15), (j, r)
    pts = _cyl(np.full(64, 4.0), np.linspace(-np.pi, np.pi, 64, endpoint=False), np.zeros(64))
    br, bp = _radial_azimuthal(oracle.gmf_at(g, pts), pts)
    assert np.max(np.abs(br)) < 1e-15 and np.allclose(bp, p["ring_b"] * (1 - L0), rtol=1e-13)
    inner = _cyl(np.full(8, 2.5), np.linspace(0, 6, 8), np.zeros(8))
    outer = _cyl(np.full(8, 20.5), np.linspace(0, 6, 8), np.zeros(8))
    assert not oracle.gmf_at(_gmf(oracle, **DISK_ONLY, r_cut_out=0.0), np.vstack([inner, outer])).any()


def test_gmf_halo_limits(oracle):
    """Toroidal only; far above the disk (L(z) = 1 to 1e-9) and well inside
    r_n, r_s the strength falls as e^{-|z|/z0} with halo_bn north and halo_bs
    south; beyond r_n it falls off on the scale halo_wh."""
    p = workloads.multiarm_gmf_params()
    g = _gmf(oracle, **HALO_ONLY, r_cut_in=0.0, r_cut_out=0.0)
    phi = np.linspace(-3, 3, 7)
    for z in (3.0, 4.0, -3.0, -4.0):
        pts = _cyl(np.full(7, 2.0), phi, np.full(7, z))
        B = oracle.gmf_at(g, pts)
        br, bp = _radial_azimuthal(B, pts)
        assert np.max(np.abs(br)) < 1e-15 and not B[:, 2].any()
        b0 = p["halo_bn"] if z > 0 else p["halo_bs"]
        assert np.allclose(bp, b0 * np.exp(-abs(z) / p["halo_z0"]), rtol=1e-8)
    far = _cyl(np.array([p["halo_rn"] + 10 * p["halo_wh"]]), np.zeros(1), np.array([3.0]))
    near = _cyl(np.array([p["halo_rn"] - 10 * p["halo_wh"]]), np.zeros(1), np.array([3.0]))
    assert abs(oracle.gmf_at(g, far)[0, 1]) < 1e-7 * abs(oracle.gmf_at(g, near)[0, 1])


def test_gmf_x_field_lines_and_midplane(oracle):
    """The X field lies in meridional planes, its lines are straight (the
    direction is unchanged a step along the line), B_z is even and B_r odd in z,
    and at the midplane |B| = x_b e^{-r/x_r} with elevation x_theta outside x_rc
    and atan(x_rc tan x_theta / r) inside."""
    p = workloads.multiarm_gmf_params()
    g = _gmf(oracle, **X_ONLY, r_cut_in=0.0, r_cut_out=0.0)
    rng = np.random.default_rng(8)
    n = 4000
    pts = _cyl(rng.uniform(0.3, 15.0, n), rng.uniform(-np.pi, np.pi, n),
               rng.choice([-1, 1], n) * rng.uniform(0.2, 8.0, n))
    B = oracle.gmf_at(g, pts)
    br, bp = _radial_azimuthal(B, pts)
    assert np.max(np.abs(bp)) < 1e-14 * np.abs(B).max()
    d = B / np.linalg.norm(B, axis=1, keepdims=True)
    # one step along the line (away from the plane, so it stays on its side)
    away = d * np.sign(d[:, 2] * pts[:, 2])[:, None]
    d2 = oracle.gmf_at(g, pts + 0.05 * away)
    d2 = d2 / np.linalg.norm(d2, axis=1, keepdims=True)
    same = np.max(np.abs(d2 - d), axis=1) < 1e-12
    assert same.mean() > 0.99
    mirror = pts * np.array([1.0, 1.0, -1.0])
    Bm = oracle.gmf_at(g, mirror)
    brm, _ = _radial_azimuthal(Bm, mirror)
    assert np.allclose(Bm[:, 2], B[:, 2], rtol=1e-14, atol=0) and np.allclose(brm, -br, rtol=1e-14, atol=0)
    r = np.linspace(0.5, 14.5, 57)
    mid = _cyl(r, np.zeros(57), np.full(57, 1e-12))
    Bmid = oracle.gmf_at(g, mid)
    brm, _ = _radial_azimuthal(Bmid, mid)
    tan_t = np.tan(p["x_theta_rad"])
    elev = np.where(r >= p["x_rc"], p["x_theta_rad"], np.arctan(p["x_rc"] * tan_t / r))
    mag = p["x_b"] * np.exp(-r / p["x_r"])
    assert np.allclose(np.hypot(brm, Bmid[:, 2]), mag, rtol=1e-9)
    assert np.allclose(np.arctan2(Bmid[:, 2], brm), elev, rtol=0, atol=1e-9)


def test_gmf_spherical_cuts(oracle):
    p = workloads.multiarm_gmf_params()
    g = _gmf(oracle)
    rng = np.random.default_rng(2)
    d = rng.normal(size=(500, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    assert not oracle.gmf_at(g, d * rng.uniform(0.01, 0.99 * p["r_cut_in"], (500, 1))).any()
    assert not oracle.gmf_at(g, d * rng.uniform(1.01 * p["r_cut_out"], 40.0, (500, 1))).any()
    assert np.abs(oracle.gmf_at(g, d * 8.0)).max() > 0.1
