"""Pins of the oracle's analytic disk + halo galactic field (the synthetic
regular field of the galactic back-tracking workload: logarithmic-spiral disk
with pitch p and exponential scale height, toroidal halo peaked at |z| = z0)
to facts fixed outside the oracle: field lines of the disk traced here by RK4
are logarithmic spirals of pitch p, numpy's exp for the vertical profiles, the
disk's radial support, the halo's parity and divergence (finite differences),
and superposition / translation.  A swapped sin/cos of the pitch, a wrong
sign of the halo, a dropped |z| or a shifted centre each fail one of them."""
import numpy as np
import pytest

import workloads

DISK = workloads.GALACTIC_LENS["disk"]


def _params(oracle, **over):
    g = dict(DISK)
    g.update(over)
    return oracle.make_params(grid_n=(2, 2, 2), spacing=1.0, flags=oracle.GALACTIC, galactic=g)


def _field(oracle, pts, **over):
    return oracle.field_at(_params(oracle, **over), np.zeros((2, 2, 2, 3)),
                           np.asarray(pts, dtype=np.float64).reshape(-1, 3))


def _cyl(r, phi, z):
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def _radial_azimuthal(B, pts):
    phi = np.arctan2(pts[:, 1], pts[:, 0])
    return (B[:, 0] * np.cos(phi) + B[:, 1] * np.sin(phi),
            -B[:, 0] * np.sin(phi) + B[:, 1] * np.cos(phi))


def test_disk_field_lines_are_log_spirals(oracle):
    """Trace a midplane field line with RK4 on the unit field direction: for a
    logarithmic spiral of pitch p, ln r grows by tan p per radian of azimuth."""
    p = DISK["disk_pitch_rad"]

    def f(x):
        b = _field(oracle, x[None, :], halo_b=0.0)[0]
        return b / np.linalg.norm(b)

    x = np.array([6.0, 0.0, 0.0])
    h, phi_prev, phi_unwrapped = 0.01, 0.0, 0.0
    for _ in range(800):
        k1 = f(x)
        k2 = f(x + 0.5 * h * k1)
        k3 = f(x + 0.5 * h * k2)
        k4 = f(x + h * k3)
        x = x + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        phi = np.arctan2(x[1], x[0])
        phi_unwrapped += (phi - phi_prev + np.pi) % (2 * np.pi) - np.pi
        phi_prev = phi
    r = np.hypot(x[0], x[1])
    assert 3.0 < r < 20.0 and phi_unwrapped > 1.0          # stayed on the disk, turned
    assert abs(x[2]) == 0.0                                  # no vertical field
    assert abs(np.log(r / 6.0) - np.tan(p) * phi_unwrapped) < 1e-9


def test_disk_vertical_profile_and_support(oracle):
    g = np.random.default_rng(4)
    n = 4000
    r = g.uniform(0.0, 25.0, n)
    phi = g.uniform(-np.pi, np.pi, n)
    z = g.uniform(-6.0, 6.0, n)
    pts = _cyl(r, phi, z)
    B = _field(oracle, pts, halo_b=0.0)
    mag = np.linalg.norm(B, axis=1)
    on = (r >= DISK["disk_rmin"]) & (r <= DISK["disk_rmax"])
    assert np.all(mag[~on] == 0.0)
    want = DISK["disk_b"] * np.exp(-np.abs(z[on]) / DISK["disk_hz"])
    assert np.max(np.abs(mag[on] - want) / want) < 1e-14
    assert np.all(B[:, 2] == 0.0)
    # even in z, outward-trailing: positive radial and azimuthal parts
    Bm = _field(oracle, _cyl(r, phi, -z), halo_b=0.0)
    assert np.array_equal(B, Bm)
    br, bp = _radial_azimuthal(B[on], pts[on])
    assert np.all(br > 0) and np.all(bp > 0)
    # the support includes both radii
    edge = _cyl(np.array([DISK["disk_rmin"], DISK["disk_rmax"]]), np.array([0.3, -2.0]),
                np.zeros(2))
    assert np.all(np.linalg.norm(_field(oracle, edge, halo_b=0.0), axis=1) > 0)
    inner = _cyl(np.array([np.nextafter(DISK["disk_rmin"], 0.0)]), np.array([0.3]), np.zeros(1))
    assert np.all(_field(oracle, inner, halo_b=0.0) == 0.0)


def test_halo_is_toroidal_odd_and_peaked(oracle):
    g = np.random.default_rng(5)
    n = 3000
    r = g.uniform(0.05, 30.0, n)
    phi = g.uniform(-np.pi, np.pi, n)
    z = g.uniform(-8.0, 8.0, n)
    pts = _cyl(r, phi, z)
    B = _field(oracle, pts, disk_b=0.0)
    br, bp = _radial_azimuthal(B, pts)
    assert np.max(np.abs(br)) < 1e-15 and np.all(B[:, 2] == 0.0)
    assert np.all(np.sign(bp) == np.sign(z))                 # north positive, south negative
    z0, s, bh = DISK["halo_z0"], DISK["halo_sigma"], DISK["halo_b"]
    want = bh * np.exp(-(np.abs(z) - z0) ** 2 / (2 * s * s))
    assert np.max(np.abs(np.abs(bp) - want)) < 1e-14 * bh
    assert np.array_equal(_field(oracle, _cyl(r, phi, -z), disk_b=0.0), -B)
    # peak bh at |z| = z0, bh e^(-1/2) one sigma either side, nothing in the midplane
    zs = np.array([z0, -z0, z0 + s, z0 - s, 0.0])
    Bz = _field(oracle, _cyl(np.full(5, 7.0), np.full(5, 1.0), zs), disk_b=0.0)
    m = np.linalg.norm(Bz, axis=1)
    assert abs(m[0] - bh) < 1e-15 and abs(m[1] - bh) < 1e-15
    assert np.allclose(m[2:4], bh * np.exp(-0.5), rtol=1e-14, atol=0) and m[4] == 0.0


def test_halo_is_divergence_free(oracle):
    """A purely azimuthal field whose strength does not depend on azimuth has
    no divergence (checked by central differences away from z = 0)."""
    g = np.random.default_rng(6)
    n, d = 400, 1e-4
    pts = _cyl(g.uniform(1.0, 20.0, n), g.uniform(-np.pi, np.pi, n),
               np.where(g.random(n) < 0.5, -1, 1) * g.uniform(0.2, 5.0, n))
    div = np.zeros(n)
    for a in range(3):
        e = np.zeros(3)
        e[a] = d
        div += (_field(oracle, pts + e, disk_b=0.0)[:, a]
                - _field(oracle, pts - e, disk_b=0.0)[:, a]) / (2 * d)
    assert np.max(np.abs(div)) < 1e-7 * DISK["halo_b"]


@pytest.mark.parametrize("center", [(0.0, 0.0, 0.0), (1.5, -2.0, 0.25)])
def test_superposition_and_centre(oracle, center):
    g = np.random.default_rng(7)
    pts = g.uniform(-22.0, 22.0, (2000, 3))
    pts[:, 2] = g.uniform(-5.0, 5.0, 2000)
    c = np.array(center)
    both = _field(oracle, pts + c, center=center)
    disk = _field(oracle, pts + c, center=center, halo_b=0.0)
    halo = _field(oracle, pts + c, center=center, disk_b=0.0)
    assert np.max(np.abs(both - (disk + halo))) < 1e-15
    # the field about a shifted centre is the centred field, shifted
    ref = _field(oracle, pts)
    assert np.max(np.abs(both - ref)) < 1e-12
