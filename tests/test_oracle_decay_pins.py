"""Pins of the oracle's decay of unstable nuclei (Sect. 2 lists nuclear decay
among the interactions) to what the physics fixes, independent of the
oracle's arithmetic:
  * survival: the probability that a nucleus of rest-frame lifetime tau and
    Lorentz factor gamma = E / (A m_p c^2) has not decayed after a path L is
    exp(-L / (gamma c tau));
  * branching: the first decay's channel is drawn with the table's
    fractions (chi-square), and the daughter is the one the channel defines
    (beta-: Z + 1; beta+: Z - 1; neutron / proton emission: A - 1 with the
    nucleon as a secondary);
  * conservation: nucleon number per lineage; energy per nucleon in nucleon
    emission; the energy of a beta decay's nucleus (mass A m_p) unchanged;
  * chains end on stable nuclides; stable nuclides never decay.
The lifetimes and branchings are the synthetic table of the workloads
(input data: no measured table is in the container)."""
import math

import numpy as np
import pytest

import workloads

MP_C2 = 938.27208816e6          # proton rest energy [eV] (CODATA 2018)
C_LIGHT = 299792458.0
MPC_M = 3.0856775814913673e22


def _one(E, A, Z, n, s_max):
    return dict(id=np.arange(n, dtype=np.uint64), x=np.zeros(n), y=np.zeros(n), z=np.zeros(n),
                ux=np.ones(n), uy=np.zeros(n), uz=np.zeros(n), E=np.full(n, E),
                A=np.full(n, A, np.int32), Z=np.full(n, Z, np.int32),
                q=np.ones(n, np.int32), s_max=np.full(n, s_max))


def _params(oracle, table, L, flags=None, seed=3):
    return oracle.make_params(grid_n=(4, 4, 4), spacing=1.0,
                              flags=oracle.DECAY if flags is None else flags, seed=seed,
                              h_max=0.25 * L, h_min=1e-9, decay_table=table)


def _field():
    return np.zeros((4, 4, 4, 3))


@pytest.fixture(scope="module")
def table():
    return workloads.synthetic_decay_table()


def _entry(table, A, Z):
    k = np.nonzero((table["A"] == A) & (table["Z"] == Z))[0]
    return (float(table["tau_s"][k[0]]), table["branching"][k[0]]) if len(k) else None


def test_survival_is_exponential_in_gamma_c_tau(oracle, table):
    A, Z = 56, 28
    tau, b = _entry(table, A, Z)
    assert b[1] == 1.0                    # pure beta+: the daughter is (56, 27)
    E = 5e19
    lam = E / (A * MP_C2) * C_LIGHT * tau / MPC_M     # decay length gamma c tau [Mpc]
    n = 5000
    for x in (0.1, 0.5, 1.0, 2.0, 3.0):
        r = oracle.propagate(_params(oracle, table, x * lam), _field(),
                             _one(E, A, Z, n, x * lam))
        assert np.all(r["generation"] == 0)
        survived = np.mean((r["A"] == A) & (r["Z"] == Z))
        p = math.exp(-x)
        assert abs(survived - p) < 4 * math.sqrt(p * (1 - p) / n) + 1e-3, (x, survived, p)


def test_branching_daughters_and_conservation(oracle):
    """A hand-made table: (20, 10) with all four channels, every daughter
    stable.  The primary's final species identifies the channel."""
    tab = dict(A=np.array([20], np.int32), Z=np.array([10], np.int32), tau_s=np.array([50.0]),
               branching=np.array([[0.2, 0.3, 0.1, 0.4]]))
    E = 2e19
    lam = E / (20 * MP_C2) * C_LIGHT * 50.0 / MPC_M
    n = 8000
    r = oracle.propagate(_params(oracle, tab, 40 * lam), _field(), _one(E, 20, 10, n, 40 * lam))
    prim = r[r["generation"] == 0]
    sec = r[r["generation"] == 1]
    assert len(prim) == n
    species = {(20, 11): 0, (20, 9): 1, (19, 10): 2, (19, 9): 3}
    ch = np.array([species[(int(a), int(z))] for a, z in zip(prim["A"], prim["Z"])])
    counts = np.bincount(ch, minlength=4)
    expect = n * np.array([0.2, 0.3, 0.1, 0.4])
    chi2 = float(np.sum((counts - expect) ** 2 / expect))
    assert chi2 < 16.3, (counts, chi2)        # 3 dof, p = 0.001
    kids = {int(s["parent_id"]): s for s in sec}
    assert len(sec) == counts[2] + counts[3]
    for p, c in zip(prim, ch):
        if c < 2:
            # beta decay: the nucleus keeps its energy; no secondary
            assert p["E"] == E and int(p["id"]) not in kids
        else:
            k = kids[int(p["id"])]
            # the nucleon: A = 1, neutron (emission) or proton, E / A; the
            # daughter: E (A - 1) / A; nucleon number conserved
            assert k["A0"] == 1 and k["Z0"] == (0 if c == 2 else 1)
            assert k["E0"] == E / 20 and p["E"] == E * 19 / 20
            assert p["A"] + k["A0"] == 20
            assert int(k["id"]) == oracle.child_id(int(p["id"]), 0)
    # one uniform per reset and one channel draw per decay: start, event, reset
    assert np.all(prim["draws"] == 3)


def test_chains_end_on_stable_nuclides(oracle, table):
    """A short-lived proton-rich iron isotope decays until it reaches a
    nuclide the table lists as stable; nucleon number is conserved per
    lineage (nucleons emitted on the way are secondaries; free neutrons
    decay to protons)."""
    unstable = set(zip(table["A"].tolist(), table["Z"].tolist()))
    A, Z = 45, 26
    assert (A, Z) in unstable
    n = 400
    r = oracle.propagate(_params(oracle, table, 1e4), _field(), _one(1e20, A, Z, n, 1e4))
    prim = r[r["generation"] == 0]
    assert len(prim) == n
    for p in prim:
        assert (int(p["A"]), int(p["Z"])) not in unstable
        assert int(p["A"]) >= 2 and 1 <= int(p["Z"]) <= int(p["A"]) - 1
    total = {}
    for rec in r:
        root = int(rec["id"]) if rec["generation"] == 0 else int(rec["parent_id"])
        total[root] = total.get(root, 0) + int(rec["A"])
    # secondaries here are nucleons emitted by the primary itself (generation 1)
    assert set(r["generation"].tolist()) <= {0, 1}
    assert all(v == A for v in total.values())
    # the stability line is approached from the proton-rich side
    assert np.all(prim["Z"] < Z)


def test_stable_nuclides_and_other_modules_unchanged(oracle, table):
    """Nuclides the table does not list never decay (one uniform drawn at
    the start); a table changes nothing for runs without DECAY."""
    for A, Z in ((56, 26), (14, 7), (4, 2), (2, 1)):
        assert _entry(table, A, Z) is None
        r = oracle.propagate(_params(oracle, table, 10.0), _field(), _one(3e19, A, Z, 20, 10.0))
        assert np.all(r["A"] == A) and np.all(r["Z"] == Z) and np.all(r["E"] == 3e19)
        assert np.all(r["draws"] == 1)
    inj = _one(5e19, 56, 28, 50, 50.0)
    P0 = oracle.make_params(grid_n=(4, 4, 4), spacing=1.0, flags=0, h_max=1.0, h_min=1e-6)
    P1 = oracle.make_params(grid_n=(4, 4, 4), spacing=1.0, flags=0, h_max=1.0, h_min=1e-6,
                            decay_table=table)
    r0 = oracle.propagate(P0, _field(), inj)
    r1 = oracle.propagate(P1, _field(), inj)
    assert r0.tobytes() == r1.tobytes() and np.all(r0["Z"] == 28)


def test_synthetic_table_recipe(table):
    """The recipe's table: the injected species are stable, fractions sum to
    one, every channel with a non-zero fraction has a valid daughter, and
    the unstable nuclides lie beyond one charge unit of Green's stability
    line (which puts iron-56, nitrogen-14 and helium-4 within it)."""
    A, Z, b = table["A"], table["Z"], table["branching"]
    assert np.allclose(b.sum(axis=1), 1.0, atol=1e-12) and np.all(b >= 0)
    assert np.all(table["tau_s"] > 0) and np.all(np.isfinite(table["tau_s"]))
    zs = workloads.beta_stability_z(A)
    assert np.all(np.abs(Z - zs) > 1.0)
    for a, z in ((56, 26), (14, 7), (4, 2)):
        assert abs(z - workloads.beta_stability_z(a)) <= 1.0
    for (a, z, bb) in zip(A, Z, b):
        for k, (ad, zd) in enumerate(((a, z + 1), (a, z - 1), (a - 1, z), (a - 1, z - 1))):
            if bb[k] > 0:
                assert ad >= 1 and 0 <= zd <= ad
                if ad >= 2:
                    assert 1 <= zd <= ad - 1
    # proton-rich nuclides decay by beta+ / proton emission, neutron-rich by beta- / n
    rich = Z > zs
    assert np.all(b[rich][:, [0, 2]] == 0) and np.all(b[~rich][:, [1, 3]] == 0)
