"""Pins of the oracle's rigid 3-site water step (the paper's bulk-water runs keep the molecules
rigid with SHAKE, Sec. 5.1): the Ewald energy with the intramolecular pairs excluded does not
depend on alpha; the forces are -grad U; the molecular virial is -dU/d eps when the molecular
centres (not the sites) scale with the box; SHAKE and RATTLE hold the distances and the velocity
constraints; the extended energy drifts by O(dt^2) without friction and noise; non-interacting
rigid molecules reach the isobaric ideal-gas volume (N_mol + 1) kT / P of their centres."""
import math

import numpy as np
import pytest

import oracle

KT = oracle.KB * 300.0
Q = np.array([-0.8476, 0.4238, 0.4238])
MASS = np.array([15.9994, 1.008, 1.008])
HALF = math.radians(109.47) / 2
LOCAL = np.array([[0.0, 0.0, 0.0], [math.sin(HALF), 0.0, math.cos(HALF)], [-math.sin(HALF), 0.0, math.cos(HALF)]])


def _rotations(n, rng):
    qt = rng.normal(size=(n, 4))
    qt /= np.linalg.norm(qt, axis=1, keepdims=True)
    w, x, y, z = qt.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1)], 1)


def _waters(n_side, L, seed, jitter=0.3, thermal=1.0):
    """n_side^3 molecules at random orientations on a jittered lattice of a cubic box L; site
    momenta at `thermal` times 300 K (not yet constrained)."""
    rng = np.random.default_rng(seed)
    g = (np.arange(n_side) + 0.5) * (L / n_side)
    c = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + rng.uniform(-jitter, jitter, (n_side ** 3, 3))
    pos = (c[:, None, :] + np.einsum("nij,sj->nsi", _rotations(len(c), rng), LOCAL)).reshape(-1, 3)
    n = len(c)
    q = np.tile(Q, n)
    m = np.tile(MASS, n)
    p = rng.normal(size=(3 * n, 3)) * np.sqrt(KT * 100 * m)[:, None] * thermal
    return np.mod(pos, L), p, q, m, np.array([L, L, L])


def _energy(pos, q, box, alpha, rc, kmax, lj=(3.166, 0.650)):
    Fk, Wk, Ek, Es = oracle.ewald_kspace(pos, q, box, alpha, kmax)
    Fr, Wr, Ec, El, Ex = oracle.water_real(pos, q, box, alpha, rc, oracle.QQR2E, *lj)
    E = oracle.QQR2E * (Ek + Es) + Ec + El + Ex
    return E, oracle.QQR2E * Fk + Fr, oracle.QQR2E * np.trace(Wk) + Wr


def test_excluded_ewald_energy_is_alpha_independent():
    """Ewald over all sites minus the intramolecular erf terms is the Coulomb energy between
    molecules (and their images): the same for any splitting alpha."""
    pos, _, q, m, box = _waters(3, 9.3, 1)
    # both splittings converged: erfc(sqrt(a) rc) < 2e-14 and exp(-pi^2 kmax^2 / (a L^2)) < 1e-14
    E1 = _energy(pos, q, box, 1.4, 4.6, 21, lj=(3.166, 0.0))[0]
    E2 = _energy(pos, q, box, 2.0, 4.6, 25, lj=(3.166, 0.0))[0]
    assert abs(E1 - E2) < 1e-9 * abs(E1), (E1, E2)
    # without the exclusion the two differ by the alpha dependence of the intramolecular terms
    Ex = [oracle.water_real(pos, q, box, a, 4.6, oracle.QQR2E, 3.166, 0.0)[4] for a in (1.4, 2.0)]
    assert abs((E1 - Ex[0]) - (E2 - Ex[1])) > 10.0


def test_forces_are_the_gradient():
    pos, _, q, m, box = _waters(3, 9.3, 2)
    alpha, rc, kmax = 0.6, 4.6, 20
    E0, F, _ = _energy(pos, q, box, alpha, rc, kmax)
    h = 1e-6
    for i, t in [(0, 0), (4, 1), (11, 2), (25, 0)]:
        xp, xm = pos.copy(), pos.copy()
        xp[i, t] += h
        xm[i, t] -= h
        d = -(_energy(xp, q, box, alpha, rc, kmax)[0] - _energy(xm, q, box, alpha, rc, kmax)[0]) / (2 * h)
        assert abs(d - F[i, t]) < 1e-6 * np.abs(F).max(), (i, t, d, F[i, t])


def test_molecular_virial_is_the_volume_derivative():
    """Centres scaled by (1 + e) with the box, shapes kept: W_mol = -dU/de."""
    pos, _, q, m, box = _waters(3, 9.3, 3)
    alpha, rc, kmax = 0.6, 4.6, 20
    _, F, W = _energy(pos, q, box, alpha, rc, kmax)
    Wmol = W + oracle.water_virial_corr(pos, m, box, F)
    n = len(q) // 3

    def scaled(e):
        x = pos.reshape(n, 3, 3).copy()
        x[:, 1:] = x[:, :1] + (x[:, 1:] - x[:, :1] + box / 2) % box - box / 2  # whole molecules
        R = np.einsum("s,nsi->ni", MASS, x) / MASS.sum()
        x = x + (e * R)[:, None, :]
        return np.mod(x.reshape(-1, 3), box * (1 + e)), box * (1 + e)

    h = 1e-6
    Up = _energy(*scaled(h)[:1], q, scaled(h)[1], alpha, rc, kmax)[0]
    Um = _energy(*scaled(-h)[:1], q, scaled(-h)[1], alpha, rc, kmax)[0]
    d = -(Up - Um) / (2 * h)
    assert abs(d - Wmol) < 1e-6 * max(1.0, abs(Wmol)), (d, Wmol, W)
    assert abs(Wmol - W) > 1.0  # the intramolecular part of the atomic virial is not small here


def _cold_lattice(seed=5):
    """27 molecules on a 6 A lattice in an 18 A box, cold: O-O neighbours at ~6 A, the next shell
    beyond 8.4 A, rc = 8 A between them (no oxygen pair crosses the LJ cutoff), alpha = 0.6 so that
    the Coulomb terms are nil at rc."""
    return _waters(3, 18.0, seed, jitter=0.05, thermal=0.1)


def _drift(dt, ps=0.3):
    pos, p, q, m, box = _cold_lattice()
    prm = oracle.npt_params(dt=dt, gamma=0.0, gamma_V=0.0, noise=0, kspace=0, real=1, alpha=0.6, rc=8.0,
                            lj_sigma=3.166, lj_eps=0.650, barostat=1, M_V=oracle.piston_mass(0.5, 0.75, 18.0 ** 3),
                            P_ext=oracle.BAR)
    wp = oracle.water_params()
    st = oracle.WaterState(pos, p, q, m, box)
    oracle.water_forces(st, 0, prm)
    V, Pi, H = oracle.water_run(st, 0, int(round(ps / dt)), prm, wp)
    return np.abs(H - H[0]).max(), V, st, wp


def test_constraints_hold():
    _, _, st, wp = _drift(0.001, ps=0.05)
    dv, vv = oracle.water_violation(st, wp)
    assert dv < 1e-13 and vv < 1e-12, (dv, vv)


def test_extended_energy_drift_is_second_order():
    d1, V, _, _ = _drift(0.001)
    d2, _, _, _ = _drift(0.0005)
    assert V.max() / V.min() > 1.005  # the cell moves (a lighter piston moves an oxygen pair across rc)
    assert d1 < 1e-7, d1
    assert d2 < d1 / 3.5, (d1, d2)


@pytest.mark.slow
def test_rigid_ideal_gas_volume():
    """U = 0: only the molecular centres feel the cell, so <V> = (N_mol + 1) kT / P."""
    n = 8
    V0 = 2000.0
    P = (n + 1) * KT / V0
    rng = np.random.default_rng(4)
    L = V0 ** (1 / 3)
    c = rng.random((n, 3)) * L
    pos = np.mod((c[:, None, :] + np.einsum("nij,sj->nsi", _rotations(n, rng), LOCAL)).reshape(-1, 3), L)
    m = np.tile(MASS, n)
    p = rng.normal(size=(3 * n, 3)) * np.sqrt(KT * 100 * m)[:, None]
    prm = oracle.npt_params(kspace=0, real=0, noise=1, gamma=5.0, gamma_V=20.0, M_V=oracle.piston_mass(0.2, 1.0 / P, V0),
                            P_ext=P, dt=0.002, seed=21, barostat=1)
    wp = oracle.water_params()
    st = oracle.WaterState(pos, p, np.tile(Q, n), m, [L, L, L])
    oracle.water_forces(st, 0, prm)
    oracle.water_run(st, 0, 5000, prm, wp)
    V, Pi, _ = oracle.water_run(st, 5000, 100000, prm, wp)
    nb = 100
    bm = V.reshape(nb, -1).mean(1)
    se = bm.std(ddof=1) / math.sqrt(nb)
    assert abs(V.mean() - V0) < 4 * se + 0.002 * V0, (V.mean(), V0, se)
    # with the sites' kinetic energy in the pressure instead, <V> would sit near (3n + 1) kT / P
