"""Pins of the oracle's Langevin NPT step (Sec. 3.2-3.3) and its real-space forces, against
facts fixed by the equations: derivatives of the potential, exact free flight, the
Ornstein--Uhlenbeck law, the isobaric ideal gas, the virial theorem, and conservation of the
extended energy without friction and noise."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle

KT = oracle.KB * 300.0


def _lattice(n_side, L, jitter, seed):
    rng = np.random.default_rng(seed)
    g = (np.arange(n_side) + 0.5) * (L / n_side)
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    pos = pos + rng.uniform(-jitter, jitter, pos.shape)
    q = np.where(np.arange(pos.shape[0]) % 2 == 0, 1.0, -1.0)
    return np.mod(pos, L), q


def test_pair_real_force_and_virial_are_derivatives():
    box = np.array([15.0, 16.0, 17.0])
    pos, q = _lattice(3, 15.0, 1.5, 0)
    args = (0.2, 7.0, oracle.QQR2E, 2.0, 0.5)
    F, W, Ec, El = oracle.pair_real(pos, q, box, *args)
    U = lambda x, b=box: sum(oracle.pair_real(x, q, b, *args)[2:])
    h = 1e-6
    for i, t in [(0, 0), (5, 1), (11, 2)]:
        xp = pos.copy(); xp[i, t] += h
        xm = pos.copy(); xm[i, t] -= h
        assert abs(F[i, t] + (U(xp) - U(xm)) / (2 * h)) < 1e-6 * max(1.0, abs(F[i, t]))
    s = pos / box
    for a in range(3):
        e = np.ones(3); e[a] += 1e-6
        e2 = np.ones(3); e2[a] -= 1e-6
        d = -(U(s * box * e, box * e) - U(s * box * e2, box * e2)) / 2e-6
        assert abs(W[a, a] - d) < 1e-6 * max(1.0, abs(d))
    assert np.abs(W - W.T).max() < 1e-10 * np.abs(W).max()
    assert np.abs(F.sum(0)).max() < 1e-9 * np.abs(F).sum()
    # with unit Coulomb constant and no LJ it is the Ewald real-space sum
    F0, W0, E0 = oracle.ewald_real(pos, q, box, 0.2, 7.0)
    F1, W1, Ec1, _ = oracle.pair_real(pos, q, box, 0.2, 7.0, 1.0, 2.0, 0.0)
    assert np.allclose(F1, F0, rtol=1e-12, atol=1e-14) and abs(Ec1 - E0) < 1e-12 * abs(E0)


def test_free_flight_is_exact():
    rng = np.random.default_rng(1)
    N, L = 50, 20.0
    r = rng.random((N, 3)) * L
    m = rng.uniform(10, 40, N)
    p = rng.normal(size=(N, 3)) * np.sqrt(KT * 100 * m)[:, None]
    st = oracle.NptState(r, p, np.zeros(N), m, [L, L, L])
    prm = oracle.npt_params(kspace=0, real=0, noise=0, gamma=0.0, barostat=0, dt=0.002)
    oracle.npt_forces(st, 0, prm)
    for s in range(25):
        oracle.npt_step(st, s, prm)
    expect = np.mod(r + p / m[:, None] * 25 * 0.002, L)
    d = st.r - expect
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-10
    assert np.array_equal(st.p, p)


def test_ornstein_uhlenbeck_step():
    """O: p <- e^{-g dt} p + sqrt(kT m (1 - e^{-2 g dt})) R (Sec. 3.3), R standard normal."""
    N = 40000
    m = np.full(N, 20.0)
    p0 = np.random.default_rng(2).normal(size=(N, 3)) * 30.0
    st = oracle.NptState(np.zeros((N, 3)), p0, np.zeros(N), m, [50.0, 50.0, 50.0])
    g, dt = 10.0, 0.001
    prm = oracle.npt_params(kspace=0, real=0, noise=1, gamma=g, barostat=0, dt=dt, seed=77)
    oracle.npt_step(st, 5, prm)
    a = math.exp(-g * dt)
    sig = math.sqrt(KT * 100 * 20.0 * (1 - a * a))
    z = (st.p - a * p0) / sig
    assert stats.kstest(z.ravel(), "norm").pvalue > 1e-3
    assert abs(z.mean()) < 5 / math.sqrt(z.size) and abs(z.var() - 1) < 5 * math.sqrt(2 / z.size)
    # without noise the momenta decay exactly
    st2 = oracle.NptState(np.zeros((N, 3)), p0, np.zeros(N), m, [50.0, 50.0, 50.0])
    prm.noise = 0
    oracle.npt_step(st2, 5, prm)
    assert np.allclose(st2.p, a * p0, rtol=1e-14)


def test_box_muller_normals_law():
    z = np.concatenate([oracle.npt_normals(3, 1, 9, i) for i in range(20000)])
    assert stats.kstest(z, "norm").pvalue > 1e-3


@pytest.mark.slow
def test_isobaric_ideal_gas():
    """U = 0: the stationary law in V is proportional to V^N exp(-P V / kT), so <V> = (N+1) kT / P;
    the pressure virial theorem gives <P_ins> = P (Sec. 3.1)."""
    N = 16
    V0 = 1000.0
    P = (N + 1) * KT / V0
    rng = np.random.default_rng(3)
    L = V0 ** (1 / 3)
    m = np.full(N, 20.0)
    p = rng.normal(size=(N, 3)) * np.sqrt(KT * 100 * m)[:, None]
    st = oracle.NptState(rng.random((N, 3)) * L, p, np.zeros(N), m, [L, L, L])
    M = oracle.piston_mass(0.2, 1.0 / P, V0)
    prm = oracle.npt_params(kspace=0, real=0, noise=1, gamma=5.0, gamma_V=20.0, M_V=M, P_ext=P, dt=0.002, seed=11)
    oracle.npt_forces(st, 0, prm)
    oracle.npt_run(st, 0, 5000, prm)
    V, Pi, _ = oracle.npt_run(st, 5000, 100000, prm)
    # batch means for the standard error
    nb = 100
    bm = V.reshape(nb, -1).mean(1)
    se = bm.std(ddof=1) / math.sqrt(nb)
    assert abs(V.mean() - V0) < 4 * se + 0.002 * V0, (V.mean(), V0, se)
    pb = Pi.reshape(nb, -1).mean(1)
    assert abs(Pi.mean() - P) < 4 * pb.std(ddof=1) / math.sqrt(nb) + 0.003 * P


def test_extended_energy_conserved_without_friction():
    """gamma = gamma_V = 0, no noise: K + U + P V + p_V^2 / (2M) is conserved up to O(dt^2).
    A cold lattice (neighbours at 5.3 and 7.5 A, cutoff 6.3 A) keeps every pair on one side of
    the cutoff, where the plain truncated potential would otherwise jump."""
    pos, q = _lattice(3, 16.0, 0.1, 4)
    N = pos.shape[0]
    m = np.full(N, 20.0)
    rng = np.random.default_rng(5)
    p0 = rng.normal(size=(N, 3)) * np.sqrt(KT * 100 * m)[:, None] * 0.1
    V0 = 16.0 ** 3
    drift = []
    for dt in (0.001, 0.0005):
        st = oracle.NptState(pos, p0, q * 0.3, m, [16.0] * 3, pV=0.0)
        prm = oracle.npt_params(kspace=0, real=1, noise=0, gamma=0.0, gamma_V=0.0,
                                M_V=oracle.piston_mass(0.5, 4.5e-5 / oracle.BAR, V0), P_ext=100 * oracle.BAR,
                                dt=dt, rc=6.3)
        oracle.npt_forces(st, 0, prm)
        n = int(round(0.4 / dt))
        V, Pi, H = oracle.npt_run(st, 0, n, prm)
        drift.append(np.abs(H - H[0]).max())
        assert V.max() / V.min() > 1.0001  # the cell does move
    assert drift[0] < 1e-5
    assert drift[1] < drift[0] / 3.5  # second order in dt
