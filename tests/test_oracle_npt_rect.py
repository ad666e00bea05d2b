"""Pins of the oracle's rectangular-cell NPT step (appendix: the rectangular cell with
anisotropic fluctuation, and the semi-isotropic constant surface-tension case), against facts
the equations of motion fix: conservation of the extended energy without friction and noise
(second order in dt), time reversibility of the deterministic splitting, the per-axis
decoupling of an ideal gas, equipartition of the cell momenta, and the reduction of the
semi-isotropic cell with a frozen area to the anisotropic cell with two frozen axes."""
import math

import numpy as np
import pytest

import oracle

KT = oracle.KB * 300.0


def _lattice(n_side, L, jitter, seed):
    rng = np.random.default_rng(seed)
    g = (np.arange(n_side) + 0.5) * (L / n_side)
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    pos = pos + rng.uniform(-jitter, jitter, pos.shape)
    q = np.where(np.arange(pos.shape[0]) % 2 == 0, 1.0, -1.0)
    return np.mod(pos, L), q


def _cold_system(seed=5):
    """27 particles on a jittered 16 A lattice (neighbours at 5.3 and 7.5 A, cutoff 6.3 A: no
    pair crosses the cutoff, where the truncated potential would jump)."""
    pos, q = _lattice(3, 16.0, 0.1, 4)
    N = pos.shape[0]
    m = np.full(N, 20.0)
    rng = np.random.default_rng(seed)
    p0 = rng.normal(size=(N, 3)) * np.sqrt(KT * 100 * m)[:, None] * 0.1
    return pos, p0, q * 0.3, m


def _energy_drift(mode, dt, pc0, gamma0=0.0):
    pos, p0, q, m = _cold_system()
    box = [16.0] * 3
    M = oracle.piston_masses_rect(mode, 0.5, 4.5e-5 / oracle.BAR, box)
    st = oracle.NptRectState(pos, p0, q, m, box, pc=pc0)
    prm = oracle.npt_params(kspace=0, real=1, noise=0, gamma=0.0, gamma_V=0.0, P_ext=100 * oracle.BAR, dt=dt,
                            rc=6.3, barostat=mode, M_cell=M, gamma0=gamma0)
    oracle.npt_forces_rect(st, 0, prm)
    n = int(round(0.4 / dt))
    L, Pd, H = oracle.npt_run_rect(st, 0, n, prm)
    return np.abs(H - H[0]).max(), L


def test_anisotropic_extended_energy_conserved():
    """gamma = gamma_V = 0, no noise: K + U + P V + sum_j pc_j^2/(2 M_j) is conserved up to O(dt^2);
    the three edges move differently."""
    pc0 = (0.05, 0.0, -0.08)
    d1, L1 = _energy_drift(2, 0.001, pc0)
    d2, _ = _energy_drift(2, 0.0005, pc0)
    span = L1.max(0) - L1.min(0)
    assert np.all(span > 1e-3)  # every edge moves
    assert np.abs(np.diff(L1[-1])).min() > 1e-4  # and the box is no longer cubic
    assert d1 < 1e-4
    assert d2 < d1 / 3.5  # second order in dt


def test_semi_isotropic_extended_energy_conserved():
    """Semi-isotropic with surface tension: K + U + P A L - gamma0 A + (p^A)^2/(2M_A) + (p^L)^2/(2M_L)
    is conserved up to O(dt^2), and l_x = l_y holds exactly."""
    pc0 = (0.02, 0.0, -0.05)
    g0 = 2e-3  # kJ/mol/A^2: g0 times the area change is far above the drift bound
    d1, L1 = _energy_drift(3, 0.001, pc0, gamma0=g0)
    d2, _ = _energy_drift(3, 0.0005, pc0, gamma0=g0)
    assert np.array_equal(L1[:, 0], L1[:, 1])
    A = L1[:, 0] * L1[:, 1]
    assert g0 * (A.max() - A.min()) > 100 * d1  # the surface term matters at this tolerance
    assert (L1[:, 2].max() - L1[:, 2].min()) > 1e-3
    assert d1 < 1e-4
    assert d2 < d1 / 3.5
    # with the surface term dropped from the force, the same H is no longer conserved
    pos, p0, q, m = _cold_system()
    M = oracle.piston_masses_rect(3, 0.5, 4.5e-5 / oracle.BAR, [16.0] * 3)
    st = oracle.NptRectState(pos, p0, q, m, [16.0] * 3, pc=pc0)
    prm = oracle.npt_params(kspace=0, real=1, noise=0, gamma=0.0, gamma_V=0.0, P_ext=100 * oracle.BAR,
                            dt=0.001, rc=6.3, barostat=3, M_cell=M, gamma0=0.0)
    oracle.npt_forces_rect(st, 0, prm)
    L0, _, H0 = oracle.npt_run_rect(st, 0, 400, prm)
    H_with = H0 - g0 * L0[:, 0] * L0[:, 1]  # the energy of the g0 ensemble along a g0 = 0 path
    assert np.abs(H_with - H_with[0]).max() > 10 * d1


@pytest.mark.parametrize("mode", [2, 3])
def test_deterministic_step_is_reversible(mode):
    """Without friction and noise the splitting is a symmetric composition of exact flows, so
    flipping every momentum (particles and cell) retraces the path."""
    pos, p0, q, m = _cold_system(7)
    box = [16.0] * 3
    M = oracle.piston_masses_rect(mode, 0.5, 4.5e-5 / oracle.BAR, box)
    st = oracle.NptRectState(pos, p0 * 3, q, m, box, pc=(0.03, 0.0 if mode == 3 else 0.01, -0.02))
    prm = oracle.npt_params(kspace=0, real=1, noise=0, gamma=0.0, gamma_V=0.0, P_ext=100 * oracle.BAR, dt=0.002,
                            rc=6.3, barostat=mode, M_cell=M, gamma0=1e-3)
    oracle.npt_forces_rect(st, 0, prm)
    r0, L0 = st.r.copy(), st.L.copy()
    oracle.npt_run_rect(st, 0, 60, prm)
    assert np.abs(st.L - L0).max() > 1e-3
    st.p *= -1
    st.pc *= -1
    oracle.npt_run_rect(st, 60, 60, prm)
    d = st.r - r0
    d -= st.L * np.round(d / st.L)
    assert np.abs(d).max() < 1e-9
    assert np.abs(st.L - L0).max() < 1e-10
    assert np.abs(st.p + p0 * 3).max() < 1e-8 * np.abs(p0 * 3).max()


def test_uniaxial_ideal_gas_moves_one_edge():
    """No forces, P = 0, momenta only along x: the pressure on y and z is zero, so their cell
    momenta, edges and coordinates stay exactly as they were; x and its piston exchange energy
    (sum p_x^2/(2m) + pc_x^2/(2 M_x) conserved to O(dt^2))."""
    rng = np.random.default_rng(8)
    N, L = 40, 30.0
    r = rng.random((N, 3)) * L
    m = rng.uniform(10, 40, N)
    p = np.zeros((N, 3))
    p[:, 0] = rng.normal(size=N) * np.sqrt(KT * 100 * m)
    M = (50.0, 70.0, 90.0)
    drift = []
    for dt in (0.002, 0.001):
        st = oracle.NptRectState(r, p, np.zeros(N), m, [L, L, L])
        prm = oracle.npt_params(kspace=0, real=0, noise=0, gamma=0.0, gamma_V=0.0, P_ext=0.0, dt=dt, barostat=2,
                                M_cell=M)
        oracle.npt_forces_rect(st, 0, prm)
        Lh, Pd, H = oracle.npt_run_rect(st, 0, int(round(1.0 / dt)), prm)
        assert np.all(Lh[:, 1] == L) and np.all(Lh[:, 2] == L)
        assert st.pc[1] == 0.0 and st.pc[2] == 0.0
        assert np.array_equal(st.r[:, 1:], r[:, 1:]) and np.all(st.p[:, 1:] == 0.0)
        assert Lh[:, 0].max() - L > 0.02  # pushed out by the gas: N kT / (l M) ~ 0.07 A/ps^2 for 1 ps
        assert np.all(Pd[:, 1:] == 0.0) and np.all(Pd[:, 0] > 0.0)
        drift.append(np.abs(H - H[0]).max() / abs(H[0]))
    assert drift[0] < 1e-3 and drift[1] < drift[0] / 3.5


@pytest.mark.parametrize("mode", [2, 3])
def test_cell_momenta_equipartition(mode):
    """One particle at rest, no forces, P = 0: the cell force vanishes and each cell momentum is an
    exact Ornstein--Uhlenbeck process whose stationary variance is kT M_j (the fluctuation-dissipation
    balance of O^p).  The masses differ by 10x per slot, so a slot given another slot's mass or
    normal fails."""
    M = (1e4, 1e5, 1e6) if mode == 2 else (1e4, 0.0, 1e6)
    st = oracle.NptRectState(np.full((1, 3), 50.0), np.zeros((1, 3)), np.zeros(1), np.full(1, 20.0),
                             [100.0] * 3)
    prm = oracle.npt_params(kspace=0, real=0, noise=1, gamma=0.0, gamma_V=100.0, P_ext=0.0, dt=0.002,
                            barostat=mode, M_cell=M, seed=21)
    oracle.npt_forces_rect(st, 0, prm)
    oracle.npt_run_rect(st, 0, 50, prm)
    n, samples = 20000, []
    for s in range(n):
        oracle.npt_step_rect(st, 50 + s, prm)
        samples.append(st.pc.copy())
    pc = np.array(samples)
    assert np.all(st.p == 0.0)
    # exp(-gamma_V dt) = e^-0.2 per step: about 10 steps between independent samples
    neff = n / 10.0
    for j in range(3):
        if M[j] == 0.0:
            assert np.all(pc[:, j] == 0.0)
            continue
        v = np.mean(pc[:, j] ** 2) / (KT * M[j])
        assert abs(v - 1.0) < 5 * math.sqrt(2.0 / neff), (j, v)
    if mode == 2:
        c = np.corrcoef(pc.T)
        assert np.abs(c[np.triu_indices(3, 1)]).max() < 5 / math.sqrt(neff)


def test_semi_with_frozen_area_is_anisotropic_with_frozen_xy():
    """With M_A (and M_x = M_y) so large that the x and y edges cannot move, the semi-isotropic L
    equation A ((P_ins)_zz - P) equals the anisotropic z equation V ((P_ins)_zz - P)/l_z, and slot 2 of
    both uses the same cell normal: the two runs agree (noise, RBE k-space and real space on)."""
    pos, q = _lattice(3, 16.0, 0.4, 9)
    N = pos.shape[0]
    m = np.full(N, 20.0)
    rng = np.random.default_rng(10)
    p0 = rng.normal(size=(N, 3)) * np.sqrt(KT * 100 * m)[:, None]
    box = [16.0, 16.0, 17.0]
    ML = oracle.piston_masses_rect(3, 0.5, 4.5e-5 / oracle.BAR, box)[2]
    out = []
    for mode, M in ((3, (1e300, 0.0, ML)), (2, (1e300, 1e300, ML))):
        st = oracle.NptRectState(pos, p0, q * 0.5, m, box, pc=(0.0, 0.0, 0.02))
        prm = oracle.npt_params(barostat=mode, M_cell=M, P_ext=50 * oracle.BAR, rc=6.0, P=60, seed=3, dt=0.002)
        oracle.npt_forces_rect(st, 0, prm)
        Lh, _, _ = oracle.npt_run_rect(st, 0, 20, prm)
        out.append((st, Lh))
    (a, La), (b, Lb) = out
    assert np.all(La[:, :2] == 16.0) and np.all(Lb[:, :2] == 16.0)
    assert La[:, 2].max() - La[:, 2].min() > 1e-4
    assert np.abs(La[:, 2] - Lb[:, 2]).max() < 1e-12 * 17.0
    assert abs(a.pc[2] - b.pc[2]) < 1e-9 * abs(a.pc[2])
    assert np.abs(a.r - b.r).max() < 1e-10 and np.abs(a.p - b.p).max() < 1e-9 * np.abs(a.p).max()


def test_rect_rejects_bad_parameters():
    st = oracle.NptRectState(np.zeros((2, 3)), np.zeros((2, 3)), np.zeros(2), np.ones(2), [10.0, 11.0, 12.0])
    prm = oracle.npt_params(kspace=0, real=0, barostat=3, M_cell=(1.0, 0.0, 1.0))
    with pytest.raises(RuntimeError):
        oracle.npt_step_rect(st, 0, prm)  # the semi-isotropic cell needs l_x = l_y
    prm = oracle.npt_params(kspace=0, real=0, barostat=2, M_cell=(1.0, 0.0, 1.0))
    with pytest.raises(RuntimeError):
        oracle.npt_step_rect(st, 0, prm)  # every anisotropic mass must be positive
    prm = oracle.npt_params(kspace=0, real=0, barostat=1)
    with pytest.raises(RuntimeError):
        oracle.npt_step_rect(st, 0, prm)
    iso = oracle.NptState(np.zeros((2, 3)), np.zeros((2, 3)), np.zeros(2), np.ones(2), [10.0] * 3)
    with pytest.raises(RuntimeError):
        oracle.npt_step(iso, 0, oracle.npt_params(kspace=0, real=0, barostat=2))


@pytest.mark.parametrize("mode", [1, 2])
def test_cap_leaves_the_dilation_alone(mode):
    """The displacement cap holds the peculiar motion (p/m) only: particles at rest in a fast
    expanding cell follow its dilation whatever the cap, so a run with a tiny cap equals the run
    without one, and the particles far from the origin keep their scaled coordinates."""
    rng = np.random.default_rng(12)
    N, L = 30, 60.0
    r = rng.random((N, 3)) * L
    out = []
    for cap in (0.0, 1e-6):
        kw = dict(kspace=0, real=0, noise=0, gamma=0.0, gamma_V=0.0, P_ext=0.0, dt=0.002, max_disp=cap,
                  barostat=mode)
        if mode == 1:
            st = oracle.NptState(r, np.zeros((N, 3)), np.zeros(N), np.full(N, 20.0), [L] * 3, pV=270.0)
            prm = oracle.npt_params(M_V=1e-3, **kw)
            oracle.npt_forces(st, 0, prm)
            oracle.npt_run(st, 0, 20, prm)
        else:
            st = oracle.NptRectState(r, np.zeros((N, 3)), np.zeros(N), np.full(N, 20.0), [L] * 3, pc=(50.0, 40.0, 60.0))
            prm = oracle.npt_params(M_cell=(1.0, 1.0, 1.0), **kw)
            oracle.npt_forces_rect(st, 0, prm)
            oracle.npt_run_rect(st, 0, 20, prm)
        out.append((st.r.copy(), st.L.copy()))
    (r0, L0), (r1, L1) = out
    assert np.all(L0 - L > 0.5)  # the cell grows fast: far particles move ~ 1 A per sub-step
    assert np.array_equal(r0, r1) and np.array_equal(L0, L1)
    assert np.abs(r0 / L0 - r / L).max() < 1e-3
