"""Pins of the oracle's fully flexible cell Langevin NPT step (App. A, fully flexible cells): with
chi = 0 and the off-diagonal cell entries frozen it is the anisotropic rectangular step (noise,
RBE and real space on); without friction and noise the extended energy K + U + P V + chi kT ln V +
sum (p^h)^2/2M is conserved to O(dt^2) with all nine cell entries moving (and the chi term is
needed for that); the deterministic splitting is time reversible."""
import numpy as np
import pytest

import oracle

KT = oracle.KB * 300.0


def _rocksalt(counts, density=0.1, jitter=0.3, seed=0):
    a = density ** (-1 / 3)
    box = a * np.asarray(counts, dtype=np.float64)
    rng = np.random.default_rng(seed)
    idx = np.stack(np.meshgrid(*[np.arange(n) for n in counts], indexing="ij"), -1).reshape(-1, 3)
    pos = np.mod((idx + 0.5) * a + rng.uniform(-jitter, jitter, idx.shape), box)
    q = np.where(idx.sum(1) % 2 == 0, 1.0, -1.0)
    m = np.full(len(q), 20.0)
    mom = rng.normal(size=(len(q), 3)) * np.sqrt(KT * 100 * m)[:, None]
    return pos, mom, q, m, box


def test_frozen_shear_without_chi_is_the_rectangular_step():
    pos, mom, q, m, box = _rocksalt((5, 5, 6))
    Md = oracle.piston_masses_rect(2, 0.5, 4.5e-5 / oracle.BAR, box)
    rates = (0.5, -0.3, 0.2)
    pc = tuple(Md[j] * rates[j] for j in range(3))
    common = dict(dt=0.001, kT=KT, P_ext=oracle.BAR, gamma=10.0, alpha=0.2, rc=5.0, qqr2e=oracle.QQR2E / 78.5,
                  lj_sigma=2.0, lj_eps=0.5, max_disp=0.05, P=60, kspace=1, real=1, noise=1, seed=19)
    rect = oracle.npt_params(barostat=2, M_cell=Md, gamma_V=2.0, M_V=0.0, **common)
    st_r = oracle.NptRectState(pos, mom, q, m, box, pc=pc)
    oracle.npt_forces_rect(st_r, 0, rect)
    M = np.full((3, 3), 1e300)
    M[np.diag_indices(3)] = Md
    flex = oracle.flex_params(gamma_h=2.0, M=M, chi=0.0, **common)
    st_f = oracle.FlexState(pos, mom, q, m, np.diag(box), ph=np.diag(pc), P=60)
    oracle.flex_forces(st_f, 0, flex)
    assert np.abs(st_f.F - st_r.F).max() < 1e-12 * np.abs(st_r.F).max()
    assert np.abs(np.diag(st_f.W) - st_r.Wd).max() < 1e-12 * np.abs(st_r.Wd).max()
    for s in range(8):
        oracle.npt_step_rect(st_r, s, rect)
        oracle.flex_step(st_f, s, flex)
    assert np.abs(np.diag(st_f.h) - st_r.L).max() < 1e-12 * st_r.L.max()
    assert np.abs(st_f.h - np.diag(np.diag(st_f.h))).max() < 1e-100
    d = st_f.r - st_r.r
    d -= st_r.L * np.round(d / st_r.L)
    assert np.abs(d).max() < 1e-10 * st_r.L.max()
    assert np.abs(st_f.p - st_r.p).max() < 1e-10 * np.abs(st_r.p).max()
    assert np.abs(np.diag(st_f.ph) - st_r.pc).max() < 1e-10 * np.abs(st_r.pc).max()


def _cold_sheared(seed=5):
    """27 particles on a jittered lattice in a sheared 16 A cell: nearest neighbours near 5.3 A, the
    next shell beyond 7 A, the cutoff 6.2 A between them, so that over the few per cent of volume
    change below no pair crosses the cutoff (where the truncated potential jumps)."""
    rng = np.random.default_rng(seed)
    h = np.array([[16.0, 1.5, -1.0], [0.0, 16.0, 2.0], [0.0, 0.0, 16.0]])
    u = (np.arange(3) + 0.5) / 3
    s = np.stack(np.meshgrid(u, u, u, indexing="ij"), -1).reshape(-1, 3) + rng.uniform(-0.004, 0.004, (27, 3))
    q = np.where(np.arange(27) % 2 == 0, 0.3, -0.3)
    m = np.full(27, 20.0)
    p = rng.normal(size=(27, 3)) * np.sqrt(KT * 100 * m)[:, None] * 0.1
    return s @ h.T, p, q, m, h


def _flex_energy_drift(dt, chi=2.0, steps_ps=0.4):
    pos, p, q, m, h = _cold_sheared()
    prm = oracle.flex_params(dt=dt, gamma=0.0, gamma_h=0.0, noise=0, kspace=0, real=1, rc=6.2, P_ext=oracle.BAR,
                             M=np.full((3, 3), 5.0), chi=chi, lj_sigma=2.0, lj_eps=0.5)
    ph = np.array([[2.0, 1.0, -1.5], [1.2, -2.0, 1.0], [-1.0, 1.5, 1.8]])
    st = oracle.FlexState(pos, p, q, m, h, ph=ph)
    oracle.flex_forces(st, 0, prm)
    hs, Ps, H = oracle.flex_run(st, 0, int(round(steps_ps / dt)), prm)
    return np.abs(H - H[0]).max(), hs, H, st


def test_extended_energy_conserved_with_all_cell_entries_moving():
    d1, hs, H, _ = _flex_energy_drift(0.001)
    d2, _, _, _ = _flex_energy_drift(0.0005)
    span = hs.max(0) - hs.min(0)
    assert np.all(span > 0.05), span  # all nine entries move (including the rotation-like ones)
    assert d1 < 1e-6, d1
    assert d2 < d1 / 3.5, (d1, d2)  # second order: halving dt quarters the drift


def test_chi_term_is_part_of_the_conserved_energy():
    """Along the chi = 2 trajectory the energy without chi kT ln V is not conserved at the same
    tolerance (the volume changes), so the cell force and H carry the same chi term."""
    d1, hs, H, _ = _flex_energy_drift(0.001)
    V = np.array([np.linalg.det(x) for x in hs])
    H_no_chi = H - 2.0 * KT * np.log(V)
    assert np.abs(H_no_chi - H_no_chi[0]).max() > 1e4 * d1
    assert V.max() / V.min() > 1.004


@pytest.mark.parametrize("chi", [0.0, 2.0])
def test_flexible_step_is_reversible(chi):
    pos, p, q, m, h = _cold_sheared(7)
    prm = oracle.flex_params(dt=0.002, gamma=0.0, gamma_h=0.0, noise=0, kspace=0, real=1, rc=6.0,
                             P_ext=100 * oracle.BAR, M=np.full((3, 3), 0.05), chi=chi)
    st = oracle.FlexState(pos, p * 3, q, m, h, ph=np.array([[0.02, 0.01, 0], [0, -0.02, 0.01], [0.01, 0, 0.02]]))
    oracle.flex_forces(st, 0, prm)
    r0, h0 = st.r.copy(), st.h.copy()
    oracle.flex_run(st, 0, 50, prm)
    assert np.abs(st.h - h0).max() > 1e-3
    st.p *= -1
    st.ph *= -1
    oracle.flex_run(st, 50, 50, prm)
    assert np.abs(st.h - h0).max() < 1e-10
    s = (st.r - r0) @ np.linalg.inv(h0).T
    s -= np.round(s)
    assert np.abs(s @ h0.T).max() < 1e-9
    assert np.abs(st.p + p * 3).max() < 1e-8 * np.abs(p * 3).max()


def test_free_particles_keep_the_canonical_momentum():
    """Without forces the momentum conjugate to the scaled coordinates, pi = h^T p, is constant
    along the flexible-cell flow (pi' = h^T F); the splitting keeps it to O(dt^2).  This fixes the
    transpose in dp/dt = -A^T p, which the energy (p^T A p = p^T A^T p) does not see."""
    pos, p, q, m, h = _cold_sheared(3)
    p = p * 30
    out = []
    for dt in (0.002, 0.001):
        prm = oracle.flex_params(dt=dt, gamma=0.0, gamma_h=0.0, noise=0, kspace=0, real=0, P_ext=oracle.BAR,
                                 M=np.full((3, 3), 5.0), chi=2.0)
        st = oracle.FlexState(pos, p, q, m, h, ph=np.array([[2.0, 1.0, -1.5], [1.2, -2.0, 1.0], [-1.0, 1.5, 1.8]]))
        oracle.flex_forces(st, 0, prm)
        pi0 = p @ h
        oracle.flex_run(st, 0, int(round(0.4 / dt)), prm)
        assert np.abs(st.h - h).max() > 0.1
        out.append(np.abs(st.p @ st.h - pi0).max() / np.abs(pi0).max())
    assert out[0] < 1e-5 and out[1] < out[0] / 3.5, out


@pytest.mark.slow
def test_cell_momenta_equipartition():
    """Ideal gas (no forces) with friction and noise on every cell entry: at stationarity each of the
    nine cell momenta is Gaussian with <(p^h_te)^2> = kT M_te (the extended energy is separable in
    p^h), whatever the cell does; masses 10x apart pin the amplitude and the mass of every entry's
    noise, the off-diagonal ones included."""
    rng = np.random.default_rng(12)
    n = 8
    L = 20.0
    h = np.diag([L, L, L])
    M = np.array([[1.0, 2.0, 4.0], [6.0, 10.0, 1.5], [3.0, 0.8, 5.0]])
    pos = rng.random((n, 3)) * L
    p = rng.normal(size=(n, 3)) * np.sqrt(KT * 100 * 20.0)
    prm = oracle.flex_params(dt=0.002, gamma=5.0, gamma_h=20.0, noise=1, kspace=0, real=0, M=M, chi=2.0,
                             P_ext=(n + 1) * KT / L ** 3, seed=31)
    st = oracle.FlexState(pos, p, np.zeros(n), np.full(n, 20.0), h)
    oracle.flex_forces(st, 0, prm)
    oracle.flex_run(st, 0, 2000, prm)
    acc = np.zeros((3, 3))
    nblk, per = 40, 1000
    blocks = np.zeros((nblk, 3, 3))
    for b in range(nblk):
        for k in range(per):
            oracle.flex_step(st, 2000 + b * per + k, prm)
            blocks[b] += st.ph ** 2
        blocks[b] /= per * KT * M
    mean = blocks.mean(0)
    se = blocks.std(0, ddof=1) / np.sqrt(nblk)
    assert np.all(np.abs(mean - 1.0) < 4 * se + 0.03), (mean, se)
