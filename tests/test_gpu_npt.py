"""GPU parity of the Langevin NPT step (Sec. 3.2-3.3) with RBE k-space and real-space forces,
through the C ABI, against the oracle's step on the same inputs, noise and RBE batches.
Tolerances: FP64 path 1e-10 relative on positions, momenta, forces, box, p_V and virial after
a few steps; FP32-phase path 1e-5 relative RMS on forces and momenta."""
import math

import numpy as np
import pytest

import oracle
import paper_2110_14362_gb300 as rbe

from gpu_util import cuda_device

pytestmark = pytest.mark.gpu

SEED = 4242
ALPHA = 0.2
P = 100


def _system(n_side, density=0.1, jitter=0.3, seed=0):
    N = n_side ** 3
    L = (N / density) ** (1 / 3)
    rng = np.random.default_rng(seed)
    g = (np.arange(n_side) + 0.5) * (L / n_side)
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    pos = np.mod(pos + rng.uniform(-jitter, jitter, pos.shape), L)
    q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    m = np.full(N, 20.0)
    mom = rng.normal(size=(N, 3)) * np.sqrt(oracle.KB * 300 * 100 * m)[:, None]
    return pos, mom, q, m, np.array([L, L, L])


def _params(box, rc, **kw):
    V0 = float(np.prod(box))
    base = dict(dt=0.001, kT=oracle.KB * 300.0, P_ext=1.0 * oracle.BAR, gamma=10.0, gamma_V=2.0,
                M_V=oracle.piston_mass(0.5, 4.5e-5 / oracle.BAR, V0), rc=rc, qqr2e=oracle.QQR2E, lj_sigma=2.0,
                lj_eps=0.5, max_disp=0.05, kspace=1, real=1, noise=1, barostat=1)
    base.update(kw)
    dev = rbe.NptParams(**base)
    orc = oracle.npt_params(alpha=ALPHA, P=P, seed=SEED, **base)
    return dev, orc


def _run_both(n_side, rc, nsteps, precision, skin=0.0, **kw):
    pos, mom, q, m, box = _system(n_side)
    prm_d, prm_o = _params(box, rc, **kw)
    prm_d.skin = skin
    dev = cuda_device()
    with rbe.Context(box, ALPHA, P, SEED, precision) as ctx:
        rep = rbe.NptReplica(pos, mom, q, m, box, prm_d, dev, step=0)
        rep.init(ctx, batch=0)
        rep.step(ctx, nsteps)
        ctx.sync()
        r_d, p_d, F_d, L_d, cell = rep.state()
    st = oracle.NptState(pos, mom, q, m, box)
    oracle.npt_forces(st, 0, prm_o)
    for s in range(nsteps):
        oracle.npt_step(st, s, prm_o)
    return (r_d, p_d, F_d, L_d, cell), st


def _rel(a, b):
    return np.sqrt(np.mean((a - b) ** 2) / np.mean(b ** 2))


@pytest.mark.parametrize("n_side,rc", [(6, 6.0), (10, 7.0), (16, 7.0)])  # 2, 3 and 5 cells per axis
def test_npt_fp64_parity(n_side, rc):
    (r, p, F, L, cell), st = _run_both(n_side, rc, 3, rbe.RBE_FP64)
    assert np.allclose(L, st.L, rtol=1e-12, atol=0)
    d = r - st.r
    d -= st.L * np.round(d / st.L)
    assert np.abs(d).max() < 1e-10 * st.L[0]
    assert np.abs(p - st.p).max() < 1e-10 * np.abs(st.p).max()
    assert np.abs(F - st.F).max() < 1e-10 * np.abs(st.F).max()
    assert abs(cell[3] - st.pV.value) < 1e-10 * max(abs(st.pV.value), 1e-30) + 1e-20
    assert abs(cell[4] - st.W.value) < 1e-10 * abs(st.W.value)


def test_npt_fp32_phase_parity():
    (r, p, F, L, cell), st = _run_both(10, 7.0, 3, rbe.RBE_FP32_PHASE)
    assert np.allclose(L, st.L, rtol=1e-9)
    d = r - st.r
    d -= st.L * np.round(d / st.L)
    assert np.abs(d).max() < 1e-7
    assert _rel(F, st.F) < 1e-5
    assert _rel(p, st.p) < 1e-5
    assert abs(cell[4] - st.W.value) < 1e-5 * abs(st.W.value)


def test_npt_components_off():
    """k-space only, real space only, no barostat, no noise: each against the oracle."""
    for kw in (dict(real=0), dict(kspace=0), dict(barostat=0), dict(noise=0, gamma=0.0, gamma_V=0.0)):
        (r, p, F, L, cell), st = _run_both(8, 6.5, 2, rbe.RBE_FP64, **kw)
        assert np.abs(F - st.F).max() < 1e-10 * np.abs(st.F).max(), kw
        assert np.abs(p - st.p).max() < 1e-10 * np.abs(st.p).max(), kw


def test_npt_energy_conservation_device():
    """gamma = 0, no noise, real space only on a cold lattice: the extended energy K + U + P V
    + p_V^2 / 2M stays constant to O(dt^2) over 400 steps on the device."""
    pos, mom, q, m, box = _system(3, density=27 / 16.0 ** 3, jitter=0.1, seed=4)
    mom = mom * 0.1
    q = q * 0.3
    prm_d, _ = _params(box, 6.3, kspace=0, noise=0, gamma=0.0, gamma_V=0.0, max_disp=0.0, P_ext=100 * oracle.BAR)
    dev = cuda_device()
    H = []
    with rbe.Context(box, ALPHA, P, SEED, rbe.RBE_FP64) as ctx:
        rep = rbe.NptReplica(pos, mom, q, m, box, prm_d, dev)
        rep.init(ctx)
        for _ in range(40):
            rep.step(ctx, 10)
            c = rep.cell.cpu().numpy()
            V = c[0] * c[1] * c[2]
            H.append(0.5 * c[5] + c[8] + c[9] + prm_d.P_ext * V + c[3] ** 2 / (2 * prm_d.M_V))
    H = np.array(H)
    assert np.abs(H - H[0]).max() < 1e-5


@pytest.mark.parametrize("scale", [2.5, 0.7, float("inf"), float("nan")])
def test_npt_box_out_of_range_is_reported(scale):
    """A device box beyond the range rbe_npt_init prepared (edges above twice the initial
    ones, rc > l/2, or not finite) is flagged by the step and reported as an error status by
    the next synchronisation; the context stays usable."""
    pos, mom, q, m, box = _system(6)  # l = 12.9, rc = 6
    prm_d, _ = _params(box, 6.0)
    dev = cuda_device()
    with rbe.Context(box, ALPHA, P, SEED, rbe.RBE_FP32_PHASE) as ctx:
        rep = rbe.NptReplica(pos, mom, q, m, box, prm_d, dev)
        rep.init(ctx, batch=0)
        ctx.sync()
        rep.cell[:3] = float(box[0]) * scale
        rep.step(ctx, 1)
        with pytest.raises(rbe.RBEError) as e:
            ctx.sync()
        assert e.value.status in (rbe.RBE_ESTATE, rbe.RBE_ENONFINITE)
        # the context still works on a sane box
        rep2 = rbe.NptReplica(pos, mom, q, m, box, prm_d, dev)
        rep2.init(ctx, batch=0)
        rep2.step(ctx, 2)
        ctx.sync()
        assert np.isfinite(rep2.cell.cpu().numpy()[:11]).all()


@pytest.mark.parametrize("n_side,rc,skin", [(10, 7.0, 1.0), (16, 7.0, 1.0), (10, 7.0, 0.02), (6, 5.0, 1.2)])
def test_npt_neighbour_list_fp64_parity(n_side, rc, skin):
    """Real-space pairs from the neighbour list (rebuilt when the displacements and the box
    change require it; skin 0.02 A rebuilds every few steps) against the oracle's all-pairs
    nearest image after 6 steps: positions, momenta and forces at 1e-10 as for the cell
    search.  The virial trace is a small difference of large LJ and Coulomb terms, and the
    r^-12 terms amplify the 1e-11 relative position differences that 6 steps of dynamics
    leave: it is checked at 1e-9 here (a single evaluation meets 1e-10 in the 3-step tests)."""
    (r, p, F, L, cell), st = _run_both(n_side, rc, 6, rbe.RBE_FP64, skin=skin)
    assert np.allclose(L, st.L, rtol=1e-12, atol=0)
    d = r - st.r
    d -= st.L * np.round(d / st.L)
    assert np.abs(d).max() < 1e-10 * st.L[0]
    assert np.abs(p - st.p).max() < 1e-10 * np.abs(st.p).max()
    assert np.abs(F - st.F).max() < 1e-10 * np.abs(st.F).max()
    assert abs(cell[4] - st.W.value) < 1e-9 * abs(st.W.value)


def test_npt_neighbour_list_fp32_parity():
    (r, p, F, L, cell), st = _run_both(16, 7.0, 3, rbe.RBE_FP32_PHASE, skin=1.0)
    assert _rel(F, st.F) < 1e-5
    assert _rel(p, st.p) < 1e-5


@pytest.mark.parametrize("precision", [rbe.RBE_FP64, rbe.RBE_FP32_PHASE])
def test_npt_list_matches_cell_search(precision):
    """60 steps of the serving system with and without the list: the same pairs, so the
    trajectories agree to rounding (the order of the pair sums differs)."""
    from paper_2110_14362_gb300 import inputs
    pos, mom, q, m, box = inputs.npt_replica(3000, 5)
    base = _params(box, 7.0, qqr2e=oracle.QQR2E / 78.5)[0]
    dev = cuda_device()
    out = []
    for skin in (0.0, 0.8):
        base.skin = skin
        with rbe.Context(box, ALPHA, P, SEED, precision) as ctx:
            rep = rbe.NptReplica(pos, mom, q, m, box, base, dev)
            rep.init(ctx, batch=0)
            rep.step(ctx, 60)
            ctx.sync()
            out.append(rep.state())
    (r0, p0, F0, L0, c0), (r1, p1, F1, L1, c1) = out
    tol = 1e-9 if precision == rbe.RBE_FP64 else 1e-4
    assert np.allclose(L1, L0, rtol=tol, atol=0)
    d = r1 - r0
    d -= L0 * np.round(d / L0)
    assert np.abs(d).max() < tol * L0[0]
    assert _rel(p1, p0) < tol
