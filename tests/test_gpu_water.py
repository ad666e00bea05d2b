"""GPU parity of the rigid 3-site water Langevin NPT step through the C ABI against the oracle's
water step (same inputs, noise and RBE batches): FP64 1e-10 on sites, momenta, forces, box,
piston momentum, molecular virial and energies after a few steps, each component switched off in
turn; FP32-phase k-space at 1e-5; the constraints held on the device; the extended energy
conserved on the device like the oracle's; bad input rejected."""
import math

import numpy as np
import pytest

import oracle
import paper_2110_14362_gb300 as rbe

from gpu_util import cuda_device

pytestmark = pytest.mark.gpu

SEED = 4242
ALPHA = 0.25
P = 100
KT = oracle.KB * 300.0
Q = np.array([-0.8476, 0.4238, 0.4238])
MASS = np.array([15.9994, 1.008, 1.008])
HALF = math.radians(109.47) / 2
LOCAL = np.array([[0.0, 0.0, 0.0], [math.sin(HALF), 0.0, math.cos(HALF)], [-math.sin(HALF), 0.0, math.cos(HALF)]])


def _waters(n_side, L, seed, jitter=0.3, thermal=1.0):
    """n_side^3 molecules at random orientations on a jittered lattice of a cubic box L, each
    moved by the lattice vector that brings its oxygen into the box (whole molecules)."""
    rng = np.random.default_rng(seed)
    g = (np.arange(n_side) + 0.5) * (L / n_side)
    c = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + rng.uniform(-jitter, jitter, (n_side ** 3, 3))
    qt = rng.normal(size=(len(c), 4))
    qt /= np.linalg.norm(qt, axis=1, keepdims=True)
    w, x, y, z = qt.T
    R = np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
                  np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
                  np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1)], 1)
    mol = c[:, None, :] + np.einsum("nij,sj->nsi", R, LOCAL)
    mol -= L * np.floor(mol[:, :1, :] / L)
    n = len(c)
    m = np.tile(MASS, n)
    p = rng.normal(size=(3 * n, 3)) * np.sqrt(KT * 100 * m)[:, None] * thermal
    return mol.reshape(-1, 3), p, np.tile(Q, n), m, np.array([L, L, L])


def _box_1gcc(n_mol):
    return (n_mol * 18.01528 / (0.602214076 * 1.0)) ** (1 / 3)


def _params(L, rc, **kw):
    base = dict(dt=0.001, kT=KT, P_ext=oracle.BAR, gamma=10.0, gamma_V=2.0,
                M_V=oracle.piston_mass(0.5, 4.5e-5 / oracle.BAR, L ** 3), rc=rc, qqr2e=oracle.QQR2E,
                lj_sigma=3.166, lj_eps=0.650, max_disp=0.0, kspace=1, real=1, noise=1, barostat=1)
    base.update(kw)
    skin = base.pop("skin", 0.0)
    return rbe.NptParams(skin=skin, **base), oracle.npt_params(alpha=ALPHA, P=P, seed=SEED, **base)


def _run_both(n_side, rc, nsteps, precision, pV=0.0, **kw):
    L = _box_1gcc(n_side ** 3)
    pos, mom, q, m, box = _waters(n_side, L, n_side)
    prm_d, prm_o = _params(L, rc, **kw)
    dev = cuda_device()
    with rbe.Context(box, ALPHA, P, SEED, precision) as ctx:
        rep = rbe.WaterReplica(pos, mom, q, m, box, prm_d, dev, step=0, pV=pV)
        rep.init(ctx, batch=0)
        rep.step(ctx, nsteps)
        ctx.sync()
        got = rep.state()
    st = oracle.WaterState(pos, mom, q, m, box, pV=pV)
    E = oracle.water_forces(st, 0, prm_o)
    for s in range(nsteps):
        E = oracle.water_step(st, s, prm_o, oracle.water_params())
    return got, st, E


def _mi(a, b, L):
    d = a - b
    return np.abs(d - L * np.round(d / L)).max()


@pytest.mark.parametrize("n_side,rc", [(4, 6.0), (6, 9.0)])
def test_water_fp64_parity(n_side, rc):
    (r, p, F, L, cell), st, E = _run_both(n_side, rc, 4, rbe.RBE_FP64, pV=0.01)
    assert np.abs(L - st.L).max() < 1e-12 * st.L.max(), (L, st.L)
    assert _mi(r, st.r, st.L) < 1e-10 * st.L.max()
    assert np.abs(p - st.p).max() < 1e-10 * np.abs(st.p).max()
    assert np.abs(F - st.F).max() < 1e-10 * np.abs(st.F).max()
    assert abs(cell[3] - st.pV.value) < 1e-10 * abs(st.pV.value), (cell[3], st.pV.value)
    assert abs(cell[4] - st.W.value) < 1e-10 * abs(st.W.value), (cell[4], st.W.value)
    for a, b in ((cell[7], E[0]), (cell[8], E[1]), (cell[9], E[2]), (cell[rbe.CELL_EXCL], E[3])):
        assert abs(a - b) < 1e-10 * abs(b), (a, b)
    # molecules stay whole in storage: every H within a bond of its oxygen without images
    mol = r.reshape(-1, 3, 3)
    assert np.abs(np.linalg.norm(mol[:, 1:] - mol[:, :1], axis=2) - 1.0).max() < 1e-12


@pytest.mark.parametrize("kw", [dict(kspace=0), dict(real=0), dict(noise=0), dict(barostat=0),
                                dict(gamma=0.0, gamma_V=0.0, noise=0)])
def test_water_fp64_components(kw):
    (r, p, F, L, cell), st, E = _run_both(4, 6.0, 3, rbe.RBE_FP64, **kw)
    assert np.abs(L - st.L).max() < 1e-12 * st.L.max()
    assert _mi(r, st.r, st.L) < 1e-10 * st.L.max()
    assert np.abs(p - st.p).max() < 1e-10 * np.abs(st.p).max()
    assert np.abs(F - st.F).max() < 1e-10 * np.abs(st.F).max()
    assert abs(cell[4] - st.W.value) < 1e-10 * max(1.0, abs(st.W.value))


def test_water_fp32_phase_kspace():
    """The k-space in FP32 phase (the rest FP64): forces and momenta to 1e-5 relative RMS."""
    (r, p, F, L, cell), st, E = _run_both(4, 6.0, 4, rbe.RBE_FP32_PHASE)
    rel = lambda a, b: np.sqrt(np.mean((a - b) ** 2) / np.mean(b ** 2))  # noqa: E731
    assert rel(F, st.F) < 1e-5
    assert rel(p, st.p) < 1e-5
    assert abs(L[0] - st.L[0]) < 1e-6 * st.L[0]


def test_water_constraints_and_energy_on_the_device():
    """Cold lattice of 27 molecules (no oxygen pair crosses rc), no friction, noise or k-space:
    the device's distances stay exact and its extended energy follows the oracle's, which drifts
    by O(dt^2)."""
    L = 18.0
    pos, p, q, m, box = _waters(3, L, 5, jitter=0.05, thermal=0.1)
    kw = dict(gamma=0.0, gamma_V=0.0, noise=0, kspace=0, M_V=oracle.piston_mass(0.5, 0.75, L ** 3))
    prm_d, prm_o = _params(L, 8.0, **kw)
    # alpha = 0.6: no Coulomb term is left at rc (the context's alpha is the Ewald splitting)
    dev = cuda_device()
    H_dev = []
    with rbe.Context(box, 0.6, P, SEED, rbe.RBE_FP64) as ctx:
        rep = rbe.WaterReplica(pos, p, q, m, box, prm_d, dev)
        rep.init(ctx, batch=0)
        for _ in range(30):
            rep.step(ctx, 10)
            r_, p_, F_, L_, c_ = rep.state()
            K = np.sum(p_ ** 2 / m[:, None]) / 200.0
            H_dev.append(K + c_[8] + c_[9] + c_[rbe.CELL_EXCL] + oracle.BAR * c_[10] + c_[3] ** 2 / (2 * prm_d.M_V))
    st = oracle.WaterState(pos, p, q, m, box)
    prm_o = oracle.npt_params(alpha=0.6, P=P, seed=SEED, dt=0.001, kT=KT, P_ext=oracle.BAR, gamma=0.0, gamma_V=0.0,
                              M_V=prm_d.M_V, rc=8.0, qqr2e=oracle.QQR2E, lj_sigma=3.166, lj_eps=0.650, kspace=0,
                              real=1, noise=0, barostat=1)
    oracle.water_forces(st, 0, prm_o)
    _, _, H = oracle.water_run(st, 0, 300, prm_o, oracle.water_params())
    H_dev = np.array(H_dev)
    assert np.abs(H_dev - H[9::10]).max() < 1e-8, np.abs(H_dev - H[9::10]).max()
    assert np.abs(H_dev - H_dev[0]).max() < 1e-6
    mol = r_.reshape(-1, 3, 3)
    d = np.linalg.norm(mol[:, 1:] - mol[:, :1], axis=2)
    dhh = np.linalg.norm(mol[:, 2] - mol[:, 1], axis=1)
    assert np.abs(d - 1.0).max() < 1e-12 and np.abs(dhh - oracle.water_params().d_HH).max() < 1e-12


def test_water_rejects_bad_input():
    import torch
    L = _box_1gcc(64)
    pos, mom, q, m, box = _waters(4, L, 1)
    dev = cuda_device()
    with rbe.Context(box, ALPHA, P, SEED, rbe.RBE_FP64) as ctx:
        good, _ = _params(L, 6.0)
        for prm, wp, sl in ((good, rbe.water_params(), slice(0, 190)),
                            (_params(L, 6.0, barostat=2, M_cell=(1.0, 1.0, 1.0))[0], rbe.water_params(), slice(None)),
                            (_params(L, 6.0, skin=1.0)[0], rbe.water_params(), slice(None)),
                            (good, rbe.water_params(shake_tol=0.0), slice(None)),
                            (good, rbe.water_params(shake_max_iter=0), slice(None))):
            rep = rbe.WaterReplica(pos[sl], mom[sl], q[sl], m[sl], box, prm, dev, wp=wp)
            with pytest.raises(rbe.RBEError) as e:
                rep.init(ctx)
            assert e.value.status == rbe.RBE_EINVAL
        rep = rbe.WaterReplica(pos, mom, q, m, box, good, dev)
        with pytest.raises(rbe.RBEError) as e:
            rep.step(ctx, 1)
        assert e.value.status == rbe.RBE_ESTATE
        rep.init(ctx)
        rep.step(ctx, 2)
        ctx.sync()
        assert torch.isfinite(rep.pos).all()


def test_water_graph_replay_equals_direct_steps():
    """One water step captured in a CUDA graph and replayed three times ends bit for bit where three
    direct steps end."""
    import torch
    L = _box_1gcc(64)
    pos, mom, q, m, box = _waters(4, L, 3)
    prm, _ = _params(L, 6.0)
    dev = cuda_device()
    out = []
    for use_graph in (False, True):
        s = torch.cuda.Stream()
        with rbe.Context(box, ALPHA, P, SEED, rbe.RBE_FP64, stream=s.cuda_stream) as ctx:
            rep = rbe.WaterReplica(pos, mom, q, m, box, prm, dev)
            rep.init(ctx, batch=0)
            ctx.sync()
            if use_graph:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
                    rep.step(ctx, 1)
                for _ in range(3):
                    g.replay()
                torch.cuda.synchronize()
            else:
                rep.step(ctx, 3)
            ctx.sync()
            out.append(rep.state())
    (r1, p1, F1, L1, c1), (r2, p2, F2, L2, c2) = out
    assert np.array_equal(r1, r2) and np.array_equal(p1, p2) and np.array_equal(F1, F2)
    assert np.array_equal(c1, c2)


def test_water_unconverged_constraints_are_reported():
    """A constraint solve limited to one iteration cannot converge: the step flags it, the next
    sync reports RBE_ESTATE, and the context runs a good system afterwards."""
    L = _box_1gcc(64)
    pos, mom, q, m, box = _waters(4, L, 2)
    prm, _ = _params(L, 6.0)
    dev = cuda_device()
    with rbe.Context(box, ALPHA, P, SEED, rbe.RBE_FP64) as ctx:
        rep = rbe.WaterReplica(pos, mom, q, m, box, prm, dev, wp=rbe.water_params(shake_max_iter=1))
        rep.init(ctx)
        rep.step(ctx, 1)
        with pytest.raises(rbe.RBEError) as e:
            ctx.sync()
        assert e.value.status == rbe.RBE_ESTATE and "SHAKE" in str(e.value)
        rep = rbe.WaterReplica(pos, mom, q, m, box, prm, dev)
        rep.init(ctx)
        rep.step(ctx, 2)
        ctx.sync()


def test_water_single_molecule_matches_oracle():
    """One molecule: no pairs between molecules, the exclusion and the k-space of its own three
    sites only; the device follows the oracle."""
    L = 12.0
    rng = np.random.default_rng(9)
    pos = np.array([[5.0, 6.0, 7.0]]) + LOCAL
    m = MASS.copy()
    mom = rng.normal(size=(3, 3)) * np.sqrt(KT * 100 * m)[:, None]
    box = np.array([L, L, L])
    prm_d, prm_o = _params(L, 5.0, M_V=oracle.piston_mass(0.5, 4.5e-5 / oracle.BAR, L ** 3))
    dev = cuda_device()
    with rbe.Context(box, ALPHA, P, SEED, rbe.RBE_FP64) as ctx:
        rep = rbe.WaterReplica(pos, mom, Q, m, box, prm_d, dev)
        rep.init(ctx, batch=0)
        rep.step(ctx, 3)
        ctx.sync()
        r, p, F, Lb, cell = rep.state()
    st = oracle.WaterState(pos, mom, Q, m, box)
    oracle.water_forces(st, 0, prm_o)
    for s in range(3):
        E = oracle.water_step(st, s, prm_o, oracle.water_params())
    assert np.abs(Lb - st.L).max() < 1e-12 * L
    assert _mi(r, st.r, st.L) < 1e-10 * L
    assert np.abs(p - st.p).max() < 1e-10 * np.abs(st.p).max()
    assert np.abs(F - st.F).max() < 1e-10 * np.abs(st.F).max()
    assert abs(cell[rbe.CELL_EXCL] - E[3]) < 1e-10 * abs(E[3])
