"""GPU parity of the rectangular-cell Langevin NPT step (appendix: the anisotropic
rectangular cell, barostat 2, and the semi-isotropic cell at constant surface tension,
barostat 3) through the C ABI, against the oracle's rectangular step on the same inputs, noise
and RBE batches.  Tolerances as for the isotropic step: FP64 path 1e-10 relative on positions,
momenta, forces, box, cell momenta and virial diagonal after a few steps; FP32-phase path 1e-5
relative RMS on forces and momenta."""
import time

import numpy as np
import pytest

import oracle
import paper_2110_14362_gb300 as rbe

from gpu_util import cuda_device

pytestmark = pytest.mark.gpu

SEED = 5151
ALPHA = 0.2
P = 100
KT = oracle.KB * 300.0


def _system(counts, density=0.1, jitter=0.3, seed=0):
    """A jittered rock-salt lattice (charge (-1)^(i+j+k) at site (i, j, k)) of counts[0] x
    counts[1] x counts[2] sites at the spacing of the density: uneven edges, the same local
    structure on every axis, so the stress is nearly isotropic."""
    a = density ** (-1 / 3)
    box = a * np.asarray(counts, dtype=np.float64)
    rng = np.random.default_rng(seed)
    idx = np.stack(np.meshgrid(*[np.arange(n) for n in counts], indexing="ij"), -1).reshape(-1, 3)
    N = idx.shape[0]
    pos = np.mod((idx + 0.5) * a + rng.uniform(-jitter, jitter, idx.shape), box)
    q = np.where(idx.sum(1) % 2 == 0, 1.0, -1.0)
    m = np.full(N, 20.0)
    mom = rng.normal(size=(N, 3)) * np.sqrt(KT * 100 * m)[:, None]
    return pos, mom, q, m, box


def _params(mode, box, rc, rates=(0.5, -0.3, 0.2), **kw):
    """Parameters and initial cell momenta giving edge j the rate of change rates[j] (A/ps; the
    semi-isotropic x and y edges move together at rates[0])."""
    M = oracle.piston_masses_rect(mode, 0.5, 4.5e-5 / oracle.BAR, box)
    # Coulomb screened by a water-like relative permittivity of 78.5: about 2e4 bar on the
    # lattice below, where the unscreened ionic lattice sits near -3e5 bar and collapses the
    # edges by an angstrom within a few femtoseconds
    base = dict(dt=0.001, kT=KT, P_ext=1.0 * oracle.BAR, gamma=10.0, gamma_V=2.0, M_V=0.0, rc=rc,
                qqr2e=oracle.QQR2E / 78.5, lj_sigma=2.0, lj_eps=0.5, max_disp=0.05, kspace=1, real=1, noise=1,
                barostat=mode, M_cell=M, gamma0=2e-3 if mode == 3 else 0.0)
    base.update(kw)
    pc = tuple(M[j] * rates[j] for j in range(3))
    if mode == 3:
        pc = (M[0] * rates[0] * 2.0 * box[0], 0.0, M[2] * rates[2])  # dA/dt = 2 l dl/dt
    skin = base.pop("skin", 0.0)
    dev = rbe.NptParams(skin=skin, **base)
    orc = oracle.npt_params(alpha=ALPHA, P=P, seed=SEED, **base)
    return dev, orc, pc


def _run_both(mode, counts, rc, nsteps, precision, skin=0.0, **kw):
    pos, mom, q, m, box = _system(counts)
    prm_d, prm_o, pc = _params(mode, box, rc, skin=skin, **kw)
    dev = cuda_device()
    with rbe.Context(box, ALPHA, P, SEED, precision) as ctx:
        rep = rbe.NptReplica(pos, mom, q, m, box, prm_d, dev, step=0, pc=pc)
        rep.init(ctx, batch=0)
        rep.step(ctx, nsteps)
        ctx.sync()
        got = rep.state()
    st = oracle.NptRectState(pos, mom, q, m, box, pc=pc)
    oracle.npt_forces_rect(st, 0, prm_o)
    for s in range(nsteps):
        oracle.npt_step_rect(st, s, prm_o)
    return got, st


def _rel(a, b):
    return np.sqrt(np.mean((a - b) ** 2) / np.mean(b ** 2))


def _oracle_pd(st):
    K2 = np.sum(st.p ** 2 / st.m[:, None], axis=0) / 100.0
    return (K2 + st.Wd) / np.prod(st.L)


CASES = [  # (mode, lattice counts, rc): 2 to 5 cells per axis, uneven edges
    (2, (8, 9, 6), 6.0),
    (2, (10, 12, 9), 7.0),
    (3, (10, 10, 13), 7.0),
    (3, (16, 16, 12), 7.0),
]


@pytest.mark.parametrize("mode,counts,rc", CASES)
@pytest.mark.parametrize("skin", [0.0, 1.0])
def test_rect_fp64_parity(mode, counts, rc, skin):
    (r, p, F, L, cell), st = _run_both(mode, counts, rc, 4, rbe.RBE_FP64, skin=skin)
    assert np.allclose(L, st.L, rtol=1e-12, atol=0), (L, st.L)
    if mode == 3:
        assert L[0] == L[1]
    d = r - st.r
    d -= st.L * np.round(d / st.L)
    assert np.abs(d).max() < 1e-10 * st.L.max(), np.abs(d).max()
    assert np.abs(p - st.p).max() < 1e-10 * np.abs(st.p).max(), np.abs(p - st.p).max() / np.abs(st.p).max()
    assert np.abs(F - st.F).max() < 1e-10 * np.abs(st.F).max(), np.abs(F - st.F).max() / np.abs(st.F).max()
    pc = cell[rbe.CELL_PC:rbe.CELL_PC + 3]
    assert np.abs(pc - st.pc).max() < 1e-10 * np.abs(st.pc).max(), (pc, st.pc)
    if mode == 3:
        assert pc[1] == 0.0
    Wd = cell[rbe.CELL_WD:rbe.CELL_WD + 3]
    assert np.abs(Wd - st.Wd).max() < 1e-10 * np.abs(st.Wd).max(), (Wd, st.Wd)
    Pd = cell[rbe.CELL_PD:rbe.CELL_PD + 3]
    assert np.abs(Pd - _oracle_pd(st)).max() < 1e-10 * np.abs(_oracle_pd(st)).max()
    assert abs(cell[4] - st.Wd.sum()) < 1e-10 * np.abs(st.Wd).sum()
    assert cell[3] == 0.0


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("skin", [0.0, 1.0])
def test_rect_fp32_phase_parity(mode, skin):
    """The FP32-phase path computes the virial to about 1e-6 of its magnitude, while the force on
    a cell variable is V ((P_ins)_jj - P) / l_j: a small difference of 2K_j + W_jj and P V.  So the
    cell momenta are held to 1e-5 of the kicks' scale, sum over the kicks of (dt/2) (2K_j + |W_jj|
    + P V) / l_j, not to 1e-5 of their own (small) size, and the edges to what that moves them."""
    counts = (10, 11, 9) if mode == 2 else (10, 10, 12)
    nsteps, dt = 4, 0.001
    (r, p, F, L, cell), st = _run_both(mode, counts, 7.0, nsteps, rbe.RBE_FP32_PHASE, skin=skin)
    assert _rel(F, st.F) < 1e-5
    assert _rel(p, st.p) < 1e-5
    Wd = cell[rbe.CELL_WD:rbe.CELL_WD + 3]
    assert np.abs(Wd - st.Wd).max() < 1e-5 * np.abs(st.Wd).max(), (Wd, st.Wd)
    K2 = np.sum(st.p ** 2 / st.m[:, None], axis=0) / 100.0
    V = np.prod(st.L)
    kick = 2 * nsteps * 0.5 * dt * (K2 + np.abs(st.Wd) + oracle.BAR * V) / st.L
    M = np.array(_params(mode, _system(counts)[4], 7.0)[0].M_cell)
    if mode == 3:
        kick[0] = 2 * nsteps * 0.5 * dt * ((K2[0] + K2[1] + np.abs(st.Wd[:2]).sum()) / (2 * st.L[0] * st.L[1]) +
                                           oracle.BAR * st.L[2])
    pc = cell[rbe.CELL_PC:rbe.CELL_PC + 3]
    for j in ((0, 1, 2) if mode == 2 else (0, 2)):
        assert abs(pc[j] - st.pc[j]) < 1e-5 * kick[j], (j, pc[j], st.pc[j], kick[j])
    dL = 1e-5 * kick * nsteps * dt / np.where(M > 0, M, 1.0)
    if mode == 3:
        dL[0] = dL[1] = dL[0] / (2 * st.L[0])
    assert np.all(np.abs(L - st.L) < dL + 1e-12 * st.L), (L - st.L, dL)
    d = r - st.r
    d -= st.L * np.round(d / st.L)
    assert np.abs(d).max() < 1e-7 + 2 * dL.max(), (np.abs(d).max(), dL)


@pytest.mark.parametrize("mode", [2, 3])
def test_rect_components_off(mode):
    """k-space only, real space only, no noise: each against the oracle."""
    for kw in (dict(real=0), dict(kspace=0), dict(noise=0, gamma=0.0, gamma_V=0.0)):
        (r, p, F, L, cell), st = _run_both(mode, (7, 7, 8), 6.5, 2, rbe.RBE_FP64, **kw)
        assert np.abs(F - st.F).max() < 1e-10 * np.abs(st.F).max(), kw
        assert np.abs(p - st.p).max() < 1e-10 * np.abs(st.p).max(), kw
        assert np.allclose(L, st.L, rtol=1e-12, atol=0), kw


@pytest.mark.parametrize("mode", [2, 3])
def test_rect_energy_conservation_device(mode):
    """gamma = gamma_V = 0, no noise, real space only on a cold lattice: K + U + P V + the cell
    kinetic energy (minus gamma0 A when semi-isotropic) stays constant over 400 device steps."""
    pos, mom, q, m, box = _system((3, 3, 3), density=27 / 16.0 ** 3, jitter=0.1, seed=4)
    mom = mom * 0.1
    q = q * 0.3
    prm_d, _, pc = _params(mode, box, 6.3, rates=(0.3, -0.2, 0.25), kspace=0, noise=0, gamma=0.0, gamma_V=0.0,
                           max_disp=0.0, P_ext=100 * oracle.BAR)
    M = list(prm_d.M_cell)
    dev = cuda_device()
    H, Ls = [], []
    with rbe.Context(box, ALPHA, P, SEED, rbe.RBE_FP64) as ctx:
        rep = rbe.NptReplica(pos, mom, q, m, box, prm_d, dev, pc=pc)
        rep.init(ctx)
        for _ in range(40):
            rep.step(ctx, 10)
            c = rep.cell.cpu().numpy()
            V = c[0] * c[1] * c[2]
            pcs = c[rbe.CELL_PC:rbe.CELL_PC + 3]
            e = 0.5 * c[5] + c[8] + c[9] + prm_d.P_ext * V
            if mode == 2:
                e += sum(pcs[j] ** 2 / (2 * M[j]) for j in range(3))
            else:
                e += -prm_d.gamma0 * c[0] * c[1] + pcs[0] ** 2 / (2 * M[0]) + pcs[2] ** 2 / (2 * M[2])
            H.append(e)
            Ls.append(c[:3].copy())
    H = np.array(H)
    Ls = np.array(Ls)
    assert np.all(Ls.max(0) - Ls.min(0) > 1e-3), Ls  # every edge moves
    assert np.abs(H - H[0]).max() < 1e-4, np.abs(H - H[0]).max()


def test_rect_rejects_bad_parameters():
    pos, mom, q, m, box = _system((6, 7, 6))
    dev = cuda_device()
    with rbe.Context(box, ALPHA, P, SEED, rbe.RBE_FP64) as ctx:
        prm_d, _, pc = _params(3, box, 6.0)  # semi-isotropic with l_x != l_y
        rep = rbe.NptReplica(pos, mom, q, m, box, prm_d, dev, pc=pc)
        with pytest.raises(rbe.RBEError) as e:
            rep.init(ctx, batch=0)
        assert e.value.status == rbe.RBE_EINVAL
        prm_d, _, pc = _params(2, box, 6.0)
        prm_d.M_cell[1] = 0.0
        rep = rbe.NptReplica(pos, mom, q, m, box, prm_d, dev, pc=pc)
        with pytest.raises(rbe.RBEError) as e:
            rep.init(ctx, batch=0)
        assert e.value.status == rbe.RBE_EINVAL
        prm_d, _, pc = _params(2, box, 6.0)
        prm_d.barostat = 4
        rep = rbe.NptReplica(pos, mom, q, m, box, prm_d, dev, pc=pc)
        with pytest.raises(rbe.RBEError):
            rep.init(ctx, batch=0)
        # the context still runs a valid rectangular replica
        prm_d, _, pc = _params(2, box, 6.0)
        rep = rbe.NptReplica(pos, mom, q, m, box, prm_d, dev, pc=pc)
        rep.init(ctx, batch=0)
        rep.step(ctx, 2)
        ctx.sync()


@pytest.mark.parametrize("precision", [rbe.RBE_FP64, rbe.RBE_FP32_PHASE])
def test_rect_served_equals_direct(precision):
    """An anisotropic and a semi-isotropic replica through the serving loop (captured chunk
    graphs) end bit for bit where the same steps launched directly end."""
    cases = [(2, (8, 9, 7), 21, 9), (3, (7, 7, 9), 22, 7)]
    cuda_device()
    srv = rbe.Server(ALPHA, P, precision, max_slots=4, chunk_steps=4, use_graphs=True)
    ids = []
    try:
        for mode, counts, pseed, nsteps in cases:
            pos, mom, q, m, box = _system(counts, seed=pseed)
            prm_d, _, pc = _params(mode, box, 6.0)
            ids.append(srv.submit(pos, mom, q, m, box, prm_d, pseed, nsteps, pc=pc))
        t_end = time.monotonic() + 300.0
        while srv.progress(wait=True)[2] < len(ids):
            assert time.monotonic() < t_end
        served = [srv.result(i) for i in ids]
    finally:
        srv.close()
    dev = cuda_device()
    for (mode, counts, pseed, nsteps), (pos_s, mom_s, cell_s) in zip(cases, served):
        pos, mom, q, m, box = _system(counts, seed=pseed)
        prm_d, _, pc = _params(mode, box, 6.0)
        with rbe.Context(box, ALPHA, P, pseed, precision) as ctx:
            rep = rbe.NptReplica(pos, mom, q, m, box, prm_d, dev, pc=pc)
            rep.init(ctx, batch=0)
            rep.step(ctx, nsteps)
            ctx.sync()
            r, p, _, L, cell = rep.state()
        assert np.array_equal(r, pos_s) and np.array_equal(p, mom_s)
        assert np.array_equal(cell[:3], cell_s[:3])
        assert np.array_equal(cell[rbe.CELL_PC:rbe.CELL_PC + 3], cell_s[rbe.CELL_PC:rbe.CELL_PC + 3])
