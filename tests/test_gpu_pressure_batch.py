"""GPU parity of the separate pressure batch (Eq. (apppress) with its own p~): forces from the
force batch (slots [0, P) of the sampler, weights S/P), virial and energy from the pressure batch
(slots [P, P + p~), weights S/p~), against the oracle's estimators on the same frequencies, through
the device and host-buffer calls and inside the NPT step."""
import numpy as np
import pytest

import oracle
import paper_2110_14362_gb300 as rbe

from gpu_util import cuda_device

pytestmark = pytest.mark.gpu

ALPHA = 0.2


def _charges(N, box, seed):
    rng = np.random.default_rng(seed)
    pos = rng.random((N, 3)) * np.asarray(box)
    q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    return pos, q


@pytest.mark.parametrize("precision,tol", [(rbe.RBE_FP64, 1e-10), (rbe.RBE_FP32_PHASE, 1e-5)])
@pytest.mark.parametrize("P,Pt", [(100, 37), (129, 300)])
def test_pressure_batch_parity(precision, tol, P, Pt):
    import torch
    dev = cuda_device()
    N, box, seed = 5003, (21.0, 23.0, 26.0), 17
    pos, q = _charges(N, box, 3)
    tp, tq = torch.as_tensor(pos).to(dev), torch.as_tensor(q).to(dev)
    out = {}
    with rbe.Context(box, ALPHA, P, seed, precision) as ctx:
        ctx.set_stream(torch.cuda.current_stream().cuda_stream)
        for pt in (0, Pt):
            ctx.set_pressure_batch(pt)
            F = torch.empty((N, 3), dtype=torch.float64, device=dev)
            W = torch.empty(9, dtype=torch.float64, device=dev)
            E = torch.empty(2, dtype=torch.float64, device=dev)
            ctx.forces_virial(tp, tq, 5, F, W, E)
            ctx.sync()
            out[pt] = (F.cpu().numpy(), W.cpu().numpy().reshape(3, 3), E.cpu().numpy())
        Fh, Wh, Eh = ctx.forces_virial_host(pos, q, 5)
    m, S = oracle.sample_k(box, ALPHA, P + Pt, seed, 5)
    F0, _, _, _, _ = oracle.rbe_kspace(pos, q, box, ALPHA, m[:P], S / P)
    _, W1, Ek1, Es1, _ = oracle.rbe_kspace(pos, q, box, ALPHA, m[P:], S / Pt)
    Fd, Wd, Ed = out[Pt]
    rms = np.sqrt(np.mean(F0 ** 2))
    err = np.abs(Fd - F0).max() if precision == rbe.RBE_FP64 else np.sqrt(np.mean((Fd - F0) ** 2))
    assert err < tol * rms
    assert np.linalg.norm(Wd - W1) < tol * np.linalg.norm(W1)
    assert abs(Ed[0] - Ek1) < tol * abs(Ek1) and abs(Ed[1] - Es1) < tol * abs(Es1)
    # the force batch is the same draws as without a pressure batch: forces bit for bit
    assert np.array_equal(Fd, out[0][0])
    assert not np.allclose(Wd, out[0][1])
    # the host-buffer call takes the same path
    assert np.array_equal(np.asarray(Fh).reshape(N, 3), Fd)
    assert np.array_equal(np.asarray(Wh).reshape(3, 3), Wd)


@pytest.mark.parametrize("sampler", [rbe.RBE_SAMPLER_EXACT, rbe.RBE_SAMPLER_MH])
def test_npt_with_pressure_batch(sampler):
    """The NPT step with p~ = 60 besides P = 100 (and the MH chain over both batches) against the
    oracle's NPT step with the same batches, at 1e-10 on the FP64 path after four steps."""
    n_side, P, Pt, seed = 8, 100, 60, 777
    N = n_side ** 3
    L = (N / 0.1) ** (1 / 3)
    rng = np.random.default_rng(1)
    g = (np.arange(n_side) + 0.5) * (L / n_side)
    pos = np.mod(np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
                 + rng.uniform(-0.3, 0.3, (N, 3)), L)
    q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    m = np.full(N, 20.0)
    mom = rng.normal(size=(N, 3)) * np.sqrt(oracle.KB * 300 * 100 * m)[:, None]
    box = np.array([L, L, L])
    base = dict(dt=0.001, kT=oracle.KB * 300.0, P_ext=oracle.BAR, gamma=10.0, gamma_V=2.0,
                M_V=oracle.piston_mass(0.5, 4.5e-5 / oracle.BAR, L ** 3), rc=6.5, qqr2e=oracle.QQR2E / 78.5,
                lj_sigma=2.0, lj_eps=0.5, max_disp=0.05, kspace=1, real=1, noise=1, barostat=1)
    dev = cuda_device()
    with rbe.Context(box, ALPHA, P, seed, rbe.RBE_FP64) as ctx:
        ctx.set_sampler(sampler)
        ctx.set_pressure_batch(Pt)
        rep = rbe.NptReplica(pos, mom, q, m, box, rbe.NptParams(**base), dev, step=0)
        rep.init(ctx, batch=0)
        rep.step(ctx, 4)
        ctx.sync()
        r_d, p_d, F_d, L_d, cell = rep.state()
    chain = np.zeros((P + Pt, 3), dtype=np.int32)
    prm = oracle.npt_params(alpha=ALPHA, P=P, seed=seed, sampler=sampler, chain=chain.ctypes.data, Ptilde=Pt,
                            **base)
    st = oracle.NptState(pos, mom, q, m, box)
    oracle.npt_forces(st, 0, prm)
    for s in range(4):
        oracle.npt_step(st, s, prm)
    assert np.allclose(L_d, st.L, rtol=1e-12, atol=0)
    assert np.abs(p_d - st.p).max() < 1e-10 * np.abs(st.p).max()
    assert np.abs(F_d - st.F).max() < 1e-10 * np.abs(st.F).max()
    assert abs(cell[4] - st.W.value) < 1e-10 * abs(st.W.value)
    assert abs(cell[3] - st.pV.value) < 1e-10 * max(abs(st.pV.value), 1e-30)


def test_pressure_batch_rejects_bad_sizes():
    cuda_device()
    with rbe.Context((10.0, 10.0, 10.0), ALPHA, 16, 1, rbe.RBE_FP64) as ctx:
        for bad in (-1, 2 ** 20 + 1):
            with pytest.raises(rbe.RBEError) as e:
                ctx.set_pressure_batch(bad)
            assert e.value.status == rbe.RBE_EINVAL


def _npt_lattice(n_side=8, seed=2):
    N = n_side ** 3
    L = (N / 0.1) ** (1 / 3)
    rng = np.random.default_rng(seed)
    g = (np.arange(n_side) + 0.5) * (L / n_side)
    pos = np.mod(np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
                 + rng.uniform(-0.3, 0.3, (N, 3)), L)
    q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    m = np.full(N, 20.0)
    mom = rng.normal(size=(N, 3)) * np.sqrt(oracle.KB * 300 * 100 * m)[:, None]
    base = dict(dt=0.001, kT=oracle.KB * 300.0, P_ext=oracle.BAR, gamma=10.0, gamma_V=2.0,
                M_V=oracle.piston_mass(0.5, 4.5e-5 / oracle.BAR, L ** 3), rc=6.5, qqr2e=oracle.QQR2E / 78.5,
                lj_sigma=2.0, lj_eps=0.5, max_disp=0.05, kspace=1, real=1, noise=1, barostat=1)
    return pos, mom, q, m, np.array([L, L, L]), base


@pytest.mark.parametrize("sampler,Pt", [(rbe.RBE_SAMPLER_EXACT, 0), (rbe.RBE_SAMPLER_OFFLINE, 40)])
def test_npt_sample_reuse(sampler, Pt):
    """Samples drawn every M = 4 steps from the box of the drawing step (Sec. 4.3): nine NPT steps
    (three refreshes) against the oracle's NPT step with the same reuse, at 1e-10; the run differs
    from the one without reuse (the kept batches are really used)."""
    P, seed, M, n = 100, 99, 4, 9
    pos, mom, q, m, box, base = _npt_lattice()
    dev = cuda_device()
    res = {}
    for reuse in (1, M):
        with rbe.Context(box, ALPHA, P, seed, rbe.RBE_FP64) as ctx:
            ctx.set_sampler(sampler)
            ctx.set_pressure_batch(Pt)
            ctx.set_sample_reuse(reuse)
            rep = rbe.NptReplica(pos, mom, q, m, box, rbe.NptParams(**base), dev, step=0)
            rep.init(ctx, batch=0)
            rep.step(ctx, n)
            ctx.sync()
            res[reuse] = rep.state()
    r_d, p_d, F_d, L_d, cell = res[M]
    buf = np.zeros((M * (P + Pt), 3), dtype=np.int32)
    prm = oracle.npt_params(alpha=ALPHA, P=P, seed=seed, sampler=sampler, Ptilde=Pt, reuse=M,
                            reuse_m=buf.ctypes.data, **base)
    st = oracle.NptState(pos, mom, q, m, box)
    oracle.npt_forces(st, 0, prm)
    for s in range(n):
        oracle.npt_step(st, s, prm)
    assert np.allclose(L_d, st.L, rtol=1e-12, atol=0)
    assert np.abs(p_d - st.p).max() < 1e-10 * np.abs(st.p).max()
    assert np.abs(F_d - st.F).max() < 1e-10 * np.abs(st.F).max()
    assert abs(cell[4] - st.W.value) < 1e-10 * abs(st.W.value)
    assert np.abs(res[1][2] - F_d).max() > 1e-6 * np.abs(F_d).max()


def test_sample_reuse_and_mh_exclude_each_other():
    cuda_device()
    with rbe.Context((20.0, 20.0, 20.0), ALPHA, 16, 1, rbe.RBE_FP64) as ctx:
        ctx.set_sampler(rbe.RBE_SAMPLER_MH)
        with pytest.raises(rbe.RBEError):
            ctx.set_sample_reuse(4)
        ctx.set_sampler(rbe.RBE_SAMPLER_EXACT)
        ctx.set_sample_reuse(4)
        with pytest.raises(rbe.RBEError):
            ctx.set_sampler(rbe.RBE_SAMPLER_MH)
        for bad in (0, 1025):
            with pytest.raises(rbe.RBEError):
                ctx.set_sample_reuse(bad)
