"""GPU parity of the paper's own frequency samplers (Sec. 4.3) through the C ABI: the offline
rounded-Gaussian draws and the online Metropolis--Hastings chain give the oracle's m bit for bit
(ragged P, several boxes, seeds and steps, the chain across box changes), the k-space forces of
those frequencies match the oracle at 1e-10 (FP64), and the NPT step driven by either sampler
matches the oracle's NPT step at 1e-10."""
import numpy as np
import pytest

import oracle
import paper_2110_14362_gb300 as rbe

from gpu_util import cuda_device

pytestmark = pytest.mark.gpu

ALPHA = 0.2


@pytest.mark.parametrize("P", [1, 129, 1000])
@pytest.mark.parametrize("box,seed", [((10.0, 12.0, 14.0), 3), ((4.5, 4.5, 4.5), 77), ((80.0, 80.0, 120.0), 2**40 + 5)])
def test_offline_m_bit_exact(P, box, seed):
    cuda_device()
    with rbe.Context(box, ALPHA, P, seed, rbe.RBE_FP64) as ctx:
        ctx.set_sampler(rbe.RBE_SAMPLER_OFFLINE)
        for step in (0, 1, 12345, 2**40 + 17):
            m, S = ctx.sample_k(step)
            m0, S0 = oracle.sample_k_offline(box, ALPHA, P, seed, step)
            assert np.array_equal(m, m0), step
            assert S == S0


@pytest.mark.parametrize("P", [3, 257, 2000])
def test_mh_chain_bit_exact_across_box_changes(P):
    """Ten MH steps with the box changing between them (as in an NPT run): the device chain equals
    the oracle chain after every step; a second rbe_set_sampler resets it to the exact draw."""
    cuda_device()
    boxes = [(10.0 + 0.3 * s, 12.0 - 0.2 * s, 14.0 + 0.1 * s) for s in range(10)]
    seed = 91
    state = np.zeros((P, 3), dtype=np.int32)
    with rbe.Context(boxes[0], ALPHA, P, seed, rbe.RBE_FP64) as ctx:
        ctx.set_sampler(rbe.RBE_SAMPLER_MH)
        moved = 0
        for s, box in enumerate(boxes):
            ctx.set_box(box)
            m, S = ctx.sample_k(100 + s)
            prev = state.copy()
            oracle.sample_k_mh(box, ALPHA, P, seed, 100 + s, state)
            assert np.array_equal(m, state), s
            if s > 0:
                moved += int(np.any(state != prev, axis=1).sum())
        assert moved > 0.3 * 9 * P  # the chain does move
        ctx.set_sampler(rbe.RBE_SAMPLER_MH)
        m, _ = ctx.sample_k(500)
        assert np.array_equal(m, oracle.sample_k(boxes[-1], ALPHA, P, seed, 500)[0])
        ctx.set_sampler(rbe.RBE_SAMPLER_EXACT)
        m, _ = ctx.sample_k(501)
        assert np.array_equal(m, oracle.sample_k(boxes[-1], ALPHA, P, seed, 501)[0])


@pytest.mark.parametrize("sampler", [rbe.RBE_SAMPLER_OFFLINE, rbe.RBE_SAMPLER_MH])
def test_forces_with_variant_samplers(sampler):
    """rbe_kspace_forces_virial with the offline or MH frequencies: forces and virial of the
    oracle's RBE estimator on the same m with weights S/P, at 1e-10 (FP64), over three steps."""
    import torch
    dev = cuda_device()
    rng = np.random.default_rng(4)
    N, P, box, seed = 3001, 129, (20.0, 22.0, 25.0), 61
    pos = rng.random((N, 3)) * np.array(box)
    q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    state = np.zeros((P, 3), dtype=np.int32)
    with rbe.Context(box, ALPHA, P, seed, rbe.RBE_FP64) as ctx:
        ctx.set_stream(torch.cuda.current_stream().cuda_stream)
        ctx.set_sampler(sampler)
        tp, tq = torch.as_tensor(pos).to(dev), torch.as_tensor(q).to(dev)
        for step in range(3):
            F = torch.empty((N, 3), dtype=torch.float64, device=dev)
            W = torch.empty(9, dtype=torch.float64, device=dev)
            ctx.forces_virial(tp, tq, step, F, W)
            ctx.sync()
            if sampler == rbe.RBE_SAMPLER_OFFLINE:
                m, S = oracle.sample_k_offline(box, ALPHA, P, seed, step)
            else:
                m, S = oracle.sample_k_mh(box, ALPHA, P, seed, step, state)
            F0, W0, _, _, _ = oracle.rbe_kspace(pos, q, box, ALPHA, m, S / P)
            Fd = F.cpu().numpy()
            assert np.abs(Fd - F0).max() < 1e-10 * np.sqrt(np.mean(F0 ** 2)), step
            assert np.linalg.norm(W.cpu().numpy().reshape(3, 3) - W0) < 1e-10 * np.linalg.norm(W0), step


@pytest.mark.parametrize("sampler", [rbe.RBE_SAMPLER_OFFLINE, rbe.RBE_SAMPLER_MH])
def test_npt_with_variant_samplers(sampler):
    """The NPT step (box changing every step, step index on the device) with the offline or MH
    frequencies against the oracle's NPT step with the same sampler, at 1e-10 after five steps."""
    n_side, P, seed = 8, 100, 4242
    N = n_side ** 3
    L = (N / 0.1) ** (1 / 3)
    rng = np.random.default_rng(0)
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
        rep = rbe.NptReplica(pos, mom, q, m, box, rbe.NptParams(**base), dev, step=0)
        rep.init(ctx, batch=0)
        rep.step(ctx, 5)
        ctx.sync()
        r_d, p_d, F_d, L_d, cell = rep.state()
    chain = np.zeros((P, 3), dtype=np.int32)
    prm = oracle.npt_params(alpha=ALPHA, P=P, seed=seed, sampler=sampler, chain=chain.ctypes.data, **base)
    st = oracle.NptState(pos, mom, q, m, box)
    oracle.npt_forces(st, 0, prm)
    for s in range(5):
        oracle.npt_step(st, s, prm)
    assert np.allclose(L_d, st.L, rtol=1e-12, atol=0)
    d = r_d - st.r
    d -= st.L * np.round(d / st.L)
    assert np.abs(d).max() < 1e-10 * L
    assert np.abs(p_d - st.p).max() < 1e-10 * np.abs(st.p).max()
    assert np.abs(F_d - st.F).max() < 1e-10 * np.abs(st.F).max()


@pytest.mark.parametrize("sampler", [rbe.RBE_SAMPLER_EXACT, rbe.RBE_SAMPLER_OFFLINE, rbe.RBE_SAMPLER_MH])
def test_sampler_bias_on_the_device(sampler):
    """The mean device force over 400 steps (P = 500, sigma = 0.5 per axis) converges to the exact
    expectation of its sampler: the Ewald force for the exact and MH samplers, the offline
    expectation (21 % of the force RMS away from it) for the offline one.  Standard errors from 20
    batch means of 20 steps (the MH chain correlates consecutive steps)."""
    import torch
    from test_oracle_samplers import offline_bias_case
    pos, q, box, alpha, F_off, F_ew, _, _ = offline_bias_case()
    dev = cuda_device()
    N, P, n = q.shape[0], 500, 400
    tp, tq = torch.as_tensor(pos).to(dev), torch.as_tensor(q).to(dev)
    Fs = np.zeros((n, N, 3))
    with rbe.Context(box, alpha, P, 5, rbe.RBE_FP64) as ctx:
        ctx.set_stream(torch.cuda.current_stream().cuda_stream)
        ctx.set_sampler(sampler)
        F = torch.empty((N, 3), dtype=torch.float64, device=dev)
        for s in range(n):
            ctx.forces_virial(tp, tq, s, F)
            Fs[s] = F.cpu().numpy()
    bm = Fs.reshape(20, 20, N, 3).mean(1)
    mean, se = bm.mean(0), bm.std(0, ddof=1) / np.sqrt(20)
    target, other = (F_off, F_ew) if sampler == rbe.RBE_SAMPLER_OFFLINE else (F_ew, F_off)
    chi_t = np.mean(((mean - target) / se) ** 2)
    chi_o = np.mean(((mean - other) / se) ** 2)
    assert chi_t < 2.0, chi_t  # about 1.1-1.3 for the right expectation (t with 19 dof, correlated components)
    assert chi_o > 10 * chi_t, (chi_t, chi_o)
