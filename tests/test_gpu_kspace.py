"""GPU parity of the RBE k-space path (through the C ABI) against the FP64 oracle.

Tolerances: sampled m and S bit-exact; FP64 path max|dF|/RMS(F), |dW|_F/|W|_F and
|dE|/|E| <= 1e-10; FP32-phase path RMS(dF)/RMS(F) <= 1e-5 with the same bound on the
virial and the energy."""
import functools

import numpy as np
import pytest

import oracle
import paper_2110_14362_gb300 as rbe
from paper_2110_14362_gb300 import inputs

from gpu_util import cuda_device, rel_frob, rel_max_force, rel_rms_force, to_dev

pytestmark = pytest.mark.gpu

SEED = 12345


def _run(sys_, P, step, precision, accum=rbe.RBE_RHO_COMP32, seed=SEED, box=None):
    import torch
    box = sys_.box if box is None else box
    dev = cuda_device()
    pos = to_dev(sys_.pos)
    q = to_dev(sys_.q)
    F = torch.full((sys_.N, 3), float("nan"), dtype=torch.float64, device=dev)
    W = torch.full((9,), float("nan"), dtype=torch.float64, device=dev)
    E = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    with rbe.Context(box, sys_.alpha, P, seed, precision, accum) as ctx:
        ctx.set_stream(torch.cuda.current_stream().cuda_stream)
        ctx.forces_virial(pos, q, step, F, W, E)
        ctx.sync()
        rho = ctx.rho()
    return F.cpu().numpy(), W.cpu().numpy().reshape(3, 3), E.cpu().numpy(), rho


@pytest.mark.parametrize("box,alpha,P,seed,step", [
    ((10.0, 10.0, 10.0), 1.0, 100, 12345, 0),
    ((80.0, 80.0, 120.0), 0.2, 200, 12345, 7),
    ((342.0, 342.0, 342.0), 0.2, 2000, 3, 1 << 40),
    ((1.0, 1.0, 1.0), 1.5, 64, 1, 0),          # almost every draw is m = 0: many redraws
    ((3.0, 40.0, 5.0), 0.7, 4096, 2**63 + 5, 123456789),
])
def test_sampled_frequencies_bit_exact(box, alpha, P, seed, step):
    m0, S0 = oracle.sample_k(np.array(box), alpha, P, seed, step)
    h = rbe.rbe_create(box, alpha, P, seed)
    try:
        m, S = rbe.rbe_sample_k(h, step, P)
    finally:
        rbe.rbe_destroy(h)
    assert np.array_equal(m, m0)
    assert S == S0


def test_fp64_snapshot_parity_small():
    s = inputs.small_snapshot()
    F, W, E, rho = _run(s, s.P, 0, rbe.RBE_FP64)
    F0, W0, Ek0, Es0, m0, S0 = oracle.rbe_snapshot(s.pos, s.q, s.box, s.alpha, s.P, SEED, 0)
    assert rel_max_force(F, F0) <= 1e-10
    assert rel_frob(W, W0) <= 1e-10
    assert abs(E[0] - Ek0) <= 1e-10 * abs(Ek0)
    assert abs(E[1] - Es0) <= 1e-12 * abs(Es0)
    _, _, _, _, rho0 = oracle.rbe_kspace(s.pos, s.q, s.box, s.alpha, m0, S0 / s.P)
    assert np.max(np.abs(rho - rho0)) <= 1e-10 * np.max(np.abs(rho0))


@pytest.mark.parametrize("N", [1, 2, 7, 127, 128, 129, 257, 1000, 3001])
@pytest.mark.parametrize("P", [1, 3, 129, 300, 700])
def test_fp64_ragged_sizes(N, P):
    box = np.array([9.0, 10.0, 11.5])
    pos, q = inputs.uniform_pm1(N, box, seed=N * 7 + P)
    if N == 1:
        q = np.array([1.0])
    s = inputs.System(pos, q, box, 0.8, P, 4.0, "ragged")
    F, W, E, _ = _run(s, P, 3, rbe.RBE_FP64)
    F0, W0, Ek0, Es0, _, _ = oracle.rbe_snapshot(pos, q, box, 0.8, P, SEED, 3)
    # unit charges in a box of side ~10: forces are O(1) unless they cancel exactly (N = 1),
    # so the bound is relative with an absolute floor of 1e-13
    scale = np.sqrt(np.mean(np.sum(F0 * F0, 1)))
    assert np.max(np.abs(F - F0)) <= 1e-10 * scale + 1e-13
    assert np.max(np.abs(W - W0)) <= 1e-10 * np.abs(W0).max() + 1e-13
    assert abs(E[0] - Ek0) <= 1e-10 * abs(Ek0) + 1e-13


@pytest.mark.parametrize("precision", [rbe.RBE_FP64, rbe.RBE_FP32_PHASE])
def test_empty_system(precision):
    import torch
    dev = cuda_device()
    pos = torch.zeros((0, 3), dtype=torch.float64, device=dev)
    q = torch.zeros((0,), dtype=torch.float64, device=dev)
    F = torch.zeros((0, 3), dtype=torch.float64, device=dev)
    W = torch.full((9,), float("nan"), dtype=torch.float64, device=dev)
    E = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    with rbe.Context([10.0, 10.0, 10.0], 1.0, 50, 1, precision) as ctx:
        ctx.forces_virial(pos, q, 0, F, W, E)
        ctx.sync()
    assert torch.all(W == 0) and torch.all(E == 0)


@pytest.mark.parametrize("precision", [rbe.RBE_FP64, rbe.RBE_FP32_PHASE])
def test_vanishing_structure_factor(precision):
    """A neutral pair at one point has rho(k) = 0 for every k: forces, k-space energy and
    virial are exactly zero (the FP32-phase force pass then shifts its phase by arg 0 with a
    zero amplitude), and the self energy is -sqrt(alpha/pi) sum q^2."""
    import torch
    dev = cuda_device()
    alpha = 0.7
    pos = torch.tensor([[1.3, 2.7, 4.1], [1.3, 2.7, 4.1]], dtype=torch.float64, device=dev)
    q = torch.tensor([1.0, -1.0], dtype=torch.float64, device=dev)
    F = torch.full((2, 3), float("nan"), dtype=torch.float64, device=dev)
    W = torch.full((9,), float("nan"), dtype=torch.float64, device=dev)
    E = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    with rbe.Context([9.0, 10.0, 11.0], alpha, 300, 5, precision) as ctx:
        ctx.forces_virial(pos, q, 3, F, W, E)
        ctx.sync()
        rho = ctx.rho()
    assert np.all(np.asarray(rho) == 0)
    assert torch.all(F == 0) and torch.all(W == 0) and E[0].item() == 0.0
    _, _, _, Es, _ = oracle.rbe_kspace(pos.cpu().numpy(), q.cpu().numpy(), [9.0, 10.0, 11.0], alpha,
                                       np.array([[1, 0, 0]], dtype=np.int32), 1.0)
    assert abs(E[1].item() - Es) <= 1e-6 * abs(Es)


def test_weighted_full_k_equals_ewald():
    import torch
    s = inputs.small_snapshot()
    pos, q = s.pos[:500], s.q[:500]
    box = np.array([10.0, 10.0, 12.0])
    kmax = 8
    import itertools
    m = np.array([v for v in itertools.product(range(-kmax, kmax + 1), repeat=3) if any(v)], dtype=np.int32)
    k = 2 * np.pi * m / box
    w = np.exp(-(k * k).sum(1) / (4 * s.alpha))
    dev = cuda_device()
    F = torch.empty((500, 3), dtype=torch.float64, device=dev)
    W = torch.empty(9, dtype=torch.float64, device=dev)
    E = torch.empty(2, dtype=torch.float64, device=dev)
    with rbe.Context(box, s.alpha, 10, 1, rbe.RBE_FP64) as ctx:
        ctx.weighted(to_dev(pos), to_dev(q), to_dev(m), to_dev(w), F, W, E)
        ctx.sync()
    F0, W0, Ek0, Es0 = oracle.ewald_kspace(pos, q, box, s.alpha, kmax)
    assert rel_max_force(F.cpu().numpy(), F0) <= 1e-10
    assert rel_frob(W.cpu().numpy().reshape(3, 3), W0) <= 1e-10
    assert abs(E[0].item() - Ek0) <= 1e-10 * abs(Ek0)


@pytest.mark.parametrize("accum", [rbe.RBE_RHO_FP32, rbe.RBE_RHO_COMP32, rbe.RBE_RHO_FP64])
def test_fp32_phase_parity_small(accum):
    s = inputs.small_snapshot()
    F, W, E, _ = _run(s, s.P, 0, rbe.RBE_FP32_PHASE, accum)
    F0, W0, Ek0, Es0, _, _ = oracle.rbe_snapshot(s.pos, s.q, s.box, s.alpha, s.P, SEED, 0)
    assert rel_rms_force(F, F0) <= 1e-5
    assert rel_frob(W, W0) <= 1e-5
    assert abs(E[0] - Ek0) <= 1e-5 * abs(Ek0)


@pytest.mark.parametrize("N,P", [(20000, 200), (5003, 517), (64, 4096), (100000, 300), (100003, 450)])
def test_fp32_phase_parity_mid(N, P):
    """FP32-phase path against the oracle; (100000, 300) and (100003, 450) run the wide
    two-frequency rho tiles with one particle sub-stream (150 and 225 lanes)."""
    s = inputs.uniform_density(N, P=P)
    F, W, E, _ = _run(s, P, 11, rbe.RBE_FP32_PHASE)
    F0, W0, Ek0, Es0, _, _ = oracle.rbe_snapshot(s.pos, s.q, s.box, s.alpha, P, SEED, 11)
    assert rel_rms_force(F, F0) <= 1e-5
    assert rel_frob(W, W0) <= 1e-5
    assert abs(E[0] - Ek0) <= 1e-5 * abs(Ek0)


@functools.lru_cache(maxsize=1)
def _slab_oracle():
    s = inputs.slab()
    return s, oracle.rbe_snapshot(s.pos, s.q, s.box, s.alpha, s.P, SEED, 0)


def test_full_size_slab_fp64():
    """The slab workload at full size (300k charges, P = 200): every output of the FP64 path
    against the oracle."""
    s, (F0, W0, Ek0, Es0, m0, S0) = _slab_oracle()
    F, W, E, _ = _run(s, s.P, 0, rbe.RBE_FP64)
    assert rel_max_force(F, F0) <= 1e-10
    assert rel_frob(W, W0) <= 1e-10
    assert abs(E[0] - Ek0) <= 1e-10 * abs(Ek0)


@pytest.mark.parametrize("accum", [rbe.RBE_RHO_COMP32, rbe.RBE_RHO_FP32, rbe.RBE_RHO_FP64])
def test_full_size_slab_fp32_phase(accum):
    """The slab workload at full size on the FP32-phase path with each rho accumulation, in
    the launch configuration the benchmark times: forces, Pxx, Pyy, Pzz and E_k against the
    oracle."""
    s, (F0, W0, Ek0, Es0, m0, S0) = _slab_oracle()
    F, W, E, _ = _run(s, s.P, 0, rbe.RBE_FP32_PHASE, accum)
    assert rel_rms_force(F, F0) <= 1e-5
    for a in range(3):  # Pxx, Pyy, Pzz separately
        assert abs(W[a, a] - W0[a, a]) <= 1e-5 * np.abs(np.diag(W0)).max()
    assert abs(E[0] - Ek0) <= 1e-5 * abs(Ek0)


def test_host_api_matches_device_api():
    s = inputs.small_snapshot()
    F, W, E, _ = _run(s, s.P, 5, rbe.RBE_FP32_PHASE)
    with rbe.Context(s.box, s.alpha, s.P, SEED, rbe.RBE_FP32_PHASE) as ctx:
        Fh, Wh, Eh = ctx.forces_virial_host(s.pos, s.q, 5)
    assert np.array_equal(F, Fh) and np.array_equal(W, Wh) and np.array_equal(E, Eh)


@pytest.mark.parametrize("pinned", [True, False])
def test_host_api_pipelined(pinned):
    """The host-buffer call on the full slab (N = 300000: copies pipelined with two groups of
    full-GPU passes), with page-locked or pageable buffers: the device API's result to FP32
    rounding (a different chunk partition), the oracle's within the path's 1e-5, and the same
    bits on every call."""
    import torch
    s = inputs.slab()
    F, W, E, _ = _run(s, s.P, 3, rbe.RBE_FP32_PHASE)
    if pinned:
        pos = torch.empty((s.N, 3), dtype=torch.float64, pin_memory=True)
        q = torch.empty((s.N,), dtype=torch.float64, pin_memory=True)
        pos.copy_(torch.as_tensor(s.pos))
        q.copy_(torch.as_tensor(s.q))
        pos_h, q_h = pos.numpy(), q.numpy()
        Fout = torch.zeros((s.N, 3), dtype=torch.float64, pin_memory=True).numpy()
    else:
        pos_h, q_h, Fout = s.pos, s.q, np.zeros((s.N, 3))
    first = None
    with rbe.Context(s.box, s.alpha, s.P, SEED, rbe.RBE_FP32_PHASE) as ctx:
        for _ in range(2):  # the second call reuses the staging and the copy stream
            Fout[:] = np.nan
            Fh, Wh, Eh = rbe.rbe_kspace_forces_virial_host(ctx.h, pos_h, q_h, 3, Fout)
            out = (Fh.copy(), Wh.copy(), Eh.copy())
            if first is None:
                first = out
            for a, b in zip(first, out):
                assert np.array_equal(a, b)
    Fh, Wh, Eh = first
    assert rel_rms_force(Fh, F) < 2e-6
    assert rel_frob(Wh, W) < 2e-6
    assert abs(Eh[0] - E[0]) < 2e-6 * abs(E[0]) and abs(Eh[1] - E[1]) < 2e-6 * abs(E[1])
    m, S = oracle.sample_k(s.box, s.alpha, s.P, SEED, 3)
    Fo, Wo, Eko, Eso, _ = oracle.rbe_kspace(s.pos, s.q, s.box, s.alpha, m, S / s.P)
    assert rel_rms_force(Fh, Fo) < 1e-5
    for a in range(3):
        assert abs(Wh[a, a] - Wo[a, a]) <= 1e-5 * np.abs(np.diag(Wo)).max()


def test_host_api_four_groups():
    """The host-buffer call from 2^19 particles pipelines four groups of uneven size (an eighth,
    three eighths, three eighths, an eighth): N = 600000, P = 100 with page-locked buffers, against
    the device API to FP32 rounding, the oracle within 1e-5, and the same bits on a second call."""
    import torch
    s = inputs.uniform_density(600000, P=100)
    F, W, E, _ = _run(s, 100, 7, rbe.RBE_FP32_PHASE)
    pos = torch.empty((s.N, 3), dtype=torch.float64, pin_memory=True)
    q = torch.empty((s.N,), dtype=torch.float64, pin_memory=True)
    pos.copy_(torch.as_tensor(s.pos))
    q.copy_(torch.as_tensor(s.q))
    Fout = torch.zeros((s.N, 3), dtype=torch.float64, pin_memory=True).numpy()
    outs = []
    with rbe.Context(s.box, s.alpha, 100, SEED, rbe.RBE_FP32_PHASE) as ctx:
        for _ in range(2):
            Fout[:] = np.nan
            Fh, Wh, Eh = rbe.rbe_kspace_forces_virial_host(ctx.h, pos.numpy(), q.numpy(), 7, Fout)
            outs.append((Fh.copy(), Wh.copy(), Eh.copy()))
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    Fh, Wh, Eh = outs[0]
    assert rel_rms_force(Fh, F) < 2e-6
    assert rel_frob(Wh, W) < 2e-6
    assert abs(Eh[0] - E[0]) < 2e-6 * abs(E[0])
    m, S = oracle.sample_k(s.box, s.alpha, 100, SEED, 7)
    Fo, Wo, Eko, Eso, _ = oracle.rbe_kspace(s.pos, s.q, s.box, s.alpha, m, S / 100)
    assert rel_rms_force(Fh, Fo) < 1e-5
    for a in range(3):
        assert abs(Wh[a, a] - Wo[a, a]) <= 1e-5 * np.abs(np.diag(Wo)).max()
    assert abs(Eh[0] - Eko) <= 1e-5 * abs(Eko)


@pytest.mark.parametrize("precision", [rbe.RBE_FP64, rbe.RBE_FP32_PHASE])
def test_bitwise_reproducible(precision):
    s = inputs.uniform_density(30000, P=300)
    a = _run(s, 300, 2, precision)
    b = _run(s, 300, 2, precision)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)


def test_nonzero_stream():
    import torch
    s = inputs.small_snapshot()
    ref = _run(s, s.P, 1, rbe.RBE_FP64)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        got = _run(s, s.P, 1, rbe.RBE_FP64)
    assert np.array_equal(ref[0], got[0])


def test_argument_errors():
    import torch
    dev = cuda_device()
    s = inputs.small_snapshot()
    with rbe.Context(s.box, s.alpha, s.P, 1) as ctx:
        pos = to_dev(s.pos)
        q = to_dev(s.q)
        F = torch.empty((s.N, 3), dtype=torch.float64, device=dev)
        lib = rbe._binding.load()
        host_pos = torch.as_tensor(s.pos)
        st = lib.rbe_kspace_forces_virial(ctx.h, s.N, rbe._binding.ctypes.c_void_p(host_pos.data_ptr()),
                                          rbe._binding._ptr(q), 0, rbe._binding._ptr(F), None, None)
        assert st == rbe.RBE_EINVAL
        with pytest.raises(rbe.RBEError) as e:
            ctx.forces_virial(pos, q, 1 << 56, F)
        assert e.value.status == rbe.RBE_EINVAL
        mis = torch.empty(3 * s.N + 1, dtype=torch.float64, device=dev)
        misaligned = rbe._binding.ctypes.c_void_p(mis.data_ptr() + 4)
        st = lib.rbe_kspace_forces_virial(ctx.h, s.N, misaligned, rbe._binding._ptr(q), 0,
                                          rbe._binding._ptr(F), None, None)
        assert st == rbe.RBE_EINVAL
        st = lib.rbe_kspace_forces_virial(ctx.h, -1, rbe._binding._ptr(pos), rbe._binding._ptr(q), 0,
                                          rbe._binding._ptr(F), None, None)
        assert st == rbe.RBE_EINVAL
    for bad in [dict(box=[10, 10, 0], alpha=1.0, P=10), dict(box=[10, 10, 10], alpha=0.0, P=10),
                dict(box=[10, 10, 10], alpha=1.0, P=0), dict(box=[0.01, 10, 10], alpha=1.0, P=10)]:
        with pytest.raises(rbe.RBEError) as e:
            rbe.rbe_create(bad["box"], bad["alpha"], bad["P"], 1)
        assert e.value.status == rbe.RBE_EINVAL


def test_nonfinite_input_is_reported():
    s = inputs.small_snapshot()
    pos = s.pos.copy()
    pos[17, 1] = np.nan
    with rbe.Context(s.box, s.alpha, s.P, 1, rbe.RBE_FP64) as ctx:
        with pytest.raises(rbe.RBEError) as e:
            ctx.forces_virial_host(pos, s.q, 0)
        assert e.value.status == rbe.RBE_ENONFINITE
        # the context stays usable and clean afterwards
        F, W, E = ctx.forces_virial_host(s.pos, s.q, 0)
        assert np.all(np.isfinite(F))


def test_water_charges_parity():
    """The 3000-molecule water charge set (9000 partial charges at 1 g/cm^3, alpha = 0.25,
    P = 100): FP64 path at 1e-10 and FP32-phase path at 1e-5 against the oracle on the same
    frequencies."""
    s = inputs.water()
    m, S = oracle.sample_k(s.box, s.alpha, s.P, SEED, 11)
    F0, W0, Ek0, Es0, _ = oracle.rbe_kspace(s.pos, s.q, s.box, s.alpha, m, S / s.P)
    F, W, E, _ = _run(s, s.P, 11, rbe.RBE_FP64)
    assert rel_max_force(F, F0) <= 1e-10
    assert rel_frob(W, W0) <= 1e-10
    assert abs(E[0] - Ek0) <= 1e-10 * abs(Ek0) and abs(E[1] - Es0) <= 1e-12 * abs(Es0)
    F, W, E, _ = _run(s, s.P, 11, rbe.RBE_FP32_PHASE)
    assert rel_rms_force(F, F0) <= 1e-5
    assert rel_frob(W, W0) <= 1e-5
    assert abs(E[0] - Ek0) <= 1e-5 * abs(Ek0)


def _xyzq(pos, q):
    import torch
    return to_dev(np.concatenate([pos, q[:, None]], axis=1).astype(np.float32))


@pytest.mark.parametrize("N,P", [(20000, 200), (5003, 517), (1, 64), (300000, 100)])
def test_xyzq_input(N, P):
    """float4 (x, y, z, q) input: bit for bit the evaluation of the float-rounded positions given
    as doubles, and within 1e-5 of the oracle fed the same float-rounded positions (the compute
    error); the rounding of the input itself is a separate, larger error.  (300000, 100) runs
    the wide two-frequency rho tiles on the float4 records."""
    import torch
    s = inputs.uniform_density(N, P=P)
    pos32, q32 = s.pos.astype(np.float32), s.q.astype(np.float32)
    pos_r, q_r = pos32.astype(np.float64), q32.astype(np.float64)
    dev = cuda_device()
    F = torch.full((N, 3), float("nan"), dtype=torch.float64, device=dev)
    W = torch.full((9,), float("nan"), dtype=torch.float64, device=dev)
    E = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    with rbe.Context(s.box, s.alpha, P, SEED, rbe.RBE_FP32_PHASE) as ctx:
        ctx.set_stream(torch.cuda.current_stream().cuda_stream)
        ctx.forces_virial_xyzq(_xyzq(s.pos, s.q), 4, F, W, E)
        ctx.sync()
    Fx, Wx, Ex = F.cpu().numpy(), W.cpu().numpy().reshape(3, 3), E.cpu().numpy()
    sr = inputs.System(pos_r, q_r, s.box, s.alpha, P, s.rc, "rounded")
    Fd, Wd, Ed, _ = _run(sr, P, 4, rbe.RBE_FP32_PHASE)
    assert np.array_equal(Fx, Fd) and np.array_equal(Wx, Wd) and np.array_equal(Ex, Ed)
    if N > 1:
        m, S = oracle.sample_k(s.box, s.alpha, P, SEED, 4)
        F0, W0, Ek0, _, _ = oracle.rbe_kspace(pos_r, q_r, s.box, s.alpha, m, S / P)
        assert rel_rms_force(Fx, F0) <= 1e-5
        assert rel_frob(Wx, W0) <= 1e-5
        assert abs(Ex[0] - Ek0) <= 1e-5 * abs(Ek0)


def test_xyzq_rejections():
    import torch
    dev = cuda_device()
    s = inputs.small_snapshot()
    F = torch.empty((s.N, 3), dtype=torch.float64, device=dev)
    buf = torch.zeros(4 * s.N + 4, dtype=torch.float32, device=dev)
    lib = rbe._binding.load()
    with rbe.Context(s.box, s.alpha, s.P, 1, rbe.RBE_FP64) as ctx:
        with pytest.raises(rbe.RBEError) as e:  # the FP64 path takes no float input
            ctx.forces_virial_xyzq(_xyzq(s.pos, s.q), 0, F)
        assert e.value.status == rbe.RBE_EINVAL
        ctx.set_precision(rbe.RBE_FP32_PHASE)
        st = lib.rbe_kspace_forces_virial_xyzq(ctx.h, s.N, rbe._binding.ctypes.c_void_p(buf.data_ptr() + 8), 0,
                                               rbe._binding._ptr(F), None, None)
        assert st == rbe.RBE_EINVAL  # 8 but not 16-byte aligned
        bad = np.concatenate([s.pos, s.q[:, None]], axis=1).astype(np.float32)
        bad[5, 2] = np.inf
        with pytest.raises(rbe.RBEError) as e:
            ctx.forces_virial_xyzq(to_dev(bad), 0, F)
            ctx.sync()
        assert e.value.status == rbe.RBE_ENONFINITE
