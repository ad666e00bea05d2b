"""GPU parity of the general-cell (triclinic) RBE k-space path (App. C) through the C ABI: forces,
virial and energy against the oracle's estimator on the oracle's own MH frequencies (so the
device chain draws the oracle's m: a different m moves the forces by O(1)), FP64 at 1e-10 and
FP32-phase at 1e-5, over several steps with the cell changing between them; a rectangular cell
through the general path equals the rectangular path; bad cells are rejected."""
import numpy as np
import pytest

import oracle
import paper_2110_14362_gb300 as rbe

from gpu_util import cuda_device

pytestmark = pytest.mark.gpu

ALPHA = 0.3


def _cell(step, base=(12.0, 13.0, 14.0), tilt=(2.5, -1.8, 3.1)):
    """An upper-triangular cell that shears a little more every step."""
    f = 1.0 + 0.01 * step
    return np.array([[base[0], tilt[0] * f, tilt[1] * f], [0.0, base[1], tilt[2] * f], [0.0, 0.0, base[2]]])


def _run(N, P, precision, steps=4, seed=17):
    import torch
    dev = cuda_device()
    rng = np.random.default_rng(N)
    s0 = rng.random((N, 3))
    q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    if N % 2:
        q[-1] = 0.5
    state = np.zeros((P, 3), dtype=np.int32)
    out = []
    with rbe.Context((12.0, 13.0, 14.0), ALPHA, P, seed, precision) as ctx:
        ctx.set_stream(torch.cuda.current_stream().cuda_stream)
        tq = torch.as_tensor(q).to(dev)
        for step in range(steps):
            h = _cell(step)
            pos = s0 @ h.T
            tp = torch.as_tensor(pos).to(dev)
            F = torch.empty((N, 3), dtype=torch.float64, device=dev)
            W = torch.empty(9, dtype=torch.float64, device=dev)
            E = torch.empty(2, dtype=torch.float64, device=dev)
            ctx.forces_virial_general(tp, tq, h, step, F, W, E)
            ctx.sync()
            m, S = oracle.gen_sample_k_mh(h, ALPHA, P, seed, step, state)
            F0, W0, Ek0, Es0 = oracle.gen_kspace(pos, q, h, ALPHA, m, S / P)
            out.append((F.cpu().numpy(), W.cpu().numpy().reshape(3, 3), E.cpu().numpy(), F0, W0, Ek0, Es0))
    return out


@pytest.mark.parametrize("N,P", [(1, 1), (257, 129), (3001, 500)])
def test_general_fp64_parity(N, P):
    for step, (F, W, E, F0, W0, Ek0, Es0) in enumerate(_run(N, P, rbe.RBE_FP64)):
        # a single charge's force is exactly zero in the oracle (Im(e^{-ik.r} rho) cancels) and
        # rounding on the device: an absolute floor far below any force of two charges
        assert np.abs(F - F0).max() < 1e-10 * np.abs(F0).max() + 1e-15, step
        assert np.linalg.norm(W - W0) < 1e-10 * np.linalg.norm(W0), step
        assert abs(E[0] - Ek0) < 1e-10 * abs(Ek0) and abs(E[1] - Es0) < 1e-12 * abs(Es0), step
        assert np.abs(W - W.T).max() == 0.0


def test_general_fp32_phase_parity():
    for step, (F, W, E, F0, W0, Ek0, Es0) in enumerate(_run(3001, 500, rbe.RBE_FP32_PHASE)):
        assert np.sqrt(np.mean((F - F0) ** 2) / np.mean(F0 ** 2)) < 1e-5, step
        assert np.linalg.norm(W - W0) < 1e-5 * np.linalg.norm(W0), step
        assert abs(E[0] - Ek0) < 1e-5 * abs(Ek0), step


def test_rectangular_cell_through_the_general_path():
    """A diagonal h: the product proposal is the target, every proposal is accepted, and the
    general path gives the rectangular path's forces, virial and energy (to rounding)."""
    import torch
    dev = cuda_device()
    N, P, box, seed = 2000, 200, (15.0, 16.0, 17.0), 9
    rng = np.random.default_rng(1)
    pos = rng.random((N, 3)) * np.array(box)
    q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    tp, tq = torch.as_tensor(pos).to(dev), torch.as_tensor(q).to(dev)
    with rbe.Context(box, ALPHA, P, seed, rbe.RBE_FP64) as ctx:
        ctx.set_stream(torch.cuda.current_stream().cuda_stream)
        for step in range(3):
            res = []
            for general in (False, True):
                F = torch.empty((N, 3), dtype=torch.float64, device=dev)
                W = torch.empty(9, dtype=torch.float64, device=dev)
                E = torch.empty(2, dtype=torch.float64, device=dev)
                if general:
                    ctx.forces_virial_general(tp, tq, np.diag(box), step, F, W, E)
                else:
                    ctx.forces_virial(tp, tq, step, F, W, E)
                ctx.sync()
                res.append((F.cpu().numpy(), W.cpu().numpy(), E.cpu().numpy()))
            (Fa, Wa, Ea), (Fb, Wb, Eb) = res
            assert np.abs(Fa - Fb).max() < 1e-11 * np.abs(Fa).max(), step
            assert np.abs(Wa - Wb).max() < 1e-11 * np.abs(Wa).max(), step
            assert abs(Ea[0] - Eb[0]) < 1e-11 * abs(Ea[0]), step


def test_general_rejects_bad_cells():
    import torch
    dev = cuda_device()
    with rbe.Context((10.0, 10.0, 10.0), ALPHA, 8, 1, rbe.RBE_FP64) as ctx:
        tp = torch.zeros((2, 3), dtype=torch.float64, device=dev)
        tq = torch.ones(2, dtype=torch.float64, device=dev)
        F = torch.empty((2, 3), dtype=torch.float64, device=dev)
        for h in (np.zeros((3, 3)), np.diag([10.0, 10.0, -10.0]), np.array([[10.0, 10.0, 0], [0, 0, 1.0], [0, 0, 10.0]]),
                  np.diag([10.0, np.nan, 10.0])):
            with pytest.raises(rbe.RBEError) as e:
                ctx.forces_virial_general(tp, tq, h, 0, F)
            assert e.value.status == rbe.RBE_EINVAL
