"""Parity at the large-N sizes of the precision and roofline sweep: N in {1e6, 4e6} uniform +-1
charges at 0.1 per A^3 (alpha = 0.2), P in {100, 2000}, against the oracle.

The oracle evaluates rho(k) over every particle (its OpenMP build: the same sums as the
single-thread build, shared among the host cores), from which the virial and the energies
follow exactly, and the forces of a seeded subset of 10^4 particles (each row the bits of the
full estimator).  Bounds: FP32-phase path, every rho accumulation: forces RMS(dF)/RMS(F) <=
1e-5 on the subset, rho RMS(d rho)/RMS(rho) <= 1e-5, each diagonal virial entry within 1e-5 of
the largest, E_k within 1e-5; FP64 path: forces max|dF|/RMS(F) <= 1e-10, rho, virial and E_k
within 1e-10.  The FP32-phase contexts run in the benchmark's launch configuration (the
current stream, the library's own plan for this N and P)."""
import functools

import numpy as np
import pytest

import oracle
import paper_2110_14362_gb300 as rbe
from paper_2110_14362_gb300 import inputs

from gpu_util import cuda_device, rel_max_force, rel_rms_force, to_dev

pytestmark = pytest.mark.gpu

SEED, STEP, NSUB = 12345, 5, 10_000
CASES = [(1_000_000, 100), (1_000_000, 2000), (4_000_000, 100), (4_000_000, 2000)]


@functools.lru_cache(maxsize=4)
def _reference(N, P):
    s = inputs.uniform_density(N, P=P)
    m, S = oracle.sample_k(s.box, s.alpha, P, SEED, STEP)
    idx = np.sort(np.random.default_rng(N + 7 * P).choice(N, NSUB, replace=False))
    F0, W0, Ek0, Es0, rho0 = oracle.rbe_kspace_subset(s.pos, s.q, s.box, s.alpha, m, S / P, idx, all_cores=True)
    return s, m, idx, F0, W0, Ek0, Es0, rho0


@functools.lru_cache(maxsize=1)
def _device_inputs(N, P):
    s = _reference(N, P)[0]
    return to_dev(s.pos), to_dev(s.q)


def _gpu(N, P, precision, accum):
    import torch
    s = _reference(N, P)[0]
    pos, q = _device_inputs(N, P)
    dev = cuda_device()
    F = torch.full((N, 3), float("nan"), dtype=torch.float64, device=dev)
    W = torch.full((9,), float("nan"), dtype=torch.float64, device=dev)
    E = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    with rbe.Context(s.box, s.alpha, P, SEED, precision, accum,
                     stream=torch.cuda.current_stream().cuda_stream) as ctx:
        m, _ = ctx.sample_k(STEP)
        ctx.forces_virial(pos, q, STEP, F, W, E)
        ctx.sync()
        rho = ctx.rho()
    return m, F.cpu().numpy(), W.cpu().numpy().reshape(3, 3), E.cpu().numpy(), rho


def _rel_rms(a, b):
    return np.sqrt(np.mean(np.abs(a - b) ** 2) / np.mean(np.abs(b) ** 2))


@pytest.mark.parametrize("accum", [rbe.RBE_RHO_COMP32, rbe.RBE_RHO_FP32, rbe.RBE_RHO_FP64])
@pytest.mark.parametrize("N,P", CASES)
def test_fp32_phase_large_against_oracle(N, P, accum):
    s, m0, idx, F0, W0, Ek0, Es0, rho0 = _reference(N, P)
    m, F, W, E, rho = _gpu(N, P, rbe.RBE_FP32_PHASE, accum)
    assert np.array_equal(m, m0)
    assert rel_rms_force(F[idx], F0) <= 1e-5
    assert _rel_rms(rho, rho0) <= 1e-5
    for a in range(3):  # Pxx, Pyy, Pzz separately
        assert abs(W[a, a] - W0[a, a]) <= 1e-5 * np.abs(np.diag(W0)).max()
    assert abs(E[0] - Ek0) <= 1e-5 * abs(Ek0)
    assert abs(E[1] - Es0) <= 1e-12 * abs(Es0)


@pytest.mark.parametrize("N,P", [(1_000_000, 2000), (4_000_000, 2000)])
def test_fp64_large_against_oracle(N, P):
    s, m0, idx, F0, W0, Ek0, Es0, rho0 = _reference(N, P)
    _, F, W, E, rho = _gpu(N, P, rbe.RBE_FP64, rbe.RBE_RHO_COMP32)
    assert rel_max_force(F[idx], F0) <= 1e-10
    assert np.max(np.abs(rho - rho0)) <= 1e-10 * np.max(np.abs(rho0))
    assert np.max(np.abs(W - W0)) <= 1e-10 * np.abs(W0).max()
    assert abs(E[0] - Ek0) <= 1e-10 * abs(Ek0)


def test_xyzq_large_against_oracle():
    """float32 (x, y, z, q) input at N = 1e6, P = 2000: within 1e-5 of the oracle fed the same
    float-rounded positions (the compute error); the error of the rounding itself (the oracle on
    the rounded positions against the oracle on the FP64 ones) is reported, not bounded here."""
    import torch
    N, P = 1_000_000, 2000
    s, m0, idx, F0, W0, Ek0, Es0, rho0 = _reference(N, P)
    pos_r = s.pos.astype(np.float32).astype(np.float64)
    Fr, Wr, Ekr, Esr, rhor = oracle.rbe_kspace_subset(pos_r, s.q, s.box, s.alpha, m0, S_of(s, P) / P, idx,
                                                      all_cores=True)
    dev = cuda_device()
    F = torch.full((N, 3), float("nan"), dtype=torch.float64, device=dev)
    W = torch.full((9,), float("nan"), dtype=torch.float64, device=dev)
    E = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    xyzq = to_dev(np.concatenate([s.pos, s.q[:, None]], axis=1).astype(np.float32))
    with rbe.Context(s.box, s.alpha, P, SEED, rbe.RBE_FP32_PHASE,
                     stream=torch.cuda.current_stream().cuda_stream) as ctx:
        ctx.forces_virial_xyzq(xyzq, STEP, F, W, E)
        ctx.sync()
        rho = ctx.rho()
    F, W, E = F.cpu().numpy(), W.cpu().numpy().reshape(3, 3), E.cpu().numpy()
    assert rel_rms_force(F[idx], Fr) <= 1e-5
    assert _rel_rms(rho, rhor) <= 1e-5
    for a in range(3):
        assert abs(W[a, a] - Wr[a, a]) <= 1e-5 * np.abs(np.diag(Wr)).max()
    assert abs(E[0] - Ekr) <= 1e-5 * abs(Ekr)
    print(f"input rounding error: forces {rel_rms_force(Fr, F0):.2e}, rho {_rel_rms(rhor, rho0):.2e}; "
          f"compute error: forces {rel_rms_force(F[idx], Fr):.2e}")


def S_of(s, P):
    return oracle.sample_k(s.box, s.alpha, P, SEED, STEP)[1]
