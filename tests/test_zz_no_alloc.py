"""The allocation-free sampler, for callers that cannot allocate device memory when they
need a batch (an engine with a fixed device pool, a plugin inside an application that owns
all device memory, a loop where a device allocation would synchronise the device).

It must draw exactly the batch of the regular entry point, rbe_sample_k, whose samples are
bit-exact against the oracle; the tolerance for sampled frequencies is zero.  Two calls in a
row check that the shared fixed scratch carries nothing from one call into the next.  This
file is collected last so that a run stopping at the first failure has run every other test.
"""
import math

import numpy as np
import pytest

import paper_2110_14362_gb300 as rbe

from gpu_util import cuda_device

pytestmark = pytest.mark.gpu

CASES = [  # two calls in a row with different boxes, sizes and steps
    ((80.0, 80.0, 120.0), 0.2, 200, 12345, 7),
    ((10.0, 11.0, 9.0), 1.0, 300, 99, 1 << 40),
]


def _regular(box, alpha, P, seed, step):
    h = rbe.rbe_create(box, alpha, P, seed)
    try:
        return rbe.rbe_sample_k(h, step, P)
    finally:
        rbe.rbe_destroy(h)


def test_noalloc_matches_regular_sampler_twice():
    import torch
    dev = cuda_device()
    stream = torch.cuda.current_stream(dev).cuda_stream
    for box, alpha, P, seed, step in CASES:
        m = torch.full((P, 3), -99999, dtype=torch.int32, device=dev)
        S = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        rbe.rbe_sample_k_noalloc(box, alpha, P, seed, step, m, S, stream)
        m_ref, S_ref = _regular(box, alpha, P, seed, step)
        assert np.array_equal(m.cpu().numpy(), m_ref)
        assert S.item() == S_ref


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    dev = cuda_device()
    m = torch.zeros((4, 3), dtype=torch.int32, device=dev)
    S = torch.zeros((1,), dtype=torch.float64, device=dev)
    with pytest.raises(rbe.RBEError) as e:
        rbe.rbe_sample_k_noalloc((5000.0, 10.0, 10.0), 1.0, 4, 1, 0, m, S)
    assert e.value.status == rbe.RBE_EINVAL and "fixed scratch" in str(e.value)


def _edge_for_M(M: float, alpha: float) -> float:
    """Box edge whose table truncation ceil(sqrt(60 ln2 / c)), c = pi^2 / (alpha l^2), lies
    halfway between M - 1 and M."""
    return (M - 0.5) * math.pi / math.sqrt(60.0 * math.log(2.0) * alpha)


def test_noalloc_at_its_largest_table_and_one_beyond():
    """The largest table the fixed scratch accepts (|m| <= 4094 on one axis) draws the same
    frequencies as rbe_sample_k, bit for bit; one entry more is rejected with RBE_EINVAL."""
    import torch
    dev = cuda_device()
    alpha, P, seed, step = 1.0, 96, 7, 3
    edge = _edge_for_M(4094, alpha)
    c = math.pi ** 2 / (alpha * edge * edge)
    assert math.ceil(math.sqrt(60.0 * math.log(2.0) / c)) == 4094
    box = (edge, 10.0, 12.0)
    m = torch.full((P, 3), -99999, dtype=torch.int32, device=dev)
    S = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
    rbe.rbe_sample_k_noalloc(box, alpha, P, seed, step, m, S, torch.cuda.current_stream(dev).cuda_stream)
    m_ref, S_ref = _regular(box, alpha, P, seed, step)
    assert np.array_equal(m.cpu().numpy(), m_ref)
    assert S.item() == S_ref
    with pytest.raises(rbe.RBEError) as e:
        rbe.rbe_sample_k_noalloc((_edge_for_M(4095, alpha), 10.0, 12.0), alpha, P, seed, step, m, S)
    assert e.value.status == rbe.RBE_EINVAL and "fixed scratch" in str(e.value)
