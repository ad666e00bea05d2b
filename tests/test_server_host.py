"""Host-side logic of the serving loop (rbe_server_*): configuration and request validation,
the memory-budget rejection and the result-state errors.  None of these calls reaches the
GPU: submission only copies the request into the host queue."""
import ctypes

import numpy as np
import pytest

import paper_2110_14362_gb300 as rbe
from paper_2110_14362_gb300 import _binding as b


def _cfg(**kw):
    base = dict(alpha=0.2, P=100, precision=rbe.RBE_FP32_PHASE, max_slots=4, chunk_steps=10,
                mem_budget=1 << 30, use_graphs=1, batched=0)
    base.update(kw)
    return b.ServerConfig(**base)


def _create(cfg):
    h = ctypes.c_void_p()
    st = b.load().rbe_server_create(ctypes.byref(cfg), ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("bad", [dict(alpha=0.0), dict(P=0), dict(max_slots=0), dict(max_slots=5000),
                                 dict(chunk_steps=0), dict(mem_budget=0), dict(precision=7),
                                 dict(batched=3), dict(batched=1, precision=rbe.RBE_FP64)])
def test_config_rejected(bad):
    st, h = _create(_cfg(**bad))
    assert st == rbe.RBE_EINVAL
    assert not h.value


def _request(N=64, nsteps=5, box=(20.0, 20.0, 20.0)):
    rng = np.random.default_rng(1)
    arrs = dict(pos=rng.uniform(0, 20, (N, 3)), mom=np.zeros((N, 3)), q=np.ones(N), m=np.full(N, 10.0))
    req = b.Request(N=N, pos=arrs["pos"].ctypes.data, mom=arrs["mom"].ctypes.data, charge=arrs["q"].ctypes.data,
                    mass=arrs["m"].ctypes.data, box=(ctypes.c_double * 3)(*box), pV=0.0, seed=3, nsteps=nsteps,
                    pad=0, params=rbe.NptParams(dt=0.001, rc=5.0, kspace=1, real=1))
    return req, arrs


def test_submit_validation_and_budget():
    lib = b.load()
    st, h = _create(_cfg(mem_budget=64 << 20))
    assert st == rbe.RBE_OK
    try:
        rid = ctypes.c_int64(-1)
        req, keep = _request()
        assert lib.rbe_server_submit(h, ctypes.byref(req), ctypes.byref(rid)) == rbe.RBE_OK
        assert rid.value == 0
        assert lib.rbe_server_submit(h, ctypes.byref(req), ctypes.byref(rid)) == rbe.RBE_OK
        assert rid.value == 1
        # a request that alone needs more than the budget is refused at submission
        big, keep2 = _request(N=1_000_000)
        assert lib.rbe_server_submit(h, ctypes.byref(big), ctypes.byref(rid)) == rbe.RBE_ENOMEM
        assert b"budget" in lib.rbe_server_last_error(h)
        for bad in (dict(nsteps=0), dict(box=(20.0, 0.0, 20.0))):
            r2, keep3 = _request(**bad)
            assert lib.rbe_server_submit(h, ctypes.byref(r2), ctypes.byref(rid)) == rbe.RBE_EINVAL
        r3, keep4 = _request()
        r3.pos = None
        assert lib.rbe_server_submit(h, ctypes.byref(r3), ctypes.byref(rid)) == rbe.RBE_EINVAL
        # results: unknown ids and unfinished requests
        out = np.zeros(64 * 3)
        dp = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        assert lib.rbe_server_result(h, 5, dp, None, None) == rbe.RBE_EINVAL
        assert lib.rbe_server_result(h, 0, dp, None, None) == rbe.RBE_ESTATE
        n, steps, span = ctypes.c_int64(-1), ctypes.c_int64(-1), ctypes.c_double(-1)
        assert lib.rbe_server_stats(h, None, 0, ctypes.byref(n), ctypes.byref(steps), ctypes.byref(span)) == 0
        assert (n.value, steps.value, span.value) == (0, 0, 0.0)
    finally:
        lib.rbe_server_destroy(h)


def test_null_arguments():
    lib = b.load()
    rid = ctypes.c_int64()
    assert lib.rbe_server_create(None, None) == rbe.RBE_EINVAL
    assert lib.rbe_server_submit(None, None, ctypes.byref(rid)) == rbe.RBE_EINVAL
    assert lib.rbe_server_progress(None, 0, None, None, None) == rbe.RBE_EINVAL
    assert lib.rbe_server_destroy(None) == rbe.RBE_OK
    assert lib.rbe_server_last_error(None) == b""


def test_cancel_queued_request_on_the_host():
    """Cancelling a queued request is host logic: it leaves the queue, counts as done, reports
    state 4 with RBE_ESTATE, its result is RBE_ESTATE, and a second cancel is refused; the other
    queued request is untouched."""
    lib = b.load()
    st, h = _create(_cfg())
    assert st == rbe.RBE_OK
    try:
        rid = ctypes.c_int64(-1)
        req, keep = _request()
        assert lib.rbe_server_submit(h, ctypes.byref(req), ctypes.byref(rid)) == rbe.RBE_OK
        assert lib.rbe_server_submit(h, ctypes.byref(req), ctypes.byref(rid)) == rbe.RBE_OK
        state, err = ctypes.c_int32(-1), ctypes.c_int(-1)
        assert lib.rbe_server_request_state(h, 0, ctypes.byref(state), ctypes.byref(err)) == rbe.RBE_OK
        assert (state.value, err.value) == (0, rbe.RBE_OK)
        assert lib.rbe_server_cancel(h, 0) == rbe.RBE_OK
        assert lib.rbe_server_request_state(h, 0, ctypes.byref(state), ctypes.byref(err)) == rbe.RBE_OK
        assert (state.value, err.value) == (4, rbe.RBE_ESTATE)
        assert lib.rbe_server_result(h, 0, None, None, None) == rbe.RBE_ESTATE
        assert b"cancelled" in lib.rbe_server_last_error(h)
        assert lib.rbe_server_cancel(h, 0) == rbe.RBE_ESTATE
        assert lib.rbe_server_request_state(h, 1, ctypes.byref(state), None) == rbe.RBE_OK and state.value == 0
        assert lib.rbe_server_cancel(h, 9) == rbe.RBE_EINVAL
        assert lib.rbe_server_request_state(h, 9, None, None) == rbe.RBE_EINVAL
    finally:
        lib.rbe_server_destroy(h)
