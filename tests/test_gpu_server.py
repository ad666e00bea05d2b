"""GPU tests of the serving loop (rbe_server_*): a replica's result does not depend on what
else is resident, graph replay equals direct launches, admission respects the memory budget,
and the served FP64 trajectory matches the oracle's NPT step (Sec. 3.2-3.3)."""
import sys
import time

import numpy as np
import pytest

import oracle
import paper_2110_14362_gb300 as rbe

from gpu_util import cuda_device

pytestmark = pytest.mark.gpu

ALPHA = 0.2
P = 100
DEADLINE_S = 300.0


def _system(n_side, seed, density=0.1):
    N = n_side ** 3
    L = (N / density) ** (1 / 3)
    rng = np.random.default_rng(seed)
    g = (np.arange(n_side) + 0.5) * (L / n_side)
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    pos = np.mod(pos + rng.uniform(-0.3, 0.3, pos.shape), L)
    q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    m = np.full(N, 20.0)
    mom = rng.normal(size=(N, 3)) * np.sqrt(oracle.KB * 300 * 100 * m)[:, None]
    return pos, mom, q, m, np.array([L, L, L])


SKIN = 0.0  # set per test: 0 = cell search every step, > 0 = neighbour list


def _base(box, rc=6.0):
    V0 = float(np.prod(box))
    return dict(dt=0.001, kT=oracle.KB * 300.0, P_ext=1.0 * oracle.BAR, gamma=10.0, gamma_V=2.0,
                M_V=oracle.piston_mass(0.5, 4.5e-5 / oracle.BAR, V0), rc=rc, qqr2e=oracle.QQR2E, lj_sigma=2.0,
                lj_eps=0.5, max_disp=0.05, kspace=1, real=1, noise=1, barostat=1)


def _dev_params(box):
    prm = rbe.NptParams(**_base(box))
    prm.skin = SKIN
    return prm


REQS = [  # (n_side, seed of the system, Philox seed, steps)
    (6, 1, 11, 9),
    (10, 2, 22, 14),
    (8, 3, 33, 7),
    (7, 4, 44, 12),
]


def _serve(reqs, precision, max_slots, chunk_steps=4, use_graphs=True, mem_budget=8 << 30, order=None):
    """Run `reqs` through one server; returns {index: (pos, mom, cell)} and the largest number
    of replicas seen resident at once."""
    cuda_device()
    srv = rbe.Server(ALPHA, P, precision, max_slots=max_slots, chunk_steps=chunk_steps,
                     mem_budget=mem_budget, use_graphs=use_graphs)
    try:
        ids = {}
        for i in (order if order is not None else range(len(reqs))):
            n_side, sseed, pseed, nsteps = reqs[i]
            pos, mom, q, m, box = _system(n_side, sseed)
            ids[i] = srv.submit(pos, mom, q, m, box, _dev_params(box), pseed, nsteps)
        t_end = time.monotonic() + DEADLINE_S
        peak = 0
        while True:
            nq, na, nd = srv.progress(wait=True)
            peak = max(peak, na)
            if nd == len(ids):
                break
            assert time.monotonic() < t_end, "serving loop did not finish"
        lat, steps, span = srv.stats()
        assert steps == sum(reqs[i][3] for i in ids)
        assert len(lat) == sum(-(-reqs[i][3] // chunk_steps) for i in ids)
        assert np.all(lat > 0) and span > 0
        return {i: srv.result(r) for i, r in ids.items()}, peak
    finally:
        srv.close()


def _direct(req, precision):
    n_side, sseed, pseed, nsteps = req
    pos, mom, q, m, box = _system(n_side, sseed)
    with rbe.Context(box, ALPHA, P, pseed, precision) as ctx:
        rep = rbe.NptReplica(pos, mom, q, m, box, _dev_params(box), cuda_device(), step=0)
        rep.init(ctx, batch=0)
        rep.step(ctx, nsteps)
        ctx.sync()
        r, p, F, L, cell = rep.state()
    return r, p, cell


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("precision", [rbe.RBE_FP64, rbe.RBE_FP32_PHASE])
def test_served_equals_direct_steps(precision):
    # chunks of 4 steps: graph replays for the whole chunks, direct launches for the tail
    out, _ = _serve(REQS[:2], precision, max_slots=2)
    for i in range(2):
        _same(out[i], _direct(REQS[i], precision))


@pytest.mark.parametrize("precision", [rbe.RBE_FP64, rbe.RBE_FP32_PHASE])
def test_alone_equals_mixed(precision):
    alone = {i: _serve([REQS[i]], precision, max_slots=1)[0][0] for i in (0, 2)}
    mixed, peak = _serve(REQS, precision, max_slots=4, order=[3, 0, 1, 2])
    assert peak >= 2
    for i in (0, 2):
        _same(mixed[i], alone[i])


def test_graphs_equal_direct_launches():
    a, _ = _serve(REQS, rbe.RBE_FP32_PHASE, max_slots=4, use_graphs=True)
    b, _ = _serve(REQS, rbe.RBE_FP32_PHASE, max_slots=4, use_graphs=False)
    for i in a:
        _same(a[i], b[i])


def test_budget_limits_residency():
    # the budget fits one replica of the largest request, not two
    big = max(r[0] ** 3 for r in REQS)
    one = big * 196 + (P + 1) * 32768 + (4 << 20)
    tight, peak = _serve(REQS, rbe.RBE_FP32_PHASE, max_slots=4, mem_budget=one + one // 2)
    assert peak == 1
    free, peak_free = _serve(REQS, rbe.RBE_FP32_PHASE, max_slots=4)
    assert peak_free >= 2
    for i in free:
        _same(tight[i], free[i])


def test_served_fp64_matches_oracle():
    req = REQS[0]
    out, _ = _serve([req], rbe.RBE_FP64, max_slots=1)
    r, p, cell = out[0]
    n_side, sseed, pseed, nsteps = req
    pos, mom, q, m, box = _system(n_side, sseed)
    prm = oracle.npt_params(alpha=ALPHA, P=P, seed=pseed, **_base(box))
    st = oracle.NptState(pos, mom, q, m, box)
    oracle.npt_forces(st, 0, prm)
    for s in range(nsteps):
        oracle.npt_step(st, s, prm)
    assert np.allclose(cell[:3], st.L, rtol=1e-12, atol=0)
    d = r - st.r
    d -= st.L * np.round(d / st.L)
    assert np.abs(d).max() < 1e-10 * st.L[0]
    assert np.abs(p - st.p).max() < 1e-10 * np.abs(st.p).max()


@pytest.mark.parametrize("precision", [rbe.RBE_FP64, rbe.RBE_FP32_PHASE])
def test_served_with_neighbour_lists(precision, monkeypatch):
    """With neighbour lists (rebuilt on the device when needed): served == direct steps and a
    request alone == the same request in a mix, bit for bit, as for the cell search."""
    monkeypatch.setattr(sys.modules[__name__], "SKIN", 0.5)
    mixed, _ = _serve(REQS, precision, max_slots=4, order=[3, 0, 1, 2])
    alone = _serve([REQS[1]], precision, max_slots=1)[0][0]
    _same(mixed[1], alone)
    _same(mixed[0], _direct(REQS[0], precision))


@pytest.mark.parametrize("kw", [dict(sampler=rbe.RBE_SAMPLER_MH, ptilde=40), dict(sampler=rbe.RBE_SAMPLER_OFFLINE),
                                dict(reuse=4, ptilde=20)])
def test_served_sampler_variants_equal_direct(kw):
    """A request carrying the paper's sampler variants (Sec. 4.3), a pressure batch or sample reuse
    is served bit for bit as the same settings stepped directly; a slot reused by requests with
    different settings (an MH chain after reuse and back) applies each request's own."""
    precision = rbe.RBE_FP32_PHASE
    cuda_device()
    srv = rbe.Server(ALPHA, P, precision, max_slots=1, chunk_steps=4, mem_budget=8 << 30, use_graphs=True)
    try:
        n_side, sseed, pseed, nsteps = REQS[0]
        pos, mom, q, m, box = _system(n_side, sseed)
        rid_plain = srv.submit(pos, mom, q, m, box, _dev_params(box), pseed, nsteps)
        rid = srv.submit(pos, mom, q, m, box, _dev_params(box), pseed, nsteps, **kw)
        rid_back = srv.submit(pos, mom, q, m, box, _dev_params(box), pseed, nsteps)
        while srv.progress(wait=True)[2] < 3:
            pass
        served = srv.result(rid)
        plain, back = srv.result(rid_plain), srv.result(rid_back)
    finally:
        srv.close()
    with rbe.Context(box, ALPHA, P, pseed, precision) as ctx:
        ctx.set_sampler(kw.get("sampler", rbe.RBE_SAMPLER_EXACT))
        ctx.set_pressure_batch(kw.get("ptilde", 0))
        ctx.set_sample_reuse(kw.get("reuse", 1))
        rep = rbe.NptReplica(pos, mom, q, m, box, _dev_params(box), cuda_device(), step=0)
        rep.init(ctx, batch=0)
        rep.step(ctx, nsteps)
        ctx.sync()
        r, p, F, L, cell = rep.state()
    _same(served, (r, p, cell))
    _same(plain, back)  # the settings did not leak into the next request
    assert not np.array_equal(served[1], plain[1])


def test_server_rejects_bad_sampling_settings():
    cuda_device()
    srv = rbe.Server(ALPHA, P, rbe.RBE_FP32_PHASE, max_slots=1, chunk_steps=4, mem_budget=8 << 30)
    try:
        pos, mom, q, m, box = _system(*REQS[0][:2])
        for kw in (dict(sampler=3), dict(ptilde=-1), dict(reuse=2000), dict(sampler=rbe.RBE_SAMPLER_MH, reuse=4)):
            with pytest.raises(rbe.RBEError) as e:
                srv.submit(pos, mom, q, m, box, _dev_params(box), 1, 4, **kw)
            assert e.value.status == rbe.RBE_EINVAL
    finally:
        srv.close()


def _run_until_done(srv, n, t_end):
    while True:
        nq, na, nd = srv.progress(wait=True)
        if nd == n:
            return
        assert time.monotonic() < t_end, "serving loop did not finish"


@pytest.mark.parametrize("precision", [rbe.RBE_FP64, rbe.RBE_FP32_PHASE])
def test_nonfinite_request_is_evicted_and_the_others_run_on(precision):
    """A request whose host positions hold a NaN latches RBE_ENONFINITE on its replica's device
    status word; the server reads it after the first chunk, evicts that replica with the error
    as its result, and the three good requests resident beside it end bit for bit as when each
    runs alone (its direct steps)."""
    cuda_device()
    srv = rbe.Server(ALPHA, P, precision, max_slots=4, chunk_steps=4, mem_budget=8 << 30)
    try:
        ids = {}
        for i, (n_side, sseed, pseed, nsteps) in enumerate(REQS):
            pos, mom, q, m, box = _system(n_side, sseed)
            if i == 2:
                pos = pos.copy()
                pos[5, 1] = np.nan
            ids[i] = srv.submit(pos, mom, q, m, box, _dev_params(box), pseed, nsteps)
        _run_until_done(srv, len(ids), time.monotonic() + DEADLINE_S)
        assert srv.state(ids[2]) == (3, rbe.RBE_ENONFINITE)
        with pytest.raises(rbe.RBEError) as e:
            srv.result(ids[2])
        assert e.value.status == rbe.RBE_ENONFINITE
        lat, steps, _ = srv.stats()
        good = [0, 1, 3]
        # the bad replica ran one chunk and left
        assert len(lat) == sum(-(-REQS[i][3] // 4) for i in good) + 1
        for i in good:
            assert srv.state(ids[i]) == (2, rbe.RBE_OK)
            _same(srv.result(ids[i]), _direct(REQS[i], precision))
    finally:
        srv.close()


def test_cancel_queued_and_resident_requests():
    """rbe_server_cancel takes a queued request out of the queue at once and a resident one out
    of its slot at the end of its chunk in flight; cancelled requests report RBE_ESTATE, the
    freed slot serves a later request, and the requests that ran are bit for bit their direct
    steps."""
    cuda_device()
    precision = rbe.RBE_FP32_PHASE
    srv = rbe.Server(ALPHA, P, precision, max_slots=2, chunk_steps=4, mem_budget=8 << 30)
    try:
        def submit(i):
            n_side, sseed, pseed, nsteps = REQS[i]
            pos, mom, q, m, box = _system(n_side, sseed)
            return srv.submit(pos, mom, q, m, box, _dev_params(box), pseed, nsteps)
        a, b, c = submit(0), submit(1), submit(3)
        srv.progress(wait=False)  # a and b resident with a chunk in flight, c queued
        assert srv.state(a)[0] == 1 and srv.state(b)[0] == 1 and srv.state(c)[0] == 0
        srv.cancel(c)
        srv.cancel(b)
        assert srv.state(c) == (4, rbe.RBE_ESTATE)
        d = submit(2)  # takes b's slot once b has left
        _run_until_done(srv, 4, time.monotonic() + DEADLINE_S)
        for rid in (b, c):
            assert srv.state(rid) == (4, rbe.RBE_ESTATE)
            with pytest.raises(rbe.RBEError) as e:
                srv.result(rid)
            assert e.value.status == rbe.RBE_ESTATE
        with pytest.raises(rbe.RBEError) as e:
            srv.cancel(a)  # finished
        assert e.value.status == rbe.RBE_ESTATE
        _same(srv.result(a), _direct(REQS[0], precision))
        _same(srv.result(d), _direct(REQS[2], precision))
    finally:
        srv.close()


def _serve_lockstep(idx, max_slots, chunk_steps=4, nan_in=None, batched=1):
    """Run requests REQS[idx] through a server of lockstep groups (the batched k-space); returns
    {i: result or the RBEError}, the chunk count and the steps done."""
    cuda_device()
    srv = rbe.Server(ALPHA, P, rbe.RBE_FP32_PHASE, max_slots=max_slots, chunk_steps=chunk_steps,
                     mem_budget=8 << 30, batched=batched)
    try:
        ids = {}
        for i in idx:
            n_side, sseed, pseed, nsteps = REQS[i]
            pos, mom, q, m, box = _system(n_side, sseed)
            if i == nan_in:
                pos = pos.copy()
                pos[3, 0] = np.nan
            ids[i] = srv.submit(pos, mom, q, m, box, _dev_params(box), pseed, nsteps)
        _run_until_done(srv, len(ids), time.monotonic() + DEADLINE_S)
        out = {}
        for i, rid in ids.items():
            try:
                out[i] = srv.result(rid)
            except rbe.RBEError as e:
                out[i] = e
        lat, steps, _ = srv.stats()
        return out, len(lat), steps
    finally:
        srv.close()


def test_lockstep_group_alone_equals_in_the_group():
    """Lockstep serving (every step's k-space of the resident replicas in one persistent
    batched launch, the group captured as one CUDA graph once it is stable): each replica ends
    bit for bit as when it is served alone, whatever the other members and the chunking they
    impose; the steps are all done."""
    mix, nchunks, steps = _serve_lockstep([0, 1, 2, 3], max_slots=4)
    assert steps == sum(r[3] for r in REQS)
    for i in range(4):
        alone, _, _ = _serve_lockstep([i], max_slots=1)
        _same(mix[i], alone[i])


def test_lockstep_close_to_direct_steps():
    """The batched k-space tiles its sums differently from the single-system path, so a
    lockstep-served trajectory agrees with the replica's direct steps to FP32 rounding only:
    positions within 1e-6 A, momenta within 1e-5 relative.  The box moves by the integrated
    virial, which each FP32-phase evaluation gives within 1e-5 relative, so the two boxes'
    displacements from the common initial box agree within 2e-5 of the displacement."""
    out, _, _ = _serve_lockstep([0, 1], max_slots=2)
    for i in range(2):
        r, p, cell = out[i]
        r0, p0, cell0 = _direct(REQS[i], rbe.RBE_FP32_PHASE)
        box_init = _system(REQS[i][0], REQS[i][1])[4]
        assert np.max(np.abs(r - r0)) < 1e-6
        assert np.max(np.abs(p - p0)) <= 1e-5 * np.max(np.abs(p0))
        assert np.all(np.abs(cell[:3] - cell0[:3]) <= 2e-5 * np.abs(cell0[:3] - box_init) + 1e-12 * cell0[:3])


def test_lockstep_nonfinite_member_is_evicted():
    """A NaN in one member's positions is latched in that replica's own status word (the
    batched k-space writes each item's errors to its context), so only that replica fails
    (RBE_ENONFINITE) while the others end bit for bit as when served alone."""
    out, _, _ = _serve_lockstep([0, 1, 2, 3], max_slots=4, nan_in=1)
    assert isinstance(out[1], rbe.RBEError) and out[1].status == rbe.RBE_ENONFINITE
    for i in (0, 2, 3):
        alone, _, _ = _serve_lockstep([i], max_slots=1)
        _same(out[i], alone[i])


def test_lockstep_autotuned_tiles():
    """With the tiles autotuned on the first captured group (batched = 2) every request still
    completes and stays within FP32 rounding of its direct steps."""
    out, _, steps = _serve_lockstep([0, 1, 2, 3], max_slots=4, batched=2)
    assert steps == sum(r[3] for r in REQS)
    for i in range(4):
        r, p, cell = out[i]
        r0, p0, cell0 = _direct(REQS[i], rbe.RBE_FP32_PHASE)
        assert np.max(np.abs(r - r0)) < 1e-6
