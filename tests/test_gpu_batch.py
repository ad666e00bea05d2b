"""GPU tests of the batched k-space evaluation (rbe_batch_*, the batched form of Sec. 4.2):
every item against the FP64 oracle on the same Philox-drawn frequencies (FP32-phase bound
1e-5), against the single-system path, alone versus in a mix (bitwise), over tile shapes,
after autotuning, and replayed from a captured CUDA graph."""
import numpy as np
import pytest

import oracle
import paper_2110_14362_gb300 as rbe
from paper_2110_14362_gb300 import inputs

from gpu_util import cuda_device, to_dev, rel_rms_force, rel_frob

pytestmark = pytest.mark.gpu

ALPHA = 0.2
SIZES = [1, 2, 127, 1000, 3001, 20000]  # N = 1 carries q = 0 (odd N)


def _systems(sizes, seed0=0, step0=0):
    out = []
    for k, N in enumerate(sizes):
        L = (max(N, 8) / 0.1) ** (1 / 3)
        box = np.array([L, 0.9 * L, 1.1 * L])
        pos, q = inputs.uniform_pm1(N, box, seed0 + k)
        out.append(dict(N=N, pos_h=pos, q_h=q, box=box, seed=1000 + seed0 + k, step=step0 + 3 * k))
    return out


def _dev(systems):
    import torch
    dev = cuda_device()
    items = []
    for sy in systems:
        items.append(dict(pos=to_dev(sy["pos_h"]), q=to_dev(sy["q_h"]),
                          F=torch.zeros((sy["N"], 3), dtype=torch.float64, device=dev),
                          W=torch.zeros(9, dtype=torch.float64, device=dev),
                          E=torch.zeros(2, dtype=torch.float64, device=dev),
                          box=sy["box"], seed=sy["seed"], step=sy["step"]))
    return items


def _out(it):
    return it["F"].cpu().numpy(), it["W"].cpu().numpy(), it["E"].cpu().numpy()


def _oracle(sy, P):
    m, S = oracle.sample_k(sy["box"], ALPHA, P, sy["seed"], sy["step"])
    return oracle.rbe_kspace(sy["pos_h"], sy["q_h"], sy["box"], ALPHA, m, S / P)


def _check_vs_oracle(F, W, E, ref, tol=1e-5):
    Fo, Wo, Eo = ref[0], ref[1], (ref[2], ref[3])
    scale = np.sqrt(np.mean(Fo ** 2)) + 1e-300
    assert np.sqrt(np.mean((F - Fo) ** 2)) <= tol * scale + 1e-12
    assert np.linalg.norm(W - Wo.reshape(-1)) <= tol * np.linalg.norm(Wo) + 1e-12
    assert abs(E[0] - Eo[0]) <= tol * abs(Eo[0]) + 1e-12
    assert abs(E[1] - Eo[1]) <= 1e-6 * abs(Eo[1]) + 1e-12


@pytest.mark.parametrize("P", [100, 257])
def test_batched_matches_oracle(P):
    systems = _systems(SIZES)
    items = _dev(systems)
    with rbe.Batch(ALPHA, P, len(items), 100.0) as b:
        b.evaluate(items)
        b.sync()
    for sy, it in zip(systems, items):
        _check_vs_oracle(*_out(it), _oracle(sy, P))


def test_batched_vs_single_system():
    systems = _systems([500, 4000, 20000], seed0=7)
    items = _dev(systems)
    P = 200
    with rbe.Batch(ALPHA, P, 3, 100.0) as b:
        b.evaluate(items)
        b.sync()
    for sy, it in zip(systems, items):
        F, W, E = _out(it)
        import torch
        F1t = torch.zeros_like(it["F"])
        W1t = torch.zeros_like(it["W"])
        with rbe.Context(sy["box"], ALPHA, P, sy["seed"], rbe.RBE_FP32_PHASE) as ctx:
            ctx.forces_virial(it["pos"], it["q"], sy["step"], F1t, W1t)
            ctx.sync()
        F1, W1 = F1t.cpu().numpy(), W1t.cpu().numpy()
        assert rel_rms_force(F, F1) < 2e-6
        assert rel_frob(W, W1) < 2e-6


def test_item_alone_equals_in_mix():
    systems = _systems([3001, 20000, 127, 1000, 2], seed0=3)
    mix = _dev(systems)
    alone = _dev([systems[1]])
    with rbe.Batch(ALPHA, 100, 8, 100.0) as b:
        b.set_tiles(128, 256, 256)
        b.evaluate(mix)
        b.evaluate(alone)
        b.sync()
    for a, c in zip(_out(alone[0]), _out(mix[1])):
        assert np.array_equal(a, c)


@pytest.mark.parametrize("tiles", [(32, 64, 128), (64, 100, 384), (128, 2048, 1024), (256, 33, 128),
                                   (50, 64, 128), (75, 256, 256), (16, 100, 128), (150, 1000, 512)])
def test_tile_shapes(tiles):
    systems = _systems([1, 999, 5000], seed0=11)
    ref = _dev(systems)
    cur = _dev(systems)
    with rbe.Batch(ALPHA, 150, 3, 100.0) as b:
        b.evaluate(ref)
        b.set_tiles(*tiles)
        assert b.tiles() == tiles
        b.evaluate(cur)
        b.sync()
    for sy, r, c in zip(systems, ref, cur):
        F0, W0, _ = _out(r)
        F1, W1, E1 = _out(c)
        if np.abs(F0).max() > 0:  # the N = 1 item has q = 0 and zero force
            assert rel_rms_force(F1, F0) < 2e-6
        _check_vs_oracle(F1, W1, E1, _oracle(sy, 150))


@pytest.mark.parametrize("tiles", [(50, 64, 128), (64, 256, 256), (16, 100, 128), (38, 512, 384), (128, 33, 128)])
def test_two_frequencies_per_lane(tiles):
    """Rho tiles whose lanes hold two frequencies each (a tile of rho_k lanes covers 2 rho_k
    frequencies; P = 150 leaves ragged tiles) agree with the one-frequency tiles and the oracle,
    and an item's result is the same alone and in a mix."""
    systems = _systems([1, 999, 5000, 20000], seed0=13)
    ref = _dev(systems)
    cur = _dev(systems)
    alone = _dev([systems[2]])
    with rbe.Batch(ALPHA, 150, 4, 100.0) as b:
        b.evaluate(ref)
        b.set_tiles(*tiles)
        b.set_rho_f(2)
        assert b.rho_f() == 2 and b.tiles() == tiles
        b.evaluate(cur)
        b.evaluate(alone)
        b.set_persistent(False)
        per_pass = _dev([systems[2]])
        b.evaluate(per_pass)
        b.sync()
    for a, c, d in zip(_out(alone[0]), _out(cur[2]), _out(per_pass[0])):
        assert np.array_equal(a, c)
        assert np.array_equal(a, d)
    for sy, r, c in zip(systems, ref, cur):
        F0, W0, _ = _out(r)
        F1, W1, E1 = _out(c)
        if np.abs(F0).max() > 0:
            assert rel_rms_force(F1, F0) < 2e-6
        _check_vs_oracle(F1, W1, E1, _oracle(sy, 150))


def test_autotune_then_evaluate():
    systems = _systems([1000, 2000, 8000, 30000], seed0=5)
    items = _dev(systems)
    with rbe.Batch(ALPHA, 100, 4, 100.0) as b:
        ms = b.autotune(items, reps=2)
        assert ms > 0
        k, c, f = b.tiles()
        assert 16 <= k <= 256 and c >= 32 and f % 128 == 0
        b.evaluate(items)
        b.sync()
    for sy, it in zip(systems, items):
        _check_vs_oracle(*_out(it), _oracle(sy, 100))


def test_graph_capture_replay():
    import torch
    systems = _systems([700, 4000, 9000], seed0=21)
    items = _dev(systems)
    s = torch.cuda.Stream()
    with rbe.Batch(ALPHA, 100, 3, 100.0, stream=s.cuda_stream) as b:
        arr = b.items(items)
        b.evaluate(arr)
        b.sync()
        direct = [_out(it) for it in items]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            b.evaluate(arr)
        for it in items:
            it["F"].zero_()
            it["W"].zero_()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        b.sync()
    for d, it in zip(direct, items):
        for a, c in zip(d, _out(it)):
            assert np.array_equal(a, c)


def test_batch_argument_errors():
    systems = _systems([10, 20])
    items = _dev(systems)
    with rbe.Batch(ALPHA, 64, 2, 50.0) as b:
        for bad in ((8, 64, 128), (257, 64, 128), (64, 16, 128), (64, 64, 100)):
            with pytest.raises(rbe.RBEError) as e:
                b.set_tiles(*bad)
            assert e.value.status == rbe.RBE_EINVAL
        for bad in (0, 3, -1):
            with pytest.raises(rbe.RBEError) as e:
                b.set_rho_f(bad)
            assert e.value.status == rbe.RBE_EINVAL
        b.set_rho_f(2)
        b.set_tiles(0, 0, 0)  # the defaults: one frequency per lane
        assert b.rho_f() == 1
        arr = b.items(items)
        arr[0].N = 0
        with pytest.raises(rbe.RBEError):
            b.evaluate(arr)
        arr = b.items(items)
        arr[1].box[2] = 80.0  # beyond max_box's tables
        with pytest.raises(rbe.RBEError):
            b.evaluate(arr)
        arr = b.items(items * 2)  # more than max_items
        with pytest.raises(rbe.RBEError):
            b.evaluate(arr)
        b.evaluate(items)  # still usable
        b.sync()


def test_persistent_launch_equals_one_launch_per_pass():
    """The persistent form (one cooperative launch whose resident blocks run the five passes
    with grid barriers between them) and one launch per pass run the same tile bodies on the same
    work lists: every output is the same bits."""
    systems = _systems([5, 1000, 4001, 20000], seed0=31)
    a = _dev(systems)
    c = _dev(systems)
    with rbe.Batch(ALPHA, 100, 4, 100.0) as b:
        b.set_tiles(128, 512, 512)
        b.evaluate(a)
        b.set_persistent(False)
        b.evaluate(c)
        b.sync()
    for x, y in zip(a, c):
        for u, v in zip(_out(x), _out(y)):
            assert np.array_equal(u, v)


def test_device_resident_box_and_step():
    """Items whose box and batch index live in device memory (box_dev, step_dev: an NPT
    replica's cell block) give the bits of items that pass the same values from the host, and a
    graph captured once follows new device values at replay."""
    import torch
    dev = cuda_device()
    systems = _systems([800, 6000], seed0=41)
    host_items = _dev(systems)
    dev_items = _dev(systems)
    for it in dev_items:
        it["box_dev"] = torch.as_tensor(np.asarray(it["box"], dtype=np.float64)).to(dev)
        it["step_dev"] = torch.tensor([it["step"]], dtype=torch.int64, device=dev)
        it["box"] = [99.0, 99.0, 99.0]  # the host box only bounds the table size check now
        it["step"] = 7777
    s = torch.cuda.Stream()
    with rbe.Batch(ALPHA, 100, 2, 100.0, stream=s.cuda_stream) as b:
        b.evaluate(host_items)
        arr = b.items(dev_items)
        b.evaluate(arr)
        b.sync()
        for x, y in zip(host_items, dev_items):
            for u, v in zip(_out(x), _out(y)):
                assert np.array_equal(u, v)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            b.evaluate(arr)
        # new boxes and indices on the device; the replay reads them
        new_box = [np.asarray(sy["box"]) * 1.03 for sy in systems]
        for it, nb in zip(dev_items, new_box):
            it["box_dev"].copy_(torch.as_tensor(nb))
            it["step_dev"].add_(5)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        b.sync()
    for sy, it, nb in zip(systems, dev_items, new_box):
        moved = dict(sy, box=nb, step=sy["step"] + 5)
        _check_vs_oracle(*_out(it), _oracle(moved, 100))


def test_persistent_barrier_timeout_is_reported_and_recovered():
    """The failure path of the persistent launch, without a fault: the test hook makes every
    grid barrier wait for one block more than the grid has, so each wait runs out after its
    one-second limit, the blocks leave the kernel and rbe_batch_sync reports RBE_ETIMEOUT; with
    the hook off the next evaluation on the same batch is complete and equals the one before."""
    import time
    systems = _systems([900, 5000], seed0=51)
    ref = _dev(systems)
    cur = _dev(systems)
    with rbe.Batch(ALPHA, 100, 2, 100.0) as b:
        b.evaluate(ref)
        b.sync()
        b.test_barrier_timeout(True)
        t0 = time.monotonic()
        b.evaluate(cur)
        with pytest.raises(rbe.RBEError) as e:
            b.sync()
        assert e.value.status == rbe.RBE_ETIMEOUT
        assert time.monotonic() - t0 < 30.0
        b.test_barrier_timeout(False)
        b.evaluate(cur)
        b.sync()
    for x, y in zip(ref, cur):
        for u, v in zip(_out(x), _out(y)):
            assert np.array_equal(u, v)
