"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/rbe.h declares; argument errors are reported before any device work."""
import ctypes
import os
import re

import pytest

import paper_2110_14362_gb300 as rbe
from paper_2110_14362_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(rbe_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = _build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert {"rbe_create", "rbe_sample_k", "rbe_kspace_forces_virial"} <= declared
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    bound = {name for name, _, _ in rbe._binding.SIGNATURES}
    assert declared <= bound, declared - bound


def test_argument_validation_without_gpu():
    lib = rbe.load()
    h = ctypes.c_void_p()
    box = (ctypes.c_double * 3)(10.0, 10.0, 10.0)
    assert lib.rbe_create(box, -1.0, 10, 1, ctypes.byref(h)) == rbe.RBE_EINVAL
    assert lib.rbe_create(box, 1.0, 0, 1, ctypes.byref(h)) == rbe.RBE_EINVAL
    assert lib.rbe_create(box, 1.0, 70000, 1, ctypes.byref(h)) == rbe.RBE_EINVAL
    bad = (ctypes.c_double * 3)(10.0, float("nan"), 10.0)
    assert lib.rbe_create(bad, 1.0, 10, 1, ctypes.byref(h)) == rbe.RBE_EINVAL
    tiny = (ctypes.c_double * 3)(0.05, 10.0, 10.0)
    assert lib.rbe_create(tiny, 1.0, 10, 1, ctypes.byref(h)) == rbe.RBE_EINVAL
    assert b"600" in lib.rbe_last_error(None)
    assert lib.rbe_create(box, 1.0, 10, 1, None) == rbe.RBE_EINVAL
    assert lib.rbe_sync(None) == rbe.RBE_EINVAL
    assert lib.rbe_destroy(None) == rbe.RBE_OK
    assert lib.rbe_measure_pipe(7, 10, None) == rbe.RBE_EINVAL
    for st in range(8):
        assert lib.rbe_status_string(st).startswith(b"RBE_")
    # the sampler, pressure-batch, reuse and general-cell entries refuse a NULL context
    assert lib.rbe_set_sampler(None, rbe.RBE_SAMPLER_MH) == rbe.RBE_EINVAL
    assert lib.rbe_set_pressure_batch(None, 10) == rbe.RBE_EINVAL
    assert lib.rbe_set_sample_reuse(None, 4) == rbe.RBE_EINVAL
    cell = (ctypes.c_double * 9)(10.0, 0, 0, 0, 10.0, 0, 0, 0, 10.0)
    assert lib.rbe_kspace_forces_virial_general(None, 0, None, None, cell, 0, None, None, None) == rbe.RBE_EINVAL
    assert lib.rbe_flex_init(None, None, 0) == rbe.RBE_EINVAL
    assert lib.rbe_water_init(None, None, None, 0) == rbe.RBE_EINVAL
    assert lib.rbe_water_step(None, None, None, 1) == rbe.RBE_EINVAL
    assert lib.rbe_flex_step(None, None, 1) == rbe.RBE_EINVAL
    # the batch's tile setters refuse a NULL batch (or a NULL output) before any device work
    f = ctypes.c_int32()
    assert lib.rbe_batch_set_rho_f(None, 2) == rbe.RBE_EINVAL
    assert lib.rbe_batch_get_rho_f(None, ctypes.byref(f)) == rbe.RBE_EINVAL
    assert lib.rbe_batch_set_tiles(None, 64, 256, 512) == rbe.RBE_EINVAL


def test_python_binding_raises_without_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("checks the no-GPU behaviour")
    with pytest.raises(rbe.RBEError) as e:
        rbe.Context([10.0, 10.0, 10.0], 1.0, 10, 1)
    assert e.value.status == rbe.RBE_ECUDA
