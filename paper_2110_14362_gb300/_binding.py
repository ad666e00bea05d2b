"""ctypes binding of librbe.so (the C ABI in include/rbe.h).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels.  Functions carry the C names; ``Context`` wraps a handle for convenience.
Device buffers are passed as torch CUDA tensors (their data pointers); host buffers as
NumPy arrays.  If the library is missing or fails to load, every call raises -- there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

from . import _build

RBE_OK, RBE_EINVAL, RBE_ENOMEM, RBE_ECUDA, RBE_ETIMEOUT, RBE_ENONFINITE, RBE_ESTATE, RBE_ESAMPLE = range(8)
RBE_FP64, RBE_FP32_PHASE = 0, 1
RBE_RHO_FP64, RBE_RHO_COMP32, RBE_RHO_FP32 = 0, 1, 2
RBE_SAMPLER_EXACT, RBE_SAMPLER_OFFLINE, RBE_SAMPLER_MH = 0, 1, 2

_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)

class NptParams(ctypes.Structure):
    """rbe_npt_params (include/rbe.h)."""
    _fields_ = [("dt", ctypes.c_double), ("kT", ctypes.c_double), ("P_ext", ctypes.c_double),
                ("gamma", ctypes.c_double), ("gamma_V", ctypes.c_double), ("M_V", ctypes.c_double),
                ("rc", ctypes.c_double), ("qqr2e", ctypes.c_double), ("lj_sigma", ctypes.c_double),
                ("lj_eps", ctypes.c_double), ("max_disp", ctypes.c_double), ("kspace", ctypes.c_int32),
                ("real", ctypes.c_int32), ("noise", ctypes.c_int32), ("barostat", ctypes.c_int32),
                ("skin", ctypes.c_double), ("M_cell", ctypes.c_double * 3), ("gamma0", ctypes.c_double)]

    def __init__(self, **kw):
        if "M_cell" in kw and not isinstance(kw["M_cell"], ctypes.Array):
            kw["M_cell"] = (ctypes.c_double * 3)(*[float(x) for x in kw["M_cell"]])
        super().__init__(**kw)


class System(ctypes.Structure):
    """rbe_system (include/rbe.h): device pointers of one replica, the next step index and
    the NPT parameters."""
    _fields_ = [("N", ctypes.c_int64), ("pos", ctypes.c_void_p), ("mom", ctypes.c_void_p),
                ("force", ctypes.c_void_p), ("charge", ctypes.c_void_p), ("mass", ctypes.c_void_p),
                ("cell", ctypes.c_void_p), ("step", ctypes.c_uint64), ("params", NptParams)]


class FlexParams(ctypes.Structure):
    """rbe_flex_params (include/rbe.h): the fully flexible cell."""
    _fields_ = [("dt", ctypes.c_double), ("kT", ctypes.c_double), ("P_ext", ctypes.c_double),
                ("gamma", ctypes.c_double), ("gamma_h", ctypes.c_double), ("M", ctypes.c_double * 9),
                ("rc", ctypes.c_double), ("qqr2e", ctypes.c_double), ("lj_sigma", ctypes.c_double),
                ("lj_eps", ctypes.c_double), ("max_disp", ctypes.c_double), ("chi", ctypes.c_double),
                ("kspace", ctypes.c_int32), ("real", ctypes.c_int32), ("noise", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("skin", ctypes.c_double)]

    def __init__(self, **kw):
        if "M" in kw and not isinstance(kw["M"], ctypes.Array):
            kw["M"] = (ctypes.c_double * 9)(*[float(x) for x in np.asarray(kw["M"], dtype=np.float64).reshape(9)])
        super().__init__(**kw)


class FlexSystem(ctypes.Structure):
    """rbe_flex_system (include/rbe.h)."""
    _fields_ = [("N", ctypes.c_int64), ("pos", ctypes.c_void_p), ("mom", ctypes.c_void_p),
                ("force", ctypes.c_void_p), ("charge", ctypes.c_void_p), ("mass", ctypes.c_void_p),
                ("cell", ctypes.c_void_p), ("step", ctypes.c_uint64), ("params", FlexParams)]


class WaterParams(ctypes.Structure):
    """rbe_water_params (include/rbe.h): the rigid 3-site water constraints."""
    _fields_ = [("d_OH", ctypes.c_double), ("d_HH", ctypes.c_double), ("shake_tol", ctypes.c_double),
                ("shake_max_iter", ctypes.c_int32), ("pad", ctypes.c_int32)]


def water_params(d_OH: float = 1.0, angle_deg: float = 109.47, shake_tol: float = 1e-14,
                 shake_max_iter: int = 500) -> WaterParams:
    """O-H length and H-O-H angle (the H-H length follows), SHAKE tolerance and sweep limit."""
    return WaterParams(d_OH=d_OH, d_HH=2.0 * d_OH * math.sin(math.radians(angle_deg) / 2.0), shake_tol=shake_tol,
                       shake_max_iter=shake_max_iter, pad=0)


CELL_EXCL = 25  # rigid water: the exclusion energy in the cell block

RBE_FLEX_CELL_DOUBLES = 64
# slots of the flexible cell block (include/rbe.h)
FLEX_H, FLEX_PH, FLEX_W, FLEX_KT, FLEX_PT = 0, 9, 18, 27, 36
FLEX_EK, FLEX_EC, FLEX_EL, FLEX_V, FLEX_HAM, FLEX_STEP, FLEX_BUILDS = 45, 46, 47, 48, 49, 50, 51

RBE_CELL_DOUBLES = 32
RBE_BAROSTAT_NONE, RBE_BAROSTAT_ISO, RBE_BAROSTAT_ANISO, RBE_BAROSTAT_SEMI = 0, 1, 2, 3
# slots of the cell block (include/rbe.h)
CELL_PC, CELL_WD, CELL_K2D, CELL_PD = 12, 16, 19, 22


class BatchItem(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("pos", ctypes.c_void_p), ("charge", ctypes.c_void_p),
                ("forces", ctypes.c_void_p), ("virial", ctypes.c_void_p), ("energy", ctypes.c_void_p),
                ("box", ctypes.c_double * 3), ("seed", ctypes.c_uint64), ("step", ctypes.c_uint64),
                ("box_dev", ctypes.c_void_p), ("step_dev", ctypes.c_void_p), ("status_dev", ctypes.c_void_p)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("P", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("max_slots", ctypes.c_int32), ("chunk_steps", ctypes.c_int32), ("mem_budget", ctypes.c_int64),
                ("use_graphs", ctypes.c_int32), ("batched", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("pos", ctypes.c_void_p), ("mom", ctypes.c_void_p),
                ("charge", ctypes.c_void_p), ("mass", ctypes.c_void_p), ("box", ctypes.c_double * 3),
                ("pV", ctypes.c_double), ("seed", ctypes.c_uint64), ("nsteps", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("params", NptParams), ("pc", ctypes.c_double * 3),
                ("sampler", ctypes.c_int32), ("ptilde", ctypes.c_int32), ("reuse", ctypes.c_int32),
                ("pad2", ctypes.c_int32)]

# (name, restype, argtypes) of every exported symbol
SIGNATURES = [
    ("rbe_create", ctypes.c_int, [_dp, ctypes.c_double, ctypes.c_int32, ctypes.c_uint64, ctypes.POINTER(_vp)]),
    ("rbe_destroy", ctypes.c_int, [_vp]),
    ("rbe_set_stream", ctypes.c_int, [_vp, _vp]),
    ("rbe_set_precision", ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32]),
    ("rbe_set_sampler", ctypes.c_int, [_vp, ctypes.c_int32]),
    ("rbe_set_pressure_batch", ctypes.c_int, [_vp, ctypes.c_int32]),
    ("rbe_set_sample_reuse", ctypes.c_int, [_vp, ctypes.c_int32]),
    ("rbe_kspace_forces_virial_general", ctypes.c_int, [_vp, ctypes.c_int64, _vp, _vp, _dp, ctypes.c_uint64, _vp, _vp,
                                                        _vp]),
    ("rbe_set_seed", ctypes.c_int, [_vp, ctypes.c_uint64]),
    ("rbe_set_box", ctypes.c_int, [_vp, _dp]),
    ("rbe_sample_k", ctypes.c_int, [_vp, ctypes.c_uint64, _ip, _dp]),
    ("rbe_kspace_forces_virial", ctypes.c_int, [_vp, ctypes.c_int64, _vp, _vp, ctypes.c_uint64, _vp, _vp, _vp]),
    ("rbe_kspace_forces_virial_xyzq", ctypes.c_int, [_vp, ctypes.c_int64, _vp, ctypes.c_uint64, _vp, _vp, _vp]),
    ("rbe_kspace_forces_virial_host", ctypes.c_int,
     [_vp, ctypes.c_int64, _dp, _dp, ctypes.c_uint64, _dp, _dp, _dp]),
    ("rbe_kspace_weighted", ctypes.c_int,
     [_vp, ctypes.c_int64, _vp, _vp, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp]),
    ("rbe_get_rho", ctypes.c_int, [_vp, _dp, ctypes.c_int32]),
    ("rbe_sync", ctypes.c_int, [_vp]),
    ("rbe_set_kernel_timing", ctypes.c_int, [_vp, ctypes.c_int32]),
    ("rbe_get_kernel_times", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_float)]),
    ("rbe_measure_pipe", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _dp]),
    ("rbe_sample_k_noalloc", ctypes.c_int,
     [_dp, ctypes.c_double, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, _vp, _vp, _vp]),
    ("rbe_npt_init", ctypes.c_int, [_vp, ctypes.POINTER(System), ctypes.c_uint64]),
    ("rbe_npt_step", ctypes.c_int, [_vp, ctypes.POINTER(System), ctypes.c_int32]),
    ("rbe_water_init", ctypes.c_int, [_vp, ctypes.POINTER(System), ctypes.POINTER(WaterParams), ctypes.c_uint64]),
    ("rbe_water_step", ctypes.c_int, [_vp, ctypes.POINTER(System), ctypes.POINTER(WaterParams), ctypes.c_int32]),
    ("rbe_flex_init", ctypes.c_int, [_vp, ctypes.POINTER(FlexSystem), ctypes.c_uint64]),
    ("rbe_flex_step", ctypes.c_int, [_vp, ctypes.POINTER(FlexSystem), ctypes.c_int32]),
    ("rbe_batch_create", ctypes.c_int, [ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                        ctypes.POINTER(_vp)]),
    ("rbe_batch_destroy", ctypes.c_int, [_vp]),
    ("rbe_batch_set_stream", ctypes.c_int, [_vp, _vp]),
    ("rbe_batch_set_tiles", ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    ("rbe_batch_set_rho_f", ctypes.c_int, [_vp, ctypes.c_int32]),
    ("rbe_batch_get_rho_f", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32)]),
    ("rbe_batch_set_persistent", ctypes.c_int, [_vp, ctypes.c_int32]),
    ("rbe_batch_test_barrier_timeout", ctypes.c_int, [_vp, ctypes.c_int32]),
    ("rbe_batch_get_tiles", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int32)]),
    ("rbe_kspace_forces_virial_batched", ctypes.c_int, [_vp, ctypes.POINTER(BatchItem), ctypes.c_int32]),
    ("rbe_batch_autotune", ctypes.c_int, [_vp, ctypes.POINTER(BatchItem), ctypes.c_int32, ctypes.c_int32, _dp]),
    ("rbe_batch_sync", ctypes.c_int, [_vp]),
    ("rbe_batch_last_error", ctypes.c_char_p, [_vp]),
    ("rbe_server_create", ctypes.c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(_vp)]),
    ("rbe_server_destroy", ctypes.c_int, [_vp]),
    ("rbe_server_submit", ctypes.c_int, [_vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_int64)]),
    ("rbe_server_progress", ctypes.c_int, [_vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]),
    ("rbe_server_result", ctypes.c_int, [_vp, ctypes.c_int64, _dp, _dp, _dp]),
    ("rbe_server_cancel", ctypes.c_int, [_vp, ctypes.c_int64]),
    ("rbe_server_request_state", ctypes.c_int, [_vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                                ctypes.POINTER(ctypes.c_int)]),
    ("rbe_server_stats", ctypes.c_int, [_vp, _dp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64), _dp]),
    ("rbe_server_last_error", ctypes.c_char_p, [_vp]),
    ("rbe_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("rbe_last_error", ctypes.c_char_p, [_vp]),
    ("rbe_version", ctypes.c_int32, []),
]


class RBEError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(message)
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load librbe.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"librbe.so not found at {path}: build it with __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(st: int, ctx=None):
    if st != RBE_OK:
        lib = load()
        msg = lib.rbe_last_error(ctx).decode() if lib.rbe_last_error(ctx) else ""
        raise RBEError(st, f"{lib.rbe_status_string(st).decode()}: {msg}")


def _ptr(t):
    """Device pointer of a torch tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


# ---------------------------------------------------------------------------------
# Functions with the C names.

def rbe_create(box, alpha: float, P: int, seed: int):
    lib = load()
    b = _host(box, np.float64).reshape(3)
    h = ctypes.c_void_p()
    _check(lib.rbe_create(b.ctypes.data_as(_dp), float(alpha), int(P), int(seed), ctypes.byref(h)))
    return h


def rbe_destroy(h):
    load().rbe_destroy(h)


def rbe_set_stream(h, stream_handle: int):
    _check(load().rbe_set_stream(h, ctypes.c_void_p(stream_handle)), h)


def rbe_set_precision(h, precision: int, rho_accum: int = RBE_RHO_COMP32):
    _check(load().rbe_set_precision(h, int(precision), int(rho_accum)), h)


def rbe_set_sampler(h, sampler: int):
    _check(load().rbe_set_sampler(h, int(sampler)), h)


def rbe_set_pressure_batch(h, Ptilde: int):
    _check(load().rbe_set_pressure_batch(h, int(Ptilde)), h)


def rbe_set_sample_reuse(h, M: int):
    _check(load().rbe_set_sample_reuse(h, int(M)), h)


def rbe_set_seed(h, seed: int):
    _check(load().rbe_set_seed(h, int(seed)), h)


def rbe_set_box(h, box):
    b = _host(box, np.float64).reshape(3)
    _check(load().rbe_set_box(h, b.ctypes.data_as(_dp)), h)


def rbe_sample_k(h, step: int, P: int):
    m = np.zeros((P, 3), dtype=np.int32)
    S = ctypes.c_double(0.0)
    _check(load().rbe_sample_k(h, int(step), m.ctypes.data_as(_ip), ctypes.byref(S)), h)
    return m, S.value


def rbe_kspace_forces_virial(h, positions, charges, step: int, forces_out, virial_out=None, energy_out=None):
    N = int(charges.shape[0])
    _check(load().rbe_kspace_forces_virial(h, N, _ptr(positions), _ptr(charges), int(step), _ptr(forces_out),
                                           _ptr(virial_out), _ptr(energy_out)), h)


def rbe_kspace_forces_virial_xyzq(h, xyzq, step: int, forces_out, virial_out=None, energy_out=None):
    """Evaluation on float32 positions and charges: xyzq a torch float32 CUDA tensor (N, 4)."""
    import torch
    if xyzq.dtype != torch.float32 or xyzq.dim() != 2 or xyzq.shape[1] != 4:
        raise ValueError("xyzq must be a float32 tensor of shape (N, 4)")
    N = int(xyzq.shape[0])
    _check(load().rbe_kspace_forces_virial_xyzq(h, N, _ptr(xyzq), int(step), _ptr(forces_out), _ptr(virial_out),
                                                _ptr(energy_out)), h)


def rbe_kspace_forces_virial_host(h, positions, charges, step: int, forces_out=None):
    pos = _host(positions, np.float64)
    q = _host(charges, np.float64)
    N = int(q.shape[0])
    F = np.zeros((N, 3)) if forces_out is None else forces_out
    W = np.zeros(9)
    E = np.zeros(2)
    _check(load().rbe_kspace_forces_virial_host(h, N, pos.ctypes.data_as(_dp), q.ctypes.data_as(_dp), int(step),
                                                F.ctypes.data_as(_dp), W.ctypes.data_as(_dp),
                                                E.ctypes.data_as(_dp)), h)
    return F, W.reshape(3, 3), E


def rbe_kspace_weighted(h, positions, charges, m, weights, forces_out, virial_out=None, energy_out=None):
    N = int(charges.shape[0])
    K = int(weights.shape[0])
    _check(load().rbe_kspace_weighted(h, N, _ptr(positions), _ptr(charges), K, _ptr(m), _ptr(weights),
                                      _ptr(forces_out), _ptr(virial_out), _ptr(energy_out)), h)


def rbe_get_rho(h, K: int):
    out = np.zeros(2 * K)
    _check(load().rbe_get_rho(h, out.ctypes.data_as(_dp), 2 * K), h)
    return out[0::2] + 1j * out[1::2]


def rbe_sync(h):
    _check(load().rbe_sync(h), h)


def rbe_set_kernel_timing(h, enable: bool):
    _check(load().rbe_set_kernel_timing(h, int(bool(enable))), h)


def rbe_get_kernel_times(h):
    out = (ctypes.c_float * 4)()
    _check(load().rbe_get_kernel_times(h, out), h)
    return list(out)


def rbe_measure_pipe(kind: int, iters: int = 4096) -> float:
    v = ctypes.c_double(0.0)
    _check(load().rbe_measure_pipe(int(kind), int(iters), ctypes.byref(v)))
    return v.value


def rbe_sample_k_noalloc(box, alpha: float, P: int, seed: int, step: int, m_out, S_out, stream_handle: int = 0):
    """Allocation-free sampling into caller device buffers: m_out a torch int32 tensor of at
    least 3 P elements, S_out a float64 tensor of at least one, both contiguous and on one CUDA
    device; the call runs with that device current."""
    import torch
    if m_out.dtype != torch.int32 or m_out.numel() < 3 * int(P):
        raise ValueError("m_out must be an int32 tensor of at least 3 P elements")
    if S_out.dtype != torch.float64 or S_out.numel() < 1:
        raise ValueError("S_out must be a float64 tensor of at least one element")
    if not (m_out.is_cuda and S_out.is_cuda) or m_out.device != S_out.device:
        raise ValueError("m_out and S_out must be CUDA tensors on the same device")
    b = _host(box, np.float64).reshape(3)
    with torch.cuda.device(m_out.device):
        _check(load().rbe_sample_k_noalloc(b.ctypes.data_as(_dp), float(alpha), int(P), int(seed), int(step),
                                           _ptr(m_out), _ptr(S_out), ctypes.c_void_p(stream_handle)))


def rbe_npt_init(h, sys_: "System", batch: int):
    _check(load().rbe_npt_init(h, ctypes.byref(sys_), int(batch)), h)


def rbe_npt_step(h, sys_: "System", nsteps: int):
    _check(load().rbe_npt_step(h, ctypes.byref(sys_), int(nsteps)), h)


class NptReplica:
    """One device-resident NPT replica: torch CUDA tensors for r, p, F, q, m and the cell
    block, and the rbe_system that points at them."""

    def __init__(self, pos, mom, charge, mass, box, params: NptParams, device, step: int = 0, pV: float = 0.0,
                 pc=(0.0, 0.0, 0.0)):
        import torch
        f64 = torch.float64
        self.pos = torch.as_tensor(np.ascontiguousarray(pos), dtype=f64).to(device).contiguous()
        self.mom = torch.as_tensor(np.ascontiguousarray(mom), dtype=f64).to(device).contiguous()
        self.force = torch.zeros_like(self.pos)
        self.charge = torch.as_tensor(np.ascontiguousarray(charge), dtype=f64).to(device).contiguous()
        self.mass = torch.as_tensor(np.ascontiguousarray(mass), dtype=f64).to(device).contiguous()
        cell = np.zeros(RBE_CELL_DOUBLES)
        cell[:3] = np.asarray(box, dtype=np.float64).reshape(3)
        cell[3] = pV
        cell[CELL_PC:CELL_PC + 3] = np.asarray(pc, dtype=np.float64).reshape(3)
        self.cell = torch.as_tensor(cell).to(device).contiguous()
        self.sys = System(N=int(self.charge.shape[0]), pos=self.pos.data_ptr(), mom=self.mom.data_ptr(),
                          force=self.force.data_ptr(), charge=self.charge.data_ptr(), mass=self.mass.data_ptr(),
                          cell=self.cell.data_ptr(), step=int(step), params=params)

    def init(self, ctx: "Context", batch: int | None = None):
        rbe_npt_init(ctx.h, self.sys, self.sys.step if batch is None else batch)

    def step(self, ctx: "Context", nsteps: int = 1):
        rbe_npt_step(ctx.h, self.sys, nsteps)

    def state(self):
        """(pos, mom, force, box, cell block) as NumPy arrays (synchronises)."""
        c = self.cell.cpu().numpy()
        return (self.pos.cpu().numpy(), self.mom.cpu().numpy(), self.force.cpu().numpy(), c[:3].copy(), c)


def rbe_water_init(h, sys_: "System", wp: WaterParams, batch: int):
    _check(load().rbe_water_init(h, ctypes.byref(sys_), ctypes.byref(wp), int(batch)), h)


def rbe_water_step(h, sys_: "System", wp: WaterParams, nsteps: int):
    _check(load().rbe_water_step(h, ctypes.byref(sys_), ctypes.byref(wp), int(nsteps)), h)


class WaterReplica(NptReplica):
    """A device-resident rigid-water system (sites O, H, H per molecule) on the NPT replica's
    buffers, stepped by rbe_water_init / rbe_water_step."""

    def __init__(self, pos, mom, charge, mass, box, params: NptParams, device, wp: WaterParams | None = None,
                 step: int = 0, pV: float = 0.0):
        super().__init__(pos, mom, charge, mass, box, params, device, step=step, pV=pV)
        self.wp = wp if wp is not None else water_params()

    def init(self, ctx: "Context", batch: int | None = None):
        rbe_water_init(ctx.h, self.sys, self.wp, self.sys.step if batch is None else batch)

    def step(self, ctx: "Context", nsteps: int = 1):
        rbe_water_step(ctx.h, self.sys, self.wp, nsteps)


def rbe_flex_init(h, sys_: "FlexSystem", batch: int):
    _check(load().rbe_flex_init(h, ctypes.byref(sys_), int(batch)), h)


def rbe_flex_step(h, sys_: "FlexSystem", nsteps: int):
    _check(load().rbe_flex_step(h, ctypes.byref(sys_), int(nsteps)), h)


class FlexReplica:
    """One device-resident replica with a fully flexible cell: torch CUDA tensors for r, p, F, q,
    m and the cell block (h and p^h row-major, the cell vectors as the columns of h), and the
    rbe_flex_system that points at them."""

    def __init__(self, pos, mom, charge, mass, h, params: FlexParams, device, step: int = 0, ph=None):
        import torch
        f64 = torch.float64
        self.pos = torch.as_tensor(np.ascontiguousarray(pos), dtype=f64).to(device).contiguous()
        self.mom = torch.as_tensor(np.ascontiguousarray(mom), dtype=f64).to(device).contiguous()
        self.force = torch.zeros_like(self.pos)
        self.charge = torch.as_tensor(np.ascontiguousarray(charge), dtype=f64).to(device).contiguous()
        self.mass = torch.as_tensor(np.ascontiguousarray(mass), dtype=f64).to(device).contiguous()
        cell = np.zeros(RBE_FLEX_CELL_DOUBLES)
        cell[FLEX_H:FLEX_H + 9] = np.asarray(h, dtype=np.float64).reshape(9)
        if ph is not None:
            cell[FLEX_PH:FLEX_PH + 9] = np.asarray(ph, dtype=np.float64).reshape(9)
        self.cell = torch.as_tensor(cell).to(device).contiguous()
        self.sys = FlexSystem(N=int(self.charge.shape[0]), pos=self.pos.data_ptr(), mom=self.mom.data_ptr(),
                              force=self.force.data_ptr(), charge=self.charge.data_ptr(), mass=self.mass.data_ptr(),
                              cell=self.cell.data_ptr(), step=int(step), params=params)

    def init(self, ctx: "Context", batch: int | None = None):
        rbe_flex_init(ctx.h, self.sys, self.sys.step if batch is None else batch)

    def step(self, ctx: "Context", nsteps: int = 1):
        rbe_flex_step(ctx.h, self.sys, nsteps)

    def state(self):
        """dict of NumPy arrays: r, p, F, h, ph, W, Kt, Pt (3x3), Ek, Ec, El, V, H, the step index and the
        neighbour-list builds so far (synchronises)."""
        c = self.cell.cpu().numpy()
        m = lambda o: c[o:o + 9].reshape(3, 3).copy()  # noqa: E731
        return {"r": self.pos.cpu().numpy(), "p": self.mom.cpu().numpy(), "F": self.force.cpu().numpy(),
                "h": m(FLEX_H), "ph": m(FLEX_PH), "W": m(FLEX_W), "Kt": m(FLEX_KT), "Pt": m(FLEX_PT),
                "Ek": c[FLEX_EK], "Ec": c[FLEX_EC], "El": c[FLEX_EL], "V": c[FLEX_V], "H": c[FLEX_HAM],
                "step": int(c[FLEX_STEP:FLEX_STEP + 1].view(np.int64)[0]), "builds": int(c[FLEX_BUILDS])}


class Batch:
    """Batched k-space evaluation of many systems (rbe_batch_*): FP32-phase path, persistent
    work-list kernels, tile shapes set by hand or by the autotuner."""

    def __init__(self, alpha: float, P: int, max_items: int, max_box: float, stream=None):
        lib = load()
        self.h = ctypes.c_void_p()
        st = lib.rbe_batch_create(float(alpha), int(P), int(max_items), float(max_box), ctypes.byref(self.h))
        if st != RBE_OK:
            raise RBEError(st, lib.rbe_last_error(None).decode())
        self.P = int(P)
        if stream is not None:
            self._check(lib.rbe_batch_set_stream(self.h, stream))

    def _check(self, st):
        if st != RBE_OK:
            lib = load()
            raise RBEError(st, f"{lib.rbe_status_string(st).decode()}: {lib.rbe_batch_last_error(self.h).decode()}")

    def close(self):
        if self.h:
            load().rbe_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def items(systems):
        """ctypes array of BatchItem from dicts with torch CUDA tensors pos (N x 3), q (N),
        F (N x 3), W (9), optional E (2), and box, seed, step."""
        arr = (BatchItem * len(systems))()
        for k, sy in enumerate(systems):
            E = sy.get("E")
            bd, sd = sy.get("box_dev"), sy.get("step_dev")
            arr[k] = BatchItem(N=int(sy["q"].shape[0]), pos=sy["pos"].data_ptr(), charge=sy["q"].data_ptr(),
                               forces=sy["F"].data_ptr(), virial=sy["W"].data_ptr(),
                               energy=E.data_ptr() if E is not None else None,
                               box=(ctypes.c_double * 3)(*[float(b) for b in sy["box"]]), seed=int(sy["seed"]),
                               step=int(sy["step"]), box_dev=bd.data_ptr() if bd is not None else None,
                               step_dev=sd.data_ptr() if sd is not None else None)
        return arr

    def evaluate(self, items):
        arr = items if isinstance(items, ctypes.Array) else self.items(items)
        self._check(load().rbe_kspace_forces_virial_batched(self.h, arr, len(arr)))

    def autotune(self, items, reps: int = 5) -> float:
        arr = items if isinstance(items, ctypes.Array) else self.items(items)
        ms = ctypes.c_double()
        self._check(load().rbe_batch_autotune(self.h, arr, len(arr), int(reps), ctypes.byref(ms)))
        return ms.value

    def test_barrier_timeout(self, enable: bool):
        self._check(load().rbe_batch_test_barrier_timeout(self.h, int(bool(enable))))

    def set_persistent(self, enable: bool):
        self._check(load().rbe_batch_set_persistent(self.h, int(bool(enable))))

    def set_tiles(self, rho_k: int, rho_chunk: int, force_block: int):
        self._check(load().rbe_batch_set_tiles(self.h, int(rho_k), int(rho_chunk), int(force_block)))

    def tiles(self):
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(load().rbe_batch_get_tiles(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def set_rho_f(self, rho_f: int):
        self._check(load().rbe_batch_set_rho_f(self.h, int(rho_f)))

    def rho_f(self) -> int:
        f = ctypes.c_int32()
        self._check(load().rbe_batch_get_rho_f(self.h, ctypes.byref(f)))
        return f.value

    def set_stream(self, stream_handle: int):
        self._check(load().rbe_batch_set_stream(self.h, stream_handle))

    def sync(self):
        self._check(load().rbe_batch_sync(self.h))


def piston_mass(tau_P: float, beta_T: float, V0: float) -> float:
    """Barostat mass giving a harmonic volume oscillation of period tau_P (ps) for an
    isothermal compressibility beta_T (per kJ/mol/A^3) about V0 (A^3): M = tau_P^2 / (4 pi^2
    beta_T V0), in the units of the Langevin NPT equations of Sec. 3.2."""
    return tau_P * tau_P / (4.0 * math.pi * math.pi * beta_T * V0)


def piston_masses_rect(mode: int, tau_P: float, beta_T: float, box) -> tuple:
    """Cell masses of the rectangular barostats (NptParams.M_cell) for a harmonic oscillation of
    period tau_P (ps) of each cell variable, when a strain of one edge (or of the area) changes
    the pressure on it by the relative volume change over beta_T (per kJ/mol/A^3).
    Anisotropic (mode 2): M_j = V tau^2 / (4 pi^2 beta_T l_j^2).  Semi-isotropic (mode 3):
    M_A = L tau^2 / (4 pi^2 beta_T A) in [0], M_L = A tau^2 / (4 pi^2 beta_T L) in [2]."""
    lx, ly, lz = (float(x) for x in box)
    c = tau_P * tau_P / (4.0 * math.pi * math.pi * beta_T)
    if mode == RBE_BAROSTAT_ANISO:
        V = lx * ly * lz
        return (c * V / (lx * lx), c * V / (ly * ly), c * V / (lz * lz))
    if mode == RBE_BAROSTAT_SEMI:
        A = lx * ly
        return (c * lz / A, 0.0, c * A / lz)
    raise ValueError("mode must be RBE_BAROSTAT_ANISO or RBE_BAROSTAT_SEMI")


class Server:
    """The C++ serving loop (rbe_server_*): submit requests, call progress() until all are
    done, read results and chunk-latency statistics."""

    def __init__(self, alpha, P, precision=RBE_FP32_PHASE, max_slots=32, chunk_steps=10,
                 mem_budget=8 << 30, use_graphs=True, batched=0):
        """batched: 0 every replica on its own chunks; 1 lockstep groups with the batched k-space
        (default tiles); 2 the same with tiles autotuned on the first captured group."""
        cfg = ServerConfig(alpha=float(alpha), P=int(P), precision=int(precision), max_slots=int(max_slots),
                           chunk_steps=int(chunk_steps), mem_budget=int(mem_budget),
                           use_graphs=int(bool(use_graphs)), batched=int(batched))
        self.h = ctypes.c_void_p()
        lib = load()
        st = lib.rbe_server_create(ctypes.byref(cfg), ctypes.byref(self.h))
        if st != RBE_OK:
            raise RBEError(st, lib.rbe_last_error(None).decode())
        self._n = {}

    def _check(self, st):
        if st != RBE_OK:
            lib = load()
            raise RBEError(st, f"{lib.rbe_status_string(st).decode()}: {lib.rbe_server_last_error(self.h).decode()}")

    def close(self):
        if self.h:
            load().rbe_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, pos, mom, charge, mass, box, params: NptParams, seed: int, nsteps: int, pV: float = 0.0,
               pc=(0.0, 0.0, 0.0), sampler: int = 0, ptilde: int = 0, reuse: int = 1):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (pos, mom, charge, mass)]
        req = Request(N=int(arrs[2].shape[0]), pos=arrs[0].ctypes.data, mom=arrs[1].ctypes.data,
                      charge=arrs[2].ctypes.data, mass=arrs[3].ctypes.data,
                      box=(ctypes.c_double * 3)(*[float(b) for b in box]), pV=float(pV), seed=int(seed),
                      nsteps=int(nsteps), pad=0, params=params,
                      pc=(ctypes.c_double * 3)(*[float(x) for x in pc]), sampler=int(sampler), ptilde=int(ptilde),
                      reuse=int(reuse), pad2=0)
        rid = ctypes.c_int64()
        self._check(load().rbe_server_submit(self.h, ctypes.byref(req), ctypes.byref(rid)))
        self._n[rid.value] = req.N
        return rid.value

    def progress(self, wait: bool = False):
        q, a, d = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        self._check(load().rbe_server_progress(self.h, int(bool(wait)), ctypes.byref(q), ctypes.byref(a),
                                               ctypes.byref(d)))
        return q.value, a.value, d.value

    def result(self, rid: int):
        N = self._n[rid]
        pos = np.zeros((N, 3))
        mom = np.zeros((N, 3))
        cell = np.zeros(RBE_CELL_DOUBLES)
        self._check(load().rbe_server_result(self.h, rid, pos.ctypes.data_as(_dp), mom.ctypes.data_as(_dp),
                                             cell.ctypes.data_as(_dp)))
        return pos, mom, cell

    def cancel(self, rid: int):
        self._check(load().rbe_server_cancel(self.h, int(rid)))

    def state(self, rid: int):
        """(state, error): state 0 queued, 1 resident, 2 finished, 3 failed, 4 cancelled."""
        st, err = ctypes.c_int32(), ctypes.c_int()
        self._check(load().rbe_server_request_state(self.h, int(rid), ctypes.byref(st), ctypes.byref(err)))
        return st.value, err.value

    def stats(self):
        n, steps, span = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        load().rbe_server_stats(self.h, None, 0, ctypes.byref(n), ctypes.byref(steps), ctypes.byref(span))
        lat = np.zeros(max(n.value, 1))
        load().rbe_server_stats(self.h, lat.ctypes.data_as(_dp), n.value, ctypes.byref(n), ctypes.byref(steps),
                                ctypes.byref(span))
        return lat[:n.value], steps.value, span.value


def rbe_version() -> int:
    return int(load().rbe_version())


# ---------------------------------------------------------------------------------
class Context:
    """Owns one librbe context: box, alpha, batch size P and Philox seed."""

    def __init__(self, box, alpha: float, P: int, seed: int, precision: int = RBE_FP64,
                 rho_accum: int = RBE_RHO_COMP32, stream=None):
        self.P = int(P)
        self.alpha = float(alpha)
        self.h = rbe_create(box, alpha, P, seed)
        rbe_set_precision(self.h, precision, rho_accum)
        if stream is not None:
            rbe_set_stream(self.h, stream)

    def close(self):
        if self.h is not None:
            rbe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream_handle: int):
        rbe_set_stream(self.h, stream_handle)

    def set_precision(self, precision: int, rho_accum: int = RBE_RHO_COMP32):
        rbe_set_precision(self.h, precision, rho_accum)

    def set_sampler(self, sampler: int):
        """RBE_SAMPLER_EXACT, _OFFLINE or _MH (Sec. 4.3); resets the MH chain."""
        rbe_set_sampler(self.h, sampler)

    def set_pressure_batch(self, Ptilde: int):
        """A separate batch of Ptilde frequencies for the virial and energy (0: the force batch)."""
        rbe_set_pressure_batch(self.h, Ptilde)

    def forces_virial_general(self, positions, charges, h, step: int, forces_out, virial_out=None, energy_out=None):
        """k-space forces/virial/energy in the general cell h (3x3, cell vectors as columns); torch
        CUDA float64 tensors for positions (N, 3), charges (N,), forces_out (N, 3), virial_out (9,),
        energy_out (2,)."""
        hh = np.ascontiguousarray(np.asarray(h, dtype=np.float64).reshape(3, 3))
        N = int(charges.shape[0])
        ptr = lambda t: None if t is None else t.data_ptr()
        _check(load().rbe_kspace_forces_virial_general(self.h, N, ptr(positions), ptr(charges),
                                                       hh.ctypes.data_as(_dp), int(step), ptr(forces_out),
                                                       ptr(virial_out), ptr(energy_out)), self.h)

    def set_sample_reuse(self, M: int):
        """NPT: draw the frequencies of M steps at once, every M steps (1: every step)."""
        rbe_set_sample_reuse(self.h, M)

    def set_box(self, box):
        rbe_set_box(self.h, box)

    def sample_k(self, step: int):
        return rbe_sample_k(self.h, step, self.P)

    def forces_virial(self, positions, charges, step: int, forces_out, virial_out=None, energy_out=None):
        rbe_kspace_forces_virial(self.h, positions, charges, step, forces_out, virial_out, energy_out)

    def forces_virial_xyzq(self, xyzq, step: int, forces_out, virial_out=None, energy_out=None):
        rbe_kspace_forces_virial_xyzq(self.h, xyzq, step, forces_out, virial_out, energy_out)

    def forces_virial_host(self, positions, charges, step: int):
        return rbe_kspace_forces_virial_host(self.h, positions, charges, step)

    def weighted(self, positions, charges, m, weights, forces_out, virial_out=None, energy_out=None):
        rbe_kspace_weighted(self.h, positions, charges, m, weights, forces_out, virial_out, energy_out)

    def rho(self, K: int | None = None):
        return rbe_get_rho(self.h, self.P if K is None else K)

    def sync(self):
        rbe_sync(self.h)

    def set_kernel_timing(self, enable: bool = True):
        rbe_set_kernel_timing(self.h, enable)

    def kernel_times(self):
        return rbe_get_kernel_times(self.h)
