"""FP64 CPU oracle for the random batch Ewald k-space path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import this package.  It wraps ``rbe_oracle.c`` (plain C, FP64,
index-order loops) through ctypes and never touches the CUDA library.

Functions follow the paper's Sec. 4.1 (Ewald sum), Sec. 4.2 (RBE estimators, the
normaliser S and the importance distribution), Sec. 4.3 (sampling) and App. C (the
pressure tensor); each C function states the equation it restates.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rbe_oracle.c")
_SRC_NPT = os.path.join(_HERE, "npt_oracle.c")
_SRC_SMP = os.path.join(_HERE, "sampler_oracle.c")
_SRC_GEN = os.path.join(_HERE, "general_oracle.c")
_SRC_FLX = os.path.join(_HERE, "flexible_oracle.c")
_SRC_WAT = os.path.join(_HERE, "water_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_int32_p = ctypes.POINTER(ctypes.c_int32)
_c_uint32_p = ctypes.POINTER(ctypes.c_uint32)
_c_int64_p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build/liboracle.so`` and return its path."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [s for s in (_SRC, _SRC_NPT, _SRC_SMP, _SRC_GEN, _SRC_FLX, _SRC_WAT) if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "npt_params.h")])
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp] + srcs + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib_omp = None


def build_omp(force: bool = False) -> str:
    """Compile ``rbe_oracle.c`` alone with ``-fopenmp`` into ``oracle/_build/liboracle_omp.so``
    (the all-cores timing build of the k-space oracle; the same loops and results as the
    single-thread build, its outer loops shared among the threads).  Raises
    ``subprocess.CalledProcessError`` where the compiler has no OpenMP runtime."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC):
        tmp = _LIB_OMP + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True, capture_output=True)
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def _load_omp():
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            lib = ctypes.CDLL(build_omp())
            lib.orc_rbe_kspace.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p,
                                           ctypes.c_double, ctypes.c_int32, _c_int32_p, _c_double_p,
                                           _c_double_p, _c_double_p, _c_double_p, _c_double_p]
            lib.orc_rbe_kspace.restype = ctypes.c_int
            lib.orc_rbe_kspace_subset.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p,
                                                  ctypes.c_double, ctypes.c_int32, _c_int32_p, _c_double_p,
                                                  ctypes.c_int64, _c_int64_p, _c_double_p, _c_double_p,
                                                  _c_double_p, _c_double_p]
            lib.orc_rbe_kspace_subset.restype = ctypes.c_int
            _lib_omp = lib
    return _lib_omp


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_philox4x32_10.argtypes = [_c_uint32_p, _c_uint32_p, _c_uint32_p]
            lib.orc_philox4x32_10.restype = None
            lib.orc_uniform53.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            lib.orc_uniform53.restype = ctypes.c_double
            lib.orc_exp.argtypes = [ctypes.c_double]
            lib.orc_exp.restype = ctypes.c_double
            lib.orc_axis_M.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.orc_axis_M.restype = ctypes.c_int32
            lib.orc_axis_table.argtypes = [ctypes.c_double, ctypes.c_double, _c_double_p,
                                           ctypes.POINTER(ctypes.c_uint64)]
            lib.orc_axis_table.restype = ctypes.c_double
            lib.orc_axis_shift.argtypes = [ctypes.c_int32]
            lib.orc_axis_shift.restype = ctypes.c_int
            lib.orc_sample_k.argtypes = [_c_double_p, ctypes.c_double, ctypes.c_int32, ctypes.c_uint64,
                                         ctypes.c_uint64, _c_int32_p, _c_double_p]
            lib.orc_sample_k.restype = ctypes.c_int
            lib.orc_ewald_kspace.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p,
                                             ctypes.c_double, ctypes.c_int32, _c_double_p, _c_double_p,
                                             _c_double_p]
            lib.orc_ewald_kspace.restype = ctypes.c_int
            lib.orc_rbe_kspace.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p,
                                           ctypes.c_double, ctypes.c_int32, _c_int32_p, _c_double_p,
                                           _c_double_p, _c_double_p, _c_double_p, _c_double_p]
            lib.orc_rbe_kspace.restype = ctypes.c_int
            lib.orc_rbe_kspace_subset.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p,
                                                  ctypes.c_double, ctypes.c_int32, _c_int32_p, _c_double_p,
                                                  ctypes.c_int64, _c_int64_p, _c_double_p, _c_double_p,
                                                  _c_double_p, _c_double_p]
            lib.orc_rbe_kspace_subset.restype = ctypes.c_int
            lib.orc_rbe_snapshot.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p,
                                             ctypes.c_double, ctypes.c_int32, ctypes.c_uint64,
                                             ctypes.c_uint64, _c_double_p, _c_double_p, _c_double_p,
                                             _c_int32_p, _c_double_p]
            lib.orc_rbe_snapshot.restype = ctypes.c_int
            lib.orc_ewald_real.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p,
                                           ctypes.c_double, ctypes.c_double, _c_double_p, _c_double_p,
                                           _c_double_p]
            lib.orc_ewald_real.restype = ctypes.c_int
            lib.orc_direct_sum.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p,
                                           ctypes.c_int32]
            lib.orc_direct_sum.restype = ctypes.c_double
            if hasattr(lib, "orc_npt_step"):
                _bind_npt(lib)
            if hasattr(lib, "orc_sample_k_mh"):
                _bind_samplers(lib)
            if hasattr(lib, "orc_gen_kspace"):
                _bind_general(lib)
            if hasattr(lib, "orc_flex_step"):
                _bind_flexible(lib)
            if hasattr(lib, "orc_water_step"):
                _bind_water(lib)
            _lib = lib
    return _lib


class NptParams(ctypes.Structure):
    """Parameters of the Langevin NPT step (mirrors orc_npt_params in npt_oracle.c)."""
    _fields_ = [("dt", ctypes.c_double), ("kT", ctypes.c_double), ("P_ext", ctypes.c_double),
                ("gamma", ctypes.c_double), ("gamma_V", ctypes.c_double), ("M_V", ctypes.c_double),
                ("alpha", ctypes.c_double), ("rc", ctypes.c_double), ("qqr2e", ctypes.c_double),
                ("lj_sigma", ctypes.c_double), ("lj_eps", ctypes.c_double), ("max_disp", ctypes.c_double),
                ("P", ctypes.c_int32), ("kspace", ctypes.c_int32), ("real", ctypes.c_int32),
                ("noise", ctypes.c_int32), ("barostat", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("M_cell", ctypes.c_double * 3), ("gamma0", ctypes.c_double),
                ("sampler", ctypes.c_int32), ("pad2", ctypes.c_int32), ("chain", ctypes.c_void_p),
                ("Ptilde", ctypes.c_int32), ("reuse", ctypes.c_int32), ("reuse_m", ctypes.c_void_p)]


def _bind_npt(lib):
    P = ctypes.POINTER(NptParams)
    lib.orc_npt_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, _c_double_p]
    lib.orc_npt_normals.restype = None
    lib.orc_pair_real.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _c_double_p,
                                  _c_double_p, _c_double_p]
    lib.orc_pair_real.restype = ctypes.c_int
    lib.orc_npt_forces.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, ctypes.c_uint64, P,
                                   _c_double_p, _c_double_p, _c_double_p]
    lib.orc_npt_forces.restype = ctypes.c_int
    lib.orc_npt_step.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, _c_double_p, _c_double_p,
                                 _c_double_p, _c_double_p, _c_double_p, ctypes.c_uint64, P, _c_double_p]
    lib.orc_npt_step.restype = ctypes.c_int
    lib.orc_npt_run.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, _c_double_p, _c_double_p,
                                _c_double_p, _c_double_p, _c_double_p, ctypes.c_uint64, ctypes.c_int32, P,
                                _c_double_p, _c_double_p, _c_double_p]
    lib.orc_npt_run.restype = ctypes.c_int
    lib.orc_npt_forces_diag.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, ctypes.c_uint64, P,
                                        _c_double_p, _c_double_p, _c_double_p]
    lib.orc_npt_forces_diag.restype = ctypes.c_int
    lib.orc_npt_step_rect.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, _c_double_p,
                                      _c_double_p, _c_double_p, _c_double_p, _c_double_p, ctypes.c_uint64, P,
                                      _c_double_p]
    lib.orc_npt_step_rect.restype = ctypes.c_int
    lib.orc_npt_run_rect.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, _c_double_p,
                                     _c_double_p, _c_double_p, _c_double_p, _c_double_p, ctypes.c_uint64,
                                     ctypes.c_int32, P, _c_double_p, _c_double_p, _c_double_p]
    lib.orc_npt_run_rect.restype = ctypes.c_int


def _bind_samplers(lib):
    lib.orc_own_log.argtypes = [ctypes.c_double]
    lib.orc_own_log.restype = ctypes.c_double
    lib.orc_own_erfc.argtypes = [ctypes.c_double]
    lib.orc_own_erfc.restype = ctypes.c_double
    lib.orc_rounded_gauss_mass.argtypes = [ctypes.c_int32, ctypes.c_double]
    lib.orc_rounded_gauss_mass.restype = ctypes.c_double
    lib.orc_polar_pair.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _c_double_p]
    lib.orc_polar_pair.restype = ctypes.c_int
    for name in ("orc_sample_k_offline", "orc_sample_k_mh"):
        f = getattr(lib, name)
        f.argtypes = [_c_double_p, ctypes.c_double, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, _c_int32_p,
                      _c_double_p]
        f.restype = ctypes.c_int


def _bind_general(lib):
    lib.orc_gen_inverse.argtypes = [_c_double_p, _c_double_p]
    lib.orc_gen_inverse.restype = ctypes.c_double
    lib.orc_gen_metric.argtypes = [_c_double_p, _c_double_p]
    lib.orc_gen_metric.restype = None
    lib.orc_gen_kspace.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, ctypes.c_double,
                                   ctypes.c_int32, _c_int32_p, _c_double_p, _c_double_p, _c_double_p, _c_double_p]
    lib.orc_gen_kspace.restype = ctypes.c_int
    lib.orc_gen_ewald_kspace.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, ctypes.c_double,
                                         ctypes.c_int32, _c_double_p, _c_double_p, _c_double_p]
    lib.orc_gen_ewald_kspace.restype = ctypes.c_int
    lib.orc_gen_ewald_real.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, ctypes.c_double,
                                       ctypes.c_double, _c_double_p, _c_double_p, _c_double_p]
    lib.orc_gen_ewald_real.restype = ctypes.c_int
    for name in ("orc_gen_S", "orc_gen_S_direct"):
        getattr(lib, name).argtypes = [_c_double_p, ctypes.c_double]
        getattr(lib, name).restype = ctypes.c_double
    lib.orc_gen_sample_k_mh.argtypes = [_c_double_p, ctypes.c_double, ctypes.c_int32, ctypes.c_uint64,
                                        ctypes.c_uint64, _c_int32_p, _c_double_p]
    lib.orc_gen_sample_k_mh.restype = ctypes.c_int


class FlexParams(ctypes.Structure):
    """Parameters of the flexible-cell NPT step (mirrors orc_flex_params in flexible_oracle.c)."""
    _fields_ = [("dt", ctypes.c_double), ("kT", ctypes.c_double), ("P_ext", ctypes.c_double),
                ("gamma", ctypes.c_double), ("gamma_h", ctypes.c_double), ("M", ctypes.c_double * 9),
                ("alpha", ctypes.c_double), ("rc", ctypes.c_double), ("qqr2e", ctypes.c_double),
                ("lj_sigma", ctypes.c_double), ("lj_eps", ctypes.c_double), ("max_disp", ctypes.c_double),
                ("chi", ctypes.c_double), ("P", ctypes.c_int32), ("kspace", ctypes.c_int32), ("real", ctypes.c_int32),
                ("noise", ctypes.c_int32), ("seed", ctypes.c_uint64), ("chain", ctypes.c_void_p)]


def _bind_flexible(lib):
    F = ctypes.POINTER(FlexParams)
    lib.orc_flex_pair_real.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       _c_double_p, _c_double_p, _c_double_p]
    lib.orc_flex_pair_real.restype = ctypes.c_int
    lib.orc_flex_forces.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, ctypes.c_uint64, F,
                                    _c_double_p, _c_double_p, _c_double_p]
    lib.orc_flex_forces.restype = ctypes.c_int
    lib.orc_flex_step.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, _c_double_p, _c_double_p,
                                  _c_double_p, _c_double_p, _c_double_p, ctypes.c_uint64, F, _c_double_p]
    lib.orc_flex_step.restype = ctypes.c_int
    lib.orc_flex_run.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, _c_double_p, _c_double_p,
                                 _c_double_p, _c_double_p, _c_double_p, ctypes.c_uint64, ctypes.c_int32, F,
                                 _c_double_p, _c_double_p, _c_double_p]
    lib.orc_flex_run.restype = ctypes.c_int


def _dp(a):
    return a.ctypes.data_as(_c_double_p)


def _ip(a):
    return a.ctypes.data_as(_c_int32_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class OracleError(RuntimeError):
    pass


def _check(st, what):
    if st != 0:
        raise OracleError(f"{what} failed with status {st}")


# ---------------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """Philox-4x32-10 words for one counter (4 uint32) and key (2 uint32)."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(c.ctypes.data_as(_c_uint32_p), k.ctypes.data_as(_c_uint32_p),
                          out.ctypes.data_as(_c_uint32_p))
    return out


def uniform53(a, b):
    return _load().orc_uniform53(int(a), int(b))


def exp_table(x: float) -> float:
    """The sampler's own exponential (Cody--Waite + Taylor), for x in [-700, 0]."""
    return _load().orc_exp(float(x))


def axis_table(alpha: float, ell: float):
    """(w, cum, M, H, sh) of the per-axis discrete Gaussian for box length ell: the weights,
    the integer cumulative sums of rint(w 2^sh), the truncation, H and the shift."""
    lib = _load()
    M = lib.orc_axis_M(alpha, ell)
    w = np.zeros(2 * M + 1)
    cum = np.zeros(2 * M + 1, dtype=np.uint64)
    H = lib.orc_axis_table(alpha, ell, _dp(w), cum.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return w, cum, M, H, lib.orc_axis_shift(M)


def sample_k(box, alpha: float, P: int, seed: int, step: int):
    """m[P,3] (int32) and S for one step of the k-sampling stream."""
    lib = _load()
    b = _f64(box, (3,))
    m = np.zeros((P, 3), dtype=np.int32)
    S = ctypes.c_double(0.0)
    _check(lib.orc_sample_k(_dp(b), alpha, P, seed, step, _ip(m), ctypes.byref(S)), "sample_k")
    return m, S.value


def own_log(x: float) -> float:
    return _load().orc_own_log(float(x))


def own_erfc(x: float) -> float:
    return _load().orc_own_erfc(float(x))


def rounded_gauss_mass(m: int, g: float) -> float:
    """Mass of [m - 1/2, m + 1/2) under N(0, sigma^2) with g = 1/(sigma sqrt 2)."""
    return _load().orc_rounded_gauss_mass(int(m), float(g))


def polar_pair(seed: int, step: int, l: int, d: int):
    """One polar-method trial of the offline stream: (ok, z[2])."""
    z = np.zeros(2)
    ok = _load().orc_polar_pair(seed, step, l, d, _dp(z))
    return bool(ok), z


def sample_k_offline(box, alpha: float, P: int, seed: int, step: int):
    """Offline approach of Sec. 4.3: m[P,3] (rounded scaled Gaussians) and S."""
    lib = _load()
    m = np.zeros((P, 3), dtype=np.int32)
    S = ctypes.c_double(0.0)
    _check(lib.orc_sample_k_offline(_dp(_f64(box, (3,))), alpha, P, seed, step, _ip(m), ctypes.byref(S)),
           "sample_k_offline")
    return m, S.value


def sample_k_mh(box, alpha: float, P: int, seed: int, step: int, state):
    """Online approach of Sec. 4.3: one MH step per slot from state[P,3] (int32, updated in
    place; rows of zeros start from the exact draw).  Returns (state, S)."""
    lib = _load()
    assert state.dtype == np.int32 and state.shape == (P, 3) and state.flags.c_contiguous
    S = ctypes.c_double(0.0)
    _check(lib.orc_sample_k_mh(_dp(_f64(box, (3,))), alpha, P, seed, step, _ip(state), ctypes.byref(S)),
           "sample_k_mh")
    return state, S.value


def ewald_kspace(pos, q, box, alpha: float, kmax: int):
    """Full Ewald k-space sum: (F[N,3], W[3,3], E_k, E_self)."""
    lib = _load()
    pos = _f64(pos)
    q = _f64(q)
    N = q.shape[0]
    b = _f64(box, (3,))
    F = np.zeros((N, 3))
    W = np.zeros((3, 3))
    E = np.zeros(2)
    _check(lib.orc_ewald_kspace(N, _dp(pos), _dp(q), _dp(b), alpha, kmax, _dp(F), _dp(W), _dp(E)),
           "ewald_kspace")
    return F, W, E[0], E[1]


def rbe_kspace(pos, q, box, alpha: float, m, weights, all_cores: bool = False):
    """RBE estimators on a given batch: (F[N,3], W[3,3], E_k, E_self, rho[P] complex).
    ``all_cores`` runs the OpenMP build (``OMP_NUM_THREADS`` threads, else every core); the
    results are the same bits."""
    lib = _load_omp() if all_cores else _load()
    pos = _f64(pos)
    q = _f64(q)
    N = q.shape[0]
    m = np.ascontiguousarray(m, dtype=np.int32).reshape(-1, 3)
    P = m.shape[0]
    wl = np.asarray(weights, dtype=np.float64)
    wl = np.full(P, float(wl)) if wl.ndim == 0 else np.ascontiguousarray(wl)
    if wl.shape != (P,):
        raise ValueError("weights must be a scalar or have one entry per frequency")
    b = _f64(box, (3,))
    F = np.zeros((N, 3))
    W = np.zeros((3, 3))
    E = np.zeros(2)
    rho = np.zeros(2 * P)
    _check(lib.orc_rbe_kspace(N, _dp(pos), _dp(q), _dp(b), alpha, P, _ip(m), _dp(wl), _dp(F), _dp(W),
                              _dp(E), _dp(rho)), "rbe_kspace")
    return F, W, E[0], E[1], rho[0::2] + 1j * rho[1::2]


def rbe_kspace_subset(pos, q, box, alpha: float, m, weights, idx, all_cores: bool = False):
    """The RBE estimators with the forces of the particles ``idx`` only: (F[len(idx),3],
    W[3,3], E_k, E_self, rho[P] complex); rho, W and E over all particles.  Each force row is
    the bits ``rbe_kspace`` gives for that particle."""
    lib = _load_omp() if all_cores else _load()
    pos = _f64(pos)
    q = _f64(q)
    N = q.shape[0]
    m = np.ascontiguousarray(m, dtype=np.int32).reshape(-1, 3)
    P = m.shape[0]
    wl = np.asarray(weights, dtype=np.float64)
    wl = np.full(P, float(wl)) if wl.ndim == 0 else np.ascontiguousarray(wl)
    if wl.shape != (P,):
        raise ValueError("weights must be a scalar or have one entry per frequency")
    ix = np.ascontiguousarray(idx, dtype=np.int64).reshape(-1)
    b = _f64(box, (3,))
    F = np.zeros((ix.shape[0], 3))
    W = np.zeros((3, 3))
    E = np.zeros(2)
    rho = np.zeros(2 * P)
    _check(lib.orc_rbe_kspace_subset(N, _dp(pos), _dp(q), _dp(b), alpha, P, _ip(m), _dp(wl), ix.shape[0],
                                     ix.ctypes.data_as(_c_int64_p), _dp(F), _dp(W), _dp(E), _dp(rho)),
           "rbe_kspace_subset")
    return F, W, E[0], E[1], rho[0::2] + 1j * rho[1::2]


def rbe_snapshot(pos, q, box, alpha: float, P: int, seed: int, step: int):
    """Sample and evaluate: (F, W, E_k, E_self, m, S)."""
    lib = _load()
    pos = _f64(pos)
    q = _f64(q)
    N = q.shape[0]
    b = _f64(box, (3,))
    F = np.zeros((N, 3))
    W = np.zeros((3, 3))
    E = np.zeros(2)
    m = np.zeros((P, 3), dtype=np.int32)
    S = ctypes.c_double(0.0)
    _check(lib.orc_rbe_snapshot(N, _dp(pos), _dp(q), _dp(b), alpha, P, seed, step, _dp(F), _dp(W),
                                _dp(E), _ip(m), ctypes.byref(S)), "rbe_snapshot")
    return F, W, E[0], E[1], m, S.value


def ewald_real(pos, q, box, alpha: float, rc: float):
    """Nearest-image erfc real-space part: (F[N,3], W[3,3], E_r)."""
    lib = _load()
    pos = _f64(pos)
    q = _f64(q)
    N = q.shape[0]
    b = _f64(box, (3,))
    F = np.zeros((N, 3))
    W = np.zeros((3, 3))
    E = ctypes.c_double(0.0)
    _check(lib.orc_ewald_real(N, _dp(pos), _dp(q), _dp(b), alpha, rc, _dp(F), _dp(W), ctypes.byref(E)),
           "ewald_real")
    return F, W, E.value


def direct_sum(pos, q, box, R: int) -> float:
    """Brute-force image sum over whole cells with |n| <= R."""
    lib = _load()
    pos = _f64(pos)
    q = _f64(q)
    b = _f64(box, (3,))
    return lib.orc_direct_sum(q.shape[0], _dp(pos), _dp(q), _dp(b), R)


# ---------------------------------------------------------------------------------
# Langevin NPT (npt_oracle.c)

KB = 0.00831446261815324        # kJ/mol/K
BAR = 6.02214076e-5              # kJ/mol/A^3 per bar
QQR2E = 1389.35457644382         # kJ/mol A / e^2


def npt_params(**kw) -> NptParams:
    """NptParams with the defaults of the point-charge NPT system (reading 17): 300 K,
    1 bar, dt = 1 fs, gamma = 10/ps, gamma_V = 2/ps, alpha = 0.2, rc = 7, LJ 2 A / 0.5 kJ/mol."""
    d = dict(dt=0.001, kT=KB * 300.0, P_ext=1.0 * BAR, gamma=10.0, gamma_V=2.0, M_V=1.0, alpha=0.2, rc=7.0,
             qqr2e=QQR2E, lj_sigma=2.0, lj_eps=0.5, max_disp=0.0, P=100, kspace=1, real=1, noise=1,
             barostat=1, pad=0, seed=1, M_cell=(1.0, 1.0, 1.0), gamma0=0.0, sampler=0, pad2=0, chain=None,
             Ptilde=0, reuse=1, reuse_m=None)
    d.update(kw)
    d["M_cell"] = (ctypes.c_double * 3)(*[float(x) for x in d["M_cell"]])
    return NptParams(**d)


def piston_mass(tau_p: float, beta_T: float, V0: float) -> float:
    """M = tau_P^2 / (4 pi^2 beta_T V0): a harmonic volume oscillation of period tau_P (reading 13)."""
    return tau_p ** 2 / (4.0 * np.pi ** 2 * beta_T * V0)


def piston_masses_rect(mode: int, tau_p: float, beta_T: float, box) -> tuple:
    """Cell masses of the rectangular barostats for a harmonic oscillation of period tau_P of
    each cell variable, taking a strain of one axis (or of the area) to change its pressure
    by the relative volume change over beta_T: anisotropic (mode 2) M_j = V tau^2 /
    (4 pi^2 beta_T l_j^2); semi-isotropic (mode 3) M_A = L tau^2 / (4 pi^2 beta_T A) in [0],
    M_L = A tau^2 / (4 pi^2 beta_T L) in [2]."""
    lx, ly, lz = (float(x) for x in box)
    c = tau_p ** 2 / (4.0 * np.pi ** 2 * beta_T)
    V = lx * ly * lz
    if mode == 2:
        return (c * V / lx ** 2, c * V / ly ** 2, c * V / lz ** 2)
    if mode == 3:
        A = lx * ly
        return (c * lz / A, 0.0, c * A / lz)
    raise ValueError("mode must be 2 (anisotropic) or 3 (semi-isotropic)")


def npt_normals(seed: int, stream: int, step: int, index: int):
    z = np.zeros(4)
    _load().orc_npt_normals(seed, stream, step, index, _dp(z))
    return z


def pair_real(pos, q, box, alpha, rc, qqr2e, lj_sigma, lj_eps):
    """Nearest-image erfc Coulomb + LJ: (F[N,3], W[3,3], E_coul, E_lj)."""
    lib = _load()
    pos = _f64(pos)
    q = _f64(q)
    N = q.shape[0]
    b = _f64(box, (3,))
    F = np.zeros((N, 3))
    W = np.zeros((3, 3))
    E = np.zeros(2)
    _check(lib.orc_pair_real(N, _dp(pos), _dp(q), _dp(b), alpha, rc, qqr2e, lj_sigma, lj_eps, _dp(F), _dp(W),
                             _dp(E)), "pair_real")
    return F, W, E[0], E[1]


class NptState:
    """Device-free NPT state for the oracle: positions, momenta, forces, box, p_V, virial trace."""

    def __init__(self, r, p, q, m, L, pV=0.0):
        self.r = _f64(r).copy()
        self.p = _f64(p).copy()
        self.q = _f64(q)
        self.m = _f64(m)
        self.L = _f64(L, (3,)).copy()
        self.F = np.zeros_like(self.r)
        self.pV = ctypes.c_double(pV)
        self.W = ctypes.c_double(0.0)

    @property
    def N(self):
        return self.q.shape[0]


def npt_forces(st: NptState, step: int, prm: NptParams):
    E = np.zeros(3)
    _check(_load().orc_npt_forces(st.N, _dp(st.r), _dp(st.q), _dp(st.L), step, ctypes.byref(prm), _dp(st.F),
                                  ctypes.byref(st.W), _dp(E)), "npt_forces")
    return E


def npt_step(st: NptState, step: int, prm: NptParams):
    E = np.zeros(3)
    _check(_load().orc_npt_step(st.N, _dp(st.r), _dp(st.p), _dp(st.F), _dp(st.q), _dp(st.m), _dp(st.L),
                                ctypes.byref(st.pV), ctypes.byref(st.W), step, ctypes.byref(prm), _dp(E)),
           "npt_step")
    return E


def npt_run(st: NptState, step0: int, nsteps: int, prm: NptParams):
    """nsteps steps; returns (V, P_ins, extended energy) per step."""
    V = np.zeros(nsteps)
    Pi = np.zeros(nsteps)
    H = np.zeros(nsteps)
    _check(_load().orc_npt_run(st.N, _dp(st.r), _dp(st.p), _dp(st.F), _dp(st.q), _dp(st.m), _dp(st.L),
                               ctypes.byref(st.pV), ctypes.byref(st.W), step0, nsteps, ctypes.byref(prm), _dp(V),
                               _dp(Pi), _dp(H)), "npt_run")
    return V, Pi, H


class NptRectState:
    """Oracle state of the rectangular-cell NPT step: positions, momenta, forces, box, cell
    momenta pc[3] and the virial diagonal Wd[3] at the current positions."""

    def __init__(self, r, p, q, m, L, pc=(0.0, 0.0, 0.0)):
        self.r = _f64(r).copy()
        self.p = _f64(p).copy()
        self.q = _f64(q)
        self.m = _f64(m)
        self.L = _f64(L, (3,)).copy()
        self.F = np.zeros_like(self.r)
        self.pc = _f64(pc, (3,)).copy()
        self.Wd = np.zeros(3)

    @property
    def N(self):
        return self.q.shape[0]


def npt_forces_rect(st: NptRectState, step: int, prm: NptParams):
    E = np.zeros(3)
    _check(_load().orc_npt_forces_diag(st.N, _dp(st.r), _dp(st.q), _dp(st.L), step, ctypes.byref(prm), _dp(st.F),
                                       _dp(st.Wd), _dp(E)), "npt_forces_diag")
    return E


def npt_step_rect(st: NptRectState, step: int, prm: NptParams):
    E = np.zeros(3)
    _check(_load().orc_npt_step_rect(st.N, _dp(st.r), _dp(st.p), _dp(st.F), _dp(st.q), _dp(st.m), _dp(st.L),
                                     _dp(st.pc), _dp(st.Wd), step, ctypes.byref(prm), _dp(E)), "npt_step_rect")
    return E


def npt_run_rect(st: NptRectState, step0: int, nsteps: int, prm: NptParams):
    """nsteps steps; returns (box[n,3], diagonal pressure[n,3], extended energy[n])."""
    L = np.zeros((nsteps, 3))
    Pd = np.zeros((nsteps, 3))
    H = np.zeros(nsteps)
    _check(_load().orc_npt_run_rect(st.N, _dp(st.r), _dp(st.p), _dp(st.F), _dp(st.q), _dp(st.m), _dp(st.L),
                                    _dp(st.pc), _dp(st.Wd), step0, nsteps, ctypes.byref(prm), _dp(L), _dp(Pd),
                                    _dp(H)), "npt_run_rect")
    return L, Pd, H


def ewald_total(pos, q, box, alpha: float, rc: float, kmax: int):
    """Total Ewald energy, force and virial (k-space + self + real space)."""
    Fk, Wk, Ek, Es = ewald_kspace(pos, q, box, alpha, kmax)
    Fr, Wr, Er = ewald_real(pos, q, box, alpha, rc)
    return Fk + Fr, Wk + Wr, Ek + Es + Er


# ---------------------------------------------------------------------------------
# General (triclinic) cell (general_oracle.c): h is 3x3 with the cell vectors as columns.
def gen_kspace(pos, q, h, alpha: float, m, weights):
    """k-space sums over the listed m with the given weights: (F[N,3], W[3,3], E_k, E_self)."""
    lib = _load()
    pos, q = _f64(pos), _f64(q)
    N = q.shape[0]
    m = np.ascontiguousarray(m, dtype=np.int32).reshape(-1, 3)
    K = m.shape[0]
    w = np.asarray(weights, dtype=np.float64)
    w = np.full(K, float(w)) if w.ndim == 0 else np.ascontiguousarray(w)
    F, W, E = np.zeros((N, 3)), np.zeros((3, 3)), np.zeros(2)
    _check(lib.orc_gen_kspace(N, _dp(pos), _dp(q), _dp(_f64(h, (3, 3))), alpha, K, _ip(m), _dp(w), _dp(F), _dp(W),
                              _dp(E)), "gen_kspace")
    return F, W, E[0], E[1]


def gen_ewald_kspace(pos, q, h, alpha: float, kmax: int):
    lib = _load()
    pos, q = _f64(pos), _f64(q)
    N = q.shape[0]
    F, W, E = np.zeros((N, 3)), np.zeros((3, 3)), np.zeros(2)
    _check(lib.orc_gen_ewald_kspace(N, _dp(pos), _dp(q), _dp(_f64(h, (3, 3))), alpha, kmax, _dp(F), _dp(W), _dp(E)),
           "gen_ewald_kspace")
    return F, W, E[0], E[1]


def gen_ewald_real(pos, q, h, alpha: float, rc: float):
    lib = _load()
    pos, q = _f64(pos), _f64(q)
    N = q.shape[0]
    F, W, E = np.zeros((N, 3)), np.zeros((3, 3)), ctypes.c_double(0.0)
    _check(lib.orc_gen_ewald_real(N, _dp(pos), _dp(q), _dp(_f64(h, (3, 3))), alpha, rc, _dp(F), _dp(W),
                                  ctypes.byref(E)), "gen_ewald_real")
    return F, W, E.value


def gen_S(h, alpha: float, direct: bool = False) -> float:
    lib = _load()
    f = lib.orc_gen_S_direct if direct else lib.orc_gen_S
    return f(_dp(_f64(h, (3, 3))), alpha)


def gen_metric(h):
    G = np.zeros((3, 3))
    _load().orc_gen_metric(_dp(_f64(h, (3, 3))), _dp(G))
    return G


def gen_sample_k_mh(h, alpha: float, P: int, seed: int, step: int, state):
    """General-cell MH sampler: state[P,3] int32 updated in place; returns (state, S)."""
    assert state.dtype == np.int32 and state.shape == (P, 3) and state.flags.c_contiguous
    S = ctypes.c_double(0.0)
    _check(_load().orc_gen_sample_k_mh(_dp(_f64(h, (3, 3))), alpha, P, seed, step, _ip(state), ctypes.byref(S)),
           "gen_sample_k_mh")
    return state, S.value


# ---------------------------------------------------------------------------------
# Flexible-cell Langevin NPT (flexible_oracle.c)
def flex_params(**kw) -> FlexParams:
    d = dict(dt=0.001, kT=KB * 300.0, P_ext=1.0 * BAR, gamma=10.0, gamma_h=2.0, M=(1.0,) * 9, alpha=0.2, rc=7.0,
             qqr2e=QQR2E, lj_sigma=2.0, lj_eps=0.5, max_disp=0.0, chi=2.0, P=100, kspace=1, real=1, noise=1, seed=1,
             chain=None)
    d.update(kw)
    d["M"] = (ctypes.c_double * 9)(*[float(x) for x in np.asarray(d["M"], dtype=float).reshape(9)])
    return FlexParams(**d)


class FlexState:
    """Oracle state of the flexible-cell step: r, p, F, h (3x3), p^h (3x3), W (3x3), and the MH chain."""

    def __init__(self, r, p, q, m, h, ph=None, P=100):
        self.r = _f64(r).copy()
        self.p = _f64(p).copy()
        self.q = _f64(q)
        self.m = _f64(m)
        self.h = _f64(h, (3, 3)).copy()
        self.ph = np.zeros((3, 3)) if ph is None else _f64(ph, (3, 3)).copy()
        self.F = np.zeros_like(self.r)
        self.W = np.zeros((3, 3))
        self.chain = np.zeros((max(P, 1), 3), dtype=np.int32)

    @property
    def N(self):
        return self.q.shape[0]

    def bind(self, prm: FlexParams):
        prm.chain = self.chain.ctypes.data
        return prm


def flex_forces(st: FlexState, step: int, prm: FlexParams):
    E = np.zeros(3)
    _check(_load().orc_flex_forces(st.N, _dp(st.r), _dp(st.q), _dp(st.h), step, ctypes.byref(st.bind(prm)),
                                   _dp(st.F), _dp(st.W), _dp(E)), "flex_forces")
    return E


def flex_step(st: FlexState, step: int, prm: FlexParams):
    E = np.zeros(3)
    _check(_load().orc_flex_step(st.N, _dp(st.r), _dp(st.p), _dp(st.F), _dp(st.q), _dp(st.m), _dp(st.h), _dp(st.ph),
                                 _dp(st.W), step, ctypes.byref(st.bind(prm)), _dp(E)), "flex_step")
    return E


def flex_run(st: FlexState, step0: int, n: int, prm: FlexParams):
    """n steps; returns (h[n,3,3], P_ins[n,3,3], extended energy[n])."""
    hs, Ps, H = np.zeros((n, 3, 3)), np.zeros((n, 3, 3)), np.zeros(n)
    _check(_load().orc_flex_run(st.N, _dp(st.r), _dp(st.p), _dp(st.F), _dp(st.q), _dp(st.m), _dp(st.h), _dp(st.ph),
                                _dp(st.W), step0, n, ctypes.byref(st.bind(prm)), _dp(hs), _dp(Ps), _dp(H)), "flex_run")
    return hs, Ps, H


# ---------------------------------------------------------------------------------
# Rigid 3-site water (water_oracle.c)
class WaterParams(ctypes.Structure):
    """Constraint settings of the rigid-water step (mirrors orc_water_params)."""
    _fields_ = [("d_OH", ctypes.c_double), ("d_HH", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("pad", ctypes.c_int32)]


def water_params(d_OH=1.0, angle_deg=109.47, tol=1e-14, max_iter=500) -> WaterParams:
    """O-H length, H-O-H angle (the H-H length follows), SHAKE tolerance and sweep limit."""
    d_HH = 2.0 * d_OH * math.sin(math.radians(angle_deg) / 2.0)
    return WaterParams(d_OH=d_OH, d_HH=d_HH, tol=tol, max_iter=max_iter, pad=0)


def _bind_water(lib):
    P = ctypes.POINTER(NptParams)
    Wp = ctypes.POINTER(WaterParams)
    lib.orc_water_real.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _c_double_p,
                                   _c_double_p, _c_double_p]
    lib.orc_water_real.restype = ctypes.c_int
    lib.orc_water_virial_corr.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, _c_double_p]
    lib.orc_water_virial_corr.restype = ctypes.c_double
    lib.orc_water_forces.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, _c_double_p,
                                     ctypes.c_uint64, P, _c_double_p, _c_double_p, _c_double_p]
    lib.orc_water_forces.restype = ctypes.c_int
    lib.orc_water_step.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, _c_double_p, _c_double_p,
                                   _c_double_p, _c_double_p, _c_double_p, ctypes.c_uint64, P, Wp, _c_double_p]
    lib.orc_water_step.restype = ctypes.c_int
    lib.orc_water_run.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, _c_double_p, _c_double_p,
                                  _c_double_p, _c_double_p, _c_double_p, ctypes.c_uint64, ctypes.c_int32, P, Wp,
                                  _c_double_p, _c_double_p, _c_double_p]
    lib.orc_water_run.restype = ctypes.c_int
    lib.orc_water_violation.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p, _c_double_p, Wp,
                                        _c_double_p]
    lib.orc_water_violation.restype = None


def water_real(pos, q, box, alpha, rc, qqr2e, lj_sigma, lj_eps):
    """Real space between molecules plus the exclusions: (F[3n,3], W trace, E_coul, E_lj, E_excl)."""
    pos = _f64(pos)
    q = _f64(q)
    F = np.zeros_like(pos)
    W = ctypes.c_double(0.0)
    E = np.zeros(3)
    _check(_load().orc_water_real(q.shape[0] // 3, _dp(pos), _dp(q), _dp(_f64(box, (3,))), alpha, rc, qqr2e,
                                  lj_sigma, lj_eps, _dp(F), ctypes.byref(W), _dp(E)), "water_real")
    return F, W.value, E[0], E[1], E[2]


def water_virial_corr(pos, m, box, F):
    """-sum_i F_i . d_i (d_i the site's offset from its molecule's centre)."""
    pos = _f64(pos)
    return _load().orc_water_virial_corr(pos.shape[0] // 3, _dp(pos), _dp(_f64(m)), _dp(_f64(box, (3,))),
                                         _dp(_f64(F)))


class WaterState:
    """Oracle state of the rigid-water step: sites (O, H, H per molecule), momenta, forces, box,
    piston momentum and molecular virial."""

    def __init__(self, r, p, q, m, L, pV=0.0):
        self.r = _f64(r).copy()
        self.p = _f64(p).copy()
        self.q = _f64(q)
        self.m = _f64(m)
        self.L = _f64(L, (3,)).copy()
        self.F = np.zeros_like(self.r)
        self.pV = ctypes.c_double(pV)
        self.W = ctypes.c_double(0.0)

    @property
    def Nmol(self):
        return self.q.shape[0] // 3


def water_forces(st: WaterState, step: int, prm: NptParams):
    E = np.zeros(4)
    _check(_load().orc_water_forces(st.Nmol, _dp(st.r), _dp(st.q), _dp(st.m), _dp(st.L), step, ctypes.byref(prm),
                                    _dp(st.F), ctypes.byref(st.W), _dp(E)), "water_forces")
    return E


def water_step(st: WaterState, step: int, prm: NptParams, wp: WaterParams):
    E = np.zeros(4)
    _check(_load().orc_water_step(st.Nmol, _dp(st.r), _dp(st.p), _dp(st.F), _dp(st.q), _dp(st.m), _dp(st.L),
                                  ctypes.byref(st.pV), ctypes.byref(st.W), step, ctypes.byref(prm), ctypes.byref(wp),
                                  _dp(E)), "water_step")
    return E


def water_run(st: WaterState, step0: int, n: int, prm: NptParams, wp: WaterParams):
    """n steps; returns (V, molecular P_ins, extended energy) per step."""
    V, Pi, H = np.zeros(n), np.zeros(n), np.zeros(n)
    _check(_load().orc_water_run(st.Nmol, _dp(st.r), _dp(st.p), _dp(st.F), _dp(st.q), _dp(st.m), _dp(st.L),
                                 ctypes.byref(st.pV), ctypes.byref(st.W), step0, n, ctypes.byref(prm),
                                 ctypes.byref(wp), _dp(V), _dp(Pi), _dp(H)), "water_run")
    return V, Pi, H


def water_violation(st: WaterState, wp: WaterParams):
    """(largest relative distance violation, largest relative velocity-constraint violation)."""
    out = np.zeros(2)
    _load().orc_water_violation(st.Nmol, _dp(st.r), _dp(st.p), _dp(st.m), _dp(st.L), ctypes.byref(wp), _dp(out))
    return out
