"""Pins of the oracle's RBE estimators (Sec. 4.2 Eqs. (appforce), (apppress); Sec. 4.4
Proposition 1; App. C) against the plain Ewald sum and against the mathematics."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2110_14362_gb300 import inputs


def _cube(kmax):
    m = np.array(list(itertools.product(range(-kmax, kmax + 1), repeat=3)), dtype=np.int32)
    return m[np.any(m != 0, axis=1)]


def test_weighted_full_k_equals_ewald():
    """Every m of the cube with weight exp(-|k|^2/4a) turns the estimator into the Ewald sum."""
    s = inputs.small_snapshot()
    pos, q = s.pos[:200], s.q[:200]
    box = np.array([10.0, 10.0, 12.0])
    alpha, kmax = 1.0, 10
    m = _cube(kmax)
    k = 2 * np.pi * m / box
    w = np.exp(-(k * k).sum(1) / (4 * alpha))
    F, W, Ek, Es, _ = oracle.rbe_kspace(pos, q, box, alpha, m, w)
    F0, W0, Ek0, Es0 = oracle.ewald_kspace(pos, q, box, alpha, kmax)
    assert abs(Ek - Ek0) < 1e-12 * abs(Ek0)
    assert Es == Es0
    assert np.abs(F - F0).max() < 1e-11 * np.abs(F0).max()
    assert np.abs(W - W0).max() < 1e-12 * np.abs(W0).max()


def test_zero_net_force_per_frequency():
    """sum_i q_i Im(e^{-ik.r_i} rho(k)) = Im(conj(rho) rho) = 0 for each sampled k."""
    s = inputs.small_snapshot()
    m, S = oracle.sample_k(s.box, s.alpha, 16, 12345, 0)
    for l in range(16):
        F, *_ = oracle.rbe_kspace(s.pos, s.q, s.box, s.alpha, m[l:l + 1], S)
        assert np.abs(F.sum(0)).max() < 1e-12 * np.abs(F).sum()


def test_trace_equals_scalar_pressure():
    """tr(W)/3V equals P_2* of Eq. (apppress) (isotropic remark of App. C)."""
    s = inputs.small_snapshot()
    box = np.array([10.0, 11.0, 9.0])
    m, S = oracle.sample_k(box, s.alpha, 50, 7, 1)
    F, W, Ek, Es, rho = oracle.rbe_kspace(s.pos, s.q, box, s.alpha, m, S / 50)
    V = box.prod()
    k = 2 * np.pi * m / box
    kk = (k * k).sum(1)
    P2 = 2 * np.pi / V ** 2 * np.sum(S / 50 * np.abs(rho) ** 2 / kk * (1 / 3 - kk / (6 * s.alpha)))
    assert abs(np.trace(W) / (3 * V) - P2) < 1e-12 * abs(P2)
    assert np.abs(W - W.T).max() < 1e-12 * np.abs(W).max()


def test_snapshot_is_sample_then_evaluate():
    s = inputs.small_snapshot()
    F, W, Ek, Es, m, S = oracle.rbe_snapshot(s.pos, s.q, s.box, s.alpha, s.P, 12345, 4)
    m2, S2 = oracle.sample_k(s.box, s.alpha, s.P, 12345, 4)
    F2, W2, Ek2, Es2, _ = oracle.rbe_kspace(s.pos, s.q, s.box, s.alpha, m2, S2 / s.P)
    assert np.array_equal(m, m2) and S == S2
    assert np.array_equal(F, F2) and np.array_equal(W, W2) and Ek == Ek2


def test_unbiased_with_proposition_1_variance():
    """E F* = F_{i,1} and E P_2* = P_2 (Eq. (EE)); the Monte-Carlo error of the batch mean is
    bounded with the exact single-sample variances of Eqs. (ForceExp), (PressExp)."""
    N, P, B = 40, 32, 3000
    box = np.array([8.0, 8.0, 9.0])
    rng = np.random.default_rng(4)
    pos = rng.random((N, 3)) * box
    q = np.where(np.arange(N) < N // 2, 1.0, -1.0)
    alpha, kmax = 1.0, 14
    V = box.prod()
    # exact target and the per-frequency terms for the variances
    mm = _cube(kmax)
    k = 2 * np.pi * mm / box
    kk = (k * k).sum(1)
    g = np.exp(-kk / (4 * alpha))
    S = g.sum()
    ph = k @ pos.T                                     # (K, N)
    rho = (np.exp(1j * ph) * q).sum(1)
    imt = np.cos(ph) * rho.imag[:, None] - np.sin(ph) * rho.real[:, None]  # Im(e^{-ik.r} rho)
    # one-sample estimator X_k = S * (-(4 pi q_i k/(V kk)) imt), drawn with prob g/S
    X = -S * (4 * np.pi / V) * (q[None, :, None] * k[:, None, :]) / kk[:, None, None] * imt[:, :, None]
    pk = g / S
    F_exact = np.einsum("k,kid->id", pk, X)
    var1 = np.einsum("k,kid->id", pk, X * X) - F_exact ** 2
    Fk, Wk, _, _ = oracle.ewald_kspace(pos, q, box, alpha, kmax)
    assert np.abs(F_exact - Fk).max() < 1e-11 * np.abs(Fk).max()
    # the variance of Eq. (ForceExp), summed over components, equals the per-component sum
    var_prop = (1.0 / 1) * (np.einsum("k,ki->i", (4 * np.pi * 1.0) ** 2 * S / (V ** 2 * kk) * g,
                                      (q[None, :] ** 2) * imt ** 2) - (Fk ** 2).sum(1))
    assert np.allclose(var_prop, var1.sum(1), rtol=1e-9, atol=1e-12 * var_prop.max())
    Y = S * 2 * np.pi / V ** 2 * np.abs(rho) ** 2 / kk * (1 / 3 - kk / (6 * alpha))
    P2 = np.trace(Wk) / (3 * V)
    varP = (pk * Y * Y).sum() - P2 ** 2
    acc = np.zeros((N, 3))
    accP = 0.0
    for b in range(B):
        F, W, Ek, Es, m, Sb = oracle.rbe_snapshot(pos, q, box, alpha, P, 99, b)
        acc += F
        accP += np.trace(W) / (3 * V)
    mean = acc / B
    sig = np.sqrt(var1 / (P * B))
    z = np.abs(mean - Fk) / sig
    assert z.max() < 5.0, z.max()
    zP = abs(accP / B - P2) / math.sqrt(varP / (P * B))
    assert zP < 5.0, zP


def test_all_cores_build_returns_the_same_bits():
    """The OpenMP timing build shares the frequencies (rho) and the particles (forces) among
    threads without changing any sum's order: every output equals the single-thread build's."""
    import subprocess
    try:
        oracle.build_omp()
    except (subprocess.CalledProcessError, OSError) as e:
        pytest.skip(f"no OpenMP runtime for gcc here: {e}")
    s = inputs.small_snapshot()
    m, S = oracle.sample_k(s.box, s.alpha, 37, 12345, 2)
    a = oracle.rbe_kspace(s.pos, s.q, s.box, s.alpha, m, S / 37)
    b = oracle.rbe_kspace(s.pos, s.q, s.box, s.alpha, m, S / 37, all_cores=True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("all_cores", [False, True])
def test_subset_forces_are_the_full_estimators_rows(all_cores):
    """The subset variant (rho over all particles, forces of listed particles only; the check of
    the largest workloads) returns, for any list of indices (repeats and any order allowed),
    the very rows of the full estimator, and the same rho, virial and energies bit for bit."""
    import subprocess
    if all_cores:
        try:
            oracle.build_omp()
        except (subprocess.CalledProcessError, OSError) as e:
            pytest.skip(f"no OpenMP runtime for gcc here: {e}")
    s = inputs.uniform_density(3000, P=64)
    m, S = oracle.sample_k(s.box, s.alpha, 64, 12345, 9)
    F, W, Ek, Es, rho = oracle.rbe_kspace(s.pos, s.q, s.box, s.alpha, m, S / 64)
    idx = np.random.default_rng(4).integers(0, 3000, 257)
    idx[:3] = [2999, 0, 2999]
    Fs, Ws, Eks, Ess, rhos = oracle.rbe_kspace_subset(s.pos, s.q, s.box, s.alpha, m, S / 64, idx, all_cores)
    assert np.array_equal(Fs, F[idx])
    assert np.array_equal(Ws, W) and Eks == Ek and Ess == Es and np.array_equal(rhos, rho)
    with pytest.raises(RuntimeError):
        oracle.rbe_kspace_subset(s.pos, s.q, s.box, s.alpha, m, S / 64, [3000])
