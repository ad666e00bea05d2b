"""Pins of the oracle's general-cell (triclinic) k-space sums, dual-sum S and MH sampler (App. C,
the fully flexible cell): the rectangular limit, invariance under a unimodular change of lattice
basis, the NaCl Madelung constant in the two-ion primitive (rhombohedral) cell, the virial as the
strain derivative of the energy (shear included), S by Poisson summation against the direct
sum, the MH chain's stationary law against exact enumeration, and RBE unbiasedness."""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _sheared(L=(10.0, 11.0, 12.0), xy=2.0, xz=-1.5, yz=3.0):
    """Upper-triangular h: a = (lx, 0, 0), b = (xy, ly, 0), c = (xz, yz, lz) as columns."""
    return np.array([[L[0], xy, xz], [0.0, L[1], yz], [0.0, 0.0, L[2]]])


def _charges(N, h, seed):
    rng = np.random.default_rng(seed)
    s = rng.random((N, 3))
    q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    return s @ h.T, q


def test_rectangular_limit():
    box = np.array([9.0, 10.0, 11.0])
    pos, q = _charges(30, np.diag(box), 1)
    F0, W0, E0, Es0 = oracle.ewald_kspace(pos, q, box, 0.6, 8)
    F1, W1, E1, Es1 = oracle.gen_ewald_kspace(pos, q, np.diag(box), 0.6, 8)
    assert np.abs(F1 - F0).max() < 1e-12 * np.abs(F0).max()
    assert np.abs(W1 - W0).max() < 1e-12 * np.abs(W0).max()
    assert abs(E1 - E0) < 1e-12 * abs(E0) and Es1 == Es0


def test_unimodular_basis_change_is_invisible():
    """h' = h U with an integer U of determinant 1 spans the same lattice: the Ewald k-space and
    real-space sums (every image within rc) are the same (k sets agree once the cube holds every
    k that matters)."""
    h = _sheared()
    U = np.array([[1, 1, 0], [0, 1, 0], [1, 1, 1]])
    assert round(np.linalg.det(U)) == 1
    h2 = h @ U
    pos, q = _charges(24, h, 2)
    alpha = 0.35
    a = oracle.gen_ewald_kspace(pos, q, h, alpha, 16)
    b = oracle.gen_ewald_kspace(pos, q, h2, alpha, 24)
    assert np.abs(a[0] - b[0]).max() < 1e-11 * np.abs(a[0]).max()
    assert np.abs(a[1] - b[1]).max() < 1e-11 * np.abs(a[1]).max()
    assert abs(a[2] - b[2]) < 1e-11 * abs(a[2])
    ra = oracle.gen_ewald_real(pos, q, h, alpha, 7.0)
    rb = oracle.gen_ewald_real(pos, q, h2, alpha, 7.0)
    assert np.abs(ra[0] - rb[0]).max() < 1e-11 * np.abs(ra[0]).max() and abs(ra[2] - rb[2]) < 1e-11 * abs(ra[2])


def test_nacl_madelung_in_the_primitive_cell():
    """Rock salt with conventional constant a = 2 (nearest neighbours at d = 1) as the two-ion FCC
    primitive cell: the Ewald energy is -M / d, M the NaCl Madelung constant of the golden file."""
    gold = json.load(open(os.path.join(HERE, "golden", "lattice_constants.json")))
    M = gold["NaCl"]["madelung"]
    a = 2.0
    h = 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])  # columns: FCC vectors
    pos = np.array([[0.0, 0.0, 0.0], [0.5 * a, 0.0, 0.0]])
    q = np.array([1.0, -1.0])
    alpha = 2.0
    _, _, Ek, Es = oracle.gen_ewald_kspace(pos, q, h, alpha, 12)
    _, _, Er = oracle.gen_ewald_real(pos, q, h, alpha, 4.0)
    assert abs((Ek + Es + Er) + M / (0.5 * a)) < 2e-6 * M


@pytest.mark.parametrize("a,b", [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)])
def test_virial_is_the_strain_derivative(a, b):
    """W_ab = -dE_k/d eps_ab at fixed scaled coordinates, h -> (I + eps E_ab) h with the symmetric
    unit strain E_ab (shears included), central differences."""
    h = _sheared()
    s = np.random.default_rng(3).random((20, 3))
    q = np.where(np.arange(20) % 2 == 0, 1.0, -1.0)
    alpha, kmax = 0.3, 9
    _, W, _, _ = oracle.gen_ewald_kspace(s @ h.T, q, h, alpha, kmax)
    E = np.zeros((3, 3))
    E[a, b] = E[b, a] = 1.0 if a == b else 0.5
    eps = 1e-6
    Ep = []
    for sg in (1, -1):
        h2 = (np.eye(3) + sg * eps * E) @ h
        Ep.append(oracle.gen_ewald_kspace(s @ h2.T, q, h2, alpha, kmax)[2])
    d = -(Ep[0] - Ep[1]) / (2 * eps)
    expect = W[a, b] if a == b else 0.5 * (W[a, b] + W[b, a])
    assert abs(d - expect) < 1e-6 * max(1.0, np.abs(W).max()), (d, expect)


@pytest.mark.parametrize("alpha", [0.05, 0.3, 1.5])
def test_S_dual_sum_matches_direct_sum(alpha):
    h = _sheared()
    S, Sd = oracle.gen_S(h, alpha), oracle.gen_S(h, alpha, direct=True)
    assert abs(S - Sd) < 1e-12 * Sd, (S, Sd)


def _target_pairs(h, alpha, R):
    """Exact law of (m_x, m_y) under exp(-pi^2 m^T G m / alpha) on Z^3 \\ {0}, by enumeration."""
    G = oracle.gen_metric(h)
    r = np.arange(-R, R + 1)
    mm = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    w = np.exp(-(math.pi ** 2) / alpha * np.einsum("ni,ij,nj->n", mm, G, mm))
    w[np.all(mm == 0, axis=1)] = 0.0
    w /= w.sum()
    return mm, w


def _pair_chi2(samples, mm, w):
    keys = {}
    for (a, b, _), p in zip(mm, w):
        keys[(a, b)] = keys.get((a, b), 0.0) + p
    n = samples.shape[0]
    obs, ex = [], []
    rest_o, rest_e = 0.0, 0.0
    counts = {}
    for a, b in map(tuple, samples[:, :2]):
        counts[(a, b)] = counts.get((a, b), 0) + 1
    for k, p in keys.items():
        if p * n >= 5:
            obs.append(counts.get(k, 0))
            ex.append(p * n)
        else:
            rest_o += counts.get(k, 0)
            rest_e += p * n
    obs.append(rest_o)
    ex.append(rest_e)
    return stats.chisquare(obs, ex).pvalue


H_SMALL = np.array([[4.0, 2.2, 1.0], [0.0, 4.5, -1.6], [0.0, 0.0, 5.0]])  # strongly sheared


def test_general_mh_reaches_the_exact_law():
    """Independent chains (one per slot) from the product proposal's first draw: after eight MH
    steps the joint law of (m_x, m_y) is the exact non-factorised target (chi-square against
    enumeration), while the first draws (0.31 in total variation from the target in this strongly
    sheared cell) are not.  The proposal's precision is below the target's, so the ratio of the
    laws is bounded and the distance reaches the sampling noise within five steps (a proposal with
    the diagonal of the target's precision, too narrow, needed over a hundred)."""
    alpha, P = 0.3, 20000
    mm, w = _target_pairs(H_SMALL, alpha, 8)
    st = np.zeros((P, 3), dtype=np.int32)
    oracle.gen_sample_k_mh(H_SMALL, alpha, P, 7, 0, st)
    assert _pair_chi2(st, mm, w) < 1e-6  # the proposal alone ignores the shear
    moved = 0
    for s in range(1, 9):
        prev = st.copy()
        oracle.gen_sample_k_mh(H_SMALL, alpha, P, 7, s, st)
        moved += np.any(st != prev, axis=1).sum()
    assert _pair_chi2(st, mm, w) > 1e-4
    assert moved > 0.4 * 8 * P
    assert not np.any(np.all(st == 0, axis=1))


def test_general_rbe_is_unbiased():
    """The RBE force with the stationary MH frequencies and weights S/P (S by the dual sum) has the
    Ewald force as its mean: 20 groups of 1000 slots give the standard error."""
    alpha, P = 0.3, 20000
    h = H_SMALL * 2.0
    pos, q = _charges(16, h, 9)
    st = np.zeros((P, 3), dtype=np.int32)
    for s in range(10):
        _, S = oracle.gen_sample_k_mh(h, alpha, P, 11, s, st)
    Fg = np.stack([oracle.gen_kspace(pos, q, h, alpha, st[g * 1000:(g + 1) * 1000], S / 1000)[0] for g in range(20)])
    F_ew = oracle.gen_ewald_kspace(pos, q, h, alpha, 12)[0]
    mean, se = Fg.mean(0), Fg.std(0, ddof=1) / math.sqrt(20)
    chi = np.mean(((mean - F_ew) / se) ** 2)
    assert chi < 2.0, chi
    assert np.sqrt(np.mean((mean - F_ew) ** 2)) < 0.05 * np.sqrt(np.mean(F_ew ** 2))
