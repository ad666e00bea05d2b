"""Pins of the oracle's plain Ewald sum (Sec. 4.1; App. C) against facts fixed outside it:
textbook Madelung constants, independence of the splitting parameter alpha, a brute-force
image sum, and finite-difference derivatives of the energy with respect to the cell."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_2110_14362_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lattice_constants.json")


def _nacl():
    fcc = np.array([[0, 0, 0], [1, 1, 0], [1, 0, 1], [0, 1, 1]], float)
    pos = np.vstack([fcc, (fcc + [1, 0, 0]) % 2.0])
    q = np.array([1.0] * 4 + [-1.0] * 4)
    return pos, q, np.array([2.0, 2.0, 2.0])


def _cscl():
    base = np.array([[0, 0, 0], [0.5, 0.5, 0.5]])
    cells = np.array(list(itertools.product([0, 1], [0, 1], [0, 1])), float)
    pos = np.vstack([base + c for c in cells])
    q = np.tile([1.0, -1.0], 8)
    return pos, q, np.array([2.0, 2.0, 2.0])


@pytest.mark.parametrize("crystal", ["NaCl", "CsCl"])
@pytest.mark.parametrize("alpha", [25.0, 40.0])
def test_madelung(crystal, alpha):
    g = json.load(open(GOLDEN))[crystal]
    pos, q, box = _nacl() if crystal == "NaCl" else _cscl()
    F, W, E = oracle.ewald_total(pos, q, box, alpha, 1.0, 28)
    expect = -g["ion_pairs_per_cell"] * g["madelung"] / g["nn_distance"]
    assert abs(E / expect - 1.0) < 1e-9
    # every ion sits at a centre of symmetry: zero force
    assert np.abs(F).max() < 1e-12
    # cubic symmetry: isotropic virial, equal to the energy for a 1/r potential (W = -3V dE/dV / 3 = E/3 per axis)
    assert np.allclose(np.diag(W), E / 3.0, rtol=1e-9)
    assert np.abs(W - np.diag(np.diag(W))).max() < 1e-9 * abs(E)


def _random_neutral(N, box, seed):
    rng = np.random.default_rng(seed)
    pos = rng.random((N, 3)) * box
    q = rng.uniform(-1, 1, N)
    q -= q.mean()
    return pos, q


def test_alpha_independence():
    box = np.array([10.0, 10.0, 10.0])
    pos, q = _random_neutral(20, box, 3)
    ref = None
    for alpha in (1.2, 2.0, 3.0):
        F, W, E = oracle.ewald_total(pos, q, box, alpha, 5.0, 38)
        if ref is None:
            ref = (F, W, E)
            continue
        assert abs(E - ref[2]) < 1e-10 * abs(ref[2])
        assert np.abs(F - ref[0]).max() < 1e-9 * np.abs(ref[0]).max()
        assert np.abs(W - ref[1]).max() < 1e-9 * np.abs(ref[1]).max()


@pytest.mark.parametrize("box", [(10.0, 10.0, 10.0), (8.0, 10.0, 12.0)])
def test_brute_force_image_sum(box):
    box = np.array(box)
    pos, q = inputs.dipole_free_cluster(2, box, seed=11)
    assert abs(q.sum()) < 1e-15 and np.abs(q @ pos).max() < 1e-12
    _, _, E_ewald = oracle.ewald_total(pos, q, box, 1.5, 5.0 if box.min() >= 10 else 4.0, 40)
    Rs = np.array([16, 20, 24, 28, 32])
    Es = np.array([oracle.direct_sum(pos, q, box, int(R)) for R in Rs])
    # neutral, dipole-free cells interact as quadrupoles: the tail falls like R^-2
    A = np.column_stack([np.ones_like(Rs, dtype=float), 1.0 / Rs.astype(float) ** 2])
    coef, *_ = np.linalg.lstsq(A, Es, rcond=None)
    assert abs(coef[0] - E_ewald) < 2e-6 * np.abs(q).sum()


def _energy_scaled(pos, q, box, scale, alpha, rc, kmax):
    s = pos / box
    b2 = box * scale
    Fk, Wk, Ek, Es = oracle.ewald_kspace(s * b2, q, b2, alpha, kmax)
    Fr, Wr, Er = oracle.ewald_real(s * b2, q, b2, alpha, rc)
    return Ek + Es, Er


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_virial_is_length_derivative(axis):
    """W_tt = -l_t dE/dl_t at fixed scaled coordinates (Sec. 4.1; App. C Eq. (pressurerect)),
    separately for the k-space and the real-space parts."""
    box = np.array([9.0, 10.0, 11.0])
    pos, q = _random_neutral(24, box, 5)
    alpha, rc, kmax = 1.0, 4.4, 30
    _, Wk, _, _ = oracle.ewald_kspace(pos, q, box, alpha, kmax)
    _, Wr, _ = oracle.ewald_real(pos, q, box, alpha, rc)
    h = 1e-5
    up = np.ones(3); up[axis] += h
    dn = np.ones(3); dn[axis] -= h
    Ekp, Erp = _energy_scaled(pos, q, box, up, alpha, rc, kmax)
    Ekm, Erm = _energy_scaled(pos, q, box, dn, alpha, rc, kmax)
    dk = -(Ekp - Ekm) / (2 * h)
    dr = -(Erp - Erm) / (2 * h)
    assert abs(Wk[axis, axis] - dk) < 1e-7 * max(1.0, abs(dk))
    assert abs(Wr[axis, axis] - dr) < 1e-7 * max(1.0, abs(dr))


def _triclinic_kspace_energy(s, q, h, alpha, kmax):
    """U_1 for a general cell, k = 2 pi h^-T m (App. C), evaluated in NumPy for the shear pin."""
    m = np.array(list(itertools.product(range(-kmax, kmax + 1), repeat=3)), float)
    m = m[np.any(m != 0, axis=1)]
    k = 2 * np.pi * m @ np.linalg.inv(h)  # rows: (h^-T m)^T = m^T h^-1
    r = s @ h.T
    kk = (k * k).sum(1)
    rho = np.exp(1j * (k @ r.T)) @ q
    return 2 * np.pi / abs(np.linalg.det(h)) * np.sum(np.exp(-kk / (4 * alpha)) / kk * np.abs(rho) ** 2)


def _triclinic_real_energy(s, q, h, alpha, rc):
    from scipy.special import erfc
    E = 0.0
    N = len(q)
    shifts = np.array(list(itertools.product([-1, 0, 1], repeat=3)), float)
    for i in range(N):
        for j in range(i + 1, N):
            ds = s[j] - s[i]
            ds -= np.round(ds)
            d = (ds[None, :] + shifts) @ h.T
            r = np.linalg.norm(d, axis=1)
            r = r[r < rc]
            E += q[i] * q[j] * np.sum(erfc(np.sqrt(alpha) * r) / r)
    return E


@pytest.mark.parametrize("ab", [(0, 1), (0, 2), (1, 2)])
def test_offdiagonal_virial_is_shear_derivative(ab):
    """W_ab = -sum_g dU/dh_ag h_bg (App. C Eq. (pressuretensorflexible)): the derivative of
    the energy under the shear h -> (I + eps e_a e_b^T) h at fixed scaled coordinates."""
    a, b = ab
    box = np.array([9.0, 10.0, 11.0])
    pos, q = _random_neutral(12, box, 9)
    alpha, rc, kmax = 1.0, 4.0, 16
    _, Wk, _, _ = oracle.ewald_kspace(pos, q, box, alpha, kmax)
    _, Wr, _ = oracle.ewald_real(pos, q, box, alpha, rc)
    s = pos / box
    h0 = np.diag(box)
    eps = 1e-5
    S = np.zeros((3, 3)); S[a, b] = 1.0
    hp = (np.eye(3) + eps * S) @ h0
    hm = (np.eye(3) - eps * S) @ h0
    dk = -(_triclinic_kspace_energy(s, q, hp, alpha, kmax) - _triclinic_kspace_energy(s, q, hm, alpha, kmax)) / (2 * eps)
    dr = -(_triclinic_real_energy(s, q, hp, alpha, rc) - _triclinic_real_energy(s, q, hm, alpha, rc)) / (2 * eps)
    assert abs(Wk[a, b] - dk) < 1e-6 * max(1.0, np.abs(Wk).max())
    assert abs(Wr[a, b] - dr) < 1e-6 * max(1.0, np.abs(Wr).max())
    assert abs(Wk[a, b] - Wk[b, a]) < 1e-12 * np.abs(Wk).max()


def test_total_force_vanishes():
    box = np.array([10.0, 10.0, 10.0])
    pos, q = _random_neutral(40, box, 1)
    F, W, E = oracle.ewald_total(pos, q, box, 1.0, 4.0, 14)
    assert np.abs(F.sum(0)).max() < 1e-11 * np.abs(F).sum()


def test_force_is_position_gradient():
    """F_i = -grad_i U (Sec. 4.1 Eq. (force)) by central differences on one particle."""
    box = np.array([10.0, 10.0, 10.0])
    pos, q = _random_neutral(10, box, 2)
    alpha, rc, kmax = 1.0, 4.5, 24
    F, _, _ = oracle.ewald_total(pos, q, box, alpha, rc, kmax)
    h = 1e-6
    for t in range(3):
        pp = pos.copy(); pp[3, t] += h
        pm = pos.copy(); pm[3, t] -= h
        Ep = oracle.ewald_total(pp, q, box, alpha, rc, kmax)[2]
        Em = oracle.ewald_total(pm, q, box, alpha, rc, kmax)[2]
        assert abs(F[3, t] + (Ep - Em) / (2 * h)) < 1e-6 * max(1.0, abs(F[3, t]))
