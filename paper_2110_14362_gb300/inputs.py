"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method: only NumPy ``default_rng`` draws of
positions, charges and request streams with the shapes of the paper's workloads
(bulk water at 1 g/cm^3, a membrane-like slab, uniform +-1 charges at 0.1 per A^3).
Both the CUDA path and the FP64 oracle consume exactly these arrays.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class System:
    pos: np.ndarray      # (N, 3) float64, inside [0, box)
    q: np.ndarray        # (N,) float64
    box: np.ndarray      # (3,) float64
    alpha: float
    P: int
    rc: float
    name: str

    @property
    def N(self) -> int:
        return int(self.q.shape[0])


def _alternating(n: int) -> np.ndarray:
    q = np.ones(n)
    q[1::2] = -1.0
    return q


def uniform_pm1(N: int, box, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """N charges uniform in the box; the first half +1, the rest -1 (N even => neutral)."""
    box = np.asarray(box, dtype=np.float64).reshape(3)
    rng = np.random.default_rng(seed)
    pos = rng.random((N, 3)) * box
    q = np.where(np.arange(N) < N // 2, 1.0, -1.0)
    if N % 2:
        q[-1] = 0.0
    return pos, q


def small_snapshot(seed: int = 0) -> System:
    """1000 point charges (500 of +1, 500 of -1) uniform in a cubic box L = 10 (reduced
    units); alpha = 1, rc = 4, P = 100."""
    pos, q = uniform_pm1(1000, [10.0, 10.0, 10.0], seed)
    return System(pos, q, np.array([10.0, 10.0, 10.0]), 1.0, 100, 4.0, "snapshot-N1000-P100")


def slab(N: int = 300_000, seed: int = 0, box=(80.0, 80.0, 120.0), frac_slab: float = 0.6,
         sigma_z: float = 10.0, half_width: float = 20.0, P: int = 200, alpha: float = 0.2) -> System:
    """Membrane-like slab: ``frac_slab`` of the charges have z ~ N(Lz/2, sigma_z) truncated
    to |z - Lz/2| <= half_width, x and y uniform; the others are uniform in the box.  Charges
    alternate +-1 within each group, so each group is neutral."""
    box = np.asarray(box, dtype=np.float64)
    rng = np.random.default_rng(seed)
    ns = int(round(frac_slab * N))
    ns -= ns % 2
    nu = N - ns
    xy = rng.random((ns, 2)) * box[:2]
    z = np.empty(ns)
    filled = 0
    while filled < ns:
        cand = rng.normal(box[2] / 2, sigma_z, size=2 * (ns - filled) + 16)
        cand = cand[np.abs(cand - box[2] / 2) <= half_width]
        take = min(cand.size, ns - filled)
        z[filled:filled + take] = cand[:take]
        filled += take
    pos_s = np.column_stack([xy, z])
    pos_u = rng.random((nu, 3)) * box
    pos = np.vstack([pos_s, pos_u])
    q = np.concatenate([_alternating(ns), _alternating(nu)])
    return System(pos, q, box, alpha, P, 10.0, f"slab-N{N}-P{P}")


def uniform_density(N: int, density: float = 0.1, seed: int = 0, P: int = 100,
                    alpha: float = 0.2, rc: float = 7.0) -> System:
    """N neutral +-1 charges uniform in a cube at the given number density (per A^3)."""
    L = (N / density) ** (1.0 / 3.0)
    box = np.array([L, L, L])
    pos, q = uniform_pm1(N, box, seed)
    return System(pos, q, box, alpha, P, rc, f"uniform-N{N}-P{P}")


# SPC/E-like rigid water: O -0.8476 e, H +0.4238 e, O-H 1.0 A, H-O-H 109.47 deg.
WATER_Q = np.array([-0.8476, 0.4238, 0.4238])
WATER_MASS_G_PER_MOL = 18.01528
AVOGADRO_E_MINUS_24 = 0.602214076  # N_A * 1e-24 (A^3 per cm^3)


def water_box_length(n_mol: int, density_g_cm3: float = 1.0) -> float:
    return (n_mol * WATER_MASS_G_PER_MOL / (AVOGADRO_E_MINUS_24 * density_g_cm3)) ** (1.0 / 3.0)


def water(n_mol: int = 3000, seed: int = 0, P: int = 100, alpha: float = 0.25) -> System:
    """Rigid 3-site water molecules at random orientations on a jittered cubic lattice
    (the first n_mol sites of a seeded shuffle of the smallest n^3 >= n_mol lattice,
    jitter +-0.1 A), cubic box at 1.0 g/cm^3.  Returns the 3*n_mol site charges."""
    rng = np.random.default_rng(seed)
    L = water_box_length(n_mol)
    n = int(math.ceil(n_mol ** (1.0 / 3.0) - 1e-9))
    a = L / n
    grid = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1)
    grid = grid.reshape(-1, 3).astype(np.float64)
    sites = grid[rng.permutation(grid.shape[0])[:n_mol]]
    centres = (sites + 0.5) * a + rng.uniform(-0.1, 0.1, size=(n_mol, 3))
    half = math.radians(109.47) / 2
    local = np.array([[0.0, 0.0, 0.0],
                      [math.sin(half), 0.0, math.cos(half)],
                      [-math.sin(half), 0.0, math.cos(half)]])  # O-H = 1.0 A
    # random rotation per molecule from a normalised Gaussian quaternion
    qt = rng.normal(size=(n_mol, 4))
    qt /= np.linalg.norm(qt, axis=1, keepdims=True)
    w, x, y, z = qt.T
    R = np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], 1)
    pos = centres[:, None, :] + np.einsum("nij,sj->nsi", R, local)
    pos = np.mod(pos.reshape(-1, 3), L)
    q = np.tile(WATER_Q, n_mol)
    return System(pos, q, np.array([L, L, L]), alpha, P, 10.0, f"water-{n_mol}mol-P{P}")


def dipole_free_cluster(n_quartets: int, box, seed: int = 0, spread: float = 0.15):
    """Neutral, dipole-free charge sets: each quartet puts +q at c +- d and -q at c +- e
    (centre c, small d and e), so charge and dipole moment both vanish.  Positions are
    left unwrapped inside the box."""
    box = np.asarray(box, dtype=np.float64)
    rng = np.random.default_rng(seed)
    pos, q = [], []
    for _ in range(n_quartets):
        c = box * rng.uniform(0.35, 0.65, size=3)
        d = box * rng.uniform(-spread, spread, size=3)
        e = box * rng.uniform(-spread, spread, size=3)
        qq = rng.uniform(0.5, 1.5)
        pos += [c + d, c - d, c + e, c - e]
        q += [qq, qq, -qq, -qq]
    return np.array(pos), np.array(q)


@dataclass
class Request:
    rid: int
    arrival_s: float
    N: int
    seed: int


K_B_KJ_MOL_K = 0.00831446261815324  # Boltzmann constant, kJ/mol/K


def npt_replica(N: int, seed: int, density: float = 0.1, T: float = 300.0, mass: float = 20.0,
                jitter: float = 0.1):
    """Initial state of one NPT replica: N +-1 charges at `density` per A^3 in a cube, on the
    sites of a jittered cubic lattice (the smallest n^3 >= N grid of spacing a = L/n; N sites
    drawn without replacement; each displaced uniformly by up to +-jitter*a per axis), so
    that no two particles overlap; +1 on the first half of the drawn sites, -1 on the rest;
    masses `mass` g/mol and Maxwell-Boltzmann momenta at T (units g/mol A/ps, so that
    p^2/m/100 is in kJ/mol).  Returns pos, mom, q, m, box."""
    L = (N / density) ** (1.0 / 3.0)
    box = np.array([L, L, L])
    n = int(math.ceil(N ** (1.0 / 3.0) - 1e-9))
    a = L / n
    rng = np.random.default_rng(seed)
    grid = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    sites = grid[rng.permutation(n ** 3)[:N]].astype(np.float64)
    pos = np.mod((sites + 0.5 + rng.uniform(-jitter, jitter, (N, 3))) * a, L)
    q = np.where(np.arange(N) < N // 2, 1.0, -1.0)
    if N % 2:
        q[-1] = 0.0
    m = np.full(N, float(mass))
    mom = rng.standard_normal((N, 3)) * np.sqrt(K_B_KJ_MOL_K * T * 100.0 * m)[:, None]
    return pos, mom, q, m, box


def request_stream(n_req: int = 256, rate_per_s: float = 20.0, seed: int = 0,
                   n_lo: float = 1e3, n_hi: float = 1e5) -> list[Request]:
    """Poisson arrivals (exponential gaps) and per-request N = 2 floor(exp(U(ln lo, ln hi))/2)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=n_req)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for r in range(n_req):
        rr = np.random.default_rng(r)
        N = 2 * int(math.floor(math.exp(rr.uniform(math.log(n_lo), math.log(n_hi))) / 2))
        out.append(Request(r, float(t[r]), max(N, 2), r))
    return out
