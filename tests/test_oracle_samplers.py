"""Pins of the oracle's variant samplers (Sec. 4.3: the offline rounded Gaussian and the online
Metropolis--Hastings chain) and of the arithmetic they decide integers with: the own logarithm
and erfc against libm / SciPy, the polar normals against the normal law, the offline draws
against the rounded-Gaussian law (and not the discrete Gaussian: the bias the paper points
out), and the chain against the exact discrete Gaussian, from an exact start and from a far one."""
import math

import numpy as np
import pytest
from scipy import special, stats

import oracle

ALPHA = 0.2


def _sigmas(box, alpha=ALPHA):
    return np.sqrt(alpha / 2.0) * np.asarray(box, dtype=np.float64) / math.pi


def _support(sig):
    A = int(math.ceil(12 * max(sig))) + 2
    return np.arange(-A, A + 1)


def _exact_marginal(box, axis, alpha=ALPHA):
    """P(m_axis = a) under exp(-pi^2 |m / l|^2 / alpha) on Z^3 without 0 (Eq. (probexpression)),
    from the definition (summed with NumPy)."""
    a = _support(_sigmas(box))
    w = [np.exp(-(math.pi ** 2) * a.astype(float) ** 2 / (alpha * l * l)) for l in box]
    H = [x.sum() for x in w]
    others = np.prod([H[j] for j in range(3) if j != axis])
    p = w[axis] * others
    p[a == 0] -= 1.0  # remove m = 0 (all three weights are 1 there)
    return a, p / (np.prod(H) - 1.0)


def _rounded_marginal(box, axis, alpha=ALPHA):
    """P(m_axis = a) when each m_j = rint(sigma_j z_j), z standard normal, redrawn on m = 0."""
    sig = _sigmas(box, alpha)
    a = _support(sig)
    q = [stats.norm.cdf((a + 0.5) / s) - stats.norm.cdf((a - 0.5) / s) for s in sig]
    q0 = [x[a == 0][0] for x in q]
    p = q[axis].copy()
    p[a == 0] -= q0[0] * q0[1] * q0[2]
    return a, p / (1.0 - q0[0] * q0[1] * q0[2])


def _chi2_pvalue(samples, a, p):
    n = samples.size
    counts = np.array([(samples == v).sum() for v in a], dtype=float)
    exp = p * n
    keep = exp >= 5
    # lump the sparse tails into one bin
    obs = np.append(counts[keep], counts[~keep].sum())
    ex = np.append(exp[keep], exp[~keep].sum())
    if ex[-1] < 5:
        obs[-2] += obs[-1]
        ex[-2] += ex[-1]
        obs, ex = obs[:-1], ex[:-1]
    assert abs(obs.sum() - ex.sum()) < 1e-6 * n
    return stats.chisquare(obs, ex).pvalue


def test_own_log_within_2_ulp():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.random(20000), 10.0 ** rng.uniform(-300, 300, 2000),
                         [2.0 ** -1074, 2.0 ** -1022, 0.5, 1 - 2.0 ** -53, 1.0, 2.0, 1e308]])
    for x in xs:
        got, ref = oracle.own_log(x), math.log(x)
        assert abs(got - ref) <= 2 * math.ulp(ref) + (0.0 if ref else 0.0), (x, got, ref)


def test_own_erfc_against_scipy():
    """On [0, 2] erfc = 1 - erf with erf summed from terms up to ~10 in size (near x = 2), so its
    error is absolute, a few times 10 ulp(1); beyond, the continued fraction is relative to 1e-15."""
    xs = np.linspace(0.0, 25.99, 30001)
    got = np.array([oracle.own_erfc(x) for x in xs])
    ref = special.erfc(xs)
    assert np.all(np.abs(got - ref) <= 3e-15 + 1e-14 * ref)
    assert oracle.own_erfc(26.0) == 0.0 and oracle.own_erfc(40.0) == 0.0


def test_rounded_gauss_mass():
    for sigma in (0.3, 1.0, 2.7, 15.0):
        g = 1.0 / (sigma * math.sqrt(2.0))
        ms = np.arange(-int(12 * sigma) - 3, int(12 * sigma) + 4)
        got = np.array([oracle.rounded_gauss_mass(int(m), g) for m in ms])
        # reference from the survival function on the positive side (no cancellation in the tail)
        am = np.abs(ms)
        ref = np.where(am > 0, stats.norm.sf((am - 0.5) / sigma) - stats.norm.sf((am + 0.5) / sigma),
                       special.erf(0.5 / (sigma * math.sqrt(2.0))))
        # a difference of two erfc values, each with the absolute error above
        assert np.all(np.abs(got - ref) <= 1e-13 * ref + 3e-15)
        assert abs(got.sum() - 1.0) < 1e-13
        assert np.array_equal(got, got[::-1])  # symmetric by construction


def test_polar_normals_law():
    z, trials, ok = [], 40000, 0
    for d in range(trials):
        good, pr = oracle.polar_pair(9, 3, d % 7, d, )
        if good:
            ok += 1
            z.extend(pr)
    # acceptance pi/4 within 5 sigma of a binomial
    assert abs(ok / trials - math.pi / 4) < 5 * math.sqrt((math.pi / 4) * (1 - math.pi / 4) / trials)
    assert stats.kstest(np.array(z), "norm").pvalue > 1e-3


@pytest.mark.parametrize("box", [(10.0, 12.0, 14.0), (4.0, 5.0, 30.0)])
def test_offline_follows_the_rounded_gaussian(box):
    m = np.concatenate([oracle.sample_k_offline(box, ALPHA, 4000, 11, s)[0] for s in range(5)])
    assert not np.any(np.all(m == 0, axis=1))
    for axis in range(3):
        a, p = _rounded_marginal(box, axis)
        assert _chi2_pvalue(m[:, axis], a, p) > 1e-4, axis


def test_offline_is_biased_where_the_rounding_matters():
    """sigma_x = 0.32 (l = 4.5): the rounded Gaussian puts visibly more mass on m_x = 0 than the
    discrete Gaussian does; the offline draws follow the former and fail the latter."""
    box = (4.5, 4.5, 4.5)
    m = np.concatenate([oracle.sample_k_offline(box, ALPHA, 5000, 5, s)[0] for s in range(6)])
    a, p_ex = _exact_marginal(box, 0)
    a2, p_rd = _rounded_marginal(box, 0)
    assert np.array_equal(a, a2)
    tv = 0.5 * np.abs(p_ex - p_rd).sum()
    assert tv > 0.01  # a real bias at this size
    assert _chi2_pvalue(m[:, 0], a, p_rd) > 1e-4
    assert _chi2_pvalue(m[:, 0], a, p_ex) < 1e-8


@pytest.mark.parametrize("box", [(4.5, 4.5, 4.5), (10.0, 12.0, 14.0)])
def test_mh_chain_keeps_the_exact_law(box):
    """Started from exact draws, each MH step leaves the discrete Gaussian invariant: after every
    step the slots (independent chains) follow it; most proposals are accepted."""
    P = 12000
    st = np.zeros((P, 3), dtype=np.int32)
    oracle.sample_k_mh(box, ALPHA, P, 21, 0, st)  # exact start
    prev = st.copy()
    moved = 0
    for s in range(1, 5):
        oracle.sample_k_mh(box, ALPHA, P, 21, s, st)
        moved += np.any(st != prev, axis=1).sum()
        prev = st.copy()
        for axis in range(3):
            a, p = _exact_marginal(box, axis)
            assert _chi2_pvalue(st[:, axis], a, p) > 1e-4, (s, axis)
    assert moved / (4 * P) > 0.5


def test_mh_chain_forgets_a_far_start_and_corrects_the_bias():
    """From m = (3, 0, 0) in every slot the chain reaches the discrete Gaussian within a few
    steps at l = 4.5, where the offline law (its proposal) is measurably different."""
    box = (4.5, 4.5, 4.5)
    P = 15000
    st = np.tile(np.array([3, 0, 0], dtype=np.int32), (P, 1))
    for s in range(12):
        oracle.sample_k_mh(box, ALPHA, P, 33, s, st)
    a, p_ex = _exact_marginal(box, 0)
    _, p_rd = _rounded_marginal(box, 0)
    assert _chi2_pvalue(st[:, 0], a, p_ex) > 1e-4
    assert _chi2_pvalue(st[:, 0], a, p_rd) < 1e-6
    assert not np.any(np.all(st == 0, axis=1))


def test_mh_slot_starts_from_the_exact_draw():
    box = (10.0, 12.0, 14.0)
    st = np.zeros((64, 3), dtype=np.int32)
    oracle.sample_k_mh(box, ALPHA, 64, 8, 3, st)
    m, S = oracle.sample_k(box, ALPHA, 64, 8, 3)
    assert np.array_equal(st, m)
    _, S2 = oracle.sample_k_offline(box, ALPHA, 1, 8, 3)
    assert S2 == S


def _offline_expectation_weights(box, alpha, kmax):
    """m over the cube |m_j| <= kmax without 0 and the weights S P_off(m) that make the weighted
    RBE sum the expectation of the offline estimator (S = sum of exp(-k^2/4 alpha) over m != 0)."""
    sig = _sigmas(box, alpha)
    r = np.arange(-kmax, kmax + 1)
    q = [stats.norm.sf((np.abs(r) - 0.5) / s) - stats.norm.sf((np.abs(r) + 0.5) / s) for s in sig]
    for j, s in enumerate(sig):
        q[j][r == 0] = special.erf(0.5 / (s * math.sqrt(2.0)))
    mm = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    mm = mm[np.any(mm != 0, axis=1)]
    p = q[0][mm[:, 0] + kmax] * q[1][mm[:, 1] + kmax] * q[2][mm[:, 2] + kmax]
    p0 = q[0][kmax] * q[1][kmax] * q[2][kmax]
    w = [np.exp(-(math.pi ** 2) * r.astype(float) ** 2 / (alpha * l * l)) for l in box]
    S = w[0].sum() * w[1].sum() * w[2].sum() - 1.0
    return mm.astype(np.int32), S * p / (1.0 - p0)


def offline_bias_case(alpha=0.05):
    """200 +-1 charges in a box of 10 (alpha = 0.05: sigma = 0.50 per axis; alpha = 1: sigma = 2.25):
    returns positions, charges, box, alpha and the exact expectations of the offline and the exact
    (Ewald) force and virial."""
    rng = np.random.default_rng(12)
    box, N = (10.0, 10.0, 10.0), 200
    pos = rng.random((N, 3)) * 10.0
    q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    kmax = 8 if alpha < 0.5 else 16
    m, w = _offline_expectation_weights(box, alpha, kmax)
    F_off, W_off, *_ = oracle.rbe_kspace(pos, q, box, alpha, m, w)
    F_ew, W_ew, *_ = oracle.ewald_kspace(pos, q, box, alpha, kmax)
    return pos, q, box, alpha, F_off, F_ew, W_off, W_ew


def test_offline_bias_is_exactly_computable_and_real():
    """The expectation of the offline estimator (weights S P_off(m) over the full cube) differs from
    the Ewald force by 21 % of its RMS at sigma = 0.5 and still by 1.8 % at sigma = 2.25: rounding a
    continuous Gaussian adds 1/12 to its variance, so the masses of the two laws differ at relative
    order 1/(24 sigma^2), not exponentially; the exact sampler's expectation (weights S P(m) =
    exp(-k^2/4 alpha)) is the Ewald force itself."""
    pos, q, box, alpha, F_off, F_ew, W_off, W_ew = offline_bias_case()
    rel = np.sqrt(np.mean((F_off - F_ew) ** 2) / np.mean(F_ew ** 2))
    assert rel > 0.1, rel
    *_, F_off2, F_ew2, _, _ = offline_bias_case(alpha=1.0)
    rel2 = np.sqrt(np.mean((F_off2 - F_ew2) ** 2) / np.mean(F_ew2 ** 2))
    assert 5e-3 < rel2 < rel / 4, (rel, rel2)
    r = np.arange(-8, 9)
    mm = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    mm = mm[np.any(mm != 0, axis=1)].astype(np.int32)
    k2 = ((2 * math.pi * mm / np.array(box)) ** 2).sum(1)
    F_ex, *_ = oracle.rbe_kspace(pos, q, box, alpha, mm, np.exp(-k2 / (4 * alpha)))
    assert np.abs(F_ex - F_ew).max() < 1e-12 * np.abs(F_ew).max()
    # the Monte-Carlo mean of the oracle's own offline draws heads for F_off, not F_ew
    acc = np.zeros_like(F_off)
    n = 60
    for s in range(n):
        m, S = oracle.sample_k_offline(box, alpha, 500, 3, s)
        acc += oracle.rbe_kspace(pos, q, box, alpha, m, S / 500)[0]
    mean = acc / n
    assert np.sqrt(np.mean((mean - F_off) ** 2)) < 0.5 * np.sqrt(np.mean((mean - F_ew) ** 2))
