"""GPU parity of the fully flexible cell Langevin NPT step (App. A, the fully flexible cells; the
general-cell k-space of App. C) through the C ABI, against the oracle's flexible step on the same
inputs, noise and RBE batches: FP64 path 1e-10 relative on positions, momenta, forces, the cell,
its momenta and the full virial after a few steps of a sheared cell; FP32-phase path 1e-5.  With
the shear frozen and no chi term the device step equals the device's anisotropic rectangular
step; without friction and noise the device conserves the extended energy; bad input is
rejected."""
import numpy as np
import pytest

import oracle
import paper_2110_14362_gb300 as rbe

from gpu_util import cuda_device

pytestmark = pytest.mark.gpu

SEED = 777
ALPHA = 0.2
P = 80
KT = oracle.KB * 300.0
QQ = oracle.QQR2E / 78.5  # Coulomb screened by a water-like permittivity (see the rectangular tests)


def _system(counts, tilt, density=0.1, jitter=0.3, seed=0):
    """A jittered rock-salt lattice in the cell h = L (I + T), T strictly upper triangular with
    the entries of `tilt` (xy, xz, yz) times the edge of their column."""
    a = density ** (-1 / 3)
    L = a * np.asarray(counts, dtype=np.float64)
    h = np.diag(L)
    h[0, 1], h[0, 2], h[1, 2] = tilt[0] * L[1], tilt[1] * L[2], tilt[2] * L[2]
    rng = np.random.default_rng(seed)
    idx = np.stack(np.meshgrid(*[np.arange(n) for n in counts], indexing="ij"), -1).reshape(-1, 3)
    s = (idx + 0.5 + rng.uniform(-jitter / a, jitter / a, idx.shape)) / np.asarray(counts)
    pos = (s - np.floor(s)) @ h.T
    q = np.where(idx.sum(1) % 2 == 0, 1.0, -1.0)
    m = np.full(len(q), 20.0)
    mom = rng.normal(size=(len(q), 3)) * np.sqrt(KT * 100 * m)[:, None]
    return pos, mom, q, m, h


def _masses(h):
    """Cell masses of the rectangular barostat's scale on the diagonal, their geometric means off it."""
    Md = np.asarray(oracle.piston_masses_rect(2, 0.5, 4.5e-5 / oracle.BAR, np.diag(h)))
    return np.sqrt(np.outer(Md, Md))


def _params(h, rc, **kw):
    M = kw.pop("M", _masses(h))
    base = dict(dt=0.001, kT=KT, P_ext=oracle.BAR, gamma=10.0, gamma_h=2.0, M=M, rc=rc, qqr2e=QQ, lj_sigma=2.0,
                lj_eps=0.5, max_disp=0.05, chi=2.0, kspace=1, real=1, noise=1)
    base.update(kw)
    skin = base.pop("skin", 0.0)
    dev = rbe.FlexParams(skin=skin, **base)
    orc = oracle.flex_params(alpha=ALPHA, P=P, seed=SEED, **base)
    rates = np.array([[0.4, 0.3, -0.2], [-0.25, -0.3, 0.2], [0.15, -0.1, 0.2]])  # dh/dt, A/ps
    return dev, orc, np.asarray(M) * rates


def _run_both(counts, tilt, rc, nsteps, precision, **kw):
    pos, mom, q, m, h = _system(counts, tilt)
    prm_d, prm_o, ph = _params(h, rc, **kw)
    dev = cuda_device()
    with rbe.Context(np.diag(h), ALPHA, P, SEED, precision) as ctx:
        rep = rbe.FlexReplica(pos, mom, q, m, h, prm_d, dev, step=0, ph=ph)
        rep.init(ctx, batch=0)
        rep.step(ctx, nsteps)
        ctx.sync()
        got = rep.state()
    st = oracle.FlexState(pos, mom, q, m, h, ph=ph, P=P)
    E = oracle.flex_forces(st, 0, prm_o)
    for s in range(nsteps):
        E = oracle.flex_step(st, s, prm_o)
    return got, st, E


def _mi_dist(a, b, h):
    """Largest distance between the positions a and b by the minimum image of the cell h."""
    s = (a - b) @ np.linalg.inv(h).T
    s -= np.round(s)
    return np.abs(s @ h.T).max()


def _rel(a, b):
    return np.sqrt(np.mean((a - b) ** 2) / np.mean(b ** 2))


CASES = [  # (lattice counts, tilts xy, xz, yz, rc): 2 to 4 cells per axis of the cell list
    ((6, 6, 7), (0.15, -0.1, 0.12), 5.0),
    ((9, 8, 10), (-0.2, 0.18, 0.1), 6.0),
    ((12, 11, 13), (0.3, 0.05, -0.22), 6.0),
]


@pytest.mark.parametrize("counts,tilt,rc", CASES)
@pytest.mark.parametrize("skin", [0.0, 1.0])
def test_flex_fp64_parity(counts, tilt, rc, skin):
    got, st, E = _run_both(counts, tilt, rc, 4, rbe.RBE_FP64, skin=skin)
    assert got["builds"] == (1 if skin > 0 else 0)
    assert np.abs(got["h"] - st.h).max() < 1e-12 * np.abs(st.h).max(), (got["h"], st.h)
    assert np.abs(np.tril(got["h"], -1) - np.tril(st.h, -1)).max() < 1e-12 * np.abs(st.h).max()
    assert _mi_dist(got["r"], st.r, st.h) < 1e-10 * np.abs(st.h).max()
    assert np.abs(got["p"] - st.p).max() < 1e-10 * np.abs(st.p).max()
    assert np.abs(got["F"] - st.F).max() < 1e-10 * np.abs(st.F).max()
    assert np.abs(got["ph"] - st.ph).max() < 1e-10 * np.abs(st.ph).max(), (got["ph"], st.ph)
    assert np.abs(got["W"] - st.W).max() < 1e-10 * np.abs(st.W).max(), (got["W"], st.W)
    assert np.abs(got["W"] - got["W"].T).max() <= 1e-12 * np.abs(st.W).max()
    for a, b in ((got["Ek"], E[0]), (got["Ec"], E[1]), (got["El"], E[2])):
        assert abs(a - b) < 1e-10 * abs(b), (a, b)
    Kt = np.einsum("ia,ib->ab", st.p, st.p / st.m[:, None]) / 100.0
    V = np.linalg.det(st.h)
    assert abs(got["V"] - V) < 1e-12 * V
    assert np.abs(got["Pt"] - (Kt + st.W) / V).max() < 1e-10 * np.abs((Kt + st.W) / V).max()
    M = _masses(_system(counts, tilt)[4])
    H = 0.5 * np.trace(Kt) + E.sum() + oracle.BAR * V + 2.0 * KT * np.log(V) + np.sum(st.ph ** 2 / (2 * M))
    assert abs(got["H"] - H) < 1e-9 * abs(H), (got["H"], H)
    assert got["step"] == 4


@pytest.mark.parametrize("kw", [dict(kspace=0), dict(real=0), dict(noise=0), dict(chi=0.0),
                                dict(gamma=0.0, gamma_h=0.0, noise=0)])
def test_flex_fp64_components(kw):
    got, st, E = _run_both((8, 8, 9), (0.2, -0.15, 0.1), 6.0, 3, rbe.RBE_FP64, **kw)
    assert np.abs(got["h"] - st.h).max() < 1e-12 * np.abs(st.h).max()
    assert _mi_dist(got["r"], st.r, st.h) < 1e-10 * np.abs(st.h).max()
    assert np.abs(got["p"] - st.p).max() < 1e-10 * np.abs(st.p).max()
    assert np.abs(got["F"] - st.F).max() < 1e-10 * np.abs(st.F).max()
    assert np.abs(got["ph"] - st.ph).max() < 1e-10 * np.abs(st.ph).max()
    assert np.abs(got["W"] - st.W).max() < 1e-10 * np.abs(st.W).max()


@pytest.mark.parametrize("skin", [0.0, 1.0])
def test_flex_fp32_phase_parity(skin):
    """FP32 real space and FP32-phase k-space: forces and momenta to 1e-5 relative RMS, the virial
    to 1e-5 of its largest entry, the cell momenta to 1e-5 of the scale of their kicks (the force
    on p^h is a small difference of Kt + W and P V) and the cell to what that moves it."""
    nsteps, dt = 4, 0.001
    got, st, E = _run_both((10, 9, 11), (0.2, -0.1, 0.15), 6.0, nsteps, rbe.RBE_FP32_PHASE, skin=skin)
    assert _rel(got["F"], st.F) < 1e-5
    assert _rel(got["p"], st.p) < 1e-5
    assert np.abs(got["W"] - st.W).max() < 1e-5 * np.abs(st.W).max()
    Kt = np.einsum("ia,ib->ab", st.p, st.p / st.m[:, None]) / 100.0
    V = np.linalg.det(st.h)
    kick = 2 * nsteps * 0.5 * dt * (np.abs(Kt).max() + np.abs(st.W).max() + oracle.BAR * V) * \
        np.abs(np.linalg.inv(st.h)).max() * 3
    assert np.abs(got["ph"] - st.ph).max() < 1e-5 * kick
    M = _masses(_system((10, 9, 11), (0.2, -0.1, 0.15))[4])
    assert np.abs(got["h"] - st.h).max() < 1e-5 * kick * nsteps * dt / M.min() + 1e-12 * np.abs(st.h).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_neighbour_list_rebuilds_and_matches_the_cell_search(precision):
    """200 steps of a cell deforming at several A/ps with a thin skin: the list is rebuilt many
    times (displacements and the deformation h h_ref^{-1} both count), and the trajectory is the
    cell search's to rounding."""
    prec = rbe.RBE_FP64 if precision == "fp64" else rbe.RBE_FP32_PHASE
    pos, mom, q, m, h = _system((8, 8, 9), (0.2, -0.15, 0.1))
    dev = cuda_device()
    out = []
    for skin in (0.0, 0.4):
        prm, _, ph = _params(h, 6.0, skin=skin)
        with rbe.Context(np.diag(h), ALPHA, P, SEED, prec) as ctx:
            rep = rbe.FlexReplica(pos, mom, q, m, h, prm, dev, step=0, ph=ph * 4.0)
            rep.init(ctx, batch=0)
            rep.step(ctx, 200)
            ctx.sync()
            out.append(rep.state())
    a, b = out
    assert a["builds"] == 0 and b["builds"] >= 5, b["builds"]
    assert np.abs(b["h"] - h).max() > 0.2  # the cell moved by more than the skin
    tol = 1e-8 if precision == "fp64" else 2e-3
    assert np.abs(a["h"] - b["h"]).max() < tol * np.abs(a["h"]).max()
    assert _rel(b["p"], a["p"]) < tol
    assert _rel(b["F"], a["F"]) < tol * 10


def test_frozen_shear_without_chi_is_the_rectangular_device_step():
    """A diagonal h, chi = 0, off-diagonal masses of 1e300: the general-cell MH chain proposes the
    exact product law (every proposal accepted), and the flexible step is the anisotropic
    rectangular step on the device to rounding."""
    pos, mom, q, m, h = _system((8, 9, 10), (0.0, 0.0, 0.0))
    box = np.diag(h).copy()
    Md = np.asarray(oracle.piston_masses_rect(2, 0.5, 4.5e-5 / oracle.BAR, box))
    rates = np.array([0.4, -0.3, 0.2])
    common = dict(dt=0.001, kT=KT, P_ext=oracle.BAR, gamma=10.0, rc=6.0, qqr2e=QQ, lj_sigma=2.0, lj_eps=0.5,
                  max_disp=0.05, kspace=1, real=1, noise=1)
    M = np.full((3, 3), 1e300)
    M[np.diag_indices(3)] = Md
    dev = cuda_device()
    with rbe.Context(box, ALPHA, P, SEED, rbe.RBE_FP64) as ctx:
        rect = rbe.NptReplica(pos, mom, q, m, box, rbe.NptParams(barostat=2, M_cell=Md, gamma_V=2.0, M_V=0.0, **common),
                              dev, step=0, pc=Md * rates)
        rect.init(ctx, batch=0)
        rect.step(ctx, 5)
        ctx.sync()
        r1, p1, F1, L1, c1 = rect.state()
    with rbe.Context(box, ALPHA, P, SEED, rbe.RBE_FP64) as ctx:
        flex = rbe.FlexReplica(pos, mom, q, m, h, rbe.FlexParams(gamma_h=2.0, M=M, chi=0.0, **common), dev, step=0,
                               ph=np.diag(Md * rates))
        flex.init(ctx, batch=0)
        flex.step(ctx, 5)
        ctx.sync()
        got = flex.state()
    assert np.abs(np.diag(got["h"]) - L1).max() < 1e-12 * L1.max()
    assert np.abs(got["h"] - np.diag(np.diag(got["h"]))).max() < 1e-100
    assert _mi_dist(got["r"], r1, np.diag(L1)) < 1e-10 * L1.max()
    assert np.abs(got["p"] - p1).max() < 1e-10 * np.abs(p1).max()
    assert np.abs(got["F"] - F1).max() < 1e-10 * np.abs(F1).max()
    pc = c1[rbe.CELL_PC:rbe.CELL_PC + 3]
    assert np.abs(np.diag(got["ph"]) - pc).max() < 1e-10 * np.abs(pc).max()
    assert np.abs(np.diag(got["W"]) - c1[rbe.CELL_WD:rbe.CELL_WD + 3]).max() < 1e-10 * np.abs(np.diag(got["W"])).max()


def test_flex_energy_conservation_on_device():
    """No friction or noise, real space only (the RBE force is a random batch): the extended
    energy with chi kT ln V drifts by O(dt^2), as in the oracle, over 400 steps with all nine
    cell entries moving, and the device's energy follows the oracle's."""
    rng = np.random.default_rng(5)
    h = np.array([[16.0, 1.5, -1.0], [0.0, 16.0, 2.0], [0.0, 0.0, 16.0]])
    u = (np.arange(3) + 0.5) / 3
    s = np.stack(np.meshgrid(u, u, u, indexing="ij"), -1).reshape(-1, 3) + rng.uniform(-0.004, 0.004, (27, 3))
    q = np.where(np.arange(27) % 2 == 0, 0.3, -0.3)
    m = np.full(27, 20.0)
    p = rng.normal(size=(27, 3)) * np.sqrt(KT * 100 * m)[:, None] * 0.1
    ph = np.array([[2.0, 1.0, -1.5], [1.2, -2.0, 1.0], [-1.0, 1.5, 1.8]])
    kw = dict(dt=0.001, kT=KT, P_ext=oracle.BAR, gamma=0.0, gamma_h=0.0, M=np.full((3, 3), 5.0), rc=6.2,
              qqr2e=oracle.QQR2E, lj_sigma=2.0, lj_eps=0.5, max_disp=0.0, chi=2.0, kspace=0, real=1, noise=0)
    # (the widths of this 16 A cell leave no room for a skin: rc already fills half of them)
    dev = cuda_device()
    Hd = []
    with rbe.Context(np.diag(h), ALPHA, P, SEED, rbe.RBE_FP64) as ctx:
        rep = rbe.FlexReplica(s @ h.T, p, q, m, h, rbe.FlexParams(**kw), dev, step=0, ph=ph)
        rep.init(ctx, batch=0)
        for _ in range(40):
            rep.step(ctx, 10)
            Hd.append(float(rep.cell[rbe.FLEX_HAM].item()))
        ctx.sync()
        got = rep.state()
    st = oracle.FlexState(s @ h.T, p, q, m, h, ph=ph)
    prm = oracle.flex_params(alpha=ALPHA, P=P, seed=SEED, **kw)
    oracle.flex_forces(st, 0, prm)
    hs, _, H = oracle.flex_run(st, 0, 400, prm)
    Hd = np.array(Hd)
    assert np.abs(Hd - Hd[0]).max() < 1e-6, np.abs(Hd - Hd[0]).max()
    assert np.abs(Hd - H[9::10]).max() < 1e-8
    assert np.abs(got["h"] - st.h).max() < 1e-9 * 16


def test_flex_rejects_bad_input():
    import torch
    pos, mom, q, m, h = _system((6, 6, 7), (0.1, 0.0, 0.0))
    dev = cuda_device()
    with rbe.Context(np.diag(h), ALPHA, P, SEED, rbe.RBE_FP64) as ctx:
        good = _params(h, 5.0)[0]
        for bad_h in (np.zeros((3, 3)), np.diag([13.0, 13.0, -15.0]), np.diag([13.0, np.nan, 15.0])):
            rep = rbe.FlexReplica(pos, mom, q, m, bad_h, good, dev)
            with pytest.raises(rbe.RBEError) as e:
                rep.init(ctx)
            assert e.value.status == rbe.RBE_EINVAL
        # rc beyond half the smallest width
        rep = rbe.FlexReplica(pos, mom, q, m, h, _params(h, 7.0)[0], dev)
        with pytest.raises(rbe.RBEError):
            rep.init(ctx)
        Mbad = _masses(h)
        Mbad[1, 2] = 0.0
        rep = rbe.FlexReplica(pos, mom, q, m, h, _params(h, 5.0, M=Mbad)[0], dev)
        with pytest.raises(rbe.RBEError):
            rep.init(ctx)
        # stepping before init is refused; the context stays usable
        rep = rbe.FlexReplica(pos, mom, q, m, h, good, dev)
        with pytest.raises(rbe.RBEError) as e:
            rep.step(ctx, 1)
        assert e.value.status == rbe.RBE_ESTATE
        rep.init(ctx)
        rep.step(ctx, 2)
        ctx.sync()
        assert torch.isfinite(rep.pos).all()


def test_flex_graph_replay_equals_direct_steps():
    """One step captured in a CUDA graph and replayed three times ends bit for bit where three
    direct steps end (the step index lives on the device; every sum runs in a fixed order)."""
    import torch
    pos, mom, q, m, h = _system((8, 8, 9), (0.2, -0.15, 0.1))
    prm, _, ph = _params(h, 6.0, skin=1.0)
    dev = cuda_device()
    out = []
    for use_graph in (False, True):
        s = torch.cuda.Stream()
        with rbe.Context(np.diag(h), ALPHA, P, SEED, rbe.RBE_FP32_PHASE, stream=s.cuda_stream) as ctx:
            rep = rbe.FlexReplica(pos, mom, q, m, h, prm, dev, step=0, ph=ph)
            rep.init(ctx, batch=0)
            ctx.sync()
            if use_graph:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
                    rep.step(ctx, 1)
                for _ in range(3):
                    g.replay()
                torch.cuda.synchronize()
            else:
                rep.step(ctx, 3)
            ctx.sync()
            out.append(rep.state())
    a, b = out
    assert b["step"] == 3
    for k in ("r", "p", "F", "h", "ph", "W"):
        assert np.array_equal(a[k], b[k]), k


def test_flex_cell_leaving_the_prepared_range_is_reported():
    """A cell edge driven down at 1000 A/ps (a light mass on h_xx; no interactions, so nothing
    pushes back, but the real-space cell list still runs) falls below 2 rc within a few steps: the
    step flags it and the next sync reports RBE_ESTATE (no fault: the cell list keeps at least one
    cell per axis and every index in range)."""
    pos, mom, q, m, h = _system((6, 6, 7), (0.15, -0.1, 0.12))
    M = _masses(h)
    M[0, 0] = 0.01
    prm, _, _ = _params(h, 5.0, M=M, noise=0, lj_eps=0.0, qqr2e=0.0, kspace=0)
    ph = np.zeros((3, 3))
    ph[0, 0] = -1000.0 * M[0, 0]
    dev = cuda_device()
    with rbe.Context(np.diag(h), ALPHA, P, SEED, rbe.RBE_FP64) as ctx:
        rep = rbe.FlexReplica(pos, mom, q, m, h, prm, dev, ph=ph)
        rep.init(ctx)
        rep.step(ctx, 4)
        with pytest.raises(rbe.RBEError) as e:
            ctx.sync()
        assert e.value.status == rbe.RBE_ESTATE
        st = rep.state()
        assert st["h"][0, 0] < 12.0 and np.isfinite(st["r"]).all()


def test_flex_single_particle_matches_oracle():
    """One charge in a sheared cell: no pairs, a k-space force of zero up to rounding (the batch's
    Im(e^{-ik.r} rho) cancels) but a k-space virial and energy; the cell and the particle follow the
    oracle."""
    h = np.array([[12.0, 2.0, -1.0], [0.0, 13.0, 1.5], [0.0, 0.0, 14.0]])
    pos, mom = np.array([[3.0, 4.0, 5.0]]), np.array([[10.0, -5.0, 3.0]])
    q, m = np.array([1.0]), np.array([20.0])
    prm_d, prm_o, ph = _params(h, 5.0)
    dev = cuda_device()
    with rbe.Context(np.diag(h), ALPHA, P, SEED, rbe.RBE_FP64) as ctx:
        rep = rbe.FlexReplica(pos, mom, q, m, h, prm_d, dev, step=0, ph=ph)
        rep.init(ctx, batch=0)
        rep.step(ctx, 3)
        ctx.sync()
        got = rep.state()
    st = oracle.FlexState(pos, mom, q, m, h, ph=ph, P=P)
    oracle.flex_forces(st, 0, prm_o)
    for s in range(3):
        E = oracle.flex_step(st, s, prm_o)
    assert np.abs(got["h"] - st.h).max() < 1e-12 * np.abs(st.h).max()
    assert _mi_dist(got["r"], st.r, st.h) < 1e-10 * np.abs(st.h).max()
    assert np.abs(got["p"] - st.p).max() < 1e-10 * np.abs(st.p).max()
    assert np.abs(got["F"]).max() < 1e-9 and np.abs(st.F).max() < 1e-9
    assert np.abs(got["W"] - st.W).max() < 1e-10 * np.abs(st.W).max()
    assert abs(got["Ek"] - E[0]) < 1e-10 * abs(E[0])
