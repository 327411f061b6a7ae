"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Tolerances (FP64 on both sides; they differ only in rounding order and FMA
contraction):
  * conservative variables after a number of steps: relative L-inf <= 1e-11
    per component, momenta normalised by the largest momentum component;
  * L(Q): relative L-inf <= 1e-11 (normalised by max |L| of the component);
  * dL/dt(Q): <= 1e-8; F^n_t = 4 (I(dt) - 2 I(dt/2)) / dt^2 cancels about
    four to five digits, so its rounding error is that much larger;
  * diagnostics: <= 1e-12 relative.
"""
import numpy as np
import pytest

from tests.inputs import rough_state, smooth_state

pytestmark = pytest.mark.gpu
GAMMA = 1.4


@pytest.fixture(scope="module")
def hg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2207_01173_gb300 import hgks
    return hgks


def rel_err(a, b, group_momenta=True):
    """per-component max |a - b| / max |b|; momenta share one normaliser."""
    scale = np.abs(b).reshape(5, -1).max(axis=1)
    if group_momenta:
        scale[1:4] = scale[1:4].max()
    scale = np.where(scale > 0, scale, 1.0)
    return np.abs(a - b).reshape(5, -1).max(axis=1) / scale


def pair(hg, oracle, n, **kw):
    return hg.Solver(n, **kw), oracle.RefSolver(n, **kw)


TGV_KW = dict(visc=(1, 1.0 / 1600, 1.0 / (GAMMA * 0.01), 0.7), Pr=0.72)


def channel_kw(Ma=0.5, Reb=2800.0):
    Tw = 1.0 / (GAMMA * Ma * Ma)
    return dict(lengths=(2 * np.pi, 2.0, np.pi), origin=(0.0, -1.0, 0.0), y_stretch_b=2.0,
                visc=(1, 1.0 / Reb, Tw, 0.7), Pr=0.7, bc_lo=(0, 1, 0), bc_hi=(0, 1, 0), T_wall=Tw,
                body_force=((180.0 / 2800.0) ** 2, 0.0, 0.0))


@pytest.mark.parametrize("n,seed", [((13, 11, 9), 1), ((8, 8, 8), 2), ((33, 5, 7), 3), ((6, 17, 4), 4)])
def test_rhs_smooth_periodic(hg, oracle, n, seed):
    g, c = pair(hg, oracle, n, visc=(0, 2e-3, 1.0, 0.0), Pr=0.72)
    q = smooth_state(n, seed)
    g.set_state(q)
    c.set_state(q)
    Lg, dLg = g.rhs(2e-3)
    Lc, dLc = c.rhs(2e-3)
    assert rel_err(Lg, Lc, False).max() < 1e-11
    assert rel_err(dLg, dLc, False).max() < 1e-8


def test_rhs_rough_power_law(hg, oracle):
    n = (10, 12, 11)
    g, c = pair(hg, oracle, n, **TGV_KW)
    q = rough_state(n, 9)
    g.set_state(q)
    c.set_state(q)
    Lg, dLg = g.rhs(1e-3)
    Lc, dLc = c.rhs(1e-3)
    assert rel_err(Lg, Lc, False).max() < 1e-11
    assert rel_err(dLg, dLc, False).max() < 1e-8


def test_rhs_channel_walls_stretched_force(hg, oracle):
    n = (9, 14, 7)
    g, c = pair(hg, oracle, n, **channel_kw())
    g.init_channel(0.5, 0.1, 2800)
    c.init_channel(0.5, 0.1, 2800)
    assert rel_err(g.get_state(), c.get_state()).max() < 1e-15
    Lg, dLg = g.rhs(5e-4)
    Lc, dLc = c.rhs(5e-4)
    assert rel_err(Lg, Lc, False).max() < 1e-11
    assert rel_err(dLg, dLc, False).max() < 1e-8


@pytest.mark.parametrize("n", [(16, 1, 1), (1, 12, 1), (1, 1, 10), (9, 7, 1), (1, 5, 6)])
def test_degenerate_directions(hg, oracle, n):
    """Grids one cell thick in some directions (periodic ghosts are copies of
    that single cell)."""
    kw = dict(lengths=(2.0, 2.0, 2.0), visc=(0, 0.0, 1.0, 0.0), Pr=1.0)
    g, c = pair(hg, oracle, n, **kw)
    g.init_density_wave(0.2)
    c.init_density_wave(0.2)
    assert rel_err(g.get_state(), c.get_state()).max() < 1e-14
    g.step(3, 0.5)
    c.step(3, 0.5)
    assert rel_err(g.get_state(), c.get_state()).max() < 1e-11


def test_dt_parity(hg, oracle):
    n = (20, 18, 16)
    g, c = pair(hg, oracle, n, **TGV_KW)
    g.init_tgv(0.1, 1.0, 1.0)
    c.init_tgv(0.1, 1.0, 1.0)
    assert g.compute_dt(0.5) == pytest.approx(c.compute_dt(0.5), rel=1e-15)


def test_tgv_32_ten_steps(hg, oracle):
    """Taylor-Green vortex 32^3 FP64, Ma 0.1, Re 1600, Pr 0.72, power-law
    viscosity, 10 steps at CFL 0.5: the GPU state matches the oracle within
    1e-11 relative L-inf, and the diagnostics within 1e-12."""
    n = (32, 32, 32)
    g, c = pair(hg, oracle, n, **TGV_KW)
    g.init_tgv(0.1, 1.0, 1.0)
    c.init_tgv(0.1, 1.0, 1.0)
    g.step(10, 0.5)
    c.step(10, 0.5)
    err = rel_err(g.get_state(), c.get_state())
    assert err.max() < 1e-11, err
    sg, sc = g.stats(), c.stats()
    assert sg["step"] == sc["step"] == 10
    assert sg["t"] == pytest.approx(sc["t"], rel=1e-14)
    for k in ("Ek", "enstrophy", "eps_com", "mass", "energy", "max_mach"):
        assert sg[k] == pytest.approx(sc[k], rel=1e-12), k


def test_channel_ten_steps(hg, oracle):
    """Compressible channel (Ma_b 0.5, Re_b 2800, stretched y, isothermal
    walls, body force, seeded noise) at reduced size, 10 steps."""
    n = (16, 24, 12)
    g, c = pair(hg, oracle, n, **channel_kw())
    g.init_channel(0.5, 0.1, 2800)
    c.init_channel(0.5, 0.1, 2800)
    g.step(10, 0.5)
    c.step(10, 0.5)
    err = rel_err(g.get_state(), c.get_state())
    assert err.max() < 1e-11, err
    sg, sc = g.stats(), c.stats()
    assert sg["wall_shear"] == pytest.approx(sc["wall_shear"], rel=1e-10)
    assert sg["Ek"] == pytest.approx(sc["Ek"], rel=1e-12)


def test_free_stream_bitwise(hg):
    n = (7, 5, 6)
    g = hg.Solver(n, lengths=(1.0, 2.0, 1.5), visc=(0, 1e-3, 1.0, 0.0))
    q = np.empty((5, 6, 5, 7))
    for c, v in enumerate((1.3, 0.52, -0.325, 0.13, 2.4)):
        q[c] = v
    g.set_state(q)
    g.step(5, 0.5)
    assert np.array_equal(g.get_state(), q)


def test_nonfinite_keeps_last_good_state(hg):
    """A non-finite cell: the step reports HGKS_ERR_NONFINITE and leaves
    state, time and step counter unchanged.  (A cell with negative internal
    energy alone is not enough: the neighbouring fluxes refill it within a
    stage, because WENO keeps the hole out of the neighbours' stencils.)"""
    n = (8, 8, 8)
    g = hg.Solver(n, **TGV_KW)
    g.init_tgv(0.1, 1.0, 1.0)
    g.step(2, 0.5)
    before = g.get_state()
    st0 = g.stats()
    bad = before.copy()
    bad[4, 3, 4, 5] = np.nan
    g.set_state(bad)
    with pytest.raises(hg.HgksError) as e:
        g.step(3, 0.5)
    assert e.value.status == hg.HGKS_ERR_NONFINITE
    assert np.array_equal(g.get_state(), bad, equal_nan=True)
    st1 = g.stats()
    assert st1["step"] == st0["step"] and st1["t"] == st0["t"]
    # the handle stays usable
    g.set_state(before)
    g.step(1, 0.5)
    assert g.stats()["step"] == st0["step"] + 1


def test_pinned_host_roundtrip(hg):
    import torch
    n = (12, 10, 8)
    g = hg.Solver(n, **TGV_KW)
    q = torch.from_numpy(smooth_state(n, 5)).pin_memory()
    g.set_state(q)
    out = torch.empty(q.shape, dtype=torch.float64).pin_memory()
    g.get_state(out)
    assert torch.equal(out, q)


def test_full_size_tgv_256(hg, oracle):
    """TGV 256^3 in the configuration the benchmark times: the GPU right-hand
    side at sampled cells (corners, edges, interior) equals the oracle's, and
    mass / energy are conserved over the steps."""
    n = (256, 256, 256)
    g = hg.Solver(n, **TGV_KW)
    g.init_tgv(0.1, 1.0, 1.0)
    s0 = g.stats()
    g.step(2, 0.5)
    s1 = g.stats()
    assert abs(s1["mass"] - s0["mass"]) <= 1e-13 * s0["mass"]
    assert abs(s1["energy"] - s0["energy"]) <= 1e-13 * s0["energy"]
    q = g.get_state()
    dt = s1["dt"]
    Lg, dLg = g.rhs(dt)
    c = oracle.RefSolver(n, **TGV_KW)
    c.set_state(q)
    rng = np.random.default_rng(256)
    N = 256
    pts = [(0, 0, 0), (255, 255, 255), (0, 255, 128), (255, 0, 1), (128, 128, 0)]
    pts += [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(19)]
    cells = [(k * N + j) * N + i for (i, j, k) in pts]
    Lc, dLc = c.rhs_cells(dt, cells)
    Lgs = Lg.reshape(5, -1)[:, cells].T
    dLgs = dLg.reshape(5, -1)[:, cells].T
    # L is a difference of face fluxes divided by a cell width: at 256^3 it
    # cancels four to five digits, so the errors are measured against the
    # flux-divergence scale (rounding acts on it): mass rho (|u| + c), momenta
    # |rho u| (|u| + c) + p, energy (rho E + p)(|u| + c), over h
    Qm = np.abs(q).reshape(5, -1).max(axis=1)
    rho, mom = q[0], q[1:4]
    u = np.abs(mom / rho).max()
    pr = (GAMMA - 1) * (q[4] - 0.5 * (mom ** 2).sum(axis=0) / rho)
    cmax = np.sqrt(GAMMA * pr / rho).max()
    h = 2 * np.pi / N
    S = np.empty(5)
    S[0] = Qm[0] * (u + cmax) / h
    S[1:4] = (Qm[1:4].max() * (u + cmax) + pr.max()) / h
    S[4] = (Qm[4] + pr.max()) * (u + cmax) / h
    assert (np.abs(Lgs - Lc) / S).max() < 1e-13
    assert (np.abs(dLgs - dLc) / (S / dt)).max() < 1e-11


def test_full_size_channel_128(hg, oracle):
    """The channel at its full 128^3 size (stretched walls, body force): the
    GPU right-hand side at sampled cells, the wall-adjacent rows included,
    equals the oracle's after two steps, measured against the flux-divergence
    scale of each cell's smallest width."""
    n = (128, 128, 128)
    kw = channel_kw()
    g = hg.Solver(n, **kw)
    g.init_channel(0.5, 0.1, 2800)
    g.step(2, 0.5)
    q = g.get_state()
    dt = g.stats()["dt"]
    Lg, dLg = g.rhs(dt)
    c = oracle.RefSolver(n, **kw)
    c.set_state(q)
    rng = np.random.default_rng(128)
    N = 128
    pts = [(0, 0, 0), (127, 127, 127), (5, 0, 64), (64, 1, 3), (17, 2, 99), (100, 126, 0), (33, 127, 50)]
    pts += [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(17)]
    cells = [(k * N + j) * N + i for (i, j, k) in pts]
    Lc, dLc = c.rhs_cells(dt, cells)
    Lgs = Lg.reshape(5, -1)[:, cells].T
    dLgs = dLg.reshape(5, -1)[:, cells].T
    # mesh: y(s) = -1 + (1 + tanh(b (s - 1)) / tanh b), s = 2 j / ny, b = 2
    s_ = 2.0 * np.arange(N + 1) / N
    yf = -1.0 + (1.0 + np.tanh(2.0 * (s_ - 1.0)) / np.tanh(2.0))
    hy = np.diff(yf)
    hmin = np.array([min(2 * np.pi / N, hy[j], np.pi / N) for (_, j, _) in pts])
    rho, mom = q[0], q[1:4]
    u = np.abs(mom / rho).max()
    pr = (GAMMA - 1) * (q[4] - 0.5 * (mom ** 2).sum(axis=0) / rho)
    cmax = np.sqrt(GAMMA * pr / rho).max()
    Qm = np.abs(q).reshape(5, -1).max(axis=1)
    S = np.empty((len(pts), 5))
    S[:, 0] = Qm[0] * (u + cmax) / hmin
    S[:, 1:4] = ((Qm[1:4].max() * (u + cmax) + pr.max()) / hmin)[:, None]
    S[:, 4] = (Qm[4] + pr.max()) * (u + cmax) / hmin
    assert (np.abs(Lgs - Lc) / S).max() < 1e-13
    assert (np.abs(dLgs - dLc) / (S / dt)).max() < 1e-11


def test_full_size_channel_128_mixed_vs_fp64(hg):
    """The channel configuration in both precisions: 40 steps at 128^3 from the
    same field; the mixed run stays within the FP32 error budget of the FP64
    run (state, wall shear, kinetic energy) and conserves mass to the FP64
    update's roundoff in the periodic directions."""
    n = (128, 128, 128)
    kw = channel_kw()
    runs = {}
    for name, prec in (("fp64", hg.FP64), ("mixed", hg.MIXED)):
        s = hg.Solver(n, precision=prec, **kw)
        s.init_channel(0.5, 0.1, 2800)
        s.step(40, 0.5)
        runs[name] = (s.get_state(), s.stats())
        s.close()
    (q64, s64), (qmx, smx) = runs["fp64"], runs["mixed"]
    scale = np.abs(q64).reshape(5, -1).max(axis=1)
    scale[1:4] = scale[1:4].max()
    err = (np.abs(qmx - q64).reshape(5, -1).max(axis=1) / scale).max()
    print("channel 128^3 mixed vs FP64 after 40 steps: state %.3e, wall shear %.3e, Ek %.3e" % (
        err, abs(smx["wall_shear"] - s64["wall_shear"]) / abs(s64["wall_shear"]),
        abs(smx["Ek"] - s64["Ek"]) / s64["Ek"]))
    assert smx["step"] == s64["step"] == 40
    # observed on GB300: state 8.8e-7, wall shear 1.2e-8, E_k 3.4e-10.  The
    # state bound is the FP32 unit roundoff (6e-8) times the growth of the
    # rounding of the small flux terms over the steps near the stretched
    # walls (h_min = 2.4e-3); the integrals average it out.
    assert err < 1e-5
    assert abs(smx["wall_shear"] - s64["wall_shear"]) < 1e-6 * abs(s64["wall_shear"])
    assert abs(smx["Ek"] - s64["Ek"]) < 5e-9 * s64["Ek"]
