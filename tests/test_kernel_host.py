"""CPU parity of the CUDA path's arithmetic with the oracle.

The flux path's arithmetic templates (hgks_device.cuh) are host-device code,
so tests/kernel_host.cu instantiates them on the host:
- the Gauss-point GKS flux, closed-form Jacobians and differentiated
  half-range moments, with no slope systems;
- WENO-Z at cell edges and Gauss points;
- the quartic value and slope weights.

They are compared here, case by case, with the oracle's independent
versions:
- the sparse-polynomial moment engine with Gaussian-elimination slopes;
- polynomial-fit WENO candidates and weights.

The inputs are thousands of seeded states and slopes, including strong
jumps, tau -> 0 and the power-law viscosity.  Only the device's libm
differs: host erfc/exp/sqrt/pow stand in for CUDA's.  This does not
replace the GPU parity tests (memory layout, tiling, staging); it pins the
arithmetic those kernels run, on every CPU run.
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GAMMA = 1.4
G = np.sqrt(3.0) / 6.0


@pytest.fixture(scope="module")
def kh(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("kh") / "libkernel_host.so")
    # host lambdas passed to the host-device pass bodies: diagnostics 20011/20014
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    "--expt-relaxed-constexpr", "-diag-suppress", "20011,20014", "-shared", "-Xcompiler",
                    "-fPIC,-ffp-contract=off",
                    "-I" + os.path.join(ROOT, "include"), "-o", out, os.path.join(ROOT, "tests", "kernel_host.cu")],
                   check=True)
    L = C.CDLL(out)
    dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
    L.kh_point_flux.argtypes = [C.c_int, dp, dp, dp, dp, dp, C.c_double, C.c_double, C.c_int, C.c_double,
                                C.c_double, C.c_double, C.c_double, dp, dp]
    L.kh_reconstruct.argtypes = [C.c_int, dp, dp, dp]
    L.kh_side_time_rate.argtypes = [C.c_int, dp, dp, C.c_double, dp]
    fp = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    L.kh_point_flux_mixed.argtypes = [C.c_int] + [fp] * 7 + [C.c_double, C.c_double, C.c_int, C.c_double,
                                                              C.c_double, C.c_double, C.c_double, dp, dp, C.c_int]
    L.kh_compat_mixed.argtypes = [C.c_int, fp, fp, fp, fp, C.c_double, dp]
    from oracle import ref
    L.kh_face_flux.argtypes = [dp, C.POINTER(ref.Grid), C.c_double, C.c_double, C.c_int, C.c_double, C.c_double,
                               C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, dp, dp]
    return L


def _cons(rho, u, v, w, p):
    return np.stack([rho, rho * u, rho * v, rho * w, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v + w * w)], -1)


def _states(rng, n, jump):
    rho = rng.uniform(0.5, 2.0, n)
    vel = rng.uniform(-1.0, 1.0, (n, 3))
    p = rng.uniform(0.5, 2.0, n)
    Ql = _cons(rho, *vel.T, p)
    f = np.exp(rng.uniform(-jump, jump, (n, 3)))
    Qr = _cons(rho * f[:, 0], *(vel + jump * rng.uniform(-1, 1, (n, 3))).T, p * f[:, 1])
    return Ql, Qr


VISC = {"const": (0, 1e-3, 1.0, 0.0), "power": (1, 2e-3, 1.3, 0.7), "inviscid": (0, 0.0, 1.0, 0.0),
        "kinetic": (0, 0.05, 1.0, 0.0)}


@pytest.mark.parametrize("jump", [0.0, 0.05, 0.5, 1.6])
@pytest.mark.parametrize("visc", sorted(VISC))
def test_point_flux_matches_oracle(oracle, kh, jump, visc):
    """F^n and dF^n/dt of one Gauss point: the CUDA path's closed forms equal
    the oracle's moment sums to 1e-13 of the flux scale (the worst case seen
    is 1e-14).  The cases run from smooth (jump 0) to strong jumps (density
    and pressure ratios up to 5, velocity jumps of 1.6).  The viscosity is inviscid (tau = 0), near the
    Navier-Stokes limit, power-law, or kinetic (tau comparable to dt)."""
    rng = np.random.default_rng([int(round(jump * 100)), sorted(VISC).index(visc)])
    n = 200
    Ql, Qr = _states(rng, n, jump)
    dl, dr, d0 = (0.5 * rng.standard_normal((n, 15)) for _ in range(3))
    dt, Pr = 0.01, 0.72
    kind, mu, Tref, om = VISC[visc]
    Fn, dFn = np.empty((n, 5)), np.empty((n, 5))
    kh.kh_point_flux(n, Ql, Qr, dl, dr, d0, GAMMA, Pr, kind, mu, Tref, om, dt, Fn, dFn)
    for i in range(n):
        _, _, F_ref, dF_ref = oracle.point_flux(Ql[i], Qr[i], dl[i], dr[i], d0[i], GAMMA, Pr, (kind, mu, Tref, om), dt)
        scale = max(np.abs(F_ref).max(), 1.0)
        np.testing.assert_allclose(Fn[i], F_ref, rtol=0, atol=1e-13 * scale)
        np.testing.assert_allclose(dFn[i], dF_ref, rtol=0, atol=1e-13 * max(np.abs(dF_ref).max(), scale / dt))


def _euler_flux(Q, d):
    """Euler flux along direction d of conservative states Q [..., 5]; plain
    arithmetic only, so it also takes complex arguments."""
    rho, m, E = Q[..., 0], Q[..., 1:4], Q[..., 4]
    u = m / rho[..., None]
    p = (GAMMA - 1.0) * (E - 0.5 * (m * u).sum(-1))
    F = np.empty_like(Q)
    F[..., 0] = m[..., d]
    F[..., 1:4] = m[..., d, None] * u
    F[..., 1 + d] += p
    F[..., 4] = u[..., d] * (E + p)
    return F


def _primitives(Q):
    rho = Q[..., 0]
    u = Q[..., 1:4] / rho[..., None]
    p = (GAMMA - 1.0) * (Q[..., 4] - 0.5 * rho * (u * u).sum(-1))
    return np.concatenate([rho[..., None], u, (p / rho)[..., None]], -1)


def test_side_time_slope_is_the_euler_time_derivative(kh):
    """A side's time slope enters the flux through the time change of its
    primitives (rho, U, V, W, T), which the kernels sum from the Euler
    equations in primitive form.  Reference: the conservative form
    d_t Q = -sum_d dF_d/dQ . d_d Q, differentiated by the complex step (exact
    to rounding) and taken to primitives the same way."""
    rng = np.random.default_rng(2207)
    n = 500
    Q, _ = _states(rng, n, 0.0)
    dq = rng.normal(size=(n, 3, 5)) * np.abs(Q)[:, None, :]
    out = np.zeros((n, 5))
    kh.kh_side_time_rate(n, Q, np.ascontiguousarray(dq.reshape(n, 15)), GAMMA, out)
    h = 1e-30
    dtq = -sum(_euler_flux(Q + 1j * h * dq[:, d], d).imag / h for d in range(3))
    ref = _primitives(Q + 1j * h * dtq).imag / h
    # per-case scale: the size of the terms that the Euler equations sum
    scale = np.abs(dq).sum(axis=(1, 2))[:, None] * (1.0 + np.abs(Q).max(axis=1))[:, None]
    assert np.max(np.abs(out - ref) / scale) < 1e-14
    assert np.max(np.abs(ref) / scale) > 1e-3  # the comparison is not of vanishing quantities


@pytest.mark.parametrize("kind", ["smooth", "rough", "step"])
def test_reconstruction_matches_oracle(oracle, kh, kind):
    """WENO-Z at -1/2, +1/2, -sqrt3/6 and +sqrt3/6, and the quartic's value
    and slope at -+sqrt3/6: the CUDA path's closed forms (one reciprocal per
    point pair) equal the oracle's fitted polynomials and weights."""
    rng = np.random.default_rng({"smooth": 1, "rough": 2, "step": 3}[kind])
    n = 2000
    if kind == "smooth":
        x0, hh = rng.uniform(0, 2 * np.pi, n), rng.uniform(0.01, 0.5, n)
        X = np.stack([np.sin(x0 + j * hh) for j in range(-2, 3)], -1) + rng.uniform(-2, 2, (n, 1))
    elif kind == "rough":
        X = rng.standard_normal((n, 5)) * np.exp2(rng.integers(-10, 10, (n, 1)))
    else:
        X = np.where(np.arange(5)[None, :] >= rng.integers(1, 5, (n, 1)), 1.0, 0.1) * rng.uniform(0.5, 2, (n, 1))
    X = np.ascontiguousarray(X)
    weno, quart = np.empty((n, 4)), np.empty((n, 4))
    kh.kh_reconstruct(n, X, weno, quart)
    Lm, Dm = oracle.quartic_coeffs(-G)
    Lp, Dp = oracle.quartic_coeffs(G)
    for i in range(n):
        scale = max(np.abs(X[i]).max(), 1e-300)
        ref = [oracle.weno_z(X[i], s) for s in (-0.5, 0.5, -G, G)]
        np.testing.assert_allclose(weno[i], ref, rtol=0, atol=2e-14 * scale)
        np.testing.assert_allclose(quart[i], [Lm @ X[i], Lp @ X[i], Dm @ X[i], Dp @ X[i]], rtol=0, atol=2e-14 * scale)


def _split(x):
    hi = x.astype(np.float32)
    return hi, (x - hi.astype(np.float64)).astype(np.float32)


@pytest.mark.parametrize("t64", [0, 1], ids=["mixed", "mixed_t64"])
@pytest.mark.parametrize("jump", [0.0, 1e-4, 1e-3, 0.5, 1.6])
@pytest.mark.parametrize("visc", sorted(VISC))
def test_mixed_point_flux_error(oracle, kh, jump, visc, t64):
    """The mixed-precision Gauss-point flux (R-MX) against the FP64 oracle on
    the same inputs: float-float states and FP32 slopes, passed to the oracle
    as the FP64 values they represent.

    Inviscid with a jump below the compatibility switch (1e-3), the flux is
    the float-float Euler flux of the float-float Q0: within 1e-10 (a
    float-only B1 would be off by ~1e-7).  Otherwise F^n is within 1e-5 of the
    flux scale (FP32 small terms, the FP32 direct compatibility sum at larger
    jumps) and dF^n/dt within 2e-3 of its scale (FP32 throughout, with the
    cancellation of the time slope of Q0).  The same bounds hold for the
    HGKS_MIXED_T64 variant (FP64 temperature, collision time and time
    coefficients)."""
    rng = np.random.default_rng([int(round(jump * 1e4)), sorted(VISC).index(visc), 7])
    n = 150
    Ql, Qr = _states(rng, n, jump)
    if jump == 0.0:
        Qr = Ql.copy()
    dl, dr, d0 = (np.ascontiguousarray((0.5 * rng.standard_normal((n, 15))).astype(np.float32)) for _ in range(3))
    (lh, ll), (rh, rl) = _split(Ql), _split(Qr)
    kind, mu, Tref, om = VISC[visc]
    dt = 0.01
    Fn, dFn = np.empty((n, 5)), np.empty((n, 5))
    kh.kh_point_flux_mixed(n, lh, ll, rh, rl, dl, dr, d0, GAMMA, 0.72, kind, mu, Tref, om, dt, Fn, dFn, t64)
    ff_only = visc == "inviscid" and jump <= 1e-4
    for i in range(n):
        ql, qr = lh[i] + ll[i].astype(np.float64), rh[i] + rl[i].astype(np.float64)
        _, _, F, dF = oracle.point_flux(ql, qr, dl[i].astype(np.float64), dr[i].astype(np.float64),
                                        d0[i].astype(np.float64), GAMMA, 0.72, (kind, mu, Tref, om), dt)
        scale = np.abs(F).max()
        np.testing.assert_allclose(Fn[i], F, rtol=0, atol=(1e-10 if ff_only else 1e-5) * scale)
        np.testing.assert_allclose(dFn[i], dF, rtol=0, atol=2e-3 * np.abs(dF).max())


FACE_CASES = {
    # name: solver keyword arguments, grid, state
    "periodic_noncubic": (dict(lengths=(1.0, 2.0, 1.5), visc=(1, 2e-3, 1.3, 0.7), Pr=0.72), (7, 6, 5), "smooth"),
    "periodic_rough": (dict(visc=(0, 1e-3, 1.0, 0.0), Pr=0.72), (6, 6, 6), "rough"),
    "channel_walls": (dict(lengths=(2 * np.pi, 2.0, np.pi), origin=(0.0, -1.0, 0.0), y_stretch_b=2.0,
                           visc=(1, 1.0 / 2800, 2.857, 0.7), Pr=0.7, bc_lo=(0, 1, 0), bc_hi=(0, 1, 0), T_wall=2.857),
                      (5, 9, 4), "channel"),
}


@pytest.mark.parametrize("case", sorted(FACE_CASES))
def test_face_flux_through_the_pass_bodies(oracle, kh, case):
    """One interface's F^n and dF^n/dt through the CUDA path's three pass
    bodies (normal, first tangential, flux), with the library's y-mesh tables
    and face geometry, equal the oracle's face flux on the same ghost-filled
    state.  Every face of every direction is checked, on a non-cubic periodic
    grid, a rough state and the stretched wall-bounded channel (faces next to
    the walls included)."""
    from tests.inputs import rough_state, smooth_state
    kw, n, kind = FACE_CASES[case]
    s = oracle.RefSolver(n, **kw)
    if kind == "channel":
        s.init_channel(0.5, 0.1, 5)
    else:
        s.set_state((smooth_state if kind == "smooth" else rough_state)(n, 11))
    seen = []
    s.set_hooks(halo=lambda q: seen.append(q.copy()))
    g = oracle.Grid(n[0], n[1], n[2], *kw.get("lengths", (2 * np.pi,) * 3), *kw.get("origin", (0.0, 0.0, 0.0)),
                    kw.get("y_stretch_b", 0.0))
    kind_v, mu, Tref, om = kw["visc"]
    dt = 2e-3
    tdirs = {0: (1, 2), 1: (0, 2), 2: (0, 1)}
    for d in range(3):
        e1, e2 = tdirs[d]
        for f in range(n[d] + 1):
            for a in range(n[e1]):
                for b in range(n[e2]):
                    F_ref, dF_ref = s.face_flux(dt, d, f, a, b)
                    q = np.ascontiguousarray(seen[-1])
                    F, dF = np.empty(5), np.empty(5)
                    kh.kh_face_flux(q.ravel(), C.byref(g), GAMMA, kw["Pr"], kind_v, mu, Tref, om, d, f, a, b, dt, F, dF)
                    scale = np.abs(F_ref).max()
                    np.testing.assert_allclose(F, F_ref, rtol=0, atol=1e-13 * scale)
                    np.testing.assert_allclose(dF, dF_ref, rtol=0, atol=1e-11 * max(np.abs(dF_ref).max(), scale / dt))


def test_mixed_compatibility_error_by_jump(oracle, kh):
    """R-MX's equilibrium state Q0 against the FP64 compatibility of the
    oracle, by the relative jump between the l/r states.  Below the 1e-3
    switch the mixed path forms Qm + C in float-float with the correction C
    in FP32, so the error is the FP32 rounding of C, about 1e-7 x jump.  The
    trapezoidal truncation, O(jump^3), lies below that.  Above the switch
    the direct FP32 sum Phi+(Ql) + Phi-(Qr) keeps FP32 accuracy."""
    K = (5 - 3 * GAMMA) / (GAMMA - 1)
    rng = np.random.default_rng(21)
    n = 60
    worst = {}
    for jump in (1e-6, 1e-5, 1e-4, 4e-4, 3e-3, 3e-2):
        Ql = _cons(rng.uniform(0.8, 1.2, n), *rng.uniform(-0.5, 0.5, (3, n)), rng.uniform(0.8, 1.2, n))
        # a jump of this relative size in density, velocity and pressure
        Qr = _cons(Ql[:, 0] * (1 + jump * rng.uniform(-1, 1, n)),
                   *(Ql[:, 1:4] / Ql[:, :1] + jump * rng.uniform(-1, 1, (n, 3))).T,
                   (GAMMA - 1) * (Ql[:, 4] - 0.5 * (Ql[:, 1:4] ** 2).sum(1) / Ql[:, 0]) * (1 + jump * rng.uniform(-1, 1, n)))
        (lh, ll), (rh, rl) = _split(Ql), _split(Qr)
        Q0 = np.empty((n, 5))
        kh.kh_compat_mixed(n, lh, ll, rh, rl, GAMMA, Q0)
        err = 0.0
        for i in range(n):
            ref = oracle.compat(lh[i] + ll[i].astype(np.float64), rh[i] + rl[i].astype(np.float64), K)
            err = max(err, np.abs(Q0[i] - ref).max() / np.abs(ref).max())
        worst[jump] = err
    for jump in (1e-6, 1e-5, 1e-4, 4e-4):  # measured: 0.9e-7 x jump
        assert worst[jump] < 2e-7 * jump + 1e-13, (jump, worst[jump])
    assert worst[3e-3] < 1e-6 and worst[3e-2] < 1e-6  # direct FP32 sum, measured 1.4e-7


@pytest.mark.parametrize("x", [100.0, 1.0, 0.01, 1e-3])
def test_mixed_time_coefficients_fp32_against_fp64(oracle, kh, x):
    """The time-integration coefficients at dt / tau = x.  Written in closed
    form, the equilibrium coefficients q1 ~ -dt^3 / (6 tau) and
    q2 ~ dt^3 / (6 tau) cancel to O(x^3) when x << 1 and lose ~2 log10(1/x)
    digits in FP32 (measured before the change: F^n 1.4e-4, dF^n/dt 2e-2 of
    their scales at x = 0.01, against 2.6e-6 and 1.2e-4 with FP64
    coefficients).  HGKS_MIXED sums their Taylor series for x < 1, so its FP32
    coefficients cost at most a factor 2.5 in accuracy against the FP64
    coefficients of HGKS_MIXED_T64 at every x; for x >= 0.01 both stay within
    the mixed-path bounds against the FP64 oracle.  (At x = 1e-3 the other
    FP32 terms put dF^n/dt of both variants near 3e-3: the near-free-molecular
    limit is outside the workloads, whose dt / tau lies between 5 and 130.)"""
    rng = np.random.default_rng([11, int(-np.log10(x) + 10)])
    n = 120
    Ql, Qr = _states(rng, n, 0.05)
    dl, dr, d0 = (np.ascontiguousarray((0.5 * rng.standard_normal((n, 15))).astype(np.float32)) for _ in range(3))
    (lh, ll), (rh, rl) = _split(Ql), _split(Qr)
    dt = 0.01
    # constant viscosity mu = tau p with p ~ 1: tau ~ dt / x
    kind, mu, Tref, om = 0, dt / x, 1.0, 0.0
    out = {}
    for t64 in (0, 1):
        Fn, dFn = np.empty((n, 5)), np.empty((n, 5))
        kh.kh_point_flux_mixed(n, lh, ll, rh, rl, dl, dr, d0, GAMMA, 0.72, kind, mu, Tref, om, dt, Fn, dFn, t64)
        out[t64] = (Fn, dFn)
    worst = {0: [0.0, 0.0], 1: [0.0, 0.0]}
    for i in range(n):
        ql, qr = lh[i] + ll[i].astype(np.float64), rh[i] + rl[i].astype(np.float64)
        _, _, F, dF = oracle.point_flux(ql, qr, dl[i].astype(np.float64), dr[i].astype(np.float64),
                                        d0[i].astype(np.float64), GAMMA, 0.72, (kind, mu, Tref, om), dt)
        for t64 in (0, 1):
            worst[t64][0] = max(worst[t64][0], np.abs(out[t64][0][i] - F).max() / np.abs(F).max())
            worst[t64][1] = max(worst[t64][1], np.abs(out[t64][1][i] - dF).max() / np.abs(dF).max())
    print("dt/tau = %g: FP32 coefficients F %.2e dF %.2e; FP64 coefficients F %.2e dF %.2e"
          % (x, worst[0][0], worst[0][1], worst[1][0], worst[1][1]))
    for j in (0, 1):
        assert worst[0][j] <= 2.5 * worst[1][j] + 1e-6
    if x >= 0.01:
        for t64 in (0, 1):
            assert worst[t64][0] < 1e-5 and worst[t64][1] < 2e-3
