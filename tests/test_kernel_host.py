"""CPU parity of the CUDA path's FP64 arithmetic with the oracle.

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
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    "--expt-relaxed-constexpr", "-shared", "-Xcompiler", "-fPIC,-ffp-contract=off",
                    "-I" + os.path.join(ROOT, "include"), "-o", out, os.path.join(ROOT, "tests", "kernel_host.cu")],
                   check=True)
    L = C.CDLL(out)
    dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
    L.kh_point_flux.argtypes = [C.c_int, dp, dp, dp, dp, dp, C.c_double, C.c_double, C.c_int, C.c_double,
                                C.c_double, C.c_double, C.c_double, dp, dp]
    L.kh_reconstruct.argtypes = [C.c_int, dp, dp, dp]
    fp = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    L.kh_point_flux_mixed.argtypes = [C.c_int] + [fp] * 7 + [C.c_double, C.c_double, C.c_int, C.c_double,
                                                              C.c_double, C.c_double, C.c_double, dp, dp]
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


@pytest.mark.parametrize("jump", [0.0, 1e-4, 1e-3, 0.5, 1.6])
@pytest.mark.parametrize("visc", sorted(VISC))
def test_mixed_point_flux_error(oracle, kh, jump, visc):
    """The mixed-precision Gauss-point flux (R-MX) against the FP64 oracle on
    the same inputs: float-float states and FP32 slopes, passed to the oracle
    as the FP64 values they represent.

    Inviscid with a jump below the compatibility switch (1e-3), the flux is
    the float-float Euler flux of the float-float Q0: within 1e-10 (a
    float-only B1 would be off by ~1e-7).  Otherwise F^n is within 1e-5 of the
    flux scale (FP32 small terms, the FP32 direct compatibility sum at larger
    jumps) and dF^n/dt within 2e-3 of its scale (FP32 throughout, with the
    cancellation of the time slope of Q0)."""
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
    kh.kh_point_flux_mixed(n, lh, ll, rh, rl, dl, dr, d0, GAMMA, 0.72, kind, mu, Tref, om, dt, Fn, dFn)
    ff_only = visc == "inviscid" and jump <= 1e-4
    for i in range(n):
        ql, qr = lh[i] + ll[i].astype(np.float64), rh[i] + rl[i].astype(np.float64)
        _, _, F, dF = oracle.point_flux(ql, qr, dl[i].astype(np.float64), dr[i].astype(np.float64),
                                        d0[i].astype(np.float64), GAMMA, 0.72, (kind, mu, Tref, om), dt)
        scale = np.abs(F).max()
        np.testing.assert_allclose(Fn[i], F, rtol=0, atol=(1e-10 if ff_only else 1e-5) * scale)
        np.testing.assert_allclose(dFn[i], dF, rtol=0, atol=2e-3 * np.abs(dF).max())
