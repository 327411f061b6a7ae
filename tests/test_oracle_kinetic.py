"""Pins of the oracle's kinetic building blocks (Sec. 2 of arXiv 2207.01173).

Each check compares the oracle with something other than itself: numerical
quadrature, closed forms that follow from the BGK model, or the
Navier-Stokes limit of the gas-kinetic flux.
"""
import numpy as np
import pytest
from scipy.integrate import quad

from tests.quadrature import VelocityGrid, brute_point_flux

GAMMA = 1.4
K = (5 - 3 * GAMMA) / (GAMMA - 1)  # internal degrees of freedom, Sec. 2 (N = 2 at gamma = 1.4)


def _gauss_1d(U, lam):
    return lambda u: np.sqrt(lam / np.pi) * np.exp(-lam * (u - U) ** 2)


@pytest.mark.parametrize("U,lam", [(0.0, 0.5), (0.3, 0.7), (-1.2, 2.0), (2.5, 0.05)])
def test_velocity_moments_against_quadrature(oracle, U, lam):
    """<u^n> over the full line and the two half lines (Sec. 2 compatibility
    integrals) equal direct numerical integration of u^n g."""
    g = _gauss_1d(U, lam)
    for rng, (a, b) in ((0, (-np.inf, np.inf)), (1, (0, np.inf)), (2, (-np.inf, 0))):
        m = oracle.moments_1d(U, lam, rng, 8)
        for n in range(8):
            ref = quad(lambda u: u ** n * g(u), a, b, epsabs=1e-14, epsrel=1e-13, limit=400)[0]
            assert m[n] == pytest.approx(ref, rel=1e-10, abs=1e-12 * (1 + abs(U) + 1 / np.sqrt(lam)) ** n)


def test_half_moments_sum_to_full(oracle):
    for U, lam in [(0.1, 0.5), (-0.7, 3.0), (1.9, 0.2)]:
        full = oracle.moments_1d(U, lam, 0, 8)
        s = oracle.moments_1d(U, lam, 1, 8) + oracle.moments_1d(U, lam, 2, 8)
        np.testing.assert_allclose(s, full, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("lam", [0.3, 1.0, 4.0])
def test_internal_moments_against_quadrature(oracle, lam):
    """<xi^2>, <xi^4> for K = 2 internal degrees of freedom (radial quadrature)."""
    m = oracle.moments_xi(lam, 2.0)
    for d in range(3):
        ref = quad(lambda r: (r * r) ** d * 2 * np.pi * r * (lam / np.pi) * np.exp(-lam * r * r), 0, np.inf,
                   epsabs=0, epsrel=1e-13)[0]
        assert m[d] == pytest.approx(ref, rel=1e-11)


def test_primitive_lambda(oracle):
    # rho E = p/(gamma-1) + rho |U|^2 / 2 and lambda = rho / (2 p)
    rho, U, V, W, p = 1.3, 0.4, -0.2, 0.1, 2.1
    Q = [rho, rho * U, rho * V, rho * W, p / (GAMMA - 1) + 0.5 * rho * (U * U + V * V + W * W)]
    Wp = oracle.prim(Q, K)
    np.testing.assert_allclose(Wp, [rho, U, V, W, rho / (2 * p)], rtol=1e-14)


def test_micro_slope_against_quadrature(oracle):
    """<a psi> = dQ: the oracle's solution reproduces dQ under brute-force
    velocity quadrature (Sec. 2 slope equations)."""
    G = VelocityGrid()
    Wp = np.array([1.2, 0.3, -0.1, 0.2, 0.6])
    dQ = np.array([0.3, -0.2, 0.5, 0.1, 1.7])
    a = oracle.micro_slope(Wp, K, dQ)
    g = G.maxwellian(Wp)
    field = a[0] + a[1] * G.U + a[2] * G.V + a[3] * G.W + a[4] * 0.5 * (G.U ** 2 + G.V ** 2 + G.W ** 2 + G.XI2)
    got = np.array([G.integrate(p * field * g) for p in G.psi()])
    np.testing.assert_allclose(got, dQ, rtol=1e-9, atol=1e-10)
    # and the exported left-hand side agrees
    np.testing.assert_allclose(oracle.slope_moments(Wp, K, a), dQ, rtol=1e-12, atol=1e-12)


def test_compat_equal_states(oracle):
    """Q0 = Q when the left and right states coincide (compatibility)."""
    Q = np.array([1.1, 0.3, 0.2, -0.4, 4.0])
    np.testing.assert_allclose(oracle.compat(Q, Q, K), Q, rtol=1e-14)


def test_compat_against_quadrature(oracle):
    G = VelocityGrid()
    Ql = np.array([1.0, 0.4, 0.1, 0.0, 3.0])
    Qr = np.array([0.8, -0.2, 0.0, 0.3, 2.2])
    from tests.quadrature import prim
    gl, gr = G.maxwellian(prim(Ql, GAMMA)), G.maxwellian(prim(Qr, GAMMA))
    ref = np.array([G.integrate(p * (gl * G.H + gr * (1 - G.H))) for p in G.psi()])
    np.testing.assert_allclose(oracle.compat(Ql, Qr, K), ref, rtol=1e-10)


@pytest.mark.parametrize("tau,delta", [(1e-3, 1e-2), (0.05, 0.01), (1.0, 0.3), (0.0, 0.02)])
def test_time_coefficients_against_quadrature(oracle, tau, delta):
    """Closed-form time integrals of the factors in Eq. (flux) over [0, delta]."""
    from tests.quadrature import time_factors
    np.testing.assert_allclose(oracle.time_coeffs(tau, delta), time_factors(tau, delta), rtol=1e-11, atol=1e-18)


def test_time_fit_recovers_linear_flux(oracle):
    """Eq. (expansion-1): for F(t) = F + F' t the two integrals give back F, F'."""
    rng = np.random.default_rng(3)
    F, dF = rng.normal(size=5), rng.normal(size=5)
    dt = 0.013
    If = F * dt + 0.5 * dF * dt * dt
    Ih = 0.5 * F * dt + 0.125 * dF * dt * dt
    Fn, dFn = oracle.time_fit(If, Ih, dt)
    np.testing.assert_allclose(Fn, F, rtol=1e-12)
    np.testing.assert_allclose(dFn, dF, rtol=1e-9)


def _cons(rho, U, V, W, p):
    return np.array([rho, rho * U, rho * V, rho * W, p / (GAMMA - 1) + 0.5 * rho * (U * U + V * V + W * W)])


@pytest.mark.parametrize("mu", [0.0, 1e-3])
def test_uniform_state_gives_euler_flux(oracle, mu):
    """A uniform state with zero slopes: the time-integrated flux is delta times
    the Euler flux (rho U, rho U^2 + p, rho U V, rho U W, (rho E + p) U)."""
    rho, U, V, W, p = 1.2, 0.35, -0.2, 0.1, 1.7
    Q = _cons(rho, U, V, W, p)
    z = np.zeros(15)
    dt = 0.01
    If, Ih, Fn, dFn = oracle.point_flux(Q, Q, z, z, z, GAMMA, 0.72, (0, mu, 1.0, 0.0), dt)
    euler = np.array([rho * U, rho * U * U + p, rho * U * V, rho * U * W, (Q[4] + p) * U])
    np.testing.assert_allclose(If, euler * dt, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Ih, euler * dt / 2, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Fn, euler, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(dFn, 0.0, atol=1e-9)


@pytest.mark.parametrize("Pr", [1.0, 0.72])
def test_navier_stokes_limit(oracle, Pr):
    """Chapman-Enskog limit of the BGK flux (Sec. 2, tau = mu/p): a normal
    gradient of tangential velocity gives the shear stress -mu du_t/dn; a
    temperature gradient at constant pressure gives the Fourier heat flux
    -mu c_p / Pr dT/dn once the Prandtl correction is applied."""
    mu, s = 1e-3, 0.5
    Q = _cons(1.0, 0.0, 0.0, 0.0, 1.0)
    z = np.zeros(15)
    d = z.copy()
    d[2] = s  # d(rho u_t1)/dn
    _, _, Fn, _ = oracle.point_flux(Q, Q, d, d, d, GAMMA, Pr, (0, mu, 1.0, 0.0), 1e-2)
    assert Fn[2] == pytest.approx(-mu * s, rel=1e-9)
    assert Fn[1] == pytest.approx(1.0, rel=1e-12)
    d = z.copy()
    d[0] = -s  # T = p/rho with p fixed: dT/dn = s at rho = T = 1 needs drho/dn = -s, d(rho E)/dn = 0
    _, _, Fn, _ = oracle.point_flux(Q, Q, d, d, d, GAMMA, Pr, (0, mu, 1.0, 0.0), 1e-2)
    cp = GAMMA / (GAMMA - 1)
    assert Fn[4] == pytest.approx(-mu * cp / Pr * s, rel=1e-9)


@pytest.mark.parametrize("T", [0.5, 2.0])
def test_power_law_viscosity_in_shear_stress(oracle, T):
    """The power law mu = mu_ref (T / T_ref)^omega (Sec. 4.1) enters the
    collision time: at rest, rho = 1 and temperature T, a normal gradient of
    tangential momentum gives the shear stress -mu_ref T^omega du_t/dn."""
    mu_ref, omega, s = 1e-3, 0.7, 0.5
    Q = _cons(1.0, 0.0, 0.0, 0.0, T)
    d = np.zeros(15)
    d[2] = s
    _, _, Fn, _ = oracle.point_flux(Q, Q, d, d, d, GAMMA, 0.72, (1, mu_ref, 1.0, omega), 1e-2)
    assert Fn[2] == pytest.approx(-mu_ref * T ** omega * s, rel=1e-9)


@pytest.mark.slow
def test_point_flux_against_brute_force(oracle):
    """Full interface flux with different left/right states and all slopes
    nonzero equals direct quadrature of the time-integrated distribution of
    Eq. (flux), including the Prandtl correction."""
    rng = np.random.default_rng(11)
    Ql = _cons(1.05, 0.3, 0.1, -0.05, 1.2)
    Qr = _cons(0.95, 0.2, -0.1, 0.08, 1.05)
    dQl, dQr, dQ0 = (0.3 * rng.normal(size=15) for _ in range(3))
    mu, dt, Pr = 0.02, 0.05, 0.72
    If, Ih, Fn, dFn = oracle.point_flux(Ql, Qr, dQl, dQr, dQ0, GAMMA, Pr, (0, mu, 1.0, 0.0), dt)
    Bf, Bh, tau = brute_point_flux(Ql, Qr, dQl, dQr, dQ0, GAMMA, Pr, mu, dt)
    assert tau > 0.1 * dt  # the non-equilibrium terms are not negligible here
    scale = np.abs(Bf).max()
    np.testing.assert_allclose(If, Bf, rtol=0, atol=1e-9 * scale)
    np.testing.assert_allclose(Ih, Bh, rtol=0, atol=1e-9 * scale)
