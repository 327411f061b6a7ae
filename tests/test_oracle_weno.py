"""Pins of the oracle's reconstruction (fifth-order WENO, Sec. 2 last paragraph).

Checks against textbook values (Jiang-Shu linear weights and smoothness
indicators), exact rational/surd derivations done here with sympy, and
polynomial reproduction.
"""
import numpy as np
import pytest
import sympy as sp

G = np.sqrt(3.0) / 6.0  # 2-point Gauss-Legendre abscissae on a unit cell, +-sqrt(3)/6


def _avg_poly(coeffs, c):
    """cell average over [c-1/2, c+1/2] of sum_n coeffs[n] x^n (exact)."""
    return sum(a * ((c + 0.5) ** (n + 1) - (c - 0.5) ** (n + 1)) / (n + 1) for n, a in enumerate(coeffs))


def test_linear_weights_at_faces(oracle):
    # Jiang & Shu (1996): d = (1/10, 6/10, 3/10) at the right face, mirrored at the left
    np.testing.assert_allclose(oracle.weno_linear_weights(0.5), [0.1, 0.6, 0.3], rtol=1e-13)
    np.testing.assert_allclose(oracle.weno_linear_weights(-0.5), [0.3, 0.6, 0.1], rtol=1e-13)


def _sym_linear_weights(sigma):
    """exact linear weights at sigma from sympy polynomial fits to cell averages."""
    x = sp.symbols("x")
    X = sp.symbols("X0:5")  # cells -2..2

    def fit(cells, vals):
        n = len(cells)
        cs = sp.symbols("c0:%d" % n)
        P = sum(cs[k] * x ** k for k in range(n))
        eqs = [sp.integrate(P, (x, c - sp.Rational(1, 2), c + sp.Rational(1, 2))) - v for c, v in zip(cells, vals)]
        sol = sp.solve(eqs, cs)
        return P.subs(sol)

    quart = sp.expand(fit([-2, -1, 0, 1, 2], X).subs(x, sigma))
    cands = [sp.expand(fit(c, [X[i + 2] for i in c]).subs(x, sigma)) for c in ([-2, -1, 0], [-1, 0, 1], [0, 1, 2])]
    d = sp.symbols("d0:3")
    comb = sp.expand(sum(d[k] * cands[k] for k in range(3)) - quart)
    eqs = [sp.Eq(comb.coeff(Xi), 0) for Xi in X]
    sol = sp.solve(eqs, d, dict=True)
    assert len(sol) == 1  # the five equations are consistent
    return [sp.nsimplify(sp.simplify(sol[0][dk])) for dk in d]


def test_linear_weights_at_gauss_points_exact(oracle):
    s3 = sp.sqrt(3)
    exact = _sym_linear_weights(s3 / 6)
    # closed form (210 -+ sqrt3)/1080, 11/18, all positive
    assert sp.simplify(exact[0] - (210 - s3) / 1080) == 0
    assert sp.simplify(exact[1] - sp.Rational(11, 18)) == 0
    assert sp.simplify(exact[2] - (210 + s3) / 1080) == 0
    np.testing.assert_allclose(oracle.weno_linear_weights(G), [float(e) for e in exact], rtol=1e-13)
    np.testing.assert_allclose(oracle.weno_linear_weights(-G), [float(e) for e in exact[::-1]], rtol=1e-13)


def test_smoothness_indicators_jiang_shu(oracle):
    """beta_k equal the published Jiang-Shu closed forms."""
    rng = np.random.default_rng(0)
    for _ in range(5):
        X = rng.normal(size=5)
        a, b, c, d, e = X
        ref = [13 / 12 * (a - 2 * b + c) ** 2 + 0.25 * (a - 4 * b + 3 * c) ** 2,
               13 / 12 * (b - 2 * c + d) ** 2 + 0.25 * (b - d) ** 2,
               13 / 12 * (c - 2 * d + e) ** 2 + 0.25 * (3 * c - 4 * d + e) ** 2]
        _, beta = oracle.weno_candidates(X, 0.5)
        np.testing.assert_allclose(beta, ref, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("sigma", [0.5, -0.5, G, -G])
def test_weno_z_exact_for_quadratics(oracle, sigma):
    """every candidate reproduces a quadratic, so WENO-Z does at any weights."""
    coeffs = [0.3, -1.1, 0.7]
    X = [_avg_poly(coeffs, c) for c in range(-2, 3)]
    exact = sum(a * sigma ** n for n, a in enumerate(coeffs))
    assert oracle.weno_z(X, sigma) == pytest.approx(exact, rel=1e-13, abs=1e-14)


@pytest.mark.parametrize("sigma", [0.5, -0.5, G, -G, 0.0])
def test_quartic_value_and_derivative(oracle, sigma):
    coeffs = [0.2, 0.5, -0.3, 0.8, -0.6]
    X = np.array([_avg_poly(coeffs, c) for c in range(-2, 3)])
    Lc, Dc = oracle.quartic_coeffs(sigma)
    val = sum(a * sigma ** n for n, a in enumerate(coeffs))
    der = sum(n * a * sigma ** (n - 1) for n, a in enumerate(coeffs) if n > 0)
    assert Lc @ X == pytest.approx(val, rel=1e-13)
    assert Dc @ X == pytest.approx(der, rel=1e-12)
    # linear weights combine the candidates into the quartic value
    d = oracle.weno_linear_weights(sigma) if sigma != 0.0 else None
    if d is not None:
        p, _ = oracle.weno_candidates(X, sigma)
        assert d @ p == pytest.approx(val, rel=1e-13)


def test_weno_z_smooth_data_is_fifth_order(oracle):
    """on smooth data WENO-Z converges at fifth order to the point value."""
    errs = []
    for h in (0.2, 0.1, 0.05):
        X = [(np.cos(h * (c - 0.5)) - np.cos(h * (c + 0.5))) / h for c in range(-2, 3)]  # averages of sin(h x)/h... scaled
        exact = np.sin(h * 0.5)
        errs.append(abs(oracle.weno_z(X, 0.5) * 1.0 - exact))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 4.5)


def test_weno_z_avoids_discontinuous_stencil(oracle):
    """with a jump inside the right part of the stencil the left-biased value
    stays on the smooth side (essentially non-oscillatory)."""
    X = [1.0, 1.0, 1.0, 1.0, 10.0]
    v = oracle.weno_z(X, 0.5)
    assert abs(v - 1.0) < 1e-3
