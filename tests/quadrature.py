"""Brute-force velocity-space quadrature for pinning the oracle.

Independent of the oracle's moment engine: every integral over particle
velocity (u, v, w) and internal variables xi (K = 2, radial) is done with
Gauss-Legendre rules on a truncated box, split at u = 0 for half-range
integrals.  Used only by tests.
"""
import numpy as np


class VelocityGrid:
    def __init__(self, center=(0.0, 0.0, 0.0), X=8.0, nu=40, nv=40, nr=30, K=2.0):
        assert K == 2.0, "radial xi quadrature assumes two internal degrees of freedom"
        xg, wg = np.polynomial.legendre.leggauss(nu)
        # u in [-X, 0] and [0, X] (absolute, so the split at u = 0 is exact)
        un = -X * (xg + 1.0) / 2.0
        up = X * (xg + 1.0) / 2.0
        self.u = np.concatenate([un, up])
        self.wu = np.concatenate([wg * X / 2.0, wg * X / 2.0])
        self.pos = np.concatenate([np.zeros(nu, bool), np.ones(nu, bool)])
        xv, wv = np.polynomial.legendre.leggauss(nv)
        self.v = center[1] + X * xv
        self.wv = wv * X
        self.w = center[2] + X * xv
        self.ww = wv * X
        xr, wr = np.polynomial.legendre.leggauss(nr)
        R = X
        self.r = R * (xr + 1.0) / 2.0
        self.wr = wr * R / 2.0 * 2.0 * np.pi * self.r  # d^2 xi = 2 pi r dr
        U, V, W, Rr = np.meshgrid(self.u, self.v, self.w, self.r, indexing="ij")
        self.U, self.V, self.W, self.XI2 = U, V, W, Rr ** 2
        self.weight = (self.wu[:, None, None, None] * self.wv[None, :, None, None]
                       * self.ww[None, None, :, None] * self.wr[None, None, None, :])
        self.H = self.pos[:, None, None, None].astype(float) * np.ones_like(U)
        self.K = K

    def psi(self):
        return [np.ones_like(self.U), self.U, self.V, self.W,
                0.5 * (self.U ** 2 + self.V ** 2 + self.W ** 2 + self.XI2)]

    def maxwellian(self, Wp):
        rho, U, V, W, lam = Wp
        return rho * (lam / np.pi) ** ((self.K + 3) / 2) * np.exp(
            -lam * ((self.U - U) ** 2 + (self.V - V) ** 2 + (self.W - W) ** 2 + self.XI2))

    def integrate(self, f, mask=None):
        if mask is not None:
            f = f * mask
        return float(np.sum(f * self.weight))


def prim(Q, gamma):
    rho = Q[0]
    U, V, W = Q[1] / rho, Q[2] / rho, Q[3] / rho
    p = (gamma - 1.0) * (Q[4] - 0.5 * rho * (U * U + V * V + W * W))
    return np.array([rho, U, V, W, rho / (2.0 * p)])


def moment_matrix(G, g, rho):
    ps = G.psi()
    return np.array([[G.integrate(ps[i] * ps[j] * g) / rho for j in range(5)] for i in range(5)])


def slope_field(G, a):
    return a[0] + a[1] * G.U + a[2] * G.V + a[3] * G.W + a[4] * 0.5 * (G.U ** 2 + G.V ** 2 + G.W ** 2 + G.XI2)


def time_factors(tau, delta):
    """Time integrals of the five time factors of the GKS distribution over [0, delta]."""
    from scipy.integrate import quad
    if tau == 0.0:
        return np.array([delta, 0.0, 0.5 * delta * delta, 0.0, 0.0])
    f = [lambda t: 1.0 - np.exp(-t / tau),
         lambda t: (t + tau) * np.exp(-t / tau) - tau,
         lambda t: t - tau + tau * np.exp(-t / tau),
         lambda t: np.exp(-t / tau),
         lambda t: (tau + t) * np.exp(-t / tau)]
    return np.array([quad(fi, 0.0, delta, epsabs=0, epsrel=1e-13, limit=200)[0] for fi in f])


def brute_point_flux(Ql, Qr, dQl, dQr, dQ0, gamma, Pr, mu, dt, G=None):
    """I(dt), I(dt/2) through a unit-area interface point by direct quadrature of
    the time-integrated second-order GKS distribution (rotated frame, constant mu)."""
    if G is None:
        G = VelocityGrid()
    ps = G.psi()
    Wl, Wr = prim(Ql, gamma), prim(Qr, gamma)
    gl, gr = G.maxwellian(Wl), G.maxwellian(Wr)
    H = G.H
    Q0 = np.array([G.integrate(ps[i] * (gl * H + gr * (1 - H))) for i in range(5)])
    W0 = prim(Q0, gamma)
    g0 = G.maxwellian(W0)
    p0 = W0[0] / (2 * W0[4])
    tau = mu / p0

    def slopes(g, rho, dQ):
        M = moment_matrix(G, g, rho)
        a = [np.linalg.solve(M, np.asarray(dQ[d]) / rho) for d in range(3)]
        au = slope_field(G, a[0]) * G.U + slope_field(G, a[1]) * G.V + slope_field(G, a[2]) * G.W
        rhs = np.array([-G.integrate(ps[i] * au * g) / rho for i in range(5)])
        A = np.linalg.solve(M, rhs)
        return au, slope_field(G, A)

    dQl, dQr, dQ0 = (np.asarray(x).reshape(3, 5) for x in (dQl, dQr, dQ0))
    au_l, A_l = slopes(gl, Wl[0], dQl)
    au_r, A_r = slopes(gr, Wr[0], dQr)
    au_0, A_0 = slopes(g0, W0[0], dQ0)
    heat = (G.U - W0[1]) * 0.5 * ((G.U - W0[1]) ** 2 + (G.V - W0[2]) ** 2 + (G.W - W0[3]) ** 2 + G.XI2)
    out = []
    for delta in (dt, 0.5 * dt):
        q = time_factors(tau, delta)
        f = (q[0] * g0 + q[1] * au_0 * g0 + q[2] * A_0 * g0
             + q[3] * (gl * H + gr * (1 - H))
             - q[4] * (au_l * gl * H + au_r * gr * (1 - H))
             - tau * q[3] * (A_l * gl * H + A_r * gr * (1 - H)))
        I = np.array([G.integrate(G.U * ps[i] * f) for i in range(5)])
        qh = G.integrate(heat * f)
        I[4] += (1.0 / Pr - 1.0) * qh
        out.append(I)
    return out[0], out[1], tau
