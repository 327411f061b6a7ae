"""ctypes binding of the C oracle (test infrastructure only).

Mirrors the product binding's shape with `hgks_ref_` names so tests can diff
the two.  Only the test suite, the smoke check and the benchmark's CPU
baseline may use it.
"""
import ctypes as C
import os

import numpy as np

from .build import build_oracle

BC_PERIODIC, BC_WALL, BC_EXTERNAL = 0, 1, 2
HALO_FN = C.CFUNCTYPE(None, C.c_void_p, C.POINTER(C.c_double))
MIN_FN = C.CFUNCTYPE(C.c_double, C.c_void_p, C.c_double)
NG = 3
VISC_CONSTANT, VISC_POWER = 0, 1


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("y_stretch_b", C.c_double)]


class Visc(C.Structure):
    _fields_ = [("kind", C.c_int), ("mu_ref", C.c_double), ("T_ref", C.c_double),
                ("omega", C.c_double)]


class Bcs(C.Structure):
    _fields_ = [("lo", C.c_int * 3), ("hi", C.c_int * 3), ("T_wall", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("t", C.c_double), ("step", C.c_int64), ("dt", C.c_double),
                ("Ek", C.c_double), ("enstrophy", C.c_double), ("eps_com", C.c_double),
                ("mass", C.c_double), ("mom", C.c_double * 3), ("energy", C.c_double),
                ("max_mach", C.c_double), ("wall_shear", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "mom"}
        d["mom"] = list(self.mom)
        return d


_lib = None
_D = C.POINTER(C.c_double)


def lib():
    """The oracle library: oracle/_build/libhgks_ref.so, or the library named
    by HGKS_REF_LIB (the pin suite's own check that planted mistakes in a
    copy of the oracle make its pins fail)."""
    global _lib
    if _lib is None:
        L = C.CDLL(os.environ.get("HGKS_REF_LIB") or build_oracle())
        L.hgks_ref_create.argtypes = [C.POINTER(Grid), C.c_double, C.c_double, C.POINTER(Visc),
                                      C.POINTER(Bcs), _D, C.POINTER(C.c_void_p)]
        L.hgks_ref_init_tgv.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double]
        L.hgks_ref_init_channel.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_uint64]
        L.hgks_ref_init_density_wave.argtypes = [C.c_void_p, C.c_double]
        L.hgks_ref_set_state.argtypes = [C.c_void_p, _D]
        L.hgks_ref_get_state.argtypes = [C.c_void_p, _D]
        L.hgks_ref_set_time.argtypes = [C.c_void_p, C.c_double, C.c_int64]
        L.hgks_ref_step.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.hgks_ref_step_dt.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.hgks_ref_compute_dt.argtypes = [C.c_void_p, C.c_double, _D]
        L.hgks_ref_rhs.argtypes = [C.c_void_p, C.c_double, _D, _D]
        L.hgks_ref_rhs_cells.argtypes = [C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_int64), _D, _D]
        L.hgks_ref_stats.argtypes = [C.c_void_p, C.POINTER(Stats)]
        L.hgks_ref_face_flux.argtypes = [C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, _D, _D]
        L.hgks_ref_last_error.argtypes = [C.c_void_p]
        L.hgks_ref_last_error.restype = C.c_char_p
        L.hgks_ref_destroy.argtypes = [C.c_void_p]
        L.hgks_ref_destroy.restype = None
        L.hgks_ref_moments_1d.argtypes = [C.c_double, C.c_double, C.c_int, C.c_int, _D]
        L.hgks_ref_moments_1d.restype = None
        L.hgks_ref_moments_xi.argtypes = [C.c_double, C.c_double, _D]
        L.hgks_ref_moments_xi.restype = None
        for name in ("hgks_ref_prim",):
            getattr(L, name).argtypes = [_D, C.c_double, _D]
            getattr(L, name).restype = None
        L.hgks_ref_micro_slope.argtypes = [_D, C.c_double, _D, _D]
        L.hgks_ref_micro_slope.restype = None
        L.hgks_ref_slope_moments.argtypes = [_D, C.c_double, _D, _D]
        L.hgks_ref_slope_moments.restype = None
        L.hgks_ref_compat.argtypes = [_D, _D, C.c_double, _D]
        L.hgks_ref_compat.restype = None
        L.hgks_ref_time_coeffs.argtypes = [C.c_double, C.c_double, _D]
        L.hgks_ref_time_coeffs.restype = None
        L.hgks_ref_time_fit.argtypes = [_D, _D, C.c_double, _D, _D]
        L.hgks_ref_time_fit.restype = None
        L.hgks_ref_point_flux.argtypes = [_D, _D, _D, _D, _D, C.c_double, C.c_double,
                                          C.POINTER(Visc), C.c_double, _D, _D, _D, _D]
        L.hgks_ref_point_flux.restype = None
        L.hgks_ref_weno_z.argtypes = [_D, C.c_double, C.c_double]
        L.hgks_ref_weno_z.restype = C.c_double
        L.hgks_ref_weno_linear_weights.argtypes = [C.c_double, _D]
        L.hgks_ref_weno_linear_weights.restype = None
        L.hgks_ref_weno_candidates.argtypes = [_D, C.c_double, _D, _D]
        L.hgks_ref_weno_candidates.restype = None
        L.hgks_ref_quartic_coeffs.argtypes = [C.c_double, _D, _D]
        L.hgks_ref_quartic_coeffs.restype = None
        L.hgks_ref_splitmix64.argtypes = [C.c_uint64]
        L.hgks_ref_splitmix64.restype = C.c_uint64
        L.hgks_ref_set_hooks.argtypes = [C.c_void_p, HALO_FN, MIN_FN, C.c_void_p]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_D)


def _arr(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))
    if n is not None:
        assert a.size == n
    return a


class RefSolver:
    """Oracle HGKS solver on the CPU (FP64)."""

    def __init__(self, n, lengths=(2 * np.pi, 2 * np.pi, 2 * np.pi), origin=(0.0, 0.0, 0.0),
                 y_stretch_b=0.0, gamma=1.4, Pr=0.72, visc=(VISC_CONSTANT, 0.0, 1.0, 0.0),
                 bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), T_wall=0.0, body_force=(0.0, 0.0, 0.0)):
        self.n = tuple(int(v) for v in n)
        g = Grid(self.n[0], self.n[1], self.n[2], *lengths, *origin, y_stretch_b)
        v = Visc(*visc)
        b = Bcs((C.c_int * 3)(*bc_lo), (C.c_int * 3)(*bc_hi), T_wall)
        bf = _arr(body_force, 3)
        h = C.c_void_p()
        st = lib().hgks_ref_create(C.byref(g), gamma, Pr, C.byref(v), C.byref(b), _p(bf), C.byref(h))
        if st != 0:
            raise ValueError("hgks_ref_create failed: %d" % st)
        self.h = h
        self.gamma, self.Pr = gamma, Pr

    def _check(self, st, what):
        if st != 0:
            raise RuntimeError("%s failed (%d): %s" % (what, st, lib().hgks_ref_last_error(self.h).decode()))

    def close(self):
        if self.h:
            lib().hgks_ref_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        nx, ny, nz = self.n
        return (5, nz, ny, nx)

    def init_tgv(self, Ma=0.1, U0=1.0, rho0=1.0):
        self._check(lib().hgks_ref_init_tgv(self.h, Ma, U0, rho0), "init_tgv")

    def init_channel(self, Ma_b=0.5, noise_amp=0.1, seed=2800):
        self._check(lib().hgks_ref_init_channel(self.h, Ma_b, noise_amp, seed), "init_channel")

    def init_density_wave(self, amp=0.2):
        self._check(lib().hgks_ref_init_density_wave(self.h, amp), "init_density_wave")

    def set_state(self, q):
        a = _arr(q, int(np.prod(self.shape)))
        self._check(lib().hgks_ref_set_state(self.h, _p(a)), "set_state")

    def get_state(self):
        a = np.empty(self.shape, dtype=np.float64)
        self._check(lib().hgks_ref_get_state(self.h, _p(a)), "get_state")
        return a

    def set_time(self, t, step):
        self._check(lib().hgks_ref_set_time(self.h, t, step), "set_time")

    def set_hooks(self, halo=None, dtmin=None):
        """halo(q) receives every ghost-filled padded state as a writable
        array [5][nz+6][ny+6][nx+6]; dtmin(m) maps this rank's CFL minimum to
        the global one.  None removes a hook."""
        nx, ny, nz = self.n
        shape = (5, nz + 2 * NG, ny + 2 * NG, nx + 2 * NG)

        def _halo(user, ptr):
            halo(np.ctypeslib.as_array(ptr, shape=shape))

        def _min(user, m):
            return float(dtmin(m))

        self._hooks = (HALO_FN(_halo) if halo else HALO_FN(), MIN_FN(_min) if dtmin else MIN_FN())
        self._check(lib().hgks_ref_set_hooks(self.h, self._hooks[0], self._hooks[1], None), "set_hooks")

    def step(self, nsteps=1, cfl=0.5):
        self._check(lib().hgks_ref_step(self.h, nsteps, cfl), "step")

    def step_dt(self, nsteps, dt):
        self._check(lib().hgks_ref_step_dt(self.h, nsteps, dt), "step_dt")

    def compute_dt(self, cfl):
        d = C.c_double()
        self._check(lib().hgks_ref_compute_dt(self.h, cfl, C.byref(d)), "compute_dt")
        return d.value

    def rhs(self, dt):
        L = np.empty(self.shape)
        dL = np.empty(self.shape)
        self._check(lib().hgks_ref_rhs(self.h, dt, _p(L), _p(dL)), "rhs")
        return L, dL

    def rhs_cells(self, dt, cells):
        """L, dL at interior cells given by linear index (k ny + j) nx + i; returns [n][5] arrays."""
        idx = np.ascontiguousarray(np.asarray(cells, dtype=np.int64))
        L = np.empty((idx.size, 5))
        dL = np.empty((idx.size, 5))
        self._check(lib().hgks_ref_rhs_cells(self.h, dt, idx.size, idx.ctypes.data_as(C.POINTER(C.c_int64)),
                                             _p(L), _p(dL)), "rhs_cells")
        return L, dL

    def face_flux(self, dt, d, f, a, b):
        """F^n and dF^n/dt (times the face area) of one interface: direction d,
        between cells f-1 and f along d, tangential cell indices (a, b)."""
        F, dF = np.empty(5), np.empty(5)
        self._check(lib().hgks_ref_face_flux(self.h, dt, d, f, a, b, _p(F), _p(dF)), "face_flux")
        return F, dF

    def stats(self):
        s = Stats()
        self._check(lib().hgks_ref_stats(self.h, C.byref(s)), "stats")
        return s.as_dict()


# ---- unit-level helpers -------------------------------------------------
def moments_1d(U, lam, rng, nmax=8):
    out = np.empty(nmax)
    lib().hgks_ref_moments_1d(U, lam, rng, nmax, _p(out))
    return out


def moments_xi(lam, K):
    out = np.empty(3)
    lib().hgks_ref_moments_xi(lam, K, _p(out))
    return out


def prim(Q, K):
    Q = _arr(Q, 5)
    W = np.empty(5)
    lib().hgks_ref_prim(_p(Q), K, _p(W))
    return W


def micro_slope(W, K, dQ):
    W, dQ = _arr(W, 5), _arr(dQ, 5)
    a = np.empty(5)
    lib().hgks_ref_micro_slope(_p(W), K, _p(dQ), _p(a))
    return a


def slope_moments(W, K, a):
    W, a = _arr(W, 5), _arr(a, 5)
    out = np.empty(5)
    lib().hgks_ref_slope_moments(_p(W), K, _p(a), _p(out))
    return out


def compat(Ql, Qr, K):
    Ql, Qr = _arr(Ql, 5), _arr(Qr, 5)
    out = np.empty(5)
    lib().hgks_ref_compat(_p(Ql), _p(Qr), K, _p(out))
    return out


def time_coeffs(tau, delta):
    out = np.empty(5)
    lib().hgks_ref_time_coeffs(tau, delta, _p(out))
    return out


def time_fit(If, Ih, dt):
    If, Ih = _arr(If, 5), _arr(Ih, 5)
    Fn, dFn = np.empty(5), np.empty(5)
    lib().hgks_ref_time_fit(_p(If), _p(Ih), dt, _p(Fn), _p(dFn))
    return Fn, dFn


def point_flux(Ql, Qr, dQl, dQr, dQ0, gamma, Pr, visc, dt):
    """GKS flux at one interface point (rotated frame); returns If, Ih, Fn, dFn."""
    Ql, Qr = _arr(Ql, 5), _arr(Qr, 5)
    dQl, dQr, dQ0 = _arr(dQl, 15), _arr(dQr, 15), _arr(dQ0, 15)
    v = Visc(*visc)
    outs = [np.empty(5) for _ in range(4)]
    lib().hgks_ref_point_flux(_p(Ql), _p(Qr), _p(dQl), _p(dQr), _p(dQ0), gamma, Pr, C.byref(v), dt,
                              *[_p(o) for o in outs])
    return tuple(outs)


def weno_z(X, sigma, eps=1e-6):
    X = _arr(X, 5)
    return lib().hgks_ref_weno_z(_p(X), sigma, eps)


def weno_linear_weights(sigma):
    d = np.empty(3)
    lib().hgks_ref_weno_linear_weights(sigma, _p(d))
    return d


def weno_candidates(X, sigma):
    X = _arr(X, 5)
    p, b = np.empty(3), np.empty(3)
    lib().hgks_ref_weno_candidates(_p(X), sigma, _p(p), _p(b))
    return p, b


def quartic_coeffs(sigma):
    Lc, Dc = np.empty(5), np.empty(5)
    lib().hgks_ref_quartic_coeffs(sigma, _p(Lc), _p(Dc))
    return Lc, Dc


def splitmix64(x):
    return lib().hgks_ref_splitmix64(x)
