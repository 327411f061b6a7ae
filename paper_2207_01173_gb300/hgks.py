"""Python binding of the HGKS C-ABI (include/hgks.h): argument marshalling only.

Every step of the solver runs in the CUDA kernels of libhgks.so; this module
converts arguments, passes PyTorch's current CUDA stream by default and turns
status codes into exceptions.  There is no CPU fallback: importing works
without a GPU (so the library can be inspected), but creating a solver on a
machine without a usable CUDA device raises.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

HGKS_OK, HGKS_ERR_INVALID_ARG, HGKS_ERR_OOM, HGKS_ERR_CUDA, HGKS_ERR_NONFINITE, HGKS_ERR_TIMEOUT, HGKS_ERR_STATE = range(7)
BC_PERIODIC, BC_WALL, BC_EXTERNAL = 0, 1, 2
STATE_CURRENT, STATE_STAGE = 0, 1
VISC_CONSTANT, VISC_POWER = 0, 1
FP64, MIXED, MIXED_T64 = 0, 1, 2

_STATUS_NAMES = {0: "HGKS_OK", 1: "HGKS_ERR_INVALID_ARG", 2: "HGKS_ERR_OOM", 3: "HGKS_ERR_CUDA",
                 4: "HGKS_ERR_NONFINITE", 5: "HGKS_ERR_TIMEOUT", 6: "HGKS_ERR_STATE"}


class HgksError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS_NAMES.get(status, status), msg))
        self.status = status


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("y_stretch_b", C.c_double)]


class Visc(C.Structure):
    _fields_ = [("kind", C.c_int), ("mu_ref", C.c_double), ("T_ref", C.c_double), ("omega", C.c_double)]


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


class StepTimes(C.Structure):
    _fields_ = [("total_ms", C.c_double), ("ghost_ms", C.c_double), ("dt_ms", C.c_double),
                ("normal_ms", C.c_double), ("tan1_ms", C.c_double), ("flux_ms", C.c_double),
                ("update_ms", C.c_double), ("other_ms", C.c_double), ("launches", C.c_int),
                ("flux_launches", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FlopModel(C.Structure):
    _fields_ = [("normal_per_face", C.c_double), ("tan1_per_pos", C.c_double), ("flux_per_face", C.c_double),
                ("div_per_face_flux", C.c_double), ("special_per_face_flux", C.c_double),
                ("per_step", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchInfo(C.Structure):
    _fields_ = [("problems", C.c_int), ("tile_sweep", C.c_int), ("tile_cells", C.c_int),
                ("launches_per_step", C.c_int), ("tiles", C.c_longlong), ("last_ms", C.c_double),
                ("last_steps", C.c_int), ("tile_normal", C.c_int), ("tile_tan1", C.c_int),
                ("tile_normal_mx", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_D = C.POINTER(C.c_double)
_lib = None

# every entry point declared in include/hgks.h
EXPORTS = ("hgks_create", "hgks_init_tgv", "hgks_init_channel", "hgks_init_density_wave", "hgks_set_state",
           "hgks_get_state", "hgks_set_time", "hgks_step", "hgks_step_dt", "hgks_compute_dt", "hgks_rhs",
           "hgks_stats", "hgks_footprint_bytes", "hgks_last_error", "hgks_synchronize", "hgks_destroy",
           "hgks_step_timed", "hgks_fp64_probe", "hgks_flop_model", "hgks_cfl_dt_noalloc",
           "hgks_batch_create", "hgks_batch_step", "hgks_batch_tune", "hgks_batch_steps", "hgks_batch_info",
           "hgks_batch_last_error", "hgks_batch_destroy", "hgks_fill_ghosts", "hgks_halo_count", "hgks_halo_get",
           "hgks_halo_set", "hgks_stage")


def library_path():
    return _build.LIB


def lib(build_if_missing=True):
    """Load libhgks.so (building it in-tree when missing)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise ImportError("libhgks.so not found at %s (run __graft_entry__.build())" % path)
        L = C.CDLL(path)
        S = C.c_int
        L.hgks_create.argtypes = [C.POINTER(Grid), C.c_double, C.c_double, C.POINTER(Visc), C.POINTER(Bcs), _D,
                                  C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]
        L.hgks_init_tgv.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double]
        L.hgks_init_channel.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_uint64]
        L.hgks_init_density_wave.argtypes = [C.c_void_p, C.c_double]
        L.hgks_set_state.argtypes = [C.c_void_p, C.c_void_p]
        L.hgks_get_state.argtypes = [C.c_void_p, C.c_void_p]
        L.hgks_set_time.argtypes = [C.c_void_p, C.c_double, C.c_int64]
        L.hgks_step.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.hgks_step_dt.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.hgks_compute_dt.argtypes = [C.c_void_p, C.c_double, _D]
        L.hgks_rhs.argtypes = [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]
        L.hgks_stats.argtypes = [C.c_void_p, C.POINTER(Stats)]
        L.hgks_footprint_bytes.argtypes = [C.POINTER(Grid), C.c_int]
        L.hgks_footprint_bytes.restype = C.c_size_t
        L.hgks_last_error.argtypes = [C.c_void_p]
        L.hgks_last_error.restype = C.c_char_p
        L.hgks_synchronize.argtypes = [C.c_void_p]
        L.hgks_destroy.argtypes = [C.c_void_p]
        L.hgks_destroy.restype = None
        L.hgks_step_timed.argtypes = [C.c_void_p, C.c_double, C.POINTER(StepTimes)]
        L.hgks_fp64_probe.argtypes = [_D]
        L.hgks_flop_model.argtypes = [C.POINTER(Grid), C.c_int, C.POINTER(FlopModel)]
        L.hgks_cfl_dt_noalloc.argtypes = [C.POINTER(Grid), C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                          C.c_void_p]
        L.hgks_batch_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p)]
        L.hgks_batch_step.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.hgks_batch_tune.argtypes = [C.c_void_p, C.c_double, _D]
        L.hgks_batch_info.argtypes = [C.c_void_p, C.POINTER(BatchInfo)]
        L.hgks_batch_steps.argtypes = [C.c_void_p, C.POINTER(C.c_longlong)]
        L.hgks_batch_last_error.argtypes = [C.c_void_p]
        L.hgks_batch_last_error.restype = C.c_char_p
        L.hgks_batch_destroy.argtypes = [C.c_void_p]
        L.hgks_batch_destroy.restype = None
        L.hgks_fill_ghosts.argtypes = [C.c_void_p, C.c_int]
        L.hgks_halo_count.argtypes = [C.c_void_p, C.c_int]
        L.hgks_halo_count.restype = C.c_size_t
        L.hgks_halo_get.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p]
        L.hgks_halo_set.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p]
        L.hgks_stage.argtypes = [C.c_void_p, C.c_int, C.c_double]
        for name in EXPORTS:
            if name not in ("hgks_footprint_bytes", "hgks_last_error", "hgks_destroy", "hgks_batch_last_error",
                            "hgks_batch_destroy", "hgks_halo_count"):
                getattr(L, name).restype = S
        _lib = L
    return _lib


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return C.c_void_p(0)


def make_grid(n, lengths=(2 * np.pi, 2 * np.pi, 2 * np.pi), origin=(0.0, 0.0, 0.0), y_stretch_b=0.0):
    return Grid(int(n[0]), int(n[1]), int(n[2]), *[float(v) for v in lengths], *[float(v) for v in origin],
                float(y_stretch_b))


def footprint_bytes(n, precision=FP64, **grid_kw):
    g = make_grid(n, **grid_kw)
    return int(lib().hgks_footprint_bytes(C.byref(g), precision))


def flop_model(n, precision=FP64, **grid_kw):
    """Algorithmic flops of the step (host-side count of the kernels' arithmetic)."""
    g = make_grid(n, **grid_kw)
    m = FlopModel()
    st = lib().hgks_flop_model(C.byref(g), precision, C.byref(m))
    if st != HGKS_OK:
        raise HgksError(st, "flop model")
    return m.as_dict()


def fp64_probe():
    """Measured FP64 FMA throughput of the current device, TFLOP/s."""
    v = C.c_double()
    st = lib().hgks_fp64_probe(C.byref(v))
    if st != HGKS_OK:
        raise HgksError(st, lib().hgks_last_error(None).decode())
    return v.value


NOALLOC_MAX_CELLS = 33554432


def cfl_dt_noalloc(n, d_q, d_dt, cfl=0.5, gamma=1.4, stream=None, **grid_kw):
    """CFL time step of a caller-owned device state without device allocation.

    d_q, d_dt: device pointers (ints) to double[5][nz][ny][nx] and to one
    double.  Asynchronous on `stream` (default: PyTorch's current stream).
    """
    g = make_grid(n, **grid_kw)
    st = lib().hgks_cfl_dt_noalloc(C.byref(g), gamma, cfl, C.c_void_p(d_q), C.c_void_p(d_dt),
                                   stream if stream is not None else _current_stream())
    if st != HGKS_OK:
        raise HgksError(st, lib().hgks_last_error(None).decode())


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


class Solver:
    """One HGKS problem on the GPU (device-resident state owned by libhgks)."""

    def __init__(self, n, lengths=(2 * np.pi, 2 * np.pi, 2 * np.pi), origin=(0.0, 0.0, 0.0), y_stretch_b=0.0,
                 gamma=1.4, Pr=0.72, visc=(VISC_CONSTANT, 0.0, 1.0, 0.0), bc_lo=(0, 0, 0), bc_hi=(0, 0, 0),
                 T_wall=0.0, body_force=(0.0, 0.0, 0.0), precision=FP64, stream=None):
        L = lib()
        self.n = tuple(int(v) for v in n)
        self._grid = make_grid(self.n, lengths, origin, y_stretch_b)
        v = Visc(*visc)
        b = Bcs((C.c_int * 3)(*bc_lo), (C.c_int * 3)(*bc_hi), T_wall)
        bf = _f64(body_force, 3)
        h = C.c_void_p()
        self.h = None
        st = L.hgks_create(C.byref(self._grid), gamma, Pr, C.byref(v), C.byref(b), bf.ctypes.data_as(_D),
                           precision, stream if stream is not None else _current_stream(), C.byref(h))
        if st != HGKS_OK:
            raise HgksError(st, L.hgks_last_error(None).decode())
        self.h = h

    # -- helpers --------------------------------------------------------
    def _check(self, st):
        if st != HGKS_OK:
            raise HgksError(st, lib().hgks_last_error(self.h).decode())

    @property
    def shape(self):
        nx, ny, nz = self.n
        return (5, nz, ny, nx)

    def close(self):
        if self.h:
            lib().hgks_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C-ABI mirror ---------------------------------------------------
    def init_tgv(self, Ma=0.1, U0=1.0, rho0=1.0):
        self._check(lib().hgks_init_tgv(self.h, Ma, U0, rho0))

    def init_channel(self, Ma_b=0.5, noise_amp=0.1, seed=2800):
        self._check(lib().hgks_init_channel(self.h, Ma_b, noise_amp, seed))

    def init_density_wave(self, amp=0.2):
        self._check(lib().hgks_init_density_wave(self.h, amp))

    def set_state(self, q):
        """q: numpy float64 [5][nz][ny][nx] or a pinned/contiguous CPU torch tensor."""
        ptr, keep = self._host_ptr(q, writable=False)
        self._check(lib().hgks_set_state(self.h, ptr))
        del keep

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.float64)
        ptr, keep = self._host_ptr(out, writable=True)
        self._check(lib().hgks_get_state(self.h, ptr))
        return out

    def set_time(self, t, step):
        self._check(lib().hgks_set_time(self.h, t, step))

    def step(self, nsteps=1, cfl=0.5):
        self._check(lib().hgks_step(self.h, nsteps, cfl))

    def step_dt(self, nsteps, dt):
        self._check(lib().hgks_step_dt(self.h, nsteps, dt))

    def step_timed(self, cfl=0.5):
        """One step with per-kernel-kind device times (ms)."""
        t = StepTimes()
        self._check(lib().hgks_step_timed(self.h, cfl, C.byref(t)))
        return t.as_dict()

    def compute_dt(self, cfl):
        d = C.c_double()
        self._check(lib().hgks_compute_dt(self.h, cfl, C.byref(d)))
        return d.value

    def rhs(self, dt):
        Lh = np.empty(self.shape)
        dLh = np.empty(self.shape)
        self._check(lib().hgks_rhs(self.h, dt, Lh.ctypes.data_as(C.c_void_p), dLh.ctypes.data_as(C.c_void_p)))
        return Lh, dLh

    def stats(self):
        s = Stats()
        self._check(lib().hgks_stats(self.h, C.byref(s)))
        return s.as_dict()

    def synchronize(self):
        self._check(lib().hgks_synchronize(self.h))

    # -- sub-domains (EXTERNAL z sides): the step in phases ---------------
    def fill_ghosts(self, state=STATE_CURRENT):
        self._check(lib().hgks_fill_ghosts(self.h, state))

    def halo_count(self, dir=2):
        """Doubles of one halo buffer of direction dir ([5][3][ny+6][nx+6] for z)."""
        return int(lib().hgks_halo_count(self.h, dir))

    def halo_get(self, state, side, d_buf, dir=2):
        """Three boundary layers of `side` (0 low, 1 high) into device pointer d_buf (int)."""
        self._check(lib().hgks_halo_get(self.h, state, dir, side, C.c_void_p(d_buf)))

    def halo_set(self, state, side, d_buf, dir=2):
        """Device buffer d_buf (int) into the three ghost layers of `side`."""
        self._check(lib().hgks_halo_set(self.h, state, dir, side, C.c_void_p(d_buf)))

    def stage(self, stage, dt):
        self._check(lib().hgks_stage(self.h, stage, dt))

    def _host_ptr(self, a, writable):
        size = int(np.prod(self.shape))
        if isinstance(a, np.ndarray):
            if a.dtype != np.float64 or a.size != size or not a.flags["C_CONTIGUOUS"]:
                if writable:
                    raise ValueError("output must be a C-contiguous float64 array of shape %s" % (self.shape,))
                a = _f64(a, size)
            return C.c_void_p(a.ctypes.data), a
        # torch CPU tensor (e.g. pinned host memory)
        if getattr(a, "is_cuda", False) or a.numel() != size or not a.is_contiguous():
            raise ValueError("expected a contiguous CPU tensor with %d elements" % size)
        import torch
        if a.dtype != torch.float64:
            raise ValueError("expected float64")
        return C.c_void_p(a.data_ptr()), a


class Batch:
    """Several Solver problems advanced together: one persistent kernel per
    pass over a tile work-list spanning all of them, one CUDA graph per step.

    Keep the solvers alive while the batch exists; close the batch first."""

    def __init__(self, solvers):
        self.b = None
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[sv.h.value for sv in self.solvers])
        b = C.c_void_p()
        st = lib().hgks_batch_create(arr, len(self.solvers), C.byref(b))
        if st != HGKS_OK:
            raise HgksError(st, lib().hgks_last_error(None).decode())
        self.b = b

    def _check(self, st):
        if st != HGKS_OK:
            raise HgksError(st, lib().hgks_batch_last_error(self.b).decode())

    def step(self, nsteps=1, cfl=0.5):
        self._check(lib().hgks_batch_step(self.b, nsteps, cfl))

    def tune(self, cfl=0.5):
        """Pick the tile size of each tunable pass by timing it; returns the
        summed time (ms) of the tuned passes in one timing run."""
        ms = C.c_double()
        self._check(lib().hgks_batch_tune(self.b, cfl, C.byref(ms)))
        return ms.value

    def steps(self):
        """Step counter of each problem after the last step call."""
        a = (C.c_longlong * len(self.solvers))()
        self._check(lib().hgks_batch_steps(self.b, a))
        return list(a)

    def info(self):
        i = BatchInfo()
        self._check(lib().hgks_batch_info(self.b, C.byref(i)))
        return i.as_dict()

    def close(self):
        if self.b:
            lib().hgks_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
