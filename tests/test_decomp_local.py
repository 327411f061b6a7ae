"""Host logic of the one-process slab driver (decomp.exchange_local_slabs,
step_local_slabs, local_slab_stats) on fake slabs, without a GPU.

A fake slab holds a padded column of z planes (3 ghost planes per side) and
implements the calls the driver makes; "device buffers" are integer keys into
a dict of numpy arrays.  After an exchange every slab's ghost planes must hold
its periodic neighbours' boundary planes, exactly as a ghost fill of the
undivided column would; the driver must fill x / y ghosts before packing,
pack every slab before unpacking any, take the minimum time step over slabs,
and weight volume averages by slab length.
"""
import numpy as np

from paper_2207_01173_gb300 import decomp

NG = 3


class FakeSlab:
    def __init__(self, planes, bufs, log, name, dt, stats):
        self.q = {0: np.zeros(len(planes) + 2 * NG), 1: np.zeros(len(planes) + 2 * NG)}
        self.q[0][NG:-NG] = planes
        self.bufs, self.log, self.name, self.dt, self._stats = bufs, log, name, dt, stats

    def fill_ghosts(self, state):
        self.log.append(("fill", self.name, state))

    def halo_get(self, state, side, ptr):
        self.log.append(("get", self.name, state))
        q = self.q[state]
        self.bufs[ptr][:] = q[NG:2 * NG] if side == 0 else q[-2 * NG:-NG]

    def halo_set(self, state, side, ptr):
        self.log.append(("set", self.name, state))
        q = self.q[state]
        if side == 0:
            q[:NG] = self.bufs[ptr]
        else:
            q[-NG:] = self.bufs[ptr]

    def compute_dt(self, cfl):
        return cfl * self.dt

    def stage(self, stage, dt):
        self.log.append(("stage", self.name, stage, dt))
        if stage == 1:
            self.q[1][:] = self.q[0]  # the stage state starts as a copy

    def stats(self):
        return dict(self._stats)


def make(sizes, log):
    col = np.arange(sum(sizes), dtype=float) + 1.0
    bufs, slabs, k0 = {}, [], 0
    for i, nk in enumerate(sizes):
        lo, hi = 2 * i, 2 * i + 1
        bufs[lo], bufs[hi] = np.zeros(NG), np.zeros(NG)
        st = {"Ek": float(i + 1), "enstrophy": 2.0, "eps_com": 1.0 + i, "wall_shear": 0.5 * i, "mass": 10.0,
              "energy": 3.0, "mom": [1.0, 2.0, 3.0], "max_mach": 0.1 * (i + 1), "t": 0.0, "step": 0, "dt": 0.0}
        slabs.append(FakeSlab(col[k0:k0 + nk], bufs, log, i, dt=1.0 + (i * 7 % 3), stats=st))
        k0 += nk
    ptrs = [(2 * i, 2 * i + 1) for i in range(len(sizes))]
    return col, slabs, ptrs


def test_exchange_fills_ghosts_from_the_periodic_ring():
    for sizes in ((8, 4), (3, 5, 4), (6,)):
        log = []
        col, slabs, ptrs = make(sizes, log)
        decomp.exchange_local_slabs(slabs, 0, ptrs)
        n = len(col)
        k0 = 0
        for s, nk in zip(slabs, sizes):
            below = [col[(k0 - NG + m) % n] for m in range(NG)]
            above = [col[(k0 + nk + m) % n] for m in range(NG)]
            assert np.array_equal(s.q[0][:NG], below)
            assert np.array_equal(s.q[0][-NG:], above)
            assert np.array_equal(s.q[0][NG:-NG], col[k0:k0 + nk])
            k0 += nk
        kinds = [e[0] for e in log]
        k = len(sizes)
        # every slab fills its x / y ghosts, then all pack, then all unpack
        assert kinds == ["fill"] * k + ["get"] * (2 * k) + ["set"] * (2 * k)


def test_step_takes_the_global_minimum_and_exchanges_each_stage():
    log = []
    _, slabs, ptrs = make((3, 5, 4), log)
    dts = decomp.step_local_slabs(slabs, ptrs, 2, 0.5)
    assert dts == [0.5 * min(s.dt for s in slabs)] * 2
    stages = [e for e in log if e[0] == "stage"]
    assert [e[2] for e in stages] == [1, 1, 1, 2, 2, 2] * 2
    assert all(e[3] == dts[0] for e in stages)
    # the stage state's halos are exchanged before stage 2
    first2 = next(i for i, e in enumerate(log) if e[0] == "stage" and e[2] == 2)
    assert any(e[0] == "set" and e[2] == 1 for e in log[:first2])


def test_stats_weight_averages_by_slab_length():
    log = []
    _, slabs, ptrs = make((3, 5, 4), log)
    lz = [3.0, 5.0, 4.0]
    out = decomp.local_slab_stats(slabs, ptrs, lz)
    assert out["Ek"] == (1 * 3 + 2 * 5 + 3 * 4) / 12.0
    assert out["eps_com"] == (1 * 3 + 2 * 5 + 3 * 4) / 12.0
    assert out["wall_shear"] == (0 * 3 + 0.5 * 5 + 1.0 * 4) / 12.0
    assert out["mass"] == 30.0 and out["energy"] == 9.0 and out["mom"] == [3.0, 6.0, 9.0]
    assert out["max_mach"] == 0.1 * 3
    assert log[0][0] == "fill"  # the current state's halos first (vorticity stencils)
