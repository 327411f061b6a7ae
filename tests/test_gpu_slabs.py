"""The domain decomposition of the CUDA path on one GPU (Sec. 3.2, Alg. 2).

One domain is split into z slabs, each a solver handle whose z sides are
EXTERNAL; before each stage the slabs' ghost layers are exchanged device to
device through caller-owned buffers (hgks_halo_get / hgks_halo_set), and the
time step is the minimum over slabs of each slab's CFL limit.  The stepped
slabs must reproduce the undivided run bit for bit (same arithmetic on the
same padded values), and the diagnostics assembled from the slabs must match
the undivided ones to rounding of the sums.
"""
import numpy as np
import pytest

from tests.test_gpu_parity import TGV_KW, channel_kw

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2207_01173_gb300 import hgks
    return hgks


def make_slabs(hg, n, sizes, kw, precision):
    import torch
    lengths = kw.get("lengths", (2 * np.pi,) * 3)
    origin = kw.get("origin", (0.0, 0.0, 0.0))
    dz = lengths[2] / n[2]
    solvers, bufs, lz, k0 = [], [], [], 0
    for nk in sizes:
        assert (dz * nk) / nk == dz  # every slab keeps the global cell size
        skw = dict(kw)
        skw["lengths"] = (lengths[0], lengths[1], dz * nk)
        skw["origin"] = (origin[0], origin[1], origin[2] + k0 * dz)
        lo, hi = list(kw.get("bc_lo", (0, 0, 0))), list(kw.get("bc_hi", (0, 0, 0)))
        lo[2] = hi[2] = hg.BC_EXTERNAL
        skw["bc_lo"], skw["bc_hi"] = tuple(lo), tuple(hi)
        sv = hg.Solver((n[0], n[1], nk), precision=precision, **skw)
        m = sv.halo_count()
        assert m == 5 * 3 * (n[0] + 6) * (n[1] + 6)
        pair = (torch.empty(m, dtype=torch.float64, device="cuda"), torch.empty(m, dtype=torch.float64, device="cuda"))
        solvers.append(sv)
        bufs.append(pair)
        lz.append(dz * nk)
        k0 += nk
    return solvers, bufs, lz


def run_case(hg, n, sizes, kw, init, steps, precision):
    from paper_2207_01173_gb300 import decomp
    whole = hg.Solver(n, precision=precision, **kw)
    init(whole)
    q0 = whole.get_state()
    solvers, bufs, lz = make_slabs(hg, n, sizes, kw, precision)
    k0 = 0
    for sv, nk in zip(solvers, sizes):
        sv.set_state(np.ascontiguousarray(q0[:, k0:k0 + nk]))
        k0 += nk
    ptrs = [(lo.data_ptr(), hi.data_ptr()) for lo, hi in bufs]
    dts = decomp.step_local_slabs(solvers, ptrs, steps, 0.5)
    dts_whole = []
    for _ in range(steps):
        whole.step(1, 0.5)
        dts_whole.append(whole.stats()["dt"])
    q_split = np.concatenate([sv.get_state() for sv in solvers], axis=1)
    q_whole = whole.get_state()
    s_split = decomp.local_slab_stats(solvers, ptrs, lz)
    s_whole = whole.stats()
    for sv in solvers:
        sv.close()
    whole.close()
    return dts, dts_whole, q_split, q_whole, s_split, s_whole


CASES = [
    # grid, slab sizes: two uneven slabs, three uneven slabs
    ((12, 10, 16), (10, 6)),
    ((12, 10, 16), (4, 7, 5)),
]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("n,sizes", CASES)
def test_tgv_slabs_equal_undivided(hg, n, sizes, precision):
    dts, dts_whole, qs, qw, ss, sw = run_case(hg, n, sizes, TGV_KW, lambda s: s.init_tgv(0.1, 1.0, 1.0), 3, precision)
    assert dts == dts_whole  # global CFL minimum, bit for bit
    assert np.array_equal(qs, qw)
    assert ss["step"] == sw["step"] == 3 and ss["t"] == sw["t"]
    for k in ("Ek", "enstrophy", "eps_com", "mass", "energy"):
        assert ss[k] == pytest.approx(sw[k], rel=1e-13, abs=1e-300), k
    assert ss["max_mach"] == sw["max_mach"]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("sizes", [(5, 7), (3, 4, 5)])
def test_channel_slabs_equal_undivided(hg, sizes, precision):
    n = (8, 16, 12)
    dts, dts_whole, qs, qw, ss, sw = run_case(hg, n, sizes, channel_kw(), lambda s: s.init_channel(0.5, 0.1, 2800), 3,
                                              precision)
    assert dts == dts_whole
    assert np.array_equal(qs, qw)
    for k in ("Ek", "enstrophy", "eps_com", "mass", "energy", "wall_shear"):
        assert ss[k] == pytest.approx(sw[k], rel=1e-12), k


def test_stage_order_and_batch_rejection(hg):
    import torch
    kw = dict(TGV_KW, bc_lo=(0, 0, hg.BC_EXTERNAL), bc_hi=(0, 0, hg.BC_EXTERNAL))
    sv = hg.Solver((8, 8, 6), **kw)
    sv.init_tgv(0.1, 1.0, 1.0)
    with pytest.raises(hg.HgksError) as e:
        sv.stage(2, 1e-3)  # stage 2 before stage 1
    assert e.value.status == hg.HGKS_ERR_STATE
    # one slab alone is its own periodic neighbour: set its halos, run stage 1
    lo = torch.empty(sv.halo_count(), dtype=torch.float64, device="cuda")
    hi = torch.empty_like(lo)
    sv.fill_ghosts(0)
    sv.halo_get(0, 0, lo.data_ptr())
    sv.halo_get(0, 1, hi.data_ptr())
    sv.halo_set(0, 0, hi.data_ptr())
    sv.halo_set(0, 1, lo.data_ptr())
    sv.stage(1, 1e-3)
    sv.set_state(sv.get_state())  # a new state in between cancels the pending stage 1
    with pytest.raises(hg.HgksError) as e:
        sv.stage(2, 1e-3)
    assert e.value.status == hg.HGKS_ERR_STATE
    with pytest.raises(hg.HgksError) as e:
        sv.halo_get(0, 0, 0)  # NULL buffer
    assert e.value.status == hg.HGKS_ERR_INVALID_ARG
    buf = torch.empty(sv.halo_count(), dtype=torch.float64, device="cuda")
    with pytest.raises(hg.HgksError) as e:
        sv.halo_get(0, 0, buf.data_ptr(), dir=1)
    assert e.value.status == hg.HGKS_ERR_INVALID_ARG
    with pytest.raises(hg.HgksError) as e:
        hg.Batch([sv])
    assert e.value.status == hg.HGKS_ERR_INVALID_ARG
    sv.close()
