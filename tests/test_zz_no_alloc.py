"""hgks_cfl_dt_noalloc: the CFL time step of a caller-owned device state with
no device allocation.

It serves callers that cannot allocate device memory when they need a time
step (a memory manager that reserved the device at start-up, a solver
embedded in another program's loop, a loop that cannot afford cudaMalloc's
implicit synchronisation).  Its scratch is a fixed file-scope device array
shared by all calls.  This file is collected last, so a run that stops at the
first failure has run every other test before it; it also passes alone.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
GAMMA = 1.4


def test_noalloc_dt_matches_allocating_entry_point():
    import torch
    assert torch.cuda.is_available(), "GPU test"
    from paper_2207_01173_gb300 import hgks

    kw = dict(visc=(1, 1.0 / 1600, 1.0 / (GAMMA * 0.01), 0.7), Pr=0.72)
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    # two calls in a row on different states (the shared scratch keeps the
    # previous call's partial minima in between)
    cases = [((40, 36, 24), 0.5, 0), ((33, 17, 9), 0.35, 2)]
    for n, cfl, nsteps in cases:
        s = hgks.Solver(n, **kw)
        s.init_tgv(0.1, 1.0, 1.0)
        if nsteps:
            s.step(nsteps, 0.5)
        expected = s.compute_dt(cfl)
        q = torch.from_numpy(s.get_state()).cuda()
        hgks.cfl_dt_noalloc(n, q.data_ptr(), dt_dev.data_ptr(), cfl=cfl, gamma=GAMMA)
        torch.cuda.synchronize()
        got = float(dt_dev.item())
        assert got == pytest.approx(expected, rel=1e-15)
        s.close()


def channel_kw(Ma=0.5, Reb=2800.0):
    Tw = 1.0 / (GAMMA * Ma * Ma)
    return dict(lengths=(2 * np.pi, 2.0, np.pi), origin=(0.0, -1.0, 0.0), y_stretch_b=2.0,
                visc=(1, 1.0 / Reb, Tw, 0.7), Pr=0.7, bc_lo=(0, 1, 0), bc_hi=(0, 1, 0), T_wall=Tw,
                body_force=((180.0 / 2800.0) ** 2, 0.0, 0.0))


def test_noalloc_dt_stretched_channel():
    """The wall-stretched channel grid (b = 2): the allocation-free call takes
    its cell heights from the device tanh, the allocating one from a host
    table; they agree to the stated 1e-13 relative, on two calls in a row."""
    import torch
    from paper_2207_01173_gb300 import hgks

    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    for n, nsteps in (((32, 48, 24), 0), ((24, 64, 16), 3)):
        kw = channel_kw()
        s = hgks.Solver(n, **kw)
        s.init_channel(0.5, 0.1, 2800)
        if nsteps:
            s.step(nsteps, 0.5)
        expected = s.compute_dt(0.5)
        q = torch.from_numpy(s.get_state()).cuda()
        hgks.cfl_dt_noalloc(n, q.data_ptr(), dt_dev.data_ptr(), cfl=0.5, gamma=GAMMA,
                            lengths=kw["lengths"], origin=kw["origin"], y_stretch_b=kw["y_stretch_b"])
        torch.cuda.synchronize()
        assert float(dt_dev.item()) == pytest.approx(expected, rel=1e-13)
        s.close()


def test_noalloc_dt_invalid_state_gives_nan():
    """A cell with negative pressure yields NaN, not a step that skips it;
    the next call on a valid state is finite again."""
    import torch
    from paper_2207_01173_gb300 import hgks

    n = (20, 12, 10)
    q = torch.zeros((5, n[2], n[1], n[0]), dtype=torch.float64, device="cuda")
    q[0] = 1.0
    q[4] = 2.5
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    q[4, 3, 5, 7] = -1.0
    hgks.cfl_dt_noalloc(n, q.data_ptr(), dt_dev.data_ptr(), cfl=0.5, gamma=GAMMA)
    torch.cuda.synchronize()
    assert np.isnan(float(dt_dev.item()))
    q[4, 3, 5, 7] = 2.5
    hgks.cfl_dt_noalloc(n, q.data_ptr(), dt_dev.data_ptr(), cfl=0.5, gamma=GAMMA)
    torch.cuda.synchronize()
    c = np.sqrt(GAMMA * 0.4 * 2.5)  # p = (gamma - 1) rho E at rest
    assert float(dt_dev.item()) == pytest.approx(0.5 * (2 * np.pi / 20) / c, rel=1e-15)


def test_noalloc_rejects_oversize_grid():
    import torch
    from paper_2207_01173_gb300 import hgks

    n = (512, 512, 256)  # 67M cells > HGKS_NOALLOC_MAX_CELLS
    assert np.prod(n) > hgks.NOALLOC_MAX_CELLS
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(hgks.HgksError) as e:
        hgks.cfl_dt_noalloc(n, dummy.data_ptr(), dummy.data_ptr())
    assert e.value.status == hgks.HGKS_ERR_INVALID_ARG
    assert "33554432" in str(e.value)
