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
