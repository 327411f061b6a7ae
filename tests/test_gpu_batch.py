"""Batched stepping (hgks_batch_*): many problems with uneven grids, gas
parameters and precisions advanced by one work-list kernel per pass and one
CUDA graph per step.  Every position runs the same arithmetic as in the
single-problem kernels, so a batch must reproduce the problems stepped one by
one bit for bit."""
import numpy as np
import pytest

from tests.test_gpu_parity import TGV_KW, channel_kw

pytestmark = pytest.mark.gpu
GAMMA = 1.4


@pytest.fixture(scope="module")
def hg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2207_01173_gb300 import hgks
    return hgks


def tgv_kw(Ma, Re):
    from paper_2207_01173_gb300.workloads import tgv_solver_kwargs
    return tgv_solver_kwargs(Ma, Re)


PROBLEMS = [((12, 16, 10), 0.1, 1600.0, 0), ((20, 12, 8), 0.3, 800.0, 0), ((8, 8, 8), 0.5, 3200.0, 1),
            ((24, 10, 14), 0.2, 400.0, 1), ((9, 7, 1), 0.15, 1000.0, 0)]


def make(hg, spec):
    n, Ma, Re, prec = spec
    s = hg.Solver(n, precision=prec, **tgv_kw(Ma, Re))
    s.init_tgv(Ma, 1.0, 1.0)
    return s


def test_batch_matches_individual_steps_bitwise(hg):
    single = [make(hg, p) for p in PROBLEMS]
    for s in single:
        s.step(4, 0.5)
    batched = [make(hg, p) for p in PROBLEMS]
    b = hg.Batch(batched)
    assert b.info()["problems"] == len(PROBLEMS)
    b.step(4, 0.5)
    for s1, s2 in zip(single, batched):
        assert np.array_equal(s1.get_state(), s2.get_state())
        a, c = s1.stats(), s2.stats()
        assert a["step"] == c["step"] == 4 and a["t"] == c["t"]
    # the handles keep working on their own after batch steps
    b.close()
    for s1, s2 in zip(single, batched):
        s1.step(1, 0.5)
        s2.step(1, 0.5)
        assert np.array_equal(s1.get_state(), s2.get_state())


def test_batch_with_walls_matches_and_tunes(hg, oracle):
    kw = channel_kw()
    ch1 = hg.Solver((10, 16, 8), **kw)
    ch2 = hg.Solver((10, 16, 8), **kw)
    for s in (ch1, ch2):
        s.init_channel(0.5, 0.1, 2800)
    tg = make(hg, PROBLEMS[0])
    ch1.step(3, 0.5)
    b = hg.Batch([ch2, tg])
    ms = b.tune(0.5)
    assert ms > 0.0
    info = b.info()
    # one tile size per pass group, each from its candidate set
    assert info["tile_sweep"] in (256, 1024, 4096, 16384)
    assert info["tile_normal"] in (256, 1024, 4096, 16384) and info["tile_tan1"] in (256, 1024, 4096, 16384)
    assert info["tile_cells"] in (2048, 8192, 32768)
    # tuning left the states where they were
    assert ch2.stats()["step"] == 0
    b.step(3, 0.5)
    assert np.array_equal(ch1.get_state(), ch2.get_state())
    assert ch1.stats()["wall_shear"] == ch2.stats()["wall_shear"]
    # and against the oracle
    c = oracle.RefSolver((10, 16, 8), **kw)
    c.init_channel(0.5, 0.1, 2800)
    c.step(3, 0.5)
    q = c.get_state()
    scale = np.abs(q).reshape(5, -1).max(axis=1)
    scale[1:4] = scale[1:4].max()
    assert (np.abs(ch2.get_state() - q).reshape(5, -1).max(axis=1) / scale).max() < 1e-11
    b.close()


def test_batch_bad_problem_stops_alone(hg):
    good = make(hg, PROBLEMS[1])
    ref = make(hg, PROBLEMS[1])
    bad = make(hg, PROBLEMS[0])
    q = bad.get_state()
    q[4, 2, 3, 4] = np.nan
    bad.set_state(q)
    b = hg.Batch([bad, good])
    with pytest.raises(hg.HgksError) as e:
        b.step(2, 0.5)
    assert e.value.status == hg.HGKS_ERR_NONFINITE
    ref.step(2, 0.5)
    assert np.array_equal(good.get_state(), ref.get_state())
    assert bad.stats()["step"] == 0
    assert np.array_equal(bad.get_state(), q, equal_nan=True)
    b.close()


def test_batch_of_the_uneven_workload(hg):
    """Twelve problems of the seeded uneven-grid workload, FP64 and mixed
    interleaved, several steps with a tuned tile size."""
    from paper_2207_01173_gb300.workloads import batch_tgv_problems
    probs = [(n, Ma, Re, i % 2) for i, (n, Ma, Re) in enumerate(batch_tgv_problems(count=12))]
    single = [make(hg, p) for p in probs]
    for s in single:
        s.step(3, 0.5)
    batched = [make(hg, p) for p in probs]
    b = hg.Batch(batched)
    b.tune(0.5)
    b.step(3, 0.5)
    info = b.info()
    assert info["last_steps"] == 3 and info["last_ms"] > 0.0
    assert info["launches_per_step"] == 12 + 36 + 2
    for s1, s2 in zip(single, batched):
        assert np.array_equal(s1.get_state(), s2.get_state())
    b.close()


def test_batch_rejects_bad_arguments(hg):
    a = make(hg, PROBLEMS[4])
    with pytest.raises(hg.HgksError):
        hg.Batch([a, a])
    with pytest.raises(hg.HgksError):
        hg.Batch([])
