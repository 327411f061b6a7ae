"""The serving loop on the GPU: requests that arrive while others run join
the running batch, and each result is the same alone and in the mix (bit
for bit, since a batch reproduces single-problem steps exactly)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2207_01173_gb300 import hgks
    return hgks


def small_stream():
    rng = np.random.default_rng(5)
    out = []
    t = 0.0
    for i in range(10):
        t += float(rng.exponential(0.02))
        if i % 3 == 2:
            n = int(rng.choice([12, 16]))
            out.append(dict(id=i, t=t, kind="channel", n=(n, n, n), Ma=0.5, Re=2800.0, seed=2800 + i,
                            steps=int(rng.integers(3, 10))))
        else:
            n = int(rng.choice([12, 16, 20]))
            out.append(dict(id=i, t=t, kind="tgv", n=(n, n, n), Ma=0.1, Re=1600.0, steps=int(rng.integers(3, 10))))
    return out


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_serve_results_same_alone_and_in_the_mix(hg, precision):
    from paper_2207_01173_gb300.serve import CudaEngine, Server
    prec = hg.MIXED if precision == "mixed" else hg.FP64
    reqs = small_stream()
    eng = CudaEngine(precision=prec, cfl=0.5)
    # room for about three of the larger problems at once
    budget = 3 * hg.footprint_bytes((20, 20, 20), prec)
    srv = Server(eng, budget, max_chunk=3, keep_state=True)
    res, summ = srv.run(reqs)
    eng.close()
    assert summ["done"] == len(reqs), summ
    assert summ["peak_bytes"] <= budget
    assert summ["mean_concurrency"] > 1.0 and eng.rebuilds > 1
    for r in reqs:
        alone = eng.create(r)
        alone.step(r["steps"], 0.5)
        out = res[r["id"]]
        assert np.array_equal(alone.get_state(), out["state"]), r
        s = alone.stats()
        assert s["step"] == out["stats"]["step"] == r["steps"]
        assert s["Ek"] == out["stats"]["Ek"] and s["t"] == out["stats"]["t"]
        alone.close()
