"""Slab decomposition along z emulated with CPU ranks (gloo): two processes,
each advancing its slab with the oracle, exchanging three ghost planes per
side before every stage and taking the global CFL minimum, must reproduce
the undivided oracle run bit for bit.  Also the partition rules and the
max-over-ranks timing reduction used by the benchmark."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

from paper_2207_01173_gb300.decomp import NG, slab_sizes
from tests.decomp_ranks import CASES, global_solver, initial_state, rank_main


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def run_ranks(case, world, tmp_path):
    from oracle.build import build_oracle
    build_oracle()  # once, before the ranks load it
    ctx = mp.get_context("spawn")
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, world, port, case, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0] * world, codes
    return [dict(np.load(os.path.join(tmp_path, "rank%d.npz" % r))) for r in range(world)]


def test_slab_sizes():
    assert slab_sizes(12, 2) == [6, 6]
    assert slab_sizes(13, 3) == [5, 4, 4]
    assert slab_sizes(12, 2, (8, 4)) == [8, 4]
    with pytest.raises(ValueError):
        slab_sizes(12, 2, (10, 2))  # a slab thinner than the ghost width
    with pytest.raises(ValueError):
        slab_sizes(12, 2, (8, 5))


@pytest.mark.parametrize("case", sorted(CASES))
def test_split_equals_unsplit(case, oracle, tmp_path):
    world = len(CASES[case][1])  # two ranks, or three (distinct left and right neighbours)
    res = run_ranks(case, world, tmp_path)
    n, sizes, _, _, steps = CASES[case]
    whole = global_solver(oracle, case)
    whole.set_state(initial_state(oracle, case))
    whole.step(steps, 0.5)
    q = whole.get_state()
    st = whole.stats()
    split = np.concatenate([r["q"] for r in sorted(res, key=lambda r: int(r["k0"]))], axis=1)
    assert [int(r["nk"]) for r in res] == list(sizes)
    assert np.array_equal(split, q)  # bit for bit
    for r in res:
        assert float(r["t"]) == st["t"]
        assert float(r["slowest"]) == 1.5 + (world - 1)  # max of 1.5 + rank
        np.testing.assert_allclose(r["sums"], [st["mass"], st["energy"]], rtol=1e-13)
        # two exchanges per step (one per stage) plus one for the statistics,
        # NG planes of the padded x-y plane each way, 5 components
        plane = (n[0] + 2 * NG) * (n[1] + 2 * NG) * 5 * 8
        assert int(r["sent"]) == (2 * steps + 1) * 2 * NG * plane
