"""Rank body of the slab-decomposition tests: each process owns a z slab,
advances it with the oracle through the ghost-plane exchange and the global
CFL minimum of paper_2207_01173_gb300.decomp, and writes its slab to disk."""
import os

import numpy as np

CASES = {
    # name: (grid, slab sizes, solver kwargs, init, steps)
    "tgv_uneven": ((8, 6, 12), (8, 4), dict(visc=(1, 1.0 / 1600, 1.0 / (1.4 * 0.01), 0.7), Pr=0.72),
                   ("tgv", 0.1), 3),
    "tgv_three": ((6, 5, 12), (3, 5, 4), dict(visc=(1, 1.0 / 1600, 1.0 / (1.4 * 0.01), 0.7), Pr=0.72),
                  ("tgv", 0.1), 2),
    # one tag for every message: the exchange must match by posting order
    # alone, as under NCCL (two ranks: left and right neighbour coincide)
    "tgv_untagged": ((6, 5, 8), (4, 4), dict(visc=(1, 1.0 / 1600, 1.0 / (1.4 * 0.01), 0.7), Pr=0.72),
                     ("tgv", 0.1), 2),
    "channel": ((6, 16, 8), (4, 4), dict(lengths=(2.0, 2.0, 1.0), origin=(0.0, -1.0, 0.0), y_stretch_b=1.5,
                                         visc=(1, 1.0 / 2800, 1.0 / (1.4 * 0.25), 0.7), Pr=0.72,
                                         bc_lo=(0, 1, 0), bc_hi=(0, 1, 0), T_wall=1.0 / (1.4 * 0.25),
                                         body_force=(0.05, 0.0, 0.0)),
                ("channel", 0.5), 3),
}


def global_solver(ref, case, lengths_override=None, nz=None, bc_z=None):
    n, _, kw, _, _ = CASES[case]
    kw = dict(kw)
    if lengths_override is not None:
        kw["lengths"] = lengths_override
    if bc_z is not None:
        lo, hi = list(kw.get("bc_lo", (0, 0, 0))), list(kw.get("bc_hi", (0, 0, 0)))
        lo[2] = hi[2] = bc_z
        kw["bc_lo"], kw["bc_hi"] = tuple(lo), tuple(hi)
    return ref.RefSolver((n[0], n[1], nz if nz is not None else n[2]), **kw)


def initial_state(ref, case):
    s = global_solver(ref, case)
    kind, a = CASES[case][3]
    if kind == "tgv":
        s.init_tgv(a, 1.0, 1.0)
    else:
        s.init_channel(a, 0.1, 2800)
    q = s.get_state()
    s.close()
    return q


def rank_main(rank, world, port, case, outdir):
    os.environ.setdefault("OMP_NUM_THREADS", "2")
    import torch.distributed as dist

    from oracle import ref
    from paper_2207_01173_gb300.decomp import NG, ZSlabs, max_over_ranks

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        n, sizes, kw, _, steps = CASES[case]
        slabs = ZSlabs(n[2], sizes=sizes if world == len(sizes) else None, tagged=(case != "tgv_untagged"))
        lengths = kw.get("lengths", (2 * np.pi,) * 3)
        dz = lengths[2] / n[2]
        # the slab's length: nk whole cells of the global size
        local = global_solver(ref, case, lengths_override=(lengths[0], lengths[1], dz * slabs.nk), nz=slabs.nk,
                              bc_z=ref.BC_EXTERNAL)
        assert (dz * slabs.nk) / slabs.nk == dz  # same cell size as the global grid
        local.set_state(np.ascontiguousarray(slabs.local(initial_state(ref, case))))
        local.set_hooks(halo=slabs.exchange, dtmin=slabs.min)
        local.step(steps, 0.5)
        q = local.get_state()
        st = local.stats()
        sums = slabs.sum([st["mass"], st["energy"]])
        slowest = max_over_ranks(1.5 + rank)
        np.savez(os.path.join(outdir, "rank%d.npz" % rank), q=q, k0=slabs.k0, nk=slabs.nk, t=st["t"],
                 sums=sums, slowest=slowest, sent=slabs.bytes_sent, planes=NG)
        local.close()
    finally:
        dist.destroy_process_group()
