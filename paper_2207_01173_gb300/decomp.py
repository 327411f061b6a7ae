"""Host-side logic of a slab decomposition along z across ranks.

The method shards naturally (Section 4.3 of the paper distributes the grid
over GPUs): each rank owns a contiguous range of z planes and, before each
stage of the two-stage step, needs three ghost planes from each neighbour,
because the normal reconstruction along z reads three cells on either side
of a face and the tangential reconstructions of x and y faces read two
planes up and down.  The time step is the minimum over all ranks of the CFL
limit, and the domain statistics are sums over ranks.

This module holds that logic and nothing of the method's arithmetic: the
partition of the planes, the periodic ring exchange of ghost planes through
torch.distributed (any backend; CPU tensors with gloo, device tensors with
NCCL), and the min / sum / max reductions.  A rank's local solve is whatever
engine the caller plugs in; the exchange expects the engine's padded state
layout [5][nz_local + 6][ny + 6][nx + 6], with the x and y ghosts of every
plane already filled, so that the planes it sends carry their x/y ghosts
along and the corners of the stencil are right.
"""
import numpy as np
import torch
import torch.distributed as dist

NG = 3  # ghost planes per side


def slab_sizes(nz, world, sizes=None):
    """Planes per rank: balanced (the first nz % world ranks take one more),
    or the explicit `sizes`.  Every rank needs at least NG planes, since its
    neighbours' ghost planes come from it alone."""
    if sizes is None:
        sizes = [nz // world + (1 if r < nz % world else 0) for r in range(world)]
    sizes = [int(v) for v in sizes]
    if len(sizes) != world or sum(sizes) != nz:
        raise ValueError("slab sizes %r do not split %d planes over %d ranks" % (sizes, nz, world))
    if min(sizes) < NG:
        raise ValueError("every slab needs at least %d planes, got %r" % (NG, sizes))
    return sizes


class ZSlabs:
    """This rank's slab of a z-periodic grid and its exchanges."""

    def __init__(self, nz, sizes=None, group=None, tagged=True):
        """tagged=False sends every message with one tag, so that the exchange
        relies on posting order alone, as it does under NCCL."""
        self.group = group
        self.tags = (0, 1) if tagged else (0, 0)
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.sizes = slab_sizes(nz, self.world, sizes)
        self.k0 = sum(self.sizes[:self.rank])
        self.nk = self.sizes[self.rank]
        self.left = (self.rank - 1) % self.world   # owns the planes below k0
        self.right = (self.rank + 1) % self.world  # owns the planes above k0 + nk
        self.bytes_sent = 0

    def local(self, q_global):
        """This rank's planes of a global [5][nz][ny][nx] array."""
        return q_global[:, self.k0:self.k0 + self.nk]

    def exchange(self, qpad):
        """Fill the NG ghost planes on both z sides of the padded local state
        qpad [5][nk+6][ny+6][nx+6] (numpy array or torch tensor, written in
        place) from the neighbours' boundary planes; periodic in z."""
        q = torch.from_numpy(qpad) if isinstance(qpad, np.ndarray) else qpad
        nk = self.nk
        bottom = q[:, NG:2 * NG].contiguous()          # -> left neighbour's top ghosts
        top = q[:, nk:nk + NG].contiguous()            # -> right neighbour's bottom ghosts
        if self.world == 1:
            q[:, :NG] = top
            q[:, nk + NG:] = bottom
            return
        lo = torch.empty_like(bottom)
        hi = torch.empty_like(top)
        # Every rank sends its bottom planes (tag 0) before its top planes
        # (tag 1), and receives its high ghosts (the right neighbour's bottom
        # planes) before its low ghosts (the left neighbour's top planes).
        # With two ranks the left and right neighbour are the same rank: gloo
        # tells the two messages apart by tag, NCCL (which ignores tags) by
        # their order, which this posting order makes agree.  One batch, so
        # that NCCL never blocks on a send whose receive is not yet posted.
        tb, tt = self.tags
        ops = [dist.P2POp(dist.isend, bottom, self.left, group=self.group, tag=tb),
               dist.P2POp(dist.isend, top, self.right, group=self.group, tag=tt),
               dist.P2POp(dist.irecv, hi, self.right, group=self.group, tag=tb),
               dist.P2POp(dist.irecv, lo, self.left, group=self.group, tag=tt)]
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        q[:, :NG] = lo
        q[:, nk + NG:] = hi
        self.bytes_sent += (bottom.numel() + top.numel()) * bottom.element_size()

    def min(self, x):
        """Global minimum of a scalar (the CFL limit)."""
        return reduce_scalar(x, dist.ReduceOp.MIN, self.group)

    def sum(self, values):
        """Global sums of a vector of partial sums (domain statistics)."""
        t = torch.tensor(np.asarray(values, dtype=np.float64))
        if self.world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t.numpy()


# ---------------------------------------------------------------------------
# several slabs of one domain in one process (one device): each slab is a
# solver handle with EXTERNAL z sides, and its halos travel device to device
# through caller-owned buffers.  This is the same exchange as ZSlabs's, run
# without a process group, so that the decomposition of the CUDA path can be
# checked on a single GPU against the undivided run.
# ---------------------------------------------------------------------------
def exchange_local_slabs(solvers, state, bufs):
    """Fill the z ghost layers of `state` on every slab from its neighbours
    (periodic ring in z).  solvers: slab handles ordered by z; bufs: per slab
    a pair (lo, hi) of device buffers of solver.halo_count() doubles each,
    given as integer device pointers."""
    k = len(solvers)
    for sv in solvers:
        sv.fill_ghosts(state)  # x / y ghosts first: they travel with the planes
    for sv, (lo, hi) in zip(solvers, bufs):
        sv.halo_get(state, 0, lo)
        sv.halo_get(state, 1, hi)
    for i, sv in enumerate(solvers):
        sv.halo_set(state, 0, bufs[(i - 1) % k][1])  # low ghosts: the lower slab's top layers
        sv.halo_set(state, 1, bufs[(i + 1) % k][0])  # high ghosts: the upper slab's bottom layers


def step_local_slabs(solvers, bufs, nsteps, cfl):
    """nsteps steps of the decomposed domain: the global CFL time step (the
    minimum over slabs), then per stage the halo exchange and the stage on
    every slab (Alg. 2).  Returns the time steps taken."""
    dts = []
    for _ in range(nsteps):
        dt = min(sv.compute_dt(cfl) for sv in solvers)
        for stage in (1, 2):
            exchange_local_slabs(solvers, stage - 1, bufs)
            for sv in solvers:
                sv.stage(stage, dt)
        dts.append(dt)
    return dts


def local_slab_stats(solvers, bufs, lz):
    """Diagnostics of the whole domain from its slabs: volume averages
    weighted by each slab's z length (lz: per slab), sums added, the Mach
    number maximised; the halos of the current state are exchanged first
    because the vorticity stencils reach into them."""
    exchange_local_slabs(solvers, 0, bufs)
    st = [sv.stats() for sv in solvers]
    L = float(sum(lz))
    out = dict(st[0])
    for k in ("Ek", "enstrophy", "eps_com", "wall_shear"):
        out[k] = sum(s[k] * l for s, l in zip(st, lz)) / L
    for k in ("mass", "energy"):
        out[k] = sum(s[k] for s in st)
    out["mom"] = [sum(s["mom"][c] for s in st) for c in range(3)]
    out["max_mach"] = max(s["max_mach"] for s in st)
    return out


def reduce_scalar(x, op, group=None, device="cpu"):
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op, group=group)
    return float(t.item())


def max_over_ranks(x, device="cpu"):
    """Maximum over ranks (the elapsed time of a multi-rank run)."""
    return reduce_scalar(x, dist.ReduceOp.MAX, device=device)
