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


def reduce_scalar(x, op, group=None, device="cpu"):
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op, group=group)
    return float(t.item())


def max_over_ranks(x, device="cpu"):
    """Maximum over ranks (the elapsed time of a multi-rank run)."""
    return reduce_scalar(x, dist.ReduceOp.MAX, device=device)
