"""Time-slab sharding of the all-at-once space-time system across ranks.

Section 2.1 splits the time axis into groups of consecutive slabs, one per process
group: the block-bidiagonal L couples a group only to the one before it (forward
communication of one slab), and the nodal correction's time integration Sigma_t /
L_t^{-1} (eq. AuxNodalSm) is a recurrence that runs through all groups.  Here each
rank owns one contiguous slab range (one library handle set up for that range: same
mesh, materials and tau) and two exchanges make its local steps equal to the
corresponding rows of the unsharded ones:

  residual          send the last slab of x to rank + 1, receive the halo from rank - 1,
                    then st_mg_residual_halo (slab 0 gets -(N_t (x) M) x_halo);
  time integration  every rank integrates its range from a zero carry, all ranks gather
                    the end states (one slab of nodal values each), each rank composes
                    its carry from those of the ranks before it (st_mg_time_carry:
                    an exclusive scan c_{k+1} = end_k + T c_k, T = -K_t^{-1} N_t) and
                    integrates again from it (st_mg_time_integrate_carry).

Block-Jacobi slab solves, G^T, the nodal solves and G w are local.  This module holds
only the rank arithmetic and the exchanges (torch.distributed point-to-point and
all_gather; NCCL between GPUs, gloo between CPU processes); the arithmetic of a range
is the `ops` object's: DeviceRangeOps calls the library.
"""
from __future__ import annotations


def slab_ranges(N_t: int, world: int):
    """Contiguous slab ranges (first slab, count) of `world` ranks: equal counts, which
    keeps every range's time coarsening local (pairs of slabs never straddle ranks)."""
    if world < 1 or N_t % world:
        raise ValueError("N_t must be a multiple of the number of ranks")
    c = N_t // world
    return [(r * c, c) for r in range(world)]


class TimeSlabShard:
    """One rank's view of the sharded time axis.  `dist` is torch.distributed (an
    initialised process group), `group` an optional sub-group."""

    def __init__(self, dist, N_t: int, group=None):
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group) if group is not None else dist.get_rank()
        self.world = dist.get_world_size(group) if group is not None else dist.get_world_size()
        self.slab0, self.count = slab_ranges(N_t, self.world)[self.rank]

    def _peer(self, r):
        return self.dist.get_global_rank(self.group, r) if self.group is not None else r

    def halo_exchange(self, last_slab):
        """Send this range's last slab to the next rank; return the previous rank's
        (None on rank 0).  `last_slab` is a contiguous tensor of one slab of rows."""
        import torch
        reqs = []
        halo = None
        if self.rank + 1 < self.world:
            reqs.append(self.dist.isend(last_slab, self._peer(self.rank + 1), group=self.group))
        if self.rank > 0:
            halo = torch.empty_like(last_slab)
            reqs.append(self.dist.irecv(halo, self._peer(self.rank - 1), group=self.group))
        for q in reqs:
            q.wait()
        return halo

    def gather_ends(self, end):
        """Every rank's end state, in rank (= time) order."""
        import torch
        ends = [torch.empty_like(end) for _ in range(self.world)]
        self.dist.all_gather(ends, end, group=self.group)
        return ends

    def residual(self, ops, f, x, level=0):
        """r = f - L x on this range, with the coupling to the range before it."""
        halo = self.halo_exchange(ops.last_slab(x, level, nodal=False))
        return ops.residual_halo(f, x, halo, level)

    def time_integrate(self, ops, z, level=0):
        """w = L_t^{-1} z on this range, continued from the state the earlier ranges end in."""
        w = ops.time_integrate(z, None, level)
        if self.world == 1:
            return w
        ends = self.gather_ends(ops.last_slab(w, level, nodal=True))
        if self.rank == 0:
            return w
        carry = ops.carry(ends[:self.rank], level)
        return ops.time_integrate(z, carry, level)


class DeviceRangeOps:
    """The arithmetic of one rank's slab range through the library (C ABI): `solver` is
    a SpaceTimeSolver set up for the range (its N_t = the range's slab count, T = that
    count times tau, n_batch 1)."""

    def __init__(self, solver):
        self.S = solver

    def last_slab(self, v, level, nodal):
        import torch
        from . import binding as B
        L = self.S.levels[level]
        rows = L["n_node"] if nodal else L["n_edge"]
        out = torch.empty((rows, self.S.q), dtype=torch.float64, device=v.device)
        B.st_mg_slab_copy(self.S.h, level, nodal, v, L["N_t"] - 1, out)
        return out

    def residual_halo(self, f, x, halo, level):
        from . import binding as B
        r = self.S.zeros(level)
        B.st_mg_residual_halo(self.S.h, level, f, x, halo, r)
        return r

    def time_integrate(self, z, carry, level):
        from . import binding as B
        w = self.S.zeros(level, nodal=True)
        B.st_mg_time_integrate_carry(self.S.h, level, z, carry, w)
        return w

    def carry(self, ends, level):
        import torch
        from . import binding as B
        e = torch.stack(ends).contiguous()
        c = torch.empty_like(ends[0])
        B.st_mg_time_carry(self.S.h, level, e, len(ends), c)
        return c
