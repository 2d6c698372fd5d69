"""Time-slab sharding (paper_1911_09548_gb300/shard.py) on two and four gloo ranks on the
CPU, against the unsharded oracle.

Each rank owns a contiguous range of the slabs.  The exchange logic under test is the
module's own (halo send/receive of one slab of x, all_gather of one slab of nodal end
states and the carry composition order); the arithmetic of a range is supplied by the
test from the oracle's operators (the library's kernels for it need a GPU and are
checked on one GPU, both ranges in one process, in test_gpu_shard.py).  The residual and
the time integration L_t^{-1} of every range must equal the matching slabs of the
single-range oracle (Section 2.1's block-bidiagonal L; eq. AuxNodalSm's Sigma_t)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

N_CUBE, N_T = 3, 8


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleRangeOps:
    """Arithmetic of one slab range from the oracle's operators (test infrastructure).
    Vectors are torch CPU tensors in the oracle's layout (slabs, q, rows)."""

    def __init__(self, space, p, tau):
        from oracle.timeblocks import time_blocks
        self.space, self.p = space, p
        self.Kt, self.Mt, self.Nt = time_blocks(p, tau)

    def last_slab(self, v, level, nodal):
        return v[-1].clone().contiguous()

    def residual_halo(self, f, x, halo, level):
        from oracle.spacetime import residual
        r = residual(self.space, self.Kt, self.Mt, self.Nt, f.numpy(), x.numpy())
        if halo is not None:
            # the coupling block of L below the diagonal, applied to the previous slab
            Mh = (self.space.M @ halo.numpy().T).T          # (q, N_e)
            r[0] -= self.Nt @ Mh
        return torch.from_numpy(r)

    def time_integrate(self, z, carry, level):
        Ktinv = np.linalg.inv(self.Kt)
        zn = z.numpy()
        w = np.zeros_like(zn)
        prev = np.zeros_like(zn[0]) if carry is None else carry.numpy()
        for n in range(zn.shape[0]):
            w[n] = Ktinv @ (zn[n] - self.Nt @ prev)
            prev = w[n]
        return torch.from_numpy(w)

    def carry(self, ends, level):
        # c_{k+1} = end_k + T^{len_k} c_k, T = -K_t^{-1} N_t, with the general matrix power
        T = -np.linalg.solve(self.Kt, self.Nt)
        c = np.zeros_like(ends[0].numpy())
        for e in ends:
            c = e.numpy() + np.linalg.matrix_power(T, N_T // self.world) @ c
        return torch.from_numpy(c)


def _rank_main(rank, world, port, p, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import st_inputs
        from oracle.spacetime import build_space_hierarchy, residual, time_integrate
        from oracle.timeblocks import time_blocks
        from paper_1911_09548_gb300.shard import TimeSlabShard

        nu, sigma = st_inputs.materials(N_CUBE, "two_material", 3)
        space = build_space_hierarchy(N_CUBE, 1, nu, sigma)[0]
        tau = 1.0 / N_T
        qd = p + 1
        rng = np.random.Generator(np.random.PCG64(42))      # the same global data on every rank
        f = rng.normal(size=(N_T, qd, space.ne))
        x = rng.normal(size=(N_T, qd, space.ne))
        z = rng.normal(size=(N_T, qd, space.nn))
        Kt, Mt, Nt = time_blocks(p, tau)
        r_all = residual(space, Kt, Mt, Nt, f, x)
        w_all = time_integrate(Kt, Nt, z)

        sh = TimeSlabShard(dist, N_T)
        ops = OracleRangeOps(space, p, tau)
        ops.world = world
        a, c = sh.slab0, sh.count
        sl = slice(a, a + c)
        r = sh.residual(ops, torch.from_numpy(f[sl].copy()), torch.from_numpy(x[sl].copy()))
        w = sh.time_integrate(ops, torch.from_numpy(z[sl].copy()))
        er = np.max(np.abs(r.numpy() - r_all[sl])) / np.max(np.abs(r_all))
        ew = np.max(np.abs(w.numpy() - w_all[sl])) / np.max(np.abs(w_all))
        # without the exchanges a range other than the first would be wrong
        r0 = ops.residual_halo(torch.from_numpy(f[sl].copy()), torch.from_numpy(x[sl].copy()), None, 0)
        w0 = ops.time_integrate(torch.from_numpy(z[sl].copy()), None, 0)
        miss = (np.max(np.abs(r0.numpy() - r_all[sl])) + np.max(np.abs(w0.numpy() - w_all[sl]))) if a > 0 else 1.0
        q.put((rank, a, c, er, ew, miss))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,p", [(2, 0), (2, 1), (4, 1)])
def test_sharded_residual_and_time_integration_match_one_range(world, p):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, p, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert [o[1] for o in out] == [r * (N_T // world) for r in range(world)]
    for rank, a, c, er, ew, miss in out:
        assert er <= 1e-14 and ew <= 1e-14, (rank, er, ew)
        assert miss > 1e-3, rank          # the halo and the carry matter on every later range


def test_slab_ranges():
    from paper_1911_09548_gb300.shard import slab_ranges
    assert slab_ranges(8, 2) == [(0, 4), (4, 4)]
    assert slab_ranges(256, 4)[3] == (192, 64)
    with pytest.raises(ValueError):
        slab_ranges(10, 4)
