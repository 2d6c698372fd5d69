"""Time-slab sharding kernels on one GPU: every rank's slab range as its own library
handle in one process (no rank waits on another: the exchanges are host-side copies
here), through the C ABI via DeviceRangeOps, against the unsharded handle.

  st_mg_residual_halo   range residual + the coupling of its first slab to the halo
  st_mg_slab_copy       the halo / end-state slab
  st_mg_time_carry      exclusive scan of the ranges' end states
  st_mg_time_integrate_carry

The range results must equal the matching slabs of the one-range results to 1e-14
(element-wise, relative to the largest entry): only the first slab of a later range
adds its coupling term in a separate pass."""
import numpy as np
import pytest

import st_inputs
from helpers import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_CUBE, N_T = 4, 16


@pytest.fixture(scope="module")
def stmg():
    from paper_1911_09548_gb300._build import build
    build()
    import paper_1911_09548_gb300
    return paper_1911_09548_gb300


@pytest.mark.parametrize("world,p", [(2, 0), (2, 1), (4, 1)])
def test_range_handles_reproduce_one_range(stmg, world, p):
    from paper_1911_09548_gb300.shard import DeviceRangeOps, slab_ranges
    nu, sigma = st_inputs.materials(N_CUBE, "two_material", 8)
    q = p + 1
    G = stmg.SpaceTimeSolver(N_CUBE, nu, sigma, 1.0, N_T, p)
    ranges = slab_ranges(N_T, world)
    H = [stmg.SpaceTimeSolver(N_CUBE, nu, sigma, c / N_T, c, p) for _, c in ranges]
    ops = [DeviceRangeOps(h) for h in H]
    rng = np.random.default_rng(7)
    f = torch.from_numpy(rng.normal(size=G.level_shape())).cuda()
    x = torch.from_numpy(rng.normal(size=G.level_shape())).cuda()
    z = torch.from_numpy(rng.normal(size=G.level_shape(nodal=True))).cuda()
    r_all = G.residual(f, x)
    w_all = G.time_integrate(z)

    def cols(v, k):
        a, c = ranges[k]
        return v[:, a * q:(a + c) * q].contiguous()

    # residual: range k takes the last slab of range k - 1 as its halo
    for k in range(world):
        halo = ops[k - 1].last_slab(cols(x, k - 1), 0, nodal=False) if k > 0 else None
        r_k = ops[k].residual_halo(cols(f, k), cols(x, k), halo, 0)
        torch.cuda.synchronize()
        assert rel(r_k.cpu().numpy(), cols(r_all, k).cpu().numpy()) <= 1e-14, k
    # time integration: zero-carry pass, end states gathered, carry composed, second pass
    w0 = [ops[k].time_integrate(cols(z, k), None, 0) for k in range(world)]
    ends = [ops[k].last_slab(w0[k], 0, nodal=True) for k in range(world)]
    for k in range(world):
        w_k = ops[k].time_integrate(cols(z, k), ops[k].carry(ends[:k], 0), 0) if k > 0 else w0[k]
        torch.cuda.synchronize()
        assert rel(w_k.cpu().numpy(), cols(w_all, k).cpu().numpy()) <= 1e-14, k
        if k > 0:   # the carry matters
            assert rel(w0[k].cpu().numpy(), cols(w_all, k).cpu().numpy()) > 1e-3
    # no preceding range: the carry is zero
    c0 = torch.full_like(ends[0], float("nan"))
    stmg.st_mg_time_carry(H[0].h, 0, None, 0, c0)
    torch.cuda.synchronize()
    assert torch.all(c0 == 0)
    for h in H:
        h.close()
    G.close()
