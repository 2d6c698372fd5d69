"""Parity at the benchmark's full size (Kuhn 16^3, two materials, T = 1, N_t = 256, DG(1),
V(2,2), tiled/split-K thresholds autotuned as in bench.py) where the oracle cannot run
V-cycles: every quantity below is recomputed by the oracle's own operators (its sparse
M_sigma, K_nu and DG(1) time blocks), not taken from the library.

  * the space-time residual r = f - L x on all 13.5 M DoFs (1e-13);
  * the finest-level slab solve, through the residual of the slab block system
    K_t (x) M + M_t (x) K that the oracle assembles (1e-12);
  * the bench's three solve paths (FP64, FP32 factor, BF16 tensor cores) to a 1e-8
    relative residual: the oracle's FP64 residual of each final iterate is <= 1e-8 and
    the mixed-precision solutions agree with the FP64 one to 1e-8."""
import numpy as np
import pytest

import st_inputs
from helpers import from_lib, rel, to_lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.load import spacetime_load  # noqa: E402
from oracle.spacetime import apply_L, build_space_hierarchy  # noqa: E402
from oracle.timeblocks import time_blocks  # noqa: E402

N, N_T, P = 16, 256, 1


@pytest.fixture(scope="module")
def setup():
    from paper_1911_09548_gb300._build import build
    build()
    import paper_1911_09548_gb300 as stmg
    nu, sigma = st_inputs.materials(N, "two_material", 0)
    sl = build_space_hierarchy(N, 1, nu, sigma)
    stream = torch.cuda.Stream()
    return stmg, nu, sigma, sl[0], stream


def solver(setup, **opts):
    stmg, nu, sigma, _, stream = setup
    return stmg.SpaceTimeSolver(N, nu, sigma, 1.0, N_T, P, nu_pre=2, nu_post=2, stream=stream.cuda_stream,
                                autotune=1, **opts)


def test_fullsize_residual(setup):
    _, _, _, space, _ = setup
    S = solver(setup)
    Kt, Mt, Nt = time_blocks(P, 1.0 / N_T)
    x = st_inputs.random_iterate((N_T, P + 1, space.ne), 3)
    f = spacetime_load(space.mesh, st_inputs.excitation(0), P, N_T, 1.0)
    r = S.residual(torch.from_numpy(to_lib(f)).cuda(), torch.from_numpy(to_lib(x)).cuda())
    torch.cuda.synchronize()
    ro = f - apply_L(space, Kt, Mt, Nt, x)
    assert rel(from_lib(r.cpu().numpy(), P + 1), ro) < 1e-13
    S.close()


def test_fullsize_slab_solve(setup):
    _, _, _, space, _ = setup
    S = solver(setup)
    Kt, Mt, _ = time_blocks(P, 1.0 / N_T)
    r = st_inputs.random_iterate((N_T, P + 1, space.ne), 4) - 0.5
    y = S.slab_solve(torch.from_numpy(to_lib(r)).cuda())
    torch.cuda.synchronize()
    Y = from_lib(y.cpu().numpy(), P + 1)                 # (N_t, 2, ne)
    X = Y.reshape(-1, space.ne).T
    MY = (space.M @ X).T.reshape(Y.shape)
    KY = (space.K @ X).T.reshape(Y.shape)
    AY = np.einsum("ij,nje->nie", Kt, MY) + np.einsum("ij,nje->nie", Mt, KY)
    assert rel(AY, r) < 1e-12
    S.close()


def test_fullsize_solves_reach_oracle_residual(setup):
    _, _, _, space, _ = setup
    Kt, Mt, Nt = time_blocks(P, 1.0 / N_T)
    exc = st_inputs.excitation(100)
    fo = spacetime_load(space.mesh, exc, P, N_T, 1.0)
    sols = {}
    for prec in (0, 1, 3):
        S = solver(setup, slab_prec=prec)
        f = S.load(exc)
        x = S.zeros()
        out = S.solve(f, x, rtol=1e-8, maxit=60)
        torch.cuda.synchronize()
        assert out["status"] == 0 and out["iters"] <= 10, (prec, out)
        X = from_lib(x.cpu().numpy(), P + 1)
        res = np.linalg.norm(fo - apply_L(space, Kt, Mt, Nt, X)) / np.linalg.norm(fo)
        assert res <= 1.0001e-8, (prec, res)
        sols[prec] = X
        S.close()
    for prec in (1, 3):
        assert rel(sols[prec], sols[0]) < 1e-8, prec
