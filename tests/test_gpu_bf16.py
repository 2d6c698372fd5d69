"""BF16 slab solve on the tensor cores (slab_prec = 3, DG(1)).

The case has enough slabs (N_t = 1024, 8 column blocks of 128) that the deep
tree depths run the tcgen05 kernels and the top ones the split-K kernels.  The
BF16 factor is a preconditioner-quality inverse: its error is BF16-sized (checked
against the oracle's exact slab solve), and the V-cycle still converges to the
FP64 solution because the residual is FP64-accurate and the coarsest solve FP64
(the nodal correction runs in FP32)."""
import numpy as np
import pytest

import st_inputs
from helpers import from_lib, oracle_mg, rel, to_lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.spacetime import sequential_solve  # noqa: E402

N_CUBE, N_T = 8, 1024


@pytest.fixture(scope="module")
def setup():
    from paper_1911_09548_gb300._build import build
    build()
    import paper_1911_09548_gb300 as stmg
    nu, sigma = st_inputs.materials(N_CUBE, "two_material", 6)
    S = stmg.SpaceTimeSolver(N_CUBE, nu, sigma, 1.0, N_T, 1, slab_prec=3)
    sl, tl, mg = oracle_mg(N_CUBE, 1, nu, sigma, 1.0, N_T, 1, max_levels=2)
    yield stmg, S, sl, mg, nu, sigma
    S.close()


def test_bf16_slab_solve_accuracy(setup):
    stmg, S, sl, mg, nu, sigma = setup
    rng = np.random.default_rng(0)
    L = S.levels[0]
    ro = rng.normal(size=(L["N_t"], 2, L["n_edge"]))
    y = S.slab_solve(torch.from_numpy(to_lib(ro)).cuda(), level=0)
    torch.cuda.synchronize()
    err = rel(from_lib(y.cpu().numpy(), 2), mg.slabs[0].solve(ro))
    assert 1e-6 < err < 5e-2, err


def test_bf16_solve_reaches_fp64_solution(setup):
    stmg, S, sl, mg, nu, sigma = setup
    f = S.load(st_inputs.excitation(11))
    x = S.zeros()
    out = S.solve(f, x, rtol=1e-10, maxit=80)
    torch.cuda.synchronize()
    assert out["status"] == 0 and out["rel_res"] <= 1e-10, out
    xs = sequential_solve(mg.slabs[0], from_lib(f.cpu().numpy(), 2))
    assert rel(from_lib(x.cpu().numpy(), 2), xs) < 1e-8
