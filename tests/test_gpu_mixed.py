"""Mixed-precision slab solve (slab_prec = 1): the FP64 factor is rounded to FP32 and
applied in FP32; the residual is FP64-accurate (double-float) and the coarsest
solve FP64, so the V-cycle iteration refines to the FP64 solution (the nodal
correction, an inner part of the preconditioner, runs in FP32).  Checked against the oracle: the
FP32 slab apply to FP32 accuracy, and the final solution to 1e-8 relative."""
import numpy as np
import pytest

import st_inputs
from helpers import from_lib, oracle_mg, rel, to_lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.spacetime import sequential_solve  # noqa: E402

CASES = {
    "dg1": (8, 1, 1, 32, "two_material", dict(nu_pre=2, nu_post=2)),
    "dg0": (4, 1, 0, 16, "unit", dict(max_levels=2)),
}


@pytest.fixture(scope="module")
def stmg():
    from paper_1911_09548_gb300._build import build
    build()
    import paper_1911_09548_gb300
    return paper_1911_09548_gb300


def make(stmg, name, prec):
    n, nsl, p, N_t, mat, opts = CASES[name]
    nu, sigma = st_inputs.materials(n, mat, 4)
    S = stmg.SpaceTimeSolver(n, nu, sigma, 1.0, N_t, p, n_space_levels=nsl, slab_prec=prec, **opts)
    return S, nu, sigma


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_slab_solve_fp32_accuracy(stmg, name):
    S, nu, sigma = make(stmg, name, 1)
    n, nsl, p, N_t, mat, opts = CASES[name]
    sl, tl, mg = oracle_mg(n, nsl, nu, sigma, 1.0, N_t, p, max_levels=opts.get("max_levels", 0),
                           nu_pre=opts.get("nu_pre", 1), nu_post=opts.get("nu_post", 1))
    rng = np.random.default_rng(0)
    for lvl in range(S.n_levels):
        L = S.levels[lvl]
        ro = rng.normal(size=(L["N_t"], p + 1, L["n_edge"]))
        y = S.slab_solve(torch.from_numpy(to_lib(ro)).cuda(), level=lvl)
        torch.cuda.synchronize()
        err = rel(from_lib(y.cpu().numpy(), p + 1), mg.slabs[lvl].solve(ro))
        if lvl == S.n_levels - 1:
            assert err < 1e-12          # coarsest level stays FP64
        else:
            assert 1e-12 < err < 1e-4   # FP32 apply: FP32-level error, not FP64
    S.close()


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_solve_reaches_fp64_solution(stmg, name):
    n, nsl, p, N_t, mat, opts = CASES[name]
    res = {}
    for prec in (0, 1):
        S, nu, sigma = make(stmg, name, prec)
        f = S.load(st_inputs.excitation(9))
        x = S.zeros()
        out = S.solve(f, x, rtol=1e-10, maxit=60)
        torch.cuda.synchronize()
        res[prec] = (out, x.cpu().numpy(), f.cpu().numpy())
        S.close()
    sl, tl, mg = oracle_mg(n, nsl, nu, sigma, 1.0, N_t, p, max_levels=opts.get("max_levels", 0))
    xs = sequential_solve(mg.slabs[0], from_lib(res[0][2], p + 1))
    for prec in (0, 1):
        out, x, _ = res[prec]
        assert out["status"] == 0 and out["rel_res"] <= 1e-10
        assert rel(from_lib(x, p + 1), xs) < 1e-8
    # the FP32 slab apply costs at most a couple of extra V-cycles
    assert res[1][0]["iters"] <= res[0][0]["iters"] + 2


@pytest.mark.parametrize("slab_prec", [1, 3])
def test_fp32_residual_correction_form_reaches_fp64_solution(stmg, slab_prec):
    """residual_prec 1: every residual inside the V-cycle in FP32, each V-cycle in correction
    form around a double-float residual.  The iteration still reaches the FP64 solution (to
    1e-8 of the exact space-time solution) in at most two more V-cycles than the FP64 path."""
    n, nsl, p, N_t, mat, opts = CASES["dg1"]
    nu, sigma = st_inputs.materials(n, mat, 4)
    res = {}
    for prec, rp in ((0, -1), (slab_prec, 1)):
        S = stmg.SpaceTimeSolver(n, nu, sigma, 1.0, N_t, p, n_space_levels=nsl, slab_prec=prec, residual_prec=rp,
                                 **opts)
        f = S.load(st_inputs.excitation(9))
        x = S.zeros()
        out = S.solve(f, x, rtol=1e-10, maxit=60)
        torch.cuda.synchronize()
        res[rp] = (out, x.cpu().numpy(), f.cpu().numpy())
        S.close()
    sl, tl, mg = oracle_mg(n, nsl, nu, sigma, 1.0, N_t, p)
    xs = sequential_solve(mg.slabs[0], from_lib(res[-1][2], p + 1))
    out, x, _ = res[1]
    assert out["status"] == 0 and out["rel_res"] <= 1e-10, out
    assert rel(from_lib(x, p + 1), xs) < 1e-8
    assert out["iters"] <= res[-1][0]["iters"] + 2
