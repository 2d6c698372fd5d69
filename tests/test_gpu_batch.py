"""Batched solves (n_batch > 1): several excitations on one mesh and time grid in one
handle, every kernel running over all problems' slabs at once.  Each problem of the
batch must behave exactly as if it were solved alone (the history coupling and the
time transfers never cross problem boundaries), and reach the oracle's solution."""
import numpy as np
import pytest

import st_inputs
from helpers import from_lib, oracle_mg, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.spacetime import sequential_solve  # noqa: E402

CASES = {
    "dg1": (8, 1, 16, "two_material", dict(nu_pre=2, nu_post=2)),
    "dg0": (4, 0, 16, "unit", dict()),
    "dg1_df": (8, 1, 16, "two_material", dict(slab_prec=2)),
    "dg1_bf16": (8, 1, 64, "two_material", dict(slab_prec=3)),
}
NB = 3


@pytest.fixture(scope="module")
def stmg():
    from paper_1911_09548_gb300._build import build
    build()
    import paper_1911_09548_gb300
    return paper_1911_09548_gb300


def cols(x, b, N_t, q):
    """Problem b's block of a batched vector (rows = edges)."""
    return x[:, b * N_t * q:(b + 1) * N_t * q]


@pytest.mark.parametrize("name", list(CASES))
def test_batch_equals_separate_solves(stmg, name):
    n, p, N_t, mat, opts = CASES[name]
    q = p + 1
    nu, sigma = st_inputs.materials(n, mat, 2)
    SB = stmg.SpaceTimeSolver(n, nu, sigma, 1.0, N_t, p, n_batch=NB, **opts)
    fb = SB.zeros()
    for b in range(NB):
        SB.load(st_inputs.excitation(30 + b), f=fb, batch=b)
    xb = SB.zeros()
    for _ in range(2):
        SB.vcycle(fb, xb)
    torch.cuda.synchronize()
    XB, FB = xb.cpu().numpy(), fb.cpu().numpy()
    S1 = stmg.SpaceTimeSolver(n, nu, sigma, 1.0, N_t, p, **opts)
    for b in range(NB):
        f1 = S1.load(st_inputs.excitation(30 + b))
        assert np.array_equal(f1.cpu().numpy(), cols(FB, b, N_t, q))
        x1 = S1.zeros()
        for _ in range(2):
            S1.vcycle(f1, x1)
        torch.cuda.synchronize()
        # BF16: batched and single runs split K differently (different column-tile
        # counts), and a last-bit FP32 difference can flip a later BF16 rounding of an
        # intermediate (2^-8 relative), so they agree to BF16 level only
        tol = 2e-3 if opts.get("slab_prec", 0) == 3 else 1e-12
        assert rel(cols(XB, b, N_t, q), x1.cpu().numpy()) < tol
    S1.close()
    SB.close()


@pytest.mark.parametrize("name", ["dg1", "dg0"])
def test_batch_solve_reaches_time_stepping(stmg, name):
    n, p, N_t, mat, opts = CASES[name]
    q = p + 1
    nu, sigma = st_inputs.materials(n, mat, 2)
    SB = stmg.SpaceTimeSolver(n, nu, sigma, 1.0, N_t, p, n_batch=NB, **opts)
    fb = SB.zeros()
    for b in range(NB):
        SB.load(st_inputs.excitation(40 + b), f=fb, batch=b)
    xb = SB.zeros()
    out = SB.solve(fb, xb, rtol=1e-10, maxit=40)
    assert out["status"] == 0
    sl, tl, mg = oracle_mg(n, 1, nu, sigma, 1.0, N_t, p)
    XB, FB = xb.cpu().numpy(), fb.cpu().numpy()
    for b in range(NB):
        xs = sequential_solve(mg.slabs[0], from_lib(cols(FB, b, N_t, q).copy(), q))
        assert rel(from_lib(cols(XB, b, N_t, q).copy(), q), xs) < 1e-8
    SB.close()


def test_batch_rejects_hierarchy_without_single_slab(stmg):
    nu, sigma = st_inputs.materials(4, "unit")
    with pytest.raises(stmg.StMgError):
        stmg.SpaceTimeSolver(4, nu, sigma, 1.0, 16, 0, n_batch=2, max_levels=2)


# ---------------------------------------------------------------- ragged batches
# problems with different slab counts over one horizon T (N_t divided by powers of two),
# given in no particular order
RAGGED = [16, 4, 8, 16, 2, 8]


def _ragged(stmg, n, p, mat, batch_nt, **opts):
    nu, sigma = st_inputs.materials(n, mat, 3)
    S = stmg.SpaceTimeSolver(n, nu, sigma, 1.0, max(batch_nt), p, n_batch=len(batch_nt), batch_nt=batch_nt,
                             **opts)
    f = S.zeros()
    for b in range(len(batch_nt)):
        S.load(st_inputs.excitation(60 + b), f=f, batch=b)
    return S, f, nu, sigma


@pytest.mark.parametrize("p", [1, 0])
def test_ragged_batch_equals_separate_handles(stmg, p):
    """One V-cycle of a ragged batch advances every problem by exactly its own V-cycle: the
    problem's columns after three V-cycles equal those of a handle of its own (N_t = its
    slab count, the same horizon), and its load equals that handle's load."""
    n, mat = 4, "two_material"
    S, f, nu, sigma = _ragged(stmg, n, p, mat, RAGGED)
    assert S.level_shape() == (S.n_edge, sum(RAGGED) * (p + 1))
    x = S.zeros()
    for _ in range(3):
        S.vcycle(f, x)
    torch.cuda.synchronize()
    X, F = x.cpu().numpy(), f.cpu().numpy()
    for b, nt in enumerate(RAGGED):
        S1 = stmg.SpaceTimeSolver(n, nu, sigma, 1.0, nt, p)
        f1 = S1.load(st_inputs.excitation(60 + b))
        assert np.array_equal(f1.cpu().numpy(), F[:, S.problem_cols(b)]), b
        x1 = S1.zeros()
        for _ in range(3):
            S1.vcycle(f1, x1)
        torch.cuda.synchronize()
        # the same operations; a level's kernels may split their sums differently for
        # the batch's column count than for one problem's (rounding level)
        assert rel(X[:, S.problem_cols(b)], x1.cpu().numpy()) < 1e-12, b
        S1.close()
    S.close()


@pytest.mark.parametrize("opts", [dict(), dict(slab_prec=3, residual_prec=1)])
def test_ragged_batch_solve_reaches_time_stepping(stmg, opts):
    """A ragged batch solved to 1e-10: every problem reaches its own time stepping (the
    oracle's sequential solve with step T / N_t,b); FP64, and the BF16 tensor-core slab
    apply with FP32 residuals in correction form."""
    n, p, mat = 4, 1, "two_material"
    batch_nt = [32, 8, 16, 32]
    S, f, nu, sigma = _ragged(stmg, n, p, mat, batch_nt, **opts)
    x = S.zeros()
    out = S.solve(f, x, rtol=1e-10, maxit=60)
    torch.cuda.synchronize()
    assert out["status"] == 0 and out["rel_res"] <= 1e-10, out
    X, F = x.cpu().numpy(), f.cpu().numpy()
    for b, nt in enumerate(batch_nt):
        sl, tl, mg = oracle_mg(n, 1, nu, sigma, 1.0, nt, p, max_levels=1)
        xs = sequential_solve(mg.slabs[0], from_lib(F[:, S.problem_cols(b)].copy(), p + 1))
        assert rel(from_lib(X[:, S.problem_cols(b)].copy(), p + 1), xs) < 1e-8, b
    S.close()


def test_ragged_batch_rejects_bad_counts(stmg):
    nu, sigma = st_inputs.materials(4, "unit")
    for bad in ([16, 12], [16, 32], [16, 0]):
        with pytest.raises(stmg.StMgError):
            stmg.SpaceTimeSolver(4, nu, sigma, 1.0, 16, 1, n_batch=2, batch_nt=bad)
