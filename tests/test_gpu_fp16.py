"""FP16 slab solve on the tensor cores (slab_prec = 4, DG(1)).

The same tcgen05 kernels as the BF16 path with FP16 operands (11 significant bits,
5 exponent bits).  Every right-hand-side column of a slab solve is scaled by a power of
two into [1, 2) before the solve and back after it, so the residuals of a converging
iteration (they shrink by many orders over a solve) keep FP16's precision instead of
falling below its range.  Checks of the slab solve (eq. StandardSmoother's slab inverse):

  * differential: the tensor-core kernels against the same FP16 factor on the CUDA cores
    with the same operand rounding (st_mg_set_tc_mode 1), element by element, depths
    forced tiled and forced split-K;
  * against the oracle's exact slab solve, to a bound set by FP16 rounding;
  * scale invariance: a right-hand side 2^-40 (about 1e-12) times as large gives the
    same solution times 2^-40, bit for bit (without the column scaling it would flush to
    zero in FP16);
  * the V-cycle iteration reaches the exact space-time solution (FP64-accurate residual,
    FP64 coarsest solve)."""
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
    S = stmg.SpaceTimeSolver(N_CUBE, nu, sigma, 1.0, N_T, 1, slab_prec=4)
    sl, tl, mg = oracle_mg(N_CUBE, 1, nu, sigma, 1.0, N_T, 1, max_levels=2)
    yield stmg, S, sl, mg, nu, sigma
    S.close()


def _solve(stmg, S, r, level):
    y = S.slab_solve(r, level=level)
    torch.cuda.synchronize()
    stmg.st_mg_check(S.h)
    return y.cpu().numpy()


@pytest.mark.parametrize("level", [0, 2])
def test_fp16_tensor_cores_match_cuda_core_reference(setup, level):
    stmg, S, sl, mg, nu, sigma = setup
    rng = np.random.default_rng(11 + level)
    L = S.levels[level]
    ro = rng.normal(size=(L["N_t"], 2, L["n_edge"]))
    r = torch.from_numpy(to_lib(ro)).cuda()
    w0 = stmg.st_mg_split_waves(S.h, level)
    try:
        stmg.st_mg_set_tc_mode(S.h, level, 1)
        y_ref = _solve(stmg, S, r, level)
        stmg.st_mg_set_tc_mode(S.h, level, 0)
        for waves in (0, 64):
            stmg.st_mg_set_split_waves(S.h, level, waves)
            y_tc = _solve(stmg, S, r, level)
            d = rel(y_tc, y_ref)
            print(f"fp16 tc vs cuda-core reference, level {level}, split waves {waves}: {d:.3e}")
            # an FP16 rounding flip of a gathered operand is 2^-11 relative (8x less than BF16's)
            assert d < 5e-4, (level, waves, d)
    finally:
        stmg.st_mg_set_tc_mode(S.h, level, 0)
        stmg.st_mg_set_split_waves(S.h, level, w0)



@pytest.mark.parametrize("level", [0, 2])
def test_fp16_persistent_tiled_depths_match_per_tile_kernel(setup, level):
    """Tensor-core mode 0 (default): every tiled depth runs as one persistent CTA per SM
    that walks the depth's (row tile, column block) tasks with a bulk-copy ring that
    never drains and two TMEM accumulators; mode 2 runs one CTA per tile.  The MMAs of a task are issued in the same order on the
    same operand tiles as in the one-CTA-per-tile kernel, and the epilogue does the same
    arithmetic, so with every depth forced tiled the two solves agree bit for bit; both
    stay within the operand-rounding bound of the CUDA-core reference."""
    stmg, S, *_ = setup
    rng = np.random.default_rng(21 + level)
    L = S.levels[level]
    ro = rng.normal(size=(L["N_t"], 2, L["n_edge"]))
    r = torch.from_numpy(to_lib(ro)).cuda()
    w0 = stmg.st_mg_split_waves(S.h, level)
    try:
        stmg.st_mg_set_tc_mode(S.h, level, 1)
        y_ref = _solve(stmg, S, r, level)
        stmg.st_mg_set_split_waves(S.h, level, 0)
        stmg.st_mg_set_tc_mode(S.h, level, 2)
        y_tile = _solve(stmg, S, r, level)
        stmg.st_mg_set_tc_mode(S.h, level, 0)
        y_pers = _solve(stmg, S, r, level)
        d = rel(y_pers, y_ref)
        print(f"fp16 persistent tiled vs cuda-core reference, level {level}: {d:.3e}")
        neq = y_pers != y_tile
        assert not neq.any(), (int(neq.sum()), int(neq.any(axis=1).sum()), int(neq.any(axis=0).sum()),
                               rel(y_pers, y_tile))
        assert d < 5e-4, (level, d)
        # the default split threshold: split-K depths unchanged, tiled ones persistent
        stmg.st_mg_set_split_waves(S.h, level, w0)
        y_mix = _solve(stmg, S, r, level)
        assert rel(y_mix, y_ref) < 5e-4
    finally:
        stmg.st_mg_set_tc_mode(S.h, level, 0)
        stmg.st_mg_set_split_waves(S.h, level, w0)

def test_fp16_slab_solve_accuracy_and_scale_invariance(setup):
    stmg, S, sl, mg, nu, sigma = setup
    rng = np.random.default_rng(0)
    L = S.levels[0]
    ro = rng.normal(size=(L["N_t"], 2, L["n_edge"]))
    exact = mg.slabs[0].solve(ro)
    y = _solve(stmg, S, torch.from_numpy(to_lib(ro)).cuda(), 0)
    err = rel(from_lib(y, 2), exact)
    print(f"fp16 slab solve vs oracle exact slab solve: {err:.3e}")
    # FP16 keeps 11 significant bits (unit roundoff 2^-12 = 2.4e-4)
    assert 1e-7 < err < 3e-3, err
    # the same right-hand side 2^-40 times as large (a late residual of a solve): every
    # column is scaled back into [1, 2) by a power of two, so the FP16 computation is the
    # same and the solution is y 2^-40 exactly
    ys = _solve(stmg, S, torch.from_numpy(to_lib(ro * 2.0 ** -40)).cuda(), 0)
    assert np.array_equal(ys * 2.0 ** 40, y)


def test_fp16_solve_reaches_fp64_solution(setup):
    stmg, S, sl, mg, nu, sigma = setup
    f = S.load(st_inputs.excitation(11))
    x = S.zeros()
    out = S.solve(f, x, rtol=1e-10, maxit=80)
    torch.cuda.synchronize()
    assert out["status"] == 0 and out["rel_res"] <= 1e-10, out
    xs = sequential_solve(mg.slabs[0], from_lib(f.cpu().numpy(), 2))
    assert rel(from_lib(x.cpu().numpy(), 2), xs) < 1e-8
