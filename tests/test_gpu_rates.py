"""Convergence rates of the GPU path by the power iteration of Section 5.1, against the
oracle's rates on the same operators and against what the paper reports:
  * with spatial coarsening the plain S smoother does not converge (rate ~ 1,
    Section 3.1) while the hybrid SAS converges (Section 4.1);
  * for large lambda the two-grid SAS rate is 2^-4 (Section 5.1);
  * two materials: raising nu on one subdomain (larger local lambda) does not slow
    the method down (Section 5.2, Table TestCase2)."""
import numpy as np
import pytest

import st_inputs
from helpers import oracle_mg, to_lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stmg():
    from paper_1911_09548_gb300._build import build
    build()
    import paper_1911_09548_gb300
    return paper_1911_09548_gb300


def rate_gpu(stmg, n, nsl, nu, sigma, T, N_t, p, iters, **opts):
    S = stmg.SpaceTimeSolver(n, nu, sigma, T, N_t, p, n_space_levels=nsl, **opts)
    x0 = st_inputs.random_iterate((N_t, p + 1, S.n_edge), 0)
    x = torch.from_numpy(to_lib(x0)).cuda()
    r, rates = S.convergence_rate(x, max_iter=iters)
    S.close()
    return r, rates, x0


def test_spatial_coarsening_needs_A(stmg):
    nf, N_t = 8, 64
    nu, sigma = st_inputs.materials(nf, "unit")
    T = N_t / 512.0
    r_S, rs_S, x0 = rate_gpu(stmg, nf, 2, nu, sigma, T, N_t, 0, 8, coarsen=2, max_levels=2, use_A=0)
    r_SAS, rs_SAS, _ = rate_gpu(stmg, nf, 2, nu, sigma, T, N_t, 0, 8, coarsen=2, max_levels=2)
    assert r_S > 0.9 and r_SAS < 0.5
    # the oracle, same operators and start: same per-cycle reductions
    sl, tl, mg = oracle_mg(nf, 2, nu, sigma, T, N_t, 0, coarsen=2, max_levels=2)
    _, rs_o = mg.convergence_rate(x0, max_iter=8)
    assert np.allclose(rs_SAS, rs_o, rtol=1e-9)


def test_high_lambda_rate_is_two_to_minus_four(stmg):
    nf, N_t = 8, 16
    nu, sigma = st_inputs.materials(nf, "unit")
    r, rates, _ = rate_gpu(stmg, nf, 1, nu, sigma, 64.0, N_t, 0, 12, coarsen=1, max_levels=2)
    assert abs(r - 2.0 ** -4) < 0.01


def test_two_materials_rate_does_not_degrade(stmg):
    """Table TestCase2 analogue on the Kuhn cube: nu_2 on the cubes with x > 1/2."""
    nf, N_t = 8, 32
    sigma = np.ones(6 * nf ** 3)
    c = np.arange(nf ** 3)
    right = np.repeat((c % nf) >= nf // 2, 6)
    T = N_t * 0.25 * 3.0 / nf ** 2        # min lambda = 0.25 at level 0 -> "Full" from the top
    out = []
    for nu2 in (1.0, 1e2, 1e4):
        nu = np.where(right, nu2, 1.0)
        r, _, _ = rate_gpu(stmg, nf, 2, nu, sigma, T, N_t, 0, 10, max_levels=2)
        out.append(r)
    assert out[0] < 0.5
    assert max(out[1:]) <= out[0] * 1.05     # raising the larger lambda only helps


def test_lambda_sweep_full_vs_semi_time(stmg):
    """The E1 analogue on the Kuhn cube (Section 5.1 experiment, power iteration of the
    two-grid method): Full tracks Semi-time for large lambda and deteriorates for small
    lambda; at lambda = 1/3 the GPU rates reproduce the oracle's per-cycle reductions."""
    nf, N_t = 8, 16
    nu, sigma = st_inputs.materials(nf, "unit")
    r = {}
    for tau in (2.0 ** -10, 2.0 ** -6, 1.0):
        for coarsen in (1, 2):
            r[tau, coarsen] = rate_gpu(stmg, nf, 2, nu, sigma, tau * N_t, N_t, 0, 15, coarsen=coarsen, max_levels=2)
    assert r[2.0 ** -10, 2][0] > 1.5 * r[2.0 ** -10, 1][0]
    assert abs(r[1.0, 2][0] / r[1.0, 1][0] - 1.0) < 0.1
    assert r[2.0 ** -6, 2][0] < 0.5
    _, rs_gpu, x0 = r[2.0 ** -6, 2]
    sl, tl, mg = oracle_mg(nf, 2, nu, sigma, 2.0 ** -6 * N_t, N_t, 0, coarsen=2, max_levels=2)
    _, rs_o = mg.convergence_rate(x0, max_iter=15)
    assert np.allclose(rs_gpu, rs_o, rtol=1e-9)


@pytest.mark.parametrize("pattern", ["SA", "SSASS"])
def test_smoother_orderings_match_oracle(stmg, pattern):
    """Rates of other hybrid-smoother orderings (Section 4) through the library equal the
    oracle's, cycle by cycle."""
    nf, N_t = 4, 16
    nu, sigma = st_inputs.materials(nf, "unit")
    r, rs_gpu, x0 = rate_gpu(stmg, nf, 1, nu, sigma, 16 / 512.0, N_t, 0, 10, coarsen=1, max_levels=2,
                             smoother=pattern)
    sl, tl, mg = oracle_mg(nf, 1, nu, sigma, 16 / 512.0, N_t, 0, coarsen=1, max_levels=2, pattern=pattern)
    _, rs_o = mg.convergence_rate(x0, max_iter=10)
    assert np.allclose(rs_gpu, rs_o, rtol=1e-9)


def test_neumann_rates(stmg):
    """The paper's rate experiments use Neumann conditions: with them, the large-lambda
    two-grid rate is again 2^-4, Full matches Semi-time there, and the GPU reproduces the
    oracle cycle by cycle."""
    nf, N_t = 8, 16
    nu, sigma = st_inputs.materials(nf, "unit")
    r1, rs1, x0 = rate_gpu(stmg, nf, 2, nu, sigma, float(N_t), N_t, 0, 12, coarsen=1, max_levels=2, bc=1)
    r2, _, _ = rate_gpu(stmg, nf, 2, nu, sigma, float(N_t), N_t, 0, 12, coarsen=2, max_levels=2, bc=1)
    assert abs(r1 - 2.0 ** -4) < 0.01
    assert abs(r2 / r1 - 1.0) < 0.1
    sl, tl, mg = oracle_mg(nf, 2, nu, sigma, float(N_t), N_t, 0, coarsen=1, max_levels=2, bc=1)
    _, rs_o = mg.convergence_rate(x0, max_iter=12)
    assert np.allclose(rs1, rs_o, rtol=1e-9)
