"""The allocation-free norm entry point (st_mg_norm2_noalloc) against the solver's own
norm (st_mg_residual with x = 0 returns ||f||) and an independent host norm, through
the C ABI, on calls in a row that share the entry point's fixed scratch array.

The entry point exists for callers that cannot allocate device memory where they
need the norm: it keeps its scratch in a fixed device array instead of allocating.
Collected last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

import st_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_norm2_noalloc_matches_solver_norm_twice():
    from paper_1911_09548_gb300._build import build
    build()
    import paper_1911_09548_gb300 as stmg
    from paper_1911_09548_gb300 import binding as B

    nu, sigma = st_inputs.materials(8, "two_material", 2)
    S = stmg.SpaceTimeSolver(8, nu, sigma, 1.0, 20, 1)
    stream = torch.cuda.current_stream().cuda_stream
    x0 = S.zeros()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    # first call: the whole vector (121280 doubles: 30 partial sums, the last one ragged)
    f = S.load(st_inputs.excitation(7))
    _, ref = S.residual(f, x0, want_norm=True)          # ||f - L 0|| = ||f||
    B.st_mg_norm2_noalloc(f, f.numel(), stream, out)
    torch.cuda.synchronize()
    got = out.item()
    # equal to the solver's norm up to rounding (the two reductions sum in different orders)
    assert np.isfinite(got) and abs(got - ref) <= 1e-13 * ref, (got, ref)
    assert abs(got - np.linalg.norm(f.cpu().numpy())) <= 1e-13 * ref
    # second call right after: a different vector with fewer elements, not a multiple of
    # the 4096 elements per partial sum, so most scratch entries of the first call are
    # left over and must not enter the result
    g = (S.load(st_inputs.excitation(8)) * 2.0).reshape(-1)
    m = g.numel() // 3 + 5
    B.st_mg_norm2_noalloc(g, m, stream, out)
    torch.cuda.synchronize()
    got2 = out.item()
    ref2 = float(np.linalg.norm(g[:m].cpu().numpy()))
    assert np.isfinite(got2) and abs(got2 - ref2) <= 1e-13 * ref2, (got2, ref2)
    # an empty vector has norm exactly 0 (only the final sum runs, over no partials)
    out.fill_(float("nan"))
    B.st_mg_norm2_noalloc(g, 0, stream, out)
    torch.cuda.synchronize()
    assert out.item() == 0.0
    # sizes beyond the fixed scratch are rejected with a clear error, before any launch
    with pytest.raises(B.StMgError, match="maximum"):
        B.st_mg_norm2_noalloc(f, 32768 * 4096 + 1, stream, out)
    S.close()
