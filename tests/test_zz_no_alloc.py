"""The allocation-free norm entry point (st_mg_norm2_noalloc) against the solver's own
norm (st_mg_residual with x = 0 returns ||f||), on two calls in a row through the C ABI.

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
    # two calls in a row with different inputs: the second must not see the first's scratch
    for call, seed in enumerate((7, 8)):
        f = S.load(st_inputs.excitation(seed)) * (1.0 + call)
        _, ref = S.residual(f, x0, want_norm=True)          # ||f - L 0|| = ||f||
        B.st_mg_norm2_noalloc(f, f.numel(), stream, out)
        torch.cuda.synchronize()
        got = out.item()
        assert np.isfinite(got) and abs(got - ref) <= 1e-13 * ref, (call, got, ref)
        # cross-check with an independent host norm
        assert abs(got - np.linalg.norm(f.cpu().numpy())) <= 1e-13 * ref
    # sizes beyond the fixed scratch are rejected with a clear error, before any launch
    with pytest.raises(B.StMgError, match="maximum"):
        B.st_mg_norm2_noalloc(f, 32768 * 4096 + 1, stream, out)
    S.close()
