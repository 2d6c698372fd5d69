"""GPU parity on general start meshes (Section 5.1: the spatial hierarchy by uniform
refinement of a coarse tetrahedral mesh) against the oracle's independent construction:
load, residual, slab solve and V-cycle iterates (1e-11 per iterate), on a refined two-tet
mesh with space coarsening (DG(1)), a sheared five-tet cube (DG(0)) and a Kuhn mesh
with a moved centre vertex (Neumann)."""
import numpy as np
import pytest

import st_inputs
from helpers import from_lib, oracle_mg_mesh, rel, to_lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.load import spacetime_load  # noqa: E402
from oracle.spacetime import sequential_solve  # noqa: E402

CASES = {
    # name: (start mesh, n_refine, n_space_levels, degree, N_t, options)
    "two_tet_dg1_full": ("two_tet", 3, 2, 1, 16, dict(coarsen=2)),
    "cube5_dg0": ("cube5", 3, 2, 0, 24, dict(nu_pre=2, nu_post=2)),
    "kuhn2_jitter_neumann": ("kuhn2_jitter", 2, 2, 1, 8, dict(bc=1, coarsen=2)),
}


@pytest.fixture(scope="module")
def lib_built():
    from paper_1911_09548_gb300._build import build
    build()
    import paper_1911_09548_gb300
    assert torch.cuda.is_available()
    return paper_1911_09548_gb300


_cache = {}


def setup_case(name, stmg):
    if name in _cache:
        return _cache[name]
    kind, nr, nsl, p, N_t, opts = CASES[name]
    xyz, tets = st_inputs.start_mesh(kind, 0)
    nu, sigma = st_inputs.materials_tets(len(tets) * 8 ** nr, "two_material", 2)
    S = stmg.SpaceTimeSolver(0, nu, sigma, 1.0, N_t, p, n_space_levels=nsl, mesh=(xyz, tets, nr), **opts)
    sl, tl, mg = oracle_mg_mesh(xyz, tets, nr, nsl, nu, sigma, 1.0, N_t, p, coarsen=opts.get("coarsen", 0),
                                nu_pre=opts.get("nu_pre", 1), nu_post=opts.get("nu_post", 1), bc=opts.get("bc", 0))
    assert [(L["space_level"], L["N_t"]) for L in S.levels] == [(t.s, t.N_t) for t in tl]
    _cache[name] = (S, sl, tl, mg, p)
    return _cache[name]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("name", list(CASES))
def test_load_residual_slab_solve(name, lib_built):
    S, sl, tl, mg, p = setup_case(name, lib_built)
    exc = st_inputs.excitation(3)
    fo = spacetime_load(sl[0].mesh, exc, p, tl[0].N_t, 1.0)
    assert rel(host(S.load(exc)), to_lib(fo)) < 1e-13
    rng = np.random.default_rng(1)
    for lvl in range(S.n_levels):
        L = S.levels[lvl]
        shape = (L["N_t"], p + 1, L["n_edge"])
        f, x = rng.normal(size=shape), rng.normal(size=shape)
        r = S.residual(dev(to_lib(f)), dev(to_lib(x)), level=lvl)
        assert rel(host(r), to_lib(mg.residual(lvl, f, x))) < 1e-13
        y = host(S.slab_solve(dev(to_lib(f)), level=lvl))
        assert rel(from_lib(y, p + 1), mg.slabs[lvl].solve(f)) < 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_vcycle_iterates(name, lib_built):
    S, sl, tl, mg, p = setup_case(name, lib_built)
    f = S.load(st_inputs.excitation(4))
    fo = from_lib(host(f), p + 1)
    x = S.zeros()
    xo = np.zeros_like(fo)
    for it in range(3):
        S.vcycle(f, x)
        xo = mg.vcycle(fo, xo)
        assert rel(from_lib(host(x), p + 1), xo) < 1e-11, it


def test_solve_reaches_time_stepping(lib_built):
    S, sl, tl, mg, p = setup_case("two_tet_dg1_full", lib_built)
    f = S.load(st_inputs.excitation(5))
    x = S.zeros()
    out = S.solve(f, x, rtol=1e-10, maxit=60)
    assert out["status"] == 0
    xs = sequential_solve(mg.slabs[0], from_lib(host(f), p + 1))
    assert rel(from_lib(host(x), p + 1), xs) < 1e-8
