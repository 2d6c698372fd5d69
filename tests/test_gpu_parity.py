"""GPU parity of every step of the hot path against the CPU oracle, through the C ABI.

Cases span several tiles and ragged tails: N_t not a power of two (coarsest level
solved by forward substitution over an odd number of slabs), N_t beyond one
residual pass (256 slabs), DG(0) and DG(1), a hierarchy that coarsens space
(eq. CoarseningRule admits it), two-material coefficients, and the nodal Jacobi
variant.  Tolerances: 1e-11 relative per V-cycle iterate (FP64 path, native FP64 or the
FP64-accurate double-float slab solve); single operators to 1e-12 (they involve one
factorisation solve at most).
"""
import numpy as np
import pytest

import st_inputs
from helpers import from_lib, oracle_mg, rel, to_lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.load import spacetime_load  # noqa: E402
from oracle.spacetime import (apply_L, restrict_space, restrict_time, prolong_space,  # noqa: E402
                              prolong_time, sequential_solve, time_integrate)

CASES = {
    # name: (n, nsl, p, N_t, materials, options)
    "dg0_two_grid": (4, 1, 0, 16, "unit", dict(max_levels=2)),
    "dg1_ragged": (8, 1, 1, 20, "two_material", dict(nu_pre=2, nu_post=2)),
    "dg1_space": (8, 2, 1, 16, "unit", dict()),
    "dg0_long": (8, 1, 0, 300, "two_material", dict()),
    "dg1_jacobi": (4, 1, 1, 8, "two_material", dict(nodal_solve=1, nodal_jacobi_sweeps=3)),
    # FP64-accurate double-float slab solve (slab_prec = 2) on the same parity bar
    "dg1_ragged_df": (8, 1, 1, 20, "two_material", dict(nu_pre=2, nu_post=2, slab_prec=2)),
    "dg1_space_df": (8, 2, 1, 16, "unit", dict(slab_prec=2)),
    "dg0_long_df": (8, 1, 0, 300, "two_material", dict(slab_prec=2)),
    # coarse-level solves as persistent cooperative launches (grid barriers between depths)
    "dg1_ragged_persistent": (8, 1, 1, 20, "two_material", dict(nu_pre=2, nu_post=2, persistent_split=1)),
    "dg0_long_df_persistent": (8, 1, 0, 300, "two_material", dict(slab_prec=2, persistent_split=1)),
    # coarse-level solves as dataflow launches (every task waits only for what it reads)
    "dg1_ragged_dataflow": (8, 1, 1, 20, "two_material", dict(nu_pre=2, nu_post=2, persistent_split=2)),
    "dg0_long_df_dataflow": (8, 1, 0, 300, "two_material", dict(slab_prec=2, persistent_split=2)),
    # other hybrid-smoother orderings (Section 4): "SSA" (pre A, S, S; post S, S, A), "SA"
    "dg1_ragged_SSA": (8, 1, 1, 20, "two_material", dict(smoother="SSA")),
    "dg0_two_grid_SA": (4, 1, 0, 16, "unit", dict(max_levels=2, smoother="SA")),
    # Neumann boundary (all edges, grounded vertex 0), space coarsening on the first transition
    "dg1_neumann_full": (8, 2, 1, 16, "two_material", dict(bc=1, coarsen=2)),
    # degenerate hierarchies: one slab (the V-cycle is the exact coarse solve), the smallest
    # Kuhn mesh (2^3 cubes), a prime number of slabs (no time coarsening at all)
    "dg1_single_slab": (4, 1, 1, 1, "two_material", dict()),
    "dg0_n2": (2, 1, 0, 8, "unit", dict()),
    "dg1_prime": (4, 1, 1, 7, "two_material", dict()),
    # tiled / split-K thresholds chosen per level by timing at setup
    "dg1_long_autotune": (8, 1, 1, 128, "two_material", dict(nu_pre=2, nu_post=2, autotune=1)),
}


@pytest.fixture(scope="module")
def lib_built():
    from paper_1911_09548_gb300._build import build
    build()
    import paper_1911_09548_gb300
    paper_1911_09548_gb300.lib()
    assert torch.cuda.is_available()
    return paper_1911_09548_gb300


_cache = {}


def setup_case(name, lib_built):
    if name in _cache:
        return _cache[name]
    n, nsl, p, N_t, mat, opts = CASES[name]
    nu, sigma = st_inputs.materials(n, mat, 1)
    S = lib_built.SpaceTimeSolver(n, nu, sigma, 1.0, N_t, p, n_space_levels=nsl, **opts)
    okw = dict(coarsen=opts.get("coarsen", 0), max_levels=opts.get("max_levels", 0),
               nu_pre=opts.get("nu_pre", 1), nu_post=opts.get("nu_post", 1),
               nodal="exact" if opts.get("nodal_solve", 0) == 0 else "jacobi",
               jacobi_sweeps=opts.get("nodal_jacobi_sweeps", 0), pattern=opts.get("smoother", ""),
               bc=opts.get("bc", 0))
    sl, tl, mg = oracle_mg(n, nsl, nu, sigma, 1.0, N_t, p, **okw)
    assert [(L["space_level"], L["N_t"]) for L in S.levels] == [(t.s, t.N_t) for t in tl]
    _cache[name] = (S, sl, tl, mg, p)
    return _cache[name]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("name", list(CASES))
def test_load(name, lib_built):
    S, sl, tl, mg, p = setup_case(name, lib_built)
    exc = st_inputs.excitation(3)
    f = host(S.load(exc))
    fo = spacetime_load(sl[0].mesh, exc, p, tl[0].N_t, 1.0)
    assert rel(f, to_lib(fo)) < 1e-13


@pytest.mark.parametrize("name", list(CASES))
def test_residual_and_norm(name, lib_built):
    S, sl, tl, mg, p = setup_case(name, lib_built)
    rng = np.random.default_rng(1)
    for lvl in range(S.n_levels):
        L = S.levels[lvl]
        shape = (L["N_t"], p + 1, L["n_edge"])
        fo, xo = rng.normal(size=shape), rng.normal(size=shape)
        r, nrm = S.residual(dev(to_lib(fo)), dev(to_lib(xo)), level=lvl, want_norm=True)
        ro = mg.residual(lvl, fo, xo)
        assert rel(host(r), to_lib(ro)) < 1e-13
        assert abs(nrm - np.linalg.norm(ro)) <= 1e-13 * np.linalg.norm(ro)


@pytest.mark.parametrize("name", list(CASES))
def test_slab_solve(name, lib_built):
    S, sl, tl, mg, p = setup_case(name, lib_built)
    rng = np.random.default_rng(2)
    for lvl in range(S.n_levels):
        L = S.levels[lvl]
        ro = rng.normal(size=(L["N_t"], p + 1, L["n_edge"]))
        y = host(S.slab_solve(dev(to_lib(ro)), level=lvl))
        assert rel(from_lib(y, p + 1), mg.slabs[lvl].solve(ro)) < 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_nodal_correction_parts(name, lib_built):
    S, sl, tl, mg, p = setup_case(name, lib_built)
    rng = np.random.default_rng(3)
    lvl = 0
    L = S.levels[lvl]
    sp_ = sl[L["space_level"]]
    q, N_t, ne, nn = p + 1, L["N_t"], L["n_edge"], L["n_node"]
    ro = rng.normal(size=(N_t, q, ne))
    y = host(S.grad_T(dev(to_lib(ro))))
    yo = (sp_.G.T @ ro.reshape(-1, ne).T).T.reshape(N_t, q, nn)
    assert rel(from_lib(y, q), yo) < 1e-14
    z = host(S.nodal_solve(dev(to_lib(yo))))
    if S.opt.nodal_solve == 0:
        zo = sp_.kn_solve(np.ascontiguousarray(yo.reshape(-1, nn).T)).T.reshape(N_t, q, nn)
    else:
        d = sp_.Kn.diagonal()[:, None]
        Y = yo.reshape(-1, nn).T
        Z = np.zeros_like(Y)
        for _ in range(S.opt.nodal_jacobi_sweeps):
            Z = Z + (2.0 / 3.0) * (Y - sp_.Kn @ Z) / d
        zo = Z.T.reshape(N_t, q, nn)
    assert rel(from_lib(z, q), zo) < 1e-12
    w = host(S.time_integrate(dev(to_lib(zo))))
    slab = mg.slabs[lvl]
    wo = time_integrate(slab.Kt, slab.Nt, zo)
    assert rel(from_lib(w, q), wo) < 1e-14
    xo = rng.normal(size=(N_t, q, ne))
    x = dev(to_lib(xo))
    S.grad_add(dev(to_lib(wo)), x)
    xw = xo + (sp_.G @ wo.reshape(-1, nn).T).T.reshape(N_t, q, ne)
    assert rel(from_lib(host(x), q), xw) < 1e-14


@pytest.mark.parametrize("name", list(CASES))
def test_smoothers(name, lib_built):
    from oracle.spacetime import correction_A, smoother_S
    S, sl, tl, mg, p = setup_case(name, lib_built)
    rng = np.random.default_rng(4)
    for lvl in range(S.n_levels):
        L = S.levels[lvl]
        shape = (L["N_t"], p + 1, L["n_edge"])
        fo, xo = rng.normal(size=shape), rng.normal(size=shape)
        x = dev(to_lib(xo))
        S.smooth_S(dev(to_lib(fo)), x, level=lvl)
        assert rel(from_lib(host(x), p + 1), smoother_S(mg.slabs[lvl], fo, xo, 0.5)) < 1e-12
        x = dev(to_lib(xo))
        S.correct_A(dev(to_lib(fo)), x, level=lvl)
        want = correction_A(mg.slabs[lvl], fo, xo, mg.nodal, mg.jacobi_sweeps)
        assert rel(from_lib(host(x), p + 1), want) < 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_transfers_and_coarse_solve(name, lib_built):
    S, sl, tl, mg, p = setup_case(name, lib_built)
    rng = np.random.default_rng(5)
    for lvl in range(S.n_levels - 1):
        L, C = S.levels[lvl], S.levels[lvl + 1]
        ro = rng.normal(size=(L["N_t"], p + 1, L["n_edge"]))
        rc = host(S.restrict(dev(to_lib(ro)), level=lvl))
        want = restrict_time(p, ro)
        space = C["space_level"] != L["space_level"]
        if space:
            want = restrict_space(sl[L["space_level"]].Px, want)
        assert rel(from_lib(rc, p + 1), want) < 1e-14
        eo = rng.normal(size=(C["N_t"], p + 1, C["n_edge"]))
        xo = rng.normal(size=(L["N_t"], p + 1, L["n_edge"]))
        x = dev(to_lib(xo))
        S.prolong_add(dev(to_lib(eo)), x, level=lvl)
        e = prolong_space(sl[L["space_level"]].Px, eo) if space else eo
        assert rel(from_lib(host(x), p + 1), xo + prolong_time(p, e)) < 1e-14
    Lc = S.levels[-1]
    fo = rng.normal(size=(Lc["N_t"], p + 1, Lc["n_edge"]))
    xc = host(S.coarse_solve(dev(to_lib(fo))))
    assert rel(from_lib(xc, p + 1), sequential_solve(mg.slabs[-1], fo)) < 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_vcycle_iterates(name, lib_built):
    S, sl, tl, mg, p = setup_case(name, lib_built)
    exc = st_inputs.excitation(4)
    f = S.load(exc)
    fo = from_lib(host(f), p + 1)
    x = S.zeros()
    xo = np.zeros_like(fo)
    for it in range(3):
        S.vcycle(f, x)
        xo = mg.vcycle(fo, xo)
        assert rel(from_lib(host(x), p + 1), xo) < 1e-11, it


@pytest.mark.parametrize("name", ["dg0_two_grid", "dg1_space", "dg1_space_df"])
def test_solve_reaches_time_stepping_solution(name, lib_built):
    S, sl, tl, mg, p = setup_case(name, lib_built)
    f = S.load(st_inputs.excitation(5))
    x = S.zeros()
    out = S.solve(f, x, rtol=1e-10, maxit=40)
    assert out["status"] == 0 and out["rel_res"] <= 1e-10
    fo = from_lib(host(f), p + 1)
    xs = sequential_solve(mg.slabs[0], fo)
    assert rel(from_lib(host(x), p + 1), xs) < 1e-8
    # history is monotone and matches an oracle-side residual of the final iterate
    h = out["history"]
    assert np.all(np.diff(h) < 0)
    ro = fo - apply_L(sl[0], mg.slabs[0].Kt, mg.slabs[0].Mt, mg.slabs[0].Nt, from_lib(host(x), p + 1))
    assert abs(np.linalg.norm(ro) / np.linalg.norm(fo) - out["rel_res"]) < 1e-12


def test_solve_host_buffers_match_device(lib_built):
    S, sl, tl, mg, p = setup_case("dg1_space", lib_built)
    f = S.load(st_inputs.excitation(6))
    x = S.zeros()
    out_d = S.solve(f, x, rtol=1e-9, maxit=30)
    fh = host(f).copy()
    xh = np.zeros_like(fh)
    out_h = S.solve_host(fh, xh, rtol=1e-9, maxit=30)
    assert out_h["iters"] == out_d["iters"]
    assert np.array_equal(xh, host(x))       # same kernels, same order: bit-identical


def test_graph_replay_matches_direct_launches(lib_built):
    """A V-cycle replayed from its captured CUDA graph is bit-identical to launching
    the same kernels one by one, and the launch counter counts replayed kernels."""
    n, nsl, p, N_t, mat, opts = CASES["dg1_ragged"]
    nu, sigma = st_inputs.materials(n, mat, 1)
    side = torch.cuda.Stream()
    out = {}
    with torch.cuda.stream(side):
        for g in (0, 1):
            S = lib_built.SpaceTimeSolver(n, nu, sigma, 1.0, N_t, p, stream=side.cuda_stream, use_graph=g, **opts)
            f = S.load(st_inputs.excitation(12))
            x = S.zeros()
            c0 = lib_built.st_mg_launch_count()
            for _ in range(3):
                S.vcycle(f, x)
            side.synchronize()
            out[g] = (x.cpu().numpy(), lib_built.st_mg_launch_count() - c0)
            S.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1] > 0


@pytest.mark.parametrize("slab_prec", [0, 1, 2, 3, 4])
def test_persistent_split_matches_per_depth_launches(slab_prec, lib_built):
    """The persistent split-K solve (grid barriers between depths) and the dataflow one
    (every task waits only for the tasks it reads from) run the same items, partial
    layout and summation order as the per-depth kernels: a V-cycle must agree bit for
    bit, for the slab solves of the coarse time levels and the nodal solves alike."""
    nu, sigma = st_inputs.materials(8, "two_material", 4)
    xs = []
    for ps in (0, 1, 2):
        S = lib_built.SpaceTimeSolver(8, nu, sigma, 1.0, 64, 1, nu_pre=2, nu_post=2, slab_prec=slab_prec,
                                      persistent_split=ps)
        f = S.load(st_inputs.excitation(6))
        x = S.zeros()
        for _ in range(2):
            S.vcycle(f, x)
        xs.append(host(x))
        S.close()
    assert np.array_equal(xs[0], xs[1])
    assert np.array_equal(xs[0], xs[2])


def test_autotune_choices_valid(lib_built):
    S, sl, tl, mg, p = setup_case("dg1_long_autotune", lib_built)
    ws = [lib_built.st_mg_split_waves(S.h, l) for l in range(S.n_levels)]
    assert all(w in (0, 1, 2, 4, 8) for w in ws)


def test_split_waves_set_between_graph_replays(lib_built):
    """Thresholds set after the V-cycle graph was captured (all tiled, then all split-K)
    take effect on the next V-cycle: each iterate still matches the oracle."""
    n, nsl, p, N_t, mat, opts = CASES["dg1_long_autotune"]
    _, sl, tl, mg, _ = setup_case("dg1_long_autotune", lib_built)
    nu, sigma = st_inputs.materials(n, mat, 1)
    stream = torch.cuda.Stream()
    S = lib_built.SpaceTimeSolver(n, nu, sigma, 1.0, N_t, p, nu_pre=2, nu_post=2, stream=stream.cuda_stream)
    with torch.cuda.stream(stream):
        f = S.load(st_inputs.excitation(6))
        x = S.zeros()
    for bad in (-1, 65):
        with pytest.raises(lib_built.StMgError) as e:
            lib_built.st_mg_set_split_waves(S.h, 0, bad)
        assert e.value.status == 1
    fo = from_lib(host(f), p + 1)
    xo = np.zeros_like(fo)
    for waves in (2, 0, 64):
        for l in range(S.n_levels):
            lib_built.st_mg_set_split_waves(S.h, l, waves)
        S.vcycle(f, x)
        xo = mg.vcycle(fo, xo)
        assert rel(from_lib(host(x), p + 1), xo) < 1e-11, waves
    S.close()
