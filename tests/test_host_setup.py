"""CPU checks of the C-ABI library: it loads, exports every declared symbol, and its
host-side setup (mesh, numbering, G, CSR, P_x, matrices, slab factors) agrees with
the oracle -- bit-exact for integer and dyadic data, to rounding for the rest."""
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import st_inputs
from helpers import from_lib, oracle_mg, rel, to_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_1911_09548_gb300._build import build
    build()
    import paper_1911_09548_gb300.binding as binding
    binding.lib()
    return binding


def test_exports_every_declared_symbol(B):
    inc = os.path.join(ROOT, "include")
    header = "".join(open(os.path.join(inc, h)).read() for h in sorted(os.listdir(inc)) if h.endswith(".h"))
    declared = set(re.findall(r"\b(st_mg_\w+)\s*\(", header))
    assert len(declared) >= 45
    L = B.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert declared <= set(B.exported_symbols())


def test_invalid_arguments_rejected(B):
    nu, sigma = st_inputs.materials(4, "unit")
    opt = B.st_mg_default_options()
    bad = B.make_problem(4, 1, nu, sigma, 1.0, 0, 0)          # N_t = 0
    with pytest.raises(B.StMgError) as e:
        B.st_mg_setup_host(bad, opt)
    assert e.value.status == 1
    sig2 = sigma.copy(); sig2[5] = -1.0
    with pytest.raises(B.StMgError):
        B.st_mg_setup_host(B.make_problem(4, 1, nu, sig2, 1.0, 4, 0), opt)
    with pytest.raises(B.StMgError):
        B.st_mg_setup_host(B.make_problem(6, 3, *st_inputs.materials(6, "unit"), 1.0, 4, 0), opt)  # 6 / 4
    h = B.st_mg_setup_host(B.make_problem(4, 1, nu, sigma, 1.0, 4, 0), opt)
    try:
        with pytest.raises(B.StMgError):     # host-only handles reject device calls
            B.st_mg_vcycle(h, 16, 16)
    finally:
        B.st_mg_destroy(h)
    assert B.st_mg_strerror(5) == "not converged"


@pytest.mark.parametrize("n,nsl,p,coarsen,bc", [(4, 1, 0, 0, 0), (8, 2, 1, 2, 0), (4, 2, 1, 2, 1)])
def test_host_setup_matches_oracle(B, n, nsl, p, coarsen, bc):
    """bc = 1: Neumann (all edges; vertex 0 grounds the nodal matrix)."""
    from paper_1911_09548_gb300 import SpaceTimeSolver
    nu, sigma = st_inputs.materials(n, "two_material", 3)
    S = SpaceTimeSolver(n, nu, sigma, 1.0, 8, p, n_space_levels=nsl, host_only=True, coarsen=coarsen, bc=bc)
    sl, tl, mg = oracle_mg(n, nsl, nu, sigma, 1.0, 8, p, coarsen=coarsen, bc=bc)
    assert [(L["space_level"], L["N_t"]) for L in S.levels] == [(t.s, t.N_t) for t in tl]
    for s in range(nsl):
        m = sl[s].mesh
        assert np.array_equal(S.debug(1, s).reshape(-1, 2), m.edges)
        assert np.array_equal(S.debug(2, s), m.interior_edges)
        assert np.array_equal(S.debug(3, s), m.interior_verts)
        M = sl[s].M.tocsr(); M.sort_indices()
        K = sl[s].K.tocsr(); K.sort_indices()
        rp, cols = S.debug(4, s), S.debug(5, s)
        assert np.array_equal(rp, M.indptr) and np.array_equal(cols, M.indices)
        assert rel(S.debug(6, s), M.data) < 1e-14
        # the oracle's sparse product drops entries that cancel to exactly zero, so K is
        # compared as a matrix on the library's (structural) pattern
        Kl = sp.csr_matrix((S.debug(7, s), cols, rp), shape=K.shape)
        assert abs(Kl - K).max() <= 1e-14 * abs(K).max()
        g = S.debug(8, s).reshape(-1, 2)
        G = sl[s].G.tocsr()
        for e in range(G.shape[0]):
            row = dict(zip(G.indices[G.indptr[e]:G.indptr[e + 1]], G.data[G.indptr[e]:G.indptr[e + 1]]))
            want = {}
            if g[e, 0] >= 0:
                want[g[e, 0]] = -1.0
            if g[e, 1] >= 0:
                want[g[e, 1]] = 1.0
            assert row == want
        Kn = sl[s].Kn.tocsr(); Kn.sort_indices()
        knl = sp.csr_matrix((S.debug(11, s), S.debug(10, s), S.debug(9, s)), shape=Kn.shape)
        if s == 0:   # assembled: same pattern
            assert np.array_equal(S.debug(9, s), Kn.indptr) and np.array_equal(S.debug(10, s), Kn.indices)
        assert abs(knl - Kn).max() <= 1e-13 * abs(Kn).max()
    if nsl > 1:
        P = sl[0].Px
        assert np.array_equal(S.debug(12), P.indptr) and np.array_equal(S.debug(13), P.indices)
        assert np.array_equal(S.debug(14), P.data)                 # dyadic: bit-exact
    rng = np.random.default_rng(0)
    for lvl, L in enumerate(S.levels):
        r = rng.normal(size=(L["n_edge"], L["N_t"] * (p + 1)))
        y = S.host_slab_solve(r, lvl)
        yo = mg.slabs[lvl].solve(from_lib(r, p + 1))
        assert rel(from_lib(y, p + 1), yo) < 1e-13
    S.close()


def test_server_options_validated(B):
    o = B.st_mg_server_default_options()
    assert (o.slots, o.max_cycles, o.slab_prec, o.nu, o.omega, o.keep_x, o.max_builds) == (4, 50, 3, 2, 0.5, 1, 2)
    for field, bad in (("slots", 0), ("max_cycles", 0), ("slab_prec", 5), ("omega", 0.0), ("mem_budget", -1),
                       ("max_builds", 0)):
        o = B.st_mg_server_default_options()
        setattr(o, field, bad)
        with pytest.raises(B.StMgError) as e:
            B.st_mg_server_create(o)
        assert e.value.status == 1


def test_smoother_pattern_validated(B):
    nu, sigma = st_inputs.materials(4, "unit")
    prob = B.make_problem(4, 1, nu, sigma, 1.0, 8, 0)
    for bad in (b"SXA", b"S A"):
        opt = B.st_mg_default_options()
        opt.smoother = bad
        with pytest.raises(B.StMgError) as e:
            B.st_mg_setup_host(prob, opt)
        assert e.value.status == 1
    opt = B.st_mg_default_options()
    opt.smoother = b"SSA"
    B.st_mg_destroy(B.st_mg_setup_host(prob, opt))



def test_split_solve_mode_validated(B):
    """persistent_split selects how few-right-hand-side solves walk the tree depths: 0 per-depth
    launches, 1 grid barriers, 2 dataflow; other values are rejected at setup."""
    nu, sigma = st_inputs.materials(4, "unit")
    prob = B.make_problem(4, 1, nu, sigma, 1.0, 8, 1)
    for ok in (0, 1, 2):
        opt = B.st_mg_default_options()
        opt.persistent_split = ok
        B.st_mg_destroy(B.st_mg_setup_host(prob, opt))
    for bad in (-1, 3):
        opt = B.st_mg_default_options()
        opt.persistent_split = bad
        with pytest.raises(B.StMgError) as e:
            B.st_mg_setup_host(prob, opt)
        assert e.value.status == 1


def test_split_waves_setter_needs_device_state(B):
    """The tiled / split-K threshold is device state: host-only handles reject both calls."""
    nu, sigma = st_inputs.materials(4, "unit")
    h = B.st_mg_setup_host(B.make_problem(4, 1, nu, sigma, 1.0, 8, 1), B.st_mg_default_options())
    try:
        for call in (lambda: B.st_mg_split_waves(h, 0), lambda: B.st_mg_set_split_waves(h, 0, 8)):
            with pytest.raises(B.StMgError) as e:
                call()
            assert e.value.status == 1
    finally:
        B.st_mg_destroy(h)


@pytest.mark.parametrize("kind,n_refine,nsl,p,bc", [("two_tet", 3, 2, 1, 0), ("cube5", 3, 2, 0, 0),
                                                    ("kuhn2_jitter", 2, 2, 1, 1)])
def test_general_mesh_setup_matches_oracle(B, kind, n_refine, nsl, p, bc):
    """General start mesh refined uniformly: meshes, unknowns, matrices, P_x (bit-exact:
    dyadic) and the slab factors agree with the oracle's independent construction."""
    from helpers import oracle_mg_mesh
    from paper_1911_09548_gb300 import SpaceTimeSolver
    xyz, tets = st_inputs.start_mesh(kind, 0)
    nt = len(tets) * 8 ** n_refine
    nu, sigma = st_inputs.materials_tets(nt, "two_material", 1)
    S = SpaceTimeSolver(0, nu, sigma, 1.0, 8, p, n_space_levels=nsl, host_only=True, coarsen=2, bc=bc,
                        mesh=(xyz, tets, n_refine))
    sl, tl, mg = oracle_mg_mesh(xyz, tets, n_refine, nsl, nu, sigma, 1.0, 8, p, coarsen=2, bc=bc)
    assert [(L["space_level"], L["N_t"]) for L in S.levels] == [(t.s, t.N_t) for t in tl]
    for s in range(nsl):
        m = sl[s].mesh
        assert np.array_equal(S.debug(1, s).reshape(-1, 2), m.edges)
        assert np.array_equal(S.debug(2, s), m.interior_edges)
        assert np.array_equal(S.debug(3, s), m.interior_verts)
        M = sl[s].M.tocsr(); M.sort_indices()
        K = sl[s].K.tocsr(); K.sort_indices()
        rp, cols = S.debug(4, s), S.debug(5, s)
        Ml = sp.csr_matrix((S.debug(6, s), cols, rp), shape=M.shape)
        Kl = sp.csr_matrix((S.debug(7, s), cols, rp), shape=K.shape)
        assert abs(Ml - M).max() <= 1e-13 * abs(M).max()
        assert abs(Kl - K).max() <= 1e-13 * abs(K).max()
        Kn = sl[s].Kn.tocsr()
        knl = sp.csr_matrix((S.debug(11, s), S.debug(10, s), S.debug(9, s)), shape=Kn.shape)
        assert abs(knl - Kn).max() <= 1e-12 * abs(Kn).max()
    P = sl[0].Px
    assert np.array_equal(S.debug(12), P.indptr) and np.array_equal(S.debug(13), P.indices)
    assert np.array_equal(S.debug(14), P.data)
    rng = np.random.default_rng(0)
    for lvl, L in enumerate(S.levels):
        r = rng.normal(size=(L["n_edge"], L["N_t"] * (p + 1)))
        assert rel(from_lib(S.host_slab_solve(r, lvl), p + 1), mg.slabs[lvl].solve(from_lib(r, p + 1))) < 1e-12
    S.close()


def test_general_mesh_rejected_when_invalid(B):
    xyz, tets = st_inputs.start_mesh("two_tet", 0)
    opt = B.st_mg_default_options()
    nu, sigma = st_inputs.materials_tets(2 * 8 ** 3, "unit")
    for bad_tets, n_refine, nsl in ((np.array([[0, 1, 2, 2], [0, 1, 2, 4]]), 3, 1),     # repeated vertex
                                    (np.array([[0, 1, 2, 7], [0, 1, 2, 4]]), 3, 1),     # id out of range
                                    (tets, 3, 5),                                       # too many levels
                                    (tets, 1, 1)):                                      # no interior unknowns
        n = len(bad_tets) * 8 ** n_refine
        prob = B.make_problem(0, nsl, nu[:n], sigma[:n], 1.0, 4, 0, mesh=(xyz, bad_tets, n_refine))
        with pytest.raises(B.StMgError) as e:
            B.st_mg_setup_host(prob, opt)
        assert e.value.status == 1
    extra = np.vstack([xyz, [[2.0, 2.0, 2.0]]])                                         # unused vertex
    prob = B.make_problem(0, 1, nu, sigma, 1.0, 4, 0, mesh=(extra, tets, 3))
    with pytest.raises(B.StMgError) as e:
        B.st_mg_setup_host(prob, opt)
    assert e.value.status == 1
    flat = xyz.copy(); flat[3] = [0.5, 0.5, 0.0]                                          # zero volume
    prob = B.make_problem(0, 1, nu, sigma, 1.0, 4, 0, mesh=(flat, tets, 3))
    with pytest.raises(B.StMgError):
        B.st_mg_setup_host(prob, opt)


@pytest.mark.parametrize("p,bc", [(1, 0), (0, 1)])
def test_kuhn_mesh_as_general_mesh_matches_kuhn_path(B, p, bc):
    """The Kuhn mesh handed in as a general mesh (coordinates and tets, no refinement) gives
    the Kuhn path's numbering and unknowns exactly and its matrices and slab solves to
    rounding: the general builder (face-based boundary, coordinate geometry) against the
    Kuhn builder (lattice rules, reference element matrices)."""
    from oracle.mesh import kuhn_mesh
    from paper_1911_09548_gb300 import SpaceTimeSolver
    n = 4
    km = kuhn_mesh(n)
    nu, sigma = st_inputs.materials(n, "two_material", 4)
    A = SpaceTimeSolver(n, nu, sigma, 1.0, 8, p, host_only=True, bc=bc)
    G = SpaceTimeSolver(0, nu, sigma, 1.0, 8, p, host_only=True, bc=bc, mesh=(km.xyz, km.tets, 0))
    for what in (1, 2, 3, 4, 5, 8, 9, 10):
        assert np.array_equal(A.debug(what, 0), G.debug(what, 0)), what
    for what in (6, 7, 11):
        a, g = A.debug(what, 0), G.debug(what, 0)
        assert np.abs(a - g).max() <= 1e-13 * np.abs(a).max(), what
    rng = np.random.default_rng(5)
    for lvl, L in enumerate(A.levels):
        r = rng.normal(size=(L["n_edge"], L["N_t"] * (p + 1)))
        assert rel(G.host_slab_solve(r, lvl), A.host_slab_solve(r, lvl)) < 1e-12
    A.close()
    G.close()
