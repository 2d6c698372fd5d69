"""Pins of the oracle's general-mesh path (a coarse tetrahedral start mesh refined
uniformly, Section 5.1) against geometry and exact identities, not against itself:

  * red refinement: every child has 1/8 of its parent's volume, its vertices are parent
    vertices or edge midpoints, the refined mesh is conforming (every face belongs to one
    or two tets) with the same boundary area, and V - E + F - T = 1 (a ball);
  * boundary detection by faces agrees with the Kuhn criterion on a Kuhn mesh;
  * Whitney elements on the distorted meshes: K G = 0, G^T M G = K_n, affine-field
    energies exact;
  * nested prolongations: interpolation of affine (edge) and linear (node) fields
    commutes with prolongation, P_x G_c = G_f P_n, and with coefficients constant on
    coarse tets the Galerkin products equal the coarse assembled matrices exactly;
  * the coarsening rule's h_T on a Kuhn mesh reduces to sqrt(3)/n.
"""
import numpy as np
import pytest

import st_inputs
from oracle.fem import assemble_edge_matrices, discrete_gradient, nodal_stiffness, tet_geometry
from oracle.mesh import LOCAL_EDGES, TET_FACES, kuhn_mesh, refine_times, tet_mesh
from oracle.multigrid import coarsening_lambda, coarsening_lambda_mesh
from oracle.spacetime import ancestor_longest_edge, build_space_hierarchy_mesh
from oracle.transfer import edge_prolongation_nested, node_prolongation_nested, round_dyadic

KINDS = ["two_tet", "cube5", "kuhn2_jitter"]


def _faces(mesh):
    count = {}
    for tv in mesh.tets:
        for f in TET_FACES:
            key = tuple(sorted(int(tv[i]) for i in f))
            count[key] = count.get(key, 0) + 1
    return count


def _boundary_area(mesh):
    area = 0.0
    for key, c in _faces(mesh).items():
        if c == 1:
            p = mesh.xyz[list(key)]
            area += 0.5 * np.linalg.norm(np.cross(p[1] - p[0], p[2] - p[0]))
    return area


@pytest.mark.parametrize("kind", KINDS)
def test_red_refinement_geometry(kind):
    xyz, tets = st_inputs.start_mesh(kind, 1)
    ms = refine_times(xyz, tets, 2)
    for c, f in zip(ms[:-1], ms[1:]):
        vc, _ = tet_geometry(c)
        vf, _ = tet_geometry(f)
        assert len(f.tets) == 8 * len(c.tets)
        assert np.allclose(vf, vc[f.parent] / 8.0, rtol=1e-12, atol=0)
        # child vertices: parent vertices or midpoints of parent edges
        for t in range(len(f.tets)):
            P = c.xyz[c.tets[f.parent[t]]]
            for v in f.tets[t]:
                x = f.xyz[v]
                cands = [P[i] for i in range(4)] + [0.5 * (P[a] + P[b]) for a, b in LOCAL_EDGES]
                assert min(np.linalg.norm(x - y) for y in cands) < 1e-14
        counts = _faces(f)
        assert set(counts.values()) <= {1, 2}
        assert abs(_boundary_area(f) - _boundary_area(c)) < 1e-12 * _boundary_area(c)
        V, E, F, T = len(f.xyz), len(f.edges), len(counts), len(f.tets)
        assert V - E + F - T == 1


def test_face_boundary_matches_kuhn_criterion():
    for n in (2, 3):
        k = kuhn_mesh(n)
        g = tet_mesh(k.xyz, k.tets)
        assert np.array_equal(g.edges, k.edges) and np.array_equal(g.tet_edges, k.tet_edges)
        assert np.array_equal(g.edge_interior, k.edge_interior)
        assert np.array_equal(g.vert_interior, k.vert_interior)
        assert np.allclose(g.longest_edge, np.sqrt(3.0) / n, rtol=1e-15)


@pytest.mark.parametrize("kind", KINDS)
def test_whitney_identities_on_distorted_mesh(kind):
    xyz, tets = st_inputs.start_mesh(kind, 2)
    m = refine_times(xyz, tets, 2)[-1]
    nu, sigma = st_inputs.materials_tets(len(m.tets), "two_material", 5)
    M, K = assemble_edge_matrices(m, nu, sigma)
    G = discrete_gradient(m)
    Kn = nodal_stiffness(m, sigma)
    assert abs(K @ G).max() <= 1e-12 * abs(K).max()
    assert abs(G.T @ M @ G - Kn).max() <= 1e-12 * abs(Kn).max()
    # affine field a + b x x: curl energy exact (curl = 2b)
    Mf, Kf = assemble_edge_matrices(m, nu, sigma, interior=False)
    rng = np.random.default_rng(3)
    a, b = rng.normal(size=3), rng.normal(size=3)
    xa, xb = m.xyz[m.edges[:, 0]], m.xyz[m.edges[:, 1]]
    mid = 0.5 * (xa + xb)
    u = np.einsum("ed,ed->e", a[None, :] + np.cross(b[None, :], mid), xb - xa)
    vol, _ = tet_geometry(m)
    assert abs(u @ Kf @ u - np.sum(nu * vol) * 4 * b @ b) < 1e-11 * max(1.0, np.sum(nu * vol) * 4 * b @ b)


def _all_unknowns(mesh):
    mesh.edge_interior[:] = True
    mesh.vert_interior[:] = True
    return mesh


@pytest.mark.parametrize("kind", KINDS)
def test_nested_prolongations_reproduce_and_commute(kind):
    xyz, tets = st_inputs.start_mesh(kind, 3)
    r = 2 if kind == "kuhn2_jitter" else 3   # the others have interior vertices from 2 refinements on
    c, f = refine_times(xyz, tets, r)[r - 1:]
    Px = round_dyadic(edge_prolongation_nested(c, f))
    Pn = round_dyadic(node_prolongation_nested(c, f))
    assert abs(Px @ discrete_gradient(c) - discrete_gradient(f) @ Pn).max() == 0.0
    assert np.all(Px.data * 4 == np.round(Px.data * 4))
    c, f = _all_unknowns(c), _all_unknowns(f)
    Pa = edge_prolongation_nested(c, f)
    Pna = node_prolongation_nested(c, f)
    rng = np.random.default_rng(4)
    a, b = rng.normal(size=3), rng.normal(size=3)

    def interp(m):
        xa, xb = m.xyz[m.edges[:, 0]], m.xyz[m.edges[:, 1]]
        mid = 0.5 * (xa + xb)
        return np.einsum("ed,ed->e", a[None, :] + np.cross(b[None, :], mid), xb - xa)

    assert abs(Pa @ interp(c) - interp(f)).max() < 1e-13
    w = np.array([0.3, -1.2, 2.0])
    assert abs(Pna @ (c.xyz @ w + 0.7) - (f.xyz @ w + 0.7)).max() < 1e-13


@pytest.mark.parametrize("kind", KINDS)
def test_galerkin_equals_coarse_assembly(kind):
    """Coefficients constant on each coarse tet: nested Whitney spaces make P^T A_f P the
    matrix assembled on the coarse mesh."""
    xyz, tets = st_inputs.start_mesh(kind, 4)
    r = 2 if kind == "kuhn2_jitter" else 3
    ms = refine_times(xyz, tets, r)
    nu_c, sig_c = st_inputs.materials_tets(len(ms[r - 1].tets), "two_material", 6)
    f = ms[r]
    nu_f, sig_f = nu_c[f.parent], sig_c[f.parent]
    L = build_space_hierarchy_mesh(xyz, tets, r, 2, nu_f, sig_f)
    Mc, Kc = assemble_edge_matrices(ms[r - 1], nu_c, sig_c)
    assert abs(L[1].M - Mc).max() <= 1e-13 * abs(Mc).max()
    assert abs(L[1].K - Kc).max() <= 1e-13 * abs(Kc).max()
    assert abs(L[1].Kn - nodal_stiffness(ms[r - 1], sig_c)).max() <= 1e-13 * abs(L[1].Kn).max()


def test_coarsening_rule_general_reduces_to_kuhn():
    xyz, tets = st_inputs.start_mesh("kuhn2_jitter", 0)
    xyz = np.array([[i, j, k] for k in range(3) for j in range(3) for i in range(3)], float) / 2
    L = build_space_hierarchy_mesh(xyz, tets, 2, 3, *st_inputs.materials_tets(8 ** 2 * 48, "two_material", 1))
    h = ancestor_longest_edge(L)
    nu, sigma = st_inputs.materials_tets(8 ** 2 * 48, "two_material", 1)
    for s, n in enumerate((8, 4, 2)):
        assert np.allclose(h[s], np.sqrt(3.0) / n, rtol=1e-15)
        assert abs(coarsening_lambda_mesh(h[s], 0.01, nu, sigma) - coarsening_lambda(n, 0.01, nu, sigma)) < 1e-15


@pytest.mark.parametrize("p", [0, 1])
def test_vcycles_on_general_mesh_reach_time_stepping(p):
    """Space-time V-cycles with space coarsening on a refined two-tet start mesh converge
    to the sequential DG(p) time-stepping solution (the plain definition of the result)."""
    from helpers import oracle_mg_mesh
    from oracle.load import spacetime_load
    from oracle.spacetime import sequential_solve
    xyz, tets = st_inputs.start_mesh("two_tet", 0)
    nu, sigma = st_inputs.materials_tets(2 * 8 ** 3, "two_material", 2)
    sl, tl, mg = oracle_mg_mesh(xyz, tets, 3, 2, nu, sigma, 1.0, 8, p, coarsen=2)
    assert tl[1].s == 1
    f = spacetime_load(sl[0].mesh, st_inputs.excitation(1), p, 8, 1.0)
    xs = sequential_solve(mg.slabs[0], f)
    x = np.zeros_like(f)
    for _ in range(40):
        x = mg.vcycle(f, x)
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)
