"""Kuhn tetrahedral meshes of the unit cube and their nested hierarchy (CPU oracle).

TEST INFRASTRUCTURE ONLY. This package is the slow, plain reference that the CUDA
path is checked against. Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import it; the product path never does.

The paper discretises the eddy-current problem on a tetrahedral mesh with
lowest-order Nedelec (edge) elements (Section 3, eq. EddyCurrent) and refines the
mesh uniformly to build the spatial hierarchy (Section 5.1).  The paper's
two-tetrahedron start mesh is not specified further, so the benchmark workloads use
the Kuhn (Freudenthal) cube mesh, whose uniform refinement is again a Kuhn mesh;
general start meshes and their red refinement are at the end of this file.

Conventions (shared with the C library through the published problem statement,
not through code):
  * vertex (i, j, k), 0 <= i, j, k <= n, has id i + (n+1)*(j + (n+1)*k) and
    coordinates (i, j, k) / n;
  * cubes are numbered c = ci + n*(cj + n*ck); cube c holds the six tets
    6*c + p, p indexing the permutations of the axes (x, y, z) in lexicographic
    order; the tet of permutation (a, b, c) is the vertex chain
    v0 = cube corner, v1 = v0 + e_a, v2 = v1 + e_b, v3 = v2 + e_c;
  * edges are the sorted vertex pairs (lo, hi), numbered in lexicographic
    order and oriented lo -> hi;
  * an edge lies on the boundary iff both end points lie on one face plane;
    a vertex is interior iff none of its indices is 0 or n.
Boundary conditions (Section 3 offers both): Dirichlet u x n = 0 keeps the interior
edges and vertices as unknowns; Neumann keeps every edge, and every vertex but
vertex 0 (the nodal matrix of the Neumann problem is singular with the constants as
kernel; G annihilates constants, so fixing one vertex changes no correction G z).
The flags edge_interior / vert_interior mark the unknowns in both cases.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

PERMS = list(itertools.permutations(range(3)))  # lexicographic order


@dataclass
class KuhnMesh:
    n: int                 # cubes per side
    xyz: np.ndarray        # (nv, 3) float64 coordinates
    ijk: np.ndarray        # (nv, 3) int64 lattice indices
    tets: np.ndarray       # (nt, 4) int64 vertex ids (chain order)
    edges: np.ndarray      # (ne, 2) int64 sorted vertex pairs
    tet_edges: np.ndarray  # (nt, 6) int64 edge ids of local edges (i<j pairs)
    edge_interior: np.ndarray  # (ne,) bool
    vert_interior: np.ndarray  # (nv,) bool

    @property
    def h(self) -> float:
        return 1.0 / self.n

    @property
    def interior_edges(self) -> np.ndarray:
        return np.nonzero(self.edge_interior)[0]

    @property
    def interior_verts(self) -> np.ndarray:
        return np.nonzero(self.vert_interior)[0]


LOCAL_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def kuhn_mesh(n: int, bc: str = "dirichlet") -> KuhnMesh:
    """Build the Kuhn mesh of [0,1]^3 with n cubes per side (plain loops); bc selects
    the unknowns ("dirichlet" or "neumann")."""
    nv = (n + 1) ** 3
    ijk = np.zeros((nv, 3), dtype=np.int64)
    for k in range(n + 1):
        for j in range(n + 1):
            for i in range(n + 1):
                ijk[i + (n + 1) * (j + (n + 1) * k)] = (i, j, k)
    xyz = ijk.astype(np.float64) / n

    def vid(p):
        return p[0] + (n + 1) * (p[1] + (n + 1) * p[2])

    tets = []
    for ck in range(n):
        for cj in range(n):
            for ci in range(n):
                for perm in PERMS:
                    p = [ci, cj, ck]
                    chain = [vid(p)]
                    for ax in perm:
                        p = list(p)
                        p[ax] += 1
                        chain.append(vid(p))
                    tets.append(chain)
    tets = np.array(tets, dtype=np.int64)

    pairs = set()
    for t in tets:
        for a, b in LOCAL_EDGES:
            lo, hi = sorted((int(t[a]), int(t[b])))
            pairs.add((lo, hi))
    edges = np.array(sorted(pairs), dtype=np.int64)
    index = {(int(a), int(b)): e for e, (a, b) in enumerate(edges)}
    tet_edges = np.zeros((len(tets), 6), dtype=np.int64)
    for t, tv in enumerate(tets):
        for le, (a, b) in enumerate(LOCAL_EDGES):
            lo, hi = sorted((int(tv[a]), int(tv[b])))
            tet_edges[t, le] = index[(lo, hi)]

    on_bdry = (ijk == 0) | (ijk == n)            # (nv, 3) per-axis face flags
    vert_interior = ~on_bdry.any(axis=1)
    a, b = edges[:, 0], edges[:, 1]
    same_face = ((ijk[a] == 0) & (ijk[b] == 0)) | ((ijk[a] == n) & (ijk[b] == n))
    edge_interior = ~same_face.any(axis=1)
    if bc == "neumann":
        edge_interior = np.ones(len(edges), dtype=bool)
        vert_interior = np.ones(nv, dtype=bool)
        vert_interior[0] = False
    elif bc != "dirichlet":
        raise ValueError(bc)
    return KuhnMesh(n, xyz, ijk, tets, edges, tet_edges, edge_interior, vert_interior)


def tet_barycentres(mesh: KuhnMesh) -> np.ndarray:
    return mesh.xyz[mesh.tets].mean(axis=1)


def locate_point(n: int, x: np.ndarray) -> int:
    """Index of a Kuhn tet of mesh n that contains point x (closed tets).

    Cube = floor(n x) (clamped), and inside the cube the tet of permutation
    (a, b, c) is {u_a >= u_b >= u_c} in local coordinates u.  Ties (points on
    shared faces) go to the lowest permutation index that contains the point.
    """
    u = np.asarray(x, dtype=np.float64) * n
    c = np.minimum(np.floor(u + 0.0), n - 1).astype(np.int64)
    c = np.maximum(c, 0)
    loc = u - c
    cube = int(c[0] + n * (c[1] + n * c[2]))
    for p, (a, b, cc) in enumerate(PERMS):
        if loc[a] >= loc[b] - 1e-12 and loc[b] >= loc[cc] - 1e-12:
            return 6 * cube + p
    raise AssertionError("point not located")


def fine_tet_parents(coarse_n: int) -> np.ndarray:
    """Parent coarse tet of every tet of the Kuhn mesh 2*coarse_n (by barycentre)."""
    fine = kuhn_mesh(2 * coarse_n)
    bc = tet_barycentres(fine)
    return np.array([locate_point(coarse_n, b) for b in bc], dtype=np.int64)


# ----------------------------------------------------------------- general tet meshes
# Section 5.1 builds the spatial hierarchy by uniform refinement of a coarse start mesh.
# Besides the Kuhn cube meshes the oracle takes any conforming tetrahedral mesh and
# refines it with the red refinement of J. Bey (Computing 55, 1995): every tet is cut
# into its four corner tets and four tets around one diagonal of the inner octahedron.
# Conventions (shared with the C library through the published problem statement):
#   * a tet keeps the vertex order it is given in; edges are the sorted vertex pairs,
#     numbered lexicographically and oriented lo -> hi, as for Kuhn meshes;
#   * refinement keeps the coarse vertex ids and gives the midpoint of coarse edge e the
#     id nv + e; child k of coarse tet t is tet 8 t + k, with vertex lists (x_ij = the
#     midpoint of the parent's local vertices i and j, in the parent's vertex order)
#       k=0 (x0, x01, x02, x03)  k=1 (x01, x1, x12, x13)  k=2 (x02, x12, x2, x23)
#       k=3 (x03, x13, x23, x3)  k=4 (x01, x02, x03, x13) k=5 (x01, x02, x12, x13)
#       k=6 (x02, x03, x13, x23) k=7 (x02, x12, x13, x23)
#   * the boundary is the set of faces that belong to one tet only; Dirichlet keeps the
#     edges and vertices that lie on no boundary face, Neumann keeps every edge and every
#     vertex but vertex 0.

@dataclass
class TetMesh:
    xyz: np.ndarray            # (nv, 3) float64
    tets: np.ndarray           # (nt, 4) int64, as given / as refined
    edges: np.ndarray          # (ne, 2) int64 sorted vertex pairs, lexicographic
    tet_edges: np.ndarray      # (nt, 6) int64 edge ids of the local edges LOCAL_EDGES
    edge_interior: np.ndarray  # (ne,) bool: unknowns
    vert_interior: np.ndarray  # (nv,) bool: unknowns
    parent: np.ndarray | None = None   # (nt,) coarse tet of every tet of a refined mesh
    n: int = 0                 # 0: not a Kuhn mesh

    @property
    def interior_edges(self) -> np.ndarray:
        return np.nonzero(self.edge_interior)[0]

    @property
    def interior_verts(self) -> np.ndarray:
        return np.nonzero(self.vert_interior)[0]

    @property
    def longest_edge(self) -> np.ndarray:
        """h_T of eq. CoarseningRule read as the diameter of T (its longest edge)."""
        P = self.xyz[self.tets]
        return np.max([np.linalg.norm(P[:, a] - P[:, b], axis=1) for a, b in LOCAL_EDGES], axis=0)


TET_FACES = [(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)]
BEY_CHILDREN = [  # entries: parent-local vertex i (int) or midpoint (i, j)
    (0, (0, 1), (0, 2), (0, 3)),
    ((0, 1), 1, (1, 2), (1, 3)),
    ((0, 2), (1, 2), 2, (2, 3)),
    ((0, 3), (1, 3), (2, 3), 3),
    ((0, 1), (0, 2), (0, 3), (1, 3)),
    ((0, 1), (0, 2), (1, 2), (1, 3)),
    ((0, 2), (0, 3), (1, 3), (2, 3)),
    ((0, 2), (1, 2), (1, 3), (2, 3)),
]


def tet_mesh(xyz, tets, bc: str = "dirichlet", parent=None) -> TetMesh:
    """Edges, local edge ids and unknowns of a conforming tetrahedral mesh (plain loops)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    pairs = set()
    for t in tets:
        for a, b in LOCAL_EDGES:
            pairs.add(tuple(sorted((int(t[a]), int(t[b])))))
    edges = np.array(sorted(pairs), dtype=np.int64).reshape(-1, 2)
    index = {(int(a), int(b)): e for e, (a, b) in enumerate(edges)}
    tet_edges = np.zeros((len(tets), 6), dtype=np.int64)
    for t, tv in enumerate(tets):
        for le, (a, b) in enumerate(LOCAL_EDGES):
            tet_edges[t, le] = index[tuple(sorted((int(tv[a]), int(tv[b]))))]
    count = {}
    for tv in tets:
        for f in TET_FACES:
            key = tuple(sorted(int(tv[i]) for i in f))
            count[key] = count.get(key, 0) + 1
    bverts, bedges = set(), set()
    for key, c in count.items():
        if c == 1:
            bverts.update(key)
            for i, j in ((0, 1), (0, 2), (1, 2)):
                bedges.add(index[(key[i], key[j])])
    nv = len(xyz)
    if bc == "dirichlet":
        vert_interior = np.array([v not in bverts for v in range(nv)], dtype=bool)
        edge_interior = np.array([e not in bedges for e in range(len(edges))], dtype=bool)
    elif bc == "neumann":
        vert_interior = np.ones(nv, dtype=bool)
        vert_interior[0] = False
        edge_interior = np.ones(len(edges), dtype=bool)
    else:
        raise ValueError(bc)
    return TetMesh(xyz, tets, edges, tet_edges, edge_interior, vert_interior,
                   None if parent is None else np.asarray(parent, dtype=np.int64))


def refine_uniform(mesh: TetMesh, bc: str = "dirichlet") -> TetMesh:
    """One red refinement (conventions above)."""
    nv = len(mesh.xyz)
    index = {(int(a), int(b)): e for e, (a, b) in enumerate(mesh.edges)}
    mids = 0.5 * (mesh.xyz[mesh.edges[:, 0]] + mesh.xyz[mesh.edges[:, 1]])
    xyz = np.concatenate([mesh.xyz, mids])
    tets, parent = [], []
    for t, tv in enumerate(mesh.tets):
        def vid(s):
            if isinstance(s, int):
                return int(tv[s])
            i, j = s
            return nv + index[tuple(sorted((int(tv[i]), int(tv[j]))))]
        for child in BEY_CHILDREN:
            tets.append([vid(s) for s in child])
            parent.append(t)
    return tet_mesh(xyz, np.array(tets, dtype=np.int64), bc, parent)


def refine_times(xyz, tets, n_refine: int, bc: str = "dirichlet"):
    """Meshes [coarse, refined once, ..., refined n_refine times]."""
    out = [tet_mesh(xyz, tets, bc)]
    for _ in range(n_refine):
        out.append(refine_uniform(out[-1], bc))
    return out
