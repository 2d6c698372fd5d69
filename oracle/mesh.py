"""Kuhn tetrahedral meshes of the unit cube and their nested hierarchy (CPU oracle).

TEST INFRASTRUCTURE ONLY. This package is the slow, plain reference that the CUDA
path is checked against. Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import it; the product path never does.

The paper discretises the eddy-current problem on a tetrahedral mesh with
lowest-order Nedelec (edge) elements (Section 3, eq. EddyCurrent) and refines the
mesh uniformly to build the spatial hierarchy (Section 5.1).  The paper's
two-tetrahedron start mesh is not specified further, so the oracle uses the
Kuhn (Freudenthal) cube mesh, whose uniform refinement is again a Kuhn mesh.

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
