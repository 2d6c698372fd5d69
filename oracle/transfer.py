"""Spatial prolongations between nested Kuhn meshes n -> 2n (CPU oracle).

TEST INFRASTRUCTURE ONLY (see oracle/mesh.py).

Section 2.2 coarsens in space inside the time V-cycle, and Section 5 notes that
the method only needs spatial prolongation/restriction through an interface.
For nested Whitney spaces the natural prolongation is interpolation:
  * edges:  P_x[f, c] = line integral over fine edge f of the coarse Whitney
    function w_c; because w_c is linear inside a coarse tet, that is
    w_c(midpoint of f) . (x_head - x_tail);
  * nodes:  P_n[v, c] = value at fine vertex v of the coarse P1 hat function c.
Restriction is the transpose.  Both act on interior (Dirichlet) unknowns.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import KuhnMesh, LOCAL_EDGES, kuhn_mesh, locate_point
from .fem import whitney_field, barycentric


def edge_prolongation(coarse: KuhnMesh, fine: KuhnMesh) -> sp.csr_matrix:
    assert fine.n == 2 * coarse.n
    rows, cols, vals = [], [], []
    for f, (a, b) in enumerate(fine.edges):
        xa, xb = fine.xyz[a], fine.xyz[b]
        mid = 0.5 * (xa + xb)
        t = locate_point(coarse.n, mid)
        for le in range(6):
            c = coarse.tet_edges[t, le]
            v = float(np.dot(whitney_field(coarse, t, le, mid), xb - xa))
            if abs(v) > 1e-13:
                rows.append(f)
                cols.append(c)
                vals.append(v)
    P = sp.coo_matrix((vals, (rows, cols)), shape=(len(fine.edges), len(coarse.edges))).tocsr()
    P.sum_duplicates()
    return P[fine.interior_edges][:, coarse.interior_edges].tocsr()


def node_prolongation(coarse: KuhnMesh, fine: KuhnMesh) -> sp.csr_matrix:
    assert fine.n == 2 * coarse.n
    rows, cols, vals = [], [], []
    for v, x in enumerate(fine.xyz):
        t = locate_point(coarse.n, x)
        lam = barycentric(coarse, t, x)
        for i in range(4):
            if abs(lam[i]) > 1e-13:
                rows.append(v)
                cols.append(coarse.tets[t, i])
                vals.append(lam[i])
    P = sp.coo_matrix((vals, (rows, cols)), shape=(len(fine.xyz), len(coarse.xyz))).tocsr()
    return P[fine.interior_verts][:, coarse.interior_verts].tocsr()


def round_dyadic(P: sp.csr_matrix, bits: int = 20) -> sp.csr_matrix:
    """Snap entries to the dyadic grid 2^-bits (entries are dyadic exactly; this
    removes the O(1e-16) noise of evaluating them through barycentric solves)."""
    Q = P.copy()
    Q.data = np.round(Q.data * (1 << bits)) / (1 << bits)
    Q.eliminate_zeros()
    return Q


def _first_tet_of(items_of_tet: np.ndarray, n_items: int) -> np.ndarray:
    """For every item (edge or vertex) the first tet, in tet order, that has it."""
    first = np.full(n_items, -1, dtype=np.int64)
    for t in range(len(items_of_tet)):
        for i in items_of_tet[t]:
            if first[i] < 0:
                first[i] = t
    return first


def edge_prolongation_nested(coarse, fine) -> sp.csr_matrix:
    """P_x between a mesh and its red refinement (fine.parent gives each fine tet's coarse
    tet): the same line integral of the coarse Whitney function as above, evaluated in the
    parent of a fine tet that contains the fine edge."""
    first = _first_tet_of(fine.tet_edges, len(fine.edges))
    rows, cols, vals = [], [], []
    for f, (a, b) in enumerate(fine.edges):
        xa, xb = fine.xyz[a], fine.xyz[b]
        mid = 0.5 * (xa + xb)
        t = int(fine.parent[first[f]])
        for le in range(6):
            v = float(np.dot(whitney_field(coarse, t, le, mid), xb - xa))
            if abs(v) > 1e-13:
                rows.append(f)
                cols.append(coarse.tet_edges[t, le])
                vals.append(v)
    P = sp.coo_matrix((vals, (rows, cols)), shape=(len(fine.edges), len(coarse.edges))).tocsr()
    P.sum_duplicates()
    return P[fine.interior_edges][:, coarse.interior_edges].tocsr()


def node_prolongation_nested(coarse, fine) -> sp.csr_matrix:
    """P1 interpolation between a mesh and its red refinement."""
    first = _first_tet_of(fine.tets, len(fine.xyz))
    rows, cols, vals = [], [], []
    for v, x in enumerate(fine.xyz):
        t = int(fine.parent[first[v]])
        lam = barycentric(coarse, t, x)
        for i in range(4):
            if abs(lam[i]) > 1e-13:
                rows.append(v)
                cols.append(coarse.tets[t, i])
                vals.append(lam[i])
    P = sp.coo_matrix((vals, (rows, cols)), shape=(len(fine.xyz), len(coarse.xyz))).tocsr()
    return P[fine.interior_verts][:, coarse.interior_verts].tocsr()
