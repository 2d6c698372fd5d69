"""Edge-element (lowest-order Nedelec) and nodal (P1) matrices (CPU oracle).

TEST INFRASTRUCTURE ONLY (see oracle/mesh.py).

Section 3 (below eq. EddyCurrent) defines the two spatial matrices of the
discrete eddy-current problem through the Nedelec basis (phi_i):
    (M_h)_ij = int sigma phi_i . phi_j,    (K_h)_ij = int mu^{-1} curl phi_i . curl phi_j.
The oracle writes the Whitney basis out directly: for the edge a -> b of a tet,
    w_ab = lam_a grad lam_b - lam_b grad lam_a,   curl w_ab = 2 grad lam_a x grad lam_b,
with lam the barycentric coordinates, and integrates products of barycentric
coordinates with  int_T lam_i lam_j = |T| (1 + delta_ij) / 20.
Coefficients are constant per tet.  nu = mu^{-1} throughout.

Section 3.3 (eq. AuxNodalSm) needs the discrete gradient G from the H^1 (P1)
space into the Nedelec space and K_n, the nodal stiffness matrix of div sigma grad.
G has -1 at the tail and +1 at the head of every edge.  K_n is assembled here
directly from the P1 basis, so that the identity K_n = G^T M_sigma G is a check,
not a definition.

Dirichlet conditions (u x n = 0) remove the boundary edges and nodes; all
matrices below are returned on the interior degrees of freedom.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import KuhnMesh, LOCAL_EDGES


def tet_geometry(mesh: KuhnMesh):
    """Volumes (nt,) and barycentric gradients (nt, 4, 3) of every tet."""
    P = mesh.xyz[mesh.tets]                      # (nt, 4, 3)
    D = P[:, 1:, :] - P[:, :1, :]                # rows: v1-v0, v2-v0, v3-v0
    vol = np.abs(np.linalg.det(D)) / 6.0
    Dinv = np.linalg.inv(D)                      # columns: grad lam_1..3
    grads = np.zeros((len(P), 4, 3))
    grads[:, 1:, :] = np.transpose(Dinv, (0, 2, 1))
    grads[:, 0, :] = -grads[:, 1:, :].sum(axis=1)
    return vol, grads


def _local_orientation(mesh: KuhnMesh):
    """For each tet and local edge: (tail local index, head local index)."""
    nt = len(mesh.tets)
    tail = np.zeros((nt, 6), dtype=np.int64)
    head = np.zeros((nt, 6), dtype=np.int64)
    for le, (a, b) in enumerate(LOCAL_EDGES):
        va, vb = mesh.tets[:, a], mesh.tets[:, b]
        forward = va < vb
        tail[:, le] = np.where(forward, a, b)
        head[:, le] = np.where(forward, b, a)
    return tail, head


def element_matrices(mesh: KuhnMesh, nu: np.ndarray, sigma: np.ndarray):
    """Element mass (sigma) and curl-curl (nu) matrices, each (nt, 6, 6)."""
    vol, g = tet_geometry(mesh)
    tail, head = _local_orientation(mesh)
    nt = len(mesh.tets)
    Me = np.zeros((nt, 6, 6))
    Ke = np.zeros((nt, 6, 6))
    idx = np.arange(nt)

    def lamlam(i, j):  # int_T lam_i lam_j / |T|
        return np.where(i == j, 2.0, 1.0) / 20.0

    for p in range(6):
        a, b = tail[:, p], head[:, p]
        ga, gb = g[idx, a], g[idx, b]
        curl_p = 2.0 * np.cross(ga, gb)
        for q in range(6):
            c, d = tail[:, q], head[:, q]
            gc, gd = g[idx, c], g[idx, d]
            dot = lambda u, v: np.einsum("ij,ij->i", u, v)
            m = (lamlam(a, c) * dot(gb, gd) - lamlam(a, d) * dot(gb, gc)
                 - lamlam(b, c) * dot(ga, gd) + lamlam(b, d) * dot(ga, gc))
            Me[:, p, q] = sigma * vol * m
            curl_q = 2.0 * np.cross(gc, gd)
            Ke[:, p, q] = nu * vol * dot(curl_p, curl_q)
    return Me, Ke


def assemble_edge_matrices(mesh: KuhnMesh, nu, sigma, interior: bool = True):
    """Global M_sigma and K_nu (CSR, float64), on interior edges unless interior=False."""
    Me, Ke = element_matrices(mesh, np.asarray(nu, float), np.asarray(sigma, float))
    ne = len(mesh.edges)
    rows = np.repeat(mesh.tet_edges, 6, axis=1).ravel()
    cols = np.tile(mesh.tet_edges, (1, 6)).ravel()
    M = sp.coo_matrix((Me.ravel(), (rows, cols)), shape=(ne, ne)).tocsr()
    K = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(ne, ne)).tocsr()
    if not interior:
        return M, K
    ie = mesh.interior_edges
    return M[ie][:, ie].tocsr(), K[ie][:, ie].tocsr()


def discrete_gradient(mesh: KuhnMesh, interior: bool = True):
    """G: nodal (P1) coefficients -> edge coefficients, -1 at tail, +1 at head."""
    ne, nv = len(mesh.edges), len(mesh.xyz)
    r = np.repeat(np.arange(ne), 2)
    c = mesh.edges.ravel()
    v = np.tile([-1.0, 1.0], ne)
    G = sp.coo_matrix((v, (r, c)), shape=(ne, nv)).tocsr()
    if interior:
        G = G[mesh.interior_edges][:, mesh.interior_verts].tocsr()
    return G


def nodal_stiffness(mesh: KuhnMesh, sigma):
    """P1 stiffness of -div(sigma grad) on interior nodes, assembled from the P1 basis."""
    vol, g = tet_geometry(mesh)
    sigma = np.asarray(sigma, float)
    Ke = sigma[:, None, None] * vol[:, None, None] * np.einsum("tid,tjd->tij", g, g)
    nv = len(mesh.xyz)
    rows = np.repeat(mesh.tets, 4, axis=1).ravel()
    cols = np.tile(mesh.tets, (1, 4)).ravel()
    K = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(nv, nv)).tocsr()
    iv = mesh.interior_verts
    return K[iv][:, iv].tocsr()


def whitney_field(mesh: KuhnMesh, t: int, le: int, x: np.ndarray) -> np.ndarray:
    """Value at point x of the global-oriented Whitney function of local edge le of tet t."""
    vol, g = tet_geometry_one(mesh, t)
    lam = barycentric(mesh, t, x)
    a, b = LOCAL_EDGES[le]
    va, vb = mesh.tets[t, a], mesh.tets[t, b]
    if va > vb:
        a, b = b, a
    return lam[a] * g[b] - lam[b] * g[a]


def tet_geometry_one(mesh: KuhnMesh, t: int):
    P = mesh.xyz[mesh.tets[t]]
    D = P[1:] - P[:1]
    Dinv = np.linalg.inv(D)
    g = np.zeros((4, 3))
    g[1:] = Dinv.T
    g[0] = -g[1:].sum(axis=0)
    return abs(np.linalg.det(D)) / 6.0, g


def barycentric(mesh: KuhnMesh, t: int, x: np.ndarray) -> np.ndarray:
    P = mesh.xyz[mesh.tets[t]]
    D = (P[1:] - P[:1]).T
    l123 = np.linalg.solve(D, np.asarray(x, float) - P[0])
    return np.concatenate([[1.0 - l123.sum()], l123])
