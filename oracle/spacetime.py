"""Space-time operators of the all-at-once system (CPU oracle).

TEST INFRASTRUCTURE ONLY (see oracle/mesh.py).

Vectors are arrays of shape (N_t, p+1, N_e): slab n, time basis index i, interior
edge e.  (The C library stores the same numbers edge-major; the tests convert.)

  * apply_L        : the block lower-bidiagonal matrix L_{tau,h} of Section 2.1,
                     diagonal K_t (x) M + M_t (x) K, sub-diagonal N_t (x) M.
  * slab solve     : A_slab^{-1} with A_slab = K_t (x) M + M_t (x) K, factorised
                     once per (space level, tau) by SuperLU on the real
                     (p+1) N_e system (no complex transformation here).
  * smoother_S     : eq. StandardSmoother, x <- x + omega (I (x) A^{-1})(f - L x).
  * correction_A   : eq. AuxNodalSm, x <- x + G Sigma_t K_n^{-1} G^T (f - L x);
                     for DG(p) Sigma_t generalises to L_t^{-1}, the inverse of the
                     time-only bidiagonal matrix (K_t diagonal, N_t below), because
                     G^T L G = L_t (x) K_n exactly (G^T K_nu G = 0, G^T M G = K_n).
  * time/space transfers of the coarse-grid correction (Section 2.1, 2.2).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .mesh import KuhnMesh, kuhn_mesh, refine_times
from .fem import assemble_edge_matrices, discrete_gradient, nodal_stiffness
from .transfer import (edge_prolongation, edge_prolongation_nested, node_prolongation,
                       node_prolongation_nested, round_dyadic)
from .timeblocks import time_blocks, time_prolongation_block

NODAL_JACOBI_WEIGHT = 2.0 / 3.0  # damping of the nodal Jacobi variant (our constant)


@dataclass
class SpaceLevel:
    mesh: KuhnMesh
    M: sp.csr_matrix
    K: sp.csr_matrix
    G: sp.csr_matrix
    Kn: sp.csr_matrix
    Px: sp.csr_matrix | None = None   # prolongation from the next coarser space level
    Pn: sp.csr_matrix | None = None
    _kn_lu: object = None

    @property
    def ne(self):
        return self.M.shape[0]

    @property
    def nn(self):
        return self.Kn.shape[0]

    def kn_solve(self, y):
        if self._kn_lu is None:
            self._kn_lu = spla.splu(self.Kn.tocsc())
        return self._kn_lu.solve(y)


def build_space_hierarchy(n_fine: int, n_levels: int, nu, sigma, bc: str = "dirichlet"):
    """Space levels, finest first.  nu, sigma are per tet of the finest mesh; bc is
    "dirichlet" or "neumann" (which unknowns, see oracle.mesh).

    The finest matrices are assembled from the element integrals; each coarser
    level uses Galerkin products with the interpolation prolongations (the
    coefficients vary per fine tet, so re-discretisation would be ambiguous).
    """
    levels = []
    mesh = kuhn_mesh(n_fine, bc)
    M, K = assemble_edge_matrices(mesh, nu, sigma)
    G = discrete_gradient(mesh)
    Kn = nodal_stiffness(mesh, sigma)
    levels.append(SpaceLevel(mesh, M, K, G, Kn))
    n = n_fine
    for _ in range(1, n_levels):
        assert n % 2 == 0
        cmesh = kuhn_mesh(n // 2, bc)
        fine = levels[-1]
        Px = round_dyadic(edge_prolongation(cmesh, fine.mesh))
        Pn = round_dyadic(node_prolongation(cmesh, fine.mesh))
        fine.Px, fine.Pn = Px, Pn
        Mc = (Px.T @ fine.M @ Px).tocsr()
        Kc = (Px.T @ fine.K @ Px).tocsr()
        Gc = discrete_gradient(cmesh)
        Knc = (Pn.T @ fine.Kn @ Pn).tocsr()
        levels.append(SpaceLevel(cmesh, Mc, Kc, Gc, Knc))
        n //= 2
    return levels


def build_space_hierarchy_mesh(xyz, tets, n_refine: int, n_levels: int, nu, sigma, bc: str = "dirichlet"):
    """Space levels, finest first, of a general start mesh (xyz, tets) refined n_refine
    times (oracle.mesh conventions); nu, sigma per tet of the finest mesh.  Matrices as in
    build_space_hierarchy: assembled on the finest mesh, Galerkin below it."""
    assert 1 <= n_levels <= n_refine + 1
    meshes = refine_times(xyz, tets, n_refine, bc)[::-1]     # finest first
    mesh = meshes[0]
    M, K = assemble_edge_matrices(mesh, nu, sigma)
    levels = [SpaceLevel(mesh, M, K, discrete_gradient(mesh), nodal_stiffness(mesh, sigma))]
    for s in range(1, n_levels):
        cmesh, fine = meshes[s], levels[-1]
        Px = round_dyadic(edge_prolongation_nested(cmesh, fine.mesh))
        Pn = round_dyadic(node_prolongation_nested(cmesh, fine.mesh))
        fine.Px, fine.Pn = Px, Pn
        levels.append(SpaceLevel(cmesh, (Px.T @ fine.M @ Px).tocsr(), (Px.T @ fine.K @ Px).tocsr(),
                                 discrete_gradient(cmesh), (Pn.T @ fine.Kn @ Pn).tocsr()))
    return levels


def ancestor_longest_edge(levels) -> list:
    """Per space level s: for every finest tet, the longest edge of its ancestor on level s
    (h_T of eq. CoarseningRule on the coarser mesh; nu, sigma stay per finest tet)."""
    out = []
    anc = np.arange(len(levels[0].mesh.tets))
    for s, L in enumerate(levels):
        if s > 0:
            anc = levels[s - 1].mesh.parent[anc]
        out.append(L.mesh.longest_edge[anc])
    return out


class SlabOperator:
    """A_slab = K_t (x) M + M_t (x) K and its exact inverse (SuperLU, real)."""

    def __init__(self, space: SpaceLevel, p: int, tau: float):
        self.space, self.p, self.tau = space, p, tau
        self.Kt, self.Mt, self.Nt = time_blocks(p, tau)
        A = sp.kron(self.Kt, space.M) + sp.kron(self.Mt, space.K)
        self.A = A.tocsc()
        self.lu = spla.splu(self.A)

    def solve(self, g):
        """g: (..., p+1, N_e) -> A_slab^{-1} g, slab by slab."""
        q, ne = self.p + 1, self.space.ne
        flat = g.reshape(-1, q * ne).T
        return self.lu.solve(np.ascontiguousarray(flat)).T.reshape(g.shape)


def apply_L(space: SpaceLevel, Kt, Mt, Nt, x):
    """L x for x of shape (N_t, q, N_e)."""
    Nt_, q, ne = x.shape
    X = x.reshape(-1, ne).T                       # (ne, N_t*q)
    Mx = (space.M @ X).T.reshape(Nt_, q, ne)
    Kx = (space.K @ X).T.reshape(Nt_, q, ne)
    y = np.einsum("ij,nje->nie", Kt, Mx) + np.einsum("ij,nje->nie", Mt, Kx)
    y[1:] += np.einsum("ij,nje->nie", Nt, Mx[:-1])
    return y


def residual(space, Kt, Mt, Nt, f, x):
    return f - apply_L(space, Kt, Mt, Nt, x)


def sequential_solve(slab: SlabOperator, f):
    """Time stepping: x_n = A_slab^{-1}(f_n - (N_t (x) M) x_{n-1}), x_0-history = 0."""
    x = np.zeros_like(f)
    M = slab.space.M
    for n in range(f.shape[0]):
        g = f[n].copy()
        if n > 0:
            Mxp = (M @ x[n - 1].T).T
            g -= slab.Nt @ Mxp
        x[n] = slab.solve(g[None])[0]
    return x


def smoother_S(slab: SlabOperator, f, x, omega):
    r = residual(slab.space, slab.Kt, slab.Mt, slab.Nt, f, x)
    return x + omega * slab.solve(r)


def time_integrate(Kt, Nt, z):
    """w = L_t^{-1} z along time, L_t = bidiag(K_t, N_t); z: (N_t, q, N_n)."""
    w = np.zeros_like(z)
    Ktinv = np.linalg.inv(Kt)
    for n in range(z.shape[0]):
        rhs = z[n] - (Nt @ w[n - 1] if n > 0 else 0.0)
        w[n] = Ktinv @ rhs
    return w


def correction_A(slab: SlabOperator, f, x, nodal="exact", jacobi_sweeps=0):
    sp_ = slab.space
    r = residual(sp_, slab.Kt, slab.Mt, slab.Nt, f, x)
    Nt_, q, ne = r.shape
    y = (sp_.G.T @ r.reshape(-1, ne).T)           # (nn, N_t*q)
    if nodal == "exact":
        z = sp_.kn_solve(np.ascontiguousarray(y))
    else:
        d = sp_.Kn.diagonal()[:, None]
        z = np.zeros_like(y)
        for _ in range(jacobi_sweeps):
            z = z + NODAL_JACOBI_WEIGHT * (y - sp_.Kn @ z) / d
    z = z.T.reshape(Nt_, q, -1)
    w = time_integrate(slab.Kt, slab.Nt, z)
    return x + (sp_.G @ w.reshape(-1, sp_.nn).T).T.reshape(Nt_, q, ne)


def restrict_time(p, r):
    P0, P1 = time_prolongation_block(p)
    return np.einsum("ji,nje->nie", P0, r[0::2]) + np.einsum("ji,nje->nie", P1, r[1::2])


def prolong_time(p, e):
    P0, P1 = time_prolongation_block(p)
    Nc, q, ne = e.shape
    out = np.zeros((2 * Nc, q, ne))
    out[0::2] = np.einsum("ij,nje->nie", P0, e)
    out[1::2] = np.einsum("ij,nje->nie", P1, e)
    return out


def restrict_space(Px, r):
    Nt_, q, ne = r.shape
    return (Px.T @ r.reshape(-1, ne).T).T.reshape(Nt_, q, -1)


def prolong_space(Px, e):
    Nt_, q, nc = e.shape
    return (Px @ e.reshape(-1, nc).T).T.reshape(Nt_, q, -1)


def spacetime_matrix(space: SpaceLevel, p: int, tau: float, N_t: int) -> sp.csr_matrix:
    """The whole L_{tau,h} as one sparse matrix (tiny problems only)."""
    Kt, Mt, Nt = time_blocks(p, tau)
    diag = sp.kron(Kt, space.M) + sp.kron(Mt, space.K)
    sub = sp.kron(Nt, space.M)
    L = sp.kron(sp.identity(N_t), diag) + sp.kron(sp.diags([np.ones(N_t - 1)], [-1]), sub)
    return L.tocsr()
