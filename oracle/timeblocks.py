"""Discontinuous-Galerkin-in-time blocks and time transfers (CPU oracle).

TEST INFRASTRUCTURE ONLY (see oracle/mesh.py).

Section 2.1 (eq. timeStepping) states the method for implicit Euler:
    -M u^k + (M + tau K) u^{k+1} = tau f^{k+1},
i.e. a block lower-bidiagonal space-time matrix with A_tau = M + tau K on the
diagonal and -M below it.  Implicit Euler is DG(0) in time.  The configurations
also use DG(1); the paper only writes the Euler case and refers to its cited
space-time framework for the rest, so the oracle takes the standard upwind DG(p)
discretisation (reading recorded in the design notes):
on slab I_n = (t_{n-1}, t_n) with local coordinate s in [0, 1] and basis
phi_0 = 1, phi_1 = 2s - 1 (Legendre), test index i, trial index j,
    K_t[i,j] = int_0^1 phi_j' phi_i ds + phi_j(0) phi_i(0)   (time derivative + inflow jump)
    M_t[i,j] = tau int_0^1 phi_j phi_i ds
    N_t[i,j] = -phi_j(1) phi_i(0)                              (coupling to slab n-1)
and the slab block is K_t (x) M_sigma + M_t (x) K_nu, the coupling block N_t (x) M_sigma.
For p = 0 this is exactly eq. timeStepping.

The blocks are computed here by exact Gauss-Legendre quadrature of the
polynomials above, not typed in.
"""
from __future__ import annotations

import numpy as np


def _basis(p: int, s: np.ndarray):
    """Legendre basis on [0,1] and derivatives, degree <= 1."""
    s = np.asarray(s, float)
    if p == 0:
        return np.ones((1,) + s.shape), np.zeros((1,) + s.shape)
    if p == 1:
        return np.stack([np.ones_like(s), 2 * s - 1]), np.stack([np.zeros_like(s), 2 * np.ones_like(s)])
    raise ValueError("degree must be 0 or 1")


def time_blocks(p: int, tau: float):
    """Return (K_t, M_t, N_t), each (p+1, p+1), rows = test, cols = trial."""
    xg, wg = np.polynomial.legendre.leggauss(4)
    s, w = 0.5 * (xg + 1), 0.5 * wg
    phi, dphi = _basis(p, s)
    phi0, _ = _basis(p, np.array(0.0))
    phi1, _ = _basis(p, np.array(1.0))
    q = p + 1
    Kt = np.zeros((q, q))
    Mt = np.zeros((q, q))
    Nt = np.zeros((q, q))
    for i in range(q):
        for j in range(q):
            Kt[i, j] = np.sum(w * dphi[j] * phi[i]) + phi0[j] * phi0[i]
            Mt[i, j] = tau * np.sum(w * phi[j] * phi[i])
            Nt[i, j] = -phi1[j] * phi0[i]
    return Kt, Mt, Nt


def time_prolongation_block(p: int):
    """Coarse slab -> its two fine halves: (P_first, P_second), each (p+1, p+1).

    P_half[i_f, j_c] = coefficients of coarse basis function j_c restricted to
    the fine half, expanded in the fine basis (exact L2 projection of a
    polynomial that already lies in the fine space).
    """
    xg, wg = np.polynomial.legendre.leggauss(4)
    s, w = 0.5 * (xg + 1), 0.5 * wg
    phi_f, _ = _basis(p, s)
    gram = np.einsum("iq,jq,q->ij", phi_f, phi_f, w)
    blocks = []
    for half in (0, 1):
        sc = 0.5 * (s + half)                 # coarse coordinate of fine point s
        phi_c, _ = _basis(p, sc)
        rhs = np.einsum("iq,jq,q->ij", phi_f, phi_c, w)
        blocks.append(np.linalg.solve(gram, rhs))
    return blocks[0], blocks[1]


def time_load_weights(p: int, N_t: int, T: float, g, nquad: int = 3):
    """c[n, i] = int_{I_n} g(t) phi_i dt by nquad-point Gauss-Legendre per slab."""
    tau = T / N_t
    xg, wg = np.polynomial.legendre.leggauss(nquad)
    s, w = 0.5 * (xg + 1), 0.5 * wg
    phi, _ = _basis(p, s)
    c = np.zeros((N_t, p + 1))
    for n in range(N_t):
        t = n * tau + s * tau
        for i in range(p + 1):
            c[n, i] = tau * np.sum(w * g(t) * phi[i])
    return c
