"""Right-hand side of the space-time system from the source J (CPU oracle).

TEST INFRASTRUCTURE ONLY (see oracle/mesh.py).

Section 3 (semi-variational form) puts int_Omega f(t) . v on the right; Section 2.1
integrates it over each time step.  With J(x, t) = g(t) j(x) separable,
    f[n, i, e] = (int_{I_n} g(t) phi_i(t) dt) * (int_Omega j(x) . w_e(x) dx),
the time integral by 3-point Gauss-Legendre per slab and the space integral by
the symmetric 4-point degree-2 tet rule (barycentric (a, b, b, b), a = (5+3 sqrt5)/20,
b = (5 - sqrt5)/20, weights |T|/4), both our fixed quadrature choices.
j(x) = curl psi(x) = sum_m pi cos(pi k_m . x + phi_m) (k_m x a_m).
"""
from __future__ import annotations

import numpy as np

from .mesh import KuhnMesh, LOCAL_EDGES
from .fem import tet_geometry, _local_orientation
from .timeblocks import time_load_weights


def source_space(x, exc):
    """j(x) for points x (npts, 3)."""
    a, k, ph = exc["a"], exc["k"], exc["phase"]
    out = np.zeros_like(x)
    for m in range(len(ph)):
        amp = np.pi * np.cos(np.pi * x @ k[m] + ph[m])
        out += amp[:, None] * np.cross(k[m], a[m])[None, :]
    return out


def source_time(t, T):
    return np.sin(np.pi * t / T) + 1.0


def space_load(mesh: KuhnMesh, exc) -> np.ndarray:
    """b[e] on interior edges."""
    vol, g = tet_geometry(mesh)
    tail, head = _local_orientation(mesh)
    sq5 = np.sqrt(5.0)
    alpha, beta = (5 + 3 * sq5) / 20, (5 - sq5) / 20
    P = mesh.xyz[mesh.tets]
    b = np.zeros(len(mesh.edges))
    idx = np.arange(len(mesh.tets))
    for q in range(4):
        lam = np.full(4, beta)
        lam[q] = alpha
        x = np.einsum("v,tvd->td", lam, P)
        jx = source_space(x, exc)
        for le in range(6):
            ta, hb = tail[:, le], head[:, le]
            w = lam[ta][:, None] * g[idx, hb] - lam[hb][:, None] * g[idx, ta]
            np.add.at(b, mesh.tet_edges[:, le], vol / 4 * np.einsum("td,td->t", jx, w))
    return b[mesh.interior_edges]


def spacetime_load(mesh: KuhnMesh, exc, p: int, N_t: int, T: float) -> np.ndarray:
    b = space_load(mesh, exc)
    c = time_load_weights(p, N_t, T, lambda t: source_time(t, T))
    return c[:, :, None] * b[None, None, :]
