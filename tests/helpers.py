"""Shared test helpers: layout conversion and oracle set-ups (test infrastructure)."""
import numpy as np

import st_inputs
from oracle.multigrid import SpaceTimeMG, build_time_hierarchy
from oracle.spacetime import ancestor_longest_edge, build_space_hierarchy, build_space_hierarchy_mesh

MODES = {0: "rule", 1: "semi_time", 2: "full_top"}


def to_lib(v):
    """Oracle (N_t, q, N_e) -> library layout (N_e, N_t*q)."""
    nt, q, ne = v.shape
    return np.ascontiguousarray(v.transpose(2, 0, 1).reshape(ne, nt * q))


def from_lib(v, q):
    """Library layout (N_e, N_t*q) -> oracle (N_t, q, N_e)."""
    ne, c = v.shape
    return np.ascontiguousarray(v.reshape(ne, c // q, q).transpose(1, 2, 0))


def rel(a, b):
    """Relative difference of a from b, the larger of the norm-wise ||a - b|| / ||b|| and
    the element-wise max |a - b| / max |b|: a block of wrong entries that a norm would
    average away (one bad supernode row block, one slab) still shows in the second."""
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    mb = np.max(np.abs(b)) if b.size else 0.0
    d = a - b
    norm_wise = np.linalg.norm(d) / (nb if nb > 0 else 1.0)
    elem_wise = (np.max(np.abs(d)) if d.size else 0.0) / (mb if mb > 0 else 1.0)
    return max(norm_wise, elem_wise)


def oracle_mg(n, nsl, nu, sigma, T, N_t, p, coarsen=0, max_levels=0, nu_pre=1, nu_post=1, lambda_crit=0.1,
              nodal="exact", jacobi_sweeps=0, use_A=True, omega=0.5, pattern="", bc=0):
    sl = build_space_hierarchy(n, nsl, nu, sigma, bc=("dirichlet", "neumann")[bc])
    tl = build_time_hierarchy(N_t, T, n, nsl, nu, sigma, mode=MODES[coarsen], lambda_crit=lambda_crit,
                              max_levels=max_levels if max_levels > 0 else 64)
    mg = SpaceTimeMG(sl, tl, p, omega, nu_pre, nu_post, nodal=nodal, jacobi_sweeps=jacobi_sweeps, use_A=use_A,
                     pattern=pattern)
    return sl, tl, mg


def oracle_mg_mesh(xyz, tets, n_refine, nsl, nu, sigma, T, N_t, p, coarsen=0, max_levels=0, nu_pre=1, nu_post=1,
                   lambda_crit=0.1, nodal="exact", jacobi_sweeps=0, omega=0.5, pattern="", bc=0):
    """oracle_mg on a general start mesh refined n_refine times (nu, sigma per finest tet)."""
    sl = build_space_hierarchy_mesh(xyz, tets, n_refine, nsl, nu, sigma, bc=("dirichlet", "neumann")[bc])
    tl = build_time_hierarchy(N_t, T, 0, nsl, nu, sigma, mode=MODES[coarsen], lambda_crit=lambda_crit,
                              max_levels=max_levels if max_levels > 0 else 64, h_levels=ancestor_longest_edge(sl))
    mg = SpaceTimeMG(sl, tl, p, omega, nu_pre, nu_post, nodal=nodal, jacobi_sweeps=jacobi_sweeps, pattern=pattern)
    return sl, tl, mg


def materials(n, kind, seed=0):
    return st_inputs.materials(n, kind, seed)
