"""Space-time V-cycle with the hybrid smoother (CPU oracle).

TEST INFRASTRUCTURE ONLY (see oracle/mesh.py).

Section 2.1: pre-smoothing, a recursive coarse time-grid correction, then
post-smoothing; the coarse level halves the number of slabs (tau doubles).
Section 2.2 (eq. CoarseningRule): the coarse level also uses the next coarser
spatial mesh iff  min_T nu_T tau / (sigma_T h_T^2) >= lambda_crit  with h_T the
longest tet edge (sqrt(3)/n for every Kuhn tet); otherwise only time is coarsened.
Section 4: the hybrid smoother is S^nu A S^nu (A = nodal correction applied
once, between the block-Jacobi sweeps S), the same sequence before and after
the coarse correction.  The coarsest level is solved exactly: one slab by the
slab factor, more slabs by forward substitution.

Modes of the hierarchy: "rule" (eq. CoarseningRule), "semi_time" (never coarsen
space) and "full_top" (coarsen space on the first transition only, Table FullMethod).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .spacetime import (SlabOperator, apply_L, smoother_S, correction_A, sequential_solve,
                        restrict_time, prolong_time, restrict_space, prolong_space)


@dataclass
class TimeLevel:
    s: int        # spatial level index (0 = finest)
    N_t: int
    tau: float


def coarsening_lambda(n_space: int, tau: float, nu, sigma) -> float:
    """lambda of eq. CoarseningRule on a Kuhn mesh with n_space cubes per side.

    nu, sigma are per finest tet; a coarser tet's minimum over its points is the
    minimum over the finest tets it contains, and all Kuhn tets of one mesh share
    the longest edge sqrt(3)/n_space, so the rule's minimum is global.
    """
    h = np.sqrt(3.0) / n_space
    return float(np.min(np.asarray(nu) / np.asarray(sigma)) * tau / h ** 2)


def coarsening_lambda_mesh(h_anc, tau: float, nu, sigma) -> float:
    """lambda of eq. CoarseningRule on a general mesh: h_anc[t] is the longest edge of the
    tet of that level containing finest tet t, nu and sigma are per finest tet."""
    return float(np.min(np.asarray(nu) / (np.asarray(sigma) * np.asarray(h_anc) ** 2)) * tau)


def build_time_hierarchy(N_t, T, n_fine, n_space_levels, nu, sigma, mode="rule",
                         lambda_crit=0.1, min_coarse_slabs=1, max_levels=64, h_levels=None):
    """n_fine: Kuhn cubes per side of the finest mesh; on a general mesh h_levels[s] gives,
    per finest tet, the longest edge of its ancestor on space level s (n_fine unused)."""
    levels = [TimeLevel(0, N_t, T / N_t)]
    while len(levels) < max_levels:
        cur = levels[-1]
        if cur.N_t <= min_coarse_slabs or cur.N_t % 2:
            break
        n_cur = n_fine >> cur.s
        can_space = cur.s + 1 < n_space_levels
        if mode == "rule":
            lam = (coarsening_lambda(n_cur, cur.tau, nu, sigma) if h_levels is None
                   else coarsening_lambda_mesh(h_levels[cur.s], cur.tau, nu, sigma))
            coarsen = can_space and lam >= lambda_crit
        elif mode == "semi_time":
            coarsen = False
        elif mode == "full_top":
            coarsen = can_space and len(levels) == 1
        else:
            raise ValueError(mode)
        levels.append(TimeLevel(cur.s + int(coarsen), cur.N_t // 2, cur.tau * 2))
    return levels


class SpaceTimeMG:
    def __init__(self, space_levels, time_levels, p, omega=0.5, nu_pre=1, nu_post=1,
                 nodal="exact", jacobi_sweeps=0, use_A=True, pattern=""):
        self.space, self.levels, self.p = space_levels, time_levels, p
        self.use_A = use_A
        # Section 4: a hybrid smoother written as a product of S and A, read right to
        # left ("SA": A, then S); the post-smoother applies the same factors in the
        # reverse order.  Empty: S^nu A S^nu with nu = nu_pre / nu_post.
        if any(c not in "SA" for c in pattern):
            raise ValueError(pattern)
        self.pattern = pattern
        self.omega, self.nu_pre, self.nu_post = omega, nu_pre, nu_post
        self.nodal, self.jacobi_sweeps = nodal, jacobi_sweeps
        self.slabs = [SlabOperator(space_levels[L.s], p, L.tau) for L in time_levels]

    def _apply(self, li, f, x, op):
        slab = self.slabs[li]
        if op == "S":
            return smoother_S(slab, f, x, self.omega)
        return correction_A(slab, f, x, self.nodal, self.jacobi_sweeps)

    # one level's smoothing sequence: the pattern (pre: right to left, post: left to
    # right), else S^k A S^k
    def _smooth(self, li, f, x, k, post=False):
        if self.pattern:
            for op in (self.pattern if post else self.pattern[::-1]):
                x = self._apply(li, f, x, op)
            return x
        slab = self.slabs[li]
        for _ in range(k):
            x = smoother_S(slab, f, x, self.omega)
        if self.use_A:
            x = correction_A(slab, f, x, self.nodal, self.jacobi_sweeps)
        for _ in range(k):
            x = smoother_S(slab, f, x, self.omega)
        return x

    def residual(self, li, f, x):
        s = self.slabs[li]
        return f - apply_L(s.space, s.Kt, s.Mt, s.Nt, x)

    def vcycle(self, f, x, li=0):
        slab = self.slabs[li]
        if li == len(self.levels) - 1:
            return sequential_solve(slab, f)
        x = self._smooth(li, f, x, self.nu_pre)
        r = self.residual(li, f, x)
        rc = restrict_time(self.p, r)
        coarse = self.levels[li + 1]
        space_coarsened = coarse.s != self.levels[li].s
        if space_coarsened:
            rc = restrict_space(self.space[self.levels[li].s].Px, rc)
        ec = self.vcycle(rc, np.zeros_like(rc), li + 1)
        if space_coarsened:
            ec = prolong_space(self.space[self.levels[li].s].Px, ec)
        x = x + prolong_time(self.p, ec)
        x = self._smooth(li, f, x, self.nu_post, post=True)
        return x

    def solve(self, f, x0=None, rtol=1e-8, maxit=50):
        x = np.zeros_like(f) if x0 is None else x0.copy()
        nf = np.linalg.norm(f)
        hist = [np.linalg.norm(self.residual(0, f, x)) / nf]
        while hist[-1] > rtol and len(hist) <= maxit:
            x = self.vcycle(f, x)
            hist.append(np.linalg.norm(self.residual(0, f, x)) / nf)
        return x, hist

    def convergence_rate(self, x0, max_iter=200, floor=1e-100):
        """Section 5.1 power iteration: f = 0, the largest per-iteration reduction
        of the l2 norm; stops when the total reduction falls below `floor`."""
        f = np.zeros_like(x0)
        x = x0.copy()
        n0 = nprev = np.linalg.norm(x)
        rates = []
        for _ in range(max_iter):
            x = self.vcycle(f, x)
            nx = np.linalg.norm(x)
            rates.append(nx / nprev)
            nprev = nx
            if nx / n0 < floor or nx == 0.0:
                break
        return max(rates), rates
