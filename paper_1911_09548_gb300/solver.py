"""Convenience wrapper around one library handle with torch CUDA buffers.

Marshalling only: every method is one C-ABI call (include/st_mg.h).  torch
provides device memory and the current CUDA stream.
"""
from __future__ import annotations

import numpy as np

from . import binding as B


class SpaceTimeSolver:
    def __init__(self, n_cube, nu, sigma, T, N_t, degree, n_space_levels=1, stream=None, host_only=False,
                 n_batch=1, bc=0, mesh=None, batch_nt=None, **options):
        """n_cube: Kuhn cubes per side, or mesh = (xyz, tets, n_refine) for a general start mesh
        refined n_refine times (n_cube ignored; nu, sigma per finest tet, child k of tet t = 8 t + k).
        batch_nt: per-problem slab counts of a ragged batch (N_t divided by powers of two)."""
        self.prob = B.make_problem(n_cube, n_space_levels, nu, sigma, T, N_t, degree, n_batch, bc, mesh, batch_nt)
        self.n_batch = n_batch
        self.batch_nt = None if batch_nt is None else [int(v) for v in batch_nt]
        self.opt = B.st_mg_default_options()
        for k, v in options.items():
            if not hasattr(self.opt, k):
                raise KeyError(k)
            setattr(self.opt, k, v.encode() if isinstance(v, str) else v)
        self.host_only = host_only
        if host_only:
            self.h = B.st_mg_setup_host(self.prob, self.opt)
            self.stream = 0
        else:
            import torch
            if stream is None:
                stream = torch.cuda.current_stream().cuda_stream
            self.stream = stream
            self.h = B.st_mg_setup(self.prob, self.opt, stream)
        self.n_edge, self.n_node, self.n_dof, self.n_levels = B.st_mg_sizes(self.h)
        self.degree, self.q = degree, degree + 1
        self.levels = [B.st_mg_level_info(self.h, l) for l in range(self.n_levels)]

    def close(self):
        if getattr(self, "h", None):
            B.st_mg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- buffers
    def level_shape(self, level=0, nodal=False):
        """Shape of a vector of a level; level 0 of a ragged batch: the caller's layout (the
        problems' own slab counts one after the other per edge row)."""
        L = self.levels[level]
        rows = L["n_node"] if nodal else L["n_edge"]
        if self.batch_nt is not None and level == 0:
            return (rows, sum(self.batch_nt) * self.q)
        return (rows, self.n_batch * L["N_t"] * self.q)

    def problem_cols(self, b):
        """Columns of problem b in a caller's vector (ragged or not)."""
        nts = self.batch_nt or [self.levels[0]["N_t"]] * self.n_batch
        a = sum(nts[:b]) * self.q
        return slice(a, a + nts[b] * self.q)

    def zeros(self, level=0, nodal=False):
        import torch
        return torch.zeros(self.level_shape(level, nodal), dtype=torch.float64, device="cuda")

    # ---- C-ABI calls
    def load(self, exc, f=None, batch=0):
        f = self.zeros() if f is None else f
        B.st_mg_assemble_load_batch(self.h, batch, exc["a"], exc["k"], exc["phase"], f)
        return f

    def residual(self, f, x, r=None, level=0, want_norm=False):
        r = self.zeros(level) if r is None else r
        nrm = B.st_mg_residual(self.h, level, f, x, r, want_norm)
        return (r, nrm) if want_norm else r

    def slab_solve(self, r, level=0):
        y = self.zeros(level)
        B.st_mg_slab_solve(self.h, level, r, y)
        return y

    def smooth_S(self, f, x, level=0):
        B.st_mg_smooth_S(self.h, level, f, x)

    def correct_A(self, f, x, level=0):
        B.st_mg_correct_A(self.h, level, f, x)

    def grad_T(self, r, level=0):
        y = self.zeros(level, nodal=True)
        B.st_mg_grad_T(self.h, level, r, y)
        return y

    def nodal_solve(self, y, level=0):
        z = self.zeros(level, nodal=True)
        B.st_mg_nodal_solve(self.h, level, y, z)
        return z

    def time_integrate(self, z, level=0):
        w = self.zeros(level, nodal=True)
        B.st_mg_time_integrate(self.h, level, z, w)
        return w

    def grad_add(self, w, x, level=0):
        B.st_mg_grad_add(self.h, level, w, x)

    def restrict(self, r, level=0):
        rc = self.zeros(level + 1)
        B.st_mg_restrict(self.h, level, r, rc)
        return rc

    def prolong_add(self, ec, x, level=0):
        B.st_mg_prolong_add(self.h, level, ec, x)

    def coarse_solve(self, f):
        x = self.zeros(self.n_levels - 1)
        B.st_mg_coarse_solve(self.h, f, x)
        return x

    def vcycle(self, f, x, want_res=False):
        return B.st_mg_vcycle(self.h, f, x, want_res)

    def solve(self, f, x, rtol=1e-8, maxit=50):
        return B.st_mg_solve(self.h, f, x, rtol, maxit)

    def solve_host(self, f_host: np.ndarray, x_host: np.ndarray, rtol=1e-8, maxit=50):
        return B.st_mg_solve_host(self.h, f_host, x_host, rtol, maxit)

    def convergence_rate(self, x0, max_iter=200, floor=1e-100):
        """Section 5.1's power iteration (st_mg_convergence_rate): V-cycles with f = 0 from
        the start x0 (device tensor, overwritten); returns (largest per-cycle reduction of
        the l2 norm, all per-cycle reductions)."""
        import torch
        # x0 was written on torch's current stream; the V-cycles run on the handle's
        torch.cuda.current_stream().synchronize()
        return B.st_mg_convergence_rate(self.h, x0, max_iter, floor)

    def debug(self, what, space_level=0):
        return B.st_mg_debug_get(self.h, what, space_level)

    def host_slab_solve(self, r_host, level=0):
        return B.st_mg_debug_host_slab_solve(self.h, level, r_host)
