"""Request loop over the library (include/st_mg_serve.h): marshalling only.

The scheduler (class handles, slots, admission by device memory, one stream per
class, V-cycles and per-slot convergence) is native code in the library; this class
holds the server handle and converts arguments and results.
"""
from __future__ import annotations

import numpy as np

from . import binding as B


class SpaceTimeServer:
    def __init__(self, **options):
        self.opt = B.st_mg_server_default_options()
        for k, v in options.items():
            if not hasattr(self.opt, k):
                raise KeyError(k)
            setattr(self.opt, k, v)
        self.h = B.st_mg_server_create(self.opt)

    def close(self):
        if getattr(self, "h", None):
            B.st_mg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def register(self, n_cube, n_space_levels, nu, sigma):
        B.st_mg_server_set_materials(self.h, n_cube, n_space_levels, nu, sigma)

    def submit(self, n_cube, degree, N_t, tau, sigma_scale, exc, rtol, t_arrival=0.0) -> int:
        return B.st_mg_server_submit(self.h, n_cube, degree, N_t, tau, sigma_scale, exc, rtol, t_arrival)

    def step(self):
        """One scheduling round; returns the ids of the requests it finished."""
        return B.st_mg_server_step(self.h)

    def result(self, rid, want_x=True):
        """Result record of a finished request (released afterwards); x: (n_edge, N_t (p+1))."""
        r = B.st_mg_server_result(self.h, rid)
        if r["state"] != 2:
            return r
        x = np.zeros(r["n_values"]) if want_x else None
        r = B.st_mg_server_result(self.h, rid, x, release=True)
        if x is not None and r["n_edge"] > 0:
            r["x"] = x.reshape(r["n_edge"], -1)
        return r

    def stats(self):
        return B.st_mg_server_stats_get(self.h)

    def run_until_idle(self, timeout_s=3600.0):
        """Step until nothing is queued, building or on the device; returns finished ids.
        (A step with only builds pending waits a few ms for them inside the library.)"""
        import time
        done = []
        t_end = time.monotonic() + timeout_s
        while time.monotonic() < t_end:
            done += self.step()
            s = self.stats()
            if s["queued"] == 0 and s["active"] == 0 and s["building"] == 0:
                return done
        raise TimeoutError("server not idle after %.0f s" % timeout_s)
