"""Request loop with continuous batching (include/st_mg_serve.h).

Requests of several meshes, DG degrees, N_t, tau and conductivity scalings arrive in
two waves; later ones join while earlier ones are on the device, some wait for a
slot of a full class, and requests whose tau / s agree share one class.  Each
result must equal the solve of the same problem alone on its own handle (same
V-cycle count, same solution to rounding), and the mixed-precision server must
reach the FP64 solution to the 1e-8 tolerance of the mixed path."""
import numpy as np
import pytest

import st_inputs
from helpers import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MESHES = {4: 2, 8: 2}            # n_cube -> n_space_levels
RTOL = 1e-10
# (n_cube, degree, N_t, tau, sigma_scale, excitation seed)
WAVE1 = [
    (4, 1, 16, 1 / 16, 1.0, 0),
    (4, 1, 16, 1 / 8, 2.0, 1),    # tau / s = 1/16: the class of the first
    (4, 1, 16, 1 / 32, 0.5, 2),   # the same class again (waits for a slot with 2 slots)
    (8, 0, 8, 1 / 8, 1.0, 3),
    (4, 1, 32, 1 / 16, 1.0, 4),   # N_t = 32, tau / s = 1/16: shares the factors of the first class
]
WAVE2 = [
    (8, 1, 16, 1 / 16, 4.0, 5),
    (4, 0, 16, 1 / 16, 1.0, 6),
    (4, 1, 16, 1 / 16, 1.0, 7),
]


@pytest.fixture(scope="module")
def stmg():
    from paper_1911_09548_gb300._build import build
    build()
    import paper_1911_09548_gb300
    return paper_1911_09548_gb300


def mats(n):
    return st_inputs.materials(n, "two_material", 5)


def alone(stmg, req, slab_prec=0):
    """The request solved on its own handle with its own conductivity and time grid."""
    n, p, N_t, tau, s, seed = req
    nu, sigma = mats(n)
    S = stmg.SpaceTimeSolver(n, nu, sigma * s, N_t * tau, N_t, p, n_space_levels=MESHES[n], nu_pre=1, nu_post=1,
                             slab_prec=slab_prec)
    f = S.load(st_inputs.excitation(seed))
    x = S.zeros()
    out = S.solve(f, x, rtol=RTOL, maxit=80)
    torch.cuda.synchronize()
    X = x.cpu().numpy()
    S.close()
    return out, X


def serve(stmg, slab_prec, slots=2, mem_budget=0, waves=(WAVE1, WAVE2)):
    srv = stmg.SpaceTimeServer(slots=slots, slab_prec=slab_prec, nu=1, max_cycles=80, mem_budget=mem_budget)
    for n, nsl in MESHES.items():
        srv.register(n, nsl, *mats(n))
    ids = {}
    results = {}
    for w, wave in enumerate(waves):
        for req in wave:
            n, p, N_t, tau, s, seed = req
            ids[srv.submit(n, p, N_t, tau, s, st_inputs.excitation(seed), RTOL)] = req
        steps = 3 if w + 1 < len(waves) else 1000000
        for _ in range(steps):
            for rid in srv.step():
                results[ids[rid]] = srv.result(rid)
            st = srv.stats()
            if st["queued"] == 0 and st["active"] == 0 and st["building"] == 0 and w + 1 == len(waves):
                break
    stats = srv.stats()
    srv.close()
    return results, stats


def test_fp64_server_results_equal_alone(stmg):
    stmg.binding.st_mg_cache_trim(0)
    results, stats = serve(stmg, slab_prec=0)
    assert len(results) == len(WAVE1) + len(WAVE2)
    # three requests share the first class; N_t = 32 reuses its factors
    assert stats["cache_hits"] > 0
    assert stats["completed"] == stats["submitted"] == len(results)
    for req, r in results.items():
        assert r["status"] == 0, (req, r)
        assert r["rel_res"] <= RTOL
        out, X = alone(stmg, req)
        assert out["status"] == 0
        assert r["cycles"] == out["iters"], req
        assert r["x"].shape == X.shape
        assert rel(r["x"], X) < 1e-9, req


def test_mixed_precision_server_reaches_fp64_solution(stmg):
    results, stats = serve(stmg, slab_prec=3)
    for req, r in results.items():
        assert r["status"] == 0, (req, r)
        out, X = alone(stmg, req)
        assert rel(r["x"], X) < 1e-8, req


def test_admission_by_device_memory(stmg):
    """A budget that holds about one class at a time: later classes wait (deferred),
    idle classes and their unused factors are evicted, every result still equals the
    solve alone."""
    B = stmg.binding
    B.st_mg_cache_trim(0)
    one = [(4, 1, 16, 1 / 16, 1.0, 0)]
    _, st1 = serve(stmg, slab_prec=0, waves=(one,))
    per_class = st1["class_bytes"] + st1["cache_bytes"]
    B.st_mg_cache_trim(0)
    reqs = [(4, 1, 16, 1 / 16, 1.0, 10), (4, 1, 16, 1 / 64, 1.0, 11), (4, 1, 16, 1 / 256, 1.0, 12)]
    results, stats = serve(stmg, slab_prec=0, mem_budget=int(1.5 * per_class), waves=(reqs,))
    assert stats["deferrals"] > 0
    assert stats["evictions"] > 0
    for req, r in results.items():
        assert r["status"] == 0
        out, X = alone(stmg, req)
        assert r["cycles"] == out["iters"]
        assert rel(r["x"], X) < 1e-9
    B.st_mg_cache_trim(0)


def test_factor_cache_shares_levels(stmg):
    """Two handles on one mesh and tau ladder: the second takes every slab factor of the
    first from the cache and references, not copies, them."""
    B = stmg.binding
    B.st_mg_cache_trim(0)
    nu, sigma = mats(4)
    c0 = B.st_mg_cache_stats()
    S1 = stmg.SpaceTimeSolver(4, nu, sigma, 16 / 16, 16, 1, n_space_levels=2, factor_cache=1)
    c1 = B.st_mg_cache_stats()
    S2 = stmg.SpaceTimeSolver(4, nu, sigma, 32 / 16, 32, 1, n_space_levels=2, factor_cache=1)
    c2 = B.st_mg_cache_stats()
    # S1's time levels: tau = 1/16 .. 1 (5 slab factors) + 2 nodal factors, all misses
    assert c1["misses"] - c0["misses"] == S1.n_levels + 2 and c1["hits"] == c0["hits"]
    # S2 (tau = 1/16 .. 2): S1's 5 slab factors and 2 nodal factors are hits, one new level
    assert c2["hits"] - c1["hits"] == S1.n_levels + 2
    assert c2["misses"] - c1["misses"] == S2.n_levels - S1.n_levels
    own1, fac1 = B.st_mg_memory(S1.h)
    own2, fac2 = B.st_mg_memory(S2.h)
    assert fac2 > fac1 > 0
    assert c2["bytes"] < fac1 + fac2            # shared, not duplicated
    # the cached factors give the same V-cycle as private ones
    S3 = stmg.SpaceTimeSolver(4, nu, sigma, 32 / 16, 32, 1, n_space_levels=2)
    f = S2.load(st_inputs.excitation(3))
    x2, x3 = S2.zeros(), S3.zeros()
    S2.vcycle(f, x2)
    S3.vcycle(f, x3)
    torch.cuda.synchronize()
    assert rel(x2.cpu().numpy(), x3.cpu().numpy()) < 1e-13
    for S in (S1, S2, S3):
        S.close()
    assert B.st_mg_cache_stats()["in_use"] == 0
    assert B.st_mg_cache_trim(0) == 0


def test_request_failures_reported(stmg):
    """A request that reaches max_cycles comes back ST_MG_ERR_NOT_CONVERGED (5) with its
    last iterate; invalid submissions are rejected at submit time."""
    srv = stmg.SpaceTimeServer(slots=2, slab_prec=0, nu=1, max_cycles=2)
    srv.register(4, 2, *mats(4))
    exc = st_inputs.excitation(1)
    rid = srv.submit(4, 1, 16, 1 / 16, 1.0, exc, 1e-12)
    done = {}
    for _ in range(100000):
        for d in srv.step():
            done[d] = srv.result(d)
        if rid in done:
            break
    r = done[rid]
    assert r["status"] == 5 and r["cycles"] == 2 and 1e-12 < r["rel_res"] < 1.0
    B = stmg.binding
    for args in ((8, 1, 16, 1 / 16, 1.0), (4, 2, 16, 1 / 16, 1.0), (4, 1, 12, 1 / 16, 1.0),
                 (4, 1, 16, -1.0, 1.0), (4, 1, 16, 1 / 16, 0.0)):
        with pytest.raises(B.StMgError):
            srv.submit(*args, exc, 1e-8)   # unregistered mesh, degree, N_t, tau, sigma scale
    srv.close()


def test_served_request_with_conductivity_scale_matches_oracle_time_stepping(stmg):
    """A request (s sigma, tau) is served as (sigma, tau / s) by the time rescaling t = s t'
    (the substitution divides the whole space-time system and its load by s).  The served
    solution is compared directly with the oracle's sequential time stepping (Section
    2.1, eq. timeStepping, and its DG(1) form) of the original problem: conductivity
    s sigma, N_t slabs of step tau, T = N_t tau, both degrees."""
    from helpers import from_lib
    from oracle.load import spacetime_load
    from oracle.spacetime import SlabOperator, build_space_hierarchy, sequential_solve

    n = 4
    nu, sigma = mats(n)
    srv = stmg.SpaceTimeServer(slots=2, slab_prec=0, nu=1, max_cycles=80)
    srv.register(n, MESHES[n], nu, sigma)
    reqs = [(1, 16, 1 / 16, 4.0, 9), (0, 8, 1 / 4, 0.25, 10)]     # (degree, N_t, tau, s, seed)
    ids = {srv.submit(n, p, N_t, tau, s, st_inputs.excitation(seed), 1e-12): (p, N_t, tau, s, seed)
           for p, N_t, tau, s, seed in reqs}
    done = {}
    for _ in range(100000):
        for rid in srv.step():
            done[ids[rid]] = srv.result(rid)
        if len(done) == len(reqs):
            break
    srv.close()
    for (p, N_t, tau, s, seed), r in done.items():
        assert r["status"] == 0 and r["rel_res"] <= 1e-12, r
        space = build_space_hierarchy(n, 1, nu, s * sigma)[0]
        f = spacetime_load(space.mesh, st_inputs.excitation(seed), p, N_t, N_t * tau)
        xs = sequential_solve(SlabOperator(space, p, tau), f)
        err = rel(from_lib(r["x"], p + 1), xs)
        assert err < 1e-9, (p, N_t, tau, s, err)
