"""ctypes binding of libstmg (include/st_mg.h): argument marshalling only.

Every function below has the name of the C entry point it calls and raises
StMgError on a non-zero status.  Device buffers are passed as torch CUDA tensors
(float64, contiguous) or raw integer addresses; the library does all the work.
The binding loads the in-tree library and fails loudly if it has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build import LIB_PATH

_i32, _i64, _dbl, _vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
_P = ctypes.POINTER


class StMgError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        super().__init__(f"{fn}: status {status} ({msg})")
        self.status = status


class Mesh(ctypes.Structure):
    _fields_ = [("n_vert", _i32), ("n_tet", _i32), ("xyz", _P(_dbl)), ("tet", _P(_i32)), ("n_refine", _i32)]


class Problem(ctypes.Structure):
    _fields_ = [("n_cube", _i32), ("n_space_levels", _i32), ("nu", _P(_dbl)), ("sigma", _P(_dbl)),
                ("T", _dbl), ("N_t", _i32), ("degree", _i32), ("n_batch", _i32), ("bc", _i32),
                ("mesh", _P(Mesh)), ("batch_nt", _P(_i32))]


class Options(ctypes.Structure):
    _fields_ = [("omega", _dbl), ("nu_pre", _i32), ("nu_post", _i32), ("lambda_crit", _dbl),
                ("coarsen", _i32), ("max_levels", _i32), ("min_coarse_slabs", _i32),
                ("nodal_solve", _i32), ("nodal_jacobi_sweeps", _i32), ("use_A", _i32),
                ("setup_threads", _i32), ("slab_prec", _i32), ("residual_prec", _i32), ("use_graph", _i32),
                ("smoother", ctypes.c_char * 16), ("persistent_split", _i32), ("factor_cache", _i32),
                ("autotune", _i32), ("nd_leaf", _i32), ("split_k", _i32), ("tc_split_k", _i32)]


class ServerOptions(ctypes.Structure):
    _fields_ = [("slots", _i32), ("mem_budget", _i64), ("max_cycles", _i32), ("slab_prec", _i32), ("nu", _i32),
                ("omega", _dbl), ("setup_threads", _i32), ("keep_x", _i32), ("max_builds", _i32)]


class Request(ctypes.Structure):
    _fields_ = [("n_cube", _i32), ("degree", _i32), ("N_t", _i32), ("tau", _dbl), ("sigma_scale", _dbl),
                ("n_modes", _i32), ("a", _P(_dbl)), ("k", _P(_dbl)), ("phase", _P(_dbl)), ("rtol", _dbl),
                ("t_arrival", _dbl)]


class Result(ctypes.Structure):
    _fields_ = [("id", _i64), ("state", _i32), ("status", _i32), ("cycles", _i32), ("rel_res", _dbl),
                ("t_arrival", _dbl), ("t_admit", _dbl), ("t_done", _dbl), ("n_edge", _i64), ("n_values", _i64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", _i64), ("completed", _i64), ("queued", _i64), ("active", _i64),
                ("classes", _i32), ("building", _i32), ("class_bytes", _i64), ("cache_bytes", _i64),
                ("cache_entries", _i32), ("cache_hits", _i64), ("cache_misses", _i64), ("vcycles", _i64),
                ("slot_cycles", _i64), ("dofs_smoothed", _i64), ("evictions", _i64), ("deferrals", _i64)]


_SIGS = {
    "st_mg_default_options": [_P(Options)],
    "st_mg_setup": [_P(Problem), _P(Options), _vp, _P(_vp)],
    "st_mg_setup_host": [_P(Problem), _P(Options), _P(_vp)],
    "st_mg_setup_begin": [_P(Problem), _P(Options), _vp, _P(_vp)],
    "st_mg_setup_finish": [_vp],
    "st_mg_destroy": [_vp],
    "st_mg_sizes": [_vp, _P(_i64), _P(_i64), _P(_i64), _P(_i32)],
    "st_mg_level_info": [_vp, _i32, _P(_i32), _P(_i32), _P(_dbl), _P(_i64), _P(_i64)],
    "st_mg_assemble_load": [_vp, _i32, _P(_dbl), _P(_dbl), _P(_dbl), _vp],
    "st_mg_assemble_load_batch": [_vp, _i32, _i32, _P(_dbl), _P(_dbl), _P(_dbl), _vp],
    "st_mg_residual": [_vp, _i32, _vp, _vp, _vp, _P(_dbl)],
    "st_mg_slab_solve": [_vp, _i32, _vp, _vp],
    "st_mg_smooth_S": [_vp, _i32, _vp, _vp],
    "st_mg_correct_A": [_vp, _i32, _vp, _vp],
    "st_mg_grad_T": [_vp, _i32, _vp, _vp],
    "st_mg_nodal_solve": [_vp, _i32, _vp, _vp],
    "st_mg_time_integrate": [_vp, _i32, _vp, _vp],
    "st_mg_grad_add": [_vp, _i32, _vp, _vp],
    "st_mg_restrict": [_vp, _i32, _vp, _vp],
    "st_mg_prolong_add": [_vp, _i32, _vp, _vp],
    "st_mg_coarse_solve": [_vp, _vp, _vp],
    "st_mg_vcycle": [_vp, _vp, _vp, _P(_dbl)],
    "st_mg_solve": [_vp, _vp, _vp, _dbl, _i32, _P(_i32), _P(_dbl), _P(_dbl)],
    "st_mg_solve_host": [_vp, _P(_dbl), _P(_dbl), _dbl, _i32, _P(_i32), _P(_dbl), _P(_dbl)],
    "st_mg_debug_get": [_vp, _i32, _i32, _vp, _P(_i64)],
    "st_mg_debug_host_slab_solve": [_vp, _i32, _P(_dbl), _P(_dbl)],
    "st_mg_probe_fp64": [_vp, _P(_dbl)],
    "st_mg_batch_norms": [_vp, _vp, _P(_dbl)],
    "st_mg_vcycle_residual_async": [_vp, _vp, _vp, _vp],
    "st_mg_batch_norms_async": [_vp, _vp, _vp],
    "st_mg_check": [_vp],
    "st_mg_memory": [_vp, _P(_i64), _P(_i64)],
    "st_mg_split_waves": [_vp, _i32, _P(_i32)],
    "st_mg_set_split_waves": [_vp, _i32, _i32],
    "st_mg_set_tc_mode": [_vp, _i32, _i32],
    "st_mg_set_launch_overlap": [_i32],
    "st_mg_convergence_rate": [_vp, _vp, _i32, _dbl, _P(_dbl), _P(_i32), _P(_dbl)],
    "st_mg_slab_copy": [_vp, _i32, _i32, _vp, _i32, _vp],
    "st_mg_residual_halo": [_vp, _i32, _vp, _vp, _vp, _vp],
    "st_mg_time_integrate_carry": [_vp, _i32, _vp, _vp, _vp],
    "st_mg_time_carry": [_vp, _i32, _vp, _i32, _vp],
    "st_mg_cache_stats": [_P(_i64), _P(_i32), _P(_i32), _P(_i64), _P(_i64)],
    "st_mg_cache_trim": [_i64, _P(_i64)],
    "st_mg_batch_zero": [_vp, _i32, _vp],
    "st_mg_launch_count": [_P(_i64)],
    "st_mg_factor_stats": [_vp, _i32, _P(_dbl), _P(_i64), _P(_i32)],
    "st_mg_norm2_noalloc": [_vp, _i64, _vp, _vp],
    "st_mg_server_default_options": [_P(ServerOptions)],
    "st_mg_server_create": [_P(ServerOptions), _P(_vp)],
    "st_mg_server_set_materials": [_vp, _i32, _i32, _P(_dbl), _P(_dbl)],
    "st_mg_server_submit": [_vp, _P(Request), _P(_i64)],
    "st_mg_server_step": [_vp, _P(_i64), _i32, _P(_i32)],
    "st_mg_server_result": [_vp, _i64, _P(Result), _P(_dbl), _i64, _i32],
    "st_mg_server_stats_get": [_vp, _P(ServerStats)],
    "st_mg_server_destroy": [_vp],
    "st_mg_strerror": [ctypes.c_int],
    "st_mg_last_error": [],
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libstmg.so (built by __graft_entry__.build() or `python -m paper_1911_09548_gb300._build`)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libstmg is not built ({LIB_PATH} missing); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_char_p if name in ("st_mg_strerror", "st_mg_last_error") else (
                None if name in ("st_mg_destroy", "st_mg_server_destroy") else ctypes.c_int)
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(status: int, fn: str):
    if status != 0:
        raise StMgError(status, fn, lib().st_mg_last_error().decode())
    return status


def _addr(t) -> int:
    """Device (or host) address of a torch tensor / numpy array / int."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        if hasattr(t, "dtype") and str(t.dtype) != "torch.float64":
            raise TypeError("buffers must be float64")
        if not t.is_contiguous():
            raise ValueError("buffers must be contiguous")
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    raise TypeError(type(t))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_P(_dbl))


# ----------------------------------------------------------------- thin wrappers
def st_mg_default_options() -> Options:
    o = Options()
    _check(lib().st_mg_default_options(ctypes.byref(o)), "st_mg_default_options")
    return o


def make_problem(n_cube, n_space_levels, nu, sigma, T, N_t, degree, n_batch=1, bc=0, mesh=None, batch_nt=None):
    """mesh: None (Kuhn mesh with n_cube cubes per side) or (xyz, tets, n_refine), a general
    start mesh refined n_refine times (n_cube is then ignored).  batch_nt: per-problem slab
    counts of a ragged batch (None: every problem has N_t)."""
    nu = np.ascontiguousarray(nu, dtype=np.float64)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    p = Problem(n_cube, n_space_levels, _dptr(nu), _dptr(sigma), float(T), N_t, degree, n_batch, bc, None, None)
    keep = [nu, sigma]
    if batch_nt is not None:
        bnt = np.ascontiguousarray(batch_nt, dtype=np.int32)
        p.batch_nt = bnt.ctypes.data_as(_P(_i32))
        keep.append(bnt)
    if mesh is not None:
        xyz, tets, n_refine = mesh
        xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        tets = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
        m = Mesh(len(xyz), len(tets), _dptr(xyz), tets.ctypes.data_as(_P(_i32)), int(n_refine))
        p.mesh = ctypes.pointer(m)
        keep += [xyz, tets, m]
    p._keep = keep
    return p


def st_mg_setup(prob: Problem, opt: Options, stream: int = 0) -> int:
    h = _vp()
    _check(lib().st_mg_setup(ctypes.byref(prob), ctypes.byref(opt), _vp(stream), ctypes.byref(h)), "st_mg_setup")
    return h.value


def st_mg_setup_host(prob: Problem, opt: Options) -> int:
    h = _vp()
    _check(lib().st_mg_setup_host(ctypes.byref(prob), ctypes.byref(opt), ctypes.byref(h)), "st_mg_setup_host")
    return h.value


def st_mg_destroy(h: int):
    lib().st_mg_destroy(_vp(h))


def st_mg_sizes(h):
    ne, nn, nd, nl = _i64(), _i64(), _i64(), _i32()
    _check(lib().st_mg_sizes(_vp(h), ctypes.byref(ne), ctypes.byref(nn), ctypes.byref(nd), ctypes.byref(nl)),
           "st_mg_sizes")
    return ne.value, nn.value, nd.value, nl.value


def st_mg_level_info(h, level):
    s, nt, tau, ne, nn = _i32(), _i32(), _dbl(), _i64(), _i64()
    _check(lib().st_mg_level_info(_vp(h), level, ctypes.byref(s), ctypes.byref(nt), ctypes.byref(tau),
                                  ctypes.byref(ne), ctypes.byref(nn)), "st_mg_level_info")
    return {"space_level": s.value, "N_t": nt.value, "tau": tau.value, "n_edge": ne.value, "n_node": nn.value}


def st_mg_assemble_load(h, a, k, phase, f_dev):
    a = np.ascontiguousarray(a, np.float64).ravel()
    k = np.ascontiguousarray(k, np.float64).ravel()
    phase = np.ascontiguousarray(phase, np.float64).ravel()
    _check(lib().st_mg_assemble_load(_vp(h), len(phase), _dptr(a), _dptr(k), _dptr(phase), _vp(_addr(f_dev))),
           "st_mg_assemble_load")


def st_mg_assemble_load_batch(h, batch, a, k, phase, f_dev):
    a = np.ascontiguousarray(a, np.float64).ravel()
    k = np.ascontiguousarray(k, np.float64).ravel()
    phase = np.ascontiguousarray(phase, np.float64).ravel()
    _check(lib().st_mg_assemble_load_batch(_vp(h), batch, len(phase), _dptr(a), _dptr(k), _dptr(phase),
                                           _vp(_addr(f_dev))), "st_mg_assemble_load_batch")


def st_mg_residual(h, level, f, x, r, want_norm=False):
    nrm = _dbl()
    _check(lib().st_mg_residual(_vp(h), level, _vp(_addr(f)), _vp(_addr(x)), _vp(_addr(r)),
                                ctypes.byref(nrm) if want_norm else None), "st_mg_residual")
    return nrm.value if want_norm else None


def _two(name):
    def fn(h, level, a, b):
        _check(getattr(lib(), name)(_vp(h), level, _vp(_addr(a)), _vp(_addr(b))), name)
    fn.__name__ = name
    return fn


st_mg_slab_solve = _two("st_mg_slab_solve")
st_mg_smooth_S = _two("st_mg_smooth_S")
st_mg_correct_A = _two("st_mg_correct_A")
st_mg_grad_T = _two("st_mg_grad_T")
st_mg_nodal_solve = _two("st_mg_nodal_solve")
st_mg_time_integrate = _two("st_mg_time_integrate")
st_mg_grad_add = _two("st_mg_grad_add")
st_mg_restrict = _two("st_mg_restrict")
st_mg_prolong_add = _two("st_mg_prolong_add")


def st_mg_coarse_solve(h, f, x):
    _check(lib().st_mg_coarse_solve(_vp(h), _vp(_addr(f)), _vp(_addr(x))), "st_mg_coarse_solve")


def st_mg_vcycle(h, f, x, want_res=False):
    rr = _dbl()
    _check(lib().st_mg_vcycle(_vp(h), _vp(_addr(f)), _vp(_addr(x)), ctypes.byref(rr) if want_res else None),
           "st_mg_vcycle")
    return rr.value if want_res else None


def _solve_outputs(maxit):
    return _i32(), _dbl(), np.zeros(maxit + 1)


def st_mg_solve(h, f, x, rtol, maxit):
    it, rr, hist = _solve_outputs(maxit)
    st = lib().st_mg_solve(_vp(h), _vp(_addr(f)), _vp(_addr(x)), rtol, maxit, ctypes.byref(it), ctypes.byref(rr),
                           _dptr(hist))
    if st not in (0, 5):
        _check(st, "st_mg_solve")
    return {"status": st, "iters": it.value, "rel_res": rr.value, "history": hist[:it.value + 1]}


def st_mg_solve_host(h, f_host: np.ndarray, x_host: np.ndarray, rtol, maxit):
    assert f_host.dtype == np.float64 and x_host.dtype == np.float64
    assert f_host.flags.c_contiguous and x_host.flags.c_contiguous
    it, rr, hist = _solve_outputs(maxit)
    st = lib().st_mg_solve_host(_vp(h), _dptr(f_host), _dptr(x_host), rtol, maxit, ctypes.byref(it),
                                ctypes.byref(rr), _dptr(hist))
    if st not in (0, 5):
        _check(st, "st_mg_solve_host")
    return {"status": st, "iters": it.value, "rel_res": rr.value, "history": hist[:it.value + 1]}


_DEBUG_TYPES = {1: np.int32, 2: np.int32, 3: np.int32, 4: np.int64, 5: np.int32, 6: np.float64, 7: np.float64,
                8: np.int32, 9: np.int64, 10: np.int32, 11: np.float64, 12: np.int64, 13: np.int32,
                14: np.float64}


def st_mg_debug_get(h, what, level):
    nb = _i64(0)
    _check(lib().st_mg_debug_get(_vp(h), what, level, None, ctypes.byref(nb)), "st_mg_debug_get")
    dt = _DEBUG_TYPES[what]
    out = np.zeros(nb.value // np.dtype(dt).itemsize, dtype=dt)
    _check(lib().st_mg_debug_get(_vp(h), what, level, _vp(out.ctypes.data), ctypes.byref(nb)), "st_mg_debug_get")
    return out


def st_mg_debug_host_slab_solve(h, level, r_host: np.ndarray) -> np.ndarray:
    r_host = np.ascontiguousarray(r_host, np.float64)
    y = np.zeros_like(r_host)
    _check(lib().st_mg_debug_host_slab_solve(_vp(h), level, _dptr(r_host), _dptr(y)), "st_mg_debug_host_slab_solve")
    return y


def st_mg_probe_fp64(h) -> float:
    t = _dbl()
    _check(lib().st_mg_probe_fp64(_vp(h), ctypes.byref(t)), "st_mg_probe_fp64")
    return t.value


def st_mg_batch_norms(h, v_dev, n_batch):
    out = np.zeros(n_batch)
    _check(lib().st_mg_batch_norms(_vp(h), _vp(_addr(v_dev)), _dptr(out)), "st_mg_batch_norms")
    return out


def st_mg_check(h):
    """Raises StMgError(ST_MG_ERR_TIMEOUT) if a bounded device wait of earlier work gave up."""
    _check(lib().st_mg_check(_vp(h)), "st_mg_check")


def st_mg_batch_zero(h, batch, v_dev):
    _check(lib().st_mg_batch_zero(_vp(h), batch, _vp(_addr(v_dev))), "st_mg_batch_zero")


def st_mg_split_waves(h, level):
    w = _i32(0)
    _check(lib().st_mg_split_waves(_vp(h), level, ctypes.byref(w)), "st_mg_split_waves")
    return w.value


def st_mg_set_split_waves(h, level, waves):
    _check(lib().st_mg_set_split_waves(_vp(h), level, waves), "st_mg_set_split_waves")


def _opt_addr(t):
    return None if t is None else _vp(_addr(t))


def st_mg_slab_copy(h, level, nodal, v_dev, slab, out_dev):
    _check(lib().st_mg_slab_copy(_vp(h), level, int(nodal), _vp(_addr(v_dev)), slab, _vp(_addr(out_dev))),
           "st_mg_slab_copy")


def st_mg_residual_halo(h, level, f, x, x_prev, r):
    _check(lib().st_mg_residual_halo(_vp(h), level, _vp(_addr(f)), _vp(_addr(x)), _opt_addr(x_prev),
                                     _vp(_addr(r))), "st_mg_residual_halo")


def st_mg_time_integrate_carry(h, level, z, carry, w):
    _check(lib().st_mg_time_integrate_carry(_vp(h), level, _vp(_addr(z)), _opt_addr(carry), _vp(_addr(w))),
           "st_mg_time_integrate_carry")


def st_mg_time_carry(h, level, ends, n_prev, carry):
    _check(lib().st_mg_time_carry(_vp(h), level, _opt_addr(ends) if n_prev > 0 else None, n_prev,
                                  _vp(_addr(carry))), "st_mg_time_carry")


def st_mg_convergence_rate(h, x_dev, max_iter, floor):
    rates = np.zeros(max_iter)
    n = _i32(0)
    rate = _dbl(0.0)
    _check(lib().st_mg_convergence_rate(_vp(h), _vp(_addr(x_dev)), max_iter, floor, _dptr(rates), ctypes.byref(n),
                                        ctypes.byref(rate)), "st_mg_convergence_rate")
    return rate.value, list(rates[:n.value])


def st_mg_set_launch_overlap(on):
    _check(lib().st_mg_set_launch_overlap(int(on)), "st_mg_set_launch_overlap")


def st_mg_set_tc_mode(h, level, mode):
    _check(lib().st_mg_set_tc_mode(_vp(h), level, mode), "st_mg_set_tc_mode")


def st_mg_memory(h):
    own, fac = _i64(0), _i64(0)
    _check(lib().st_mg_memory(_vp(h), ctypes.byref(own), ctypes.byref(fac)), "st_mg_memory")
    return own.value, fac.value


def st_mg_cache_stats():
    b, e, u, hi, mi = _i64(0), _i32(0), _i32(0), _i64(0), _i64(0)
    _check(lib().st_mg_cache_stats(ctypes.byref(b), ctypes.byref(e), ctypes.byref(u), ctypes.byref(hi),
                                   ctypes.byref(mi)), "st_mg_cache_stats")
    return {"bytes": b.value, "entries": e.value, "in_use": u.value, "hits": hi.value, "misses": mi.value}


def st_mg_cache_trim(max_bytes=0):
    after = _i64(0)
    _check(lib().st_mg_cache_trim(max_bytes, ctypes.byref(after)), "st_mg_cache_trim")
    return after.value


def st_mg_launch_count() -> int:
    c = _i64()
    _check(lib().st_mg_launch_count(ctypes.byref(c)), "st_mg_launch_count")
    return c.value


def st_mg_factor_stats(h, level):
    m, b, d = _dbl(), _i64(), _i32()
    _check(lib().st_mg_factor_stats(_vp(h), level, ctypes.byref(m), ctypes.byref(b), ctypes.byref(d)),
           "st_mg_factor_stats")
    return {"macs_per_rhs": m.value, "factor_bytes": b.value, "depth": d.value}


def st_mg_norm2_noalloc(v_dev, n, stream, norm_dev):
    _check(lib().st_mg_norm2_noalloc(_vp(_addr(v_dev)), n, _vp(stream), _vp(_addr(norm_dev))),
           "st_mg_norm2_noalloc")


def st_mg_strerror(status: int) -> str:
    return lib().st_mg_strerror(status).decode()


# ----------------------------------------------------------------- request loop (st_mg_serve.h)
def st_mg_server_default_options() -> ServerOptions:
    o = ServerOptions()
    _check(lib().st_mg_server_default_options(ctypes.byref(o)), "st_mg_server_default_options")
    return o


def st_mg_server_create(opt: ServerOptions) -> int:
    h = _vp()
    _check(lib().st_mg_server_create(ctypes.byref(opt), ctypes.byref(h)), "st_mg_server_create")
    return h.value


def st_mg_server_set_materials(srv, n_cube, n_space_levels, nu, sigma):
    nu = np.ascontiguousarray(nu, dtype=np.float64)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    _check(lib().st_mg_server_set_materials(_vp(srv), n_cube, n_space_levels, _dptr(nu), _dptr(sigma)),
           "st_mg_server_set_materials")


def st_mg_server_submit(srv, n_cube, degree, N_t, tau, sigma_scale, exc, rtol, t_arrival=0.0) -> int:
    a = np.ascontiguousarray(exc["a"], np.float64).ravel()
    k = np.ascontiguousarray(exc["k"], np.float64).ravel()
    ph = np.ascontiguousarray(exc["phase"], np.float64).ravel()
    r = Request(n_cube, degree, N_t, float(tau), float(sigma_scale), len(ph), _dptr(a), _dptr(k), _dptr(ph),
                float(rtol), float(t_arrival))
    i = _i64()
    _check(lib().st_mg_server_submit(_vp(srv), ctypes.byref(r), ctypes.byref(i)), "st_mg_server_submit")
    return i.value


def st_mg_server_step(srv, cap=4096):
    ids = np.zeros(cap, dtype=np.int64)
    n = _i32()
    _check(lib().st_mg_server_step(_vp(srv), ids.ctypes.data_as(_P(_i64)), cap, ctypes.byref(n)),
           "st_mg_server_step")
    return [int(v) for v in ids[:min(n.value, cap)]]


def st_mg_server_result(srv, rid, x_out: np.ndarray | None = None, release=False):
    r = Result()
    cap = 0 if x_out is None else x_out.size
    _check(lib().st_mg_server_result(_vp(srv), rid, ctypes.byref(r), None if x_out is None else _dptr(x_out), cap,
                                     1 if release else 0), "st_mg_server_result")
    return {f: getattr(r, f) for f, _ in Result._fields_}


def st_mg_server_stats_get(srv):
    s = ServerStats()
    _check(lib().st_mg_server_stats_get(_vp(srv), ctypes.byref(s)), "st_mg_server_stats_get")
    return {f: getattr(s, f) for f, _ in ServerStats._fields_}


def st_mg_server_destroy(srv):
    lib().st_mg_server_destroy(_vp(srv))
