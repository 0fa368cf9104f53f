"""ctypes binding of the serial oracle (``liboracle.so``).

TEST INFRASTRUCTURE ONLY.  Every function here is a thin call into the C++
oracle; the arithmetic lives in ``rdsplit_oracle.cpp`` (Algorithm 1 and its
samplers) and ``issa.cpp`` (exact spatial SSA).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None

_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_philox4x32.argtypes = [_u32p, _u32p, _u32p]
        L.orc_philox4x64.argtypes = [_u64p, _u64p, _u64p]
        for name in ("orc_log_many", "orc_exp_many"):
            getattr(L, name).argtypes = [_f64p, _f64p, C.c_int64]
        L.orc_log_factorial_many.argtypes = [_i64p, _f64p, C.c_int64]
        L.orc_threshold.argtypes = [C.c_double]
        L.orc_threshold.restype = C.c_uint32
        L.orc_stream_u32.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, _u32p, C.c_int64]
        L.orc_stream_u01.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, _f64p, C.c_int64, C.c_int]
        L.orc_binomial_many.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_double, _i64p, C.c_int64]
        L.orc_tau.argtypes = [C.c_int32, _i32p, _f64p, _f64p, _f64p, C.c_int32, _f64p, C.c_double]
        L.orc_tau.restype = C.c_double
        L.orc_run.argtypes = [C.c_int32, _i32p, _f64p, _f64p, _f64p, C.c_int32, _f64p, C.c_int32,
                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                              _i32p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_double,
                              C.c_uint64, C.c_int64]
        L.orc_run.restype = C.c_int
        L.orc_run_rule.argtypes = L.orc_run.argtypes + [C.c_int32]
        L.orc_run_rule.restype = C.c_int
        L.orc_run_opts.argtypes = L.orc_run.argtypes + [C.c_int32, C.c_int32]
        L.orc_run_opts.restype = C.c_int
        L.orc_tau_outliers.argtypes = L.orc_tau.argtypes + [C.c_int32]
        L.orc_tau_outliers.restype = C.c_double
        L.orc_run_foil.argtypes = [C.c_int32, _i32p, _f64p, _f64p, _f64p, C.c_int32, _f64p, C.c_double,
                                   _i32p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_double, C.c_uint64,
                                   C.c_int64, C.c_int32]
        L.orc_run_foil.restype = C.c_int
        L.orc_issa_run.argtypes = [C.c_int32, _i32p, _f64p, _f64p, _f64p, C.c_int32, _f64p, C.c_int32,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, _i32p, C.c_double,
                                   C.c_uint64]
        L.orc_issa_run.restype = C.c_int
        L.orc_period_tets.argtypes = [C.c_int32, _i32p, _f64p, _f64p, _f64p, C.c_int32, _f64p, C.c_int32,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, _i32p,
                                      C.c_int64, C.c_double, C.c_uint64, C.c_int32, C.c_int32, _i32p, _i32p]
        L.orc_period_tets.restype = C.c_int
        _lib = L
    return _lib


def philox4x32(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def philox4x64(ctr, key):
    out = np.zeros(4, np.uint64)
    lib().orc_philox4x64(np.asarray(ctr, np.uint64), np.asarray(key, np.uint64), out)
    return out


def own_log(x):
    x = np.ascontiguousarray(x, np.float64)
    y = np.empty_like(x)
    lib().orc_log_many(x.reshape(-1), y.reshape(-1), x.size)
    return y


def own_exp(x):
    x = np.ascontiguousarray(x, np.float64)
    y = np.empty_like(x)
    lib().orc_exp_many(x.reshape(-1), y.reshape(-1), x.size)
    return y


def log_factorial(k):
    k = np.ascontiguousarray(k, np.int64)
    y = np.empty(k.shape, np.float64)
    lib().orc_log_factorial_many(k.reshape(-1), y.reshape(-1), k.size)
    return y


def threshold(y: float) -> int:
    return int(lib().orc_threshold(float(y)))


def stream_u32(seed, tet, period, purpose, species, n):
    out = np.zeros(n, np.uint32)
    lib().orc_stream_u32(seed, tet, period, purpose, species, out, n)
    return out


def stream_u01(seed, tet, period, purpose, species, n, open0=False):
    out = np.zeros(n, np.float64)
    lib().orc_stream_u01(seed, tet, period, purpose, species, out, n, int(open0))
    return out


def binomial_many(n: int, p: float, count: int, seed: int = 1, period: int = 0):
    out = np.zeros(count, np.int64)
    lib().orc_binomial_many(seed, period, n, p, out, count)
    return out


def _ptr(a):
    return None if a is None else a.ctypes.data


def _model_arrays(model):
    S = model.n_species
    R = model.n_reactions
    D = np.ascontiguousarray(model.D, np.float64)
    lhs = np.ascontiguousarray(model.lhs, np.int32).reshape(R, S) if R else np.zeros((1, S), np.int32)
    rhs = np.ascontiguousarray(model.rhs, np.int32).reshape(R, S) if R else np.zeros((1, S), np.int32)
    k = np.ascontiguousarray(model.k, np.float64) if R else np.zeros(1)
    mask = None if model.mask is None else np.ascontiguousarray(model.mask, np.uint8)
    return S, R, D, lhs, rhs, k, mask


def tau(mesh, model, outliers: int = 0) -> float:
    """tau of Algorithm 1; with outliers = k > 0, taken from the (k+1)-th
    fastest tet (the outlier option of Sec. II.A)."""
    S, R, D, *_ = _model_arrays(model)
    if outliers:
        return lib().orc_tau_outliers(mesh.n_tets, mesh.adj, mesh.vol, mesh.area, mesh.dist, S, D,
                                      float(model.tau_scale), int(outliers))
    return lib().orc_tau(mesh.n_tets, mesh.adj, mesh.vol, mesh.area, mesh.dist, S, D,
                         float(model.tau_scale))


class OracleError(RuntimeError):
    pass


# Transfer rules (Sec. II.C): the count the diffusion draw of a period uses.
RULE_MEAN = 0   # N-bar, the mean occupancy (Eq. 3): the method
RULE_END = 1    # N(tau_k): first-order splitting (Sec. III.B, Fig. 7)
RULE_MID = 2    # N(tau_k / 2): the half-step ("median") reading


def run(mesh, model, counts, t_end: float, seed: int, t0: float = 0.0, period0: int = 0,
        max_periods: int = -1, rule: int = RULE_MEAN, outliers: int = 0):
    """Algorithm 1 from ``t0`` towards ``t_end`` (at most ``max_periods``
    periods) with the given transfer rule and tau taken from the
    (outliers + 1)-th fastest tet.  Returns (counts [T][S] int32, t,
    period)."""
    S, R, D, lhs, rhs, k, mask = _model_arrays(model)
    c = np.ascontiguousarray(counts, np.int32).copy()
    assert c.shape == (mesh.n_tets, S)
    t = C.c_double(t0)
    p = C.c_int64(period0)
    rc = lib().orc_run_opts(mesh.n_tets, mesh.adj, mesh.vol, mesh.area, mesh.dist, S, D, R,
                            lhs.ctypes.data, rhs.ctypes.data, k.ctypes.data, _ptr(mask),
                            float(model.tau_scale), c, C.byref(t), C.byref(p), float(t_end),
                            int(seed), int(max_periods), int(rule), int(outliers))
    if rc != 0:
        raise OracleError(f"orc_run_opts failed with code {rc}")
    return c, t.value, p.value


# Validation foils (Sec. II.A, Fig. 2), test-only diffusion counts.
FOIL_MEAN_N = 1   # n = discrete mean of the gross transfer (Fig. 2(b))
FOIL_NET = 2      # transfer binomial on the net flux only (Fig. 2(c))


def run_foil(mesh, model, counts, t_end: float, seed: int, foil: int, t0: float = 0.0, period0: int = 0,
             max_periods: int = -1):
    """Pure diffusion with a validation foil in place of the binomial count.
    Returns (counts [T][S] int32, t, period)."""
    S, R, D, *_ = _model_arrays(model)
    assert R == 0, "the foils are defined for pure diffusion"
    c = np.ascontiguousarray(counts, np.int32).copy()
    assert c.shape == (mesh.n_tets, S)
    t = C.c_double(t0)
    p = C.c_int64(period0)
    rc = lib().orc_run_foil(mesh.n_tets, mesh.adj, mesh.vol, mesh.area, mesh.dist, S, D, float(model.tau_scale),
                            c, C.byref(t), C.byref(p), float(t_end), int(seed), int(max_periods), int(foil))
    if rc != 0:
        raise OracleError(f"orc_run_foil failed with code {rc}")
    return c, t.value, p.value


def issa_run(mesh, model, counts, t_end: float, seed: int):
    """Exact whole-mesh SSA to ``t_end``; returns counts [T][S]."""
    S, R, D, lhs, rhs, k, mask = _model_arrays(model)
    c = np.ascontiguousarray(counts, np.int32).copy()
    rc = lib().orc_issa_run(mesh.n_tets, mesh.adj, mesh.vol, mesh.area, mesh.dist, S, D, R,
                            lhs.ctypes.data, rhs.ctypes.data, k.ctypes.data, _ptr(mask), c,
                            float(t_end), int(seed))
    if rc != 0:
        raise OracleError(f"orc_issa_run failed with code {rc}")
    return c


def period_tets(mesh, model, counts, period: int, tau_k: float, seed: int, t_begin: int, t_end: int):
    """Steps 2-3 of one period for tets t_begin..t_end-1: returns
    (out [n][S][4], rem [n][S])."""
    S, R, D, lhs, rhs, k, mask = _model_arrays(model)
    c = np.ascontiguousarray(counts, np.int32)
    n = t_end - t_begin
    out = np.zeros((n, S, 4), np.int32)
    rem = np.zeros((n, S), np.int32)
    rc = lib().orc_period_tets(mesh.n_tets, mesh.adj, mesh.vol, mesh.area, mesh.dist, S, D, R,
                               lhs.ctypes.data, rhs.ctypes.data, k.ctypes.data, _ptr(mask),
                               float(model.tau_scale), c, int(period), float(tau_k), int(seed),
                               int(t_begin), int(t_end), out, rem)
    if rc != 0:
        raise OracleError(f"orc_period_tets failed with code {rc}")
    return out, rem
