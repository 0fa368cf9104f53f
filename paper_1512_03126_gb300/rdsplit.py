"""Python binding of the C ABI in include/rdsplit.h (argument marshalling only).

Every step of the method runs in the CUDA kernels of ``librdsplit.so``; this
module converts numpy arrays / torch tensors to pointers and error codes to
exceptions.  There is no fallback: if the library is missing or cannot be
loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librdsplit.so")

RDSPLIT_OK = 0
RDSPLIT_EINVAL = -1
RDSPLIT_ENOMEM = -2
RDSPLIT_ECUDA = -3
RDSPLIT_ETIMEOUT = -4
RDSPLIT_EOVERFLOW = -5
RDSPLIT_ESTATE = -6

_lib = None


class RdsplitError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rdsplit error {code}: {msg}")
        self.code = code


def _declare(L):
    vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    sig = {
        "rdsplit_last_error": ([], C.c_char_p),
        "rdsplit_kernel_launches": ([], i64),
        "rdsplit_mesh_create": ([i32, vp, vp, vp, vp, i32, C.POINTER(vp)], C.c_int),
        "rdsplit_mesh_create_ex": ([i32, vp, vp, vp, vp, vp, i32, C.POINTER(vp)], C.c_int),
        "rdsplit_get_order": ([vp, vp], C.c_int),
        "rdsplit_set_model": ([vp, i32, vp, i32, vp, vp, vp, vp, dbl], C.c_int),
        "rdsplit_set_counts": ([vp, vp], C.c_int),
        "rdsplit_set_counts_device": ([vp, vp], C.c_int),
        "rdsplit_run": ([vp, dbl, u64], C.c_int),
        "rdsplit_run_periods": ([vp, i64, u64], C.c_int),
        "rdsplit_get_counts": ([vp, vp], C.c_int),
        "rdsplit_get_counts_device": ([vp, vp], C.c_int),
        "rdsplit_get_time": ([vp, C.POINTER(dbl), C.POINTER(i64)], C.c_int),
        "rdsplit_set_time": ([vp, dbl, i64], C.c_int),
        "rdsplit_get_tau": ([vp, C.POINTER(dbl)], C.c_int),
        "rdsplit_get_shape": ([vp, C.POINTER(i32), C.POINTER(i32)], C.c_int),
        "rdsplit_set_stream": ([vp, vp], C.c_int),
        "rdsplit_mesh_destroy": ([vp], C.c_int),
        "rdsplit_set_allocator": ([vp, vp, vp], C.c_int),
        "rdsplit_set_timing": ([vp, i32], C.c_int),
        "rdsplit_set_period_kernel": ([vp, i32, i32], C.c_int),
        "rdsplit_partition_set": ([vp, i32, i32], C.c_int),
        "rdsplit_partition_step": ([vp, dbl, u64, C.POINTER(i32)], C.c_int),
        "rdsplit_inbox_export": ([vp, vp, i32, vp], C.c_int),
        "rdsplit_inbox_import": ([vp, vp, i32, vp], C.c_int),
        "rdsplit_partition_end": ([vp], C.c_int),
        "rdsplit_get_period_kernel": ([vp, C.POINTER(i32), C.POINTER(i32)], C.c_int),
        "rdsplit_static_scratch_bytes": ([i32, i32, i32], C.c_size_t),
        "rdsplit_engine_create": ([i32, i64, C.POINTER(vp)], C.c_int),
        "rdsplit_engine_set_stream": ([vp, vp], C.c_int),
        "rdsplit_engine_add": ([vp, vp, dbl, u64, C.POINTER(i32)], C.c_int),
        "rdsplit_engine_step": ([vp, i64], C.c_int),
        "rdsplit_engine_poll": ([vp, vp, i32, C.POINTER(i32)], C.c_int),
        "rdsplit_engine_active": ([vp, C.POINTER(i32), C.POINTER(i64)], C.c_int),
        "rdsplit_engine_destroy": ([vp], C.c_int),
        "rdsplit_ensemble_run": ([i32, vp, vp, vp], C.c_int),
        "rdsplit_engine_set_timing": ([vp, i32], C.c_int),
        "rdsplit_set_zeta_outliers": ([vp, i32], C.c_int),
        "rdsplit_zeta_histogram": ([vp, i32, vp, C.POINTER(dbl), C.POINTER(dbl)], C.c_int),
        "rdsplit_set_transfer_rule": ([vp, i32], C.c_int),
        "rdsplit_engine_set_concurrency": ([vp, i32, i32], C.c_int),
        "rdsplit_engine_stats": ([vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(dbl), C.POINTER(i64)], C.c_int),
        "rdsplit_engine_slot_times": ([vp, vp, i32], C.c_int),
        "rdsplit_engine_schedule": ([vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)], C.c_int),
        "rdsplit_engine_set_slice_work": ([vp, i64], C.c_int),
        "rdsplit_run_static": ([i32, vp, vp, vp, vp, i32, vp, i32, vp, vp, vp, vp, dbl, vp,
                                C.POINTER(dbl), C.POINTER(i64), dbl, u64, vp], C.c_int),
        "rdsplit_get_timing": ([vp, C.POINTER(dbl), C.POINTER(i64)], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res


def lib():
    """Load librdsplit.so (built by ``build.build()``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1512_03126_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        _declare(L)
        _lib = L
    return _lib


def _check(rc: int):
    if rc != RDSPLIT_OK:
        raise RdsplitError(rc, lib().rdsplit_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def _c(a, dtype, shape=None):
    a = np.ascontiguousarray(a, dtype=dtype)
    if shape is not None and a.shape != tuple(shape):
        a = a.reshape(shape)
    return a


# ---------------------------------------------------------------- C ABI ----

def rdsplit_last_error() -> str:
    return lib().rdsplit_last_error().decode()


def rdsplit_kernel_launches() -> int:
    return int(lib().rdsplit_kernel_launches())


def rdsplit_mesh_create(n_tets, adj, vol, face_area, centroid_dist, flags=0):
    adj = _c(adj, np.int32, (n_tets, 4))
    vol = _c(vol, np.float64, (n_tets,))
    face_area = _c(face_area, np.float64, (n_tets, 4))
    centroid_dist = _c(centroid_dist, np.float64, (n_tets, 4))
    h = C.c_void_p()
    _check(lib().rdsplit_mesh_create(int(n_tets), _ptr(adj), _ptr(vol), _ptr(face_area),
                                     _ptr(centroid_dist), int(flags), C.byref(h)))
    return h


RDSPLIT_REORDER_SFC = 1


def rdsplit_mesh_create_ex(n_tets, adj, vol, face_area, centroid_dist, centroid=None, flags=0):
    adj = _c(adj, np.int32, (n_tets, 4))
    vol = _c(vol, np.float64, (n_tets,))
    face_area = _c(face_area, np.float64, (n_tets, 4))
    centroid_dist = _c(centroid_dist, np.float64, (n_tets, 4))
    centroid = None if centroid is None else _c(centroid, np.float64, (n_tets, 3))
    h = C.c_void_p()
    _check(lib().rdsplit_mesh_create_ex(int(n_tets), _ptr(adj), _ptr(vol), _ptr(face_area), _ptr(centroid_dist),
                                        _ptr(centroid), int(flags), C.byref(h)))
    return h


def rdsplit_get_order(h):
    T, _ = rdsplit_get_shape(h)
    out = np.empty(T, np.int32)
    _check(lib().rdsplit_get_order(h, _ptr(out)))
    return out


def rdsplit_set_model(h, n_species, D, n_reactions, lhs, rhs, k, rxn_tet_mask=None, tau_scale=1.0):
    D = _c(D, np.float64, (n_species,))
    R = int(n_reactions)
    lhs = _c(lhs, np.int32, (R, n_species)) if R else None
    rhs = _c(rhs, np.int32, (R, n_species)) if R else None
    k = _c(k, np.float64, (R,)) if R else None
    mask = None if rxn_tet_mask is None else _c(rxn_tet_mask, np.uint8)
    _check(lib().rdsplit_set_model(h, int(n_species), _ptr(D), R, _ptr(lhs), _ptr(rhs), _ptr(k),
                                   _ptr(mask), float(tau_scale)))


def rdsplit_set_counts(h, counts):
    counts = _c(counts, np.int32)
    _check(lib().rdsplit_set_counts(h, _ptr(counts)))


def rdsplit_set_counts_device(h, tensor):
    _check(lib().rdsplit_set_counts_device(h, _ptr(tensor)))


def rdsplit_run(h, t_end: float, seed: int):
    _check(lib().rdsplit_run(h, float(t_end), int(seed)))


def rdsplit_run_periods(h, n_periods: int, seed: int):
    _check(lib().rdsplit_run_periods(h, int(n_periods), int(seed)))


def rdsplit_get_shape(h):
    T, S = C.c_int32(), C.c_int32()
    _check(lib().rdsplit_get_shape(h, C.byref(T), C.byref(S)))
    return T.value, S.value


def rdsplit_get_counts(h, out=None):
    T, S = rdsplit_get_shape(h)
    if out is None:
        out = np.empty((T, S), np.int32)
    _check(lib().rdsplit_get_counts(h, _ptr(out)))
    return out


def rdsplit_get_counts_device(h, tensor):
    _check(lib().rdsplit_get_counts_device(h, _ptr(tensor)))
    return tensor


def rdsplit_get_time(h):
    t, p = C.c_double(), C.c_int64()
    _check(lib().rdsplit_get_time(h, C.byref(t), C.byref(p)))
    return t.value, p.value


def rdsplit_set_time(h, t: float, period: int):
    _check(lib().rdsplit_set_time(h, float(t), int(period)))


def rdsplit_get_tau(h) -> float:
    t = C.c_double()
    _check(lib().rdsplit_get_tau(h, C.byref(t)))
    return t.value


def rdsplit_set_stream(h, stream):
    """``stream``: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(lib().rdsplit_set_stream(h, C.c_void_p(stream or 0)))


def rdsplit_mesh_destroy(h):
    _check(lib().rdsplit_mesh_destroy(h))


def rdsplit_partition_set(h, t0: int, t1: int):
    _check(lib().rdsplit_partition_set(h, int(t0), int(t1)))


def rdsplit_partition_step(h, t_end: float, seed: int) -> bool:
    """One period of the own tets; True while t < t_end."""
    more = C.c_int32()
    _check(lib().rdsplit_partition_step(h, float(t_end), int(seed), C.byref(more)))
    return bool(more.value)


def rdsplit_inbox_export(h, d_slots, d_buf):
    """d_slots: int32 device tensor [n]; d_buf: int32 device tensor [n][S]."""
    _check(lib().rdsplit_inbox_export(h, _ptr(d_slots), int(d_slots.numel()), _ptr(d_buf)))
    return d_buf


def rdsplit_inbox_import(h, d_slots, d_buf):
    _check(lib().rdsplit_inbox_import(h, _ptr(d_slots), int(d_slots.numel()), _ptr(d_buf)))


def rdsplit_partition_end(h):
    _check(lib().rdsplit_partition_end(h))


def rdsplit_set_period_kernel(h, mode: int = 0, block: int = 0):
    """mode 0 automatic, 1 one pass, 2 two passes (light + deferred); block
    0 = chosen from the mesh size."""
    _check(lib().rdsplit_set_period_kernel(h, int(mode), int(block)))


def rdsplit_get_period_kernel(h):
    """(1 if runs use two passes else 0, light-pass block size)."""
    a, b = C.c_int32(), C.c_int32()
    _check(lib().rdsplit_get_period_kernel(h, C.byref(a), C.byref(b)))
    return a.value, b.value


def rdsplit_set_timing(h, stride: int):
    _check(lib().rdsplit_set_timing(h, int(stride)))


def rdsplit_get_timing(h):
    ms, n = C.c_double(), C.c_int64()
    _check(lib().rdsplit_get_timing(h, C.byref(ms), C.byref(n)))
    return ms.value, n.value


def rdsplit_engine_create(max_slots: int, max_active_tets: int):
    e = C.c_void_p()
    _check(lib().rdsplit_engine_create(int(max_slots), int(max_active_tets), C.byref(e)))
    return e


def rdsplit_engine_set_stream(e, stream):
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(lib().rdsplit_engine_set_stream(e, C.c_void_p(stream or 0)))


def rdsplit_engine_add(e, h, t_end: float, seed: int) -> int:
    slot = C.c_int32()
    _check(lib().rdsplit_engine_add(e, h, float(t_end), int(seed), C.byref(slot)))
    return slot.value


def rdsplit_engine_step(e, n_steps: int):
    _check(lib().rdsplit_engine_step(e, int(n_steps)))


def rdsplit_engine_poll(e, max_slots: int = 4096):
    buf = np.zeros(max_slots, np.int32)
    n = C.c_int32()
    _check(lib().rdsplit_engine_poll(e, _ptr(buf), int(max_slots), C.byref(n)))
    return [int(x) for x in buf[:n.value]]


def rdsplit_engine_active(e):
    ns, nt = C.c_int32(), C.c_int64()
    _check(lib().rdsplit_engine_active(e, C.byref(ns), C.byref(nt)))
    return ns.value, nt.value


def rdsplit_engine_destroy(e):
    _check(lib().rdsplit_engine_destroy(e))


RDSPLIT_TRANSFER_MEAN = 0   # N-bar, the mean occupancy (Eq. 3): the method
RDSPLIT_TRANSFER_END = 1    # N(tau_k): first-order splitting
RDSPLIT_TRANSFER_MID = 2    # N(tau_k / 2): the half-step reading


def rdsplit_set_zeta_outliers(h, k: int):
    _check(lib().rdsplit_set_zeta_outliers(h, int(k)))


def rdsplit_zeta_histogram(h, nbins: int):
    """Returns (counts int64[nbins], mean, max) of zeta over the tets."""
    counts = np.zeros(int(nbins), np.int64)
    mean, mx = C.c_double(), C.c_double()
    _check(lib().rdsplit_zeta_histogram(h, int(nbins), _ptr(counts), C.byref(mean), C.byref(mx)))
    return counts, mean.value, mx.value


def rdsplit_set_transfer_rule(h, rule: int):
    _check(lib().rdsplit_set_transfer_rule(h, int(rule)))


def rdsplit_engine_set_concurrency(e, in_flight: int, cluster: int):
    _check(lib().rdsplit_engine_set_concurrency(e, int(in_flight), int(cluster)))


def rdsplit_engine_set_timing(e, stride: int):
    _check(lib().rdsplit_engine_set_timing(e, int(stride)))


def rdsplit_engine_stats(e):
    """(global steps, processed entries, sampled ms, sampled launches)."""
    st, pr, ms, n = C.c_int64(), C.c_int64(), C.c_double(), C.c_int64()
    _check(lib().rdsplit_engine_stats(e, C.byref(st), C.byref(pr), C.byref(ms), C.byref(n)))
    return st.value, pr.value, ms.value, n.value


def rdsplit_engine_slot_times(e, n_slots: int):
    """int64 [n_slots][3]: device-clock start and end (ns) and entries
    processed of each slot's last timed slice."""
    out = np.zeros((int(n_slots), 3), np.int64)
    _check(lib().rdsplit_engine_slot_times(e, _ptr(out), int(n_slots)))
    return out


def rdsplit_engine_set_slice_work(e, max_tet_periods: int):
    _check(lib().rdsplit_engine_set_slice_work(e, int(max_tet_periods)))


def rdsplit_engine_schedule(e):
    """(simulations in flight, CTAs per cluster, clusters that fit at once)
    of the last launch."""
    a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().rdsplit_engine_schedule(e, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def rdsplit_ensemble_run(meshes, t_end, seeds):
    """Run mesh handles to t_end[i] with seeds[i] in one lockstep engine."""
    n = len(meshes)
    hs = (C.c_void_p * n)(*[m.value if hasattr(m, "value") else m for m in meshes])
    te = np.ascontiguousarray(t_end, np.float64)
    sd = np.ascontiguousarray(seeds, np.uint64)
    _check(lib().rdsplit_ensemble_run(n, C.cast(hs, C.c_void_p), _ptr(te), _ptr(sd)))


RDSPLIT_STATIC_SCRATCH_BYTES = 32 * 1024 * 1024


def rdsplit_static_scratch_bytes(n_tets: int, n_species: int, masked: bool = False) -> int:
    return int(lib().rdsplit_static_scratch_bytes(int(n_tets), int(n_species), int(bool(masked))))


def rdsplit_run_static(n_tets, d_adj, d_vol, d_face_area, d_centroid_dist, n_species, D, n_reactions,
                       lhs, rhs, k, d_rxn_tet_mask, tau_scale, d_counts, t, period, t_end, seed,
                       stream=None):
    """Allocation-free run: mesh arrays, mask and counts are device tensors
    (caller-owned); the model arrays are host arrays.  Returns (t, period)."""
    R = int(n_reactions)
    D = _c(D, np.float64, (n_species,))
    lhs = _c(lhs, np.int32, (R, n_species)) if R else None
    rhs = _c(rhs, np.int32, (R, n_species)) if R else None
    k = _c(k, np.float64, (R,)) if R else None
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    tt, pp = C.c_double(t), C.c_int64(period)
    _check(lib().rdsplit_run_static(int(n_tets), _ptr(d_adj), _ptr(d_vol), _ptr(d_face_area),
                                    _ptr(d_centroid_dist), int(n_species), _ptr(D), R, _ptr(lhs), _ptr(rhs),
                                    _ptr(k), _ptr(d_rxn_tet_mask), float(tau_scale), _ptr(d_counts),
                                    C.byref(tt), C.byref(pp), float(t_end), int(seed),
                                    C.c_void_p(stream or 0)))
    return tt.value, pp.value


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
_allocator_refs = None


def rdsplit_set_allocator(alloc=None, free=None, ctx=None):
    """Route the library's device allocations through Python callables
    ``alloc(nbytes) -> int pointer`` and ``free(ptr)``; ``None`` restores
    cudaMalloc / cudaFree."""
    global _allocator_refs
    if alloc is None:
        _check(lib().rdsplit_set_allocator(None, None, None))
        _allocator_refs = None
        return
    a = ALLOC_FN(lambda n, _c: int(alloc(int(n))) or None)
    f = FREE_FN(lambda p, _c: free(int(p)) if p else None)
    _check(lib().rdsplit_set_allocator(C.cast(a, C.c_void_p), C.cast(f, C.c_void_p), ctx))
    _allocator_refs = (a, f)


def use_torch_allocator():
    """Serve the library's device memory from PyTorch's caching allocator."""
    import torch

    def alloc(n):
        return torch.cuda.caching_allocator_alloc(n, device=torch.cuda.current_device())

    def free(p):
        torch.cuda.caching_allocator_delete(p)

    rdsplit_set_allocator(alloc, free)


# ------------------------------------------------------------ convenience --

class Simulation:
    """One mesh + model handle: ``Simulation(mesh, model)``, then
    ``set_counts``, ``run``, ``counts``."""

    def __init__(self, mesh, model, counts=None, stream=None, rule: int = RDSPLIT_TRANSFER_MEAN,
                 reorder: bool = False):
        if reorder:
            self.h = rdsplit_mesh_create_ex(mesh.n_tets, mesh.adj, mesh.vol, mesh.area, mesh.dist, mesh.centroid,
                                            RDSPLIT_REORDER_SFC)
        else:
            self.h = rdsplit_mesh_create(mesh.n_tets, mesh.adj, mesh.vol, mesh.area, mesh.dist)
        try:
            rdsplit_set_model(self.h, model.n_species, model.D, model.n_reactions, model.lhs, model.rhs,
                              model.k, model.mask, model.tau_scale)
            if rule != RDSPLIT_TRANSFER_MEAN:
                rdsplit_set_transfer_rule(self.h, rule)
            if stream is not None:
                rdsplit_set_stream(self.h, stream)
            if counts is not None:
                rdsplit_set_counts(self.h, counts)
        except Exception:
            rdsplit_mesh_destroy(self.h)
            self.h = None
            raise

    def set_counts(self, counts):
        rdsplit_set_counts(self.h, counts)

    def run(self, t_end: float, seed: int):
        rdsplit_run(self.h, t_end, seed)

    def run_periods(self, n: int, seed: int):
        rdsplit_run_periods(self.h, n, seed)

    def counts(self):
        return rdsplit_get_counts(self.h)

    @property
    def tau(self) -> float:
        return rdsplit_get_tau(self.h)

    @property
    def time(self):
        return rdsplit_get_time(self.h)

    def close(self):
        if self.h is not None:
            rdsplit_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
