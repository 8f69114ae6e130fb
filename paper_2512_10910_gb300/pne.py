"""ctypes binding of libpne (include/pne.h): the same calls, argument marshalling only.

Every step of the expansion runs inside the CUDA library; this module only
packs arrays, pointers and streams.  It raises if the compiled library is
missing -- there is no fallback path.

Low-level names mirror the C ABI (``pne_ctx_create``, ``pne_build_partition``,
``pne_enumerate_terms``, ``pne_contract_terms``, ``pne_sum`` ...).  ``Context``
and ``run`` wrap one full pass for convenience.
"""
from __future__ import annotations

import ctypes
import collections.abc
import os

import numpy as np

__all__ = [
    "PNE_OK", "PNE_F64", "PNE_F32", "PNE_TF32", "PNE_BF16", "PNE_MODE_LOOP", "PNE_MODE_ALL",
    "PneError", "load_library", "lib_path", "exported_symbols",
    "pne_ctx_create", "pne_ctx_destroy", "pne_last_error", "pne_ctx_set_allocator",
    "pne_build_partition", "pne_partition_destroy", "pne_enumerate_terms", "pne_terms_destroy",
    "pne_contract_terms", "pne_sum", "pne_terms_n_results", "pne_terms_export",
    "pne_ctx_profile", "pne_ctx_profile_read", "pne_ctx_trace_read", "pne_terms_work", "pne_measure_fma_peak",
    "pne_bp_messages_noalloc", "pne_partition_update", "pne_batch_create", "pne_batch_run", "pne_batch_n_results", "pne_batch_config",
    "pne_batch_schedule", "pne_batch_destroy", "BatchOpts", "PNE_SCHED_HANDLE", "PNE_SCHED_LARGEST_FIRST",
    "pne_server_create", "pne_server_submit", "pne_server_poll",
    "pne_server_drain", "pne_server_stats", "pne_server_first_error", "pne_server_destroy", "ServerOpts", "RequestInfo",
    "Network", "PartitionOpts", "user_projector_opts", "EnumOpts", "Result", "Context", "run", "network_struct",
    "pne_strip_expansion", "StripOpts", "StripResult", "PNE_STRIP_MAX_L", "PNE_STRIP_MAX_CHI",
    "pne_dense_gemm", "pne_grid_contract", "pne_rank_r_expand_grid", "pne_rank_r_expand",
    "pne_recursive_expand_grid", "pne_weight_passing", "pne_weights_read", "pne_weights_destroy",
]

PNE_OK, PNE_EINVAL, PNE_ENOMEM, PNE_ECUDA, PNE_ENOCONV, PNE_EDEGENERATE, PNE_ETIMEOUT, PNE_EOVERFLOW, PNE_EBUSY = range(9)
PNE_F64, PNE_F32, PNE_TF32, PNE_BF16 = range(4)
PNE_MODE_LOOP, PNE_MODE_ALL, PNE_MODE_COMB = 0, 1, 2
PNE_MAX_ORDER = 32
MAX_ORDER = 32
DTYPES = {"f64": PNE_F64, "f32": PNE_F32, "tf32": PNE_TF32, "bf16": PNE_BF16}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libpne.so")
_lib = None


class PneError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class Network(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int32), ("n_bonds", ctypes.c_int32),
                ("bond_site", ctypes.POINTER(ctypes.c_int32)),
                ("bond_dim", ctypes.POINTER(ctypes.c_int32)),
                ("site_ptr", ctypes.POINTER(ctypes.c_int32)),
                ("site_bonds", ctypes.POINTER(ctypes.c_int32)),
                ("data", ctypes.c_void_p),
                ("data_off", ctypes.POINTER(ctypes.c_int64)),
                ("data_on_device", ctypes.c_int32),
                ("n_batch", ctypes.c_int32)]


class PartitionOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("damping", ctypes.c_double),
                ("arithmetic", ctypes.c_int32), ("async_status", ctypes.c_int32),
                ("use_user_projectors", ctypes.c_int32), ("user_u", ctypes.POINTER(ctypes.c_double)),
                ("user_v", ctypes.POINTER(ctypes.c_double))]


def user_projector_opts(u, v, **kw):
    """PartitionOpts with user projectors P_b = u_b v_b^T / (u_b . v_b): u and v
    are FP64 arrays laid out [tensor set][closed bonds in id order][bond_dim[b]]
    (flattened).  Returns (opts, keep): keep holds the arrays for the call."""
    u = np.ascontiguousarray(u, dtype=np.float64).ravel()
    v = np.ascontiguousarray(v, dtype=np.float64).ravel()
    if u.shape != v.shape:
        raise ValueError("user_u and user_v must have the same length")
    o = PartitionOpts(kw.get("tol", 1e-13), kw.get("max_iter", 10000), kw.get("damping", 0.0),
                      kw.get("arithmetic", 0), kw.get("async_status", 0))
    o.use_user_projectors = 1
    o.user_u = u.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    o.user_v = v.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return o, (u, v)


class EnumOpts(ctypes.Structure):
    _fields_ = [("max_order", ctypes.c_int32), ("mode", ctypes.c_int32), ("use_cache", ctypes.c_int32),
                ("max_cluster", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("sign", ctypes.c_int32), ("log_abs", ctypes.c_double), ("value", ctypes.c_double),
                ("c", ctypes.c_double * (MAX_ORDER + 1)), ("abs_c", ctypes.c_double * (MAX_ORDER + 1)),
                ("n_orders", ctypes.c_int32), ("log_abs_zref", ctypes.c_double), ("sign_zref", ctypes.c_int32),
                ("n_zero_sites", ctypes.c_int32), ("log_series", ctypes.c_double),
                ("err_bound", ctypes.c_double), ("n_terms", ctypes.c_uint64), ("n_clusters", ctypes.c_uint64),
                ("bp_iters", ctypes.c_int32), ("bp_residual", ctypes.c_double)]

    def as_dict(self) -> dict:
        n = self.n_orders
        return dict(sign=self.sign, log_abs=self.log_abs, value=self.value,
                    c=np.array(self.c[:n]), abs_c=np.array(self.abs_c[:n]),
                    log_abs_zref=self.log_abs_zref, sign_zref=self.sign_zref,
                    n_zero_sites=self.n_zero_sites, log_series=self.log_series,
                    err_bound=self.err_bound, n_terms=int(self.n_terms), n_clusters=int(self.n_clusters),
                    bp_iters=self.bp_iters, bp_residual=self.bp_residual)


class BatchOpts(ctypes.Structure):
    _fields_ = [("warps_per_block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("schedule", ctypes.c_int32)]


PNE_SCHED_HANDLE, PNE_SCHED_LARGEST_FIRST = 0, 1


class ServerOpts(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_int32),
                ("n_prep_streams", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("warps_per_block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("t_arrival", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_ready", ctypes.c_double),
                ("t_done", ctypes.c_double), ("device_bytes", ctypes.c_uint64), ("batch_size", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


PNE_STRIP_MAX_L, PNE_STRIP_MAX_CHI = 12, 8


class StripOpts(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("two_d", ctypes.c_int32), ("bp_tol", ctypes.c_double),
                ("eig_tol", ctypes.c_double), ("bp_max_iter", ctypes.c_int32), ("eig_max_iter", ctypes.c_int32),
                ("arithmetic", ctypes.c_int32)]


_SM1 = PNE_STRIP_MAX_L + 1


class StripResult(ctypes.Structure):
    _fields_ = [("f", ctypes.c_double), ("f_bp", ctypes.c_double),
                ("log_lambda", ctypes.c_double * _SM1), ("log_gamma", ctypes.c_double * _SM1),
                ("log_z", ctypes.c_double * (_SM1 * _SM1)), ("sign_z", ctypes.c_int32 * (_SM1 * _SM1)),
                ("messages", ctypes.c_double * (4 * PNE_STRIP_MAX_CHI)), ("eig_change", ctypes.c_double),
                ("bp_sweeps", ctypes.c_int32), ("eig_iters", ctypes.c_int32), ("status", ctypes.c_int),
                ("iters", ctypes.c_int32 * (2 * _SM1))]

    def as_dict(self, L, chi):
        lz = np.ctypeslib.as_array(self.log_z).reshape(_SM1, _SM1)
        sz = np.ctypeslib.as_array(self.sign_z).reshape(_SM1, _SM1)
        msg = np.ctypeslib.as_array(self.messages).reshape(4, PNE_STRIP_MAX_CHI)[:, :chi]
        return {"f": self.f, "f_bp": self.f_bp,
                "log_lam": [None] + list(self.log_lambda[1:L + 1]),
                "log_gam": [None] + list(self.log_gamma[1:L + 1]),
                "log_z": [None] + [[None] + list(lz[w, 1:L + 1]) for w in range(1, L + 1)],
                "sign_z": [None] + [[None] + [int(x) for x in sz[w, 1:L + 1]] for w in range(1, L + 1)],
                "msgs": tuple(np.array(m) for m in msg), "eig_change": self.eig_change,
                "bp_sweeps": self.bp_sweeps, "eig_iters": self.eig_iters, "status": self.status,
                "iters": [list(self.iters[0:L + 1]), list(self.iters[_SM1:_SM1 + L + 1])]}


class ProfileEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class TraceEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("kind", ctypes.c_int32), ("stream", ctypes.c_int32),
                ("t0_ms", ctypes.c_double), ("t1_ms", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


def lib_path() -> str:
    return _LIB_PATH


def load_library():
    """Load libpne.so; raise if it was not built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libpne.so not built at {_LIB_PATH}; run paper_2512_10910_gb300.build.build()")
    lib = ctypes.CDLL(_LIB_PATH)
    vp = ctypes.c_void_p
    lib.pne_ctx_create.argtypes = [ctypes.c_int, ctypes.POINTER(vp)]
    lib.pne_ctx_create.restype = ctypes.c_int
    lib.pne_ctx_destroy.argtypes = [vp]
    lib.pne_ctx_destroy.restype = None
    lib.pne_last_error.argtypes = [vp]
    lib.pne_last_error.restype = ctypes.c_char_p
    lib.pne_ctx_set_allocator.argtypes = [vp, ALLOC_FN, FREE_FN, vp]
    lib.pne_ctx_set_allocator.restype = ctypes.c_int
    lib.pne_build_partition.argtypes = [vp, ctypes.POINTER(Network), ctypes.POINTER(PartitionOpts), vp, ctypes.POINTER(vp)]
    lib.pne_build_partition.restype = ctypes.c_int
    lib.pne_partition_destroy.argtypes = [vp]
    lib.pne_partition_destroy.restype = None
    lib.pne_enumerate_terms.argtypes = [vp, vp, ctypes.POINTER(EnumOpts), vp, ctypes.POINTER(vp),
                                        ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
    lib.pne_enumerate_terms.restype = ctypes.c_int
    lib.pne_terms_destroy.argtypes = [vp]
    lib.pne_terms_destroy.restype = None
    lib.pne_contract_terms.argtypes = [vp, vp, ctypes.c_int, vp]
    lib.pne_contract_terms.restype = ctypes.c_int
    lib.pne_sum.argtypes = [vp, vp, vp, ctypes.POINTER(Result)]
    lib.pne_sum.restype = ctypes.c_int
    lib.pne_terms_n_results.argtypes = [vp]
    lib.pne_terms_n_results.restype = ctypes.c_int64
    lib.pne_enumerate_combinatorial.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, vp,
                                                ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_uint64),
                                                ctypes.POINTER(ctypes.c_uint64)]
    lib.pne_enumerate_combinatorial.restype = ctypes.c_int
    lib.pne_weight_passing.argtypes = [vp, ctypes.POINTER(Network), ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                       vp, ctypes.POINTER(vp)]
    lib.pne_weight_passing.restype = ctypes.c_int
    lib.pne_weights_read.argtypes = [vp, vp, vp, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.pne_weights_read.restype = ctypes.c_int
    lib.pne_weights_destroy.argtypes = [vp]
    lib.pne_weights_destroy.restype = None
    lib.pne_rank_r_expand.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.c_void_p, vp, ctypes.POINTER(Result)]
    lib.pne_rank_r_expand.restype = ctypes.c_int
    lib.pne_strip_expansion.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                        ctypes.POINTER(StripOpts), vp, ctypes.POINTER(StripResult)]
    lib.pne_strip_expansion.restype = ctypes.c_int
    lib.pne_dense_gemm.argtypes = [vp, ctypes.c_int, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                   ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, vp]
    lib.pne_dense_gemm.restype = ctypes.c_int
    lib.pne_grid_contract.argtypes = [vp, ctypes.POINTER(Network), ctypes.c_int32, ctypes.c_int32, ctypes.c_int, vp,
                                      ctypes.POINTER(Result)]
    lib.pne_grid_contract.restype = ctypes.c_int
    lib.pne_rank_r_expand_grid.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int, vp,
                                           ctypes.POINTER(Result)]
    lib.pne_rank_r_expand_grid.restype = ctypes.c_int
    lib.pne_recursive_expand_grid.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_int32, ctypes.c_int, vp, ctypes.POINTER(Result),
                                              ctypes.POINTER(ctypes.c_uint64)]
    lib.pne_recursive_expand_grid.restype = ctypes.c_int
    lib.pne_open_tensor.argtypes = [vp, vp, vp, ctypes.c_void_p, ctypes.c_void_p]
    lib.pne_open_tensor.restype = ctypes.c_int
    lib.pne_open_tensor_assemble.argtypes = [ctypes.POINTER(Result), ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                             ctypes.c_void_p]
    lib.pne_open_tensor_assemble.restype = ctypes.c_int
    lib.pne_terms_export.argtypes = [vp, vp, vp, ctypes.c_void_p, ctypes.c_void_p]
    lib.pne_terms_export.restype = ctypes.c_int
    lib.pne_bp_messages_noalloc.argtypes = [ctypes.POINTER(Network), ctypes.c_double, ctypes.c_int32, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, vp]
    lib.pne_bp_messages_noalloc.restype = ctypes.c_int
    lib.pne_partition_update.argtypes = [vp, vp, ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(PartitionOpts), vp]
    lib.pne_partition_update.restype = ctypes.c_int
    lib.pne_batch_create.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(BatchOpts), vp,
                                     ctypes.POINTER(vp)]
    lib.pne_batch_create.restype = ctypes.c_int
    lib.pne_batch_run.argtypes = [vp, vp, vp, ctypes.POINTER(Result)]
    lib.pne_batch_run.restype = ctypes.c_int
    lib.pne_batch_n_results.argtypes = [vp]
    lib.pne_batch_n_results.restype = ctypes.c_int64
    lib.pne_batch_config.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_double)]
    lib.pne_batch_config.restype = ctypes.c_int
    lib.pne_batch_schedule.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
    lib.pne_batch_schedule.restype = ctypes.c_int
    lib.pne_batch_destroy.argtypes = [vp]
    lib.pne_batch_destroy.restype = None
    lib.pne_server_create.argtypes = [vp, ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]
    lib.pne_server_create.restype = ctypes.c_int
    lib.pne_server_submit.argtypes = [vp, ctypes.POINTER(Network), ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64)]
    lib.pne_server_submit.restype = ctypes.c_int
    lib.pne_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(Result), ctypes.POINTER(RequestInfo)]
    lib.pne_server_poll.restype = ctypes.c_int
    lib.pne_server_drain.argtypes = [vp]
    lib.pne_server_drain.restype = ctypes.c_int
    lib.pne_server_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double)]
    lib.pne_server_stats.restype = ctypes.c_int
    lib.pne_server_first_error.argtypes = [vp]
    lib.pne_server_first_error.restype = ctypes.c_char_p
    lib.pne_server_destroy.argtypes = [vp]
    lib.pne_server_destroy.restype = None
    lib.pne_ctx_profile.argtypes = [vp, ctypes.c_int]
    lib.pne_ctx_profile.restype = ctypes.c_int
    lib.pne_ctx_profile_read.argtypes = [vp, ctypes.POINTER(ProfileEntry), ctypes.c_int]
    lib.pne_ctx_profile_read.restype = ctypes.c_int
    lib.pne_ctx_trace_read.argtypes = [vp, ctypes.POINTER(TraceEntry), ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.pne_ctx_trace_read.restype = ctypes.c_int
    lib.pne_terms_work.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.pne_terms_work.restype = ctypes.c_int
    lib.pne_measure_fma_peak.argtypes = [vp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_double)]
    lib.pne_measure_fma_peak.restype = ctypes.c_int
    _lib = lib
    return lib


def exported_symbols() -> list:
    """Names of the ``pne_*`` functions ``include/pne.h`` declares, found in the library."""
    lib = load_library()
    names = ["pne_ctx_create", "pne_ctx_destroy", "pne_last_error", "pne_ctx_set_allocator",
             "pne_build_partition", "pne_partition_destroy", "pne_enumerate_terms", "pne_terms_destroy",
             "pne_enumerate_combinatorial", "pne_contract_terms", "pne_sum", "pne_terms_n_results", "pne_open_tensor", "pne_open_tensor_assemble",
             "pne_terms_export",
             "pne_ctx_profile", "pne_ctx_profile_read", "pne_ctx_trace_read", "pne_terms_work", "pne_measure_fma_peak",
             "pne_bp_messages_noalloc", "pne_partition_update", "pne_batch_create", "pne_batch_run",
             "pne_batch_n_results", "pne_batch_config", "pne_batch_schedule", "pne_batch_destroy", "pne_server_create",
             "pne_server_submit", "pne_server_poll", "pne_server_drain", "pne_server_stats", "pne_server_first_error",
             "pne_server_destroy", "pne_weight_passing", "pne_weights_read", "pne_weights_destroy",
             "pne_rank_r_expand", "pne_strip_expansion", "pne_dense_gemm", "pne_grid_contract",
             "pne_rank_r_expand_grid", "pne_recursive_expand_grid"]
    return [n for n in names if hasattr(lib, n)]


def _check(st, ctx=None):
    if st != PNE_OK:
        msg = load_library().pne_last_error(ctx).decode() if ctx is not None else "pne call failed"
        raise PneError(st, msg)


# ------------------------------------------------------------------ the C calls
def pne_ctx_create(device=0):
    h = ctypes.c_void_p()
    _check(load_library().pne_ctx_create(int(device), ctypes.byref(h)))
    return h


def pne_ctx_destroy(ctx):
    load_library().pne_ctx_destroy(ctx)


def pne_last_error(ctx=None) -> str:
    return load_library().pne_last_error(ctx).decode()


def pne_ctx_set_allocator(ctx, alloc_fn, free_fn, user=None):
    _check(load_library().pne_ctx_set_allocator(ctx, alloc_fn, free_fn, user), ctx)


def pne_build_partition(ctx, net: Network, opts: PartitionOpts, stream=None, allow_noconv=False):
    h = ctypes.c_void_p()
    st = load_library().pne_build_partition(ctx, ctypes.byref(net), ctypes.byref(opts), stream, ctypes.byref(h))
    if st == PNE_ENOCONV and allow_noconv:
        return h, st
    _check(st, ctx)
    return h, st


def pne_partition_destroy(p):
    load_library().pne_partition_destroy(p)


def pne_enumerate_terms(ctx, part, opts: EnumOpts, stream=None):
    h = ctypes.c_void_p()
    nc, nt = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load_library().pne_enumerate_terms(ctx, part, ctypes.byref(opts), stream, ctypes.byref(h),
                                              ctypes.byref(nc), ctypes.byref(nt)), ctx)
    return h, nc.value, nt.value


def pne_enumerate_combinatorial(ctx, part, partitions, stream=None):
    """Combinatorial-form handle over multi-index partitions (each a list of
    bond ids of the network).  Returns (terms, n_components, n_terms)."""
    ptr = np.zeros(len(partitions) + 1, dtype=np.int32)
    for i, S in enumerate(partitions):
        ptr[i + 1] = ptr[i] + len(S)
    bonds = np.ascontiguousarray(np.concatenate([np.asarray(S, dtype=np.int32) for S in partitions]), dtype=np.int32)
    h = ctypes.c_void_p()
    nc, nt = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load_library().pne_enumerate_combinatorial(ctx, part, len(partitions), ptr.ctypes.data, bonds.ctypes.data,
                                                      stream, ctypes.byref(h), ctypes.byref(nc), ctypes.byref(nt)), ctx)
    return h, int(nc.value), int(nt.value)


def pne_weight_passing(ctx, net: Network, alpha=0.8, tol=1e-12, max_sweeps=5000, stream=None, allow_noconv=False):
    """Weight passing (App. C) on the device; returns the handle."""
    h = ctypes.c_void_p()
    st = load_library().pne_weight_passing(ctx, ctypes.byref(net), float(alpha), float(tol), int(max_sweeps), stream,
                                           ctypes.byref(h))
    if not (st == PNE_ENOCONV and allow_noconv):
        _check(st, ctx)
    return h


def pne_weights_read(ctx, w, n_sets, n_bonds, stream=None):
    """(weights [n_sets, n_bonds, 16], sweeps [n_sets], log_scale [n_sets])."""
    wts = np.zeros((n_sets, max(n_bonds, 1), 16))
    sw = np.zeros(n_sets, dtype=np.int32)
    ls = np.zeros(n_sets)
    _check(load_library().pne_weights_read(ctx, w, stream, wts.ctypes.data, sw.ctypes.data, ls.ctypes.data), ctx)
    return wts[:, :n_bonds], sw, ls


def pne_weights_destroy(w):
    load_library().pne_weights_destroy(w)


def pne_rank_r_expand(ctx, w, rank, form, partitions, n_sets, stream=None):
    """The rank-r expansion (form 0 linear, 1 combinatorial) on the weights:
    one result dict per tensor set."""
    ptr = np.zeros(len(partitions) + 1, dtype=np.int32)
    for i, S in enumerate(partitions):
        ptr[i + 1] = ptr[i] + len(S)
    bonds = np.ascontiguousarray(np.concatenate([np.asarray(S, dtype=np.int32) for S in partitions]), dtype=np.int32)
    out = (Result * n_sets)()
    _check(load_library().pne_rank_r_expand(ctx, w, int(rank), int(form), len(partitions), ptr.ctypes.data,
                                            bonds.ctypes.data, stream, out), ctx)
    return [r.as_dict() for r in out]


def pne_strip_expansion(ctx, A, L, two_d=True, bp_tol=0.0, eig_tol=0.0, bp_max_iter=0, eig_max_iter=0,
                        arithmetic=0, stream=None, allow_noconv=False):
    """The infinite-lattice strip expansion (Sec. IV.C) of uniform tensors:
    ``A`` a [n, chi, chi, chi, chi] (or one [chi]*4) host array or a CUDA
    tensor; one result dict per tensor (log lists indexed from 1)."""
    dev = hasattr(A, "data_ptr")
    if dev:
        if A.dim() == 4:
            A = A.unsqueeze(0)
        A = A.contiguous()
        n, chi = int(A.shape[0]), int(A.shape[1])
        ptr = A.data_ptr()
    else:
        A = np.ascontiguousarray(A, dtype=np.float64)
        if A.ndim == 4:
            A = A[None]
        n, chi = A.shape[0], A.shape[1]
        ptr = A.ctypes.data
    opts = StripOpts(int(L), 1 if two_d else 0, float(bp_tol), float(eig_tol), int(bp_max_iter), int(eig_max_iter),
                     int(arithmetic))
    out = (StripResult * n)()
    st = load_library().pne_strip_expansion(ctx, int(chi), int(n), ptr, 1 if dev else 0, ctypes.byref(opts), stream,
                                            out)
    if not (st == PNE_ENOCONV and allow_noconv):
        _check(st, ctx)
    return [r.as_dict(int(L), int(chi)) for r in out]


def pne_dense_gemm(ctx, dtype, A, B, C, stream=None):
    """C[b] = A[b] B[b]^T for CUDA tensors A [batch, M, K], B [batch, N, K],
    C [batch, M, N] (FP32 for TF32/BF16, FP64 for F64; contiguous rows)."""
    batch, M, K = (int(x) for x in A.shape)
    N = int(B.shape[1])
    _check(load_library().pne_dense_gemm(ctx, int(dtype), batch, M, N, K, A.data_ptr(), A.stride(1), A.stride(0),
                                         B.data_ptr(), B.stride(1), B.stride(0), C.data_ptr(), C.stride(1),
                                         C.stride(0), stream), ctx)


def pne_grid_contract(ctx, net, lx, ly, dtype, data=None, n_batch=None, stream=None):
    """Exact contraction of a closed lx x ly grid network (site id = y * lx +
    x); one result dict per tensor set."""
    ns, keep = network_struct(net, data=data, n_batch=n_batch or 1)
    nb = int(ns.n_batch)
    out = (Result * nb)()
    _check(load_library().pne_grid_contract(ctx, ctypes.byref(ns), int(lx), int(ly), int(dtype), stream, out), ctx)
    del keep
    return [r.as_dict() for r in out]


def pne_rank_r_expand_grid(ctx, w, rank, form, partitions, n_sets, lx, ly, dtype, stream=None):
    """The rank-r expansion with every term contracted as a grid (row-by-row
    GEMMs; F64, TF32 or BF16): one result dict per tensor set."""
    ptr = np.zeros(len(partitions) + 1, dtype=np.int32)
    for i, S in enumerate(partitions):
        ptr[i + 1] = ptr[i] + len(S)
    bonds = np.ascontiguousarray(np.concatenate([np.asarray(S, dtype=np.int32) for S in partitions]), dtype=np.int32)
    out = (Result * n_sets)()
    _check(load_library().pne_rank_r_expand_grid(ctx, w, int(rank), int(form), len(partitions), ptr.ctypes.data,
                                                 bonds.ctypes.data, int(lx), int(ly), int(dtype), stream, out), ctx)
    return [r.as_dict() for r in out]


def _csr(partitions):
    ptr = np.zeros(len(partitions) + 1, dtype=np.int32)
    for i, S in enumerate(partitions):
        ptr[i + 1] = ptr[i] + len(S)
    bonds = (np.ascontiguousarray(np.concatenate([np.asarray(S, dtype=np.int32) for S in partitions]), dtype=np.int32)
             if partitions else np.zeros(1, dtype=np.int32))
    return ptr, bonds


def pne_recursive_expand_grid(ctx, w, rank, partitions, sub_partitions, max_side, n_sets, lx, ly, dtype,
                              stream=None):
    """Recursive partitioning on the weights' rank-r projectors: (results, networks contracted)."""
    p1, b1 = _csr(partitions)
    p2, b2 = _csr(sub_partitions)
    out = (Result * n_sets)()
    n = ctypes.c_uint64()
    _check(load_library().pne_recursive_expand_grid(ctx, w, int(rank), len(partitions), p1.ctypes.data,
                                                    b1.ctypes.data, len(sub_partitions), p2.ctypes.data,
                                                    b2.ctypes.data, int(max_side), int(lx), int(ly), int(dtype),
                                                    stream, out, ctypes.byref(n)), ctx)
    return [r.as_dict() for r in out], int(n.value)


def pne_terms_destroy(t):
    load_library().pne_terms_destroy(t)


def pne_contract_terms(ctx, terms, dtype, stream=None):
    _check(load_library().pne_contract_terms(ctx, terms, int(dtype), stream), ctx)


def pne_terms_n_results(terms) -> int:
    return int(load_library().pne_terms_n_results(terms))


def pne_terms_export(ctx, terms, n_clusters, K, with_values=True, stream=None):
    """(edges [n_clusters, K] int32, w [n_results, n_clusters] float64 or None)."""
    edges = np.full((max(n_clusters, 1), max(K, 1)), -1, dtype=np.int32)
    w = np.zeros((pne_terms_n_results(terms), max(n_clusters, 1))) if with_values else None
    _check(load_library().pne_terms_export(ctx, terms, stream, edges.ctypes.data,
                                           w.ctypes.data if w is not None else None), ctx)
    return edges[:n_clusters], (w[:, :n_clusters] if w is not None else None)


def pne_bp_messages_noalloc(net: Network, msg_out_ptr, tol=1e-13, max_iter=10000, stream=None):
    """Allocation-free BP (see include/pne.h): fixed-point messages written to
    the caller's device buffer ``msg_out_ptr`` ([n_batch][n_legs][8] doubles).
    Returns (iters, residuals) per tensor set."""
    B = int(net.n_batch)
    iters = np.zeros(B, dtype=np.int32)
    res = np.zeros(B, dtype=np.float64)
    st = load_library().pne_bp_messages_noalloc(ctypes.byref(net), float(tol), int(max_iter), ctypes.c_void_p(msg_out_ptr),
                                                 iters.ctypes.data, res.ctypes.data, stream)
    _check(st, ctypes.c_void_p(0))
    return iters, res


def pne_partition_update(ctx, part, data, opts: PartitionOpts = None, stream=None):
    """Re-run a partition on new tensors (host numpy or device torch tensor)."""
    opts = opts or PartitionOpts(1e-13, 10000, 0.0)
    if hasattr(data, "data_ptr"):
        ptr, dev = data.data_ptr(), int(bool(data.is_cuda))
    else:
        data = np.ascontiguousarray(data, dtype=np.float64)
        ptr, dev = data.ctypes.data, 0
    _check(load_library().pne_partition_update(ctx, part, ctypes.c_void_p(ptr), dev, ctypes.byref(opts), stream), ctx)


def pne_batch_create(ctx, terms_list, dtype, opts: BatchOpts = None, stream=None):
    arr = (ctypes.c_void_p * len(terms_list))(*[t.value if isinstance(t, ctypes.c_void_p) else t for t in terms_list])
    h = ctypes.c_void_p()
    _check(load_library().pne_batch_create(ctx, len(terms_list), arr, int(dtype),
                                           ctypes.byref(opts) if opts is not None else None, stream, ctypes.byref(h)), ctx)
    return h


def pne_batch_n_results(b) -> int:
    return int(load_library().pne_batch_n_results(b))


def pne_batch_run(ctx, b, stream=None):
    n = pne_batch_n_results(b)
    out = (Result * n)()
    _check(load_library().pne_batch_run(ctx, b, stream, out), ctx)
    return [r.as_dict() for r in out]


def pne_batch_config(b):
    w, k, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(load_library().pne_batch_config(b, ctypes.byref(w), ctypes.byref(k), ctypes.byref(ms)))
    return int(w.value), int(k.value), float(ms.value)


def pne_batch_schedule(b) -> int:
    v = ctypes.c_int32()
    _check(load_library().pne_batch_schedule(b, ctypes.byref(v)))
    return int(v.value)


def pne_batch_destroy(b):
    load_library().pne_batch_destroy(b)


def pne_server_create(ctx, opts: ServerOpts = None):
    h = ctypes.c_void_p()
    _check(load_library().pne_server_create(ctx, ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)), ctx)
    return h


def pne_server_submit(srv, net: Network, max_order) -> int:
    i = ctypes.c_uint64()
    _check(load_library().pne_server_submit(srv, ctypes.byref(net), int(max_order), ctypes.byref(i)))
    return int(i.value)


def pne_server_poll(srv, rid):
    """(status, result dict or None, info dict or None); status PNE_EBUSY while pending."""
    r, info = Result(), RequestInfo()
    st = load_library().pne_server_poll(srv, ctypes.c_uint64(rid), ctypes.byref(r), ctypes.byref(info))
    if st == PNE_EBUSY:
        return st, None, None
    return st, (r.as_dict() if st == PNE_OK else None), info.as_dict()


def pne_server_drain(srv):
    _check(load_library().pne_server_drain(srv))


def pne_server_stats(srv):
    b, t = ctypes.c_uint64(), ctypes.c_double()
    _check(load_library().pne_server_stats(srv, ctypes.byref(b), ctypes.byref(t)))
    return int(b.value), float(t.value)


def pne_server_first_error(srv) -> str:
    """Error text of the first failed request ('' while none has)."""
    return (load_library().pne_server_first_error(srv) or b"").decode()


def pne_server_destroy(srv):
    load_library().pne_server_destroy(srv)


def pne_ctx_profile(ctx, enable=True, trace=False):
    """Turn the per-kernel event timing on or off; ``trace`` also keeps a timeline."""
    _check(load_library().pne_ctx_profile(ctx, 2 if (enable and trace) else int(bool(enable))), ctx)


def pne_ctx_profile_read(ctx) -> dict:
    """{kernel family: (launches, total_ms)}, largest total first."""
    lib = load_library()
    buf = (ProfileEntry * 64)()
    n = lib.pne_ctx_profile_read(ctx, buf, 64)
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(min(n, 64))}


def pne_ctx_trace_read(ctx):
    """(entries, host_origin_ms): the timeline since ``pne_ctx_profile(ctx, trace=True)``
    as dicts {name, kind ('gpu'|'host'), stream, t0_ms, t1_ms}, sorted by start."""
    lib = load_library()
    origin = ctypes.c_double()
    n = lib.pne_ctx_trace_read(ctx, None, 0, ctypes.byref(origin))
    buf = (TraceEntry * max(n, 1))()
    n = min(n, lib.pne_ctx_trace_read(ctx, buf, max(n, 1), ctypes.byref(origin)))
    out = [{"name": buf[i].name.decode(), "kind": "gpu" if buf[i].kind == 0 else "host",
            "stream": int(buf[i].stream), "t0_ms": float(buf[i].t0_ms), "t1_ms": float(buf[i].t1_ms)}
           for i in range(n)]
    return out, float(origin.value)


def pne_terms_work(ctx, terms, stream=None) -> int:
    v = ctypes.c_uint64()
    _check(load_library().pne_terms_work(ctx, terms, stream, ctypes.byref(v)), ctx)
    return int(v.value)


def pne_measure_fma_peak(ctx, dtype, stream=None) -> float:
    v = ctypes.c_double()
    _check(load_library().pne_measure_fma_peak(ctx, int(dtype), stream, ctypes.byref(v)), ctx)
    return float(v.value)


def pne_sum(ctx, terms, stream=None, allow_noconv=False):
    """Results of every tensor set and open-index assignment.  With a partition
    built with async_status, a BP record that shows non-convergence makes this
    raise unless allow_noconv (then the results carry bp_iters == 0)."""
    n = pne_terms_n_results(terms)
    out = (Result * n)()
    st = load_library().pne_sum(ctx, terms, stream, out)
    if not (st == PNE_ENOCONV and allow_noconv):
        _check(st, ctx)
    return Results(out)


def pne_open_tensor(ctx, terms, n_sets, open_dims, stream=None, allow_noconv=False):
    """The open-index tensors of every tensor set through the C call: returns
    (mantissa [n_sets, *open_dims], log_scale [n_sets]); the tensor of set b is
    mantissa[b] * exp(log_scale[b])."""
    n = pne_terms_n_results(terms)
    out = np.zeros(n, dtype=np.float64)
    ls = np.zeros(n_sets, dtype=np.float64)
    st = load_library().pne_open_tensor(ctx, terms, stream, out.ctypes.data, ls.ctypes.data)
    if not (st == PNE_ENOCONV and allow_noconv):
        _check(st, ctx)
    return out.reshape((n_sets,) + tuple(open_dims)), ls


def pne_open_tensor_assemble(results, n_sets, open_dims):
    """The assembly step alone (host only) from pne_sum's results."""
    arr = results._arr if isinstance(results, Results) else results
    n_open = int(np.prod(open_dims)) if len(open_dims) else 1
    out = np.zeros(n_sets * n_open, dtype=np.float64)
    ls = np.zeros(n_sets, dtype=np.float64)
    _check(load_library().pne_open_tensor_assemble(arr, int(n_sets), n_open, out.ctypes.data, ls.ctypes.data))
    return out.reshape((n_sets,) + tuple(open_dims)), ls


class Results(collections.abc.Sequence):
    """The results of a pne_sum call as a sequence of dicts (``Result.as_dict``).
    The values are already in host memory; each dict is built on first access."""

    def __init__(self, arr):
        self._arr = arr
        self._dicts = {}

    def __len__(self):
        return len(self._arr)

    def __getitem__(self, i):
        if isinstance(i, slice):
            return [self[j] for j in range(*i.indices(len(self)))]
        if i < 0:
            i += len(self)
        if not 0 <= i < len(self):
            raise IndexError(i)
        d = self._dicts.get(i)
        if d is None:
            d = self._dicts[i] = self._arr[i].as_dict()
        return d

    def __repr__(self):
        return repr(list(self))


# ------------------------------------------------------------------ marshalling helpers
def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def network_struct(net, data=None, n_batch=1, data_on_device=False):
    """pne_network for an ``inputs.Network``.  ``data``: a flat FP64 array of
    n_batch tensor sets (numpy for host, a torch CUDA tensor for device), or
    None to use the network's own tensors.  Returns (struct, keepalive)."""
    bs, p_bs = _i32(net.bond_site.reshape(-1))
    bd, p_bd = _i32(net.bond_dim)
    sp, p_sp = _i32(net.site_ptr)
    sb, p_sb = _i32(net.site_bonds)
    if data is None:
        flat, off = net.flat_data()
        data = flat
    else:
        _, off = _offsets(net)
    off = np.ascontiguousarray(off, dtype=np.int64)
    if hasattr(data, "data_ptr"):
        ptr = data.data_ptr()
        data_on_device = bool(data.is_cuda)
    else:
        data = np.ascontiguousarray(data, dtype=np.float64)
        ptr = data.ctypes.data
    s = Network(net.n_sites, net.n_bonds, p_bs, p_bd, p_sp, p_sb, ctypes.c_void_p(ptr),
                off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(data_on_device), int(n_batch))
    return s, (bs, bd, sp, sb, off, data)


def _offsets(net):
    """Per-site tensor sizes (product of the leg dimensions) and their offsets,
    vectorised: one segmented product over the CSR legs."""
    ptr = np.asarray(net.site_ptr, dtype=np.int64)
    dims = np.asarray(net.bond_dim, dtype=np.int64)[np.asarray(net.site_bonds, dtype=np.int64)]
    sizes = np.ones(net.n_sites, dtype=np.int64)
    nonempty = np.diff(ptr) > 0
    if dims.size:
        sizes[nonempty] = np.multiply.reduceat(dims, ptr[:-1][nonempty])
    off = np.zeros(net.n_sites + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    return sizes, off


class Context:
    """Owns a pne_ctx on one device.  ``torch_alloc=True`` routes the library's
    device memory through PyTorch's caching allocator."""

    def __init__(self, device=0, torch_alloc=False):
        self.device = device
        self.h = pne_ctx_create(device)
        self._cbs = None
        if torch_alloc:
            import torch

            def _alloc(nbytes, stream, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0)
                except Exception:
                    return None

            def _free(ptr, nbytes, stream, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._cbs = (ALLOC_FN(_alloc), FREE_FN(_free))
            pne_ctx_set_allocator(self.h, self._cbs[0], self._cbs[1], None)

    def close(self):
        if self.h is not None:
            pne_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def expand(self, net, K, mode=PNE_MODE_LOOP, dtype=PNE_F64, data=None, n_batch=1, stream=None,
               tol=1e-13, max_iter=10000, damping=0.0, use_cache=True, allow_noconv=False,
               export=False, arithmetic=0, projectors=None, max_cluster=0):
        """One pass: partition -> enumerate -> contract -> sum.  Returns the
        list of result dicts (one per tensor set and open-index assignment);
        with export=True also (edges, w) of the clusters.  projectors=(u, v)
        replaces BP by user projectors (see user_projector_opts)."""
        if isinstance(dtype, str):
            dtype = DTYPES[dtype]
        ns, keep = network_struct(net, data=data, n_batch=n_batch)
        if projectors is not None:
            popts, pkeep = user_projector_opts(*projectors, arithmetic=arithmetic)
        else:
            popts, pkeep = PartitionOpts(tol, max_iter, damping, arithmetic), None
        part, st = pne_build_partition(self.h, ns, popts, stream, allow_noconv)
        del pkeep
        try:
            terms, nc, nt = pne_enumerate_terms(self.h, part, EnumOpts(K, mode, int(use_cache), max_cluster), stream)
            try:
                pne_contract_terms(self.h, terms, dtype, stream)
                res = pne_sum(self.h, terms, stream)
                if export:
                    res = (res, pne_terms_export(self.h, terms, nc, K, True, stream))
            finally:
                pne_terms_destroy(terms)
        finally:
            pne_partition_destroy(part)
        del keep
        return res


def _context_open_tensor(self, net, K, mode=PNE_MODE_LOOP, dtype=PNE_F64, data=None, n_batch=1, stream=None,
                         arithmetic=0):
    """One pass (partition -> enumerate -> contract) and the open-index tensor
    through pne_open_tensor: (mantissa [n_batch, *open_dims], log_scale)."""
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    open_dims = [int(net.bond_dim[b]) for b in range(net.n_bonds) if int(net.bond_site[b][1]) < 0]
    ns, keep = network_struct(net, data=data, n_batch=n_batch)
    part, _ = pne_build_partition(self.h, ns, PartitionOpts(1e-13, 10000, 0.0, arithmetic), stream)
    try:
        terms, _, _ = pne_enumerate_terms(self.h, part, EnumOpts(K, mode, 1), stream)
        try:
            pne_contract_terms(self.h, terms, dtype, stream)
            return pne_open_tensor(self.h, terms, n_batch, open_dims, stream)
        finally:
            pne_terms_destroy(terms)
    finally:
        pne_partition_destroy(part)
        del keep


Context.open_tensor = _context_open_tensor


def _context_combinatorial(self, net, partitions, dtype=PNE_F64, data=None, n_batch=1, stream=None, arithmetic=0,
                           export=False):
    """One pass of the combinatorial form (partition -> sub-network components
    -> contraction -> signed sums).  Returns the result dicts (one per tensor
    set); with export=True also (component edges, component values)."""
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    ns, keep = network_struct(net, data=data, n_batch=n_batch)
    part, _ = pne_build_partition(self.h, ns, PartitionOpts(1e-13, 10000, 0.0, arithmetic), stream)
    try:
        terms, nc, nt = pne_enumerate_combinatorial(self.h, part, partitions, stream)
        try:
            pne_contract_terms(self.h, terms, dtype, stream)
            res = pne_sum(self.h, terms, stream)
            if export:
                res = (res, pne_terms_export(self.h, terms, nc, PNE_MAX_ORDER, True, stream))
            return res
        finally:
            pne_terms_destroy(terms)
    finally:
        pne_partition_destroy(part)
        del keep


Context.combinatorial = _context_combinatorial


def _context_rank_r(self, net, partitions, rank, form, alpha=0.8, tol=1e-12, max_sweeps=5000, data=None, n_batch=1,
                    stream=None, grid=None, dtype=PNE_F64):
    """Weight passing then the rank-r expansion (form 0 linear over single-index
    partitions, 1 combinatorial): (results, weights, sweeps, log_scale).
    ``grid=(lx, ly)`` contracts the terms row by row as GEMMs (dtype F64 on the
    CUDA cores, TF32 / BF16 on the tensor cores)."""
    ns, keep = network_struct(net, data=data, n_batch=n_batch)
    w = pne_weight_passing(self.h, ns, alpha, tol, max_sweeps, stream)
    try:
        if grid is None:
            res = pne_rank_r_expand(self.h, w, rank, form, partitions, n_batch, stream)
        else:
            res = pne_rank_r_expand_grid(self.h, w, rank, form, partitions, n_batch, grid[0], grid[1], dtype, stream)
        wts, sw, ls = pne_weights_read(self.h, w, n_batch, int(net.n_bonds), stream)
        return res, wts, sw, ls
    finally:
        pne_weights_destroy(w)
        del keep


Context.rank_r = _context_rank_r


def run(net, K, mode=PNE_MODE_LOOP, dtype=PNE_F64, device=0, **kw):
    ctx = Context(device)
    try:
        return ctx.expand(net, K, mode, dtype, **kw)
    finally:
        ctx.close()


def open_tensor(results, open_dims, n_sets=1):
    """The open-index tensors (n_sets, *open_dims) from pne_sum's results,
    assembled by the library (pne_open_tensor_assemble) and scaled back to
    plain values; entries beyond the FP64 range become +-inf (use
    pne_open_tensor_assemble for the mantissa and its log scale)."""
    mant, ls = pne_open_tensor_assemble(results, n_sets, open_dims)
    with np.errstate(over="ignore", invalid="ignore"):
        scale = np.exp(np.where(np.isfinite(ls), ls, 0.0))
    return mant * scale.reshape((n_sets,) + (1,) * len(open_dims))
