"""B300-native bulk trace analysis (arxiv 2605.03561, the hpcanalysis trace path).

A thin ctypes binding over ``libta.so`` (C ABI in ``include/ta.h``).  Every
step of the analysis runs in the library's CUDA kernels; this module only
marshals arguments.  PyTorch supplies device memory (the library allocates
through torch's caching allocator) and the CUDA stream.  There is no CPU
fallback: if the extension cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libta.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "ta.h")

OK, INVALID_ARG, NOT_SORTED, BAD_CTX, BAD_CCT, OOM, CAPACITY, TIMEOUT, CUDA, STATE = range(10)
MEM_HOST, MEM_DEVICE = 0, 1
EXCLUSIVE, INCLUSIVE = 0, 1
LOAD_BORROW, LOAD_NO_INCLUSIVE, LOAD_KEEP_TRACES = 1, 2, 4
NO_PARENT = 0xFFFFFFFF
STATUS_NAMES = {0: "ok", 1: "invalid_arg", 2: "not_sorted", 3: "bad_ctx", 4: "bad_cct", 5: "oom",
                6: "capacity", 7: "timeout", 8: "cuda", 9: "state"}

P = C.c_void_p
u32, u64 = C.c_uint32, C.c_uint64


class TraceDesc(C.Structure):
    _fields_ = [("n_ranks", u32), ("n_ctx", u32), ("marker_ctx", u32), ("mem_kind", u32),
                ("n_records", u64), ("rank_off", P), ("ts", P), ("ctx", P), ("parent", P),
                ("flags", u32), ("reserved", u32), ("nnz_hint", u64), ("rows_hint", u64)]


class ExperimentInfo(C.Structure):
    _fields_ = [("n_ranks", u32), ("n_ctx", u32), ("marker_ctx", u32), ("max_depth", u32),
                ("n_records", u64), ("n_rows", u64), ("tensor_nnz", u64), ("excl_nnz", u64),
                ("incl_nnz", u64), ("device_bytes", u64)]


class TensorOut(C.Structure):
    _fields_ = [("mem_kind", u32), ("reserved", u32), ("n_iter", P), ("row_off_of_rank", P),
                ("entry_off", P), ("e_ctx", P), ("e_time", P), ("e_cnt", P), ("rows_cap", u64),
                ("nnz_cap", u64), ("rows", u64), ("nnz", u64)]


class CsrOut(C.Structure):
    _fields_ = [("mem_kind", u32), ("reserved", u32), ("off", P), ("ctx", P), ("time", P),
                ("cnt", P), ("nnz_cap", u64), ("nnz", u64)]


class TensorView(C.Structure):
    _fields_ = [("n_iter", P), ("row_off_of_rank", P), ("entry_off", P), ("e_ctx", P),
                ("e_time", P), ("e_cnt", P), ("span", P), ("rows", u64), ("nnz", u64)]


class CsrView(C.Structure):
    _fields_ = [("off", P), ("ctx", P), ("time", P), ("cnt", P), ("nnz", u64)]


class StatsArgs(C.Structure):
    _fields_ = [("metric", u32), ("mem_kind", u32), ("ranks", P), ("n_ranks_subset", u32),
                ("n_ctxs", u32), ("ctxs", P), ("tau_num", u32), ("tau_den", u32)]


class CtxStats(C.Structure):
    _fields_ = [("n", u32), ("present", u32), ("argmax", u32), ("reserved", u32), ("min", u64),
                ("max", u64), ("s1", u64), ("s2_lo", u64), ("s2_hi", u64), ("mean", C.c_double),
                ("std", C.c_double), ("cv", C.c_double), ("balance", C.c_double)]


class Outlier(C.Structure):
    _fields_ = [("ctx", u32), ("rank", u32), ("z", C.c_double)]


class StatsOut(C.Structure):
    _fields_ = [("stats", P), ("outliers", P), ("outlier_cap", u64), ("n_outliers", u64),
                ("z", P)]


class Topology(C.Structure):
    _fields_ = [("n_nodes", u32), ("n_chassis", u32), ("n_racks", u32), ("mem_kind", u32),
                ("node_of_rank", P), ("rack_of_node", P), ("chassis_of_node", P)]


class TopoArgs(C.Structure):
    _fields_ = [("metric", u32), ("ctx", u32), ("tau_num", u32), ("tau_den", u32),
                ("min_ranks", u32), ("n_ranks_subset", u32), ("ranks", P)]


class TopoOut(C.Structure):
    _fields_ = [("mem_kind", u32), ("n_flagged_racks", u32), ("node_outliers", P),
                ("node_sum", P), ("node_ranks", P), ("node_flag", P), ("chassis_flagged", P),
                ("chassis_nodes", P), ("chassis_sum", P), ("rack_flagged", P),
                ("rack_nodes", P), ("rack_sum", P), ("flagged_racks", P)]


class SpeedupArgs(C.Structure):
    _fields_ = [("mem_kind", u32), ("n_ctxs", u32), ("ctxs", P), ("ranks", P),
                ("n_ranks_subset", u32), ("reserved", u32), ("app_time_ns", u64)]


class SpeedupCtx(C.Structure):
    _fields_ = [("A", u64), ("B", u64), ("G_lo", u64), ("G_hi", u64), ("avg_mean", C.c_double),
                ("avg_max", C.c_double), ("savings_per_iter", C.c_double),
                ("total_reduction", C.c_double), ("share", C.c_double),
                ("cv_across", C.c_double), ("cv_within", C.c_double)]


class SpeedupTotal(C.Structure):
    _fields_ = [("i_star", u32), ("reserved", u32), ("excluded_iterations", u64),
                ("sum_G_lo", u64), ("sum_G_hi", u64), ("t_app", u64),
                ("total_reduction", C.c_double), ("speedup_fraction", C.c_double)]


class ShardStatsParts(C.Structure):
    _fields_ = [("sums", P), ("mins", P), ("maxs", P)]


class ShardMerged(C.Structure):
    _fields_ = [("metric", u32), ("rank_base", u32), ("n_total", u32), ("tau_num", u32),
                ("tau_den", u32), ("sums", P), ("mins", P), ("maxs", P)]


class ShardStatsOut(C.Structure):
    _fields_ = [("stats", P), ("argmax", P), ("outliers", P), ("outlier_cap", u64),
                ("n_outliers", u64)]


class ShardSpeedupParts(C.Structure):
    _fields_ = [("cells", P), ("cell_max", P), ("within", P)]


class Profile(C.Structure):
    _fields_ = [("validate_ms", C.c_double), ("tensor_count_ms", C.c_double),
                ("tensor_ms", C.c_double),
                ("exclusive_ms", C.c_double), ("inclusive_ms", C.c_double),
                ("stats_ms", C.c_double), ("topology_ms", C.c_double), ("speedup_ms", C.c_double),
                ("tensor_launches", u64), ("tensor_records", u64), ("tensor_entries", u64),
                ("tensor_rows", u64), ("interval_ms", C.c_double),
                ("interval_samples", u64), ("interval_entries", u64)]


class BatchSetArgs(C.Structure):
    _fields_ = [("speedup_ctxs", P), ("n_speedup_ctxs", u32), ("topo_ctx", u32),
                ("app_time_ns", u64), ("node_of_rank", P), ("rack_of_node", P),
                ("chassis_of_node", P), ("n_nodes", u32), ("n_chassis", u32), ("n_racks", u32),
                ("topo_tau_num", u32), ("topo_tau_den", u32), ("topo_min_ranks", u32)]


class BatchArgs(C.Structure):
    _fields_ = [("tau_num", u32), ("tau_den", u32), ("outlier_cap", u64), ("set_args", P)]


class BatchInfo(C.Structure):
    _fields_ = [("n_sets", u32), ("n_ranks", u32), ("n_records", u64), ("n_rows", u64),
                ("tensor_nnz", u64), ("excl_nnz", u64), ("incl_nnz", u64), ("n_outliers", u64),
                ("graph_nodes", u64), ("graph_kernels", u64), ("device_bytes", u64),
                ("count_warps", u32), ("count_grid", u32), ("write_warps", u32),
                ("write_grid", u32), ("tune_trials", u32), ("tile_width", u32),
                ("tune_ms", C.c_double)]


class BatchSetView(C.Structure):
    _fields_ = [("n_ranks", u32), ("n_ctx", u32), ("tensor", TensorView),
                ("exclusive", CsrView), ("inclusive", CsrView), ("stats", P), ("outliers", P),
                ("n_outliers", u64), ("speedup", P), ("speedup_total", P), ("n_speedup", u32),
                ("n_flagged_racks", u32), ("n_nodes", u32), ("n_chassis", u32), ("n_racks", u32),
                ("reserved", u32), ("node_outliers", P), ("node_sum", P), ("node_ranks", P),
                ("node_flag", P), ("chassis_flagged", P), ("chassis_nodes", P),
                ("chassis_sum", P), ("rack_flagged", P), ("rack_nodes", P), ("rack_sum", P),
                ("flagged_racks", P)]


class ServeConfig(C.Structure):
    _fields_ = [("max_batch", u32), ("n_streams", u32), ("max_inflight", u32), ("reserved", u32),
                ("result_bytes", u64), ("scratch_bytes", u64), ("staging_bytes", u64),
                ("device_budget", u64)]


class Query(C.Structure):
    _fields_ = [("kind", u32), ("experiment", u32), ("metric", u32), ("ctx", u32),
                ("tau_num", u32), ("tau_den", u32), ("k", u32), ("min_ranks", u32), ("r0", u32),
                ("r1", u32), ("i0", u32), ("i1", u32), ("ranks", P), ("n_ranks", u32),
                ("reserved", u32), ("t0", u64), ("t1", u64)]


class QueryResult(C.Structure):
    _fields_ = [("status", u32), ("kind", u32), ("t_submit_ns", u64), ("t_admit_ns", u64),
                ("t_launch_ns", u64), ("t_done_ns", u64), ("bytes", u64), ("data", P)]


class SpeedupOut(C.Structure):
    _fields_ = [("per_ctx", P), ("total", P)]


class PruneArgs(C.Structure):
    _fields_ = [("mem_kind", u32), ("keep_num", u32), ("keep_den", u32), ("reserved", u32),
                ("drop", P)]


class IntervalArgs(C.Structure):
    _fields_ = [("t0", u64), ("t1", u64), ("r0", u32), ("r1", u32), ("metric", u32),
                ("reserved", u32)]


class ClusterArgs(C.Structure):
    _fields_ = [("method", u32), ("metric", u32), ("ctx", u32), ("mem_kind", u32),
                ("ranks", P), ("n_ranks_subset", u32), ("min_pts", u32), ("eps", u64),
                ("k", u32), ("max_iter", u32), ("node_of_rank", P), ("n_nodes", u32),
                ("reserved", u32)]


class ClusterInfo(C.Structure):
    _fields_ = [("n", u64), ("sum", u64), ("min", u64), ("max", u64), ("mean", C.c_double),
                ("centroid", C.c_double)]


class ClusterOut(C.Structure):
    _fields_ = [("labels", P), ("clusters", P), ("cluster_nodes", P), ("pair_nodes", P),
                ("cluster_cap", u32), ("n_clusters", u32), ("n_noise", u64), ("iterations", u32),
                ("noise_nodes", u32), ("node_view", u32), ("reserved", u32)]


CLUSTER_DBSCAN, CLUSTER_KMEANS = 1, 2


class PruneOut(C.Structure):
    _fields_ = [("kept", P), ("summary", P), ("n_kept", u32), ("reserved", u32),
                ("excl_nnz", u64), ("incl_nnz", u64)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

class QStats(C.Structure):
    _fields_ = [("stats", CtxStats), ("n_outliers", u64)]


class QTopkEntry(C.Structure):
    _fields_ = [("rank", u32), ("reserved", u32), ("x", u64), ("z", C.c_double)]


class QRacks(C.Structure):
    _fields_ = [("n_racks", u32), ("n_flagged_racks", u32)]


Q_STATS, Q_SLICE, Q_TOPK, Q_RACKS, Q_WINDOW = 1, 2, 3, 4, 5

_SIGS = {
    "ta_create": (C.c_int, [C.c_int, P, C.POINTER(P)]),
    "ta_destroy": (C.c_int, [P]),
    "ta_set_allocator": (C.c_int, [P, ALLOC_FN, FREE_FN, P]),
    "ta_sync": (C.c_int, [P]),
    "ta_last_error_message": (C.c_char_p, []),
    "ta_status_string": (C.c_char_p, [C.c_int]),
    "ta_kernel_launches": (u64, [P]),
    "ta_get_profile": (C.c_int, [P, C.POINTER(Profile), C.c_int]),
    "ta_load_traces": (C.c_int, [P, C.POINTER(TraceDesc), C.POINTER(P)]),
    "ta_experiment_free": (C.c_int, [P]),
    "ta_experiment_get_info": (C.c_int, [P, C.POINTER(ExperimentInfo)]),
    "ta_iteration_tensor": (C.c_int, [P, C.POINTER(TensorOut)]),
    "ta_exclusive": (C.c_int, [P, C.POINTER(CsrOut)]),
    "ta_inclusive_rollup": (C.c_int, [P, C.POINTER(CsrOut)]),
    "ta_tensor_get_view": (C.c_int, [P, C.POINTER(TensorView)]),
    "ta_csr_get_view": (C.c_int, [P, u32, C.POINTER(CsrView)]),
    "ta_context_stats": (C.c_int, [P, C.POINTER(StatsArgs), C.POINTER(StatsOut)]),
    "ta_topology_rollup": (C.c_int, [P, C.POINTER(Topology), C.POINTER(TopoArgs),
                                     C.POINTER(TopoOut)]),
    "ta_potential_speedup": (C.c_int, [P, C.POINTER(SpeedupArgs), C.POINTER(SpeedupOut)]),
    "ta_prune_profiles": (C.c_int, [P, C.POINTER(PruneArgs), C.POINTER(PruneOut)]),
    "ta_interval_profile": (C.c_int, [P, C.POINTER(IntervalArgs), C.POINTER(CsrOut)]),
    "ta_call_chains": (C.c_int, [P, u32, P, u32, P, P, u64, C.POINTER(u64)]),
    "ta_cluster_ranks": (C.c_int, [P, C.POINTER(ClusterArgs), C.POINTER(ClusterOut)]),
    "ta_events_table": (C.c_int, [P, u32, u32, P, P, P, P, C.POINTER(u64)]),
    "ta_col_sort": (C.c_int, [P, P, u64, P, P]),
    "ta_col_filter": (C.c_int, [P, P, u64, u64, u64, P, C.POINTER(u64)]),
    "ta_col_group": (C.c_int, [P, P, u32, P, u32, P, u64, P, P, P, P, u64, C.POINTER(u64)]),
    "ta_col_gather": (C.c_int, [P, P, u64, P, u32, P]),
    "ta_col_compare": (C.c_int, [P, P, u64, u64, P]),
    "ta_col_add": (C.c_int, [P, P, P, u64, P]),
    "ta_col_scale": (C.c_int, [P, P, u64, u64]),
    "ta_col_sum": (C.c_int, [P, P, u64, C.POINTER(u64)]),
    "ta_col_cumsum": (C.c_int, [P, P, u64, P]),
    "ta_context_stats_noalloc": (C.c_int, [P, P, P, P, u32, u32, P, u32, u32, u32, P, P, u64,
                                           C.POINTER(u64)]),
    "ta_shard_stats_partials": (C.c_int, [P, u32, C.POINTER(ShardStatsParts)]),
    "ta_shard_stats_finalize": (C.c_int, [P, C.POINTER(ShardMerged), C.POINTER(ShardStatsOut)]),
    "ta_shard_set_argmax": (C.c_int, [P, P, P, u32]),
    "ta_shard_topology_partials": (C.c_int, [P, C.POINTER(ShardMerged), u32, P, u32, P]),
    "ta_topology_finalize": (C.c_int, [P, P, C.POINTER(Topology), u32, C.POINTER(TopoOut)]),
    "ta_shard_speedup_bounds": (C.c_int, [P, C.POINTER(u64)]),
    "ta_shard_speedup_partials": (C.c_int, [P, P, u32, u32, C.POINTER(ShardSpeedupParts)]),
    "ta_speedup_finalize": (C.c_int, [P, u32, u32, u32, u64, u64, C.POINTER(ShardSpeedupParts),
                                      P, P]),
    "ta_batch_plan": (C.c_int, [P, C.POINTER(TraceDesc), u32, C.POINTER(BatchArgs),
                                C.POINTER(P)]),
    "ta_batch_run": (C.c_int, [P]),
    "ta_batch_free": (C.c_int, [P]),
    "ta_batch_get_info": (C.c_int, [P, C.POINTER(BatchInfo)]),
    "ta_batch_get_set": (C.c_int, [P, u32, C.POINTER(BatchSetView)]),
    "ta_serve_open": (C.c_int, [P, C.POINTER(ServeConfig), C.POINTER(P)]),
    "ta_serve_close": (C.c_int, [P]),
    "ta_serve_add_experiment": (C.c_int, [P, P, C.POINTER(Topology), C.POINTER(u32)]),
    "ta_serve_submit": (C.c_int, [P, C.POINTER(Query), C.POINTER(u64)]),
    "ta_serve_poll": (C.c_int, [P, u64, C.c_int64, C.POINTER(QueryResult)]),
    "ta_serve_release": (C.c_int, [P, u64]),
    "ta_serve_replay": (C.c_int, [P, P, P, u64, P, C.POINTER(u64)]),
}

_lib = None


def declared_symbols():
    """Names of the functions include/ta.h declares."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:ta_status|const char\*|uint64_t)\s+(ta_\w+)\s*\(",
                                 text, re.M)))


def lib():
    """Load libta.so (building it first if needed); raises if unavailable."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            from . import build as _b
            _b.build()
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class _CudaArray:
    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = dict(shape=(n,), typestr=typestr, data=(ptr, False),
                                             version=3, strides=None)


def device_array(ptr, n, dtype, device=0):
    """Zero-copy torch view of n elements of library-owned device memory
    (64-bit unsigned values are viewed as int64; reinterpret on the host)."""
    torch = _torch()
    typestr = {np.uint64: "<i8", np.uint32: "<i4", np.float64: "<f8", np.uint8: "|u1"}[dtype]
    return torch.as_tensor(_CudaArray(int(ptr), int(n), typestr), device=f"cuda:{device}")


class TaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(s):
    if s != OK:
        raise TaError(s, lib().ta_last_error_message().decode())


def _ptr(a):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _is_dev(a):
    return a is not None and not isinstance(a, np.ndarray) and a.is_cuda


def _torch():
    import torch
    return torch


class Context:
    """A library context bound to a CUDA device and a torch stream."""

    def __init__(self, device: int = 0, stream=None, use_torch_allocator: bool = True):
        torch = _torch()
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = P()
        _check(lib().ta_create(device, self.stream.cuda_stream, C.byref(h)))
        self.h = h
        self._cb = None
        if use_torch_allocator:
            dev = device

            def _alloc(n, stream, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(n), dev, stream)
                except Exception:
                    return None

            def _free(p, n, stream, user):
                torch.cuda.caching_allocator_delete(p)

            self._cb = (ALLOC_FN(_alloc), FREE_FN(_free))
            _check(lib().ta_set_allocator(self.h, self._cb[0], self._cb[1], None))

    def launches(self) -> int:
        return int(lib().ta_kernel_launches(self.h))

    def sync(self):
        _check(lib().ta_sync(self.h))

    def profile(self, reset: bool = False) -> dict:
        p = Profile()
        _check(lib().ta_get_profile(self.h, C.byref(p), 1 if reset else 0))
        return {f: getattr(p, f) for f, _ in Profile._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().ta_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, rank_off, ts, ctx, parent, marker: int, borrow: bool = False,
             inclusive: bool = True, nnz_hint: int = 0, rows_hint: int = 0,
             keep_traces: bool = False) -> "Experiment":
        return Experiment(self, rank_off, ts, ctx, parent, marker, borrow, inclusive, nnz_hint,
                          rows_hint, keep_traces)


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _as_py_ints(a):
    """A struct field column with the dtype np.array would give the same
    values as Python numbers: integers as int64, or uint64 when one exceeds
    int64's range; floats unchanged."""
    if a.dtype.kind not in "ui":
        return a.copy()
    if a.dtype == np.uint64 and a.size and int(a.max()) > np.iinfo(np.int64).max:
        return a.copy()
    return a.astype(np.int64)


class Columns:
    """The column operations of include/ta.h (ta_events_table, ta_col_*) on
    torch device tensors of this context's device."""

    def __init__(self, ctx: "Context"):
        self.ctx = ctx

    def _t(self, n, dtype):
        torch = _torch()
        return torch.empty(max(int(n), 1), dtype=dtype, device=f"cuda:{self.ctx.device}")[:int(n)]

    def events(self, e: "Experiment", r0=0, r1=None):
        """dict(rank, ts, ctx, dur) of the events of ranks [r0, r1)."""
        torch = _torch()
        r1 = e.R if r1 is None else r1
        n = u64()
        _check(lib().ta_events_table(e.h, r0, r1, None, None, None, None, C.byref(n)))
        out = dict(rank=self._t(n.value, torch.uint32), ts=self._t(n.value, torch.uint64),
                   ctx=self._t(n.value, torch.uint32), dur=self._t(n.value, torch.uint64))
        _check(lib().ta_events_table(e.h, r0, r1, out["rank"].data_ptr(), out["ts"].data_ptr(),
                                     out["ctx"].data_ptr(), out["dur"].data_ptr(), C.byref(n)))
        return out

    def sort(self, keys):
        torch = _torch()
        n = keys.numel()
        ko, perm = self._t(n, torch.uint64), self._t(n, torch.uint32)
        _check(lib().ta_col_sort(self.ctx.h, keys.data_ptr(), n, ko.data_ptr(), perm.data_ptr()))
        return ko, perm

    def filter(self, col, lo, hi):
        torch = _torch()
        n = col.numel()
        idx = self._t(n, torch.uint32)
        m = u64()
        _check(lib().ta_col_filter(self.ctx.h, col.data_ptr(), n, int(lo), int(hi),
                                   idx.data_ptr(), C.byref(m)))
        return idx[:m.value]

    def group(self, seg_off, key, n_keys, val):
        torch = _torch()
        n_seg = seg_off.numel() - 1
        off = self._t(n_seg + 1, torch.uint64)
        m = u64()
        args = (self.ctx.h, seg_off.data_ptr(), n_seg, key.data_ptr(), int(n_keys), val.data_ptr(),
                key.numel(), off.data_ptr())
        _check(lib().ta_col_group(*args, None, None, None, 0, C.byref(m)))
        k, sm, cn = (self._t(m.value, torch.uint32), self._t(m.value, torch.uint64),
                     self._t(m.value, torch.uint32))
        _check(lib().ta_col_group(*args, k.data_ptr(), sm.data_ptr(), cn.data_ptr(), m.value,
                                  C.byref(m)))
        return dict(off=off, key=k, sum=sm, cnt=cn)

    def gather(self, key, dim):
        torch = _torch()
        out = self._t(key.numel(), torch.uint32)
        _check(lib().ta_col_gather(self.ctx.h, key.data_ptr(), key.numel(), dim.data_ptr(),
                                   dim.numel(), out.data_ptr()))
        return out

    def compare(self, col, c):
        torch = _torch()
        m = self._t(col.numel(), torch.uint8)
        _check(lib().ta_col_compare(self.ctx.h, col.data_ptr(), col.numel(), int(c), m.data_ptr()))
        return m

    def add(self, a, b):
        torch = _torch()
        out = self._t(a.numel(), torch.uint64)
        _check(lib().ta_col_add(self.ctx.h, a.data_ptr(), b.data_ptr(), a.numel(), out.data_ptr()))
        return out

    def scale(self, a, s):
        _check(lib().ta_col_scale(self.ctx.h, a.data_ptr(), a.numel(), int(s)))
        return a

    def sum(self, a):
        v = u64()
        _check(lib().ta_col_sum(self.ctx.h, a.data_ptr(), a.numel(), C.byref(v)))
        return int(v.value)

    def cumsum(self, a):
        torch = _torch()
        out = self._t(a.numel(), torch.uint64)
        _check(lib().ta_col_cumsum(self.ctx.h, a.data_ptr(), a.numel(), out.data_ptr()))
        return out


class Experiment:
    """Resident analysis products of one trace set (see ta_load_traces)."""

    def __init__(self, ctx: Context, rank_off, ts, cx, parent, marker, borrow=False,
                 inclusive=True, nnz_hint=0, rows_hint=0, keep_traces=False):
        self.ctx = ctx
        dev = _is_dev(ts) or _is_dev(rank_off)
        if dev:
            torch = _torch()
            rank_off = rank_off.contiguous()
            ts, cx, parent = ts.contiguous(), cx.contiguous(), parent.contiguous()
            assert rank_off.dtype == torch.uint64 and ts.dtype == torch.uint64
            assert cx.dtype == torch.uint32 and parent.dtype == torch.uint32
        else:
            rank_off, ts, cx = _np(rank_off, np.uint64), _np(ts, np.uint64), _np(cx, np.uint32)
            parent = _np(parent, np.uint32)
        self._keep = (rank_off, ts, cx, parent) if borrow else None
        d = TraceDesc()
        d.n_ranks = rank_off.shape[0] - 1
        d.n_ctx = parent.shape[0]
        d.marker_ctx = int(marker)
        d.mem_kind = MEM_DEVICE if dev else MEM_HOST
        d.n_records = ts.shape[0]
        d.rank_off, d.ts, d.ctx, d.parent = _ptr(rank_off), _ptr(ts), _ptr(cx), _ptr(parent)
        d.flags = ((LOAD_BORROW if borrow else 0) | (0 if inclusive else LOAD_NO_INCLUSIVE)
                   | (LOAD_KEEP_TRACES if keep_traces else 0))
        d.nnz_hint, d.rows_hint = nnz_hint, rows_hint
        h = P()
        _check(lib().ta_load_traces(ctx.h, C.byref(d), C.byref(h)))
        self.h = h
        self.R = int(d.n_ranks)
        self.C = int(d.n_ctx)
        self.has_incl = inclusive

    def free(self):
        if getattr(self, "h", None):
            lib().ta_experiment_free(self.h)
            self.h = None
            self._keep = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self) -> dict:
        i = ExperimentInfo()
        _check(lib().ta_experiment_get_info(self.h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in ExperimentInfo._fields_}

    # ---- products copied to host (numpy) or device (torch) -----------------
    def _alloc(self, n, dtype, device):
        if device:
            torch = _torch()
            tdt = {np.uint32: torch.uint32, np.uint64: torch.uint64, np.float64: torch.float64,
                   np.uint8: torch.uint8}[dtype]
            return torch.empty(max(n, 1), dtype=tdt, device=f"cuda:{self.ctx.device}")[:n]
        return np.empty(n, dtype)

    def tensor(self, device: bool = False) -> dict:
        o = TensorOut()
        _check(lib().ta_iteration_tensor(self.h, C.byref(o)))
        rows, nnz = int(o.rows), int(o.nnz)
        out = dict(n_iter=self._alloc(self.R, np.uint32, device),
                   row_off_of_rank=self._alloc(self.R + 1, np.uint64, device),
                   entry_off=self._alloc(rows + 1, np.uint64, device),
                   e_ctx=self._alloc(nnz, np.uint32, device),
                   e_time=self._alloc(nnz, np.uint64, device),
                   e_cnt=self._alloc(nnz, np.uint32, device))
        o = TensorOut()
        o.mem_kind = MEM_DEVICE if device else MEM_HOST
        for k, v in out.items():
            setattr(o, k, _ptr(v))
        o.rows_cap, o.nnz_cap = rows + 1, nnz
        _check(lib().ta_iteration_tensor(self.h, C.byref(o)))
        return out

    def csr(self, metric=EXCLUSIVE, device: bool = False) -> dict:
        fn = lib().ta_exclusive if metric == EXCLUSIVE else lib().ta_inclusive_rollup
        o = CsrOut()
        _check(fn(self.h, C.byref(o)))
        nnz = int(o.nnz)
        out = dict(off=self._alloc(self.R + 1, np.uint64, device),
                   ctx=self._alloc(nnz, np.uint32, device),
                   time=self._alloc(nnz, np.uint64, device), cnt=self._alloc(nnz, np.uint32, device))
        o = CsrOut()
        o.mem_kind = MEM_DEVICE if device else MEM_HOST
        o.off, o.ctx, o.time, o.cnt = (_ptr(out[k]) for k in ("off", "ctx", "time", "cnt"))
        o.nnz_cap = nnz
        _check(fn(self.h, C.byref(o)))
        return out

    def tensor_view(self) -> TensorView:
        v = TensorView()
        _check(lib().ta_tensor_get_view(self.h, C.byref(v)))
        return v

    def span(self) -> np.ndarray:
        """Per-rank span (ts_last - ts_first), read through the tensor view."""
        v = self.tensor_view()
        return device_array(v.span, self.R, np.uint64, self.ctx.device).cpu().numpy().view(np.uint64)

    def stats(self, metric=EXCLUSIVE, ranks=None, ctxs=None, tau=(3, 1), outlier_cap=1 << 20,
              want_z=False, device=False):
        torch = _torch() if device else None
        k = self.C if ctxs is None else len(ctxs)
        a = StatsArgs()
        a.metric, a.mem_kind = metric, MEM_DEVICE if device else MEM_HOST
        if device:
            rk = None if ranks is None else torch.as_tensor(np.asarray(ranks, np.uint32)).cuda()
            cx = None if ctxs is None else torch.as_tensor(np.asarray(ctxs, np.uint32)).cuda()
        else:
            rk = None if ranks is None else _np(ranks, np.uint32)
            cx = None if ctxs is None else _np(ctxs, np.uint32)
        a.ranks, a.n_ranks_subset = _ptr(rk), 0 if ranks is None else len(ranks)
        a.ctxs, a.n_ctxs = _ptr(cx), 0 if ctxs is None else len(ctxs)
        a.tau_num, a.tau_den = tau
        st = np.zeros(max(k, 1), np.dtype(CtxStats))
        outl = np.empty(max(outlier_cap, 1), np.dtype(Outlier))
        nnz = 0
        if want_z:
            v = CsrView()
            _check(lib().ta_csr_get_view(self.h, metric, C.byref(v)))
            nnz = int(v.nnz)
        z = np.zeros(max(nnz, 1), np.float64) if want_z else None
        o = StatsOut()
        if device:
            dst = torch.empty(max(k, 1) * C.sizeof(CtxStats), dtype=torch.uint8, device="cuda")
            dout = torch.empty(max(outlier_cap, 1) * C.sizeof(Outlier), dtype=torch.uint8,
                               device="cuda")
            dz = torch.zeros(max(nnz, 1), dtype=torch.float64, device="cuda") if want_z else None
            o.stats, o.outliers, o.z = dst.data_ptr(), dout.data_ptr(), _ptr(dz)
        else:
            o.stats, o.outliers, o.z = st.ctypes.data, outl.ctypes.data, _ptr(z)
        o.outlier_cap = outlier_cap
        s = lib().ta_context_stats(self.h, C.byref(a), C.byref(o))
        n_out = int(o.n_outliers)
        if s not in (OK, CAPACITY):
            _check(s)
        m = min(n_out, outlier_cap) if s == OK else 0
        if device:
            C.memmove(st.ctypes.data, dst.cpu().numpy().ctypes.data, max(k, 1) * C.sizeof(CtxStats))
            if m:
                C.memmove(outl.ctypes.data, dout[: m * C.sizeof(Outlier)].cpu().numpy().ctypes.data,
                          m * C.sizeof(Outlier))
            if want_z:
                z = dz.cpu().numpy()
        stats = {f: _as_py_ints(st[f][:k]) for f, _ in CtxStats._fields_ if f != "reserved"}
        outliers = dict(ctx=outl["ctx"][:m].copy(), rank=outl["rank"][:m].copy(),
                        z=outl["z"][:m].copy())
        if s == CAPACITY:
            raise TaError(s, f"{n_out} outliers exceed capacity {outlier_cap}")
        return stats, outliers, n_out, (z[:nnz] if want_z else None)

    def topology(self, ctx, node_of_rank, rack_of_node, chassis_of_node, n_racks, n_chassis,
                 metric=EXCLUSIVE, tau=(3, 1), min_ranks=1, ranks=None):
        nn = len(rack_of_node)
        t = Topology()
        t.n_nodes, t.n_chassis, t.n_racks, t.mem_kind = nn, n_chassis, n_racks, MEM_HOST
        arrs = [_np(node_of_rank, np.uint32), _np(rack_of_node, np.uint32),
                _np(chassis_of_node, np.uint32)]
        t.node_of_rank, t.rack_of_node, t.chassis_of_node = (_ptr(x) for x in arrs)
        a = TopoArgs()
        a.metric, a.ctx, a.tau_num, a.tau_den, a.min_ranks = metric, ctx, tau[0], tau[1], min_ranks
        rk = None if ranks is None else _np(ranks, np.uint32)
        a.ranks, a.n_ranks_subset = _ptr(rk), 0 if ranks is None else len(ranks)
        out = dict(node_outliers=np.zeros(nn, np.uint32), node_sum=np.zeros(nn, np.uint64),
                   node_ranks=np.zeros(nn, np.uint32), node_flag=np.zeros(nn, np.uint8),
                   chassis_flagged=np.zeros(n_chassis, np.uint32),
                   chassis_nodes=np.zeros(n_chassis, np.uint32),
                   chassis_sum=np.zeros(n_chassis, np.uint64),
                   rack_flagged=np.zeros(n_racks, np.uint32), rack_nodes=np.zeros(n_racks, np.uint32),
                   rack_sum=np.zeros(n_racks, np.uint64), flagged_racks=np.zeros(n_racks, np.uint32))
        o = TopoOut()
        o.mem_kind = MEM_HOST
        for k, v in out.items():
            setattr(o, k, _ptr(v))
        _check(lib().ta_topology_rollup(self.h, C.byref(t), C.byref(a), C.byref(o)))
        out["flagged_racks"] = out["flagged_racks"][: int(o.n_flagged_racks)]
        return out

    def speedup(self, ctxs, ranks=None, app_time_ns=0):
        cx = _np(ctxs, np.uint32)
        rk = None if ranks is None else _np(ranks, np.uint32)
        a = SpeedupArgs()
        a.mem_kind, a.n_ctxs, a.ctxs = MEM_HOST, len(cx), _ptr(cx)
        a.ranks, a.n_ranks_subset = _ptr(rk), 0 if ranks is None else len(ranks)
        a.app_time_ns = app_time_ns
        per = (SpeedupCtx * len(cx))()
        tot = SpeedupTotal()
        o = SpeedupOut()
        o.per_ctx, o.total = C.addressof(per), C.addressof(tot)
        _check(lib().ta_potential_speedup(self.h, C.byref(a), C.byref(o)))
        d = {f: np.array([getattr(x, f) for x in per]) for f, _ in SpeedupCtx._fields_}
        d["G"] = [int(lo) + (int(hi) << 64) for lo, hi in zip(d["G_lo"], d["G_hi"])]
        t = {f: getattr(tot, f) for f, _ in SpeedupTotal._fields_ if f != "reserved"}
        t["sum_G"] = t["sum_G_lo"] + (t["sum_G_hi"] << 64)
        return d, t

    def interval(self, t0, t1, r0=0, r1=None, metric=EXCLUSIVE, device=False):
        """ta_interval_profile: per-rank profiles of the time window [t0, t1)
        for ranks [r0, r1) (the experiment must keep its traces).  Returns a
        CSR dict like csr(), over r1 - r0 ranks."""
        a = IntervalArgs()
        a.t0, a.t1 = int(t0), int(t1)
        a.r0, a.r1 = int(r0), self.R if r1 is None else int(r1)
        a.metric = metric
        o = CsrOut()
        o.mem_kind = MEM_DEVICE if device else MEM_HOST
        _check(lib().ta_interval_profile(self.h, C.byref(a), C.byref(o)))
        nnz = int(o.nnz)
        n = a.r1 - a.r0
        out = dict(off=self._alloc(n + 1, np.uint64, device), ctx=self._alloc(nnz, np.uint32, device),
                   time=self._alloc(nnz, np.uint64, device), cnt=self._alloc(nnz, np.uint32, device))
        o.off, o.ctx, o.time, o.cnt = (_ptr(out[k]) for k in ("off", "ctx", "time", "cnt"))
        o.nnz_cap = nnz
        _check(lib().ta_interval_profile(self.h, C.byref(a), C.byref(o)))
        return out

    def call_chains(self, ctxs):
        """ta_call_chains: the bottom-up calling context of each context id.
        Returns a list of uint32 arrays (context, parent, ..., root)."""
        cx = _np(ctxs, np.uint32)
        n = len(cx)
        off = np.zeros(n + 1, np.uint64)
        total = u64()
        _check(lib().ta_call_chains(self.h, MEM_HOST, _ptr(cx), n, _ptr(off), None, 0,
                                    C.byref(total)))
        chain = np.zeros(max(int(total.value), 1), np.uint32)
        _check(lib().ta_call_chains(self.h, MEM_HOST, _ptr(cx), n, _ptr(off), _ptr(chain),
                                    int(total.value), C.byref(total)))
        return [chain[int(off[i]):int(off[i + 1])] for i in range(n)]

    def cluster(self, ctx, method="dbscan", eps=0, min_pts=1, k=2, max_iter=0, metric=EXCLUSIVE,
                ranks=None, node_of_rank=None, n_nodes=0):
        """ta_cluster_ranks: DBSCAN (eps ns, min_pts) or K-Means (k, max_iter)
        over the ranks' values of ctx.  Returns dict(labels int32[n], clusters
        (dict of arrays n, sum, min, max, mean, centroid, in ascending value),
        n_clusters, n_noise, iterations, and with node_of_rank: cluster_nodes,
        pair_nodes [nc, nc] (entry i, j for i < j), noise_nodes)."""
        a = ClusterArgs()
        a.method = CLUSTER_DBSCAN if method == "dbscan" else CLUSTER_KMEANS
        a.metric, a.ctx, a.mem_kind = metric, int(ctx), MEM_HOST
        rk = None if ranks is None else _np(ranks, np.uint32)
        a.ranks, a.n_ranks_subset = _ptr(rk), 0 if rk is None else len(rk)
        a.min_pts, a.eps, a.k, a.max_iter = int(min_pts), int(eps), int(k), int(max_iter)
        nd = None if node_of_rank is None else _np(node_of_rank, np.uint32)
        a.node_of_rank, a.n_nodes = _ptr(nd), int(n_nodes)
        n = self.R if rk is None else len(rk)
        labels = np.zeros(max(n, 1), np.int32)
        o = ClusterOut()
        o.labels = _ptr(labels)
        _check(lib().ta_cluster_ranks(self.h, C.byref(a), C.byref(o)))
        nc = int(o.n_clusters)
        cl = (ClusterInfo * max(nc, 1))()
        per = np.zeros(max(nc, 1), np.uint32)
        pair = np.zeros((max(nc, 1), max(nc, 1)), np.uint32)
        o = ClusterOut()
        o.labels, o.clusters, o.cluster_cap = _ptr(labels), C.addressof(cl), nc
        if nd is not None:
            o.cluster_nodes, o.pair_nodes = _ptr(per), _ptr(pair)
        _check(lib().ta_cluster_ranks(self.h, C.byref(a), C.byref(o)))
        out = dict(labels=labels[:n], n_clusters=nc, n_noise=int(o.n_noise),
                   iterations=int(o.iterations),
                   clusters={f: np.array([getattr(x, f) for x in cl[:nc]])
                             for f, _ in ClusterInfo._fields_})
        if o.node_view:
            out.update(cluster_nodes=per[:nc], pair_nodes=pair[:nc, :nc],
                       noise_nodes=int(o.noise_nodes))
        return out

    def prune(self, keep=(1, 100), drop=None):
        """ta_prune_profiles: keep the contexts whose summary inclusive time is
        at least keep[0]/keep[1] of the total and not flagged in drop; this
        experiment's exclusive and inclusive CSRs are compacted in place.
        Returns dict(kept u8[C], summary u64[C], n_kept, excl_nnz, incl_nnz)."""
        a = PruneArgs()
        a.mem_kind, a.keep_num, a.keep_den = MEM_HOST, int(keep[0]), int(keep[1])
        dr = None if drop is None else _np(drop, np.uint8)
        a.drop = _ptr(dr)
        kept = np.zeros(self.C, np.uint8)
        summary = np.zeros(self.C, np.uint64)
        o = PruneOut()
        o.kept, o.summary = _ptr(kept), _ptr(summary)
        _check(lib().ta_prune_profiles(self.h, C.byref(a), C.byref(o)))
        return dict(kept=kept, summary=summary, n_kept=int(o.n_kept), excl_nnz=int(o.excl_nnz),
                    incl_nnz=int(o.incl_nnz))


def _dev_to_np(ptr, n, dtype, device):
    """Host copy of n elements of library-owned device memory."""
    if n == 0 or not ptr:
        return np.zeros(0, dtype)
    return device_array(ptr, n, dtype, device).cpu().numpy().view(dtype)


def _dev_structs(ptr, n, ctype, device):
    """Host ctypes array copied from n device structs."""
    arr = (ctype * max(n, 1))()
    if n and ptr:
        raw = _dev_to_np(ptr, n * C.sizeof(ctype), np.uint8, device)
        C.memmove(arr, raw.ctypes.data, n * C.sizeof(ctype))
    return arr


class Batch:
    """Many independent trace sets analysed as one unit (ta_batch_plan): the
    whole analysis is one captured CUDA graph, replayed by run()."""

    def __init__(self, ctx: Context, sets, tau=(3, 1), outlier_cap=1 << 20, set_args=None):
        """sets: sequence of (rank_off, ts, ctx, parent, marker), either all
        numpy arrays (host) or all torch CUDA tensors (device).  set_args:
        optional per-set dicts (or None) with keys speedup_ctxs, app_time_ns,
        and topology (node_of_rank, rack_of_node, chassis_of_node, n_racks,
        n_chassis) with topo_ctx, topo_tau, min_ranks."""
        self.ctx = ctx
        keep, descs = [], (TraceDesc * len(sets))()
        for d, (rank_off, ts, cx, parent, marker) in zip(descs, sets):
            dev = _is_dev(ts) or _is_dev(rank_off)
            if dev:
                torch = _torch()
                rank_off, ts = rank_off.contiguous(), ts.contiguous()
                cx, parent = cx.contiguous(), parent.contiguous()
                assert rank_off.dtype == torch.uint64 and ts.dtype == torch.uint64
                assert cx.dtype == torch.uint32 and parent.dtype == torch.uint32
            else:
                rank_off, ts = _np(rank_off, np.uint64), _np(ts, np.uint64)
                cx, parent = _np(cx, np.uint32), _np(parent, np.uint32)
            keep.append((rank_off, ts, cx, parent))
            d.n_ranks = rank_off.shape[0] - 1
            d.n_ctx = parent.shape[0]
            d.marker_ctx = int(marker)
            d.mem_kind = MEM_DEVICE if dev else MEM_HOST
            d.n_records = ts.shape[0]
            d.rank_off, d.ts, d.ctx, d.parent = _ptr(rank_off), _ptr(ts), _ptr(cx), _ptr(parent)
        a = BatchArgs()
        a.tau_num, a.tau_den = tau
        a.outlier_cap = outlier_cap
        sargs = None
        if set_args is not None:
            sargs = (BatchSetArgs * len(sets))()
            for x, sa in zip(sargs, set_args):
                if not sa:
                    continue
                if sa.get("speedup_ctxs") is not None:
                    kc = _np(sa["speedup_ctxs"], np.uint32)
                    keep.append(kc)
                    x.speedup_ctxs, x.n_speedup_ctxs = kc.ctypes.data, len(kc)
                x.app_time_ns = int(sa.get("app_time_ns", 0))
                topo = sa.get("topology")
                if topo is not None:
                    arrs = [_np(topo[k], np.uint32)
                            for k in ("node_of_rank", "rack_of_node", "chassis_of_node")]
                    keep.extend(arrs)
                    x.node_of_rank, x.rack_of_node, x.chassis_of_node = (
                        z.ctypes.data for z in arrs)
                    x.n_nodes, x.n_racks = len(arrs[1]), int(topo["n_racks"])
                    x.n_chassis = int(topo["n_chassis"])
                    x.topo_ctx = int(sa.get("topo_ctx", 0))
                    x.topo_tau_num, x.topo_tau_den = sa.get("topo_tau", (3, 1))
                    x.topo_min_ranks = int(sa.get("min_ranks", 1))
            a.set_args = C.cast(sargs, P)
        h = P()
        _check(lib().ta_batch_plan(ctx.h, descs, len(sets), C.byref(a), C.byref(h)))
        self.h = h
        self.S = len(sets)

    def run(self):
        _check(lib().ta_batch_run(self.h))

    def free(self):
        if getattr(self, "h", None):
            lib().ta_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self) -> dict:
        i = BatchInfo()
        _check(lib().ta_batch_get_info(self.h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in BatchInfo._fields_}

    def view(self, s: int) -> BatchSetView:
        v = BatchSetView()
        _check(lib().ta_batch_get_set(self.h, s, C.byref(v)))
        return v

    def products(self, s: int) -> dict:
        """Host copies of every product of set s (offsets relative to the set)."""
        v = self.view(s)
        dev = self.ctx.device
        R, Cn = int(v.n_ranks), int(v.n_ctx)
        t = v.tensor
        rows, nnz = int(t.rows), int(t.nnz)
        out = dict(R=R, C=Cn)
        out["tensor"] = dict(n_iter=_dev_to_np(t.n_iter, R, np.uint32, dev),
                             row_off_of_rank=_dev_to_np(t.row_off_of_rank, R + 1, np.uint64, dev),
                             entry_off=_dev_to_np(t.entry_off, rows + 1, np.uint64, dev),
                             e_ctx=_dev_to_np(t.e_ctx, nnz, np.uint32, dev),
                             e_time=_dev_to_np(t.e_time, nnz, np.uint64, dev),
                             e_cnt=_dev_to_np(t.e_cnt, nnz, np.uint32, dev),
                             span=_dev_to_np(t.span, R, np.uint64, dev))
        for name in ("exclusive", "inclusive"):
            c = getattr(v, name)
            n = int(c.nnz)
            out[name] = dict(off=_dev_to_np(c.off, R + 1, np.uint64, dev),
                             ctx=_dev_to_np(c.ctx, n, np.uint32, dev),
                             time=_dev_to_np(c.time, n, np.uint64, dev),
                             cnt=_dev_to_np(c.cnt, n, np.uint32, dev))
        st = _dev_structs(v.stats, Cn, CtxStats, dev)
        out["stats"] = {f: np.array([getattr(x, f) for x in st[:Cn]]) for f, _ in CtxStats._fields_
                        if f != "reserved"}
        m = int(v.n_outliers)
        ol = _dev_structs(v.outliers, m, Outlier, dev)
        out["outliers"] = dict(ctx=np.array([x.ctx for x in ol[:m]], np.uint32),
                               rank=np.array([x.rank for x in ol[:m]], np.uint32),
                               z=np.array([x.z for x in ol[:m]], np.float64))
        if v.n_speedup:
            ns = int(v.n_speedup)
            sp = _dev_structs(v.speedup, ns, SpeedupCtx, dev)
            d = {f: np.array([getattr(x, f) for x in sp[:ns]]) for f, _ in SpeedupCtx._fields_}
            d["G"] = [int(lo) + (int(hi) << 64) for lo, hi in zip(d["G_lo"], d["G_hi"])]
            tt = _dev_structs(v.speedup_total, 1, SpeedupTotal, dev)[0]
            t = {f: getattr(tt, f) for f, _ in SpeedupTotal._fields_ if f != "reserved"}
            t["sum_G"] = t["sum_G_lo"] + (t["sum_G_hi"] << 64)
            out["speedup"] = (d, t)
        if v.n_nodes:
            nn, nc, nr = int(v.n_nodes), int(v.n_chassis), int(v.n_racks)
            out["topology"] = dict(
                node_outliers=_dev_to_np(v.node_outliers, nn, np.uint32, dev),
                node_sum=_dev_to_np(v.node_sum, nn, np.uint64, dev),
                node_ranks=_dev_to_np(v.node_ranks, nn, np.uint32, dev),
                node_flag=_dev_to_np(v.node_flag, nn, np.uint8, dev),
                chassis_flagged=_dev_to_np(v.chassis_flagged, nc, np.uint32, dev),
                chassis_nodes=_dev_to_np(v.chassis_nodes, nc, np.uint32, dev),
                chassis_sum=_dev_to_np(v.chassis_sum, nc, np.uint64, dev),
                rack_flagged=_dev_to_np(v.rack_flagged, nr, np.uint32, dev),
                rack_nodes=_dev_to_np(v.rack_nodes, nr, np.uint32, dev),
                rack_sum=_dev_to_np(v.rack_sum, nr, np.uint64, dev),
                flagged_racks=_dev_to_np(v.flagged_racks, int(v.n_flagged_racks), np.uint32, dev))
        return out


def make_query(kind, experiment=0, ctx=0, metric=EXCLUSIVE, ranks=None, tau=(3, 1), k=10,
               min_ranks=1, r0=0, r1=0, i0=0, i1=0, t0=0, t1=0):
    """A ta_query; keeps the rank subset alive on the returned object."""
    q = Query()
    q.kind, q.experiment, q.metric, q.ctx = kind, experiment, metric, ctx
    q.tau_num, q.tau_den, q.k, q.min_ranks = tau[0], tau[1], k, min_ranks
    q.r0, q.r1, q.i0, q.i1 = r0, r1, i0, i1
    q.t0, q.t1 = int(t0), int(t1)
    if ranks is not None:
        arr = _np(ranks, np.uint32)
        q._ranks = arr
        q.ranks, q.n_ranks = arr.ctypes.data, len(arr)
    return q


def parse_payload(kind, data, nbytes):
    """Decode a query payload (bytes) into numpy / dict form."""
    if kind == Q_STATS:
        r = QStats.from_buffer_copy(data[: C.sizeof(QStats)])
        d = {f: getattr(r.stats, f) for f, _ in CtxStats._fields_ if f != "reserved"}
        d["n_outliers"] = r.n_outliers
        return d
    if kind == Q_SLICE:
        return np.frombuffer(data, np.uint64).copy()
    if kind == Q_WINDOW:
        v = np.frombuffer(data[:nbytes], np.uint64).copy()
        return dict(time=v[: len(v) // 2], cnt=v[len(v) // 2:])
    if kind == Q_TOPK:
        n = int(np.frombuffer(data[:8], np.uint64)[0])
        ent = (QTopkEntry * max(n, 1)).from_buffer_copy(data[8: 8 + max(n, 1) * C.sizeof(QTopkEntry)]
                                                       if n else bytes(C.sizeof(QTopkEntry)))
        return dict(rank=np.array([e.rank for e in ent[:n]], np.uint32),
                    x=np.array([e.x for e in ent[:n]], np.uint64),
                    z=np.array([e.z for e in ent[:n]], np.float64))
    h = QRacks.from_buffer_copy(data[:8])
    nr, nf = h.n_racks, h.n_flagged_racks
    o = 8
    rack_sum = np.frombuffer(data[o: o + 8 * nr], np.uint64).copy()
    o += 8 * nr
    rack_flagged = np.frombuffer(data[o: o + 4 * nr], np.uint32).copy()
    o += 4 * nr
    rack_nodes = np.frombuffer(data[o: o + 4 * nr], np.uint32).copy()
    o += 4 * nr
    flagged = np.frombuffer(data[o: o + 4 * nf], np.uint32).copy()
    return dict(rack_sum=rack_sum, rack_flagged=rack_flagged, rack_nodes=rack_nodes,
                flagged_racks=flagged)


class Server:
    """Query server over resident experiments (ta_serve_*)."""

    def __init__(self, ctx: Context, max_batch=0, n_streams=0, max_inflight=0, result_bytes=0,
                 scratch_bytes=0, staging_bytes=0, device_budget=0):
        self.ctx = ctx
        c = ServeConfig()
        c.max_batch, c.n_streams, c.max_inflight = max_batch, n_streams, max_inflight
        c.result_bytes, c.scratch_bytes, c.staging_bytes = result_bytes, scratch_bytes, staging_bytes
        c.device_budget = device_budget
        h = P()
        _check(lib().ta_serve_open(ctx.h, C.byref(c), C.byref(h)))
        self.h = h
        self._exps = []

    def close(self):
        if getattr(self, "h", None):
            lib().ta_serve_close(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, e: "Experiment", topo=None) -> int:
        t = None
        if topo is not None:
            t = Topology()
            keep = [_np(topo["node_of_rank"], np.uint32), _np(topo["rack_of_node"], np.uint32),
                    _np(topo["chassis_of_node"], np.uint32)]
            t.n_nodes, t.n_chassis, t.n_racks = len(keep[1]), int(topo["n_chassis"]), int(topo["n_racks"])
            t.mem_kind = MEM_HOST
            t.node_of_rank, t.rack_of_node, t.chassis_of_node = (a.ctypes.data for a in keep)
        i = u32(0)
        _check(lib().ta_serve_add_experiment(self.h, e.h, C.byref(t) if t is not None else None,
                                             C.byref(i)))
        self._exps.append(e)
        return int(i.value)

    def submit(self, q: Query) -> int:
        t = u64(0)
        _check(lib().ta_serve_submit(self.h, C.byref(q), C.byref(t)))
        return int(t.value)

    def poll(self, ticket: int, wait_ns: int = -1):
        """(payload, timings) when done, None while pending."""
        r = QueryResult()
        s = lib().ta_serve_poll(self.h, ticket, wait_ns, C.byref(r))
        if s == STATE:
            return None
        _check(s)
        if r.status != OK:
            raise TaError(r.status, "query failed on the device")
        data = C.string_at(r.data, r.bytes)
        times = dict(submit=r.t_submit_ns, admit=r.t_admit_ns, launch=r.t_launch_ns,
                     done=r.t_done_ns)
        return parse_payload(r.kind, data, r.bytes), times

    def release(self, ticket: int):
        _check(lib().ta_serve_release(self.h, ticket))

    def query(self, q: Query):
        t = self.submit(q)
        out, _ = self.poll(t, -1)
        self.release(t)
        return out

    def replay(self, queries, arrival_ns):
        """Open-loop replay; returns (latency_ns array, wall_ns)."""
        n = len(queries)
        arr = (Query * max(n, 1))(*queries)
        arrival = _np(arrival_ns, np.uint64)
        lat = np.zeros(max(n, 1), np.uint64)
        wall = u64(0)
        _check(lib().ta_serve_replay(self.h, C.cast(arr, P), arrival.ctypes.data, n,
                                     lat.ctypes.data, C.byref(wall)))
        return lat[:n], int(wall.value)


class Shard:
    """One contiguous rank range [rank_base, rank_base + R) of a job of
    n_total ranks, loaded as its own experiment: the sharded form's calls
    (include/ta.h, "sharded form").  Partials are int64 device tensors holding
    the library's u64 words (two's complement views: SUM, MIN and MAX over
    them equal the unsigned ones, every value being below 2^63), so any
    all-reduce merges them, e.g. torch.distributed.all_reduce or a sum over
    shards on one GPU."""

    def __init__(self, exp: Experiment, rank_base: int, n_total: int):
        self.e, self.rank_base, self.n_total = exp, int(rank_base), int(n_total)

    def _i64(self, n):
        torch = _torch()
        return torch.zeros(max(int(n), 1), dtype=torch.int64, device="cuda")

    def stats_partials(self, metric=EXCLUSIVE):
        """dict(sums [6 C] SUM, mins [C] MIN, maxs [C] MAX)."""
        C_ = self.e.C
        out = dict(sums=self._i64(6 * C_), mins=self._i64(C_), maxs=self._i64(C_))
        p = ShardStatsParts()
        p.sums, p.mins, p.maxs = (out[k].data_ptr() for k in ("sums", "mins", "maxs"))
        _check(lib().ta_shard_stats_partials(self.e.h, metric, C.byref(p)))
        return out

    def _merged(self, merged, metric, tau):
        m = ShardMerged()
        m.metric, m.rank_base, m.n_total = metric, self.rank_base, self.n_total
        m.tau_num, m.tau_den = tau
        m.sums, m.mins, m.maxs = (merged[k].data_ptr() for k in ("sums", "mins", "maxs"))
        return m

    def stats_finalize(self, merged, metric=EXCLUSIVE, tau=(3, 1), outlier_cap=1 << 20):
        """The job's statistics (device bytes of ta_ctx_stats[C]), this
        shard's argmax candidates (int64 [C], MIN) and outliers (host arrays,
        global rank ids)."""
        torch = _torch()
        C_ = self.e.C
        m = self._merged(merged, metric, tau)
        stats = torch.zeros(C_ * C.sizeof(CtxStats), dtype=torch.uint8, device="cuda")
        arg32 = torch.zeros(max(C_, 1), dtype=torch.int32, device="cuda")
        outl = torch.zeros(max(outlier_cap, 1) * C.sizeof(Outlier), dtype=torch.uint8,
                           device="cuda")
        o = ShardStatsOut()
        o.stats, o.argmax, o.outliers = stats.data_ptr(), arg32.data_ptr(), outl.data_ptr()
        o.outlier_cap = outlier_cap
        _check(lib().ta_shard_stats_finalize(self.e.h, C.byref(m), C.byref(o)))
        k = int(o.n_outliers)
        ol = (Outlier * max(k, 1)).from_buffer_copy(outl[: max(k, 1) * C.sizeof(Outlier)]
                                                    .cpu().numpy().tobytes())
        outliers = dict(ctx=np.array([x.ctx for x in ol[:k]], np.uint32),
                        rank=np.array([x.rank for x in ol[:k]], np.uint32),
                        z=np.array([x.z for x in ol[:k]], np.float64))
        argmax = arg32.to(torch.int64) & 0xFFFFFFFF
        return stats, argmax, outliers

    def set_argmax(self, stats, argmax):
        """Writes the merged argmax candidates into the statistics; returns
        them as a host dict like Experiment.stats()."""
        torch = _torch()
        a32 = argmax.to(torch.int32).contiguous()
        _check(lib().ta_shard_set_argmax(self.e.ctx.h, stats.data_ptr(), a32.data_ptr(),
                                         self.e.C))
        st = (CtxStats * self.e.C).from_buffer_copy(stats.cpu().numpy().tobytes())
        return {f: np.array([getattr(x, f) for x in st]) for f, _ in CtxStats._fields_
                if f != "reserved"}

    def topology_partials(self, merged, ctx, node_of_rank, n_nodes, metric=EXCLUSIVE, tau=(3, 1)):
        """node_parts int64 [3 n_nodes] (SUM); node_of_rank: this shard's
        ranks' global node ids."""
        torch = _torch()
        m = self._merged(merged, metric, tau)
        node = torch.as_tensor(np.asarray(node_of_rank, np.uint32).view(np.int32)).cuda()
        parts = self._i64(3 * n_nodes)
        _check(lib().ta_shard_topology_partials(self.e.h, C.byref(m), int(ctx), node.data_ptr(),
                                                int(n_nodes), parts.data_ptr()))
        return parts

    def speedup_bounds(self):
        """(min n_iter, sum of n_iter, longest span) of this shard."""
        b = (u64 * 3)()
        _check(lib().ta_shard_speedup_bounds(self.e.h, b))
        return int(b[0]), int(b[1]), int(b[2])

    def speedup_partials(self, ctxs, i_star):
        """dict(cells [5 I* nk] SUM, cell_max [I* nk] MAX, within [nk] f64 SUM)."""
        torch = _torch()
        cx = torch.as_tensor(np.asarray(ctxs, np.uint32).view(np.int32)).cuda()
        nk = len(ctxs)
        out = dict(cells=self._i64(5 * i_star * nk), cell_max=self._i64(i_star * nk),
                   within=torch.zeros(nk, dtype=torch.float64, device="cuda"))
        p = ShardSpeedupParts()
        p.cells, p.cell_max, p.within = (out[k].data_ptr() for k in ("cells", "cell_max", "within"))
        _check(lib().ta_shard_speedup_partials(self.e.h, cx.data_ptr(), nk, int(i_star),
                                               C.byref(p)))
        return out


def topology_finalize(ctx: Context, node_parts, rack_of_node, chassis_of_node, n_racks,
                      n_chassis, min_ranks=1):
    """The rack rollup from merged node partials (host dict like
    Experiment.topology())."""
    torch = _torch()
    nn = len(rack_of_node)
    rack = torch.as_tensor(np.asarray(rack_of_node, np.uint32).view(np.int32)).cuda()
    ch = torch.as_tensor(np.asarray(chassis_of_node, np.uint32).view(np.int32)).cuda()
    t = Topology()
    t.n_nodes, t.n_chassis, t.n_racks, t.mem_kind = nn, int(n_chassis), int(n_racks), MEM_DEVICE
    t.node_of_rank, t.rack_of_node, t.chassis_of_node = None, rack.data_ptr(), ch.data_ptr()
    spec = dict(node_outliers=(nn, np.uint32), node_sum=(nn, np.uint64),
                node_ranks=(nn, np.uint32), node_flag=(nn, np.uint8),
                chassis_flagged=(n_chassis, np.uint32), chassis_nodes=(n_chassis, np.uint32),
                chassis_sum=(n_chassis, np.uint64), rack_flagged=(n_racks, np.uint32),
                rack_nodes=(n_racks, np.uint32), rack_sum=(n_racks, np.uint64),
                flagged_racks=(n_racks, np.uint32))
    dev = {k: torch.zeros(max(int(n), 1) * np.dtype(dt).itemsize, dtype=torch.uint8,
                          device="cuda") for k, (n, dt) in spec.items()}
    o = TopoOut()
    o.mem_kind = MEM_DEVICE
    for k, v in dev.items():
        setattr(o, k, v.data_ptr())
    _check(lib().ta_topology_finalize(ctx.h, node_parts.data_ptr(), C.byref(t), int(min_ranks),
                                      C.byref(o)))
    out = {k: np.frombuffer(dev[k].cpu().numpy().tobytes(), dt)[: int(n)]
           for k, (n, dt) in spec.items()}
    out["flagged_racks"] = out["flagged_racks"][: int(o.n_flagged_racks)]
    return out


def speedup_finalize(ctx: Context, merged, n_total, i_star, excluded, t_app, nk):
    """The job's speedup from merged partials (host dicts like
    Experiment.speedup())."""
    torch = _torch()
    per = torch.zeros(nk * C.sizeof(SpeedupCtx), dtype=torch.uint8, device="cuda")
    tot = torch.zeros(C.sizeof(SpeedupTotal), dtype=torch.uint8, device="cuda")
    p = ShardSpeedupParts()
    p.cells, p.cell_max, p.within = (merged[k].data_ptr() for k in ("cells", "cell_max", "within"))
    _check(lib().ta_speedup_finalize(ctx.h, nk, int(n_total), int(i_star), int(excluded),
                                     int(t_app), C.byref(p), per.data_ptr(), tot.data_ptr()))
    pc = (SpeedupCtx * nk).from_buffer_copy(per.cpu().numpy().tobytes())
    tc = SpeedupTotal.from_buffer_copy(tot.cpu().numpy().tobytes())
    d = {f: np.array([getattr(x, f) for x in pc]) for f, _ in SpeedupCtx._fields_}
    d["G"] = [int(lo) + (int(hi) << 64) for lo, hi in zip(d["G_lo"], d["G_hi"])]
    t = {f: getattr(tc, f) for f, _ in SpeedupTotal._fields_ if f != "reserved"}
    t["sum_G"] = t["sum_G_lo"] + (t["sum_G_hi"] << 64)
    return d, t
