"""CPU oracle for the trace-analysis path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``oracle.cpp`` (plain,
single-threaded C++, written from the paper's definitions; see the header of
that file for the section each function follows) through ctypes; pruning, time
windows, call chains, the clustering of ranks (DBSCAN, K-Means, node view) and
the column operations are plain Python loops in this file.  It shares no
code with the CUDA path and never imports it.

Parity pins live in ``tests/test_oracle_*.py``.  The per-group CV definitions
(``cv_across``, ``cv_within``) are parity unpinned against the paper's printed
numbers (the data behind Table IV is not available); their arithmetic is pinned
by closed-form cases only.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, INVALID, NOT_SORTED, BAD_CTX, BAD_CCT = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "ok", 1: "invalid_arg", 2: "not_sorted", 3: "bad_ctx", 4: "bad_cct"}
EXCL, INCL = 0, 1


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain g++, no fast-math, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", _LIB + ".tmp", _SRC]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Input(C.Structure):
    _fields_ = [("n_ranks", C.c_uint32), ("n_ctx", C.c_uint32), ("marker_ctx", C.c_uint32),
                ("pad", C.c_uint32), ("n_records", C.c_uint64), ("rank_off", C.c_void_p),
                ("ts", C.c_void_p), ("ctx", C.c_void_p), ("parent", C.c_void_p)]


class CtxStats(C.Structure):
    _fields_ = [("n", C.c_uint32), ("present", C.c_uint32), ("argmax", C.c_uint32),
                ("pad", C.c_uint32), ("min", C.c_uint64), ("max", C.c_uint64),
                ("s1", C.c_uint64), ("s2_lo", C.c_uint64), ("s2_hi", C.c_uint64),
                ("mean", C.c_double), ("std", C.c_double), ("cv", C.c_double),
                ("balance", C.c_double)]


class Outlier(C.Structure):
    _fields_ = [("ctx", C.c_uint32), ("rank", C.c_uint32), ("z", C.c_double)]


class SpeedupCtx(C.Structure):
    _fields_ = [("A", C.c_uint64), ("B", C.c_uint64), ("G_lo", C.c_uint64), ("G_hi", C.c_uint64),
                ("avg_mean", C.c_double), ("avg_max", C.c_double),
                ("savings_per_iter", C.c_double), ("total_reduction", C.c_double),
                ("share", C.c_double), ("cv_across", C.c_double), ("cv_within", C.c_double)]


class SpeedupTotal(C.Structure):
    _fields_ = [("i_star", C.c_uint32), ("pad", C.c_uint32), ("excluded_iterations", C.c_uint64),
                ("sum_G_lo", C.c_uint64), ("sum_G_hi", C.c_uint64), ("t_app", C.c_uint64),
                ("total_reduction", C.c_double), ("speedup_fraction", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.or_validate.restype = C.c_int
        L.or_validate.argtypes = [C.POINTER(_Input)]
        L.or_u128_to_double.restype = C.c_double
        L.or_u128_to_double.argtypes = [C.c_uint64, C.c_uint64]
        L.or_analyze.restype = C.c_void_p
        L.or_analyze.argtypes = [C.POINTER(_Input), C.c_uint32, C.c_uint32, C.c_int, C.c_int,
                                 C.POINTER(C.c_int)]
        L.or_free.argtypes = [C.c_void_p]
        L.or_tensor_sizes.argtypes = [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
        L.or_tensor_get.argtypes = [C.c_void_p] + [C.c_void_p] * 6
        L.or_csr_nnz.restype = C.c_uint64
        L.or_csr_nnz.argtypes = [C.c_void_p, C.c_int]
        L.or_csr_get.argtypes = [C.c_void_p, C.c_int] + [C.c_void_p] * 4
        L.or_span_get.argtypes = [C.c_void_p, C.c_void_p]
        L.or_stats.restype = C.c_int
        L.or_stats.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_uint32, C.c_void_p,
                               C.c_uint32, C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p,
                               C.c_uint64, C.POINTER(C.c_uint64), C.c_void_p]
        L.or_topology.restype = C.c_int
        L.or_topology.argtypes = ([C.c_void_p, C.c_int, C.c_uint32, C.c_uint32, C.c_uint32,
                                   C.c_uint32, C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint32,
                                   C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint32]
                                  + [C.c_void_p] * 12)
        L.or_speedup.restype = C.c_int
        L.or_speedup.argtypes = [C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint32,
                                 C.c_uint64, C.c_void_p, C.POINTER(SpeedupTotal)]
        L.or_slice.restype = C.c_int
        L.or_slice.argtypes = [C.c_void_p] + [C.c_uint32] * 5 + [C.c_void_p]
        L.or_topk.restype = C.c_int
        L.or_topk.argtypes = [C.c_void_p, C.c_int, C.c_uint32, C.c_uint32, C.c_void_p,
                              C.c_void_p, C.c_void_p, C.POINTER(C.c_uint32)]
        L.or_savings_from_averages.argtypes = [C.c_void_p, C.c_void_p, C.c_uint32, C.c_uint32,
                                               C.c_double, C.c_void_p, C.c_void_p,
                                               C.POINTER(C.c_double), C.POINTER(C.c_double)]
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _u32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.uint32)


class Traces:
    """Host arrays of one experiment (kept alive for the oracle handle)."""

    def __init__(self, rank_off, ts, ctx, parent, marker):
        self.rank_off = np.ascontiguousarray(rank_off, dtype=np.uint64)
        self.ts = np.ascontiguousarray(ts, dtype=np.uint64)
        self.ctx = np.ascontiguousarray(ctx, dtype=np.uint32)
        self.parent = np.ascontiguousarray(parent, dtype=np.uint32)
        self.marker = int(marker)
        self.R = len(self.rank_off) - 1
        self.C = len(self.parent)
        self.N = int(self.rank_off[-1]) if self.R >= 0 and len(self.rank_off) else 0

    def struct(self):
        s = _Input()
        s.n_ranks, s.n_ctx, s.marker_ctx = self.R, self.C, self.marker
        s.n_records = len(self.ts)
        s.rank_off, s.ts = _p(self.rank_off), _p(self.ts)
        s.ctx, s.parent = _p(self.ctx), _p(self.parent)
        return s


def validate(tr: Traces) -> int:
    s = tr.struct()
    return lib().or_validate(C.byref(s))


def u128_to_double(v: int) -> float:
    return lib().or_u128_to_double(v & (2**64 - 1), v >> 64)


class Analysis:
    """Oracle results for ranks [r0, r1) of one experiment."""

    def __init__(self, tr: Traces, r0=0, r1=None, rows=True, incl=True, validate=True):
        self.tr = tr
        self.r0 = r0
        self.r1 = tr.R if r1 is None else r1
        s = tr.struct()
        st = C.c_int(0)
        want = (1 if rows else 0) | (2 if incl else 0)
        self.h = lib().or_analyze(C.byref(s), r0, self.r1, want, 1 if validate else 0, C.byref(st))
        self.status = st.value
        if not self.h:
            raise OracleError(self.status)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().or_free(h)
            self.h = None

    def tensor(self):
        rows, nnz = C.c_uint64(0), C.c_uint64(0)
        lib().or_tensor_sizes(self.h, C.byref(rows), C.byref(nnz))
        n = self.r1 - self.r0
        out = dict(row_off_of_rank=np.zeros(n + 1, np.uint64),
                   entry_off=np.zeros(rows.value + 1, np.uint64),
                   e_ctx=np.zeros(nnz.value, np.uint32), e_time=np.zeros(nnz.value, np.uint64),
                   e_cnt=np.zeros(nnz.value, np.uint32), n_iter=np.zeros(n, np.uint32))
        lib().or_tensor_get(self.h, _p(out["row_off_of_rank"]), _p(out["entry_off"]),
                            _p(out["e_ctx"]), _p(out["e_time"]), _p(out["e_cnt"]),
                            _p(out["n_iter"]))
        return out

    def csr(self, which=EXCL):
        nnz = lib().or_csr_nnz(self.h, which)
        n = self.r1 - self.r0
        out = dict(off=np.zeros(n + 1, np.uint64), ctx=np.zeros(nnz, np.uint32),
                   time=np.zeros(nnz, np.uint64), cnt=np.zeros(nnz, np.uint32))
        lib().or_csr_get(self.h, which, _p(out["off"]), _p(out["ctx"]), _p(out["time"]),
                         _p(out["cnt"]))
        return out

    def span(self):
        out = np.zeros(self.r1 - self.r0, np.uint64)
        lib().or_span_get(self.h, _p(out))
        return out

    def interval(self, t0, t1, incl=False):
        """Per-rank profiles of the time window [t0, t1) (Section III-A's
        trace slices; Section II-A samples: sample i of a rank is in ctx_i
        during [ts_i, ts_{i+1}), the rank's last sample lasts 0 ns).  A sample
        adds to its context the length of its interval inside the window and
        counts as a sample iff ts_i lies in the window; a (rank, context) is
        listed iff it gets time or samples.  With incl, every value is also
        added along the context's path to the root.  Returns a CSR over the
        analysed ranks (contexts ascending).  Plain loops; small inputs."""
        tr = self.tr
        parent = np.asarray(tr.parent).tolist()
        off, ctx, time, cnt = [0], [], [], []
        for r in range(self.r0, self.r1):
            b, e = int(tr.rank_off[r]), int(tr.rank_off[r + 1])
            acc = {}
            for i in range(b, e):
                ts = int(tr.ts[i])
                nxt = int(tr.ts[i + 1]) if i + 1 < e else ts
                d = max(0, min(nxt, t1) - max(ts, t0))
                n = 1 if t0 <= ts < t1 else 0
                if d == 0 and n == 0:
                    continue
                c = int(tr.ctx[i])
                while True:
                    v = acc.setdefault(c, [0, 0])
                    v[0] += d
                    v[1] += n
                    if not incl or parent[c] == 0xFFFFFFFF:
                        break
                    c = parent[c]
            for c in sorted(acc):
                ctx.append(c)
                time.append(acc[c][0])
                cnt.append(acc[c][1])
            off.append(len(ctx))
        return dict(off=np.array(off, np.uint64), ctx=np.array(ctx, np.uint32),
                    time=np.array(time, np.uint64), cnt=np.array(cnt, np.uint32))

    def call_chain(self, c):
        """The calling context of node c, bottom up (Section VI-B, "Obtaining
        Calling Context"): c, its parent, ..., the root."""
        parent = np.asarray(self.tr.parent).tolist()
        out = [int(c)]
        while parent[out[-1]] != 0xFFFFFFFF:
            out.append(parent[out[-1]])
        return np.array(out, np.uint32)

    def values(self, ctx, metric=EXCL, ranks=None):
        """Per-rank value of context ctx over a rank subset (relative rank ids;
        None: every analysed rank), 0 where the rank has no sample of it --
        the per-rank series the paper clusters (Section VI-B)."""
        csr = self.csr(metric)
        ranks = range(self.r1 - self.r0) if ranks is None else ranks
        out = []
        for r in ranks:
            v = 0
            for j in range(int(csr["off"][r]), int(csr["off"][r + 1])):
                if int(csr["ctx"][j]) == ctx:
                    v = int(csr["time"][j])
                    break
            out.append(v)
        return out

    def prune(self, keep_num, keep_den, drop=None):
        """Pruning of the calling context tree on the summary profile (Section
        III-A, "Pruning Large Calling Context Trees": a strategy is evaluated
        once on the summary profile, the aggregate of all parallel profiles,
        then propagated to every parallel profile; Section VI-B drops the
        regions under 1 % of the total runtime, and MPI internals and line
        statements by class).

        The summary profile holds, per context, its inclusive time summed
        over the ranks; the total is the root's.  Context c is kept iff
        summary[c] * keep_den >= total * keep_num (exact integers) and not
        drop[c].  Every rank's exclusive and inclusive profile keeps the
        entries of kept contexts, in order; a dropped context's time is not
        moved elsewhere.  Returns (kept u8[C], summary u64[C], exclusive CSR,
        inclusive CSR).  Written as plain loops; for small inputs."""
        n_ctx = self.tr.C
        inc = self.csr(INCL)
        summary = [0] * n_ctx
        for c, t in zip(inc["ctx"].tolist(), inc["time"].tolist()):
            summary[c] += int(t)
        parent = np.asarray(self.tr.parent).tolist()
        root = parent.index(0xFFFFFFFF)
        total = summary[root]
        kept = [1 if summary[c] * keep_den >= total * keep_num and not (drop is not None and drop[c])
                else 0 for c in range(n_ctx)]

        def restrict(csr):
            off, ctx, time, cnt = [0], [], [], []
            for r in range(self.r1 - self.r0):
                for j in range(int(csr["off"][r]), int(csr["off"][r + 1])):
                    if kept[int(csr["ctx"][j])]:
                        ctx.append(int(csr["ctx"][j]))
                        time.append(int(csr["time"][j]))
                        cnt.append(int(csr["cnt"][j]))
                off.append(len(ctx))
            return dict(off=np.array(off, np.uint64), ctx=np.array(ctx, np.uint32),
                        time=np.array(time, np.uint64), cnt=np.array(cnt, np.uint32))

        return (np.array(kept, np.uint8), np.array(summary, np.uint64),
                restrict(self.csr(EXCL)), restrict(inc))

    def stats(self, metric=EXCL, ranks=None, ctxs=None, tau=(3, 1), cap=1 << 20, want_z=False):
        ranks, ctxs = _u32(ranks), _u32(ctxs)
        k = self.tr.C if ctxs is None else len(ctxs)
        st = (CtxStats * max(k, 1))()
        outl = (Outlier * max(cap, 1))()
        n_out = C.c_uint64(0)
        z = np.zeros(lib().or_csr_nnz(self.h, metric), np.float64) if want_z else None
        s = lib().or_stats(self.h, metric, _p(ranks), 0 if ranks is None else len(ranks),
                           _p(ctxs), 0 if ctxs is None else len(ctxs), tau[0], tau[1],
                           C.cast(st, C.c_void_p), C.cast(outl, C.c_void_p), cap,
                           C.byref(n_out), _p(z))
        if s != OK:
            raise OracleError(s)
        stats = _structs_to_dict(st[:k], CtxStats)
        m = min(n_out.value, cap)
        outliers = dict(ctx=np.array([o.ctx for o in outl[:m]], np.uint32),
                        rank=np.array([o.rank for o in outl[:m]], np.uint32),
                        z=np.array([o.z for o in outl[:m]], np.float64))
        return stats, outliers, n_out.value, z

    def topology(self, ctx, node_of_rank, rack_of_node, chassis_of_node, n_racks, n_chassis,
                 metric=EXCL, tau=(3, 1), min_ranks=1, ranks=None):
        node_of_rank, rack_of_node = _u32(node_of_rank), _u32(rack_of_node)
        chassis_of_node, ranks = _u32(chassis_of_node), _u32(ranks)
        nn = len(rack_of_node)
        o = dict(node_outliers=np.zeros(nn, np.uint32), node_sum=np.zeros(nn, np.uint64),
                 node_ranks=np.zeros(nn, np.uint32), node_flag=np.zeros(nn, np.uint8),
                 chassis_flagged=np.zeros(n_chassis, np.uint32),
                 chassis_nodes=np.zeros(n_chassis, np.uint32),
                 chassis_sum=np.zeros(n_chassis, np.uint64),
                 rack_flagged=np.zeros(n_racks, np.uint32), rack_nodes=np.zeros(n_racks, np.uint32),
                 rack_sum=np.zeros(n_racks, np.uint64), flagged_racks=np.zeros(n_racks, np.uint32))
        nf = np.zeros(1, np.uint32)
        s = lib().or_topology(self.h, metric, ctx, tau[0], tau[1], min_ranks, _p(ranks),
                              0 if ranks is None else len(ranks), _p(node_of_rank), nn,
                              _p(rack_of_node), n_racks, _p(chassis_of_node), n_chassis,
                              _p(o["node_outliers"]), _p(o["node_sum"]), _p(o["node_ranks"]),
                              _p(o["node_flag"]), _p(o["chassis_flagged"]),
                              _p(o["chassis_nodes"]), _p(o["chassis_sum"]),
                              _p(o["rack_flagged"]), _p(o["rack_nodes"]), _p(o["rack_sum"]),
                              _p(o["flagged_racks"]), _p(nf))
        if s != OK:
            raise OracleError(s)
        o["flagged_racks"] = o["flagged_racks"][: int(nf[0])]
        return o

    def slice(self, ctx, r0, r1, i0, i1):
        """Dense [r1 - r0, i1 - i0] time of ctx per (rank, iteration)."""
        out = np.zeros((r1 - r0) * (i1 - i0), np.uint64)
        s = lib().or_slice(self.h, ctx, r0, r1, i0, i1, _p(out))
        if s != OK:
            raise OracleError(s)
        return out.reshape(r1 - r0, i1 - i0)

    def topk(self, ctx, k, metric=EXCL):
        """(ranks, x, z) of the k largest values of ctx, ties to lower rank."""
        n = self.r1 - self.r0
        rk = np.zeros(max(min(k, n), 1), np.uint32)
        x = np.zeros(max(min(k, n), 1), np.uint64)
        z = np.zeros(max(min(k, n), 1), np.float64)
        m = C.c_uint32(0)
        s = lib().or_topk(self.h, metric, ctx, k, _p(rk), _p(x), _p(z), C.byref(m))
        if s != OK:
            raise OracleError(s)
        return rk[: m.value], x[: m.value], z[: m.value]

    def speedup(self, ctxs, ranks=None, app_time_ns=0):
        ctxs, ranks = _u32(ctxs), _u32(ranks)
        per = (SpeedupCtx * len(ctxs))()
        tot = SpeedupTotal()
        s = lib().or_speedup(self.h, _p(ctxs), len(ctxs), _p(ranks),
                             0 if ranks is None else len(ranks), app_time_ns,
                             C.cast(per, C.c_void_p), C.byref(tot))
        if s != OK:
            raise OracleError(s)
        d = _structs_to_dict(per[:], SpeedupCtx)
        d["G"] = [int(lo) + (int(hi) << 64) for lo, hi in zip(d["G_lo"], d["G_hi"])]
        t = {f: getattr(tot, f) for f, _ in SpeedupTotal._fields_ if f != "pad"}
        t["sum_G"] = t["sum_G_lo"] + (t["sum_G_hi"] << 64)
        return d, t


def dbscan(x, eps, min_pts):
    """DBSCAN (Ester et al., as applied to per-rank times in Section VI-B) on
    integer scalars.  The eps-neighbourhood of a point holds every point q
    with |x_q - x_p| <= eps, itself included; a point is a core point when
    its neighbourhood has at least min_pts points; clusters are the connected
    components of core points, two cores being connected when they are
    neighbours; a non-core point within eps of a core is a border point and
    joins the cluster of its nearest core (equal distances: the cluster of
    smaller values); every other point is noise (-1).  Clusters are numbered
    in ascending order of value.  Returns (labels, core flags)."""
    import bisect
    n = len(x)
    order = sorted(range(n), key=lambda i: x[i])
    xs = [x[i] for i in order]

    def region(p):
        lo = bisect.bisect_left(xs, x[p] - eps)
        hi = bisect.bisect_right(xs, x[p] + eps)
        return [order[j] for j in range(lo, hi)]

    core = []
    for p in range(n):
        lo = bisect.bisect_left(xs, x[p] - eps)
        hi = bisect.bisect_right(xs, x[p] + eps)
        core.append(hi - lo >= min_pts)
    comp = [-1] * n
    n_comp = 0
    for p in order:  # expansion from the smallest unvisited core
        if not core[p] or comp[p] >= 0:
            continue
        comp[p] = n_comp
        stack = [p]
        while stack:
            q = stack.pop()
            for o in region(q):
                if core[o] and comp[o] < 0:
                    comp[o] = n_comp
                    stack.append(o)
        n_comp += 1
    labels = []
    for p in range(n):
        if core[p]:
            labels.append(comp[p])
            continue
        best = None
        for o in region(p):
            if core[o]:
                key = (abs(x[o] - x[p]), comp[o])
                if best is None or key < best:
                    best = key
        labels.append(-1 if best is None else best[1])
    return labels, core


def kmeans(x, k, max_iter):
    """K-Means (Lloyd's iteration; Section VI-B's stability check) on integer
    scalars in exact rational arithmetic.  Start: centroid j is the value at
    sorted position floor((2j + 1) n / (2k)).  Each assignment step orders
    the clusters by centroid (stably) and gives every point to the first
    cluster in that order at the smallest distance; each update step moves a
    non-empty cluster's centroid to its mean (an empty one keeps its
    centroid).  Stops when an assignment repeats the previous one or after
    max_iter updates.  Returns (labels as positions in the final order,
    centroids in that order as Fractions, updates made, the centroids as
    unreduced (sum, count) pairs)."""
    from fractions import Fraction
    n = len(x)
    xs = sorted(x)
    pairs = [(xs[(2 * j + 1) * n // (2 * k)], 1) for j in range(k)]

    def assign(pairs):
        order = sorted(range(k), key=lambda j: Fraction(*pairs[j]))  # stable
        pairs = [pairs[j] for j in order]
        cents = [Fraction(*p) for p in pairs]
        lab = [min(range(k), key=lambda j: (abs(v - cents[j]), j)) for v in x]
        return pairs, lab

    pairs, labels = assign(pairs)
    it = 0
    while it < max_iter:
        for j in range(k):
            members = [v for v, l in zip(x, labels) if l == j]
            if members:
                pairs[j] = (sum(members), len(members))
        it += 1
        pairs, new = assign(pairs)
        same = new == labels
        labels = new
        if same:
            break
    return labels, [Fraction(*p) for p in pairs], it, pairs


def cluster_nodes(labels, node_of_rank, n_nodes, n_clusters):
    """Node view of a rank clustering (Section VI-B maps rank clusters to
    compute nodes): per cluster the nodes holding at least one of its ranks,
    per pair of clusters i < j the nodes holding ranks of both, and the nodes
    holding a noise rank."""
    sets = [set() for _ in range(n_nodes)]
    for l, nd in zip(labels, node_of_rank):
        sets[nd].add(l)
    per = [0] * n_clusters
    pair = [[0] * n_clusters for _ in range(n_clusters)]
    noise = 0
    for s in sets:
        if -1 in s:
            noise += 1
        ls = sorted(l for l in s if l >= 0)
        for a in ls:
            per[a] += 1
        for i in range(len(ls)):
            for j in range(i + 1, len(ls)):
                pair[ls[i]][ls[j]] += 1
    return per, pair, noise


# ---------------------------------------------------------------------------
# Column operations (Section IV, Tables I-III: the DataFrame operation classes
# the paper times on trace events).  Plain definitions over numpy arrays.

def events_table(tr, r0, r1):
    """The trace events of ranks [r0, r1) as columns: rank, ts, ctx and the
    duration (next timestamp of the rank minus this one; 0 for a rank's last
    event, Section II-A)."""
    rank, ts, ctx, dur = [], [], [], []
    for r in range(r0, r1):
        b, e = int(tr.rank_off[r]), int(tr.rank_off[r + 1])
        for i in range(b, e):
            rank.append(r)
            ts.append(int(tr.ts[i]))
            ctx.append(int(tr.ctx[i]))
            dur.append(int(tr.ts[i + 1]) - int(tr.ts[i]) if i + 1 < e else 0)
    return dict(rank=np.array(rank, np.uint32), ts=np.array(ts, np.uint64),
                ctx=np.array(ctx, np.uint32), dur=np.array(dur, np.uint64))


def col_sort(keys):
    """Stable ascending sort: (sorted keys, permutation)."""
    perm = np.argsort(np.asarray(keys, np.uint64), kind="stable").astype(np.uint32)
    return np.asarray(keys, np.uint64)[perm], perm


def col_filter(col, lo, hi):
    """Ascending indices i with lo <= col[i] <= hi."""
    return np.array([i for i, v in enumerate(np.asarray(col).tolist()) if lo <= v <= hi],
                    np.uint32)


def col_group(seg_off, key, val):
    """Per segment s (rows [seg_off[s], seg_off[s+1])) and key: the sum of val
    and the row count, keys ascending within a segment (a group-by on
    (segment, key))."""
    off, keys, sums, cnts = [0], [], [], []
    key, val = np.asarray(key).tolist(), np.asarray(val).tolist()
    for s in range(len(seg_off) - 1):
        acc = {}
        for i in range(int(seg_off[s]), int(seg_off[s + 1])):
            a = acc.setdefault(key[i], [0, 0])
            a[0] += val[i]
            a[1] += 1
        for k in sorted(acc):
            keys.append(k)
            sums.append(acc[k][0])
            cnts.append(acc[k][1])
        off.append(len(keys))
    return dict(off=np.array(off, np.uint64), key=np.array(keys, np.uint32),
                sum=np.array(sums, np.uint64), cnt=np.array(cnts, np.uint32))


def col_gather(key, dim):
    """The merge of a fact column with a dimension table on its row id:
    out[i] = dim[key[i]]."""
    return np.array([dim[k] for k in np.asarray(key).tolist()], np.uint32)


def savings_from_averages(avg_mean, avg_max, iterations, app_time):
    a = np.ascontiguousarray(avg_mean, np.float64)
    b = np.ascontiguousarray(avg_max, np.float64)
    s = np.zeros(len(a)), np.zeros(len(a))
    tot, frac = C.c_double(0), C.c_double(0)
    lib().or_savings_from_averages(_p(a), _p(b), len(a), iterations, app_time, _p(s[0]),
                                   _p(s[1]), C.byref(tot), C.byref(frac))
    return s[0], s[1], tot.value, frac.value


def _structs_to_dict(items, cls):
    names = [f for f, _ in cls._fields_ if f != "pad"]
    return {f: np.array([getattr(it, f) for it in items]) for f in names}


class OracleError(RuntimeError):
    def __init__(self, status):
        super().__init__(f"oracle status {status} ({STATUS_NAMES.get(status, '?')})")
        self.status = status
