"""The C-ABI library loads on a machine without a GPU, exports every function
include/ta.h declares, and the Python binding's struct layouts match the C
header's (sizes and field offsets, checked by compiling the header)."""
import ctypes as C
import os
import subprocess
import tempfile

import pytest

import paper_2605_03561_b300 as ta
from paper_2605_03561_b300 import build as tabuild

STRUCTS = {"ta_trace_desc": ta.TraceDesc, "ta_experiment_info": ta.ExperimentInfo,
           "ta_tensor_out": ta.TensorOut, "ta_csr_out": ta.CsrOut, "ta_tensor_view": ta.TensorView,
           "ta_csr_view": ta.CsrView, "ta_stats_args": ta.StatsArgs, "ta_ctx_stats": ta.CtxStats,
           "ta_outlier": ta.Outlier, "ta_stats_out": ta.StatsOut, "ta_topology": ta.Topology,
           "ta_topo_args": ta.TopoArgs, "ta_topo_out": ta.TopoOut,
           "ta_speedup_args": ta.SpeedupArgs, "ta_speedup_ctx": ta.SpeedupCtx,
           "ta_speedup_total": ta.SpeedupTotal, "ta_speedup_out": ta.SpeedupOut,
           "ta_prune_args": ta.PruneArgs, "ta_prune_out": ta.PruneOut,
           "ta_interval_args": ta.IntervalArgs, "ta_cluster_args": ta.ClusterArgs,
           "ta_cluster_info": ta.ClusterInfo, "ta_cluster_out": ta.ClusterOut,
           "ta_profile": ta.Profile, "ta_batch_args": ta.BatchArgs,
           "ta_batch_info": ta.BatchInfo, "ta_batch_set_view": ta.BatchSetView,
           "ta_batch_set_args": ta.BatchSetArgs,
           "ta_shard_stats_parts": ta.ShardStatsParts, "ta_shard_merged": ta.ShardMerged,
           "ta_shard_stats_out": ta.ShardStatsOut,
           "ta_shard_speedup_parts": ta.ShardSpeedupParts,
           "ta_serve_config": ta.ServeConfig, "ta_query": ta.Query,
           "ta_query_result": ta.QueryResult, "ta_q_stats": ta.QStats,
           "ta_q_topk_entry": ta.QTopkEntry, "ta_q_racks": ta.QRacks}


def test_library_builds_and_exports_every_declared_symbol():
    path = tabuild.build()
    L = C.CDLL(path)
    names = ta.declared_symbols()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(names) == set(ta._SIGS), "binding signatures out of sync with ta.h"
    assert ta.lib().ta_status_string(ta.CAPACITY) == b"TA_ERR_CAPACITY"


def test_struct_layouts_match_header():
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ta.h"', "int main(void){"]
    for cname, py in STRUCTS.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        open(src, "w").write("\n".join(lines))
        subprocess.check_call(["gcc", "-I", os.path.join(ta._HERE, "..", "include"), src, "-o", exe])
        out = subprocess.check_output([exe]).decode().split("\n")
    got = dict(l.split() for l in out if l)
    for cname, py in STRUCTS.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)


def test_error_text_without_gpu():
    # Creating a context without a GPU fails cleanly with a CUDA status.
    import torch
    if torch.cuda.is_available():
        pytest.skip("has a GPU")
    h = C.c_void_p()
    s = ta.lib().ta_create(0, None, C.byref(h))
    assert s in (ta.CUDA, ta.INVALID_ARG)
    assert ta.lib().ta_last_error_message()
