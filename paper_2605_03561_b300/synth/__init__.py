"""Seeded synthetic trace sets (Python side of ``tagen.cpp``).

Stand-in for the paper's missing AMG / GAMESS trace databases (Section VI).
The recipe is documented in ``tagen.cpp``.  This module draws inputs only; it
holds none of the analysis method's arithmetic, and both the CUDA path's tests
and the CPU oracle consume what it produces.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "tagen.cpp"), os.path.join(_HERE, "tagen.h")]
_LIB = os.path.join(_HERE, "libtagen.so")

LEN_FIXED, LEN_LOGNORMAL = 0, 1
SLOW_NONE, SLOW_RANKS, SLOW_JITTER, SLOW_RACK_COMM = 0, 1, 2, 3


class Config(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("n_ranks", C.c_uint32), ("n_ctx", C.c_uint32),
                ("max_depth", C.c_uint32), ("n_iter", C.c_uint32), ("n_segments", C.c_uint32),
                ("prologue_len", C.c_uint32), ("marker_ctx", C.c_uint32), ("len_kind", C.c_uint32),
                ("len_mean", C.c_double), ("len_sigma", C.c_double), ("gap_mean_ns", C.c_double),
                ("slow_model", C.c_uint32), ("n_slow_ranks", C.c_uint32),
                ("slow_factor", C.c_double), ("jitter_sigma", C.c_double),
                ("jitter_clip", C.c_double), ("imb_rank_frac", C.c_double),
                ("imb_iter_prob", C.c_double), ("imb_lo", C.c_double), ("imb_hi", C.c_double),
                ("comm_frac", C.c_double), ("ranks_per_node", C.c_uint32),
                ("n_racks", C.c_uint32), ("nodes_per_chassis", C.c_uint32),
                ("n_slow_racks", C.c_uint32), ("shuffle_segments", C.c_uint32)]


class Info(C.Structure):
    _fields_ = [("n_segments", C.c_uint32), ("prologue_ctx", C.c_uint32),
                ("n_nodes", C.c_uint32), ("n_chassis", C.c_uint32),
                ("n_records", C.c_uint64), ("max_len", C.c_uint32)]


def build(force: bool = False) -> str:
    newest = max(os.path.getmtime(s) for s in _SRC)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread",
                               "-o", _LIB + ".tmp", _SRC[0]])
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.tagen_preset.argtypes = [C.c_int, C.POINTER(Config)]
        _lib.tagen_plan.argtypes = [C.POINTER(Config), C.c_void_p, C.c_void_p, C.POINTER(Info)]
        _lib.tagen_fill.argtypes = [C.POINTER(Config), C.c_void_p, C.c_uint32, C.c_uint32,
                                    C.c_void_p, C.c_void_p, C.c_int]
        _lib.tagen_topology.argtypes = [C.POINTER(Config), C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.tagen_truth.argtypes = [C.POINTER(Config)] + [C.c_void_p] * 4
    return _lib


def preset(n: int, seed: int = 1, **overrides) -> Config:
    """Config family n (0 tiny, 1: 64 ranks, 2: 4096 ranks, 3: 100,000 ranks)."""
    cfg = Config()
    if lib().tagen_preset(n, C.byref(cfg)) != 0:
        raise ValueError(f"unknown preset {n}")
    cfg.seed = seed
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def plan(cfg: Config):
    """rank_off[R+1], parent[C], info."""
    rank_off = np.zeros(cfg.n_ranks + 1, np.uint64)
    parent = np.zeros(cfg.n_ctx, np.uint32)
    info = Info()
    if lib().tagen_plan(C.byref(cfg), rank_off.ctypes.data, parent.ctypes.data,
                        C.byref(info)) != 0:
        raise ValueError("invalid generator config")
    return rank_off, parent, info


def fill(cfg: Config, rank_off: np.ndarray, r0: int, r1: int, ts_ptr: int, ctx_ptr: int,
         n_threads: int = 0) -> None:
    """Write the records of ranks [r0, r1) at raw host addresses ts_ptr/ctx_ptr."""
    if lib().tagen_fill(C.byref(cfg), rank_off.ctypes.data, r0, r1, ts_ptr, ctx_ptr,
                        n_threads) != 0:
        raise ValueError("tagen_fill failed")


def topology(cfg: Config, info: Info):
    node = np.zeros(cfg.n_ranks, np.uint32)
    rack = np.zeros(info.n_nodes, np.uint32)
    chassis = np.zeros(info.n_nodes, np.uint32)
    lib().tagen_topology(C.byref(cfg), node.ctypes.data, rack.ctypes.data, chassis.ctypes.data)
    return dict(node_of_rank=node, rack_of_node=rack, chassis_of_node=chassis,
                n_nodes=info.n_nodes, n_chassis=info.n_chassis, n_racks=max(cfg.n_racks, 1))


def truth(cfg: Config, info: Info):
    slowed_rank = np.zeros(cfg.n_ranks, np.uint8)
    slowed_rack = np.zeros(max(cfg.n_racks, 1), np.uint8)
    comm = np.zeros(max(info.n_segments, 1), np.uint8)
    seg = np.zeros(max(info.n_segments, 1), np.uint32)
    lib().tagen_truth(C.byref(cfg), slowed_rank.ctypes.data, slowed_rack.ctypes.data,
                      comm.ctypes.data, seg.ctypes.data)
    return dict(slowed_rank=slowed_rank, slowed_rack=slowed_rack,
                comm_segment=comm[: info.n_segments], segment_ctx=seg[: info.n_segments])


def generate(cfg: Config, n_threads: int = 0):
    """Whole experiment in numpy arrays (for sizes that fit host memory)."""
    rank_off, parent, info = plan(cfg)
    n = int(rank_off[-1])
    ts = np.empty(n, np.uint64)
    ctx = np.empty(n, np.uint32)
    if n:
        fill(cfg, rank_off, 0, cfg.n_ranks, ts.ctypes.data, ctx.ctypes.data, n_threads)
    return dict(rank_off=rank_off, ts=ts, ctx=ctx, parent=parent, marker=cfg.marker_ctx,
                info=info, cfg=cfg)
