"""RAKS-CPU: the paper's multi-core CPU search (OpenMP), a parallel baseline.

Reported next to the GPU library by the benchmark; neither the oracle nor
part of the library's product path.  See raks_cpu.c.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "raks_cpu.c")
_LIB = os.path.join(_HERE, "_raks_cpu.so")
_lib = None


def build_lib(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_lib())
        P, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        _lib.raks_activation.argtypes = [i32, i64, P, P, P, i32, f64, f64, P]
        _lib.raks_activation.restype = ctypes.c_int
        _lib.raks_search.argtypes = [i32, P, P, P, P, P, P, i32, P, i32, i32, i32, f64, P, P, P, P]
        _lib.raks_search.restype = i32
        _lib.raks_threads.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    return int(_L().raks_threads())


def activation(ds) -> np.ndarray:
    g = ds.graph
    a = np.empty(g.m2, np.uint8)
    rc = _L().raks_activation(g.n, g.m2, _p(g.row_ptr), _p(g.col), _p(g.label), g.n_labels, ds.alpha, ds.abar, _p(a))
    if rc != 0:
        raise ValueError("graph is not bi-directed")
    return a


def search(ds, a, central, marginal, k, max_depth, gamma=0.5):
    g = ds.graph
    c = np.ascontiguousarray(central, np.int32)
    m = np.ascontiguousarray(marginal, np.int32)
    node = np.zeros(max(k, 1), np.int64)
    sc = np.zeros(max(k, 1), np.int32)
    sm = np.zeros(max(k, 1), np.int32)
    sr = np.zeros(max(k, 1), np.float64)
    nr = _L().raks_search(g.n, _p(g.row_ptr), _p(g.col), _p(a), _p(ds.kw_ptr), _p(ds.kw_nodes), _p(c), len(c),
                          _p(m) if len(m) else None, len(m), int(k), int(max_depth), float(gamma),
                          _p(node), _p(sc), _p(sm), _p(sr))
    return node[:nr], sc[:nr], sm[:nr], sr[:nr]
