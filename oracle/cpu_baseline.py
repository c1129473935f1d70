"""The paper's multicore scheme (Section 5) on the host cores: a CPU baseline.

BENCHMARK INFRASTRUCTURE ONLY (used by ``bench.py``).  It is not a parity oracle:
its threads race by design, so runs are not reproducible.  The arithmetic lives in
``cpu_baseline_mt.c`` (pthreads, FP32, atomic adds by compare-and-swap); this module
builds it and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpu_baseline_mt.c")
_LIB = os.path.join(_HERE, "libcpu_baseline.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O3", "-std=gnu11", "-fPIC", "-shared", "-pthread", "-o",
                               tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, i64 = ctypes.c_void_p, ctypes.c_int64
        lib.cpu_asyrk_mt.argtypes = [i64, P, P, P, P, P, P, ctypes.c_float, ctypes.c_int, i64,
                                     ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]
        lib.cpu_asyrk_mt.restype = i64
        _lib = lib
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def run(m, row_ptr, col, val, b, x, gamma=1.0, threads=None, scans=1, seed=1):
    """Runs ``scans`` scans of every thread's row slice; x (float32) is updated in place.

    Returns (projections, seconds, threads)."""
    threads = threads or len(os.sched_getaffinity(0)) or 1
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    c = np.ascontiguousarray(col, dtype=np.int32)
    v = np.ascontiguousarray(val, dtype=np.float32)
    bb = np.ascontiguousarray(b, dtype=np.float32)
    v64 = v.astype(np.float64)
    w = np.add.reduceat(v64 * v64, rp[:-1]) if v.size else np.zeros(m)
    inv_w = (1.0 / w).astype(np.float32)
    assert x.dtype == np.float32 and x.flags.c_contiguous
    secs = ctypes.c_double()
    done = _load().cpu_asyrk_mt(m, _p(rp), _p(c), _p(v), _p(bb), _p(inv_w), _p(x), float(gamma),
                                int(threads), int(scans), int(seed), ctypes.byref(secs))
    if done < 0:
        raise RuntimeError("could not start the CPU baseline threads")
    return int(done), secs.value, threads
