"""Builds and loads the C++/OpenMP oracle CGLS (``cpu_cgls.cpp``), the timed CPU baseline.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: used by the tests, by
``__graft_entry__.build()`` (which compiles it) and by ``bench.py``'s CPU legs.  It is the same
CGLS on the same operator as ``wri_oracle.cgls`` (pinned against it in tests/), written as plain
OpenMP loops so that the CPU baseline uses every host core.
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpu_cgls.cpp")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libcpu_cgls.so")


def build() -> str:
    """Compile the shared library in-tree (g++, OpenMP) if it is missing or older than its source."""
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cxx = os.environ.get("CXX") or shutil.which("g++") or "g++"
    os.makedirs(BUILD, exist_ok=True)
    tmp = f"{LIB}.{os.getpid()}.tmp"
    r = subprocess.run([cxx, "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("g++ failed on the CPU oracle:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        dp, i32 = C.c_void_p, C.c_int
        lib.oracle_cgls.argtypes = [i32, i32, i32, i32, C.c_double, C.c_double, C.c_double, C.c_double, dp,
                                    C.c_longlong, i32, dp, i32, dp, dp, C.c_double, i32, C.c_double, i32, dp,
                                    C.POINTER(C.c_int), C.POINTER(C.c_double)]
        lib.oracle_cgls.restype = C.c_int
        lib.oracle_threads.restype = C.c_int
        _lib = lib
    return _lib


def threads() -> int:
    """Threads the OpenMP loops use (all cores of the process's affinity unless OMP_NUM_THREADS says)."""
    return int(_load().oracle_threads())


def cgls(shape, h, omega, m, npml, v_max, src, rec, d, lam, alpha=None, source_free=True, tol=0.0, max_iter=10,
         R=1e-3, nthreads=0):
    """x, iterations, relres of the CGLS solve of one system (see cpu_cgls.cpp); shape = (nz, ny, nx)."""
    nz, ny, nx = shape
    n = nx * ny * nz
    m = np.ascontiguousarray(m, dtype=np.float64).ravel()
    rec = np.ascontiguousarray(rec, dtype=np.int32)
    d = np.ascontiguousarray(np.asarray(d, dtype=np.complex128)).view(np.float64)
    al = None
    if not source_free:
        al = np.array([complex(alpha).real, complex(alpha).imag], dtype=np.float64)
    x = np.zeros(2 * n, dtype=np.float64)
    it = C.c_int(0)
    rr = C.c_double(0.0)
    rc = _load().oracle_cgls(nx, ny, nz, npml, h, omega, R, v_max, m.ctypes.data, int(src), int(bool(source_free)),
                             None if al is None else al.ctypes.data, len(rec), rec.ctypes.data if len(rec) else None,
                             d.ctypes.data if len(rec) else None, lam, int(max_iter), float(tol), int(nthreads),
                             x.ctypes.data, C.byref(it), C.byref(rr))
    if rc != 0:
        raise ValueError("oracle_cgls: invalid argument")
    return x.view(np.complex128), int(it.value), float(rr.value)
