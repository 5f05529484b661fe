"""The oracle spread over the host's cores (``cg_oracle_omp.c``, OpenMP).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: the benchmark's multi-core CPU
baseline and its per-workload error legs, and the tests that hold it to the
single-thread oracle.  The same definitions as ``cg_oracle.c`` (locate and deposition
give the same bits; the diffusion differs only in the order of the conjugate-gradient
dot products: fixed chunks, so the result does not depend on the thread count).

:func:`available` is False where the compiler has no OpenMP; nothing else in the
project needs this module.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cg_oracle_omp.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_err = None

_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_intp = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile cg_oracle_omp.c next to it (gcc -fopenmp); raises if that fails."""
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True, capture_output=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib, _err
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.omp_num_threads_used.restype = ctypes.c_int
        lib.omp_use_threads.restype = None
        lib.omp_use_threads.argtypes = [ctypes.c_int]
        lib.omp_locate_structured.restype = ctypes.c_int64
        lib.omp_locate_structured.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _f64p,
                                              ctypes.c_double, ctypes.c_int64, _f64p, _i32p]
        lib.omp_deposit.restype = None
        lib.omp_deposit.argtypes = [ctypes.c_int64, _i32p, ctypes.c_int, _f64p, ctypes.c_int64,
                                    _f64p, ctypes.c_double, ctypes.c_int, _intp, _f64p]
        lib.omp_diffuse_structured.restype = ctypes.c_int
        lib.omp_diffuse_structured.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_double, ctypes.c_int, _f64p,
                                               ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_double, ctypes.c_int, _i64p]
        lib.omp_diffuse_csr.restype = ctypes.c_int
        lib.omp_diffuse_csr.argtypes = [ctypes.c_int64, _f64p, _i64p, _i32p, _f64p, ctypes.c_int,
                                        _f64p, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_int, _i64p]
        lib.omp_locate_tet_bucketed.restype = ctypes.c_int64
        lib.omp_locate_tet_bucketed.argtypes = [ctypes.c_int64, _f64p, ctypes.c_int64, _i32p,
                                                ctypes.c_int64, _f64p, _i32p, ctypes.c_int]
        _lib = lib
        return lib


def available() -> bool:
    """Whether the OpenMP build compiles and loads here."""
    global _err
    try:
        _load()
        return True
    except (OSError, subprocess.CalledProcessError) as e:
        _err = str(e)
        return False


def threads() -> int:
    """Threads the parallel regions use (OMP_NUM_THREADS, else every core)."""
    return int(_load().omp_num_threads_used())


def use_threads(n: int) -> None:
    """Run the following calls on n threads."""
    _load().omp_use_threads(int(n))


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def locate_structured(dims, origin, dx, pos):
    nx, ny, nz = (int(d) for d in dims)
    pos = _f64(pos)
    n = pos.shape[1]
    cell = np.empty(n, dtype=np.int32)
    org = _f64(origin)
    out = _load().omp_locate_structured(nx, ny, nz, _p(org, ctypes.c_double), float(dx), n,
                                        _p(pos, ctypes.c_double), _p(cell, ctypes.c_int32))
    return cell, int(out)


def deposit(cell, w, ncells, vc=None, vc_uniform=1.0, mode=0, fbits=None):
    """mode 1 needs the scale exponents F per field (oracle.fixed_point_bits)."""
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    w = _f64(np.atleast_2d(w))
    nf, n = w.shape
    out = np.empty((nf, ncells), dtype=np.float64)
    fb = np.zeros(nf, dtype=np.intc) if fbits is None else np.ascontiguousarray(fbits, dtype=np.intc)
    vcp = None
    if vc is not None:
        vc = _f64(vc)
        vcp = _p(vc, ctypes.c_double)
    _load().omp_deposit(n, _p(cell, ctypes.c_int32), nf, _p(w, ctypes.c_double), int(ncells), vcp,
                        float(vc_uniform), int(mode), _p(fb, ctypes.c_int), _p(out, ctypes.c_double))
    return out


def diffuse_structured(u, dims, dx, T, nsteps, scheme=0, tol=1e-14, max_iter=100000):
    nx, ny, nz = (int(d) for d in dims)
    squeeze = np.ndim(u) == 1
    u = np.array(np.atleast_2d(u), dtype=np.float64, order="C", copy=True)
    iters = ctypes.c_int64(0)
    st = _load().omp_diffuse_structured(nx, ny, nz, float(dx), u.shape[0], _p(u, ctypes.c_double),
                                        float(T), int(nsteps), int(scheme), float(tol),
                                        int(max_iter), ctypes.byref(iters))
    if st != 0:
        raise RuntimeError("multi-core oracle CG did not converge (status %d)" % st)
    return (u[0] if squeeze else u), int(iters.value)


def diffuse_csr(u, vc, rowptr, col, val, T, nsteps, scheme=0, tol=1e-14, max_iter=100000):
    squeeze = np.ndim(u) == 1
    u = np.array(np.atleast_2d(u), dtype=np.float64, order="C", copy=True)
    vc = _f64(vc)
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = _f64(val)
    iters = ctypes.c_int64(0)
    st = _load().omp_diffuse_csr(vc.shape[0], _p(vc, ctypes.c_double), _p(rowptr, ctypes.c_int64),
                                 _p(col, ctypes.c_int32), _p(val, ctypes.c_double), u.shape[0],
                                 _p(u, ctypes.c_double), float(T), int(nsteps), int(scheme),
                                 float(tol), int(max_iter), ctypes.byref(iters))
    if st != 0:
        raise RuntimeError("multi-core oracle CG did not converge (status %d)" % st)
    return (u[0] if squeeze else u), int(iters.value)


def locate_tet_bucketed(xyz, tets, pos, nb=None):
    xyz = _f64(xyz)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    pos = _f64(pos)
    n = pos.shape[1]
    if nb is None:
        nb = max(1, int(round((tets.shape[0] / 6.0) ** (1.0 / 3.0))))
    cell = np.empty(n, dtype=np.int32)
    out = _load().omp_locate_tet_bucketed(xyz.shape[0], _p(xyz, ctypes.c_double), tets.shape[0],
                                          _p(tets, ctypes.c_int32), n, _p(pos, ctypes.c_double),
                                          _p(cell, ctypes.c_int32), int(nb))
    return cell, int(out)
