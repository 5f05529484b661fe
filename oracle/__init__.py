"""FP64 CPU oracle for diffusion-based coarse graining (Sun & Xiao).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of
the benchmark use it; the CUDA library never does.  The arithmetic lives in
``cg_oracle.c`` (plain C, compiled with ``-ffp-contract=off``); this module only
builds it and marshals numpy arrays.  It shares no code with the CUDA path.

Functions follow the paper's steps:

* :func:`locate_structured`, :func:`locate_tet` -- host cell of each particle
  centroid (Section 2.2, Section 3.1).
* :func:`deposit` -- particle centroid method, Eq. (pcm-k).
* :func:`diffuse_structured`, :func:`diffuse_csr` -- pseudo-time integration of
  Eq. (diffusion) to T = b^2/4 with zero-flux walls (Section 2.6 step 2,
  Section 3.2), implicit Euler / Crank-Nicolson (Section 5.1) / explicit Euler.
* :func:`tet_build` -- two-point-flux finite-volume Laplacian on tetrahedra.
* :func:`kernel_sum` -- brute-force Gaussian kernel with wall images,
  Eq. (hi), Eq. (hi-bound), Eq. (diffHalf).
* :func:`coarse_grain_structured` -- the whole method (Section 2.6).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_intp = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile cg_oracle.c into a shared library next to it (plain gcc)."""
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.orc_locate_structured.restype = ctypes.c_int64
        lib.orc_locate_structured.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _f64p,
                                              ctypes.c_double, ctypes.c_int64, _f64p, _i32p]
        lib.orc_fixed_point_bits.restype = ctypes.c_int
        lib.orc_fixed_point_bits.argtypes = [ctypes.c_int64, ctypes.c_double]
        lib.orc_deposit.restype = None
        lib.orc_deposit.argtypes = [ctypes.c_int64, _i32p, ctypes.c_int, _f64p, ctypes.c_int64,
                                    _f64p, ctypes.c_double, ctypes.c_int, _intp, _f64p]
        lib.orc_diffuse_structured.restype = ctypes.c_int
        lib.orc_diffuse_structured.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_double, ctypes.c_int, _f64p,
                                               ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_double, ctypes.c_int, _i64p]
        lib.orc_diffuse_structured_p.restype = ctypes.c_int
        lib.orc_diffuse_structured_p.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                                 _f64p, ctypes.c_double, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                                 _i64p]
        lib.orc_solid_velocity.restype = None
        lib.orc_solid_velocity.argtypes = [ctypes.c_int64, ctypes.c_int, _f64p, _f64p,
                                           ctypes.c_double, _f64p]
        lib.orc_hex_build.restype = ctypes.c_int64
        lib.orc_hex_build.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _f64p, _f64p,
                                      _f64p, _f64p, _f64p, _i64p, _i32p, _f64p]
        lib.orc_locate_hex.restype = ctypes.c_int64
        lib.orc_locate_hex.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _f64p, _f64p,
                                       _f64p, ctypes.c_int64, _f64p, _i32p]
        lib.orc_tet_build.restype = ctypes.c_int64
        lib.orc_tet_build.argtypes = [ctypes.c_int64, _f64p, ctypes.c_int64, _i32p, _f64p, _f64p,
                                      _i64p, _i32p, _f64p]
        lib.orc_diffuse_csr.restype = ctypes.c_int
        lib.orc_diffuse_csr.argtypes = [ctypes.c_int64, _f64p, _i64p, _i32p, _f64p, ctypes.c_int,
                                        _f64p, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_int, _i64p]
        lib.orc_tet_min_bary.restype = ctypes.c_double
        lib.orc_tet_min_bary.argtypes = [_f64p, _i32p, ctypes.c_int64, _f64p]
        lib.orc_locate_tet.restype = ctypes.c_int64
        lib.orc_locate_tet.argtypes = [ctypes.c_int64, _f64p, ctypes.c_int64, _i32p,
                                       ctypes.c_int64, _f64p, _i32p]
        lib.orc_locate_tet_bucketed.restype = ctypes.c_int64
        lib.orc_locate_tet_bucketed.argtypes = [ctypes.c_int64, _f64p, ctypes.c_int64, _i32p,
                                                ctypes.c_int64, _f64p, _i32p, ctypes.c_int]
        lib.orc_kernel_sum.restype = None
        lib.orc_kernel_sum.argtypes = [ctypes.c_int64, _f64p, _f64p, ctypes.c_int64, _f64p, _f64p,
                                       ctypes.c_double, ctypes.c_int, _f64p]
        _lib = lib
        return lib


def _p(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def bandwidth_to_time(b: float) -> float:
    """Pseudo-time of the diffusion equivalent to a Gaussian kernel of bandwidth b:
    b = sqrt(4 T) (Section 3.2.1), i.e. T = b^2 / 4."""
    return b * b / 4.0


# ----------------------------------------------------------------------------- locate
def locate_structured(dims, origin, dx, pos):
    """Host cell of each particle centroid on a uniform mesh (Section 3.1).

    pos is [3, n] FP64.  Returns (cell int32 [n], number out of domain); a particle
    outside the closed box gets cell -1."""
    nx, ny, nz = (int(d) for d in dims)
    pos = _f64(pos)
    n = pos.shape[1]
    cell = np.empty(n, dtype=np.int32)
    org = _f64(origin)
    out = _load().orc_locate_structured(nx, ny, nz, _p(org, ctypes.c_double), float(dx), n,
                                        _p(pos, ctypes.c_double), _p(cell, ctypes.c_int32))
    return cell, int(out)


def locate_tet(xyz, tets, pos):
    """Host tetrahedron of each particle centroid, by brute force over all tets
    (rule in cg_oracle.c).  Returns (cell int32 [n], number out of domain)."""
    xyz = _f64(xyz)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    pos = _f64(pos)
    n = pos.shape[1]
    cell = np.empty(n, dtype=np.int32)
    out = _load().orc_locate_tet(xyz.shape[0], _p(xyz, ctypes.c_double), tets.shape[0],
                                 _p(tets, ctypes.c_int32), n, _p(pos, ctypes.c_double),
                                 _p(cell, ctypes.c_int32))
    return cell, int(out)


def locate_tet_bucketed(xyz, tets, pos, nb=None):
    """The rule of locate_tet, searching only the tets listed in the point's bucket of a
    uniform nb^3 grid over the mesh's box (every tet whose box holds the point is listed
    there), for meshes too large for the brute force.  nb defaults to round((ntets/6)^(1/3))."""
    xyz = _f64(xyz)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    pos = _f64(pos)
    n = pos.shape[1]
    if nb is None:
        nb = max(1, int(round((tets.shape[0] / 6.0) ** (1.0 / 3.0))))
    cell = np.empty(n, dtype=np.int32)
    out = _load().orc_locate_tet_bucketed(xyz.shape[0], _p(xyz, ctypes.c_double), tets.shape[0],
                                          _p(tets, ctypes.c_int32), n, _p(pos, ctypes.c_double),
                                          _p(cell, ctypes.c_int32), int(nb))
    return cell, int(out)


def tet_min_bary(xyz, tets, t, x):
    xyz = _f64(xyz)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    x = _f64(x)
    return _load().orc_tet_min_bary(_p(xyz, ctypes.c_double), _p(tets, ctypes.c_int32), int(t),
                                    _p(x, ctypes.c_double))


# ----------------------------------------------------------------------------- deposit
def fixed_point_bits(n: int, maxabs: float) -> int:
    """Scale exponent F of the 64-bit fixed-point deposition (see cg_oracle.c)."""
    return int(_load().orc_fixed_point_bits(int(n), float(maxabs)))


def deposit(cell, w, ncells, vc=None, vc_uniform=1.0, mode=0):
    """Particle centroid method, Eq. (pcm-k).  w is [nf, n]; returns (eps [nf, ncells],
    fbits list).  mode 0 sums in ascending particle index; mode 1 is 64-bit fixed point."""
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    w = _f64(np.atleast_2d(w))
    nf, n = w.shape
    out = np.empty((nf, ncells), dtype=np.float64)
    fbits = np.zeros(nf, dtype=np.intc)
    if mode == 1:
        for f in range(nf):
            m = float(np.max(np.abs(w[f]))) if n else 0.0
            fbits[f] = fixed_point_bits(n, m)
    vcp = None
    if vc is not None:
        vc = _f64(vc)
        vcp = _p(vc, ctypes.c_double)
    _load().orc_deposit(n, _p(cell, ctypes.c_int32), nf, _p(w, ctypes.c_double), int(ncells), vcp,
                        float(vc_uniform), int(mode), _p(fbits, ctypes.c_int),
                        _p(out, ctypes.c_double))
    return out, [int(x) for x in fbits]


# ----------------------------------------------------------------------------- diffuse
def diffuse_structured(u, dims, dx, T, nsteps, scheme=0, tol=1e-14, max_iter=100000,
                       periodic=(False, False, False)):
    """Pseudo-time integration of Eq. (diffusion) on a uniform mesh with zero-flux walls
    (or periodic axes where periodic[a] is set, Section 3.1).  u is [nf, ncells] (or
    [ncells]); returns (u(T), total CG iterations)."""
    nx, ny, nz = (int(d) for d in dims)
    per = sum(1 << a for a in range(3) if periodic[a])
    squeeze = np.ndim(u) == 1
    u = np.array(np.atleast_2d(u), dtype=np.float64, order="C", copy=True)
    iters = ctypes.c_int64(0)
    st = _load().orc_diffuse_structured_p(nx, ny, nz, per, float(dx), u.shape[0],
                                          _p(u, ctypes.c_double), float(T), int(nsteps),
                                          int(scheme), float(tol), int(max_iter),
                                          ctypes.byref(iters))
    if st != 0:
        raise RuntimeError("oracle CG did not converge")
    return (u[0] if squeeze else u), int(iters.value)


def tet_build(xyz, tets):
    """Cell volumes, centroids and the CSR two-point-flux Laplacian of a tet mesh."""
    xyz = _f64(xyz)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    nt = tets.shape[0]
    vc = np.empty(nt)
    cent = np.empty((nt, 3))
    rowptr = np.empty(nt + 1, dtype=np.int64)
    col = np.empty(5 * nt, dtype=np.int32)
    val = np.empty(5 * nt)
    nnz = _load().orc_tet_build(xyz.shape[0], _p(xyz, ctypes.c_double), nt,
                                _p(tets, ctypes.c_int32), _p(vc, ctypes.c_double),
                                _p(cent, ctypes.c_double), _p(rowptr, ctypes.c_int64),
                                _p(col, ctypes.c_int32), _p(val, ctypes.c_double))
    if nnz < 0:
        raise ValueError("invalid tet mesh (code %d)" % nnz)
    return vc, cent, rowptr, col[:nnz].copy(), val[:nnz].copy()


def diffuse_csr(u, vc, rowptr, col, val, T, nsteps, scheme=0, tol=1e-14, max_iter=100000):
    """Pseudo-time integration on a general cell-centred mesh: M = diag(vc), L in CSR."""
    squeeze = np.ndim(u) == 1
    u = np.array(np.atleast_2d(u), dtype=np.float64, order="C", copy=True)
    vc = _f64(vc)
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = _f64(val)
    iters = ctypes.c_int64(0)
    st = _load().orc_diffuse_csr(vc.shape[0], _p(vc, ctypes.c_double), _p(rowptr, ctypes.c_int64),
                                 _p(col, ctypes.c_int32), _p(val, ctypes.c_double), u.shape[0],
                                 _p(u, ctypes.c_double), float(T), int(nsteps), int(scheme),
                                 float(tol), int(max_iter), ctypes.byref(iters))
    if st != 0:
        raise RuntimeError("oracle CG did not converge")
    return (u[0] if squeeze else u), int(iters.value)


def kernel_sum(src, w, evals, L, b, mmax=2):
    """Brute-force Gaussian kernel of bandwidth b with wall images (box [0,L])."""
    src = _f64(src).reshape(-1, 3)
    w = _f64(w)
    evals = _f64(evals).reshape(-1, 3)
    Lv = _f64(L)
    out = np.empty(evals.shape[0])
    _load().orc_kernel_sum(src.shape[0], _p(src, ctypes.c_double), _p(w, ctypes.c_double),
                           evals.shape[0], _p(evals, ctypes.c_double), _p(Lv, ctypes.c_double),
                           float(b), int(mmax), _p(out, ctypes.c_double))
    return out


# ----------------------------------------------------------------------------- whole method
def coarse_grain_structured(dims, origin, dx, pos, w, b, nsteps, scheme=0, mode=0, tol=1e-14):
    """Section 2.6: PCM deposition (step 1) then diffusion to T = b^2/4 (step 2).
    Returns (eps0 [nf, ncells], eps(T) [nf, ncells], n_out_of_domain, cg iterations)."""
    nx, ny, nz = (int(d) for d in dims)
    cell, nout = locate_structured(dims, origin, dx, pos)
    vcu = (dx * dx) * dx
    eps0, _ = deposit(cell, w, nx * ny * nz, vc_uniform=vcu, mode=mode)
    epsT, iters = diffuse_structured(eps0, dims, dx, bandwidth_to_time(b), nsteps, scheme, tol)
    return eps0, epsT, nout, iters


def solid_velocity(eps, mom, eps_min=0.0):
    """Solid velocity as diffused momentum over diffused solid fraction (conclusions of
    the paper: momentum, not velocity, is diffused); 0 where eps <= eps_min.  eps is
    [ncells], mom [ncomp, ncells]."""
    eps = _f64(eps)
    mom = np.array(np.atleast_2d(mom), dtype=np.float64, order="C")
    out = np.empty_like(mom)
    _load().orc_solid_velocity(eps.shape[0], mom.shape[0], _p(eps, ctypes.c_double),
                               _p(mom, ctypes.c_double), float(eps_min), _p(out, ctypes.c_double))
    return out


def hex_build(xf, yf, zf, D=None):
    """Cell volumes and the CSR two-point-flux Laplacian of a stretched Cartesian mesh
    with face coordinates xf, yf, zf and a cell diffusion constant D (default 1; the face
    value is the harmonic mean).  Returns (vc, rowptr, col, val)."""
    xf, yf, zf = _f64(xf), _f64(yf), _f64(zf)
    nx, ny, nz = len(xf) - 1, len(yf) - 1, len(zf) - 1
    n = nx * ny * nz
    d = None if D is None else _f64(D)
    vc = np.empty(n)
    rowptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(7 * n, dtype=np.int32)
    val = np.empty(7 * n)
    nnz = _load().orc_hex_build(nx, ny, nz, _p(xf, ctypes.c_double), _p(yf, ctypes.c_double),
                                _p(zf, ctypes.c_double),
                                None if d is None else _p(d, ctypes.c_double),
                                _p(vc, ctypes.c_double), _p(rowptr, ctypes.c_int64),
                                _p(col, ctypes.c_int32), _p(val, ctypes.c_double))
    return vc, rowptr, col[:nnz].copy(), val[:nnz].copy()


def locate_hex(xf, yf, zf, pos):
    """Cell of each point on a stretched Cartesian mesh (-1 outside); returns (cell, nout)."""
    xf, yf, zf = _f64(xf), _f64(yf), _f64(zf)
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = pos.shape[1]
    cell = np.empty(n, dtype=np.int32)
    nout = _load().orc_locate_hex(len(xf) - 1, len(yf) - 1, len(zf) - 1, _p(xf, ctypes.c_double),
                                  _p(yf, ctypes.c_double), _p(zf, ctypes.c_double), n,
                                  _p(pos, ctypes.c_double), _p(cell, ctypes.c_int32))
    return cell, int(nout)
