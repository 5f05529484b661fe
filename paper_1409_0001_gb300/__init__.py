"""Python binding of the GB300 diffusion-based coarse-graining library (include/cg.h).

Argument marshalling only: every step of the method runs in the CUDA library
``libcgdiff.so``.  PyTorch supplies device memory and the stream.  There is no CPU
fallback: if the library is missing or no GPU is present, calls raise.

    import paper_1409_0001_gb300 as cg
    mesh = cg.StructuredMesh((128, 128, 128), (0, 0, 0), 1 / 128)
    eps = cg.coarse_grain(mesh, pos, w, cg.Params(bandwidth=2 / 128, nsteps=10))

Method (Section 2.6): particle centroid deposition, Eq. (pcm-k), then diffusion,
Eq. (diffusion), to pseudo-time T = b^2/4 with zero-flux walls.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = _build.LIB_PATH

SCHEME_IMPLICIT_EULER, SCHEME_CRANK_NICOLSON, SCHEME_EXPLICIT_EULER = 0, 1, 2
PREC_FP64, PREC_FP32_REFINE, PREC_BF16_REFINE, PREC_FP32_DF_REFINE, PREC_BF16_DF_REFINE = 0, 1, 2, 3, 4
DEPOSIT_ORDERED, DEPOSIT_FIXED_POINT = 0, 1
MAX_REPORT_FIELDS = 8

STATUS = {0: "CG_OK", 1: "CG_EINVAL", 2: "CG_ENOMEM", 3: "CG_ECUDA", 4: "CG_ENOCONV",
          5: "CG_ETIMEOUT", 6: "CG_EDOMAIN"}


class CgParams(ctypes.Structure):
    _fields_ = [("bandwidth", ctypes.c_double), ("T", ctypes.c_double), ("nsteps", ctypes.c_int),
                ("scheme", ctypes.c_int), ("precision", ctypes.c_int),
                ("deposit_mode", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("max_rounds", ctypes.c_int),
                ("fused_k", ctypes.c_int), ("sweep_shape", ctypes.c_int),
                ("barrier_budget", ctypes.c_longlong)]


class CgReport(ctypes.Structure):
    _fields_ = [("ms_locate", ctypes.c_double), ("ms_deposit", ctypes.c_double),
                ("ms_diffuse", ctypes.c_double), ("iters", ctypes.c_longlong),
                ("refine_rounds", ctypes.c_longlong), ("cell_updates", ctypes.c_longlong),
                ("final_rel_residual", ctypes.c_double),
                ("mass_in", ctypes.c_double * MAX_REPORT_FIELDS),
                ("mass_out", ctypes.c_double * MAX_REPORT_FIELDS),
                ("n_out_of_domain", ctypes.c_longlong),
                ("fixed_point_bits", ctypes.c_int * MAX_REPORT_FIELDS),
                ("inner_iters_per_round", ctypes.c_int), ("sweep_shape_used", ctypes.c_int)]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


class CGError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        self.code = STATUS.get(status, "CG_UNKNOWN")
        super().__init__("%s: %s (%s)" % (where, self.code, detail))


_lib = None


def load_library(path: str | None = None):
    """Load libcgdiff.so (built in-tree by build.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libcgdiff.so not found at %s: run paper_1409_0001_gb300.build.build() "
                           "(there is no CPU fallback)" % path)
    lib = ctypes.CDLL(path)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    P = ctypes.POINTER
    sigs = {
        "cg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "cg_last_error": (ctypes.c_char_p, []),
        "cg_params_default": (None, [P(CgParams)]),
        "cg_create_mesh_structured": (i32, [i32, i32, i32, P(dbl), dbl, P(vp)]),
        "cg_create_mesh_tet": (i32, [i64, vp, i64, vp, P(vp)]),
        "cg_destroy_mesh": (i32, [vp]),
        "cg_mesh_num_cells": (i64, [vp]),
        "cg_mesh_cell_volumes": (i32, [vp, vp]),
        "cg_mesh_tet_operator": (i32, [vp, vp, vp, vp, P(i64)]),
        "cg_locate": (i32, [vp, i64, vp, vp, P(i64), vp]),
        "cg_deposit": (i32, [vp, i64, vp, i32, vp, vp, P(CgParams), P(CgReport), vp]),
        "cg_diffuse": (i32, [vp, i32, vp, P(CgParams), P(CgReport), vp]),
        "cg_coarse_grain": (i32, [vp, i64, vp, i32, vp, vp, P(CgParams), P(CgReport), vp]),
        "cg_coarse_grain_host": (i32, [vp, i64, vp, i32, vp, vp, P(CgParams), P(CgReport), vp]),
        "cg_profile_enable": (i32, [i32]),
        "cg_profile_reset": (None, []),
        "cg_profile_count": (i32, []),
        "cg_profile_get": (i32, [i32, ctypes.c_char_p, i32, P(ctypes.c_longlong), P(dbl), P(dbl)]),
        "cg_launch_count": (ctypes.c_longlong, []),
        "cg_diffuse_batched": (i32, [i32, vp, i32, vp, P(CgParams), vp, P(CgReport), vp]),
        "cg_coarse_grain_batched": (i32, [i32, vp, vp, vp, i32, vp, vp, P(CgParams), vp,
                                          P(CgReport), vp]),
        "cg_deposit_fixed_noalloc": (i32, [i32, i32, i32, P(dbl), dbl, i64, vp, i32, vp, vp,
                                           P(ctypes.c_int), vp]),
        "cg_launch_count_reset": (None, []),
        "cg_mesh_set_periodic": (i32, [vp, i32, i32, i32]),
        "cg_create_mesh_hex": (i32, [i32, i32, i32, vp, vp, vp, vp, P(vp)]),
        "cg_solid_velocity": (i32, [vp, i32, vp, vp, dbl, vp, vp]),
        "cg_coarse_grain_concurrent": (i32, [i32, vp, vp, vp, i32, vp, vp, vp, vp, vp, i32]),
        "cg_set_workspace_limit": (i32, [ctypes.c_longlong]),
        "cg_workspace_bytes": (ctypes.c_longlong, []),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names the C header declares (used by the ABI test)."""
    return ["cg_status_string", "cg_last_error", "cg_params_default", "cg_create_mesh_structured",
            "cg_create_mesh_tet", "cg_destroy_mesh", "cg_mesh_num_cells", "cg_mesh_cell_volumes",
            "cg_mesh_tet_operator", "cg_locate", "cg_deposit", "cg_diffuse", "cg_coarse_grain",
            "cg_coarse_grain_host", "cg_profile_enable", "cg_profile_reset", "cg_profile_count",
            "cg_profile_get", "cg_launch_count", "cg_launch_count_reset",
            "cg_deposit_fixed_noalloc", "cg_diffuse_batched", "cg_coarse_grain_batched",
            "cg_mesh_set_periodic", "cg_solid_velocity", "cg_create_mesh_hex",
            "cg_coarse_grain_concurrent", "cg_set_workspace_limit", "cg_workspace_bytes"]


def set_workspace_limit(nbytes: int) -> None:
    """Cap the device bytes the library's workspaces may hold (0: no cap); a call that
    would exceed it raises CGError CG_ENOMEM before allocating (cg_set_workspace_limit)."""
    _check(load_library().cg_set_workspace_limit(int(nbytes)), "cg_set_workspace_limit")


def workspace_bytes() -> int:
    """Device bytes the library's workspaces hold now (cg_workspace_bytes)."""
    return int(load_library().cg_workspace_bytes())


def _check(status: int, where: str):
    if status != 0:
        detail = load_library().cg_last_error().decode(errors="replace")
        raise CGError(status, where, detail)


@dataclass
class Params:
    """Mirror of cg_params (see include/cg.h)."""
    bandwidth: float = 0.0
    T: float = 0.0
    nsteps: int = 10
    scheme: int = SCHEME_IMPLICIT_EULER
    precision: int = PREC_FP64
    deposit_mode: int = DEPOSIT_ORDERED
    tol: float = 1e-13
    max_iter: int = 10000
    max_rounds: int = 12
    fused_k: int = 0
    sweep_shape: int = 0
    barrier_budget: int = 0

    def to_c(self) -> CgParams:
        p = CgParams()
        load_library().cg_params_default(ctypes.byref(p))
        for k in ("bandwidth", "T", "nsteps", "scheme", "precision", "deposit_mode", "tol",
                  "max_iter", "max_rounds", "fused_k", "sweep_shape", "barrier_budget"):
            setattr(p, k, getattr(self, k))
        return p


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_f64(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError("%s must be a CUDA float64 tensor" % name)
    if not t.is_contiguous():
        raise TypeError("%s must be contiguous" % name)
    return t


class _MeshBase:
    _h = None

    @property
    def handle(self):
        return self._h

    @property
    def ncells(self) -> int:
        return int(load_library().cg_mesh_num_cells(self._h))

    def cell_volumes(self):
        import numpy as np
        out = np.empty(self.ncells, dtype=np.float64)
        _check(load_library().cg_mesh_cell_volumes(self._h, out.ctypes.data), "cg_mesh_cell_volumes")
        return out

    def close(self):
        if self._h:
            load_library().cg_destroy_mesh(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class StructuredMesh(_MeshBase):
    """Uniform Cartesian hex mesh (cg_create_mesh_structured); periodic = (px, py, pz)
    marks periodic axes (cg_mesh_set_periodic)."""

    def __init__(self, dims, origin, dx, periodic=(False, False, False)):
        lib = load_library()
        self.dims = tuple(int(d) for d in dims)
        self.origin = tuple(float(o) for o in origin)
        self.dx = float(dx)
        h = ctypes.c_void_p()
        org = (ctypes.c_double * 3)(*self.origin)
        _check(lib.cg_create_mesh_structured(self.dims[0], self.dims[1], self.dims[2], org, self.dx,
                                             ctypes.byref(h)), "cg_create_mesh_structured")
        self._h = h
        if any(periodic):
            self.set_periodic(*periodic)

    def set_periodic(self, px, py, pz):
        _check(load_library().cg_mesh_set_periodic(self.handle, int(bool(px)), int(bool(py)),
                                                   int(bool(pz))), "cg_mesh_set_periodic")


class HexMesh(_MeshBase):
    """Stretched Cartesian mesh with a cell diffusion constant (cg_create_mesh_hex):
    face coordinates xf, yf, zf (strictly increasing), diffusivity [ncells] or None."""

    def __init__(self, xf, yf, zf, diffusivity=None):
        import numpy as np
        lib = load_library()
        self.faces = tuple(np.ascontiguousarray(f, dtype=np.float64) for f in (xf, yf, zf))
        self.dims = tuple(len(f) - 1 for f in self.faces)
        self.diffusivity = None if diffusivity is None else np.ascontiguousarray(diffusivity,
                                                                                 dtype=np.float64)
        h = ctypes.c_void_p()
        _check(lib.cg_create_mesh_hex(self.dims[0], self.dims[1], self.dims[2],
                                      self.faces[0].ctypes.data, self.faces[1].ctypes.data,
                                      self.faces[2].ctypes.data,
                                      None if self.diffusivity is None else self.diffusivity.ctypes.data,
                                      ctypes.byref(h)), "cg_create_mesh_hex")
        self._h = h

    def operator(self):
        return TetMesh.operator(self)


class TetMesh(_MeshBase):
    """Unstructured tetrahedral mesh (cg_create_mesh_tet); xyz [nv,3] f64, tets [nt,4] i32."""

    def __init__(self, xyz, tets):
        import numpy as np
        lib = load_library()
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.tets = np.ascontiguousarray(tets, dtype=np.int32)
        h = ctypes.c_void_p()
        _check(lib.cg_create_mesh_tet(self.xyz.shape[0], self.xyz.ctypes.data, self.tets.shape[0],
                                      self.tets.ctypes.data, ctypes.byref(h)), "cg_create_mesh_tet")
        self._h = h

    def operator(self):
        import numpy as np
        lib = load_library()
        nnz = ctypes.c_int64()
        _check(lib.cg_mesh_tet_operator(self._h, None, None, None, ctypes.byref(nnz)), "operator")
        rp = np.empty(self.ncells + 1, dtype=np.int64)
        col = np.empty(nnz.value, dtype=np.int32)
        val = np.empty(nnz.value, dtype=np.float64)
        _check(lib.cg_mesh_tet_operator(self._h, rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                                        ctypes.byref(nnz)), "operator")
        return rp, col, val


def locate(mesh, pos, out=None, stream=None):
    """Host cell per particle (cg_locate).  pos: CUDA f64 [3, n].  Returns (cell i32, n_out)."""
    import torch
    _dev_f64(pos, "pos")
    n = pos.shape[1]
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=pos.device)
    nout = ctypes.c_int64()
    _check(load_library().cg_locate(mesh.handle, n, pos.data_ptr(), out.data_ptr(),
                                    ctypes.byref(nout), _stream_handle(stream)), "cg_locate")
    return out, int(nout.value)


def deposit(mesh, pos, w, params: Params | None = None, out=None, stream=None, report=False):
    """Particle centroid deposition, Eq. (pcm-k).  pos [3,n], w [nf,n] CUDA f64."""
    import torch
    params = params or Params()
    _dev_f64(pos, "pos")
    _dev_f64(w, "w")
    nf, n = w.shape
    if out is None:
        out = torch.empty((nf, mesh.ncells), dtype=torch.float64, device=w.device)
    rep = CgReport()
    cp = params.to_c()
    _check(load_library().cg_deposit(mesh.handle, n, pos.data_ptr(), nf, w.data_ptr(),
                                     out.data_ptr(), ctypes.byref(cp), ctypes.byref(rep),
                                     _stream_handle(stream)), "cg_deposit")
    return (out, rep.as_dict()) if report else out


def diffuse(mesh, cells, params: Params, stream=None, report=False):
    """Diffusion smoothing in place, Eq. (diffusion) to T.  cells [nf, ncells] CUDA f64."""
    _dev_f64(cells, "cells")
    nf = cells.shape[0] if cells.dim() == 2 else 1
    rep = CgReport()
    cp = params.to_c()
    _check(load_library().cg_diffuse(mesh.handle, nf, cells.data_ptr(), ctypes.byref(cp),
                                     ctypes.byref(rep), _stream_handle(stream)), "cg_diffuse")
    return (cells, rep.as_dict()) if report else cells


def coarse_grain(mesh, pos, w, params: Params, out=None, stream=None, report=False):
    """The whole method (Section 2.6): deposition then diffusion."""
    import torch
    _dev_f64(pos, "pos")
    _dev_f64(w, "w")
    nf, n = w.shape
    if out is None:
        out = torch.empty((nf, mesh.ncells), dtype=torch.float64, device=w.device)
    rep = CgReport()
    cp = params.to_c()
    _check(load_library().cg_coarse_grain(mesh.handle, n, pos.data_ptr(), nf, w.data_ptr(),
                                          out.data_ptr(), ctypes.byref(cp), ctypes.byref(rep),
                                          _stream_handle(stream)), "cg_coarse_grain")
    return (out, rep.as_dict()) if report else out


def solid_velocity(mesh, eps, mom, eps_min=0.0, out=None, stream=None):
    """Solid velocity (cg_solid_velocity): mom / eps per cell where eps > eps_min, else 0.
    eps: CUDA f64 [ncells]; mom: CUDA f64 [ncomp, ncells]; returns [ncomp, ncells]."""
    import torch
    _dev_f64(eps, "eps")
    _dev_f64(mom, "mom")
    if out is None:
        out = torch.empty_like(mom)
    _check(load_library().cg_solid_velocity(mesh.handle, mom.shape[0], eps.data_ptr(),
                                            mom.data_ptr(), float(eps_min), out.data_ptr(),
                                            _stream_handle(stream)), "cg_solid_velocity")
    return out


def coarse_grain_host(mesh, pos, w, params: Params, out=None, stream=None, report=False):
    """The whole method on HOST arrays (numpy or CPU tensors, f64, contiguous)."""
    import numpy as np
    pos = np.ascontiguousarray(pos, dtype=np.float64) if not hasattr(pos, "data_ptr") else pos
    w = np.ascontiguousarray(w, dtype=np.float64) if not hasattr(w, "data_ptr") else w
    nf, n = w.shape

    def ptr(a):
        return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data

    if out is None:
        out = np.empty((nf, mesh.ncells), dtype=np.float64)
    rep = CgReport()
    cp = params.to_c()
    _check(load_library().cg_coarse_grain_host(mesh.handle, n, ptr(pos), nf, ptr(w), ptr(out),
                                               ctypes.byref(cp), ctypes.byref(rep),
                                               _stream_handle(stream)), "cg_coarse_grain_host")
    return (out, rep.as_dict()) if report else out


def profile_enable(on: bool = True):
    """Per-kernel device timing (cg_profile_enable)."""
    load_library().cg_profile_enable(1 if on else 0)


def profile_reset():
    load_library().cg_profile_reset()


def profile_read() -> dict:
    """{kernel name: {"launches", "ms", "bytes"}} accumulated while profiling was on."""
    lib = load_library()
    out = {}
    for i in range(lib.cg_profile_count()):
        name = ctypes.create_string_buffer(64)
        n = ctypes.c_longlong()
        ms = ctypes.c_double()
        by = ctypes.c_double()
        _check(lib.cg_profile_get(i, name, 64, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)),
               "cg_profile_get")
        out[name.value.decode()] = {"launches": int(n.value), "ms": ms.value, "bytes": by.value}
    return out


NOALLOC_MAX_FIELDS = 8
NOALLOC_MAX_CELL_FIELDS = 2097152


def deposit_fixed_noalloc(dims, origin, dx, pos, w, out=None, stream=None):
    """Fixed-point deposition that allocates nothing inside the library
    (cg_deposit_fixed_noalloc); returns (cells [nf, ncells], F per field)."""
    import torch
    _dev_f64(pos, "pos")
    _dev_f64(w, "w")
    nf, n = w.shape
    ncells = int(dims[0]) * int(dims[1]) * int(dims[2])
    if out is None:
        out = torch.empty((nf, ncells), dtype=torch.float64, device=w.device)
    bits = (ctypes.c_int * max(nf, 1))()
    org = (ctypes.c_double * 3)(*[float(o) for o in origin])
    _check(load_library().cg_deposit_fixed_noalloc(int(dims[0]), int(dims[1]), int(dims[2]), org,
                                                   float(dx), n, pos.data_ptr(), nf, w.data_ptr(),
                                                   out.data_ptr(), bits, _stream_handle(stream)),
           "cg_deposit_fixed_noalloc")
    return out, list(bits)[:nf]


def _ptr_array(ptrs, ctype=ctypes.c_void_p):
    arr = (ctype * len(ptrs))()
    for i, v in enumerate(ptrs):
        arr[i] = v
    return arr


def diffuse_batched(meshes, cells, params: Params, bandwidths=None, stream=None, report=False):
    """Batched diffusion (cg_diffuse_batched): cells[s] is a CUDA f64 [nf, ncells_s] tensor."""
    import numpy as np
    for c in cells:
        _dev_f64(c, "cells")
    nf = cells[0].shape[0]
    ms = _ptr_array([m.handle.value for m in meshes])
    cs = _ptr_array([c.data_ptr() for c in cells])
    bw = None
    if bandwidths is not None:
        bw = np.ascontiguousarray(bandwidths, dtype=np.float64)
    rep = CgReport()
    cp = params.to_c()
    _check(load_library().cg_diffuse_batched(len(meshes), ms, nf, cs, ctypes.byref(cp),
                                             None if bw is None else bw.ctypes.data,
                                             ctypes.byref(rep), _stream_handle(stream)),
           "cg_diffuse_batched")
    return (cells, rep.as_dict()) if report else cells


def coarse_grain_batched(meshes, pos, w, params: Params, bandwidths=None, out=None, stream=None,
                         report=False):
    """The whole method for a batch (cg_coarse_grain_batched).  pos[s] [3, n_s] and w[s]
    [nf, n_s] CUDA f64 tensors; returns the list of cell tensors."""
    import numpy as np
    import torch
    nf = w[0].shape[0]
    for t in list(pos) + list(w):
        _dev_f64(t, "pos/w")
    if out is None:
        out = [torch.empty((nf, m.ncells), dtype=torch.float64, device=w[0].device) for m in meshes]
    ms = _ptr_array([m.handle.value for m in meshes])
    ns = _ptr_array([int(p_.shape[1]) for p_ in pos], ctypes.c_int64)
    ps = _ptr_array([p_.data_ptr() for p_ in pos])
    ws = _ptr_array([w_.data_ptr() for w_ in w])
    cs = _ptr_array([c.data_ptr() for c in out])
    bw = None if bandwidths is None else np.ascontiguousarray(bandwidths, dtype=np.float64)
    rep = CgReport()
    cp = params.to_c()
    _check(load_library().cg_coarse_grain_batched(len(meshes), ms, ns, ps, nf, ws, cs,
                                                  ctypes.byref(cp),
                                                  None if bw is None else bw.ctypes.data,
                                                  ctypes.byref(rep), _stream_handle(stream)),
           "cg_coarse_grain_batched")
    return (out, rep.as_dict()) if report else out


def coarse_grain_concurrent(meshes, pos, w, params, out=None, streams=None, max_concurrent=2,
                            report=False):
    """Independent coarse-grainings run concurrently (cg_coarse_grain_concurrent): problem
    i is coarse_grain(meshes[i], pos[i], w[i], params[i]) on streams[i] (one new stream per
    problem by default).  pos[i] [3, n_i] and w[i] [nf, n_i] are f64 tensors (they may be
    shared between problems): all CUDA tensors, or all host tensors (pinned for fast
    copies), in which case every problem copies its inputs in and its result out as
    coarse_grain_host does (problems given the same host tensors share one copy).  params is one Params or a list.  Returns the list of
    [nf, ncells_i] cell tensors (and the reports)."""
    import torch
    k = len(meshes)
    params = list(params) if isinstance(params, (list, tuple)) else [params] * k
    nf = w[0].shape[0]
    on_host = not w[0].is_cuda
    for t in list(pos) + list(w):
        if on_host:
            if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
                raise ValueError("pos/w: contiguous float64 host tensors expected")
        else:
            _dev_f64(t, "pos/w")
    if out is None:
        out = [torch.empty((nf, m.ncells), dtype=torch.float64, device=w[0].device,
                           pin_memory=on_host) for m in meshes]
    if streams is None:
        streams = [torch.cuda.Stream() for _ in range(k)]
    # the problems' streams start after the work already queued on the current stream
    cur = torch.cuda.current_stream()
    for s_ in streams:
        s_.wait_stream(cur)
    ms = _ptr_array([m.handle.value for m in meshes])
    ns = _ptr_array([int(p_.shape[1]) for p_ in pos], ctypes.c_int64)
    ps = _ptr_array([p_.data_ptr() for p_ in pos])
    ws = _ptr_array([w_.data_ptr() for w_ in w])
    cs = _ptr_array([c.data_ptr() for c in out])
    ss = _ptr_array([s_.cuda_stream for s_ in streams])
    cps = (CgParams * k)(*[p_.to_c() for p_ in params])
    reps = (CgReport * k)()
    _check(load_library().cg_coarse_grain_concurrent(k, ms, ns, ps, nf, ws, cs, cps, reps, ss,
                                                     int(max_concurrent)),
           "cg_coarse_grain_concurrent")
    for s_ in streams:   # later work on the current stream sees the results
        cur.wait_stream(s_)
    return (out, [r.as_dict() for r in reps]) if report else out
