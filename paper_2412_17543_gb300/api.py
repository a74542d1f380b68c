"""Python binding of the GB300 DD solver: marshals torch tensors to the C ABI.

Every numerical step runs in the native library (libdd_gb300.so); this module only
passes device pointers, sizes and the current CUDA stream, and owns the handles.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as nat


def _mesh_desc(mesh, keep: list) -> nat.MeshDesc:
    """MeshDesc from an object with nx, ny, nz, xc, yc, zc, sub, dirichlet, coef (host arrays)."""
    def dptr(a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        keep.append(a)
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d = nat.MeshDesc()
    d.nx, d.ny, d.nz = int(mesh.nx), int(mesh.ny), int(mesh.nz)
    d.xc, d.yc, d.zc = dptr(mesh.xc), dptr(mesh.yc), dptr(mesh.zc)
    d.coef = dptr(np.asarray(mesh.coef).ravel()) if getattr(mesh, "coef", None) is not None else None
    d.sub_x, d.sub_y, d.sub_z = (int(v) for v in mesh.sub)
    d.dirichlet_faces = int(mesh.dirichlet)
    return d


def make_options(**kw) -> nat.Options:
    """dd_options from keyword arguments (names as in the C struct; weights/precisions by name)."""
    lib = nat.load()
    o = nat.Options()
    nat.check(lib.dd_default_options(ctypes.byref(o)), "dd_default_options")
    for k, v in kw.items():
        if k == "weights" and isinstance(v, str):
            v = nat.WEIGHTS[v]
        if k in ("precond_prec", "schur_prec") and isinstance(v, str):
            v = nat.PREC[v]
        if not hasattr(o, k):
            raise KeyError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def plan(mesh, **opts):
    """Host-only setup (no GPU): returns (info dict, interface free-node indices)."""
    lib = nat.load()
    keep = []
    d = _mesh_desc(mesh, keep)
    o = make_options(**opts)
    info = nat.Info()
    nat.check(lib.dd_plan(ctypes.byref(d), ctypes.byref(o), ctypes.byref(info), None, 0), "dd_plan")
    nodes = np.empty(info.n_gamma, dtype=np.int64)
    nat.check(lib.dd_plan(ctypes.byref(d), ctypes.byref(o), ctypes.byref(info),
                          nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), nodes.size), "dd_plan")
    return _info_dict(info), nodes


def _info_dict(info) -> dict:
    return {f: getattr(info, f) for f, _ in nat.Info._fields_}


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """A set-up DD/BDDC solver for one matrix (dd_setup / dd_destroy)."""

    def __init__(self, mesh, **opts):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the DD solver needs a CUDA device")
        self.lib = nat.load()
        keep = []
        d = _mesh_desc(mesh, keep)
        self.options = make_options(**opts)
        h = ctypes.c_void_p()
        nat.check(self.lib.dd_setup(ctypes.byref(d), ctypes.byref(self.options), _stream_ptr(), ctypes.byref(h)),
                  "dd_setup")
        self.handle = h
        info = nat.Info()
        nat.check(self.lib.dd_get_info(self.handle, ctypes.byref(info)), "dd_get_info")
        self.info = _info_dict(info)
        self.n_free = int(info.n_free)
        self.n_gamma = int(info.n_gamma)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.dd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def interface_nodes(self) -> np.ndarray:
        out = np.empty(self.n_gamma, dtype=np.int64)
        nat.check(self.lib.dd_interface_nodes(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
                  "dd_interface_nodes")
        return out

    def _vec(self, n, like):
        import torch
        return torch.empty(n, dtype=torch.float64, device=like.device)

    def schur_apply(self, x, out=None):
        y = out if out is not None else self._vec(self.n_gamma, x)
        nat.check(self.lib.dd_schur_apply(self.handle, _dptr(x), _dptr(y), _stream_ptr()), "dd_schur_apply")
        return y

    def precond_apply(self, r, out=None):
        z = out if out is not None else self._vec(self.n_gamma, r)
        nat.check(self.lib.dd_precond_apply(self.handle, _dptr(r), _dptr(z), _stream_ptr()), "dd_precond_apply")
        return z

    def condense(self, f, out=None):
        b = out if out is not None else self._vec(self.n_gamma, f)
        nat.check(self.lib.dd_condense(self.handle, _dptr(f), _dptr(b), _stream_ptr()), "dd_condense")
        return b

    def recover(self, f, xg, out=None):
        x = out if out is not None else self._vec(self.n_free, f)
        nat.check(self.lib.dd_recover(self.handle, _dptr(f), _dptr(xg), _dptr(x), _stream_ptr()), "dd_recover")
        return x

    def profile(self, enable: bool, read: bool = True):
        """Starts/stops kernel timing; returns ({class: (ms, launches, alg_bytes)}, kernel launches) if read."""
        if not read:
            nat.check(self.lib.dd_profile(self.handle, int(enable), None, None, _stream_ptr()), "dd_profile")
            return None
        prof = (nat.KernelProf * len(nat.PROF_CLASSES))()
        nl = ctypes.c_int64()
        nat.check(self.lib.dd_profile(self.handle, int(enable), prof, ctypes.byref(nl), _stream_ptr()), "dd_profile")
        out = {name: (prof[i].ms, prof[i].launches, prof[i].alg_bytes) for i, name in enumerate(nat.PROF_CLASSES)}
        return out, nl.value

    def recycler(self, k=0, strategy="B4", freeze_tol=1e-5) -> "Recycler":
        return Recycler(self, k, strategy, freeze_tol)

    def solve(self, f, rec: "Recycler", rtol=1e-8, out=None, allow_not_converged=False):
        """x = K^{-1} f (device float64 [n_free]); returns (x, stats dict)."""
        x = out if out is not None else self._vec(self.n_free, f)
        st = nat.Stats()
        allow = (nat.DD_OK, nat.DD_NOT_CONVERGED) if allow_not_converged else (nat.DD_OK,)
        code = nat.check(self.lib.dd_solve(self.handle, _dptr(f), _dptr(x), ctypes.c_double(rtol), rec.handle,
                                           ctypes.byref(st), _stream_ptr()), "dd_solve", allow)
        stats = {f: getattr(st, f) for f, _ in nat.Stats._fields_}
        stats["status"] = nat.STATUS_NAMES[code]
        return x, stats


class Recycler:
    """Recycle state of a sequence of solves (dd_recycle_create / dd_recycle_destroy)."""

    def __init__(self, solver: Solver, k=0, strategy="B4", freeze_tol=1e-5):
        self.solver = solver
        h = ctypes.c_void_p()
        nat.check(solver.lib.dd_recycle_create(solver.handle, int(k), nat.STRATEGY[strategy],
                                               ctypes.c_double(freeze_tol), ctypes.byref(h)), "dd_recycle_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self.solver.lib.dd_recycle_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
