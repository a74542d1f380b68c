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
        if k == "local_solver" and isinstance(v, str):
            v = nat.LOCAL[v]
        if k == "ens_nmm" and isinstance(v, str):
            v = nat.ENS_NMM[v]
        if k == "adaptive_solver" and isinstance(v, str):
            v = nat.EIG[v]
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
        info = self.info
        self.n_free = int(info["n_free"])
        self.n_gamma = int(info["n_gamma"])
        self.n_elem = int(mesh.nx) * int(mesh.ny) * int(mesh.nz)

    @property
    def info(self) -> dict:
        """dd_get_info of the context (current: includes the ensemble kernel once selected)."""
        info = nat.Info()
        nat.check(self.lib.dd_get_info(self.handle, ctypes.byref(info)), "dd_get_info")
        d = _info_dict(info)
        for f in ("ens_nmm_ms", "tune_symv_ms", "tune_kii_ms", "tune_schur_ms"):
            d[f] = list(getattr(info, f))
        return d

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
        """Starts/stops kernel timing; returns ({class: (ms, launches, alg_bytes, alg_flops)}, kernel launches)
        if read."""
        if not read:
            nat.check(self.lib.dd_profile(self.handle, int(enable), None, None, _stream_ptr()), "dd_profile")
            return None
        prof = (nat.KernelProf * len(nat.PROF_CLASSES))()
        nl = ctypes.c_int64()
        nat.check(self.lib.dd_profile(self.handle, int(enable), prof, ctypes.byref(nl), _stream_ptr()), "dd_profile")
        out = {name: (prof[i].ms, prof[i].launches, prof[i].alg_bytes, prof[i].alg_flops)
               for i, name in enumerate(nat.PROF_CLASSES)}
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


    def ensemble_recycler(self, k=0, strategy="B4", freeze_tol=1e-5) -> "Recycler":
        """Recycle state for ensemble solves (dd_recycle_create_batch)."""
        return Recycler(self, k, strategy, freeze_tol, ensemble=True)

    def schur_apply_batch(self, X, out=None):
        """Y[m] = A X[m] for interface vectors X (device float64 [nrhs][n_gamma])."""
        Y = out if out is not None else X.new_empty(X.shape)
        nat.check(self.lib.dd_schur_apply_batch(self.handle, int(X.shape[0]), _dptr(X), _dptr(Y), _stream_ptr()),
                  "dd_schur_apply_batch")
        return Y

    def precond_apply_batch(self, R, out=None):
        """Z[m] = M^{-1} R[m] (BDDC) for interface vectors R (device float64 [nrhs][n_gamma])."""
        Z = out if out is not None else R.new_empty(R.shape)
        nat.check(self.lib.dd_precond_apply_batch(self.handle, int(R.shape[0]), _dptr(R), _dptr(Z), _stream_ptr()),
                  "dd_precond_apply_batch")
        return Z

    def solve_batch(self, F, rec: "Recycler", rtol=1e-8, out=None, allow_not_converged=False):
        """X[m] = K^{-1} F[m] for an ensemble F (device float64 [nrhs][n_free], nrhs <= 32);
        returns (X, list of per-member stats dicts)."""
        nrhs = int(F.shape[0])
        X = out if out is not None else F.new_empty(F.shape)
        st = (nat.Stats * nrhs)()
        allow = (nat.DD_OK, nat.DD_NOT_CONVERGED) if allow_not_converged else (nat.DD_OK,)
        code = nat.check(self.lib.dd_solve_batch(self.handle, nrhs, _dptr(F), _dptr(X), ctypes.c_double(rtol),
                                                 rec.handle, st, _stream_ptr()), "dd_solve_batch", allow)
        stats = []
        for m in range(nrhs):
            d = {f: getattr(st[m], f) for f, _ in nat.Stats._fields_}
            d["status"] = nat.STATUS_NAMES[code]
            stats.append(d)
        return X, stats

    def adjoint(self, grad_x, x=None, rec: "Recycler" = None, rtol=1e-10, coef_grad=True, log_coef=False):
        """lambda = K^{-1} grad_x (K symmetric); returns (dL/df = lambda, dL/dk per element or None, stats).
        With log_coef the coefficient gradient is taken with respect to g = log k (computed in the
        library). rec (optional) deflates the adjoint solve with its basis, which is not updated."""
        import torch
        gf = self._vec(self.n_free, grad_x)
        gk = None
        if coef_grad:
            if x is None:
                raise ValueError("the coefficient gradient needs the forward solution x")
            gk = torch.empty(self.n_elem, dtype=torch.float64, device=grad_x.device)
        st = nat.Stats()
        nat.check(self.lib.dd_adjoint(self.handle, _dptr(grad_x), _dptr(x) if x is not None else None, _dptr(gf),
                                      _dptr(gk) if gk is not None else None, int(bool(log_coef)),
                                      ctypes.c_double(rtol), rec.handle if rec is not None else None,
                                      ctypes.byref(st), _stream_ptr()), "dd_adjoint")
        return gf, gk, {f: getattr(st, f) for f, _ in nat.Stats._fields_}

    def coef_mismatch(self, coef, log=False) -> float:
        """max_e |k_e - c_e| / |k_e| between the set-up coefficients and coef (exp(coef) if log)."""
        out = ctypes.c_double()
        nat.check(self.lib.dd_coef_mismatch(self.handle, _dptr(coef.reshape(-1)), int(bool(log)), ctypes.byref(out),
                                            _stream_ptr()), "dd_coef_mismatch")
        return out.value


class PoissonSolve:
    """x = K(k)^{-1} f as a differentiable operation (torch.autograd.Function).

    forward(f, g): solves with the set-up solver, whose coefficient field must be k = exp(g)
    (checked in the library: a field that differs by more than 1e-12 relative raises,
    since the solver's operator is fixed at setup); backward: the adjoint solve with the same
    operator, preconditioner and deflation basis returns dL/df = lambda and
    dL/dg_e = k_e * (-lambda_e^T K_e^0 x_e), both computed by the library.
    """

    COEF_TOL = 1e-12

    @staticmethod
    def apply(f, g, solver: "Solver", rec: "Recycler", rtol: float = 1e-10, adjoint_rtol: float = 1e-10):
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, f_, g_):
                gd = g_.detach().contiguous()
                diff = solver.coef_mismatch(gd, log=True)
                if not diff <= PoissonSolve.COEF_TOL:
                    raise ValueError(f"PoissonSolve: exp(g) differs from the solver's coefficients by {diff:.3e} "
                                     "(relative); set up a solver for this field")
                x, _ = solver.solve(f_.detach().contiguous(), rec, rtol)
                ctx.save_for_backward(x)
                ctx.g_shape = g_.shape
                return x

            @staticmethod
            def backward(ctx, grad_x):
                (x,) = ctx.saved_tensors
                gf, gg, _ = solver.adjoint(grad_x.contiguous(), x, rec, adjoint_rtol,
                                           coef_grad=ctx.needs_input_grad[1], log_coef=True)
                return gf, (gg.reshape(ctx.g_shape) if gg is not None else None)

        return _Fn.apply(f, g)


class Recycler:
    """Recycle state of a sequence of solves (dd_recycle_create / dd_recycle_destroy)."""

    def __init__(self, solver: Solver, k=0, strategy="B4", freeze_tol=1e-5, ensemble=False):
        self.solver = solver
        h = ctypes.c_void_p()
        fn = "dd_recycle_create_batch" if ensemble else "dd_recycle_create"
        nat.check(getattr(solver.lib, fn)(solver.handle, int(k), nat.STRATEGY[strategy], ctypes.c_double(freeze_tol),
                                          ctypes.byref(h)), fn)
        self.handle = h

    def export(self) -> bytes:
        """Checkpoint of the recycle state (host bytes)."""
        lib = self.solver.lib
        n = ctypes.c_size_t(0)
        nat.check(lib.dd_recycle_export(self.handle, None, ctypes.byref(n)), "dd_recycle_export")
        buf = ctypes.create_string_buffer(n.value)
        nat.check(lib.dd_recycle_export(self.handle, buf, ctypes.byref(n)), "dd_recycle_export")
        return buf.raw[: n.value]

    def state(self) -> dict:
        """Basis size, frozen flag, step count and the selected harmonic Ritz values, read
        from the checkpoint header (layout of dd_recycle_export)."""
        import struct
        blob = self.export()
        magic, n_gamma, kmax, strategy, k, frozen, step, ntheta, tol = struct.unpack_from("<8sq6id", blob, 0)
        theta = np.frombuffer(blob, dtype=np.float64, count=ntheta, offset=struct.calcsize("<8sq6id"))
        return dict(k=k, frozen=bool(frozen), step=step, theta=theta.copy(), kmax=kmax, freeze_tol=tol)

    @classmethod
    def restore(cls, solver: "Solver", data: bytes) -> "Recycler":
        obj = cls.__new__(cls)
        obj.solver = solver
        h = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(data, len(data))
        nat.check(solver.lib.dd_recycle_import(solver.handle, buf, len(data), ctypes.byref(h)), "dd_recycle_import")
        obj.handle = h
        return obj

    def close(self):
        if getattr(self, "handle", None):
            self.solver.lib.dd_recycle_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
