"""Sparse Cholesky of the global Q1 matrix by nested dissection + multifrontal elimination.

Oracle (test infrastructure). It solves K x = f (eq. 5) directly, so the
result is the exact discrete solution that the iterative method approaches.

Ordering: the free nodes form a box of a structured grid whose matrix graph is
the 27-point stencil. A box is split by the middle node plane of its longest
axis (a separator: nodes on either side share no element), recursively, until a
box holds at most `leaf` nodes. Elimination follows the tree bottom-up; each tree
node assembles a dense frontal matrix over its own variables plus its boundary
(the grid nodes in the one-node shell around its box, all of which lie in
ancestor separators), factors its own variables and passes the Schur complement
of the boundary to its parent (extend-add). Dense steps use numpy/scipy LAPACK
routines as library primitives.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
from scipy.linalg import blas, lapack
import scipy.sparse as sp


class _Front:
    __slots__ = ("vars", "bnd", "children", "L11", "L21")

    def __init__(self, vars_, bnd, children):
        self.vars = vars_
        self.bnd = bnd
        self.children = children
        self.L11 = None
        self.L21 = None


def _box_nodes(dims, box):
    Nx, Ny, Nz = dims
    x0, x1, y0, y1, z0, z1 = box
    z, y, x = np.meshgrid(np.arange(z0, z1), np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
    return (x + Nx * (y + Ny * z)).ravel()


def _shell_nodes(dims, box):
    """Grid nodes in the one-node shell around box (inside the grid, outside the box), sorted."""
    Nx, Ny, Nz = dims
    x0, x1, y0, y1, z0, z1 = box
    X0, X1 = max(x0 - 1, 0), min(x1 + 1, Nx)
    Y0, Y1 = max(y0 - 1, 0), min(y1 + 1, Ny)
    Z0, Z1 = max(z0 - 1, 0), min(z1 + 1, Nz)
    z, y, x = np.meshgrid(np.arange(Z0, Z1), np.arange(Y0, Y1), np.arange(X0, X1), indexing="ij")
    inside = (x >= x0) & (x < x1) & (y >= y0) & (y < y1) & (z >= z0) & (z < z1)
    return np.sort((x + Nx * (y + Ny * z))[~inside].ravel())


class NDCholesky:
    """K = L L^T with nested-dissection ordering on a structured (Nx, Ny, Nz) node grid."""

    def __init__(self, K: sp.spmatrix, dims, leaf: int = 512):
        self.K = sp.csr_matrix(K)
        self.dims = tuple(int(d) for d in dims)
        self.n = self.K.shape[0]
        assert self.n == self.dims[0] * self.dims[1] * self.dims[2]
        self.leaf = leaf
        self.root = self._build((0, self.dims[0], 0, self.dims[1], 0, self.dims[2]))
        self.postorder = []
        self._post(self.root)
        self._factor()

    # -- ordering ---------------------------------------------------------
    def _build(self, box):
        x0, x1, y0, y1, z0, z1 = box
        sizes = [x1 - x0, y1 - y0, z1 - z0]
        bnd = _shell_nodes(self.dims, box)
        if sizes[0] * sizes[1] * sizes[2] <= self.leaf or max(sizes) < 3:
            return _Front(_box_nodes(self.dims, box), bnd, [])
        ax = int(np.argmax(sizes))
        lo, hi = box[2 * ax], box[2 * ax + 1]
        mid = lo + (hi - lo) // 2
        sep = list(box)
        sep[2 * ax], sep[2 * ax + 1] = mid, mid + 1
        left = list(box)
        left[2 * ax + 1] = mid
        right = list(box)
        right[2 * ax] = mid + 1
        children = [self._build(tuple(b)) for b in (left, right) if b[2 * ax + 1] > b[2 * ax]]
        return _Front(_box_nodes(self.dims, tuple(sep)), bnd, children)

    def _post(self, f):
        stack = [(f, False)]
        while stack:
            node, done = stack.pop()
            if done:
                self.postorder.append(node)
            else:
                stack.append((node, True))
                for c in reversed(node.children):
                    stack.append((c, False))

    # -- numeric factorization -------------------------------------------
    def _factor(self):
        updates = {}
        Kc = self.K.tocsc()
        for f in self.postorder:
            nv, nb = len(f.vars), len(f.bnd)
            idx = np.concatenate([f.vars, f.bnd])
            F = np.zeros((nv + nb, nv + nb))
            # original entries in the columns of this front's own variables
            blk = Kc[:, f.vars][idx, :].toarray()  # [(nv+nb), nv]
            F[:, :nv] = blk
            F[:nv, nv:] = blk[nv:, :].T
            # extend-add of the children's boundary Schur complements
            if f.children:
                order = np.argsort(idx)
                sidx = idx[order]
                for c in f.children:
                    U = updates.pop(id(c))
                    p = order[np.searchsorted(sidx, c.bnd)]
                    F[np.ix_(p, p)] += U
            L11 = np.linalg.cholesky(F[:nv, :nv])
            if nb:
                # L21 = F21 L11^{-T}; the triangular inverse turns the solve into one GEMM
                Linv, info = lapack.dtrtri(L11, lower=1)
                assert info == 0
                L21 = F[nv:, :nv] @ Linv.T  # [nb, nv]
                # U = F22 - L21 L21^T (lower triangle by SYRK, then mirrored)
                U = blas.dsyrk(-1.0, L21, beta=1.0, c=np.asfortranarray(F[nv:, nv:]), lower=1)
                U = np.tril(U) + np.tril(U, -1).T
                updates[id(f)] = U
            else:
                L21 = np.zeros((0, nv))
            f.L11, f.L21 = L11, L21

    # -- triangular solves -------------------------------------------------
    def solve(self, b: np.ndarray) -> np.ndarray:
        """x = K^{-1} b for b of shape [n] or [n, m]."""
        y = np.array(b, dtype=np.float64, copy=True)
        for f in self.postorder:
            yv = sla.solve_triangular(f.L11, y[f.vars], lower=True)
            y[f.vars] = yv
            if len(f.bnd):
                y[f.bnd] -= f.L21 @ yv
        x = y
        for f in reversed(self.postorder):
            rhs = x[f.vars]
            if len(f.bnd):
                rhs = rhs - f.L21.T @ x[f.bnd]
            x[f.vars] = sla.solve_triangular(f.L11, rhs, lower=True, trans="T")
        return x

    def nnz_L(self) -> int:
        return int(sum(f.L11.shape[0] * (f.L11.shape[0] + 1) // 2 + f.L21.size for f in self.postorder))


def symbolic_counts(dims, leaf: int = 64):
    """(nnz(L), multiply-adds of the factorization) of the nested-dissection multifrontal
    Cholesky of a structured (Nx, Ny, Nz) grid, from the front sizes alone (no numeric work)."""
    class _Sym(NDCholesky):
        def __init__(self, dims, leaf):
            self.dims = tuple(int(d) for d in dims)
            self.leaf = leaf
            self.root = self._build((0, self.dims[0], 0, self.dims[1], 0, self.dims[2]))
            self.postorder = []
            self._post(self.root)
    sym = _Sym(dims, leaf)
    nnz = sum(len(f.vars) * (len(f.vars) + 1) // 2 + len(f.vars) * len(f.bnd) for f in sym.postorder)
    madds = sum(len(f.vars) ** 3 / 3 + len(f.vars) ** 2 * len(f.bnd) + len(f.vars) * len(f.bnd) ** 2 / 2
                for f in sym.postorder)
    return int(nnz), float(madds)


def factor_mesh(mesh, K=None, leaf: int = 64) -> NDCholesky:
    """Factor the assembled Q1 matrix of `mesh` (free nodes)."""
    from . import q1
    if K is None:
        K = q1.assemble(mesh)
    x0, x1, y0, y1, z0, z1 = mesh.free_box
    return NDCholesky(K, (x1 - x0, y1 - y0, z1 - z0), leaf)
