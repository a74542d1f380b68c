"""Pure-Neumann variant of the pressure problem (oracle; test infrastructure).

With no Dirichlet part of the boundary (Sect. 2) the stiffness matrix K is only
semidefinite: its null space is spanned by the constant vector (the constant functions of
the finite element space). Sect. 4.1 handles this in the deflated CG by taking the constant
vector into the deflation basis; the null space of the interface Schur complement A is the
restriction of the constants to the interface.

The paper gives no more detail; this module follows these readings.
  * A load vector is made consistent by its l2 projection onto range(K) = 1^perp (K is
    symmetric and K 1 = 0): its mean is removed.
  * The solution reported is the representative orthogonal to the null space (mean zero).
  * A consistent singular system is solved in its grounded form K + e_g e_g^T, which is
    SPD for a connected mesh and keeps the sparsity pattern of K: its solution y has
    y_g = 0 and K y = f (multiply by 1^T: 1^T K y + y_g = 1^T f = 0).
  * In BDDC the constrained local problems stay nonsingular (the coarse dofs fix the
    constants). The coarse matrix is singular in the constant coarse vector but the coarse
    right-hand side of a residual orthogonal to 1 is consistent (the coarse basis
    reproduces constants and the weights are a partition of unity), so the coarse problem
    is solved in grounded form. Two levels only.
  * The constant column of W is orthogonal to the range of A (A 1 = 0), so it takes no
    part in the A-orthogonal deflation of Algorithm 1 (its Galerkin row is zero). It acts
    as an l2 projection: the preconditioned residuals, and with them the search
    directions, are kept orthogonal to the constants (W^T p_j = 0 for that column), and the
    constant is removed from the initial guess and from the result.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import cholesky, dd, pcg, q1


def consistent(f: np.ndarray) -> np.ndarray:
    """l2 projection of a load vector onto range(K) = 1^perp."""
    f = np.asarray(f, dtype=np.float64)
    return f - f.mean()


def grounded(K, g: int = 0):
    """K + e_g e_g^T (sparse or dense)."""
    if sp.issparse(K):
        n = K.shape[0]
        return (K + sp.csr_matrix(([1.0], ([g], [g])), shape=(n, n))).tocsr()
    Kg = np.array(K, dtype=np.float64, copy=True)
    Kg[g, g] += 1.0
    return Kg


class Solver:
    """Mean-free solutions of K x = P f on a mesh without Dirichlet faces, by the oracle's
    nested-dissection sparse Cholesky of the grounded matrix."""

    def __init__(self, mesh, K=None):
        self.K = q1.assemble(mesh) if K is None else K
        self.ch = cholesky.factor_mesh(mesh, grounded(self.K))

    def solve(self, f: np.ndarray) -> np.ndarray:
        y = self.ch.solve(consistent(f))
        return y - y.mean()


def null_projector(n: np.ndarray):
    """v -> v - n (n^T v) / (n^T n): the l2 projection onto n^perp."""
    n = np.asarray(n, dtype=np.float64)
    nn = float(n @ n)
    return lambda v: v - n * (float(n @ v) / nn)


class Preconditioner(dd.Preconditioner):
    """Two-level BDDC whose coarse problem is solved in grounded form."""

    def __init__(self, subs: dd.Substructures, kinds=(dd.CORNER, dd.EDGE, dd.FACE), weights="diag"):
        super().__init__(subs, 2, kinds, weights)
        self.KCg = grounded(self.l1.KC)

    def coarse_solve(self, g):
        return np.linalg.solve(self.KCg, g)


def deflated_pcg(A, Minv, b, x_init, W=None, AW=None, rtol=1e-8, maxit=1000, stop="rhs", flexible=False,
                 reorth=False):
    """Algorithm 1 on the consistent singular interface problem, with the constant
    interface vector as the null-space column of the deflation basis (see the module
    readings); W, AW: the other (recycled) columns, orthogonal to the constants."""
    P = null_projector(np.ones(len(b)))
    x, info = pcg.deflated_pcg(A, lambda r: P(Minv(r)), b, P(np.asarray(x_init, dtype=np.float64)), W, AW, rtol,
                               maxit, stop, flexible, reorth)
    return P(x), info


def solve_sequence(A, Minv, rhs_list, R=0, strategy="B4", rtol=1e-8, freeze_tol=1e-5, flexible=False):
    """A sequence of consistent interface problems with the previous solution as the initial
    guess and the deflation basis recycled between them (Sect. 4.2); returns (xs, infos,
    recycler). The recycled columns come from search directions, hence are orthogonal to
    the constants."""
    rec = pcg.Recycler(R, strategy, freeze_tol)
    P = null_projector(np.ones(len(rhs_list[0])))
    Mp = lambda r: P(Minv(r))
    x = np.zeros(len(rhs_list[0]))
    xs, infos = [], []
    for b in rhs_list:
        x, info = deflated_pcg(A, Minv, b, x, rec.W, rec.AW, rtol, flexible=flexible)
        rec.update(info, Mp)
        xs.append(x)
        infos.append(info)
    return xs, infos, rec
