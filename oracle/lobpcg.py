"""Block LOBPCG for the largest eigenpairs of a symmetric pencil (oracle; test infrastructure).

Sect. 3.3: the paper obtains the adaptive coarse dofs from the face eigenproblems (eq. 10)
by LOBPCG, with at most 15 iterations and at most 10 vectors per face. This module restates
the locally optimal block preconditioned conjugate gradient method (Knyazev, SIAM J. Sci.
Comput. 23, 2001) for A x = lambda B x with A symmetric and B symmetric positive definite,
maximizing the Rayleigh quotient, without a preconditioner (T = I), in this form:

  * the iterate block X (n x k) spans the current approximation; the residuals
    R = A X - B X diag(theta) are the new directions W; P holds the previous step's
    W- and P-components (the "conjugate" directions);
  * each step runs Rayleigh-Ritz on S = [X, W, P] (first step [X, W]): the columns are
    scaled to unit B-norm, an in-order Cholesky of S^T B S drops columns whose pivot is
    below drop_tol (1e-8) of the largest diagonal entry, and the k largest eigenpairs of
    L^{-1} (S^T A S) L^{-T} give the next X. A Cholesky factor of a Gram matrix carries
    about half the working digits, so columns independent of the others by less than
    1e-4 (pivot 1e-8) are treated as dependent: with smaller thresholds the B-orthogonality
    of the iterates decays once residuals reach rounding level;
  * the start block is the unit vectors of the k largest ratios A_ii / B_ii (a stable
    order: ties by index), and exactly `iters` steps are taken.

A, B: dense symmetric arrays (B semidefinite allowed: directions of zero B-norm are dropped
from every Rayleigh-Ritz basis). The CUDA path implements the same steps in the same order.
"""
from __future__ import annotations

import numpy as np


def start_block(A, B, k):
    """Unit vectors at the k largest A_ii / B_ii (ties: smaller index first; indices with
    B_ii = 0 last)."""
    a, b = np.diag(A), np.diag(B)
    r = [a[i] / b[i] if b[i] > 0 else -np.inf for i in range(len(a))]
    order = sorted(range(len(r)), key=lambda i: (-r[i], i))[:k]
    X = np.zeros((A.shape[0], k))
    for j, i in enumerate(order):
        X[i, j] = 1.0
    return X


def _rayleigh_ritz(S, AS, BS, k, drop_tol):
    """k largest Ritz pairs of (A, B) on span(S): (theta descending, Y with X = S Y)."""
    GA = S.T @ AS
    GB = S.T @ BS
    GA, GB = 0.5 * (GA + GA.T), 0.5 * (GB + GB.T)
    q = S.shape[1]
    # columns of (numerically) zero B-norm are dropped: B may be semidefinite (the face
    # pencil's B vanishes on the constrained jumps and on common constants)
    gmax = max(GB[j, j] for j in range(q))
    d = np.array([1.0 / np.sqrt(GB[j, j]) if GB[j, j] > 1e-14 * gmax else 0.0 for j in range(q)])
    GA = d[:, None] * GA * d[None, :]
    GB = d[:, None] * GB * d[None, :]
    # in-order Cholesky of GB, dropping columns with a small pivot
    keep, L = [], np.zeros((q, q))
    scale = max(GB[j, j] for j in range(q))
    for j in range(q):
        row = np.zeros(len(keep))  # forward substitution: L_kept row = GB[keep, j]
        for a, i in enumerate(keep):
            row[a] = (GB[j, i] - np.dot(L[a, :a], row[:a])) / L[a, a]
        piv = GB[j, j] - np.dot(row, row)
        if piv > drop_tol * scale:
            t = len(keep)
            L[t, :t] = row
            L[t, t] = np.sqrt(piv)
            keep.append(j)
    r = len(keep)
    L = L[:r, :r]
    Li = np.linalg.inv(L)
    C = Li @ GA[np.ix_(keep, keep)] @ Li.T
    theta, U = np.linalg.eigh(0.5 * (C + C.T))
    m = min(k, r)
    theta, U = theta[::-1][:m], U[:, ::-1][:, :m]
    Y = np.zeros((q, m))
    Y[keep, :] = d[keep, None] * (Li.T @ U)
    return theta, Y


def lobpcg_largest(A, B, k, iters=15, drop_tol=1e-8, X0=None, history=None, project=None):
    """theta (descending, k values) and X (n x k, B-orthonormal) after `iters` steps.

    project (optional): a projector onto a subspace on which B is definite, applied to the
    start block and to every new direction W, so that the iteration stays in it (the face
    pencil is posed on such a subspace of its 2m unknowns)."""
    n = A.shape[0]
    k = min(k, n)
    X = start_block(A, B, k) if X0 is None else X0
    if project is not None:
        X = project(X)
    theta, Y = _rayleigh_ritz(X, A @ X, B @ X, k, drop_tol)
    X = X @ Y
    AX, BX = A @ X, B @ X
    P = AP = BP = None
    if history is not None:
        history.append(theta.copy())
    for _ in range(iters):
        W = AX - BX * theta[None, :]
        if project is not None:
            W = project(W)
        AW, BW = A @ W, B @ W
        if P is None:
            S, AS, BS = np.hstack([X, W]), np.hstack([AX, AW]), np.hstack([BX, BW])
        else:
            S, AS, BS = np.hstack([X, W, P]), np.hstack([AX, AW, AP]), np.hstack([BX, BW, BP])
        kx = X.shape[1]
        theta, Y = _rayleigh_ritz(S, AS, BS, k, drop_tol)
        Yd = Y.copy()
        Yd[:kx, :] = 0.0  # the W- and P-components of the step
        P, AP, BP = S @ Yd, AS @ Yd, BS @ Yd
        X, AX, BX = S @ Y, AS @ Y, BS @ Y
        if history is not None:
            history.append(theta.copy())
    return theta, X
