"""Pins for the oracle's block LOBPCG (the paper's face eigensolver, Sect. 3.3).

* Converged, the k Ritz values are the k largest generalized eigenvalues of the pencil
  (scipy.linalg.eigh) and agree with scipy.sparse.linalg.lobpcg, a library implementation.
* At every step the Ritz values do not decrease and stay below the eigenvalues they
  approximate (Courant-Fischer: the search space only grows by the previous iterate).
* The iterates are B-orthonormal.
* On a semidefinite B, restricting the iteration to a subspace where B is definite gives
  the eigenvalues of the pencil restricted to it (as the face problems of eq. 10 need).
* For the adaptive constraints of a mesh with jumping coefficients, 60 steps give the same
  constraint count and essentially the same preconditioner as the dense eigensolver, and
  15 steps (the paper's limit) keep the BDDC bounds lambda_min >= 1, lambda_max at most
  the non-adaptive one.
"""
import numpy as np
import pytest
import scipy.linalg as sla
from scipy.sparse.linalg import lobpcg as scipy_lobpcg

from oracle import dd, lobpcg
from workload import make_mesh


def _pencil(n, seed):
    rng = np.random.default_rng(seed)
    Q = rng.standard_normal((n, n))
    A = Q @ np.diag(np.geomspace(1e-2, 50, n)) @ Q.T
    Bq = rng.standard_normal((n, n))
    B = Bq @ Bq.T + n * np.eye(n)
    return A, B


@pytest.mark.parametrize("n,k", [(40, 3), (80, 10), (12, 12)])
def test_converged_ritz_values_are_the_largest_eigenvalues(n, k):
    A, B = _pencil(n, n)
    ev = sla.eigh(A, B, eigvals_only=True)[::-1][:k]
    th, X = lobpcg.lobpcg_largest(A, B, k, iters=300)
    assert np.allclose(th, ev, rtol=1e-9, atol=1e-12 * ev[0])
    assert np.allclose(X.T @ B @ X, np.eye(k), atol=1e-9)
    if k < n // 2:
        th_s, _ = scipy_lobpcg(A, lobpcg.start_block(A, B, k), B=B, largest=True, maxiter=500, tol=1e-12)
        assert np.allclose(np.sort(th_s)[::-1], th, rtol=1e-7)


def test_ritz_values_rise_monotonically_and_stay_below_the_eigenvalues():
    A, B = _pencil(60, 7)
    ev = sla.eigh(A, B, eigvals_only=True)[::-1]
    hist = []
    lobpcg.lobpcg_largest(A, B, 5, iters=15, history=hist)
    for a, b in zip(hist[:-1], hist[1:]):
        assert np.all(b >= a - 1e-10 * abs(ev[0]))
    for th in hist:
        assert np.all(th <= ev[: len(th)] + 1e-10 * abs(ev[0]))
    assert hist[-1][0] > hist[0][0]  # it makes progress


def test_semidefinite_pencil_restricted_by_a_projector():
    # B vanishes on span(Z); A vanishes there too. On the complement the pencil is definite
    rng = np.random.default_rng(3)
    n, nz, k = 30, 4, 4
    Z, _ = np.linalg.qr(rng.standard_normal((n, nz)))
    Pz = np.eye(n) - Z @ Z.T
    A0, B0 = _pencil(n, 11)
    A, B = Pz @ A0 @ Pz, Pz @ B0 @ Pz
    A, B = 0.5 * (A + A.T), 0.5 * (B + B.T)
    Cc = np.linalg.qr(np.column_stack([Z, rng.standard_normal((n, n - nz))]))[0][:, nz:]  # basis of the complement
    ev = sla.eigh(Cc.T @ A @ Cc, Cc.T @ B @ Cc, eigvals_only=True)[::-1][:k]
    th, X = lobpcg.lobpcg_largest(A, B, k, iters=200, project=lambda V: V - Z @ (Z.T @ V))
    assert np.allclose(th, ev, rtol=1e-9)
    assert np.abs(Z.T @ X).max() <= 1e-10


def test_adaptive_constraints_by_lobpcg_match_the_dense_eigensolver():
    rng = np.random.default_rng(5)
    n = 8
    coef = np.exp(2.0 * rng.standard_normal((n, n, n)))
    m = make_mesh(n, 4, 1.08, 20.0, coef=coef)
    subs = dd.q1_substructures(m)
    kinds = (dd.CORNER, dd.EDGE, dd.FACE)
    base = dd.Preconditioner(subs, 2, kinds, "diag")
    A = subs.dense_schur()
    L = np.linalg.cholesky(A)
    N = len(subs.gamma)
    e0 = np.linalg.eigvalsh(L.T @ base.dense(N) @ L)
    for tau in (1.5, 2.0, 3.0):
        dense = dd.adaptive_face_constraints(subs, base.l1.D, tau=tau)
        r60 = dd.adaptive_face_constraints(subs, base.l1.D, tau=tau, method="lobpcg", lobpcg_iters=60)
        r15 = dd.adaptive_face_constraints(subs, base.l1.D, tau=tau, method="lobpcg", lobpcg_iters=15)
        assert sorted(dense) == sorted(r60)
        assert all(len(dense[g]) == len(r60[g]) for g in dense)
        Md = dd.Preconditioner(subs, 2, kinds, "diag", extra_rows=dense).dense(N)
        M60 = dd.Preconditioner(subs, 2, kinds, "diag", extra_rows=r60).dense(N)
        assert np.abs(M60 - Md).max() <= 1e-6 * np.abs(Md).max()
        e15 = np.linalg.eigvalsh(L.T @ dd.Preconditioner(subs, 2, kinds, "diag", extra_rows=r15).dense(N) @ L)
        assert e15[0] >= 1 - 1e-10 and e15[-1] <= e0[-1] + 1e-9
