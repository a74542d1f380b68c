"""Adjoint of the Poisson solve (oracle; test infrastructure).

K(k) x = f with K = sum_e k_e K_e^0 symmetric positive definite (eq. 5).
For a loss L(x): lambda = K^{-1} dL/dx, dL/df = lambda, and
dL/dk_e = -lambda_e^T K_e^0 x_e (derivative of K^{-1} f with respect to k_e);
with k_e = exp(g_e), dL/dg_e = k_e dL/dk_e.
"""
from __future__ import annotations

import numpy as np

from . import q1


def coefficient_gradient(mesh, x: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """dL/dk_e = -lambda_e^T K_e^0 x_e per element (x fastest), Dirichlet values zero."""
    conn, Ke0 = q1.element_arrays(mesh, with_coef=False)
    xe = np.where(conn >= 0, x[np.maximum(conn, 0)], 0.0)
    le = np.where(conn >= 0, lam[np.maximum(conn, 0)], 0.0)
    return -np.einsum("ea,eab,eb->e", le, Ke0, xe)


def adjoint(mesh, chol, x: np.ndarray, grad_x: np.ndarray):
    """Returns (dL/df, dL/dk) for dL/dx = grad_x at the solution x = K^{-1} f."""
    lam = chol.solve(grad_x)
    return lam, coefficient_gradient(mesh, x, lam)
