"""Deflated PCG with Krylov subspace recycling (oracle; test infrastructure).

Algorithm 1 (deflated PCG, Sect. 4.1) with the optional residual
re-orthogonalization, the stopping criteria of Sect. 5 (eq. 18,
default, and eq. 17), and the recycling strategies of Sect. 4.2:
B1 (first R search vectors), B2 (last R search vectors), B3/B4 (R smallest /
largest harmonic Ritz vectors of eq. 15 on V = [W, P]) with the
freezing criterion eq. 16.

A flexible (Polak-Ribiere) beta is available for inexact preconditioners; it is
not in the paper and equals the paper's beta whenever the preconditioner is an
exact fixed SPD operator and r_j^T z_{j-1} = 0.

A and Minv are callables on vectors; every product is formed explicitly.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla


@dataclass
class SolveInfo:
    iters: int
    rel_res0: float
    rel_res: float
    res_history: list
    P: np.ndarray      # search vectors p_0..p_{l-1} as columns
    AP: np.ndarray     # A p_j
    Z: np.ndarray      # preconditioned residuals z_0..z_l (z_l computed only if needed)
    alphas: np.ndarray
    wtr: list = field(default_factory=list)  # ||W^T r_j|| per iteration


class Deflation:
    """The deflation space U = range(W) of Sect. 4.1 with G = W^T A W (k x k, SPD).

    coarse_correct: x + W G^{-1} W^T (b - A x), the A-orthogonal projection of the
    error onto U, after which W^T (b - A x) = 0.
    project: Q v = v - W G^{-1} (AW)^T v, the A-orthogonal projector onto the
    complement of U (eq. 13).
    orthogonalize: v - W (W^T W)^{-1} W^T v (the optional residual
    re-orthogonalization of Sect. 4.1).
    """

    def __init__(self, W, AW):
        self.W, self.AW = W, AW
        G = W.T @ AW
        self.G = sla.cho_factor(0.5 * (G + G.T))
        self._WW = None

    def coarse_correct(self, x, r):
        return x + self.W @ sla.cho_solve(self.G, self.W.T @ r)

    def project(self, v):
        return v - self.W @ sla.cho_solve(self.G, self.AW.T @ v)

    def orthogonalize(self, v):
        if self._WW is None:
            self._WW = sla.cho_factor(self.W.T @ self.W)
        return v - self.W @ sla.cho_solve(self._WW, self.W.T @ v)


def deflated_pcg(A, Minv, b, x_init, W=None, AW=None, rtol=1e-8, maxit=1000, stop="rhs",
                 flexible=False, reorth=False):
    """Deflated PCG (Sect. 4.1, Algorithm 1). Returns (x, SolveInfo); W, AW are [n, k] or None.

    The method: the initial guess is corrected on U = range(W) so that the residual is
    orthogonal to W; then PCG runs with every preconditioned residual passed through Q
    (eq. 13), so the search directions stay A-orthogonal to U and the iterates minimize
    the A-norm error over x_0 + U + K_j(QAQ, r_0). With flexible=True the step length
    of the new direction uses r_j^T (z_j - z_{j-1}) (Polak-Ribiere) instead of r_j^T z_j.
    """
    b = np.asarray(b, dtype=np.float64)
    x = np.array(x_init, dtype=np.float64, copy=True)
    U = Deflation(W, AW) if (W is not None and W.shape[1] > 0) else None
    if U is not None:
        x = U.coarse_correct(x, b - A(x))
    r = b - A(x)
    nb = np.linalg.norm(b)
    nr0 = np.linalg.norm(r)
    ref = nb if stop == "rhs" else nr0
    if ref == 0.0:
        ref = 1.0
    P, AP, Z, alphas, hist, wtr = [], [], [], [], [np.linalg.norm(r) / ref], []
    p = None
    z_prev = None
    rz_prev = None
    its = 0
    while hist[-1] >= rtol and its < maxit:
        z = Minv(r)
        Z.append(z)
        rz = r @ z
        d = U.project(z) if U is not None else z
        if p is None:
            p = d.copy() if U is None else d
        else:
            num = rz - r @ z_prev if flexible else rz
            p = d + (num / rz_prev) * p
        q = A(p)
        alpha = rz / (p @ q)
        P.append(p); AP.append(q); alphas.append(alpha)
        x = x + alpha * p
        r = r - alpha * q
        if U is not None and reorth:
            r = U.orthogonalize(r)
        its += 1
        if U is not None:
            wtr.append(float(np.linalg.norm(U.W.T @ r)))
        hist.append(np.linalg.norm(r) / ref)
        z_prev, rz_prev = z, rz
    n = len(b)
    stack = lambda L: np.column_stack(L) if L else np.zeros((n, 0))
    info = SolveInfo(its, nr0 / ref, hist[-1], hist, stack(P), stack(AP), stack(Z), np.array(alphas), wtr)
    return x, info


def harmonic_ritz(V, AV, MAV):
    """Solve V^T A M^{-1} A V y = theta V^T A V y (Sect. 4.2, eq. 15).

    Returns theta (ascending) and Y with Y^T (V^T A V) Y = I. The pencil's eigenpairs
    do not depend on the scaling of V's columns, so the columns are first scaled to
    unit A-norm (search vectors shrink with the residual, by many orders of magnitude
    within one solve); the problem is then restricted to the numerically nonsingular
    part of the scaled V^T A V (eigenvalues above 1e-12 of the largest), which drops
    only directions that are numerically dependent.
    """
    F = V.T @ AV
    F = 0.5 * (F + F.T)
    Gh = AV.T @ MAV
    Gh = 0.5 * (Gh + Gh.T)
    d = 1.0 / np.sqrt(np.diag(F))
    Fs = d[:, None] * F * d[None, :]
    lam, Q = np.linalg.eigh(Fs)
    keep = lam > 1e-12 * lam.max()
    T = d[:, None] * (Q[:, keep] / np.sqrt(lam[keep]))
    theta, U = np.linalg.eigh(T.T @ Gh @ T)
    return theta, T @ U


def ritz_settled(theta_new, theta_old, tol):
    """Freezing test of Sect. 4.2, eq. 16: ||theta^(i) - theta^(i-1)||_2 / ||theta^(i)||_2 <= tol.

    theta_new, theta_old: the R selected harmonic Ritz values of two consecutive
    systems, in the order of selection. Returns (settled, ratio).
    """
    ratio = np.linalg.norm(np.asarray(theta_new) - np.asarray(theta_old)) / np.linalg.norm(theta_new)
    return bool(ratio <= tol), float(ratio)


class Recycler:
    """Deflation basis W across a sequence of solves (Sect. 4.2).

    crit_history records, per update that applied the freezing test, (step, ratio).
    """

    def __init__(self, R: int, strategy: str = "B4", freeze_tol: float = 1e-5):
        self.R = R
        self.strategy = strategy
        self.freeze_tol = freeze_tol
        self.W = None
        self.AW = None
        self.MAW = None
        self.theta = None
        self.frozen = False
        self.frozen_at = None
        self.step = 0
        self.crit_history = []

    def update(self, info: SolveInfo, Minv):
        """Update W after a solve from its search vectors (P, AP) and M^{-1} A P."""
        self.step += 1
        if self.frozen or self.R == 0 or info.P.shape[1] == 0:
            return
        P, AP = info.P, info.AP
        if self.strategy == "B1":
            have = 0 if self.W is None else self.W.shape[1]
            take = min(self.R - have, P.shape[1])
            self.W = P[:, :take] if self.W is None else np.hstack([self.W, P[:, :take]])
            self.AW = AP[:, :take] if self.AW is None else np.hstack([self.AW, AP[:, :take]])
            if self.W.shape[1] >= self.R:
                self.frozen = True
                self.frozen_at = self.step
            return
        if self.strategy == "B2":
            W = P if self.W is None else np.hstack([self.W, P])
            AW = AP if self.AW is None else np.hstack([self.AW, AP])
            self.W, self.AW = W[:, -self.R:], AW[:, -self.R:]
            return
        MAP = np.column_stack([Minv(AP[:, j]) for j in range(AP.shape[1])])
        if self.W is None:
            V, AV, MAV = P, AP, MAP
        else:
            V, AV, MAV = np.hstack([self.W, P]), np.hstack([self.AW, AP]), np.hstack([self.MAW, MAP])
        theta, Y = harmonic_ritz(V, AV, MAV)
        m = min(self.R, len(theta))
        sel = np.arange(len(theta))[::-1][:m] if self.strategy == "B4" else np.arange(m)
        new_theta = np.array(theta[sel])  # B4: descending, B3: ascending
        if (self.theta is not None and len(self.theta) == self.R and len(new_theta) == self.R):
            settled, ratio = ritz_settled(new_theta, self.theta, self.freeze_tol)
            self.crit_history.append((self.step, ratio))
            if settled:
                self.frozen = True
                self.frozen_at = self.step
        self.theta = new_theta
        Ys = Y[:, sel]
        self.W, self.AW, self.MAW = V @ Ys, AV @ Ys, MAV @ Ys


def solve_sequence(A, Minv, rhs_list, R=0, strategy="B4", rtol=1e-8, stop="rhs", x0="prev",
                   flexible=False, reorth=False, maxit=1000, freeze_tol=1e-5):
    """Solve A x_t = b_t for a sequence with recycling; returns (xs, infos, recycler)."""
    rec = Recycler(R, strategy, freeze_tol)
    x = np.zeros_like(rhs_list[0])
    xs, infos = [], []
    for b in rhs_list:
        xin = x if x0 == "prev" else np.zeros_like(b)
        x, info = deflated_pcg(A, Minv, b, xin, rec.W, rec.AW, rtol, maxit, stop, flexible, reorth)
        rec.update(info, Minv)
        xs.append(x)
        infos.append(info)
    return xs, infos, rec
