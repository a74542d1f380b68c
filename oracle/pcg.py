"""Deflated PCG with Krylov subspace recycling (oracle; test infrastructure).

Algorithm 1 (deflated PCG, Sect. 4.1) with the optional residual
re-orthogonalization, the stopping criteria of Sect. 5 (eq. stopping_rhs,
default, and eq. stopping_residual), and the recycling strategies of Sect. 4.2:
B1 (first R search vectors), B2 (last R search vectors), B3/B4 (R smallest /
largest harmonic Ritz vectors of eq. harmonicRitz on V = [W, P]) with the
freezing criterion eq. harmritzstopcrit.

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


def deflated_pcg(A, Minv, b, x_init, W=None, AW=None, rtol=1e-8, maxit=1000, stop="rhs",
                 flexible=False, reorth=False):
    """Algorithm 1. Returns (x, SolveInfo). W, AW are [n, k] arrays or None."""
    b = np.asarray(b, dtype=np.float64)
    x = np.array(x_init, dtype=np.float64, copy=True)
    k = 0 if W is None else W.shape[1]
    if k:
        G = W.T @ AW
        G = 0.5 * (G + G.T)
        Gf = sla.cho_factor(G)
        x = x + W @ sla.cho_solve(Gf, W.T @ (b - A(x)))       # first projection: W^T r_0 = 0
        if reorth:
            WWf = sla.cho_factor(W.T @ W)
    r = b - A(x)
    nb = np.linalg.norm(b)
    nr0 = np.linalg.norm(r)
    ref = nb if stop == "rhs" else nr0
    if ref == 0.0:
        ref = 1.0
    P, AP, Z, alphas, hist, wtr = [], [], [], [], [np.linalg.norm(r) / ref], []
    if hist[0] < rtol:
        return x, SolveInfo(0, nr0 / ref, hist[0], hist, np.zeros((len(b), 0)), np.zeros((len(b), 0)),
                            np.zeros((len(b), 0)), np.zeros(0), wtr)
    z = Minv(r)
    Z.append(z)
    p = z - W @ sla.cho_solve(Gf, AW.T @ z) if k else z.copy()
    rz = r @ z
    its = 0
    while its < maxit:
        q = A(p)
        alpha = rz / (p @ q)
        P.append(p); AP.append(q); alphas.append(alpha)
        x = x + alpha * p
        r = r - alpha * q
        if k and reorth:
            r = r - W @ sla.cho_solve(WWf, W.T @ r)
        its += 1
        if k:
            wtr.append(float(np.linalg.norm(W.T @ r)))
        rel = np.linalg.norm(r) / ref
        hist.append(rel)
        if rel < rtol:
            break
        z_new = Minv(r)
        Z.append(z_new)
        rz_new = r @ z_new
        beta = (rz_new - r @ z) / rz if flexible else rz_new / rz
        p = z_new + beta * p
        if k:
            p = p - W @ sla.cho_solve(Gf, AW.T @ z_new)
        z, rz = z_new, rz_new
    info = SolveInfo(its, nr0 / ref, hist[-1], hist, np.column_stack(P), np.column_stack(AP),
                     np.column_stack(Z), np.array(alphas), wtr)
    return x, info


def harmonic_ritz(V, AV, MAV):
    """Solve V^T A M^{-1} A V y = theta V^T A V y (eq. harmonicRitz).

    Returns theta (ascending) and Y with Y^T (V^T A V) Y = I. The problem is
    restricted to the numerically nonsingular part of V^T A V.
    """
    F = V.T @ AV
    F = 0.5 * (F + F.T)
    Gh = AV.T @ MAV
    Gh = 0.5 * (Gh + Gh.T)
    lam, Q = np.linalg.eigh(F)
    keep = lam > 1e-12 * lam.max()
    T = Q[:, keep] / np.sqrt(lam[keep])
    theta, U = np.linalg.eigh(T.T @ Gh @ T)
    return theta, T @ U


class Recycler:
    """Deflation basis W across a sequence of solves (Sect. 4.2)."""

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
            crit = np.linalg.norm(new_theta - self.theta) / np.linalg.norm(new_theta)
            if crit <= self.freeze_tol:
                self.frozen = True
                self.frozen_at = self.step
        self.theta = new_theta
        Ys = Y[:, sel]
        self.W, self.AW, self.MAW = V @ Ys, AV @ Ys, MAV @ Ys


def solve_sequence(A, Minv, rhs_list, R=0, strategy="B4", rtol=1e-8, stop="rhs", x0="prev",
                   flexible=False, reorth=False, maxit=1000):
    """Solve A x_t = b_t for a sequence with recycling; returns (xs, infos, recycler)."""
    rec = Recycler(R, strategy)
    x = np.zeros_like(rhs_list[0])
    xs, infos = [], []
    for b in rhs_list:
        xin = x if x0 == "prev" else np.zeros_like(b)
        x, info = deflated_pcg(A, Minv, b, xin, rec.W, rec.AW, rtol, maxit, stop, flexible, reorth)
        rec.update(info, Minv)
        xs.append(x)
        infos.append(info)
    return xs, infos, rec
