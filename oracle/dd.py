"""Substructuring and BDDC, written densely from the paper's definitions (oracle; test infrastructure).

Sect. 3.1: the free nodes are split into subdomains of s^3 elements; a node is an
*interface* node if it belongs to more than one subdomain and an *interior* node
otherwise. The global Schur complement A = sum_i R_i^T S_i R_i with
S_i = K_GG - K_GI K_II^{-1} K_IG is applied per subdomain and never assembled
(eq. 6), and the reduced right-hand side is b = f_G - sum_i R_i^T K_GI K_II^{-1} f_I.

Sect. 3.2: the BDDC preconditioner (eqs. 7-9) with card or diag weights, coarse degrees of freedom
at corners and arithmetic averages over edges and faces, and the multilevel
variant in which the coarse problem is itself preconditioned by BDDC with the
level-1 subdomains playing the role of elements.

Sect. 3.3: adaptive face constraints from the generalized eigenproblem
(eq. 10) with the constraint row of eq. 12.

Interface vectors are indexed by the interface nodes in increasing free-node
index. Each subdomain problem is solved with dense LAPACK factorizations.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import q1

FACE, EDGE, CORNER = 0, 1, 2


def glob_type(mult: int) -> int:
    """Glob class from the number of subdomains sharing it: 2 -> face, 3..7 -> edge, >= 8 -> corner."""
    if mult <= 2:
        return FACE
    if mult < 8:
        return EDGE
    return CORNER


# ---------------------------------------------------------------------------
# Generic substructured system (used at level 1 with Q1 subdomain matrices and
# at level 2 with coarse subdomain matrices)
# ---------------------------------------------------------------------------

class Substructures:
    """An SPD system given as a sum of dense subdomain matrices over shared global dofs."""

    def __init__(self, n_global: int, local_dofs: list, local_K: list):
        self.n = n_global
        self.dofs = [np.asarray(d, dtype=np.int64) for d in local_dofs]
        self.K = local_K
        self.S = len(self.dofs)
        mult = np.zeros(n_global, dtype=np.int64)
        for d in self.dofs:
            mult[d] += 1
        self.mult = mult
        self.gamma = np.nonzero(mult >= 2)[0]              # interface dofs (sorted)
        self.interior_dofs = np.nonzero(mult == 1)[0]
        self.gpos = -np.ones(n_global, dtype=np.int64)
        self.gpos[self.gamma] = np.arange(len(self.gamma))
        self.locG, self.locI, self.RG = [], [], []
        for d in self.dofs:
            isG = mult[d] >= 2
            self.locG.append(np.nonzero(isG)[0])
            self.locI.append(np.nonzero(~isG)[0])
            self.RG.append(self.gpos[d[isG]])               # local interface -> global interface index
        # sharing sets of interface dofs -> globs
        pairs_dof = np.concatenate([d[mult[d] >= 2] for d in self.dofs])
        pairs_sub = np.concatenate([np.full(int((mult[d] >= 2).sum()), i) for i, d in enumerate(self.dofs)])
        order = np.lexsort((pairs_sub, pairs_dof))
        pd, ps = pairs_dof[order], pairs_sub[order]
        sets = {}
        starts = np.concatenate([[0], np.nonzero(np.diff(pd))[0] + 1, [len(pd)]])
        for a, b in zip(starts[:-1], starts[1:]):
            key = tuple(ps[a:b].tolist())
            sets.setdefault(key, []).append(int(pd[a]))
        globs = [(min(v), k, np.array(sorted(v), dtype=np.int64)) for k, v in sets.items()]
        globs.sort(key=lambda g: g[0])
        self.glob_subs = [g[1] for g in globs]               # sharing set (tuple of subdomain ids)
        self.glob_dofs = [g[2] for g in globs]               # global dof ids (sorted)
        self.glob_kind = [glob_type(len(g[1])) for g in globs]

    # Schur complement pieces ------------------------------------------------
    def local_schur(self, i: int) -> np.ndarray:
        K = self.K[i]
        I, G = self.locI[i], self.locG[i]
        if len(I) == 0:
            return K[np.ix_(G, G)].copy()
        X = np.linalg.solve(K[np.ix_(I, I)], K[np.ix_(I, G)])
        return K[np.ix_(G, G)] - K[np.ix_(G, I)] @ X

    def schur_apply(self, x: np.ndarray) -> np.ndarray:
        """A x = sum_i R_i^T S_i R_i x (eq. 6), S_i formed densely."""
        y = np.zeros(len(self.gamma))
        for i in range(self.S):
            S = self.local_schur(i)
            np.add.at(y, self.RG[i], S @ x[self.RG[i]])
        return y

    def dense_schur(self) -> np.ndarray:
        A = np.zeros((len(self.gamma), len(self.gamma)))
        for i in range(self.S):
            A[np.ix_(self.RG[i], self.RG[i])] += self.local_schur(i)
        return A

    def condense(self, f: np.ndarray) -> np.ndarray:
        """Reduced right-hand side b = f_G - sum_i R_i^T K_GI K_II^{-1} f_I (Sect. 3.1)."""
        b = f[self.gamma].copy()
        for i in range(self.S):
            K, I, G = self.K[i], self.locI[i], self.locG[i]
            if len(I):
                y = np.linalg.solve(K[np.ix_(I, I)], f[self.dofs[i][I]])
                np.add.at(b, self.RG[i], -K[np.ix_(G, I)] @ y)
        return b

    def recover(self, f: np.ndarray, x_gamma: np.ndarray) -> np.ndarray:
        """Full solution: interface values x_G and interior x_I = K_II^{-1}(f_I - K_IG x_G)."""
        x = np.zeros(self.n)
        x[self.gamma] = x_gamma
        for i in range(self.S):
            K, I, G = self.K[i], self.locI[i], self.locG[i]
            if len(I):
                rhs = f[self.dofs[i][I]] - K[np.ix_(I, G)] @ x_gamma[self.RG[i]]
                x[self.dofs[i][I]] = np.linalg.solve(K[np.ix_(I, I)], rhs)
        return x


# ---------------------------------------------------------------------------
# Level 1: Q1 subdomains of a block-partitioned structured mesh
# ---------------------------------------------------------------------------

def q1_substructures(mesh) -> Substructures:
    """Level-1 substructures: subdomain i = block of sx*sy*sz elements, x fastest."""
    conn, Ke = q1.element_arrays(mesh, with_coef=True)
    sx, sy, sz = mesh.sub
    Sx, Sy, Sz = mesh.nx // sx, mesh.ny // sy, mesh.nz // sz
    ez, ey, ex = np.meshgrid(np.arange(mesh.nz), np.arange(mesh.ny), np.arange(mesh.nx), indexing="ij")
    sub_of_elem = ((ex // sx) + Sx * ((ey // sy) + Sy * (ez // sz))).ravel()
    order = np.argsort(sub_of_elem, kind="stable")
    bounds = np.searchsorted(sub_of_elem[order], np.arange(Sx * Sy * Sz + 1))
    dofs, Ks = [], []
    for i in range(Sx * Sy * Sz):
        els = order[bounds[i]:bounds[i + 1]]
        c = conn[els]
        d = np.unique(c[c >= 0])
        pos = np.searchsorted(d, np.where(c >= 0, c, d[0]))
        K = np.zeros((len(d), len(d)))
        for e in range(len(els)):
            keep = c[e] >= 0
            p = pos[e][keep]
            K[np.ix_(p, p)] += Ke[els[e]][np.ix_(keep, keep)]
        dofs.append(d)
        Ks.append(K)
    subs = Substructures(mesh.n_free, dofs, Ks)
    subs.grid = (Sx, Sy, Sz)
    return subs


# ---------------------------------------------------------------------------
# BDDC on one level
# ---------------------------------------------------------------------------

class BDDC:
    """Two-level BDDC for the interface problem of `subs` (Sect. 3.2).

    kinds: which glob classes give coarse dofs ({CORNER, EDGE, FACE}); corners
    are point values, edges and faces arithmetic averages. extra_rows maps a
    face glob index to additional constraint rows (adaptive BDDC, Sect. 3.3),
    each an array over that glob's dofs. weights: 'card' or 'diag'.
    """

    def __init__(self, subs: Substructures, kinds=(CORNER, EDGE, FACE), weights="diag", extra_rows=None):
        self.subs = subs
        self.weights = weights
        extra_rows = extra_rows or {}
        # coarse dofs: (glob index, row over glob dofs)
        self.cdofs = []
        for gi, (kind, gd) in enumerate(zip(subs.glob_kind, subs.glob_dofs)):
            if kind not in kinds:
                continue
            row = np.full(len(gd), 1.0 / len(gd))  # point value if one dof, else average
            self.cdofs.append((gi, row))
            for r in extra_rows.get(gi, []):
                self.cdofs.append((gi, np.asarray(r, dtype=np.float64)))
        self.nC = len(self.cdofs)
        # per-subdomain constraint matrices over local dofs, coarse maps
        glob_of_sub = [[] for _ in range(subs.S)]
        for c, (gi, row) in enumerate(self.cdofs):
            for s in subs.glob_subs[gi]:
                glob_of_sub[s].append(c)
        self.cmap, self.C = [], []
        for i in range(subs.S):
            cs = glob_of_sub[i]
            C = np.zeros((len(cs), len(subs.dofs[i])))
            for r, c in enumerate(cs):
                gi, row = self.cdofs[c]
                loc = np.searchsorted(subs.dofs[i], subs.glob_dofs[gi])
                C[r, loc] = row
            self.cmap.append(np.array(cs, dtype=np.int64))
            self.C.append(C)
        # weights D_i on local interface dofs
        self.D = []
        if weights == "card":
            for i in range(subs.S):
                self.D.append(1.0 / subs.mult[subs.dofs[i][subs.locG[i]]])
        else:
            dsum = np.zeros(subs.n)
            for i in range(subs.S):
                np.add.at(dsum, subs.dofs[i], np.diag(subs.K[i]))
            for i in range(subs.S):
                g = subs.dofs[i][subs.locG[i]]
                self.D.append(np.diag(subs.K[i])[subs.locG[i]] / dsum[g])
        # saddle-point factorizations, coarse basis, coarse matrix (eqs. 8-9)
        self.lu, self.Phi, self.KCi = [], [], []
        KC = np.zeros((self.nC, self.nC))
        for i in range(subs.S):
            K, C = subs.K[i], self.C[i]
            n, m = K.shape[0], C.shape[0]
            Sad = np.zeros((n + m, n + m))
            Sad[:n, :n], Sad[:n, n:], Sad[n:, :n] = K, C.T, C
            lu = sla.lu_factor(Sad)
            rhs = np.zeros((n + m, m)); rhs[n:, :] = np.eye(m)
            Phi = sla.lu_solve(lu, rhs)[:n]
            KCi = Phi.T @ K @ Phi
            self.lu.append(lu); self.Phi.append(Phi); self.KCi.append(KCi)
            KC[np.ix_(self.cmap[i], self.cmap[i])] += KCi
        self.KC = KC

    def coarse_substructure_dofs(self, groups):
        """Level-2 subdomains: union of the coarse dofs of each group of level-1 subdomains."""
        dofs, Ks = [], []
        for grp in groups:
            d = np.unique(np.concatenate([self.cmap[i] for i in grp]))
            K = np.zeros((len(d), len(d)))
            for i in grp:
                p = np.searchsorted(d, self.cmap[i])
                K[np.ix_(p, p)] += self.KCi[i]
            dofs.append(d); Ks.append(K)
        return dofs, Ks

    def apply(self, r: np.ndarray, coarse_solve=None) -> np.ndarray:
        """z = M_BDDC^{-1} r on the interface (eqs. 7, 8, 9)."""
        subs = self.subs
        if coarse_solve is None:
            coarse_solve = lambda g: np.linalg.solve(self.KC, g)
        g = np.zeros(self.nC)
        us = []
        for i in range(subs.S):
            n = len(subs.dofs[i])
            m = self.C[i].shape[0]
            rhs = np.zeros(n + m)
            rhs[subs.locG[i]] = self.D[i] * r[subs.RG[i]]
            u = sla.lu_solve(self.lu[i], rhs)[:n]
            us.append(u)
            np.add.at(g, self.cmap[i], self.Phi[i].T @ rhs[:n])
        uC = coarse_solve(g)
        z = np.zeros(len(subs.gamma))
        for i in range(subs.S):
            v = us[i] + self.Phi[i] @ uC[self.cmap[i]]
            np.add.at(z, subs.RG[i], self.D[i] * v[subs.locG[i]])
        return z

    def apply_full(self, g: np.ndarray, coarse_solve=None) -> np.ndarray:
        """BDDC for the whole (uncondensed) system sum_i K_i u = g: interior correction,
        BDDC on the interface Schur complement, harmonic extension."""
        subs = self.subs
        u = np.zeros(subs.n)
        rG = g[subs.gamma].copy()
        u0s = []
        for i in range(subs.S):
            K, I, G = subs.K[i], subs.locI[i], subs.locG[i]
            if len(I):
                u0 = np.linalg.solve(K[np.ix_(I, I)], g[subs.dofs[i][I]])
                np.add.at(rG, subs.RG[i], -K[np.ix_(G, I)] @ u0)
            else:
                u0 = np.zeros(0)
            u0s.append(u0)
        zG = self.apply(rG, coarse_solve)
        u[subs.gamma] = zG
        for i in range(subs.S):
            K, I, G = subs.K[i], subs.locI[i], subs.locG[i]
            if len(I):
                u[subs.dofs[i][I]] = u0s[i] - np.linalg.solve(K[np.ix_(I, I)], K[np.ix_(I, G)] @ zG[subs.RG[i]])
        return u


def group_subdomains(grid, group: int):
    """Groups of group^3 level-1 subdomains (x fastest) forming the level-2 subdomains."""
    Sx, Sy, Sz = grid
    Gx, Gy, Gz = -(-Sx // group), -(-Sy // group), -(-Sz // group)
    groups = [[] for _ in range(Gx * Gy * Gz)]
    for k in range(Sz):
        for j in range(Sy):
            for i in range(Sx):
                gidx = (i // group) + Gx * ((j // group) + Gy * (k // group))
                groups[gidx].append(i + Sx * (j + Sy * k))
    return groups


class Preconditioner:
    """Two- or three-level BDDC preconditioner for the level-1 interface problem."""

    def __init__(self, subs: Substructures, levels=2, kinds=(CORNER, EDGE, FACE), weights="diag",
                 group=4, kinds2=(CORNER, EDGE, FACE), extra_rows=None):
        self.l1 = BDDC(subs, kinds, weights, extra_rows)
        self.levels = levels
        if levels == 3:
            groups = group_subdomains(subs.grid, group)
            d2, K2 = self.l1.coarse_substructure_dofs(groups)
            self.subs2 = Substructures(self.l1.nC, d2, K2)
            self.l2 = BDDC(self.subs2, kinds2, weights)

    def coarse_solve(self, g):
        if self.levels == 2:
            return np.linalg.solve(self.l1.KC, g)
        return self.l2.apply_full(g)

    def apply(self, r):
        return self.l1.apply(r, self.coarse_solve)

    def dense(self, n):
        return np.column_stack([self.apply(e) for e in np.eye(n)])


# ---------------------------------------------------------------------------
# Adaptive face constraints (Sect. 3.3)
# ---------------------------------------------------------------------------

def face_schur(subs: Substructures, i: int, face_dofs: np.ndarray) -> np.ndarray:
    """Schur complement of subdomain matrix K_i onto the given dofs (all other local dofs eliminated)."""
    d = subs.dofs[i]
    F = np.searchsorted(d, face_dofs)
    R = np.setdiff1d(np.arange(len(d)), F)
    K = subs.K[i]
    X = np.linalg.solve(K[np.ix_(R, R)], K[np.ix_(R, F)])
    S = K[np.ix_(F, F)] - K[np.ix_(F, R)] @ X
    return 0.5 * (S + S.T)


def adaptive_face_constraints(subs: Substructures, bddc_weights: list, tau: float, max_per_face: int = 10,
                              drop_tol: float = 1e-10, kinds=(CORNER, EDGE, FACE), method: str = "dense",
                              lobpcg_iters: int = 15):
    """Extra face constraints from eq. 10, one problem per face shared by two subdomains s, t.

    Reading used here: the pair problem lives on the common interface of s and t
    (the face together with the edges and corners it touches, i.e. every glob whose
    sharing set contains both). A_s, A_t are the Schur complements of the two
    subdomain matrices onto those dofs; Pi is the orthogonal projection onto the
    space where the two copies agree in every initial coarse dof of the common
    interface (corner values, edge and face averages); E averages the two copies
    with the BDDC weights. Eigenvectors with lambda > tau (at most max_per_face,
    largest first) give c = w^T Pi (I-E)^T A (I-E) Pi (eq. 12); its entries on
    the face itself, first copy, form the new row, orthogonalized against the face
    average and the rows before it (rows whose remaining relative norm is below
    drop_tol are dropped). Returns {face glob index: [rows]}.
    Parity unpinned against the paper (which uses a limited LOBPCG).
    """
    out = {}
    for gi, (kind, gd, sset) in enumerate(zip(subs.glob_kind, subs.glob_dofs, subs.glob_subs)):
        if kind != FACE or len(sset) != 2 or len(gd) < 2:
            continue
        s, t = sset
        closure = [g2 for g2, ss in enumerate(subs.glob_subs) if s in ss and t in ss]
        dofs = np.sort(np.concatenate([subs.glob_dofs[g2] for g2 in closure]))
        m = len(dofs)
        As, At = face_schur(subs, s, dofs), face_schur(subs, t, dofs)
        A = sla.block_diag(As, At)
        ws = bddc_weights[s][np.searchsorted(subs.dofs[s][subs.locG[s]], dofs)]
        wt = bddc_weights[t][np.searchsorted(subs.dofs[t][subs.locG[t]], dofs)]
        E = np.block([[np.diag(ws), np.diag(wt)], [np.diag(ws), np.diag(wt)]])
        IE = np.eye(2 * m) - E
        Q = []
        for g2 in closure:
            if subs.glob_kind[g2] in kinds:
                a = np.zeros(m)
                a[np.searchsorted(dofs, subs.glob_dofs[g2])] = 1.0 / len(subs.glob_dofs[g2])
                Q.append(np.concatenate([a, -a]))
        Qo, _ = np.linalg.qr(np.array(Q).T)
        Pi = np.eye(2 * m) - Qo @ Qo.T
        Lhs = Pi @ IE.T @ A @ IE @ Pi
        Rhs = Pi @ A @ Pi
        Lhs, Rhs = 0.5 * (Lhs + Lhs.T), 0.5 * (Rhs + Rhs.T)
        if method == "lobpcg":
            # the paper's solver: block LOBPCG for the largest eigenpairs, max_per_face vectors,
            # lobpcg_iters steps, on the subspace where Rhs is definite: the range of Pi, less
            # the common constant (1, 1) when both subdomains float (A_s 1 = A_t 1 = 0), on
            # which both sides of eq. 10 vanish
            from . import lobpcg
            ones = np.ones(m)
            floating = (np.linalg.norm(As @ ones) <= 1e-10 * np.linalg.norm(As) * np.sqrt(m) and
                        np.linalg.norm(At @ ones) <= 1e-10 * np.linalg.norm(At) * np.sqrt(m))
            Nc = np.ones(2 * m) / np.sqrt(2 * m) if floating else None

            def project(V):
                V = V - Qo @ (Qo.T @ V)
                return V - np.outer(Nc, Nc @ V) if Nc is not None else V

            # start block: unit vectors at the largest ratios of the diagonals of
            # (I-E)^T A (I-E) and A (the pencil before Pi; they need only diagonals of A)
            da = np.concatenate([np.diag(As), np.diag(At)])
            a1 = np.concatenate([(1 - ws) ** 2 * np.diag(As) + ws ** 2 * np.diag(At),
                                 wt ** 2 * np.diag(As) + (1 - wt) ** 2 * np.diag(At)])
            X0 = lobpcg.start_block(np.diag(a1), np.diag(da), min(max_per_face, 2 * m))
            lam_l, Xl = lobpcg.lobpcg_largest(Lhs, Rhs, max_per_face, iters=lobpcg_iters, X0=X0,
                                              project=project)
            order = np.argsort(lam_l, kind="stable")
            lam, V, T = lam_l[order], Xl[:, order], np.eye(2 * m)
        else:
            # restrict to the range of Rhs (drops ker Pi and the common null space)
            lam_r, U = np.linalg.eigh(Rhs)
            keep = lam_r > 1e-12 * lam_r.max()
            T = U[:, keep] / np.sqrt(lam_r[keep])
            lam, V = np.linalg.eigh(T.T @ Lhs @ T)
        sel = np.nonzero(lam > tau)[0][::-1][:max_per_face]
        fpos = np.searchsorted(dofs, gd)
        rows = []
        basis = [np.full(len(gd), 1.0 / np.sqrt(len(gd)))]
        for k in sel:
            w = T @ V[:, k]
            r = (w @ Lhs)[:m][fpos]
            nr0 = np.linalg.norm(r)
            if nr0 == 0:
                continue
            for bvec in basis:
                r = r - (bvec @ r) * bvec
            if np.linalg.norm(r) < drop_tol * nr0:
                continue
            r = r / np.linalg.norm(r)
            basis.append(r)
            rows.append(r)
        if rows:
            out[gi] = rows
    return out
