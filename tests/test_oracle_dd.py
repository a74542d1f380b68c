"""Pins for the oracle's substructuring and BDDC (Sect. 3.1-3.3)."""
import os

import numpy as np
import pytest

from oracle import cholesky, dd, q1
from workload import load_sequence, make_mesh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def small():
    m = make_mesh(8, 4, 1.08, 20.0)
    return m, dd.q1_substructures(m)


def test_cube16_partition_counts():
    ref = dict(l.split() for l in open(os.path.join(GOLDEN, "cube16_globs.txt")) if l.strip() and not l.startswith("#"))
    m = make_mesh(16, 4)
    subs = dd.q1_substructures(m)
    assert m.n_free == int(ref["free_nodes"])
    assert len(subs.gamma) == int(ref["interface_nodes"])
    kinds = np.array(subs.glob_kind)
    assert (kinds == dd.FACE).sum() == int(ref["faces"])
    assert (kinds == dd.EDGE).sum() == int(ref["edges"])
    assert (kinds == dd.CORNER).sum() == int(ref["corners"])


def test_schur_complement_equals_global_elimination(small):
    m, subs = small
    K = q1.assemble(m).toarray()
    G, I = subs.gamma, subs.interior_dofs
    S_glob = K[np.ix_(G, G)] - K[np.ix_(G, I)] @ np.linalg.solve(K[np.ix_(I, I)], K[np.ix_(I, G)])
    A = subs.dense_schur()
    assert np.allclose(A, S_glob, rtol=1e-12, atol=1e-12 * np.abs(S_glob).max())
    x = np.random.default_rng(1).standard_normal(len(G))
    assert np.allclose(subs.schur_apply(x), S_glob @ x, rtol=1e-12, atol=1e-12 * np.abs(S_glob @ x).max())


def test_condense_solve_recover_equals_direct(small):
    m, subs = small
    f = load_sequence(m, 1, 1)[0]
    x_direct = cholesky.factor_mesh(m).solve(f)
    b = subs.condense(f)
    xg = np.linalg.solve(subs.dense_schur(), b)
    assert np.allclose(xg, x_direct[subs.gamma], rtol=1e-11, atol=1e-12 * np.abs(x_direct).max())
    x = subs.recover(f, xg)
    assert np.allclose(x, x_direct, rtol=1e-11, atol=1e-12 * np.abs(x_direct).max())


@pytest.mark.parametrize("weights", ["card", "diag"])
def test_bddc_lambda_min_and_constraint_monotonicity(small, weights):
    m, subs = small
    A = subs.dense_schur()
    n = len(subs.gamma)
    lmax = []
    for kinds in [(dd.CORNER,), (dd.CORNER, dd.FACE), (dd.CORNER, dd.EDGE, dd.FACE)]:
        P = dd.Preconditioner(subs, 2, kinds, weights)
        M = P.dense(n)
        assert np.allclose(M, M.T, atol=1e-12 * np.abs(M).max())
        Lc = np.linalg.cholesky(A)
        ev = np.linalg.eigvalsh(Lc.T @ M @ Lc)  # spectrum of M^{-1}-preconditioned A
        assert ev[0] >= 1 - 1e-10
        lmax.append(ev[-1])
        # coarse basis reproduces the coarse dofs: C_i Phi_i = I
        for i in range(subs.S):
            assert np.allclose(P.l1.C[i] @ P.l1.Phi[i], np.eye(P.l1.C[i].shape[0]), atol=1e-10)
    assert lmax[0] > lmax[1] > lmax[2] - 1e-12


def test_bddc_card_weights_partition_of_unity(small):
    m, subs = small
    for w in ("card", "diag"):
        P = dd.Preconditioner(subs, 2, (dd.CORNER, dd.EDGE, dd.FACE), w)
        tot = np.zeros(len(subs.gamma))
        for i in range(subs.S):
            np.add.at(tot, subs.RG[i], P.l1.D[i])
        assert np.allclose(tot, 1.0, atol=1e-14)


def test_three_level_bddc_bounds():
    m = make_mesh(8, 2, 1.08, 20.0)
    subs = dd.q1_substructures(m)  # 4^3 subdomains of 2^3 elements, groups of 2^3 -> 8 coarse subdomains
    A = subs.dense_schur()
    L = np.linalg.cholesky(A)
    n = len(subs.gamma)
    P2 = dd.Preconditioner(subs, 2)
    P3 = dd.Preconditioner(subs, 3, group=2)
    assert P3.subs2.S == 8
    e2 = np.linalg.eigvalsh(L.T @ P2.dense(n) @ L)
    M3 = P3.dense(n)
    assert np.allclose(M3, M3.T, atol=1e-11 * np.abs(M3).max())
    e3 = np.linalg.eigvalsh(L.T @ M3 @ L)
    assert e2[0] >= 1 - 1e-10 and e3[0] >= 1 - 1e-10
    assert e3[-1] >= e2[-1] - 1e-9  # an approximate coarse solve cannot lower lambda_max


def test_level2_full_system_bddc_dominates_exact_inverse():
    # M_C^{-1} >= K_C^{-1} in the SPD order (level-2 BDDC has lambda_min >= 1 on K_C)
    m = make_mesh(8, 2, 1.08, 20.0)
    subs = dd.q1_substructures(m)
    P3 = dd.Preconditioner(subs, 3, group=2)
    KC = P3.l1.KC
    MC = np.column_stack([P3.l2.apply_full(e) for e in np.eye(KC.shape[0])])
    L = np.linalg.cholesky(KC)
    ev = np.linalg.eigvalsh(L.T @ (0.5 * (MC + MC.T)) @ L)
    assert ev[0] >= 1 - 1e-9


def test_adaptive_constraints_invariants():
    # variable coefficients make some faces need more than the average (Sect. 3.3)
    rng = np.random.default_rng(5)
    n = 8
    coef = np.exp(2.0 * rng.standard_normal((n, n, n)))
    m = make_mesh(n, 4, 1.08, 20.0, coef=coef)
    subs = dd.q1_substructures(m)
    A = subs.dense_schur()
    L = np.linalg.cholesky(A)
    N = len(subs.gamma)
    base = dd.Preconditioner(subs, 2, (dd.CORNER, dd.EDGE, dd.FACE), "diag")
    e0 = np.linalg.eigvalsh(L.T @ base.dense(N) @ L)
    counts, lmax = [], []
    for tau in (3.0, 2.0, 1.5):
        rows = dd.adaptive_face_constraints(subs, base.l1.D, tau=tau)
        counts.append(sum(len(r) for r in rows.values()))
        ad = dd.Preconditioner(subs, 2, (dd.CORNER, dd.EDGE, dd.FACE), "diag", extra_rows=rows)
        e1 = np.linalg.eigvalsh(L.T @ ad.dense(N) @ L)
        assert e1[0] >= 1 - 1e-10          # lambda_min >= 1 is kept (Sect. 3.2)
        assert e1[-1] <= e0[-1] + 1e-9     # added constraints cannot raise lambda_max
        lmax.append(e1[-1])
    assert counts[0] > 0
    # a smaller threshold adds at least the constraints of a larger one and lowers lambda_max
    assert counts[0] <= counts[1] <= counts[2]
    assert lmax[0] >= lmax[1] - 1e-9 >= lmax[2] - 2e-9
