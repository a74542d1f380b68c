"""Pins for the oracle's deflated PCG (Algorithm 1), recycling (Sect. 4.2) and adjoint."""
import numpy as np
import pytest

from oracle import adjoint, cholesky, dd, pcg, q1
from workload import load_sequence, make_mesh


@pytest.fixture(scope="module")
def problem():
    m = make_mesh(8, 4, 1.08, 20.0)
    subs = dd.q1_substructures(m)
    P = dd.Preconditioner(subs, 2, (dd.CORNER, dd.FACE), "diag")
    A = subs.dense_schur()
    M = P.dense(len(subs.gamma))
    F = load_sequence(m, 1, 6)
    bs = [subs.condense(f) for f in F]
    return m, subs, A, M, F, bs


def _textbook_pcg(A, M, b, x0, rtol, ref):
    """Hestenes-Stiefel PCG with dense matrices (independent restatement for the k=0 pin)."""
    x = x0.copy(); r = b - A @ x; z = M @ r; p = z.copy(); rz = r @ z; xs = [x.copy()]
    while np.linalg.norm(r) / ref >= rtol:
        q = A @ p; a = rz / (p @ q); x = x + a * p; r = r - a * q; xs.append(x.copy())
        if np.linalg.norm(r) / ref < rtol:
            break
        z = M @ r; rz2 = r @ z; p = z + (rz2 / rz) * p; rz = rz2
    return xs


def test_k0_equals_textbook_pcg(problem):
    m, subs, A, M, F, bs = problem
    b = bs[0]
    x, info = pcg.deflated_pcg(lambda v: A @ v, lambda v: M @ v, b, np.zeros_like(b), rtol=1e-10)
    xs = _textbook_pcg(A, M, b, np.zeros_like(b), 1e-10, np.linalg.norm(b))
    assert info.iters == len(xs) - 1
    assert np.allclose(x, xs[-1], rtol=1e-12, atol=1e-14 * np.abs(x).max())
    # converged solution equals the direct solve within the rtol-implied bound
    xe = np.linalg.solve(A, b)
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(x - xe) <= kappa * 1e-10 * np.linalg.norm(xe)


def test_stop_criteria_coincide_from_zero(problem):
    # from x0 = 0, r0 = b, so eqs. 17, 18 give the same iterations
    m, subs, A, M, F, bs = problem
    for b in bs[:3]:
        _, i1 = pcg.deflated_pcg(lambda v: A @ v, lambda v: M @ v, b, np.zeros_like(b), rtol=1e-8, stop="rhs")
        _, i2 = pcg.deflated_pcg(lambda v: A @ v, lambda v: M @ v, b, np.zeros_like(b), rtol=1e-8, stop="r0")
        assert i1.iters == i2.iters


def test_deflation_invariants(problem):
    m, subs, A, M, F, bs = problem
    Av, Mv = (lambda v: A @ v), (lambda v: M @ v)
    rng = np.random.default_rng(3)
    W = rng.standard_normal((A.shape[0], 5))
    x, info = pcg.deflated_pcg(Av, Mv, bs[1], rng.standard_normal(A.shape[0]), W, A @ W, rtol=1e-10)
    # W^T r_j = 0 and W^T A p_j = 0 (Sect. 4.1), checked on every stored vector
    nW = np.linalg.norm(W)
    for j in range(info.P.shape[1]):
        assert np.linalg.norm(W.T @ info.AP[:, j]) <= 1e-10 * nW * np.linalg.norm(info.AP[:, j])
    assert max(info.wtr) <= 1e-10 * nW * np.linalg.norm(bs[1])
    # search vectors are A-orthogonal
    Gp = info.P.T @ info.AP
    off = Gp - np.diag(np.diag(Gp))
    assert np.abs(off).max() <= 1e-8 * np.abs(np.diag(Gp)).max()
    xe = np.linalg.solve(A, bs[1])
    assert np.linalg.norm(x - xe) <= np.linalg.cond(A) * 1e-10 * np.linalg.norm(xe)


def test_deflation_space_containing_solution_needs_no_iteration(problem):
    m, subs, A, M, F, bs = problem
    b = bs[2]
    xe = np.linalg.solve(A, b)
    W = np.column_stack([xe, np.random.default_rng(0).standard_normal(len(b))])
    x, info = pcg.deflated_pcg(lambda v: A @ v, lambda v: M @ v, b, np.zeros_like(b), W, A @ W, rtol=1e-9)
    assert info.iters == 0
    assert np.allclose(x, xe, rtol=1e-9, atol=1e-12 * np.abs(xe).max())


def test_harmonic_ritz_values(problem):
    m, subs, A, M, F, bs = problem
    L = np.linalg.cholesky(A)
    lam = np.linalg.eigvalsh(L.T @ M @ L)  # spectrum of M^{-1}A (similar matrices)
    _, info = pcg.deflated_pcg(lambda v: A @ v, lambda v: M @ v, bs[0], np.zeros_like(bs[0]), rtol=1e-10)
    V = info.P
    theta, Y = pcg.harmonic_ritz(V, A @ V, M @ (A @ V))
    # Rayleigh quotients of M^{-1} relative to A^{-1}: inside [lambda_min, lambda_max] of M^{-1}A
    assert theta.min() >= lam[0] * (1 - 1e-10) and theta.max() <= lam[-1] * (1 + 1e-10)
    assert np.allclose(Y.T @ (V.T @ A @ V) @ Y, np.eye(len(theta)), atol=1e-8)
    # exact for an invariant subspace: V = eigenvectors of M^{-1}A
    ev, U = np.linalg.eigh(L.T @ M @ L)
    Vinv = np.linalg.solve(L.T, U[:, -4:])  # A-orthonormal eigenvectors of M A  (M^{-1}A in paper notation)
    th2, _ = pcg.harmonic_ritz(Vinv, A @ Vinv, M @ (A @ Vinv))
    assert np.allclose(np.sort(th2), np.sort(ev[-4:]), rtol=1e-9)


def test_b4_recycling_reduces_iterations_and_freezes():
    m = make_mesh(8, 4, 1.08, 20.0)
    subs = dd.q1_substructures(m)
    P = dd.Preconditioner(subs, 2, (dd.CORNER,), "diag")
    A = subs.dense_schur()
    M = P.dense(len(subs.gamma))
    F = load_sequence(m, 2, 12)
    bs = [subs.condense(f) for f in F]
    Av, Mv = (lambda v: A @ v), (lambda v: M @ v)
    _, inf0, _ = pcg.solve_sequence(Av, Mv, bs, R=0, rtol=1e-8)
    xs, inf4, rec = pcg.solve_sequence(Av, Mv, bs, R=8, strategy="B4", rtol=1e-8)
    its0 = np.array([i.iters for i in inf0])
    its4 = np.array([i.iters for i in inf4])
    assert its4[0] == its0[0]               # the first solve has no deflation space
    assert its4[1:].sum() < its0[1:].sum()  # B4 recycling cuts iterations (Sect. 4.2)
    for x, b in zip(xs, bs):
        assert np.linalg.norm(A @ x - b) <= 1.001e-8 * np.linalg.norm(b)
    # the retained Ritz values are the largest ones, all >= 1 (BDDC spectrum, Sect. 3.2)
    assert rec.theta.min() >= 1 - 1e-8
    for strat in ("B1", "B2", "B3"):
        xs2, inf, _ = pcg.solve_sequence(Av, Mv, bs, R=8, strategy=strat, rtol=1e-8)
        for x, b in zip(xs2, bs):
            assert np.linalg.norm(A @ x - b) <= 1.001e-8 * np.linalg.norm(b)


def test_adjoint_central_differences():
    rng = np.random.default_rng(11)
    n = 4
    coef = np.exp(rng.standard_normal((n, n, n)))
    m = make_mesh(n, 2, 1.08, 20.0, coef=coef)
    f = load_sequence(m, 4, 1)[0]
    target = rng.standard_normal(m.n_free)

    def loss(mm, ff):
        x = cholesky.factor_mesh(mm, leaf=16).solve(ff)
        return np.sum((x - target) ** 2), x

    L0, x = loss(m, f)
    ch = cholesky.factor_mesh(m, leaf=16)
    gf, gk = adjoint.adjoint(m, ch, x, 2 * (x - target))
    h = 1e-6
    for i in rng.choice(m.n_free, 5, replace=False):
        e = np.zeros_like(f); e[i] = h
        fd = (loss(m, f + e)[0] - loss(m, f - e)[0]) / (2 * h)
        assert abs(fd - gf[i]) <= 1e-6 * max(1.0, abs(gf[i]))
    for e_idx in rng.choice(n ** 3, 5, replace=False):
        cp, cm = coef.copy().ravel(), coef.copy().ravel()
        cp[e_idx] += h; cm[e_idx] -= h
        mp = make_mesh(n, 2, 1.08, 20.0, coef=cp.reshape(coef.shape))
        mm = make_mesh(n, 2, 1.08, 20.0, coef=cm.reshape(coef.shape))
        fd = (loss(mp, f)[0] - loss(mm, f)[0]) / (2 * h)
        assert abs(fd - gk[e_idx]) <= 1e-6 * max(1.0, abs(gk[e_idx]))
    # dense adjoint restatement: lambda = K^{-1} g
    K = q1.assemble(m).toarray()
    assert np.allclose(gf, np.linalg.solve(K, 2 * (x - target)), rtol=1e-10)
