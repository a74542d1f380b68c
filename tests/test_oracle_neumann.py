"""Pins for the oracle's pure-Neumann variant (no Dirichlet face; Sect. 2 and 4.1):
null space of K, the grounded solve against the pseudo-inverse, a manufactured solution,
the interface problem's null space and consistency, BDDC with a grounded coarse problem,
and Algorithm 1 with the constants in the deflation basis."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import dd, neumann, q1
from workload import load_sequence, make_mesh

KINDS = (dd.CORNER, dd.EDGE, dd.FACE)


def _mesh(n, sub, ratio=1.08, aspect=20.0):
    return make_mesh(n, sub, ratio, aspect, dirichlet=0)


def test_stiffness_null_space_is_the_constants():
    m = _mesh(3, 1)
    K = q1.assemble(m).toarray()
    assert np.abs(K - K.T).max() < 1e-15
    assert np.abs(K @ np.ones(K.shape[0])).max() < 1e-13 * np.abs(K).max()
    lam = np.linalg.eigvalsh(K)
    assert abs(lam[0]) < 1e-12 * lam[-1]          # semidefinite ...
    assert lam[1] > 1e-4 * lam[-1]                 # ... with a one-dimensional null space (connected mesh)


@pytest.mark.parametrize("n,ratio", [(4, 1.0), (5, 1.3)])
def test_grounded_solve_equals_pseudo_inverse(n, ratio):
    m = _mesh(n, 1, ratio)
    K = q1.assemble(m)
    f = np.random.default_rng(n).standard_normal(K.shape[0])
    x = neumann.Solver(m, K).solve(f)
    xp = np.linalg.pinv(K.toarray(), rcond=1e-10, hermitian=True) @ f  # minimum-norm solution
    assert np.allclose(x, xp, rtol=0, atol=1e-10 * np.abs(xp).max())
    fc = neumann.consistent(f)
    assert abs(fc.sum()) < 1e-12 * np.abs(f).sum()
    assert np.linalg.norm(K @ x - fc) <= 1e-12 * np.linalg.norm(fc)
    assert abs(x.mean()) < 1e-14 * np.abs(x).max()


def _bisect(m):
    from workload import Mesh
    mid = lambda c: np.sort(np.concatenate([c, 0.5 * (c[1:] + c[:-1])]))
    return Mesh(2 * m.nx, 2 * m.ny, 2 * m.nz, mid(m.xc), mid(m.yc), mid(m.zc), m.sub, m.dirichlet)


@pytest.mark.parametrize("ratio,aspect", [(1.0, None), (1.3, 8.0)])
def test_manufactured_solution_second_order(ratio, aspect):
    # p = cos(pi x) cos(pi y) cos(pi z): dp/dn = 0 on every face of the unit cube,
    # -lap p = 3 pi^2 p; the discrete solution is defined up to a constant, so both sides
    # are compared with their nodal means removed
    p = lambda x, y, z: np.cos(np.pi * x) * np.cos(np.pi * y) * np.cos(np.pi * z)
    f = lambda x, y, z: 3 * np.pi ** 2 * p(x, y, z)
    errs = []
    m = make_mesh(8, 4, ratio, aspect, dirichlet=0)
    for level in range(3):
        if level:
            m = _bisect(m)
        x = neumann.Solver(m).solve(q1.load_vector(m, f))
        pts = m.free_node_coords()
        pe = p(pts[:, 0], pts[:, 1], pts[:, 2])
        errs.append(np.abs(x - (pe - pe.mean())).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.4 < r1 < 4.6 and 3.4 < r2 < 4.6, errs


@pytest.fixture(scope="module")
def problem():
    m = _mesh(12, 4, 1.2, 20.0)
    subs = dd.q1_substructures(m)
    K = q1.assemble(m)
    return m, subs, K, neumann.Solver(m, K)


def test_interface_problem_null_space_and_consistency(problem):
    m, subs, K, ns = problem
    A = subs.dense_schur()
    one = np.ones(len(subs.gamma))
    assert np.abs(A @ one).max() < 1e-12 * np.abs(A).max()       # null(A) = constants on the interface
    f = neumann.consistent(load_sequence(m, 3, 1)[0])
    b = subs.condense(f)
    assert abs(one @ b) < 1e-12 * np.abs(b).sum()                # consistent condensed right-hand side
    x = ns.solve(f)
    xg = x[subs.gamma]
    assert np.linalg.norm(A @ xg - b) <= 1e-10 * np.linalg.norm(b)
    # recovery from the interface values gives the full solution (any constant carries over)
    c = 0.37
    xr = subs.recover(f, xg + c)
    assert np.allclose(xr - c, x, rtol=0, atol=1e-10 * np.abs(x).max())


def test_bddc_coarse_basis_reproduces_constants_and_bound(problem):
    m, subs, K, ns = problem
    Pc = neumann.Preconditioner(subs, KINDS)
    for i in range(subs.S):
        Phi, C = Pc.l1.Phi[i], Pc.l1.C[i]
        assert np.allclose(C @ Phi, np.eye(C.shape[0]), atol=1e-10)
        assert np.allclose(Phi @ np.ones(Phi.shape[1]), 1.0, atol=1e-10)   # constants are coarse functions
    n = len(subs.gamma)
    A = subs.dense_schur()
    # on the complement of the constants, lambda_min(M^{-1} A) >= 1
    Q = sla.null_space(np.ones((1, n)))
    Pr = neumann.null_projector(np.ones(n))
    M = np.column_stack([Pr(Pc.apply(Q[:, j])) for j in range(n - 1)])
    Mq = Q.T @ M
    Mq = 0.5 * (Mq + Mq.T)
    lam = sla.eigh(Q.T @ A @ Q, np.linalg.inv(Mq), eigvals_only=True)
    assert lam.min() >= 1 - 1e-10


def test_deflated_pcg_converges_to_the_mean_free_solution(problem):
    m, subs, K, ns = problem
    Pc = neumann.Preconditioner(subs, KINDS)
    F = [neumann.consistent(f) for f in load_sequence(m, 5, 4)]
    bs = [subs.condense(f) for f in F]
    xs, infos, rec = neumann.solve_sequence(subs.schur_apply, Pc.apply, bs, R=6, strategy="B4", rtol=1e-10)
    one = np.ones(len(subs.gamma))
    for f, xg, info in zip(F, xs, infos):
        x = ns.solve(f)
        xo = x[subs.gamma] - x[subs.gamma].mean()                  # mean-free interface representative
        assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)
        assert abs(one @ xg) < 1e-12 * np.abs(xg).sum()
        assert np.abs(one @ info.P).max() < 1e-10 * np.abs(info.P).max()   # search directions orthogonal to 1
    assert rec.W.shape[1] == 6 and np.abs(one @ rec.W).max() < 1e-10 * np.abs(rec.W).max()
    assert infos[-1].iters < infos[0].iters                            # the recycled basis deflates
