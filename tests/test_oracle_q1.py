"""Pins for the oracle's Q1 discretization (Sect. 2, eq. 5) and its sparse Cholesky."""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import cholesky, q1
from workload import FACE_X1, make_mesh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_matrix(name):
    rows = [l.split() for l in open(os.path.join(GOLDEN, name)) if l.strip() and not l.startswith("#")]
    return np.array(rows, dtype=np.float64)


def test_cube_element_closed_form():
    ref = _golden_matrix("q1_cube_element.txt") / 12.0
    for h in (1.0, 0.37):
        K = q1.element_stiffness(h, h, h)
        assert np.allclose(K, h * ref, rtol=0, atol=1e-14 * h)


def test_brick_element_kronecker_form():
    # 1D stiffness/mass on [0,h]: (1/h)[[1,-1],[-1,1]], h[[1/3,1/6],[1/6,1/3]]; a brick is a sum of
    # Kronecker products (node a = ax + 2 ay + 4 az, so z is the slowest factor).
    K1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
    M1 = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    hx, hy, hz, k = 0.3, 0.05, 1.7, 2.5
    ref = k * ((hy * hz / hx) * np.kron(M1, np.kron(M1, K1)) + (hx * hz / hy) * np.kron(M1, np.kron(K1, M1))
               + (hx * hy / hz) * np.kron(K1, np.kron(M1, M1)))
    K = q1.element_stiffness(hx, hy, hz, k)
    assert np.allclose(K, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    assert np.allclose(K.sum(axis=1), 0.0, atol=1e-13 * np.abs(K).max())
    Kb = q1.element_stiffness_batch([hx], [hy], [hz], [k])[0]
    assert np.allclose(Kb, K, rtol=1e-14, atol=1e-14)
    Me = q1.element_mass(hx, hy, hz)
    assert np.allclose(Me, hx * hy * hz * np.kron(M1, np.kron(M1, M1)), rtol=1e-13)


def test_assembly_constant_nullspace_and_symmetry():
    m = make_mesh(6, 2, 1.08, 20.0, dirichlet=FACE_X1)
    K = q1.assemble(m)
    assert abs(K - K.T).max() < 1e-15
    # interior rows (not touching the removed Dirichlet layer) annihilate constants
    fmap = q1.free_index_map(m)
    rows = fmap[:, :, : m.nx - 1].ravel()
    assert np.abs((K @ np.ones(K.shape[0]))[rows]).max() < 1e-13


def _bisect(m):
    """Nested refinement: every element split in two along each axis."""
    from workload import Mesh
    mid = lambda c: np.sort(np.concatenate([c, 0.5 * (c[1:] + c[:-1])]))
    return Mesh(2 * m.nx, 2 * m.ny, 2 * m.nz, mid(m.xc), mid(m.yc), mid(m.zc), m.sub, m.dirichlet)


@pytest.mark.parametrize("ratio,aspect", [(1.0, None), (1.3, 8.0)])
def test_manufactured_solution_second_order(ratio, aspect):
    # p = cos(pi x/2) cos(pi y) cos(pi z): p = 0 on x=1, dp/dn = 0 on the other faces, -lap p = 9 pi^2/4 p
    p = lambda x, y, z: np.cos(np.pi * x / 2) * np.cos(np.pi * y) * np.cos(np.pi * z)
    f = lambda x, y, z: 9 * np.pi ** 2 / 4 * p(x, y, z)
    errs = []
    m = make_mesh(8, 4, ratio, aspect)
    for level in range(3):
        if level:
            m = _bisect(m)
        K = q1.assemble(m)
        x = cholesky.factor_mesh(m, K).solve(q1.load_vector(m, f))
        pts = m.free_node_coords()
        errs.append(np.abs(x - p(pts[:, 0], pts[:, 1], pts[:, 2])).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.4 < r1 < 4.6 and 3.4 < r2 < 4.6, errs


@pytest.mark.parametrize("n,leaf", [(3, 8), (4, 16), (5, 27)])
def test_cholesky_equals_dense(n, leaf):
    m = make_mesh(n, 1, 1.08, 20.0)
    K = q1.assemble(m)
    b = np.random.default_rng(n).standard_normal((K.shape[0], 2))
    x = cholesky.factor_mesh(m, K, leaf).solve(b)
    xd = np.linalg.solve(K.toarray(), b)
    assert np.allclose(x, xd, rtol=1e-12, atol=1e-12 * np.abs(xd).max())


def test_cholesky_residual_and_library_solve():
    m = make_mesh(16, 4, 1.08, 20.0)
    K = q1.assemble(m)
    b = np.random.default_rng(0).standard_normal(K.shape[0])
    ch = cholesky.factor_mesh(m, K)
    x = ch.solve(b)
    assert np.linalg.norm(K @ x - b) <= 1e-13 * np.linalg.norm(b)
    xs = spla.spsolve(K.tocsc(), b)
    assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)
