"""Q1 (trilinear) finite elements for the pressure Poisson problem (oracle; test infrastructure).

The pressure space is continuous piecewise trilinear on hexahedra (Sect. 2,
Taylor-Hood Q2-Q1, pressure part), and the Poisson problem for the pressure
corrector with Dirichlet data on the outflow part and Neumann data elsewhere
gives the SPD system K x = f (eq. 5).

Written from the definition: K_ab = sum_e int_e k_e grad(phi_a) . grad(phi_b) dx,
integrated on each brick by 2x2x2 Gauss quadrature (exact for these integrands).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# local node a = ax + 2*ay + 4*az, (ax, ay, az) in {0,1}^3
_LOCAL = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)])


def element_stiffness(hx: float, hy: float, hz: float, k: float = 1.0) -> np.ndarray:
    """8x8 stiffness matrix of the brick [0,hx]x[0,hy]x[0,hz] with coefficient k.

    Integrates k grad(phi_a).grad(phi_b) with 2-point Gauss rules per axis.
    """
    g = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])  # on [0,1]
    h = np.array([hx, hy, hz])
    Ke = np.zeros((8, 8))
    for qx in g:
        for qy in g:
            for qz in g:
                q = np.array([qx, qy, qz])
                grads = np.zeros((8, 3))
                for a in range(8):
                    s = _LOCAL[a]
                    # phi_a(q) = prod_d (s_d ? q_d : 1 - q_d) in reference coordinates
                    f = np.where(s == 1, q, 1.0 - q)
                    df = np.where(s == 1, 1.0, -1.0) / h  # derivative in physical coordinates
                    grads[a] = [df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2]]
                Ke += (k * hx * hy * hz / 8.0) * grads @ grads.T
    return Ke


def element_mass(hx: float, hy: float, hz: float) -> np.ndarray:
    """8x8 consistent mass matrix of the brick (2x2x2 Gauss, exact)."""
    g = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    Me = np.zeros((8, 8))
    for qx in g:
        for qy in g:
            for qz in g:
                q = np.array([qx, qy, qz])
                phi = np.array([np.prod(np.where(_LOCAL[a] == 1, q, 1.0 - q)) for a in range(8)])
                Me += (hx * hy * hz / 8.0) * np.outer(phi, phi)
    return Me


def element_stiffness_batch(hx, hy, hz, k=None) -> np.ndarray:
    """[E, 8, 8] stiffness matrices of bricks with sizes (hx[e], hy[e], hz[e]) and coefficients k[e].

    Same 2x2x2 Gauss quadrature of k grad(phi_a).grad(phi_b) as `element_stiffness`,
    evaluated for all elements at once.
    """
    hx, hy, hz = (np.asarray(v, dtype=np.float64) for v in (hx, hy, hz))
    E = hx.shape[0]
    h = np.stack([hx, hy, hz], axis=1)  # [E,3]
    g = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    sgn = np.where(_LOCAL == 1, 1.0, -1.0)  # [8,3]
    Ke = np.zeros((E, 8, 8))
    vol = (hx * hy * hz / 8.0)[:, None, None]
    for qx in g:
        for qy in g:
            for qz in g:
                q = np.array([qx, qy, qz])
                f = np.where(_LOCAL == 1, q, 1.0 - q)  # [8,3] basis factors per axis
                grads = np.empty((E, 8, 3))
                grads[:, :, 0] = (sgn[:, 0] * f[:, 1] * f[:, 2])[None, :] / h[:, 0:1]
                grads[:, :, 1] = (f[:, 0] * sgn[:, 1] * f[:, 2])[None, :] / h[:, 1:2]
                grads[:, :, 2] = (f[:, 0] * f[:, 1] * sgn[:, 2])[None, :] / h[:, 2:3]
                Ke += vol * np.einsum("ead,ebd->eab", grads, grads)
    if k is not None:
        Ke *= np.asarray(k, dtype=np.float64)[:, None, None]
    return Ke


def free_index_map(mesh) -> np.ndarray:
    """Array [nz+1][ny+1][nx+1] giving the free-node index of each mesh node, -1 if Dirichlet."""
    x0, x1, y0, y1, z0, z1 = mesh.free_box
    idx = -np.ones((mesh.nz + 1, mesh.ny + 1, mesh.nx + 1), dtype=np.int64)
    nxf, nyf = x1 - x0, y1 - y0
    zz, yy, xx = np.meshgrid(np.arange(z0, z1), np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
    idx[zz, yy, xx] = (xx - x0) + nxf * ((yy - y0) + nyf * (zz - z0))
    return idx


def element_arrays(mesh, with_coef: bool = False):
    """Per-element free-node indices [E, 8] (-1 for Dirichlet) and 8x8 matrices [E, 8, 8].

    Elements are ordered x fastest; local node a = ax + 2 ay + 4 az. The matrices
    are K_e^0 (coefficient 1) unless with_coef, then k_e K_e^0.
    """
    fmap = free_index_map(mesh)
    ez, ey, ex = np.meshgrid(np.arange(mesh.nz), np.arange(mesh.ny), np.arange(mesh.nx), indexing="ij")
    ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
    conn = np.empty((ex.size, 8), dtype=np.int64)
    for a in range(8):
        s = _LOCAL[a]
        conn[:, a] = fmap[ez + s[2], ey + s[1], ex + s[0]]
    hx, hy, hz = np.diff(mesh.xc), np.diff(mesh.yc), np.diff(mesh.zc)
    k = None
    if with_coef and mesh.coef is not None:
        k = np.asarray(mesh.coef, dtype=np.float64).ravel()
    Ke = element_stiffness_batch(hx[ex], hy[ey], hz[ez], k)
    return conn, Ke


def assemble(mesh) -> sp.csr_matrix:
    """Global stiffness K on the free nodes (Dirichlet rows/columns removed), CSR, float64."""
    conn, Ke = element_arrays(mesh, with_coef=True)
    rows = np.broadcast_to(conn[:, :, None], Ke.shape).ravel()
    cols = np.broadcast_to(conn[:, None, :], Ke.shape).ravel()
    vals = Ke.ravel()
    keep = (rows >= 0) & (cols >= 0)
    n = mesh.n_free
    K = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(n, n))
    return K.tocsr()


def load_vector(m, f) -> np.ndarray:
    """Consistent load vector b_i = integral of f phi_i over the free nodes' hat functions
    (trilinear phi_i), by 3x3x3 Gauss quadrature per brick; f is a callable f(x, y, z) on
    arrays (manufactured-solution checks of the discretization, Sect. 2)."""
    gp = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)]) * 0.5 + 0.5
    gw = np.array([5 / 9, 8 / 9, 5 / 9]) * 0.5
    conn, _ = element_arrays(m)
    ez, ey, ex = np.meshgrid(np.arange(m.nz), np.arange(m.ny), np.arange(m.nx), indexing="ij")
    ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
    x0, hx = m.xc[ex], np.diff(m.xc)[ex]
    y0, hy = m.yc[ey], np.diff(m.yc)[ey]
    z0, hz = m.zc[ez], np.diff(m.zc)[ez]
    b = np.zeros(m.n_free)
    for i, qx in enumerate(gp):
        for j, qy in enumerate(gp):
            for k, qz in enumerate(gp):
                w = gw[i] * gw[j] * gw[k] * hx * hy * hz
                fv = f(x0 + qx * hx, y0 + qy * hy, z0 + qz * hz) * w
                for a in range(8):
                    sx, sy, sz = a & 1, (a >> 1) & 1, (a >> 2) & 1
                    phi = (qx if sx else 1 - qx) * (qy if sy else 1 - qy) * (qz if sz else 1 - qz)
                    c = conn[:, a]
                    ok = c >= 0
                    np.add.at(b, c[ok], (fv * phi)[ok])
    return b
