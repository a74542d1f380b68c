"""Seeded synthetic inputs for the Poisson-sequence workloads.

This module is the only code shared by the oracle and the CUDA path: it builds
the inputs (mesh coordinates, partition sizes, coefficient fields, right-hand
side sequences) and holds none of the solver's arithmetic.

The paper's workload (pressure-corrector Poisson solves behind a sphere, Sect. 6)
needs Navier-Stokes flow data that is not available, so these generators stand
in for it with the structure that matters to the solver: one constant SPD
matrix (Q1 Laplacian, Dirichlet p=0 on the outflow face x=1, Neumann elsewhere,
as for the pressure corrector in Sect. 2) and a slowly varying right-hand side
(advected Gaussian bumps plus white noise, time step 0.05 as in Sect. 6).

Node numbering used everywhere: a mesh with nx*ny*nz hexahedral elements has
(nx+1)*(ny+1)*(nz+1) nodes; nodes on Dirichlet faces are removed, the remaining
("free") nodes form a box [x0,x1)x[y0,y1)x[z0,z1) of node indices and are
numbered lexicographically with x fastest.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Dirichlet face bits: x=0, x=1, y=0, y=1, z=0, z=1
FACE_X0, FACE_X1, FACE_Y0, FACE_Y1, FACE_Z0, FACE_Z1 = 1, 2, 4, 8, 16, 32


@dataclass
class Mesh:
    """Tensor-product hexahedral mesh of the unit cube with a block partition."""
    nx: int
    ny: int
    nz: int
    xc: np.ndarray  # node coordinates per axis, float64 [nx+1]
    yc: np.ndarray
    zc: np.ndarray
    sub: tuple      # elements per subdomain per axis (sx, sy, sz)
    dirichlet: int = FACE_X1
    coef: np.ndarray | None = None   # per-element coefficient k_e [nz][ny][nx] (x fastest) or None (=1)
    name: str = ""
    info: dict = field(default_factory=dict)

    @property
    def free_box(self):
        """Half-open node index box of the free (non-Dirichlet) nodes."""
        d = self.dirichlet
        x0 = 1 if d & FACE_X0 else 0
        x1 = self.nx if d & FACE_X1 else self.nx + 1
        y0 = 1 if d & FACE_Y0 else 0
        y1 = self.ny if d & FACE_Y1 else self.ny + 1
        z0 = 1 if d & FACE_Z0 else 0
        z1 = self.nz if d & FACE_Z1 else self.nz + 1
        return (x0, x1, y0, y1, z0, z1)

    @property
    def n_free(self) -> int:
        x0, x1, y0, y1, z0, z1 = self.free_box
        return (x1 - x0) * (y1 - y0) * (z1 - z0)

    def free_node_coords(self) -> np.ndarray:
        """Coordinates [n_free, 3] of the free nodes in free-node order."""
        x0, x1, y0, y1, z0, z1 = self.free_box
        Z, Y, X = np.meshgrid(self.zc[z0:z1], self.yc[y0:y1], self.xc[x0:x1], indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def n_subdomains(self) -> int:
        sx, sy, sz = self.sub
        return (self.nx // sx) * (self.ny // sy) * (self.nz // sz)


def graded_coords(n: int, ratio: float, max_aspect: float | None) -> tuple[np.ndarray, float]:
    """Node coordinates on [0,1] for n elements graded geometrically toward the centre.

    Element i has size proportional to r**d_i with d_i = |i - (n-1)/2| - 1/2, so the
    two central elements are the finest; r = ratio, lowered so that the largest
    to smallest element size ratio r**(n/2-1) does not exceed max_aspect.
    Returns (coords[n+1], r).
    """
    if ratio == 1.0 or n < 4:
        return np.linspace(0.0, 1.0, n + 1), 1.0
    r = ratio
    if max_aspect is not None:
        r = min(ratio, max_aspect ** (1.0 / (n / 2 - 1)))
    d = np.abs(np.arange(n) - (n - 1) / 2.0) - 0.5
    h = r ** d
    h /= h.sum()
    c = np.concatenate([[0.0], np.cumsum(h)])
    c[-1] = 1.0
    return c, r


def make_mesh(n: int, sub: int, ratio: float = 1.0, max_aspect: float | None = None,
              dirichlet: int = FACE_X1, coef: np.ndarray | None = None, name: str = "") -> Mesh:
    c, r = graded_coords(n, ratio, max_aspect)
    h = np.diff(c)
    aspect = float(h.max() / h.min())
    return Mesh(n, n, n, c.copy(), c.copy(), c.copy(), (sub, sub, sub), dirichlet, coef, name,
                {"ratio": r, "max_aspect": aspect})


def gaussian_random_field(n: int, seed: int, corr_len: float = 0.1, std: float = 1.0) -> np.ndarray:
    """Per-element Gaussian random field g_e on a uniform n^3 element grid.

    Squared-exponential covariance with the given correlation length, realised by
    FFT filtering of seeded white noise on a periodic grid padded 2x per axis,
    sampled at element centroids (index space) and rescaled to sample std `std`.
    Returns g[nz][ny][nx] (x fastest), float64.
    """
    rng = np.random.default_rng(seed)
    m = 2 * n
    noise = rng.standard_normal((m, m, m))
    k = np.fft.fftfreq(m, d=1.0 / m)  # integer wave numbers on the padded period (length 2)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    # physical period of the padded grid is 2 (unit cube doubled); omega = pi*k
    w2 = (np.pi ** 2) * (kx ** 2 + ky ** 2 + kz ** 2)
    filt = np.exp(-0.25 * corr_len ** 2 * w2)  # sqrt of the SE spectral density (up to scale)
    g = np.real(np.fft.ifftn(np.fft.fftn(noise) * filt))[:n, :n, :n]
    g = g - g.mean()
    g = g / g.std() * std
    return np.ascontiguousarray(g)


# ---------------------------------------------------------------------------
# Right-hand sides: advected Gaussian bumps + white noise, lumped nodal volumes
# ---------------------------------------------------------------------------

@dataclass
class BumpSequence:
    """f_t(x) = sum_m a_m exp(-|x - c_m(t)|^2 / (2 w_m^2)), c_m(t) advected periodically."""
    seed: int
    nbumps: int = 8
    dt: float = 0.05
    speed: float = 0.5
    noise: float = 1e-3

    def __post_init__(self):
        rng = np.random.default_rng(self.seed)
        self.a = rng.standard_normal(self.nbumps)
        self.w = rng.uniform(0.05, 0.2, self.nbumps)
        self.c0 = rng.uniform(0.0, 1.0, (self.nbumps, 3))
        v = rng.standard_normal((self.nbumps, 3))
        self.v = self.speed * v / np.linalg.norm(v, axis=1, keepdims=True)

    def centres(self, t: int) -> np.ndarray:
        return np.mod(self.c0 + self.v * (t * self.dt), 1.0)

    def f(self, pts: np.ndarray, t: int) -> np.ndarray:
        c = self.centres(t)
        out = np.zeros(pts.shape[0])
        for m in range(self.nbumps):
            d2 = np.sum((pts - c[m]) ** 2, axis=1)
            out += self.a[m] * np.exp(-d2 / (2.0 * self.w[m] ** 2))
        return out

    def f_grid(self, xs: np.ndarray, ys: np.ndarray, zs: np.ndarray, t: int) -> np.ndarray:
        """f_t on the tensor grid zs x ys x xs (x fastest), using that each bump is a
        product of one-dimensional Gaussians."""
        c = self.centres(t)
        out = np.zeros((len(zs), len(ys), len(xs)))
        for m in range(self.nbumps):
            s2 = 2.0 * self.w[m] ** 2
            gx = np.exp(-((xs - c[m, 0]) ** 2) / s2)
            gy = np.exp(-((ys - c[m, 1]) ** 2) / s2)
            gz = self.a[m] * np.exp(-((zs - c[m, 2]) ** 2) / s2)
            out += gz[:, None, None] * (gy[:, None] * gx[None, :])[None, :, :]
        return out.ravel()


def lumped_nodal_volumes(mesh: Mesh) -> np.ndarray:
    """Volume share of each free node: product over axes of half the adjacent element sizes."""
    def axis_vol(c, lo, hi):
        h = np.diff(c)
        v = np.zeros(len(c))
        v[:-1] += 0.5 * h
        v[1:] += 0.5 * h
        return v[lo:hi]
    x0, x1, y0, y1, z0, z1 = mesh.free_box
    vx, vy, vz = axis_vol(mesh.xc, x0, x1), axis_vol(mesh.yc, y0, y1), axis_vol(mesh.zc, z0, z1)
    return (vz[:, None, None] * vy[None, :, None] * vx[None, None, :]).ravel()


def load_vector(mesh: Mesh, seq: BumpSequence, t: int, _cache: dict | None = None) -> np.ndarray:
    """b_i = V_i (f_t(x_i) + noise * xi_{t,i}) on the free nodes (float64)."""
    pts = mesh.free_node_coords()
    vol = lumped_nodal_volumes(mesh)
    xi = np.random.default_rng([seq.seed, t, 7]).standard_normal(pts.shape[0])
    return vol * (seq.f(pts, t) + seq.noise * xi)


def load_sequence(mesh: Mesh, seed: int, steps: int, start: int = 0) -> np.ndarray:
    """[steps, n_free] float64 load vectors for t = start .. start+steps-1."""
    seq = BumpSequence(seed)
    x0, x1, y0, y1, z0, z1 = mesh.free_box
    xs, ys, zs = mesh.xc[x0:x1], mesh.yc[y0:y1], mesh.zc[z0:z1]
    vol = lumped_nodal_volumes(mesh)
    out = np.empty((steps, vol.shape[0]))
    for i in range(steps):
        t = start + i
        xi = np.random.default_rng([seq.seed, t, 7]).standard_normal(vol.shape[0])
        out[i] = vol * (seq.f_grid(xs, ys, zs, t) + seq.noise * xi)
    return out


# ---------------------------------------------------------------------------
# Named workloads (sizes, grading, partition, solver options)
# ---------------------------------------------------------------------------

WORKLOADS = {
    # uniform 16^3, 64 subdomains of 4^3, two-level BDDC corners + face averages, plain PCG
    "cube16": dict(n=16, sub=4, ratio=1.0, max_aspect=None, levels=2, corners=1, edges=0, faces=1,
                   adaptive=0, k=0, rtol=1e-8, steps=10, seed=1),
    # 64^3 graded (1.08, aspect <= 20), 512 subdomains, three-level, k=20
    "graded64": dict(n=64, sub=8, ratio=1.08, max_aspect=20.0, levels=3, corners=1, edges=1, faces=1,
                     adaptive=0, k=20, rtol=1e-8, steps=200, seed=2),
    # 128^3 graded (aspect <= 40), 4096 subdomains, three-level + adaptive tau=10, k=40
    "graded128": dict(n=128, sub=8, ratio=1.08, max_aspect=40.0, levels=3, corners=1, edges=1, faces=1,
                      adaptive=1, tau=10.0, k=40, rtol=1e-8, steps=500, seed=3),
    # 64^3 graded with k_e = exp(g_e), gradients
    "graded64_coef": dict(n=64, sub=8, ratio=1.08, max_aspect=20.0, levels=3, corners=1, edges=1, faces=1,
                          adaptive=0, k=20, rtol=1e-8, steps=50, seed=4, field_seed=40, target_seed=41),
    # 96^3 graded, 1728 subdomains, 32-member ensemble
    "graded96_ens": dict(n=96, sub=8, ratio=1.08, max_aspect=40.0, levels=3, corners=1, edges=1, faces=1,
                         adaptive=0, k=40, rtol=1e-8, steps=100, seed=500, nrhs=32),
}


def workload_mesh(name: str, n: int | None = None, sub: int | None = None) -> Mesh:
    """Mesh of a named workload (optionally with n/sub overridden for small test cases)."""
    w = WORKLOADS[name]
    nn = n if n is not None else w["n"]
    ss = sub if sub is not None else w["sub"]
    coef = None
    if "field_seed" in w:
        coef = np.exp(gaussian_random_field(nn, w["field_seed"]))
    return make_mesh(nn, ss, w["ratio"], w["max_aspect"], FACE_X1, coef, name)
