"""Writes graded64_coef_fd.txt: central finite differences, on the oracle, of the loss of the
differentiation workload (64^3 graded mesh, k_e = exp(g_e), g a seeded Gaussian random field).

Loss: L(g) = sum_t ||x_t(g) - target_t||^2 over T = 3 steps of the workload's right-hand-side
sequence, x_t = K(exp g)^{-1} f_t by the oracle's sparse Cholesky (exact solves), targets
seeded standard normal fields scaled to the solution's rms value.

Central differences with step h = 1e-6 along (a) a seeded random direction d of unit RMS per
element and (b) 16 seeded single elements. The difference of losses is evaluated as
sum_t (x_t^+ - x_t^-) . (x_t^+ + x_t^- - 2 target_t) / (2 h), algebraically the same as
(L(g + h d) - L(g - h d)) / (2 h) but free of the cancellation of two large losses.

Test infrastructure: calls only oracle/ and workload/. Run: python tests/golden/make_graded64_coef_fd.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import adjoint, cholesky  # noqa: E402
from workload import WORKLOADS, gaussian_random_field, load_sequence, make_mesh  # noqa: E402

T_STEPS = 3
H = 1e-6
DIR_SEED = 42
ELEM_SEED = 43
N_ELEM = 16


def problem():
    w = WORKLOADS["graded64_coef"]
    n = w["n"]
    g = gaussian_random_field(n, w["field_seed"])
    mesh = make_mesh(n, w["sub"], w["ratio"], w["max_aspect"], coef=np.exp(g))
    F = load_sequence(mesh, w["seed"], T_STEPS)
    return w, n, g, mesh, F


def targets(n_free, scale, seed):
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal((T_STEPS, n_free))


def solve_all(mesh_g, F):
    ch = cholesky.factor_mesh(mesh_g)
    return ch, [ch.solve(f) for f in F]


def main():
    w, n, g, mesh, F = problem()
    t0 = time.time()
    ch, X = solve_all(mesh, F)
    scale = float(np.sqrt(np.mean(np.square(X[0]))))
    tg = targets(mesh.n_free, scale, w["target_seed"])
    loss = sum(float(np.sum((X[t] - tg[t]) ** 2)) for t in range(T_STEPS))
    # oracle adjoint gradient with respect to g (for the record; the GPU test recomputes it)
    grad_g = np.zeros(n ** 3)
    for t in range(T_STEPS):
        _, gk = adjoint.adjoint(mesh, ch, X[t], 2 * (X[t] - tg[t]))
        grad_g += np.exp(g).ravel() * gk
    d = np.random.default_rng(DIR_SEED).standard_normal(n ** 3)
    elems = np.sort(np.random.default_rng(ELEM_SEED).choice(n ** 3, N_ELEM, replace=False))

    def fd(direction):
        xs = []
        for sgn in (+1.0, -1.0):
            gp = g.ravel() + sgn * H * direction
            m2 = make_mesh(n, w["sub"], w["ratio"], w["max_aspect"], coef=np.exp(gp).reshape(g.shape))
            xs.append(solve_all(m2, F)[1])
        return sum(float(np.dot(xs[0][t] - xs[1][t], xs[0][t] + xs[1][t] - 2 * tg[t])) for t in range(T_STEPS)) / (2 * H)

    rows = [("direction", -1, fd(d), float(np.dot(grad_g, d)))]
    for e in elems:
        u = np.zeros(n ** 3)
        u[e] = 1.0
        rows.append(("element", int(e), fd(u), float(grad_g[e])))
        print(rows[-1], time.time() - t0, flush=True)
    with open(os.path.join(HERE, "graded64_coef_fd.txt"), "w") as out:
        out.write("# Central finite differences of L(g) = sum_t ||x_t - target_t||^2 on the oracle (sparse Cholesky),\n")
        out.write(f"# 64^3 graded mesh of the differentiation workload, k = exp(g); T = {T_STEPS} steps, h = {H},\n")
        out.write(f"# direction seed {DIR_SEED} (standard normal per element), element seed {ELEM_SEED}, targets = "
                  f"rms(x_0) * N(0,1) with seed {w['target_seed']}.\n")
        out.write("# Written by tests/golden/make_graded64_coef_fd.py (oracle only). Columns: kind, element "
                  "(-1: direction), finite difference, oracle adjoint value.\n")
        out.write(f"target_scale {scale!r}\nloss {loss!r}\n")
        for kind, e, v, a in rows:
            out.write(f"{kind} {e} {v!r} {a!r}\n")
    print("done", time.time() - t0)


if __name__ == "__main__":
    main()
