"""The differentiation workload at its stated size: 64^3 graded mesh, k_e = exp(g_e) with g a
seeded Gaussian random field, 512 subdomains, three-level BDDC, B4 recycling with k = 20 over
the forward sequence, mixed precision (df64 Schur operator, FP32 BDDC, flexible PCG).

The backward pass is the adjoint solve with the same operator and preconditioner, deflated
by the basis recycled over the forward steps. Checked through the C ABI:
  * dL/df_t = lambda_t and dL/dg (summed over the steps, with k = exp(g) applied in the
    library) against the oracle's adjoint (sparse Cholesky) on the full vectors;
  * the directional derivative along a seeded direction and 16 seeded single elements
    against central finite differences of the loss on the oracle, stored in
    tests/golden/graded64_coef_fd.txt by tests/golden/make_graded64_coef_fd.py;
  * the autograd wrapper gives the same gradients and refuses a coefficient field that is
    not the one the solver was set up with.
"""
import os

import numpy as np
import pytest

from oracle import adjoint, cholesky
from workload import WORKLOADS, gaussian_random_field, load_sequence, make_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2412_17543_gb300 as P  # noqa: E402

DEV = "cuda:0"
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "graded64_coef_fd.txt")
T_STEPS = 3


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _golden():
    rows, meta = [], {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] in ("target_scale", "loss"):
            meta[f[0]] = float(f[1])
        else:
            rows.append((f[0], int(f[1]), float(f[2]), float(f[3])))
    return meta, rows


@pytest.fixture(scope="module")
def case():
    w = WORKLOADS["graded64_coef"]
    n = w["n"]
    g = gaussian_random_field(n, w["field_seed"])
    mesh = make_mesh(n, w["sub"], w["ratio"], w["max_aspect"], coef=np.exp(g))
    F = load_sequence(mesh, w["seed"], T_STEPS)
    meta, rows = _golden()
    tg = meta["target_scale"] * np.random.default_rng(w["target_seed"]).standard_normal((T_STEPS, mesh.n_free))
    ch = cholesky.factor_mesh(mesh)
    Xo = [ch.solve(f) for f in F]
    lam_o, grad_o = [], np.zeros(n ** 3)
    for t in range(T_STEPS):
        lo, gk = adjoint.adjoint(mesh, ch, Xo[t], 2 * (Xo[t] - tg[t]))
        lam_o.append(lo)
        grad_o += np.exp(g).ravel() * gk
    S = P.Solver(mesh, levels=3, coarse_group=4, use_corners=1, use_edges=1, use_faces=1, weights="diag",
                 schur_prec="df64", precond_prec="fp32", flexible=1)
    yield dict(w=w, n=n, g=g, mesh=mesh, F=F, tg=tg, Xo=Xo, lam_o=lam_o, grad_o=grad_o, rows=rows, meta=meta, S=S)
    S.close()


def test_adjoint_deflated_by_forward_basis_matches_oracle_and_fd(case):
    S, F, tg, n = case["S"], case["F"], case["tg"], case["n"]
    rec = S.recycler(20, "B4")
    X = []
    for t in range(T_STEPS):
        x, st = S.solve(T(F[t]), rec, rtol=1e-10)
        X.append(x)
        err = np.linalg.norm(x.cpu().numpy() - case["Xo"][t]) / np.linalg.norm(case["Xo"][t])
        assert err <= 1e-8, (t, err)
    assert rec.state()["k"] > 0  # the backward pass is deflated by the forward basis
    grad = torch.zeros(n ** 3, dtype=torch.float64, device=DEV)
    for t in reversed(range(T_STEPS)):
        gf, gg, st = S.adjoint(2 * (X[t] - T(tg[t])), X[t], rec, 1e-10, log_coef=True)
        assert st["recycled_k"] > 0
        lam_o = case["lam_o"][t]
        assert np.linalg.norm(gf.cpu().numpy() - lam_o) <= 1e-7 * np.linalg.norm(lam_o), t
        grad += gg
    grad = grad.cpu().numpy()
    go = case["grad_o"]
    assert np.linalg.norm(grad - go) <= 1e-7 * np.linalg.norm(go)
    # central finite differences on the oracle (directional and 16 single elements). A single
    # element's derivative is small next to the rounding of two independent factorizations
    # (about kappa * eps * ||x|| in each solution), which leaves the finite difference itself
    # noisy at up to ~1e-3 relative; the GPU gradient must agree with it as closely as the
    # oracle's exact adjoint does, up to the GPU-vs-oracle tolerance
    d = np.random.default_rng(42).standard_normal(n ** 3)
    for kind, e, fd, oracle_val in case["rows"]:
        val = float(np.dot(grad, d)) if kind == "direction" else float(grad[e])
        assert abs(oracle_val - fd) <= 1e-3 * abs(fd), (kind, e, oracle_val, fd)  # the FD noise level
        slack = 1e-6 * abs(fd) + (1e-7 * np.linalg.norm(go) * np.linalg.norm(d) if kind == "direction"
                                  else 1e-7 * np.linalg.norm(go))
        assert abs(val - fd) <= abs(oracle_val - fd) + slack, (kind, e, val, oracle_val, fd)


def test_autograd_wrapper_matches_and_refuses_another_field(case):
    S, F, tg, g = case["S"], case["F"], case["tg"], case["g"]
    rec = S.recycler(20, "B4")
    fT = T(F[0]).requires_grad_(True)
    gT = T(g).requires_grad_(True)
    x = P.PoissonSolve.apply(fT, gT, S, rec, 1e-10, 1e-10)
    loss = ((x - T(tg[0])) ** 2).sum()
    loss.backward()
    lam_o = case["lam_o"][0]
    assert np.linalg.norm(fT.grad.cpu().numpy() - lam_o) <= 1e-7 * np.linalg.norm(lam_o)
    # the single-step gradient with respect to g: k_e times the oracle's coefficient gradient
    g0 = np.exp(g).ravel() * adjoint.coefficient_gradient(case["mesh"], case["Xo"][0], lam_o)
    assert np.linalg.norm(gT.grad.cpu().numpy().ravel() - g0) <= 1e-7 * np.linalg.norm(g0)
    # a field the solver was not set up with is refused (its operator is fixed at setup)
    g2 = T(g + 1e-3)
    with pytest.raises(ValueError):
        P.PoissonSolve.apply(T(F[0]), g2.requires_grad_(True), S, rec, 1e-10, 1e-10)
