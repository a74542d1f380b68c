"""Full-size checks in the configuration bench.py times (128^3 graded mesh, 4096
subdomains, three-level adaptive BDDC, B4 recycling with k = 40, df64 Schur operator
and FP32 BDDC in flexible PCG; and the 96^3 ensemble of 32 sequences).

The oracle cannot factor these sizes within a test, so the check is a property that
holds at any size: the returned free-node solution satisfies K x = f, with K the
oracle's own assembled stiffness matrix, to a relative residual of 1e-7. The interior
unknowns come from exact local solves, so the full residual is the interface
residual, which the solver drives below rtol = 1e-8 of the condensed right-hand side.
"""
import os
import sys

import numpy as np
import pytest

from oracle import q1
from workload import WORKLOADS, load_sequence, workload_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2412_17543_gb300 as P  # noqa: E402

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

DEV = "cuda:0"
TOL = 1e-7


def _rel_residual(K, x, f):
    return np.linalg.norm(f - K @ x) / np.linalg.norm(f)


def test_graded128_bench_configuration_satisfies_the_equations():
    wl = WORKLOADS["graded128"]
    mesh = workload_mesh("graded128")
    S = P.Solver(mesh, **bench.solver_options(wl, True))
    assert S.info["n_sub"] == 4096 and S.info["n_adaptive"] > 0
    rec = S.recycler(wl["k"], "B4")
    F = load_sequence(mesh, wl["seed"], 3)
    K = q1.assemble(mesh)
    for t in range(F.shape[0]):
        x, st = S.solve(torch.as_tensor(F[t], device=DEV), rec, rtol=wl["rtol"])
        assert st["rel_res"] < wl["rtol"]
        res = _rel_residual(K, x.cpu().numpy(), F[t])
        assert res <= TOL, (t, res)
    assert st["recycled_k"] > 0  # the later steps ran deflated
    rec.close()
    S.close()


def test_graded96_ensemble_satisfies_the_equations():
    wl = WORKLOADS["graded96_ens"]
    mesh = workload_mesh("graded96_ens")
    S = P.Solver(mesh, **bench.solver_options(wl, True))
    rec = S.ensemble_recycler(wl["k"], "B4")
    R = wl["nrhs"]
    F = np.stack([load_sequence(mesh, wl["seed"] + j, 2) for j in range(R)], axis=1)  # [steps][R][n]
    K = q1.assemble(mesh)
    for t in range(F.shape[0]):
        X, st = S.solve_batch(torch.as_tensor(F[t], device=DEV), rec, rtol=wl["rtol"])
        X = X.cpu().numpy()
        for j in range(R):
            assert st[j]["rel_res"] < wl["rtol"]
            res = _rel_residual(K, X[j], F[t, j])
            assert res <= TOL, (t, j, res)
    rec.close()
    S.close()
