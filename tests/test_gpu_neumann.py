"""The pure-Neumann variant (no Dirichlet face; Sect. 2 and 4.1) through the C ABI against
the oracle of oracle/neumann.py: the library projects the load vector onto the range of K,
keeps the preconditioned residuals orthogonal to the constants and returns the mean-free
solution, which must match the oracle's grounded sparse-Cholesky solution to 1e-7 at
rtol 1e-9 (the solution tolerance of the other parity tests)."""
import numpy as np
import pytest

from oracle import neumann
from workload import load_sequence, make_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2412_17543_gb300 as P  # noqa: E402
from paper_2412_17543_gb300 import DDError  # noqa: E402

DEV = "cuda:0"


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def N(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _opts(levels, **kw):
    o = dict(levels=levels, coarse_group=4, use_corners=1, use_edges=1, use_faces=1, weights="diag")
    o.update(kw)
    return o


@pytest.mark.parametrize("levels,sub,mixed", [(2, 4, False), (2, 4, True), (3, 2, True)])
def test_neumann_sequence_matches_oracle(levels, sub, mixed):
    m = make_mesh(16, sub, 1.08, 20.0, dirichlet=0)
    prec = dict(schur_prec="df64", precond_prec="fp32", flexible=1) if mixed else {}
    S = P.Solver(m, **_opts(levels, **prec))
    assert S.info["neumann"] == 1
    rec = S.recycler(6, "B4")
    ns = neumann.Solver(m)
    F = load_sequence(m, 21, 4)
    for t in range(F.shape[0]):
        x, st = S.solve(T(F[t]), rec, rtol=1e-9)
        x = N(x)
        xo = ns.solve(F[t])
        assert abs(x.mean()) <= 1e-12 * np.abs(x).max()
        assert np.linalg.norm(x - xo) <= 1e-7 * np.linalg.norm(xo), t
    assert st["recycled_k"] > 0
    S.close()


def test_neumann_rejects_ensembles_and_adjoint():
    m = make_mesh(16, 4, 1.08, 20.0, dirichlet=0)
    S = P.Solver(m, **_opts(2))
    with pytest.raises(DDError):
        S.solve_batch(T(np.zeros((2, S.n_free))), S.ensemble_recycler(0))
    with pytest.raises(DDError):
        S.adjoint(T(np.ones(S.n_free)), coef_grad=False)
    S.close()
