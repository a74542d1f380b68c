"""Solver options through the C ABI: the initial guess (previous solution or zero) and the
two stopping criteria (eq. 18 and eq. 17, Sect. 5)."""
import numpy as np
import pytest

from oracle import cholesky
from workload import load_sequence, make_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2412_17543_gb300 as P  # noqa: E402

DEV = "cuda:0"


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _opts(**kw):
    o = dict(levels=2, coarse_group=4, use_corners=1, use_edges=1, use_faces=1, weights="diag")
    o.update(kw)
    return o


def test_zero_initial_guess_and_stopping_criteria():
    """From x = 0 the residual-norm and right-hand-side-norm criteria coincide (r_0 = b), so
    both stop after the same iterations with the same iterate; from the previous solution
    the first step starts closer (fewer iterations on a slowly varying sequence)."""
    m = make_mesh(16, 4, 1.08, 20.0)
    F = load_sequence(m, 31, 3)
    ch = cholesky.factor_mesh(m)
    runs = {}
    for name, kw in {"zero_rhs": dict(zero_initial_guess=1, stop_rhs_norm=1),
                     "zero_r0": dict(zero_initial_guess=1, stop_rhs_norm=0),
                     "prev_rhs": dict(zero_initial_guess=0, stop_rhs_norm=1)}.items():
        S = P.Solver(m, **_opts(**kw))
        rec = S.recycler(0)
        out = []
        for f in F:
            x, st = S.solve(T(f), rec, rtol=1e-9)
            xo = ch.solve(f)
            assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-7 * np.linalg.norm(xo)
            out.append((st["iters"], st["rel_res0"], x.cpu().numpy()))
        runs[name] = out
        S.close()
    for (i1, r1, x1), (i2, r2, x2) in zip(runs["zero_rhs"], runs["zero_r0"]):
        assert i1 == i2 and r2 == 1.0 and abs(r1 - 1.0) < 1e-12
        assert np.array_equal(x1, x2)
    assert runs["prev_rhs"][1][1] < 1.0 and runs["prev_rhs"][2][0] <= runs["zero_rhs"][2][0]
