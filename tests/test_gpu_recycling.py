"""The recycling update (Sect. 4.2) and the residual re-orthogonalization (Sect. 4.1) of the
CUDA path against the oracle, through the C ABI.

* B4 with an FP64 operator and preconditioner: after every step the selected harmonic Ritz
  values (eq. 15) agree with the oracle's within 1e-8 relative, and the basis freezes
  (eq. 16) after the same step. The tolerances are chosen where the oracle's freezing
  ratios are decisive (at least a factor 3 from the tolerance), so rounding differences
  between the two sides cannot move the decision.
* Re-orthogonalization: the deflated solve with a recycled basis matches the oracle's
  solution and keeps W^T r at rounding level.
"""
import numpy as np
import pytest

from oracle import cholesky, dd, pcg
from workload import load_sequence, make_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2412_17543_gb300 as P  # noqa: E402

DEV = "cuda:0"
KINDS = dict(levels=2, use_corners=1, use_edges=0, use_faces=0, weights="diag", schur_prec="fp64",
             precond_prec="fp64")


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


_case = {}


def _oracle_sequence(R, tol, steps=8):
    key = (R, tol, steps)
    if key not in _case:
        m = make_mesh(16, 8, 1.08, 20.0)
        subs = dd.q1_substructures(m)
        Po = dd.Preconditioner(subs, 2, (dd.CORNER,), "diag")
        F = load_sequence(m, 2, steps)
        rec = pcg.Recycler(R, "B4", tol)
        x = np.zeros(len(subs.gamma))
        thetas, frozen = [], []
        for f in F:
            x, info = pcg.deflated_pcg(subs.schur_apply, Po.apply, subs.condense(f), x, rec.W, rec.AW, 1e-9)
            rec.update(info, Po.apply)
            thetas.append(None if rec.theta is None else rec.theta.copy())
            frozen.append(rec.frozen)
        _case[key] = (m, F, thetas, frozen, rec)
    return _case[key]


@pytest.mark.parametrize("tol,freeze_step", [(1e-5, 3), (1e-7, 4)])
def test_b4_ritz_values_and_freezing_match_oracle(tol, freeze_step):
    m, F, thetas, frozen, rec_o = _oracle_sequence(8, tol)
    # the decision is decisive on the oracle's side
    for step, ratio in rec_o.crit_history:
        assert ratio <= tol / 3 or ratio >= 3 * tol, (step, ratio)
    assert rec_o.frozen_at == freeze_step
    S = P.Solver(m, **KINDS)
    rec = S.recycler(8, "B4", tol)
    for t, f in enumerate(F):
        _, st = S.solve(T(f), rec, rtol=1e-9)
        state = rec.state()
        assert state["frozen"] == frozen[t] == bool(st["frozen"]), t
        th_o = thetas[t]
        assert len(state["theta"]) == len(th_o)
        assert np.abs(state["theta"] - th_o).max() <= 1e-8 * np.abs(th_o).max(), (t, state["theta"], th_o)
    S.close()


@pytest.mark.parametrize("schur,pre,flex", [("fp64", "fp64", 0), ("df64", "fp32", 1)])
def test_reorthogonalized_recycled_solves_match_oracle(schur, pre, flex):
    m = make_mesh(16, 8, 1.08, 20.0)
    F = load_sequence(m, 6, 5)
    ch = cholesky.factor_mesh(m)
    subs = dd.q1_substructures(m)
    Po = dd.Preconditioner(subs, 2, (dd.CORNER,), "diag")
    S = P.Solver(m, **dict(KINDS, schur_prec=schur, precond_prec=pre, flexible=flex, reorth=1))
    rec = S.recycler(6, "B4")
    rec_o = pcg.Recycler(6, "B4")
    x_o = np.zeros(len(subs.gamma))
    for t, f in enumerate(F):
        x, st = S.solve(T(f), rec, rtol=1e-9)
        xe = ch.solve(f)
        err = np.linalg.norm(x.cpu().numpy() - xe) / np.linalg.norm(xe)
        assert err <= 1e-7, (t, err)
        # the oracle with re-orthogonalization: same iteration count within one
        x_o, info = pcg.deflated_pcg(subs.schur_apply, Po.apply, subs.condense(f), x_o, rec_o.W, rec_o.AW, 1e-9,
                                     reorth=True, flexible=bool(flex))
        if rec_o.W is not None:
            nW = np.linalg.norm(rec_o.W, 2)
            ref = np.linalg.norm(subs.condense(f))
            assert max(info.wtr) <= 1e-12 * nW * ref
        rec_o.update(info, Po.apply)
        if schur == "fp64":
            assert abs(st["iters"] - info.iters) <= 1, (t, st["iters"], info.iters)
    S.close()


def test_fp32_valued_basis_is_exact_for_its_own_span():
    """With an FP32 preconditioner the recycled basis is rounded to FP32-representable values
    when it is formed and A W recomputed for it (the update streams W as floats). The
    checkpoint holds the state as the solver uses it: every entry of W is a float, A W is
    the Schur operator applied to that W bit for bit, and the solves match the oracle."""
    import struct
    m = make_mesh(16, 8, 1.08, 20.0)
    F = load_sequence(m, 4, 5)
    ch = cholesky.factor_mesh(m)
    S = P.Solver(m, **dict(KINDS, schur_prec="df64", precond_prec="fp32", flexible=1))
    rec = S.recycler(6, "B4")
    for t, f in enumerate(F):
        x, st = S.solve(T(f), rec, rtol=1e-9)
        xe = ch.solve(f)
        assert np.linalg.norm(x.cpu().numpy() - xe) <= 1e-7 * np.linalg.norm(xe), t
    blob = rec.export()
    fmt = "<8sq6id"
    _, n, kmax, _, k, _, _, ntheta, _ = struct.unpack_from(fmt, blob, 0)
    assert k > 0
    off = struct.calcsize(fmt) + 8 * ntheta + 8 * n  # theta, previous solution
    W = np.frombuffer(blob, dtype=np.float64, count=k * n, offset=off).reshape(k, n)
    AW = np.frombuffer(blob, dtype=np.float64, count=k * n, offset=off + 8 * k * n).reshape(k, n)
    assert np.array_equal(W, W.astype(np.float32).astype(np.float64))
    for j in range(k):
        y = S.schur_apply(T(W[j])).cpu().numpy()
        assert np.array_equal(y, AW[j]), j
    rec.close()
    S.close()


@pytest.mark.parametrize("pre", ["fp64", "fp32"])
def test_wide_recycled_basis_matches_oracle(pre):
    """A basis of 100 columns (the deflation dots' last-block reduction then gives each thread
    a segment of half the blocks, and the update walks 25 groups of four columns) on the
    FP64 and the mixed-precision path: every step's solution against the sparse Cholesky."""
    m = make_mesh(16, 4, 1.08, 20.0)
    F = load_sequence(m, 8, 6)
    ch = cholesky.factor_mesh(m)
    mixed = pre == "fp32"
    S = P.Solver(m, **dict(KINDS, schur_prec="df64" if mixed else "fp64", precond_prec=pre, flexible=int(mixed)))
    rec = S.recycler(100, "B4")
    for t, f in enumerate(F):
        x, st = S.solve(T(f), rec, rtol=1e-9)
        xe = ch.solve(f)
        err = np.linalg.norm(x.cpu().numpy() - xe) / np.linalg.norm(xe)
        assert err <= 1e-7, (t, err)
    assert rec.state()["k"] > 40
    rec.close()
    S.close()
