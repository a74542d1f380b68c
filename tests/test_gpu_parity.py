"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (derived from the arithmetic):
  * FP64 operators: a sum of <= ~800 products per output in a different order than
    the oracle's LAPACK-based dense path: |y - y_oracle| <= 1e-12 * max|y_oracle|.
  * DF64 Schur operator (float pairs, ~2^-44 per operation): 1e-11 * max|y|.
  * FP32 preconditioner: 1e-4 * max|z| (single-precision storage, FP32 sums).
  * Solutions (the stated solution tolerance): relative 2-norm error vs the sparse Cholesky
    solution <= 1e-7 at rtol 1e-9.
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


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def N(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


CASES = {
    # name: (n, sub, ratio, aspect, levels, kinds)
    "cube16_cf": (16, 4, 1.0, None, 2, (dd.CORNER, dd.FACE)),
    "graded16_s8": (16, 8, 1.08, 20.0, 2, (dd.CORNER, dd.EDGE, dd.FACE)),
    "graded24_s8": (24, 8, 1.3, 20.0, 2, (dd.CORNER, dd.EDGE, dd.FACE)),
    "graded16_s2_3l": (16, 2, 1.08, 20.0, 3, (dd.CORNER, dd.EDGE, dd.FACE)),
}


def _opts(levels, kinds, **kw):
    o = dict(levels=levels, coarse_group=4, use_corners=int(dd.CORNER in kinds), use_edges=int(dd.EDGE in kinds),
             use_faces=int(dd.FACE in kinds), weights="diag")
    o.update(kw)
    return o


_oracles = {}


def oracle_case(name):
    if name not in _oracles:
        n, sub, ratio, aspect, levels, kinds = CASES[name]
        m = make_mesh(n, sub, ratio, aspect)
        subs = dd.q1_substructures(m)
        _oracles[name] = (m, subs, kinds, levels)
    return _oracles[name]


@pytest.mark.parametrize("name", ["cube16_cf", "graded16_s8", "graded24_s8"])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("df64", 1e-11)])
@pytest.mark.parametrize("local", ["dense", "fdm"])
def test_schur_apply(name, prec, tol, local):
    m, subs, kinds, levels = oracle_case(name)
    S = P.Solver(m, **_opts(2, kinds, schur_prec=prec, local_solver=local))
    assert S.info["local_solver"] == (1 if local == "dense" else 2)
    assert np.array_equal(S.interface_nodes(), subs.gamma)
    rng = np.random.default_rng(0)
    for _ in range(2):
        x = rng.standard_normal(len(subs.gamma))
        y = N(S.schur_apply(T(x)))
        yo = subs.schur_apply(x)
        assert np.abs(y - yo).max() <= tol * np.abs(yo).max()


@pytest.mark.parametrize("name", ["cube16_cf", "graded24_s8"])
@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("local", ["dense", "fdm"])
def test_condense_and_recover(name, prec, local):
    m, subs, kinds, levels = oracle_case(name)
    S = P.Solver(m, **_opts(2, kinds, schur_prec=prec, local_solver=local))
    f = load_sequence(m, 1, 1)[0]
    b = N(S.condense(T(f)))
    bo = subs.condense(f)
    assert np.abs(b - bo).max() <= 1e-11 * np.abs(bo).max()
    xg = np.random.default_rng(2).standard_normal(len(subs.gamma))
    x = N(S.recover(T(f), T(xg)))
    xo = subs.recover(f, xg)
    assert np.abs(x - xo).max() <= 1e-11 * np.abs(xo).max()


@pytest.mark.parametrize("name", ["cube16_cf", "graded16_s8", "graded16_s2_3l"])
@pytest.mark.parametrize("weights", ["card", "diag"])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_precond_apply(name, weights, prec, tol):
    m, subs, kinds, levels = oracle_case(name)
    S = P.Solver(m, **_opts(levels, kinds, weights=weights, precond_prec=prec))
    Po = dd.Preconditioner(subs, levels, kinds, weights, group=4)
    rng = np.random.default_rng(1)
    r = rng.standard_normal(len(subs.gamma))
    z = N(S.precond_apply(T(r)))
    zo = Po.apply(r)
    assert np.abs(z - zo).max() <= tol * np.abs(zo).max()


def _direct(m, F):
    ch = cholesky.factor_mesh(m)
    return [ch.solve(f) for f in F]


@pytest.mark.parametrize("schur,pre,flex", [("fp64", "fp64", 0), ("df64", "fp32", 1)])
def test_solve_sequence_plain(schur, pre, flex):
    m, subs, kinds, levels = oracle_case("cube16_cf")
    F = load_sequence(m, 1, 10)
    X = _direct(m, F)
    S = P.Solver(m, **_opts(2, kinds, schur_prec=schur, precond_prec=pre, flexible=flex))
    rec = S.recycler(0)
    Po = dd.Preconditioner(subs, 2, kinds, "diag")
    xs_o, infos_o, _ = pcg.solve_sequence(subs.schur_apply, Po.apply, [subs.condense(f) for f in F], R=0, rtol=1e-9)
    for t, f in enumerate(F):
        x, st = S.solve(T(f), rec, rtol=1e-9)
        x = N(x)
        err = np.linalg.norm(x - X[t]) / np.linalg.norm(X[t])
        assert err <= 1e-7, (t, err)
        assert st["rel_res"] < 1e-9
        if schur == "fp64" and pre == "fp64":
            assert abs(st["iters"] - infos_o[t].iters) <= 1, (t, st["iters"], infos_o[t].iters)


@pytest.mark.parametrize("strategy", ["B4", "B3", "B2", "B1"])
def test_solve_sequence_recycled(strategy):
    m, subs, kinds, levels = oracle_case("graded16_s8")
    F = load_sequence(m, 2, 8)
    X = _direct(m, F)
    S = P.Solver(m, **_opts(2, (dd.CORNER,), schur_prec="fp64", precond_prec="fp64"))
    rec = S.recycler(6, strategy)
    Po = dd.Preconditioner(subs, 2, (dd.CORNER,), "diag")
    _, infos_o, _ = pcg.solve_sequence(subs.schur_apply, Po.apply, [subs.condense(f) for f in F], R=6,
                                       strategy=strategy, rtol=1e-9)
    its = []
    for t, f in enumerate(F):
        x, st = S.solve(T(f), rec, rtol=1e-9)
        x = N(x)
        err = np.linalg.norm(x - X[t]) / np.linalg.norm(X[t])
        assert err <= 1e-7, (t, err)
        its.append(st["iters"])
    its_o = [i.iters for i in infos_o]
    assert its[0] == its_o[0]
    assert sum(its) <= sum(its_o) + len(F), (its, its_o)


@pytest.mark.parametrize("local", ["dense", "fdm"])
def test_solve_mixed_recycled_three_level(local):
    m, subs, kinds, levels = oracle_case("graded16_s2_3l")
    F = load_sequence(m, 3, 6)
    X = _direct(m, F)
    S = P.Solver(m, **_opts(3, kinds, schur_prec="df64", precond_prec="fp32", flexible=1, local_solver=local))
    rec = S.recycler(8, "B4")
    for t, f in enumerate(F):
        x, st = S.solve(T(f), rec, rtol=1e-9)
        err = np.linalg.norm(N(x) - X[t]) / np.linalg.norm(X[t])
        assert err <= 1e-7, (t, err)


@pytest.mark.parametrize("tau", [1.5, 3.0])
@pytest.mark.parametrize("solver,tol", [("dense", 1e-9), ("lobpcg", 1e-6)])
def test_precond_apply_adaptive(tau, solver, tol):
    # random coefficients make some faces need extra constraints (Sect. 3.3); the face
    # eigenproblems by the dense eigensolver, or by the paper's LOBPCG (15 steps, 10 vectors)
    # batched on the device against the oracle's LOBPCG with the same steps (the tolerance
    # allows for the rounding that 15 steps of an inexact eigensolver carry into the rows)
    rng = np.random.default_rng(5)
    n = 8
    coef = np.exp(2.0 * rng.standard_normal((n, n, n)))
    m = make_mesh(n, 4, 1.08, 20.0, coef=coef)
    subs = dd.q1_substructures(m)
    kinds = (dd.CORNER, dd.EDGE, dd.FACE)
    base = dd.Preconditioner(subs, 2, kinds, "diag")
    rows = dd.adaptive_face_constraints(subs, base.l1.D, tau=tau, method=solver, lobpcg_iters=15)
    Po = dd.Preconditioner(subs, 2, kinds, "diag", extra_rows=rows)
    S = P.Solver(m, **_opts(2, kinds, adaptive=1, tau=tau, adaptive_solver=solver, lobpcg_iters=15))
    assert S.info["n_adaptive"] == sum(len(r) for r in rows.values()) > 0
    r = np.random.default_rng(3).standard_normal(len(subs.gamma))
    z = N(S.precond_apply(T(r)))
    zo = Po.apply(r)
    assert np.abs(z - zo).max() <= tol * np.abs(zo).max()


def test_adaptive_lobpcg_on_the_bench_mesh_family():
    """Device LOBPCG constraints on a graded 32^3 member of the timed workload's family (FDM
    local solves, three levels): the count equals the oracle's LOBPCG count, and the solution
    sequence still matches the sparse Cholesky."""
    m = make_mesh(32, 8, 1.3, 40.0)
    subs = dd.q1_substructures(m)
    kinds = (dd.CORNER, dd.EDGE, dd.FACE)
    base = dd.Preconditioner(subs, 2, kinds, "diag")
    rows = dd.adaptive_face_constraints(subs, base.l1.D, tau=4.0, method="lobpcg", lobpcg_iters=15)
    S = P.Solver(m, levels=3, coarse_group=2, use_corners=1, use_edges=1, use_faces=1, weights="diag", adaptive=1,
                 tau=4.0, adaptive_solver="lobpcg", schur_prec="df64", precond_prec="fp32", flexible=1)
    assert S.info["n_adaptive"] == sum(len(r) for r in rows.values()) > 0
    F = load_sequence(m, 3, 3)
    ch = cholesky.factor_mesh(m)
    rec = S.recycler(8, "B4")
    for t, f in enumerate(F):
        x, st = S.solve(T(f), rec, rtol=1e-9)
        xe = ch.solve(f)
        assert np.linalg.norm(N(x) - xe) <= 1e-7 * np.linalg.norm(xe), t
    S.close()


def test_adjoint_and_autograd_match_oracle():
    from oracle import adjoint
    rng = np.random.default_rng(11)
    n = 16
    from workload import gaussian_random_field
    g = gaussian_random_field(n, 40)
    m = make_mesh(n, 4, 1.08, 20.0, coef=np.exp(g))
    f = load_sequence(m, 4, 1)[0]
    target = rng.standard_normal(m.n_free)
    ch = cholesky.factor_mesh(m)
    x_o = ch.solve(f)
    gf_o, gk_o = adjoint.adjoint(m, ch, x_o, 2 * (x_o - target))
    S = P.Solver(m, levels=2, use_edges=1, schur_prec="fp64", precond_prec="fp64")
    rec = S.recycler(0)
    # C ABI adjoint
    gf, gk, st = S.adjoint(T(2 * (x_o - target)), T(x_o), None, 1e-12)
    assert np.abs(N(gf) - gf_o).max() <= 1e-9 * np.abs(gf_o).max()
    assert np.abs(N(gk) - gk_o).max() <= 1e-9 * np.abs(gk_o).max()
    # autograd through the binding: loss = ||x - target||^2, gradients w.r.t. f and g = log k
    fT = T(f).requires_grad_(True)
    gT = T(g).requires_grad_(True)
    x = P.PoissonSolve.apply(fT, gT, S, rec, 1e-12, 1e-12)
    loss = ((x - T(target)) ** 2).sum()
    loss.backward()
    gg_o = (np.exp(g).ravel() * gk_o).reshape(g.shape)
    assert np.abs(N(fT.grad) - gf_o).max() <= 1e-8 * np.abs(gf_o).max()
    assert np.abs(N(gT.grad) - gg_o).max() <= 1e-8 * np.abs(gg_o).max()


def test_recycle_checkpoint_resume_is_bitwise_identical():
    m, subs, kinds, levels = oracle_case("graded16_s8")
    F = load_sequence(m, 5, 10)
    S = P.Solver(m, **_opts(2, kinds, schur_prec="df64", precond_prec="fp32", flexible=1))
    recA = S.recycler(6, "B4")
    xa = [N(S.solve(T(f), recA, rtol=1e-9)[0]) for f in F]
    recB = S.recycler(6, "B4")
    xb = [N(S.solve(T(f), recB, rtol=1e-9)[0]) for f in F[:5]]
    blob = recB.export()
    recB.close()
    recC = P.Recycler.restore(S, blob)
    xb += [N(S.solve(T(f), recC, rtol=1e-9)[0]) for f in F[5:]]
    for t in range(10):
        assert np.array_equal(xa[t], xb[t]), t


def test_bench_options_at_32cubed_every_step_against_sparse_cholesky():
    """The timed configuration's options on a small member of its mesh family: 32^3 graded to
    aspect 40 with 8^3 subdomains (FDM local solves, fused Schur operator), three levels
    (groups of 2^3), adaptive face constraints at tau = 10, df64 Schur operator, FP32 BDDC,
    flexible PCG, B4 recycling; every step's full solution against the oracle's sparse
    Cholesky: relative 2-norm error <= 1e-7 at rtol 1e-9."""
    m = make_mesh(32, 8, 1.3, 40.0)
    S = P.Solver(m, levels=3, coarse_group=2, use_corners=1, use_edges=1, use_faces=1, weights="diag", adaptive=1,
                 tau=10.0, schur_prec="df64", precond_prec="fp32", flexible=1)
    assert S.info["n_adaptive"] > 0 and S.info["local_solver"] == 2
    F = load_sequence(m, 3, 8)
    ch = cholesky.factor_mesh(m)
    rec = S.recycler(16, "B4")
    for t, f in enumerate(F):
        x, st = S.solve(T(f), rec, rtol=1e-9)
        xe = ch.solve(f)
        err = np.linalg.norm(N(x) - xe) / np.linalg.norm(xe)
        assert err <= 1e-7, (t, err, st)
        assert st["rel_res"] < 1e-9
    assert rec.state()["k"] > 0
    S.close()
