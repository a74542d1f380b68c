"""Ensemble path (dd_solve_batch and the batched operators) against the FP64 oracle.

Every member of an ensemble is an independent problem, so the oracle is the
single-vector oracle applied member by member: the dense-restated Schur complement
and BDDC of oracle/dd.py for the operators, the sparse Cholesky for the solutions.
Tolerances as in test_gpu_parity.py (FP64 1e-12, df64 1e-11, FP32 BDDC 1e-4 of the
largest entry; solutions 1e-7 relative at rtol 1e-9).
"""
import numpy as np
import pytest

from oracle import cholesky, dd
from workload import load_sequence, make_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2412_17543_gb300 as P  # noqa: E402
from paper_2412_17543_gb300 import DDError  # noqa: E402

DEV = "cuda:0"
W = 32


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def N(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _opts(levels, kinds, **kw):
    o = dict(levels=levels, coarse_group=4, use_corners=int(dd.CORNER in kinds), use_edges=int(dd.EDGE in kinds),
             use_faces=int(dd.FACE in kinds), weights="diag")
    o.update(kw)
    return o


CASES = {
    "cube16_cf": (16, 4, 1.0, None, 2, (dd.CORNER, dd.FACE)),
    "graded24_s8": (24, 8, 1.3, 20.0, 2, (dd.CORNER, dd.EDGE, dd.FACE)),
    "graded16_s2_3l": (16, 2, 1.08, 20.0, 3, (dd.CORNER, dd.EDGE, dd.FACE)),
}
_cache = {}


def case(name):
    if name not in _cache:
        n, sub, ratio, aspect, levels, kinds = CASES[name]
        m = make_mesh(n, sub, ratio, aspect)
        _cache[name] = (m, dd.q1_substructures(m), kinds, levels)
    return _cache[name]


@pytest.mark.parametrize("name", ["cube16_cf", "graded24_s8"])
@pytest.mark.parametrize("prec,local,tol", [("fp64", "dense", 1e-12), ("fp64", "fdm", 1e-12),
                                            ("df64", "fdm", 1e-11)])
@pytest.mark.parametrize("nrhs", [3, W])
def test_schur_apply_batch(name, prec, local, tol, nrhs):
    m, subs, kinds, _ = case(name)
    S = P.Solver(m, **_opts(2, kinds, schur_prec=prec, local_solver=local))
    X = np.random.default_rng(nrhs).standard_normal((nrhs, len(subs.gamma)))
    Y = N(S.schur_apply_batch(T(X)))
    for j in range(nrhs):
        yo = subs.schur_apply(X[j])
        assert np.abs(Y[j] - yo).max() <= tol * np.abs(yo).max()
    S.close()


@pytest.mark.parametrize("elem_rc,fdm_rc", [(4, 4), (8, 8), (16, 4), (16, 8)])
def test_schur_apply_batch_launch_shapes(elem_rc, fdm_rc):
    """Every members-per-pass choice of the df64 element kernels and per-block choice of
    the ensemble fast diagonalization gives the same operator (8^3 subdomains, all 32
    members, tolerance of the df64 operator)."""
    m, subs, kinds, _ = case("graded24_s8")
    S = P.Solver(m, **_opts(2, kinds, schur_prec="df64", local_solver="fdm", ens_elem_rc=elem_rc,
                            ens_fdm_rc=fdm_rc))
    X = np.random.default_rng(elem_rc + fdm_rc).standard_normal((W, len(subs.gamma)))
    Y = N(S.schur_apply_batch(T(X)))
    for j in range(W):
        yo = subs.schur_apply(X[j])
        assert np.abs(Y[j] - yo).max() <= 1e-11 * np.abs(yo).max()
    assert (S.info["ens_elem_rc"], S.info["ens_fdm_rc"]) == (elem_rc, fdm_rc)
    S.close()


def test_schur_apply_batch_rejects_df64_dense():
    m, subs, kinds, _ = case("cube16_cf")
    S = P.Solver(m, **_opts(2, kinds, schur_prec="df64", local_solver="dense"))
    with pytest.raises(DDError):
        S.schur_apply_batch(T(np.ones((2, len(subs.gamma)))))
    S.close()


@pytest.mark.parametrize("name", ["cube16_cf", "graded24_s8", "graded16_s2_3l"])
@pytest.mark.parametrize("weights", ["card", "diag"])
@pytest.mark.parametrize("prec,nmm,tol", [("fp64", "auto", 1e-10), ("fp32", "simt", 1e-4), ("fp32", "tc", 1e-4),
                                          ("fp32", "bf16x3", 1e-4)])
def test_precond_apply_batch(name, weights, prec, nmm, tol):
    """BDDC of the ensemble; with FP32 every N_i kernel (CUDA-core tiles, tensor-core
    3xTF32 and BF16x3, including the partial 128-row block of 386-row operators) is checked."""
    m, subs, kinds, levels = case(name)
    S = P.Solver(m, **_opts(levels, kinds, weights=weights, precond_prec=prec, ens_nmm=nmm))
    Po = dd.Preconditioner(subs, levels, kinds, weights, group=4)
    R = np.random.default_rng(5).standard_normal((7, len(subs.gamma)))
    Z = N(S.precond_apply_batch(T(R)))
    for j in range(R.shape[0]):
        zo = Po.apply(R[j])
        assert np.abs(Z[j] - zo).max() <= tol * np.abs(zo).max()
    if prec == "fp32":
        assert S.info["ens_nmm"] == {"simt": 1, "tc": 2, "bf16x3": 3}[nmm]
    S.close()


def test_nmm_autotune_picks_a_kernel():
    m, subs, kinds, levels = case("graded24_s8")
    S = P.Solver(m, **_opts(2, kinds, precond_prec="fp32", ens_nmm="auto"))
    S.precond_apply_batch(T(np.ones((2, len(subs.gamma)))))
    info = S.info
    assert info["ens_nmm"] in (1, 2, 3) and min(info["ens_nmm_ms"]) > 0.0
    S.close()


def test_launch_shapes_are_tuned_on_first_call():
    """Members per pass of the df64 element kernels and per block of the ensemble
    fast diagonalization are chosen by timing on the context's own mesh; every choice
    gives the same operator (checked in test_schur_apply_batch)."""
    m, subs, kinds, levels = case("graded24_s8")
    S = P.Solver(m, **_opts(2, kinds, schur_prec="df64", local_solver="fdm", precond_prec="fp32"))
    assert S.info["ens_elem_rc"] == 0
    S.schur_apply_batch(T(np.ones((2, len(subs.gamma)))))
    info = S.info
    assert info["ens_elem_rc"] in (4, 8, 16) and info["ens_fdm_rc"] in (4, 8)
    S.close()


def _member_sequences(m, nrhs, steps, seed0):
    return [load_sequence(m, seed0 + j, steps) for j in range(nrhs)]


@pytest.mark.parametrize("name", ["cube16_cf", "graded16_s2_3l", "graded24_s8"])
@pytest.mark.parametrize("schur,pre,flex,nmm", [("fp64", "fp64", 0, "auto"), ("df64", "fp32", 1, "simt"),
                                                ("df64", "fp32", 1, "tc"), ("df64", "fp32", 1, "bf16x3")])
@pytest.mark.parametrize("k", [0, 6])
def test_solve_batch_matches_direct(name, schur, pre, flex, nmm, k):
    m, subs, kinds, levels = case(name)
    nrhs, steps = 5, 4
    seqs = _member_sequences(m, nrhs, steps, 30)
    ch = cholesky.factor_mesh(m)
    S = P.Solver(m, **_opts(levels, kinds, schur_prec=schur, precond_prec=pre, flexible=flex, ens_nmm=nmm))
    rec = S.ensemble_recycler(k, "B4")
    iters = []
    for t in range(steps):
        F = np.stack([seqs[j][t] for j in range(nrhs)])
        X, st = S.solve_batch(T(F), rec, rtol=1e-9)
        X = N(X)
        for j in range(nrhs):
            xo = ch.solve(F[j])
            err = np.linalg.norm(X[j] - xo) / np.linalg.norm(xo)
            assert err <= 1e-7, (t, j, err)
            assert st[j]["rel_res"] < 1e-9
        iters.append([s["iters"] for s in st])
    if k:
        assert st[0]["recycled_k"] > 0
    rec.close()
    S.close()


def test_solve_batch_equals_single_sequences():
    """Without deflation every member runs exactly the single-sequence PCG: same
    iteration counts (up to one from rounding order) and the same solutions."""
    m, subs, kinds, levels = case("graded24_s8")
    nrhs = 4
    seqs = _member_sequences(m, nrhs, 2, 50)
    S = P.Solver(m, **_opts(2, kinds))
    recb = S.ensemble_recycler(0)
    singles = [S.recycler(0) for _ in range(nrhs)]
    for t in range(2):
        F = np.stack([seqs[j][t] for j in range(nrhs)])
        X, st = S.solve_batch(T(F), recb, rtol=1e-10)
        X = N(X)
        for j in range(nrhs):
            x1, s1 = S.solve(T(F[j]), singles[j], rtol=1e-10)
            x1 = N(x1)
            assert abs(st[j]["iters"] - s1["iters"]) <= 1
            assert np.linalg.norm(X[j] - x1) <= 1e-9 * np.linalg.norm(x1)
    S.close()


def test_solve_batch_padding_and_single_member():
    m, subs, kinds, levels = case("cube16_cf")
    S = P.Solver(m, **_opts(2, kinds))
    rec = S.ensemble_recycler(4)
    ch = cholesky.factor_mesh(m)
    f = load_sequence(m, 77, 1)[0]
    X, st = S.solve_batch(T(f[None, :]), rec, rtol=1e-10)
    xo = ch.solve(f)
    assert np.linalg.norm(N(X)[0] - xo) <= 1e-8 * np.linalg.norm(xo)
    # a zero right-hand side is solved by zero without iterations
    X, st = S.solve_batch(T(np.stack([f, 0 * f])), rec, rtol=1e-10)
    assert st[1]["iters"] == 0 and np.abs(N(X)[1]).max() == 0.0
    S.close()


def test_solve_batch_invalid_arguments():
    m, subs, kinds, levels = case("cube16_cf")
    S = P.Solver(m, **_opts(2, kinds))
    rec_b = S.ensemble_recycler(0)
    rec_1 = S.recycler(0)
    F = torch.zeros((W + 1, S.n_free), dtype=torch.float64, device=DEV)
    with pytest.raises(DDError):
        S.solve_batch(F, rec_b)                       # more members than the block width
    with pytest.raises(DDError):
        S.solve_batch(F[:0], rec_b)                   # no member
    with pytest.raises(DDError):
        S.solve_batch(F[:2], rec_1)                   # single-sequence state
    S.close()


@pytest.mark.parametrize("nmm", ["tc", "bf16x3"])
def test_precond_apply_batch_persistent_items(nmm):
    """125 subdomains give 500 (subdomain, 128-row block) items, more than the GPU has
    SMs: each persistent CTA walks several items, so the copy ring runs across item
    boundaries and both accumulator slots are used. All 32 members against the oracle."""
    m = make_mesh(40, 8, 1.2, 20.0)
    subs = dd.q1_substructures(m)
    kinds = (dd.CORNER, dd.EDGE, dd.FACE)
    S = P.Solver(m, **_opts(2, kinds, precond_prec="fp32", ens_nmm=nmm))
    Po = dd.Preconditioner(subs, 2, kinds, "diag", group=4)
    R = np.random.default_rng(9).standard_normal((W, len(subs.gamma)))
    Z = N(S.precond_apply_batch(T(R)))
    for j in range(W):
        zo = Po.apply(R[j])
        assert np.abs(Z[j] - zo).max() <= 1e-4 * np.abs(zo).max(), j
    S.close()
