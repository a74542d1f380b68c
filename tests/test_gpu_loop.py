"""The device-resident PCG loop (one CUDA-graph launch per solve, conditional WHILE node,
stopping test in a kernel) against the host-issued loop of the same kernels.

Both forms launch the same kernels in the same order on the same data, so every
iterate, iteration count, residual and recycled basis must agree bit for bit: the
comparisons below are exact. Correctness against the oracle of the solves themselves
is checked in test_gpu_parity.py and test_gpu_ensemble.py (which run the graph form,
the default).
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

DEV = "cuda:0"
KINDS = (dd.CORNER, dd.EDGE, dd.FACE)


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def N(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _opts(levels, **kw):
    o = dict(levels=levels, coarse_group=4, use_corners=1, use_edges=1, use_faces=1, weights="diag")
    o.update(kw)
    return o


MESHES = {"graded24_s8": (24, 8, 1.3, 20.0, 2), "graded16_s2_3l": (16, 2, 1.08, 20.0, 3)}
_m = {}


def mesh(name):
    if name not in _m:
        n, sub, ratio, aspect, levels = MESHES[name]
        _m[name] = (make_mesh(n, sub, ratio, aspect), levels)
    return _m[name]


def _same_stats(a, b):
    for key in ("iters", "rel_res0", "rel_res", "recycled_k", "frozen", "status"):
        assert a[key] == b[key], (key, a[key], b[key])


@pytest.mark.parametrize("name", ["graded24_s8", "graded16_s2_3l"])
@pytest.mark.parametrize("mixed,reorth", [(False, 0), (True, 0), (True, 1)])
def test_graph_loop_equals_host_loop(name, mixed, reorth):
    m, levels = mesh(name)
    prec = dict(schur_prec="df64", precond_prec="fp32", flexible=1) if mixed else {}
    Sg = P.Solver(m, **_opts(levels, reorth=reorth, **prec))
    Sh = P.Solver(m, **_opts(levels, reorth=reorth, loop_graph=0, **prec))
    rg, rh = Sg.recycler(6, "B4"), Sh.recycler(6, "B4")
    F = load_sequence(m, 11, 5)
    for t in range(F.shape[0]):
        xg, sg = Sg.solve(T(F[t]), rg, rtol=1e-9)
        xh, sh = Sh.solve(T(F[t]), rh, rtol=1e-9)
        _same_stats(sg, sh)
        assert np.array_equal(N(xg), N(xh)), t
    assert sg["recycled_k"] > 0
    # the recycled bases agree too: the checkpoints are byte-identical
    assert rg.export() == rh.export()
    Sg.close()
    Sh.close()


def test_graph_loop_not_converged_and_zero_rhs():
    m, levels = mesh("graded24_s8")
    Sg = P.Solver(m, **_opts(levels, maxit=3))
    Sh = P.Solver(m, **_opts(levels, maxit=3, loop_graph=0))
    rg, rh = Sg.recycler(0), Sh.recycler(0)
    f = load_sequence(m, 12, 1)[0]
    xg, sg = Sg.solve(T(f), rg, rtol=1e-12, allow_not_converged=True)
    xh, sh = Sh.solve(T(f), rh, rtol=1e-12, allow_not_converged=True)
    assert sg["status"] == "DD_NOT_CONVERGED" and sg["iters"] == 3
    _same_stats(sg, sh)
    assert np.array_equal(N(xg), N(xh))
    # a zero right-hand side stops before the first iteration
    z = np.zeros_like(f)
    x0, s0 = Sg.solve(T(z), Sg.recycler(0), rtol=1e-9)
    assert s0["iters"] == 0 and not np.any(N(x0))
    Sg.close()
    Sh.close()


def test_graph_loop_solution_matches_oracle():
    m, levels = mesh("graded16_s2_3l")
    S = P.Solver(m, **_opts(levels, schur_prec="df64", precond_prec="fp32", flexible=1))
    rec = S.recycler(6, "B4")
    ch = cholesky.factor_mesh(m)
    F = load_sequence(m, 13, 4)
    for t in range(F.shape[0]):
        x, st = S.solve(T(F[t]), rec, rtol=1e-9)
        xo = ch.solve(F[t])
        assert np.linalg.norm(N(x) - xo) <= 1e-7 * np.linalg.norm(xo)
    S.close()


def test_graph_loop_counts_replayed_launches():
    """Kernels replayed by the graph are counted like launched ones: the graph form
    launches exactly one kernel more per solve than the host form (the gate that seeds
    the loop condition)."""
    m, levels = mesh("graded24_s8")
    counts = []
    for lg in (1, 0):
        S = P.Solver(m, **_opts(levels, loop_graph=lg))
        rec = S.recycler(4, "B4")
        F = load_sequence(m, 14, 3)
        S.profile(False, read=True)
        for t in range(F.shape[0]):
            S.solve(T(F[t]), rec, rtol=1e-9)
        counts.append(S.profile(False, read=True)[1])
        S.close()
    assert counts[0] == counts[1] + 3, counts


def test_profiling_uses_host_loop_with_same_results():
    m, levels = mesh("graded24_s8")
    S = P.Solver(m, **_opts(levels))
    Sref = P.Solver(m, **_opts(levels))
    r1, r2 = S.recycler(4, "B4"), Sref.recycler(4, "B4")
    F = load_sequence(m, 15, 3)
    S.profile(True, read=True)
    for t in range(F.shape[0]):
        x1, s1 = S.solve(T(F[t]), r1, rtol=1e-9)
        x2, s2 = Sref.solve(T(F[t]), r2, rtol=1e-9)
        _same_stats(s1, s2)
        assert np.array_equal(N(x1), N(x2))
    prof, _ = S.profile(False, read=True)
    assert prof["schur_apply"][1] > 0 and prof["precond_apply"][1] > 0
    S.close()
    Sref.close()


@pytest.mark.parametrize("mixed,nmm", [(False, "auto"), (True, "tc"), (True, "bf16x3")])
def test_graph_loop_equals_host_loop_ensemble(mixed, nmm):
    m, levels = mesh("graded24_s8")
    prec = dict(schur_prec="df64", precond_prec="fp32", flexible=1, local_solver="fdm") if mixed else {}
    Sg = P.Solver(m, **_opts(levels, ens_nmm=nmm, **prec))
    Sh = P.Solver(m, **_opts(levels, ens_nmm=nmm, loop_graph=0, **prec))
    rg, rh = Sg.ensemble_recycler(6, "B4"), Sh.ensemble_recycler(6, "B4")
    nrhs = 5
    seqs = [load_sequence(m, 40 + j, 4) for j in range(nrhs)]
    for t in range(4):
        F = T(np.stack([seqs[j][t] for j in range(nrhs)]))
        Xg, sg = Sg.solve_batch(F, rg, rtol=1e-9)
        Xh, sh = Sh.solve_batch(F, rh, rtol=1e-9)
        for j in range(nrhs):
            _same_stats(sg[j], sh[j])
        assert np.array_equal(N(Xg), N(Xh)), t
    assert sg[0]["recycled_k"] > 0
    Sg.close()
    Sh.close()
