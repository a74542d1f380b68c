"""Failure detection through the C ABI, with every failure made on the host.

* A non-finite load vector (a NaN or an infinity placed on the host) must end the solve
  with DD_BREAKDOWN instead of a silent "converged" result, and must leave the recycle
  state as it was: the next valid step gives bit for bit the result of a sequence in
  which the bad step never happened.
* A bounded device-side wait that runs out (an mbarrier that nothing arrives at, the
  same wait the streaming kernels use for their bulk copies) is reported as DD_TIMEOUT
  once; the context stays usable and the next call on it returns DD_OK.
"""
import ctypes

import numpy as np
import pytest

from workload import load_sequence, make_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2412_17543_gb300 as P  # noqa: E402
from paper_2412_17543_gb300 import _native as nat  # noqa: E402

DEV = "cuda:0"


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
@pytest.mark.parametrize("graph", [1, 0])
def test_nonfinite_load_vector_is_a_breakdown_and_leaves_state_unchanged(bad, graph):
    m = make_mesh(16, 4, 1.08, 20.0)
    F = load_sequence(m, 7, 5)
    opts = dict(levels=2, use_edges=1, schur_prec="df64", precond_prec="fp32", flexible=1, loop_graph=graph)
    S = P.Solver(m, **opts)
    clean = S.recycler(4, "B4")
    ref = [S.solve(T(f), clean, rtol=1e-9)[0].cpu().numpy() for f in F]
    rec = S.recycler(4, "B4")
    out = []
    for t, f in enumerate(F):
        if t == 2:
            g = f.copy()
            g[len(g) // 3] = bad
            gd = T(g)
            xd = torch.empty(S.n_free, dtype=torch.float64, device=DEV)
            code = S.lib.dd_solve(S.handle, ctypes.c_void_p(gd.data_ptr()), ctypes.c_void_p(xd.data_ptr()),
                                  ctypes.c_double(1e-9), rec.handle, None,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
            torch.cuda.synchronize()
            assert code == nat.DD_BREAKDOWN, nat.STATUS_NAMES[code]
            assert "breakdown" in S.lib.dd_last_error().decode().lower()
        x, st = S.solve(T(f), rec, rtol=1e-9)
        assert st["status"] == "DD_OK"
        out.append(x.cpu().numpy())
    for t in range(len(F)):
        assert np.array_equal(out[t], ref[t]), t
    S.close()


@pytest.mark.parametrize("schur_prec", ["fp64", "df64"])
def test_bounded_wait_timeout_is_reported_once(schur_prec):
    m = make_mesh(16, 8, 1.08, 20.0)
    S = P.Solver(m, levels=2, schur_prec=schur_prec, local_solver="dense")
    x = T(np.random.default_rng(1).standard_normal(S.n_gamma))
    y0 = S.schur_apply(x).cpu().numpy()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for polls in (1, 1000):
        code = S.lib.dd_selftest_bounded_wait(S.handle, polls, stream)
        assert code == nat.DD_TIMEOUT, nat.STATUS_NAMES[code]
        assert "timed out" in S.lib.dd_last_error().decode()
        # the error word was cleared when it was read: the streaming kernels run clean
        y1 = S.schur_apply(x).cpu().numpy()
        assert np.array_equal(y0, y1)
    assert S.lib.dd_selftest_bounded_wait(S.handle, 0, stream) == nat.DD_INVALID_ARG
    S.close()
