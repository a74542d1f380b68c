"""dd_schur_apply_noalloc: the Schur-complement application for callers that must not
allocate device memory on the call path (fixed device-memory budgets, or code that
cannot take cudaMalloc's implicit synchronization). It keeps its scratch in a static
device array, so two calls in a row must give the same result as the context-buffer
entry point dd_schur_apply, within the FP64 operator tolerance of the parity tests.
This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from workload import make_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2412_17543_gb300 as P  # noqa: E402
from paper_2412_17543_gb300 import _native as nat  # noqa: E402

TOL = 1e-12  # FP64 operator tolerance used by the Schur-apply parity tests


def _noalloc(S, x, y):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return S.lib.dd_schur_apply_noalloc(S.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                        stream)


@pytest.mark.parametrize("n,sub,levels,prec", [(16, 4, 2, "fp64"), (24, 8, 2, "df64"), (32, 8, 3, "fp64")])
def test_noalloc_matches_schur_apply_twice(n, sub, levels, prec):
    m = make_mesh(n, sub, 1.3, 20.0)
    S = P.Solver(m, levels=levels, coarse_group=2, schur_prec=prec)
    x = torch.as_tensor(np.random.default_rng(n).standard_normal(S.n_gamma), device="cuda:0")
    ref = S.schur_apply(x)
    torch.cuda.synchronize()
    scale = ref.abs().max().item()
    for _ in range(2):
        y = torch.full_like(x, float("nan"))
        assert _noalloc(S, x, y) == nat.DD_OK, S.lib.dd_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(y).all()
        assert (y - ref).abs().max().item() <= TOL * scale
    S.close()


def test_noalloc_rejects_problem_beyond_scratch():
    m = make_mesh(88, 8, 1.08, 20.0)  # about 11 MiB of scratch needed
    S = P.Solver(m, levels=3)
    need = 8 * (2 * (S.n_free - S.n_gamma))
    assert need > 0
    x = torch.zeros(S.n_gamma, dtype=torch.float64, device="cuda:0")
    y = torch.zeros_like(x)
    code = _noalloc(S, x, y)
    assert code == nat.DD_INVALID_ARG
    msg = S.lib.dd_last_error().decode()
    assert "scratch" in msg and "bytes" in msg
    S.close()
