"""CPU-side checks of the native library: exports and host-side setup against the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import dd
from workload import FACE_X1, make_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    import paper_2412_17543_gb300 as P
    try:
        return P.load()
    except RuntimeError as e:
        pytest.skip(str(e))


def _declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(dd_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = _lib()
    names = _declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    from paper_2412_17543_gb300 import _native
    assert set(names) == set(_native.SIGNATURES), "binding must declare exactly the header's functions"


def test_binding_struct_layouts_match_the_library():
    """The ctypes mirrors of the public structs have the C sizes (a field added on one side
    only would shift every later field); the defaults read back through them."""
    lib = _lib()
    from paper_2412_17543_gb300 import _native as nat
    sizes = (ctypes.c_size_t * 5)()
    lib.dd_abi_struct_sizes(sizes)
    mine = [ctypes.sizeof(c) for c in (nat.MeshDesc, nat.Options, nat.Info, nat.Stats, nat.KernelProf)]
    assert list(sizes) == mine
    o = nat.Options()
    assert lib.dd_default_options(ctypes.byref(o)) == 0
    assert (o.levels, o.maxit, o.loop_graph, o.ens_nmm, o.ens_elem_rc, o.ens_fdm_rc) == (3, 500, 1, 0, 0, 0)


@pytest.mark.parametrize("n,sub,levels,kinds,dirichlet", [(16, 4, 2, dict(use_edges=0), FACE_X1), (16, 2, 3, {}, FACE_X1),
                                                          (12, 4, 2, {}, FACE_X1), (16, 4, 2, {}, 0), (16, 2, 3, {}, 0)])
def test_plan_matches_oracle_partition(n, sub, levels, kinds, dirichlet):
    """Host setup against the oracle's partition; dirichlet = 0 is the pure-Neumann case
    (semidefinite K: the coarse matrices are inverted in grounded form)."""
    _lib()
    import paper_2412_17543_gb300 as P
    m = make_mesh(n, sub, 1.08, 20.0, dirichlet=dirichlet)
    info, nodes = P.plan(m, levels=levels, coarse_group=4, **kinds)
    assert info["neumann"] == (dirichlet == 0)
    subs = dd.q1_substructures(m)
    assert info["n_free"] == m.n_free
    assert info["n_gamma"] == len(subs.gamma)
    assert np.array_equal(nodes, subs.gamma)
    sel = (dd.CORNER, dd.FACE) if kinds.get("use_edges", 1) == 0 else (dd.CORNER, dd.EDGE, dd.FACE)
    nC = sum(1 for k in subs.glob_kind if k in sel)
    assert info["n_coarse"] == nC
    if levels == 3:
        Pc = dd.Preconditioner(subs, 3, sel, group=4)
        assert info["n_sub2"] == Pc.subs2.S
        assert info["n_coarse3"] == Pc.l2.nC


def test_plan_rejects_bad_input():
    _lib()
    import paper_2412_17543_gb300 as P
    m = make_mesh(10, 4)  # 4 does not divide 10
    with pytest.raises(P.DDError) as e:
        P.plan(m, levels=2)
    assert e.value.code == 1
    m = make_mesh(8, 4, dirichlet=0)  # pure Neumann takes no adaptive constraints
    with pytest.raises(P.DDError):
        P.plan(m, levels=2, adaptive=1)
    m = make_mesh(8, 4, coef=-np.ones((8, 8, 8)))
    with pytest.raises(P.DDError):
        P.plan(m, levels=2)


@pytest.mark.parametrize("tau", [1.5, 3.0])
def test_plan_adaptive_count_matches_oracle(tau):
    _lib()
    import paper_2412_17543_gb300 as P
    rng = np.random.default_rng(5)
    n = 8
    coef = np.exp(2.0 * rng.standard_normal((n, n, n)))
    m = make_mesh(n, 4, 1.08, 20.0, coef=coef)
    subs = dd.q1_substructures(m)
    base = dd.Preconditioner(subs, 2, (dd.CORNER, dd.EDGE, dd.FACE), "diag")
    rows = dd.adaptive_face_constraints(subs, base.l1.D, tau=tau)
    info, _ = P.plan(m, levels=2, adaptive=1, tau=tau, weights="diag")
    assert info["n_adaptive"] == sum(len(r) for r in rows.values())


@pytest.mark.parametrize("field,value", [("loop_graph", 2), ("zero_initial_guess", -1), ("ens_elem_rc", 3),
                                         ("ens_fdm_rc", 16), ("ens_nmm", 7), ("maxit", 0), ("schur_prec", 1)])
def test_setup_validates_options_before_any_device_work(field, value):
    """dd_setup rejects an invalid option with DD_INVALID_ARG and a message naming it; the
    checks come before any device call, so they run without a GPU."""
    lib = _lib()
    from paper_2412_17543_gb300 import _native as nat
    from paper_2412_17543_gb300.api import _mesh_desc, make_options
    keep = []
    d = _mesh_desc(make_mesh(8, 4), keep)
    o = make_options()
    setattr(o, field, value)
    h = ctypes.c_void_p()
    code = lib.dd_setup(ctypes.byref(d), ctypes.byref(o), None, ctypes.byref(h))
    assert code == 1 and not h.value
    msg = lib.dd_last_error().decode()
    assert field.split("_")[0] in msg or field in msg, msg


@pytest.mark.parametrize("bad", [0.0, -1e-3, float("nan"), float("inf")])
def test_plan_rejects_nonpositive_or_nonfinite_coefficient(bad):
    """One bad k_e among valid ones makes K indefinite, singular or undefined: setup refuses
    it with DD_INVALID_ARG before any factorization (host-side failure detection)."""
    _lib()
    import paper_2412_17543_gb300 as P
    coef = np.ones((8, 8, 8))
    coef[3, 5, 2] = bad
    with pytest.raises(P.DDError) as e:
        P.plan(make_mesh(8, 4, coef=coef), levels=2)
    assert e.value.code == 1
    assert "coefficient" in str(e.value)
