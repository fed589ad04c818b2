"""The C ABI library loads without a GPU and exports every entry point that
include/pa_elasticity.h declares; host-only entry points validate their
arguments.  No compute call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pa_elasticity.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pa_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def pa():
    path = os.path.join(ROOT, "paper_2601_08374_gb300", "_build", "libpa_elasticity.so")
    if not os.path.exists(path):
        import importlib.util
        spec = importlib.util.spec_from_file_location("_pa_build", os.path.join(ROOT, "paper_2601_08374_gb300", "build.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        mod.build()
    import paper_2601_08374_gb300 as pa
    return pa


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ["pa_mesh_create", "pa_op_setup", "pa_op_apply", "pa_op_diag", "pa_gmg_pcg_solve",
                 "pa_solver_create", "pa_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(pa):
    missing = [n for n in declared_functions() if not hasattr(pa.lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_host_only_entry_points(pa):
    assert pa.pa_version() >= 100
    lam, mu = pa.pa_lame(1.0, 0.3)
    assert abs(lam - 0.3 / (1.3 * 0.4)) < 1e-15 and abs(mu - 1 / 2.6) < 1e-15
    with pytest.raises(pa.PAError) as ei:
        pa.pa_lame(1.0, 0.5)
    assert ei.value.code == pa.PA_EINVAL
    with pytest.raises(pa.PAError) as ei:
        pa.pa_mesh_create(0, 1, 1)
    assert ei.value.code == pa.PA_EINVAL and "dimensions" in str(ei.value)
    bad = np.zeros((2, 12))
    bad[:, [0, 4, 8]] = 1.0
    bad[1, 8] = -1.0  # det J < 0 in element 1
    with pytest.raises(pa.PAError) as ei:
        pa.pa_mesh_create(2, 1, 1, affine=bad)
    assert "element 1" in str(ei.value)
    h = pa.pa_mesh_create(3, 2, 1, box=[0, 0, 0, 3, 2, 1])
    pa.pa_mesh_destroy(h)


def test_argument_checks_before_any_device_call(pa):
    """Null handles, negative counts and bad level lists are refused with
    PA_EINVAL and a message before any CUDA call (so without a GPU)."""
    import ctypes
    lib = pa.lib
    assert lib.pa_op_apply_add(None, None, None, None) == pa.PA_EINVAL
    assert lib.pa_op_apply_host_batch(None, None, None, -1, None) == pa.PA_EINVAL
    assert lib.pa_op_apply_host_batch(None, None, None, 0, None) == pa.PA_OK
    assert lib.pa_gmg_pcg_solve_batch(None, None, None, -1, 1e-10, 10, None, None) == pa.PA_EINVAL
    assert lib.pa_op_prolong(None, None, None, None, None) == pa.PA_EINVAL
    assert lib.pa_op_restrict(None, None, None, None, None) == pa.PA_EINVAL
    out = ctypes.c_void_p()
    lv = (ctypes.c_int * 3)(4, 2, 1)
    assert lib.pa_solver_create_hp(None, 3, lv, 1, 2, 1e-2, 10, 0, ctypes.byref(out)) == pa.PA_EINVAL
    assert not out.value
    assert lib.pa_solver_create_hp(None, 3, lv, 1, 2, 1e-2, 10, 0, None) == pa.PA_EINVAL
    assert b"null" in lib.pa_last_error()


def test_flop_model_reproduces_table6():
    """bench.flops_per_element against the per-element counts printed in
    Table 6 of the paper (tests/golden/table6_flops.txt)."""
    import bench
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "table6_flops.txt"))
            if l.strip() and not l.startswith("#")]
    for p, D, Q, fe, fd in rows:
        p = int(p)
        assert bench.flops_per_element(p) == int(fe)
        assert round(bench.flops_per_element(p) / (3 * p ** 3)) == int(fd)
