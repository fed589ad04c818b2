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
    assert lib.pa_server_cancel(None, 1) == pa.PA_EINVAL
    assert lib.pa_op_set_wait_limit(None, 1.0) == pa.PA_EINVAL
    assert lib.pa_solver_set_option(None, pa.PA_SOLVER_OPT_WAIT_LIMIT, 1.0) == pa.PA_EINVAL
    t = ctypes.c_double()
    assert lib.pa_measure_fma_rate(7, ctypes.byref(t), None) == pa.PA_EINVAL
    assert lib.pa_measure_fma_rate(0, None, None) == pa.PA_EINVAL
    assert lib.pa_op_set_geometry_mode(None, pa.PA_GEOMETRY_UA) == pa.PA_EINVAL


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


def test_noalloc_refuses_overflowing_sizes_and_overlaps(pa):
    """pa_apply_noalloc checks the mesh sizes with overflow-safe products and
    refuses overlapping x / y / mask / affine ranges, all before any device
    call (the pointers below are never dereferenced)."""
    lib = pa.lib
    fake = [ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 30), ctypes.c_void_p(1 << 40)]
    big = 1 << 21  # 2^63 elements as a product: must not wrap past the limits
    for dims in [(big, big, big), (1 << 30, 1 << 30, 1), ((1 << 31) - 1, 1, 1), (1 << 16, 1 << 16, 2)]:
        rc = lib.pa_apply_noalloc(*dims, 8, 1.0, 1.0, pa.PA_FP64, fake[0], None, fake[1], fake[2], None)
        assert rc == pa.PA_EINVAL, dims
        assert b"too many" in lib.pa_last_error() or b"exceed" in lib.pa_last_error()
    # x and y overlapping by one entry (2 x 2 x 2 elements, p = 1: 81 dofs)
    x = ctypes.c_void_p(1 << 20)
    y = ctypes.c_void_p((1 << 20) + 80 * 8)
    rc = lib.pa_apply_noalloc(2, 2, 2, 1, 1.0, 1.0, pa.PA_FP64, ctypes.c_void_p(1 << 30), None, x, y, None)
    assert rc == pa.PA_EINVAL and b"x and y overlap" in lib.pa_last_error()
    rc = lib.pa_apply_noalloc(2, 2, 2, 1, 1.0, 1.0, pa.PA_FP64, ctypes.c_void_p((1 << 20) + 8), None,
                              ctypes.c_void_p(1 << 30), ctypes.c_void_p(1 << 20), None)
    assert rc == pa.PA_EINVAL and b"affine and y overlap" in lib.pa_last_error()
    rc = lib.pa_apply_noalloc(2, 2, 2, 1, 1.0, 1.0, pa.PA_FP64, ctypes.c_void_p(1 << 30),
                              ctypes.c_void_p((1 << 20) + 640), ctypes.c_void_p(1 << 40), ctypes.c_void_p(1 << 20), None)
    assert rc == pa.PA_EINVAL and b"ess_mask and y overlap" in lib.pa_last_error()


def test_noalloc_binding_checks_tensors(pa):
    """The Python wrapper of pa_apply_noalloc refuses tensors of the wrong
    dtype, shape, length, layout or device with ValueError (CPU tensors
    reach the device check last)."""
    torch = pytest.importorskip("torch")
    nx, ny, nz, p = 2, 1, 1, 2
    ne, nd = 2, 3 * 5 * 3 * 3
    good = dict(affine=torch.zeros(ne, 12, dtype=torch.float64), x=torch.zeros(nd, dtype=torch.float64),
                y=torch.zeros(nd, dtype=torch.float64), ess_mask=torch.zeros(nd, dtype=torch.uint8))
    bad_cases = [
        ("affine", torch.zeros(ne, 12, dtype=torch.float32), "float64"),
        ("affine", torch.zeros(ne * 12, dtype=torch.float64), "shape"),
        ("affine", torch.zeros(12, ne, dtype=torch.float64).t(), "contiguous"),
        ("x", torch.zeros(nd, dtype=torch.float32), "float64"),
        ("x", torch.zeros(nd + 1, dtype=torch.float64), "entries"),
        ("y", torch.zeros(nd - 3, dtype=torch.float64), "entries"),
        ("y", torch.zeros(2 * nd, dtype=torch.float64)[::2], "contiguous"),
        ("ess_mask", torch.zeros(nd, dtype=torch.bool), "uint8"),
        ("ess_mask", torch.zeros(nd - 1, dtype=torch.uint8), "entries"),
        ("x", None, "CUDA"),  # every tensor right but on the CPU
    ]
    for name, t, word in bad_cases:
        args = dict(good)
        if t is not None:
            args[name] = t
        with pytest.raises(ValueError) as ei:
            pa.pa_apply_noalloc(nx, ny, nz, p, 1.0, 1.0, pa.PA_FP64, args["affine"], args["x"], args["y"],
                                ess_mask=args["ess_mask"])
        assert word in str(ei.value), (name, word, str(ei.value))
    with pytest.raises(ValueError):
        pa.pa_apply_noalloc(nx, ny, nz, p, 1.0, 1.0, 7, good["affine"], good["x"], good["y"])


def test_noalloc_rejects_meshes_beyond_the_scratch(pa):
    """A mesh whose scratch exceeds the fixed 64 MiB array is refused with
    PA_EINVAL and the required size, before any device call (the pointers
    are placeholders that are never dereferenced)."""
    lib = pa.lib
    n = 40  # p = 8: 64000 elements x 2199 doubles each, far above 64 MiB
    rc = lib.pa_apply_noalloc(n, n, n, 8, 1.0, 1.0, pa.PA_FP64, ctypes.c_void_p(1 << 44), None,
                              ctypes.c_void_p(1 << 40), ctypes.c_void_p(1 << 42), None)
    assert rc == pa.PA_EINVAL and b"64 MiB" in lib.pa_last_error()
