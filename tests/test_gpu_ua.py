"""UA geometry (the element kernel recomputes J^-1, detJ and the material
factors from the 9 entries of J, Sec. 2's unassembled evaluation of the
data D): parity with the oracle element by element, agreement with the
stored-record apply to FP32 rounding, the mode's admission rules, and the
batched path taking UA operators one by one."""
import numpy as np
import pytest

import oracle
import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MESH_DIMS = {1: (5, 4, 3), 2: (5, 3, 2), 3: (3, 3, 2), 4: (3, 2, 2), 5: (3, 2, 1), 6: (2, 2, 1)}


@pytest.fixture(scope="module")
def pa():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08374_gb300 as pa
    return pa


def _relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("p", range(1, 7))
def test_ua_apply_matches_oracle(pa, p):
    nx, ny, nz = MESH_DIMS[p]
    m = syn.random_affine_cube(nx, seed=300 + p, ny=ny, nz=nz)
    lam, mu = syn.lame(1.0, 0.3)
    ess = syn.clamp_mask(m, p) if p % 2 == 0 else None
    op = pa.Operator(nx, ny, nz, m.affine, p, lam, mu, precision=pa.PA_FP32, ess_mask=ess)
    x = syn.uniform_vector(op.ndofs, seed=30 + p)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    y_rec = op.apply(xt).double().cpu().numpy()
    pa.pa_op_set_geometry_mode(op.h, pa.PA_GEOMETRY_UA)
    assert pa.pa_op_get_launch(op.h)[0] == 5
    y_ua = op.apply(xt).double().cpu().numpy()
    yo = oracle.apply(p, nx, ny, nz, m.affine, lam, mu, x, ess=ess)
    assert _relerr(y_ua, yo) <= 1e-5
    # the same sums from records rounded differently: FP32 rounding apart
    assert _relerr(y_ua, y_rec) <= 2e-6
    if ess is not None:
        e = ess.astype(bool)
        np.testing.assert_array_equal(y_ua[e], x[e].astype(np.float32))
    # back to the stored records: the stored apply's bits again
    pa.pa_op_set_geometry_mode(op.h, pa.PA_GEOMETRY_STORED)
    np.testing.assert_array_equal(op.apply(xt).double().cpu().numpy(), y_rec)
    op.close()


def test_ua_launch_shapes_and_autotune(pa):
    p = 4
    m = syn.random_affine_cube(6, seed=321)
    lam, mu = syn.lame(2.0, 0.35)
    op = pa.Operator(6, 6, 6, m.affine, p, lam, mu, precision=pa.PA_FP32)
    pa.pa_op_set_geometry_mode(op.h, pa.PA_GEOMETRY_UA)
    with pytest.raises(pa.PAError):
        pa.pa_op_set_launch(op.h, 2, 2, 128)
    x = syn.uniform_vector(op.ndofs, seed=32)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    yo = oracle.apply(p, 6, 6, 6, m.affine, lam, mu, x)
    for epb, th in [(1, 64), (3, 96), (8, 128), (13, 256)]:
        pa.pa_op_set_launch(op.h, 5, epb, th)
        assert _relerr(op.apply(xt).double().cpu().numpy(), yo) <= 1e-5
    pa.pa_op_autotune(op.h)
    assert pa.pa_op_get_launch(op.h)[0] == 5
    assert _relerr(op.apply(xt).double().cpu().numpy(), yo) <= 1e-5
    op.close()


def test_ua_admission_rules(pa):
    m = syn.random_affine_cube(2, seed=322)
    lam, mu = syn.lame(1.0, 0.3)
    op64 = pa.Operator(2, 2, 2, m.affine, 2, lam, mu, precision=pa.PA_FP64)
    with pytest.raises(pa.PAError):
        pa.pa_op_set_geometry_mode(op64.h, pa.PA_GEOMETRY_UA)
    op64.close()
    op8 = pa.Operator(2, 2, 2, m.affine, 8, lam, mu, precision=pa.PA_FP32)
    with pytest.raises(pa.PAError):
        pa.pa_op_set_geometry_mode(op8.h, pa.PA_GEOMETRY_UA)
    op8.close()
    op = pa.Operator(2, 2, 2, m.affine, 2, lam, mu, precision=pa.PA_FP32)
    with pytest.raises(pa.PAError):
        pa.pa_op_set_geometry_mode(op.h, 7)
    mat = np.tile([lam, mu], (8, 1))
    pa.pa_op_set_material(op.h, mat)
    with pytest.raises(pa.PAError):
        pa.pa_op_set_geometry_mode(op.h, pa.PA_GEOMETRY_UA)
    pa.pa_op_set_material(op.h, None)
    pa.pa_op_set_geometry_mode(op.h, pa.PA_GEOMETRY_UA)
    with pytest.raises(pa.PAError):
        pa.pa_op_set_material(op.h, mat)
    op.close()


def test_ua_operator_in_a_batch(pa):
    """A batch holding a UA operator and stored-record operators: each
    member's output is bitwise its own apply's."""
    lam, mu = syn.lame(1.0, 0.3)
    ops, xs = [], []
    for k, (p, n) in enumerate([(2, 4), (4, 3), (2, 5), (6, 2)]):
        m = syn.random_affine_cube(n, seed=330 + k)
        op = pa.Operator(n, n, n, m.affine, p, lam, mu, precision=pa.PA_FP32)
        if k == 1:
            pa.pa_op_set_geometry_mode(op.h, pa.PA_GEOMETRY_UA)
        ops.append(op)
        xs.append(torch.tensor(syn.uniform_vector(op.ndofs, seed=40 + k), dtype=torch.float32, device="cuda"))
    solo = [o.apply(x).clone() for o, x in zip(ops, xs)]
    ys = [torch.empty_like(x) for x in xs]
    pa.pa_op_apply_batch([o.h for o in ops], xs, ys)
    torch.cuda.synchronize()
    for a, b in zip(ys, solo):
        assert torch.equal(a, b)
    for o in ops:
        o.close()
