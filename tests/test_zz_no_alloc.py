"""pa_apply_noalloc -- the operator apply for callers that cannot call
cudaMalloc (their framework owns all device memory, or they must not block on
the allocator) -- gives the same result as the regular pa_op_setup +
pa_op_apply path, on two calls in a row that share its fixed scratch array.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}  # the tolerances of the operator parity tests


@pytest.fixture(scope="module")
def pa():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08374_gb300 as pa
    return pa


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p,dims", [(2, (5, 3, 2)), (4, (3, 3, 2)), (8, (2, 2, 1))])
def test_noalloc_matches_regular_apply_twice(pa, p, dims, prec):
    nx, ny, nz = dims
    m = syn.random_affine_cube(nx, seed=500 + p, ny=ny, nz=nz)
    lam, mu = syn.lame(1.0, 0.3)
    ess = syn.clamp_mask(m, p)
    op = pa.Operator(nx, ny, nz, m.affine, p, lam, mu, precision=prec, ess_mask=ess)
    aff = torch.tensor(m.affine, dtype=torch.float64, device="cuda")
    mask = torch.tensor(ess, dtype=torch.uint8, device="cuda")
    for call, seed in enumerate((11, 12)):  # two calls in a row, different inputs
        x = torch.tensor(syn.uniform_vector(op.ndofs, seed=seed), dtype=op.dtype, device="cuda")
        y_ref = op.apply(x)
        y = torch.full_like(x, float("nan"))
        pa.pa_apply_noalloc(nx, ny, nz, p, lam, mu, prec, aff, x, y, ess_mask=mask)
        torch.cuda.synchronize()
        a, b = y.double().cpu().numpy(), y_ref.double().cpu().numpy()
        err = np.max(np.abs(a - b)) / np.max(np.abs(b))
        assert err <= TOL[prec], (call, err)
    op.close()


def test_noalloc_rejects_meshes_beyond_the_scratch(pa):
    n = 40  # p = 8: 64000 elements x 2199 doubles each, far above 64 MiB
    aff = torch.zeros((n ** 3, 12), dtype=torch.float64, device="cuda")
    x = torch.zeros(3, dtype=torch.float64, device="cuda")
    y = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(pa.PAError) as ei:
        pa.pa_apply_noalloc(n, n, n, 8, 1.0, 1.0, pa.PA_FP64, aff, x, y)
    assert ei.value.code == pa.PA_EINVAL and "64 MiB" in str(ei.value)
