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


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_oracle(pa, prec):
    """The allocation-free path on its own scratch layout (geometry records
    from the caller's maps, the 256-byte-rounded element-vector offset)
    against the CPU oracle, at the operator tolerances."""
    import oracle
    nx, ny, nz, p = 3, 2, 2, 3  # 12 elements: geometry part 576 / 1152 bytes, not a multiple of 256
    m = syn.random_affine_cube(nx, seed=77, ny=ny, nz=nz)
    lam, mu = syn.lame(1.0, 0.3)
    ess = syn.clamp_mask(m, p)
    n = m.n_dofs(p)
    xh = syn.uniform_vector(n, seed=78)
    dt = torch.float64 if prec == 0 else torch.float32
    aff = torch.tensor(m.affine, dtype=torch.float64, device="cuda")
    mask = torch.tensor(ess, dtype=torch.uint8, device="cuda")
    x = torch.tensor(xh, dtype=dt, device="cuda")
    y = torch.full_like(x, float("nan"))
    pa.pa_apply_noalloc(nx, ny, nz, p, lam, mu, prec, aff, x, y, ess_mask=mask)
    torch.cuda.synchronize()
    xin = x.double().cpu().numpy()  # the FP32 path's input as the oracle sees it
    yo = oracle.apply(p, nx, ny, nz, m.affine, lam, mu, xin, ess=ess)
    err = np.max(np.abs(y.double().cpu().numpy() - yo)) / np.max(np.abs(yo))
    assert err <= TOL[prec], err


def test_noalloc_bad_map_gives_nan(pa):
    """An element map with det J <= 0 turns every entry of y into NaN (the
    entry point has no host round trip to report it otherwise); the next
    call with good maps is clean again."""
    nx, ny, nz, p = 2, 2, 1, 2
    m = syn.box_mesh(nx, ny, nz)
    aff_h = m.affine.copy()
    aff_h[3, 8] = -aff_h[3, 8]  # element 3 mirrored: det J < 0
    x = torch.tensor(syn.uniform_vector(m.n_dofs(p), seed=5), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    pa.pa_apply_noalloc(nx, ny, nz, p, 1.0, 1.0, pa.PA_FP64, torch.tensor(aff_h, device="cuda"), x, y)
    torch.cuda.synchronize()
    assert torch.isnan(y).all()
    pa.pa_apply_noalloc(nx, ny, nz, p, 1.0, 1.0, pa.PA_FP64, torch.tensor(m.affine, device="cuda"), x, y)
    torch.cuda.synchronize()
    assert torch.isfinite(y).all()
