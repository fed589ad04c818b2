"""Parity of the CUDA operator (apply, diagonal, load vector) with the CPU
oracle, element by element, through the C ABI.

Tolerances (relative max-norm, against max |oracle|): FP64 1e-12, FP32 1e-5.
"""
import numpy as np
import pytest

import oracle
import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def pa():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08374_gb300 as pa
    return pa


def _relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _run_apply(pa, mesh, p, lam, mu, x, prec, ess=None):
    op = pa.Operator(mesh.nx, mesh.ny, mesh.nz, mesh.affine, p, lam, mu, precision=prec, ess_mask=ess)
    xt = torch.tensor(x, dtype=op.dtype, device="cuda")
    y = op.apply(xt)
    torch.cuda.synchronize()
    out = y.double().cpu().numpy()
    op.close()
    return out


# meshes with several CTAs and a ragged last CTA for every degree
MESH_DIMS = {1: (5, 4, 3), 2: (5, 3, 2), 3: (3, 3, 2), 4: (3, 2, 2), 5: (3, 2, 1), 6: (2, 2, 1), 7: (3, 1, 1),
             8: (2, 1, 1)}


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", range(1, 9))
def test_apply_random_affine(pa, p, prec):
    nx, ny, nz = MESH_DIMS[p]
    m = syn.random_affine_cube(nx, seed=100 + p, ny=ny, nz=nz)
    lam, mu = syn.lame(1.0, 0.3)
    x = syn.uniform_vector(m.n_dofs(p), seed=p)
    y = _run_apply(pa, m, p, lam, mu, x, prec)
    yo = oracle.apply(p, nx, ny, nz, m.affine, lam, mu, x)
    assert _relerr(y, yo) <= TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_config_small_cube_clamped(pa, prec):
    # 4x4x4 unit cube, p = 2, E = 1, nu = 0.3, x = 0 face clamped, x ~ U[-1,1] seed 0
    m = syn.box_mesh(4, 4, 4)
    p = 2
    lam, mu = syn.lame(1.0, 0.3)
    ess = syn.clamp_mask(m, p)
    x = syn.uniform_vector(m.n_dofs(p), seed=0)
    assert len(x) == 2187
    y = _run_apply(pa, m, p, lam, mu, x, prec, ess)
    yo = oracle.apply(p, 4, 4, 4, m.affine, lam, mu, x, ess=ess)
    assert _relerr(y, yo) <= TOL[prec]
    e = ess.astype(bool)
    if prec == 0:
        np.testing.assert_array_equal(y[e], x[e])


@pytest.mark.parametrize("p", [1, 4, 8])
def test_single_element_and_thin_meshes(pa, p):
    lam, mu = 0.8, 0.5
    for dims in [(1, 1, 1), (1, 3, 1), (2, 1, 3)]:
        m = syn.random_affine_cube(dims[0], seed=7, ny=dims[1], nz=dims[2])
        x = syn.uniform_vector(m.n_dofs(p), seed=3)
        y = _run_apply(pa, m, p, lam, mu, x, 0)
        yo = oracle.apply(p, *dims, m.affine, lam, mu, x)
        assert _relerr(y, yo) <= 1e-12


@pytest.mark.parametrize("p", [1, 2, 4, 6, 8])
def test_apply_full_size_sweep_sampled(pa, p):
    """Operator-sweep size (~3M dofs, the benchmark's launch configuration):
    sampled rows checked one by one against the oracle's element-matrix rows."""
    n = syn.sweep_n(p)
    m = syn.random_affine_cube(n, seed=1000 + p)
    lam, mu = syn.lame(1.0, 0.3)
    N = m.n_dofs(p)
    x = syn.uniform_vector(N, seed=2000 + p)
    for prec in (0, 1):
        y = _run_apply(pa, m, p, lam, mu, x, prec)
        rng = np.random.default_rng(p)
        rows = np.concatenate([rng.choice(N, 1500, replace=False), [0, N - 1, N // 3, N // 3 - 1]])
        yo = oracle.apply_rows(p, n, n, n, m.affine, lam, mu, x, rows)
        scale = np.max(np.abs(yo))
        assert np.max(np.abs(y[rows] - yo)) <= TOL[prec] * scale


def test_apply_is_deterministic_and_host_path(pa):
    p = 3
    m = syn.random_affine_cube(3, seed=5)
    lam, mu = syn.lame(1.0, 0.3)
    op = pa.Operator(m.nx, m.ny, m.nz, m.affine, p, lam, mu)
    x = torch.tensor(syn.uniform_vector(m.n_dofs(p), 1), device="cuda", dtype=torch.float64)
    y1 = op.apply(x)
    y2 = op.apply(x)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    pa.pa_op_apply_host(op.h, xh, yh)
    assert torch.equal(yh, y1.cpu())
    with pytest.raises(pa.PAError):
        pa.pa_op_apply(op.h, x, x)
    op.close()


def test_host_batch_apply_equals_device_applies(pa):
    """Several operators (both precisions, several degrees) applied from
    pinned host buffers with the copies overlapped: the same bits as one
    device apply each; a repeated operator is refused."""
    ops, xs, ys_dev, probs = [], [], [], []
    for k, (p, prec) in enumerate([(2, pa.PA_FP64), (4, pa.PA_FP32), (1, pa.PA_FP64), (3, pa.PA_FP32)]):
        m = syn.random_affine_cube(3 + k, seed=60 + k)
        op = pa.Operator(m.nx, m.ny, m.nz, m.affine, p, 1.0, 0.5, precision=prec)
        dt = torch.float64 if prec == pa.PA_FP64 else torch.float32
        x = torch.tensor(syn.uniform_vector(op.ndofs, seed=k), dtype=dt, device="cuda")
        ops.append(op)
        xs.append(x)
        ys_dev.append(op.apply(x))
        probs.append((p, prec, m))
    torch.cuda.synchronize()
    xh = [x.cpu().pin_memory() for x in xs]
    yh = [torch.full_like(h, float("nan")).pin_memory() for h in xh]
    pa.pa_op_apply_host_batch([o.h for o in ops], xh, yh)
    for a, b in zip(yh, ys_dev):
        assert torch.equal(a, b.cpu())
    # each member against the oracle's apply
    for a, x, (p, prec, m) in zip(yh, xh, probs):
        yo = oracle.apply(p, m.nx, m.ny, m.nz, m.affine, 1.0, 0.5, x.double().numpy())
        assert _relerr(a.double().numpy(), yo) <= TOL[prec], (p, prec)
    with pytest.raises(pa.PAError) as ei:
        pa.pa_op_apply_host_batch([ops[0].h, ops[0].h], xh[:1] * 2, yh[:1] * 2)
    assert ei.value.code == pa.PA_EINVAL
    for op in ops:
        op.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 4, 8])
def test_diag(pa, p, prec):
    m = syn.random_affine_cube(2, seed=40 + p, ny=2, nz=1)
    lam, mu = syn.lame(2.0, 0.45)
    ess = syn.clamp_mask(m, p)
    op = pa.Operator(m.nx, m.ny, m.nz, m.affine, p, lam, mu, precision=prec, ess_mask=ess)
    d = op.diag().double().cpu().numpy()
    op.close()
    do = oracle.diag(p, m.nx, m.ny, m.nz, m.affine, lam, mu, ess=ess)
    assert _relerr(d, do) <= TOL[prec]


@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_rhs(pa, p):
    m = syn.random_affine_cube(3, seed=60 + p, nz=2)
    ess = syn.clamp_mask(m, p)
    modes = syn.smooth_force_modes(seed=p)
    op = pa.Operator(m.nx, m.ny, m.nz, m.affine, p, 1.0, 1.0, ess_mask=ess)
    F = op.rhs(f0=(0.0, 0.0, -1.0), modes=modes).cpu().numpy()
    op.close()
    Fo = oracle.load(p, m.nx, m.ny, m.nz, m.affine, f0=(0.0, 0.0, -1.0), modes=modes, ess=ess)
    assert _relerr(F, Fo) <= 1e-12


LINE_OK = {0: range(1, 5), 1: range(1, 9)}


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", range(1, 9))
def test_apply_register_tiled_variant(pa, p, prec, variant):
    """The register-tiled kernels (variant 1; variant 2 with the gather and
    the store fused into the X sweeps; variant 3, variant 2 with three lanes
    per quadrature column) against the oracle, with several CTA shapes (some
    leaving a ragged last CTA or a partly idle last warp)."""
    if variant in (1, 2) and p not in LINE_OK[prec]:
        pytest.skip("variants 1 and 2 not instantiated for this degree in FP64")
    nx, ny, nz = MESH_DIMS[p]
    m = syn.random_affine_cube(nx, seed=300 + p, ny=ny, nz=nz)
    lam, mu = syn.lame(1.0, 0.3)
    ess = syn.clamp_mask(m, p)
    x = syn.uniform_vector(m.n_dofs(p), seed=7 + p)
    yo = oracle.apply(p, nx, ny, nz, m.affine, lam, mu, x, ess=ess)
    op = pa.Operator(nx, ny, nz, m.affine, p, lam, mu, precision=prec, ess_mask=ess)
    xt = torch.tensor(x, dtype=op.dtype, device="cuda")
    ran = 0
    for epb, th in [(1, 128), (7, 256), (3, 256), (2, 32)]:
        try:
            pa.pa_op_set_launch(op.h, variant, epb, th)
        except pa.PAError as e:  # shape beyond the shared-memory limit for this degree
            assert e.code == pa.PA_EINVAL
            continue
        y = op.apply(xt).double().cpu().numpy()
        assert _relerr(y, yo) <= TOL[prec], (epb, th)
        ran += 1
    assert ran >= 2
    op.close()


@pytest.mark.parametrize("p", range(1, 9))
def test_apply_two_pass_column_variant(pa, p):
    """Variant 7 (FP32 line kernel whose fused Z stage runs in two passes
    through shared memory) against the oracle with several CTA shapes,
    constrained, and bitwise against variant 2 (the same terms in the same
    order); in a batched launch it equals its single applies."""
    nx, ny, nz = MESH_DIMS[p]
    m = syn.random_affine_cube(nx, seed=360 + p, ny=ny, nz=nz)
    lam, mu = syn.lame(1.0, 0.3)
    ess = syn.clamp_mask(m, p)
    op = pa.Operator(nx, ny, nz, m.affine, p, lam, mu, precision=pa.PA_FP32, ess_mask=ess)
    xt = torch.tensor(syn.uniform_vector(op.ndofs, seed=27 + p), dtype=op.dtype, device="cuda")
    yo = oracle.apply(p, nx, ny, nz, m.affine, lam, mu, xt.double().cpu().numpy(), ess=ess)
    pa.pa_op_set_launch(op.h, 2, 1, 128)
    y2 = op.apply(xt).clone()
    ran = 0
    for epb, th in [(1, 64), (3, 96), (2, 128), (5, 256)]:
        try:
            pa.pa_op_set_launch(op.h, 7, epb, th)
        except pa.PAError as e:
            assert e.code == pa.PA_EINVAL
            continue
        y = op.apply(xt)
        assert _relerr(y.double().cpu().numpy(), yo) <= TOL[1], (epb, th)
        assert torch.equal(y, y2), (epb, th)
        ran += 1
    assert ran >= 2
    pa.pa_op_set_launch(op.h, 7, 1, 128)
    ys = torch.full_like(xt, float("nan"))
    pa.pa_op_apply_batch([op.h], [xt], [ys])
    torch.cuda.synchronize()
    assert torch.equal(ys, y2)
    op.close()


@pytest.mark.parametrize("variant", [5, 6])
@pytest.mark.parametrize("p", range(1, 9))
def test_apply_plane_fused_variant(pa, p, variant):
    """The plane-fused FP32 kernels (variant 5: X+Y and Y^T+X^T sweeps per
    plane in registers, one thread per column in the fused Z stage; variant
    6: three lanes per column) against the oracle with several CTA shapes
    (ragged last CTA, partly idle warps), constrained; they sum in the order
    of the line variants 2 and 3 (same column code), so their results are
    bitwise those; the batched launch of variant 5/6 operators equals their
    single applies."""
    if variant == 5 and p > 6:
        pytest.skip("variant 5 is instantiated for p <= 6")
    nx, ny, nz = MESH_DIMS[p]
    m = syn.random_affine_cube(nx, seed=330 + p, ny=ny, nz=nz)
    lam, mu = syn.lame(1.0, 0.3)
    ess = syn.clamp_mask(m, p)
    x = syn.uniform_vector(m.n_dofs(p), seed=17 + p)
    op = pa.Operator(nx, ny, nz, m.affine, p, lam, mu, precision=pa.PA_FP32, ess_mask=ess)
    xt = torch.tensor(x, dtype=op.dtype, device="cuda")
    yo = oracle.apply(p, nx, ny, nz, m.affine, lam, mu, xt.double().cpu().numpy(), ess=ess)
    pa.pa_op_set_launch(op.h, 2 if variant == 5 else 3, 1, 128)
    y2 = op.apply(xt).clone()
    ran = 0
    for epb, th in [(1, 64), (5, 256), (3, 96), (2, 32), (16, 256)]:
        try:
            pa.pa_op_set_launch(op.h, variant, epb, th)
        except pa.PAError as e:  # shape beyond the shared-memory limit for this degree
            assert e.code == pa.PA_EINVAL
            continue
        y = op.apply(xt)
        assert _relerr(y.double().cpu().numpy(), yo) <= TOL[1], (epb, th)
        assert torch.equal(y, y2), (epb, th)
        ran += 1
    assert ran >= 3
    with pytest.raises(pa.PAError):
        pa.pa_op_set_launch(op.h, variant, 1, 512)  # at most 256 threads
    # two operators of this degree in one batched launch of the variant
    pa.pa_op_set_launch(op.h, variant, 3, 128)
    op2 = pa.Operator(nx, ny, nz, m.affine, p, 2.0, 0.5, precision=pa.PA_FP32)
    pa.pa_op_set_launch(op2.h, variant, 3, 128)
    x2 = torch.tensor(syn.uniform_vector(op2.ndofs, seed=3), dtype=op2.dtype, device="cuda")
    r1, r2 = op.apply(xt).clone(), op2.apply(x2).clone()
    ys = [torch.full_like(xt, float("nan")), torch.full_like(x2, float("nan"))]
    pa.pa_op_apply_batch([op.h, op2.h], [xt, x2], ys)
    torch.cuda.synchronize()
    assert torch.equal(ys[0], r1) and torch.equal(ys[1], r2)
    op.close()
    op2.close()


def test_plane_variants_are_fp32_only(pa):
    m = syn.box_mesh(2, 2, 2)
    op = pa.Operator(2, 2, 2, m.affine, 2, 1.0, 1.0, precision=pa.PA_FP64)
    for v in (5, 6, 7):
        with pytest.raises(pa.PAError) as ei:
            pa.pa_op_set_launch(op.h, v, 2, 128)
        assert ei.value.code == pa.PA_EINVAL
    op.close()


def test_autotune_keeps_parity(pa):
    p = 4
    m = syn.random_affine_cube(4, seed=9)
    lam, mu = syn.lame(1.0, 0.3)
    x = syn.uniform_vector(m.n_dofs(p), seed=1)
    yo = oracle.apply(p, 4, 4, 4, m.affine, lam, mu, x)
    for prec in (0, 1):
        op = pa.Operator(4, 4, 4, m.affine, p, lam, mu, precision=prec)
        cfg = pa.pa_op_autotune(op.h)
        assert cfg[0] in range(8) and cfg[1] >= 1 and cfg[2] % 32 == 0  # any admissible variant 0-7
        y = op.apply(torch.tensor(x, dtype=op.dtype, device="cuda")).double().cpu().numpy()
        assert _relerr(y, yo) <= TOL[prec]
        op.close()


@pytest.mark.parametrize("pc,pf", [(1, 2), (2, 4), (4, 8), (1, 3), (3, 6)])
def test_transfers_against_oracle(pa, pc, pf):
    m = syn.random_affine_cube(3, seed=pc + pf, ny=2, nz=2)
    opc = pa.Operator(m.nx, m.ny, m.nz, m.affine, pc, 1.0, 1.0)
    opf = pa.Operator(m.nx, m.ny, m.nz, m.affine, pf, 1.0, 1.0)
    rng = np.random.default_rng(pc * 7 + pf)
    u = rng.normal(size=opc.ndofs)
    v = rng.normal(size=opf.ndofs)
    xf = torch.empty(opf.ndofs, dtype=torch.float64, device="cuda")
    rc = torch.empty(opc.ndofs, dtype=torch.float64, device="cuda")
    pa.pa_op_prolong(opc.h, opf.h, torch.tensor(u, device="cuda"), xf)
    pa.pa_op_restrict(opc.h, opf.h, torch.tensor(v, device="cuda"), rc)
    Pu = oracle.prolong(pc, pf, m.nx, m.ny, m.nz, u)
    Rv = oracle.restrict(pc, pf, m.nx, m.ny, m.nz, v)
    assert _relerr(xf.cpu().numpy(), Pu) <= 1e-13
    assert _relerr(rc.cpu().numpy(), Rv) <= 1e-13
    opc.close()
    opf.close()


@pytest.mark.parametrize("nx,ny,nz", [(1, 1, 1), (3, 2, 1), (8, 2, 2)])
def test_h_transfers_against_oracle(pa, nx, ny, nz):
    """p = 1 prolongation to the uniformly refined mesh and its transpose
    (the h-level transfers) against the oracle's evaluation of the coarse
    trilinear field at the fine nodes."""
    mc = syn.box_mesh(nx, ny, nz, hi=(2.0, 1.0, 1.5))
    mf = syn.box_mesh(2 * nx, 2 * ny, 2 * nz, hi=(2.0, 1.0, 1.5))
    opc = pa.Operator(mc.nx, mc.ny, mc.nz, mc.affine, 1, 1.0, 1.0)
    opf = pa.Operator(mf.nx, mf.ny, mf.nz, mf.affine, 1, 1.0, 1.0)
    rng = np.random.default_rng(nx + 5 * ny + 25 * nz)
    u = rng.normal(size=opc.ndofs)
    v = rng.normal(size=opf.ndofs)
    xf = torch.empty(opf.ndofs, dtype=torch.float64, device="cuda")
    rc = torch.empty(opc.ndofs, dtype=torch.float64, device="cuda")
    pa.pa_op_prolong(opc.h, opf.h, torch.tensor(u, device="cuda"), xf)
    pa.pa_op_restrict(opc.h, opf.h, torch.tensor(v, device="cuda"), rc)
    assert _relerr(xf.cpu().numpy(), oracle.prolong_h(nx, ny, nz, u)) <= 1e-15
    assert _relerr(rc.cpu().numpy(), oracle.restrict_h(nx, ny, nz, v)) <= 1e-14
    opc.close()
    opf.close()


def test_h_coarse_operator_is_galerkin_product_on_gpu(pa):
    """The p = 1 operator on the coarse mesh equals R A_fine P (nested
    spaces, exact quadrature, material constant per coarse element), all
    three factors applied by the library: a property that holds at any
    size, checked here on a sheared domain with two materials."""
    M = np.array([[1.3, 0.2, -0.1], [0.1, 0.9, 0.3], [-0.2, 0.15, 1.1]])
    mc = syn.globally_affine_mesh(6, 4, 2, M, t=(0.3, -0.2, 0.5))
    mf = syn.globally_affine_mesh(12, 8, 4, M, t=(0.3, -0.2, 0.5))
    rng = np.random.default_rng(4)
    mat_c = rng.uniform(0.5, 3.0, size=(mc.ne, 2))
    ef = np.arange(mf.ne)
    ex, ey, ez = ef % 12, (ef // 12) % 8, ef // 96
    mat_f = mat_c[ex // 2 + 6 * (ey // 2 + 4 * (ez // 2))]
    opc = pa.Operator(mc.nx, mc.ny, mc.nz, mc.affine, 1, 1.0, 1.0, mat=mat_c)
    opf = pa.Operator(mf.nx, mf.ny, mf.nz, mf.affine, 1, 1.0, 1.0, mat=mat_f)
    x = torch.tensor(rng.uniform(-1, 1, size=opc.ndofs), device="cuda")
    y = opc.apply(x)
    xf = torch.empty(opf.ndofs, dtype=torch.float64, device="cuda")
    pa.pa_op_prolong(opc.h, opf.h, x, xf)
    yf = opf.apply(xf)
    g = torch.empty_like(y)
    pa.pa_op_restrict(opc.h, opf.h, yf, g)
    assert _relerr(g.cpu().numpy(), y.cpu().numpy()) <= 1e-12
    opc.close()
    opf.close()


def test_assembled_p1_stencil_against_oracle_matrix(pa):
    """The assembled coarse matrix (27-point stencil) against the oracle's
    assembled global matrix, entry by entry."""
    m = syn.random_affine_cube(3, seed=77, ny=2, nz=2)
    lam, mu = syn.lame(1.0, 0.35)
    op = pa.Operator(m.nx, m.ny, m.nz, m.affine, 1, lam, mu)
    N = op.ndofs
    vals = torch.zeros(81 * N, dtype=torch.float64, device="cuda")
    pa.pa_op_assemble_p1(op.h, vals)
    V = vals.cpu().numpy().reshape(81, N)
    A = oracle.assemble_dense(1, m.nx, m.ny, m.nz, m.affine, lam, mu)
    Nn = N // 3
    Mx, My, Mz = m.nx + 1, m.ny + 1, m.nz + 1
    S = np.zeros_like(A)
    for row in range(N):
        c, i = divmod(row, Nn)
        ix, iy, iz = i % Mx, (i // Mx) % My, i // (Mx * My)
        for k in range(81):
            s, d = divmod(k, 3)
            dx, dy, dz = s % 3 - 1, (s // 3) % 3 - 1, s // 9 - 1
            jx, jy, jz = ix + dx, iy + dy, iz + dz
            if 0 <= jx < Mx and 0 <= jy < My and 0 <= jz < Mz:
                S[row, d * Nn + jx + Mx * (jy + My * jz)] = V[k, row]
            else:
                assert V[k, row] == 0.0
    assert np.max(np.abs(S - A)) <= 1e-13 * np.max(np.abs(A))
    op.close()


def test_batched_apply_matches_individual_applies(pa):
    """One batched launch over operators of uneven sizes, degrees and
    precisions (more than 24 in one group) equals the one-by-one applies,
    and every member matches the oracle's apply at the operator tolerance."""
    rng = np.random.default_rng(31)
    ops, xs, refs, probs = [], [], [], []
    specs = [(int(rng.choice([2, 4, 8])), int(rng.integers(0, 2)), tuple(int(v) for v in rng.integers(1, 4, 3)))
             for _ in range(12)]
    specs += [(2, 0, (2, 1, 1))] * 26  # one group larger than a launch
    for k, (p, prec, dims) in enumerate(specs):
        m = syn.random_affine_cube(dims[0], seed=900 + k, ny=dims[1], nz=dims[2])
        ess = syn.clamp_mask(m, p) if k % 3 == 0 else None
        op = pa.Operator(*dims, m.affine, p, 1.0, 0.7, precision=prec, ess_mask=ess)
        x = torch.tensor(syn.uniform_vector(op.ndofs, seed=k), dtype=op.dtype, device="cuda")
        ops.append(op)
        xs.append(x)
        refs.append(op.apply(x).clone())
        probs.append((p, prec, m, ess))
    ys = [torch.full_like(x, float("nan")) for x in xs]
    pa.pa_op_apply_batch([o.h for o in ops], xs, ys)
    torch.cuda.synchronize()
    for y, r in zip(ys, refs):
        assert torch.equal(y, r)
    for y, x, (p, prec, m, ess) in zip(ys, xs, probs):
        yo = oracle.apply(p, m.nx, m.ny, m.nz, m.affine, 1.0, 0.7, x.double().cpu().numpy(), ess=ess)
        assert _relerr(y.double().cpu().numpy(), yo) <= TOL[prec], (p, prec, m.nx, m.ny, m.nz)
    with pytest.raises(pa.PAError):
        pa.pa_op_apply_batch([ops[0].h, ops[0].h], [xs[0], xs[0]], [ys[0], ys[1]])
    for o in ops:
        o.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_per_element_material_apply_and_diag(pa, p, prec):
    """Per-element material (the PA data D with lambda(alpha, e), mu(alpha, e)
    constant per element) against the oracle's apply and diagonal; None
    restores the constant material."""
    nx, ny, nz = 3, 2, 2
    m = syn.random_affine_cube(nx, seed=600 + p, ny=ny, nz=nz)
    rng = np.random.default_rng(p)
    mat = rng.uniform(0.5, 50.0, (m.ne, 2))
    ess = syn.clamp_mask(m, p)
    x = syn.uniform_vector(m.n_dofs(p), seed=61 + p)
    op = pa.Operator(nx, ny, nz, m.affine, p, 1.0, 0.7, precision=prec, ess_mask=ess, mat=mat)
    xt = torch.tensor(x, dtype=op.dtype, device="cuda")
    yo = oracle.apply(p, nx, ny, nz, m.affine, 0.0, 0.0, x, ess=ess, mat=mat)
    assert _relerr(op.apply(xt).double().cpu().numpy(), yo) <= TOL[prec]
    do = oracle.diag(p, nx, ny, nz, m.affine, 0.0, 0.0, ess=ess, mat=mat)
    assert _relerr(op.diag().double().cpu().numpy(), do) <= TOL[prec]
    pa.pa_op_set_material(op.h, None)
    yc = oracle.apply(p, nx, ny, nz, m.affine, 1.0, 0.7, x, ess=ess)
    assert _relerr(op.apply(xt).double().cpu().numpy(), yc) <= TOL[prec]
    op.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p,face", [(1, 1), (2, 0), (3, 3), (4, 5), (8, 1)])
def test_traction_load_against_oracle(pa, p, face, prec):
    """Body force plus a constant traction on one face (clamped at x = 0):
    the load vector against the oracle's volume and surface integrals."""
    m = syn.random_affine_cube(2, seed=700 + p, ny=2, nz=1)
    ess = syn.clamp_mask(m, p)
    t = (0.1, -0.3, -1e-2)
    op = pa.Operator(m.nx, m.ny, m.nz, m.affine, p, 1.0, 1.0, precision=prec, ess_mask=ess)
    F = op.rhs(f0=(0.0, 0.0, -1.0), traction=(face, t)).double().cpu().numpy()
    Fo = oracle.load(p, m.nx, m.ny, m.nz, m.affine, f0=(0.0, 0.0, -1.0), ess=ess) + \
        oracle.traction(p, m.nx, m.ny, m.nz, m.affine, face, t, ess=ess)
    assert _relerr(F, Fo) <= TOL[prec]
    op.close()


@pytest.mark.parametrize("stage", [0, 1, 2, 3])
@pytest.mark.parametrize("p", [1, 2, 4])
def test_optimisation_stack_stages_against_oracle(pa, p, stage):
    """Every stage of the Table 8 ladder on the GPU (baseline with dense
    contractions, full 81-term stress and the Q values through HBM; + sum
    factorisation; + Voigt; + fusion) is the same operator: FP64 parity with
    the oracle, constrained, on uneven elements with per-element material."""
    nx, ny, nz = MESH_DIMS[p]
    m = syn.random_affine_cube(nx, seed=800 + p, ny=ny, nz=nz)
    mat = np.random.default_rng(p).uniform(0.5, 5.0, (m.ne, 2))
    ess = syn.clamp_mask(m, p)
    x = syn.uniform_vector(m.n_dofs(p), seed=81 + p)
    yo = oracle.apply(p, nx, ny, nz, m.affine, 0.0, 0.0, x, ess=ess, mat=mat)
    op = pa.Operator(nx, ny, nz, m.affine, p, 1.0, 1.0, ess_mask=ess, mat=mat)
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    y = torch.full_like(xt, float("nan"))
    pa.pa_op_apply_stage(op.h, stage, xt, y)
    assert _relerr(y.cpu().numpy(), yo) <= TOL[0]
    op.close()


def test_optimisation_stack_rejects_fp32_and_bad_stage(pa):
    m = syn.random_affine_cube(2, seed=5)
    op = pa.Operator(2, 2, 2, m.affine, 2, 1.0, 1.0, precision=pa.PA_FP32)
    x = torch.zeros(op.ndofs, dtype=torch.float32, device="cuda")
    y = torch.zeros_like(x)
    pa.pa_op_apply_stage(op.h, 3, x, y)  # the production apply: any precision
    for stage in (0, 4, -1):
        with pytest.raises(pa.PAError) as ei:
            pa.pa_op_apply_stage(op.h, stage, x, y)
        assert ei.value.code == pa.PA_EINVAL
    op.close()


def _spd_voigt_stack(ne, seed):
    rng = np.random.default_rng(seed)
    out = np.empty((ne, 6, 6))
    for e in range(ne):
        L = rng.uniform(-1, 1, (6, 6))
        out[e] = L @ L.T + 2.0 * np.eye(6)
    return out


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 4, 7])
def test_anisotropic_apply_and_diag(pa, p, prec):
    """A general symmetric 6x6 Voigt matrix per element (Eq. 2) against the
    oracle's full-tensor apply and diagonal, constrained; None restores the
    isotropic material."""
    nx, ny, nz = MESH_DIMS[p]
    m = syn.random_affine_cube(nx, seed=900 + p, ny=ny, nz=nz)
    Cv = _spd_voigt_stack(m.ne, p)
    ct = np.stack([oracle.voigt_to_tensor(c) for c in Cv])
    ess = syn.clamp_mask(m, p)
    x = syn.uniform_vector(m.n_dofs(p), seed=91 + p)
    op = pa.Operator(nx, ny, nz, m.affine, p, 1.0, 0.7, precision=prec, ess_mask=ess, cvoigt=Cv)
    xt = torch.tensor(x, dtype=op.dtype, device="cuda")
    yo = oracle.apply(p, nx, ny, nz, m.affine, 0.0, 0.0, x, ess=ess, ctens=ct)
    assert _relerr(op.apply(xt).double().cpu().numpy(), yo) <= TOL[prec]
    do = oracle.diag(p, nx, ny, nz, m.affine, 0.0, 0.0, ess=ess, ctens=ct)
    assert _relerr(op.diag().double().cpu().numpy(), do) <= TOL[prec]
    pa.pa_op_set_anisotropic(op.h, None)
    yc = oracle.apply(p, nx, ny, nz, m.affine, 1.0, 0.7, x, ess=ess)
    assert _relerr(op.apply(xt).double().cpu().numpy(), yc) <= TOL[prec]
    bad = Cv.copy()
    bad[0, 0, 1] += 1.0
    with pytest.raises(pa.PAError):
        pa.pa_op_set_anisotropic(op.h, bad)
    op.close()


@pytest.mark.parametrize("p", range(1, 7))
def test_tensor_core_variant_against_oracle(pa, p):
    """Variant 4 (FP32): the six 1D contractions on the tensor cores
    (tcgen05.mma kind::tf32, three TF32 products per contraction), against
    the oracle at the FP32 tolerance, constrained, on a mesh whose element
    count leaves a ragged last batch; no tensor-core wait timed out."""
    nx, ny, nz = {1: (5, 4, 3), 2: (5, 3, 2), 3: (3, 3, 2), 4: (5, 2, 1), 5: (3, 1, 1), 6: (3, 1, 1)}[p]
    m = syn.random_affine_cube(nx, seed=950 + p, ny=ny, nz=nz)
    ess = syn.clamp_mask(m, p)
    x = syn.uniform_vector(m.n_dofs(p), seed=95 + p)
    yo = oracle.apply(p, nx, ny, nz, m.affine, 1.0, 0.7, x, ess=ess)
    op = pa.Operator(nx, ny, nz, m.affine, p, 1.0, 0.7, precision=pa.PA_FP32, ess_mask=ess)
    E = 128 // (p + 2) ** 2
    assert op.nelem % E != 0
    pa.pa_op_set_launch(op.h, 4, E, 384)
    with pytest.raises(pa.PAError):
        pa.pa_op_set_launch(op.h, 4, E + 1, 384)  # the one admissible shape
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    y = op.apply(xt)
    torch.cuda.synchronize()
    pa.pa_op_check(op.h)
    assert _relerr(y.double().cpu().numpy(), yo) <= TOL[1]
    op.close()


def test_tensor_core_variant_is_fp32_and_low_degree_only(pa):
    m = syn.random_affine_cube(2, seed=3)
    op64 = pa.Operator(2, 2, 2, m.affine, 2, 1.0, 1.0)
    with pytest.raises(pa.PAError):
        pa.pa_op_set_launch(op64.h, 4, 8, 384)
    op64.close()
    op = pa.Operator(2, 1, 1, m.affine[:2], 7, 1.0, 1.0, precision=pa.PA_FP32)
    with pytest.raises(pa.PAError):
        pa.pa_op_set_launch(op.h, 4, 1, 384)
    op.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", [1, 3, 8])
def test_degenerate_inputs(pa, p, prec):
    """Degenerate cases of the method: zero input gives exactly zero; every
    dof essential gives the identity; rigid translations (any geometry) and,
    on a globally affine mesh, rigid rotations lie in the kernel of the
    unconstrained operator to rounding of the operator's scale."""
    dt = torch.float64 if prec == 0 else torch.float32
    m = syn.random_affine_cube(3, seed=90 + p, ny=2, nz=2)
    op = pa.Operator(m.nx, m.ny, m.nz, m.affine, p, 1.0, 0.7, precision=prec)
    N = op.ndofs
    z = torch.zeros(N, dtype=dt, device="cuda")
    assert torch.count_nonzero(op.apply(z)) == 0
    xr = torch.tensor(syn.uniform_vector(N, seed=5), dtype=dt, device="cuda")
    scale = float(op.apply(xr).abs().max())
    Nn = N // 3
    for c in range(3):
        t = torch.zeros(N, dtype=dt, device="cuda")
        t[c * Nn:(c + 1) * Nn] = 1.0
        assert float(op.apply(t).abs().max()) <= TOL[prec] * scale
    op.close()
    allm = np.ones(N, dtype=np.uint8)
    opc = pa.Operator(m.nx, m.ny, m.nz, m.affine, p, 1.0, 0.7, precision=prec, ess_mask=allm)
    assert torch.equal(opc.apply(xr), xr)
    opc.close()
    M = np.array([[1.3, 0.2, -0.1], [0.1, 0.9, 0.3], [-0.2, 0.15, 1.1]])
    mg = syn.globally_affine_mesh(3, 2, 2, M, t=(0.3, -0.2, 0.5))
    opg = pa.Operator(mg.nx, mg.ny, mg.nz, mg.affine, p, 1.0, 0.7, precision=prec)
    X = oracle.node_coords_box(3, 2, 2, p) @ M.T + np.array([0.3, -0.2, 0.5])
    sg = float(opg.apply(torch.tensor(syn.uniform_vector(N, seed=6), dtype=dt, device="cuda")).abs().max())
    for w in np.eye(3):
        u = np.cross(w, X)  # rotation field w x X
        y = opg.apply(torch.tensor(u.T.reshape(-1), dtype=dt, device="cuda"))
        assert float(y.abs().max()) <= 10 * TOL[prec] * sg * np.abs(X).max()
    opg.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 5])
def test_apply_add_accumulates(pa, p, prec):
    """pa_op_apply_add: y0 + A x against the oracle (constrained rows add x)."""
    dt = torch.float64 if prec == 0 else torch.float32
    m = syn.random_affine_cube(3, seed=70 + p, ny=2, nz=2)
    lam, mu = syn.lame(1.0, 0.3)
    ess = syn.clamp_mask(m, p)
    op = pa.Operator(m.nx, m.ny, m.nz, m.affine, p, lam, mu, precision=prec, ess_mask=ess)
    x = syn.uniform_vector(op.ndofs, seed=1)
    y0 = syn.uniform_vector(op.ndofs, seed=2)
    y = torch.tensor(y0, dtype=dt, device="cuda")
    pa.pa_op_apply_add(op.h, torch.tensor(x, dtype=dt, device="cuda"), y)
    yo = y0 + oracle.apply(p, m.nx, m.ny, m.nz, m.affine, lam, mu, x, ess=ess)
    assert _relerr(y.cpu().double().numpy(), yo) <= TOL[prec]
    with pytest.raises(pa.PAError):
        pa.pa_op_apply_add(op.h, y, y)
    op.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_apply_largest_served_size_sampled(pa, prec):
    """The largest request of the served stream (32^3 elements at p = 8,
    50.9M dofs), clamped at x = 0: sampled rows (both faces, edges, the
    interior) against the oracle's element-matrix rows."""
    n, p = 32, 8
    m = syn.box_mesh(n, n, n)
    lam, mu = syn.lame(3.0, 0.4)
    ess = syn.clamp_mask(m, p)
    N = m.n_dofs(p)
    assert N == 3 * 257 ** 3
    x = syn.uniform_vector(N, seed=11)
    y = _run_apply(pa, m, p, lam, mu, x, prec, ess)
    rng = np.random.default_rng(12)
    rows = np.concatenate([rng.choice(N, 2000, replace=False), [0, 1, 256, 257, N // 3, N - 1]])
    yo = oracle.apply_rows(p, n, n, n, m.affine, lam, mu, x, rows, ess=ess)
    assert np.max(np.abs(y[rows] - yo)) <= TOL[prec] * np.max(np.abs(yo))


def test_multi_operator_launch_any_degrees(pa):
    """The persistent multi-operator launch: operators of every degree
    1..8, both precisions, uneven sizes (one element to a few hundred),
    constrained or not, FP32 ones in the unsplit and split forms, plus
    operators it does not hold (FP32 flat and tensor-core shapes, FP64 line
    shapes) that take the per-degree path -- all in one batched call; every
    result within the operator tolerance of the oracle and bitwise the
    operator's own apply (except tensor-core shapes, which a batch runs as
    the register-tiled line variant)."""
    rng = np.random.default_rng(57)
    ops, xs, refs, probs = [], [], [], []
    k = 0
    for p in range(1, 9):
        for prec in (0, 1):
            for launch in (None, "alt"):
                dims = tuple(int(v) for v in rng.integers(1, 5, 3)) if (p + prec) % 3 else (1, 1, 1)
                m = syn.random_affine_cube(dims[0], seed=1900 + k, ny=dims[1], nz=dims[2])
                ess = syn.clamp_mask(m, p) if k % 2 else None
                op = pa.Operator(*dims, m.affine, p, 1.3, 0.6, precision=prec, ess_mask=ess)
                if launch == "alt":
                    if prec == 1:
                        v = [6, 3, 0, 4][k % 4]
                        if v == 4 and p > 6:
                            v = 3
                        shape = (v, 128 // (p + 2) ** 2, 384) if v == 4 else (v, 2, 128)
                    else:
                        shape = (2, 1, 128) if p <= 4 else (0, 1, 128)
                    pa.pa_op_set_launch(op.h, *shape)
                x = torch.tensor(syn.uniform_vector(op.ndofs, seed=k), dtype=op.dtype, device="cuda")
                ops.append(op)
                xs.append(x)
                refs.append(op.apply(x).clone())
                probs.append((p, prec, m, ess))
                k += 1
    order = rng.permutation(len(ops))
    ys = [torch.full_like(x, float("nan")) for x in xs]
    pa.pa_op_apply_batch([ops[i].h for i in order], [xs[i] for i in order], [ys[i] for i in order])
    torch.cuda.synchronize()
    for i in range(len(ops)):
        if pa.pa_op_get_launch(ops[i].h)[0] != 4:  # a batch runs tensor-core shapes as the line variant
            assert torch.equal(ys[i], refs[i]), (i, probs[i][:2], pa.pa_op_get_launch(ops[i].h))
        p, prec, m, ess = probs[i]
        yo = oracle.apply(p, m.nx, m.ny, m.nz, m.affine, 1.3, 0.6, xs[i].double().cpu().numpy(), ess=ess)
        assert _relerr(ys[i].double().cpu().numpy(), yo) <= TOL[prec], (i, p, prec)
    for o in ops:
        o.close()
