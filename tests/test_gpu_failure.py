"""Failure detection on the GPU without a GPU fault: bounded device waits
that run out (a wait budget shorter than the work it waits for) return
PA_ETIMEOUT and leave the solver or operator usable; a breakdown reached from
host input (an indefinite material) returns PA_EBREAKDOWN; an inner-solve
failure injected on the host ends iterative refinement cleanly; the server
cancels queued and running requests and keeps serving."""
import time

import numpy as np
import pytest

import oracle
import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pa():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08374_gb300 as pa
    return pa


def _beam_op(pa, nx, ny, nz, p, mat=None):
    m = syn.box_mesh(nx, ny, nz, hi=(8.0, 1.0, 1.0))
    lam, mu = syn.lame(1.0, 0.3)
    ess = syn.clamp_mask(m, p)
    op = pa.Operator(nx, ny, nz, m.affine, p, lam, mu, ess_mask=ess, mat=mat)
    return m, lam, mu, ess, op


@pytest.mark.parametrize("graphs", [1, 0])
def test_coarse_grid_barrier_wait_runs_out(pa, graphs):
    """The persistent coarse CG (h-multigrid off) with a wait budget of a
    nanosecond: its CTAs reach a grid barrier before the others, the wait
    runs out, the kernel returns and the solve reports PA_ETIMEOUT.  With the
    default budget restored the same solver converges."""
    m, lam, mu, ess, op = _beam_op(pa, 32, 2, 2, 4)
    b = op.rhs(f0=(0.0, 0.0, -1.0))
    s = pa.pa_solver_create(op.h, [4, 2, 1], 2, 1e-4, 300, pa.PA_SOLVE_FP64)
    pa.pa_solver_set_option(s, pa.PA_SOLVER_OPT_COARSE_HMG, 0)
    pa.pa_solver_set_option(s, pa.PA_SOLVER_OPT_PERSISTENT_COARSE, 1)
    pa.pa_solver_set_option(s, pa.PA_SOLVER_OPT_GRAPHS, graphs)
    pa.pa_solver_set_option(s, pa.PA_SOLVER_OPT_WAIT_LIMIT, 1e-9)
    x = torch.zeros_like(b)
    t0 = time.perf_counter()
    with pytest.raises(pa.PAError) as ei:
        pa.pa_gmg_pcg_solve(s, b, x, 1e-10, 200)
    assert ei.value.code == pa.PA_ETIMEOUT and "barrier" in str(ei.value)
    assert time.perf_counter() - t0 < 30.0
    pa.pa_solver_set_option(s, pa.PA_SOLVER_OPT_WAIT_LIMIT, 2.0)
    code, info = pa.pa_gmg_pcg_solve(s, b, x.zero_(), 1e-10, 200)
    assert code == pa.PA_OK and info.rel_residual <= 2e-9
    with pytest.raises(pa.PAError):
        pa.pa_solver_set_option(s, pa.PA_SOLVER_OPT_WAIT_LIMIT, 0.0)
    pa.pa_solver_destroy(s)
    op.close()


def test_tensor_core_wait_runs_out(pa):
    """The tensor-core variant with a wait budget of a nanosecond: the MMAs
    in flight are drained, the apply is marked invalid and pa_op_check
    reports PA_ETIMEOUT once; with the default budget the apply matches the
    oracle again."""
    p = 2
    m = syn.random_affine_cube(3, seed=71)
    lam, mu = syn.lame(1.0, 0.3)
    op = pa.Operator(3, 3, 3, m.affine, p, lam, mu, precision=pa.PA_FP32)
    E = 128 // (p + 2) ** 2
    pa.pa_op_set_launch(op.h, 4, E, 384)
    x = torch.tensor(syn.uniform_vector(op.ndofs, seed=72), dtype=torch.float32, device="cuda")
    pa.pa_op_check(op.h)  # clear
    pa.pa_op_set_wait_limit(op.h, 1e-9)
    op.apply(x)
    torch.cuda.synchronize()
    with pytest.raises(pa.PAError) as ei:
        pa.pa_op_check(op.h)
    assert ei.value.code == pa.PA_ETIMEOUT
    pa.pa_op_check(op.h)  # reported once, then clear
    pa.pa_op_set_wait_limit(op.h, 2.0)
    y = op.apply(x).double().cpu().numpy()
    pa.pa_op_check(op.h)
    yo = oracle.apply(p, 3, 3, 3, m.affine, lam, mu, x.double().cpu().numpy())
    assert np.max(np.abs(y - yo)) <= 1e-5 * np.max(np.abs(yo))
    with pytest.raises(pa.PAError):
        pa.pa_op_set_wait_limit(op.h, -1.0)
    op.close()


def test_indefinite_material_breaks_down(pa):
    """PA_EBREAKDOWN from host input.  At creation: a material with mu < 0
    everywhere makes the assembled coarsest matrix indefinite and its
    Cholesky factorisation fails.  At solve time: the fine operator's
    material turned negative after the solver was built makes p^T A p < 0 in
    the first CG step; the solve returns PA_EBREAKDOWN with its info, and
    with the material restored the same solver converges."""
    ne = 8 * 2 * 2
    neg = np.tile([0.0, -1.0], (ne, 1))
    m, lam, mu, ess, op = _beam_op(pa, 8, 2, 2, 2, mat=neg)
    with pytest.raises(pa.PAError) as ei:
        pa.pa_solver_create(op.h, [2, 1])
    assert ei.value.code == pa.PA_EBREAKDOWN
    pa.pa_op_set_material(op.h, None)
    b = op.rhs(f0=(0.0, 0.0, -1.0))
    s = pa.pa_solver_create(op.h, [2, 1])
    pa.pa_op_set_material(op.h, neg)
    x = torch.zeros_like(b)
    code, info = pa.pa_gmg_pcg_solve(s, b, x, 1e-10, 200)
    assert code == pa.PA_EBREAKDOWN and info.status == pa.PA_EBREAKDOWN
    assert "breakdown" in pa.lib.pa_last_error().decode()
    pa.pa_op_set_material(op.h, None)
    code, info = pa.pa_gmg_pcg_solve(s, b, x.zero_(), 1e-10, 200)
    assert code == pa.PA_OK and info.tolerance_met == 1
    pa.pa_solver_destroy(s)
    op.close()


def test_injected_inner_failure_ends_refinement(pa):
    """A breakdown injected on the host into the second inner solve of
    iterative refinement: the solve returns PA_EBREAKDOWN after one
    refinement, with x the once-refined iterate (its true residual already
    reduced); the hook fires once, and the next solve converges."""
    m, lam, mu, ess, op = _beam_op(pa, 8, 2, 2, 4)
    b = op.rhs(f0=(0.0, 0.0, -1.0))
    s = pa.pa_solver_create(op.h, [4, 2, 1], 2, 1e-4, 300, pa.PA_SOLVE_MIXED)
    pa.pa_solver_set_option(s, pa.PA_SOLVER_OPT_INJECT_INNER_FAILURE, 2)
    x = torch.zeros_like(b)
    code, info = pa.pa_gmg_pcg_solve(s, b, x, 1e-10, 500)
    assert code == pa.PA_EBREAKDOWN and info.status == pa.PA_EBREAKDOWN
    assert info.refinements == 1 and "injected" in pa.lib.pa_last_error().decode()
    assert 0.0 < info.rel_residual < 0.5  # below the initial 1: one refinement was applied
    code, info = pa.pa_gmg_pcg_solve(s, b, x.zero_(), 1e-10, 500)
    assert code == pa.PA_OK and info.refinements >= 2
    pa.pa_solver_destroy(s)
    op.close()


def test_server_cancels_queued_and_running_requests(pa):
    """One slot: a long FP64 solve (a tolerance whose square underflows to 0,
    so only maxit ends it) runs while a second request waits in the queue.
    Canceling the queued one completes it at once with PA_ECANCELED;
    canceling the running one ends its solve early with PA_ECANCELED and
    releases its memory; the server then serves a new request normally."""
    srv = pa.pa_server_create(8 << 30, 1)
    pa.pa_server_set_option(srv, pa.PA_SERVER_OPT_BATCH, 0)
    long_req = pa.make_request(12, 12, 12, (0, 0, 0, 1, 1, 1), 8, 1.0, 0.45, f0=(0, 0, -1.0), rtol=1e-200,
                               maxit=400, mode=pa.PA_SOLVE_FP64)
    small = pa.make_request(4, 1, 1, (0, 0, 0, 8, 1, 1), 2, 1.0, 0.3, f0=(0, 0, -1.0), rtol=1e-10, maxit=500,
                            mode=pa.PA_SOLVE_FP64)
    ta = pa.pa_server_submit(srv, long_req)
    tb = pa.pa_server_submit(srv, small)
    time.sleep(0.2)
    pa.pa_server_cancel(srv, tb)
    code_b, info_b, tm_b, _ = pa.pa_server_wait(srv, tb)
    assert code_b == pa.PA_ECANCELED and info_b.status == pa.PA_ECANCELED
    # let the long request get past its setup into the solve, then cancel it
    time.sleep(2.0)
    t0 = time.perf_counter()
    pa.pa_server_cancel(srv, ta)
    code_a, info_a, tm_a, _ = pa.pa_server_wait(srv, ta)
    assert code_a == pa.PA_ECANCELED
    assert time.perf_counter() - t0 < 5.0
    assert info_a.iterations < 400
    st = pa.pa_server_stats(srv)
    assert st.used_bytes == 0 and st.queued == 0
    with pytest.raises(pa.PAError):
        pa.pa_server_cancel(srv, 987654)
    tc = pa.pa_server_submit(srv, small)
    code_c, info_c, _, _ = pa.pa_server_wait(srv, tc)
    assert code_c == pa.PA_OK and info_c.tolerance_met == 1
    pa.pa_server_cancel(srv, pa.pa_server_submit(srv, small))  # a queued or running one, collected below
    pa.pa_server_destroy(srv)


def test_server_cancels_a_batch_lane_member(pa):
    """A small request in the lockstep batch lane that only its iteration
    cap would end (a tolerance whose square underflows): canceled while it
    steps, it leaves the batch before the
    next tick with PA_ECANCELED; a request solved beside it is unaffected."""
    srv = pa.pa_server_create(4 << 30, 2)
    endless = pa.make_request(4, 4, 4, (0, 0, 0, 1, 1, 1), 4, 1.0, 0.3, f0=(0, 0, -1.0), rtol=1e-200, maxit=5000,
                              mode=pa.PA_SOLVE_MIXED_FCG)
    normal = pa.make_request(3, 3, 3, (0, 0, 0, 1, 1, 1), 4, 2.0, 0.3, f0=(0, 0, -1.0), rtol=1e-10, maxit=500,
                             mode=pa.PA_SOLVE_MIXED_FCG, keep_solution=True)
    te = pa.pa_server_submit(srv, endless)
    tn = pa.pa_server_submit(srv, normal)
    code_n, info_n, tm_n, xn = pa.pa_server_wait(srv, tn, x_len=3 * 13 ** 3)
    assert code_n == pa.PA_OK and tm_n.batched == 1
    time.sleep(0.5)
    pa.pa_server_cancel(srv, te)
    code_e, info_e, tm_e, _ = pa.pa_server_wait(srv, te)
    assert code_e == pa.PA_ECANCELED and tm_e.batched == 1
    assert info_e.iterations < 5000
    pa.pa_server_destroy(srv)
