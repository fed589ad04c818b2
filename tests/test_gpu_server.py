"""The solve server: continuous admission by memory footprint, overlapping
requests, and each result identical alone and in a mix."""
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


def _req(pa, k, keep=True, mode=1, p=None):
    rng = np.random.default_rng(k)
    p = int(rng.choice([2, 4])) if p is None else p
    n = int(rng.integers(2, 5))
    beam = bool(k % 2)
    dims = (4 * n, n, n) if beam else (n, n, n)
    box = (0, 0, 0, 8.0 if beam else 1.0, 1.0, 1.0)
    E = float(np.exp(rng.uniform(np.log(0.1), np.log(10.0))))
    nu = float(rng.uniform(0.2, 0.45))
    modes = syn.smooth_force_modes(seed=100 + k)
    return pa.make_request(*dims, box, p, E, nu, modes=modes, rtol=1e-10, maxit=400, mode=mode, keep_solution=keep)


def _ndofs(r):
    return 3 * (r.nx * r.p + 1) * (r.ny * r.p + 1) * (r.nz * r.p + 1)


def test_result_is_identical_alone_and_in_a_mix(pa):
    target = _req(pa, 7)
    srv = pa.pa_server_create(64 << 30, 1)
    t = pa.pa_server_submit(srv, target)
    code, info, tm, x_alone = pa.pa_server_wait(srv, t, _ndofs(target))
    pa.pa_server_destroy(srv)
    assert code == pa.PA_OK and info.rel_residual <= 1e-8
    srv = pa.pa_server_create(64 << 30, 4)
    tickets = [pa.pa_server_submit(srv, _req(pa, k, keep=False)) for k in range(3)]
    tt = pa.pa_server_submit(srv, _req(pa, 7))
    tickets += [pa.pa_server_submit(srv, _req(pa, k, keep=False)) for k in range(10, 14)]
    code, info2, tm2, x_mix = pa.pa_server_wait(srv, tt, _ndofs(target))
    others = [pa.pa_server_wait(srv, t)[0] for t in tickets]
    st = pa.pa_server_stats(srv)
    pa.pa_server_destroy(srv)
    assert code == pa.PA_OK and all(c == pa.PA_OK for c in others)
    assert np.array_equal(x_alone, x_mix)  # deterministic: the same bits
    assert info2.iterations == info.iterations
    assert st.completed == 8 and st.peak_used_bytes > 0


def test_batch_lane_gives_the_solo_lane_bits(pa):
    """Flexible-CG requests of one hierarchy solved in the lockstep batch
    lane (continuous batching, batched applies) give bitwise the results of
    the same requests solved one per worker with the lane off."""
    reqs = [_req(pa, 40 + k, mode=pa.PA_SOLVE_MIXED_FCG, p=4) for k in range(8)]
    reqs[3].mode = pa.PA_SOLVE_FP64  # another hierarchy key: its own batch

    def serve(batch):
        srv = pa.pa_server_create(64 << 30, 8)
        pa.pa_server_set_option(srv, pa.PA_SERVER_OPT_BATCH, batch)
        ts = [pa.pa_server_submit(srv, r) for r in reqs]
        out = [pa.pa_server_wait(srv, t, _ndofs(r)) for t, r in zip(ts, reqs)]
        st = pa.pa_server_stats(srv)
        pa.pa_server_destroy(srv)
        return out, st

    solo, st0 = serve(0)
    lane, st1 = serve(1)
    assert st0.batched == 0 and st1.batched == 8
    assert st1.batch_max_members >= 2 and st1.batch_member_ticks > st1.batch_ticks
    for (c0, i0, t0, x0), (c1, i1, t1, x1) in zip(solo, lane):
        assert c0 == pa.PA_OK and c1 == pa.PA_OK
        assert t0.batched == 0 and t1.batched == 1
        assert i0.iterations == i1.iterations and i0.rel_residual == i1.rel_residual
        assert np.array_equal(x0, x1)
    with pytest.raises(pa.PAError):
        srv = pa.pa_server_create(1 << 30, 1)
        try:
            pa.pa_server_set_option(srv, pa.PA_SERVER_OPT_BATCH_MAX_MEMBERS, 0)
        finally:
            pa.pa_server_destroy(srv)


def test_admission_respects_the_memory_budget(pa):
    reqs = [_req(pa, k, keep=False) for k in range(6)]
    srv = pa.pa_server_create(64 << 30, 6)
    fps = []
    for r in reqs:
        code, info, tm, _ = pa.pa_server_wait(srv, pa.pa_server_submit(srv, r))
        fps.append(tm.footprint_bytes)
    pa.pa_server_destroy(srv)
    budget = int(max(fps) * 1.5)  # room for one request at a time, sometimes two
    srv = pa.pa_server_create(budget, 6)
    ts = [pa.pa_server_submit(srv, r) for r in reqs]
    res = [pa.pa_server_wait(srv, t) for t in ts]
    st = pa.pa_server_stats(srv)
    pa.pa_server_destroy(srv)
    assert all(r[0] == pa.PA_OK for r in res)
    assert st.peak_used_bytes <= budget
    # a request larger than the whole budget is refused, not run
    srv = pa.pa_server_create(1 << 20, 2)
    code = pa.pa_server_wait(srv, pa.pa_server_submit(srv, reqs[0]))[0]
    pa.pa_server_destroy(srv)
    assert code == pa.PA_EBUSY


def test_served_solution_matches_direct_solve(pa):
    E, nu = 2.0, 0.35
    r = pa.make_request(4, 1, 1, (0, 0, 0, 8.0, 1.0, 1.0), 2, E, nu, f0=(0, 0, -1.0), rtol=1e-10, maxit=300,
                        mode=pa.PA_SOLVE_MIXED, keep_solution=True)
    srv = pa.pa_server_create(8 << 30, 2)
    code, info, tm, x = pa.pa_server_wait(srv, pa.pa_server_submit(srv, r), _ndofs(r))
    pa.pa_server_destroy(srv)
    assert code == pa.PA_OK
    m = syn.box_mesh(4, 1, 1, hi=(8.0, 1.0, 1.0))
    lam, mu = syn.lame(E, nu)
    ess = syn.clamp_mask(m, 2)
    b = oracle.load(2, 4, 1, 1, m.affine, f0=(0, 0, -1.0), ess=ess)
    xo = oracle.solve_dense(2, 4, 1, 1, m.affine, lam, mu, b, ess)
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
    assert tm.latency_s >= tm.solve_s > 0


def test_served_h_levels_match_direct_solve_and_the_p_only_hierarchy(pa):
    """A 16x2x2 beam request gets one h-level by default (its p = 1 level
    has 459 dofs); the served solution matches a direct solve, and so does
    the same request served with h-levels off."""
    E, nu = 1.0, 0.3
    m = syn.box_mesh(16, 2, 2, hi=(8.0, 1.0, 1.0))
    lam, mu = syn.lame(E, nu)
    ess = syn.clamp_mask(m, 2)
    b = oracle.load(2, 16, 2, 2, m.affine, f0=(0, 0, -1.0), ess=ess)
    xo = oracle.solve_dense(2, 16, 2, 2, m.affine, lam, mu, b, ess)
    for h_on in (1, 0):
        r = pa.make_request(16, 2, 2, (0, 0, 0, 8.0, 1.0, 1.0), 2, E, nu, f0=(0, 0, -1.0), rtol=1e-10, maxit=300,
                            mode=pa.PA_SOLVE_MIXED_FCG, keep_solution=True)
        srv = pa.pa_server_create(8 << 30, 2)
        pa.pa_server_set_option(srv, pa.PA_SERVER_OPT_H_LEVELS, h_on)
        code, info, tm, x = pa.pa_server_wait(srv, pa.pa_server_submit(srv, r), _ndofs(r))
        pa.pa_server_destroy(srv)
        assert code == pa.PA_OK, pa.lib.pa_last_error()
        assert (tm.h_levels, tm.levels) == ((1, 3) if h_on else (0, 2))
        assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
