// Lockstep engine of the GMG-PCG solver: several flexible-CG solves advanced
// one CG step per tick with their operator applies batched, and the ABI
// entry point that drives it (pa_gmg_pcg_solve_batch).
#include <algorithm>
#include <atomic>
#include <string>
#include <vector>

#include "pa_solver_state.h"

namespace pa {
namespace {

// ------------------------------------------------------------ lockstep
// Several solvers advanced together, one flexible-CG step per tick.  Each
// solver's step is captured once per phase (the kernels between two
// operator applies) into small executable graphs on its own stream; a tick
// runs phase j of every member that has one (members of different
// hierarchies have different numbers of phases), then the applies that end
// those phases -- on any levels, of any degrees -- as one batched apply (the
// persistent multi-operator launch pair) on the lockstep's stream, then
// phase j + 1.  The coarse solve of
// each member is its own device-controlled loop between the two halves of
// the step.  Members join and leave between ticks.  The kernels, their
// order per member and the applies' arithmetic are those of the solver's
// own step, so a member's iterates are bitwise those of its solo solve.
struct ApplyRec {
    pa_op *op = nullptr;
    const void *x = nullptr;
    void *y = nullptr;
};

struct Segment {
    std::vector<cudaGraphExec_t> g;  // per phase (null: nothing to launch)
    std::vector<ApplyRec> ap;        // apply ending each phase but the last (op null: none)
};

struct LockMember {
    pa_solver *s = nullptr;
    double *x_out = nullptr;
    void *tag = nullptr;
    double bb = 0.0, tol2 = 0.0;
    int maxit = 0, it = 0;
    bool started = false;
    cudaEvent_t ev = nullptr;
    Segment a[2], b[2];  // [0] first step, [1] iteration step
    cudaGraphExec_t coarse = nullptr;
    pa_solve_info info{};
};

void free_segment(Segment &sg)
{
    for (cudaGraphExec_t g : sg.g)
        if (g) cudaGraphExecDestroy(g);
    sg.g.clear();
    sg.ap.clear();
}

void free_member(LockMember &m)
{
    for (int k = 0; k < 2; ++k) {
        free_segment(m.a[k]);
        free_segment(m.b[k]);
    }
    if (m.coarse) cudaGraphExecDestroy(m.coarse);
    if (m.ev) cudaEventDestroy(m.ev);
    m.coarse = nullptr;
    m.ev = nullptr;
}

// Captures every phase of a step segment of solver s into sg.
template <typename F>
int capture_segment(pa_solver *s, F fn, Segment &sg)
{
    cudaStream_t st = s->stream;
    s->ph_on = true;
    s->ph_target = -1;  // count the phases: nothing is emitted
    s->ph_counter = 0;
    int rc = fn();
    const int napply = s->ph_counter;
    for (int j = 0; !rc && j <= napply; ++j) {
        s->ph_target = j;
        s->ph_counter = 0;
        s->ph_op = nullptr;
        s->ph_x = nullptr;
        s->ph_y = nullptr;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) {
            rc = cuda_error(e, "lockstep: cudaStreamBeginCapture");
            break;
        }
        int r = fn();
        e = cudaStreamEndCapture(st, &g);
        if (!r && e != cudaSuccess) r = cuda_error(e, "lockstep: cudaStreamEndCapture");
        if (!r && s->ph_counter != napply) r = set_error(PA_EINVAL, "lockstep: step phases differ between captures");
        cudaGraphExec_t ex = nullptr;
        if (!r) {
            size_t nn = 0;
            e = cudaGraphGetNodes(g, nullptr, &nn);
            if (e != cudaSuccess) r = cuda_error(e, "lockstep: cudaGraphGetNodes");
            else if (nn > 0 && (e = cudaGraphInstantiate(&ex, g, 0)) != cudaSuccess)
                r = cuda_error(e, "lockstep: cudaGraphInstantiate");
        }
        if (g) cudaGraphDestroy(g);
        if (r) {
            rc = r;
            break;
        }
        sg.g.push_back(ex);
        if (j < napply) sg.ap.push_back(ApplyRec{s->ph_op, s->ph_x, s->ph_y});
    }
    s->ph_on = false;
    return rc;
}

template <typename TP>
int capture_member(LockMember &m)
{
    pa_solver *s = m.s;
    FcgVecs<double> v = outer_vecs(s);
    const cudaStream_t st = s->stream;
    int rc = capture_segment(s, [&]() { return fcg_init_a<double, TP>(s, v, st); }, m.a[0]);
    if (!rc) rc = capture_segment(s, [&]() { return fcg_iter_a<double, TP>(s, v, st); }, m.a[1]);
    if (!rc) rc = capture_segment(s, [&]() { return fcg_init_b<double, TP>(s, v, st); }, m.b[0]);
    if (!rc) rc = capture_segment(s, [&]() { return fcg_iter_b<double, TP>(s, v, st); }, m.b[1]);
    if (!rc && (m.a[0].g.size() != m.a[1].g.size() || m.b[0].g.size() != m.b[1].g.size()))
        rc = set_error(PA_EINVAL, "lockstep: first and later steps have different phases");
    if (!rc) rc = build_coarse_graph(s, st, &m.coarse);
    return rc;
}

}  // namespace

struct Lockstep {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    std::vector<LockMember> m;
    std::vector<LockstepDone> done;
};

namespace {

// Finishes member m (true residual, solution copy) into L.done.
void retire(Lockstep &L, LockMember &m, int rc_loop, bool converged)
{
    LockstepDone d;
    d.tag = m.tag;
    m.info.iterations = m.it;
    int st = solve_finish(m.s, m.x_out, rc_loop, converged, m.bb, m.tol2, &m.info);
    d.status = st;
    if (st != PA_OK) d.error = pa_last_error();
    d.info = m.info;
    L.done.push_back(d);
    free_member(m);
}

// Runs phases 0 .. n-1 of one segment kind for all members, batching the
// applies between phases; the last phase is launched but not joined.
int run_segment(Lockstep &L, bool second_half)
{
    // members may have different hierarchies, so different numbers of
    // phases: phase round j runs phase j of every member that has one, then
    // the applies that end those phases as one batched launch
    auto seg = [&](LockMember &m) -> Segment & {
        return second_half ? m.b[m.started ? 1 : 0] : m.a[m.started ? 1 : 0];
    };
    size_t nph = 0;
    for (LockMember &m : L.m) nph = std::max(nph, seg(m).g.size());
    std::vector<pa_op *> ops;
    std::vector<const void *> xs;
    std::vector<void *> ys;
    for (size_t j = 0; j < nph; ++j) {
        for (LockMember &m : L.m) {
            Segment &sg = seg(m);
            if (j < sg.g.size() && sg.g[j]) PA_CUDA_TRY(cudaGraphLaunch(sg.g[j], m.s->stream));
        }
        ops.clear();
        xs.clear();
        ys.clear();
        for (LockMember &m : L.m) {
            Segment &sg = seg(m);
            if (j + 1 >= sg.g.size()) continue;  // its last phase (or none): no apply follows
            const ApplyRec &ap = sg.ap[j];
            if (!ap.op) continue;
            PA_CUDA_TRY(cudaEventRecord(m.ev, m.s->stream));
            PA_CUDA_TRY(cudaStreamWaitEvent(L.st, m.ev, 0));
            ops.push_back(ap.op);
            xs.push_back(ap.x);
            ys.push_back(ap.y);
        }
        if (ops.empty()) continue;
        int rc = apply_batch_async(ops.data(), xs.data(), ys.data(), (int)ops.size(), L.st);
        if (rc) return rc;
        PA_CUDA_TRY(cudaEventRecord(L.ev, L.st));
        for (LockMember &m : L.m) {
            Segment &sg = seg(m);
            if (j + 1 < sg.g.size() && sg.ap[j].op) PA_CUDA_TRY(cudaStreamWaitEvent(m.s->stream, L.ev, 0));
        }
    }
    return PA_OK;
}

}  // namespace

int lockstep_create(Lockstep **out)
{
    *out = nullptr;
    Lockstep *L = new (std::nothrow) Lockstep;
    if (!L) return set_error(PA_ENOMEM, "lockstep: host allocation");
    cudaError_t e = cudaStreamCreateWithFlags(&L->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        lockstep_destroy(L);
        return cuda_error(e, "lockstep: stream or event creation");
    }
    *out = L;
    return PA_OK;
}

void lockstep_destroy(Lockstep *L)
{
    if (!L) return;
    for (LockMember &m : L->m) free_member(m);
    if (L->ev) cudaEventDestroy(L->ev);
    if (L->st) cudaStreamDestroy(L->st);
    delete L;
}

int lockstep_active(const Lockstep *L) { return (int)L->m.size(); }

void lockstep_take_done(Lockstep *L, std::vector<LockstepDone> &out)
{
    for (LockstepDone &d : L->done) out.push_back(d);
    L->done.clear();
}

int lockstep_add(Lockstep *L, pa_solver *s, const double *b, double *x, double rtol, int maxit, void *tag)
{
    if (s->mode != PA_SOLVE_FP64 && s->mode != PA_SOLVE_MIXED_FCG)
        return set_error(PA_EINVAL, "lockstep: only the flexible-CG modes (FP64, MIXED_FCG) step in lockstep");
    // a grid-wide persistent coarse kernel must not run beside other members
    s->allow_coop = false;
    LockMember m;
    m.s = s;
    m.x_out = x;
    m.tag = tag;
    m.maxit = maxit;
    m.tol2 = rtol * rtol;
    bool trivial = false;
    int rc = solve_begin(s, b, x, &m.bb, &m.info, &trivial);
    if (rc || trivial) {
        LockstepDone d;
        d.tag = tag;
        d.status = rc;
        if (rc) d.error = pa_last_error();
        d.info = m.info;
        d.info.status = rc;
        L->done.push_back(d);
        return PA_OK;
    }
    rc = s->mode == PA_SOLVE_FP64 ? capture_member<double>(m) : capture_member<float>(m);
    if (!rc && cudaEventCreateWithFlags(&m.ev, cudaEventDisableTiming) != cudaSuccess)
        rc = cuda_error(cudaGetLastError(), "lockstep: cudaEventCreate");
    if (rc) {
        free_member(m);
        return rc;
    }
    L->m.push_back(m);
    return PA_OK;
}

void solver_set_cancel(pa_solver *s, const std::atomic<int> *flag) { s->cancel = flag; }

int lockstep_cancel(Lockstep *L, void *tag)
{
    for (size_t i = 0; i < L->m.size(); ++i) {
        if (L->m[i].tag != tag) continue;
        LockMember m = L->m[i];
        L->m.erase(L->m.begin() + (std::ptrdiff_t)i);
        retire(*L, m, set_error(PA_ECANCELED, "solver: solve canceled"), false);
        return PA_OK;
    }
    return set_error(PA_EINVAL, "lockstep: no member with this tag");
}

// Members of any hierarchy step together; one lockstep per solve mode keeps
// each lane's members of one precision mix.
int lockstep_key(const pa_solver *s) { return s->mode; }

int lockstep_tick(Lockstep *L)
{
    NvtxRange nvtx("lockstep_tick");
    if (L->m.empty()) return PA_OK;
    int rc = run_segment(*L, false);
    if (rc) return rc;
    for (LockMember &m : L->m) PA_CUDA_TRY(cudaGraphLaunch(m.coarse, m.s->stream));
    rc = run_segment(*L, true);
    if (rc) return rc;
    for (LockMember &m : L->m) PA_CUDA_TRY(cudaStreamSynchronize(m.s->stream));
    // convergence test of every member, as in the solo loop
    std::vector<LockMember> keep;
    for (LockMember &m : L->m) {
        pa_solver *s = m.s;
        const double rr = s->h_scal[S_RR];
        s->coarse_its += s->h_flag[F_CIT];
        if (m.started) ++m.it;
        m.started = true;
        if (s->h_flag[F_CTIMEOUT]) {
            retire(*L, m, set_error(PA_ETIMEOUT, "solver: coarse-solve grid barrier timed out"), false);
            continue;
        }
        if (s->h_flag[F_BREAK]) {
            retire(*L, m,
                   set_error(PA_EBREAKDOWN, m.it == 0 ? "solver: non-finite value in the first preconditioned residual"
                                                      : "solver: CG breakdown (p^T A p <= 0 or non-finite value)"),
                   false);
            continue;
        }
        if (rr <= m.tol2 * m.bb || m.it >= m.maxit) {
            retire(*L, m, PA_OK, rr <= m.tol2 * m.bb);
            continue;
        }
        keep.push_back(m);
    }
    L->m.swap(keep);
    return PA_OK;
}

namespace {
}  // namespace
}  // namespace pa

using namespace pa;

extern "C" {

int pa_gmg_pcg_solve_batch(pa_solver *const *solvers, const double *const *b, double *const *x, int count,
                           double rtol, int maxit, pa_solve_info *infos, void *stream)
{
    if (count < 0 || (count > 0 && (!solvers || !b || !x)))
        return set_error(PA_EINVAL, "pa_gmg_pcg_solve_batch: bad arguments");
    if (!(rtol > 0.0) || maxit < 0) return set_error(PA_EINVAL, "pa_gmg_pcg_solve_batch: bad tolerance or cap");
    for (int k = 0; k < count; ++k) {
        if (!solvers[k] || !b[k] || !x[k]) return set_error(PA_EINVAL, "pa_gmg_pcg_solve_batch: null entry");
        for (int j = 0; j < k; ++j)
            if (solvers[j] == solvers[k]) return set_error(PA_EINVAL, "pa_gmg_pcg_solve_batch: a solver appears twice");
    }
    PA_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    Lockstep *L = nullptr;
    int rc = lockstep_create(&L);
    if (rc) return rc;
    std::vector<int> status(count, PA_OK);
    std::vector<std::string> errors(count);
    for (int k = 0; k < count && !rc; ++k) rc = lockstep_add(L, solvers[k], b[k], x[k], rtol, maxit, (void *)(intptr_t)k);
    while (!rc && lockstep_active(L) > 0) rc = lockstep_tick(L);
    std::vector<LockstepDone> done;
    lockstep_take_done(L, done);
    lockstep_destroy(L);
    if (rc) return rc;
    int first = PA_OK;
    std::string first_err;
    for (const LockstepDone &d : done) {
        const int k = (int)(intptr_t)d.tag;
        if (infos) infos[k] = d.info;
        status[k] = d.status;
        errors[k] = d.error;
    }
    for (int k = 0; k < count; ++k)
        if (status[k] != PA_OK && first == PA_OK) {
            first = status[k];
            first_err = errors[k];
        }
    if (first != PA_OK) set_error(first, first_err);
    return first;
}

}  // extern "C"
