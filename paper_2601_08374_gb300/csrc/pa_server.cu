// Solve server: continuous admission of elasticity solve requests.
//
// Requests are queued in arrival order.  A request is admitted as soon as a
// setup slot is free and its estimated device footprint fits in what the
// memory budget has left; a worker thread then builds it -- mesh, operators
// on every level, diagonals, eigenvalue estimates, load vector -- on a CUDA
// stream of its own.  Small flexible-CG requests then leave the slot for the
// batch lane of their hierarchy: a stepper thread advances all of its
// requests one CG step per tick with their operator applies batched into
// one launch per (precision, degree), and new requests join between ticks
// (continuous batching).  Other requests are solved by their worker on the
// solver's own stream, overlapping with everything else.  When a request
// finishes its memory is released and the next queued requests are
// admitted.  A request's hierarchy is its p-levels (halving to 1) and,
// where its box mesh is a uniform refinement, h-levels below them
// (PA_SERVER_OPT_H_LEVELS).  Every solve is deterministic (fixed-order
// reductions, no atomics in the arithmetic, batched applies with the
// arithmetic of single ones), so a request gives the same bits alone or in
// any mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pa_internal.h"

namespace {

using clk = std::chrono::steady_clock;

constexpr int kServerChebOrder = 4;  // Chebyshev degree of the served solves

struct Ticket {
    int64_t id = 0;
    pa_request req{};
    std::vector<int> levels;
    int hlev = 0;  // h-levels below the p-levels
    size_t footprint = 0;
    int state = 0;  // 0 queued, 1 running, 2 done
    int status = PA_OK;
    std::string error;
    pa_solve_info info{};
    clk::time_point t_submit, t_start, t_end;
    double setup_s = 0.0, solve_s = 0.0;
    int batched = 0;
    std::vector<double> x;  // host copy of the solution when requested
    std::atomic<int> cancel{0};  // pa_server_cancel of a running request
};

// Device resources of one request between setup and completion.
struct Res {
    pa_op *op = nullptr;
    pa_solver *sol = nullptr;
    double *b = nullptr, *x = nullptr;
    cudaStream_t st = nullptr;
};

// A request in the batch lane.
struct BatchJob {
    std::shared_ptr<Ticket> t;
    Res res;
    clk::time_point t_join;
};

// One lockstep batch (requests of one hierarchy) and its stepper thread.
struct Stepper {
    int key = 0;
    std::thread th;
    std::deque<BatchJob *> inbox;
    int members = 0;
};

// Degrees of the p-hierarchy: halve down to 1 (8-4-2-1, 6-3-1, 4-2-1, 2-1).
std::vector<int> p_levels_for(int p)
{
    std::vector<int> lv{p};
    while (lv.back() > 1) lv.push_back(lv.back() / 2);
    return lv;
}

// h-levels under the p-hierarchy of a box mesh: halve the element counts
// while all three are even, the hierarchy has at most 8 levels, and the
// p = 1 level above still has more than 320 dofs (the size whose assembled
// matrix the solver inverts densely).
int h_levels_for(const pa_request &r, int np)
{
    int nx = r.nx, ny = r.ny, nz = r.nz, h = 0;
    while (np + h < 8 && !(nx & 1) && !(ny & 1) && !(nz & 1) && 3LL * (nx + 1) * (ny + 1) * (nz + 1) > 320) {
        nx /= 2;
        ny /= 2;
        nz /= 2;
        ++h;
    }
    return h;
}

// Device bytes that pa_op_setup + pa_solver_create + the request's own
// vectors allocate (sum of the documented allocations).
size_t footprint_bytes(const pa_request &r, const std::vector<int> &levels, int hlev)
{
    size_t total = 0, n0 = 0;
    const size_t nlev = levels.size() + (size_t)hlev;
    for (size_t l = 0; l < nlev; ++l) {
        const int p = l < levels.size() ? levels[l] : 1, D = p + 1;
        const int sh = l < levels.size() ? 0 : (int)(l + 1 - levels.size());  // halvings of the mesh
        const size_t nx = (size_t)(r.nx >> sh), ny = (size_t)(r.ny >> sh), nz = (size_t)(r.nz >> sh);
        const size_t ne = nx * ny * nz;
        const size_t N = 3 * (nx * p + 1) * (ny * p + 1) * (nz * p + 1);
        if (l == 0) n0 = N;
        auto op_bytes = [&](size_t elem) {
            return ne * 12 * elem + ne * 96 + ne * 3 * (size_t)D * D * D * elem + 2 * N * elem + N;
        };
        total += op_bytes(8) + 5 * N * 8 + (l + 1 < nlev ? 2 : 4) * N * 8;
        if (r.mode != PA_SOLVE_FP64) total += op_bytes(4) + 7 * N * 4;
    }
    total += 7 * n0 * 8 + (r.mode == PA_SOLVE_MIXED ? 6 * n0 * 4 : 0);
    total += 2 * n0 * 8;  // b and x of the request
    return total + total / 10 + ((size_t)16 << 20);
}

}  // namespace

struct pa_server {
    size_t budget = 0, used = 0, peak_used = 0;
    int max_slots = 1, running = 0, device = 0;
    int64_t next_id = 1, completed = 0;
    std::deque<std::shared_ptr<Ticket>> queue;
    std::unordered_map<int64_t, std::shared_ptr<Ticket>> tickets;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::thread> workers;
    bool stop = false;
    // batch lane
    bool batch = true;
    bool h_levels = true;  // h-levels under the p-levels where the mesh allows
    int64_t batch_max_dofs = 2000000;
    int batch_max_members = 64;
    int64_t in_lane = 0;  // handed to a stepper, not finished
    std::vector<std::unique_ptr<Stepper>> steppers;
    std::condition_variable cv_lane;
    bool stop_lanes = false;
    int64_t batched = 0, batch_ticks = 0, batch_member_ticks = 0, batch_max_seen = 0;
};

namespace {

void release(Res &r)
{
    cudaFree(r.b);
    cudaFree(r.x);
    pa_solver_destroy(r.sol);
    pa_op_destroy(r.op);
    if (r.st) cudaStreamDestroy(r.st);
    r = Res{};
}

// Builds an admitted request on the calling thread: operators, solver, load
// vector b and x = 0 (all ready on the device when it returns PA_OK).
int setup_request(pa_server *srv, Ticket &t, Res &res)
{
    pa::NvtxRange nvtx("server: request setup");
    const pa_request &r = t.req;
    pa_mesh *mesh = nullptr;
    int rc = PA_OK;
    do {
        if (cudaSetDevice(srv->device) != cudaSuccess) { rc = pa::cuda_error(cudaGetLastError(), "cudaSetDevice"); break; }
        if (cudaStreamCreateWithFlags(&res.st, cudaStreamNonBlocking) != cudaSuccess) {
            rc = pa::cuda_error(cudaGetLastError(), "cudaStreamCreate");
            break;
        }
        double lam = 0, mu = 0;
        if ((rc = pa_lame(r.E, r.nu, &lam, &mu))) break;
        if ((rc = pa_mesh_create(r.nx, r.ny, r.nz, r.box, nullptr, &mesh))) break;
        std::vector<uint8_t> ess;
        if (r.clamp_x0) {
            const int64_t Mx = (int64_t)r.nx * r.p + 1, My = (int64_t)r.ny * r.p + 1, Mz = (int64_t)r.nz * r.p + 1;
            const int64_t Nn = Mx * My * Mz;
            ess.assign((size_t)(3 * Nn), 0);
            for (int c = 0; c < 3; ++c)
                for (int64_t g = 0; g < Nn; g += Mx) ess[(size_t)(c * Nn + g)] = 1;  // gx = 0
        }
        if ((rc = pa_op_setup(mesh, r.p, 0, lam, mu, PA_FP64, ess.empty() ? nullptr : ess.data(), &res.op))) break;
        pa_mesh_destroy(mesh);
        mesh = nullptr;
        // Chebyshev degree 4 on [0.05, 1.2] lambda_max: the fastest setting of
        // the measured degree / interval sweep on beams and cubes
        if ((rc = pa_solver_create_hp(res.op, (int)t.levels.size(), t.levels.data(), t.hlev, kServerChebOrder, 1e-2, 10,
                                      r.mode, &res.sol)))
            break;
        // concurrent solvers must not each hold a grid-wide barrier
        pa_solver_set_option(res.sol, PA_SOLVER_OPT_PERSISTENT_COARSE, 0.0);
        pa::solver_set_cancel(res.sol, &t.cancel);
        const size_t n = (size_t)res.op->ndofs();
        if (cudaMalloc((void **)&res.b, n * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void **)&res.x, n * sizeof(double)) != cudaSuccess) {
            rc = pa::set_error(PA_ENOMEM, "server: device allocation for b, x");
            break;
        }
        if ((rc = pa_op_rhs(res.op, r.f0, r.nmodes, r.nmodes ? r.modes : nullptr, res.b, res.st))) break;
        if (cudaMemsetAsync(res.x, 0, n * sizeof(double), res.st) != cudaSuccess ||
            cudaStreamSynchronize(res.st) != cudaSuccess) {
            rc = pa::cuda_error(cudaGetLastError(), "server: load vector");
            break;
        }
    } while (false);
    pa_mesh_destroy(mesh);
    return rc;
}

// Records a finished solve in the ticket (solution copied to the host when
// kept) and frees the request's device resources.
void record_result(Ticket &t, Res &res, int status, const pa_solve_info &info, const std::string &err)
{
    t.status = status;
    t.info = info;
    if (status == PA_ECANCELED) t.info.status = PA_ECANCELED;
    if (status != PA_OK) t.error = err;
    if (t.req.keep_solution && res.x && status != PA_EINVAL) {
        const size_t n = (size_t)res.op->ndofs();
        t.x.resize(n);
        if (cudaMemcpy(t.x.data(), res.x, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
            t.status = pa::cuda_error(cudaGetLastError(), "cudaMemcpy solution");
            t.error = pa_last_error();
        }
    }
    release(res);
}

// Marks a ticket done and returns its memory (caller holds srv->mu).
void complete_locked(pa_server *srv, Ticket &t)
{
    t.t_end = clk::now();
    t.state = 2;
    srv->used -= t.footprint;
    ++srv->completed;
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
}

bool batchable(const pa_server *srv, const Ticket &t)
{
    const pa_request &r = t.req;
    const int64_t n = 3LL * (r.nx * (int64_t)r.p + 1) * (r.ny * (int64_t)r.p + 1) * (r.nz * (int64_t)r.p + 1);
    return srv->batch && (r.mode == PA_SOLVE_FP64 || r.mode == PA_SOLVE_MIXED_FCG) && n <= srv->batch_max_dofs;
}

void stepper_main(pa_server *srv, Stepper *sp);

// Hands a built request to the stepper of its hierarchy (caller holds
// srv->mu); the stepper is started on first use.
void hand_to_lane(pa_server *srv, BatchJob *job)
{
    const int key = pa::lockstep_key(job->res.sol);
    Stepper *sp = nullptr;
    for (auto &x : srv->steppers)
        if (x->key == key) sp = x.get();
    if (!sp) {
        srv->steppers.emplace_back(new Stepper);
        sp = srv->steppers.back().get();
        sp->key = key;
        sp->th = std::thread(stepper_main, srv, sp);
    }
    sp->inbox.push_back(job);
    srv->cv_lane.notify_all();
}

// Stepper thread: joins waiting requests between ticks, runs one lockstep
// tick for all members, completes the members that finished.
void stepper_main(pa_server *srv, Stepper *sp)
{
    cudaSetDevice(srv->device);
    pa::Lockstep *L = nullptr;
    int rc_create = pa::lockstep_create(&L);
    std::string create_err = rc_create ? pa_last_error() : "";
    std::vector<BatchJob *> active;
    std::vector<pa::LockstepDone> done;
    auto finish = [&](BatchJob *job, int status, const pa_solve_info &info, const std::string &err) {
        job->t->solve_s = std::chrono::duration<double>(clk::now() - job->t_join).count();
        record_result(*job->t, job->res, status, info, err);
        std::lock_guard<std::mutex> lk(srv->mu);
        --srv->in_lane;
        ++srv->batched;
        complete_locked(srv, *job->t);
        delete job;
    };
    std::unique_lock<std::mutex> lk(srv->mu);
    while (true) {
        srv->cv_lane.wait(lk, [&] { return srv->stop_lanes || !sp->inbox.empty() || sp->members > 0; });
        if (sp->inbox.empty() && sp->members == 0) {
            if (srv->stop_lanes) break;
            continue;
        }
        std::vector<BatchJob *> joining;
        while (!sp->inbox.empty() && (int)(active.size() + joining.size()) < srv->batch_max_members) {
            joining.push_back(sp->inbox.front());
            sp->inbox.pop_front();
        }
        lk.unlock();
        for (BatchJob *job : joining) {
            job->t_join = clk::now();
            int rc = rc_create ? rc_create
                               : pa::lockstep_add(L, job->res.sol, job->res.b, job->res.x, job->t->req.rtol,
                                                  job->t->req.maxit, job);
            if (rc) finish(job, rc, pa_solve_info{}, rc_create ? create_err : std::string(pa_last_error()));
            else active.push_back(job);
        }
        // members canceled since the last tick leave before the next one
        if (!rc_create)
            for (BatchJob *job : active)
                if (job->t->cancel.load()) pa::lockstep_cancel(L, job);
        int stepped = 0;
        if (!rc_create && pa::lockstep_active(L) > 0) {
            stepped = pa::lockstep_active(L);
            int rc = pa::lockstep_tick(L);
            if (rc) {
                // a failed launch: every member ends with the error, and the
                // batch starts afresh
                std::string err = pa_last_error();
                pa::lockstep_destroy(L);
                L = nullptr;
                for (BatchJob *job : active) finish(job, rc, pa_solve_info{}, err);
                active.clear();
                rc_create = pa::lockstep_create(&L);
                create_err = rc_create ? pa_last_error() : "";
            }
        }
        if (L) {
            done.clear();
            pa::lockstep_take_done(L, done);
            for (const pa::LockstepDone &d : done) {
                BatchJob *job = static_cast<BatchJob *>(d.tag);
                active.erase(std::find(active.begin(), active.end(), job));
                finish(job, d.status, d.info, d.error);
            }
        }
        lk.lock();
        sp->members = (int)active.size();
        if (stepped) {
            ++srv->batch_ticks;
            srv->batch_member_ticks += stepped;
            srv->batch_max_seen = std::max<int64_t>(srv->batch_max_seen, stepped);
        }
    }
    lk.unlock();
    pa::lockstep_destroy(L);
}

void worker_main(pa_server *srv)
{
    std::unique_lock<std::mutex> lk(srv->mu);
    while (true) {
        // admit the head of the queue when a slot and memory are free; a
        // request larger than the whole budget is rejected instead of waiting
        std::shared_ptr<Ticket> t;
        srv->cv_work.wait(lk, [&] {
            if (srv->stop) return true;
            if (srv->queue.empty() || srv->running >= srv->max_slots) return false;
            const auto &h = srv->queue.front();
            return h->footprint > srv->budget || srv->used + h->footprint <= srv->budget;
        });
        if (srv->stop) return;
        t = srv->queue.front();
        srv->queue.pop_front();
        if (t->footprint > srv->budget) {
            t->state = 2;
            t->status = PA_EBUSY;
            t->error = "server: request footprint exceeds the whole memory budget";
            t->t_start = t->t_end = clk::now();
            ++srv->completed;
            srv->cv_done.notify_all();
            srv->cv_work.notify_all();
            continue;
        }
        srv->used += t->footprint;
        srv->peak_used = std::max(srv->peak_used, srv->used);
        ++srv->running;
        t->state = 1;
        t->t_start = clk::now();
        const bool lane = batchable(srv, *t);
        // another request may fit as well
        srv->cv_work.notify_all();
        lk.unlock();
        Res res;
        int rc = setup_request(srv, *t, res);
        auto t_setup = clk::now();
        t->setup_s = std::chrono::duration<double>(t_setup - t->t_start).count();
        if (rc == PA_OK && lane) {
            BatchJob *job = new BatchJob{t, res, t_setup};
            lk.lock();
            t->batched = 1;
            --srv->running;
            ++srv->in_lane;
            hand_to_lane(srv, job);
            srv->cv_work.notify_all();
            continue;
        }
        if (rc == PA_OK && t->cancel.load()) {
            rc = pa::set_error(PA_ECANCELED, "server: request canceled during its setup");
            t->solve_s = 0.0;
            record_result(*t, res, rc, pa_solve_info{}, pa_last_error());
        } else if (rc == PA_OK) {
            pa_solve_info info{};
            rc = pa_gmg_pcg_solve(res.sol, res.b, res.x, t->req.rtol, t->req.maxit, &info, res.st);
            t->solve_s = std::chrono::duration<double>(clk::now() - t_setup).count();
            record_result(*t, res, rc, info, rc != PA_OK ? std::string(pa_last_error()) : std::string());
        } else {
            record_result(*t, res, rc, pa_solve_info{}, pa_last_error());
        }
        lk.lock();
        --srv->running;
        complete_locked(srv, *t);
    }
}

}  // namespace

using namespace pa;

extern "C" {

int pa_server_create(size_t budget_bytes, int max_slots, pa_server **out)
{
    if (!out) return set_error(PA_EINVAL, "pa_server_create: null output");
    *out = nullptr;
    if (max_slots < 1 || max_slots > 64) return set_error(PA_EINVAL, "pa_server_create: max_slots in 1..64");
    if (budget_bytes == 0) return set_error(PA_EINVAL, "pa_server_create: zero memory budget");
    pa_server *s = new (std::nothrow) pa_server;
    if (!s) return set_error(PA_ENOMEM, "pa_server_create: host allocation");
    s->budget = budget_bytes;
    s->max_slots = max_slots;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return cuda_error(cudaGetLastError(), "pa_server_create: cudaGetDevice");
    }
    try {
        for (int i = 0; i < max_slots; ++i) s->workers.emplace_back(worker_main, s);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        for (auto &w : s->workers) w.join();
        delete s;
        return set_error(PA_ENOMEM, "pa_server_create: could not start worker threads");
    }
    *out = s;
    return PA_OK;
}

int pa_server_submit(pa_server *s, const pa_request *req, int64_t *ticket)
{
    if (!s || !req || !ticket) return set_error(PA_EINVAL, "pa_server_submit: null argument");
    if (req->nx < 1 || req->ny < 1 || req->nz < 1 || req->p < 1 || req->p > kMaxP)
        return set_error(PA_EINVAL, "pa_server_submit: bad mesh size or degree");
    if (req->nmodes < 0 || req->nmodes > PA_REQUEST_MAX_MODES) return set_error(PA_EINVAL, "pa_server_submit: nmodes");
    if (req->mode != PA_SOLVE_FP64 && req->mode != PA_SOLVE_MIXED && req->mode != PA_SOLVE_MIXED_FCG)
        return set_error(PA_EINVAL, "pa_server_submit: mode");
    if (!(req->rtol > 0.0) || req->maxit < 1) return set_error(PA_EINVAL, "pa_server_submit: rtol or maxit");
    auto t = std::make_shared<Ticket>();
    t->req = *req;
    t->levels = p_levels_for(req->p);
    t->t_submit = clk::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        t->hlev = s->h_levels ? h_levels_for(*req, (int)t->levels.size()) : 0;
        t->footprint = footprint_bytes(*req, t->levels, t->hlev);
        t->id = s->next_id++;
        s->tickets[t->id] = t;
        s->queue.push_back(t);
    }
    s->cv_work.notify_all();
    *ticket = t->id;
    return PA_OK;
}

int pa_server_poll(pa_server *s, int64_t ticket, int *done)
{
    if (!s || !done) return set_error(PA_EINVAL, "pa_server_poll: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return set_error(PA_EINVAL, "pa_server_poll: unknown ticket");
    *done = it->second->state == 2;
    return PA_OK;
}

int pa_server_wait(pa_server *s, int64_t ticket, double *x_host, int64_t x_len, pa_solve_info *info,
                   pa_request_timing *timing)
{
    if (!s) return set_error(PA_EINVAL, "pa_server_wait: null server");
    std::shared_ptr<Ticket> t;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->tickets.find(ticket);
        if (it == s->tickets.end()) return set_error(PA_EINVAL, "pa_server_wait: unknown ticket");
        t = it->second;
        s->cv_done.wait(lk, [&] { return t->state == 2; });
        s->tickets.erase(it);
    }
    if (info) *info = t->info;
    if (timing) {
        timing->batched = t->batched;
        timing->levels = (int)t->levels.size() + t->hlev;
        timing->h_levels = t->hlev;
        timing->latency_s = std::chrono::duration<double>(t->t_end - t->t_submit).count();
        timing->queue_s = std::chrono::duration<double>(t->t_start - t->t_submit).count();
        timing->setup_s = t->setup_s;
        timing->solve_s = t->solve_s;
        timing->footprint_bytes = (int64_t)t->footprint;
    }
    if (x_host) {
        if (t->x.empty()) return set_error(PA_EINVAL, "pa_server_wait: the request did not keep its solution");
        if (x_len != (int64_t)t->x.size()) return set_error(PA_EINVAL, "pa_server_wait: x_len does not match");
        std::memcpy(x_host, t->x.data(), t->x.size() * sizeof(double));
    }
    if (t->status != PA_OK) set_error(t->status, t->error);
    return t->status;
}

int pa_server_cancel(pa_server *s, int64_t ticket)
{
    if (!s) return set_error(PA_EINVAL, "pa_server_cancel: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return set_error(PA_EINVAL, "pa_server_cancel: unknown ticket");
    Ticket &t = *it->second;
    if (t.state == 0) {
        // still queued: it holds no memory and never starts
        auto q = std::find(s->queue.begin(), s->queue.end(), it->second);
        if (q != s->queue.end()) s->queue.erase(q);
        t.state = 2;
        t.status = PA_ECANCELED;
        t.info.status = PA_ECANCELED;
        t.error = "server: request canceled before admission";
        t.t_start = t.t_end = clk::now();
        ++s->completed;
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    } else if (t.state == 1) {
        // running: its setup is skipped past, its solve ends at the next CG
        // step (worker) or before the next tick (batch lane)
        t.cancel.store(1);
        s->cv_lane.notify_all();
    }
    return PA_OK;
}

int pa_server_stats(pa_server *s, pa_server_stats_t *out)
{
    if (!s || !out) return set_error(PA_EINVAL, "pa_server_stats: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->queued = (int64_t)s->queue.size();
    out->running = s->running;
    out->completed = s->completed;
    out->used_bytes = (int64_t)s->used;
    out->peak_used_bytes = (int64_t)s->peak_used;
    out->batched = s->batched;
    out->batch_ticks = s->batch_ticks;
    out->batch_member_ticks = s->batch_member_ticks;
    out->batch_max_members = s->batch_max_seen;
    return PA_OK;
}

int pa_server_set_option(pa_server *s, int option, double value)
{
    if (!s) return set_error(PA_EINVAL, "pa_server_set_option: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    switch (option) {
    case PA_SERVER_OPT_BATCH: s->batch = value != 0.0; return PA_OK;
    case PA_SERVER_OPT_BATCH_MAX_DOFS:
        if (!(value >= 0.0)) return set_error(PA_EINVAL, "pa_server_set_option: negative dof count");
        s->batch_max_dofs = (int64_t)value;
        return PA_OK;
    case PA_SERVER_OPT_BATCH_MAX_MEMBERS:
        if (!(value >= 1.0 && value <= 256.0)) return set_error(PA_EINVAL, "pa_server_set_option: members in 1..256");
        s->batch_max_members = (int)value;
        return PA_OK;
    case PA_SERVER_OPT_H_LEVELS: s->h_levels = value != 0.0; return PA_OK;
    default: return set_error(PA_EINVAL, "pa_server_set_option: unknown option");
    }
}

int pa_server_destroy(pa_server *s)
{
    if (!s) return PA_OK;
    {
        // finish what is queued, running or batched, then stop the threads
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_done.wait(lk, [&] { return s->queue.empty() && s->running == 0 && s->in_lane == 0; });
        s->stop = true;
        s->stop_lanes = true;
    }
    s->cv_work.notify_all();
    s->cv_lane.notify_all();
    for (auto &w : s->workers) w.join();
    for (auto &sp : s->steppers) sp->th.join();
    delete s;
    return PA_OK;
}

}  // extern "C"
