// serve.cu -- a serving engine for interpolation requests with continuous batching.
//
// Requests (points, values, targets, spline order) arrive at any time from any host
// thread.  A scheduler thread admits them while job slots and the device-memory budget
// allow; host worker threads build each admitted job's plan (tree, FMM tables, QR, Vecchia
// factor) on the job's own stream and start its PCG solve (the Q_perp-projected system of
// Eq. 2.5 with the Vecchia preconditioner of Sec. 2.2); from then on the job's tree,
// factor and PCG state stay on the device until it finishes.  Every scheduler tick
// advances all active jobs by one PCG iteration: each job's FMM matvec (Sec. 2.1) and
// Vecchia apply run on its own stream, so jobs of different sizes overlap on the GPU, and
// the vector operations of all of them -- projection, CG update, inner products, direction
// update -- run as shared launches over a table of the active jobs (plan.cuh: the table
// steps).  A job's FMM matvec and Vecchia apply are captured once, at setup, into CUDA
// graphs replayed every tick (one launch each instead of the FMM's ~100 kernel launches,
// which for small jobs is what limits a tick).  One device-to-host copy per tick brings
// every job's residual; converged jobs
// leave the tick (a worker computes beta, evaluates the targets and returns the
// results), and new jobs join as slots and memory free up.  A job's arithmetic is the
// same as phs_fit's (the same begin/end and the same table steps with a table of one),
// so its result is identical whether it runs alone or in the mix.  Precision 1-4 jobs
// run phs_fit's FP64 refinement around their inner solves (a worker takes each
// refinement step between the inner solves' ticks).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "plan.cuh"

namespace phs {
namespace {

enum JobState { J_PENDING, J_SETUP, J_ACTIVE, J_REFINE, J_FINISH, J_DONE };

struct Job {
    int64_t id = 0;
    int k = 2, deg = -1, fmm_order = 0, vm = 30;
    phs_options opt{};
    int64_t n = 0, m = 0;
    std::vector<double> pts, f, tgt;    // host inputs
    std::vector<double> w, beta, pred;  // host outputs
    double t_submit = 0, t_admit = 0, t_ready = 0, t_done = 0;
    JobState state = J_PENDING;
    phs_status status = PHS_OK;
    std::string err;
    int64_t reserved = 0;  // bytes reserved against the budget
    phs_plan_t pl = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    double *dbuf = nullptr;  // inputs and outputs on the device: pts 2n, f n, tgt 2m, w n, beta 16, pred m
    size_t dbytes = 0;
    FitStart st{};
    double rr = 0;            // r . r of the current (inner) solve
    int it = 0;               // iterations of the current (inner) solve
    int iters = 0, outer = 0; // refinement: inner iterations so far, refinement steps
    double itol = 0;          // the current solve's stopping threshold
    int imax = 0;             // and its iteration limit
    double *rhs_p = nullptr, *x_p = nullptr;  // the current solve's right-hand side and iterate
    bool converged = false;
    // the iteration's per-job work captured once: y = M' p (FMM) and t2 = S~^-1 r (Vecchia)
    cudaGraphExec_t g_mv = nullptr, g_pc = nullptr;
    int64_t n_mv_kernels = 0, n_pc_kernels = 0;
    int mv_prec = 0;          // the current solve's operator (fit_precision / inner_precision)
    int g_mv_prec = -1;       // the operator g_mv was captured with
    phs_fit_info info{};
    double *pts_d() { return dbuf; }
    double *f_d() { return dbuf + 2 * n; }
    double *tgt_d() { return dbuf + 3 * n; }
    double *w_d() { return dbuf + 3 * n + 2 * m; }
    double *beta_d() { return dbuf + 4 * n + 2 * m; }
    double *pred_d() { return dbuf + 4 * n + 2 * m + 16; }
};

// a-priori device bytes of a job: plan state (coordinates, tree and lists, expansions,
// QR, Vecchia factor and its transpose, 12 work vectors) plus call temporaries and the
// job's own inputs and outputs; corrected to the plan's measured size once it exists
int64_t estimate_bytes(int64_t n, int64_t m, int vm) {
    return (64ll << 20) + n * (int64_t)(700 + 48 * vm) + 24 * m;
}

// Start the job's next PCG solve, as phs_fit does: the whole solve (precision 0: rhs =
// work vector 8, x = 9, to tol) or the next correction of the refinement (precision 1-4:
// rhs = 11, x = 8, to the inner tolerance).  Synchronises the job's stream.
void start_solve(Job *j) {
    phs_plan *pl = j->pl;
    const phs_options &o = pl->opt;
    if (fit_precision(pl) == 0) {
        j->mv_prec = 0;
        j->rhs_p = W(pl, 8);
        j->x_p = W(pl, 9);
        j->itol = j->st.stop;
        j->imax = o.maxiter;
    } else {
        j->mv_prec = inner_precision(pl, j->outer);
        j->rhs_p = W(pl, 11);
        j->x_p = W(pl, 8);
        j->itol = refine_inner_tol(o, std::sqrt(j->rr), j->st.stop);
        j->imax = refine_inner_maxiter(o, j->iters);
    }
    j->it = 0;
    j->rr = pcg_start(pl, j->rhs_p, j->x_p, j->s);
}
// the current solve has ended (converged to itol or reached imax)
bool solve_ended(const Job *j) { return std::sqrt(j->rr) <= j->itol || j->it >= j->imax; }

// Capture fn's work on the job's stream into an executable graph (thread-local capture:
// other threads keep issuing work meanwhile); *kernels receives its kernel count.
template <typename Fn>
cudaGraphExec_t capture(cudaStream_t s, int64_t *kernels, Fn &&fn) {
    cudaGraph_t g = nullptr;
    PHS_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    try {
        fn();
    } catch (...) {
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    PHS_CUDA(cudaStreamEndCapture(s, &g));
    size_t nn = 0;
    PHS_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) PHS_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
    int64_t kc = 0;
    for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType t;
        PHS_CUDA(cudaGraphNodeGetType(nodes[i], &t));
        if (t == cudaGraphNodeTypeKernel) ++kc;
    }
    *kernels = kc;
    cudaGraphExec_t ex = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    PHS_CUDA(e);
    return ex;
}

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace
}  // namespace phs

using namespace phs;

struct phs_server {
    int dev = 0;
    int64_t budget = 0;
    int max_active = 32;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    std::mutex mu;
    std::condition_variable cv_sched, cv_work, cv_done;
    std::deque<Job *> pending, work;
    std::vector<Job *> active;
    std::map<int64_t, std::unique_ptr<Job>> jobs;
    int64_t next_id = 1, reserved = 0;
    int n_setup = 0, n_finish = 0;
    bool stop = false;          // no more submissions: the scheduler drains and exits
    bool stop_workers = false;  // set once the scheduler has exited
    std::thread sched;
    std::vector<std::thread> workers;
    cudaStream_t engine = nullptr;
    double *rr_dev = nullptr, *rr_host = nullptr;
    // statistics
    int64_t ticks = 0, batched_jobs = 0, max_concurrent = 0, max_reserved = 0, completed = 0;

    void worker_loop();
    void sched_loop();
    void setup(Job *j);
    void finish(Job *j);
    void refine(Job *j);
    void tick(std::vector<Job *> &act);
};

void phs_server::setup(Job *j) {
    try {
        PHS_CUDA(cudaStreamCreateWithFlags(&j->s, cudaStreamNonBlocking));
        PHS_CUDA(cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming));
        j->dbytes = (size_t)(4 * j->n + 3 * j->m + 16) * sizeof(double);
        PHS_CUDA(cudaMallocFromPoolAsync((void **)&j->dbuf, j->dbytes, scratch_pool(), j->s));
        PHS_CUDA(cudaMemcpyAsync(j->pts_d(), j->pts.data(), 2 * j->n * sizeof(double), cudaMemcpyHostToDevice, j->s));
        PHS_CUDA(cudaMemcpyAsync(j->f_d(), j->f.data(), j->n * sizeof(double), cudaMemcpyHostToDevice, j->s));
        if (j->m)
            PHS_CUDA(cudaMemcpyAsync(j->tgt_d(), j->tgt.data(), 2 * j->m * sizeof(double), cudaMemcpyHostToDevice, j->s));
        phs_status st = phs_plan_create(j->pts_d(), j->n, j->k, j->deg, j->fmm_order, j->vm, &j->opt,
                                        (phs_stream_t)j->s, &j->pl);
        if (st != PHS_OK) throw Error{st, phs_last_error()};
        phs_plan *pl = j->pl;
        AllocScope scope(j->s, &pl->dev_bytes);
        pl->last_stream = j->s;
        j->st = fit_begin(pl, j->f_d(), j->s);
        if (!j->st.trivial) {
            if (fit_precision(pl) != 0) fit_refine_begin(pl, j->s);
            j->rr = j->st.nrm0 * j->st.nrm0;
            start_solve(j);
            // one uncaptured matvec sizes every lazily allocated buffer (its output, work
            // vector 4, is overwritten by the first tick); then both pieces are captured
            const int prec = j->mv_prec;
            matvec_norm(pl, W(pl, 2), W(pl, 4), prec, j->s);
            j->g_mv = capture(j->s, &j->n_mv_kernels, [&] { matvec_norm(pl, W(pl, 2), W(pl, 4), prec, j->s); });
            j->g_mv_prec = prec;
            j->g_pc = capture(j->s, &j->n_pc_kernels,
                              [&] { vecchia_apply(pl->vec, W(pl, 0), W(pl, 5), W(pl, 6), j->s); });
            PHS_CUDA(cudaStreamSynchronize(j->s));
        }
        // the measured plan size replaces the a-priori estimate (temporaries: a quarter more)
        const int64_t actual = pl->dev_bytes + pl->dev_bytes / 4 + (int64_t)j->dbytes;
        std::lock_guard<std::mutex> g(mu);
        reserved += actual - j->reserved;
        j->reserved = actual;
        max_reserved = std::max(max_reserved, reserved);
        j->t_ready = now_s(t0);
        if (j->st.trivial) {
            j->converged = true;
            j->state = J_FINISH;
            ++n_finish;
            work.push_back(j);
            cv_work.notify_one();
        } else if (solve_ended(j)) {
            j->state = fit_precision(pl) == 0 ? J_FINISH : J_REFINE;
            if (fit_precision(pl) == 0) j->converged = true;
            ++n_finish;
            work.push_back(j);
            cv_work.notify_one();
        } else {
            j->state = J_ACTIVE;
            active.push_back(j);
            cv_sched.notify_one();
        }
        --n_setup;
    } catch (const Error &e) {
        std::lock_guard<std::mutex> g(mu);
        j->status = e.code;
        j->err = e.msg;
        j->state = J_FINISH;
        ++n_finish;
        work.push_back(j);
        --n_setup;
        cv_work.notify_one();
    }
}

// A correction has ended (precision 1-4): x += dx and the FP64 residual; then, as in
// phs_fit's loop, finish when it meets the tolerance, or when the correction took no
// iteration, or when the refinement budget is spent; else start the next correction.
void phs_server::refine(Job *j) {
    bool again = false;
    try {
        phs_plan *pl = j->pl;
        AllocScope scope(j->s, &pl->dev_bytes);
        pl->last_stream = j->s;
        const phs_options &o = pl->opt;
        j->iters += j->it;
        ++j->outer;
        const double res = fit_refine_step(pl, j->s);
        const int it_inner = j->it;
        j->rr = res * res;
        if (res <= j->st.stop) {
            j->converged = true;
        } else if (it_inner != 0 && j->outer < o.max_refine && j->iters < o.maxiter) {
            start_solve(j);
            if (j->g_mv && j->g_mv_prec != j->mv_prec) {  // the corrections' operator differs
                PHS_CUDA(cudaGraphExecDestroy(j->g_mv));
                const int prec = j->mv_prec;
                matvec_norm(pl, W(pl, 2), W(pl, 4), prec, j->s);
                j->g_mv = capture(j->s, &j->n_mv_kernels, [&] { matvec_norm(pl, W(pl, 2), W(pl, 4), prec, j->s); });
                j->g_mv_prec = prec;
            }
            again = !solve_ended(j);
            if (!again) {  // the correction ended at once: refine again
                std::lock_guard<std::mutex> g(mu);
                work.push_back(j);
                cv_work.notify_one();
                return;
            }
        }
    } catch (const Error &e) {
        j->status = e.code;
        j->err = e.msg;
    }
    std::lock_guard<std::mutex> g(mu);
    if (again) {
        j->state = J_ACTIVE;
        active.push_back(j);
        --n_finish;
        cv_sched.notify_one();
    } else {
        j->state = J_FINISH;
        work.push_back(j);
        cv_work.notify_one();
    }
}

void phs_server::finish(Job *j) {
    if (j->pl && j->status == PHS_OK) {
        try {
            phs_plan *pl = j->pl;
            AllocScope scope(j->s, &pl->dev_bytes);
            pl->last_stream = j->s;
            const double rr_true = fit_end(pl, j->w_d(), j->beta_d(), j->s, j->outer > 0);
            if (j->m) {
                const phs_status st = phs_eval(j->pl, j->w_d(), j->beta_d(), j->tgt_d(), j->m, j->pred_d(),
                                               (phs_stream_t)j->s);
                if (st != PHS_OK) throw Error{st, phs_last_error()};
            }
            m2l_tc_check(pl->fmm, j->s);
            j->w.resize(j->n);
            j->beta.resize(pl->S);
            j->pred.resize(j->m);
            PHS_CUDA(cudaMemcpyAsync(j->w.data(), j->w_d(), j->n * sizeof(double), cudaMemcpyDeviceToHost, j->s));
            PHS_CUDA(cudaMemcpyAsync(j->beta.data(), j->beta_d(), pl->S * sizeof(double), cudaMemcpyDeviceToHost, j->s));
            if (j->m)
                PHS_CUDA(cudaMemcpyAsync(j->pred.data(), j->pred_d(), j->m * sizeof(double), cudaMemcpyDeviceToHost,
                                         j->s));
            PHS_CUDA(cudaStreamSynchronize(j->s));
            const double nrm0 = j->st.nrm0;
            j->info.iters = fit_precision(j->pl) == 0 ? j->it : j->iters;
            j->info.outer_iters = j->outer;
            j->info.converged = j->converged ? 1 : 0;
            j->info.jittered = (int)pl->vec.jittered;
            j->info.rel_res_recursive = nrm0 > 0 ? std::sqrt(j->rr) / nrm0 : 0.0;
            j->info.rel_res_true = nrm0 > 0 ? std::sqrt(rr_true) / nrm0 : 0.0;
            j->info.ms_plan = pl->ms_plan;
            if (!j->converged) {
                j->status = PHS_ERR_NOT_CONVERGED;
                j->err = "PCG did not reach the tolerance";
            }
        } catch (const Error &e) {
            j->status = e.code;
            j->err = e.msg;
        }
    }
    if (j->g_mv) cudaGraphExecDestroy(j->g_mv);
    if (j->g_pc) cudaGraphExecDestroy(j->g_pc);
    j->g_mv = j->g_pc = nullptr;
    if (j->pl) phs_plan_destroy(j->pl);
    j->pl = nullptr;
    if (j->dbuf) cudaFreeAsync(j->dbuf, j->s);
    if (j->s) cudaStreamSynchronize(j->s);
    if (j->ev) cudaEventDestroy(j->ev);
    if (j->s) cudaStreamDestroy(j->s);
    j->dbuf = nullptr;
    j->s = nullptr;
    j->ev = nullptr;
    std::vector<double>().swap(j->pts);
    std::vector<double>().swap(j->f);
    std::vector<double>().swap(j->tgt);
    std::lock_guard<std::mutex> g(mu);
    reserved -= j->reserved;
    j->reserved = 0;
    j->t_done = now_s(t0);
    j->info.ms_fit = (float)((j->t_done - j->t_ready) * 1e3);
    j->state = J_DONE;
    --n_finish;
    ++completed;
    cv_done.notify_all();
    cv_sched.notify_one();
}

void phs_server::worker_loop() {
    cudaSetDevice(dev);
    for (;;) {
        Job *j = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop_workers || !work.empty(); });
            if (work.empty()) return;  // stop_workers: the scheduler has exited, nothing more comes
            j = work.front();
            work.pop_front();
        }
        if (j->state == J_SETUP) setup(j);
        else if (j->state == J_REFINE) refine(j);
        else finish(j);
    }
}

// One PCG iteration of every active job (phs_fit's loop body, the vector steps shared).
void phs_server::tick(std::vector<Job *> &act) {
    const int nj = (int)act.size();
    BatchTable t;
    t.nj = nj;
    for (int i = 0; i < nj; ++i) t.j[i] = bjob_of(act[i]->pl, act[i]->rhs_p, act[i]->x_p);
    cudaEvent_t ev_e = ev_get();
    PHS_CUDA(cudaEventRecord(ev_e, engine));
    for (Job *j : act) {  // y = M' p on each job's stream
        phs_plan *pl = j->pl;
        AllocScope scope(j->s, &pl->dev_bytes);
        PHS_CUDA(cudaStreamWaitEvent(j->s, ev_e, 0));
        if (j->g_mv) {
            PHS_CUDA(cudaGraphLaunch(j->g_mv, j->s));
            count_launches(j->n_mv_kernels);
        } else {
            matvec_norm(pl, W(pl, 2), W(pl, 4), j->mv_prec, j->s);
        }
        PHS_CUDA(cudaEventRecord(j->ev, j->s));
        PHS_CUDA(cudaStreamWaitEvent(engine, j->ev, 0));
    }
    batch_matvec_update(t, engine);
    batch_gather(t, 2, rr_dev, engine);
    PHS_CUDA(cudaMemcpyAsync(rr_host, rr_dev, nj * sizeof(double), cudaMemcpyDeviceToHost, engine));
    PHS_CUDA(cudaStreamSynchronize(engine));
    ++ticks;
    batched_jobs += nj;
    std::vector<Job *> cont, done;
    for (int i = 0; i < nj; ++i) {
        Job *j = act[i];
        j->rr = rr_host[i];
        ++j->it;
        if (solve_ended(j)) {
            if (fit_precision(j->pl) == 0 && std::sqrt(j->rr) <= j->itol) j->converged = true;
            done.push_back(j);
        } else {
            cont.push_back(j);
        }
    }
    if (!cont.empty()) {
        BatchTable t2;
        t2.nj = (int)cont.size();
        for (int i = 0; i < t2.nj; ++i) t2.j[i] = bjob_of(cont[i]->pl, cont[i]->rhs_p, cont[i]->x_p);
        PHS_CUDA(cudaEventRecord(ev_e, engine));
        for (Job *j : cont) {  // t2 = S~^-1 r on each job's stream
            phs_plan *pl = j->pl;
            AllocScope scope(j->s, &pl->dev_bytes);
            PHS_CUDA(cudaStreamWaitEvent(j->s, ev_e, 0));
            if (j->g_pc) {
                PHS_CUDA(cudaGraphLaunch(j->g_pc, j->s));
                count_launches(j->n_pc_kernels);
            } else {
                vecchia_apply(pl->vec, W(pl, 0), W(pl, 5), W(pl, 6), j->s);
            }
            PHS_CUDA(cudaEventRecord(j->ev, j->s));
            PHS_CUDA(cudaStreamWaitEvent(engine, j->ev, 0));
        }
        batch_zproj(t2, engine);
        batch_pupdate(t2, engine);
    }
    // the jobs' streams must see the engine's last steps before their next work
    PHS_CUDA(cudaEventRecord(ev_e, engine));
    for (Job *j : act) PHS_CUDA(cudaStreamWaitEvent(j->s, ev_e, 0));
    ev_put(ev_e);
    std::lock_guard<std::mutex> g(mu);
    for (Job *j : done) {
        j->state = fit_precision(j->pl) == 0 ? J_FINISH : J_REFINE;
        act.erase(std::find(act.begin(), act.end(), j));
        ++n_finish;
        work.push_back(j);
        cv_work.notify_one();
    }
}

void phs_server::sched_loop() {
    cudaSetDevice(dev);
    for (;;) {
        std::vector<Job *> act;
        {
            std::unique_lock<std::mutex> lk(mu);
            // admission: slots and the memory budget (a job larger than the budget still
            // runs, alone)
            for (;;) {
                if (pending.empty()) break;
                const int in_flight = (int)active.size() + n_setup;
                if (in_flight >= max_active) break;
                Job *j = pending.front();
                if (reserved + j->reserved > budget && (in_flight + n_finish) > 0) break;
                pending.pop_front();
                reserved += j->reserved;
                max_reserved = std::max(max_reserved, reserved);
                j->state = J_SETUP;
                j->t_admit = now_s(t0);
                ++n_setup;
                work.push_back(j);
                cv_work.notify_one();
            }
            if (active.empty()) {
                if (stop && pending.empty() && n_setup == 0 && n_finish == 0 && work.empty()) return;
                cv_sched.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
            max_concurrent = std::max<int64_t>(max_concurrent, (int64_t)active.size());
            act.swap(active);
        }
        // at most kMaxBatch jobs per table
        std::vector<Job *> rest;
        if ((int)act.size() > kMaxBatch) {
            rest.assign(act.begin() + kMaxBatch, act.end());
            act.resize(kMaxBatch);
        }
        try {
            tick(act);
        } catch (const Error &e) {
            std::lock_guard<std::mutex> g(mu);
            for (Job *j : act) {
                j->status = e.code;
                j->err = e.msg;
                j->state = J_FINISH;
                ++n_finish;
                work.push_back(j);
            }
            act.clear();
            cv_work.notify_all();
        }
        std::lock_guard<std::mutex> g(mu);
        for (Job *j : act) active.push_back(j);
        for (Job *j : rest) active.push_back(j);
    }
}

extern "C" {

phs_status phs_server_create(const phs_server_config *cfg, phs_server_t *out) {
    PHS_TRY
    PHS_REQUIRE(out, PHS_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    phs_server_config c{};
    if (cfg) c = *cfg;
    const int max_active = c.max_active > 0 ? c.max_active : 32;
    const int threads = c.setup_threads > 0 ? c.setup_threads : 4;
    PHS_REQUIRE(max_active <= kMaxBatch, PHS_ERR_INVALID_ARG, "max_active must be at most 96");
    PHS_REQUIRE(threads <= 64, PHS_ERR_INVALID_ARG, "setup_threads must be at most 64");
    std::unique_ptr<phs_server> sv(new phs_server());
    PHS_CUDA(cudaGetDevice(&sv->dev));
    size_t fre = 0, tot = 0;
    PHS_CUDA(cudaMemGetInfo(&fre, &tot));
    sv->budget = c.memory_budget > 0 ? c.memory_budget : (int64_t)(fre / 2);
    sv->max_active = max_active;
    PHS_CUDA(cudaStreamCreateWithFlags(&sv->engine, cudaStreamNonBlocking));
    PHS_CUDA(cudaMalloc((void **)&sv->rr_dev, kMaxBatch * sizeof(double)));
    PHS_CUDA(cudaMallocHost((void **)&sv->rr_host, kMaxBatch * sizeof(double)));
    phs_server *p = sv.get();
    for (int i = 0; i < threads; ++i) sv->workers.emplace_back([p] { p->worker_loop(); });
    sv->sched = std::thread([p] { p->sched_loop(); });
    *out = sv.release();
    PHS_CATCH
}

phs_status phs_server_submit(phs_server_t sv, const double *pts_host, const double *f_host, int64_t n,
                             const double *tgt_host, int64_t m, int k, int poly_degree, int fmm_order, int vecchia_m,
                             const phs_options *opt, int64_t *job_id) {
    PHS_TRY
    PHS_REQUIRE(sv && pts_host && f_host && n > 0 && m >= 0 && (tgt_host || m == 0) && job_id, PHS_ERR_INVALID_ARG,
                "bad arguments");
    PHS_REQUIRE(k >= 1 && k <= 5 && vecchia_m >= 1 && vecchia_m <= 64, PHS_ERR_INVALID_ARG, "bad k or vecchia_m");
    std::unique_ptr<Job> j(new Job());
    j->k = k;
    j->deg = poly_degree;
    j->fmm_order = fmm_order;
    j->vm = vecchia_m;
    if (opt) j->opt = *opt;
    else phs_options_default(&j->opt, k);
    PHS_REQUIRE(j->opt.precision >= 0 && j->opt.precision <= 4, PHS_ERR_INVALID_ARG, "precision must be 0..4");
    PHS_REQUIRE(k % 2 == 0 || j->opt.precision == 0 || j->opt.precision == 4, PHS_ERR_INVALID_ARG,
                "odd spline orders run in precision 0 or 4");
    j->n = n;
    j->m = m;
    j->pts.assign(pts_host, pts_host + 2 * n);
    j->f.assign(f_host, f_host + n);
    if (m) j->tgt.assign(tgt_host, tgt_host + 2 * m);
    j->reserved = estimate_bytes(n, m, vecchia_m);
    std::lock_guard<std::mutex> g(sv->mu);
    PHS_REQUIRE(!sv->stop, PHS_ERR_INVALID_ARG, "server is shutting down");
    j->id = sv->next_id++;
    j->t_submit = now_s(sv->t0);
    *job_id = j->id;
    sv->pending.push_back(j.get());
    sv->jobs[j->id] = std::move(j);
    sv->cv_sched.notify_one();
    PHS_CATCH
}

phs_status phs_server_wait(phs_server_t sv, int64_t job_id, double *w_host, double *beta_host, double *pred_host,
                           phs_fit_info *info, double *times_host) {
    PHS_TRY
    PHS_REQUIRE(sv, PHS_ERR_INVALID_ARG, "null server");
    std::unique_ptr<Job> j;
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        auto it = sv->jobs.find(job_id);
        PHS_REQUIRE(it != sv->jobs.end(), PHS_ERR_INVALID_ARG, "unknown job id (or already collected)");
        Job *jp = it->second.get();
        sv->cv_done.wait(lk, [&] { return jp->state == J_DONE; });
        j = std::move(it->second);
        sv->jobs.erase(it);
    }
    if (w_host && !j->w.empty()) std::copy(j->w.begin(), j->w.end(), w_host);
    if (beta_host && !j->beta.empty()) std::copy(j->beta.begin(), j->beta.end(), beta_host);
    if (pred_host && !j->pred.empty()) std::copy(j->pred.begin(), j->pred.end(), pred_host);
    if (info) *info = j->info;
    if (times_host) {
        times_host[0] = j->t_submit;
        times_host[1] = j->t_admit;
        times_host[2] = j->t_ready;
        times_host[3] = j->t_done;
    }
    if (j->status != PHS_OK) throw Error{j->status, j->err};
    PHS_CATCH
}

phs_status phs_server_stats(phs_server_t sv, int64_t *stats_host) {
    PHS_TRY
    PHS_REQUIRE(sv && stats_host, PHS_ERR_INVALID_ARG, "bad arguments");
    std::lock_guard<std::mutex> g(sv->mu);
    stats_host[0] = sv->ticks;
    stats_host[1] = sv->batched_jobs;
    stats_host[2] = sv->max_concurrent;
    stats_host[3] = sv->max_reserved;
    stats_host[4] = sv->budget;
    stats_host[5] = sv->completed;
    stats_host[6] = (int64_t)sv->pending.size();
    stats_host[7] = sv->reserved;
    PHS_CATCH
}

phs_status phs_server_destroy(phs_server_t sv) {
    PHS_TRY
    if (!sv) return PHS_OK;
    {
        std::lock_guard<std::mutex> g(sv->mu);
        sv->stop = true;
    }
    sv->cv_sched.notify_all();
    if (sv->sched.joinable()) sv->sched.join();
    {
        std::lock_guard<std::mutex> g(sv->mu);
        sv->stop_workers = true;
        sv->cv_work.notify_all();
    }
    for (auto &t : sv->workers)
        if (t.joinable()) t.join();
    if (sv->engine) cudaStreamDestroy(sv->engine);
    if (sv->rr_dev) cudaFree(sv->rr_dev);
    if (sv->rr_host) cudaFreeHost(sv->rr_host);
    delete sv;
    PHS_CATCH
}

}  // extern "C"
