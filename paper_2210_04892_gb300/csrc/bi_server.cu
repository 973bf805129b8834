// Continuous-batching solve server.  A request is a surface, a wavenumber, nrhs plane waves and
// a tolerance.  Requests on the same operator (identical surface, wavenumber and parameters)
// share one set-up operator, kept in a cache after its requests finish, and are merged into
// one job: one resumable GMRES context over the columns of all of them, so every product of
// the job is one batched bi_matvec -- one launch per kernel of the product for all its
// requests.  A job takes every waiting request of its operator (up to max_batch_rhs columns),
// including those that arrive while the operator is being set up.  Jobs are admitted as device
// memory and slots allow; setup threads build operators and GMRES contexts (and tune the
// kernel forms for the job's column count) so that set-ups overlap running solves, and the serving thread advances every running job by one iteration
// per pass (their products are queued on their own streams and overlap on the device),
// retires finished jobs and admits waiting requests between passes.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <exception>
#include <list>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>

#include "bi_internal.h"

namespace {

using clk = std::chrono::steady_clock;

enum req_state { RQ_QUEUED = 0, RQ_SETUP = 1, RQ_RUNNING = 2, RQ_DONE = 3 };
enum op_state { OP_BUILDING = 0, OP_IDLE = 1, OP_BUSY = 2 };

struct job;

struct request {
    int64_t id = 0;
    std::vector<double> verts;
    std::vector<int> tris;
    double k0 = 0;
    bi_params prm{};
    uint64_t key = 0;
    int nrhs = 1;
    std::vector<double> khat, phat;
    double tol = 1e-3;
    clk::time_point t_submit, t_done;
    std::atomic<int> state{RQ_QUEUED};
    int status = BI_OK;
    std::string err;
    job* jb = nullptr;
    int col0 = 0;                       // first column of this request in its job
    std::vector<unsigned char> x_host;  // result, handle precision
    std::vector<int> iters;
    std::vector<double> relres;
    double setup_ms = 0;                // operator set-up time, when this request's job built it
};

// One set-up operator and the identity it was built for.
struct op_entry {
    uint64_t key = 0;
    std::vector<double> verts;
    std::vector<int> tris;
    double k0 = 0;
    bi_params prm{};
    int max_rhs = 1;
    int state = OP_BUILDING;
    bi_handle_s* h = nullptr;
    cudaStream_t stream = nullptr;
    int64_t bytes = 0;                  // device bytes held (estimate until built)
    double setup_ms = 0;
    clk::time_point last_use;
};

struct job {
    op_entry* op = nullptr;
    std::vector<request*> reqs;
    bool sealed = false;                // columns fixed (no more requests join)
    bool builds_op = false;             // this job triggered the operator's set-up
    int R = 0;
    void* d_rhs = nullptr;
    void* d_x = nullptr;
    gmres_ctx* ctx = nullptr;
    int64_t est_bytes = 0, held_bytes = 0;
};

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

// Operator identity: the surface, the wavenumber and every parameter that changes the operator
// or its solver (stream and max_rhs excluded: the server sets them).
uint64_t operator_key(const request* r) {
    uint64_t h = 1469598103934665603ull;
    h = fnv1a(h, r->verts.data(), r->verts.size() * sizeof(double));
    h = fnv1a(h, r->tris.data(), r->tris.size() * sizeof(int));
    h = fnv1a(h, &r->k0, sizeof(double));
    const bi_params& p = r->prm;
    const double dv[] = {p.leaf_box, p.k_im, p.eps_re, p.eps_im};
    const int iv[] = {p.digits, p.levels, p.interp_order, p.precision, p.op_mode, p.gmres_restart, p.gmres_maxit,
                      p.precond, p.core_tris};
    h = fnv1a(h, dv, sizeof(dv));
    h = fnv1a(h, iv, sizeof(iv));
    return h;
}

bool same_operator(const op_entry* e, const request* r) {
    const bi_params &a = e->prm, &b = r->prm;
    return e->key == r->key && e->k0 == r->k0 && e->verts == r->verts && e->tris == r->tris &&
           a.leaf_box == b.leaf_box && a.digits == b.digits && a.levels == b.levels &&
           a.interp_order == b.interp_order && a.precision == b.precision && a.op_mode == b.op_mode &&
           a.gmres_restart == b.gmres_restart && a.gmres_maxit == b.gmres_maxit && a.precond == b.precond &&
           a.k_im == b.k_im && a.eps_re == b.eps_re && a.eps_im == b.eps_im && a.core_tris == b.core_tris &&
           r->nrhs <= e->max_rhs;
}

int64_t n_unknowns_of(const request* r) {
    const int64_t N = (int64_t)r->tris.size() / 3 * 3 / 2;
    return N * (r->prm.op_mode == 0 ? 2 : 1);
}

// Device bytes of an operator: near blocks (~420 near pairs per RWG at a 0.25-wavelength
// leaf), leaf patterns, far-field buffers and work vectors for max_rhs columns; a 1.5x margin
// covers the tree and scratch.
int64_t estimate_op_bytes(const request* r, int max_rhs) {
    const int64_t N = (int64_t)r->tris.size() / 3 * 3 / 2;
    const int nX = r->prm.op_mode == 0 ? 2 : 1;
    const int64_t cs = r->prm.precision == 0 ? 16 : 8;
    const int64_t near = N * 420 * cs * nX;
    const int64_t pat = N * 300 * 4 * cs;
    const int64_t far = N * 300 * 2 * (int64_t)max_rhs * cs * 2;
    return (near + pat + far + N * nX * max_rhs * cs * 4) * 3 / 2 + (64 << 20);
}

// Device bytes of a job's GMRES state and vectors for R columns.
int64_t estimate_job_bytes(const request* r, int R) {
    const int64_t nun = n_unknowns_of(r);
    const int64_t cs = r->prm.precision == 0 ? 16 : 8;
    return bi_gmres_estimate_bytes(nun, R, r->prm.gmres_restart) + 2 * nun * R * cs;
}

}  // namespace

struct bi_server_s {
    bi_server_params prm{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<request*> queue;          // waiting for a job
    std::deque<job*> to_setup;           // admitted, waiting for the setup worker
    std::vector<job*> pending;           // jobs whose columns are still open (setting up)
    std::vector<job*> running;           // iterating (serving thread only)
    std::deque<job*> ready;              // set up, waiting to join `running`
    std::list<op_entry*> ops;            // every operator, in order of last use (front: oldest)
    std::vector<op_entry*> retired;      // operators to destroy outside the lock (evicted or unshared)
    std::unordered_map<int64_t, request*> all;
    int64_t next_id = 1;
    int64_t held_bytes = 0;              // operators (cached or in use) plus jobs
    int active = 0;                      // jobs admitted and not finished
    bool stop = false;
    std::thread serve_thread;
    std::vector<std::thread> setup_threads;
    std::string err;
    int64_t stats[BI_SERVER_NSTATS] = {};
};

namespace {

void destroy_op(op_entry* e) {
    if (e->h) bi_destroy(e->h);
    if (e->stream) cudaStreamDestroy(e->stream);
    delete e;
}

// Drop idle cached operators, oldest first, until `need` more bytes fit the budget.  Their
// device memory is released by destroy_retired, outside the lock (freeing synchronises the
// device, which must not hold up bi_submit and bi_poll).
void evict_locked(bi_server_s* S, int64_t need) {
    for (auto it = S->ops.begin(); it != S->ops.end() && S->held_bytes + need > S->prm.mem_budget_bytes;) {
        op_entry* e = *it;
        if (e->state == OP_IDLE) {
            S->held_bytes -= e->bytes;
            it = S->ops.erase(it);
            S->retired.push_back(e);
            S->stats[BI_STAT_EVICTIONS] += 1;
        } else {
            ++it;
        }
    }
}

// Destroy the operators retired under the lock (called without it).
void destroy_retired(bi_server_s* S) {
    std::vector<op_entry*> dead;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        dead.swap(S->retired);
    }
    for (op_entry* e : dead) destroy_op(e);
}

// Finish every request of a job with the same status; frees the job and releases its operator
// (destroyed when operators are not shared, or when it failed to build).
void finish_job(bi_server_s* S, job* jb, int code, const std::string& msg) {
    if (jb->ctx) bi_gmres_destroy(jb->ctx);
    cudaStream_t st = jb->op ? jb->op->stream : nullptr;
    if (jb->d_rhs) cudaFreeAsync(jb->d_rhs, st);
    if (jb->d_x) cudaFreeAsync(jb->d_x, st);
    std::lock_guard<std::mutex> lk(S->mu);
    const clk::time_point now = clk::now();
    for (request* r : jb->reqs) {
        if (code != BI_OK && r->status == BI_OK) {
            r->status = code;
            r->err = msg;
        }
        r->t_done = now;
        r->jb = nullptr;
        r->state = RQ_DONE;
    }
    S->held_bytes -= jb->held_bytes;
    S->active -= 1;
    op_entry* e = jb->op;
    if (e) {
        e->last_use = now;
        const bool keep = S->prm.share_operators && e->h && code != BI_ERR_CUDA;
        if (keep) {
            e->state = OP_IDLE;
            S->ops.remove(e);
            S->ops.push_back(e);
        } else {
            S->held_bytes -= e->bytes;
            S->ops.remove(e);
            S->retired.push_back(e);
        }
    }
    for (auto it = S->pending.begin(); it != S->pending.end(); ++it)
        if (*it == jb) {
            S->pending.erase(it);
            break;
        }
    delete jb;
    S->cv.notify_all();
}

// Admit waiting requests in arrival order.  A request joins the open job of its operator
// when one is setting up and has room; else it starts a job on its idle cached operator; else
// it starts a job that builds a new operator; a request whose operator is busy with a job
// that no longer takes columns waits for that job to finish.
void admit_locked(bi_server_s* S) {
    const int cap = std::max(1, S->prm.max_batch_rhs);
    for (auto it = S->queue.begin(); it != S->queue.end();) {
        request* r = *it;
        op_entry* e = nullptr;
        if (S->prm.share_operators)
            for (op_entry* o : S->ops)
                if (same_operator(o, r)) {
                    e = o;
                    break;
                }
        if (e && e->state == OP_BUSY) {
            job* open = nullptr;
            for (job* jb : S->pending)
                if (jb->op == e && !jb->sealed) open = jb;
            int cols = 0;
            if (open)
                for (request* q : open->reqs) cols += q->nrhs;
            if (open && cols + r->nrhs <= cap) {
                const int64_t more = estimate_job_bytes(r, cols + r->nrhs) - open->est_bytes;
                if (S->held_bytes + more <= S->prm.mem_budget_bytes) {
                    open->reqs.push_back(r);
                    open->est_bytes += more;
                    open->held_bytes += more;
                    S->held_bytes += more;
                    r->jb = open;
                    r->state = RQ_SETUP;
                    S->stats[BI_STAT_MERGED_REQUESTS] += 1;
                    it = S->queue.erase(it);
                    continue;
                }
            }
            ++it;   // waits for the operator's current job
            continue;
        }
        // no free job slot: later requests may still join open jobs of their operators
        if (S->active >= S->prm.max_active) {
            ++it;
            continue;
        }
        const int max_rhs = std::max(cap, r->nrhs);
        const int64_t op_bytes = e ? 0 : estimate_op_bytes(r, max_rhs);
        const int64_t jb_bytes = estimate_job_bytes(r, r->nrhs);
        if (e) e->state = OP_BUSY;      // not evictable while this request may use it
        if (S->held_bytes + op_bytes + jb_bytes > S->prm.mem_budget_bytes) evict_locked(S, op_bytes + jb_bytes);
        if (S->held_bytes + op_bytes + jb_bytes > S->prm.mem_budget_bytes && S->active > 0) {
            if (e) e->state = OP_IDLE;
            break;
        }
        job* jb = new job();
        if (!e) {
            e = new op_entry();
            e->key = r->key;
            e->verts = r->verts;
            e->tris = r->tris;
            e->k0 = r->k0;
            e->prm = r->prm;
            e->max_rhs = max_rhs;
            e->bytes = op_bytes;
            S->held_bytes += op_bytes;
            S->ops.push_back(e);
            jb->builds_op = true;
            S->stats[BI_STAT_OPERATORS_BUILT] += 1;
        } else {
            S->stats[BI_STAT_CACHE_HITS] += 1;
        }
        e->state = OP_BUSY;
        jb->op = e;
        jb->reqs.push_back(r);
        jb->est_bytes = jb->held_bytes = jb_bytes;
        S->held_bytes += jb_bytes;
        S->active += 1;
        S->stats[BI_STAT_JOBS] += 1;
        r->jb = jb;
        r->state = RQ_SETUP;
        S->pending.push_back(jb);
        S->to_setup.push_back(jb);
        it = S->queue.erase(it);
        S->cv.notify_all();
    }
}

// Build the job's operator if needed, then close its columns and create its right-hand sides
// and GMRES context (setup thread).
void setup_job(bi_server_s* S, job* jb) {
    op_entry* e = jb->op;
    if (jb->builds_op) {
        CU(cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking));
        bi_params p = e->prm;
        p.stream = e->stream;
        p.max_rhs = e->max_rhs;
        bi_handle h = nullptr;
        const int rc = bi_setup(e->verts.data(), (int)e->verts.size() / 3, e->tris.data(), (int)e->tris.size() / 3,
                                e->k0, 0, &p, &h);
        if (rc != BI_OK) throw bi_error{rc, std::string("setup: ") + bi_last_error(nullptr)};
        e->h = h;
        bi_info_t inf;
        bi_get_info(h, &inf);
        e->setup_ms = inf.setup_ms;
        std::lock_guard<std::mutex> lk(S->mu);
        S->held_bytes += inf.device_bytes - e->bytes;
        e->bytes = inf.device_bytes;
    }
    std::vector<request*> reqs;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        jb->sealed = true;
        reqs = jb->reqs;
    }
    bi_handle_s* h = e->h;
    int R = 0;
    for (request* r : reqs) {
        r->col0 = R;
        R += r->nrhs;
    }
    jb->R = R;
    const size_t vb = (size_t)h->nun * R * h->csize;
    // stream-ordered: allocating and freeing a job's vectors (and its GMRES state) does not
    // synchronise the device while other jobs run
    CU(cudaMallocAsync(&jb->d_rhs, vb, e->stream));
    CU(cudaMallocAsync(&jb->d_x, vb, e->stream));
    std::vector<double> tolv;
    for (request* r : reqs) {
        const int rc = bi_rhs_planewave(h, r->khat.data(), r->phat.data(), r->nrhs,
                                        (char*)jb->d_rhs + (size_t)r->col0 * h->nun * h->csize);
        if (rc != BI_OK) throw bi_error{rc, bi_last_error(h)};
        tolv.insert(tolv.end(), r->nrhs, r->tol);
        r->setup_ms = jb->builds_op ? e->setup_ms : 0.0;
    }
    jb->ctx = bi_gmres_create(h, jb->d_rhs, R, tolv.data(), e->stream);
    // tune the level passes for this column count here, off the serving thread (the first
    // product of a new column count would otherwise time every kernel form while the other
    // jobs wait)
    if (h->use_fast) bi_autotune(h, R, e->stream);
    CU(cudaStreamSynchronize(e->stream));
    const int64_t actual = bi_gmres_bytes(jb->ctx) + 2 * (int64_t)vb;
    std::lock_guard<std::mutex> lk(S->mu);
    S->held_bytes += actual - jb->held_bytes;
    jb->held_bytes = actual;
    for (request* r : reqs) r->state = RQ_RUNNING;
    S->ready.push_back(jb);
}

void setup_worker(bi_server_s* S) {
    cudaSetDevice(S->device);
    for (;;) {
        job* jb = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return S->stop || !S->to_setup.empty(); });
            if (S->stop) return;
            jb = S->to_setup.front();
            S->to_setup.pop_front();
        }
        try {
            setup_job(S, jb);
            S->cv.notify_all();
        } catch (const bi_error& e) {
            {
                std::lock_guard<std::mutex> lk(S->mu);
                jb->sealed = true;
            }
            finish_job(S, jb, e.code, e.msg);
        } catch (const std::exception& e) {
            // host allocation failure: fail this job, keep the worker alive
            {
                std::lock_guard<std::mutex> lk(S->mu);
                jb->sealed = true;
            }
            finish_job(S, jb, BI_ERR_OOM, std::string("setup: ") + e.what());
        }
    }
}

// Results of a finished job, split into its requests.
void retire_job(bi_server_s* S, job* jb) {
    bi_handle_s* h = jb->op->h;
    std::vector<int> its(jb->R, 0);
    std::vector<double> rel(jb->R, 0.0);
    const int st = bi_gmres_finish(jb->ctx, jb->d_x, its.data(), rel.data());
    const size_t col = (size_t)h->nun * h->csize;
    for (request* r : jb->reqs) {
        r->x_host.resize(col * r->nrhs);
        CU(cudaMemcpy(r->x_host.data(), (const char*)jb->d_x + col * r->col0, col * r->nrhs, cudaMemcpyDeviceToHost));
        r->iters.assign(its.begin() + r->col0, its.begin() + r->col0 + r->nrhs);
        r->relres.assign(rel.begin() + r->col0, rel.begin() + r->col0 + r->nrhs);
        r->status = BI_OK;
        for (int c = 0; c < r->nrhs; ++c)
            if (r->relres[c] > r->tol * 1.0001 + 1e-12) r->status = BI_ERR_NOT_CONVERGED;
        if (st != BI_OK && st != BI_ERR_NOT_CONVERGED) r->status = st;
        if (r->status == BI_ERR_NOT_CONVERGED) r->err = "GMRES did not reach tol";
    }
    finish_job(S, jb, BI_OK, "");
}

void serve_loop(bi_server_s* S) {
    cudaSetDevice(S->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            admit_locked(S);
            if (S->running.empty() && S->ready.empty())
                S->cv.wait_for(lk, std::chrono::milliseconds(2),
                               [&] { return S->stop || !S->ready.empty() || !S->queue.empty(); });
            if (S->stop) return;
            while (!S->ready.empty()) {
                S->running.push_back(S->ready.front());
                S->ready.pop_front();
            }
        }
        destroy_retired(S);
        // one pass: every running job advances as far as its completed work allows
        for (size_t i = 0; i < S->running.size();) {
            job* jb = S->running[i];
            try {
                if (bi_gmres_advance(jb->ctx)) {
                    S->running.erase(S->running.begin() + i);
                    retire_job(S, jb);
                    continue;
                }
            } catch (const bi_error& e) {
                S->running.erase(S->running.begin() + i);
                finish_job(S, jb, e.code, e.msg);
                continue;
            } catch (const std::exception& e) {
                S->running.erase(S->running.begin() + i);
                finish_job(S, jb, BI_ERR_OOM, std::string("solve: ") + e.what());
                continue;
            }
            ++i;
        }
        if (!S->running.empty()) std::this_thread::yield();
    }
}

}  // namespace

extern "C" void bi_server_default_params(bi_server_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->mem_budget_bytes = 0;
    p->max_active = 8;
    p->queue_capacity = 4096;
    p->share_operators = 1;
    p->max_batch_rhs = 64;
    p->setup_threads = 2;
}

extern "C" int bi_server_create(const bi_server_params* prm, bi_server* out) {
    if (!out) return BI_ERR_ARG;
    *out = nullptr;
    bi_server_s* S = new (std::nothrow) bi_server_s();
    if (!S) return BI_ERR_OOM;
    if (prm) S->prm = *prm;
    else bi_server_default_params(&S->prm);
    if (S->prm.max_active < 1 || S->prm.queue_capacity < 1 || S->prm.mem_budget_bytes < 0 ||
        S->prm.max_batch_rhs < 1 || (S->prm.share_operators != 0 && S->prm.share_operators != 1) ||
        S->prm.setup_threads < 1 || S->prm.setup_threads > 16) {
        delete S;
        return BI_ERR_ARG;
    }
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return BI_ERR_CUDA;
    }
    {
        // keep stream-ordered memory that jobs free in the device's pool (no unmap and remap
        // of every job's GMRES state at the next synchronisation); process-local pool setting
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, S->device) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    }
    if (S->prm.mem_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            delete S;
            return BI_ERR_CUDA;
        }
        S->prm.mem_budget_bytes = (int64_t)(fr * 0.8);
    }
    try {
        for (int i = 0; i < S->prm.setup_threads; ++i) S->setup_threads.emplace_back(setup_worker, S);
        S->serve_thread = std::thread(serve_loop, S);
    } catch (const std::exception&) {
        // a thread could not be started: stop those that started, then give up
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop = true;
        }
        S->cv.notify_all();
        for (std::thread& t : S->setup_threads)
            if (t.joinable()) t.join();
        if (S->serve_thread.joinable()) S->serve_thread.join();
        delete S;
        return BI_ERR_OOM;
    }
    *out = S;
    return BI_OK;
}

extern "C" int bi_submit(bi_server S, const double* verts, int nv, const int* tris, int nt, double k0,
                         const bi_params* opt, int nrhs, const double* khat, const double* phat, double tol,
                         int64_t* req) {
    if (!S || !verts || !tris || nv < 3 || nt < 4 || !(k0 > 0) || nrhs < 1 || !khat || !phat || !(tol > 0) || !req)
        return BI_ERR_ARG;
    if (opt && (opt->k_im != 0.0 || opt->op_mode > 1)) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->err = "bi_submit: requests are free-space C-block or PEC operators (k_im = 0, op_mode 0 or 1)";
        return BI_ERR_ARG;
    }
    std::unique_ptr<request> r;
    try {
        r.reset(new request());
        r->verts.assign(verts, verts + 3 * (size_t)nv);
        r->tris.assign(tris, tris + 3 * (size_t)nt);
        r->khat.assign(khat, khat + 3 * (size_t)nrhs);
        r->phat.assign(phat, phat + 3 * (size_t)nrhs);
    } catch (const std::exception&) {
        return BI_ERR_OOM;              // the copies of the inputs did not fit in host memory
    }
    r->k0 = k0;
    if (opt) r->prm = *opt;
    else bi_default_params(&r->prm);
    r->prm.stream = nullptr;
    r->nrhs = nrhs;
    r->tol = tol;
    r->key = operator_key(r.get());
    r->t_submit = clk::now();
    const int64_t need = estimate_op_bytes(r.get(), std::max(S->prm.max_batch_rhs, nrhs)) +
                         estimate_job_bytes(r.get(), nrhs);
    std::lock_guard<std::mutex> lk(S->mu);
    if ((int)S->queue.size() >= S->prm.queue_capacity) return BI_ERR_BUSY;
    if (need > S->prm.mem_budget_bytes) {
        S->err = "bi_submit: request needs more device memory than the whole budget";
        return BI_ERR_OOM;
    }
    const int64_t id = S->next_id;
    try {
        S->all[id] = r.get();
        S->queue.push_back(r.get());
    } catch (const std::exception&) {
        S->all.erase(id);
        return BI_ERR_OOM;
    }
    S->next_id += 1;
    r->id = id;
    *req = id;
    r.release();                        // owned by S->all from here on
    S->cv.notify_all();
    return BI_OK;
}

extern "C" int bi_poll(bi_server S, int64_t req, int* done, int* status) {
    if (!S) return BI_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(req);
    if (it == S->all.end()) return BI_ERR_ARG;
    const bool d = it->second->state.load() == RQ_DONE;
    if (done) *done = d ? 1 : 0;
    if (status) *status = d ? it->second->status : BI_OK;
    return BI_OK;
}

extern "C" int bi_result(bi_server S, int64_t req, void* x_host, int64_t x_bytes, int* iters, double* relres,
                         double* latency_ms, double* setup_ms) {
    if (!S) return BI_ERR_ARG;
    request* r = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->all.find(req);
        if (it == S->all.end()) return BI_ERR_ARG;
        r = it->second;
    }
    if (r->state.load() != RQ_DONE) return BI_ERR_BUSY;
    if (x_host) {
        if ((int64_t)r->x_host.size() > x_bytes) return BI_ERR_ARG;
        std::memcpy(x_host, r->x_host.data(), r->x_host.size());
    }
    for (int i = 0; i < r->nrhs && i < (int)r->iters.size(); ++i) {
        if (iters) iters[i] = r->iters[i];
        if (relres) relres[i] = r->relres[i];
    }
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    if (setup_ms) *setup_ms = r->setup_ms;
    return r->status;
}

extern "C" int bi_server_stats(bi_server S, int64_t* out, int n) {
    if (!S || !out || n < 1) return BI_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    int64_t cached = 0;
    for (op_entry* e : S->ops) cached += e->state == OP_IDLE;
    int64_t v[BI_SERVER_NSTATS];
    std::memcpy(v, S->stats, sizeof(v));
    v[BI_STAT_CACHED_OPERATORS] = cached;
    v[BI_STAT_HELD_BYTES] = S->held_bytes;
    for (int i = 0; i < n && i < BI_SERVER_NSTATS; ++i) out[i] = v[i];
    return BI_OK;
}

extern "C" int bi_release(bi_server S, int64_t req) {
    if (!S) return BI_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(req);
    if (it == S->all.end() || it->second->state.load() != RQ_DONE) return BI_ERR_ARG;
    delete it->second;
    S->all.erase(it);
    return BI_OK;
}

extern "C" const char* bi_server_last_error(bi_server S) { return S ? S->err.c_str() : ""; }

extern "C" void bi_server_destroy(bi_server S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->serve_thread.joinable()) S->serve_thread.join();
    for (std::thread& t : S->setup_threads)
        if (t.joinable()) t.join();
    cudaSetDevice(S->device);
    // jobs still set up or running; the threads are gone, so nothing else touches them
    std::vector<job*> jobs(S->running.begin(), S->running.end());
    jobs.insert(jobs.end(), S->ready.begin(), S->ready.end());
    jobs.insert(jobs.end(), S->to_setup.begin(), S->to_setup.end());
    for (job* jb : jobs) {
        if (jb->ctx) bi_gmres_destroy(jb->ctx);
        cudaStream_t st = jb->op ? jb->op->stream : nullptr;
        if (jb->d_rhs) cudaFreeAsync(jb->d_rhs, st);
        if (jb->d_x) cudaFreeAsync(jb->d_x, st);
        delete jb;
    }
    cudaDeviceSynchronize();
    for (op_entry* e : S->ops) destroy_op(e);
    for (op_entry* e : S->retired) destroy_op(e);
    for (auto& kv : S->all) delete kv.second;
    delete S;
}
