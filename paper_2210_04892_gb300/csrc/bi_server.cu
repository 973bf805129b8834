// Continuous-batching solve server: requests (mesh, wavenumber, plane-wave excitations,
// tolerance) are admitted as device memory and slots allow; each admitted request gets its
// own stream, operator (bi_setup, on a setup worker thread so that setups overlap the
// iterations of running solves) and resumable GMRES context.  The serving thread advances
// every running solve by one iteration per pass -- their matvec graphs and Krylov kernels
// are queued on their own streams and overlap on the device -- retires finished requests
// and admits waiting ones between passes.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <exception>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>

#include "bi_internal.h"

namespace {

using clk = std::chrono::steady_clock;

enum req_state { RQ_QUEUED = 0, RQ_SETUP = 1, RQ_RUNNING = 2, RQ_DONE = 3 };

struct request {
    int64_t id = 0;
    std::vector<double> verts;
    std::vector<int> tris;
    double k0 = 0;
    bi_params prm{};
    int nrhs = 1;
    std::vector<double> khat, phat;
    double tol = 1e-3;
    int64_t est_bytes = 0, held_bytes = 0;
    clk::time_point t_submit, t_start, t_done;
    std::atomic<int> state{RQ_QUEUED};
    int status = BI_OK;
    std::string err;
    cudaStream_t stream = nullptr;
    bi_handle_s* op = nullptr;
    void* d_rhs = nullptr;
    void* d_x = nullptr;
    gmres_ctx* ctx = nullptr;
    std::vector<unsigned char> x_host;  // result, handle precision
    std::vector<int> iters;
    std::vector<double> relres;
    double setup_ms = 0;
};

}  // namespace

struct bi_server_s {
    bi_server_params prm{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<request*> queue;          // waiting for admission
    std::deque<request*> to_setup;       // admitted, waiting for the setup worker
    std::vector<request*> running;       // set up, iterating (serving thread only)
    std::deque<request*> ready;          // set up, waiting to join `running`
    std::unordered_map<int64_t, request*> all;
    int64_t next_id = 1;
    int64_t held_bytes = 0;
    int active = 0;                      // admitted and not finished
    bool stop = false;
    std::thread serve_thread, setup_thread;
    std::string err;
};

static int64_t estimate_request_bytes(const request* r) {
    // near blocks (~400 near pairs per RWG at a 0.25-wavelength leaf), patterns, far-field
    // buffers and the Krylov basis; a 1.5x margin covers the tree and scratch
    const int64_t nt = (int64_t)r->tris.size() / 3;
    const int64_t N = nt * 3 / 2;
    const int nX = r->prm.op_mode == 0 ? 2 : 1;
    const int64_t cs = r->prm.precision == 0 ? 16 : 8;
    const int64_t nun = N * nX;
    const int64_t near = N * 420 * cs * nX;
    const int64_t pat = N * 300 * 4 * cs;
    const int64_t far = N * 300 * 2 * r->nrhs * cs * 2;
    const int64_t kry = bi_gmres_estimate_bytes(nun, r->nrhs, r->prm.gmres_restart);
    return (near + pat + far + kry + nun * r->nrhs * cs * 6) * 3 / 2 + (64 << 20);
}

static void fail_request(bi_server_s* S, request* r, int code, const std::string& msg) {
    r->status = code;
    r->err = msg;
    r->t_done = clk::now();
    if (r->ctx) { bi_gmres_destroy(r->ctx); r->ctx = nullptr; }
    if (r->op) { bi_destroy(r->op); r->op = nullptr; }
    if (r->d_rhs) { cudaFree(r->d_rhs); r->d_rhs = nullptr; }
    if (r->d_x) { cudaFree(r->d_x); r->d_x = nullptr; }
    if (r->stream) { cudaStreamDestroy(r->stream); r->stream = nullptr; }
    std::lock_guard<std::mutex> lk(S->mu);
    S->held_bytes -= r->held_bytes;
    r->held_bytes = 0;
    S->active -= 1;
    r->state = RQ_DONE;
    S->cv.notify_all();
}

// admit queued requests in arrival order while slots and the memory budget allow
static void admit_locked(bi_server_s* S) {
    while (!S->queue.empty() && S->active < S->prm.max_active) {
        request* r = S->queue.front();
        if (S->held_bytes + r->est_bytes > S->prm.mem_budget_bytes && S->active > 0) break;
        S->queue.pop_front();
        r->held_bytes = r->est_bytes;
        S->held_bytes += r->held_bytes;
        S->active += 1;
        r->state = RQ_SETUP;
        S->to_setup.push_back(r);
        S->cv.notify_all();
    }
}

static void setup_worker(bi_server_s* S) {
    cudaSetDevice(S->device);
    for (;;) {
        request* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return S->stop || !S->to_setup.empty(); });
            if (S->stop) return;
            r = S->to_setup.front();
            S->to_setup.pop_front();
        }
        r->t_start = clk::now();
        try {
            CU(cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking));
            bi_params p = r->prm;
            p.stream = r->stream;
            p.max_rhs = std::max(p.max_rhs, r->nrhs);
            bi_handle h = nullptr;
            int rc = bi_setup(r->verts.data(), (int)r->verts.size() / 3, r->tris.data(), (int)r->tris.size() / 3, r->k0,
                              0, &p, &h);
            if (rc != BI_OK) throw bi_error{rc, std::string("setup: ") + bi_last_error(nullptr)};
            r->op = h;
            bi_info_t inf;
            bi_get_info(h, &inf);
            r->setup_ms = inf.setup_ms;
            const size_t vb = (size_t)h->nun * r->nrhs * h->csize;
            CU(cudaMalloc(&r->d_rhs, vb));
            CU(cudaMalloc(&r->d_x, vb));
            rc = bi_rhs_planewave(h, r->khat.data(), r->phat.data(), r->nrhs, r->d_rhs);
            if (rc != BI_OK) throw bi_error{rc, bi_last_error(h)};
            r->ctx = bi_gmres_create(h, r->d_rhs, r->nrhs, r->tol, r->stream);
            const int64_t actual = inf.device_bytes + bi_gmres_bytes(r->ctx) + 2 * (int64_t)vb;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                S->held_bytes += actual - r->held_bytes;
                r->held_bytes = actual;
                r->state = RQ_RUNNING;
                S->ready.push_back(r);
            }
            S->cv.notify_all();
        } catch (const bi_error& e) {
            fail_request(S, r, e.code, e.msg);
        } catch (const std::exception& e) {
            // host allocation failure: fail this request, keep the worker alive
            fail_request(S, r, BI_ERR_OOM, std::string("setup: ") + e.what());
        }
    }
}

static void serve_loop(bi_server_s* S) {
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
        // one pass: every running solve advances as far as its completed work allows
        for (size_t i = 0; i < S->running.size();) {
            request* r = S->running[i];
            try {
                int fin = bi_gmres_advance(r->ctx);
                if (fin) {
                    r->iters.assign(r->nrhs, 0);
                    r->relres.assign(r->nrhs, 0.0);
                    int st = bi_gmres_finish(r->ctx, r->d_x, r->iters.data(), r->relres.data());
                    const size_t vb = (size_t)r->op->nun * r->nrhs * r->op->csize;
                    r->x_host.resize(vb);
                    CU(cudaMemcpy(r->x_host.data(), r->d_x, vb, cudaMemcpyDeviceToHost));
                    fail_request(S, r, st, st == BI_OK ? "" : "GMRES did not reach tol");
                    S->running.erase(S->running.begin() + i);
                    continue;
                }
            } catch (const bi_error& e) {
                fail_request(S, r, e.code, e.msg);
                S->running.erase(S->running.begin() + i);
                continue;
            } catch (const std::exception& e) {
                fail_request(S, r, BI_ERR_OOM, std::string("solve: ") + e.what());
                S->running.erase(S->running.begin() + i);
                continue;
            }
            ++i;
        }
        if (!S->running.empty()) std::this_thread::yield();
    }
}

extern "C" void bi_server_default_params(bi_server_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->mem_budget_bytes = 0;
    p->max_active = 8;
    p->queue_capacity = 4096;
}

extern "C" int bi_server_create(const bi_server_params* prm, bi_server* out) {
    if (!out) return BI_ERR_ARG;
    *out = nullptr;
    bi_server_s* S = new (std::nothrow) bi_server_s();
    if (!S) return BI_ERR_OOM;
    if (prm) S->prm = *prm;
    else bi_server_default_params(&S->prm);
    if (S->prm.max_active < 1 || S->prm.queue_capacity < 1 || S->prm.mem_budget_bytes < 0) {
        delete S;
        return BI_ERR_ARG;
    }
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return BI_ERR_CUDA;
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
        S->setup_thread = std::thread(setup_worker, S);
        S->serve_thread = std::thread(serve_loop, S);
    } catch (const std::exception&) {
        // a thread could not be started: stop the one that may have started, then give up
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop = true;
        }
        S->cv.notify_all();
        if (S->setup_thread.joinable()) S->setup_thread.join();
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
    r->nrhs = nrhs;
    r->tol = tol;
    r->t_submit = clk::now();
    r->est_bytes = estimate_request_bytes(r.get());
    std::lock_guard<std::mutex> lk(S->mu);
    if ((int)S->queue.size() >= S->prm.queue_capacity) return BI_ERR_BUSY;
    if (r->est_bytes > S->prm.mem_budget_bytes) {
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
    if (S->setup_thread.joinable()) S->setup_thread.join();
    cudaSetDevice(S->device);
    for (request* r : S->running) {
        if (r->ctx) bi_gmres_destroy(r->ctx);
        if (r->op) bi_destroy(r->op);
        if (r->d_rhs) cudaFree(r->d_rhs);
        if (r->d_x) cudaFree(r->d_x);
        if (r->stream) cudaStreamDestroy(r->stream);
        r->ctx = nullptr;
        r->op = nullptr;
    }
    for (request* r : S->ready) {
        if (r->ctx) bi_gmres_destroy(r->ctx);
        if (r->op) bi_destroy(r->op);
        if (r->d_rhs) cudaFree(r->d_rhs);
        if (r->d_x) cudaFree(r->d_x);
        if (r->stream) cudaStreamDestroy(r->stream);
        r->ctx = nullptr;
        r->op = nullptr;
    }
    for (auto& kv : S->all) delete kv.second;
    delete S;
}
