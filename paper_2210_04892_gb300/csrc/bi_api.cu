// C-ABI entry points (include/bi.h): argument checks, handle lifecycle, error text.
#include <complex>
#include <map>
#include <mutex>
#include <chrono>
#include <cstring>
#include <exception>
#include <string>

#include "bi_internal.h"

static thread_local std::string g_setup_error;

void* bi_handle_s::alloc(size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw bi_error{BI_ERR_OOM, "cudaMalloc(" + std::to_string(bytes) + " B): " + cudaGetErrorString(e)};
    }
    owned.push_back({p, bytes});
    info.device_bytes += (int64_t)bytes;
    return p;
}

void bi_raise_smem_limit(const void* func, size_t bytes) {
    if (bytes <= 48 * 1024) return;
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> limit;
    int dev = 0;
    CU(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = limit[{dev, func}];
    if (bytes <= cur) return;
    CU(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
}

extern "C" void bi_default_params(bi_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->digits = 3;
    p->leaf_box = 0.25;
    p->levels = 0;
    p->interp_order = 10;
    p->precision = BI_PREC_FP32;
    p->op_mode = BI_MODE_CBLOCK;
    p->max_rhs = 1;
    p->gmres_restart = 100;
    p->gmres_maxit = 1000;
    p->stream = nullptr;
    p->eps_re = 1.0;
}

static void release(bi_handle_s* h) {
    if (!h) return;
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    for (auto& b : h->owned) cudaFree(b.p);
    h->owned.clear();
    if (h->h_pinned) cudaFreeHost(h->h_pinned);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    for (int l = 0; l < BI_MAXLEV; ++l) {
        if (h->tstream[l]) cudaStreamDestroy(h->tstream[l]);
        if (h->ev_tfork[l]) cudaEventDestroy(h->ev_tfork[l]);
        if (h->ev_tjoin[l]) cudaEventDestroy(h->ev_tjoin[l]);
    }
}

bool bi_params_valid(const bi_params& P) {
    return P.digits >= 1 && P.digits <= 8 && P.leaf_box > 0 && P.interp_order >= 2 && P.interp_order <= 32 &&
           (P.precision == 0 || P.precision == 1) && P.op_mode >= 0 && P.op_mode <= 4 && P.max_rhs >= 1 &&
           P.max_rhs <= 4096 && P.gmres_restart >= 1 && P.gmres_maxit >= 1 && P.levels >= 0 && P.levels <= 21 &&
           (P.precond == 0 || P.precond == 1) && P.k_im <= 0.0;
}

static int setup_two_region(const double* verts, int nv, const int* tris, int nt, double k0, const bi_params& P,
                            bi_handle* out);

// One operator.  op_mode 3 (one medium of the two-region form) is built only by the two-region
// set-up (internal = true).
static int setup_handle(const double* verts, int nv, const int* tris, int nt, double k0, int digits, const bi_params* opt,
                        bi_handle* out, bool internal) {
    if (!out) return BI_ERR_ARG;
    *out = nullptr;
    if (opt && opt->op_mode == 3 && !internal) {
        g_setup_error = "bi_setup: op_mode must be 0, 1 or 2";
        return BI_ERR_ARG;
    }
    if (!verts || !tris || nv < 3 || nt < 4 || !(k0 > 0)) {
        g_setup_error = "bi_setup: null mesh, fewer than 4 triangles, or k0 <= 0";
        return BI_ERR_ARG;
    }
    auto t0 = std::chrono::steady_clock::now();
    bi_handle_s* h = new bi_handle_s();
    if (opt) h->prm = *opt;
    else bi_default_params(&h->prm);
    if (digits > 0) h->prm.digits = digits;
    bi_params& P = h->prm;
    if (!bi_params_valid(P)) {
        g_setup_error = "bi_setup: parameter out of range";
        delete h;
        return BI_ERR_ARG;
    }
    if (P.op_mode == 2 || P.op_mode == 4) {
        const bi_params P2 = P;
        delete h;
        return setup_two_region(verts, nv, tris, nt, k0, P2, out);
    }
    if (P.k_im < -k0) {
        g_setup_error = "bi_setup: k_im outside [-k0, 0]";
        delete h;
        return BI_ERR_ARG;
    }
    h->k = k0;
    h->ki = P.k_im;
    h->prec = P.precision;
    h->csize = P.precision == 0 ? 16 : 8;
    h->nX = (P.op_mode == 0 || P.op_mode == 3) ? 2 : 1;
    h->nF = P.op_mode == 3 ? 2 : 1;
    h->max_rhs = P.max_rhs;
    h->stream = (cudaStream_t)P.stream;
    const char* env = std::getenv("BI_NO_GRAPHS");
    h->use_graphs = !(env && env[0] == '1');
    const char* env2 = std::getenv("BI_TWO_PASS");
    h->use_fast = !(env2 && env2[0] == '1') || h->ki != 0.0;   // the reference kernels assume a real k
    const char* env3 = std::getenv("BI_LEAF_BULK");
    h->use_leaf_bulk = !(env3 && env3[0] == '0');
    const char* env4 = std::getenv("BI_ANTERP_ROWS");
    h->force_anterp_rows = env4 && env4[0] == '1';
    const char* env8 = std::getenv("BI_INTERP_VARIANT");
    h->interp_variant = env8 ? std::atoi(env8) : 0;
    const char* env9 = std::getenv("BI_ANTERP_VARIANT");
    h->anterp_variant = env9 ? std::atoi(env9) : 0;
    const char* env7 = std::getenv("BI_TRANSLATE_VARIANT");
    h->translate_variant = env7 ? std::atoi(env7) : 0;
    if (h->translate_variant < 0 || h->translate_variant > 9) h->translate_variant = 0;
    const char* env6 = std::getenv("BI_NEAR_RB");
    h->near_rb = env6 ? std::atoi(env6) : 2;
    if (h->near_rb < 0 || h->near_rb > 2) h->near_rb = 2;
    const char* env5 = std::getenv("BI_AUTOTUNE");
    h->autotune = !(env5 && env5[0] == '0') && !h->force_anterp_rows;
    try {
        bi_build_rwg(h, verts, nv, tris, nt);
        h->nun = h->nX * h->N;
        bi_build_tree(h, verts);
        bi_build_sampling(h);
        bi_build_interp(h);
        // the far-field chain is the latency-critical path of a product: its streams get the
        // highest priority, the bandwidth-bound near-field product (side stream) the lowest
        int prio_lo = 0, prio_hi = 0;
        CU(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
        CU(cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, prio_lo));
        CU(cudaStreamCreateWithPriority(&h->cap, cudaStreamNonBlocking, prio_hi));
        CU(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        CU(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
        for (int l = 3; l < h->nlev && l < BI_MAXLEV; ++l) {
            CU(cudaStreamCreateWithPriority(&h->tstream[l], cudaStreamNonBlocking, prio_hi));
            CU(cudaEventCreateWithFlags(&h->ev_tfork[l], cudaEventDisableTiming));
            CU(cudaEventCreateWithFlags(&h->ev_tjoin[l], cudaEventDisableTiming));
        }
        {
            int dev = 0;
            CU(cudaGetDevice(&dev));
            h->device = dev;
            CU(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
        }
        bi_device_geometry(h, verts, tris);
        bi_fill_near(h);
        bi_fill_patterns(h);
        bi_fill_translations(h);
        bi_build_translate_lists(h);
        bi_alloc_work(h);
        bi_build_sai(h);
        CU(cudaStreamSynchronize(h->stream));
    } catch (const bi_error& e) {
        g_setup_error = e.msg;
        release(h);
        delete h;
        return e.code;
    } catch (const std::exception& e) {
        g_setup_error = std::string("bi_setup: ") + e.what();
        release(h);
        delete h;
        return BI_ERR_OOM;
    }
    bi_info_t& I = h->info;
    I.n_rwg = h->N;
    I.n_unknowns = h->nun;
    I.levels = h->nlev;
    I.leaf_level = h->leaf;
    for (int l = 0; l < h->nlev && l < 32; ++l) {
        I.boxes[l] = h->lev[l].nbox;
        I.L[l] = h->lev[l].L;
        I.K[l] = h->lev[l].K;
        I.interactions[l] = h->lev[l].n_inter;
    }
    I.near_pairs = h->near_nnz;
    I.root_size = h->lev[0].a;
    I.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return BI_OK;
}

extern "C" int bi_setup(const double* verts, int nv, const int* tris, int nt, double k0, int digits, const bi_params* opt,
                        bi_handle* out) {
    return setup_handle(verts, nv, tris, nt, k0, digits, opt, out, false);
}

// The two-region operator: one op_mode-3 handle per medium, the exterior at k0 (a = b = 1) and
// the body at k1 = k0 sqrt(eps_r) (a = eta, b = 1/eta, eta = 1/sqrt(eps_r)); products summed.
static int setup_two_region(const double* verts, int nv, const int* tris, int nt, double k0, const bi_params& P,
                            bi_handle* out) {
    auto t0 = std::chrono::steady_clock::now();
    if (P.precond != 0 || P.k_im != 0.0 || !(P.eps_im <= 0.0) || !(P.eps_re * P.eps_re + P.eps_im * P.eps_im > 0.0)) {
        g_setup_error = "bi_setup: two-region needs precond 0, k_im 0, eps_im <= 0 and eps_r != 0";
        return BI_ERR_ARG;
    }
    std::complex<double> n = std::sqrt(std::complex<double>(P.eps_re, P.eps_im));
    if (n.real() < 0) n = -n;
    const std::complex<double> k1 = k0 * n, eta = 1.0 / n;
    if (!(k1.real() > 0) || -k1.imag() > k1.real()) {
        g_setup_error = "bi_setup: the body's wavenumber k0 sqrt(eps_r) has |Im k| > Re k";
        return BI_ERR_ARG;
    }
    const bool coated = P.op_mode == 4;
    int nt_outer = nt;
    if (coated) {
        // the core: the last core_tris triangles; every vertex of the outer surface numbered first
        if (P.core_tris < 4 || P.core_tris > nt - 4) {
            g_setup_error = "bi_setup: coated body needs 4 <= core_tris <= nt - 4";
            return BI_ERR_ARG;
        }
        nt_outer = nt - P.core_tris;
        int max_outer = -1, min_core = nv;
        for (int t = 0; t < nt; ++t)
            for (int a = 0; a < 3; ++a) {
                const int v = tris[3 * t + a];
                if (t < nt_outer) max_outer = std::max(max_outer, v);
                else min_core = std::min(min_core, v);
            }
        if (max_outer >= min_core) {
            g_setup_error = "bi_setup: coated body: number the outer surface's vertices before the core's";
            return BI_ERR_MESH;
        }
    }
    bi_params P0 = P, P1 = P;
    P0.op_mode = P1.op_mode = 3;
    P0.k_im = 0.0;
    P1.k_im = k1.imag();
    bi_handle c0 = nullptr, c1 = nullptr;
    int rc = setup_handle(verts, nv, tris, nt_outer, k0, 0, &P0, &c0, true);
    if (rc != BI_OK) return rc;
    rc = setup_handle(verts, nv, tris, nt, k1.real(), 0, &P1, &c1, true);
    if (rc != BI_OK) {
        bi_destroy(c0);
        return rc;
    }
    if (coated) {
        // the coat's RWG functions: those of the outer surface first, numbered as the outer medium's
        bool same = c1->N > c0->N;
        for (int i = 0; same && i < 2 * c0->N; ++i) same = c0->edges[i] == c1->edges[i];
        if (!same) {
            g_setup_error = "bi_setup: coated body: the outer surface's RWG functions do not come first";
            bi_destroy(c0);
            bi_destroy(c1);
            return BI_ERR_MESH;
        }
    }
    c1->pa[0] = eta.real();
    c1->pa[1] = eta.imag();
    c1->pb[0] = n.real();
    c1->pb[1] = n.imag();
    bi_handle_s* h = new bi_handle_s();
    h->prm = P;
    h->k = k0;
    h->prec = P.precision;
    h->csize = P.precision == 0 ? 16 : 8;
    h->N = c0->N;
    h->nun = c0->nun;
    h->nX = 2;
    h->nF = 2;
    h->max_rhs = P.max_rhs;
    h->stream = (cudaStream_t)P.stream;
    h->device = c0->device;
    h->med[0] = c0;
    h->med[1] = c1;
    h->edges = c0->edges;
    if (coated) {
        h->coated = 1;
        h->N1 = c0->N;
        h->N2 = c1->N - c0->N;
        h->N = c1->N;
        h->nun = 2 * h->N1 + h->N2;
        h->edges = c1->edges;
    }
    try {
        h->d_status = (int*)h->alloc(sizeof(int));
        CU(cudaMemset(h->d_status, 0, sizeof(int)));
        const size_t vec = (size_t)h->nun * h->max_rhs * h->csize;
        h->d_sx = h->alloc(vec);
        h->d_sy = h->alloc(vec);
        h->d_ysum = h->alloc(vec);
        if (coated) {
            const size_t v0 = (size_t)c0->nun * h->max_rhs * h->csize, v1 = (size_t)c1->nun * h->max_rhs * h->csize;
            h->d_xin0 = h->alloc(v0);
            h->d_y0 = h->alloc(v0);
            h->d_xin1 = h->alloc(v1);
            h->d_y1 = h->alloc(v1);
        }
    } catch (const bi_error& e) {
        g_setup_error = e.msg;
        release(h);
        delete h;
        bi_destroy(c0);
        bi_destroy(c1);
        return e.code;
    }
    h->info = c0->info;
    h->info.n_rwg = h->N;
    h->info.n_unknowns = h->nun;
    int64_t own = 0;
    for (const dbuf& b : h->owned) own += (int64_t)b.bytes;
    h->info.device_bytes = c0->info.device_bytes + c1->info.device_bytes + own;
    h->info.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return BI_OK;
}

extern "C" int bi_num_unknowns(bi_handle h, int64_t* n_rwg, int64_t* n_unknowns) {
    if (!h) return BI_ERR_ARG;
    if (n_rwg) *n_rwg = h->N;
    if (n_unknowns) *n_unknowns = h->nun;
    return BI_OK;
}

extern "C" int bi_rwg_edges(bi_handle h, int* ev) {
    if (!h || !ev) return BI_ERR_ARG;
    std::memcpy(ev, h->edges.data(), sizeof(int) * h->edges.size());
    return BI_OK;
}

extern "C" int bi_get_info(bi_handle h, bi_info_t* info) {
    if (!h || !info) return BI_ERR_ARG;
    *info = h->info;
    return BI_OK;
}

template <typename F>
static int guarded(bi_handle h, F&& f) {
    try {
        return f();
    } catch (const bi_error& e) {
        h->err = e.msg;
        return e.code;
    } catch (const std::exception& e) {
        // a host allocation failed: report it rather than let it cross the C ABI
        h->err = std::string("host: ") + e.what();
        return BI_ERR_OOM;
    }
}

// Read and clear the device status word (the caller has synchronised the work it checks).
int bi_take_device_status(bi_handle_s* h) {
    for (bi_handle_s* m : h->med)
        if (m && bi_take_device_status(m) != BI_OK) {
            h->err = m->err;
            return BI_ERR_TIMEOUT;
        }
    if (!h->d_status) return BI_OK;
    int st = 0;
    CU(cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st == 0) return BI_OK;
    CU(cudaMemset(h->d_status, 0, sizeof(int)));
    h->err = "a bounded wait on a bulk copy gave up in a product kernel (results of that product are invalid)";
    return BI_ERR_TIMEOUT;
}

extern "C" int bi_device_status(bi_handle h) {
    if (!h) return BI_ERR_ARG;
    return guarded(h, [&] {
        CU(cudaStreamSynchronize(h->stream));
        return bi_take_device_status(h);
    });
}

extern "C" int bi_matvec(bi_handle h, const void* x, void* y, int nrhs) {
    if (!h) return BI_ERR_ARG;
    if (!x || !y || nrhs < 1 || nrhs > h->max_rhs) {
        h->err = "bi_matvec: null vector or nrhs outside [1, max_rhs]";
        return BI_ERR_ARG;
    }
    size_t bytes = (size_t)h->nun * nrhs * h->csize;
    const char* xa = (const char*)x;
    const char* ya = (const char*)y;
    if (xa < ya + bytes && ya < xa + bytes) {
        h->err = "bi_matvec: x and y overlap";
        return BI_ERR_ARG;
    }
    return guarded(h, [&] {
        bi_matvec_launch(h, x, y, nrhs, h->stream);
        return (int)BI_OK;
    });
}

extern "C" int bi_set_coupling(bi_handle h, int64_t n_int, const int* dlx_ptr, const int* dlx_col, const void* dlx_val,
                               const int* dxl_ptr, const int* dxl_col, const void* dxl_val, bi_qsolve_fn qsolve,
                               void* user) {
    if (!h) return BI_ERR_ARG;
    if (h->med[0]) {
        h->err = "bi_set_coupling: not available for the two-region operator";
        return BI_ERR_ARG;
    }
    if (qsolve && (n_int < 1 || !dlx_ptr || !dlx_col || !dlx_val || !dxl_ptr || !dxl_col || !dxl_val)) {
        h->err = "bi_set_coupling: n_int < 1 or a null CSR array";
        return BI_ERR_ARG;
    }
    return guarded(h, [&] {
        bi_coupling_set(h, n_int, dlx_ptr, dlx_col, dlx_val, dxl_ptr, dxl_col, dxl_val, qsolve, user);
        return (int)BI_OK;
    });
}

extern "C" int bi_coupling_blocks(bi_handle h, int conforming, int64_t* sizes, int* dxl_ptr, int* dxl_col,
                                  void* dxl_val, int* dlx_ptr, int* dlx_col, void* dlx_val) {
    if (!h) return BI_ERR_ARG;
    if (h->med[0] || h->prm.op_mode != 0) {
        h->err = "bi_coupling_blocks: needs the C-block operator (op_mode 0: unknowns [J; M])";
        return BI_ERR_ARG;
    }
    const bool none = !dxl_ptr && !dxl_col && !dxl_val && !dlx_ptr && !dlx_col && !dlx_val;
    const bool all = dxl_ptr && dxl_col && dxl_val && dlx_ptr && dlx_col && dlx_val;
    if (!sizes || (conforming != 0 && conforming != 1) || !(none || all)) {
        h->err = "bi_coupling_blocks: null sizes, conforming not 0 or 1, or some but not all CSR arrays null";
        return BI_ERR_ARG;
    }
    return guarded(h, [&] {
        bi_coupling_blocks_impl(h, conforming, sizes, dxl_ptr, dxl_col, dxl_val, dlx_ptr, dlx_col, dlx_val);
        return (int)BI_OK;
    });
}

extern "C" int bi_matvec_coupled(bi_handle h, const void* x, void* y, int nrhs) {
    if (!h) return BI_ERR_ARG;
    if (!h->cpl.qsolve) {
        h->err = "bi_matvec_coupled: no coupling set (bi_set_coupling)";
        return BI_ERR_ARG;
    }
    if (!x || !y || nrhs < 1 || nrhs > h->max_rhs) {
        h->err = "bi_matvec_coupled: null vector or nrhs outside [1, max_rhs]";
        return BI_ERR_ARG;
    }
    return guarded(h, [&] {
        bi_operator_launch(h, x, y, nrhs, h->stream);
        return (int)BI_OK;
    });
}

extern "C" int bi_matvec_host(bi_handle h, const void* x, void* y, int nrhs) {
    if (!h) return BI_ERR_ARG;
    if (!x || !y || nrhs < 1 || nrhs > h->max_rhs) {
        h->err = "bi_matvec_host: null vector or nrhs outside [1, max_rhs]";
        return BI_ERR_ARG;
    }
    size_t bytes = (size_t)h->nun * nrhs * h->csize;
    return guarded(h, [&] {
        CU(cudaMemcpyAsync(h->d_sx, x, bytes, cudaMemcpyHostToDevice, h->stream));
        bi_matvec_launch(h, h->d_sx, h->d_sy, nrhs, h->stream);
        CU(cudaMemcpyAsync(y, h->d_sy, bytes, cudaMemcpyDeviceToHost, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        return bi_take_device_status(h);
    });
}

extern "C" int bi_rhs_planewave(bi_handle h, const double* khat, const double* phat, int nrhs, void* b) {
    if (h && h->ki != 0.0) {
        h->err = "bi_rhs_planewave: the handle's medium is lossy (k_im != 0); plane waves are built for free space";
        return BI_ERR_ARG;
    }
    if (!h) return BI_ERR_ARG;
    if (!khat || !phat || !b || nrhs < 1) {
        h->err = "bi_rhs_planewave: null argument or nrhs < 1";
        return BI_ERR_ARG;
    }
    if (nrhs > h->max_rhs && h->coated) {
        h->err = "bi_rhs_planewave: nrhs above max_rhs (coated body)";
        return BI_ERR_ARG;
    }
    return guarded(h, [&] {
        if (h->coated) {
            // the outer surface's [-<f, E>; -<f, H>], zero on the core's rows
            bi_rhs_launch(h->med[0], khat, phat, nrhs, h->d_y0);
            bi_coated_rhs(h, b, nrhs, h->stream);
            CU(cudaStreamSynchronize(h->stream));
            return (int)BI_OK;
        }
        bi_rhs_launch(h->med[0] ? h->med[0] : h, khat, phat, nrhs, b);
        return (int)BI_OK;
    });
}

extern "C" int bi_solve(bi_handle h, const void* rhs, void* x, int nrhs, double tol, int* iters, double* relres) {
    if (!h) return BI_ERR_ARG;
    if (!rhs || !x || nrhs < 1 || nrhs > h->max_rhs || !(tol > 0)) {
        h->err = "bi_solve: null vector, nrhs outside [1, max_rhs] or tol <= 0";
        return BI_ERR_ARG;
    }
    return guarded(h, [&] { return bi_gmres(h, rhs, x, nrhs, tol, iters, relres); });
}

extern "C" int bi_solve_refined(bi_handle h, bi_handle h_ref, const void* rhs, void* x, int nrhs, double tol, int* iters,
                                double* relres) {
    if (!h || !h_ref) return BI_ERR_ARG;
    if (!rhs || !x || nrhs < 1 || nrhs > h->max_rhs || nrhs > h_ref->max_rhs || !(tol > 0) || h_ref->prec != 0 ||
        h_ref->nun != h->nun || h_ref->prm.op_mode != h->prm.op_mode || h_ref->N != h->N) {
        h->err = "bi_solve_refined: null vector, nrhs outside [1, max_rhs], tol <= 0, or h_ref not an FP64 handle of "
                 "the same operator";
        return BI_ERR_ARG;
    }
    return guarded(h, [&] { return bi_solve_refined_impl(h, h_ref, rhs, x, nrhs, tol, iters, relres); });
}

extern "C" const char* bi_last_error(bi_handle h) { return h ? h->err.c_str() : g_setup_error.c_str(); }

extern "C" void bi_destroy(bi_handle h) {
    if (!h) return;
    for (bi_handle_s*& m : h->med) {
        bi_destroy(m);
        m = nullptr;
    }
    cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
}

extern "C" int bi_debug_copy(bi_handle h, int what, int level, void* host, int64_t bytes) {
    if (!h || !host || bytes < 0) return BI_ERR_ARG;
    if (h->med[0]) return bi_debug_copy(h->med[0], what, level, host, bytes);   // two-region: the exterior medium
    const void* src = nullptr;
    size_t need = 0;
    const bool far = h->leaf >= 2;
    const bool lev_ok = far && level >= 2 && level <= h->leaf;
    const int E = 2 * h->max_rhs;
    switch (what) {
        case 0:
        case 1:
            if (!far) break;
            src = what == 0 ? h->d_F : h->d_RX;
            need = (size_t)h->N * (h->lev[h->leaf].K / 2) * 2 * h->csize;
            break;
        case 2:
            if (!lev_ok) break;
            src = h->lev[level].d_T;
            need = (size_t)343 * h->lev[level].K * h->csize;
            break;
        case 3:
        case 4:
            if (!lev_ok) break;
            src = what == 3 ? h->lev[level].d_U : h->lev[level].d_V;
            need = (size_t)h->lev[level].nbox * h->lev[level].K * E * h->csize;
            break;
        case 5:
            src = h->d_perm;
            need = sizeof(int) * (size_t)h->N;
            break;
        default:
            break;
    }
    if (!src || (size_t)bytes < need) {
        h->err = "bi_debug_copy: no such buffer or host buffer too small";
        return BI_ERR_ARG;
    }
    return guarded(h, [&] {
        CU(cudaStreamSynchronize(h->stream));
        CU(cudaMemcpy(host, src, need, cudaMemcpyDeviceToHost));
        return (int)BI_OK;
    });
}

extern "C" int bi_profile_stages(bi_handle h, const void* x, void* y, int nrhs, int reps, double* stage_ms) {
    if (!h) return BI_ERR_ARG;
    if (!x || !y || !stage_ms || nrhs < 1 || nrhs > h->max_rhs || reps < 1) {
        h->err = "bi_profile_stages: null argument, nrhs outside [1, max_rhs] or reps < 1";
        return BI_ERR_ARG;
    }
    return guarded(h, [&] {
        if (h->med[0]) {
            // two-region: the stages of both media, summed
            double ms1[BI_NSTAGES];
            if (h->coated) {
                bi_coated_outer_currents(h, x, nrhs, h->stream);
                bi_profile_impl(h->med[0], h->d_xin0, h->d_y0, nrhs, reps, stage_ms);
                bi_profile_impl(h->med[1], h->d_xin1, h->d_y1, nrhs, reps, ms1);
                for (int i = 0; i < BI_NSTAGES; ++i) stage_ms[i] += ms1[i];
                return (int)BI_OK;
            }
            bi_profile_impl(h->med[0], x, y, nrhs, reps, stage_ms);
            bi_profile_impl(h->med[1], x, h->d_ysum, nrhs, reps, ms1);
            for (int i = 0; i < BI_NSTAGES; ++i) stage_ms[i] += ms1[i];
            return (int)BI_OK;
        }
        bi_profile_impl(h, x, y, nrhs, reps, stage_ms);
        return (int)BI_OK;
    });
}

extern "C" const char* bi_stage_name(int i) { return bi_stage_name_impl(i); }

extern "C" int bi_tuned_config(bi_handle h, char* buf, int64_t len) {
    if (!h || !buf || len < 1) return BI_ERR_ARG;
    static const char* pass_name[3] = {"translate", "interpolate", "anterpolate"};
    std::string out;
    for (int m = 0; m < 2; ++m) {
        const bi_handle_s* src = h->med[0] ? h->med[m] : (m == 0 ? h : nullptr);
        if (!src) continue;
        for (const auto& t : src->tuned) {
            std::string form = t.pass == 0 ? (t.variant >= 6 ? std::string(t.variant % 2 ? "2" : "1") +
                                                                    " pair(s)/thread, " + (t.variant <= 7 ? "4" : "8") +
                                                                    " child slots, pipelined loads"
                                              : t.variant == 5 ? std::string("staged sources, thread per child slot")
                                              : std::string(t.variant % 2 == 0 ? "2 pairs/thread" : "1 pair/thread") +
                                                    (t.variant >= 3 ? ", 4 child slots/thread" : ""))
                               : t.variant == 2 ? "two-pass"
                               : t.variant == 3 ? "two-pass, entry pairs"
                               : t.variant >= 200 ? "row blocks, chunk " + std::to_string(t.variant - 200)
                               : t.pass == 1 ? "rows per CTA, chunk " + std::to_string(t.variant - 100)
                                             : "per child, chunk " + std::to_string(t.variant - 100);
            if (h->med[0]) out += "medium " + std::to_string(m) + " ";
            out += std::string(pass_name[t.pass]) + " level " + std::to_string(t.level) + " E " + std::to_string(t.E) +
                   ": " + form + " (" + std::to_string((int)t.us) + " us)\n";
        }
    }
    std::strncpy(buf, out.c_str(), (size_t)len - 1);
    buf[len - 1] = 0;
    return (int64_t)out.size() < len ? BI_OK : BI_ERR_ARG;
}

extern "C" int bi_debug_set_wait_limit(bi_handle h, long long cycles) {
    if (!h) return BI_ERR_ARG;
    return guarded(h, [&] {
        CU(cudaStreamSynchronize(h->stream));
        h->wait_cycles = cycles > 0 ? cycles : (1ll << 31);
        for (bi_handle_s* m : h->med)
            if (m && bi_debug_set_wait_limit(m, cycles) != BI_OK) throw bi_error{BI_ERR_CUDA, m->err};
        // the captured products carry the old limit as a kernel argument
        for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
        h->graphs.clear();
        return (int)BI_OK;
    });
}

extern "C" int bi_farfield(bi_handle h, const void* x, int nrhs, const double* dirs, int ndir, void* F) {
    if (h && h->coated) {
        // the outer surface's currents radiate into free space
        if (!x || nrhs < 1 || nrhs > h->max_rhs) {
            h->err = "bi_farfield: null x or nrhs outside [1, max_rhs] (coated body)";
            return BI_ERR_ARG;
        }
        const int rc = guarded(h, [&] {
            bi_coated_outer_currents(h, x, nrhs, h->stream);
            return (int)BI_OK;
        });
        return rc != BI_OK ? rc : bi_farfield(h->med[0], h->d_xin0, nrhs, dirs, ndir, F);
    }
    if (h && h->med[0]) return bi_farfield(h->med[0], x, nrhs, dirs, ndir, F);   // radiated into the exterior
    if (h && h->ki != 0.0) {
        h->err = "bi_farfield: the handle's medium is lossy (k_im != 0); a far field exists in free space only";
        return BI_ERR_ARG;
    }
    if (!h) return BI_ERR_ARG;
    if (!x || !dirs || !F || nrhs < 1 || ndir < 1 || nrhs > 65535 || ndir > 65535) {
        h->err = "bi_farfield: null argument or nrhs/ndir outside [1, 65535]";
        return BI_ERR_ARG;
    }
    return guarded(h, [&] {
        size_t need = bi_farfield_scratch_bytes(h, nrhs, ndir);
        if (need > h->ffscratch_bytes) {
            // scratch is kept by the handle and reused by later calls
            CU(cudaStreamSynchronize(h->stream));
            h->d_ffscratch = h->alloc(need);
            h->ffscratch_bytes = need;
        }
        bi_farfield_launch(h, x, nrhs, dirs, ndir, F, (double*)h->d_ffscratch, h->stream);
        return (int)BI_OK;
    });
}
