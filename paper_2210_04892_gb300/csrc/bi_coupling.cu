// Coupling with an interior discretisation: the reduced operator of Eq. 52,
//   y = C x - D^{X Lambda} Q^{-1} D^{Lambda X} x,
// computed as in steps 2(a)-(e) of Sec. II.E: the multilevel product y_d = C x, x1 = D^{Lambda X} x,
// x2 = Q^{-1} x1 by the caller's solver (the paper uses the LU factors of the sparse Q), and
// y = y_d - D^{X Lambda} x2.  D^{Lambda X} (n_int x n_unknowns) and D^{X Lambda}
// (n_unknowns x n_int) are the caller's CSR matrices on the device.
#include <algorithm>
#include <vector>

#include "bi_cpx.cuh"
#include "bi_internal.h"

namespace {

// y[r][i] (+)= sign * sum_j val[j] x[r][col[j]], rows i < nrows; vectors column-major with
// leading dimensions ldx, ldy.  One warp per (row, RHS).
template <typename T>
__global__ void __launch_bounds__(256) k_csr_apply(int64_t nrows, int R, const int* __restrict__ ptr,
                                                   const int* __restrict__ col, const cpx<T>* __restrict__ val,
                                                   const cpx<T>* __restrict__ x, int64_t ldx, cpx<T>* __restrict__ y,
                                                   int64_t ldy, T sign, int accumulate) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nrows * R) return;
    const int r = (int)(w / nrows);
    const int64_t i = w - (int64_t)r * nrows;
    cpx<T> acc = czero<T>();
    for (int j = ptr[i] + lane; j < ptr[i + 1]; j += 32) cfma(acc, val[j], x[(int64_t)r * ldx + col[j]]);
    acc = warp_sum(acc);
    if (lane == 0) {
        cpx<T> v = cscale(acc, sign);
        if (accumulate) v = cadd(v, y[(int64_t)r * ldy + i]);
        y[(int64_t)r * ldy + i] = v;
    }
}

template <typename T>
void csr_apply(int64_t nrows, int R, const int* ptr, const int* col, const void* val, const void* x, int64_t ldx, void* y,
               int64_t ldy, double sign, bool accumulate, cudaStream_t s) {
    const int64_t threads = nrows * R * 32;
    k_csr_apply<T><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(nrows, R, ptr, col, (const cpx<T>*)val,
                                                                     (const cpx<T>*)x, ldx, (cpx<T>*)y, ldy, (T)sign,
                                                                     accumulate ? 1 : 0);
    CU(cudaGetLastError());
}

}  // namespace

void bi_operator_launch(bi_handle_s* h, const void* x, void* y, int R, cudaStream_t s) {
    bi_matvec_launch(h, x, y, R, s);
    const bi_handle_s::coupling_t& c = h->cpl;
    if (!c.qsolve) return;
    const int64_t nun = h->nun;
    if (h->prec == 0) {
        csr_apply<double>(c.n_int, R, c.lx_ptr, c.lx_col, c.lx_val, x, nun, c.t1, c.n_int, 1.0, false, s);
        c.qsolve(c.user, c.t1, c.t2, R, (void*)s);
        csr_apply<double>(nun, R, c.xl_ptr, c.xl_col, c.xl_val, c.t2, c.n_int, y, nun, -1.0, true, s);
    } else {
        csr_apply<float>(c.n_int, R, c.lx_ptr, c.lx_col, c.lx_val, x, nun, c.t1, c.n_int, 1.0, false, s);
        c.qsolve(c.user, c.t1, c.t2, R, (void*)s);
        csr_apply<float>(nun, R, c.xl_ptr, c.xl_col, c.xl_val, c.t2, c.n_int, y, nun, -1.0, true, s);
    }
}

void bi_coupling_set(bi_handle_s* h, int64_t n_int, const int* lx_ptr, const int* lx_col, const void* lx_val,
                     const int* xl_ptr, const int* xl_col, const void* xl_val, bi_qsolve_fn qsolve, void* user) {
    bi_handle_s::coupling_t& c = h->cpl;
    if (!qsolve) {
        c.qsolve = nullptr;
        return;
    }
    if (c.n_int != n_int || !c.t1) {
        // workspace for D^{Lambda X} x and Q^{-1} of it, max_rhs columns
        c.t1 = h->alloc((size_t)n_int * h->max_rhs * h->csize);
        c.t2 = h->alloc((size_t)n_int * h->max_rhs * h->csize);
    }
    c.n_int = n_int;
    c.lx_ptr = lx_ptr;
    c.lx_col = lx_col;
    c.lx_val = lx_val;
    c.xl_ptr = xl_ptr;
    c.xl_col = xl_col;
    c.xl_val = xl_val;
    c.user = user;
    c.qsolve = qsolve;
}

// ---------------------------------------------------------------------------------
// The sparse coupling blocks themselves (Eqs. 47, 48, 40a, 40b) on the handle's surface:
//   D^{J Lambda}_mn = -1/2 <f_m, n x eta_n>,  D^{M Lambda}_mn = 1/2 <f_m, eta_n>,
//   D^{Lambda J}_mn = -<eta_m, n x f_n>,      D^{Lambda M}_mn = -<eta_m, f_n>,
// f the RWG functions (J and M share them), eta the zeroth-order edge functions of the
// triangles, eta = l_ab (lambda_a grad lambda_b - lambda_b grad lambda_a) on the edge (a, b),
// a the smaller global vertex number.  Every integral is over one triangle of two linear
// fields, so it is exact from the vertex values: int_T u.w = A/12 sum_ij (1 + delta_ij) u_i.w_j.
// The host builds the sparsity (integer work); one GPU thread computes each entry, which is a
// sum of one or two triangle terms.
namespace {

struct cpl_term {
    int tri;    // triangle (user order)
    int code;   // RWG free vertex (bits 0-1), RWG sign on this triangle (bit 2: minus),
                // local edge of eta (bits 3-4), kind (bits 5-6)
};

__device__ double coupling_face_term(const double* __restrict__ tri9, const double* __restrict__ tri_n,
                                     const double* __restrict__ tri_area, const int* __restrict__ tri_vid, cpl_term q) {
    const int t = q.tri;
    const int lf = q.code & 3, k = (q.code >> 3) & 3, kind = (q.code >> 5) & 3;
    const double sg = (q.code & 4) ? -1.0 : 1.0;
    double P[3][3], n[3];
    for (int i = 0; i < 3; ++i)
        for (int d = 0; d < 3; ++d) P[i][d] = tri9[9 * (size_t)t + 3 * i + d];
    for (int d = 0; d < 3; ++d) n[d] = tri_n[3 * (size_t)t + d];
    const double A = tri_area[t];
    auto len = [&](int i, int j) {
        const double dx = P[i][0] - P[j][0], dy = P[i][1] - P[j][1], dz = P[i][2] - P[j][2];
        return sqrt(dx * dx + dy * dy + dz * dz);
    };
    auto cross = [](const double* a, const double* b, double* c) {
        c[0] = a[1] * b[2] - a[2] * b[1];
        c[1] = a[2] * b[0] - a[0] * b[2];
        c[2] = a[0] * b[1] - a[1] * b[0];
    };
    // RWG vertex values: sign l / (2A) (P_i - P_lf)
    double fv[3][3], g[3][3], ev[3][3] = {};
    const double cf = sg * len((lf + 1) % 3, (lf + 2) % 3) / (2.0 * A);
    for (int i = 0; i < 3; ++i)
        for (int d = 0; d < 3; ++d) fv[i][d] = cf * (P[i][d] - P[lf][d]);
    // barycentric gradients: n x (P_{i+2} - P_{i+1}) / (2A)
    for (int i = 0; i < 3; ++i) {
        double e[3];
        for (int d = 0; d < 3; ++d) e[d] = (P[(i + 2) % 3][d] - P[(i + 1) % 3][d]) / (2.0 * A);
        cross(n, e, g[i]);
    }
    int a = (k + 1) % 3, b = (k + 2) % 3;
    if (tri_vid[3 * (size_t)t + a] > tri_vid[3 * (size_t)t + b]) {
        const int w = a;
        a = b;
        b = w;
    }
    const double lk = len(a, b);
    for (int d = 0; d < 3; ++d) {
        ev[a][d] = lk * g[b][d];
        ev[b][d] = -lk * g[a][d];
    }
    // kind 0: -1/2 <f, n x eta>; 1: 1/2 <f, eta>; 2: -<eta, n x f>; 3: -<eta, f>
    double (*u)[3] = (kind < 2) ? fv : ev;
    double (*w)[3] = (kind < 2) ? ev : fv;
    double wr[3][3];
    for (int j = 0; j < 3; ++j) {
        if (kind == 0 || kind == 2) cross(n, w[j], wr[j]);
        else
            for (int d = 0; d < 3; ++d) wr[j][d] = w[j][d];
    }
    double acc = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            acc += (i == j ? 2.0 : 1.0) * (u[i][0] * wr[j][0] + u[i][1] * wr[j][1] + u[i][2] * wr[j][2]);
    const double scale = kind == 0 ? -0.5 : (kind == 1 ? 0.5 : -1.0);
    return scale * acc * A / 12.0;
}

template <typename T>
__global__ void k_coupling_values(int64_t nnz, const int4* __restrict__ terms, const double* __restrict__ tri9,
                                  const double* __restrict__ tri_n, const double* __restrict__ tri_area,
                                  const int* __restrict__ tri_vid, cpx<T>* __restrict__ val) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const int4 q = terms[e];
    double v = coupling_face_term(tri9, tri_n, tri_area, tri_vid, cpl_term{q.x, q.y});
    if (q.z >= 0) v += coupling_face_term(tri9, tri_n, tri_area, tri_vid, cpl_term{q.z, q.w});
    val[e] = cpx<T>{(T)v, (T)0};
}

inline int term_code(int lf, bool minus, int k, int kind) { return lf | (minus ? 4 : 0) | (k << 3) | (kind << 5); }

// CSR rows under construction: (column, entry terms), merged by column and sorted.
struct row_builder {
    std::vector<int> ptr{0}, col;
    std::vector<int4> terms;
    std::vector<std::pair<int, cpl_term>> cur;
    void add(int c, int tri, int code) { cur.push_back({c, cpl_term{tri, code}}); }
    void close() {
        std::stable_sort(cur.begin(), cur.end(), [](const auto& p, const auto& q) { return p.first < q.first; });
        for (size_t i = 0; i < cur.size();) {
            int4 e{cur[i].second.tri, cur[i].second.code, -1, 0};
            size_t j = i + 1;
            if (j < cur.size() && cur[j].first == cur[i].first) {
                e.z = cur[j].second.tri;
                e.w = cur[j].second.code;
                ++j;
            }
            if (j < cur.size() && cur[j].first == cur[i].first)
                throw bi_error{BI_ERR_MESH, "coupling blocks: an entry with more than two triangle terms"};
            col.push_back(cur[i].first);
            terms.push_back(e);
            i = j;
        }
        ptr.push_back((int)col.size());
        cur.clear();
    }
};

}  // namespace

void bi_coupling_blocks_impl(bi_handle_s* h, int conforming, int64_t* sizes, int* xl_ptr, int* xl_col, void* xl_val,
                             int* lx_ptr, int* lx_col, void* lx_val) {
    const int N = h->N, nt = h->nt;
    // edge of each triangle opposite each local vertex, as an RWG index
    std::vector<int> tri_edge(3 * (size_t)nt, -1);
    for (int m = 0; m < N; ++m) {
        tri_edge[3 * (size_t)h->tplus[m] + h->lplus[m]] = m;
        tri_edge[3 * (size_t)h->tminus[m] + h->lminus[m]] = m;
    }
    const int nL = conforming ? N : 3 * nt;
    auto eta_col = [&](int t, int k) { return conforming ? tri_edge[3 * (size_t)t + k] : 3 * t + k; };
    // D^{X Lambda}: rows J (kind 0) then M (kind 1); each row the edge functions of both triangles
    row_builder XL, LX;
    for (int kind = 0; kind < 2; ++kind)
        for (int m = 0; m < N; ++m) {
            for (int side = 0; side < 2; ++side) {
                const int t = side ? h->tminus[m] : h->tplus[m];
                const int lf = side ? h->lminus[m] : h->lplus[m];
                for (int k = 0; k < 3; ++k) XL.add(eta_col(t, k), t, term_code(lf, side == 1, k, kind));
            }
            XL.close();
        }
    // D^{Lambda X}: one row per edge function; columns J (kind 2) then M (kind 3) of the RWG
    // functions on its triangle(s)
    auto lx_face = [&](int t, int k) {
        for (int j = 0; j < 3; ++j) {
            const int m = tri_edge[3 * (size_t)t + j];
            const bool minus = h->tminus[m] == t;
            LX.add(m, t, term_code(j, minus, k, 2));
            LX.add(N + m, t, term_code(j, minus, k, 3));
        }
    };
    if (conforming) {
        for (int e = 0; e < N; ++e) {
            lx_face(h->tplus[e], h->lplus[e]);
            lx_face(h->tminus[e], h->lminus[e]);
            LX.close();
        }
    } else {
        for (int t = 0; t < nt; ++t)
            for (int k = 0; k < 3; ++k) {
                lx_face(t, k);
                LX.close();
            }
    }
    sizes[0] = nL;
    sizes[1] = (int64_t)XL.col.size();
    sizes[2] = (int64_t)LX.col.size();
    if (!xl_ptr) return;
    cudaStream_t s = h->stream;
    int4* d_terms = nullptr;
    const size_t nterm = XL.terms.size() + LX.terms.size();
    CU(cudaMalloc(&d_terms, sizeof(int4) * nterm));
    try {
        CU(cudaMemcpyAsync(d_terms, XL.terms.data(), sizeof(int4) * XL.terms.size(), cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(d_terms + XL.terms.size(), LX.terms.data(), sizeof(int4) * LX.terms.size(),
                           cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(xl_ptr, XL.ptr.data(), sizeof(int) * XL.ptr.size(), cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(xl_col, XL.col.data(), sizeof(int) * XL.col.size(), cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(lx_ptr, LX.ptr.data(), sizeof(int) * LX.ptr.size(), cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(lx_col, LX.col.data(), sizeof(int) * LX.col.size(), cudaMemcpyHostToDevice, s));
        const int64_t n1 = (int64_t)XL.terms.size(), n2 = (int64_t)LX.terms.size();
        const int th = 128;
        if (h->prec == 0) {
            k_coupling_values<double><<<(unsigned)((n1 + th - 1) / th), th, 0, s>>>(
                n1, d_terms, h->d_tri, h->d_tri_n, h->d_tri_area, h->d_tri_vid, (cpx<double>*)xl_val);
            k_coupling_values<double><<<(unsigned)((n2 + th - 1) / th), th, 0, s>>>(
                n2, d_terms + n1, h->d_tri, h->d_tri_n, h->d_tri_area, h->d_tri_vid, (cpx<double>*)lx_val);
        } else {
            k_coupling_values<float><<<(unsigned)((n1 + th - 1) / th), th, 0, s>>>(
                n1, d_terms, h->d_tri, h->d_tri_n, h->d_tri_area, h->d_tri_vid, (cpx<float>*)xl_val);
            k_coupling_values<float><<<(unsigned)((n2 + th - 1) / th), th, 0, s>>>(
                n2, d_terms + n1, h->d_tri, h->d_tri_n, h->d_tri_area, h->d_tri_vid, (cpx<float>*)lx_val);
        }
        CU(cudaGetLastError());
        // the host arrays above are pageable and die with this call
        CU(cudaStreamSynchronize(s));
    } catch (...) {
        cudaFree(d_terms);
        throw;
    }
    CU(cudaFree(d_terms));
}

