// Coupling with an interior discretisation: the reduced operator of Eq. 52,
//   y = C x - D^{X Lambda} Q^{-1} D^{Lambda X} x,
// computed as in steps 2(a)-(e) of Sec. II.E: the multilevel product y_d = C x, x1 = D^{Lambda X} x,
// x2 = Q^{-1} x1 by the caller's solver (the paper uses the LU factors of the sparse Q), and
// y = y_d - D^{X Lambda} x2.  D^{Lambda X} (n_int x n_unknowns) and D^{X Lambda}
// (n_unknowns x n_int) are the caller's CSR matrices on the device.
#include <algorithm>

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
