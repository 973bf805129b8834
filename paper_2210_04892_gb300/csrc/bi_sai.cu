// Sparse approximate inverse (SAI) preconditioner built from the near field of the operator
// only (the preconditioned solves of Sec. III.B use an SAI constructed from C alone).
//
// Right preconditioner M, block-diagonal over leaf boxes: for box b with unknowns T (its
// RWGs, both currents in op_mode 0) and N the unknowns of b's near boxes (the rows through
// which the near field couples to T),
//   M_b = argmin || A(N, T) M_b - I(N, T) ||_F  =>  (A_NT^H A_NT) M_b = A_TT^H,
// A the near-field operator exactly as the product applies it (stored blocks plus the Gram
// terms).  GMRES then solves A M u = b and returns x = M u, so the residual it minimises is
// the true one and the solution is that of A x = b.
//
// Set-up: one CTA per box accumulates the Hermitian normal matrix in FP64 directly from the
// near-block storage and factors it (Cholesky, small Tikhonov shift); M_b is stored in the
// handle precision.  Apply: one CTA per box, y_T = M_b x_T through the user permutation.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "bi_cpx.cuh"
#include "bi_internal.h"

namespace {

__device__ __forceinline__ cpx<double> to64(cpx<float> a) { return {(double)a.x, (double)a.y}; }
__device__ __forceinline__ cpx<double> to64(cpx<double> a) { return a; }

// Operator entry for test row (tree RWG m of box bp at local row ml, current Xr) and trial
// column c of bp's segment (current Xc), as the near-field product applies it.
template <typename T, int MODE>
__device__ cpx<double> near_entry(const cpx<T>* __restrict__ blocks, int64_t segp, int ncolp, int ml, int col, int Xr,
                                  int Xc, int m, const int* __restrict__ gptr, const int* __restrict__ gseg,
                                  const T* __restrict__ gval) {
    if (MODE == 1) {
        const cpx<double> a = to64(blocks[segp + (int64_t)ml * ncolp + col]);
        return {-a.x, -a.y};
    }
    const cpx<T>* p = blocks + 2 * (segp + (int64_t)ml * ncolp + col);
    const cpx<double> A = to64(p[0]), B = to64(p[1]);
    if (Xr == 0) return Xc == 0 ? cpx<double>{-A.x, -A.y} : cpx<double>{-B.x, -B.y};
    cpx<double> v = Xc == 0 ? B : cpx<double>{-A.x, -A.y};
    for (int g = gptr[m]; g < gptr[m + 1]; ++g)
        if (gseg[g] == col) {
            if (Xc == 0) v.x += 0.5 * (double)gval[2 * g + 1];
            else v.x -= 0.5 * (double)gval[2 * g];
        }
    return v;
}

// H_b = A_NT^H A_NT and R_b = A_TT^H for every leaf box (one CTA per box, FP64).
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_sai_normal(const int* __restrict__ leaf_start, const int* __restrict__ near_ptr,
                                                    const int* __restrict__ near_src, const int64_t* __restrict__ near_blk,
                                                    const int* __restrict__ near_col0, const int* __restrict__ near_ncol,
                                                    const int* __restrict__ near_tr, const cpx<T>* __restrict__ blocks,
                                                    const int* __restrict__ gptr, const int* __restrict__ gseg,
                                                    const T* __restrict__ gval, const int64_t* __restrict__ off,
                                                    cpx<double>* __restrict__ Hs, cpx<double>* __restrict__ Rs) {
    constexpr int NX = MODE == 0 ? 2 : 1;
    const int b = blockIdx.x;
    const int nb = leaf_start[b + 1] - leaf_start[b], n = NX * nb;
    cpx<double>* H = Hs + off[b];
    cpx<double>* Rb = Rs + off[b];
    for (int o = threadIdx.x; o < n * n; o += blockDim.x) {
        const int i = o / n, j = o - i * n;
        const int Xi = i / nb, ci = i - Xi * nb, Xj = j / nb, cj = j - Xj * nb;
        cpx<double> acc = {0.0, 0.0}, rself = {0.0, 0.0};
        for (int q = near_ptr[b]; q < near_ptr[b + 1]; ++q) {
            const int bp = near_src[q];
            const int qp = near_tr[q];                    // entry of b in bp's near list
            const int m0p = leaf_start[bp], mbp = leaf_start[bp + 1] - m0p;
            const int64_t segp = near_blk[near_ptr[bp]];
            const int ncolp = near_ncol[bp], c0p = near_col0[qp];
            for (int ml = 0; ml < mbp; ++ml)
                for (int Xr = 0; Xr < NX; ++Xr) {
                    const cpx<double> ei = near_entry<T, MODE>(blocks, segp, ncolp, ml, c0p + ci, Xr, Xi, m0p + ml, gptr, gseg, gval);
                    const cpx<double> ej = near_entry<T, MODE>(blocks, segp, ncolp, ml, c0p + cj, Xr, Xj, m0p + ml, gptr, gseg, gval);
                    acc.x += ei.x * ej.x + ei.y * ej.y;   // conj(ei) ej
                    acc.y += ei.x * ej.y - ei.y * ej.x;
                    // R = A_TT^H: R[i][j] = conj(A[(row j of T), (col i of T)])
                    if (bp == b && ml == cj && Xr == Xj) rself = {ei.x, -ei.y};
                }
        }
        H[o] = acc;
        Rb[o] = rself;
    }
}

// Cholesky H = L L^H in place (lower), then M = H^{-1} R by forward and back substitution,
// one right-hand-side column per thread; M stored row-major in the handle precision.
template <typename T>
__global__ void __launch_bounds__(256) k_sai_solve(const int* __restrict__ leaf_start, int NX, const int64_t* __restrict__ off,
                                                   cpx<double>* __restrict__ Hs, cpx<double>* __restrict__ Rs,
                                                   cpx<T>* __restrict__ Ms) {
    const int b = blockIdx.x;
    const int n = NX * (leaf_start[b + 1] - leaf_start[b]);
    cpx<double>* H = Hs + off[b];
    cpx<double>* Rb = Rs + off[b];
    __shared__ double shift;
    if (threadIdx.x == 0) {
        double tr = 0.0;
        for (int i = 0; i < n; ++i) tr += H[i * n + i].x;
        shift = 1e-12 * tr / max(n, 1) + 1e-300;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) H[i * n + i].x += shift;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) H[k * n + k] = {sqrt(fmax(H[k * n + k].x, shift)), 0.0};
        __syncthreads();
        const double d = H[k * n + k].x;
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
            H[i * n + k].x /= d;
            H[i * n + k].y /= d;
        }
        __syncthreads();
        const int w = n - k - 1;
        for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
            const int i = k + 1 + t / w, j = k + 1 + t % w;
            if (j > i) continue;
            const cpx<double> a = H[i * n + k], c = H[j * n + k];   // H_ij -= L_ik conj(L_jk)
            H[i * n + j].x -= a.x * c.x + a.y * c.y;
            H[i * n + j].y -= a.y * c.x - a.x * c.y;
        }
        __syncthreads();
    }
    cpx<T>* M = Ms + off[b];
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        // forward: L z = R[:, c]  (z kept in R's column)
        for (int i = 0; i < n; ++i) {
            cpx<double> s = Rb[i * n + c];
            for (int k = 0; k < i; ++k) {
                const cpx<double> l = H[i * n + k], z = Rb[k * n + c];
                s.x -= l.x * z.x - l.y * z.y;
                s.y -= l.x * z.y + l.y * z.x;
            }
            const double d = H[i * n + i].x;
            Rb[i * n + c] = {s.x / d, s.y / d};
        }
        // back: L^H m = z
        for (int i = n - 1; i >= 0; --i) {
            cpx<double> s = Rb[i * n + c];
            for (int k = i + 1; k < n; ++k) {
                const cpx<double> l = H[k * n + i], z = Rb[k * n + c];   // conj(L_ki) z_k
                s.x -= l.x * z.x + l.y * z.y;
                s.y -= l.x * z.y - l.y * z.x;
            }
            const double d = H[i * n + i].x;
            Rb[i * n + c] = {s.x / d, s.y / d};
        }
        for (int i = 0; i < n; ++i) M[i * n + c] = {(T)Rb[i * n + c].x, (T)Rb[i * n + c].y};
    }
}

// y = M x for vectors in user order [R][nun]; one CTA per box.
template <typename T>
__global__ void __launch_bounds__(128) k_sai_apply(int N, int nun, int NX, int R, const int* __restrict__ perm,
                                                   const int* __restrict__ leaf_start, const int64_t* __restrict__ off,
                                                   const cpx<T>* __restrict__ Ms, const cpx<T>* __restrict__ x,
                                                   cpx<T>* __restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* xs = reinterpret_cast<cpx<T>*>(smem_raw);   // [R][n]
    const int b = blockIdx.x;
    const int n0 = leaf_start[b], nb = leaf_start[b + 1] - n0, n = NX * nb;
    for (int t = threadIdx.x; t < n * R; t += blockDim.x) {
        const int r = t / n, i = t - r * n, X = i / nb, c = i - X * nb;
        xs[t] = x[(int64_t)r * nun + (int64_t)X * N + perm[n0 + c]];
    }
    __syncthreads();
    const cpx<T>* M = Ms + off[b];
    for (int t = threadIdx.x; t < n * R; t += blockDim.x) {
        const int r = t / n, i = t - r * n, X = i / nb, c = i - X * nb;
        cpx<T> acc = czero<T>();
        for (int j = 0; j < n; ++j) cfma(acc, M[(int64_t)i * n + j], xs[r * n + j]);
        y[(int64_t)r * nun + (int64_t)X * N + perm[n0 + c]] = acc;
    }
}

template <typename T>
void build_t(bi_handle_s* h) {
    const int nbox = (int)h->leaf_start.size() - 1;
    const int NX = h->nX;
    std::vector<int64_t> off(nbox + 1, 0);
    for (int b = 0; b < nbox; ++b) {
        const int64_t n = (int64_t)NX * (h->leaf_start[b + 1] - h->leaf_start[b]);
        off[b + 1] = off[b] + n * n;
    }
    // position of b in the near list of each of its near boxes (the near relation is symmetric)
    std::vector<int> tr(h->near_src.size(), -1);
    for (int b = 0; b < nbox; ++b)
        for (int q = h->near_ptr[b]; q < h->near_ptr[b + 1]; ++q) {
            const int bp = h->near_src[q];
            for (int qp = h->near_ptr[bp]; qp < h->near_ptr[bp + 1]; ++qp)
                if (h->near_src[qp] == b) tr[q] = qp;
            if (tr[q] < 0) throw bi_error{BI_ERR_ARG, "near lists are not symmetric"};
        }
    h->sai_off = (int64_t*)h->upload(off);
    int* d_tr = h->upload(tr);
    h->d_sai = h->alloc((size_t)off[nbox] * sizeof(cpx<T>));
    cpx<double>* Hs = nullptr;
    cpx<double>* Rs = nullptr;
    CU(cudaMallocAsync((void**)&Hs, (size_t)off[nbox] * sizeof(cpx<double>), h->stream));
    CU(cudaMallocAsync((void**)&Rs, (size_t)off[nbox] * sizeof(cpx<double>), h->stream));
    if (h->prm.op_mode == 0)
        k_sai_normal<T, 0><<<nbox, 256, 0, h->stream>>>(h->d_leaf_start, h->d_near_ptr, h->d_near_src, h->d_near_blk,
                                                       h->d_near_col0, h->d_near_ncol, d_tr, (const cpx<T>*)h->d_near,
                                                       h->d_gram_ptr, h->d_gram_seg, (const T*)h->d_gram_val, h->sai_off,
                                                       Hs, Rs);
    else
        k_sai_normal<T, 1><<<nbox, 256, 0, h->stream>>>(h->d_leaf_start, h->d_near_ptr, h->d_near_src, h->d_near_blk,
                                                       h->d_near_col0, h->d_near_ncol, d_tr, (const cpx<T>*)h->d_near,
                                                       nullptr, nullptr, nullptr, h->sai_off, Hs, Rs);
    CU(cudaGetLastError());
    k_sai_solve<T><<<nbox, 256, 0, h->stream>>>(h->d_leaf_start, NX, h->sai_off, Hs, Rs, (cpx<T>*)h->d_sai);
    CU(cudaGetLastError());
    CU(cudaFreeAsync(Hs, h->stream));
    CU(cudaFreeAsync(Rs, h->stream));
}

}  // namespace

void bi_build_sai(bi_handle_s* h) {
    if (h->prm.precond != 1) return;
    auto t0 = std::chrono::steady_clock::now();
    if (h->prec == 0) build_t<double>(h);
    else build_t<float>(h);
    CU(cudaStreamSynchronize(h->stream));
    h->info.setup_sai_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

void bi_sai_apply(bi_handle_s* h, const void* x, void* y, int R, cudaStream_t s) {
    const int nbox = (int)h->leaf_start.size() - 1;
    const size_t smem = (size_t)h->nX * h->max_leaf_count * R * h->csize;
    if (h->prec == 0) {
        bi_raise_smem(k_sai_apply<double>, smem);
        k_sai_apply<double><<<nbox, 128, smem, s>>>(h->N, h->nun, h->nX, R, h->d_perm, h->d_leaf_start, h->sai_off,
                                                    (const cpx<double>*)h->d_sai, (const cpx<double>*)x, (cpx<double>*)y);
    } else {
        bi_raise_smem(k_sai_apply<float>, smem);
        k_sai_apply<float><<<nbox, 128, smem, s>>>(h->N, h->nun, h->nX, R, h->d_perm, h->d_leaf_start, h->sai_off,
                                                   (const cpx<float>*)h->d_sai, (const cpx<float>*)x, (cpx<float>*)y);
    }
    CU(cudaGetLastError());
}
