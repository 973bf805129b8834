// Plane-wave right-hand sides (Eqs. 49-50) and the device-resident restarted GMRES
// (Saad and Schultz 1986) used by the hybrid solver of Sec. II.E.
//
// GMRES: x0 = 0, Arnoldi with classical Gram-Schmidt applied twice (numerically as
// robust as modified Gram-Schmidt, and two batched kernels per pass instead of j),
// FP64 basis, Hessenberg and Givens rotations, every right-hand side advanced in the
// same batched matvec; a column stops updating once its residual estimate is <= tol.
#include <algorithm>
#include <cmath>
#include <vector>

#include "bi_internal.h"

namespace {

struct z2 {
    double x, y;
};

// ------------------------------------------------------------------ plane-wave RHS
// b^J_m = <f_m, E/2 + n x H/2>, b^M_m = <f_m, H/2 - n x E/2>, E = p e, H = (k x p) e, e = exp(-jk khat.r)
template <typename T>
__global__ void k_rhs(int N, int nX, int nun, int nrhs, const int* __restrict__ perm, const int* __restrict__ rwg_t,
                      const int* __restrict__ rwg_l, const double* __restrict__ rwg_len, const double* __restrict__ tri,
                      const double* __restrict__ nrm, const double* __restrict__ area, const double* __restrict__ kp, double k,
                      int two_region, T* __restrict__ b) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * nrhs) return;
    int t = idx % N, s = idx / N;
    const double* kh = kp + 6 * s;
    const double* ph = kp + 6 * s + 3;
    double hp[3] = {kh[1] * ph[2] - kh[2] * ph[1], kh[2] * ph[0] - kh[0] * ph[2], kh[0] * ph[1] - kh[1] * ph[0]};
    const double s15 = 3.872983346207417;
    const double a1 = (6.0 - s15) / 21.0, a2 = (6.0 + s15) / 21.0;
    double bJr = 0, bJi = 0, bMr = 0, bMi = 0;
    for (int side = 0; side < 2; ++side) {
        int tr = rwg_t[2 * t + side], l = rwg_l[2 * t + side];
        const double* P = tri + 9 * tr;
        const double* n = nrm + 3 * tr;
        double cf = (side == 0 ? 1.0 : -1.0) * rwg_len[t] / (2.0 * area[tr]) * area[tr];
        double nE[3] = {n[1] * ph[2] - n[2] * ph[1], n[2] * ph[0] - n[0] * ph[2], n[0] * ph[1] - n[1] * ph[0]};
        double nH[3] = {n[1] * hp[2] - n[2] * hp[1], n[2] * hp[0] - n[0] * hp[2], n[0] * hp[1] - n[1] * hp[0]};
        for (int q = 0; q < 7; ++q) {
            double bb[3], w;
            if (q == 0) { bb[0] = bb[1] = bb[2] = 1.0 / 3.0; w = 9.0 / 40.0; }
            else {
                double a = (q <= 3) ? a1 : a2;
                w = (q <= 3) ? (155.0 - s15) / 1200.0 : (155.0 + s15) / 1200.0;
                bb[0] = bb[1] = bb[2] = a;
                bb[(q - 1) % 3] = 1.0 - 2.0 * a;
            }
            double r[3], f[3];
            for (int d = 0; d < 3; ++d) {
                r[d] = bb[0] * P[d] + bb[1] * P[3 + d] + bb[2] * P[6 + d];
                f[d] = cf * w * (r[d] - P[3 * l + d]);
            }
            double sn, cs;
            sincos(-k * (kh[0] * r[0] + kh[1] * r[1] + kh[2] * r[2]), &sn, &cs);
            double vJ, vM;
            if (two_region) {   // -<f, E_inc>, -<f, H_inc>: tangential E and H matched across the surface
                vJ = -(f[0] * ph[0] + f[1] * ph[1] + f[2] * ph[2]);
                vM = -(f[0] * hp[0] + f[1] * hp[1] + f[2] * hp[2]);
            } else {
                vJ = 0.5 * (f[0] * (ph[0] + nH[0]) + f[1] * (ph[1] + nH[1]) + f[2] * (ph[2] + nH[2]));
                vM = 0.5 * (f[0] * (hp[0] - nE[0]) + f[1] * (hp[1] - nE[1]) + f[2] * (hp[2] - nE[2]));
            }
            bJr += vJ * cs; bJi += vJ * sn;
            bMr += vM * cs; bMi += vM * sn;
        }
    }
    int u = perm[t];
    int64_t o = (int64_t)s * nun + u;
    b[2 * o] = (T)bJr;
    b[2 * o + 1] = (T)bJi;
    if (nX == 2) {
        b[2 * (o + N)] = (T)bMr;
        b[2 * (o + N) + 1] = (T)bMi;
    }
}

// ------------------------------------------------------------------ GMRES kernels
template <typename T>
__global__ void k_cvt_to(int64_t n, const z2* __restrict__ a, T* __restrict__ b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { b[2 * i] = (T)a[i].x; b[2 * i + 1] = (T)a[i].y; }
}
template <typename T>
__global__ void k_cvt_from(int64_t n, const T* __restrict__ a, z2* __restrict__ b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = z2{(double)a[2 * i], (double)a[2 * i + 1]};
}

// out[i][r] = sum_n conj(V_i[r][n]) w[r][n], one CTA per (i, r)
__global__ void k_dots(int nun, int R, const z2* __restrict__ V, int64_t vstride, const z2* __restrict__ w, z2* __restrict__ out) {
    int i = blockIdx.y, r = blockIdx.x;
    const z2* v = V + (int64_t)i * vstride + (int64_t)r * nun;
    const z2* ww = w + (int64_t)r * nun;
    double sx = 0, sy = 0;
    for (int n = threadIdx.x; n < nun; n += blockDim.x) {
        z2 a = v[n], b = ww[n];
        sx += a.x * b.x + a.y * b.y;
        sy += a.x * b.y - a.y * b.x;
    }
    __shared__ double bx[256], by[256];
    bx[threadIdx.x] = sx;
    by[threadIdx.x] = sy;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) { bx[threadIdx.x] += bx[threadIdx.x + s]; by[threadIdx.x] += by[threadIdx.x + s]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[(int64_t)i * R + r] = z2{bx[0], by[0]};
}

// w[r][n] -= sum_{i<nv} V_i[r][n] c[i][r]
__global__ void k_orth_update(int nun, int R, int nv, const z2* __restrict__ V, int64_t vstride, const z2* __restrict__ c,
                              z2* __restrict__ w) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nun * R) return;
    int r = (int)(idx / nun);
    z2 acc = w[idx];
    for (int i = 0; i < nv; ++i) {
        z2 v = V[(int64_t)i * vstride + idx], h = c[(int64_t)i * R + r];
        acc.x -= v.x * h.x - v.y * h.y;
        acc.y -= v.x * h.y + v.y * h.x;
    }
    w[idx] = acc;
}

__global__ void k_norms(int nun, const z2* __restrict__ w, double* __restrict__ out) {
    int r = blockIdx.x;
    const z2* ww = w + (int64_t)r * nun;
    double s = 0;
    for (int n = threadIdx.x; n < nun; n += blockDim.x) s += ww[n].x * ww[n].x + ww[n].y * ww[n].y;
    __shared__ double b[256];
    b[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) b[threadIdx.x] += b[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[r] = sqrt(b[0]);
}

__global__ void k_scale_into(int nun, int R, const z2* __restrict__ w, const double* __restrict__ nrm, z2* __restrict__ v) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nun * R) return;
    int r = (int)(idx / nun);
    double s = nrm[r] > 0 ? 1.0 / nrm[r] : 0.0;
    v[idx] = z2{w[idx].x * s, w[idx].y * s};
}

// Hessenberg column j for every RHS: H[r][i][j] (i <= j+1), Givens rotations (cs real, sn complex),
// g[r][.] and the residual estimate |g[j+1]|.
__global__ void k_givens(int R, int m, int j, const z2* __restrict__ hcol, const double* __restrict__ hnext, z2* __restrict__ H,
                         double* __restrict__ cs, z2* __restrict__ sn, z2* __restrict__ g, double* __restrict__ res,
                         const int* __restrict__ active) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R || !active[r]) return;
    z2* Hr = H + (int64_t)r * (m + 1) * m;
    for (int i = 0; i <= j; ++i) Hr[i * m + j] = hcol[(int64_t)i * R + r];
    Hr[(j + 1) * m + j] = z2{hnext[r], 0.0};
    // previous rotations: [c  s; -conj(s) c] acting on (h_i, h_{i+1})
    for (int i = 0; i < j; ++i) {
        double c = cs[r * m + i];
        z2 s = sn[r * m + i];
        z2 a = Hr[i * m + j], b = Hr[(i + 1) * m + j];
        z2 na = {c * a.x + s.x * b.x - s.y * b.y, c * a.y + s.x * b.y + s.y * b.x};
        z2 nb = {-(s.x * a.x + s.y * a.y) + c * b.x, -(s.x * a.y - s.y * a.x) + c * b.y};
        Hr[i * m + j] = na;
        Hr[(i + 1) * m + j] = nb;
    }
    z2 a = Hr[j * m + j], b = Hr[(j + 1) * m + j];
    double na = sqrt(a.x * a.x + a.y * a.y), nb = sqrt(b.x * b.x + b.y * b.y);
    double c;
    z2 s;
    if (nb == 0.0) { c = 1.0; s = z2{0, 0}; }
    else if (na == 0.0) { c = 0.0; s = z2{b.x / nb, -b.y / nb}; }   // s = conj(b)/|b|
    else {
        double t = sqrt(na * na + nb * nb);
        c = na / t;
        // s = (a/|a|) conj(b) / t
        z2 u = {a.x / na, a.y / na};
        s = z2{(u.x * b.x + u.y * b.y) / t, (u.y * b.x - u.x * b.y) / t};
    }
    cs[r * m + j] = c;
    sn[r * m + j] = s;
    z2 rnew = {c * a.x + s.x * b.x - s.y * b.y, c * a.y + s.x * b.y + s.y * b.x};
    Hr[j * m + j] = rnew;
    Hr[(j + 1) * m + j] = z2{0, 0};
    z2* gr = g + (int64_t)r * (m + 1);
    z2 gj = gr[j];
    gr[j] = z2{c * gj.x, c * gj.y};
    gr[j + 1] = z2{-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x)};
    res[r] = sqrt(gr[j + 1].x * gr[j + 1].x + gr[j + 1].y * gr[j + 1].y);
}

// back substitution y = H^-1 g on the first nk[r] columns
__global__ void k_backsolve(int R, int m, const z2* __restrict__ H, const z2* __restrict__ g, const int* __restrict__ nk,
                            z2* __restrict__ y) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const z2* Hr = H + (int64_t)r * (m + 1) * m;
    const z2* gr = g + (int64_t)r * (m + 1);
    z2* yr = y + (int64_t)r * m;
    int n = nk[r];
    for (int i = n - 1; i >= 0; --i) {
        z2 s = gr[i];
        for (int q = i + 1; q < n; ++q) {
            z2 h = Hr[i * m + q], v = yr[q];
            s.x -= h.x * v.x - h.y * v.y;
            s.y -= h.x * v.y + h.y * v.x;
        }
        z2 d = Hr[i * m + i];
        double dd = d.x * d.x + d.y * d.y;
        yr[i] = dd > 0 ? z2{(s.x * d.x + s.y * d.y) / dd, (s.y * d.x - s.x * d.y) / dd} : z2{0, 0};
    }
}

// x[r] += sum_{i < nk[r]} y[r][i] V_i[r]
__global__ void k_update_x(int nun, int R, int m, const z2* __restrict__ V, int64_t vstride, const z2* __restrict__ y,
                           const int* __restrict__ nk, z2* __restrict__ x) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nun * R) return;
    int r = (int)(idx / nun);
    z2 acc = x[idx];
    for (int i = 0; i < nk[r]; ++i) {
        z2 v = V[(int64_t)i * vstride + idx], c = y[(int64_t)r * m + i];
        acc.x += v.x * c.x - v.y * c.y;
        acc.y += v.x * c.y + v.y * c.x;
    }
    x[idx] = acc;
}

__global__ void k_residual(int64_t n, const z2* __restrict__ b, const z2* __restrict__ ax, z2* __restrict__ r) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = z2{b[i].x - ax[i].x, b[i].y - ax[i].y};
}

inline unsigned nb(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void bi_rhs_launch(bi_handle_s* h, const double* khat, const double* phat, int nrhs, void* b) {
    std::vector<double> kp(6 * (size_t)nrhs);
    for (int s = 0; s < nrhs; ++s)
        for (int d = 0; d < 3; ++d) {
            kp[6 * s + d] = khat[3 * s + d];
            kp[6 * s + 3 + d] = phat[3 * s + d];
        }
    double* d_kp = (double*)h->alloc(kp.size() * sizeof(double));
    CU(cudaMemcpy(d_kp, kp.data(), kp.size() * sizeof(double), cudaMemcpyHostToDevice));
    int tot = h->N * nrhs;
    if (h->prec == 0)
        k_rhs<double><<<nb(tot, 128), 128, 0, h->stream>>>(h->N, h->nX, h->nun, nrhs, h->d_perm, h->d_rwg_t, h->d_rwg_l,
                                                            h->d_rwg_len, h->d_tri, h->d_tri_n, h->d_tri_area, d_kp, h->k,
                                                            h->prm.op_mode == 3, (double*)b);
    else
        k_rhs<float><<<nb(tot, 128), 128, 0, h->stream>>>(h->N, h->nX, h->nun, nrhs, h->d_perm, h->d_rwg_t, h->d_rwg_l,
                                                           h->d_rwg_len, h->d_tri, h->d_tri_n, h->d_tri_area, d_kp, h->k,
                                                           h->prm.op_mode == 3, (float*)b);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(h->stream));
    // the small parameter buffer is released with the handle's other scratch at bi_destroy
}

// ---------------------------------------------------------------------------------
// Resumable GMRES: one context per solve.  The serving loop interleaves the iterations of
// many contexts (each on its own stream); bi_solve drives one context synchronously.
namespace {
__global__ void k_add_inplace(int64_t n, z2* __restrict__ a, const z2* __restrict__ b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { a[i].x += b[i].x; a[i].y += b[i].y; }
}
}  // namespace

struct gmres_ctx_impl {
    bi_handle_s* h = nullptr;
    int R = 1, m = 1, maxit = 1;
    std::vector<double> tolv;           // per-column tolerance
    int64_t nun = 0, nv = 0;
    cudaStream_t s = nullptr;
    std::vector<void*> mem;
    z2 *V = nullptr, *w = nullptr, *b64 = nullptr, *x64 = nullptr, *hc = nullptr, *hc2 = nullptr, *H = nullptr,
       *g = nullptr, *yv = nullptr, *sn = nullptr;
    double *cs = nullptr, *nrm = nullptr, *res = nullptr;
    int *act = nullptr, *nk = nullptr;
    void *xin = nullptr, *yout = nullptr;
    void* zbuf = nullptr;               // M v in the handle precision (right preconditioner)
    double* h_res = nullptr;  // pinned
    cudaEvent_t ev = nullptr;
    std::vector<double> bnorm, last_true;
    std::vector<int> done, its, a, kcols;
    int j = 0, total = 0;
    bool in_cycle = false, finished = false;
    int64_t bytes = 0;

    // Stream-ordered allocations on the context's stream: creating and freeing a context does
    // not synchronise the device, so the contexts of concurrent solves (the server) come and go
    // while other solves' kernels run.
    void* A(size_t n) {
        void* p = nullptr;
        CU(cudaMallocAsync(&p, n, s));
        mem.push_back(p);
        bytes += (int64_t)n;
        return p;
    }
    ~gmres_ctx_impl() {
        for (void* p : mem) cudaFreeAsync(p, s);
        if (h_res) cudaFreeHost(h_res);
        if (ev) cudaEventDestroy(ev);
    }
    static int64_t estimate_bytes(int64_t nun, int R, int m) {
        return (int64_t)sizeof(z2) * nun * R * (m + 5) + (int64_t)R * (m + 2) * (m + 4) * 32 + 2 * nun * R * 16;
    }
    // out = A M in (M the right preconditioner when the handle has one, else the identity)
    void matvec64(const z2* in, z2* out) {
        const int th = 256;
        if (h->prec == 0) k_cvt_to<double><<<nb(nv, th), th, 0, s>>>(nv, in, (double*)xin);
        else k_cvt_to<float><<<nb(nv, th), th, 0, s>>>(nv, in, (float*)xin);
        // the operator of Eq. 52 when a coupling is set, else C
        if (h->d_sai) {
            bi_sai_apply(h, xin, zbuf, R, s);
            bi_operator_launch(h, zbuf, yout, R, s);
        } else {
            bi_operator_launch(h, xin, yout, R, s);
        }
        if (h->prec == 0) k_cvt_from<double><<<nb(nv, th), th, 0, s>>>(nv, (const double*)yout, out);
        else k_cvt_from<float><<<nb(nv, th), th, 0, s>>>(nv, (const float*)yout, out);
    }
    // allocate, x0 = 0, |b| (synchronises the stream once)
    void init(bi_handle_s* hh, const void* rhs, int nrhs, const double* tol_, cudaStream_t st, void* xin_,
              void* yout_) {
        h = hh;
        R = nrhs;
        tolv.assign(tol_, tol_ + nrhs);
        s = st;
        m = std::max(1, h->prm.gmres_restart);
        maxit = std::max(1, h->prm.gmres_maxit);
        nun = h->nun;
        nv = nun * R;
        V = (z2*)A(sizeof(z2) * nv * (m + 1));
        w = (z2*)A(sizeof(z2) * nv);
        b64 = (z2*)A(sizeof(z2) * nv);
        x64 = (z2*)A(sizeof(z2) * nv);
        hc = (z2*)A(sizeof(z2) * (size_t)(m + 1) * R);
        hc2 = (z2*)A(sizeof(z2) * (size_t)(m + 1) * R);
        H = (z2*)A(sizeof(z2) * (size_t)R * (m + 1) * m);
        g = (z2*)A(sizeof(z2) * (size_t)R * (m + 1));
        yv = (z2*)A(sizeof(z2) * (size_t)R * m);
        cs = (double*)A(sizeof(double) * (size_t)R * m);
        sn = (z2*)A(sizeof(z2) * (size_t)R * m);
        nrm = (double*)A(sizeof(double) * R);
        res = (double*)A(sizeof(double) * R);
        act = (int*)A(sizeof(int) * R);
        nk = (int*)A(sizeof(int) * R);
        xin = xin_ ? xin_ : A(h->csize * nv);
        yout = yout_ ? yout_ : A(h->csize * nv);
        if (h->d_sai) zbuf = A(h->csize * nv);
        CU(cudaMallocHost(&h_res, sizeof(double) * 2 * R));
        CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        const int th = 256;
        if (h->prec == 0) k_cvt_from<double><<<nb(nv, th), th, 0, s>>>(nv, (const double*)rhs, b64);
        else k_cvt_from<float><<<nb(nv, th), th, 0, s>>>(nv, (const float*)rhs, b64);
        CU(cudaMemsetAsync(x64, 0, sizeof(z2) * nv, s));
        k_norms<<<R, 256, 0, s>>>(nun, b64, nrm);
        bnorm.assign(R, 0.0);
        CU(cudaMemcpyAsync(bnorm.data(), nrm, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        last_true.assign(R, 1e300);
        done.assign(R, 0);
        its.assign(R, 0);
        a.assign(R, 0);
        kcols.assign(R, 0);
        for (int r = 0; r < R; ++r)
            if (bnorm[r] == 0.0) done[r] = 1;
    }
    // Start a restart cycle from the true residual; false when no column is left to solve.
    bool start_cycle() {
        const int th = 256;
        if (total >= maxit) return false;
        matvec64(x64, w);
        k_residual<<<nb(nv, th), th, 0, s>>>(nv, b64, w, w);
        k_norms<<<R, 256, 0, s>>>(nun, w, nrm);
        k_scale_into<<<nb(nv, th), th, 0, s>>>(nun, R, w, nrm, V);
        std::vector<double> beta(R);
        CU(cudaMemcpyAsync(beta.data(), nrm, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        std::vector<z2> g0((size_t)R * (m + 1), z2{0, 0});
        bool any_left = false;
        for (int r = 0; r < R; ++r) {
            g0[(size_t)r * (m + 1)] = z2{beta[r], 0};
            double rel = beta[r] / std::max(bnorm[r], 1e-300);
            // the true residual decides; a column whose true residual did not drop over a
            // whole cycle by 1% has stagnated (matvec rounding floor) and stops
            if (bnorm[r] == 0.0 || rel <= tolv[r]) done[r] = 1;
            else if (done[r] == 0 && rel > 0.99 * last_true[r]) done[r] = 2;
            else if (done[r] == 1) done[r] = 0;
            last_true[r] = rel;
            a[r] = (done[r] == 0);
            kcols[r] = 0;
            any_left = any_left || a[r];
        }
        if (!any_left) return false;
        CU(cudaMemcpyAsync(g, g0.data(), sizeof(z2) * g0.size(), cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(act, a.data(), sizeof(int) * R, cudaMemcpyHostToDevice, s));
        CU(cudaStreamSynchronize(s));
        j = 0;
        in_cycle = true;
        return true;
    }
    // Queue one Arnoldi step (classical Gram-Schmidt twice, FP64) and the Givens update; the
    // residual estimates are copied to pinned memory and `ev` marks completion.
    void enqueue_iteration() {
        const int th = 256;
        matvec64(V + (int64_t)j * nv, w);
        k_dots<<<dim3(R, j + 1), 256, 0, s>>>(nun, R, V, nv, w, hc);
        k_orth_update<<<nb(nv, th), th, 0, s>>>(nun, R, j + 1, V, nv, hc, w);
        k_dots<<<dim3(R, j + 1), 256, 0, s>>>(nun, R, V, nv, w, hc2);
        k_orth_update<<<nb(nv, th), th, 0, s>>>(nun, R, j + 1, V, nv, hc2, w);
        k_add_inplace<<<nb((int64_t)(j + 1) * R, 128), 128, 0, s>>>((int64_t)(j + 1) * R, hc, hc2);
        k_norms<<<R, 256, 0, s>>>(nun, w, nrm);
        k_scale_into<<<nb(nv, th), th, 0, s>>>(nun, R, w, nrm, V + (int64_t)(j + 1) * nv);
        k_givens<<<nb(R, 64), 64, 0, s>>>(R, m, j, hc, nrm, H, cs, sn, g, res, act);
        CU(cudaMemcpyAsync(h_res, res, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
        CU(cudaEventRecord(ev, s));
        CU(cudaGetLastError());
    }
    bool iteration_ready() {
        cudaError_t e = cudaEventQuery(ev);
        if (e == cudaErrorNotReady) return false;
        CU(e);
        return true;
    }
    // Host update after an iteration completed; true when the cycle must end.
    bool complete_iteration() {
        ++total;
        bool any = false;
        for (int r = 0; r < R; ++r)
            if (a[r]) {
                kcols[r] = j + 1;
                its[r] += 1;
                if (h_res[r] / std::max(bnorm[r], 1e-300) <= tolv[r]) a[r] = 0;
                any = any || a[r];
            }
        ++j;
        if (any) CU(cudaMemcpyAsync(act, a.data(), sizeof(int) * R, cudaMemcpyHostToDevice, s));
        return !any || j >= m || total >= maxit;
    }
    // x += V y for the columns of this cycle (queued)
    void end_cycle() {
        const int th = 256;
        CU(cudaMemcpyAsync(nk, kcols.data(), sizeof(int) * R, cudaMemcpyHostToDevice, s));
        k_backsolve<<<nb(R, 64), 64, 0, s>>>(R, m, H, g, nk, yv);
        k_update_x<<<nb(nv, th), th, 0, s>>>(nun, R, m, V, nv, yv, nk, x64);
        CU(cudaGetLastError());
        CU(cudaStreamSynchronize(s));
        in_cycle = false;
    }
    // True residual, x out (device, handle precision); synchronises.
    int finish(void* xout, int* iters, double* relres) {
        const int th = 256;
        matvec64(x64, w);
        k_residual<<<nb(nv, th), th, 0, s>>>(nv, b64, w, w);
        k_norms<<<R, 256, 0, s>>>(nun, w, nrm);
        std::vector<double> rr(R);
        CU(cudaMemcpyAsync(rr.data(), nrm, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
        // x = M u (the iterate lives in the preconditioned variable)
        void* xdst = h->d_sai ? zbuf : xout;
        if (h->prec == 0) k_cvt_to<double><<<nb(nv, th), th, 0, s>>>(nv, x64, (double*)xdst);
        else k_cvt_to<float><<<nb(nv, th), th, 0, s>>>(nv, x64, (float*)xdst);
        if (h->d_sai) bi_sai_apply(h, zbuf, xout, R, s);
        CU(cudaStreamSynchronize(s));
        int status = bi_take_device_status(h);
        for (int r = 0; r < R; ++r) {
            double rel = bnorm[r] > 0 ? rr[r] / bnorm[r] : 0.0;
            if (iters) iters[r] = its[r];
            if (relres) relres[r] = rel;
            if (status == BI_OK && rel > tolv[r] * 1.0001 + 1e-12) status = BI_ERR_NOT_CONVERGED;
        }
        finished = true;
        return status;
    }
};

gmres_ctx* bi_gmres_create(bi_handle_s* h, const void* rhs, int nrhs, const double* tol, cudaStream_t s) {
    gmres_ctx_impl* c = new gmres_ctx_impl();
    try {
        c->init(h, rhs, nrhs, tol, s, nullptr, nullptr);
    } catch (...) {
        delete c;
        throw;
    }
    return reinterpret_cast<gmres_ctx*>(c);
}
void bi_gmres_destroy(gmres_ctx* c) { delete reinterpret_cast<gmres_ctx_impl*>(c); }
int64_t bi_gmres_bytes(gmres_ctx* c) { return reinterpret_cast<gmres_ctx_impl*>(c)->bytes; }
int64_t bi_gmres_estimate_bytes(int64_t nun, int R, int m) { return gmres_ctx_impl::estimate_bytes(nun, R, m); }

// Advance a context without blocking on other work: returns 1 when the solve is finished
// (then bi_gmres_finish), 0 when it needs more calls.
int bi_gmres_advance(gmres_ctx* cc) {
    gmres_ctx_impl* c = reinterpret_cast<gmres_ctx_impl*>(cc);
    if (c->finished) return 1;
    if (!c->in_cycle) {
        if (!c->start_cycle()) return 1;
        c->enqueue_iteration();
        return 0;
    }
    if (!c->iteration_ready()) return 0;
    if (c->complete_iteration()) {
        c->end_cycle();
        return 0;
    }
    c->enqueue_iteration();
    return 0;
}
int bi_gmres_finish(gmres_ctx* cc, void* xout, int* iters, double* relres) {
    return reinterpret_cast<gmres_ctx_impl*>(cc)->finish(xout, iters, relres);
}

int bi_gmres(bi_handle_s* h, const void* rhs, void* xout, int R, double tol, int* iters, double* relres) {
    gmres_ctx_impl c;
    const std::vector<double> tolv(R, tol);
    c.init(h, rhs, R, tolv.data(), h->stream, h->d_sx, h->d_sy);
    while (c.start_cycle()) {
        for (;;) {
            c.enqueue_iteration();
            CU(cudaEventSynchronize(c.ev));
            if (c.complete_iteration()) break;
        }
        c.end_cycle();
    }
    return c.finish(xout, iters, relres);
}

// ---------------------------------------------------------------------------------
// Mixed-precision iterative refinement: the working handle's GMRES (FP32 products) solves the
// correction equation C d = r to a loose tolerance, d is added to x in FP64, and the residual
// r = b - C x is recomputed with an FP64 handle of the same operator.  The working product's
// rounding floor (about 1e-4 in FP32) then limits only the inner solves, not the solution.
namespace {
template <typename T>
__global__ void k_add_to64(int64_t n, const T* __restrict__ d, z2* __restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        x[i].x += (double)d[2 * i];
        x[i].y += (double)d[2 * i + 1];
    }
}
}  // namespace

int bi_solve_refined_impl(bi_handle_s* h, bi_handle_s* href, const void* rhs, void* xout, int R, double tol, int* iters,
                          double* relres) {
    const int64_t nun = h->nun, nv = nun * R;
    const int th = 256;
    cudaStream_t s = href->stream;
    std::vector<void*> bufs;
    auto A = [&](size_t bytes) {
        void* p = nullptr;
        CU(cudaMalloc(&p, bytes));
        bufs.push_back(p);
        return p;
    };
    int status = BI_OK;
    try {
        z2* b = (z2*)rhs;
        z2* x = (z2*)xout;
        z2* r = (z2*)A(sizeof(z2) * nv);
        z2* ax = (z2*)A(sizeof(z2) * nv);
        void* rl = A(h->csize * nv);
        void* d = A(h->csize * nv);
        double* nrm = (double*)A(sizeof(double) * R);
        std::vector<double> bn(R), rn(R);
        CU(cudaMemsetAsync(x, 0, sizeof(z2) * nv, s));
        CU(cudaMemcpyAsync(r, b, sizeof(z2) * nv, cudaMemcpyDeviceToDevice, s));
        k_norms<<<R, 256, 0, s>>>((int)nun, b, nrm);
        CU(cudaMemcpyAsync(bn.data(), nrm, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        std::vector<int> its(R, 0), it1(R);
        std::vector<double> rel1(R);
        rn = bn;
        for (int step = 0; step < 20; ++step) {
            bool done = true;
            for (int c = 0; c < R; ++c) done = done && (bn[c] == 0.0 || rn[c] <= tol * bn[c]);
            if (done) break;
            // C d = r in the working precision, to 1e-3 of r (above its rounding floor)
            if (h->prec == 0) k_cvt_to<double><<<nb(nv, th), th, 0, s>>>(nv, r, (double*)rl);
            else k_cvt_to<float><<<nb(nv, th), th, 0, s>>>(nv, r, (float*)rl);
            CU(cudaGetLastError());
            CU(cudaStreamSynchronize(s));
            const int st = bi_gmres(h, rl, d, R, 1e-3, it1.data(), rel1.data());
            if (st != BI_OK && st != BI_ERR_NOT_CONVERGED) throw bi_error{st, h->err};
            for (int c = 0; c < R; ++c) its[c] += it1[c];
            CU(cudaStreamSynchronize(h->stream));
            if (h->prec == 0) k_add_to64<double><<<nb(nv, th), th, 0, s>>>(nv, (const double*)d, x);
            else k_add_to64<float><<<nb(nv, th), th, 0, s>>>(nv, (const float*)d, x);
            CU(cudaGetLastError());
            // r = b - C x with the FP64 product
            bi_operator_launch(href, x, ax, R, s);
            k_residual<<<nb(nv, th), th, 0, s>>>(nv, b, ax, r);
            k_norms<<<R, 256, 0, s>>>((int)nun, r, nrm);
            CU(cudaMemcpyAsync(rn.data(), nrm, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
        }
        status = bi_take_device_status(href);
        if (status == BI_OK) status = bi_take_device_status(h);
        for (int c = 0; c < R; ++c) {
            const double rel = bn[c] > 0 ? rn[c] / bn[c] : 0.0;
            if (iters) iters[c] = its[c];
            if (relres) relres[c] = rel;
            if (status == BI_OK && rel > tol * 1.0001 + 1e-15) status = BI_ERR_NOT_CONVERGED;
        }
    } catch (...) {
        for (void* p : bufs) cudaFree(p);
        throw;
    }
    for (void* p : bufs) cudaFree(p);
    return status;
}

