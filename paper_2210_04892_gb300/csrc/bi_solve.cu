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
                      T* __restrict__ b) {
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
            double vJ = 0.5 * (f[0] * (ph[0] + nH[0]) + f[1] * (ph[1] + nH[1]) + f[2] * (ph[2] + nH[2]));
            double vM = 0.5 * (f[0] * (hp[0] - nE[0]) + f[1] * (hp[1] - nE[1]) + f[2] * (hp[2] - nE[2]));
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
                                                            (double*)b);
    else
        k_rhs<float><<<nb(tot, 128), 128, 0, h->stream>>>(h->N, h->nX, h->nun, nrhs, h->d_perm, h->d_rwg_t, h->d_rwg_l,
                                                           h->d_rwg_len, h->d_tri, h->d_tri_n, h->d_tri_area, d_kp, h->k,
                                                           (float*)b);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(h->stream));
    // the small parameter buffer is released with the handle's other scratch at bi_destroy
}

int bi_gmres(bi_handle_s* h, const void* rhs, void* xout, int R, double tol, int* iters, double* relres) {
    const int nun = h->nun;
    const int m = std::max(1, h->prm.gmres_restart);
    const int maxit = std::max(1, h->prm.gmres_maxit);
    const int64_t nv = (int64_t)nun * R;
    cudaStream_t s = h->stream;
    // FP64 Krylov state (allocated per solve, released at the end)
    std::vector<void*> tmp;
    auto A = [&](size_t bytes) {
        void* p = nullptr;
        CU(cudaMalloc(&p, bytes));
        tmp.push_back(p);
        return p;
    };
    int status = BI_OK;
    try {
        z2* V = (z2*)A(sizeof(z2) * nv * (m + 1));
        z2* w = (z2*)A(sizeof(z2) * nv);
        z2* b64 = (z2*)A(sizeof(z2) * nv);
        z2* x64 = (z2*)A(sizeof(z2) * nv);
        z2* hc = (z2*)A(sizeof(z2) * (size_t)(m + 1) * R);
        z2* hc2 = (z2*)A(sizeof(z2) * (size_t)(m + 1) * R);
        z2* H = (z2*)A(sizeof(z2) * (size_t)R * (m + 1) * m);
        z2* g = (z2*)A(sizeof(z2) * (size_t)R * (m + 1));
        z2* yv = (z2*)A(sizeof(z2) * (size_t)R * m);
        double* cs = (double*)A(sizeof(double) * (size_t)R * m);
        z2* sn = (z2*)A(sizeof(z2) * (size_t)R * m);
        double* nrm = (double*)A(sizeof(double) * R);
        double* res = (double*)A(sizeof(double) * R);
        int* act = (int*)A(sizeof(int) * R);
        int* nk = (int*)A(sizeof(int) * R);
        // fixed staging buffers of the handle, so the captured matvec graph is reused
        void* xin = h->d_sx;
        void* yout = h->d_sy;
        const int th = 256;
        if (h->prec == 0) k_cvt_from<double><<<nb(nv, th), th, 0, s>>>(nv, (const double*)rhs, b64);
        else k_cvt_from<float><<<nb(nv, th), th, 0, s>>>(nv, (const float*)rhs, b64);
        CU(cudaMemsetAsync(x64, 0, sizeof(z2) * nv, s));
        k_norms<<<R, 256, 0, s>>>(nun, b64, nrm);
        std::vector<double> bnorm(R), rr(R);
        CU(cudaMemcpyAsync(bnorm.data(), nrm, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        std::vector<int> done(R, 0), its(R, 0);
        for (int r = 0; r < R; ++r)
            if (bnorm[r] == 0.0) done[r] = 1;
        auto matvec64 = [&](const z2* in, z2* out) {
            if (h->prec == 0) k_cvt_to<double><<<nb(nv, th), th, 0, s>>>(nv, in, (double*)xin);
            else k_cvt_to<float><<<nb(nv, th), th, 0, s>>>(nv, in, (float*)xin);
            bi_matvec_launch(h, xin, yout, R, s);
            if (h->prec == 0) k_cvt_from<double><<<nb(nv, th), th, 0, s>>>(nv, (const double*)yout, out);
            else k_cvt_from<float><<<nb(nv, th), th, 0, s>>>(nv, (const float*)yout, out);
        };
        int total = 0;
        std::vector<double> last_true(R, 1e300);
        while (total < maxit) {
            // r0 = b - A x
            matvec64(x64, w);
            k_residual<<<nb(nv, th), th, 0, s>>>(nv, b64, w, w);
            k_norms<<<R, 256, 0, s>>>(nun, w, nrm);
            k_scale_into<<<nb(nv, th), th, 0, s>>>(nun, R, w, nrm, V);
            std::vector<double> beta(R);
            CU(cudaMemcpyAsync(beta.data(), nrm, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            std::vector<z2> g0((size_t)R * (m + 1), z2{0, 0});
            std::vector<int> a(R), kcols(R, 0);
            // the true residual decides at every restart; a column whose true residual did not
            // drop by 10% over a whole cycle has stagnated (matvec rounding floor) and stops
            bool any_left = false;
            for (int r = 0; r < R; ++r) {
                g0[(size_t)r * (m + 1)] = z2{beta[r], 0};
                double rel = beta[r] / std::max(bnorm[r], 1e-300);
                if (bnorm[r] == 0.0 || rel <= tol) done[r] = 1;
                else if (done[r] == 0 && rel > 0.9 * last_true[r]) done[r] = 2;  // stagnated
                else if (done[r] == 1) done[r] = 0;                              // estimate was optimistic
                last_true[r] = rel;
                a[r] = (done[r] == 0);
                any_left = any_left || a[r];
            }
            if (!any_left) break;
            CU(cudaMemcpyAsync(g, g0.data(), sizeof(z2) * g0.size(), cudaMemcpyHostToDevice, s));
            CU(cudaMemcpyAsync(act, a.data(), sizeof(int) * R, cudaMemcpyHostToDevice, s));
            int j = 0;
            for (; j < m && total < maxit; ++j, ++total) {
                bool any = false;
                for (int r = 0; r < R; ++r) any = any || a[r];
                if (!any) break;
                matvec64(V + (int64_t)j * nv, w);
                // two passes of classical Gram-Schmidt
                k_dots<<<dim3(R, j + 1), 256, 0, s>>>(nun, R, V, nv, w, hc);
                k_orth_update<<<nb(nv, th), th, 0, s>>>(nun, R, j + 1, V, nv, hc, w);
                k_dots<<<dim3(R, j + 1), 256, 0, s>>>(nun, R, V, nv, w, hc2);
                k_orth_update<<<nb(nv, th), th, 0, s>>>(nun, R, j + 1, V, nv, hc2, w);
                // hc += hc2 (on the host side of the small arrays)
                std::vector<z2> h1((size_t)(j + 1) * R), h2((size_t)(j + 1) * R);
                CU(cudaMemcpyAsync(h1.data(), hc, sizeof(z2) * h1.size(), cudaMemcpyDeviceToHost, s));
                CU(cudaMemcpyAsync(h2.data(), hc2, sizeof(z2) * h2.size(), cudaMemcpyDeviceToHost, s));
                k_norms<<<R, 256, 0, s>>>(nun, w, nrm);
                k_scale_into<<<nb(nv, th), th, 0, s>>>(nun, R, w, nrm, V + (int64_t)(j + 1) * nv);
                CU(cudaStreamSynchronize(s));
                for (size_t q = 0; q < h1.size(); ++q) { h1[q].x += h2[q].x; h1[q].y += h2[q].y; }
                CU(cudaMemcpyAsync(hc, h1.data(), sizeof(z2) * h1.size(), cudaMemcpyHostToDevice, s));
                k_givens<<<nb(R, 64), 64, 0, s>>>(R, m, j, hc, nrm, H, cs, sn, g, res, act);
                CU(cudaMemcpyAsync(rr.data(), res, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
                CU(cudaStreamSynchronize(s));
                for (int r = 0; r < R; ++r)
                    if (a[r]) {
                        kcols[r] = j + 1;
                        its[r] += 1;
                        if (rr[r] / std::max(bnorm[r], 1e-300) <= tol) a[r] = 0;
                    }
                CU(cudaMemcpyAsync(act, a.data(), sizeof(int) * R, cudaMemcpyHostToDevice, s));
            }
            CU(cudaMemcpyAsync(nk, kcols.data(), sizeof(int) * R, cudaMemcpyHostToDevice, s));
            k_backsolve<<<nb(R, 64), 64, 0, s>>>(R, m, H, g, nk, yv);
            k_update_x<<<nb(nv, th), th, 0, s>>>(nun, R, m, V, nv, yv, nk, x64);
            CU(cudaStreamSynchronize(s));
        }
        // true residual
        matvec64(x64, w);
        k_residual<<<nb(nv, th), th, 0, s>>>(nv, b64, w, w);
        k_norms<<<R, 256, 0, s>>>(nun, w, nrm);
        CU(cudaMemcpyAsync(rr.data(), nrm, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
        if (h->prec == 0) k_cvt_to<double><<<nb(nv, th), th, 0, s>>>(nv, x64, (double*)xout);
        else k_cvt_to<float><<<nb(nv, th), th, 0, s>>>(nv, x64, (float*)xout);
        CU(cudaStreamSynchronize(s));
        for (int r = 0; r < R; ++r) {
            double rel = bnorm[r] > 0 ? rr[r] / bnorm[r] : 0.0;
            if (iters) iters[r] = its[r];
            if (relres) relres[r] = rel;
            if (rel > tol * 1.0001 + 1e-12) status = BI_ERR_NOT_CONVERGED;
        }
    } catch (...) {
        for (void* p : tmp) cudaFree(p);
        throw;
    }
    for (void* p : tmp) cudaFree(p);
    return status;
}
