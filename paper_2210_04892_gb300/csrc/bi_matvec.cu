// The matrix-vector product y = C x (step 2(a) of the hybrid solver, Sec. II.E) by a
// multilevel fast multipole algorithm.
//
// Far interactions use the plane-wave expansion of G = exp(-jkR)/(4 pi R) between
// well-separated boxes:
//   G(r, r') ~ (-jk / 16 pi^2) sum_khat w(khat) exp(-jk khat.(r - c_b)) T_L(khat; c_b - c_s) exp(+jk khat.(r' - c_s)).
// With F_n(khat) = int f_n exp(+jk khat.(r' - c)) (theta, phi components), R_m = conj(F_m)
// and RX_m(khat) = int (n x f_m) exp(-jk khat.(r - c)), the far parts of the operators
// of Eqs. 43-46 are
//   <f_m, L f_n> -> -jk c R_m.F_n,        <f_m, n x Kbar f_n> -> jk c RX_m.(khat x F_n),
//   <f_m, n x L f_n> -> jk c RX_m.F_n,    <f_m, Kbar f_n> -> -jk c R_m.(khat x F_n)     (c = -jk/16pi^2 with T, w).
// For the C block all four far blocks then depend on the single transverse field
//   U = sum_n ( -x_J,n F_n + x_M,n khat x F_n )
// (the part that radiates), so one two-component pattern per box and direction is
// aggregated, translated and disaggregated, and the leaf receive is
//   y_J,m = -(k^2/32 pi^2) sum_khat [ R_m.V - RX_m.(khat x V) ],
//   y_M,m = +(k^2/32 pi^2) sum_khat [ -R_m.(khat x V) - RX_m.V ],
// V the incoming field with the quadrature weights folded in.  The PEC mode is the
// J row with x_M = 0.
//
// Layouts (device): vectors in tree order [N][nX][R]; far-field patterns per level
// [box][direction][E] with E = 2 R (theta, phi) x RHS; directions theta-major.
#include <algorithm>
#include <cstdio>

#include "bi_internal.h"

namespace {

template <typename T>
struct cpx {
    T x, y;
};
template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {  // conj(a) * b
    return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) {
    return {a.x + b.x, a.y + b.y};
}
template <typename T>
__device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) {
    return {a.x - b.x, a.y - b.y};
}
template <typename T>
__device__ __forceinline__ cpx<T> cscale(cpx<T> a, T s) {
    return {a.x * s, a.y * s};
}
template <typename T>
__device__ __forceinline__ void cfma(cpx<T>& acc, cpx<T> a, cpx<T> b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
template <typename T>
__device__ __forceinline__ cpx<T> czero() {
    return {T(0), T(0)};
}

// ------------------------------------------------------------------ permutations
template <typename T>
__global__ void k_gather_x(int N, int nX, int R, int nun, const int* __restrict__ perm, const cpx<T>* __restrict__ x,
                           cpx<T>* __restrict__ xt) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t tot = (int64_t)N * nX * R;
    if (idx >= tot) return;
    int r = (int)(idx % R);
    int X = (int)((idx / R) % nX);
    int t = (int)(idx / ((int64_t)R * nX));
    xt[idx] = x[(int64_t)r * nun + (int64_t)X * N + perm[t]];
}

template <typename T>
__global__ void k_scatter_y(int N, int nX, int R, int nun, const int* __restrict__ perm, const cpx<T>* __restrict__ yt,
                            const cpx<T>* __restrict__ yf, cpx<T>* __restrict__ y) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t tot = (int64_t)N * nX * R;
    if (idx >= tot) return;
    int r = (int)(idx % R);
    int X = (int)((idx / R) % nX);
    int t = (int)(idx / ((int64_t)R * nX));
    cpx<T> v = yt[idx];
    if (yf) v = cadd(v, yf[idx]);
    y[(int64_t)r * nun + (int64_t)X * N + perm[t]] = v;
}

// ------------------------------------------------------------------ near field
// One CTA per test leaf box.  Thread (r, m) accumulates the row of RWG m for RHS r over
// the box's near blocks; blocks are column-major so consecutive m read consecutive entries.
//   C block:  y_J = -(A x_J + B x_M),  y_M = B x_J - A x_M + (X/2) x_J - (G/2) x_M
//   PEC:      y   = -A x
template <typename T, int MODE>
__global__ void __launch_bounds__(128) k_near(int R, const int* __restrict__ leaf_start, const int* __restrict__ near_ptr,
                                              const int* __restrict__ near_src, const int64_t* __restrict__ near_blk,
                                              const cpx<T>* __restrict__ blocks, const int* __restrict__ gptr,
                                              const int* __restrict__ gcol, const T* __restrict__ gval,
                                              const cpx<T>* __restrict__ xt, cpx<T>* __restrict__ yt) {
    const int b = blockIdx.x;
    const int m0 = leaf_start[b], mb = leaf_start[b + 1] - m0;
    const int nX = MODE == 0 ? 2 : 1;
    for (int idx = threadIdx.x; idx < mb * R; idx += blockDim.x) {
        const int ml = idx % mb, r = idx / mb;
        cpx<T> aJ = czero<T>(), aM = czero<T>();
        for (int q = near_ptr[b]; q < near_ptr[b + 1]; ++q) {
            const int s = near_src[q];
            const int n0 = leaf_start[s], nbs = leaf_start[s + 1] - n0;
            const int64_t base = near_blk[q];
            for (int nl = 0; nl < nbs; ++nl) {
                const int64_t e = base + (int64_t)nl * mb + ml;
                const int n = n0 + nl;
                if (MODE == 0) {
                    cpx<T> A = blocks[2 * e], B = blocks[2 * e + 1];
                    cpx<T> xJ = xt[((int64_t)n * 2 + 0) * R + r], xM = xt[((int64_t)n * 2 + 1) * R + r];
                    cfma(aJ, A, xJ);
                    cfma(aJ, B, xM);
                    cfma(aM, B, xJ);
                    cfma(aM, A, cpx<T>{-xM.x, -xM.y});
                } else {
                    cpx<T> A = blocks[e];
                    cpx<T> xJ = xt[(int64_t)n * R + r];
                    cfma(aJ, A, xJ);
                }
            }
        }
        const int m = m0 + ml;
        if (MODE == 0) {
            for (int q = gptr[m]; q < gptr[m + 1]; ++q) {
                const int n = gcol[q];
                const T g = gval[2 * q], x = gval[2 * q + 1];
                cpx<T> xJ = xt[((int64_t)n * 2 + 0) * R + r], xM = xt[((int64_t)n * 2 + 1) * R + r];
                aM.x += T(0.5) * (x * xJ.x - g * xM.x);
                aM.y += T(0.5) * (x * xJ.y - g * xM.y);
            }
            yt[((int64_t)m * 2 + 0) * R + r] = cpx<T>{-aJ.x, -aJ.y};
            yt[((int64_t)m * 2 + 1) * R + r] = aM;
        } else {
            yt[(int64_t)m * R + r] = cpx<T>{-aJ.x, -aJ.y};
        }
        (void)nX;
    }
}

// ------------------------------------------------------------------ leaf aggregation
// U_b(k) = sum_{n in b} ( -x_J,n F_n(k) + x_M,n khat x F_n(k) ),  (khat x F) = (-F_phi, F_theta)
template <typename T, int MODE>
__global__ void k_aggregate(int K, int R, const int* __restrict__ leaf_start, const cpx<T>* __restrict__ F,
                            const cpx<T>* __restrict__ xt, cpx<T>* __restrict__ U) {
    const int b = blockIdx.y;
    const int E = 2 * R;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)K * E) return;
    const int kk = (int)(idx / E), e = (int)(idx % E);
    const int c = e / R, r = e % R;
    cpx<T> acc = czero<T>();
    for (int n = leaf_start[b]; n < leaf_start[b + 1]; ++n) {
        cpx<T> Ft = F[((int64_t)n * K + kk) * 2 + 0], Fp = F[((int64_t)n * K + kk) * 2 + 1];
        if (MODE == 0) {
            cpx<T> xJ = xt[((int64_t)n * 2 + 0) * R + r], xM = xt[((int64_t)n * 2 + 1) * R + r];
            if (c == 0) {  // -xJ Ft - xM Fp
                acc = csub(acc, cmul(xJ, Ft));
                acc = csub(acc, cmul(xM, Fp));
            } else {       // -xJ Fp + xM Ft
                acc = csub(acc, cmul(xJ, Fp));
                acc = cadd(acc, cmul(xM, Ft));
            }
        } else {
            cpx<T> xJ = xt[(int64_t)n * R + r];
            acc = csub(acc, cmul(xJ, c == 0 ? Ft : Fp));
        }
    }
    U[((int64_t)b * K) * E + idx] = acc;
}

// ------------------------------------------------------------------ interpolation (upward)
// theta pass on great circles: tmp[cb][ip][jc][e] = sum_t w (+-) U_c[cb][src][jc or jc+half][e]
template <typename T>
__global__ void k_interp_theta(int nthp, int nphc, int Kc, int E, int pth, const int* __restrict__ src,
                               const int* __restrict__ flip, const T* __restrict__ w, const cpx<T>* __restrict__ Uc,
                               cpx<T>* __restrict__ tmp) {
    const int cb = blockIdx.y;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t tot = (int64_t)nthp * nphc * E;
    if (idx >= tot) return;
    const int e = (int)(idx % E);
    const int jc = (int)((idx / E) % nphc);
    const int ip = (int)(idx / ((int64_t)E * nphc));
    const int half = nphc / 2;
    const cpx<T>* u = Uc + (int64_t)cb * Kc * E;
    cpx<T> acc = czero<T>();
    for (int t = 0; t < pth; ++t) {
        const int i = src[ip * pth + t];
        const int f = flip[ip * pth + t];
        const int j = f ? (jc + half) % nphc : jc;
        const T ww = f ? -w[ip * pth + t] : w[ip * pth + t];
        cpx<T> v = u[((int64_t)i * nphc + j) * E + e];
        acc.x = fma(ww, v.x, acc.x);
        acc.y = fma(ww, v.y, acc.y);
    }
    tmp[(int64_t)cb * tot + idx] = acc;
}

// phi pass, phase shift to the parent center and sum over children:
//   U_p[pb][ip][jp][e] = sum_{cb} shift[oct(cb)][ip, jp] sum_q w tmp[cb][ip][src][e]
template <typename T>
__global__ void k_interp_phi(int nthp, int nphp, int nphc, int E, int pph, const int* __restrict__ src,
                             const T* __restrict__ w, const int* __restrict__ child_ptr, const int* __restrict__ octant,
                             const cpx<T>* __restrict__ shift, const cpx<T>* __restrict__ tmp, cpx<T>* __restrict__ Up) {
    const int pb = blockIdx.y;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int Kp = nthp * nphp;
    if (idx >= (int64_t)Kp * E) return;
    const int e = (int)(idx % E);
    const int kk = (int)(idx / E);
    const int ip = kk / nphp, jp = kk % nphp;
    const int64_t tsz = (int64_t)nthp * nphc * E;
    cpx<T> acc = czero<T>();
    for (int cb = child_ptr[pb]; cb < child_ptr[pb + 1]; ++cb) {
        const cpx<T>* tt = tmp + (int64_t)cb * tsz + (int64_t)ip * nphc * E;
        cpx<T> s = czero<T>();
        for (int q = 0; q < pph; ++q) {
            const T ww = w[jp * pph + q];
            cpx<T> v = tt[(int64_t)src[jp * pph + q] * E + e];
            s.x = fma(ww, v.x, s.x);
            s.y = fma(ww, v.y, s.y);
        }
        cfma(acc, shift[(int64_t)octant[cb] * Kp + kk], s);
    }
    Up[(int64_t)pb * Kp * E + idx] = acc;
}

// ------------------------------------------------------------------ translations
// V_b(k) = sum_{s in IL(b)} T[off(b,s)](k) U_s(k)   (weights folded into T)
template <typename T>
__global__ void k_translate(int K, int E, const int* __restrict__ il_ptr, const int* __restrict__ il_src,
                            const int* __restrict__ il_off, const cpx<T>* __restrict__ Top, const cpx<T>* __restrict__ U,
                            cpx<T>* __restrict__ V) {
    const int b = blockIdx.y;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)K * E) return;
    const int kk = (int)(idx / E);
    cpx<T> acc = czero<T>();
    for (int q = il_ptr[b]; q < il_ptr[b + 1]; ++q) {
        const cpx<T> t = Top[(int64_t)il_off[q] * K + kk];
        const cpx<T> u = U[(int64_t)il_src[q] * K * E + idx];
        cfma(acc, t, u);
    }
    V[(int64_t)b * K * E + idx] = acc;
}

// ------------------------------------------------------------------ anterpolation (downward)
// tmp[cb][ip][jc][e] = sum_{(jp, w) in tph(jc)} w conj(shift[oct(cb)][ip, jp]) V_p[parent(cb)][ip][jp][e]
template <typename T>
__global__ void k_anterp_phi(int nthp, int nphp, int nphc, int E, const int* __restrict__ tptr, const int* __restrict__ tdst,
                             const T* __restrict__ tw, const int* __restrict__ parent, const int* __restrict__ octant,
                             const cpx<T>* __restrict__ shift, const cpx<T>* __restrict__ Vp, cpx<T>* __restrict__ tmp) {
    const int cb = blockIdx.y;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)nthp * nphc * E;
    if (idx >= tot) return;
    const int e = (int)(idx % E);
    const int jc = (int)((idx / E) % nphc);
    const int ip = (int)(idx / ((int64_t)E * nphc));
    const int Kp = nthp * nphp;
    const cpx<T>* vp = Vp + (int64_t)parent[cb] * Kp * E;
    const cpx<T>* sh = shift + (int64_t)octant[cb] * Kp;
    cpx<T> acc = czero<T>();
    for (int q = tptr[jc]; q < tptr[jc + 1]; ++q) {
        const int jp = tdst[q];
        const int kk = ip * nphp + jp;
        cpx<T> v = cmulc(sh[kk], vp[(int64_t)kk * E + e]);
        const T ww = tw[q];
        acc.x = fma(ww, v.x, acc.x);
        acc.y = fma(ww, v.y, acc.y);
    }
    tmp[(int64_t)cb * tot + idx] = acc;
}

// V_c[cb][ic][jc][e] += sum_{(ip, flip, w) in tth(ic)} (+-) w tmp[cb][ip][jc or jc+half][e]
template <typename T>
__global__ void k_anterp_theta(int nthp, int nthc, int nphc, int E, const int* __restrict__ tptr,
                               const int* __restrict__ tdst, const int* __restrict__ tflip, const T* __restrict__ tw,
                               const cpx<T>* __restrict__ tmp, cpx<T>* __restrict__ Vc) {
    const int cb = blockIdx.y;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int Kc = nthc * nphc;
    if (idx >= (int64_t)Kc * E) return;
    const int e = (int)(idx % E);
    const int kk = (int)(idx / E);
    const int ic = kk / nphc, jc = kk % nphc;
    const int half = nphc / 2;
    const int64_t tsz = (int64_t)nthp * nphc * E;
    const cpx<T>* tt = tmp + (int64_t)cb * tsz;
    cpx<T> acc = czero<T>();
    for (int q = tptr[ic]; q < tptr[ic + 1]; ++q) {
        const int ip = tdst[q];
        const int f = tflip[q];
        const int j = f ? (jc + half) % nphc : jc;
        const T ww = f ? -tw[q] : tw[q];
        cpx<T> v = tt[((int64_t)ip * nphc + j) * E + e];
        acc.x = fma(ww, v.x, acc.x);
        acc.y = fma(ww, v.y, acc.y);
    }
    cpx<T>* out = Vc + (int64_t)cb * Kc * E + idx;
    *out = cadd(*out, acc);
}

// ------------------------------------------------------------------ leaf receive
// One warp per (tree RWG m, RHS r); lanes stride over directions, then a shuffle reduction.
template <typename T, int MODE>
__global__ void k_receive(int N, int K, int R, const int* __restrict__ leaf_of, const cpx<T>* __restrict__ F,
                          const cpx<T>* __restrict__ RX, const cpx<T>* __restrict__ V, T c, cpx<T>* __restrict__ yf) {
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= N * R) return;
    const int m = warp / R, r = warp % R;
    const int b = leaf_of[m];
    const int E = 2 * R;
    cpx<T> sJ = czero<T>(), sM = czero<T>();
    for (int kk = lane; kk < K; kk += 32) {
        const cpx<T> Ft = F[((int64_t)m * K + kk) * 2], Fp = F[((int64_t)m * K + kk) * 2 + 1];
        const cpx<T> Xt = RX[((int64_t)m * K + kk) * 2], Xp = RX[((int64_t)m * K + kk) * 2 + 1];
        const cpx<T> Vt = V[((int64_t)b * K + kk) * E + r], Vp = V[((int64_t)b * K + kk) * E + R + r];
        // R.V = conj(Ft) Vt + conj(Fp) Vp ; RX.(khat x V) = -Xt Vp + Xp Vt
        cpx<T> RV = cadd(cmulc(Ft, Vt), cmulc(Fp, Vp));
        cpx<T> XkV = csub(cmul(Xp, Vt), cmul(Xt, Vp));
        sJ = cadd(sJ, csub(RV, XkV));
        if (MODE == 0) {
            // -R.(khat x V) - RX.V = conj(Ft) Vp - conj(Fp) Vt - Xt Vt - Xp Vp
            cpx<T> t = csub(cmulc(Ft, Vp), cmulc(Fp, Vt));
            t = csub(t, cmul(Xt, Vt));
            t = csub(t, cmul(Xp, Vp));
            sM = cadd(sM, t);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sJ.x += __shfl_xor_sync(0xffffffffu, sJ.x, o);
        sJ.y += __shfl_xor_sync(0xffffffffu, sJ.y, o);
        if (MODE == 0) {
            sM.x += __shfl_xor_sync(0xffffffffu, sM.x, o);
            sM.y += __shfl_xor_sync(0xffffffffu, sM.y, o);
        }
    }
    if (lane == 0) {
        if (MODE == 0) {
            yf[((int64_t)m * 2 + 0) * R + r] = cscale(sJ, -c);
            yf[((int64_t)m * 2 + 1) * R + r] = cscale(sM, c);
        } else {
            yf[(int64_t)m * R + r] = cscale(sJ, -c);
        }
    }
}

inline unsigned nblk(int64_t n, int th) { return (unsigned)((n + th - 1) / th); }

// Stage boundaries for bi_profile_stages: when ev is non-null every stage runs on s (no
// overlap) and ev[i] is recorded after stage i; ev[-1] must be recorded by the caller.
template <typename T>
void launch_all(bi_handle_s* h, const void* xv, void* yv, int R, cudaStream_t s, cudaStream_t side,
                cudaEvent_t* ev = nullptr) {
    if (ev) side = s;
    const int N = h->N, nX = h->nX, nun = h->nun;
    const int E = 2 * R;
    const int th = 256;
    typedef cpx<T> C;
    const C* x = (const C*)xv;
    C* y = (C*)yv;
    C* xt = (C*)h->d_xt;
    C* yt = (C*)h->d_yt;
    C* yf = (C*)h->d_yfar;
    int64_t nvec = (int64_t)N * nX * R;
    k_gather_x<T><<<nblk(nvec, th), th, 0, s>>>(N, nX, R, nun, h->d_perm, x, xt);
    CU(cudaGetLastError());
    if (ev) CU(cudaEventRecord(ev[0], s));
    // near field on the side stream, concurrent with the far field
    if (!ev) {
        CU(cudaEventRecord(h->ev_fork, s));
        CU(cudaStreamWaitEvent(side, h->ev_fork, 0));
    }
    const level_t& LF = h->lev[h->leaf];
    if (h->prm.op_mode == 0)
        k_near<T, 0><<<LF.nbox, 128, 0, side>>>(R, h->d_leaf_start, h->d_near_ptr, h->d_near_src, h->d_near_blk,
                                                (const C*)h->d_near, h->d_gram_ptr, h->d_gram_col, (const T*)h->d_gram_val, xt, yt);
    else
        k_near<T, 1><<<LF.nbox, 128, 0, side>>>(R, h->d_leaf_start, h->d_near_ptr, h->d_near_src, h->d_near_blk,
                                                (const C*)h->d_near, nullptr, nullptr, nullptr, xt, yt);
    CU(cudaGetLastError());
    if (ev) CU(cudaEventRecord(ev[1], s));
    else CU(cudaEventRecord(h->ev_join, side));
    const bool far = h->leaf >= 2;
    if (far) {
        const int lf = h->leaf;
        // leaf aggregation
        {
            level_t& L = h->lev[lf];
            dim3 g(nblk((int64_t)L.K * E, th), L.nbox);
            if (h->prm.op_mode == 0)
                k_aggregate<T, 0><<<g, th, 0, s>>>(L.K, R, h->d_leaf_start, (const C*)h->d_F, xt, (C*)L.d_U);
            else
                k_aggregate<T, 1><<<g, th, 0, s>>>(L.K, R, h->d_leaf_start, (const C*)h->d_F, xt, (C*)L.d_U);
            CU(cudaGetLastError());
        }
        if (ev) CU(cudaEventRecord(ev[2], s));
        // upward pass
        for (int l = lf - 1; l >= 2; --l) {
            level_t& P = h->lev[l];
            level_t& Cc = h->lev[l + 1];
            interp_t& I = h->itp[l];
            dim3 g1(nblk((int64_t)P.nth * Cc.nph * E, th), Cc.nbox);
            k_interp_theta<T><<<g1, th, 0, s>>>(P.nth, Cc.nph, Cc.K, E, I.p_th, I.d_th_src, I.d_th_flip, (const T*)I.d_th_w,
                                                (const C*)Cc.d_U, (C*)I.d_tmp);
            CU(cudaGetLastError());
            dim3 g2(nblk((int64_t)P.K * E, th), P.nbox);
            k_interp_phi<T><<<g2, th, 0, s>>>(P.nth, P.nph, Cc.nph, E, I.p_ph, I.d_ph_src, (const T*)I.d_ph_w, P.d_child_ptr,
                                              Cc.d_octant, (const C*)P.d_shift, (const C*)I.d_tmp, (C*)P.d_U);
            CU(cudaGetLastError());
        }
        if (ev) CU(cudaEventRecord(ev[3], s));
        // translations on every level
        for (int l = 2; l <= lf; ++l) {
            level_t& L = h->lev[l];
            dim3 g(nblk((int64_t)L.K * E, th), L.nbox);
            k_translate<T><<<g, th, 0, s>>>(L.K, E, L.d_il_ptr, L.d_il_src, L.d_il_off, (const C*)L.d_T, (const C*)L.d_U,
                                            (C*)L.d_V);
            CU(cudaGetLastError());
        }
        if (ev) CU(cudaEventRecord(ev[4], s));
        // downward pass
        for (int l = 2; l < lf; ++l) {
            level_t& P = h->lev[l];
            level_t& Cc = h->lev[l + 1];
            interp_t& I = h->itp[l];
            dim3 g1(nblk((int64_t)P.nth * Cc.nph * E, th), Cc.nbox);
            k_anterp_phi<T><<<g1, th, 0, s>>>(P.nth, P.nph, Cc.nph, E, I.d_tph_ptr, I.d_tph_dst, (const T*)I.d_tph_w,
                                              Cc.d_parent, Cc.d_octant, (const C*)P.d_shift, (const C*)P.d_V, (C*)I.d_tmp);
            CU(cudaGetLastError());
            dim3 g2(nblk((int64_t)Cc.K * E, th), Cc.nbox);
            k_anterp_theta<T><<<g2, th, 0, s>>>(P.nth, Cc.nth, Cc.nph, E, I.d_tth_ptr, I.d_tth_dst, I.d_tth_flip,
                                                (const T*)I.d_tth_w, (const C*)I.d_tmp, (C*)Cc.d_V);
            CU(cudaGetLastError());
        }
        if (ev) CU(cudaEventRecord(ev[5], s));
        // leaf receive
        {
            level_t& L = h->lev[lf];
            const double pi = 3.14159265358979323846;
            T c = (T)(h->k * h->k / (32.0 * pi * pi));
            int64_t nthreads = (int64_t)N * R * 32;
            if (h->prm.op_mode == 0)
                k_receive<T, 0><<<nblk(nthreads, th), th, 0, s>>>(N, L.K, R, h->d_leaf_of, (const C*)h->d_F,
                                                                   (const C*)h->d_RX, (const C*)L.d_V, c, yf);
            else
                k_receive<T, 1><<<nblk(nthreads, th), th, 0, s>>>(N, L.K, R, h->d_leaf_of, (const C*)h->d_F,
                                                                   (const C*)h->d_RX, (const C*)L.d_V, c, yf);
            CU(cudaGetLastError());
        }
    }
    if (ev) {
        if (!far)
            for (int i = 2; i <= 5; ++i) CU(cudaEventRecord(ev[i], s));
        CU(cudaEventRecord(ev[6], s));
    } else {
        CU(cudaStreamWaitEvent(s, h->ev_join, 0));
    }
    k_scatter_y<T><<<nblk(nvec, th), th, 0, s>>>(N, nX, R, nun, h->d_perm, yt, far ? yf : nullptr, y);
    CU(cudaGetLastError());
    if (ev) CU(cudaEventRecord(ev[7], s));
}

}  // namespace

// Enqueue one product on stream s (no graph).
static void matvec_enqueue(bi_handle_s* h, const void* x, void* y, int nrhs, cudaStream_t s, cudaStream_t side) {
    if (h->prec == 0)
        launch_all<double>(h, x, y, nrhs, s, side);
    else
        launch_all<float>(h, x, y, nrhs, s, side);
}

// One product: replayed from a CUDA graph captured on first use for this (x, y, nrhs).
void bi_matvec_launch(bi_handle_s* h, const void* x, void* y, int nrhs, cudaStream_t s) {
    if (!h->use_graphs) {
        matvec_enqueue(h, x, y, nrhs, s, h->side);
        return;
    }
    for (auto& g : h->graphs)
        if (g.nrhs == nrhs && g.x == x && g.y == y) {
            CU(cudaGraphLaunch(g.exec, s));
            return;
        }
    cudaGraph_t graph;
    CU(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    try {
        matvec_enqueue(h, x, y, nrhs, h->cap, h->side);
    } catch (...) {
        cudaStreamEndCapture(h->cap, &graph);
        throw;
    }
    CU(cudaStreamEndCapture(h->cap, &graph));
    cudaGraphExec_t exec;
    CU(cudaGraphInstantiate(&exec, graph, 0));
    CU(cudaGraphDestroy(graph));
    if (h->graphs.size() >= 16) {
        cudaGraphExecDestroy(h->graphs.front().exec);
        h->graphs.erase(h->graphs.begin());
    }
    h->graphs.push_back({nrhs, x, y, exec});
    CU(cudaGraphLaunch(exec, s));
}

static const char* kStageNames[BI_NSTAGES] = {"gather", "near", "aggregate", "interpolate", "translate",
                                              "anterpolate", "receive", "scatter"};

const char* bi_stage_name_impl(int i) { return (i >= 0 && i < BI_NSTAGES) ? kStageNames[i] : ""; }

// Per-stage device time of `reps` products (serialised stages, CUDA events on the handle's stream).
void bi_profile_impl(bi_handle_s* h, const void* x, void* y, int nrhs, int reps, double* ms) {
    cudaEvent_t ev[BI_NSTAGES + 1];
    for (auto& e : ev) CU(cudaEventCreate(&e));
    for (int i = 0; i < BI_NSTAGES; ++i) ms[i] = 0.0;
    cudaStream_t s = h->stream;
    for (int r = 0; r < reps; ++r) {
        CU(cudaEventRecord(ev[0], s));
        if (h->prec == 0) launch_all<double>(h, x, y, nrhs, s, s, ev + 1);
        else launch_all<float>(h, x, y, nrhs, s, s, ev + 1);
        CU(cudaEventSynchronize(ev[BI_NSTAGES]));
        for (int i = 0; i < BI_NSTAGES; ++i) {
            float t = 0;
            CU(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
            ms[i] += t / reps;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
}
