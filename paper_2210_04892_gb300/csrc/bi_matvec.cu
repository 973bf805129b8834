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

#include "bi_cpx.cuh"
#include "bi_internal.h"

namespace {

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

// ------------------------------------------------------------------ near field (reference kernel)
// One thread per (test row, RHS) over the row-major segment of its box; tree-ordered vectors.
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
    const int64_t seg = near_blk[near_ptr[b]];
    const int ncol = (int)((near_blk[near_ptr[b + 1]] - seg) / mb);
    for (int idx = threadIdx.x; idx < mb * R; idx += blockDim.x) {
        const int ml = idx % mb, r = idx / mb;
        cpx<T> aJ = czero<T>(), aM = czero<T>();
        int c = 0;
        for (int q = near_ptr[b]; q < near_ptr[b + 1]; ++q) {
            const int s = near_src[q];
            const int n0 = leaf_start[s], nbs = leaf_start[s + 1] - n0;
            for (int nl = 0; nl < nbs; ++nl, ++c) {
                const int64_t e = seg + (int64_t)ml * ncol + c;
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
    }
}

// ------------------------------------------------------------------ leaf aggregation
// U_b(k) = sum_{n in b} ( -x_J,n F_n(k) + x_M,n khat x F_n(k) ),  (khat x F) = (-F_phi, F_theta)
template <typename T, int MODE>
__global__ void k_aggregate(int K, int nph, int R, const int* __restrict__ leaf_start, const cpx<T>* __restrict__ F,
                            const cpx<T>* __restrict__ xt, cpx<T>* __restrict__ U) {
    const int b = blockIdx.x;
    const int E = 2 * R, Kh = K / 2;
    int64_t idx = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)K * E) return;
    const int kk = (int)(idx / E), e = (int)(idx % E);
    const int c = e / R, r = e % R;
    const bool stored = kk < Kh;
    const int ks = stored ? kk : antipode(kk, K, nph);
    cpx<T> acc = czero<T>();
    for (int n = leaf_start[b]; n < leaf_start[b + 1]; ++n) {
        cpx<T> Ft = F[((int64_t)n * Kh + ks) * 2 + 0], Fp = F[((int64_t)n * Kh + ks) * 2 + 1];
        if (!stored) {
            Ft = cconj(Ft);
            Fp = cnegconj(Fp);
        }
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
// P > 0: compile-time tap count (taps hoisted and unrolled); P = 0: runtime count pth.
template <typename T, int P>
__global__ void k_interp_theta(int nthp, int nphc, int Kc, int E, int pth, const int* __restrict__ src,
                               const int* __restrict__ flip, const T* __restrict__ w, const cpx<T>* __restrict__ Uc,
                               cpx<T>* __restrict__ tmp) {
    const int cb = blockIdx.x;
    int64_t idx = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    int64_t tot = (int64_t)nthp * nphc * E;
    if (idx >= tot) return;
    const int e = (int)(idx % E);
    const int jc = (int)((idx / E) % nphc);
    const int ip = (int)(idx / ((int64_t)E * nphc));
    const int half = nphc / 2;
    const cpx<T>* u = Uc + (int64_t)cb * Kc * E;
    const int np = P > 0 ? P : pth;
    cpx<T> acc = czero<T>();
#pragma unroll
    for (int t = 0; t < (P > 0 ? P : 1); ++t) {
        if (P == 0) break;
        const int i = __ldg(src + ip * np + t);
        const int f = __ldg(flip + ip * np + t);
        const int j = f ? (jc + half) % nphc : jc;
        const T ww = f ? -__ldg(w + ip * np + t) : __ldg(w + ip * np + t);
        cpx<T> v = u[((int64_t)i * nphc + j) * E + e];
        acc.x = fma(ww, v.x, acc.x);
        acc.y = fma(ww, v.y, acc.y);
    }
    if (P == 0) {
        for (int t = 0; t < np; ++t) {
            const int i = src[ip * np + t];
            const int f = flip[ip * np + t];
            const int j = f ? (jc + half) % nphc : jc;
            const T ww = f ? -w[ip * np + t] : w[ip * np + t];
            cpx<T> v = u[((int64_t)i * nphc + j) * E + e];
            acc.x = fma(ww, v.x, acc.x);
            acc.y = fma(ww, v.y, acc.y);
        }
    }
    tmp[(int64_t)cb * tot + idx] = acc;
}

// phi pass, phase shift to the parent center and sum over children:
//   U_p[pb][ip][jp][e] = sum_{cb} shift[oct(cb)][ip, jp] sum_q w tmp[cb][ip][src][e]
template <typename T, int P>
__global__ void k_interp_phi(int nthp, int nphp, int nphc, int E, int pph, const int* __restrict__ src,
                             const T* __restrict__ w, const int* __restrict__ child_ptr, const int* __restrict__ octant,
                             const cpx<T>* __restrict__ shift, const cpx<T>* __restrict__ tmp, cpx<T>* __restrict__ Up) {
    const int pb = blockIdx.x;
    int64_t idx = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    const int Kp = nthp * nphp;
    if (idx >= (int64_t)Kp * E) return;
    const int e = (int)(idx % E);
    const int kk = (int)(idx / E);
    const int ip = kk / nphp, jp = kk % nphp;
    const int64_t tsz = (int64_t)nthp * nphc * E;
    const int np = P > 0 ? P : pph;
    int sj[P > 0 ? P : 1];
    T sw[P > 0 ? P : 1];
    if (P > 0) {
#pragma unroll
        for (int q = 0; q < (P > 0 ? P : 1); ++q) {
            sj[q] = __ldg(src + jp * np + q);
            sw[q] = __ldg(w + jp * np + q);
        }
    }
    cpx<T> acc = czero<T>();
    for (int cb = child_ptr[pb]; cb < child_ptr[pb + 1]; ++cb) {
        const cpx<T>* tt = tmp + (int64_t)cb * tsz + (int64_t)ip * nphc * E + e;
        cpx<T> s = czero<T>();
        if (P > 0) {
#pragma unroll
            for (int q = 0; q < (P > 0 ? P : 1); ++q) {
                const cpx<T> v = tt[(int64_t)sj[q] * E];
                s.x = fma(sw[q], v.x, s.x);
                s.y = fma(sw[q], v.y, s.y);
            }
        } else {
            for (int q = 0; q < np; ++q) {
                const cpx<T> v = tt[(int64_t)src[jp * np + q] * E];
                const T ww = w[jp * np + q];
                s.x = fma(ww, v.x, s.x);
                s.y = fma(ww, v.y, s.y);
            }
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
    const int b = blockIdx.x;
    int64_t idx = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
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
    const int cb = blockIdx.x;
    int64_t idx = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)nthp * nphc * E;
    if (idx >= tot) return;
    const int e = (int)(idx % E);
    const int jc = (int)((idx / E) % nphc);
    const int ip = (int)(idx / ((int64_t)E * nphc));
    const int Kp = nthp * nphp;
    const cpx<T>* vp = Vp + (int64_t)parent[cb] * Kp * E;
    const cpx<T>* sh = shift + (int64_t)octant[cb] * Kp;
    cpx<T> acc = czero<T>();
#pragma unroll 4
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
    const int cb = blockIdx.x;
    int64_t idx = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    const int Kc = nthc * nphc;
    if (idx >= (int64_t)Kc * E) return;
    const int e = (int)(idx % E);
    const int kk = (int)(idx / E);
    const int ic = kk / nphc, jc = kk % nphc;
    const int half = nphc / 2;
    const int64_t tsz = (int64_t)nthp * nphc * E;
    const cpx<T>* tt = tmp + (int64_t)cb * tsz;
    cpx<T> acc = czero<T>();
#pragma unroll 4
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
__global__ void k_receive(int N, int K, int nph, int R, const int* __restrict__ leaf_of, const cpx<T>* __restrict__ F,
                          const cpx<T>* __restrict__ RX, const cpx<T>* __restrict__ V, T c, cpx<T>* __restrict__ yf) {
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= N * R) return;
    const int m = warp / R, r = warp % R;
    const int b = leaf_of[m];
    const int E = 2 * R;
    cpx<T> sJ = czero<T>(), sM = czero<T>();
    const int Kh = K / 2;
    for (int kk = lane; kk < K; kk += 32) {
        const bool stored = kk < Kh;
        const int ks = stored ? kk : antipode(kk, K, nph);
        cpx<T> Ft = F[((int64_t)m * Kh + ks) * 2], Fp = F[((int64_t)m * Kh + ks) * 2 + 1];
        cpx<T> Xt = RX[((int64_t)m * Kh + ks) * 2], Xp = RX[((int64_t)m * Kh + ks) * 2 + 1];
        if (!stored) {
            Ft = cconj(Ft);
            Fp = cnegconj(Fp);
            Xt = cconj(Xt);
            Xp = cnegconj(Xp);
        }
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

// ------------------------------------------------------------------ near field (streaming)
// One CTA per test leaf box; x of the box's near columns (read through the user permutation)
// is staged in shared memory, then each warp streams whole rows of the row-major segment:
// lane j reads columns j, j+32, ... (coalesced 16-byte entries), a shuffle reduction gives the
// row.  RT right-hand sides per pass.
template <typename T, int MODE, int RT>
__global__ void __launch_bounds__(256, RT == 1 ? 6 : 1) k_near_stream(int N, int R, int nun, const int* __restrict__ perm,
                                                     const int2* __restrict__ work,
                                                     const int* __restrict__ leaf_start, const int* __restrict__ near_ptr,
                                                     const int* __restrict__ near_src, const int64_t* __restrict__ near_blk,
                                                     const int* __restrict__ near_col0, const int* __restrict__ near_ncol,
                                                     const cpx<T>* __restrict__ blocks, const int* __restrict__ gptr,
                                                     const int* __restrict__ gseg, const T* __restrict__ gval,
                                                     const cpx<T>* __restrict__ x, cpx<T>* __restrict__ yt,
                                                     cpx<T>* __restrict__ yuser) {
    constexpr int NX = MODE == 0 ? 2 : 1;
    extern __shared__ unsigned char smem_raw[];
    cpx<T>* xs = reinterpret_cast<cpx<T>*>(smem_raw);  // [NX][RT][ncol]
    // work item: test box and its first row; a CTA covers up to 2 * (blockDim / 32) rows
    const int b = work[blockIdx.x].x, row0 = work[blockIdx.x].y;
    const int m0 = leaf_start[b], mb = leaf_start[b + 1] - m0;
    const int q0 = near_ptr[b], q1 = near_ptr[b + 1];
    const int64_t seg = near_blk[q0];
    const int ncol = near_ncol[b];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const int row_end = min(mb, row0 + 2 * nwarp);
    for (int r0 = 0; r0 < R; r0 += RT) {
        const int rn = min(RT, R - r0);
        __syncthreads();
        // x of the near columns: one near box per warp, lanes over its RWGs
        for (int q = q0 + warp; q < q1; q += nwarp) {
            const int s = near_src[q];
            const int n0 = leaf_start[s], nbs = leaf_start[s + 1] - n0;
            const int c0 = near_col0[q];
            for (int i = lane; i < nbs; i += 32) {
                const int u = perm[n0 + i];
#pragma unroll
                for (int X = 0; X < NX; ++X)
#pragma unroll
                    for (int rr = 0; rr < RT; ++rr)
                        xs[((size_t)X * RT + rr) * ncol + c0 + i] =
                            rr < rn ? x[(int64_t)(r0 + rr) * nun + (int64_t)X * N + u] : czero<T>();
            }
        }
        __syncthreads();
        // each warp streams two rows at once (independent loads in flight for both)
        {
            const int mlA = row0 + 2 * warp, mlB = mlA + 1;
            const bool hasA = mlA < row_end, hasB = mlB < row_end;
            cpx<T> aJ[2][RT], aM[2][RT];
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2)
#pragma unroll
                for (int rr = 0; rr < RT; ++rr) { aJ[h2][rr] = czero<T>(); aM[h2][rr] = czero<T>(); }
            const int stride = (MODE == 0 ? 2 : 1);
            const cpx<T>* rowA = blocks + stride * (seg + (int64_t)(hasA ? mlA : 0) * ncol);
            const cpx<T>* rowB = blocks + stride * (seg + (int64_t)(hasB ? mlB : 0) * ncol);
            if (hasA) {
#pragma unroll 4
                for (int c = lane; c < ncol; c += 32) {
                    if (MODE == 0) {
                        cpx<T> A0, B0, A1 = czero<T>(), B1 = czero<T>();
                        load_pair(rowA + 2 * c, A0, B0);
                        if (hasB) load_pair(rowB + 2 * c, A1, B1);
#pragma unroll
                        for (int rr = 0; rr < RT; ++rr) {
                            const cpx<T> xJ = xs[(size_t)(0 * RT + rr) * ncol + c], xM = xs[(size_t)(1 * RT + rr) * ncol + c];
                            const cpx<T> nxM = {-xM.x, -xM.y};
                            cfma(aJ[0][rr], A0, xJ);
                            cfma(aJ[0][rr], B0, xM);
                            cfma(aM[0][rr], B0, xJ);
                            cfma(aM[0][rr], A0, nxM);
                            cfma(aJ[1][rr], A1, xJ);
                            cfma(aJ[1][rr], B1, xM);
                            cfma(aM[1][rr], B1, xJ);
                            cfma(aM[1][rr], A1, nxM);
                        }
                    } else {
                        const cpx<T> A0 = rowA[c];
                        const cpx<T> A1 = hasB ? rowB[c] : czero<T>();
#pragma unroll
                        for (int rr = 0; rr < RT; ++rr) {
                            cfma(aJ[0][rr], A0, xs[(size_t)rr * ncol + c]);
                            cfma(aJ[1][rr], A1, xs[(size_t)rr * ncol + c]);
                        }
                    }
                }
            }
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int ml = h2 == 0 ? mlA : mlB;
                if (ml >= row_end) continue;
                const int m = m0 + ml;
                if (MODE == 0) {
                    // Gram correction of the M row, (X/2) x_J - (G/2) x_M: one neighbour per lane, x from shared memory
                    const int g0 = gptr[m], gn = gptr[m + 1] - g0;
                    for (int qq = lane; qq < gn; qq += 32) {
                        const int c = gseg[g0 + qq];
                        const T gg = gval[2 * (g0 + qq)], xx = gval[2 * (g0 + qq) + 1];
#pragma unroll
                        for (int rr = 0; rr < RT; ++rr) {
                            const cpx<T> xJ = xs[(size_t)(0 * RT + rr) * ncol + c], xM = xs[(size_t)(1 * RT + rr) * ncol + c];
                            aM[h2][rr].x += T(0.5) * (xx * xJ.x - gg * xM.x);
                            aM[h2][rr].y += T(0.5) * (xx * xJ.y - gg * xM.y);
                        }
                    }
                }
#pragma unroll
                for (int rr = 0; rr < RT; ++rr) {
                    const cpx<T> sJ = warp_sum(aJ[h2][rr]);
                    const cpx<T> sM = MODE == 0 ? warp_sum(aM[h2][rr]) : czero<T>();
                    if (lane == 0 && rr < rn) {
                        const int r = r0 + rr;
                        const cpx<T> vJ = {-sJ.x, -sJ.y};
                        if (yuser) {
                            yuser[(int64_t)r * nun + perm[m]] = vJ;
                            if (MODE == 0) yuser[(int64_t)r * nun + N + perm[m]] = sM;
                        } else {
                            yt[((int64_t)m * NX + 0) * R + r] = vJ;
                            if (MODE == 0) yt[((int64_t)m * NX + 1) * R + r] = sM;
                        }
                    }
                }
            }
        }
    }
}

// ------------------------------------------------------------------ near field, several RHS
// Same work items and near-block segments as k_near_stream, for R >= 2: x comes from the
// tree-ordered copy xt [N][NX][R] (gathered once per product), so the x of one near box is one
// contiguous chunk and its staging is coalesced; each warp owns one row at a time (RT RHS of J
// and M in registers), lanes stride the row's columns with 16-byte block loads.
// MODE 3 (one medium of the two-region form): entries (L, K) = (<f, L f>, <f, Kbar f>) and
//   y_E = a L x_J - K x_M,   y_H = K x_J + b L x_M   (a, b: the medium's eta and 1/eta, or 1).
template <typename T, int MODE, int RT>
__global__ void __launch_bounds__(256, RT >= 8 ? 2 : 3) k_near_multi(int N, int R, int nun, const int* __restrict__ perm,
                                                      const int2* __restrict__ work,
                                                      const int* __restrict__ leaf_start, const int* __restrict__ near_ptr,
                                                      const int* __restrict__ near_src, const int64_t* __restrict__ near_blk,
                                                      const int* __restrict__ near_col0, const int* __restrict__ near_ncol,
                                                      const cpx<T>* __restrict__ blocks, const int* __restrict__ gptr,
                                                      const int* __restrict__ gseg, const T* __restrict__ gval,
                                                      const cpx<T>* __restrict__ xt, cpx<T>* __restrict__ yt,
                                                      cpx<T>* __restrict__ yuser, cpx<T> pa, cpx<T> pb) {
    constexpr int NX = (MODE == 0 || MODE == 3) ? 2 : 1;
    extern __shared__ unsigned char smem_raw[];
    cpx<T>* xs = reinterpret_cast<cpx<T>*>(smem_raw);  // [NX][RT][ncol]
    const int b = work[blockIdx.x].x, row0 = work[blockIdx.x].y;
    const int m0 = leaf_start[b], mb = leaf_start[b + 1] - m0;
    const int q0 = near_ptr[b], q1 = near_ptr[b + 1];
    const int64_t seg = near_blk[q0];
    const int ncol = near_ncol[b];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const int row_end = min(mb, row0 + 16);   // a work item holds up to 16 rows of its box
    for (int r0 = 0; r0 < R; r0 += RT) {
        const int rn = min(RT, R - r0);
        __syncthreads();
        // x of the near columns: one near box per warp; its tree-ordered x is contiguous
        for (int q = q0 + warp; q < q1; q += nwarp) {
            const int s = near_src[q];
            const int n0 = leaf_start[s], nbs = leaf_start[s + 1] - n0;
            const int c0 = near_col0[q];
            const cpx<T>* xb = xt + (int64_t)n0 * NX * R + r0;
            for (int i = lane; i < nbs * NX * RT; i += 32) {
                const int rr = i % RT, X = (i / RT) % NX, n = i / (RT * NX);
                xs[((size_t)X * RT + rr) * ncol + c0 + n] = rr < rn ? xb[((int64_t)n * NX + X) * R + rr] : czero<T>();
            }
        }
        __syncthreads();
        const int stride = ((MODE == 0 || MODE == 3) ? 2 : 1);
        for (int ml = row0 + warp; ml < row_end; ml += nwarp) {
            cpx<T> aJ[RT], aM[RT], bJ[RT], bM[RT];   // b*: the second pair of sums of MODE 3
#pragma unroll
            for (int rr = 0; rr < RT; ++rr) { aJ[rr] = czero<T>(); aM[rr] = czero<T>(); bJ[rr] = czero<T>(); bM[rr] = czero<T>(); }
            const cpx<T>* row = blocks + stride * (seg + (int64_t)ml * ncol);
#pragma unroll 2
            for (int c = lane; c < ncol; c += 32) {
                if (MODE == 3) {
                    cpx<T> A, B;   // A = L, B = K
                    load_pair(row + 2 * c, A, B);
#pragma unroll
                    for (int rr = 0; rr < RT; ++rr) {
                        const cpx<T> xJ = xs[(size_t)rr * ncol + c], xM = xs[(size_t)(RT + rr) * ncol + c];
                        cfma(aJ[rr], A, xJ);   // L x_J
                        cfma(aM[rr], B, xM);   // K x_M
                        cfma(bJ[rr], B, xJ);   // K x_J
                        cfma(bM[rr], A, xM);   // L x_M
                    }
                } else if (MODE == 0) {
                    cpx<T> A, B;
                    load_pair(row + 2 * c, A, B);
#pragma unroll
                    for (int rr = 0; rr < RT; ++rr) {
                        const cpx<T> xJ = xs[(size_t)rr * ncol + c], xM = xs[(size_t)(RT + rr) * ncol + c];
                        cfma(aJ[rr], A, xJ);
                        cfma(aJ[rr], B, xM);
                        cfma(aM[rr], B, xJ);
                        cfma(aM[rr], A, cpx<T>{-xM.x, -xM.y});
                    }
                } else {
                    const cpx<T> A = ldg_cpx(row + c);
#pragma unroll
                    for (int rr = 0; rr < RT; ++rr) cfma(aJ[rr], A, xs[(size_t)rr * ncol + c]);
                }
            }
            const int m = m0 + ml;
            if (MODE == 0) {
                const int g0 = gptr[m], gn = gptr[m + 1] - g0;
                for (int qq = lane; qq < gn; qq += 32) {
                    const int c = gseg[g0 + qq];
                    const T gg = gval[2 * (g0 + qq)], xx = gval[2 * (g0 + qq) + 1];
#pragma unroll
                    for (int rr = 0; rr < RT; ++rr) {
                        const cpx<T> xJ = xs[(size_t)rr * ncol + c], xM = xs[(size_t)(RT + rr) * ncol + c];
                        aM[rr].x += T(0.5) * (xx * xJ.x - gg * xM.x);
                        aM[rr].y += T(0.5) * (xx * xJ.y - gg * xM.y);
                    }
                }
            }
#pragma unroll
            for (int rr = 0; rr < RT; ++rr) {
                cpx<T> sJ = warp_sum(aJ[rr]);
                cpx<T> sM = (MODE == 0 || MODE == 3) ? warp_sum(aM[rr]) : czero<T>();
                if (MODE == 3) {
                    // y_E = a L x_J - K x_M,  y_H = K x_J + b L x_M (stored so that the lines below,
                    // which negate the first, write them)
                    const cpx<T> kJ = warp_sum(bJ[rr]), lM = warp_sum(bM[rr]);
                    const cpx<T> yE = csub(cmul(pa, sJ), sM), yH = cadd(kJ, cmul(pb, lM));
                    sJ = cpx<T>{-yE.x, -yE.y};
                    sM = yH;
                }
                if (lane == rr && rr < rn) {
                    const int r = r0 + rr;
                    const cpx<T> vJ = {-sJ.x, -sJ.y};
                    if (yuser) {
                        yuser[(int64_t)r * nun + perm[m]] = vJ;
                        if (NX == 2) yuser[(int64_t)r * nun + N + perm[m]] = sM;
                    } else {
                        yt[((int64_t)m * NX + 0) * R + r] = vJ;
                        if (NX == 2) yt[((int64_t)m * NX + 1) * R + r] = sM;
                    }
                }
            }
        }
    }
}

// ------------------------------------------------------------------ near field, row pairs
// Several RHS (R >= 3, MODE 0 or 1), the work items and staged x of k_near_multi: each warp
// takes two rows of its work item at once, its lanes split as 16 column lanes x 2 halves of
// the RT right-hand sides.  A lane's staged x values (RT/2 RHS of J and M) serve both rows, so
// shared-memory reads per multiply-add are half those of k_near_multi, and the row sums meet
// over 16 lanes (4 shuffle steps) for RT/2 RHS per lane instead of 32 lanes for RT.
template <typename T, int MODE, int RT>
__global__ void __launch_bounds__(256, 2) k_near_rb(int N, int R, int nun, const int* __restrict__ perm,
                                                    const int2* __restrict__ work, const int* __restrict__ leaf_start,
                                                    const int* __restrict__ near_ptr, const int* __restrict__ near_src,
                                                    const int64_t* __restrict__ near_blk, const int* __restrict__ near_col0,
                                                    const int* __restrict__ near_ncol, const cpx<T>* __restrict__ blocks,
                                                    const int* __restrict__ gptr, const int* __restrict__ gseg,
                                                    const T* __restrict__ gval, const cpx<T>* __restrict__ xt,
                                                    cpx<T>* __restrict__ yt, cpx<T>* __restrict__ yuser) {
    constexpr int NX = MODE == 0 ? 2 : 1;
    constexpr int RH = RT / 2;           // RHS per lane
    extern __shared__ unsigned char smem_raw[];
    cpx<T>* xs = reinterpret_cast<cpx<T>*>(smem_raw);  // [NX][RT][ncol]
    const int b = work[blockIdx.x].x, row0 = work[blockIdx.x].y;
    const int m0 = leaf_start[b], mb = leaf_start[b + 1] - m0;
    const int q0 = near_ptr[b], q1 = near_ptr[b + 1];
    const int64_t seg = near_blk[q0];
    const int ncol = near_ncol[b];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const int cl = lane & 15, hh = lane >> 4;      // column lane, RHS half
    const int row_end = min(mb, row0 + 16);       // a work item holds up to 16 rows of its box
    for (int r0 = 0; r0 < R; r0 += RT) {
        const int rn = min(RT, R - r0);
        __syncthreads();
        for (int q = q0 + warp; q < q1; q += nwarp) {
            const int s = near_src[q];
            const int n0 = leaf_start[s], nbs = leaf_start[s + 1] - n0;
            const int c0 = near_col0[q];
            const cpx<T>* xb = xt + (int64_t)n0 * NX * R + r0;
            for (int i = lane; i < nbs * NX * RT; i += 32) {
                const int rr = i % RT, X = (i / RT) % NX, n = i / (RT * NX);
                xs[((size_t)X * RT + rr) * ncol + c0 + n] = rr < rn ? xb[((int64_t)n * NX + X) * R + rr] : czero<T>();
            }
        }
        __syncthreads();
        const cpx<T>* xJs = xs + (size_t)(hh * RH) * ncol;
        const cpx<T>* xMs = xs + (size_t)(RT + hh * RH) * ncol;
        for (int ml = row0 + 2 * warp; ml < row_end; ml += 2 * nwarp) {
            const bool two = ml + 1 < row_end;
            cpx<T> a0[RH][NX], a1[RH][NX];
#pragma unroll
            for (int j = 0; j < RH; ++j)
#pragma unroll
                for (int X = 0; X < NX; ++X) { a0[j][X] = czero<T>(); a1[j][X] = czero<T>(); }
            const cpx<T>* rowA = blocks + (int64_t)NX * (seg + (int64_t)ml * ncol);
            const cpx<T>* rowB = two ? rowA + (int64_t)NX * ncol : rowA;   // a lone last row reads its own row twice
#pragma unroll 2
            for (int c = cl; c < ncol; c += 16) {
                if (MODE == 0) {
                    cpx<T> A0, B0, A1, B1;
                    load_pair(rowA + 2 * c, A0, B0);
                    load_pair(rowB + 2 * c, A1, B1);
#pragma unroll
                    for (int j = 0; j < RH; ++j) {
                        const cpx<T> xJ = xJs[(size_t)j * ncol + c], xM = xMs[(size_t)j * ncol + c];
                        const cpx<T> nxM = {-xM.x, -xM.y};
                        cfma(a0[j][0], A0, xJ);
                        cfma(a0[j][0], B0, xM);
                        cfma(a0[j][NX - 1], B0, xJ);
                        cfma(a0[j][NX - 1], A0, nxM);
                        cfma(a1[j][0], A1, xJ);
                        cfma(a1[j][0], B1, xM);
                        cfma(a1[j][NX - 1], B1, xJ);
                        cfma(a1[j][NX - 1], A1, nxM);
                    }
                } else {
                    const cpx<T> A0 = ldg_cpx(rowA + c), A1 = ldg_cpx(rowB + c);
#pragma unroll
                    for (int j = 0; j < RH; ++j) {
                        const cpx<T> xJ = xJs[(size_t)j * ncol + c];
                        cfma(a0[j][0], A0, xJ);
                        cfma(a1[j][0], A1, xJ);
                    }
                }
            }
            if (MODE == 0) {
                // Gram terms of the M rows: 1/2 (X x_J - G x_M), lanes over the row's entries
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    if (t == 1 && !two) break;
                    const int m = m0 + ml + t;
                    const int g0 = gptr[m], gn = gptr[m + 1] - g0;
                    for (int qq = cl; qq < gn; qq += 16) {
                        const int c = gseg[g0 + qq];
                        const T gg = gval[2 * (g0 + qq)], xx = gval[2 * (g0 + qq) + 1];
#pragma unroll
                        for (int j = 0; j < RH; ++j) {
                            const cpx<T> xJ = xJs[(size_t)j * ncol + c], xM = xMs[(size_t)j * ncol + c];
                            cpx<T>& acc = t == 0 ? a0[j][NX - 1] : a1[j][NX - 1];
                            acc.x += T(0.5) * (xx * xJ.x - gg * xM.x);
                            acc.y += T(0.5) * (xx * xJ.y - gg * xM.y);
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < RH; ++j)
#pragma unroll
                for (int X = 0; X < NX; ++X)
#pragma unroll
                    for (int o = 1; o < 16; o <<= 1) {
                        a0[j][X].x += __shfl_xor_sync(0xffffffffu, a0[j][X].x, o);
                        a0[j][X].y += __shfl_xor_sync(0xffffffffu, a0[j][X].y, o);
                        a1[j][X].x += __shfl_xor_sync(0xffffffffu, a1[j][X].x, o);
                        a1[j][X].y += __shfl_xor_sync(0xffffffffu, a1[j][X].y, o);
                    }
            // lane cl of each half writes RHS hh*RH + cl (cl < RH) of both rows
#pragma unroll
            for (int j = 0; j < RH; ++j) {
                const int rr = hh * RH + j;
                if (cl == j && rr < rn) {
                    const int r = r0 + rr;
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        if (t == 1 && !two) break;
                        const int m = m0 + ml + t;
                        const cpx<T> sJ = t == 0 ? a0[j][0] : a1[j][0];
                        const cpx<T> vJ = {-sJ.x, -sJ.y};
                        if (yuser) {
                            yuser[(int64_t)r * nun + perm[m]] = vJ;
                            if (NX == 2) yuser[(int64_t)r * nun + N + perm[m]] = t == 0 ? a0[j][NX - 1] : a1[j][NX - 1];
                        } else {
                            yt[((int64_t)m * NX + 0) * R + r] = vJ;
                            if (NX == 2) yt[((int64_t)m * NX + 1) * R + r] = t == 0 ? a0[j][NX - 1] : a1[j][NX - 1];
                        }
                    }
                }
            }
        }
    }
}

// ------------------------------------------------------------------ near field, row pairs, pipelined
// The row-pair kernel above (MODE 0, FP32) with the block entries brought into shared memory by
// per-lane cp.async copies NS column steps ahead of their use: lane (t, cl) copies the 16-byte
// (A, B) entry of row t of the pair at column step + cl into the warp's ring, so the registers
// hold no loads in flight and each warp keeps NS x 512 bytes of the block stream in flight.
__device__ __forceinline__ void near_cp16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}
template <int RT, int NS>
__global__ void __launch_bounds__(256, 2) k_near_rbp(int N, int R, int nun, const int* __restrict__ perm,
                                                     const int2* __restrict__ work, const int* __restrict__ leaf_start,
                                                     const int* __restrict__ near_ptr, const int* __restrict__ near_src,
                                                     const int64_t* __restrict__ near_blk,
                                                     const int* __restrict__ near_col0, const int* __restrict__ near_ncol,
                                                     const cpx<float>* __restrict__ blocks, const int* __restrict__ gptr,
                                                     const int* __restrict__ gseg, const float* __restrict__ gval,
                                                     const cpx<float>* __restrict__ xt, cpx<float>* __restrict__ yt,
                                                     cpx<float>* __restrict__ yuser) {
    typedef cpx<float> C;
    constexpr int NX = 2, RH = RT / 2;
    extern __shared__ float4 smem_rbp[];
    float4* ring = smem_rbp;                                    // [8 warps][NS][32]
    C* xs = reinterpret_cast<C*>(smem_rbp + 8 * NS * 32);      // [NX][RT][ncol]
    const int b = work[blockIdx.x].x, row0 = work[blockIdx.x].y;
    const int m0 = leaf_start[b], mb = leaf_start[b + 1] - m0;
    const int q0 = near_ptr[b], q1 = near_ptr[b + 1];
    const int64_t seg = near_blk[q0];
    const int ncol = near_ncol[b];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const int cl = lane & 15, hh = lane >> 4;
    const int row_end = min(mb, row0 + 16);
    float4* wr = ring + warp * NS * 32;
    const int nstep = (ncol + 15) / 16;
    for (int r0 = 0; r0 < R; r0 += RT) {
        const int rn = min(RT, R - r0);
        __syncthreads();
        for (int q = q0 + warp; q < q1; q += nwarp) {
            const int s = near_src[q];
            const int n0 = leaf_start[s], nbs = leaf_start[s + 1] - n0;
            const int c0 = near_col0[q];
            const C* xb = xt + (int64_t)n0 * NX * R + r0;
            for (int i = lane; i < nbs * NX * RT; i += 32) {
                const int rr = i % RT, X = (i / RT) % NX, n = i / (RT * NX);
                xs[((size_t)X * RT + rr) * ncol + c0 + n] = rr < rn ? xb[((int64_t)n * NX + X) * R + rr] : czero<float>();
            }
        }
        __syncthreads();
        const C* xJs = xs + (size_t)(hh * RH) * ncol;
        const C* xMs = xs + (size_t)(RT + hh * RH) * ncol;
        for (int ml = row0 + 2 * warp; ml < row_end; ml += 2 * nwarp) {
            const bool two = ml + 1 < row_end;
            // this lane copies row (ml + hh) of the pair (a lone last row: row ml twice)
            const C* crow = blocks + 2 * (seg + (int64_t)(two ? ml + hh : ml) * ncol);
            auto issue = [&](int st) {
                const int c = st * 16 + cl;
                if (st < nstep) near_cp16(&wr[(st % NS) * 32 + lane], crow + 2 * min(c, ncol - 1), c < ncol ? 16 : 0);
                asm volatile("cp.async.commit_group;" ::: "memory");
            };
#pragma unroll
            for (int st = 0; st < NS - 1; ++st) issue(st);
            C a0[RH][NX], a1[RH][NX];
#pragma unroll
            for (int j = 0; j < RH; ++j)
#pragma unroll
                for (int X = 0; X < NX; ++X) { a0[j][X] = czero<float>(); a1[j][X] = czero<float>(); }
            for (int st = 0; st < nstep; ++st) {
                issue(st + NS - 1);
                asm volatile("cp.async.wait_group %0;" ::"n"(NS - 1) : "memory");
                __syncwarp();
                const int c = st * 16 + cl;
                if (c < ncol) {
                    const float4 e0 = wr[(st % NS) * 32 + cl], e1 = wr[(st % NS) * 32 + 16 + cl];
                    const C A0 = {e0.x, e0.y}, B0 = {e0.z, e0.w}, A1 = {e1.x, e1.y}, B1 = {e1.z, e1.w};
#pragma unroll
                    for (int j = 0; j < RH; ++j) {
                        const C xJ = xJs[(size_t)j * ncol + c], xM = xMs[(size_t)j * ncol + c];
                        const C nxM = {-xM.x, -xM.y};
                        cfma(a0[j][0], A0, xJ);
                        cfma(a0[j][0], B0, xM);
                        cfma(a0[j][1], B0, xJ);
                        cfma(a0[j][1], A0, nxM);
                        cfma(a1[j][0], A1, xJ);
                        cfma(a1[j][0], B1, xM);
                        cfma(a1[j][1], B1, xJ);
                        cfma(a1[j][1], A1, nxM);
                    }
                }
                __syncwarp();   // the slot is refilled by the copy issued next step
            }
            asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                if (t == 1 && !two) break;
                const int m = m0 + ml + t;
                const int g0 = gptr[m], gn = gptr[m + 1] - g0;
                for (int qq = cl; qq < gn; qq += 16) {
                    const int c = gseg[g0 + qq];
                    const float gg = gval[2 * (g0 + qq)], xx = gval[2 * (g0 + qq) + 1];
#pragma unroll
                    for (int j = 0; j < RH; ++j) {
                        const C xJ = xJs[(size_t)j * ncol + c], xM = xMs[(size_t)j * ncol + c];
                        C& acc = t == 0 ? a0[j][1] : a1[j][1];
                        acc.x += 0.5f * (xx * xJ.x - gg * xM.x);
                        acc.y += 0.5f * (xx * xJ.y - gg * xM.y);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < RH; ++j)
#pragma unroll
                for (int X = 0; X < NX; ++X)
#pragma unroll
                    for (int o = 1; o < 16; o <<= 1) {
                        a0[j][X].x += __shfl_xor_sync(0xffffffffu, a0[j][X].x, o);
                        a0[j][X].y += __shfl_xor_sync(0xffffffffu, a0[j][X].y, o);
                        a1[j][X].x += __shfl_xor_sync(0xffffffffu, a1[j][X].x, o);
                        a1[j][X].y += __shfl_xor_sync(0xffffffffu, a1[j][X].y, o);
                    }
#pragma unroll
            for (int j = 0; j < RH; ++j) {
                const int rr = hh * RH + j;
                if (cl == j && rr < rn) {
                    const int r = r0 + rr;
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        if (t == 1 && !two) break;
                        const int m = m0 + ml + t;
                        const C sJ = t == 0 ? a0[j][0] : a1[j][0];
                        const C vJ = {-sJ.x, -sJ.y};
                        const C vM = t == 0 ? a0[j][1] : a1[j][1];
                        if (yuser) {
                            yuser[(int64_t)r * nun + perm[m]] = vJ;
                            yuser[(int64_t)r * nun + N + perm[m]] = vM;
                        } else {
                            yt[((int64_t)m * NX + 0) * R + r] = vJ;
                            yt[((int64_t)m * NX + 1) * R + r] = vM;
                        }
                    }
                }
            }
            __syncwarp();
        }
    }
}

// ------------------------------------------------------------------ leaf aggregation (fused gather)
// thread per (stored direction kk, RHS r): both components from one 16-byte pattern load give
// U at kk and at its antipode.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_aggregate2(int N, int K, int nph, int R, int nun, const int* __restrict__ perm,
                                                    const int* __restrict__ leaf_start, const cpx<T>* __restrict__ F,
                                                    const cpx<T>* __restrict__ x, cpx<T>* __restrict__ U) {
    // CTA = (box, 64 direction-RHS slots); the box's RWGs are split over 4 thread groups whose
    // partial sums meet in shared memory.  x of the box is staged once per CTA.
    extern __shared__ unsigned char smem_raw[];
    cpx<T>* xs = reinterpret_cast<cpx<T>*>(smem_raw);  // [nb][2][R]
    __shared__ cpx<T> red[4][64][4];
    const int b = blockIdx.x;
    const int Kh = K / 2;
    const int n0 = leaf_start[b], nb = leaf_start[b + 1] - n0;
    for (int i = threadIdx.x; i < nb * 2 * R; i += blockDim.x) {
        const int r = i % R, X = (i / R) % 2, n = i / (2 * R);
        xs[i] = (MODE == 0 || X == 0) ? x[(int64_t)r * nun + (int64_t)X * N + perm[n0 + n]] : czero<T>();
    }
    __syncthreads();
    const int slot = threadIdx.x & 63, grp = threadIdx.x >> 6;
    const int idx = blockIdx.y * 64 + slot;
    const bool ok = idx < Kh * R;
    const int kk = ok ? idx / R : 0, r = ok ? idx % R : 0;
    // (ut, up) at kk; (vt, vp) at the antipode, where the pattern reads (conj Ft, -conj Fp)
    cpx<T> ut = czero<T>(), up = czero<T>(), vt = czero<T>(), vp = czero<T>();
    if (ok) {
        const cpx<T>* f = F + ((int64_t)n0 * Kh + kk) * 2;
#pragma unroll 4
        for (int n = grp; n < nb; n += 4) {
            cpx<T> Ft, Fp;
            load_pair(f + (int64_t)n * Kh * 2, Ft, Fp);
            const cpx<T> xJ = xs[(n * 2 + 0) * R + r];
            ut = csub(ut, cmul(xJ, Ft));
            up = csub(up, cmul(xJ, Fp));
            vt = csub(vt, cmulc(Ft, xJ));
            vp = cadd(vp, cmulc(Fp, xJ));
            if (MODE == 0) {
                const cpx<T> xM = xs[(n * 2 + 1) * R + r];
                ut = csub(ut, cmul(xM, Fp));
                up = cadd(up, cmul(xM, Ft));
                vt = cadd(vt, cmulc(Fp, xM));
                vp = cadd(vp, cmulc(Ft, xM));
            }
        }
    }
    red[grp][slot][0] = ut;
    red[grp][slot][1] = up;
    red[grp][slot][2] = vt;
    red[grp][slot][3] = vp;
    __syncthreads();
    if (grp == 0 && ok) {
        for (int g2 = 1; g2 < 4; ++g2) {
            ut = cadd(ut, red[g2][slot][0]);
            up = cadd(up, red[g2][slot][1]);
            vt = cadd(vt, red[g2][slot][2]);
            vp = cadd(vp, red[g2][slot][3]);
        }
        cpx<T>* o = U + ((int64_t)b * K + kk) * (2 * R);
        o[r] = ut;
        o[R + r] = up;
        cpx<T>* oa = U + ((int64_t)b * K + antipode(kk, K, nph)) * (2 * R);
        oa[r] = vt;
        oa[R + r] = vp;
    }
}

// ------------------------------------------------------------------ many right-hand sides: per-box tiles
// Aggregation as a small product per leaf box, U[k][c][r] = sum_n F[n][k][.] x[n][.][r]:
// CTA = (box, 32 directions); the box's patterns for those directions and its x for all RHS
// are staged in shared memory, so every pattern entry is read from HBM once per product.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_aggregate_tile(int N, int K, int nph, int R, int nun, const int* __restrict__ perm,
                                                        const int* __restrict__ leaf_start, const cpx<T>* __restrict__ F,
                                                        const cpx<T>* __restrict__ x, cpx<T>* __restrict__ U) {
    constexpr int KT = 32;
    const int Kh = K / 2;
    extern __shared__ unsigned char smem_raw[];
    const int b = blockIdx.x, k0 = blockIdx.y * KT;
    const int n0 = leaf_start[b], nb = leaf_start[b + 1] - n0;
    cpx<T>* fs = reinterpret_cast<cpx<T>*>(smem_raw);      // [nb][KT][2]
    cpx<T>* xs = fs + (size_t)nb * KT * 2;                   // [nb][2][R]
    for (int i = threadIdx.x; i < nb * KT; i += blockDim.x) {
        const int n = i / KT, kk = k0 + i % KT;
        cpx<T> a = czero<T>(), c = czero<T>();
        if (kk < Kh) load_pair(F + ((int64_t)(n0 + n) * Kh + kk) * 2, a, c);
        fs[2 * i] = a;
        fs[2 * i + 1] = c;
    }
    for (int i = threadIdx.x; i < nb * 2 * R; i += blockDim.x) {
        const int r = i % R, X = (i / R) % 2, n = i / (2 * R);
        xs[i] = (MODE == 0 || X == 0) ? x[(int64_t)r * nun + (int64_t)X * N + perm[n0 + n]] : czero<T>();
    }
    __syncthreads();
    const int E = 2 * R;
    for (int o = threadIdx.x; o < KT * R; o += blockDim.x) {
        const int kl = o / R, r = o % R, kk = k0 + kl;
        if (kk >= Kh) continue;
        // (ut, up) at kk, (vt, vp) at its antipode
        cpx<T> ut = czero<T>(), up = czero<T>(), vt = czero<T>(), vp = czero<T>();
        for (int n = 0; n < nb; ++n) {
            const cpx<T> Ft = fs[(n * KT + kl) * 2], Fp = fs[(n * KT + kl) * 2 + 1];
            const cpx<T> xJ = xs[(n * 2 + 0) * R + r];
            ut = csub(ut, cmul(xJ, Ft));
            up = csub(up, cmul(xJ, Fp));
            vt = csub(vt, cmulc(Ft, xJ));
            vp = cadd(vp, cmulc(Fp, xJ));
            if (MODE == 0) {
                const cpx<T> xM = xs[(n * 2 + 1) * R + r];
                ut = csub(ut, cmul(xM, Fp));
                up = cadd(up, cmul(xM, Ft));
                vt = cadd(vt, cmulc(Fp, xM));
                vp = cadd(vp, cmulc(Ft, xM));
            }
        }
        cpx<T>* out = U + ((int64_t)b * K + kk) * E;
        out[r] = ut;
        out[R + r] = up;
        cpx<T>* oa = U + ((int64_t)b * K + antipode(kk, K, nph)) * E;
        oa[r] = vt;
        oa[R + r] = vp;
    }
}

// Receive as a small product per leaf box: y[m][r] = sum_k (F, RX)[m][k] . V[k][r]:
// CTA = one leaf box; directions in tiles of 32 staged in shared memory (patterns of the
// box's RWGs and V for all RHS), each thread accumulating a few (m, r) outputs.
template <typename T, int MODE, int OPT>
__global__ void __launch_bounds__(256) k_receive_tile(int N, int K, int nph, int R, int RC, int nun, const int* __restrict__ perm,
                                                      const int* __restrict__ leaf_start, const cpx<T>* __restrict__ F,
                                                      const cpx<T>* __restrict__ RX, const cpx<T>* __restrict__ V, T c,
                                                      const cpx<T>* __restrict__ yt, cpx<T>* __restrict__ y) {
    constexpr int KT = 32;
    extern __shared__ unsigned char smem_raw[];
    const int b = blockIdx.x;
    const int r0 = blockIdx.y * RC, rc = min(RC, R - r0);     // this CTA's right-hand sides
    const int n0 = leaf_start[b], nb = leaf_start[b + 1] - n0;
    const int E = 2 * R;
    const int Kh = K / 2;
    cpx<T>* fs = reinterpret_cast<cpx<T>*>(smem_raw);       // [nb][KT][4]: Ft Fp Xt Xp (stored directions)
    cpx<T>* vs = fs + (size_t)nb * KT * 4;                    // [KT][4][RC]: V at kk (t, p), at its antipode (t, p)
    // When the box has fewer (RWG, RHS) outputs than threads, G groups of threads split the
    // directions of each tile (group g takes kl = g, g + G, ...) and meet in shared memory.
    const int no = nb * rc;
    const int G = no > 0 ? max(1, min(8, (int)blockDim.x / no)) : 1;
    cpx<T> aJ[OPT], aM[OPT];
#pragma unroll
    for (int o = 0; o < OPT; ++o) { aJ[o] = czero<T>(); aM[o] = czero<T>(); }
    for (int k0 = 0; k0 < Kh; k0 += KT) {
        __syncthreads();
        for (int i = threadIdx.x; i < nb * KT; i += blockDim.x) {
            const int n = i / KT, kk = k0 + i % KT;
            cpx<T> a = czero<T>(), bb = czero<T>(), cc = czero<T>(), dd = czero<T>();
            if (kk < Kh) {
                load_pair(F + ((int64_t)(n0 + n) * Kh + kk) * 2, a, bb);
                load_pair(RX + ((int64_t)(n0 + n) * Kh + kk) * 2, cc, dd);
            }
            fs[4 * i] = a;
            fs[4 * i + 1] = bb;
            fs[4 * i + 2] = cc;
            fs[4 * i + 3] = dd;
        }
        for (int i = threadIdx.x; i < KT * 4 * RC; i += blockDim.x) {
            const int kl = i / (4 * RC), q = (i / RC) % 4, rr = i % RC, kk = k0 + kl;
            cpx<T> v = czero<T>();
            if (kk < Kh && rr < rc) {
                const int kd = q < 2 ? kk : antipode(kk, K, nph);
                v = V[((int64_t)b * K + kd) * E + (q & 1) * R + r0 + rr];
            }
            vs[i] = v;
        }
        __syncthreads();
        const int kn = min(KT, Kh - k0);
        if (G > 1) {
            const int g = threadIdx.x / no, it = threadIdx.x - g * no;
            if (g < G) {
                const int n = it / rc, r = it % rc;
                for (int kl = g; kl < kn; kl += G) {
                    const cpx<T>* f = fs + (n * KT + kl) * 4;
                    const cpx<T>* v = vs + kl * 4 * RC + r;
                    recv_terms<T, MODE>(f[0], f[1], f[2], f[3], v[0], v[RC], aJ[0], aM[0]);
                    recv_terms<T, MODE>(cconj(f[0]), cnegconj(f[1]), cconj(f[2]), cnegconj(f[3]), v[2 * RC], v[3 * RC],
                                        aJ[0], aM[0]);
                }
            }
            continue;
        }
#pragma unroll
        for (int o = 0; o < OPT; ++o) {
            const int it = threadIdx.x + o * blockDim.x;
            if (it >= nb * rc) continue;
            const int n = it / rc, r = it % rc;
            for (int kl = 0; kl < kn; ++kl) {
                const cpx<T>* f = fs + (n * KT + kl) * 4;
                const cpx<T>* v = vs + kl * 4 * RC + r;
                recv_terms<T, MODE>(f[0], f[1], f[2], f[3], v[0], v[RC], aJ[o], aM[o]);
                recv_terms<T, MODE>(cconj(f[0]), cnegconj(f[1]), cconj(f[2]), cnegconj(f[3]), v[2 * RC], v[3 * RC], aJ[o],
                                    aM[o]);
            }
        }
    }
    if (G > 1) {
        // the groups' partial sums meet in the (now free) pattern stage: [G][no][2]
        __syncthreads();
        cpx<T>* red = fs;
        const int g = threadIdx.x / no, it = threadIdx.x - g * no;
        if (g < G) {
            red[(g * no + it) * 2] = aJ[0];
            red[(g * no + it) * 2 + 1] = aM[0];
        }
        __syncthreads();
        if (threadIdx.x < no) {
            cpx<T> sJ = czero<T>(), sM = czero<T>();
            for (int gg = 0; gg < G; ++gg) {
                sJ = cadd(sJ, red[(gg * no + threadIdx.x) * 2]);
                sM = cadd(sM, red[(gg * no + threadIdx.x) * 2 + 1]);
            }
            const int n = threadIdx.x / rc, r = r0 + threadIdx.x % rc, m = n0 + n, u = perm[m];
            if (MODE == 0) {
                y[(int64_t)r * nun + u] = cadd(yt[((int64_t)m * 2 + 0) * R + r], cscale(sJ, -c));
                y[(int64_t)r * nun + N + u] = cadd(yt[((int64_t)m * 2 + 1) * R + r], cscale(sM, c));
            } else {
                y[(int64_t)r * nun + u] = cadd(yt[(int64_t)m * R + r], cscale(sJ, -c));
            }
        }
        return;
    }
#pragma unroll
    for (int o = 0; o < OPT; ++o) {
        const int it = threadIdx.x + o * blockDim.x;
        if (it >= nb * rc) continue;
        const int n = it / rc, r = r0 + it % rc, m = n0 + n, u = perm[m];
        if (MODE == 0) {
            y[(int64_t)r * nun + u] = cadd(yt[((int64_t)m * 2 + 0) * R + r], cscale(aJ[o], -c));
            y[(int64_t)r * nun + N + u] = cadd(yt[((int64_t)m * 2 + 1) * R + r], cscale(aM[o], c));
        } else {
            y[(int64_t)r * nun + u] = cadd(yt[(int64_t)m * R + r], cscale(aJ[o], -c));
        }
    }
}

// ------------------------------------------------------------------ per-child interpolation / anterpolation
// One CTA per child box; the child's pattern, the pass intermediate and the interpolation
// tables live in shared memory, so every tap is a shared-memory read.
//  upward:   U_p[parent] += shift(oct) * Interp_phi(Interp_theta(U_c))   (float atomics into U_p,
//            which the caller zeroes; 8 children per parent)
//  downward: V_c += Anterp_theta(Anterp_phi(conj(shift(oct)) * V_p[parent]))
__device__ __forceinline__ void atomic_add_c(cpx<float>* p, cpx<float> v) {
    atomicAdd(reinterpret_cast<float2*>(p), make_float2(v.x, v.y));
}
__device__ __forceinline__ void atomic_add_c(cpx<double>* p, cpx<double> v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}

template <typename T>
__global__ void __launch_bounds__(256) k_interp_child(int nthc, int nphc, int nthp, int nphp, int E, int pth, int pph,
                                                      const int* __restrict__ th_src, const int* __restrict__ th_flip,
                                                      const T* __restrict__ th_w, const int* __restrict__ ph_src,
                                                      const T* __restrict__ ph_w, const int* __restrict__ parent,
                                                      const int* __restrict__ octant, const cpx<T>* __restrict__ shift,
                                                      const int* __restrict__ order,
                                                      const cpx<T>* __restrict__ Uc, cpx<T>* __restrict__ Up) {
    extern __shared__ unsigned char smem_raw[];
    const int Kc = nthc * nphc, Kp = nthp * nphp;
    cpx<T>* s1 = reinterpret_cast<cpx<T>*>(smem_raw);        // [Kc][E]
    cpx<T>* s2 = s1 + (size_t)Kc * E;                        // [nthp][nphc][E]
    T* tw = reinterpret_cast<T*>(s2 + (size_t)nthp * nphc * E);  // theta weights (sign folded) [nthp*pth]
    T* pw = tw + nthp * pth;                                 // phi weights [nphp*pph]
    int* tsrc = reinterpret_cast<int*>(pw + nphp * pph);     // theta source row*nphc + column shift flag
    int* psrc = tsrc + nthp * pth;                           // phi source column
    const int cb = order[blockIdx.x];
    const int half = nphc / 2;
    for (int i = threadIdx.x; i < nthp * pth; i += blockDim.x) {
        const int f = th_flip[i];
        tw[i] = f ? -th_w[i] : th_w[i];
        tsrc[i] = th_src[i] * 2 + f;
    }
    for (int i = threadIdx.x; i < nphp * pph; i += blockDim.x) {
        pw[i] = ph_w[i];
        psrc[i] = ph_src[i];
    }
    const cpx<T>* u = Uc + (int64_t)cb * Kc * E;
    for (int i = threadIdx.x; i < Kc * E; i += blockDim.x) s1[i] = u[i];
    __syncthreads();
    // theta pass: thread owns one (column, component) slot of a row and walks the rows
    const int W = nphc * E, Wp = nphp * E;
    for (int cbase = 0; cbase < W; cbase += blockDim.x) {
        const int lanes = min(W - cbase, (int)blockDim.x);
        const int rpp = blockDim.x / lanes;
        const int col = cbase + threadIdx.x % lanes, r0 = threadIdx.x / lanes;
        if (r0 >= rpp) continue;
        const int jc = col / E, e = col - jc * E;
        const int off0 = col, off1 = ((jc + half) % nphc) * E + e;
        for (int ip = r0; ip < nthp; ip += rpp) {
            cpx<T> a = czero<T>();
            for (int t = 0; t < pth; ++t) {
                const int code = tsrc[ip * pth + t];
                const cpx<T> v = s1[(code >> 1) * W + ((code & 1) ? off1 : off0)];
                const T w = tw[ip * pth + t];
                a.x = fma(w, v.x, a.x);
                a.y = fma(w, v.y, a.y);
            }
            s2[ip * W + col] = a;
        }
    }
    __syncthreads();
    const cpx<T>* sh = shift + (int64_t)octant[cb] * Kp;
    cpx<T>* up = Up + (int64_t)parent[cb] * Kp * E;
    for (int cbase = 0; cbase < Wp; cbase += blockDim.x) {
        const int lanes = min(Wp - cbase, (int)blockDim.x);
        const int rpp = blockDim.x / lanes;
        const int col = cbase + threadIdx.x % lanes, r0 = threadIdx.x / lanes;
        if (r0 >= rpp) continue;
        const int jp = col / E, e = col - jp * E;
        const int* ps = psrc + jp * pph;
        const T* pwj = pw + jp * pph;
        for (int ip = r0; ip < nthp; ip += rpp) {
            const cpx<T>* row = s2 + ip * W + e;
            cpx<T> a = czero<T>();
            for (int q = 0; q < pph; ++q) {
                const cpx<T> v = row[ps[q] * E];
                a.x = fma(pwj[q], v.x, a.x);
                a.y = fma(pwj[q], v.y, a.y);
            }
            atomic_add_c(up + ip * Wp + col, cmul(sh[ip * nphp + jp], a));
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_anterp_child(int nthc, int nphc, int nthp, int nphp, int E, int ntph, int ntth,
                                                      const int* __restrict__ tph_ptr, const int* __restrict__ tph_dst,
                                                      const T* __restrict__ tph_w, const int* __restrict__ tth_ptr,
                                                      const int* __restrict__ tth_dst, const int* __restrict__ tth_flip,
                                                      const T* __restrict__ tth_w, const int* __restrict__ parent,
                                                      const int* __restrict__ octant, const cpx<T>* __restrict__ shift,
                                                      const cpx<T>* __restrict__ Vp, cpx<T>* __restrict__ Vc) {
    extern __shared__ unsigned char smem_raw[];
    const int Kc = nthc * nphc, Kp = nthp * nphp;
    cpx<T>* s0 = reinterpret_cast<cpx<T>*>(smem_raw);        // conj(shift) * V_p  [Kp][E]
    cpx<T>* s2 = s0 + (size_t)Kp * E;                        // [nthp][nphc][E]
    T* pw = reinterpret_cast<T*>(s2 + (size_t)nthp * nphc * E);   // [ntph]
    T* tw = pw + ntph;                                            // [ntth] (sign folded)
    int* pptr = reinterpret_cast<int*>(tw + ntth);                // [nphc + 1]
    int* pdst = pptr + nphc + 1;                                  // [ntph]
    int* tptr = pdst + ntph;                                      // [nthc + 1]
    int* tdst = tptr + nthc + 1;                                  // [ntth]: parent row * 2 + flip
    const int cb = blockIdx.x;
    const int half = nphc / 2;
    for (int i = threadIdx.x; i < ntph; i += blockDim.x) { pw[i] = tph_w[i]; pdst[i] = tph_dst[i]; }
    for (int i = threadIdx.x; i < ntth; i += blockDim.x) {
        const int f = tth_flip[i];
        tw[i] = f ? -tth_w[i] : tth_w[i];
        tdst[i] = tth_dst[i] * 2 + f;
    }
    for (int i = threadIdx.x; i <= nphc; i += blockDim.x) pptr[i] = tph_ptr[i];
    for (int i = threadIdx.x; i <= nthc; i += blockDim.x) tptr[i] = tth_ptr[i];
    const cpx<T>* sh = shift + (int64_t)octant[cb] * Kp;
    const cpx<T>* vp = Vp + (int64_t)parent[cb] * Kp * E;
    for (int i = threadIdx.x; i < Kp * E; i += blockDim.x) s0[i] = cmulc(sh[i / E], vp[i]);
    __syncthreads();
    const int W = nphc * E, Wp = nphp * E;
    for (int cbase = 0; cbase < W; cbase += blockDim.x) {
        const int lanes = min(W - cbase, (int)blockDim.x);
        const int rpp = blockDim.x / lanes;
        const int col = cbase + threadIdx.x % lanes, r0 = threadIdx.x / lanes;
        if (r0 >= rpp) continue;
        const int jc = col / E, e = col - jc * E;
        const int q0 = pptr[jc], q1 = pptr[jc + 1];
        for (int ip = r0; ip < nthp; ip += rpp) {
            const cpx<T>* row = s0 + ip * Wp + e;
            cpx<T> a = czero<T>();
            for (int q = q0; q < q1; ++q) {
                const cpx<T> v = row[pdst[q] * E];
                a.x = fma(pw[q], v.x, a.x);
                a.y = fma(pw[q], v.y, a.y);
            }
            s2[ip * W + col] = a;
        }
    }
    __syncthreads();
    cpx<T>* vc = Vc + (int64_t)cb * Kc * E;
    for (int cbase = 0; cbase < W; cbase += blockDim.x) {
        const int lanes = min(W - cbase, (int)blockDim.x);
        const int rpp = blockDim.x / lanes;
        const int col = cbase + threadIdx.x % lanes, r0 = threadIdx.x / lanes;
        if (r0 >= rpp) continue;
        const int jc = col / E, e = col - jc * E;
        const int off0 = col, off1 = ((jc + half) % nphc) * E + e;
        for (int ic = r0; ic < nthc; ic += rpp) {
            cpx<T> a = czero<T>();
            for (int q = tptr[ic]; q < tptr[ic + 1]; ++q) {
                const int code = tdst[q];
                const cpx<T> v = s2[(code >> 1) * W + ((code & 1) ? off1 : off0)];
                a.x = fma(tw[q], v.x, a.x);
                a.y = fma(tw[q], v.y, a.y);
            }
            vc[ic * W + col] = cadd(vc[ic * W + col], a);
        }
    }
}

// ------------------------------------------------------------------ leaf receive with the final permutation
// y_user[perm[m]] = y_near[m] + far part (the near result in tree order is added here).
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_receive2(int N, int K, int nph, int R, int nun, const int* __restrict__ perm,
                                                  const int* __restrict__ leaf_of, const cpx<T>* __restrict__ F,
                                                  const cpx<T>* __restrict__ RX, const cpx<T>* __restrict__ V, T c,
                                                  const cpx<T>* __restrict__ yt, cpx<T>* __restrict__ y) {
    // one warp per (tree RWG m, RHS r); lanes stride over directions, then a shuffle reduction
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= N * R) return;
    const int m = warp / R, r = warp % R;
    const int b = leaf_of[m];
    const int E = 2 * R;
    const int Kh = K / 2;
    cpx<T> sJ = czero<T>(), sM = czero<T>();
    // lanes over the stored directions; each pattern load serves kk and its antipode
#pragma unroll 2
    for (int kk = lane; kk < Kh; kk += 32) {
        cpx<T> Ft, Fp, Xt, Xp;
        load_pair(F + ((int64_t)m * Kh + kk) * 2, Ft, Fp);
        load_pair(RX + ((int64_t)m * Kh + kk) * 2, Xt, Xp);
        const int ka = antipode(kk, K, nph);
        const cpx<T> Vt = V[((int64_t)b * K + kk) * E + r], Vp = V[((int64_t)b * K + kk) * E + R + r];
        const cpx<T> Wt = V[((int64_t)b * K + ka) * E + r], Wp = V[((int64_t)b * K + ka) * E + R + r];
        recv_terms<T, MODE>(Ft, Fp, Xt, Xp, Vt, Vp, sJ, sM);
        recv_terms<T, MODE>(cconj(Ft), cnegconj(Fp), cconj(Xt), cnegconj(Xp), Wt, Wp, sJ, sM);
    }
    sJ = warp_sum(sJ);
    if (MODE == 0) sM = warp_sum(sM);
    if (lane == 0) {
        const int u = perm[m];
        if (MODE == 0) {
            y[(int64_t)r * nun + u] = cadd(yt[((int64_t)m * 2 + 0) * R + r], cscale(sJ, -c));
            y[(int64_t)r * nun + N + u] = cadd(yt[((int64_t)m * 2 + 1) * R + r], cscale(sM, c));
        } else {
            y[(int64_t)r * nun + u] = cadd(yt[(int64_t)m * R + r], cscale(sJ, -c));
        }
    }
}

// ------------------------------------------------------------------ complex wavenumber (lossy medium)
// The leaf patterns are stored for every direction ([N][K][2]): at complex k the receive
// pattern R_m(khat) = int f_m exp(-jk khat.(r - c)) is not conj F_m, but it is F_m at the
// antipode -khat (theta-hat the same there, phi-hat reversed): R = (F_theta, -F_phi)(-khat).
// Aggregation: U_b(k) = sum_n ( -x_J,n F_n(k) + x_M,n khat x F_n(k) ), thread per (direction, entry).
// MODE 3 (one medium of the two-region form): two fields per box, E = 4R entries per direction,
//   U_E = a x_J F - x_M khat x F,   U_H = x_J F - b x_M khat x F      ((khat x F) = (-F_phi, F_theta)).
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_aggregate_full(int N, int K, int R, int nun, const int* __restrict__ perm,
                                                        const int* __restrict__ leaf_start, const cpx<T>* __restrict__ F,
                                                        const cpx<T>* __restrict__ x, cpx<T>* __restrict__ U, cpx<T> pa,
                                                        cpx<T> pb) {
    const int b = blockIdx.x;
    const int E = (MODE == 3 ? 4 : 2) * R;
    const int64_t idx = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)K * E) return;
    const int kk = (int)(idx / E), e = (int)(idx % E);
    const int c = (e / R) & 1, r = e % R, fld = e / (2 * R);
    cpx<T> acc = czero<T>();
    for (int n = leaf_start[b]; n < leaf_start[b + 1]; ++n) {
        const cpx<T> Ft = F[((int64_t)n * K + kk) * 2], Fp = F[((int64_t)n * K + kk) * 2 + 1];
        const int u = perm[n];
        const cpx<T> xJ = x[(int64_t)r * nun + u];
        if (MODE == 3) {
            const cpx<T> xM = x[(int64_t)r * nun + N + u];
            const cpx<T> sJ = fld == 0 ? cmul(pa, xJ) : xJ;    // coefficient of F
            const cpx<T> sM = fld == 0 ? xM : cmul(pb, xM);    // coefficient of -khat x F
            // theta: sJ Ft + sM Fp;  phi: sJ Fp - sM Ft
            acc = c == 0 ? cadd(acc, cadd(cmul(sJ, Ft), cmul(sM, Fp))) : cadd(acc, csub(cmul(sJ, Fp), cmul(sM, Ft)));
        } else if (MODE == 0) {
            const cpx<T> xM = x[(int64_t)r * nun + N + u];
            acc = c == 0 ? csub(acc, cadd(cmul(xJ, Ft), cmul(xM, Fp))) : cadd(acc, csub(cmul(xM, Ft), cmul(xJ, Fp)));
        } else {
            acc = csub(acc, cmul(xJ, c == 0 ? Ft : Fp));
        }
    }
    U[((int64_t)b * K) * E + idx] = acc;
}

// Receive: y_J = yt_J - cc sum_k [ R.V - RX.(khat x V) ],  y_M = yt_M + cc sum_k [ -R.(khat x V) - RX.V ]
// with the complex constant cc = k^2 / (32 pi^2); one warp per (tree RWG m, RHS r).
// MODE 3: y_E = yt_E - cc sum_k R.V_E,  y_H = yt_H - cc sum_k R.(khat x V_H), cc = k^2 / (16 pi^2).
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_receive_full(int N, int K, int nph, int R, int nun, const int* __restrict__ perm,
                                                      const int* __restrict__ leaf_of, const cpx<T>* __restrict__ F,
                                                      const cpx<T>* __restrict__ RX, const cpx<T>* __restrict__ V,
                                                      cpx<T> cc, const cpx<T>* __restrict__ yt, cpx<T>* __restrict__ y) {
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= N * R) return;
    const int m = warp / R, r = warp % R;
    const int b = leaf_of[m];
    const int E = (MODE == 3 ? 4 : 2) * R;
    cpx<T> sJ = czero<T>(), sM = czero<T>();
    for (int kk = lane; kk < K; kk += 32) {
        const int ka = antipode(kk, K, nph);
        const cpx<T> Rt = F[((int64_t)m * K + ka) * 2];
        const cpx<T> Fa = F[((int64_t)m * K + ka) * 2 + 1];
        const cpx<T> Rp = {-Fa.x, -Fa.y};
        if (MODE == 3) {
            const cpx<T>* v = V + ((int64_t)b * K + kk) * E + r;
            const cpx<T> Et = v[0], Ep = v[R], Ht = v[2 * R], Hp = v[3 * R];
            sJ = cadd(sJ, cadd(cmul(Rt, Et), cmul(Rp, Ep)));   // R.V_E
            sM = cadd(sM, csub(cmul(Rp, Ht), cmul(Rt, Hp)));   // R.(khat x V_H)
            continue;
        }
        const cpx<T> Xt = RX[((int64_t)m * K + kk) * 2], Xp = RX[((int64_t)m * K + kk) * 2 + 1];
        const cpx<T> Vt = V[((int64_t)b * K + kk) * E + r], Vp = V[((int64_t)b * K + kk) * E + R + r];
        sJ = cadd(sJ, cadd(csub(cadd(cmul(Rt, Vt), cmul(Rp, Vp)), cmul(Xp, Vt)), cmul(Xt, Vp)));
        if (MODE == 0) sM = cadd(sM, csub(csub(cmul(Rt, Vp), cmul(Rp, Vt)), cadd(cmul(Xt, Vt), cmul(Xp, Vp))));
    }
    sJ = warp_sum(sJ);
    if (MODE == 0 || MODE == 3) sM = warp_sum(sM);
    if (lane == 0) {
        const int u = perm[m];
        const cpx<T> nc = {-cc.x, -cc.y};
        if (MODE == 3) {
            y[(int64_t)r * nun + u] = cadd(yt[((int64_t)m * 2 + 0) * R + r], cmul(nc, sJ));
            y[(int64_t)r * nun + N + u] = cadd(yt[((int64_t)m * 2 + 1) * R + r], cmul(nc, sM));
        } else if (MODE == 0) {
            y[(int64_t)r * nun + u] = cadd(yt[((int64_t)m * 2 + 0) * R + r], cmul(nc, sJ));
            y[(int64_t)r * nun + N + u] = cadd(yt[((int64_t)m * 2 + 1) * R + r], cmul(cc, sM));
        } else {
            y[(int64_t)r * nun + u] = cadd(yt[(int64_t)m * R + r], cmul(nc, sJ));
        }
    }
}

inline unsigned nblk(int64_t n, int th) { return (unsigned)((n + th - 1) / th); }

// complex wavenumber: aggregation and receive on the full pattern layout (any R)
template <typename T>
void launch_aggregate_full(bi_handle_s* h, const cpx<T>* x, int R, cudaStream_t s) {
    level_t& L = h->lev[h->leaf];
    dim3 g(L.nbox, nblk((int64_t)L.K * 2 * h->nF * R, 256));
    const cpx<T> pa = {(T)h->pa[0], (T)h->pa[1]}, pb = {(T)h->pb[0], (T)h->pb[1]};
    if (h->prm.op_mode == 3)
        k_aggregate_full<T, 3><<<g, 256, 0, s>>>(h->N, L.K, R, h->nun, h->d_perm, h->d_leaf_start, (const cpx<T>*)h->d_F, x,
                                                 (cpx<T>*)L.d_U, pa, pb);
    else if (h->prm.op_mode == 0)
        k_aggregate_full<T, 0><<<g, 256, 0, s>>>(h->N, L.K, R, h->nun, h->d_perm, h->d_leaf_start, (const cpx<T>*)h->d_F, x,
                                                 (cpx<T>*)L.d_U, pa, pb);
    else
        k_aggregate_full<T, 1><<<g, 256, 0, s>>>(h->N, L.K, R, h->nun, h->d_perm, h->d_leaf_start, (const cpx<T>*)h->d_F, x,
                                                 (cpx<T>*)L.d_U, pa, pb);
    CU(cudaGetLastError());
}
template <typename T>
void launch_receive_full(bi_handle_s* h, cpx<T>* y, int R, cudaStream_t s) {
    level_t& L = h->lev[h->leaf];
    const double pi = 3.14159265358979323846;
    // k^2 / (32 pi^2) at complex k (k^2 / (16 pi^2) for one medium of the two-region form)
    const double kr = h->k, ki = h->ki, den = (h->prm.op_mode == 3 ? 16.0 : 32.0) * pi * pi;
    const cpx<T> cc = {(T)((kr * kr - ki * ki) / den), (T)(2.0 * kr * ki / den)};
    const int64_t nthreads = (int64_t)h->N * R * 32;
    if (h->prm.op_mode == 3)
        k_receive_full<T, 3><<<nblk(nthreads, 256), 256, 0, s>>>(h->N, L.K, L.nph, R, h->nun, h->d_perm, h->d_leaf_of,
                                                                 (const cpx<T>*)h->d_F, (const cpx<T>*)h->d_RX,
                                                                 (const cpx<T>*)L.d_V, cc, (const cpx<T>*)h->d_yt, y);
    else if (h->prm.op_mode == 0)
        k_receive_full<T, 0><<<nblk(nthreads, 256), 256, 0, s>>>(h->N, L.K, L.nph, R, h->nun, h->d_perm, h->d_leaf_of,
                                                                 (const cpx<T>*)h->d_F, (const cpx<T>*)h->d_RX,
                                                                 (const cpx<T>*)L.d_V, cc, (const cpx<T>*)h->d_yt, y);
    else
        k_receive_full<T, 1><<<nblk(nthreads, 256), 256, 0, s>>>(h->N, L.K, L.nph, R, h->nun, h->d_perm, h->d_leaf_of,
                                                                 (const cpx<T>*)h->d_F, (const cpx<T>*)h->d_RX,
                                                                 (const cpx<T>*)L.d_V, cc, (const cpx<T>*)h->d_yt, y);
    CU(cudaGetLastError());
}

template <typename T>
void launch_interp_two_pass(bi_handle_s* h, int l, int E, cudaStream_t s) {
    level_t& P = h->lev[l];
    level_t& Cc = h->lev[l + 1];
    interp_t& I = h->itp[l];
    const int th = 256;
    typedef cpx<T> C;
    dim3 g1(Cc.nbox, nblk((int64_t)P.nth * Cc.nph * E, th));
    dim3 g2(P.nbox, nblk((int64_t)P.K * E, th));
#define BI_TH(PP) k_interp_theta<T, PP><<<g1, th, 0, s>>>(P.nth, Cc.nph, Cc.K, E, I.p_th, I.d_th_src, I.d_th_flip, \
                                                          (const T*)I.d_th_w, (const C*)Cc.d_U, (C*)I.d_tmp)
#define BI_PH(PP) k_interp_phi<T, PP><<<g2, th, 0, s>>>(P.nth, P.nph, Cc.nph, E, I.p_ph, I.d_ph_src, (const T*)I.d_ph_w, \
                                                        P.d_child_ptr, Cc.d_octant, (const C*)P.d_shift, \
                                                        (const C*)I.d_tmp, (C*)P.d_U)
    switch (I.p_th) {
        case 4: BI_TH(4); break;
        case 6: BI_TH(6); break;
        case 8: BI_TH(8); break;
        case 10: BI_TH(10); break;
        case 12: BI_TH(12); break;
        case 16: BI_TH(16); break;
        default: BI_TH(0); break;
    }
    CU(cudaGetLastError());
    switch (I.p_ph) {
        case 4: BI_PH(4); break;
        case 6: BI_PH(6); break;
        case 8: BI_PH(8); break;
        case 10: BI_PH(10); break;
        case 12: BI_PH(12); break;
        case 16: BI_PH(16); break;
        default: BI_PH(0); break;
    }
#undef BI_TH
#undef BI_PH
    CU(cudaGetLastError());
}



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
            dim3 g(L.nbox, nblk((int64_t)L.K * E, th));
            if (h->prm.op_mode == 0)
                k_aggregate<T, 0><<<g, th, 0, s>>>(L.K, L.nph, R, h->d_leaf_start, (const C*)h->d_F, xt, (C*)L.d_U);
            else
                k_aggregate<T, 1><<<g, th, 0, s>>>(L.K, L.nph, R, h->d_leaf_start, (const C*)h->d_F, xt, (C*)L.d_U);
            CU(cudaGetLastError());
        }
        if (ev) CU(cudaEventRecord(ev[2], s));
        // upward pass
        for (int l = lf - 1; l >= 2; --l) {
            level_t& P = h->lev[l];
            level_t& Cc = h->lev[l + 1];
            interp_t& I = h->itp[l];
            (void)P; (void)Cc; (void)I;
            launch_interp_two_pass<T>(h, l, E, s);
        }
        if (ev) CU(cudaEventRecord(ev[3], s));
        // translations on every level
        for (int l = 2; l <= lf; ++l) {
            level_t& L = h->lev[l];
            dim3 g(L.nbox, nblk((int64_t)L.K * E, th));
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
            dim3 g1(Cc.nbox, nblk((int64_t)P.nth * Cc.nph * E, th));
            k_anterp_phi<T><<<g1, th, 0, s>>>(P.nth, P.nph, Cc.nph, E, I.d_tph_ptr, I.d_tph_dst, (const T*)I.d_tph_w,
                                              Cc.d_parent, Cc.d_octant, (const C*)P.d_shift_dn, (const C*)P.d_V, (C*)I.d_tmp);
            CU(cudaGetLastError());
            dim3 g2(Cc.nbox, nblk((int64_t)Cc.K * E, th));
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
                k_receive<T, 0><<<nblk(nthreads, th), th, 0, s>>>(N, L.K, L.nph, R, h->d_leaf_of, (const C*)h->d_F,
                                                                   (const C*)h->d_RX, (const C*)L.d_V, c, yf);
            else
                k_receive<T, 1><<<nblk(nthreads, th), th, 0, s>>>(N, L.K, L.nph, R, h->d_leaf_of, (const C*)h->d_F,
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


template <typename T, int MODE, int RT>
void launch_near_stream(bi_handle_s* h, const cpx<T>* x, cpx<T>* yt, cpx<T>* yuser, int R, cudaStream_t s) {
    const int NX = MODE == 0 ? 2 : 1;
    size_t smem = (size_t)h->near_ncol_max * NX * RT * sizeof(cpx<T>);
    auto kern = k_near_stream<T, MODE, RT>;
    bi_raise_smem(kern, smem);
    kern<<<h->near_nwork, 256, smem, s>>>(h->N, R, h->nun, h->d_perm, (const int2*)h->d_near_work, h->d_leaf_start,
                                          h->d_near_ptr, h->d_near_src,
                                                 h->d_near_blk, h->d_near_col0, h->d_near_ncol, (const cpx<T>*)h->d_near,
                                                 h->d_gram_ptr, h->d_gram_seg,
                                                 (const T*)h->d_gram_val, x, yt, yuser);
    CU(cudaGetLastError());
}

template <typename T, int MODE, int RT>
void launch_near_multi(bi_handle_s* h, cpx<T>* yt, cpx<T>* yuser, int R, cudaStream_t s) {
    const int NX = (MODE == 0 || MODE == 3) ? 2 : 1;
    size_t smem = (size_t)h->near_ncol_max * NX * RT * sizeof(cpx<T>);
    auto kern = k_near_multi<T, MODE, RT>;
    bi_raise_smem(kern, smem);
    kern<<<h->near_nwork, 256, smem, s>>>(h->N, R, h->nun, h->d_perm, (const int2*)h->d_near_work, h->d_leaf_start,
                                          h->d_near_ptr, h->d_near_src, h->d_near_blk, h->d_near_col0, h->d_near_ncol,
                                          (const cpx<T>*)h->d_near, h->d_gram_ptr, h->d_gram_seg, (const T*)h->d_gram_val,
                                          (const cpx<T>*)h->d_xt, yt, yuser, cpx<T>{(T)h->pa[0], (T)h->pa[1]},
                                          cpx<T>{(T)h->pb[0], (T)h->pb[1]});
    CU(cudaGetLastError());
}

template <typename T, int MODE, int RT>
bool launch_near_rb(bi_handle_s* h, cpx<T>* yt, cpx<T>* yuser, int R, cudaStream_t s) {
    constexpr int NX = MODE == 0 ? 2 : 1;
    const size_t smem = (size_t)h->near_ncol_max * RT * NX * sizeof(cpx<T>);
    if (smem > 110 * 1024) return false;
    auto kern = k_near_rb<T, MODE, RT>;
    bi_raise_smem(kern, smem);
    kern<<<h->near_nwork, 256, smem, s>>>(h->N, R, h->nun, h->d_perm, (const int2*)h->d_near_work, h->d_leaf_start,
                                          h->d_near_ptr, h->d_near_src, h->d_near_blk, h->d_near_col0, h->d_near_ncol,
                                          (const cpx<T>*)h->d_near, h->d_gram_ptr, h->d_gram_seg, (const T*)h->d_gram_val,
                                          (const cpx<T>*)h->d_xt, yt, yuser);
    CU(cudaGetLastError());
    return true;
}

template <typename T, int MODE>
void launch_near_any(bi_handle_s* h, const cpx<T>* x, cpx<T>* yt, cpx<T>* yuser, int R, cudaStream_t s) {
    if (MODE == 3) {
        // one medium of the two-region form: the tree-ordered kernel for every R
        if ((size_t)h->near_ncol_max * 2 * 4 * sizeof(cpx<T>) > 200 * 1024)
            throw bi_error{BI_ERR_ARG, "two-region near field: a leaf box's near segment is too wide"};
        const int64_t nvec = (int64_t)h->N * h->nX * R;
        k_gather_x<T><<<nblk(nvec, 256), 256, 0, s>>>(h->N, h->nX, R, h->nun, h->d_perm, x, (cpx<T>*)h->d_xt);
        CU(cudaGetLastError());
        if (R == 1) launch_near_multi<T, 3, 1>(h, yt, yuser, R, s);
        else if (R == 2) launch_near_multi<T, 3, 2>(h, yt, yuser, R, s);
        else launch_near_multi<T, 3, 4>(h, yt, yuser, R, s);
        return;
    }
    if ((size_t)h->near_ncol_max * 2 * sizeof(cpx<T>) > 160 * 1024) {
        // rows of one box exceed the CTA: the row-per-thread kernel on tree-ordered vectors
        const int64_t nvec = (int64_t)h->N * h->nX * R;
        k_gather_x<T><<<nblk(nvec, 256), 256, 0, s>>>(h->N, h->nX, R, h->nun, h->d_perm, x, (cpx<T>*)h->d_xt);
        k_near<T, MODE><<<h->lev[h->leaf].nbox, 128, 0, s>>>(R, h->d_leaf_start, h->d_near_ptr, h->d_near_src, h->d_near_blk,
                                                            (const cpx<T>*)h->d_near, h->d_gram_ptr, h->d_gram_col,
                                                            (const T*)h->d_gram_val, (const cpx<T>*)h->d_xt, yt);
        if (yuser)
            k_scatter_y<T><<<nblk(nvec, 256), 256, 0, s>>>(h->N, h->nX, R, h->nun, h->d_perm, yt, nullptr, yuser);
        CU(cudaGetLastError());
        return;
    }
    if (R == 1) {
        launch_near_stream<T, MODE, 1>(h, x, yt, yuser, R, s);
        return;
    }
    // several right-hand sides: x gathered once into tree order, then staged per work item
    const int64_t nvec = (int64_t)h->N * h->nX * R;
    k_gather_x<T><<<nblk(nvec, 256), 256, 0, s>>>(h->N, h->nX, R, h->nun, h->d_perm, x, (cpx<T>*)h->d_xt);
    CU(cudaGetLastError());
    if constexpr (MODE == 0 && sizeof(T) == 4) {
        if (h->near_rb == 2 && R >= 6 && R <= 8) {
            constexpr int NS = 6;
            const size_t smem = (size_t)8 * NS * 32 * 16 + (size_t)h->near_ncol_max * 8 * 2 * sizeof(cpx<T>);
            if (smem <= 110 * 1024) {
                bi_raise_smem(k_near_rbp<8, NS>, smem);
                k_near_rbp<8, NS><<<h->near_nwork, 256, smem, s>>>(
                    h->N, R, h->nun, h->d_perm, (const int2*)h->d_near_work, h->d_leaf_start, h->d_near_ptr,
                    h->d_near_src, h->d_near_blk, h->d_near_col0, h->d_near_ncol, (const cpx<float>*)h->d_near,
                    h->d_gram_ptr, h->d_gram_seg, (const float*)h->d_gram_val, (const cpx<float>*)h->d_xt,
                    (cpx<float>*)yt, (cpx<float>*)yuser);
                CU(cudaGetLastError());
                return;
            }
        }
    }
    if constexpr (MODE == 0 || MODE == 1) {
        // the row-pair kernel for one chunk of right-hand sides (measured: 25% faster than the
        // per-row kernel at R = 8, 10% slower at R = 64, where x is restaged per chunk)
        if (h->near_rb && R >= 3 && R <= 8) {
            if (R >= 6 && launch_near_rb<T, MODE, 8>(h, yt, yuser, R, s)) return;
            if (launch_near_rb<T, MODE, 4>(h, yt, yuser, R, s)) return;
        }
    }
    if (R == 2) launch_near_multi<T, MODE, 2>(h, yt, yuser, R, s);
    else if (R <= 4 || (size_t)h->near_ncol_max * 2 * 8 * sizeof(cpx<T>) > 160 * 1024) launch_near_multi<T, MODE, 4>(h, yt, yuser, R, s);
    else launch_near_multi<T, MODE, 8>(h, yt, yuser, R, s);
}



template <typename T>
size_t interp_child_smem(bi_handle_s* h, int l, int E) {
    const level_t& P = h->lev[l];
    const level_t& C = h->lev[l + 1];
    const interp_t& I = h->itp[l];
    return ((size_t)C.K * E + (size_t)P.nth * C.nph * E) * sizeof(cpx<T>) +
           ((size_t)P.nth * I.p_th + (size_t)P.nph * I.p_ph) * (sizeof(T) + sizeof(int));
}
template <typename T>
size_t anterp_child_smem(bi_handle_s* h, int l, int E) {
    const level_t& P = h->lev[l];
    const level_t& C = h->lev[l + 1];
    const interp_t& I = h->itp[l];
    return ((size_t)P.K * E + (size_t)P.nth * C.nph * E) * sizeof(cpx<T>) +
           (I.tph_dst.size() + I.tth_dst.size()) * (sizeof(T) + sizeof(int)) + (size_t)(C.nph + C.nth + 2) * sizeof(int);
}

template <typename T>
bool interp_child(bi_handle_s* h, int l, int E, cudaStream_t s) {
    level_t& P = h->lev[l];
    level_t& C = h->lev[l + 1];
    interp_t& I = h->itp[l];
    size_t smem = interp_child_smem<T>(h, l, E);
    if (smem > 180 * 1024) return false;
    bi_raise_smem(k_interp_child<T>, smem);
    CU(cudaMemsetAsync(P.d_U, 0, (size_t)P.nbox * P.K * E * sizeof(cpx<T>), s));
    k_interp_child<T><<<C.nbox, 256, smem, s>>>(C.nth, C.nph, P.nth, P.nph, E, I.p_th, I.p_ph, I.d_th_src, I.d_th_flip,
                                                (const T*)I.d_th_w, I.d_ph_src, (const T*)I.d_ph_w, C.d_parent, C.d_octant,
                                                (const cpx<T>*)P.d_shift, C.d_child_order, (const cpx<T>*)C.d_U,
                                                (cpx<T>*)P.d_U);
    CU(cudaGetLastError());
    return true;
}

template <typename T>
bool anterp_child(bi_handle_s* h, int l, int E, cudaStream_t s) {
    level_t& P = h->lev[l];
    level_t& C = h->lev[l + 1];
    interp_t& I = h->itp[l];
    size_t smem = anterp_child_smem<T>(h, l, E);
    if (smem > 180 * 1024) return false;
    bi_raise_smem(k_anterp_child<T>, smem);
    k_anterp_child<T><<<C.nbox, 256, smem, s>>>(C.nth, C.nph, P.nth, P.nph, E, (int)I.tph_dst.size(), (int)I.tth_dst.size(),
                                                I.d_tph_ptr, I.d_tph_dst, (const T*)I.d_tph_w, I.d_tth_ptr, I.d_tth_dst,
                                                I.d_tth_flip, (const T*)I.d_tth_w, C.d_parent, C.d_octant,
                                                (const cpx<T>*)P.d_shift_dn, (const cpx<T>*)P.d_V, (cpx<T>*)C.d_V);
    CU(cudaGetLastError());
    return true;
}


template <typename T, int OPT>
bool launch_receive_tile_opt(bi_handle_s* h, cpx<T>* y, int R, cudaStream_t s) {
    level_t& L = h->lev[h->leaf];
    // right-hand sides per CTA so that one thread holds at most OPT outputs
    int RC = std::min(R, (256 * OPT) / std::max(1, h->max_leaf_count));
    if (RC < 1) return false;
    size_t smem = ((size_t)h->max_leaf_count * 32 * 4 + (size_t)32 * 4 * RC) * sizeof(cpx<T>);
    if (smem > 200 * 1024) return false;
    const double pi = 3.14159265358979323846;
    const T c = (T)(h->k * h->k / (32.0 * pi * pi));
    if (h->prm.op_mode == 0) {
        if (smem > 48 * 1024)
            bi_raise_smem(k_receive_tile<T, 0, OPT>, smem);
        k_receive_tile<T, 0, OPT><<<dim3(L.nbox, (R + RC - 1) / RC), 256, smem, s>>>(h->N, L.K, L.nph, R, RC, h->nun, h->d_perm,
                                                                                   h->d_leaf_start,
                                                            (const cpx<T>*)h->d_F, (const cpx<T>*)h->d_RX,
                                                            (const cpx<T>*)L.d_V, c, (const cpx<T>*)h->d_yt, y);
    } else {
        if (smem > 48 * 1024)
            bi_raise_smem(k_receive_tile<T, 1, OPT>, smem);
        k_receive_tile<T, 1, OPT><<<dim3(L.nbox, (R + RC - 1) / RC), 256, smem, s>>>(h->N, L.K, L.nph, R, RC, h->nun, h->d_perm,
                                                                                   h->d_leaf_start,
                                                            (const cpx<T>*)h->d_F, (const cpx<T>*)h->d_RX,
                                                            (const cpx<T>*)L.d_V, c, (const cpx<T>*)h->d_yt, y);
    }
    CU(cudaGetLastError());
    return true;
}

template <typename T>
bool launch_receive_tile(bi_handle_s* h, const cpx<T>* x, cpx<T>* y, int R, cudaStream_t s) {
    (void)x;
    return launch_receive_tile_opt<T, 8>(h, y, R, s);
}

// The product: near (side stream) || aggregate -> interpolate -> translate -> anterpolate ->
// receive (+ near result, + permutation to user order).  Each step takes the first kernel
// family that applies: the bulk-copy leaf kernels (bi_leaf.cu), the level passes of
// bi_interp.cu and bi_translate.cu, then the per-child, tiled and two-pass kernels of this
// file (large RHS counts, shared memory that does not fit, or non-default tap counts).
template <typename T>
void launch_fast(bi_handle_s* h, const void* xv, void* yv, int R, cudaStream_t s, cudaStream_t side, cudaEvent_t* ev) {
    if (ev) side = s;
    typedef cpx<T> C;
    const C* x = (const C*)xv;
    C* y = (C*)yv;
    C* yt = (C*)h->d_yt;
    const int N = h->N, nun = h->nun, E = 2 * h->nF * R, th = 256;
    const bool far = h->leaf >= 2;
    const bool full = h->ki != 0.0 || h->prm.op_mode == 3;   // every direction of the leaf patterns stored
    if (ev) CU(cudaEventRecord(ev[0], s));
    if (!ev) {
        CU(cudaEventRecord(h->ev_fork, s));
        CU(cudaStreamWaitEvent(side, h->ev_fork, 0));
    }
    if (h->prm.op_mode == 3) launch_near_any<T, 3>(h, x, yt, far ? nullptr : y, R, side);
    else if (h->prm.op_mode == 0) launch_near_any<T, 0>(h, x, yt, far ? nullptr : y, R, side);
    else launch_near_any<T, 1>(h, x, yt, far ? nullptr : y, R, side);
    if (ev) CU(cudaEventRecord(ev[1], s));
    else CU(cudaEventRecord(h->ev_join, side));
    if (!far) {
        if (ev)
            for (int i = 2; i < BI_NSTAGES; ++i) CU(cudaEventRecord(ev[i], s));
        else
            CU(cudaStreamWaitEvent(s, h->ev_join, 0));
        return;
    }
    const int lf = h->leaf;
    if (full) {
        launch_aggregate_full<T>(h, x, R, s);
    } else if (R < 8 && bi_leaf_aggregate_bulk(h, x, R, s)) {
    } else if (R >= 8) {
        level_t& L = h->lev[lf];
        dim3 g(L.nbox, nblk(L.K / 2, 32));
        size_t smem = ((size_t)h->max_leaf_count * 32 * 2 + (size_t)h->max_leaf_count * 2 * R) * sizeof(C);
        if (smem > 48 * 1024) {
            bi_raise_smem(k_aggregate_tile<T, 0>, smem);
            bi_raise_smem(k_aggregate_tile<T, 1>, smem);
        }
        if (h->prm.op_mode == 0)
            k_aggregate_tile<T, 0><<<g, 256, smem, s>>>(N, L.K, L.nph, R, nun, h->d_perm, h->d_leaf_start, (const C*)h->d_F, x,
                                                        (C*)L.d_U);
        else
            k_aggregate_tile<T, 1><<<g, 256, smem, s>>>(N, L.K, L.nph, R, nun, h->d_perm, h->d_leaf_start, (const C*)h->d_F, x,
                                                        (C*)L.d_U);
        CU(cudaGetLastError());
    } else {
        level_t& L = h->lev[lf];
        dim3 g(L.nbox, nblk((int64_t)(L.K / 2) * R, 64));
        size_t smem = (size_t)h->max_leaf_count * 2 * R * sizeof(C);
        if (smem > 48 * 1024) {
            bi_raise_smem(k_aggregate2<T, 0>, smem);
            bi_raise_smem(k_aggregate2<T, 1>, smem);
        }
        if (h->prm.op_mode == 0)
            k_aggregate2<T, 0><<<g, th, smem, s>>>(N, L.K, L.nph, R, nun, h->d_perm, h->d_leaf_start, (const C*)h->d_F, x, (C*)L.d_U);
        else
            k_aggregate2<T, 1><<<g, th, smem, s>>>(N, L.K, L.nph, R, nun, h->d_perm, h->d_leaf_start, (const C*)h->d_F, x, (C*)L.d_U);
        CU(cudaGetLastError());
    }
    if (ev) CU(cudaEventRecord(ev[2], s));
    // Translations of level l only need U_l: the finer levels run on their own streams while
    // the upward pass continues, and join before the downward pass adds into V_l.
    auto translate = [&](int l, cudaStream_t st) {
        if (bi_translate_level(h, l, E, st)) return;
        level_t& L = h->lev[l];
        dim3 g(L.nbox, nblk((int64_t)L.K * E, th));
        k_translate<T><<<g, th, 0, st>>>(L.K, E, L.d_il_ptr, L.d_il_src, L.d_il_off, (const C*)L.d_T, (const C*)L.d_U,
                                         (C*)L.d_V);
        CU(cudaGetLastError());
    };
    auto fork_translate = [&](int l) {
        if (ev) return;  // profiling: translations are timed as one serial stage below
        cudaStream_t st = h->tstream[l];
        CU(cudaEventRecord(h->ev_tfork[l], s));
        CU(cudaStreamWaitEvent(st, h->ev_tfork[l], 0));
        translate(l, st);
        CU(cudaEventRecord(h->ev_tjoin[l], st));
    };
    if (lf > 2) fork_translate(lf);
    for (int l = lf - 1; l >= 2; --l) {
        // one CTA per parent only pays off when the level has enough parents to fill the GPU
        if (!bi_interp_level(h, l, E, s) && !interp_child<T>(h, l, E, s)) launch_interp_two_pass<T>(h, l, E, s);
        if (l > 2) fork_translate(l);
    }
    if (ev) CU(cudaEventRecord(ev[3], s));
    if (ev)
        for (int l = 2; l <= lf; ++l) translate(l, s);
    else
        translate(2, s);
    if (ev) CU(cudaEventRecord(ev[4], s));
    for (int l = 2; l < lf; ++l) {
        if (!ev) CU(cudaStreamWaitEvent(s, h->ev_tjoin[l + 1], 0));
        if (bi_anterp_level(h, l, E, s) || anterp_child<T>(h, l, E, s)) continue;
        level_t& P = h->lev[l];
        level_t& Cc = h->lev[l + 1];
        interp_t& I = h->itp[l];
        dim3 g1(Cc.nbox, nblk((int64_t)P.nth * Cc.nph * E, th));
        k_anterp_phi<T><<<g1, th, 0, s>>>(P.nth, P.nph, Cc.nph, E, I.d_tph_ptr, I.d_tph_dst, (const T*)I.d_tph_w,
                                          Cc.d_parent, Cc.d_octant, (const C*)P.d_shift_dn, (const C*)P.d_V, (C*)I.d_tmp);
        CU(cudaGetLastError());
        dim3 g2(Cc.nbox, nblk((int64_t)Cc.K * E, th));
        k_anterp_theta<T><<<g2, th, 0, s>>>(P.nth, Cc.nth, Cc.nph, E, I.d_tth_ptr, I.d_tth_dst, I.d_tth_flip,
                                            (const T*)I.d_tth_w, (const C*)I.d_tmp, (C*)Cc.d_V);
        CU(cudaGetLastError());
    }
    if (ev) CU(cudaEventRecord(ev[5], s));
    else CU(cudaStreamWaitEvent(s, h->ev_join, 0));
    if (full) {
        launch_receive_full<T>(h, y, R, s);
    } else if (R >= 8 && launch_receive_tile<T>(h, x, y, R, s)) {
    } else if (R < 8 && bi_leaf_receive_bulk(h, y, R, s)) {
    } else {
        level_t& L = h->lev[lf];
        const double pi = 3.14159265358979323846;
        T c = (T)(h->k * h->k / (32.0 * pi * pi));
        int64_t nthreads = (int64_t)N * R * 32;
        if (h->prm.op_mode == 0)
            k_receive2<T, 0><<<nblk(nthreads, th), th, 0, s>>>(N, L.K, L.nph, R, nun, h->d_perm, h->d_leaf_of, (const C*)h->d_F,
                                                                (const C*)h->d_RX, (const C*)L.d_V, c, yt, y);
        else
            k_receive2<T, 1><<<nblk(nthreads, th), th, 0, s>>>(N, L.K, L.nph, R, nun, h->d_perm, h->d_leaf_of, (const C*)h->d_F,
                                                                (const C*)h->d_RX, (const C*)L.d_V, c, yt, y);
        CU(cudaGetLastError());
    }
    if (ev) {
        CU(cudaEventRecord(ev[6], s));
        CU(cudaEventRecord(ev[7], s));
    }
}

}  // namespace

// Autotuner of the level passes: the first product with a given E = 2 nF nrhs times every
// applicable kernel form of each level pass once on the handle's own buffers (zeroed first:
// the values do not change the timing) and keeps the fastest per (pass, level, E):
//   translation: one or two pairs of entries per thread;
//   interpolation: chunks of 16, 8, 4 or 2 entries, or the two-pass form;
//   anterpolation: per child or in row blocks, chunks of 16, 8, 4 or 2 entries, or two-pass.
// Every later launch (and every captured graph) uses the choice.  It synchronises the stream.
void bi_autotune(bi_handle_s* h, int nrhs, cudaStream_t s) {
    const int E = 2 * h->nF * nrhs;
    if (!h->autotune || E <= 2 || h->leaf < 2) return;
    if (std::find(h->tuned_E.begin(), h->tuned_E.end(), E) != h->tuned_E.end()) return;
    h->tuned_E.push_back(E);
    for (int l = 2; l <= h->leaf; ++l) {
        const level_t& L = h->lev[l];
        const size_t sz = (size_t)L.nbox * L.K * E * h->csize;
        CU(cudaMemsetAsync(L.d_U, 0, sz, s));
        CU(cudaMemsetAsync(L.d_V, 0, sz, s));
    }
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    const std::vector<int> cand[3] = {{1, 2, 3, 4, 5, 6, 7, 8, 9},
                                      {116, 108, 104, 102, 2, 3},
                                      {116, 108, 104, 102, 216, 208, 204, 202, 2, 3}};
    try {
        for (int pass = 0; pass < 3; ++pass) {
            const int lmax = pass == 0 ? h->leaf : h->leaf - 1;
            for (int l = 2; l <= lmax; ++l) {
                int best = 0;
                double best_us = 1e300;
                for (int c : cand[pass]) {
                    h->force_variant = c;
                    auto run = [&] {
                        return pass == 0 ? bi_translate_level(h, l, E, s)
                                         : pass == 1 ? bi_interp_level(h, l, E, s) : bi_anterp_level(h, l, E, s);
                    };
                    if (!run()) continue;       // not applicable at this level (shared memory, E)
                    double us = 1e300;
                    for (int rep = 0; rep < 2; ++rep) {
                        CU(cudaEventRecord(e0, s));
                        run();
                        CU(cudaEventRecord(e1, s));
                        CU(cudaEventSynchronize(e1));
                        float ms = 0;
                        CU(cudaEventElapsedTime(&ms, e0, e1));
                        us = std::min(us, 1e3 * ms);
                    }
                    if (us < best_us) {
                        best_us = us;
                        best = c;
                    }
                }
                h->force_variant = -1;
                if (best) h->tuned.push_back({pass, l, E, best, best_us});
            }
        }
    } catch (...) {
        h->force_variant = -1;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    CU(cudaEventDestroy(e0));
    CU(cudaEventDestroy(e1));
}

// Enqueue one product on stream s (no graph).
static void matvec_enqueue(bi_handle_s* h, const void* x, void* y, int nrhs, cudaStream_t s, cudaStream_t side) {
    if (h->use_fast) {
        if (h->prec == 0) launch_fast<double>(h, x, y, nrhs, s, side, nullptr);
        else launch_fast<float>(h, x, y, nrhs, s, side, nullptr);
    } else {
        if (h->prec == 0) launch_all<double>(h, x, y, nrhs, s, side);
        else launch_all<float>(h, x, y, nrhs, s, side);
    }
}

template <typename T>
__global__ void k_add_vec(int64_t n, cpx<T>* __restrict__ y, const cpx<T>* __restrict__ a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = cadd(y[i], a[i]);
}

// Coated PEC body: inputs of the two media from x = [J1, M1, J2] (column-major [R][2 N1 + N2]):
//   outer medium (S1):  [J1; M1];   coat (S1 and S2):  x_J = [J1; -J2],  x_M = [M1; 0]
template <typename T>
__global__ void k_coated_in(int N1, int N2, int R, const cpx<T>* __restrict__ x, cpx<T>* __restrict__ x0,
                            cpx<T>* __restrict__ x1) {
    const int nun = 2 * N1 + N2, n1 = 2 * (N1 + N2);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)R * n1) return;
    const int r = (int)(i / n1), j = (int)(i % n1);
    const cpx<T>* xr = x + (int64_t)r * nun;
    cpx<T> v = czero<T>();
    if (j < N1) v = xr[j];                                     // J1
    else if (j < N1 + N2) v = cpx<T>{-xr[N1 + j].x, -xr[N1 + j].y};   // -J2 (x index 2 N1 + (j - N1))
    else if (j < 2 * N1 + N2) v = xr[j - N2];                  // M1 (x index N1 + (j - N1 - N2))
    x1[i] = v;
    if (j < 2 * N1) x0[(int64_t)r * 2 * N1 + j] = xr[j];
}
// rows: E and H of S1 = outer + coat; the core's row (tangential E = 0 on S2) = -(coat's E rows of S2)
template <typename T>
__global__ void k_coated_out(int N1, int N2, int R, const cpx<T>* __restrict__ y0, const cpx<T>* __restrict__ y1,
                             cpx<T>* __restrict__ y) {
    const int nun = 2 * N1 + N2, n1 = 2 * (N1 + N2);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)R * nun) return;
    const int r = (int)(i / nun), j = (int)(i % nun);
    const cpx<T>* a = y0 + (int64_t)r * 2 * N1;
    const cpx<T>* b = y1 + (int64_t)r * n1;
    cpx<T> v;
    if (j < N1) v = cadd(a[j], b[j]);
    else if (j < 2 * N1) v = cadd(a[j], b[N2 + j]);           // H rows of S1: coat index N1 + N2 + (j - N1)
    else v = cpx<T>{-b[j - N1].x, -b[j - N1].y};              // E rows of S2: coat index N1 + (j - 2 N1)
    y[i] = v;
}
template <typename T>
__global__ void k_coated_rhs(int N1, int N2, int R, const cpx<T>* __restrict__ b0, cpx<T>* __restrict__ b) {
    const int nun = 2 * N1 + N2;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)R * nun) return;
    const int r = (int)(i / nun), j = (int)(i % nun);
    b[i] = j < 2 * N1 ? b0[(int64_t)r * 2 * N1 + j] : czero<T>();
}

void bi_coated_outer_currents(bi_handle_s* h, const void* x, int R, cudaStream_t s) {
    const int64_t n = (int64_t)R * 2 * (h->N1 + h->N2);
    if (h->prec == 0)
        k_coated_in<double><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(h->N1, h->N2, R, (const cpx<double>*)x,
                                                                        (cpx<double>*)h->d_xin0, (cpx<double>*)h->d_xin1);
    else
        k_coated_in<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(h->N1, h->N2, R, (const cpx<float>*)x,
                                                                       (cpx<float>*)h->d_xin0, (cpx<float>*)h->d_xin1);
    CU(cudaGetLastError());
}

void bi_coated_rhs(bi_handle_s* h, void* b, int R, cudaStream_t s) {
    const int64_t n = (int64_t)R * h->nun;
    if (h->prec == 0)
        k_coated_rhs<double><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(h->N1, h->N2, R, (const cpx<double>*)h->d_y0,
                                                                         (cpx<double>*)b);
    else
        k_coated_rhs<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(h->N1, h->N2, R, (const cpx<float>*)h->d_y0,
                                                                        (cpx<float>*)b);
    CU(cudaGetLastError());
}

// One product: replayed from a CUDA graph captured on first use for this (x, y, nrhs).  The
// two-region operator sums the products of its two media; the coated body maps its unknowns to
// and from theirs.
void bi_matvec_launch(bi_handle_s* h, const void* x, void* y, int nrhs, cudaStream_t s) {
    if (h->coated) {
        bi_coated_outer_currents(h, x, nrhs, s);
        bi_matvec_launch(h->med[0], h->d_xin0, h->d_y0, nrhs, s);
        bi_matvec_launch(h->med[1], h->d_xin1, h->d_y1, nrhs, s);
        const int64_t n = (int64_t)nrhs * h->nun;
        if (h->prec == 0)
            k_coated_out<double><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(h->N1, h->N2, nrhs, (const cpx<double>*)h->d_y0,
                                                                              (const cpx<double>*)h->d_y1, (cpx<double>*)y);
        else
            k_coated_out<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(h->N1, h->N2, nrhs, (const cpx<float>*)h->d_y0,
                                                                             (const cpx<float>*)h->d_y1, (cpx<float>*)y);
        CU(cudaGetLastError());
        return;
    }
    if (h->med[0]) {
        bi_matvec_launch(h->med[0], x, y, nrhs, s);
        bi_matvec_launch(h->med[1], x, h->d_ysum, nrhs, s);
        const int64_t n = (int64_t)h->nun * nrhs;
        if (h->prec == 0)
            k_add_vec<double><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, (cpx<double>*)y, (const cpx<double>*)h->d_ysum);
        else
            k_add_vec<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, (cpx<float>*)y, (const cpx<float>*)h->d_ysum);
        CU(cudaGetLastError());
        return;
    }
    if (h->use_fast) bi_autotune(h, nrhs, s);
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
    if (h->use_fast) bi_autotune(h, nrhs, h->stream);
    cudaEvent_t ev[BI_NSTAGES + 1];
    for (auto& e : ev) CU(cudaEventCreate(&e));
    for (int i = 0; i < BI_NSTAGES; ++i) ms[i] = 0.0;
    cudaStream_t s = h->stream;
    for (int r = 0; r < reps; ++r) {
        CU(cudaEventRecord(ev[0], s));
        if (h->use_fast) {
            if (h->prec == 0) launch_fast<double>(h, x, y, nrhs, s, s, ev + 1);
            else launch_fast<float>(h, x, y, nrhs, s, s, ev + 1);
        } else {
            if (h->prec == 0) launch_all<double>(h, x, y, nrhs, s, s, ev + 1);
            else launch_all<float>(h, x, y, nrhs, s, s, ev + 1);
        }
        CU(cudaEventSynchronize(ev[BI_NSTAGES]));
        for (int i = 0; i < BI_NSTAGES; ++i) {
            float t = 0;
            CU(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
            ms[i] += t / reps;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
}
