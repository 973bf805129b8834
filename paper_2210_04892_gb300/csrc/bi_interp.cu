// Interpolation (upward pass) and anterpolation (downward pass) between octree levels of
// the multilevel product, with compile-time tap counts.
//
// Upward, for a parent box p with children c (level l+1 -> l):
//   U_p(k) = sum_c exp(+jk khat.(c_c - c_p)) [Phi Theta U_c](k)
// Theta: local Lagrange interpolation in theta along great circles (a tap across a pole reads
// the column half a turn away with both components negated); Phi: local Lagrange
// interpolation in phi on the periodic grid.  One CTA per (parent, block of parent theta
// rows) computes the theta pass of every child for those rows into shared memory, then each
// thread sums one parent sample over the children: no atomics and no zeroing of U_p.
//
// Downward (anterpolation, the transpose), for each child c of p:
//   V_c += Theta^T Phi^T [ conj(exp(+jk khat.(c_c - c_p))) V_p ]
// One CTA per child: the shifted parent field, then the transposed phi pass for every parent
// row, then the transposed theta pass, each from shared memory with zero-padded tap lists.
//
// With one right-hand side (E = 2) each thread carries both components of a sample as one
// 16-byte vector; the general kernels handle any E one component at a time.
#include <algorithm>
#include <vector>

#include "bi_cpx.cuh"
#include "bi_internal.h"

namespace {

template <typename T>
struct tap {
    int c;  // index code
    T w;    // weight
};

// o / d for 0 <= o < 2^22 via a float reciprocal, corrected to the exact quotient
__device__ __forceinline__ int fdiv(int o, int d, float inv) {
    int q = __float2int_rz((float)o * inv);
    if (q * d > o) --q;
    else if ((q + 1) * d <= o) ++q;
    return q;
}

// one complex value through the read-only path as a single vector load
__device__ __forceinline__ cpx<float> ldg_c(const cpx<float>* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ cpx<double> ldg_c(const cpx<double>* p) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return {v.x, v.y};
}

template <typename T>
__device__ __forceinline__ void sts_pair(cpx<T>* p, cpx<T> a, cpx<T> b) {
    p[0] = a;
    p[1] = b;
}
template <typename T>
__device__ __forceinline__ void fma_pair(T w, cpx<T> a, cpx<T> b, cpx<T>& s, cpx<T>& t) {
    s.x = fma(w, a.x, s.x);
    s.y = fma(w, a.y, s.y);
    t.x = fma(w, b.x, t.x);
    t.y = fma(w, b.y, t.y);
}

// ---------------------------------------------------------------- general E
template <typename T, int P>
__global__ void __launch_bounds__(256) k_interp_pb(int nthc, int nphc, int nthp, int nphp, int E, int RB,
                                                   const int* __restrict__ child_ptr, const int* __restrict__ octant,
                                                   const tap<T>* __restrict__ th_tap, const tap<T>* __restrict__ ph_tap,
                                                   const cpx<T>* __restrict__ shift, const cpx<T>* __restrict__ Uc,
                                                   cpx<T>* __restrict__ Up) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int p = blockIdx.x, ip0 = blockIdx.y * RB, nr = min(RB, nthp - ip0);
    const int c0 = child_ptr[p], nc = child_ptr[p + 1] - c0;
    const int W = nphc * E, Wp = nphp * E, Kc = nthc * nphc, Kp = nthp * nphp, half = nphc / 2;
    tap<T>* tt = reinterpret_cast<tap<T>*>(smem_raw);  // [RB][P]
    tap<T>* pt = tt + RB * P;                          // [P][nphp]
    int* oc = reinterpret_cast<int*>(pt + nphp * P);   // [8]
    cpx<T>* s2 = reinterpret_cast<cpx<T>*>(oc + 8);    // [nc][nr][W]
    for (int i = threadIdx.x; i < nr * P; i += blockDim.x) tt[i] = th_tap[ip0 * P + i];
    for (int i = threadIdx.x; i < nphp * P; i += blockDim.x) {
        const int jp = i / P, q = i - jp * P;
        pt[q * nphp + jp] = ph_tap[i];
    }
    if (threadIdx.x < nc) oc[threadIdx.x] = octant[c0 + threadIdx.x];
    __syncthreads();
    const float invE = 1.0f / E, invW = 1.0f / W, invRW = 1.0f / (nr * W), invWp = 1.0f / Wp;
    for (int o = threadIdx.x; o < nc * nr * W; o += blockDim.x) {
        const int c = fdiv(o, nr * W, invRW);
        const int rem = o - c * nr * W;
        const int ipl = fdiv(rem, W, invW);
        const int col = rem - ipl * W;
        const int jc = fdiv(col, E, invE), e = col - jc * E;
        const int jf = jc + half < nphc ? jc + half : jc + half - nphc;
        const int off0 = col, off1 = jf * E + e;
        const cpx<T>* u = Uc + (int64_t)(c0 + c) * Kc * E;
        cpx<T> a = czero<T>();
#pragma unroll
        for (int t = 0; t < P; ++t) {
            const tap<T> q = tt[ipl * P + t];
            const cpx<T> v = ldg_c(u + (q.c >> 1) * W + ((q.c & 1) ? off1 : off0));
            a.x = fma(q.w, v.x, a.x);
            a.y = fma(q.w, v.y, a.y);
        }
        s2[o] = a;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < nr * Wp; o += blockDim.x) {
        const int ipl = fdiv(o, Wp, invWp);
        const int colp = o - ipl * Wp;
        const int jp = fdiv(colp, E, invE), e = colp - jp * E;
        const int ip = ip0 + ipl;
        cpx<T> acc = czero<T>();
        for (int c = 0; c < nc; ++c) {
            const cpx<T>* row = s2 + ((int64_t)c * nr + ipl) * W + e;
            cpx<T> a = czero<T>();
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const tap<T> tq = pt[q * nphp + jp];
                const cpx<T> v = row[tq.c * E];
                a.x = fma(tq.w, v.x, a.x);
                a.y = fma(tq.w, v.y, a.y);
            }
            cfma(acc, ldg_c(shift + (int64_t)oc[c] * Kp + ip * nphp + jp), a);
        }
        Up[((int64_t)p * Kp + ip * nphp) * E + colp] = acc;
    }
}

template <typename T, int PT, int PP>
__global__ void __launch_bounds__(256) k_anterp_cb(int nthc, int nphc, int nthp, int nphp, int E,
                                                   const int* __restrict__ parent, const int* __restrict__ octant,
                                                   const tap<T>* __restrict__ tth_pad, const tap<T>* __restrict__ tph_pad,
                                                   const cpx<T>* __restrict__ shift, const cpx<T>* __restrict__ Vp,
                                                   cpx<T>* __restrict__ Vc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int c = blockIdx.x;
    const int pb = parent[c], oct = octant[c];
    const int W = nphc * E, Wp = nphp * E, Kc = nthc * nphc, Kp = nthp * nphp, half = nphc / 2;
    tap<T>* tt = reinterpret_cast<tap<T>*>(smem_raw);       // [nthc][PT]
    tap<T>* pt = tt + nthc * PT;                             // [PP][nphc]
    cpx<T>* S = reinterpret_cast<cpx<T>*>(pt + nphc * PP);  // [Kp][E] conj(shift) V_p
    cpx<T>* t1 = S + (int64_t)Kp * E;                        // [nthp][W] transposed phi pass
    for (int i = threadIdx.x; i < nthc * PT; i += blockDim.x) tt[i] = tth_pad[i];
    for (int i = threadIdx.x; i < nphc * PP; i += blockDim.x) {
        const int jc = i / PP, q = i - jc * PP;
        pt[q * nphc + jc] = tph_pad[i];
    }
    const cpx<T>* sh = shift + (int64_t)oct * Kp;
    const cpx<T>* vp = Vp + (int64_t)pb * Kp * E;
    const float invE = 1.0f / E, invW = 1.0f / W;
    for (int i = threadIdx.x; i < Kp * E; i += blockDim.x) S[i] = cmulc(ldg_c(sh + fdiv(i, E, invE)), ldg_c(vp + i));
    __syncthreads();
    // t1[ip][jc][e] = sum over parent columns jp that interpolate child column jc
    for (int o = threadIdx.x; o < nthp * W; o += blockDim.x) {
        const int ip = fdiv(o, W, invW);
        const int col = o - ip * W;
        const int jc = fdiv(col, E, invE), e = col - jc * E;
        const cpx<T>* row = S + (int64_t)ip * Wp + e;
        cpx<T> a = czero<T>();
#pragma unroll
        for (int q = 0; q < PP; ++q) {
            const tap<T> tq = pt[q * nphc + jc];
            const cpx<T> v = row[tq.c * E];
            a.x = fma(tq.w, v.x, a.x);
            a.y = fma(tq.w, v.y, a.y);
        }
        t1[o] = a;
    }
    __syncthreads();
    // V_c[ic][col] += sum over parent rows ip that interpolate child row ic (pole taps read the
    // column half a turn away, sign folded into the weight)
    cpx<T>* vc = Vc + (int64_t)c * Kc * E;
    for (int o = threadIdx.x; o < nthc * W; o += blockDim.x) {
        const int ic = fdiv(o, W, invW);
        const int col = o - ic * W;
        const int jc = fdiv(col, E, invE), e = col - jc * E;
        const int jf = jc + half < nphc ? jc + half : jc + half - nphc;
        const int off0 = col, off1 = jf * E + e;
        cpx<T> a = czero<T>();
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            const tap<T> tq = tt[ic * PT + q];
            const cpx<T> v = t1[(tq.c >> 1) * W + ((tq.c & 1) ? off1 : off0)];
            a.x = fma(tq.w, v.x, a.x);
            a.y = fma(tq.w, v.y, a.y);
        }
        vc[o] = cadd(vc[o], a);
    }
}

// ---------------------------------------------------------------- several right-hand sides, chunked
// CTA = (parent p, block of nr parent rows, chunk of EC entries of the E-vector); threads work
// on pairs of adjacent entries (16-byte loads and stores).  The theta pass of every child for
// the block's rows goes to shared memory, then each thread sums one parent (sample, pair) over
// the children.  Chunking E keeps the shared memory per CTA bounded at every level.
template <typename T, int P>
__global__ void __launch_bounds__(256) k_interp_pbE(int nthc, int nphc, int nthp, int nphp, int E, int RB, int EC,
                                                    int nrb, const int* __restrict__ child_ptr,
                                                    const int* __restrict__ octant, const tap<T>* __restrict__ th_tap,
                                                    const tap<T>* __restrict__ ph_tap, const cpx<T>* __restrict__ shift,
                                                    const cpx<T>* __restrict__ Uc, cpx<T>* __restrict__ Up) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nec = E / EC;
    const int ec = blockIdx.x % nec;
    const int rb = (blockIdx.x / nec) % nrb;
    const int p = blockIdx.x / (nec * nrb);
    const int ip0 = rb * RB, nr = min(RB, nthp - ip0), e0 = ec * EC, PC = EC / 2;
    const int c0 = child_ptr[p], nc = child_ptr[p + 1] - c0;
    const int Kc = nthc * nphc, Kp = nthp * nphp, half = nphc / 2;
    tap<T>* tt = reinterpret_cast<tap<T>*>(smem_raw);  // [RB][P]
    tap<T>* pt = tt + RB * P;                          // [P][nphp]
    int* oc = reinterpret_cast<int*>(pt + nphp * P);   // [8]
    cpx<T>* s2 = reinterpret_cast<cpx<T>*>(smem_raw + (((size_t)(RB + nphp) * P * sizeof(tap<T>) + 8 * sizeof(int) + 15) / 16) * 16);
    // s2: [nc][nr][nphc][EC]
    for (int i = threadIdx.x; i < nr * P; i += blockDim.x) tt[i] = th_tap[ip0 * P + i];
    for (int i = threadIdx.x; i < nphp * P; i += blockDim.x) {
        const int jp = i / P, q = i - jp * P;
        pt[q * nphp + jp] = ph_tap[i];
    }
    if (threadIdx.x < nc) oc[threadIdx.x] = octant[c0 + threadIdx.x];
    __syncthreads();
    const int64_t E64 = E;
    const float invPC = 1.0f / PC, invCP = 1.0f / (nphc * PC), invRCP = 1.0f / (nr * nphc * PC);
    for (int o = threadIdx.x; o < nc * nr * nphc * PC; o += blockDim.x) {
        const int c = fdiv(o, nr * nphc * PC, invRCP);
        int rem = o - c * nr * nphc * PC;
        const int ipl = fdiv(rem, nphc * PC, invCP);
        rem -= ipl * nphc * PC;
        const int jc = fdiv(rem, PC, invPC), pr = rem - jc * PC;
        const int jf = jc + half < nphc ? jc + half : jc + half - nphc;
        const cpx<T>* u = Uc + (int64_t)(c0 + c) * Kc * E64 + e0 + 2 * pr;
        cpx<T> a = czero<T>(), b = czero<T>();
#pragma unroll
        for (int t = 0; t < P; ++t) {
            const tap<T> q = tt[ipl * P + t];
            cpx<T> va, vb;
            load_pair(u + ((int64_t)(q.c >> 1) * nphc + ((q.c & 1) ? jf : jc)) * E64, va, vb);
            fma_pair(q.w, va, vb, a, b);
        }
        sts_pair(s2 + 2 * (int64_t)o, a, b);
    }
    __syncthreads();
    const float invPP = 1.0f / (nphp * PC);
    for (int o = threadIdx.x; o < nr * nphp * PC; o += blockDim.x) {
        const int ipl = fdiv(o, nphp * PC, invPP);
        const int rem = o - ipl * nphp * PC;
        const int jp = fdiv(rem, PC, invPC), pr = rem - jp * PC;
        const int ip = ip0 + ipl;
        int src[P];
        T w[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const tap<T> tq = pt[q * nphp + jp];
            src[q] = tq.c;
            w[q] = tq.w;
        }
        cpx<T> A = czero<T>(), B = czero<T>();
        for (int c = 0; c < nc; ++c) {
            const cpx<T>* row = s2 + ((((int64_t)c * nr + ipl) * nphc) * PC + pr) * 2;
            cpx<T> a = czero<T>(), b = czero<T>();
#pragma unroll
            for (int q = 0; q < P; ++q) {
                cpx<T> va, vb;
                lds_pair(row + (int64_t)src[q] * EC, va, vb);
                fma_pair(w[q], va, vb, a, b);
            }
            const cpx<T> sh = ldg_c(shift + (int64_t)oc[c] * Kp + ip * nphp + jp);
            cfma(A, sh, a);
            cfma(B, sh, b);
        }
        cpx<T>* out = Up + ((int64_t)p * Kp + ip * nphp + jp) * E64 + e0 + 2 * pr;
        sts_pair(out, A, B);
    }
}

// CTA = (child c, chunk of EC entries of the E-vector): the shifted parent field for the chunk,
// the transposed phi pass for every parent row, then the transposed theta pass added into the
// child's incoming field, all on pairs of adjacent entries.
template <typename T, int PT>
__global__ void __launch_bounds__(256) k_anterp_cbE(int nthc, int nphc, int nthp, int nphp, int E, int EC,
                                                    const int* __restrict__ parent, const int* __restrict__ octant,
                                                    const tap<T>* __restrict__ tth_pad, const tap<T>* __restrict__ tph_pad,
                                                    const cpx<T>* __restrict__ shift, const cpx<T>* __restrict__ Vp,
                                                    cpx<T>* __restrict__ Vc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nec = E / EC;
    const int c = blockIdx.x / nec, ec = blockIdx.x - c * nec;
    const int e0 = ec * EC, PC = EC / 2;
    const int pb = parent[c], oct = octant[c];
    const int Kc = nthc * nphc, Kp = nthp * nphp, half = nphc / 2;
    const int64_t E64 = E;
    tap<T>* tt = reinterpret_cast<tap<T>*>(smem_raw);       // [nthc][PT]
    tap<T>* pt = tt + nthc * PT;                             // [PT][nphc]
    cpx<T>* S = reinterpret_cast<cpx<T>*>(smem_raw + (((size_t)(nthc + nphc) * PT * sizeof(tap<T>) + 15) / 16) * 16);
    cpx<T>* t1 = S + (int64_t)Kp * EC;                       // [nthp][nphc][EC]
    for (int i = threadIdx.x; i < nthc * PT; i += blockDim.x) tt[i] = tth_pad[i];
    for (int i = threadIdx.x; i < nphc * PT; i += blockDim.x) {
        const int jc = i / PT, q = i - jc * PT;
        pt[q * nphc + jc] = tph_pad[i];
    }
    const cpx<T>* sh = shift + (int64_t)oct * Kp;
    const cpx<T>* vp = Vp + (int64_t)pb * Kp * E64 + e0;
    const float invPC = 1.0f / PC;
    for (int o = threadIdx.x; o < Kp * PC; o += blockDim.x) {
        const int i = fdiv(o, PC, invPC), pr = o - i * PC;
        cpx<T> a, b;
        load_pair(vp + (int64_t)i * E64 + 2 * pr, a, b);
        const cpx<T> z = ldg_c(sh + i);
        sts_pair(S + 2 * (int64_t)o, cmulc(z, a), cmulc(z, b));
    }
    __syncthreads();
    const float invCP = 1.0f / (nphc * PC);
    for (int o = threadIdx.x; o < nthp * nphc * PC; o += blockDim.x) {
        const int ip = fdiv(o, nphc * PC, invCP);
        const int rem = o - ip * nphc * PC;
        const int jc = fdiv(rem, PC, invPC), pr = rem - jc * PC;
        const cpx<T>* row = S + ((int64_t)ip * nphp * PC + pr) * 2;
        cpx<T> a = czero<T>(), b = czero<T>();
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            const tap<T> tq = pt[q * nphc + jc];
            cpx<T> va, vb;
            lds_pair(row + (int64_t)tq.c * EC, va, vb);
            fma_pair(tq.w, va, vb, a, b);
        }
        sts_pair(t1 + 2 * (int64_t)o, a, b);
    }
    __syncthreads();
    cpx<T>* vc = Vc + (int64_t)c * Kc * E64 + e0;
    for (int o = threadIdx.x; o < Kc * PC; o += blockDim.x) {
        const int ic = fdiv(o, nphc * PC, invCP);
        const int rem = o - ic * nphc * PC;
        const int jc = fdiv(rem, PC, invPC), pr = rem - jc * PC;
        const int jf = jc + half < nphc ? jc + half : jc + half - nphc;
        cpx<T> a = czero<T>(), b = czero<T>();
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            const tap<T> tq = tt[ic * PT + q];
            cpx<T> va, vb;
            lds_pair(t1 + ((((int64_t)(tq.c >> 1) * nphc + ((tq.c & 1) ? jf : jc)) * PC) + pr) * 2, va, vb);
            fma_pair(tq.w, va, vb, a, b);
        }
        cpx<T>* g = vc + ((int64_t)ic * nphc + jc) * E64 + 2 * pr;
        cpx<T> ga, gb;
        load_pair(g, ga, gb);
        sts_pair(g, cadd(ga, a), cadd(gb, b));
    }
}

// Coarse levels, where one child's shifted parent field does not fit: CTA = (child c, block of
// nr child rows, chunk of EC entries).  Interpolation in phi commutes with the half turn that the
// pole taps apply (both grids are uniform with an even count), so the transpose can take theta
// first, on the parent's columns, then phi:
//   t[ic][jp]  = sum over the transposed theta taps (ip, w, flip) of w conj(shift) V_p[ip][jp or jp + nphp/2]
//   V_c[ic][jc] += sum over the transposed phi taps (jp, w) of w t[ic][jp]
// The shifted parent field is read from L2 per tap; only t is kept in shared memory.
template <typename T, int PT>
__global__ void __launch_bounds__(256) k_anterp_rbE(int nthc, int nphc, int nthp, int nphp, int E, int RB, int EC, int nrb,
                                                    const int* __restrict__ parent, const int* __restrict__ octant,
                                                    const tap<T>* __restrict__ tth_pad, const tap<T>* __restrict__ tph_pad,
                                                    const cpx<T>* __restrict__ shift, const cpx<T>* __restrict__ Vp,
                                                    cpx<T>* __restrict__ Vc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nec = E / EC;
    const int ec = blockIdx.x % nec;
    const int rb = (blockIdx.x / nec) % nrb;
    const int c = blockIdx.x / (nec * nrb);
    const int ic0 = rb * RB, nr = min(RB, nthc - ic0), e0 = ec * EC, PC = EC / 2;
    const int pb = parent[c], oct = octant[c];
    const int Kc = nthc * nphc, Kp = nthp * nphp, hp = nphp / 2;
    const int64_t E64 = E;
    tap<T>* tt = reinterpret_cast<tap<T>*>(smem_raw);       // [RB][PT]
    tap<T>* pt = tt + RB * PT;                               // [PT][nphc]
    cpx<T>* tS = reinterpret_cast<cpx<T>*>(smem_raw + (((size_t)(RB + nphc) * PT * sizeof(tap<T>) + 15) / 16) * 16);
    for (int i = threadIdx.x; i < nr * PT; i += blockDim.x) tt[i] = tth_pad[ic0 * PT + i];
    for (int i = threadIdx.x; i < nphc * PT; i += blockDim.x) {
        const int jc = i / PT, q = i - jc * PT;
        pt[q * nphc + jc] = tph_pad[i];
    }
    __syncthreads();
    const cpx<T>* sh = shift + (int64_t)oct * Kp;
    const cpx<T>* vp = Vp + (int64_t)pb * Kp * E64 + e0;
    const float invPC = 1.0f / PC, invPP = 1.0f / (nphp * PC), invCP = 1.0f / (nphc * PC);
    for (int o = threadIdx.x; o < nr * nphp * PC; o += blockDim.x) {
        const int icl = fdiv(o, nphp * PC, invPP);
        const int rem = o - icl * nphp * PC;
        const int jp = fdiv(rem, PC, invPC), pr = rem - jp * PC;
        const int jpf = jp + hp < nphp ? jp + hp : jp + hp - nphp;
        cpx<T> a = czero<T>(), b = czero<T>();
        for (int q = 0; q < PT; ++q) {
            const tap<T> tq = tt[icl * PT + q];
            if (tq.w == T(0)) continue;
            const int i = (tq.c >> 1) * nphp + ((tq.c & 1) ? jpf : jp);
            cpx<T> va, vb;
            load_pair(vp + (int64_t)i * E64 + 2 * pr, va, vb);
            const cpx<T> z = ldg_c(sh + i);
            fma_pair(tq.w, cmulc(z, va), cmulc(z, vb), a, b);
        }
        sts_pair(tS + 2 * (int64_t)o, a, b);
    }
    __syncthreads();
    cpx<T>* vc = Vc + ((int64_t)c * Kc + (int64_t)ic0 * nphc) * E64 + e0;
    for (int o = threadIdx.x; o < nr * nphc * PC; o += blockDim.x) {
        const int icl = fdiv(o, nphc * PC, invCP);
        const int rem = o - icl * nphc * PC;
        const int jc = fdiv(rem, PC, invPC), pr = rem - jc * PC;
        const cpx<T>* row = tS + ((int64_t)icl * nphp * PC + pr) * 2;
        cpx<T> a = czero<T>(), b = czero<T>();
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            const tap<T> tq = pt[q * nphc + jc];
            cpx<T> va, vb;
            lds_pair(row + (int64_t)tq.c * EC, va, vb);
            fma_pair(tq.w, va, vb, a, b);
        }
        cpx<T>* g = vc + ((int64_t)icl * nphc + jc) * E64 + 2 * pr;
        cpx<T> ga, gb;
        load_pair(g, ga, gb);
        sts_pair(g, cadd(ga, a), cadd(gb, b));
    }
}

// ---------------------------------------------------------------- one right-hand side (E = 2)
template <typename T, int P>
__global__ void __launch_bounds__(256, 4) k_interp_pb1(int nthc, int nphc, int nthp, int nphp, int RB,
                                                    const int* __restrict__ child_ptr, const int* __restrict__ octant,
                                                    const tap<T>* __restrict__ th_tap, const tap<T>* __restrict__ ph_tap,
                                                    const cpx<T>* __restrict__ shift, const cpx<T>* __restrict__ Uc,
                                                    cpx<T>* __restrict__ Up) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int p = blockIdx.x, ip0 = blockIdx.y * RB, nr = min(RB, nthp - ip0);
    const int c0 = child_ptr[p], nc = child_ptr[p + 1] - c0;
    const int Kc = nthc * nphc, Kp = nthp * nphp, half = nphc / 2;
    tap<T>* tt = reinterpret_cast<tap<T>*>(smem_raw);  // [RB][P]
    tap<T>* pt = tt + RB * P;                          // [P][nphp]: lanes (columns) read consecutive taps
    int* oc = reinterpret_cast<int*>(pt + nphp * P);   // [8]
    cpx<T>* s2 = reinterpret_cast<cpx<T>*>(oc + 8);    // [nc][nr][nphc][2]
    for (int i = threadIdx.x; i < nr * P; i += blockDim.x) tt[i] = th_tap[ip0 * P + i];
    for (int i = threadIdx.x; i < nphp * P; i += blockDim.x) {
        const int jp = i / P, q = i - jp * P;
        pt[q * nphp + jp] = ph_tap[i];
    }
    if (threadIdx.x < nc) oc[threadIdx.x] = octant[c0 + threadIdx.x];
    __syncthreads();
    // theta pass: one (child, row, column) per thread, both components
    const float invC = 1.0f / nphc, invRC = 1.0f / (nr * nphc);
    for (int o = threadIdx.x; o < nc * nr * nphc; o += blockDim.x) {
        const int c = fdiv(o, nr * nphc, invRC);
        const int rem = o - c * nr * nphc;
        const int ipl = fdiv(rem, nphc, invC);
        const int jc = rem - ipl * nphc;
        const int jf = jc + half < nphc ? jc + half : jc + half - nphc;
        const cpx<T>* u = Uc + (int64_t)(c0 + c) * Kc * 2;
        cpx<T> a = czero<T>(), b = czero<T>();
#pragma unroll
        for (int t = 0; t < P; ++t) {
            const tap<T> q = tt[ipl * P + t];
            cpx<T> va, vb;
            load_pair(u + ((q.c >> 1) * nphc + ((q.c & 1) ? jf : jc)) * 2, va, vb);
            fma_pair(q.w, va, vb, a, b);
        }
        sts_pair(s2 + 2 * o, a, b);
    }
    __syncthreads();
    // phi pass and sum over children: one parent sample per thread, its taps in registers for
    // every child
    for (int o = threadIdx.x; o < nr * nphp; o += blockDim.x) {
        const int ipl = o / nphp;
        const int jp = o - ipl * nphp;
        const int ip = ip0 + ipl;
        int src[P];
        T w[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const tap<T> tq = pt[q * nphp + jp];
            src[q] = tq.c;
            w[q] = tq.w;
        }
        cpx<T> A = czero<T>(), B = czero<T>();
        for (int c = 0; c < nc; ++c) {
            const cpx<T>* row = s2 + (((int64_t)c * nr + ipl) * nphc) * 2;
            cpx<T> a = czero<T>(), b = czero<T>();
#pragma unroll
            for (int q = 0; q < P; ++q) {
                cpx<T> va, vb;
                lds_pair(row + 2 * src[q], va, vb);
                fma_pair(w[q], va, vb, a, b);
            }
            const cpx<T> sh = ldg_c(shift + (int64_t)oc[c] * Kp + ip * nphp + jp);
            cfma(A, sh, a);
            cfma(B, sh, b);
        }
        cpx<T>* out = Up + ((int64_t)p * Kp + ip * nphp + jp) * 2;
        out[0] = A;
        out[1] = B;
    }
}

template <typename T, int PT>
__global__ void __launch_bounds__(256, 8) k_anterp_cb1(int nthc, int nphc, int nthp, int nphp,
                                                    const int* __restrict__ parent, const int* __restrict__ octant,
                                                    const tap<T>* __restrict__ tth_pad, const tap<T>* __restrict__ tph_pad,
                                                    const cpx<T>* __restrict__ shift, const cpx<T>* __restrict__ Vp,
                                                    cpx<T>* __restrict__ Vc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int c = blockIdx.x;
    const int pb = parent[c], oct = octant[c];
    const int Kc = nthc * nphc, Kp = nthp * nphp, half = nphc / 2;
    tap<T>* tt = reinterpret_cast<tap<T>*>(smem_raw);       // [nthc][PT]
    tap<T>* pt = tt + nthc * PT;                             // [PT][nphc]: lanes (columns) read consecutive taps
    cpx<T>* S = reinterpret_cast<cpx<T>*>(pt + nphc * PT);  // [Kp][2] conj(shift) V_p
    cpx<T>* t1 = S + (int64_t)Kp * 2;                        // [nthp][nphc][2]
    for (int i = threadIdx.x; i < nthc * PT; i += blockDim.x) tt[i] = tth_pad[i];
    for (int i = threadIdx.x; i < nphc * PT; i += blockDim.x) {
        const int jc = i / PT, q = i - jc * PT;
        pt[q * nphc + jc] = tph_pad[i];
    }
    const cpx<T>* sh = shift + (int64_t)oct * Kp;
    const cpx<T>* vp = Vp + (int64_t)pb * Kp * 2;
    for (int i = threadIdx.x; i < Kp; i += blockDim.x) {
        cpx<T> a, b;
        load_pair(vp + 2 * i, a, b);
        const cpx<T> s = ldg_c(sh + i);
        sts_pair(S + 2 * i, cmulc(s, a), cmulc(s, b));
    }
    __syncthreads();
    // transposed phi pass: one (parent row, child column) per thread
    for (int o = threadIdx.x; o < nphc * nthp; o += blockDim.x) {
        const int ip = o / nphc;
        const int jc = o - ip * nphc;
        const cpx<T>* row = S + (int64_t)ip * nphp * 2;
        cpx<T> a = czero<T>(), b = czero<T>();
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            const tap<T> tq = pt[q * nphc + jc];
            cpx<T> va, vb;
            lds_pair(row + 2 * tq.c, va, vb);
            fma_pair(tq.w, va, vb, a, b);
        }
        sts_pair(t1 + 2 * o, a, b);
    }
    __syncthreads();
    // transposed theta pass: one child sample per thread (taps of its row shared by the warp)
    cpx<T>* vc = Vc + (int64_t)c * Kc * 2;
    for (int o = threadIdx.x; o < Kc; o += blockDim.x) {
        const int ic = o / nphc;
        const int jc = o - ic * nphc;
        const int jf = jc + half < nphc ? jc + half : jc + half - nphc;
        cpx<T> a = czero<T>(), b = czero<T>();
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            const tap<T> tq = tt[ic * PT + q];
            cpx<T> va, vb;
            lds_pair(t1 + ((tq.c >> 1) * nphc + ((tq.c & 1) ? jf : jc)) * 2, va, vb);
            fma_pair(tq.w, va, vb, a, b);
        }
        cpx<T> ga, gb;
        load_pair(vc + 2 * o, ga, gb);
        sts_pair(vc + 2 * o, cadd(ga, a), cadd(gb, b));
    }
}

// ---------------------------------------------------------------- many right-hand sides (E >= 32)
// Two passes through the per-child intermediate tmp[child][ip][jc][e].  One CTA per (box, row),
// rows fastest so that the CTAs of one box run together and share its patterns in L2; the
// row's taps are uniform over the CTA; threads = 32 lanes over e x 8 over columns.
template <typename T, int P>
__global__ void __launch_bounds__(256) k_interp_theta_w(int nthc, int nphc, int nthp, int E, const tap<T>* __restrict__ th_tap,
                                                        const cpx<T>* __restrict__ Uc, cpx<T>* __restrict__ tmp) {
    const int cb = blockIdx.x / nthp, ip = blockIdx.x - cb * nthp;
    const int half = nphc / 2, Kc = nthc * nphc;
    int code[P];
    T w[P];
#pragma unroll
    for (int t = 0; t < P; ++t) {
        const tap<T> q = th_tap[ip * P + t];
        code[t] = q.c;
        w[t] = q.w;
    }
    const cpx<T>* u = Uc + (int64_t)cb * Kc * E;
    cpx<T>* out = tmp + (((int64_t)cb * nthp + ip) * nphc) * E;
    for (int jc = threadIdx.y; jc < nphc; jc += blockDim.y) {
        const int jf = jc + half < nphc ? jc + half : jc + half - nphc;
        for (int e = threadIdx.x; e < E; e += blockDim.x) {
            cpx<T> a = czero<T>();
#pragma unroll
            for (int t = 0; t < P; ++t) {
                const cpx<T> v = ldg_c(u + ((int64_t)(code[t] >> 1) * nphc + ((code[t] & 1) ? jf : jc)) * E + e);
                a.x = fma(w[t], v.x, a.x);
                a.y = fma(w[t], v.y, a.y);
            }
            out[(int64_t)jc * E + e] = a;
        }
    }
}

template <typename T, int P>
__global__ void __launch_bounds__(256) k_interp_phi_w(int nthp, int nphp, int nphc, int E, const tap<T>* __restrict__ ph_tap,
                                                      const int* __restrict__ child_ptr, const int* __restrict__ octant,
                                                      const cpx<T>* __restrict__ shift, const cpx<T>* __restrict__ tmp,
                                                      cpx<T>* __restrict__ Up) {
    const int pb = blockIdx.x / nthp, ip = blockIdx.x - pb * nthp;
    const int Kp = nthp * nphp;
    const int c0 = child_ptr[pb], nc = child_ptr[pb + 1] - c0;
    for (int jp = threadIdx.y; jp < nphp; jp += blockDim.y) {
        int src[P];
        T w[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const tap<T> tq = ph_tap[jp * P + q];
            src[q] = tq.c;
            w[q] = tq.w;
        }
        for (int e = threadIdx.x; e < E; e += blockDim.x) {
            cpx<T> acc = czero<T>();
            for (int c = 0; c < nc; ++c) {
                const cpx<T>* row = tmp + (((int64_t)(c0 + c) * nthp + ip) * nphc) * E + e;
                cpx<T> a = czero<T>();
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const cpx<T> v = ldg_c(row + (int64_t)src[q] * E);
                    a.x = fma(w[q], v.x, a.x);
                    a.y = fma(w[q], v.y, a.y);
                }
                cfma(acc, ldg_c(shift + (int64_t)octant[c0 + c] * Kp + ip * nphp + jp), a);
            }
            Up[((int64_t)pb * Kp + ip * nphp + jp) * E + e] = acc;
        }
    }
}

// tmp[cb][ip][jc][e] = sum over parent columns jp of w conj(shift(ip, jp)) V_p[ip][jp][e]
template <typename T, int PT>
__global__ void __launch_bounds__(256) k_anterp_phi_w(int nthp, int nphp, int nphc, int E, const tap<T>* __restrict__ tph_pad,
                                                      const int* __restrict__ parent, const int* __restrict__ octant,
                                                      const cpx<T>* __restrict__ shift, const cpx<T>* __restrict__ Vp,
                                                      cpx<T>* __restrict__ tmp) {
    const int cb = blockIdx.x / nthp, ip = blockIdx.x - cb * nthp;
    const int Kp = nthp * nphp;
    const int pb = parent[cb];
    const cpx<T>* sh = shift + (int64_t)octant[cb] * Kp + ip * nphp;
    const cpx<T>* vp = Vp + ((int64_t)pb * Kp + ip * nphp) * E;
    cpx<T>* out = tmp + (((int64_t)cb * nthp + ip) * nphc) * E;
    for (int jc = threadIdx.y; jc < nphc; jc += blockDim.y) {
        int dst[PT];
        T w[PT];
        cpx<T> sc[PT];
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            const tap<T> tq = tph_pad[jc * PT + q];
            dst[q] = tq.c;
            const cpx<T> z = ldg_c(sh + tq.c);
            sc[q] = {tq.w * z.x, -tq.w * z.y};   // w conj(shift)
        }
        for (int e = threadIdx.x; e < E; e += blockDim.x) {
            cpx<T> a = czero<T>();
#pragma unroll
            for (int q = 0; q < PT; ++q) cfma(a, sc[q], ldg_c(vp + (int64_t)dst[q] * E + e));
            out[(int64_t)jc * E + e] = a;
        }
    }
}

// V_c[ic][jc][e] += sum over parent rows ip of w tmp[cb][ip][jc or jc + half][e]
template <typename T, int PT>
__global__ void __launch_bounds__(256) k_anterp_theta_w(int nthc, int nphc, int nthp, int E, const tap<T>* __restrict__ tth_pad,
                                                        const cpx<T>* __restrict__ tmp, cpx<T>* __restrict__ Vc) {
    const int cb = blockIdx.x / nthc, ic = blockIdx.x - cb * nthc;
    const int half = nphc / 2, Kc = nthc * nphc;
    int code[PT];
    T w[PT];
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        const tap<T> tq = tth_pad[ic * PT + q];
        code[q] = tq.c;
        w[q] = tq.w;
    }
    const cpx<T>* t0 = tmp + (int64_t)cb * nthp * nphc * E;
    cpx<T>* vc = Vc + ((int64_t)cb * Kc + ic * nphc) * E;
    for (int jc = threadIdx.y; jc < nphc; jc += blockDim.y) {
        const int jf = jc + half < nphc ? jc + half : jc + half - nphc;
        for (int e = threadIdx.x; e < E; e += blockDim.x) {
            cpx<T> a = czero<T>();
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                const cpx<T> v = ldg_c(t0 + ((int64_t)(code[q] >> 1) * nphc + ((code[q] & 1) ? jf : jc)) * E + e);
                a.x = fma(w[q], v.x, a.x);
                a.y = fma(w[q], v.y, a.y);
            }
            vc[(int64_t)jc * E + e] = cadd(vc[(int64_t)jc * E + e], a);
        }
    }
}

// ---------------------------------------------------------------- two passes, entry pairs
// The two-pass forms above with each thread on one pair of adjacent entries (a 16-byte load in
// FP32) and E/2 pair lanes per column, so every tap reads whole contiguous E-vectors and no
// lane idles for E < 32; zero-weight entries of the padded transposed tap lists are skipped.
// For the coarse levels (few boxes, many directions), where the per-CTA forms leave most SMs
// idle or read the parent field once per tap.
template <typename T>
__device__ __forceinline__ void st_pair(cpx<T>* p, cpx<T> a, cpx<T> b) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
    } else {
        p[0] = a;
        p[1] = b;
    }
}

template <typename T, int P>
__global__ void __launch_bounds__(256) k_interp_theta_p2(int nthc, int nphc, int nthp, int E, const tap<T>* __restrict__ th_tap,
                                                         const cpx<T>* __restrict__ Uc, cpx<T>* __restrict__ tmp) {
    const int cb = blockIdx.x / nthp, ip = blockIdx.x - cb * nthp;
    const int PE = E / 2, le = threadIdx.x % PE, col0 = threadIdx.x / PE, ncols = blockDim.x / PE;
    const int half = nphc / 2, Kc = nthc * nphc;
    int code[P];
    T w[P];
#pragma unroll
    for (int t = 0; t < P; ++t) {
        const tap<T> q = th_tap[ip * P + t];
        code[t] = q.c;
        w[t] = q.w;
    }
    const cpx<T>* u = Uc + (int64_t)cb * Kc * E + 2 * le;
    cpx<T>* out = tmp + (((int64_t)cb * nthp + ip) * nphc) * E + 2 * le;
    for (int jc = col0; jc < nphc; jc += ncols) {
        const int jf = jc + half < nphc ? jc + half : jc + half - nphc;
        cpx<T> a = czero<T>(), b = czero<T>();
#pragma unroll
        for (int t = 0; t < P; ++t) {
            cpx<T> va, vb;
            load_pair(u + ((int64_t)(code[t] >> 1) * nphc + ((code[t] & 1) ? jf : jc)) * E, va, vb);
            fma_pair(w[t], va, vb, a, b);
        }
        st_pair(out + (int64_t)jc * E, a, b);
    }
}

template <typename T, int P>
__global__ void __launch_bounds__(256) k_interp_phi_p2(int nthp, int nphp, int nphc, int E, const tap<T>* __restrict__ ph_tap,
                                                       const int* __restrict__ child_ptr, const int* __restrict__ octant,
                                                       const cpx<T>* __restrict__ shift, const cpx<T>* __restrict__ tmp,
                                                       cpx<T>* __restrict__ Up) {
    const int pb = blockIdx.x / nthp, ip = blockIdx.x - pb * nthp;
    const int PE = E / 2, le = threadIdx.x % PE, col0 = threadIdx.x / PE, ncols = blockDim.x / PE;
    const int Kp = nthp * nphp;
    const int c0 = child_ptr[pb], nc = child_ptr[pb + 1] - c0;
    for (int jp = col0; jp < nphp; jp += ncols) {
        int src[P];
        T w[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const tap<T> tq = ph_tap[jp * P + q];
            src[q] = tq.c;
            w[q] = tq.w;
        }
        cpx<T> A = czero<T>(), B = czero<T>();
        for (int c = 0; c < nc; ++c) {
            const cpx<T>* row = tmp + (((int64_t)(c0 + c) * nthp + ip) * nphc) * E + 2 * le;
            cpx<T> a = czero<T>(), b = czero<T>();
#pragma unroll
            for (int q = 0; q < P; ++q) {
                cpx<T> va, vb;
                load_pair(row + (int64_t)src[q] * E, va, vb);
                fma_pair(w[q], va, vb, a, b);
            }
            const cpx<T> z = ldg_c(shift + (int64_t)octant[c0 + c] * Kp + ip * nphp + jp);
            cfma(A, z, a);
            cfma(B, z, b);
        }
        st_pair(Up + ((int64_t)pb * Kp + ip * nphp + jp) * E + 2 * le, A, B);
    }
}

template <typename T, int PT>
__global__ void __launch_bounds__(256) k_anterp_phi_p2(int nthp, int nphp, int nphc, int E, const tap<T>* __restrict__ tph_pad,
                                                       const int* __restrict__ parent, const int* __restrict__ octant,
                                                       const cpx<T>* __restrict__ shift, const cpx<T>* __restrict__ Vp,
                                                       cpx<T>* __restrict__ tmp) {
    const int cb = blockIdx.x / nthp, ip = blockIdx.x - cb * nthp;
    const int PE = E / 2, le = threadIdx.x % PE, col0 = threadIdx.x / PE, ncols = blockDim.x / PE;
    const int Kp = nthp * nphp;
    const int pb = parent[cb];
    const cpx<T>* sh = shift + (int64_t)octant[cb] * Kp + ip * nphp;
    const cpx<T>* vp = Vp + ((int64_t)pb * Kp + ip * nphp) * E + 2 * le;
    cpx<T>* out = tmp + (((int64_t)cb * nthp + ip) * nphc) * E + 2 * le;
    for (int jc = col0; jc < nphc; jc += ncols) {
        cpx<T> a = czero<T>(), b = czero<T>();
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            const tap<T> tq = tph_pad[jc * PT + q];
            if (tq.w == T(0)) continue;      // padding of the transposed list
            const cpx<T> z = ldg_c(sh + tq.c);
            const cpx<T> sc = {tq.w * z.x, -tq.w * z.y};   // w conj(shift)
            cpx<T> va, vb;
            load_pair(vp + (int64_t)tq.c * E, va, vb);
            cfma(a, sc, va);
            cfma(b, sc, vb);
        }
        st_pair(out + (int64_t)jc * E, a, b);
    }
}

template <typename T, int PT>
__global__ void __launch_bounds__(256) k_anterp_theta_p2(int nthc, int nphc, int nthp, int E, const tap<T>* __restrict__ tth_pad,
                                                         const cpx<T>* __restrict__ tmp, cpx<T>* __restrict__ Vc) {
    const int cb = blockIdx.x / nthc, ic = blockIdx.x - cb * nthc;
    const int PE = E / 2, le = threadIdx.x % PE, col0 = threadIdx.x / PE, ncols = blockDim.x / PE;
    const int half = nphc / 2, Kc = nthc * nphc;
    int code[PT];
    T w[PT];
    int nq = 0;
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        const tap<T> tq = tth_pad[ic * PT + q];
        code[q] = tq.c;
        w[q] = tq.w;
        if (tq.w != T(0)) nq = q + 1;
    }
    const cpx<T>* t0 = tmp + (int64_t)cb * nthp * nphc * E + 2 * le;
    cpx<T>* vc = Vc + ((int64_t)cb * Kc + ic * nphc) * E + 2 * le;
    for (int jc = col0; jc < nphc; jc += ncols) {
        const int jf = jc + half < nphc ? jc + half : jc + half - nphc;
        cpx<T> a = czero<T>(), b = czero<T>();
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            if (q >= nq) break;
            cpx<T> va, vb;
            load_pair(t0 + ((int64_t)(code[q] >> 1) * nphc + ((code[q] & 1) ? jf : jc)) * E, va, vb);
            fma_pair(w[q], va, vb, a, b);
        }
        cpx<T>* g = vc + (int64_t)jc * E;
        cpx<T> ga, gb;
        load_pair(g, ga, gb);
        st_pair(g, cadd(ga, a), cadd(gb, b));
    }
}

template <typename T>
bool interp_pairs(bi_handle_s* h, int l, int E, cudaStream_t s) {
    level_t& Pl = h->lev[l];
    level_t& C = h->lev[l + 1];
    interp_t& I = h->itp[l];
    if (!I.d_tmp || E % 2 != 0 || E / 2 > 256) return false;
    const int PE = E / 2, threads = (256 / PE) * PE;
    k_interp_theta_p2<T, 10><<<(unsigned)((int64_t)C.nbox * Pl.nth), threads, 0, s>>>(
        C.nth, C.nph, Pl.nth, E, (const tap<T>*)I.d_th_tap, (const cpx<T>*)C.d_U, (cpx<T>*)I.d_tmp);
    CU(cudaGetLastError());
    k_interp_phi_p2<T, 10><<<(unsigned)((int64_t)Pl.nbox * Pl.nth), threads, 0, s>>>(
        Pl.nth, Pl.nph, C.nph, E, (const tap<T>*)I.d_ph_tap, Pl.d_child_ptr, C.d_octant, (const cpx<T>*)Pl.d_shift,
        (const cpx<T>*)I.d_tmp, (cpx<T>*)Pl.d_U);
    CU(cudaGetLastError());
    return true;
}

template <typename T, int PT>
bool anterp_pairs(bi_handle_s* h, int l, int E, cudaStream_t s) {
    level_t& Pl = h->lev[l];
    level_t& C = h->lev[l + 1];
    interp_t& I = h->itp[l];
    if (!I.d_tmp || E % 2 != 0 || E / 2 > 256) return false;
    const int PE = E / 2, threads = (256 / PE) * PE;
    k_anterp_phi_p2<T, PT><<<(unsigned)((int64_t)C.nbox * Pl.nth), threads, 0, s>>>(
        Pl.nth, Pl.nph, C.nph, E, (const tap<T>*)I.d_tph_pad, C.d_parent, C.d_octant, (const cpx<T>*)Pl.d_shift_dn,
        (const cpx<T>*)Pl.d_V, (cpx<T>*)I.d_tmp);
    CU(cudaGetLastError());
    k_anterp_theta_p2<T, PT><<<(unsigned)((int64_t)C.nbox * C.nth), threads, 0, s>>>(
        C.nth, C.nph, Pl.nth, E, (const tap<T>*)I.d_tth_pad, (const cpx<T>*)I.d_tmp, (cpx<T>*)C.d_V);
    CU(cudaGetLastError());
    return true;
}

template <typename T>
bool interp_wide(bi_handle_s* h, int l, int E, cudaStream_t s) {
    level_t& Pl = h->lev[l];
    level_t& C = h->lev[l + 1];
    interp_t& I = h->itp[l];
    if (!I.d_tmp) return false;
    const dim3 blk(32, 8);
    k_interp_theta_w<T, 10><<<(unsigned)((int64_t)C.nbox * Pl.nth), blk, 0, s>>>(C.nth, C.nph, Pl.nth, E, (const tap<T>*)I.d_th_tap,
                                                                               (const cpx<T>*)C.d_U, (cpx<T>*)I.d_tmp);
    CU(cudaGetLastError());
    k_interp_phi_w<T, 10><<<(unsigned)((int64_t)Pl.nbox * Pl.nth), blk, 0, s>>>(Pl.nth, Pl.nph, C.nph, E, (const tap<T>*)I.d_ph_tap,
                                                                             Pl.d_child_ptr, C.d_octant, (const cpx<T>*)Pl.d_shift,
                                                                             (const cpx<T>*)I.d_tmp, (cpx<T>*)Pl.d_U);
    CU(cudaGetLastError());
    return true;
}

template <typename T, int PT>
bool anterp_wide(bi_handle_s* h, int l, int E, cudaStream_t s) {
    level_t& Pl = h->lev[l];
    level_t& C = h->lev[l + 1];
    interp_t& I = h->itp[l];
    if (!I.d_tmp) return false;
    const dim3 blk(32, 8);
    k_anterp_phi_w<T, PT><<<(unsigned)((int64_t)C.nbox * Pl.nth), blk, 0, s>>>(Pl.nth, Pl.nph, C.nph, E, (const tap<T>*)I.d_tph_pad,
                                                                             C.d_parent, C.d_octant, (const cpx<T>*)Pl.d_shift_dn,
                                                                             (const cpx<T>*)Pl.d_V, (cpx<T>*)I.d_tmp);
    CU(cudaGetLastError());
    k_anterp_theta_w<T, PT><<<(unsigned)((int64_t)C.nbox * C.nth), blk, 0, s>>>(C.nth, C.nph, Pl.nth, E, (const tap<T>*)I.d_tth_pad,
                                                                               (const cpx<T>*)I.d_tmp, (cpx<T>*)C.d_V);
    CU(cudaGetLastError());
    return true;
}

template <typename T>
void upload_taps_t(bi_handle_s* h) {
    for (int l = 2; l + 1 <= h->leaf; ++l) {
        interp_t& I = h->itp[l];
        const level_t& C = h->lev[l + 1];
        std::vector<tap<T>> th(I.th_src.size()), ph(I.ph_src.size());
        for (size_t i = 0; i < th.size(); ++i)
            th[i] = {I.th_src[i] * 2 + I.th_flip[i], (T)(I.th_flip[i] ? -I.th_w[i] : I.th_w[i])};
        for (size_t i = 0; i < ph.size(); ++i) ph[i] = {I.ph_src[i], (T)I.ph_w[i]};
        int mt = 0, mp = 0;
        for (int i = 0; i < C.nth; ++i) mt = std::max(mt, I.tth_ptr[i + 1] - I.tth_ptr[i]);
        for (int j = 0; j < C.nph; ++j) mp = std::max(mp, I.tph_ptr[j + 1] - I.tph_ptr[j]);
        // one padded width for both lists (the kernels are instantiated for 16 and 24)
        const int m = std::max(mt, mp);
        I.pt_th = I.pt_ph = m <= 16 ? 16 : m <= 24 ? 24 : m;
        std::vector<tap<T>> tth((size_t)C.nth * I.pt_th, tap<T>{0, T(0)}), tph((size_t)C.nph * I.pt_ph, tap<T>{0, T(0)});
        for (int i = 0; i < C.nth; ++i)
            for (int q = I.tth_ptr[i]; q < I.tth_ptr[i + 1]; ++q)
                tth[(size_t)i * I.pt_th + (q - I.tth_ptr[i])] = {I.tth_dst[q] * 2 + I.tth_flip[q],
                                                                 (T)(I.tth_flip[q] ? -I.tth_w[q] : I.tth_w[q])};
        for (int j = 0; j < C.nph; ++j)
            for (int q = I.tph_ptr[j]; q < I.tph_ptr[j + 1]; ++q)
                tph[(size_t)j * I.pt_ph + (q - I.tph_ptr[j])] = {I.tph_dst[q], (T)I.tph_w[q]};
        I.d_th_tap = h->upload(th);
        I.d_ph_tap = h->upload(ph);
        I.d_tth_pad = h->upload(tth);
        I.d_tph_pad = h->upload(tph);
    }
}

template <typename T, int P>
bool interp_t_p(bi_handle_s* h, int l, int E, cudaStream_t s) {
    level_t& Pl = h->lev[l];
    level_t& C = h->lev[l + 1];
    interp_t& I = h->itp[l];
    const int W = C.nph * E;
    // rows per CTA: shared memory for 8 children, and at least ~2 CTAs per SM overall
    const size_t per_row = (size_t)8 * W * sizeof(cpx<T>);
    int RB = (int)std::max<size_t>(1, (64 * 1024) / per_row);
    const int want_blocks = (2 * h->num_sms + Pl.nbox - 1) / Pl.nbox;
    RB = std::min(RB, std::max(1, (Pl.nth + want_blocks - 1) / want_blocks));
    RB = std::min(RB, Pl.nth);
    const size_t smem = (size_t)(RB + Pl.nph) * P * sizeof(tap<T>) + 8 * sizeof(int) + (size_t)RB * per_row;
    if (smem > 160 * 1024) return false;
    dim3 g(Pl.nbox, (Pl.nth + RB - 1) / RB);
    if (E == 2) {
        auto k1 = k_interp_pb1<T, P>;
        bi_raise_smem(k1, smem);
        k1<<<g, 256, smem, s>>>(C.nth, C.nph, Pl.nth, Pl.nph, RB, Pl.d_child_ptr, C.d_octant, (const tap<T>*)I.d_th_tap,
                                (const tap<T>*)I.d_ph_tap, (const cpx<T>*)Pl.d_shift, (const cpx<T>*)C.d_U,
                                (cpx<T>*)Pl.d_U);
        CU(cudaGetLastError());
        return true;
    }
    auto kern = k_interp_pb<T, P>;
    bi_raise_smem(kern, smem);
    kern<<<g, 256, smem, s>>>(C.nth, C.nph, Pl.nth, Pl.nph, E, RB, Pl.d_child_ptr, C.d_octant, (const tap<T>*)I.d_th_tap,
                              (const tap<T>*)I.d_ph_tap, (const cpx<T>*)Pl.d_shift, (const cpx<T>*)C.d_U,
                              (cpx<T>*)Pl.d_U);
    CU(cudaGetLastError());
    return true;
}

// Several right-hand sides: the chunked kernel.  EC (entries per chunk) is the largest of 16,
// 8, 4, 2 that divides E and leaves room for at least one parent row of 8 children in about
// 64 KB of shared memory; rows per CTA fill the rest.
template <typename T, int P>
bool interp_chunked(bi_handle_s* h, int l, int E, cudaStream_t s, int ec_force = 0) {
    level_t& Pl = h->lev[l];
    level_t& C = h->lev[l + 1];
    interp_t& I = h->itp[l];
    const size_t budget = 64 * 1024;
    int EC = 0;
    for (int ec : {16, 8, 4, 2})
        if (E % ec == 0 && (size_t)8 * C.nph * ec * sizeof(cpx<T>) <= budget / 2 && (!ec_force || ec == ec_force)) {
            EC = ec;
            break;
        }
    if (!EC) return false;
    const size_t per_row = (size_t)8 * C.nph * EC * sizeof(cpx<T>);
    int RB = (int)std::max<size_t>(1, budget / per_row);
    RB = std::min(RB, Pl.nth);
    auto smem_of = [&](int rb) {
        return (((size_t)(rb + Pl.nph) * P * sizeof(tap<T>) + 8 * sizeof(int) + 15) / 16) * 16 + (size_t)rb * per_row;
    };
    while (RB > 1 && smem_of(RB) > budget + 16 * 1024) --RB;
    const size_t smem = smem_of(RB);
    if (smem > 160 * 1024) return false;
    const int nrb = (Pl.nth + RB - 1) / RB, nec = E / EC;
    const int64_t blocks = (int64_t)Pl.nbox * nrb * nec;
    if (blocks > 0x7fffffffLL) return false;
    auto kern = k_interp_pbE<T, P>;
    bi_raise_smem(kern, smem);
    kern<<<(unsigned)blocks, 256, smem, s>>>(C.nth, C.nph, Pl.nth, Pl.nph, E, RB, EC, nrb, Pl.d_child_ptr, C.d_octant,
                                             (const tap<T>*)I.d_th_tap, (const tap<T>*)I.d_ph_tap,
                                             (const cpx<T>*)Pl.d_shift, (const cpx<T>*)C.d_U, (cpx<T>*)Pl.d_U);
    CU(cudaGetLastError());
    return true;
}

template <typename T, int PT, int PP>
bool anterp_t_p(bi_handle_s* h, int l, int E, cudaStream_t s) {
    level_t& Pl = h->lev[l];
    level_t& C = h->lev[l + 1];
    interp_t& I = h->itp[l];
    const size_t smem = (size_t)(C.nth * PT + C.nph * PP) * sizeof(tap<T>) +
                        ((size_t)Pl.K * E + (size_t)Pl.nth * C.nph * E) * sizeof(cpx<T>);
    if (smem > 160 * 1024) return false;
    if (E == 2) {
        auto k1 = k_anterp_cb1<T, PT>;
        bi_raise_smem(k1, smem);
        k1<<<C.nbox, 256, smem, s>>>(C.nth, C.nph, Pl.nth, Pl.nph, C.d_parent, C.d_octant, (const tap<T>*)I.d_tth_pad,
                                     (const tap<T>*)I.d_tph_pad, (const cpx<T>*)Pl.d_shift_dn, (const cpx<T>*)Pl.d_V,
                                     (cpx<T>*)C.d_V);
        CU(cudaGetLastError());
        return true;
    }
    auto kern = k_anterp_cb<T, PT, PP>;
    bi_raise_smem(kern, smem);
    kern<<<C.nbox, 256, smem, s>>>(C.nth, C.nph, Pl.nth, Pl.nph, E, C.d_parent, C.d_octant, (const tap<T>*)I.d_tth_pad,
                                   (const tap<T>*)I.d_tph_pad, (const cpx<T>*)Pl.d_shift_dn, (const cpx<T>*)Pl.d_V,
                                   (cpx<T>*)C.d_V);
    CU(cudaGetLastError());
    return true;
}

// Several right-hand sides: one CTA per (child, chunk of EC entries), EC the largest of 16, 8,
// 4, 2 dividing E whose shared memory (shifted parent field and transposed phi pass of the
// chunk) stays within about 80 KB; false when even EC = 2 does not fit (coarse levels).
template <typename T, int PT>
bool anterp_chunked(bi_handle_s* h, int l, int E, cudaStream_t s, int ec_force = 0) {
    level_t& Pl = h->lev[l];
    level_t& C = h->lev[l + 1];
    interp_t& I = h->itp[l];
    const size_t taps = (((size_t)(C.nth + C.nph) * PT * sizeof(tap<T>) + 15) / 16) * 16;
    int EC = 0;
    size_t smem = 0;
    for (int ec : {16, 8, 4, 2}) {
        const size_t sm = taps + ((size_t)Pl.K + (size_t)Pl.nth * C.nph) * ec * sizeof(cpx<T>);
        if (E % ec == 0 && sm <= (ec_force ? 160 : 80) * 1024 && (!ec_force || ec == ec_force)) {
            EC = ec;
            smem = sm;
            break;
        }
    }
    if (!EC) return false;
    const int64_t blocks = (int64_t)C.nbox * (E / EC);
    if (blocks > 0x7fffffffLL) return false;
    auto kern = k_anterp_cbE<T, PT>;
    bi_raise_smem(kern, smem);
    kern<<<(unsigned)blocks, 256, smem, s>>>(C.nth, C.nph, Pl.nth, Pl.nph, E, EC, C.d_parent, C.d_octant,
                                             (const tap<T>*)I.d_tth_pad, (const tap<T>*)I.d_tph_pad,
                                             (const cpx<T>*)Pl.d_shift_dn, (const cpx<T>*)Pl.d_V, (cpx<T>*)C.d_V);
    CU(cudaGetLastError());
    return true;
}

// Coarse levels: the row-blocked kernel, EC the largest of 16, 8, 4, 2 dividing E with at least
// one child row's parent-column field (nphp x EC) in about 48 KB; rows fill up to that.
template <typename T, int PT>
bool anterp_rows(bi_handle_s* h, int l, int E, cudaStream_t s, int ec_force = 0) {
    level_t& Pl = h->lev[l];
    level_t& C = h->lev[l + 1];
    interp_t& I = h->itp[l];
    const size_t budget = 48 * 1024;
    int EC = 0;
    for (int ec : {16, 8, 4, 2})
        if (E % ec == 0 && (size_t)Pl.nph * ec * sizeof(cpx<T>) * 2 <= budget && (!ec_force || ec == ec_force)) {
            EC = ec;
            break;
        }
    if (!EC) return false;
    const size_t per_row = (size_t)Pl.nph * EC * sizeof(cpx<T>);
    int RB = (int)std::max<size_t>(1, budget / per_row);
    RB = std::min(RB, C.nth);
    const size_t smem = (((size_t)(RB + C.nph) * PT * sizeof(tap<T>) + 15) / 16) * 16 + (size_t)RB * per_row;
    if (smem > 160 * 1024) return false;
    const int nrb = (C.nth + RB - 1) / RB, nec = E / EC;
    const int64_t blocks = (int64_t)C.nbox * nrb * nec;
    if (blocks > 0x7fffffffLL) return false;
    auto kern = k_anterp_rbE<T, PT>;
    bi_raise_smem(kern, smem);
    kern<<<(unsigned)blocks, 256, smem, s>>>(C.nth, C.nph, Pl.nth, Pl.nph, E, RB, EC, nrb, C.d_parent, C.d_octant,
                                             (const tap<T>*)I.d_tth_pad, (const tap<T>*)I.d_tph_pad,
                                             (const cpx<T>*)Pl.d_shift_dn, (const cpx<T>*)Pl.d_V, (cpx<T>*)C.d_V);
    CU(cudaGetLastError());
    return true;
}

template <typename T>
bool anterp_t(bi_handle_s* h, int l, int E, cudaStream_t s) {
    const interp_t& I = h->itp[l];
    if (I.pt_th == 16 && I.pt_ph == 16) return anterp_t_p<T, 16, 16>(h, l, E, s);
    if (I.pt_th == 24 && I.pt_ph == 24) return anterp_t_p<T, 24, 24>(h, l, E, s);
    return false;
}

}  // namespace

void bi_upload_taps(bi_handle_s* h) {
    if (h->prec == 0) upload_taps_t<double>(h);
    else upload_taps_t<float>(h);
}

bool bi_interp_level(bi_handle_s* h, int l, int E, cudaStream_t s) {
    const interp_t& I = h->itp[l];
    if (I.p_th != 10 || I.p_ph != 10 || !I.d_th_tap) return false;
    const int v = h->force_variant >= 0 ? h->force_variant
                  : E > 2 && h->interp_variant > 0 ? h->interp_variant : (E > 2 ? h->variant_of(1, l, E) : 0);
    if (v >= 100) return h->prec == 0 ? interp_chunked<double, 10>(h, l, E, s, v - 100) : interp_chunked<float, 10>(h, l, E, s, v - 100);
    if (v == 2) return h->prec == 0 ? interp_wide<double>(h, l, E, s) : interp_wide<float>(h, l, E, s);
    if (v == 3) return h->prec == 0 ? interp_pairs<double>(h, l, E, s) : interp_pairs<float>(h, l, E, s);
    if (E > 2 && (h->prec == 0 ? interp_chunked<double, 10>(h, l, E, s) : interp_chunked<float, 10>(h, l, E, s)))
        return true;
    if (E >= 32) return h->prec == 0 ? interp_wide<double>(h, l, E, s) : interp_wide<float>(h, l, E, s);
    return h->prec == 0 ? interp_t_p<double, 10>(h, l, E, s) : interp_t_p<float, 10>(h, l, E, s);
}

bool bi_anterp_level(bi_handle_s* h, int l, int E, cudaStream_t s) {
    const interp_t& I = h->itp[l];
    if (!I.d_tth_pad) return false;
    const int v = h->force_variant >= 0 ? h->force_variant
                  : E > 2 && h->anterp_variant > 0 ? h->anterp_variant : (E > 2 ? h->variant_of(2, l, E) : 0);
    if (v != 0 && I.pt_th == I.pt_ph && (I.pt_th == 16 || I.pt_th == 24)) {
        const bool p16 = I.pt_th == 16, dbl = h->prec == 0;
        if (v >= 200)
            return p16 ? (dbl ? anterp_rows<double, 16>(h, l, E, s, v - 200) : anterp_rows<float, 16>(h, l, E, s, v - 200))
                       : (dbl ? anterp_rows<double, 24>(h, l, E, s, v - 200) : anterp_rows<float, 24>(h, l, E, s, v - 200));
        if (v >= 100)
            return p16 ? (dbl ? anterp_chunked<double, 16>(h, l, E, s, v - 100) : anterp_chunked<float, 16>(h, l, E, s, v - 100))
                       : (dbl ? anterp_chunked<double, 24>(h, l, E, s, v - 100) : anterp_chunked<float, 24>(h, l, E, s, v - 100));
        if (v == 2)
            return p16 ? (dbl ? anterp_wide<double, 16>(h, l, E, s) : anterp_wide<float, 16>(h, l, E, s))
                       : (dbl ? anterp_wide<double, 24>(h, l, E, s) : anterp_wide<float, 24>(h, l, E, s));
        if (v == 3)
            return p16 ? (dbl ? anterp_pairs<double, 16>(h, l, E, s) : anterp_pairs<float, 16>(h, l, E, s))
                       : (dbl ? anterp_pairs<double, 24>(h, l, E, s) : anterp_pairs<float, 24>(h, l, E, s));
    }
    if (E > 2 && I.pt_th == I.pt_ph) {
        const bool whole = !h->force_anterp_rows;
        if (whole && I.pt_th == 16 && (h->prec == 0 ? anterp_chunked<double, 16>(h, l, E, s) : anterp_chunked<float, 16>(h, l, E, s)))
            return true;
        if (whole && I.pt_th == 24 && (h->prec == 0 ? anterp_chunked<double, 24>(h, l, E, s) : anterp_chunked<float, 24>(h, l, E, s)))
            return true;
        if (I.pt_th == 16 && (h->prec == 0 ? anterp_rows<double, 16>(h, l, E, s) : anterp_rows<float, 16>(h, l, E, s)))
            return true;
        if (I.pt_th == 24 && (h->prec == 0 ? anterp_rows<double, 24>(h, l, E, s) : anterp_rows<float, 24>(h, l, E, s)))
            return true;
    }
    if (E >= 32) {
        if (I.pt_th == 16) return h->prec == 0 ? anterp_wide<double, 16>(h, l, E, s) : anterp_wide<float, 16>(h, l, E, s);
        if (I.pt_th == 24) return h->prec == 0 ? anterp_wide<double, 24>(h, l, E, s) : anterp_wide<float, 24>(h, l, E, s);
        return false;
    }
    return h->prec == 0 ? anterp_t<double>(h, l, E, s) : anterp_t<float>(h, l, E, s);
}
