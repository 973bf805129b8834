// Diagonal translations of one level (the M2L step of the multilevel product):
//   V_b(k) = sum_{s in IL(b)} T[off(b, s)](k) U_s(k)     (quadrature weights folded into T)
// with IL(b) the children of the neighbours of b's parent that do not touch b.
//
// Parent-centred form: one CTA per (parent box p, 32 directions) computes V for every child of
// p.  The sources of all children of p are the children of p's neighbours; each source
// pattern U_s(k) is loaded once into registers and applied to every child that has s in its
// interaction list, the per-child offset codes coming from a host-built table (one 16-byte
// record of eight codes per (parent, source)).  The CTA's warps split the sources and meet
// in shared memory; every child's V is written once, without atomics.  One right-hand side
// (E = 2): each lane carries both components of its direction.
//
// Several right-hand sides (E = 2R > 2): thread = (direction k, one or two pairs of adjacent
// entries of the E-vector of k), so a CTA reads a contiguous tile of D directions x E entries of
// each source and the threads of a direction share every operator value (one broadcast load).
// CTAs run parents fastest: the CTAs resident at one time work on one direction tile of
// neighbouring parents, whose sources and the tile of the 343 operators stay in L2/L1.
#include <algorithm>
#include <cstdlib>
#include <unordered_map>
#include <utility>
#include <vector>

#include "bi_cpx.cuh"
#include "bi_internal.h"

namespace {

constexpr unsigned short kNone = 0xFFFF;

template <typename T, int kWarps>
__global__ void __launch_bounds__(32 * kWarps) k_translate_pc(int K, const int* __restrict__ cptr,
                                                              const int* __restrict__ tptr, const int* __restrict__ src,
                                                              const uint4* __restrict__ codes,
                                                              const cpx<T>* __restrict__ Top,
                                                              const cpx<T>* __restrict__ U, cpx<T>* __restrict__ V) {
    __shared__ cpx<T> red[kWarps][8][2][32];
    const int p = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = blockIdx.y * 32 + lane;
    const bool ok = k < K;
    const int kk = ok ? k : 0;
    const int c0 = cptr[p], nc = cptr[p + 1] - c0;
    cpx<T> a0[8], a1[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a0[j] = a1[j] = czero<T>();
    // unrolled so that several sources' loads are in flight at once
#pragma unroll 4
    for (int q = tptr[p] + warp; q < tptr[p + 1]; q += kWarps) {
        const int s = src[q];
        const uint4 cw = codes[q];
        const unsigned cc[4] = {cw.x, cw.y, cw.z, cw.w};
        cpx<T> u0, u1;
        load_pair(U + ((int64_t)s * K + kk) * 2, u0, u1);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const unsigned code = (cc[j >> 1] >> ((j & 1) * 16)) & 0xFFFFu;
            if (code != kNone) {
                const cpx<T> t = ldg_cpx(Top + (int64_t)code * K + kk);
                cfma(a0[j], t, u0);
                cfma(a1[j], t, u1);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        red[warp][j][0][lane] = a0[j];
        red[warp][j][1][lane] = a1[j];
    }
    __syncthreads();
    // thread -> (child j, lane): sum the warps' partials and write both components
    for (int t = threadIdx.x; t < nc * 32; t += blockDim.x) {
        const int j = t >> 5, l = t & 31;
        const int kd = blockIdx.y * 32 + l;
        if (kd >= K) continue;
        cpx<T> s0 = czero<T>(), s1 = czero<T>();
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            s0 = cadd(s0, red[w][j][0][l]);
            s1 = cadd(s1, red[w][j][1][l]);
        }
        cpx<T>* out = V + ((int64_t)(c0 + j) * K + kd) * 2;
        out[0] = s0;
        out[1] = s1;
    }
}

template <typename T>
__device__ __forceinline__ void store_pair(cpx<T>* p, cpx<T> a, cpx<T> b) {
    p[0] = a;
    p[1] = b;
}
__device__ __forceinline__ void store_pair(cpx<float>* p, cpx<float> a, cpx<float> b) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}

template <typename T, int VP, int CH>
__global__ void __launch_bounds__(256) k_translate_pcE(int K, int R, int D, int np, const int* __restrict__ cptr,
                                                       const int* __restrict__ tptr, const int* __restrict__ src,
                                                       const uint4* __restrict__ codes, const cpx<T>* __restrict__ Top,
                                                       const cpx<T>* __restrict__ U, cpx<T>* __restrict__ V) {
    // thread = (direction, VP consecutive pairs of entries, CH of the parent's 8 child slots);
    // the next source's entries and offset codes are loaded one iteration ahead.  CH = 4 halves
    // the accumulators (more resident warps) at the price of loading each source twice.
    constexpr int NH = 8 / CH;                 // threads sharing one (direction, pairs)
    const int p = (int)(blockIdx.x % (unsigned)np);
    const int chunk = (int)(blockIdx.x / (unsigned)np);
    const int TPP = R / VP;                    // pair groups per direction
    const int TPD = TPP * NH;                  // threads per direction
    const int d = threadIdx.x / TPD, jj = threadIdx.x - d * TPD;
    const int j = jj % TPP, half = jj / TPP;
    const int k = chunk * D + d;
    if (d >= D || k >= K) return;   // no barrier below
    const int64_t E = 2 * R;
    const int c0 = cptr[p], nc = cptr[p + 1] - c0;
    cpx<T> acc[CH][2 * VP];
#pragma unroll
    for (int i = 0; i < CH; ++i)
#pragma unroll
        for (int v = 0; v < 2 * VP; ++v) acc[i][v] = czero<T>();
    const cpx<T>* ub = U + (int64_t)k * E + 2 * VP * j;
    const cpx<T>* tk = Top + k;
    const int64_t box = (int64_t)K * E;
    const int q0 = tptr[p], q1 = tptr[p + 1];
    cpx<T> un[2 * VP];
    uint4 cn = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
    if (q0 < q1) {
        const cpx<T>* us = ub + (int64_t)src[q0] * box;
#pragma unroll
        for (int v = 0; v < VP; ++v) load_pair(us + 2 * v, un[2 * v], un[2 * v + 1]);
        cn = codes[q0];
    }
    for (int q = q0; q < q1; ++q) {
        cpx<T> u[2 * VP];
#pragma unroll
        for (int v = 0; v < 2 * VP; ++v) u[v] = un[v];
        // the 16-bit codes of this thread's child slots, indexed at compile time only
        const unsigned w0 = CH == 8 ? cn.x : (half ? cn.z : cn.x), w1 = CH == 8 ? cn.y : (half ? cn.w : cn.y);
        const unsigned w2 = cn.z, w3 = cn.w;
        if (q + 1 < q1) {
            const cpx<T>* us = ub + (int64_t)src[q + 1] * box;
#pragma unroll
            for (int v = 0; v < VP; ++v) load_pair(us + 2 * v, un[2 * v], un[2 * v + 1]);
            cn = codes[q + 1];
        }
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            const unsigned w = (i >> 1) == 0 ? w0 : (i >> 1) == 1 ? w1 : (i >> 1) == 2 ? w2 : w3;
            const unsigned code = (w >> ((i & 1) * 16)) & 0xFFFFu;
            if (code != kNone) {
                const cpx<T> t = ldg_cpx(tk + (int64_t)code * K);
#pragma unroll
                for (int v = 0; v < 2 * VP; ++v) cfma(acc[i][v], t, u[v]);
            }
        }
    }
    cpx<T>* vb = V + (int64_t)c0 * box + (int64_t)k * E + 2 * VP * j;
#pragma unroll
    for (int i = 0; i < CH; ++i) {
        const int ci = (CH == 8 ? 0 : half * CH) + i;
        if (ci < nc)
#pragma unroll
            for (int v = 0; v < VP; ++v) store_pair(vb + ci * box + 2 * v, acc[i][2 * v], acc[i][2 * v + 1]);
    }
}

// Pipelined form of the above: the offset codes are loaded two sources ahead, the operator
// values T[code](k) and the source entries one source ahead, so no load is consumed in the
// iteration that issues it.  A child slot without an interaction reads the zero row 343 of T,
// so every slot runs the same multiply-adds without a branch.  CH = 4 or 8 child slots per
// thread.
template <typename T, int VP, int CH>
__global__ void __launch_bounds__(256, CH == 4 ? 3 : 2) k_translate_pp(int K, int R, int D, int np,
                                                                       const int* __restrict__ cptr,
                                                                       const int* __restrict__ tptr,
                                                                       const int* __restrict__ src,
                                                                       const uint4* __restrict__ codes,
                                                                       const cpx<T>* __restrict__ Top,
                                                                       const cpx<T>* __restrict__ U, cpx<T>* __restrict__ V) {
    constexpr int NH = 8 / CH;
    const int p = (int)(blockIdx.x % (unsigned)np);
    const int chunk = (int)(blockIdx.x / (unsigned)np);
    const int TPP = R / VP;
    const int TPD = TPP * NH;
    const int d = threadIdx.x / TPD, jj = threadIdx.x - d * TPD;
    const int j = jj % TPP, half = jj / TPP;
    const int k = chunk * D + d;
    if (d >= D || k >= K) return;   // no barrier below
    const int64_t E = 2 * R;
    const int c0 = cptr[p], nc = cptr[p + 1] - c0;
    cpx<T> acc[CH][2 * VP];
#pragma unroll
    for (int i = 0; i < CH; ++i)
#pragma unroll
        for (int v = 0; v < 2 * VP; ++v) acc[i][v] = czero<T>();
    const cpx<T>* ub = U + (int64_t)k * E + 2 * VP * j;
    const cpx<T>* tk = Top + k;
    const int64_t box = (int64_t)K * E;
    const int q0 = tptr[p], q1 = tptr[p + 1];
    // this thread's code words (CH slots) of a source record; past the list: no interaction
    auto words = [&](int q, unsigned* w) {
        if (q < q1) {
            const uint4 c = codes[q];
            if (CH == 8) {
                w[0] = c.x; w[1] = c.y; w[2] = c.z; w[3] = c.w;
            } else {
                w[0] = half ? c.z : c.x;
                w[1] = half ? c.w : c.y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < CH / 2; ++i) w[i] = 0xFFFFFFFFu;
        }
    };
    auto load_t = [&](const unsigned* w, cpx<T>* t) {
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            const unsigned code = min((w[i >> 1] >> ((i & 1) * 16)) & 0xFFFFu, 343u);
            t[i] = ldg_cpx(tk + (int64_t)code * K);
        }
    };
    auto load_u = [&](int q, cpx<T>* u) {
        if (q < q1) {
            const cpx<T>* us = ub + (int64_t)src[q] * box;
#pragma unroll
            for (int v = 0; v < VP; ++v) load_pair(us + 2 * v, u[2 * v], u[2 * v + 1]);
        }
    };
    unsigned w1[CH / 2], w2[CH / 2];
    cpx<T> t1[CH], u1[2 * VP];
    words(q0, w1);
    words(q0 + 1, w2);
    load_t(w1, t1);
    load_u(q0, u1);
    for (int q = q0; q < q1; ++q) {
        cpx<T> t[CH], u[2 * VP];
#pragma unroll
        for (int i = 0; i < CH; ++i) t[i] = t1[i];
#pragma unroll
        for (int v = 0; v < 2 * VP; ++v) u[v] = u1[v];
        // issue the next source's operator values and entries, and the codes after that
        load_t(w2, t1);
        load_u(q + 1, u1);
        words(q + 2, w2);
#pragma unroll
        for (int i = 0; i < CH; ++i)
#pragma unroll
            for (int v = 0; v < 2 * VP; ++v) cfma(acc[i][v], t[i], u[v]);
    }
    cpx<T>* vb = V + (int64_t)c0 * box + (int64_t)k * E + 2 * VP * j;
#pragma unroll
    for (int i = 0; i < CH; ++i) {
        const int ci = (CH == 8 ? 0 : half * CH) + i;
        if (ci < nc)
#pragma unroll
            for (int v = 0; v < VP; ++v) store_pair(vb + ci * box + 2 * v, acc[i][2 * v], acc[i][2 * v + 1]);
    }
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Staged form (FP32): CTA = (parent p, 32 directions, one group of EP entries); thread =
// (direction, child slot) with the EP entries of its group in registers.  The sources' entries
// for the CTA's directions are copied into shared memory, KS sources per stage and two stages in
// flight (cp.async), so each source value is read from global memory once per CTA and then by
// the 8 child-slot threads of its direction from shared memory (a broadcast); every operator
// value T[code](k) serves EP multiply-adds.  Rows are padded by 16 bytes so the 4 directions
// of a warp read distinct banks.
constexpr int kTrDir = 32, kTrStage = 8;
template <int EP>
__global__ void __launch_bounds__(256, 3) k_translate_sm(int K, int E, int np, const int* __restrict__ cptr,
                                                         const int* __restrict__ tptr, const int* __restrict__ src,
                                                         const uint4* __restrict__ codes,
                                                         const cpx<float>* __restrict__ Top,
                                                         const cpx<float>* __restrict__ U, cpx<float>* __restrict__ V) {
    constexpr int ROW = EP + 2;                    // complex values per staged row (16-byte pad)
    extern __shared__ float4 smem_tr[];
    cpx<float>* buf = reinterpret_cast<cpx<float>*>(smem_tr);   // [2][kTrStage][kTrDir][ROW]
    const int p = (int)(blockIdx.x % (unsigned)np);
    const int k0 = (int)(blockIdx.x / (unsigned)np) * kTrDir;
    const int e0 = blockIdx.y * EP;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int dl = warp * 4 + (lane & 3), slot = lane >> 2;
    const int k = k0 + dl;
    const int q0 = tptr[p], q1 = tptr[p + 1];
    const int c0 = cptr[p], nc = cptr[p + 1] - c0;
    const int64_t box = (int64_t)K * E;
    cpx<float> acc[EP];
#pragma unroll
    for (int e = 0; e < EP; ++e) acc[e] = czero<float>();
    // copy sources qs .. qs + n - 1 (n <= kTrStage) into stage st: 16-byte chunks of (source,
    // direction, entry pair); directions past K are zero-filled
    auto stage = [&](int st, int qs) {
        const int n = min(kTrStage, q1 - qs);
        const int chunks = n * kTrDir * (EP / 2);
        for (int i = threadIdx.x; i < chunks; i += blockDim.x) {
            const int h = i % (EP / 2), d = (i / (EP / 2)) % kTrDir, sq = i / (kTrDir * (EP / 2));
            cpx<float>* dst = buf + ((size_t)(st * kTrStage + sq) * kTrDir + d) * ROW + 2 * h;
            if (k0 + d < K)
                cp_async16(dst, U + (int64_t)src[qs + sq] * box + (int64_t)(k0 + d) * E + e0 + 2 * h);
            else
                *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        cp_async_commit();
    };
    if (q0 < q1) stage(0, q0);
    for (int qs = q0, it = 0; qs < q1; qs += kTrStage, ++it) {
        const int st = it & 1;
        if (qs + kTrStage < q1) {
            stage(st ^ 1, qs + kTrStage);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int n = min(kTrStage, q1 - qs);
        for (int sq = 0; sq < n; ++sq) {
            const uint4 cw = codes[qs + sq];
            const unsigned long long half = slot < 4 ? ((unsigned long long)cw.y << 32 | cw.x)
                                                     : ((unsigned long long)cw.w << 32 | cw.z);
            const unsigned code = (unsigned)(half >> (16 * (slot & 3))) & 0xFFFFu;
            if (code != kNone && k < K) {
                const cpx<float> t = ldg_cpx(Top + (int64_t)code * K + k);
                const cpx<float>* u = buf + ((size_t)(st * kTrStage + sq) * kTrDir + dl) * ROW;
#pragma unroll
                for (int e = 0; e < EP; e += 2) {
                    cpx<float> a, b;
                    lds_pair(u + e, a, b);
                    cfma(acc[e], t, a);
                    cfma(acc[e + 1], t, b);
                }
            }
        }
        __syncthreads();   // stage st is refilled by the copy issued in the next iteration
    }
    if (slot < nc && k < K) {
        cpx<float>* vb = V + (int64_t)(c0 + slot) * box + (int64_t)k * E + e0;
#pragma unroll
        for (int e = 0; e < EP; e += 2) store_pair(vb + e, acc[e], acc[e + 1]);
    }
}

template <int EP>
bool launch_tsm(level_t& L, int E, cudaStream_t s) {
    const size_t smem = (size_t)2 * kTrStage * kTrDir * (EP + 2) * sizeof(cpx<float>);
    bi_raise_smem(k_translate_sm<EP>, smem);
    const int64_t nchunk = (L.K + kTrDir - 1) / kTrDir;
    const int64_t blocks = nchunk * L.tp_np;
    if (blocks > 0x7fffffffLL) throw bi_error{BI_ERR_ARG, "translation grid too large"};
    dim3 g((unsigned)blocks, E / EP);
    k_translate_sm<EP><<<g, 256, smem, s>>>(L.K, E, L.tp_np, L.d_tp_cptr, L.d_tp_ptr, L.d_tp_src,
                                            (const uint4*)L.d_tp_code, (const cpx<float>*)L.d_T,
                                            (const cpx<float>*)L.d_U, (cpx<float>*)L.d_V);
    CU(cudaGetLastError());
    return true;
}

// Variant codes (autotuner): 1 / 2 = one / two pairs of entries per thread over all 8 child
// slots; 3 / 4 = the same with the child slots split over two threads (4 each); 5 = the staged
// form (FP32, E a multiple of 4); 6 / 7 = the pipelined form with 4 child slots per thread, one
// or two pairs; 8 / 9 = the pipelined form with all 8 child slots, one or two pairs.
template <typename T>
bool launch_tE(bi_handle_s* h, int l, int E, cudaStream_t s, int variant) {
    level_t& L = h->lev[l];
    if (variant == 5) {
        if (sizeof(T) != 4 || E % 4 != 0) return false;
        return E % 16 == 0 ? launch_tsm<16>(L, E, s) : E % 8 == 0 ? launch_tsm<8>(L, E, s) : launch_tsm<4>(L, E, s);
    }
    const int R = E / 2;
    if (variant >= 6 && variant <= 9) {
        const int VP = (variant == 7 || variant == 9) ? 2 : 1;
        const int CH = variant <= 7 ? 4 : 8;
        if (R % VP != 0) return false;
        const int TPD = R / VP * (8 / CH);
        if (TPD > 256) return false;
        const int D = std::max(1, 256 / TPD);
        const int threads = std::min(1024, (D * TPD + 31) / 32 * 32);
        const int64_t blocks = (int64_t)((L.K + D - 1) / D) * L.tp_np;
        if (blocks > 0x7fffffffLL) throw bi_error{BI_ERR_ARG, "translation grid too large"};
        // FP64 runs only the one-pair forms: two pairs would not fit the register bounds
        auto kern = CH == 4 ? k_translate_pp<T, 1, 4> : k_translate_pp<T, 1, 8>;
        if constexpr (sizeof(T) == 4) {
            if (VP == 2) kern = CH == 4 ? k_translate_pp<T, 2, 4> : k_translate_pp<T, 2, 8>;
        } else {
            if (VP == 2) return false;
        }
        kern<<<(unsigned)blocks, threads, 0, s>>>(L.K, R, D, L.tp_np, L.d_tp_cptr, L.d_tp_ptr, L.d_tp_src,
                                                  (const uint4*)L.d_tp_code, (const cpx<T>*)L.d_T, (const cpx<T>*)L.d_U,
                                                  (cpx<T>*)L.d_V);
        CU(cudaGetLastError());
        return true;
    }
    // two pairs per thread when R is even (FP32): the code decode and operator loads serve twice
    // the multiply-adds
    int VP = (R % 2 == 0 && sizeof(T) == 4) ? 2 : 1;
    int CH = 8;
    if (variant == 1 || variant == 3) VP = 1;
    if (variant == 2 || variant == 4) {
        if (R % 2 != 0) return false;
        VP = 2;
    }
    if (variant == 3 || variant == 4) CH = 4;
    const int TPD = R / VP * (8 / CH);
    if (TPD > 256) return false;
    const int D = std::max(1, 256 / TPD);
    const int threads = std::min(1024, (D * TPD + 31) / 32 * 32);
    const int64_t nchunk = (L.K + D - 1) / D;
    const int64_t blocks = nchunk * L.tp_np;
    if (blocks > 0x7fffffffLL) throw bi_error{BI_ERR_ARG, "translation grid too large"};
    auto kern = VP == 2 ? (CH == 8 ? k_translate_pcE<T, 2, 8> : k_translate_pcE<T, 2, 4>)
                        : (CH == 8 ? k_translate_pcE<T, 1, 8> : k_translate_pcE<T, 1, 4>);
    kern<<<(unsigned)blocks, threads, 0, s>>>(L.K, R, D, L.tp_np, L.d_tp_cptr, L.d_tp_ptr, L.d_tp_src,
                                              (const uint4*)L.d_tp_code, (const cpx<T>*)L.d_T, (const cpx<T>*)L.d_U,
                                              (cpx<T>*)L.d_V);
    CU(cudaGetLastError());
    return true;
}

template <typename T>
void launch_t(bi_handle_s* h, int l, cudaStream_t s) {
    level_t& L = h->lev[l];
    dim3 g(L.tp_np, (L.K + 31) / 32);
    // levels with few (parent, chunk) CTAs split each parent's sources over more warps
    if ((int64_t)g.x * g.y < 4 * h->num_sms)
        k_translate_pc<T, 8><<<g, 256, 0, s>>>(L.K, L.d_tp_cptr, L.d_tp_ptr, L.d_tp_src, (const uint4*)L.d_tp_code,
                                               (const cpx<T>*)L.d_T, (const cpx<T>*)L.d_U, (cpx<T>*)L.d_V);
    else
        k_translate_pc<T, 4><<<g, 128, 0, s>>>(L.K, L.d_tp_cptr, L.d_tp_ptr, L.d_tp_src, (const uint4*)L.d_tp_code,
                                               (const cpx<T>*)L.d_T, (const cpx<T>*)L.d_U, (cpx<T>*)L.d_V);
    CU(cudaGetLastError());
}

inline uint64_t ckey(int x, int y, int z) {
    return ((uint64_t)(uint32_t)x << 42) | ((uint64_t)(uint32_t)y << 21) | (uint64_t)(uint32_t)z;
}

}  // namespace

void bi_plan_translate_lists(bi_handle_s* h) {
    for (int l = 2; l <= h->leaf; ++l) {
        level_t& C = h->lev[l];
        const level_t& P = h->lev[l - 1];
        std::unordered_map<uint64_t, int> pidx;
        pidx.reserve(P.nbox * 2);
        for (int b = 0; b < P.nbox; ++b) pidx[ckey(P.coords[3 * b], P.coords[3 * b + 1], P.coords[3 * b + 2])] = b;
        const int pside = 1 << (l - 1);
        std::vector<int> tptr(P.nbox + 1, 0), src;
        std::vector<unsigned short> code;
        for (int p = 0; p < P.nbox; ++p) {
            const int c0 = P.child_ptr[p], nc = P.child_ptr[p + 1] - c0;
            if (nc > 8) throw bi_error{BI_ERR_ARG, "octree parent with more than 8 children"};
            for (int dx = -1; dx <= 1; ++dx)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dz = -1; dz <= 1; ++dz) {
                        const int x = P.coords[3 * p] + dx, y = P.coords[3 * p + 1] + dy, z = P.coords[3 * p + 2] + dz;
                        if (x < 0 || y < 0 || z < 0 || x >= pside || y >= pside || z >= pside) continue;
                        auto it = pidx.find(ckey(x, y, z));
                        if (it == pidx.end()) continue;
                        const int qb = it->second;
                        for (int s = P.child_ptr[qb]; s < P.child_ptr[qb + 1]; ++s) {
                            unsigned short cs[8];
                            bool any = false;
                            for (int j = 0; j < 8; ++j) {
                                cs[j] = kNone;
                                if (j >= nc) continue;
                                const int b = c0 + j;
                                const int ox = C.coords[3 * b] - C.coords[3 * s];
                                const int oy = C.coords[3 * b + 1] - C.coords[3 * s + 1];
                                const int oz = C.coords[3 * b + 2] - C.coords[3 * s + 2];
                                if (std::abs(ox) <= 1 && std::abs(oy) <= 1 && std::abs(oz) <= 1) continue;
                                cs[j] = (unsigned short)((ox + 3) * 49 + (oy + 3) * 7 + (oz + 3));
                                any = true;
                            }
                            if (!any) continue;
                            src.push_back(s);
                            code.insert(code.end(), cs, cs + 8);
                        }
                    }
            tptr[p + 1] = (int)src.size();
        }
        C.tp_np = P.nbox;
        C.tp_ptr = std::move(tptr);
        C.tp_src = std::move(src);
        C.tp_code = std::move(code);
    }
}

void bi_build_translate_lists(bi_handle_s* h) {
    bi_plan_translate_lists(h);
    for (int l = 2; l <= h->leaf; ++l) {
        level_t& C = h->lev[l];
        const level_t& P = h->lev[l - 1];
        std::vector<int> cptr(P.child_ptr.begin(), P.child_ptr.end());
        C.d_tp_cptr = h->upload(cptr);
        C.d_tp_ptr = h->upload(C.tp_ptr);
        if (!C.tp_src.empty()) {
            C.d_tp_src = h->upload(C.tp_src);
            C.d_tp_code = h->upload(C.tp_code);
        } else {
            C.d_tp_src = (int*)h->alloc(sizeof(int));
            C.d_tp_code = h->alloc(16);
        }
    }
}

bool bi_translate_level(bi_handle_s* h, int l, int E, cudaStream_t s) {
    if (!h->lev[l].d_tp_ptr || h->lev[l].tp_np == 0) return false;
    if (E == 2) {
        if (h->prec == 0) launch_t<double>(h, l, s);
        else launch_t<float>(h, l, s);
    } else if (E <= 512) {
        const int v = h->force_variant >= 0 ? h->force_variant
                      : h->translate_variant > 0 ? h->translate_variant : h->variant_of(0, l, E);
        return h->prec == 0 ? launch_tE<double>(h, l, E, s, v) : launch_tE<float>(h, l, E, s, v);
    } else {
        return false;
    }
    return true;
}
