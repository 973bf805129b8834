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

// Variant codes (autotuner): 1 / 2 = one / two pairs of entries per thread over all 8 child
// slots; 3 / 4 = the same with the child slots split over two threads (4 each).
template <typename T>
bool launch_tE(bi_handle_s* h, int l, int E, cudaStream_t s, int variant) {
    level_t& L = h->lev[l];
    const int R = E / 2;
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
