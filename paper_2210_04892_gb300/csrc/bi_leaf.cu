// Leaf aggregation and leaf receive of the product (the two steps that read the leaf
// radiation patterns, Sec. II.E step 2(a) accelerated as in the far-field formulation of the
// product kernels) as bulk-copy pipelines.
//
// Both steps are bound by HBM: per leaf box they stream the box's rows of F (and RX) once,
// the rows of one box being contiguous in tree order.  One CTA per leaf box keeps a ring of
// S stages, each holding the rows of G RWGs, filled by cp.async.bulk (TMA) copies that
// complete on one mbarrier per stage; thread 0 refills a stage as soon as the CTA has
// consumed it, so up to S stages per CTA are in flight while the CTA computes.
//
//   aggregation: U_b(k)  = sum_{n in b} ( -x_J,n F_n(k) + x_M,n khat x F_n(k) ) at each stored
//                direction k and at its antipode (pattern (conj F_theta, -conj F_phi));
//   receive:     y_J,m = -(k^2/32 pi^2) sum_k [ R_m.V - RX_m.(khat x V) ],
//                y_M,m = +(k^2/32 pi^2) sum_k [ -R_m.(khat x V) - RX_m.V ],
//                the incoming field V of the box staged once, plus the near result, written
//                in user order.
#include <algorithm>

#include "bi_cpx.cuh"
#include "bi_internal.h"
#include "bi_tma.cuh"

namespace {

constexpr int kBarBytes = 128;  // shared-memory header: up to 16 mbarriers

// CTA = one leaf box; thread slot = (stored direction kk, RHS r), SL slots per thread.
template <typename T, int MODE, int SL>
__global__ void __launch_bounds__(256) k_aggregate_bulk(int N, int K, int nph, int R, int nun, int G, int S,
                                                        const int* __restrict__ perm, const int* __restrict__ leaf_start,
                                                        const int* __restrict__ order, const cpx<T>* __restrict__ F,
                                                        const cpx<T>* __restrict__ x, cpx<T>* __restrict__ U,
                                                        int* __restrict__ status, long long wait) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int Kh = K / 2, E = 2 * R;
    const int b = order[blockIdx.x];
    const int n0 = leaf_start[b], nb = leaf_start[b + 1] - n0;
    const int64_t row = (int64_t)Kh * 2;        // complex entries of one RWG's pattern row
    const int64_t stage = (int64_t)G * row;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    cpx<T>* ring = reinterpret_cast<cpx<T>*>(smem_raw + kBarBytes);  // [S][G][Kh][2]
    cpx<T>* xs = ring + S * stage;                                    // [nb][2][R]
    const int nch = (nb + G - 1) / G;
    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) mbar_init(&bar[i], 1);
        fence_barrier_init();
        for (int c = 0; c < min(S, nch); ++c) {
            const int cnt = min(G, nb - c * G);
            const uint32_t bytes = (uint32_t)(cnt * row * sizeof(cpx<T>));
            mbar_arrive_expect_tx(&bar[c], bytes);
            bulk_copy_g2s(ring + c * stage, F + (n0 + (int64_t)c * G) * row, bytes, &bar[c]);
        }
    }
    for (int i = threadIdx.x; i < nb * 2 * R; i += blockDim.x) {
        const int r = i % R, X = (i / R) % 2, n = i / (2 * R);
        xs[i] = (MODE == 0 || X == 0) ? x[(int64_t)r * nun + (int64_t)X * N + perm[n0 + n]] : czero<T>();
    }
    __syncthreads();
    // (ut, up) at kk, (vt, vp) at its antipode
    cpx<T> ut[SL], up[SL], vt[SL], vp[SL];
#pragma unroll
    for (int j = 0; j < SL; ++j) ut[j] = up[j] = vt[j] = vp[j] = czero<T>();
    for (int c = 0; c < nch; ++c) {
        const int st = c % S;
        const bool ok = mbar_wait_bounded(&bar[st], (c / S) & 1, wait);
        if (!__syncthreads_and(ok)) {
            bulk_give_up(bar, c, nch, S, status);
            return;
        }
        const cpx<T>* f = ring + st * stage;
        const int cnt = min(G, nb - c * G);
#pragma unroll
        for (int j = 0; j < SL; ++j) {
            const int slot = threadIdx.x + j * blockDim.x;
            if (slot < Kh * R) {
                const int kk = slot / R, r = slot - kk * R;
                for (int i = 0; i < cnt; ++i) {
                    cpx<T> Ft, Fp;
                    lds_pair(f + (i * Kh + kk) * 2, Ft, Fp);
                    const cpx<T> xJ = xs[((c * G + i) * 2 + 0) * R + r];
                    const cpx<T> xM = MODE == 0 ? xs[((c * G + i) * 2 + 1) * R + r] : czero<T>();
                    agg_pair<T, MODE>(Ft, Fp, xJ, xM, ut[j], up[j], vt[j], vp[j]);
                }
            }
        }
        __syncthreads();  // stage st consumed by every thread
        if (threadIdx.x == 0 && c + S < nch) {
            const int cn = c + S, cnt2 = min(G, nb - cn * G);
            const uint32_t bytes = (uint32_t)(cnt2 * row * sizeof(cpx<T>));
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[st], bytes);
            bulk_copy_g2s(ring + st * stage, F + (n0 + (int64_t)cn * G) * row, bytes, &bar[st]);
        }
    }
#pragma unroll
    for (int j = 0; j < SL; ++j) {
        const int slot = threadIdx.x + j * blockDim.x;
        if (slot < Kh * R) {
            const int kk = slot / R, r = slot - kk * R;
            cpx<T>* o = U + ((int64_t)b * K + kk) * E;
            o[r] = ut[j];
            o[R + r] = up[j];
            cpx<T>* oa = U + ((int64_t)b * K + antipode(kk, K, nph)) * E;
            oa[r] = vt[j];
            oa[R + r] = vp[j];
        }
    }
}

// CTA = one leaf box; warp task = (RWG of the stage, RHS r); lanes over stored directions.
template <typename T, int MODE, int R1>
__global__ void __launch_bounds__(256) k_receive_bulk(int N, int K, int nph, int R_, int nun, int G, int S,
                                                      const int* __restrict__ perm, const int* __restrict__ leaf_start,
                                                      const int* __restrict__ order, const cpx<T>* __restrict__ F,
                                                      const cpx<T>* __restrict__ RX, const cpx<T>* __restrict__ V, T cc,
                                                      const cpx<T>* __restrict__ yt, cpx<T>* __restrict__ y,
                                                      int* __restrict__ status, long long wait) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int R = R1 ? 1 : R_;   // R1: one right-hand side, (V_theta, V_phi) adjacent
    const int Kh = K / 2, E = 2 * R;
    const int b = order[blockIdx.x];
    const int n0 = leaf_start[b], nb = leaf_start[b + 1] - n0;
    const int64_t row = (int64_t)Kh * 2;
    const int64_t half = (int64_t)G * row;    // F part of a stage; RX part follows
    const int64_t stage = 2 * half;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);      // [S] stages, [S] = V
    cpx<T>* vs = reinterpret_cast<cpx<T>*>(smem_raw + kBarBytes);  // [K][E]
    cpx<T>* ring = vs + (int64_t)K * E;                           // [S][F: G][Kh][2] [RX: G][Kh][2]
    int* ap = reinterpret_cast<int*>(ring + S * stage);            // [Kh] antipode of each stored direction
    const int nch = (nb + G - 1) / G;
    for (int kk = threadIdx.x; kk < Kh; kk += blockDim.x) ap[kk] = antipode(kk, K, nph);
    if (threadIdx.x == 0) {
        for (int i = 0; i <= S; ++i) mbar_init(&bar[i], 1);
        fence_barrier_init();
        const uint32_t vbytes = (uint32_t)((int64_t)K * E * sizeof(cpx<T>));
        mbar_arrive_expect_tx(&bar[S], vbytes);
        bulk_copy_g2s(vs, V + (int64_t)b * K * E, vbytes, &bar[S]);
        for (int c = 0; c < min(S, nch); ++c) {
            const int cnt = min(G, nb - c * G);
            const uint32_t bytes = (uint32_t)(cnt * row * sizeof(cpx<T>));
            mbar_arrive_expect_tx(&bar[c], 2 * bytes);
            bulk_copy_g2s(ring + c * stage, F + (n0 + (int64_t)c * G) * row, bytes, &bar[c]);
            bulk_copy_g2s(ring + c * stage + half, RX + (n0 + (int64_t)c * G) * row, bytes, &bar[c]);
        }
    }
    __syncthreads();
    if (!__syncthreads_and(mbar_wait_bounded(&bar[S], 0, wait))) {
        if (threadIdx.x == 0) mbar_wait_bounded(&bar[S], 0);
        bulk_give_up(bar, 0, nch, S, status);
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    for (int c = 0; c < nch; ++c) {
        const int st = c % S;
        const bool ok = mbar_wait_bounded(&bar[st], (c / S) & 1, wait);
        if (!__syncthreads_and(ok)) {
            bulk_give_up(bar, c, nch, S, status);
            return;
        }
        const cpx<T>* fst = ring + st * stage;
        const int cnt = min(G, nb - c * G);
        for (int t = warp; t < cnt * R; t += nwarp) {
            const int i = t / R, r = t - i * R;
            const cpx<T>* f = fst + (int64_t)i * row;
            const cpx<T>* rx = f + half;
            // stored directions and their antipodes accumulate separately (two independent chains)
            cpx<T> sJ = czero<T>(), sM = czero<T>(), aJ = czero<T>(), aM = czero<T>();
            for (int kk = lane; kk < Kh; kk += 32) {
                cpx<T> Ft, Fp, Xt, Xp, Vt, Vp, Wt, Wp;
                lds_pair(f + 2 * kk, Ft, Fp);
                lds_pair(rx + 2 * kk, Xt, Xp);
                const int ka = ap[kk];
                if (R1) {
                    lds_pair(vs + 2 * kk, Vt, Vp);
                    lds_pair(vs + 2 * ka, Wt, Wp);
                } else {
                    Vt = vs[kk * E + r], Vp = vs[kk * E + R + r];
                    Wt = vs[ka * E + r], Wp = vs[ka * E + R + r];
                }
                recv_pair<T, MODE>(Ft, Fp, Xt, Xp, Vt, Vp, Wt, Wp, sJ, sM, aJ, aM);
            }
            sJ = warp_sum(cadd(sJ, aJ));
            if (MODE == 0) sM = warp_sum(cadd(sM, aM));
            if (lane == 0) {
                const int m = n0 + c * G + i, u = perm[m];
                if (MODE == 0) {
                    y[(int64_t)r * nun + u] = cadd(yt[((int64_t)m * 2 + 0) * R + r], cscale(sJ, -cc));
                    y[(int64_t)r * nun + N + u] = cadd(yt[((int64_t)m * 2 + 1) * R + r], cscale(sM, cc));
                } else {
                    y[(int64_t)r * nun + u] = cadd(yt[(int64_t)m * R + r], cscale(sJ, -cc));
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && c + S < nch) {
            const int cn = c + S, cnt2 = min(G, nb - cn * G);
            const uint32_t bytes = (uint32_t)(cnt2 * row * sizeof(cpx<T>));
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[st], 2 * bytes);
            bulk_copy_g2s(ring + st * stage, F + (n0 + (int64_t)cn * G) * row, bytes, &bar[st]);
            bulk_copy_g2s(ring + st * stage + half, RX + (n0 + (int64_t)cn * G) * row, bytes, &bar[st]);
        }
    }
}

constexpr size_t kStageBytes = 16 * 1024;  // target bytes of one ring stage
constexpr int kStages = 3;

template <typename T, int MODE, int SL>
void launch_aggregate(bi_handle_s* h, const cpx<T>* x, int R, int threads, int G, size_t smem, cudaStream_t s) {
    const level_t& L = h->lev[h->leaf];
    auto kern = k_aggregate_bulk<T, MODE, SL>;
    bi_raise_smem(kern, smem);
    kern<<<L.nbox, threads, smem, s>>>(h->N, L.K, L.nph, R, h->nun, G, kStages, h->d_perm, h->d_leaf_start,
                                       h->d_leaf_order, (const cpx<T>*)h->d_F, x, (cpx<T>*)L.d_U, h->d_status,
                                       h->wait_cycles);
    CU(cudaGetLastError());
}

template <typename T>
bool aggregate_bulk(bi_handle_s* h, const void* xv, int R, cudaStream_t s) {
    const level_t& L = h->lev[h->leaf];
    const int Kh = L.K / 2;
    const int slots = Kh * R;
    const int threads = std::min(256, (slots + 31) / 32 * 32);
    const int sl = (slots + threads - 1) / threads;
    const size_t rowb = (size_t)Kh * 2 * sizeof(cpx<T>);
    const int G = (int)std::max<size_t>(1, std::min<size_t>(h->max_leaf_count, kStageBytes / rowb));
    const size_t smem = kBarBytes + (size_t)kStages * G * rowb + (size_t)h->max_leaf_count * 2 * R * sizeof(cpx<T>);
    if (smem > 200 * 1024 || sl > 8) return false;
    const cpx<T>* x = (const cpx<T>*)xv;
    const int S1 = sl <= 1 ? 1 : sl <= 2 ? 2 : sl <= 4 ? 4 : 8;
    if (h->prm.op_mode == 0) {
        if (S1 == 1) launch_aggregate<T, 0, 1>(h, x, R, threads, G, smem, s);
        else if (S1 == 2) launch_aggregate<T, 0, 2>(h, x, R, threads, G, smem, s);
        else if (S1 == 4) launch_aggregate<T, 0, 4>(h, x, R, threads, G, smem, s);
        else launch_aggregate<T, 0, 8>(h, x, R, threads, G, smem, s);
    } else {
        if (S1 == 1) launch_aggregate<T, 1, 1>(h, x, R, threads, G, smem, s);
        else if (S1 == 2) launch_aggregate<T, 1, 2>(h, x, R, threads, G, smem, s);
        else if (S1 == 4) launch_aggregate<T, 1, 4>(h, x, R, threads, G, smem, s);
        else launch_aggregate<T, 1, 8>(h, x, R, threads, G, smem, s);
    }
    return true;
}

template <typename T>
bool receive_bulk(bi_handle_s* h, void* yv, int R, cudaStream_t s) {
    const level_t& L = h->lev[h->leaf];
    const int Kh = L.K / 2, E = 2 * R;
    const size_t rowb = (size_t)Kh * 2 * sizeof(cpx<T>);
    // 8 warps, one RWG each per stage; two stages
    const int S = 2;
    const int G = (int)std::max<size_t>(1, std::min<size_t>(h->max_leaf_count, (2 * kStageBytes) / (2 * rowb)));
    const size_t smem = kBarBytes + (size_t)L.K * E * sizeof(cpx<T>) + (size_t)S * G * 2 * rowb + (size_t)Kh * sizeof(int);
    if (smem > 200 * 1024) return false;
    const double pi = 3.14159265358979323846;
    const T cc = (T)(h->k * h->k / (32.0 * pi * pi));
    auto kern = h->prm.op_mode == 0 ? (R == 1 ? k_receive_bulk<T, 0, 1> : k_receive_bulk<T, 0, 0>)
                                    : (R == 1 ? k_receive_bulk<T, 1, 1> : k_receive_bulk<T, 1, 0>);
    bi_raise_smem(kern, smem);
    kern<<<L.nbox, 256, smem, s>>>(h->N, L.K, L.nph, R, h->nun, G, S, h->d_perm, h->d_leaf_start, h->d_leaf_order,
                                   (const cpx<T>*)h->d_F, (const cpx<T>*)h->d_RX, (const cpx<T>*)L.d_V, cc,
                                   (const cpx<T>*)h->d_yt, (cpx<T>*)yv, h->d_status, h->wait_cycles);
    CU(cudaGetLastError());
    return true;
}

}  // namespace

bool bi_leaf_aggregate_bulk(bi_handle_s* h, const void* x, int R, cudaStream_t s) {
    if (!h->use_leaf_bulk || h->leaf < 2) return false;
    return h->prec == 0 ? aggregate_bulk<double>(h, x, R, s) : aggregate_bulk<float>(h, x, R, s);
}

bool bi_leaf_receive_bulk(bi_handle_s* h, void* y, int R, cudaStream_t s) {
    if (!h->use_leaf_bulk || h->leaf < 2) return false;
    return h->prec == 0 ? receive_bulk<double>(h, y, R, s) : receive_bulk<float>(h, y, R, s);
}
