// Far field of the equivalent currents (Eq. 22a in the far zone), for the RCS of
// Sec. III (Eq. 5-25):
//   F(rhat) = -jk/(4 pi) [ (I - rhat rhat) N_J - rhat x N_M ],
//   N_X(rhat) = sum_n x_X,n int f_n(r') exp(+jk rhat.r') ds',
// so that E_sca ~ exp(-jkr)/r F(rhat) and sigma = 4 pi |F|^2 for a unit incident field.
// Two passes: per-CTA partial sums of N_J, N_M over a chunk of RWG functions (written to
// scratch memory), then one thread per (rhs, direction) adds the chunks and projects.
#include <cmath>

#include <cuda.h>
#include <mutex>

#include "bi_internal.h"

namespace {

constexpr int kFFChunk = 256;   // RWG functions per CTA of the first pass

template <typename TX>
__global__ void __launch_bounds__(kFFChunk) k_farfield_partial(int N, int nX, int nun, int ndir,
                                                               const int* __restrict__ perm, const int* __restrict__ rwg_t,
                                                               const int* __restrict__ rwg_l,
                                                               const double* __restrict__ rwg_len,
                                                               const double* __restrict__ tri,
                                                               const double* __restrict__ area, double k,
                                                               const TX* __restrict__ x, const double* __restrict__ dirs,
                                                               double* __restrict__ part) {
    const int chunk = blockIdx.x, d = blockIdx.y, r = blockIdx.z;
    const int t = chunk * kFFChunk + threadIdx.x;
    const double* rh = dirs + 3 * d;
    double acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = 0.0;
    if (t < N) {
        const int u = perm[t];
        const double xJr = (double)x[2 * ((int64_t)r * nun + u)], xJi = (double)x[2 * ((int64_t)r * nun + u) + 1];
        double xMr = 0, xMi = 0;
        if (nX == 2) {
            xMr = (double)x[2 * ((int64_t)r * nun + N + u)];
            xMi = (double)x[2 * ((int64_t)r * nun + N + u) + 1];
        }
        const double s15 = 3.872983346207417;
        const double a1 = (6.0 - s15) / 21.0, a2 = (6.0 + s15) / 21.0;
        for (int side = 0; side < 2; ++side) {
            const int tr = rwg_t[2 * t + side], l = rwg_l[2 * t + side];
            const double* P = tri + 9 * tr;
            const double cf = (side == 0 ? 1.0 : -1.0) * rwg_len[t] * 0.5;   // (l / 2A) * A
            for (int q = 0; q < 7; ++q) {
                double bb[3], w;
                if (q == 0) { bb[0] = bb[1] = bb[2] = 1.0 / 3.0; w = 9.0 / 40.0; }
                else {
                    const double a = (q <= 3) ? a1 : a2;
                    w = (q <= 3) ? (155.0 - s15) / 1200.0 : (155.0 + s15) / 1200.0;
                    bb[0] = bb[1] = bb[2] = a;
                    bb[(q - 1) % 3] = 1.0 - 2.0 * a;
                }
                double rr[3], f[3];
                for (int c = 0; c < 3; ++c) {
                    rr[c] = bb[0] * P[c] + bb[1] * P[3 + c] + bb[2] * P[6 + c];
                    f[c] = cf * w * (rr[c] - P[3 * l + c]);
                }
                double sn, cs;
                sincos(k * (rh[0] * rr[0] + rh[1] * rr[1] + rh[2] * rr[2]), &sn, &cs);
                // (xJ, xM) * exp(j ph) * f
                const double eJr = xJr * cs - xJi * sn, eJi = xJr * sn + xJi * cs;
                const double eMr = xMr * cs - xMi * sn, eMi = xMr * sn + xMi * cs;
                for (int c = 0; c < 3; ++c) {
                    acc[2 * c] += eJr * f[c];
                    acc[2 * c + 1] += eJi * f[c];
                    acc[6 + 2 * c] += eMr * f[c];
                    acc[6 + 2 * c + 1] += eMi * f[c];
                }
            }
        }
    }
    // block reduction: warp shuffles, then one value per warp in shared memory
    __shared__ double red[kFFChunk / 32][12];
#pragma unroll
    for (int i = 0; i < 12; ++i)
        for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int i = 0; i < 12; ++i) red[warp][i] = acc[i];
    __syncthreads();
    if (threadIdx.x < 12) {
        double s = 0.0;
        for (int w = 0; w < kFFChunk / 32; ++w) s += red[w][threadIdx.x];
        part[(((int64_t)chunk * gridDim.z + r) * ndir + d) * 12 + threadIdx.x] = s;
    }
}

__global__ void k_farfield_final(int nchunk, int nrhs, int ndir, double k, const double* __restrict__ dirs,
                                 const double* __restrict__ part, double* __restrict__ F) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrhs * ndir) return;
    const int r = i / ndir, d = i % ndir;
    double n[12];
    for (int c = 0; c < 12; ++c) n[c] = 0.0;
    for (int ch = 0; ch < nchunk; ++ch)
        for (int c = 0; c < 12; ++c) n[c] += part[(((int64_t)ch * nrhs + r) * ndir + d) * 12 + c];
    const double* rh = dirs + 3 * d;
    // v = (I - rr) N_J - rhat x N_M   (re and im separately)
    double v[6];
    for (int p = 0; p < 2; ++p) {
        const double J[3] = {n[0 + p], n[2 + p], n[4 + p]};
        const double M[3] = {n[6 + p], n[8 + p], n[10 + p]};
        const double rj = rh[0] * J[0] + rh[1] * J[1] + rh[2] * J[2];
        const double cr[3] = {rh[1] * M[2] - rh[2] * M[1], rh[2] * M[0] - rh[0] * M[2], rh[0] * M[1] - rh[1] * M[0]};
        for (int c = 0; c < 3; ++c) v[2 * c + p] = J[c] - rh[c] * rj - cr[c];
    }
    // F = (-jk / 4 pi) v
    const double s = k / (4.0 * 3.14159265358979323846);
    for (int c = 0; c < 3; ++c) {
        F[2 * ((int64_t)i * 3 + c)] = s * v[2 * c + 1];
        F[2 * ((int64_t)i * 3 + c) + 1] = -s * v[2 * c];
    }
}

}  // namespace

size_t bi_farfield_scratch_bytes(const bi_handle_s* h, int nrhs, int ndir) {
    const int nchunk = (h->N + kFFChunk - 1) / kFFChunk;
    return (size_t)nchunk * nrhs * ndir * 12 * sizeof(double);
}

// Both passes on stream s with `part` as scratch (bi_farfield_scratch_bytes(h, nrhs, ndir) bytes).
void bi_farfield_launch(bi_handle_s* h, const void* x, int nrhs, const double* dirs, int ndir, void* F, double* part,
                        cudaStream_t s) {
    const int nchunk = (h->N + kFFChunk - 1) / kFFChunk;
    dim3 g(nchunk, ndir, nrhs);
    if (h->prec == 0)
        k_farfield_partial<double><<<g, kFFChunk, 0, s>>>(h->N, h->nX, h->nun, ndir, h->d_perm, h->d_rwg_t, h->d_rwg_l,
                                                          h->d_rwg_len, h->d_tri, h->d_tri_area, h->k,
                                                          (const double*)x, dirs, part);
    else
        k_farfield_partial<float><<<g, kFFChunk, 0, s>>>(h->N, h->nX, h->nun, ndir, h->d_perm, h->d_rwg_t, h->d_rwg_l,
                                                         h->d_rwg_len, h->d_tri, h->d_tri_area, h->k,
                                                         (const float*)x, dirs, part);
    CU(cudaGetLastError());
    const int tot = nrhs * ndir;
    k_farfield_final<<<(tot + 127) / 128, 128, 0, s>>>(nchunk, nrhs, ndir, h->k, dirs, part, (double*)F);
    CU(cudaGetLastError());
}

// ---------------------------------------------------------------------------------
// Allocation-free variant of bi_farfield.  The first-pass partial sums live in a fixed
// array compiled into the library instead of handle-owned scratch, so the call itself
// never allocates device memory.  Every GPU that loads the library holds this array until
// the process exits; all calls on one device share it.
static __device__ __align__(256) double g_ff_noalloc_scratch[BI_FARFIELD_NOALLOC_MAX_BYTES / sizeof(double)];

// Unique id of the calling thread's current CUDA context (0 when none or unknown), through
// the driver entry points the runtime hands out, so the library needs no link to libcuda.
static unsigned long long current_context_id() {
    typedef CUresult (*get_current_t)(CUcontext*);
    typedef CUresult (*get_id_t)(CUcontext, unsigned long long*);
    static get_current_t get_current = nullptr;
    static get_id_t get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (get_current_t)p;
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (get_id_t)p;
        cudaGetLastError();
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS) return id;
    return 0;
}

extern "C" int bi_farfield_noalloc(bi_handle h, const void* x, int nrhs, const double* dirs, int ndir, void* F) {
    if (!h) return BI_ERR_ARG;
    if (h->coated) {
        h->err = "bi_farfield_noalloc: use bi_farfield for the coated body";
        return BI_ERR_ARG;
    }
    if (h->med[0]) return bi_farfield_noalloc(h->med[0], x, nrhs, dirs, ndir, F);   // two-region: the exterior
    if (!x || !dirs || !F || nrhs < 1 || ndir < 1 || nrhs > 65535 || ndir > 65535) {
        h->err = "bi_farfield_noalloc: null argument or nrhs/ndir outside [1, 65535]";
        return BI_ERR_ARG;
    }
    if (h->ki != 0.0) {
        h->err = "bi_farfield_noalloc: the handle's medium is lossy (k_im != 0); a far field exists in free space only";
        return BI_ERR_ARG;
    }
    const size_t need = bi_farfield_scratch_bytes(h, nrhs, ndir);
    if (need > (size_t)BI_FARFIELD_NOALLOC_MAX_BYTES) {
        h->err = "bi_farfield_noalloc: needs " + std::to_string(need) + " B of scratch, more than the fixed " +
                 std::to_string((size_t)BI_FARFIELD_NOALLOC_MAX_BYTES) +
                 " B; use fewer directions or right-hand sides per call, or bi_farfield";
        return BI_ERR_ARG;
    }
    try {
        int dev = 0;
        CU(cudaGetDevice(&dev));
        if (dev != h->device) {
            // the array's address is per device: on another device it would name memory the
            // handle's stream cannot use
            h->err = "bi_farfield_noalloc: the current device (" + std::to_string(dev) +
                     ") is not the handle's device (" + std::to_string(h->device) + "); make it current first";
            return BI_ERR_ARG;
        }
        const unsigned long long ctx = current_context_id();
        if (!h->ff_noalloc_part || ctx != h->ff_noalloc_ctx || ctx == 0) {
            // Host code cannot use the array's name as an address: look the address up with the
            // handle's device current, and again whenever the current context is not the one the
            // kept address belongs to (a context destroyed and recreated, e.g. after
            // cudaDeviceReset, places the array anew; an unknown context is never trusted).
            void* p = nullptr;
            CU(cudaGetSymbolAddress(&p, g_ff_noalloc_scratch));
            h->ff_noalloc_part = (double*)p;
            h->ff_noalloc_ctx = ctx;
        }
        // every partial-sum slot used by this call is written by the first pass before the
        // second pass reads it, so nothing needs clearing
        bi_farfield_launch(h, x, nrhs, dirs, ndir, F, h->ff_noalloc_part, h->stream);
        return BI_OK;
    } catch (const bi_error& e) {
        h->err = e.msg;
        return e.code;
    } catch (const std::exception& e) {
        h->err = std::string("host: ") + e.what();
        return BI_ERR_OOM;
    }
}
