// Internal data structures of the GB300 boundary-integral operator.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "bi.h"

#define BI_MAXLEV 24
#define BI_NSTAGES 8

// Status propagation: every CUDA call is checked, and a failure becomes BI_ERR_CUDA
// with the call text in the handle's error string.
struct bi_error {
    int code;
    std::string msg;
};

#define CU(call)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            throw bi_error{e_ == cudaErrorMemoryAllocation ? BI_ERR_OOM : BI_ERR_CUDA,                 \
                           std::string(#call) + ": " + cudaGetErrorString(e_)};                        \
    } while (0)

// Raise (never lower) a kernel's dynamic shared-memory limit on the current device.  The
// limit belongs to the function, not to one launch: products captured into graphs earlier (by
// this or another handle) keep their larger sizes, so a later, smaller request must not
// lower it.  Sizes up to the 48 KB default need no call.
void bi_raise_smem_limit(const void* func, size_t bytes);
template <typename F>
inline void bi_raise_smem(F* func, size_t bytes) {
    bi_raise_smem_limit(reinterpret_cast<const void*>(func), bytes);
}

// Device pointer with a host-side size, freed by the handle.
struct dbuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// One level of the octree.
struct level_t {
    int nbox = 0;
    double a = 0;                       // box edge
    std::vector<int> coords;            // [nbox][3]
    std::vector<double> center;         // [nbox][3]
    std::vector<uint64_t> key;          // Morton key at this level, sorted
    std::vector<int> parent;            // index in level-1
    std::vector<int> child_ptr;         // CSR into level+1 (children contiguous)
    // far-field sampling (levels >= 2 when the leaf is >= 2)
    int L = 0, nth = 0, nph = 0, K = 0;
    std::vector<double> theta, wtheta;  // [nth], theta ascending, Gauss-Legendre in cos(theta)
    // interaction list (levels >= 2)
    std::vector<int> il_ptr, il_src, il_off;
    // device
    void* d_T = nullptr;                // translation operators [344][K] complex (weights folded; row 343 zero)
    int* d_il_ptr = nullptr;
    int* d_il_src = nullptr;
    int* d_il_off = nullptr;
    int* d_parent = nullptr;
    int* d_child_ptr = nullptr;
    int* d_octant = nullptr;            // octant of each box inside its parent
    int* d_child_order = nullptr;       // boxes ordered by (slot in parent, parent): siblings far apart in a grid
    void* d_shift = nullptr;            // [8][K] exp(+jk khat.(c_child - c_parent)) for parent level
    void* d_shift_dn = nullptr;         // [8][K] conj(exp(-jk khat.(c_child - c_parent))), read conjugated by the
                                        // downward pass; the same table as d_shift when k is real
    void* d_U = nullptr;                // outgoing patterns [nbox][K][E]
    void* d_V = nullptr;                // incoming patterns [nbox][K][E]
    int64_t n_inter = 0;
    // parent-centred interaction lists (translation level l, parents at l - 1): per parent its
    // children range, and per source box the offset codes to each child (0xFFFF: near or none)
    int tp_np = 0;
    std::vector<int> tp_ptr, tp_src;    // host copies of the lists below
    std::vector<unsigned short> tp_code;
    int* d_tp_cptr = nullptr;           // [np + 1] children of each parent (level-l indices)
    int* d_tp_ptr = nullptr;            // [np + 1] source entries of each parent
    int* d_tp_src = nullptr;            // [entries] source box
    void* d_tp_code = nullptr;          // [entries][8] uint16 offset code per child slot
};

// Lagrange interpolation between level l+1 (child) and level l (parent).
struct interp_t {
    int p_th = 0, p_ph = 0;
    // forward theta pass: for every parent theta, p_th taps (child theta index, flip, weight)
    std::vector<int> th_src, th_flip;
    std::vector<double> th_w;
    // forward phi pass: for every parent phi, p_ph taps (child phi index, weight)
    std::vector<int> ph_src;
    std::vector<double> ph_w;
    // transposed (anterpolation) lists
    std::vector<int> tth_ptr, tth_dst, tth_flip;   // per child theta: parent thetas
    std::vector<double> tth_w;
    std::vector<int> tph_ptr, tph_dst;             // per child phi: parent phis
    std::vector<double> tph_w;
    // device copies (weights stored in the handle precision)
    int *d_th_src = nullptr, *d_th_flip = nullptr, *d_ph_src = nullptr;
    void *d_th_w = nullptr, *d_ph_w = nullptr;
    int *d_tth_ptr = nullptr, *d_tth_dst = nullptr, *d_tth_flip = nullptr, *d_tph_ptr = nullptr, *d_tph_dst = nullptr;
    void *d_tth_w = nullptr, *d_tph_w = nullptr;
    void* d_tmp = nullptr;              // per child box: [nbox_child][nth_parent][nph_child][E]
    // packed taps (index, weight in the handle precision) for the unrolled kernels:
    //   th_tap [nth_parent][p_th]: code = child row * 2 + flip, weight with the flip sign folded
    //   ph_tap [nph_parent][p_ph]: child column
    //   tth_pad [nth_child][pt_th]: code = parent row * 2 + flip (zero-padded lists)
    //   tph_pad [nph_child][pt_ph]: parent column (zero-padded lists)
    int pt_th = 0, pt_ph = 0;
    void *d_th_tap = nullptr, *d_ph_tap = nullptr, *d_tth_pad = nullptr, *d_tph_pad = nullptr;
};

struct bi_handle_s {
    bi_params prm{};
    double k = 0;     // Re k: sets the sampling and the box sizes in wavelengths
    double ki = 0;    // Im k (<= 0: a lossy medium; 0: free space)
    // one medium of the two-region form (op_mode 3): y_E = a L x_J - K x_M, y_H = K x_J + b L x_M
    double pa[2] = {1.0, 0.0}, pb[2] = {1.0, 0.0};
    int nF = 1;       // transverse fields per box and direction: 1, or 2 (op_mode 3: E and H)
    // the two-region operator (op_mode 2): one handle per medium, products summed
    bi_handle_s* med[2] = {nullptr, nullptr};
    void* d_ysum = nullptr;             // [max_rhs][nun] the second medium's product
    // Autotuned kernel forms of the level passes, per (pass, level, E): pass 0 translation
    // (1 or 2 pairs of entries per thread), 1 interpolation (100 + EC: chunked; 2: two-pass),
    // 2 anterpolation (100 + EC: per child; 200 + EC: row blocks; 2: two-pass); 0 = the built-in
    // choice.  Filled by the first product with a given nrhs (bi_autotune) and reported by
    // bi_tuned_config.
    struct tune_entry {
        int pass, level, E, variant;
        double us;
    };
    std::vector<tune_entry> tuned;
    std::vector<int> tuned_E;           // E values already tuned
    bool autotune = true;
    int variant_of(int pass, int level, int E) const {
        for (const tune_entry& t : tuned)
            if (t.pass == pass && t.level == level && t.E == E) return t.variant;
        return 0;
    }
    int force_variant = -1;             // set by the tuner while it times one candidate
    // the coated PEC body (op_mode 4): med[0] = free space on the outer surface (N1 RWG),
    // med[1] = the coat on both surfaces (N1 + N2 RWG); unknowns [J1, M1, J2]
    int coated = 0, N1 = 0, N2 = 0;
    void *d_xin0 = nullptr, *d_xin1 = nullptr, *d_y0 = nullptr, *d_y1 = nullptr;
    int N = 0, nt = 0, nv = 0;
    int nun = 0;      // unknowns
    int nX = 2;       // currents per RWG (2 for op_mode 0, 1 for op_mode 1)
    int prec = 1;     // 0 double, 1 float
    size_t csize = 8; // bytes of one complex
    std::string err;
    bi_info_t info{};

    cudaStream_t stream = nullptr;      // user stream (not owned)
    cudaStream_t side = nullptr;        // owned: near field runs here concurrently with the far field
    cudaStream_t cap = nullptr;         // owned: graph capture origin
    cudaStream_t tstream[BI_MAXLEV] = {};   // owned: translations of level l (l >= 3)
    cudaEvent_t ev_tfork[BI_MAXLEV] = {}, ev_tjoin[BI_MAXLEV] = {};
    bool use_graphs = true;
    bool use_fast = true;               // fused kernels (false: two-pass reference kernels)
    bool use_leaf_bulk = true;          // bulk-copy pipelines for leaf aggregation and receive
    int interp_variant = 0, anterp_variant = 0;   // level-pass forms forced on every level (test
                                                  // switches BI_INTERP_VARIANT, BI_ANTERP_VARIANT)
    int translate_variant = 0;          // translation kernel form forced on every level (test switch
                                        // BI_TRANSLATE_VARIANT=1..9; 0: tuned)
    int near_rb = 2;                    // near kernel for 3 <= R <= 8: 2 row pairs with cp.async-pipelined
                                        // block entries (FP32 C block, 6-8 RHS; else 1), 1 row pairs,
                                        // 0 per-row (switch BI_NEAR_RB)
    bool force_anterp_rows = false;     // row-blocked anterpolation on every level (test switch)
    int* d_status = nullptr;            // device status word (0: healthy; see bi_tma.cuh)
    long long wait_cycles = 1ll << 31;  // limit of the bulk-copy waits of the leaf kernels (SM clocks)
    void* d_sai = nullptr;              // near-field SAI blocks, one dense [n_b][n_b] per leaf box (precond 1)
    struct coupling_t {                 // Eq. 52 coupling (caller-owned CSR arrays and Q^{-1} solver)
        int64_t n_int = 0;
        const int *lx_ptr = nullptr, *lx_col = nullptr, *xl_ptr = nullptr, *xl_col = nullptr;
        const void *lx_val = nullptr, *xl_val = nullptr;
        bi_qsolve_fn qsolve = nullptr;
        void* user = nullptr;
        void *t1 = nullptr, *t2 = nullptr;   // work: D^{Lambda X} x, Q^{-1} of it
    } cpl;
    int64_t* sai_off = nullptr;         // [nbox + 1] offsets of the blocks (complex entries)
    int near_ncol_max = 0;
    int near_nwork = 0;                 // work items of the streaming near kernel (box, first row)
    int* d_near_work = nullptr;
    int* d_near_col0 = nullptr;         // per near entry: first column in the test box's segment
    int* d_near_ncol = nullptr;         // per leaf box: segment width (near columns)
    int num_sms = 152;
    int device = -1;                    // CUDA device current at bi_setup (the handle's buffers live there)
    double* ff_noalloc_part = nullptr;  // device address of the allocation-free far-field array on that device
    unsigned long long ff_noalloc_ctx = 0;  // id of the CUDA context that address belongs to
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

    // host mesh / RWG in user order
    std::vector<int> edges;             // [N][2]
    std::vector<int> tplus, tminus, lplus, lminus;
    std::vector<int> tri_vid_host;      // [nt][3] copy of the mesh triangles
    double margin = 0.0;                // bandwidth margin: twice the largest RWG overhang
    std::vector<double> tri_host, tri_n_host, tri_area_host, rwg_len_user;
    double* d_leaf_center = nullptr;    // [nbox_leaf][3]
    // tree order
    std::vector<int> perm;              // tree index -> user index
    int nlev = 0, leaf = 0;
    std::vector<level_t> lev;
    std::vector<interp_t> itp;          // itp[l] maps level l+1 -> l
    std::vector<int> leaf_start;        // [nbox_leaf + 1]
    int max_leaf_count = 0;
    int64_t near_nnz = 0;
    std::vector<int> near_ptr, near_src;  // per leaf box: near source boxes
    std::vector<int64_t> near_blk;        // block offset per (box, near index)

    // device data
    std::vector<dbuf> owned;
    int* d_perm = nullptr;
    int* d_leaf_start = nullptr;
    int* d_leaf_of = nullptr;           // leaf box of each tree RWG
    int* d_leaf_order = nullptr;        // leaf boxes by decreasing RWG count (launch order of per-box CTAs)
    int* d_near_ptr = nullptr;
    int* d_near_src = nullptr;
    int64_t* d_near_blk = nullptr;
    void* d_near = nullptr;             // near blocks: per pair (A, B) complex (mode 0) or A (mode 1)
    int* d_gram_ptr = nullptr;          // mode 0: Gram correction per tree row
    int* d_gram_col = nullptr;
    int* d_gram_seg = nullptr;          // column of the neighbour in the test box's near segment
    void* d_gram_val = nullptr;         // [nnz][2] real: (G, X)
    void* d_F = nullptr;                // leaf radiation patterns [N][K/2][2] (one direction of each antipodal pair)
    void* d_RX = nullptr;               // leaf twisted receive patterns [N][K/2][2]
    // geometry on device (tree order for RWG data)
    double* d_tri = nullptr;            // [nt][9]
    double* d_tri_n = nullptr;          // [nt][3]
    double* d_tri_area = nullptr;       // [nt]
    int* d_tri_vid = nullptr;           // [nt][3]
    int* d_rwg_t = nullptr;             // tree order [N][2] (T+, T-)
    int* d_rwg_l = nullptr;             // tree order [N][2] local free vertex
    double* d_rwg_len = nullptr;        // tree order [N]
    // work buffers
    int max_rhs = 1;
    void* d_xt = nullptr;               // [N][nX][R]
    void* d_yt = nullptr;               // [N][nX][R]
    void* d_yfar = nullptr;             // [N][nX][R]
    void* d_sx = nullptr;               // staging [R][nun] (host API and GMRES matvec input)
    void* d_sy = nullptr;               // staging [R][nun] (output)
    void* d_ffscratch = nullptr;        // far-field partial sums (grown on demand)
    size_t ffscratch_bytes = 0;
    void* h_pinned = nullptr;           // pinned host staging
    size_t h_pinned_bytes = 0;

    // CUDA graph of one matvec per nrhs value (captured lazily)
    struct graph_entry {
        int nrhs;
        const void* x;
        void* y;
        cudaGraphExec_t exec;
    };
    std::vector<graph_entry> graphs;

    void* alloc(size_t bytes);
    template <typename T>
    T* upload(const std::vector<T>& v) {
        if (v.empty()) return nullptr;
        T* p = (T*)alloc(sizeof(T) * v.size());
        CU(cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
        return p;
    }
};

// setup stages (host)
void bi_build_rwg(bi_handle_s* h, const double* V, int nv, const int* T, int nt);
void bi_build_tree(bi_handle_s* h, const double* V);
void bi_build_sampling(bi_handle_s* h);
void bi_build_interp(bi_handle_s* h);

// device stages
void bi_device_geometry(bi_handle_s* h, const double* V, const int* T);
void bi_fill_near(bi_handle_s* h);
void bi_fill_patterns(bi_handle_s* h);
void bi_fill_translations(bi_handle_s* h);
// Host part of the translation operators of level l: for each of the 343 offset codes the index
// of its distance |X| (-1 for touching offsets), and per distance h_n^(2)(k|X|), n = 0..L, as
// interleaved (re, im) pairs.
void bi_translation_series(const bi_handle_s* h, int l, std::vector<int>& dist_idx, std::vector<double>& hk);
void bi_alloc_work(bi_handle_s* h);
void bi_matvec_launch(bi_handle_s* h, const void* x, void* y, int nrhs, cudaStream_t s);
void bi_rhs_launch(bi_handle_s* h, const double* khat, const double* phat, int nrhs, void* b);
// coated body: the outer surface's currents [J1; M1] of x into d_xin0; the outer medium's
// right-hand sides (in d_y0) into b = [b_J1; b_M1; 0]
void bi_coated_outer_currents(bi_handle_s* h, const void* x, int R, cudaStream_t s);
void bi_coated_rhs(bi_handle_s* h, void* b, int R, cudaStream_t s);
void bi_profile_impl(bi_handle_s* h, const void* x, void* y, int nrhs, int reps, double* ms);
const char* bi_stage_name_impl(int i);
bool bi_leaf_aggregate_bulk(bi_handle_s* h, const void* x, int R, cudaStream_t s);
bool bi_interp_level(bi_handle_s* h, int l, int E, cudaStream_t s);
bool bi_anterp_level(bi_handle_s* h, int l, int E, cudaStream_t s);
void bi_upload_taps(bi_handle_s* h);
bool bi_translate_level(bi_handle_s* h, int l, int E, cudaStream_t s);
void bi_autotune(bi_handle_s* h, int nrhs, cudaStream_t s);
void bi_build_sai(bi_handle_s* h);
void bi_operator_launch(bi_handle_s* h, const void* x, void* y, int R, cudaStream_t s);
void bi_coupling_blocks_impl(bi_handle_s* h, int conforming, int64_t* sizes, int* xl_ptr, int* xl_col, void* xl_val,
                             int* lx_ptr, int* lx_col, void* lx_val);
void bi_coupling_set(bi_handle_s* h, int64_t n_int, const int* lx_ptr, const int* lx_col, const void* lx_val,
                     const int* xl_ptr, const int* xl_col, const void* xl_val, bi_qsolve_fn qsolve, void* user);
void bi_sai_apply(bi_handle_s* h, const void* x, void* y, int R, cudaStream_t s);
void bi_build_translate_lists(bi_handle_s* h);
void bi_plan_translate_lists(bi_handle_s* h);   // host part of bi_build_translate_lists
bool bi_params_valid(const bi_params& P);       // the parameter ranges bi_setup accepts
bool bi_leaf_receive_bulk(bi_handle_s* h, void* y, int R, cudaStream_t s);
int bi_take_device_status(bi_handle_s* h);
size_t bi_farfield_scratch_bytes(const bi_handle_s* h, int nrhs, int ndir);
void bi_farfield_launch(bi_handle_s* h, const void* x, int nrhs, const double* dirs, int ndir, void* F, double* part,
                        cudaStream_t s);
int bi_gmres(bi_handle_s* h, const void* rhs, void* x, int nrhs, double tol, int* iters, double* relres);
int bi_solve_refined_impl(bi_handle_s* h, bi_handle_s* href, const void* rhs, void* x, int R, double tol, int* iters,
                          double* relres);
// resumable GMRES (serving loop)
struct gmres_ctx;
// tol: host [nrhs], one tolerance per column (columns of different requests may share a context)
gmres_ctx* bi_gmres_create(bi_handle_s* h, const void* rhs, int nrhs, const double* tol, cudaStream_t s);
int bi_gmres_advance(gmres_ctx* c);
int bi_gmres_finish(gmres_ctx* c, void* xout, int* iters, double* relres);
void bi_gmres_destroy(gmres_ctx* c);
int64_t bi_gmres_bytes(gmres_ctx* c);
int64_t bi_gmres_estimate_bytes(int64_t nun, int R, int m);

// numerical helpers shared by the host setup files of the library (not by the oracle)
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);  // nodes in (-1, 1)
