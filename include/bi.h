/*
 * bi.h -- C-ABI of the GB300 boundary-integral operator library.
 *
 * The library applies the dense boundary-integral matrix C of the coupled HDG-BI
 * system (Sec. II.D, Eq. 42, lower-right block; entries Eqs. 43-46) to vectors of
 * RWG coefficients of the equivalent currents J and M on a closed triangulated
 * surface (Sec. II.B-C), accelerated by a multilevel fast multipole algorithm
 * (step 2(a) of the hybrid solver, Sec. II.E).  It also solves C X = b with a
 * device-resident GMRES (Sec. II.E, steps 2-3) and builds the plane-wave right-hand
 * sides of Eqs. 49-50.
 *
 * Conventions (fixed by the ABI):
 *   - Time dependence exp(j w t); G = exp(-j k0 R) / (4 pi R); fields normalised so
 *     that E and H carry the same amplitude (Sec. II.A).
 *   - Mesh: verts[nv][3] (float64, any length unit consistent with k0), tris[nt][3]
 *     (int32), counter-clockwise seen from outside.  Several disjoint closed
 *     components are allowed (Sec. II.F, comment 2).
 *   - RWG functions are the interior edges sorted by (min vertex, max vertex);
 *     f = (l / 2A+)(r - p+) on T+, (l / 2A-)(p- - r) on T-, where T+ is the
 *     triangle in which the edge runs from its smaller to its larger vertex.
 *   - Unknown vectors are column-major [nrhs][n_unknowns]: for op_mode 0 the J
 *     block (N entries) then the M block (N entries); for op_mode 1 only J.
 *   - Complex numbers are interleaved (re, im): complex128 for precision 0,
 *     complex64 for precision 1.
 *
 * Ownership: the caller owns every vector it passes (device memory for the
 * device entry points, host memory for *_host).  The handle owns all internal
 * device buffers.  A handle is used by one host thread at a time.
 *
 * Errors: every entry point returns a bi_status; nothing aborts.  bi_last_error()
 * gives a one-line description of the last failure on that handle.
 */
#ifndef BI_GB300_H
#define BI_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bi_handle_s* bi_handle;

typedef enum {
    BI_OK = 0,
    BI_ERR_ARG = -1,            /* invalid argument or size                          */
    BI_ERR_MESH = -2,           /* open/non-manifold edge, flipped or degenerate tri */
    BI_ERR_OOM = -3,            /* device allocation failed                          */
    BI_ERR_CUDA = -4,           /* a CUDA call failed                                */
    BI_ERR_NOT_CONVERGED = -5,  /* GMRES stopped before tol; best iterate returned   */
    BI_ERR_TIMEOUT = -6,        /* a bounded device wait gave up                     */
    BI_ERR_BUSY = -7            /* serving queue full                                */
} bi_status;

typedef enum { BI_PREC_FP64 = 0, BI_PREC_FP32 = 1 } bi_precision;

/* op_mode 2: a homogeneous penetrable body of relative permittivity eps_r = eps_re + j eps_im
 * (mu_r = 1) in free space, by the surface-only two-region (PMCHWT) equations -- tangential E
 * and H continuous across the surface (the check the paper's Mie comparisons of Sec. III.A need
 * without the HDG interior):
 *     [ L0 + eta L1        -(K0 + K1)     ] [J]      L_i = <f_m, L f_n>, K_i = <f_m, Kbar f_n>
 *     [ K0 + K1        L0 + L1 / eta      ] [M]      in medium i (k1 = k0 sqrt(eps_r), eta = 1/sqrt(eps_r)),
 *   2N unknowns (J then M: the exterior equivalent currents).  Each medium gets its own
 *   octree, sampling and near field; the two products are summed.  Right-hand sides of
 *   bi_rhs_planewave are [-<f, E_inc>; -<f, H_inc>]; bi_farfield radiates J, M into free space.
 *   precond must be 0 and k_im 0; bi_set_coupling is not available.
 * op_mode 0: the C block of Eq. 42 (2N unknowns):
 *     [ G - P     X/2 - Q ] [J]      G = <f_m, f_n>, X = <f_m, n x f_n>,
 *     [   Q       G/2 - P ] [M]      P = <f_m, C f_n>, Q = <f_m, n x C f_n>,
 *   with C = 1/2 pi_tau L + 1/2 pi_x Kbar (Eq. 27, alpha = 1/2).
 * op_mode 1: PEC combined-field equation (Eqs. 24a/24b with M = 0, alpha = 1/2):
 *     G/4 - P  (N unknowns). */
/* op_mode 4: a PEC core under a coat of relative permittivity eps_r (the coated sphere of
 *   Sec. III.A, without the HDG interior): the mesh holds two closed surfaces, the coat's outer
 *   surface S1 (the first nt - core_tris triangles) and the core S2 (the last core_tris), every
 *   vertex of S1 numbered before every vertex of S2 (so the RWG functions of S1 come first).
 *   Unknowns [J1, M1, J2] (2 N1 + N2): the exterior currents on S1 and J2 = n2 x H on the core
 *   (n2 out of the core).  Rows: tangential E and H matched on S1, tangential E = 0 on S2:
 *     [ L0 + eta L1_11      -(K0 + K1_11)       -eta L1_12 ]
 *     [ K0 + K1_11         L0 + L1_11 / eta     -K1_12     ]
 *     [ -eta L1_21          K1_21               eta L1_22  ]
 *   with the free-space operators on S1 and the coat's on both surfaces.  Right-hand sides and
 *   far fields as for op_mode 2 (zero on the core's rows). */
typedef enum { BI_MODE_CBLOCK = 0, BI_MODE_PEC = 1, BI_MODE_TWO_REGION = 2, BI_MODE_COATED_PEC = 4 } bi_op_mode;

typedef struct {
    int digits;             /* MLFMA accuracy digits d0 in the excess-bandwidth rule (default 3) */
    double leaf_box;        /* leaf box edge in wavelengths 2 pi / k0 (default 0.25) */
    int levels;             /* octree levels including the root; 0 = smallest root that holds the mesh */
    int interp_order;       /* Lagrange points per angular dimension between levels (default 10) */
    int precision;          /* bi_precision (default BI_PREC_FP32) */
    int op_mode;            /* bi_op_mode (default BI_MODE_CBLOCK) */
    int max_rhs;            /* largest nrhs of one bi_matvec call; sizes the workspace (default 1) */
    int gmres_restart;      /* GMRES(m) restart length (default 100) */
    int gmres_maxit;        /* total GMRES iterations per right-hand side (default 1000) */
    void* stream;           /* cudaStream_t for all work of this handle; NULL = legacy default stream */
    int precond;            /* bi_solve preconditioner: 0 none (default); 1 sparse approximate inverse
                               from the near field only (Sec. III.B), a right preconditioner that is
                               block-diagonal over leaf boxes, M_b = argmin ||A(N,T) M_b - I(N,T)||_F
                               with T the box's unknowns and N those of its near boxes; built at
                               bi_setup, used by bi_solve and the server, never by bi_matvec */
    double k_im;            /* imaginary part of the wavenumber, k = k0 + j k_im (default 0).  A lossy
                               medium (with exp(j w t), -k0 <= k_im < 0; Sec. III.D's coating) takes
                               the same integrals and expansions continued to complex k: sampling and
                               box sizes follow Re k, the leaf patterns are stored for every direction
                               (R_n is no longer conj F_n), the translation operators use spherical
                               Hankel functions of complex argument, and the near field is integrated
                               in FP64 throughout.  bi_rhs_planewave, bi_farfield(_noalloc) and the
                               server take free-space handles only (BI_ERR_ARG otherwise). */
    double eps_re, eps_im;  /* op_mode 2, 4: relative permittivity of the body or coat (default 1, 0); eps_im <= 0 */
    int core_tris;          /* op_mode 4: triangles of the PEC core (the last ones of the mesh) */
} bi_params;

typedef struct {
    int64_t n_rwg;              /* N */
    int64_t n_unknowns;         /* 2N (op_mode 0) or N (op_mode 1) */
    int levels;                 /* including the root */
    int leaf_level;             /* levels - 1 */
    int boxes[32];              /* non-empty boxes per level */
    int L[32];                  /* multipole truncation per level (0 where no far field) */
    int K[32];                  /* directions per level, 2 (L+1)^2 */
    int64_t near_pairs;         /* RWG pairs stored in the near-field block matrix */
    int64_t interactions[32];   /* box-to-box translations per level */
    int64_t device_bytes;       /* device memory held by the handle */
    double root_size;           /* root box edge */
    double setup_ms;            /* wall time of bi_setup */
    double setup_near_regular_ms;   /* near-field fill: separated triangle pairs (FP32) */
    double setup_near_special_ms;   /* near-field fill: singular / near-singular pairs (FP64) */
    int64_t near_special_entries;   /* triangle pairs of the near field integrated in FP64 (singular / near-singular) */
    double setup_sai_ms;            /* set-up time of the preconditioner (0 without) */
} bi_info_t;

/* Fill *p with the defaults listed above. */
void bi_default_params(bi_params* p);

/* Build the operator for mesh (verts, tris) at wavenumber k0 (Sec. II.B-D):
 * validates the mesh, builds RWG functions, the octree, the near-field block matrix
 * (singular Galerkin integrals in FP64 on the device), leaf radiation/receive
 * patterns, translation operators and interpolation tables.
 * verts, tris: host arrays.  digits overrides opt->digits when > 0.  opt may be NULL.
 * Returns BI_ERR_MESH for an invalid surface, BI_ERR_OOM / BI_ERR_CUDA on device
 * failure; *out is NULL on failure. */
int bi_setup(const double* verts, int nv, const int* tris, int nt, double k0, int digits,
             const bi_params* opt, bi_handle* out);

/* N (RWG count) and the unknown count of the handle's op_mode. */
int bi_num_unknowns(bi_handle h, int64_t* n_rwg, int64_t* n_unknowns);

/* RWG order of the ABI: edge_vertex_pairs[N][2] (host) = (min vertex, max vertex). */
int bi_rwg_edges(bi_handle h, int* edge_vertex_pairs);

/* Sizes and timings of the built operator (host struct). */
int bi_get_info(bi_handle h, bi_info_t* info);

/* y = C x for nrhs column vectors (step 2(a) of Sec. II.E).  x, y: device pointers,
 * column-major [nrhs][n_unknowns], complex of the handle's precision; x and y must
 * not overlap.  1 <= nrhs <= max_rhs.  Work is queued on the handle's stream and
 * the call returns without synchronising. */
int bi_matvec(bi_handle h, const void* x, void* y, int nrhs);

/* Same product with host buffers: copies x to the device, multiplies, copies y back
 * and synchronises the stream before returning. */
int bi_matvec_host(bi_handle h, const void* x, void* y, int nrhs);

/* Plane-wave right-hand sides of Eqs. 49-50 (op_mode 0) or the PEC combined-field
 * right-hand side <f, E/2 + n x H/2> (op_mode 1), for E = phat exp(-j k0 khat.r),
 * H = (khat x phat) exp(-j k0 khat.r) (Sec. III).  khat, phat: host [nrhs][3] unit
 * vectors.  b: device, column-major [nrhs][n_unknowns], handle precision. */
int bi_rhs_planewave(bi_handle h, const double* khat, const double* phat, int nrhs, void* b);

/* Solve C x = rhs for nrhs right-hand sides with restarted GMRES (Saad and Schultz
 * 1986; Sec. II.E), x0 = 0, stopping when ||rhs - C x|| / ||rhs|| <= tol for every
 * column or at gmres_maxit iterations.  rhs, x: device, column-major [nrhs][n_unknowns].
 * iters, relres: host arrays [nrhs] (may be NULL).  Returns BI_ERR_NOT_CONVERGED when a
 * column missed tol (x holds the last iterate). */
int bi_solve(bi_handle h, const void* rhs, void* x, int nrhs, double tol, int* iters, double* relres);

/* Mixed-precision iterative refinement of C x = rhs (Sec. II.E's GMRES, no counterpart in the
 * paper for the precision split): each step solves C d = r with h's GMRES to 1e-3 of r (h
 * normally FP32), adds d to x in FP64, and recomputes r = rhs - C x with the FP64 handle h_ref
 * of the same surface, wavenumber and operator mode; it stops when ||r|| / ||rhs|| <= tol for
 * every column or after 20 steps.  Reaches tolerances below the working product's rounding floor
 * (about 1e-4 in FP32).  rhs, x: device complex128, column-major [nrhs][n_unknowns];
 * iters: host [nrhs] inner GMRES iterations in total; relres: host [nrhs] the final FP64
 * residuals.  Allocates its work vectors for the call.  BI_ERR_NOT_CONVERGED when a column
 * missed tol; BI_ERR_ARG when h_ref is not FP64 or does not match h. */
int bi_solve_refined(bi_handle h, bi_handle h_ref, const void* rhs, void* x, int nrhs, double tol, int* iters,
                     double* relres);

/* Coupling with an interior discretisation (Eq. 52; Sec. II.E steps 2(a)-(e)).  Once set,
 * bi_solve solves the reduced system (C - D^{X Lambda} Q^{-1} D^{Lambda X}) x = rhs and
 * bi_matvec_coupled applies that operator; bi_matvec keeps applying C alone.
 *   n_int: interior (hybrid) unknowns.
 *   D^{Lambda X}: CSR, n_int rows, columns in [0, n_unknowns): dlx_ptr [n_int + 1],
 *     dlx_col [nnz], dlx_val [nnz] complex of the handle's precision (device pointers).
 *   D^{X Lambda}: CSR, n_unknowns rows, columns in [0, n_int): dxl_ptr, dxl_col, dxl_val.
 *   qsolve(user, in, out, nrhs, stream): out = Q^{-1} in for nrhs columns (device,
 *     column-major [nrhs][n_int], handle precision), its work ordered on `stream` (the
 *     handle's cudaStream_t) or finished before it returns; the paper uses the LU factors of
 *     the sparse Q from a direct solver, which the caller owns.
 * The caller keeps every array alive while the coupling is set; qsolve == NULL clears it.
 * The handle allocates two n_int x max_rhs work vectors.  BI_ERR_ARG on null arrays or
 * n_int < 1. */
typedef void (*bi_qsolve_fn)(void* user, const void* in, void* out, int nrhs, void* stream);
int bi_set_coupling(bi_handle h, int64_t n_int, const int* dlx_ptr, const int* dlx_col, const void* dlx_val,
                    const int* dxl_ptr, const int* dxl_col, const void* dxl_val, bi_qsolve_fn qsolve, void* user);
/* The coupling blocks of Eq. 42 on the handle's surface, in the CSR form bi_set_coupling takes:
 *   D^{X Lambda} = [D^{J Lambda}; D^{M Lambda}], n_unknowns rows (J rows then M rows):
 *     D^{J Lambda}_mn = -1/2 <f_m, n x eta_n>   (Eq. 47),  D^{M Lambda}_mn = 1/2 <f_m, eta_n>  (Eq. 48);
 *   D^{Lambda X} = [D^{Lambda J}, D^{Lambda M}], n_lambda rows, columns [0, n_unknowns):
 *     D^{Lambda J}_mn = -<eta_m, n x f_n>       (Eq. 40a), D^{Lambda M}_mn = -<eta_m, f_n>     (Eq. 40b).
 * f are the RWG functions of bi_rwg_edges; eta the zeroth-order edge functions of Eq. exp3 on
 * the surface triangles, eta = l_ab (lambda_a grad lambda_b - lambda_b grad lambda_a) for the
 * edge (a, b), a the smaller vertex number (tangential component 1 from a to b); n the outward
 * normal.  conforming = 0: one eta per (triangle t, local edge k opposite vertex k of t),
 * n_lambda = 3 nt, index 3 t + k (the face-wise trace space of a hybridised method);
 * conforming = 1: one eta per mesh edge in the RWG order, the sum of its two face functions,
 * n_lambda = N.  op_mode 0 only.
 * sizes: host int64 [3], set to (n_lambda, nnz of D^{X Lambda}, nnz of D^{Lambda X}).  With
 * all six arrays null only the sizes are returned; otherwise all six are device arrays:
 * *_ptr int32 [rows + 1], *_col int32 [nnz] (ascending within a row), *_val complex [nnz] of
 * the handle precision (imaginary parts 0).  Computed on the handle's stream; returns once
 * the arrays are written.  BI_ERR_ARG for another op_mode, bad conforming or a partial set
 * of arrays. */
int bi_coupling_blocks(bi_handle h, int conforming, int64_t* sizes, int* dxl_ptr, int* dxl_col, void* dxl_val,
                       int* dlx_ptr, int* dlx_col, void* dlx_val);
/* y = (C - D^{X Lambda} Q^{-1} D^{Lambda X}) x, the product of steps 2(a)-(e); same
 * arguments and stream behaviour as bi_matvec.  BI_ERR_ARG when no coupling is set. */
int bi_matvec_coupled(bi_handle h, const void* x, void* y, int nrhs);

/* Far field of the currents x (Eq. 22a in the far zone, time factor exp(-jkr)/r removed):
 *   F(rhat) = -jk/(4 pi) [ (I - rhat rhat) N_J - rhat x N_M ],  N_X = sum_n x_X,n int f_n exp(+jk rhat.r') ds',
 * so that sigma(rhat) = 4 pi |F(rhat)|^2 for a unit incident field (RCS of Sec. III, Eq. 5-25).
 * x: device, column-major [nrhs][n_unknowns] in the handle precision (op_mode 1: M = 0).
 * dirs: device float64 [ndir][3] unit vectors.  F: device complex128 [nrhs][ndir][3].
 * Partial sums go to scratch memory that the handle allocates on first use (and grows
 * when a later call needs more) and keeps until bi_destroy.  Queued on the handle's stream. */
int bi_farfield(bi_handle h, const void* x, int nrhs, const double* dirs, int ndir, void* F);

/* Allocation-free far field, for callers that cannot allocate device memory while they
 * run: real-time loops with a fixed memory budget set up in advance, or hosts whose device
 * allocator belongs to another runtime or framework that forbids outside cudaMalloc calls.
 * (The paper has no counterpart: it is a deployment variant of bi_farfield.)
 * Computes exactly what bi_farfield computes, with the same arguments, but its partial sums
 * go to a fixed array of BI_FARFIELD_NOALLOC_MAX_BYTES bytes compiled into the library: every
 * GPU that loads the library holds that array until the process exits.  Scratch needed:
 * ceil(N / 256) * nrhs * ndir * 96 bytes; larger requests return BI_ERR_ARG (split the
 * directions over several calls).  The call allocates nothing.  The handle's device (the one
 * current at bi_setup) must be current: otherwise BI_ERR_ARG.  The first call on each handle
 * looks up the array's device address (cudaGetSymbolAddress) and keeps it in the handle with
 * the id of the current CUDA context; a later call under another context (the device reset
 * and its context created anew) looks it up again.  Make the first call before any stream
 * capture.  All calls on a device share the array, which
 * keeps the last call's partial sums (each call writes every slot it reads): calls whose work
 * overlaps on the GPU (different streams, or different handles on one device) race on it --
 * order them on one stream or synchronise between them.  The handle itself must already
 * exist (bi_setup allocates). */
#define BI_FARFIELD_NOALLOC_MAX_BYTES (8u << 20)
int bi_farfield_noalloc(bi_handle h, const void* x, int nrhs, const double* dirs, int ndir, void* F);

/* Diagnostics: copy an internal device buffer of h to host memory.
 *   what 0: leaf radiation patterns F [N_tree][K_leaf/2][2] complex (tree order, theta/phi;
 *           the first K_leaf/2 directions in theta-major order, one of each antipodal pair:
 *           the antipode holds (conj F_theta, -conj F_phi))
 *   what 1: leaf twisted receive patterns RX [N_tree][K_leaf/2][2], same convention
 *   what 2: translation operators of `level` [343][K_level] (weights folded in)
 *   what 3: outgoing patterns U of `level` [boxes][K_level][2 nrhs] (last product)
 *   what 4: incoming patterns V of `level` [boxes][K_level][2 nrhs] (last product)
 *   what 5: tree order: int32 [N] user RWG index of each tree position
 * host: buffer of `bytes` bytes; returns BI_ERR_ARG when it is too small or the buffer
 * does not exist for that level.  Synchronises the handle's stream. */
int bi_debug_copy(bi_handle h, int what, int level, void* host, int64_t bytes);

/* Diagnostics: device time of each stage of one product, in milliseconds, averaged over
 * `reps` products.  Stages run one after another on the handle's stream (no graph and no
 * near/far overlap), bracketed by CUDA events; stage_ms[8] = gather, near, aggregate,
 * interpolate, translate, anterpolate, receive, scatter (names from bi_stage_name).
 * x, y as for bi_matvec.  Synchronises the stream. */
int bi_profile_stages(bi_handle h, const void* x, void* y, int nrhs, int reps, double* stage_ms);
const char* bi_stage_name(int i);

/* ---- Serving: continuous batching of solves ------------------------------------------
 * A server owns two host threads.  bi_submit queues a solve request (mesh, k0, parameters,
 * nrhs plane waves, tolerance).  Requests on the same operator (identical vertices,
 * triangles, k0 and parameters) share one set-up operator and are merged into one job: one
 * GMRES over the columns of all of them (each column keeps its request's tolerance), so each
 * product of the job is one batched bi_matvec for all its requests.  A job takes every waiting
 * request of its operator up to max_batch_rhs columns, including requests that arrive while
 * its operator is set up; later requests of a busy operator wait for the next job.  After its
 * job an operator stays cached (idle operators are dropped, oldest first, when the memory
 * budget needs room).  Jobs are admitted while fewer than max_active are set up or running
 * and the device-memory estimate fits mem_budget_bytes; setup threads build operators and
 * GMRES states (and tune the kernel forms for the job's column count) so that set-ups
 * overlap running solves, and the serving thread advances every
 * running job by one iteration per pass, so their products and Krylov kernels overlap on the
 * device.  Latency = submit to solution on the host. */
typedef struct bi_server_s* bi_server;
typedef struct {
    int64_t mem_budget_bytes;   /* device bytes for operators and jobs; 0 = 80% of free memory */
    int max_active;             /* jobs set up or iterating at once (default 8) */
    int queue_capacity;         /* waiting requests before bi_submit returns BI_ERR_BUSY (default 4096) */
    int share_operators;        /* 1 (default): cache operators and merge requests on one operator into
                                   jobs; 0: every request builds its own operator and runs alone */
    int max_batch_rhs;          /* columns of one job, and max_rhs of the operators (default 64) */
    int setup_threads;          /* host threads that build operators and jobs, 1-16 (default 2) */
} bi_server_params;

/* bi_server_stats counters */
enum {
    BI_STAT_JOBS = 0,              /* jobs started */
    BI_STAT_OPERATORS_BUILT = 1,   /* bi_setup calls */
    BI_STAT_CACHE_HITS = 2,        /* jobs started on a cached operator */
    BI_STAT_MERGED_REQUESTS = 3,   /* requests that joined another request's job */
    BI_STAT_EVICTIONS = 4,         /* cached operators dropped for memory */
    BI_STAT_CACHED_OPERATORS = 5,  /* idle operators held now */
    BI_STAT_HELD_BYTES = 6,        /* device bytes held now (operators and jobs) */
    BI_SERVER_NSTATS = 7
};

void bi_server_default_params(bi_server_params* p);
/* Create a server on the current CUDA device. */
int bi_server_create(const bi_server_params* prm, bi_server* out);
/* Queue a solve of C x = b for nrhs plane waves (khat, phat: host [nrhs][3]) on the surface
 * (verts, tris) at k0; opt as for bi_setup (stream ignored).  Copies every input.  *req
 * receives the request id.  BI_ERR_BUSY: queue full; BI_ERR_OOM: larger than the budget. */
int bi_submit(bi_server s, const double* verts, int nv, const int* tris, int nt, double k0, const bi_params* opt,
              int nrhs, const double* khat, const double* phat, double tol, int64_t* req);
/* *done = 1 once the request finished; *status = its bi_status then. */
int bi_poll(bi_server s, int64_t req, int* done, int* status);
/* Result of a finished request: x_host [nrhs][n_unknowns] complex of the request precision
 * (x_bytes = buffer size), GMRES iterations and relative residuals [nrhs], latency (submit
 * to result) and setup time in ms.  Returns the request's status, or BI_ERR_BUSY if it is not
 * finished.  Any output pointer may be NULL. */
int bi_result(bi_server s, int64_t req, void* x_host, int64_t x_bytes, int* iters, double* relres, double* latency_ms,
              double* setup_ms);
/* Copy the first n counters (BI_STAT_*) into out. */
int bi_server_stats(bi_server s, int64_t* out, int n);
/* Forget a finished request (frees its host result). */
int bi_release(bi_server s, int64_t req);
const char* bi_server_last_error(bi_server s);
/* Stop the threads and free every request and buffer. */
void bi_server_destroy(bi_server s);

/* Host-only plan (inspection of the set-up, no counterpart in the paper): the RWG numbering,
 * octree, near and interaction lists, parent-centred translation lists, angular sampling and
 * interpolation tables that bi_setup builds, computed on the host with no device and no CUDA
 * call.  Same mesh and parameter rules as bi_setup; BI_ERR_MESH / BI_ERR_ARG as there.
 * bi_plan_get copies one array to `out` (`bytes` long; NULL out only reports the element
 * count in *count).  Element type int32 unless marked (double):
 *    0 leaf_start [nbox_leaf + 1]   1 near_ptr [nbox_leaf + 1]   2 near_src
 *    3 coords [nbox][3] of `level`  4 parent [nbox] of `level` >= 1
 *    5 child_ptr [nbox + 1] of `level` (children at level + 1)
 *    6 il_ptr, 7 il_src, 8 il_off (offset code (ox+3)*49 + (oy+3)*7 + (oz+3), ox = receiver - source)
 *      of translation `level` >= 2
 *    9 parent-centred list pointers [nbox(level-1) + 1], 10 its sources, 11 its codes [entries][8]
 *      (65535: the child slot has no interaction with that source)
 *   12 perm [N] (tree position -> RWG index)
 *   13 edges [N][2] (vertex ids of the edge of each RWG), 14 T+ [N], 15 T- [N] (its triangles)
 *   20 theta nodes (double), 21 theta weights in cos(theta) (double) of `level` >= 2
 *   22 th_src, 23 th_flip, 24 th_w (double): theta taps [nth(level)][p] from level + 1 to level
 *   25 ph_src, 26 ph_w (double): phi taps [nph(level)][p]
 *   27 tth_ptr, 28 tth_dst, 29 tth_flip, 30 tth_w (double): transposed theta lists per child row
 *   31 tph_ptr, 32 tph_dst, 33 tph_w (double): transposed phi lists per child column
 *   40 distance index [343] of each offset code of translation `level` (-1: touching offset)
 *   41 spherical Hankel values (double) [distances][L + 1][2]: h_n^(2)(k|X|) as (re, im) */
typedef struct bi_plan_s* bi_plan;
/* verts, tris, opt as for bi_setup (opt may be NULL; stream and precision are ignored).
 * *out is NULL on failure. */
int bi_plan_create(const double* verts, int nv, const int* tris, int nt, double k0, const bi_params* opt, bi_plan* out);
/* Sizes of the plan (host struct; device and timing fields are 0). */
int bi_plan_info(bi_plan p, bi_info_t* info);
/* BI_ERR_ARG for an unknown `what`, a level that has no such array, or `bytes` smaller than
 * the array (nothing is copied then; *count still holds the element count). */
int bi_plan_get(bi_plan p, int what, int level, void* out, int64_t bytes, int64_t* count);
/* Text of the last failed bi_plan_create of the calling thread. */
const char* bi_plan_last_error(void);
/* Free the plan (host memory only).  NULL is ignored. */
void bi_plan_destroy(bi_plan p);

/* Text of the last error on h (or, when h is NULL, of the calling thread's last failed bi_setup). */
const char* bi_last_error(bi_handle h);

/* Diagnostics (no counterpart in the paper): the kernel forms the autotuner chose for the level
 * passes, one line per (pass, level, E): the first product with a given nrhs (bi_matvec,
 * bi_solve, bi_profile_stages) times every applicable form of each translation, interpolation
 * and anterpolation on the handle's buffers, synchronising the stream, and keeps the fastest
 * (environment BI_AUTOTUNE=0 keeps the built-in choices).  buf: host, len bytes, NUL-terminated;
 * BI_ERR_ARG when the text was cut. */
int bi_tuned_config(bi_handle h, char* buf, int64_t len);

/* Diagnostics (no counterpart in the paper): limit, in SM clock cycles, of the consumer waits of
 * the bulk-copy leaf kernels (aggregation and receive of one and few right-hand sides); cycles <= 0
 * restores the default of 2^31 (about one second).  A wait that runs out makes its CTA drain its
 * copies in flight (always with the default limit, so no copy lands after the CTA has left),
 * record BI_ERR_TIMEOUT in the handle's device status word and leave its outputs unwritten.  With
 * a limit of a few cycles a normal product gives up on its first copies: that is how the
 * give-up path is tested without a copy that never lands.  Synchronises the handle's stream. */
int bi_debug_set_wait_limit(bi_handle h, long long cycles);

/* Device status of h (implementation health, no counterpart in the paper): synchronises
 * the handle's stream, then returns BI_ERR_TIMEOUT if a product kernel gave up a bounded
 * wait on one of its bulk copies since the last check (the products enqueued before then
 * are invalid), else BI_OK; the status is cleared by the call.  bi_matvec_host and
 * bi_solve make the same check before they return. */
int bi_device_status(bi_handle h);

/* Release every device buffer of h.  NULL is ignored. */
void bi_destroy(bi_handle h);

#ifdef __cplusplus
}
#endif

#endif /* BI_GB300_H */
