/*
 * sa.h - C ABI of the GB300 semi-analytical isogeometric thermal library.
 *
 * The method (Sections 2-2.4 of the paper): the temperature of a part under
 * a scanning laser is split into T = T~ + T^ (Eq. temperature-decomposition).
 * T~ is a closed-form sum of point-source solutions over every past laser
 * position (Eqs. sum-of-point-temp, semi-temperature); T^ solves the
 * source-free heat equation on a NURBS patch (Eq. that-heat) with Neumann
 * data k dT~/dn on the lateral faces (Eq. that-bc-n) and Dirichlet data
 * T_c - T~ on the bottom face (Eq. that-bc-d), discretised by IGA
 * (Section 2.3) and advanced by the theta-scheme (Eq. theta-method).
 *
 * Conventions for every call:
 *  - Units are SI (m, s, W, J, K).
 *  - Every call returns an sa_status; nothing throws across the ABI.
 *  - Input buffers passed by the caller are copied during the call; the
 *    caller keeps ownership.  Output buffers are caller-allocated.
 *  - The library owns all device memory of a context and frees it in
 *    sa_destroy.  Device buffers are allocated during set-up
 *    (sa_create_patch, sa_set_scan, the first sa_step), never per step.
 *  - Work runs asynchronously on the stream given in sa_options (NULL = the
 *    legacy default stream) unless a call says otherwise.
 *  - After SA_ERR_CUDA the context is poisoned: every later call returns
 *    SA_ERR_STATE except sa_destroy and sa_last_error.
 *  - Calls out of order (a step before patch, material and scan) return
 *    SA_ERR_STATE.
 *  - sa_last_error(ctx) gives a one-line message for the last failure.
 */
#ifndef SA_H
#define SA_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sa_ctx sa_ctx;

typedef enum sa_status {
    SA_OK = 0,
    SA_ERR_ARG = 1,            /* invalid argument (NULL, size, range, NaN) */
    SA_ERR_GEOMETRY = 2,       /* invalid knots / weights / degenerate Jacobian */
    SA_ERR_STATE = 3,          /* call out of order, or context poisoned */
    SA_ERR_CUDA = 4,           /* a CUDA runtime call failed */
    SA_ERR_OOM = 5,            /* device allocation failed */
    SA_ERR_NOT_CONVERGED = 6,  /* PCG hit pcg_max_iter before pcg_tol */
    SA_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up */
    SA_ERR_NAN = 8             /* a non-finite value appeared in the state */
} sa_status;

/* Arithmetic of the per-step path. */
enum { SA_FP64 = 0,   /* every stage in FP64                                       */
       SA_MIXED = 1   /* history sums in FP32 (coefficients from ages relative to
                         the current step; compensated accumulation on the
                         pairwise path, per-chunk FP32 sums on the separable one)
                         and the per-step operators' values in FP32 with FP64
                         Krylov vectors, state and residual test (dot products
                         from copies scaled by 1/||b||, in FP32); assembly and
                         boundary integrals FP64                                   */ };

/* Face ids: 0 xi=0, 1 xi=1, 2 eta=0, 3 eta=1, 4 zeta=0, 5 zeta=1. */
enum { SA_FACE_NONE = 0,       /* no boundary term (top face, Section 2.1)      */
       SA_FACE_NEUMANN = 1,    /* lateral face: F_i = int (-q_N) N_i dS          */
       SA_FACE_DIRICHLET = 2   /* bottom face: T^ = T_c - T~ (L2 projection)     */ };

typedef struct sa_options {
    int precision;             /* SA_FP64 (default) or SA_MIXED                   */
    double pcg_tol;            /* stop when ||r||_2 <= pcg_tol ||b||_2; 1e-10     */
    int pcg_max_iter;          /* per solve; default 2000                         */
    double half_space_factor;  /* s_img multiplying every point source; default 2
                                  (image across the adiabatic top plane); 1 gives
                                  the printed full-space kernel                   */
    void* cuda_stream;         /* cudaStream_t to run on, NULL = default stream   */
    int use_graph;             /* 1: sa_step replays captured CUDA graphs (needs a
                                  non-default cuda_stream): 16 steps per graph while
                                  at least 16 remain in the call, then one-step
                                  graphs                                          */
    int device;                /* CUDA device ordinal; -1 = the current device   */
    int hist_points_per_lane;  /* history-sum tile: points per lane (1,2,4); 0=auto*/
    int hist_warps;            /* history-sum tile: warps splitting the sources (4,8); 0=auto */
    int stage_timing;          /* 1: CUDA events around every stage of each step (direct
                                  launches, the graph path is off while set); the step then
                                  synchronises; read the times with sa_get_stage_times   */
    int pcg_variant;           /* where both solves keep their Krylov vectors (same
                                  Jacobi-PCG recurrences, Chronopoulos-Gear form, FP64
                                  vectors, two grid barriers per iteration):
                                  SA_PCG_AUTO (0, default): shared memory when a block's
                                    rows fit, global memory otherwise;
                                  SA_PCG_SHARED (1): shared memory (SA_ERR_ARG at set-up
                                    if the rows do not fit);
                                  SA_PCG_GLOBAL (2): global memory                  */
    int initial_guess;         /* start of each theta-step solve:
                                  SA_GUESS_PREVIOUS (0, default): T^n (and g^n for
                                    the bottom projection);
                                  SA_GUESS_EXTRAPOLATE (1): T^n + (T^n - T^{n-1}),
                                    kept only when its residual is below that of
                                    T^n, and 2 g^n - g^{n-1} for the projection.  The
                                    converged step is the same to the solver tolerance;
                                    after sa_set_state the first step starts from T^n.
                                  A learned warm start (sa_set_warm_start) replaces
                                  the extrapolated proposal of the main solve.     */
    int precond;               /* preconditioner of the main theta-step solve:
                                  SA_PRECOND_AUTO (0, default): fast diagonalization
                                    (below) when the shared-memory PCG runs and the free
                                    control variables form the tensor grid, Jacobi
                                    otherwise;
                                  SA_PRECOND_JACOBI (1): D^{-1};
                                  SA_PRECOND_FD (2): fast diagonalization of the box with
                                    the patch's knot vectors and mean lengths, scaled to
                                    the diagonal of A (exact on a box), SA_ERR_ARG at
                                    set-up where it does not apply (more than 128
                                    control variables along a direction).  The bottom
                                    projection keeps Jacobi.  Same solution to the
                                    solver tolerance.                                */
    int hist_mode;             /* evaluation of the history sums (same sums):
                                  SA_HIST_AUTO (0, default): separable where every
                                    lateral and Dirichlet face is an axis-aligned
                                    rectangle (its quadrature points a tensor grid, the
                                    normal a coordinate axis), pairwise otherwise;
                                  SA_HIST_PAIRWISE (1): one exponential per
                                    (point, source) pair;
                                  SA_HIST_SEPARABLE (2): the Gaussian of each source
                                    factorised along the face's two axes, each face's
                                    sum a matrix product over the sources (one FMA a
                                    pair); SA_ERR_ARG at sa_create_patch where a face
                                    is not such a rectangle                          */
    double hist_cutoff;        /* opt-in truncation of the separable history sums
                                  (not the paper's method, which keeps the full
                                  sum; 0, the default, keeps it): with eta > 0 the
                                  product of a face tile with a unit of sources is
                                  skipped when an upper bound of that unit's
                                  contribution at every point of the tile (sum over
                                  its sources of w exp(-a d_min^2), times |n . d|
                                  on the lateral faces, d_min the distance from the
                                  source to the tile's box) is at most eta M / U,
                                  M the largest |sum| over the face kind's points
                                  at the previous step and U the units per tile.
                                  Every sum then differs from the full one by at
                                  most eta M.  Ignored by the pairwise sums;
                                  SA_ERR_ARG when negative or >= 1               */
} sa_options;

enum { SA_PCG_AUTO = 0, SA_PCG_SHARED = 1, SA_PCG_GLOBAL = 2 };
enum { SA_PRECOND_AUTO = 0, SA_PRECOND_JACOBI = 1, SA_PRECOND_FD = 2 };
enum { SA_GUESS_PREVIOUS = 0, SA_GUESS_EXTRAPOLATE = 1 };
enum { SA_HIST_AUTO = 0, SA_HIST_PAIRWISE = 1, SA_HIST_SEPARABLE = 2 };

/* Fill o (caller-owned, not NULL) with the defaults listed above; host only. */
void sa_options_default(sa_options* o);

/* Create an empty context on the chosen device.  o may be NULL (defaults);
 * the options are copied.  *out is owned by the caller and released with
 * sa_destroy.  Errors: SA_ERR_ARG (out NULL, an option out of its range),
 * SA_ERR_CUDA (device selection or query), SA_ERR_OOM. */
sa_status sa_create(const sa_options* o, sa_ctx** out);

/*
 * Geometry: one trivariate NURBS patch (Section 2.3, the map Phi and the
 * basis of degree p on the knot vectors).
 *   degree[d]   polynomial degree in parametric direction d (1..3)
 *   n_ctrl[d]   control points in direction d
 *   ctrl_xyz    n_ctrl[0]*n_ctrl[1]*n_ctrl[2]*3 doubles (host), index
 *               ((k*n1 + j)*n0 + i)*3 + c, xi index i fastest
 *   weights     same count without the *3, > 0; NULL = B-spline (all 1)
 *   knots[d]    n_knots[d] = n_ctrl[d] + degree[d] + 1 nondecreasing values,
 *               open (first and last value repeated degree+1 times)
 *   seam_dir    -1: an open patch.  0, 1 or 2: the patch is closed in that
 *               parametric direction (a ring): the control layers i_d = 0 and
 *               i_d = n_ctrl[d] - 1 coincide (points and weights) and are ONE
 *               set of control variables, so the space holds the merged
 *               functions R_0 + R_{n-1}.  Both faces of that direction must be
 *               SA_FACE_NONE (they are interior).  Control variables, fields
 *               and matrices are then indexed over the merged grid (n_ctrl[d]
 *               - 1 layers in direction d, natural order, layer n-1 = layer 0).
 * The top face (zeta = 1) must be the plane z = const: the point sources
 * lie on it.  Set-up (on the device): element and face Gauss points
 * ((p+1) per direction), the assembly of M and K in CSR form and the
 * boundary weight matrices.  Errors: SA_ERR_ARG (also: seam faces not NONE),
 * SA_ERR_GEOMETRY (non-open or decreasing knots, weights <= 0, non-planar
 * top, seam layers that do not coincide, det J <= 0 at a Gauss point),
 * SA_ERR_OOM, SA_ERR_CUDA.
 */
sa_status sa_create_patch(sa_ctx* ctx, const int degree[3], const int n_ctrl[3],
                          const double* ctrl_xyz, const double* weights,
                          const double* const knots[3], const int n_knots[3], int seam_dir);

/* Face kinds (SA_FACE_*), face ids as above (Section 2.1: Neumann data on
 * the lateral faces, Eq. that-bc-n; Dirichlet data on the bottom face, Eq.
 * that-bc-d; the top face's condition is built into the half-space point
 * source).  Default: faces 0-3 NEUMANN, face 4 DIRICHLET, face 5 NONE.
 * face_kind: 6 ints (host), copied.  Must be called before sa_create_patch
 * to take effect on set-up.  Errors: SA_ERR_ARG (NULL, unknown kind),
 * SA_ERR_STATE (after sa_create_patch, or a poisoned context). */
sa_status sa_set_boundary(sa_ctx* ctx, const int face_kind[6]);

/* Material (Section 2, Eq. linear-heat: alpha = k/(rho c_p)) and the
 * platform / initial temperature T_c (Section 2: T(x,0) = T_c).  All > 0
 * except T_c (any finite value).  Errors: SA_ERR_ARG (a value out of range or
 * not finite), SA_ERR_STATE (poisoned context). */
sa_status sa_set_material(sa_ctx* ctx, double k, double rho, double cp, double T_c);

/*
 * Scan (Section 2): the laser moves along a polyline on the top plane.
 *   path_xyz  nv*3 doubles (host), vertex coordinates; z is ignored (the
 *             sources are put on the top plane)
 *   seg_on    nv-1 flags: 1 laser on, 0 a jump that takes no time and adds
 *             no source; NULL = all on
 * A maximal run of laser-on segments is a track.  Along each track, sources
 * sit at arc lengths 0, v*dt, 2 v*dt, ... (dt of the first sa_step); source
 * I (1-based, in scan order) carries E = A P dt and is active from step I on
 * (Section 2 and 3.1).  spot_radius r enters through tau = t - r^2/(8 alpha)
 * (Eq. semi-temperature).  Errors: SA_ERR_ARG.
 */
sa_status sa_set_scan(sa_ctx* ctx, const double* path_xyz, int nv,
                      const unsigned char* seg_on, double power, double absorptivity,
                      double speed, double spot_radius);

/* Counters cover every step since the previous call that returned stats
 * (steps enqueued with stats == NULL included). */
typedef struct sa_step_stats {
    int steps_done;            /* steps enqueued by this call                      */
    int pcg_iters_last;        /* PCG iterations of the last step                  */
    int pcg_iters_total;       /* summed over the covered steps                    */
    int pcg_iters_max;
    int bot_iters_total;       /* iterations of the bottom (Dirichlet) projection  */
    double rel_res_last;       /* ||r||/||b|| at exit of the last step's PCG       */
    int n_active_sources;      /* sources in the sum at the last step              */
    long long step_index;      /* n after the call                                 */
    int ws_used_last;          /* 1: the last step's PCG started from the learned guess */
    double ws_ratio_last;      /* |r0 - A dx| / |r0| of the last learned guess           */
    long long hist_pairs_skipped;  /* (point, source) pairs dropped by hist_cutoff over
                                      the steps since the last statistics read      */
} sa_step_stats;

/*
 * Advance the correction field n_steps theta-steps of size dt (Eq.
 * theta-method, theta in [0, 1]).  Per step n -> n+1: point-source history
 * sums at the boundary quadrature points, F^{n+1} and the bottom projection,
 * the theta right-hand side, PCG with the preconditioner and initial guess
 * of sa_options (precond, initial_guess) to pcg_tol.  dt must stay the
 * same for the life of a scan (the source spacing is v*dt); a change returns
 * SA_ERR_ARG.  theta may change between calls (the operator is rebuilt).
 * stats may be NULL: the call then returns after enqueueing the work (errors
 * of the device-side solves are reported by the next call that synchronises).
 * With stats != NULL the call synchronises the stream and returns
 * SA_ERR_NOT_CONVERGED / SA_ERR_TIMEOUT / SA_ERR_NAN when a step failed.
 */
sa_status sa_step(sa_ctx* ctx, double theta, double dt, int n_steps, sa_step_stats* stats);

/*
 * Reconstruction T = T~ + T^ (Section 2.4) at n physical points at the
 * current step t_n = n dt: point inversion x -> xi by Newton's method on the
 * NURBS map, sum_i R_i(xi) T^_i, plus the history sum at t_n (FP64; in an
 * SA_MIXED context the history sum is formed in FP32 like the step's, and so
 * are the nearest-element search that seeds Newton and the point inversion
 * with its basis values: Newton in FP32 to 1e-6 of the patch size, or in
 * FP64 for a point where FP32 does not settle).  In FP64 contexts Newton
 * starts in FP32 and ends in FP64 at 1e-13 of the patch size.
 *   pts    n*3 doubles, host (on_device = 0) or device (on_device = 1)
 *   T_out  n doubles, same memory space; a point outside the patch gets NaN
 * Synchronous.  Errors: SA_ERR_ARG, SA_ERR_STATE, SA_ERR_CUDA.
 */
sa_status sa_eval_T(sa_ctx* ctx, const double* pts, int n, double* T_out, int on_device);

/*
 * T = T~ + T^ at n physical points for SEVERAL LASERS on one part, by
 * superposition (the setting of Section 2 allows several lasers; its outlook
 * names them): the problem is linear (constant material, Eq. that-heat with
 * linear boundary data in T~, and T~ a plain sum over sources, Eq.
 * sum-of-point-temp), so the temperature of lasers 1..L switched on together
 * is sum_l T_l - (L - 1) T_c, where T_l is the temperature with laser l
 * alone.  ctxs[l] is a context that carries laser l alone (sa_set_scan with
 * its path, power and speed), stepped with the same theta and dt as the
 * others (separately, or together in an sa_batch).
 *   ctxs     n_ctx >= 1 contexts on the current device: same patch (the
 *            same control-variable count), material and T_c, and the same
 *            step index (SA_ERR_ARG otherwise)
 *   pts      n*3 doubles, host (on_device = 0) or device (on_device = 1)
 *   T_out    n doubles, same memory space; NaN outside the patch
 * Each context evaluates like sa_eval_T (its own precision); the sum runs
 * on the device.  Working buffers belong to ctxs[0] (grown on demand, kept).
 * Synchronous.  Errors: SA_ERR_ARG, SA_ERR_STATE, SA_ERR_CUDA.
 */
sa_status sa_eval_T_superposed(sa_ctx* const* ctxs, int n_ctx, const double* pts, int n, double* T_out,
                               int on_device);

/*
 * Heat-loss rates at n physical points with unit normals (Section 3.1, the
 * diagnostic q~ + q^ = -k dT/dn of the adiabatic boundary): q~ = -k n . grad T~
 * (the history sum's gradient at t_n) and q^ = -k n . grad T^ (grad T^ =
 * J^{-T} sum_i T^_i grad_xi R_i at the inverted point).  On an adiabatic
 * face the exact solution has q~ + q^ = 0.
 *   pts, nrm  n*3 doubles each (nrm: unit outward normals), host or device
 *   q_tilde, q_hat  n doubles each, same memory space; NaN outside the patch
 * FP64, or FP32 history sums in an SA_MIXED context.  Synchronous.
 * Errors: SA_ERR_ARG, SA_ERR_STATE, SA_ERR_CUDA.
 */
sa_status sa_eval_flux(sa_ctx* ctx, const double* pts, const double* nrm, int n, double* q_tilde,
                       double* q_hat, int on_device);

/*
 * Allocation-free variant of sa_eval_T (this entry point has no counterpart
 * in the paper; it exists for callers that cannot allocate device memory).
 * Some callers must not call cudaMalloc/cudaFree while they run: a
 * monitoring hook inside a latency-critical loop (an allocation may
 * synchronise the device), or code inside a framework whose caching
 * allocator already holds the free device memory.  sa_eval_T may allocate
 * (its first call, a larger point count); this call never allocates.
 *   pts    n*3 doubles in DEVICE memory (caller-allocated)
 *   T_out  n doubles in DEVICE memory (caller-allocated); NaN outside the patch
 * Evaluates in FP64 in every context: in an SA_FP64 context the result
 * equals sa_eval_T's to rounding; in an SA_MIXED context (whose sa_eval_T
 * sums the sources in FP32) the two agree within 1e-4 relative and 0.05 K.
 * Working memory: one fixed file-scope device array of 5 MiB (the current
 * step's FP64 source coefficients and the element centres), held by every
 * device that loads the library until the process exits.  Limits: at most 65,536 discretised sources and 131,072 elements;
 * larger contexts get SA_ERR_ARG with a message.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  All
 * calls share the array, so calls that overlap on the GPU (different
 * streams or contexts, concurrently) race; serialise them.  Synchronous on
 * the context's stream.  Needs a context that has stepped or had its state
 * set (SA_ERR_STATE otherwise).
 */
sa_status sa_eval_T_noalloc(sa_ctx* ctx, const double* pts, int n, double* T_out);

/*
 * Self-test of the device-side bounded waits (no paper counterpart; for the
 * tests).  Launches (1) two blocks of which one leaves without arriving, so
 * the other's grid-barrier wait never completes, and (2) one block waiting on
 * an mbarrier that nothing arrives at.  Each wait gives up after its time
 * limit (2 s, 1 s), records SA_DEV_TIMEOUT in a status word and returns; no
 * fault, the device stays usable.  *barrier_flagged / *mbarrier_flagged
 * (may be NULL) get 1 when the flag was recorded.  Uses the current device;
 * synchronous.  Errors: SA_ERR_CUDA.
 */
sa_status sa_selftest_waits(int* barrier_flagged, int* mbarrier_flagged);

/* Sizes of a context after set-up (out: caller-owned).  Errors: SA_ERR_ARG
 * (out NULL), SA_ERR_STATE (before sa_create_patch, or poisoned). */
typedef struct sa_sizes {
    int n_dof, n_free, n_dir;      /* control variables; free / Dirichlet             */
    int q_lat, q_bot;              /* lateral / bottom quadrature points              */
    int n_src;                     /* discretised sources (0 before the first step)   */
    long long nnz_mk;              /* nonzeros of the M, K rows of free control vars. */
    long long nnz_a;               /* nonzeros of the free-free operator              */
    long long step_index;          /* current n                                       */
    int n_elem;                    /* volume elements                                 */
    int hist_separable;            /* 1: the history sums are evaluated separably     */
    long long sep_factors;         /* separable sums: factor exponentials per active  */
                                   /* source and step (sum over the face tiles of     */
                                   /* rows + columns); 0 for the pairwise sums        */
} sa_sizes;
sa_status sa_get_sizes(sa_ctx* ctx, sa_sizes* out);

/* Fields that can be read back (synchronous copy to host or device memory).
 * Indices are NATURAL control-point order ((k*n1 + j)*n0 + i) for dof vectors
 * and the canonical quadrature order for point vectors: faces in increasing
 * id, face elements with the lower tangential direction fastest, then the
 * Gauss points of each face element with the lower tangential direction
 * fastest. */
enum { SA_FIELD_THAT = 0,      /* T^ at control variables (n_dof)                    */
       SA_FIELD_F = 1,         /* F^n at control variables (n_dof)                   */
       SA_FIELD_DTDN_LAT = 2,  /* dT~/dn at lateral points, last step (q_lat)        */
       SA_FIELD_TT_BOT = 3,    /* T~ at bottom points, last step (q_bot)             */
       SA_FIELD_LAT_X = 4,     /* lateral points: x,y,z,nx,ny,nz,wdS (q_lat*7)       */
       SA_FIELD_BOT_X = 5      /* bottom points: x,y,z,wdS (q_bot*4)                 */ };
/* out: count >= the field's length, host (on_device = 0) or device (1);
 * synchronous.  Errors: SA_ERR_ARG (out NULL, unknown field, count too
 * small), SA_ERR_STATE (before sa_create_patch), SA_ERR_CUDA. */
sa_status sa_get_field(sa_ctx* ctx, int field, double* out, long long count, int on_device);

/* Assembled matrices (Section 2.3: M_ij = int rho c_p R_i R_j dV, K_ij = int
 * k grad R_i . grad R_j dV) in natural order, CSR over ALL control
 * variables: which = 0 mass M, 1 conductivity K.  rowptr: n_dof+1, colind
 * and vals: nnz (from sa_get_matrix_nnz).  Host buffers, caller-allocated;
 * synchronous.  Errors: SA_ERR_ARG (NULL, which not 0 or 1), SA_ERR_STATE
 * (before sa_create_patch), SA_ERR_CUDA. */
sa_status sa_get_matrix_nnz(sa_ctx* ctx, long long* nnz);
sa_status sa_get_matrix(sa_ctx* ctx, int which, long long* rowptr, int* colind, double* vals);

/* Checkpoint: the state is (n, T^ (n_dof, natural order), F^n (n_dof)).  The
 * sources are recomputed from the scan.  Host buffers (caller-owned; read by
 * sa_set_state, written by sa_get_state); synchronous.  Errors: SA_ERR_ARG
 * (NULL, n < 0), SA_ERR_STATE (before patch and material), SA_ERR_NAN (a
 * non-finite value in the state), SA_ERR_CUDA. */
sa_status sa_get_state(sa_ctx* ctx, long long* n, double* T_hat, double* F);
sa_status sa_set_state(sa_ctx* ctx, long long n, const double* T_hat, const double* F);

/*
 * Learned warm start (the paper has no learned component: this only changes
 * the initial guess of the free-block solve; PCG still converges to pcg_tol
 * and keeps the cold start x0 = T^n whenever the proposal does not lower the
 * residual).  A 4-layer perceptron of width H (BF16 weights, FP32
 * accumulation, tensor-core GEMMs):
 *   x -> silu(W1 x + b1) -> silu(W2 h + b2) -> silu(W3 h + b3) -> W4 h + b4
 * Input: the initial residual r0 = b - A T^n of the free block at the rows
 * in_idx, divided by |r0|_2; output: the increment of the free control
 * variables divided by |r0|_2 (the solve is linear, so the scaling is exact).
 */
/* Every sa_mlp call: Errors SA_ERR_ARG (NULL, sizes out of range or not
 * matching the network), SA_ERR_OOM, SA_ERR_CUDA.  *out of sa_mlp_create is
 * owned by the caller and released with sa_mlp_destroy (NULL is a no-op);
 * a network set as a warm start must outlive that use; the context keeps no
 * reference after sa_set_warm_start(ctx, NULL, ...). */
typedef struct sa_mlp sa_mlp;
sa_status sa_mlp_create(int n_in, int hidden, int n_out, unsigned long long seed, sa_mlp** out);
void sa_mlp_destroy(sa_mlp* m);
long long sa_mlp_n_params(const sa_mlp* m);
/* FP32 host arrays, per layer W_l (row-major, out x in) then b_l */
sa_status sa_mlp_get_params(sa_mlp* m, float* host);
sa_status sa_mlp_set_params(sa_mlp* m, const float* host);
/* X: rows x n_in BF16 (device); Y: rows x n_out FP32 (device); synchronous */
sa_status sa_mlp_forward(sa_mlp* m, const void* X, int rows, float* Y, void* stream);
/* loss 1/(2 rows) sum |f(x) - y|^2 and its gradient (host FP32, parameter layout) */
sa_status sa_mlp_gradients(sa_mlp* m, const void* X, const void* Y, int rows, float* grads,
                           double* loss, void* stream);
/* one Adam step (beta 0.9 / 0.999) on a minibatch; loss may be NULL (async) */
sa_status sa_mlp_train_step(sa_mlp* m, const void* X, const void* Y, int rows, float lr,
                            double* loss, void* stream);
/* use net as the warm start of sa_step (NULL: cold start); n_out must be n_free */
sa_status sa_set_warm_start(sa_ctx* ctx, sa_mlp* net, int n_in, const int* in_idx);
/* training data: every following step writes row k of X (n_in BF16: r0[in_idx]/|r0|)
 * and of Y (n_free BF16: increment/|r0|) into the caller's device buffers, up to
 * capacity rows (graph replay is off while recording).  X = NULL stops. */
sa_status sa_set_recorder(sa_ctx* ctx, void* X, void* Y, int capacity, int n_in, const int* in_idx);
sa_status sa_get_recorded(sa_ctx* ctx, int* count);

/* Stages of one step, in launch order. */
enum { SA_STAGE_PROLOGUE = 0,  /* source coefficients of the step                       */
       SA_STAGE_HISTORY = 1,   /* history sums at the lateral and bottom points          */
       SA_STAGE_GATHER = 2,    /* F^{n+1} and the bottom right-hand side                 */
       SA_STAGE_BOTTOM = 3,    /* bottom L2 projection (PCG)                             */
       SA_STAGE_RHS = 4,       /* theta right-hand side and initial residual             */
       SA_STAGE_PCG = 5,       /* free-block PCG                                         */
       SA_STAGE_FINALIZE = 6,  /* Dirichlet values, F^n <- F^{n+1}, n <- n+1            */
       SA_N_STAGES = 7 };
/* Milliseconds per stage accumulated over the steps run with stage_timing
 * since the previous call (which resets them); *steps = number of steps.
 * ms: SA_N_STAGES doubles (host). */
sa_status sa_get_stage_times(sa_ctx* ctx, double* ms, long long* steps);

/*
 * Batches: many independent instances (uneven patches, different scans and
 * powers; one material, one theta and dt) stepped together with one launch
 * per stage, replayed as one CUDA graph per step when use_graph is set and a
 * stream is given.  The instances' operators, boundary weights, points and
 * sources are concatenated (block-diagonal operators, every instance padded
 * to whole 32-row slices and 128-point tiles); the PCG keeps per-instance
 * dot products, step lengths and convergence tests (Sections 2.3-2.4 for
 * each instance, unchanged).  sa_batch_create takes contexts that have a
 * patch, material and scan and are at the same step; the batch copies their
 * state at its first step and owns it from then on (read it back with
 * sa_batch_get_field); the contexts must outlive the batch.  Options of the
 * batch: precision, pcg_tol, pcg_max_iter, cuda_stream, use_graph (one
 * graph per step), hist_points_per_lane / hist_warps (pairwise sums),
 * precond (fast diagonalization of both solves when every instance has it)
 * and hist_mode (separable sums when every instance's faces allow them, as
 * for one context; with SA_HIST_SEPARABLE otherwise the first
 * sa_batch_step returns SA_ERR_ARG).
 */
/* Errors of the batch calls: SA_ERR_ARG (NULL, n_inst < 1, an instance
 * index or field out of range, options the batch does not support),
 * SA_ERR_STATE (an instance without patch, material or scan, or instances at
 * different steps), SA_ERR_OOM, SA_ERR_CUDA, and from sa_batch_step the
 * sa_step statuses.  *out is owned by the caller (sa_batch_destroy; NULL is
 * a no-op); sa_batch_last_error gives the last message. */
typedef struct sa_batch sa_batch;
sa_status sa_batch_create(sa_ctx* const* insts, int n_inst, const sa_options* o, sa_batch** out);
sa_status sa_batch_step(sa_batch* b, double theta, double dt, int n_steps, sa_step_stats* stats);
/* fields SA_FIELD_THAT, SA_FIELD_F (natural order of instance inst),
 * SA_FIELD_DTDN_LAT, SA_FIELD_TT_BOT; host buffer */
sa_status sa_batch_get_field(sa_batch* b, int inst, int field, double* out, long long count);
/* PCG iterations of the last step per instance (main, bottom projection) */
sa_status sa_batch_get_iters(sa_batch* b, int* main_iters, int* bottom_iters);
/* Autotuner of the history-sum tile (points per lane x warps): times every
 * shape on the batch's data (CUDA events), keeps the fastest and appends the
 * choice to the JSON-lines file cache_path (NULL: no cache), keyed by the
 * batch sizes; a cached choice is reused without timing (*best_ms = -1). */
sa_status sa_batch_autotune(sa_batch* b, const char* cache_path, int* P, int* NW, double* best_ms);
/* Launch shapes of a batch: the history sums (separable product: tile
 * widths of the lateral and bottom tiles, 64 rows each, and units of sources
 * per tile; pairwise sums: points per lane and warps) and the number of
 * blocks of the batched solves (one 1024-thread block per SM at most). */
typedef struct sa_batch_shapes {
    int hist_separable;            /* 1: separable product, 0: pairwise sums          */
    int tj_lat, tj_bot;            /* separable: tile widths (64, 48 or 32)           */
    int units_per_tile;            /* separable: source units per tile (1, 2 or 4)    */
    int hist_P, hist_NW;           /* pairwise: points per lane, warps per block      */
    int pcg_grid;                  /* blocks of the batched PCG launches              */
    double step_ms;                /* sa_batch_tune: time of one step with the chosen */
                                   /* solve grid (ms); -1 when read from the cache    */
} sa_batch_shapes;
/* Tuner of the batch's launch shapes (this project's, no paper counterpart):
 * times every separable tile shape (3 x 3 widths x 1, 2, 4 units; or the
 * pairwise tiles when the faces are not rectangles) on the batch's data with
 * the sources active at step at_step (0: the next step; the work grows with
 * the step, so a mid-run step represents a run), then the solve grid (all SMs, 3/4, 1/2) over whole steps
 * from a saved copy of the batch's state, which is restored afterwards (the
 * simulation does not advance).  The choice is kept by the batch, written to
 * *out and appended to the JSON-lines file cache_path (NULL: no cache),
 * keyed by the batch's sizes and at_step; a cached choice is applied without
 * timing (step_ms = -1).  Needs a batch that has stepped (SA_ERR_STATE);
 * errors SA_ERR_ARG (at_step < 0), SA_ERR_OOM, SA_ERR_CUDA.  Synchronous. */
sa_status sa_batch_tune(sa_batch* b, const char* cache_path, long long at_step,
                        sa_batch_shapes* out);
/* The shapes the batch runs with (out: caller-owned).  Errors: SA_ERR_ARG,
 * SA_ERR_STATE (before the first step). */
sa_status sa_batch_get_shapes(sa_batch* b, sa_batch_shapes* out);
const char* sa_batch_last_error(const sa_batch* b);
void sa_batch_destroy(sa_batch* b);

/* Release every device buffer, graph and stream object of the context
 * (NULL is a no-op). */
void sa_destroy(sa_ctx* ctx);
/* Name of a status ("SA_ERR_ARG", ...); a static string. */
const char* sa_status_str(sa_status s);
/* One-line message of the context's last failure, valid until its next
 * call; "null context" for NULL. */
const char* sa_last_error(const sa_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SA_H */
