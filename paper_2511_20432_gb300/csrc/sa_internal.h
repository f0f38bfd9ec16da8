// Internal declarations shared by the translation units of libsa.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

#include "../../include/sa.h"

// ---------------------------------------------------------------------------
// limits
// ---------------------------------------------------------------------------
#define SA_MAX_DEGREE 3
#define SA_MAX_NLOC ((SA_MAX_DEGREE + 1) * (SA_MAX_DEGREE + 1) * (SA_MAX_DEGREE + 1))
#define SA_MAX_NFACE ((SA_MAX_DEGREE + 1) * (SA_MAX_DEGREE + 1))
// limits of sa_eval_T_noalloc (its fixed scratch array)
#define SA_NOALLOC_MAX_SOURCES 65536
#define SA_NOALLOC_MAX_ELEMENTS 131072

// device error flags (DevStatus::err)
enum {
    SA_DEV_NOT_CONVERGED = 1,
    SA_DEV_BOT_NOT_CONVERGED = 2,
    SA_DEV_TIMEOUT = 4,
    SA_DEV_NAN = 8,
    SA_DEV_BAD_INDEX = 16
};

// Written by kernels, read by the host after a stream synchronisation.
struct DevStatus {
    int err;
    int pcg_iters;            // last main solve
    int bot_iters;            // last bottom solve
    int n_active;             // sources in the sum at the last step
    double rel_res;           // last main solve
    double bot_rel_res;
    int ws_used;              // last main solve started from the learned guess
    int ws_pad;
    double ws_ratio;          // |r0 - A dx| / |r0| of the last learned guess
    long long n;              // step index (device copy)
    long long iters_total;    // accumulated since the last reset by the host
    long long bot_total;
    long long hist_skipped;   // (point, source) pairs the opt-in cutoff dropped
    int iters_max;
    int pad;
    unsigned bar_count[4];    // grid barrier counters (one pair per cooperative kernel slot)
    unsigned bar_gen[4];
};

// Geometry description handed to device kernels by value.
struct DevPatch {
    int p[3];
    int n[3];
    int ne[3];
    const double* U[3];       // knot vectors
    const int* espan[3];      // span index of each element, per direction
    const double4* cw;        // control points (x, y, z, w), natural order
};

// ---------------------------------------------------------------------------
// RAII device buffer
// ---------------------------------------------------------------------------
template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    cudaError_t alloc(size_t count) {
        release();
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc((void**)&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        n = count;
        return cudaSuccess;
    }
};

// Sliced ELLPACK, slice height 32, column-major inside a slice: entry k of
// row r = 32 s + l lives at sptr[s] + 32 k + l.  Padding entries have value
// 0 and column = the row itself (in range).  One warp per slice, lane = row:
// every value/column load is a coalesced 32-wide access and the lanes'
// gathers x[col] are contiguous for banded (tensor-product) matrices.
struct SellDev {
    int n = 0, n_slices = 0;
    long long n_stored = 0;
    DBuf<long long> sptr;     // n_slices + 1
    DBuf<int> col;            // n_stored (absolute columns)
    DBuf<short> col16;        // n_stored (column - row), when every offset fits
    DBuf<int> src;            // n_stored: slot in the source CSR, -1 for padding
    DBuf<int> diag;           // n: storage index of the diagonal entry
    DBuf<unsigned char> hi;   // n_slices: 1 when the slice holds a column >= n
    int dmin = 0, dmax = 0;
};

// Host copy of a SELL pattern (built on the host, kept for batching).
struct SellHost {
    int n = 0, n_slices = 0;
    std::vector<long long> sptr;
    std::vector<int> col, src, diag;
    std::vector<short> col16;   // column - row, filled when every offset fits
    int dmin = 0, dmax = 0;     // extreme column - row offsets (when col16 is filled)
};

// Per slice: 1 when a stored entry has a column >= n, i.e. for the free-row
// operators, a Dirichlet column (padding entries hold a column < n).
inline std::vector<unsigned char> sell_hi_flags(const SellHost& h) {
    std::vector<unsigned char> f(h.n_slices > 0 ? h.n_slices : 1, 0);
    if (h.col.empty()) return f;
    for (int s = 0; s < h.n_slices; ++s)
        for (long long e = h.sptr[s]; e < h.sptr[s + 1]; ++e)
            if (h.col[e] >= h.n) {
                f[s] = 1;
                break;
            }
    return f;
}

// What the kernels need of a SELL operator (no ownership).
struct SellView {
    int n, n_slices;
    const long long* sptr;
    const int* col32;         // null when col16 is used
    const short* col16;
    const unsigned char* hi;  // per slice: holds a column >= n (may be null)
    int dmin, dmax;           // extreme column - row offsets (col16 only)
};

inline SellView sell_view(const SellDev& s) {
    SellView v;
    v.n = s.n;
    v.n_slices = s.n_slices;
    v.sptr = s.sptr.p;
    v.col16 = s.col16.p;
    v.col32 = s.col16.p ? nullptr : s.col.p;
    v.hi = s.hi.p;
    v.dmin = s.dmin;
    v.dmax = s.dmax;
    return v;
}

// Fast-diagonalization preconditioner as the PCG kernel sees it (device
// pointers in the operator precision; m[d] free sizes per direction).
struct FdView {
    bool on;
    int nd;                // 3 (passes 0 1 2f 1 0) or 2 (passes 0 1f 0)
    int m[3];
    const void* U[3];      // m x m row-major: U[a][o] (columns = eigenvectors)
    const void* Ut[3];     // transposes
    const void* lamc[3];   // c_d lambda_d
    double cM;
    const void* S;         // n_free diagonal scaling
    void* Z;               // n_free work vector
    void* Z2;              // second n_free work vector (plane form, 3-D)
};

// Host and device data of one fast-diagonalization preconditioner over an
// nd-dimensional grid of control variables (m[d] per direction, m[2] = 1 for
// nd = 2): eigenvectors U_d (U_d^T M^_d U_d = I), eigenvalues, the diagonals
// of M^_d and K^_d, mean lengths, the scalings of the current (theta, dt).
struct FdData {
    bool ok = false;
    int nd = 3;
    int m[3] = {1, 1, 1};
    double L[3] = {0, 0, 0}, cM = 0, c[3] = {0, 0, 0};
    std::vector<double> U[3], lam[3], md[3], kd[3];
    DBuf<unsigned char> dU[3], dUt[3], dlamc[3], dmd[3], dkd[3], S, Z, Z2;
};

// One face of the separable history evaluation: an axis-aligned rectangle
// whose quadrature points are the tensor grid (A list) x (B list) at the
// fixed coordinate dd along axis axd (coordinates relative: x - x_ref,
// y - y_ref, z - z_top).  List index i = ea * nga + ga, j = eb * ngb + gb;
// the point's output index is q0 + ((eb * nea + ea) * ngb + gb) * nga + ga.
struct SepFace {
    int q0;
    int La, Lb;             // A and B list lengths
    int nga, nea, ngb;
    int axa, axb, axd;      // physical axes (0 x, 1 y, 2 z)
    int a_off, b_off;       // list offsets in the coordinate array
    int flux;               // 1: lateral flux (output s_lat = -sum); 0: bottom T~
    double dd;              // fixed coordinate
    double nsgn;            // outward normal along axd (flux faces), else 1
    int inst;               // instance of a batch (0 for one context)
    int pad;
};

// Separable history plan: faces, tiles (lateral tiles first), the split of
// the sources into units and the partial-sum buffers.
struct SepPlan {
    bool ok = false;
    int tj[2] = {64, 64};          // tile width of lateral / bottom tiles
    int n_tiles[2] = {0, 0};
    int unit = 0, s_max = 0;       // sources per unit; units at the full scan
    std::vector<SepFace> faces_h;
    std::vector<int4> tiles_h;     // (face, i0, j0, 0)
    std::vector<double> coord_h;
    DBuf<SepFace> faces;
    DBuf<int4> tiles;
    DBuf<double> coord64;
    DBuf<float> coord32;
    DBuf<double> part64;           // [tile][unit][64 x 64]
    DBuf<float> part32;
    // opt-in cutoff: largest |sum| per face kind at the last two steps
    // ([kind][step parity], FP32 bit patterns of non-negative values)
    DBuf<float> ref;
};

// Arguments of one PCG solve.  The grid-barrier counter st->bar_count[which]
// must be zero at launch: the step's gather kernel zeroes it on the stream
// the solve runs on.
struct PcgLaunch {
    SellView op;
    const void* val;          // operator values in the path's precision
    const double* val_hi;     // FP64 values (initial residual when r0 == null)
    const double* dinv;
    const void* dinvl;        // dinv in the path's precision (FP32 copy or = dinv)
    const double* b;
    const double* r0;         // given initial residual (x0 = x), or null
    const double* bsq;        // with r0: b_i^2 per row (norm of the right-hand side)
    double* x;
    double* w64;              // FP64 work vectors of length stride: p, r, w, s, u
    void* vpad;               // 2 padded vectors in the path's precision, each
                              // [pad | stride | pad], pad = halo entries; vector k
                              // starts at k (stride + 2 pad)
    int pad;
    size_t stride;
    int variant;              // SA_PCG_AUTO / SA_PCG_SHARED / SA_PCG_GLOBAL
    FdView fd{};              // preconditioner (fd.on false: Jacobi)
    double* partials;         // 12 x grid
    const float* dx0;         // proposed increment (mode 1), or null
    const double* dx0_scale;  // device scalar multiplying dx0
    DevStatus* st;
    int which;
    double tol;
    int max_iter;
    int grid;                 // 1: one block, no grid barrier
    int block = 0;            // threads per block (0: 1024)
    int ksplit;               // warps per SELL slice in the SpMV (1, 2, 4, 8)
    // shared-memory variant, optional: with x final, dir_out[i] = x_i - dir_old[i]
    // and dir_out[n + i] = x_i in the operator precision (the Dirichlet
    // increments the theta right-hand side needs)
    const double* dir_old = nullptr;
    void* dir_out = nullptr;
    // the right-hand side kernel's per-slice (b^2, r0^2) sums (npart_n
    // slices) and its Z = S r0 for the fast diagonalization: the solve then
    // needs no exchange for the norms (null: it forms them itself)
    const float* npart = nullptr;
    int npart_n = 0;
    // shared-memory variant, optional: the step's finalize after the solve
    // (That[n_free + d] = g[d], F0 = F1, the step counters); x must be That
    const double* fin_F1 = nullptr;
    double* fin_F0 = nullptr;
    const double* fin_g = nullptr;
    double* fin_That = nullptr;
    int fin_n_dof = 0, fin_n_dir = 0;
};

// ---------------------------------------------------------------------------
// the context
// ---------------------------------------------------------------------------
// Steps captured in one CUDA graph when a call asks for at least that many.
constexpr int kGraphSteps = 16;

struct sa_mlp;
cudaError_t mlp_forward(sa_mlp* m, const void* X, int rows, const float** out, cudaStream_t s);
int mlp_n_in(const sa_mlp* m);
int mlp_n_out(const sa_mlp* m);
int mlp_prepare(sa_mlp* m, int rows);
cudaError_t launch_norm(int n, const double* r, double* part, double* norm, cudaStream_t s);
cudaError_t launch_ws_input(int n_in, const int* idx, const double* r0, const double* norm,
                            void* out, cudaStream_t s);
cudaError_t launch_ws_target(int n, const double* xnew, const double* xold, const double* norm,
                             void* out, cudaStream_t s);

struct sa_ctx {
    sa_options opt;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    bool poisoned = false;
    int num_sms = 0;

    // patch (host copy)
    bool has_patch = false;
    int p[3] = {0, 0, 0}, n[3] = {0, 0, 0}, ne[3] = {0, 0, 0};
    std::vector<double> U[3];
    std::vector<int> espan[3];
    std::vector<int> elo[3], ehi[3];   // element range touching each 1-D basis function
    std::vector<double> ctrl, w;
    int face_kind[6] = {SA_FACE_NEUMANN, SA_FACE_NEUMANN, SA_FACE_NEUMANN, SA_FACE_NEUMANN,
                        SA_FACE_DIRICHLET, SA_FACE_NONE};
    int n_dof = 0, n_free = 0, n_dir = 0, n_elem = 0;
    int seam = -1;            // closed direction (merged end layers), or -1
    int nd[3] = {0, 0, 0};    // control-variable grid (n, minus one layer on the seam)
    std::vector<int> cmap;    // control point (natural) -> control variable (natural)
    std::vector<int> perm;    // control variable: natural -> internal (free first, then Dirichlet)
    std::vector<int> iperm;   // internal -> natural
    double z_top = 0, x_ref = 0, y_ref = 0, length_scale = 1;

    // material
    bool has_material = false;
    double k = 0, rho = 0, cp = 0, Tc = 0;

    // scan
    bool has_scan = false;
    std::vector<double> path;
    std::vector<unsigned char> seg_on;
    double power = 0, absorptivity = 0, speed = 0, spot_radius = 0;
    double src_dt = 0;        // dt the sources were discretised with (0: not yet)
    int n_src = 0;
    double E = 0;

    // stepping
    long long n_step = 0;     // host mirror of the step index
    double op_dt = 0, op_theta = -1;   // operator currently built
    bool state_dirty_graph = true;
    cudaGraphExec_t graph_exec = nullptr;    // one step
    cudaGraphExec_t graph_multi = nullptr;   // kGraphSteps steps

    // ---- device: geometry -------------------------------------------------
    DBuf<double> dU[3];
    DBuf<int> despan[3];
    DBuf<double4> dcw;
    DBuf<int> dperm;          // control point (natural) -> internal control variable
    DevPatch dp;

    // quadrature points (canonical order)
    int q_lat = 0, q_bot = 0;
    DBuf<double> lat64;       // SoA: x, y, z, nx, ny, nz, wdS   (7 * q_lat)
    DBuf<double> bot64;       // SoA: x, y, z, wdS               (4 * q_bot)
    DBuf<float> lat32;        // SoA: px, py, dz2, nzdz, nx, ny  (6 * q_lat)
    DBuf<float> bot32;        // SoA: px, py, dz2                (3 * q_bot)

    // W_lat: rows = control variables touched by lateral points
    int wlat_rows = 0;
    DBuf<int> wlat_rowdof, wlat_ptr, wlat_col;
    DBuf<double> wlat_val;
    // W_bot: rows = Dirichlet control variables (bottom-local index)
    DBuf<int> wbot_ptr, wbot_col;
    DBuf<double> wbot_val;
    // M_bot (Dirichlet x Dirichlet, bottom-local indices) and its Jacobi inverse
    long long nnz_mbot = 0;
    DBuf<int> mbot_ptr, mbot_col;
    DBuf<double> mbot_val, mbot_dinv;
    SellDev mbot_s;
    DBuf<double> mbot_sval;
    DBuf<float> mbot_sval32;

    // M, K: CSR over all control variables, natural order
    long long nnz = 0;
    DBuf<long long> mk_ptr;
    DBuf<int> mk_col;
    DBuf<double> M, K;
    // free-free operator A = M/dt + theta K, internal indices (SELL)
    long long nnz_a = 0;
    SellDev a_s;
    DBuf<double> a_val, a_dinv;
    DBuf<float> a_val32;
    // free rows of M and K over all columns (internal indices), for the
    // theta right-hand side (SELL, unit rho c_p and k)
    SellDev r_s;
    DBuf<double> r_M, r_K;
    DBuf<float> r_M32, r_K32;
    // mixed path, slices without Dirichlet columns: 16-bit column offsets
    // from the row, and M as bf16 (M enters only b, whose norm scales the
    // stopping test); empty when an offset does not fit
    DBuf<short> r_col16lo;
    DBuf<unsigned short> r_M16;
    int r_dir_sl0 = 0, r_dir_sl1 = -1;   // slices with Dirichlet columns lie in [sl0, sl1)
    // sa_eval_T_superposed (this context first in the list): points, the sum
    // and one context's values, n entries each (3 n for the points)
    DBuf<double> sup_pts, sup_acc, sup_tmp;

    // ---- device: scan and history ------------------------------------------
    DBuf<double2> src_pos;    // relative (x - x_ref, y - y_ref)
    DBuf<double4> src64T, src64F;   // (sx, sy, a, c) / (sx, sy, a, g)
    DBuf<float4> src32T, src32F;    // (sx, sy, -a log2 e, log2 c / log2 g)
    DBuf<double> s_lat;       // dT~/dn at lateral points
    DBuf<double> tt_bot;      // T~ at bottom points

    // ---- device: state and solver work ---------------------------------------
    DBuf<double> That;        // internal order (n_dof)
    DBuf<double> F0, F1;      // internal order (n_dof)
    DBuf<double> gnew, bbot;  // n_dir
    DBuf<double> r0bot, bsqbot;   // n_dir: projection's initial residual and b_bot^2
    DBuf<double> rhs, r0, bsq;   // n_free
    DBuf<double> dirv;           // 2 n_dir: Dirichlet increments for the theta RHS
    DBuf<double> work64;                 // PCG work: 5 x nwork (FP64)
    DBuf<unsigned char> workpad;         // PCG padded vectors (2 x (nwork + 2 pad) x VT)
    int work_pad = 0;
    DBuf<float> a_dinv32, mbot_dinv32;   // Jacobi inverse in FP32 (mixed path)
    size_t nwork = 0;
    DBuf<double> dev64;                  // T^n - T_c (n_dof)
    DBuf<float> dev32;
    DBuf<double> partials;    // 4 * max grid
    DBuf<float> npart;        // per slice of the free rows: (b^2, r0^2) sums of the step's
                              // right-hand side, for the main solve
    DBuf<float> npart_bot;    // per gather warp of the bottom rows: the same for the projection
    DBuf<DevStatus> st;
    int pcg_grid = 0, pcg_block = 0;
    int hist_P = 0, hist_W = 0;

    // ---- device: set-up and evaluation helpers ---------------------------------
    DBuf<int> d_elo[3], d_ehi[3];   // element range touching each 1-D basis function
    DBuf<int> d_iperm_free;         // internal free index -> natural index
    bool state_init = false;
    DBuf<double> ecent;             // physical element centres (eval initial guess)
    DBuf<double4> evT, evF;         // FP64 source coefficients at the current step
    DBuf<double> eval_pts, eval_out;
    DBuf<float> ecent32;            // FP32 element centres (the eval's search)

    // host copies of the patterns (for sa_batch)
    SellHost a_h, r_h, mbot_h;
    std::vector<int> wlat_rowdof_h, wlat_ptr_h, wlat_col_h, wbot_ptr_h, wbot_col_h;

    // fast-diagonalization preconditioners (csrc/sa_fd.cu): the main solve
    // (3-D) and the bottom projection (2-D)
    FdData fdm, fdb;

    // separable history sums (csrc/sa_sep.cu)
    SepPlan sep;
    int face_q0[2][7] = {};          // first point of each face: lateral, bottom

    // extrapolated initial guesses (sa_options::initial_guess)
    DBuf<double> x_prev;             // T^{n-1}: free part, then the Dirichlet part
    DBuf<float> dx_extrap;           // n_free: proposed increment T^n - T^{n-1}
    DBuf<double> one;                // device scalar 1.0 (scale of dx_extrap)

    // learned warm start and training-data recorder
    sa_mlp* ws_net = nullptr;
    int ws_n_in = 0;
    DBuf<int> ws_idx;
    DBuf<double> ws_norm, ws_part, ws_xold;
    DBuf<unsigned char> ws_in;       // BF16 input row (n_in)
    void* rec_X = nullptr;           // recorder: caller's device buffers (BF16)
    void* rec_Y = nullptr;
    int rec_cap = 0, rec_count = 0, rec_n_in = 0;
    DBuf<int> rec_idx;

    // stage timing (sa_options::stage_timing)
    cudaEvent_t ev[SA_N_STAGES + 1] = {};
    // second stream of a step: the bottom chain (history of the bottom
    // points, b_bot, the projection) runs beside the lateral chain
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_hist = nullptr;   // the bottom history sums done (the lateral ones wait)
    cudaEvent_t ev_lat = nullptr;    // the lateral gather done (the Dirichlet-column right-hand side waits)
    double stage_ms[SA_N_STAGES] = {};
    long long stage_steps = 0;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
sa_status sa_fail(sa_ctx* c, sa_status s, const char* fmt, ...);
sa_status sa_prepare(sa_ctx* c, double theta, double dt);
sa_status sa_cuda_fail(sa_ctx* c, cudaError_t e, const char* where);

#define SA_CUDA(ctx, call)                                           \
    do {                                                             \
        cudaError_t e__ = (call);                                    \
        if (e__ != cudaSuccess) return sa_cuda_fail(ctx, e__, #call); \
    } while (0)

#define SA_ALLOC(ctx, buf, count)                                                      \
    do {                                                                               \
        cudaError_t e__ = (buf).alloc(count);                                          \
        if (e__ != cudaSuccess) {                                                      \
            cudaGetLastError();                                                        \
            return sa_fail(ctx, e__ == cudaErrorMemoryAllocation ? SA_ERR_OOM : SA_ERR_CUDA, \
                           "allocation of %s (%zu elements): %s", #buf, (size_t)(count), \
                           cudaGetErrorString(e__));                                   \
        }                                                                              \
    } while (0)

// ---------------------------------------------------------------------------
// entry points of the kernel translation units
// ---------------------------------------------------------------------------
// sa_geom.cu
cudaError_t launch_face_points(const DevPatch& dp, int face, int pa, int pb, int nea, int neb,
                               const int* dof_of_local,  // unused placeholder (nullptr)
                               const double* xg_a, const double* wg_a, const double* xg_b,
                               const double* wg_b, int q_offset, double* pts64, int q_stride,
                               int with_normal, const int* slot_of_entry, double* w_val,
                               double* coo_R, int* coo_dof, const int* perm, cudaStream_t s);
cudaError_t launch_element_local(const DevPatch& dp, double rho_cp, double k, const double* xg,
                                 const double* wg, double* Mloc, double* Kloc, int* bad_jac,
                                 cudaStream_t s);
cudaError_t launch_mk_gather(const DevPatch& dp, const long long* ptr, const int* col,
                             const int* const* elo, const int* const* ehi, const double* Mloc,
                             const double* Kloc, double* M, double* K, cudaStream_t s);
cudaError_t launch_merge_csr(long long n, const long long* sptr, const int* sidx, const double* Mc,
                             const double* Kc, double* M, double* K, cudaStream_t s);
cudaError_t launch_elem_centers(const DevPatch& dp, double* ecent, cudaStream_t s);
cudaError_t launch_mbot_fill(int n_rows, const int* mptr, const int* mcol, const int* wptr,
                             const int* wcol, const double* wval, const int* coo_dof,
                             const double* coo_R, int nfb, int n_free, double* mval,
                             double* dinv, cudaStream_t s);
cudaError_t launch_sell_fill(long long n_stored, const int* src, const double* in1, double s1,
                            const double* in2, double s2, double* out, cudaStream_t s);
cudaError_t launch_to_f32(long long n, const double* in, float* out, cudaStream_t s);
cudaError_t launch_sell_dinv(int n, const int* diag, const double* val, double* dinv,
                             cudaStream_t s);
cudaError_t launch_points32(int q_lat, int q_bot, const double* lat64, const double* bot64,
                            double x_ref, double y_ref, double z_top, float* lat32,
                            float* bot32, cudaStream_t s);

// sa_history.cu
cudaError_t launch_prologue(const DevStatus* st_in, long long n_explicit, DevStatus* st_out,
                            int n_src, const double2* pos, double dt, double alpha,
                            double r2_8a, double coefE, int precision, double4* s64T,
                            double4* s64F, float4* s32T, float4* s32F, cudaStream_t s);
cudaError_t launch_history(int precision, int P, int warps, DevStatus* st, int q_lat,
                           int q_bot, const float* lat32, const float* bot32,
                           const double* lat64, const double* bot64, double x_ref,
                           double y_ref, double z_top, const float4* s32F,
                           const float4* s32T, const double4* s64F, const double4* s64T,
                           double* s_lat, double* tt_bot, cudaStream_t s, int part = 0);
// sa_sep.cu
sa_status sep_setup(sa_ctx* c);
sa_status sep_alloc(sa_ctx* c);
cudaError_t launch_sep(sa_ctx* c, int part, double dt, cudaStream_t s);
// Batched instances (each with its plan): one plan over all of them, faces
// shifted to the batch's point offsets, one unit per tile.  False when an
// instance has no separable plan.
bool sep_batch_plan(const std::vector<sa_ctx*>& insts, const std::vector<int>& qlat_off,
                    const std::vector<int>& qbot_off, int precision, SepPlan& P, int tj_lat = 0,
                    int tj_bot = 0, int s_max = 1);
cudaError_t launch_sep_batch(const SepPlan& P, int precision, DevStatus* st, const int* n_active,
                             const int* src_off, const float4* s32F, const float4* s32T,
                             const double4* s64F, const double4* s64T, double* s_lat,
                             double* tt_bot, cudaStream_t s);
// T = T~ + T^ at points; ecent32 (FP32 copy of the element centres) and
// s32T (FP32 source coefficients) are optional: with them the search and the
// source sum run in FP32 (mixed contexts).
// flux != null: the heat-loss rates -k n . grad T~ (into T_out) and
// -k n . grad T^ (into flux->q_hat) at the points with unit normals nrm.
struct EvalFlux {
    const double* nrm;
    const double4* s64F;
    const float4* s32F;
    double k;
    double* q_hat;
};
cudaError_t launch_eval_points(const DevPatch& dp, const double* pts, int n, const double* ecent,
                               const int* perm, const double* That, const double4* s64T,
                               int n_active, double x_ref, double y_ref, double z_top,
                               double scale, double* T_out, cudaStream_t s,
                               const float* ecent32 = nullptr, const float4* s32T = nullptr,
                               const EvalFlux* flux = nullptr);

// sa_solve.cu
// With the bottom rows of the gather, optionally the bottom projection's
// initial residual r0 = b_bot - M_bot g0 (FP64) and b_bot^2.
struct BotResid {
    const int* mptr = nullptr;    // M_bot CSR over the Dirichlet control variables
    const int* mcol = nullptr;
    const double* mval = nullptr;
    const double* g0 = nullptr;   // initial guess
    double* r0 = nullptr;
    double* bsq = nullptr;
    // for the projection solve (null: off): Z = S r0 of its 2-D fast
    // diagonalization (FP32 when f32, else FP64) and per warp of the bottom
    // rows the sums of b^2 and r0^2 ([warp][2])
    const void* fdS = nullptr;
    void* fdZ = nullptr;
    int f32 = 0;
    float* npart = nullptr;
};
cudaError_t launch_gather(int wlat_rows, const int* wlat_rowdof, const int* wlat_ptr,
                          const int* wlat_col, const double* wlat_val, const double* s_lat,
                          double k, int n_dir, const int* wbot_ptr, const int* wbot_col,
                          const double* wbot_val, const double* tt_bot, double Tc, double* F1,
                          double* bbot, int n_dof, const double* That, double* dev64,
                          float* dev32, cudaStream_t s, int part = 0,
                          const BotResid& br = BotResid(), DevStatus* st = nullptr);
cudaError_t launch_theta_rhs(int precision, const SellView& op, const void* Kval,
                             const void* Mval, const void* dev, const double* That,
                             const double* gnew, const double* F0, const double* F1,
                             double inv_dt_rhocp, double k, double theta, double Tc, double* r0,
                             double* bsq, int n_dir, void* dir_scratch, cudaStream_t s, int only = 0,
                             bool dir_ready = false, const void* fdS = nullptr, void* fdZ = nullptr,
                             float* npart = nullptr, const short* col16lo = nullptr,
                             const unsigned short* M16 = nullptr, int sl0 = 0, int sl1 = -1);
cudaError_t launch_pcg(int precision, const PcgLaunch& L, cudaStream_t s);
cudaError_t launch_to_bf16(long long n, const double* in, unsigned short* out, cudaStream_t s);
cudaError_t launch_extrap(int n_free, int n_dir, const double* That, double* Tprev, float* dx0,
                          double* gprev, double* g0, cudaStream_t s);
sa_status fd_setup(sa_ctx* c);
cudaError_t fd_prepare(sa_ctx* c, double theta, double dt, cudaStream_t s);
FdView fd_view(const sa_ctx* c, const FdData& f);
void gauss_legendre(int n, double* x, double* w);
// Whether the shared-memory PCG of this launch keeps its rows in shared memory.
bool pcg_shared_fits(int precision, const PcgLaunch& L);
cudaError_t launch_finalize(int n_dir, int n_free, int n_dof, const double* gnew, double* That,
                            const double* F1, double* F0, DevStatus* st, cudaStream_t s);
int pcg_block_size();
const void* pcg_kernel_ptr(int precision);
