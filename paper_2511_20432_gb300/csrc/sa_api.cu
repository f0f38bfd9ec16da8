// C ABI of libsa: host-side validation, set-up (element lists, CSR
// patterns, Dirichlet elimination order, scan discretisation) and the
// per-step launch sequence.  See include/sa.h for the contract of each call.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <numeric>

#include "sa_async.cuh"
#include "sa_internal.h"


// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
sa_status sa_fail(sa_ctx* c, sa_status s, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

sa_status sa_cuda_fail(sa_ctx* c, cudaError_t e, const char* where) {
    if (c) {
        c->poisoned = true;
        c->err = std::string(where) + ": " + cudaGetErrorString(e);
    }
    return SA_ERR_CUDA;
}

// Gauss-Legendre nodes and weights on [-1, 1] for 1..4 points (closed forms).
void gauss_legendre(int n, double* x, double* w) {
    switch (n) {
        case 1:
            x[0] = 0.0;
            w[0] = 2.0;
            break;
        case 2:
            x[0] = -1.0 / std::sqrt(3.0);
            x[1] = -x[0];
            w[0] = w[1] = 1.0;
            break;
        case 3:
            x[0] = -std::sqrt(0.6);
            x[1] = 0.0;
            x[2] = std::sqrt(0.6);
            w[0] = w[2] = 5.0 / 9.0;
            w[1] = 8.0 / 9.0;
            break;
        default: {
            const double a = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
            const double b = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
            const double wa = (18.0 + std::sqrt(30.0)) / 36.0;
            const double wb = (18.0 - std::sqrt(30.0)) / 36.0;
            x[0] = -b;
            x[1] = -a;
            x[2] = a;
            x[3] = b;
            w[0] = wb;
            w[1] = wa;
            w[2] = wa;
            w[3] = wb;
        }
    }
}

namespace {

bool is_fin(double v) { return std::isfinite(v); }

sa_status check_usable(sa_ctx* c) {
    if (!c) return SA_ERR_ARG;
    if (c->poisoned) return sa_fail(c, SA_ERR_STATE, "context poisoned by an earlier CUDA error: %s", c->err.c_str());
    return SA_OK;
}

int nat(const sa_ctx* c, int i, int j, int k) { return (k * c->n[1] + j) * c->n[0] + i; }

// Build one CSR (rows given as internal/bottom-local indices) from entries
// (row, q) listed in point-major order; returns slot of every entry.
void build_w_csr(int n_rows, const std::vector<int>& erow, const std::vector<int>& ecol,
                 std::vector<int>& ptr, std::vector<int>& col, std::vector<int>& slot) {
    ptr.assign(n_rows + 1, 0);
    for (int r : erow) ptr[r + 1]++;
    for (int r = 0; r < n_rows; ++r) ptr[r + 1] += ptr[r];
    col.assign(erow.size(), 0);
    slot.assign(erow.size(), 0);
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (size_t e = 0; e < erow.size(); ++e) {
        const int s = fill[erow[e]]++;
        col[s] = ecol[e];
        slot[e] = s;
    }
}

// SELL-32 layout of a row list: rows r = 0..n-1 with entries
// (col, src) in [ptr[r], ptr[r+1]); diag = storage index of col == diag_col[r]
// (diag_col may be empty: no diagonal needed).
void build_sell(int n, const std::vector<long long>& ptr, const std::vector<int>& col,
                const std::vector<int>& src, const std::vector<int>& diag_col, SellHost& out) {
    out.n = n;
    out.n_slices = (n + 31) / 32;
    out.sptr.assign(out.n_slices + 1, 0);
    for (int s = 0; s < out.n_slices; ++s) {
        long long w = 0;
        for (int l = 0; l < 32; ++l) {
            const int r = s * 32 + l;
            if (r < n) w = std::max(w, ptr[r + 1] - ptr[r]);
        }
        out.sptr[s + 1] = out.sptr[s] + 32 * w;
    }
    const long long tot = out.sptr[out.n_slices];
    out.col.assign(tot, 0);
    out.src.assign(tot, -1);
    out.diag.assign(std::max(n, 1), 0);
    for (int s = 0; s < out.n_slices; ++s) {
        const long long w = (out.sptr[s + 1] - out.sptr[s]) / 32;
        for (int l = 0; l < 32; ++l) {
            const int r = s * 32 + l;
            for (long long k = 0; k < w; ++k) {
                const long long e = out.sptr[s] + 32 * k + l;
                if (r < n && ptr[r] + k < ptr[r + 1]) {
                    const long long t = ptr[r] + k;
                    out.col[e] = col[t];
                    out.src[e] = src[t];
                    if (!diag_col.empty() && col[t] == diag_col[r]) out.diag[r] = (int)e;
                } else {
                    out.col[e] = r < n ? (diag_col.empty() ? 0 : diag_col[r]) : 0;
                    out.src[e] = -1;
                }
            }
        }
    }
    // 16-bit offsets from the row (padding lanes past n use row n-1)
    bool fits = n > 0;
    out.col16.assign(tot, 0);
    for (int s = 0; s < out.n_slices && fits; ++s) {
        const long long w = (out.sptr[s + 1] - out.sptr[s]) / 32;
        for (int l = 0; l < 32 && fits; ++l) {
            const int r = std::min(s * 32 + l, n - 1);
            for (long long k = 0; k < w; ++k) {
                const long long e = out.sptr[s] + 32 * k + l;
                const long long d = (s * 32 + l < n) ? (long long)out.col[e] - r : 0;
                if (d < -32768 || d > 32767) {
                    fits = false;
                    break;
                }
                out.col16[e] = (short)d;
            }
        }
    }
    if (!fits) out.col16.clear();
    out.dmin = out.dmax = 0;
    for (short d : out.col16) {
        out.dmin = std::min(out.dmin, (int)d);
        out.dmax = std::max(out.dmax, (int)d);
    }
}

template <class T>
cudaError_t upload(DBuf<T>& b, const std::vector<T>& v) {
    cudaError_t e = b.alloc(v.size());
    if (e != cudaSuccess) return e;
    if (v.empty()) return cudaSuccess;
    return cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

#define SA_UPLOAD_SELL(ctx, dev, host)          \
    do {                                          \
        (dev).n = (host).n;                       \
        (dev).n_slices = (host).n_slices;         \
        (dev).n_stored = (long long)(host).col.size(); \
        (dev).dmin = (host).dmin;                 \
        (dev).dmax = (host).dmax;                 \
        SA_UPLOAD(ctx, (dev).sptr, (host).sptr);  \
        if ((host).col16.empty())                 \
            SA_UPLOAD(ctx, (dev).col, (host).col);    \
        else                                      \
            SA_UPLOAD(ctx, (dev).col16, (host).col16); \
        SA_UPLOAD(ctx, (dev).src, (host).src);    \
        SA_UPLOAD(ctx, (dev).diag, (host).diag);  \
        SA_UPLOAD(ctx, (dev).hi, sell_hi_flags(host)); \
    } while (0)

#define SA_UPLOAD(ctx, buf, vec)                                                              \
    do {                                                                                      \
        cudaError_t e__ = upload(buf, vec);                                                   \
        if (e__ != cudaSuccess) {                                                             \
            cudaGetLastError();                                                               \
            return e__ == cudaErrorMemoryAllocation                                           \
                       ? sa_fail(ctx, SA_ERR_OOM, "allocation of %s failed", #buf)            \
                       : sa_cuda_fail(ctx, e__, "upload " #buf);                              \
        }                                                                                     \
    } while (0)

// Self-test kernels: waits that nothing completes (bounded, flag on give-up).
__global__ void k_selftest_barrier(unsigned* count, int* err) {
    if (blockIdx.x == 1) return;    // leaves without arriving
    unsigned nb = 0;
    sa_dev::count_barrier(count, nb, err, SA_DEV_TIMEOUT);
}

__global__ void k_selftest_mbarrier(int* err) {
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        sa_dev::mbar_init(&bar, 1);   // expects one arrival; none comes
        sa_dev::mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !sa_dev::mbar_wait_bounded(&bar, 0)) atomicOr(err, SA_DEV_TIMEOUT);
}

}  // namespace

// Captured step graphs depend on the operator, the warm start and the
// options: dropped whenever one of them changes.
void drop_graphs(sa_ctx* c) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph_multi) cudaGraphExecDestroy(c->graph_multi);
    c->graph_exec = nullptr;
    c->graph_multi = nullptr;
}

extern "C" {

void sa_options_default(sa_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = SA_FP64;
    o->pcg_tol = 1e-10;
    o->pcg_max_iter = 2000;
    o->half_space_factor = 2.0;
    o->cuda_stream = nullptr;
    o->use_graph = 0;
    o->device = -1;
    o->hist_points_per_lane = 0;
    o->hist_warps = 0;
}

sa_status sa_selftest_waits(int* barrier_flagged, int* mbarrier_flagged) {
    int* d = nullptr;   // [0] barrier counter, [1] status of (1), [2] status of (2)
    if (cudaMalloc((void**)&d, 3 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return SA_ERR_CUDA;
    }
    int h[3] = {0, 0, 0};
    cudaError_t e = cudaMemset(d, 0, 3 * sizeof(int));
    if (e == cudaSuccess) {
        k_selftest_barrier<<<2, 32>>>((unsigned*)d, d + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_selftest_mbarrier<<<1, 32>>>(d + 2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SA_ERR_CUDA;
    }
    if (barrier_flagged) *barrier_flagged = (h[1] & SA_DEV_TIMEOUT) ? 1 : 0;
    if (mbarrier_flagged) *mbarrier_flagged = (h[2] & SA_DEV_TIMEOUT) ? 1 : 0;
    return SA_OK;
}

const char* sa_status_str(sa_status s) {
    switch (s) {
        case SA_OK: return "SA_OK";
        case SA_ERR_ARG: return "SA_ERR_ARG";
        case SA_ERR_GEOMETRY: return "SA_ERR_GEOMETRY";
        case SA_ERR_STATE: return "SA_ERR_STATE";
        case SA_ERR_CUDA: return "SA_ERR_CUDA";
        case SA_ERR_OOM: return "SA_ERR_OOM";
        case SA_ERR_NOT_CONVERGED: return "SA_ERR_NOT_CONVERGED";
        case SA_ERR_TIMEOUT: return "SA_ERR_TIMEOUT";
        case SA_ERR_NAN: return "SA_ERR_NAN";
    }
    return "SA_ERR_UNKNOWN";
}

const char* sa_last_error(const sa_ctx* c) { return c ? c->err.c_str() : "null context"; }

sa_status sa_create(const sa_options* o, sa_ctx** out) {
    if (!out) return SA_ERR_ARG;
    *out = nullptr;
    sa_options opt;
    if (o)
        opt = *o;
    else
        sa_options_default(&opt);
    if (opt.precision != SA_FP64 && opt.precision != SA_MIXED) return SA_ERR_ARG;
    if (!(opt.pcg_tol > 0.0) || opt.pcg_max_iter <= 0) return SA_ERR_ARG;
    if (!(opt.half_space_factor > 0.0) || !is_fin(opt.half_space_factor)) return SA_ERR_ARG;
    if (opt.pcg_variant < SA_PCG_AUTO || opt.pcg_variant > SA_PCG_GLOBAL) return SA_ERR_ARG;
    if (opt.initial_guess != SA_GUESS_PREVIOUS && opt.initial_guess != SA_GUESS_EXTRAPOLATE)
        return SA_ERR_ARG;
    if (opt.precond < SA_PRECOND_AUTO || opt.precond > SA_PRECOND_FD) return SA_ERR_ARG;
    if (opt.hist_mode < SA_HIST_AUTO || opt.hist_mode > SA_HIST_SEPARABLE) return SA_ERR_ARG;
    if (opt.hist_points_per_lane != 0 && opt.hist_points_per_lane != 1 &&
        opt.hist_points_per_lane != 2 && opt.hist_points_per_lane != 4)
        return SA_ERR_ARG;
    if (opt.hist_warps != 0 && opt.hist_warps != 4 && opt.hist_warps != 8) return SA_ERR_ARG;
    if (!(opt.hist_cutoff >= 0.0 && opt.hist_cutoff < 1.0)) return SA_ERR_ARG;
    sa_ctx* c = new sa_ctx();
    c->opt = opt;
    if (opt.device >= 0) {
        cudaError_t e = cudaSetDevice(opt.device);
        if (e != cudaSuccess) {
            delete c;
            return SA_ERR_CUDA;
        }
    }
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        delete c;
        return SA_ERR_CUDA;
    }
    c->stream = (cudaStream_t)opt.cuda_stream;
    if (c->st.alloc(1) != cudaSuccess) {
        delete c;
        return SA_ERR_OOM;
    }
    if (cudaMemset(c->st.p, 0, sizeof(DevStatus)) != cudaSuccess) {
        delete c;
        return SA_ERR_CUDA;
    }
    if (opt.stage_timing)
        for (int i = 0; i <= SA_N_STAGES; ++i)
            if (cudaEventCreate(&c->ev[i]) != cudaSuccess) {
                delete c;
                return SA_ERR_CUDA;
            }
    // the bottom chain gets the higher priority: its projection then runs
    // beside the lateral history sums instead of after them
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (!opt.stage_timing &&
        (cudaStreamCreateWithPriority(&c->aux, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_hist, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_lat, cudaEventDisableTiming) != cudaSuccess)) {
        cudaGetLastError();
        if (c->aux) cudaStreamDestroy(c->aux);
        if (c->ev_fork) cudaEventDestroy(c->ev_fork);
        if (c->ev_join) cudaEventDestroy(c->ev_join);
        if (c->ev_hist) cudaEventDestroy(c->ev_hist);
        if (c->ev_lat) cudaEventDestroy(c->ev_lat);
        delete c;
        return SA_ERR_CUDA;
    }
    c->hist_P = opt.hist_points_per_lane ? opt.hist_points_per_lane : 4;
    c->hist_W = opt.hist_warps ? opt.hist_warps : 8;
    *out = c;
    return SA_OK;
}

void sa_destroy(sa_ctx* c) {
    if (!c) return;
    drop_graphs(c);
    for (int i = 0; i <= SA_N_STAGES; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_hist) cudaEventDestroy(c->ev_hist);
    if (c->ev_lat) cudaEventDestroy(c->ev_lat);
    if (c->aux) cudaStreamDestroy(c->aux);
    delete c;
}

sa_status sa_set_boundary(sa_ctx* c, const int face_kind[6]) {
    sa_status s = check_usable(c);
    if (s) return s;
    if (!face_kind) return sa_fail(c, SA_ERR_ARG, "face_kind is NULL");
    if (c->has_patch) return sa_fail(c, SA_ERR_STATE, "sa_set_boundary after sa_create_patch");
    for (int f = 0; f < 6; ++f)
        if (face_kind[f] < SA_FACE_NONE || face_kind[f] > SA_FACE_DIRICHLET)
            return sa_fail(c, SA_ERR_ARG, "face_kind[%d] = %d", f, face_kind[f]);
    std::memcpy(c->face_kind, face_kind, sizeof(c->face_kind));
    return SA_OK;
}

sa_status sa_set_material(sa_ctx* c, double k, double rho, double cp, double T_c) {
    sa_status s = check_usable(c);
    if (s) return s;
    if (!(k > 0) || !(rho > 0) || !(cp > 0) || !is_fin(k) || !is_fin(rho) || !is_fin(cp) ||
        !is_fin(T_c))
        return sa_fail(c, SA_ERR_ARG, "material k=%g rho=%g cp=%g T_c=%g", k, rho, cp, T_c);
    if (c->has_material && c->n_step > 0 && (k != c->k || rho != c->rho || cp != c->cp))
        return sa_fail(c, SA_ERR_STATE, "material changed after stepping");
    c->k = k;
    c->rho = rho;
    c->cp = cp;
    c->Tc = T_c;
    c->has_material = true;
    c->op_theta = -1;   // operator depends on rho c_p and k
    return SA_OK;
}

sa_status sa_set_scan(sa_ctx* c, const double* path_xyz, int nv, const unsigned char* seg_on,
                      double power, double absorptivity, double speed, double spot_radius) {
    sa_status s = check_usable(c);
    if (s) return s;
    if (!path_xyz || nv < 2) return sa_fail(c, SA_ERR_ARG, "scan needs at least 2 vertices");
    if (!(power >= 0) || !(absorptivity >= 0) || !(speed > 0) || !(spot_radius > 0) ||
        !is_fin(power) || !is_fin(absorptivity) || !is_fin(speed) || !is_fin(spot_radius))
        return sa_fail(c, SA_ERR_ARG, "scan parameters P=%g A=%g v=%g r=%g", power, absorptivity,
                       speed, spot_radius);
    for (int i = 0; i < 3 * nv; ++i)
        if (!is_fin(path_xyz[i])) return sa_fail(c, SA_ERR_ARG, "non-finite path vertex");
    if (c->n_step > 0) return sa_fail(c, SA_ERR_STATE, "sa_set_scan after stepping");
    c->path.assign(path_xyz, path_xyz + 3 * nv);
    c->seg_on.assign(nv - 1, 1);
    if (seg_on)
        for (int i = 0; i < nv - 1; ++i) c->seg_on[i] = seg_on[i] ? 1 : 0;
    c->power = power;
    c->absorptivity = absorptivity;
    c->speed = speed;
    c->spot_radius = spot_radius;
    c->has_scan = true;
    c->src_dt = 0;
    c->n_src = 0;
    return SA_OK;
}

sa_status sa_create_patch(sa_ctx* c, const int degree[3], const int n_ctrl[3],
                          const double* ctrl_xyz, const double* weights,
                          const double* const knots[3], const int n_knots[3], int seam_dir) {
    sa_status st = check_usable(c);
    if (st) return st;
    if (c->has_patch) return sa_fail(c, SA_ERR_STATE, "patch already created");
    if (!degree || !n_ctrl || !ctrl_xyz || !knots || !n_knots)
        return sa_fail(c, SA_ERR_ARG, "NULL argument");
    // ---- validation ------------------------------------------------------
    for (int d = 0; d < 3; ++d) {
        if (degree[d] < 1 || degree[d] > SA_MAX_DEGREE)
            return sa_fail(c, SA_ERR_ARG, "degree[%d] = %d (supported 1..%d)", d, degree[d], SA_MAX_DEGREE);
        if (n_ctrl[d] < degree[d] + 1)
            return sa_fail(c, SA_ERR_ARG, "n_ctrl[%d] = %d < degree+1", d, n_ctrl[d]);
        if (n_knots[d] != n_ctrl[d] + degree[d] + 1)
            return sa_fail(c, SA_ERR_ARG, "n_knots[%d] = %d != n_ctrl + degree + 1", d, n_knots[d]);
        if (!knots[d]) return sa_fail(c, SA_ERR_ARG, "knots[%d] is NULL", d);
        const double* U = knots[d];
        for (int i = 0; i < n_knots[d]; ++i)
            if (!is_fin(U[i])) return sa_fail(c, SA_ERR_GEOMETRY, "non-finite knot");
        for (int i = 0; i + 1 < n_knots[d]; ++i)
            if (U[i + 1] < U[i]) return sa_fail(c, SA_ERR_GEOMETRY, "knots[%d] decreasing at %d", d, i);
        for (int i = 1; i <= degree[d]; ++i)
            if (U[i] != U[0] || U[n_knots[d] - 1 - i] != U[n_knots[d] - 1])
                return sa_fail(c, SA_ERR_GEOMETRY, "knots[%d] not open", d);
        if (!(U[n_knots[d] - 1] > U[0])) return sa_fail(c, SA_ERR_GEOMETRY, "knots[%d] empty", d);
        for (int i = 0; i + degree[d] + 1 < n_knots[d]; ++i)
            if (U[i + degree[d] + 1] == U[i])
                return sa_fail(c, SA_ERR_GEOMETRY, "knot multiplicity > degree in direction %d", d);
    }
    const long long ndof_ll = (long long)n_ctrl[0] * n_ctrl[1] * n_ctrl[2];
    if (ndof_ll > (1ll << 28)) return sa_fail(c, SA_ERR_ARG, "patch too large");
    const int ndof = (int)ndof_ll;
    for (long long i = 0; i < 3 * ndof_ll; ++i)
        if (!is_fin(ctrl_xyz[i])) return sa_fail(c, SA_ERR_GEOMETRY, "non-finite control point");
    if (weights)
        for (int i = 0; i < ndof; ++i)
            if (!(weights[i] > 0.0) || !is_fin(weights[i]))
                return sa_fail(c, SA_ERR_GEOMETRY, "weight %d = %g must be > 0", i, weights[i]);
    // bounding box, top plane
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < ndof; ++i)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], ctrl_xyz[3 * i + d]);
            hi[d] = std::max(hi[d], ctrl_xyz[3 * i + d]);
        }
    const double scale = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                   (hi[2] - lo[2]) * (hi[2] - lo[2]));
    if (!(scale > 0)) return sa_fail(c, SA_ERR_GEOMETRY, "degenerate control net");
    const int n0 = n_ctrl[0], n1 = n_ctrl[1], n2 = n_ctrl[2];
    const double zt = ctrl_xyz[3 * ((n2 - 1) * n1 * n0) + 2];
    for (int j = 0; j < n1; ++j)
        for (int i = 0; i < n0; ++i)
            if (std::fabs(ctrl_xyz[3 * (((n2 - 1) * n1 + j) * n0 + i) + 2] - zt) > 1e-12 * scale)
                return sa_fail(c, SA_ERR_GEOMETRY, "top face (zeta = 1) is not a plane z = const");
    // closed direction: coinciding end layers, interior faces, no wrap of a support
    if (seam_dir < -1 || seam_dir > 2) return sa_fail(c, SA_ERR_ARG, "seam_dir = %d", seam_dir);
    if (seam_dir >= 0) {
        const int d = seam_dir;
        if (c->face_kind[2 * d] != SA_FACE_NONE || c->face_kind[2 * d + 1] != SA_FACE_NONE)
            return sa_fail(c, SA_ERR_ARG, "the faces of the seam direction %d must be SA_FACE_NONE", d);
        if (n_ctrl[d] <= 2 * (degree[d] + 1))
            return sa_fail(c, SA_ERR_ARG, "seam direction %d needs more than %d control points", d,
                           2 * (degree[d] + 1));
        for (int k = 0; k < n2; ++k)
            for (int j = 0; j < n1; ++j)
                for (int i = 0; i < n0; ++i) {
                    int idx[3] = {i, j, k};
                    if (idx[d] != 0) continue;
                    const int a = (k * n1 + j) * n0 + i;
                    idx[d] = n_ctrl[d] - 1;
                    const int b = (idx[2] * n1 + idx[1]) * n0 + idx[0];
                    for (int q = 0; q < 3; ++q)
                        if (std::fabs(ctrl_xyz[3 * a + q] - ctrl_xyz[3 * b + q]) > 1e-12 * scale)
                            return sa_fail(c, SA_ERR_GEOMETRY, "seam layers of direction %d do not coincide", d);
                    if (weights && std::fabs(weights[a] - weights[b]) > 1e-12 * weights[a])
                        return sa_fail(c, SA_ERR_GEOMETRY, "seam weights of direction %d differ", d);
                }
    }

    // ---- host copy and element lists -----------------------------------------
    for (int d = 0; d < 3; ++d) {
        c->p[d] = degree[d];
        c->n[d] = n_ctrl[d];
        c->U[d].assign(knots[d], knots[d] + n_knots[d]);
        c->espan[d].clear();
        for (int s = degree[d]; s < n_ctrl[d]; ++s)
            if (c->U[d][s + 1] > c->U[d][s]) c->espan[d].push_back(s);
        c->ne[d] = (int)c->espan[d].size();
        // elements touching basis i: spans s with s - p <= i <= s
        c->elo[d].assign(n_ctrl[d], 0);
        c->ehi[d].assign(n_ctrl[d], -1);
        for (int i = 0; i < n_ctrl[d]; ++i) {
            int first = -1, last = -2;
            for (int e = 0; e < c->ne[d]; ++e) {
                const int s = c->espan[d][e];
                if (s - degree[d] <= i && i <= s) {
                    if (first < 0) first = e;
                    last = e;
                }
            }
            c->elo[d][i] = first;
            c->ehi[d][i] = last;
        }
    }
    c->n_elem = c->ne[0] * c->ne[1] * c->ne[2];
    c->ctrl.assign(ctrl_xyz, ctrl_xyz + 3 * ndof_ll);
    c->w.assign(ndof, 1.0);
    if (weights) c->w.assign(weights, weights + ndof);
    // control variables: the control points, one layer fewer on the seam
    c->seam = seam_dir;
    for (int d = 0; d < 3; ++d) c->nd[d] = n_ctrl[d] - (d == seam_dir ? 1 : 0);
    const int nvar = c->nd[0] * c->nd[1] * c->nd[2];
    c->cmap.assign(ndof, 0);
    for (int k = 0; k < n2; ++k)
        for (int j = 0; j < n1; ++j)
            for (int i = 0; i < n0; ++i) {
                int idx[3] = {i, j, k};
                if (seam_dir >= 0) idx[seam_dir] %= c->nd[seam_dir];
                c->cmap[nat(c, i, j, k)] = (idx[2] * c->nd[1] + idx[1]) * c->nd[0] + idx[0];
            }
    c->n_dof = nvar;
    c->z_top = zt;
    c->x_ref = 0.5 * (lo[0] + hi[0]);
    c->y_ref = 0.5 * (lo[1] + hi[1]);
    c->length_scale = scale;

    // ---- Dirichlet control variables and the internal order -----------------
    std::vector<char> isdir(nvar, 0);
    for (int f = 0; f < 6; ++f) {
        if (c->face_kind[f] != SA_FACE_DIRICHLET) continue;
        const int d = f / 2, side = f % 2;
        const int layer = side == 0 ? 0 : c->n[d] - 1;   // open knots
        for (int k = 0; k < n2; ++k)
            for (int j = 0; j < n1; ++j)
                for (int i = 0; i < n0; ++i) {
                    const int idx[3] = {i, j, k};
                    if (idx[d] == layer) isdir[c->cmap[nat(c, i, j, k)]] = 1;
                }
    }
    c->perm.assign(nvar, 0);
    c->iperm.assign(nvar, 0);
    int nf = 0;
    for (int i = 0; i < nvar; ++i)
        if (!isdir[i]) c->iperm[nf++] = i;
    c->n_free = nf;
    int nd = nf;
    for (int i = 0; i < nvar; ++i)
        if (isdir[i]) c->iperm[nd++] = i;
    c->n_dir = nvar - nf;
    for (int i = 0; i < nvar; ++i) c->perm[c->iperm[i]] = i;

    // ---- upload geometry --------------------------------------------------
    std::vector<double4> cw(ndof);
    for (int i = 0; i < ndof; ++i)
        cw[i] = make_double4(ctrl_xyz[3 * i], ctrl_xyz[3 * i + 1], ctrl_xyz[3 * i + 2], c->w[i]);
    SA_UPLOAD(c, c->dcw, cw);
    for (int d = 0; d < 3; ++d) {
        SA_UPLOAD(c, c->dU[d], c->U[d]);
        SA_UPLOAD(c, c->despan[d], c->espan[d]);
    }
    {
        std::vector<int> cp(ndof);   // control point -> internal control variable
        for (int i = 0; i < ndof; ++i) cp[i] = c->perm[c->cmap[i]];
        SA_UPLOAD(c, c->dperm, cp);
    }
    DevPatch& dp = c->dp;
    for (int d = 0; d < 3; ++d) {
        dp.p[d] = c->p[d];
        dp.n[d] = c->n[d];
        dp.ne[d] = c->ne[d];
        dp.U[d] = c->dU[d].p;
        dp.espan[d] = c->despan[d].p;
    }
    dp.cw = c->dcw.p;
    cudaStream_t s = c->stream;

    // ---- boundary quadrature points and weight matrices ------------------------
    double gx[3][SA_MAX_DEGREE + 1], gw[3][SA_MAX_DEGREE + 1];
    for (int d = 0; d < 3; ++d) gauss_legendre(c->p[d] + 1, gx[d], gw[d]);
    for (int kind = SA_FACE_NEUMANN; kind <= SA_FACE_DIRICHLET; ++kind) {
        const bool lat = kind == SA_FACE_NEUMANN;
        // enumerate entries (point-major) to build the CSR pattern on the host
        std::vector<int> erow, ecol;
        std::vector<int> face_q0, face_e0;
        int Q = 0;
        for (int f = 0; f < 6; ++f) {
            face_q0.push_back(Q);
            face_e0.push_back((int)erow.size());
            if (c->face_kind[f] != kind) continue;
            const int d = f / 2, side = f % 2;
            const int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;
            const int nea = c->ne[ta], neb = c->ne[tb];
            const int nga = c->p[ta] + 1, ngb = c->p[tb] + 1;
            const int layer = side == 0 ? 0 : c->n[d] - 1;
            for (int eb = 0; eb < neb; ++eb)
                for (int ea = 0; ea < nea; ++ea)
                    for (int g = 0; g < nga * ngb; ++g) {
                        const int q = Q++;
                        for (int lb = 0; lb <= c->p[tb]; ++lb)
                            for (int la = 0; la <= c->p[ta]; ++la) {
                                int idx[3];
                                idx[d] = layer;
                                idx[ta] = c->espan[ta][ea] - c->p[ta] + la;
                                idx[tb] = c->espan[tb][eb] - c->p[tb] + lb;
                                const int in = c->perm[c->cmap[nat(c, idx[0], idx[1], idx[2])]];
                                erow.push_back(in);
                                ecol.push_back(q);
                            }
                    }
        }
        face_q0.push_back(Q);
        face_e0.push_back((int)erow.size());
        for (int f = 0; f <= 6; ++f) c->face_q0[lat ? 0 : 1][f] = face_q0[f];
        std::vector<int> ptr, col, slot;
        if (lat) {
            // compact rows: the distinct internal dofs, ascending
            std::vector<int> rows(erow.begin(), erow.end());
            std::sort(rows.begin(), rows.end());
            rows.erase(std::unique(rows.begin(), rows.end()), rows.end());
            std::vector<int> rmap(c->n_dof, -1);
            for (size_t r = 0; r < rows.size(); ++r) rmap[rows[r]] = (int)r;
            std::vector<int> er(erow.size());
            for (size_t e = 0; e < erow.size(); ++e) er[e] = rmap[erow[e]];
            build_w_csr((int)rows.size(), er, ecol, ptr, col, slot);
            c->wlat_rows = (int)rows.size();
            c->wlat_rowdof_h = rows;
            c->wlat_ptr_h = ptr;
            c->wlat_col_h = col;
            c->q_lat = Q;
            SA_UPLOAD(c, c->wlat_rowdof, rows);
            SA_UPLOAD(c, c->wlat_ptr, ptr);
            SA_UPLOAD(c, c->wlat_col, col);
            SA_ALLOC(c, c->wlat_val, col.size());
            SA_ALLOC(c, c->lat64, (size_t)7 * Q);
        } else {
            std::vector<int> er(erow.size());
            for (size_t e = 0; e < erow.size(); ++e) {
                er[e] = erow[e] - c->n_free;
                if (er[e] < 0) return sa_fail(c, SA_ERR_GEOMETRY, "Dirichlet face function is not a Dirichlet dof");
            }
            build_w_csr(c->n_dir, er, ecol, ptr, col, slot);
            c->wbot_ptr_h = ptr;
            c->wbot_col_h = col;
            for (int r = 0; r < c->n_dir; ++r)
                if (ptr[r + 1] == ptr[r])
                    return sa_fail(c, SA_ERR_GEOMETRY, "Dirichlet dof without support on a Dirichlet face");
            c->q_bot = Q;
            SA_UPLOAD(c, c->wbot_ptr, ptr);
            SA_UPLOAD(c, c->wbot_col, col);
            SA_ALLOC(c, c->wbot_val, col.size());
            SA_ALLOC(c, c->bot64, (size_t)4 * Q);
        }
        DBuf<int> dslot;
        SA_UPLOAD(c, dslot, slot);
        DBuf<double> cooR;
        DBuf<int> cooD;
        if (!lat && Q > 0) {
            SA_ALLOC(c, cooR, erow.size());
            SA_ALLOC(c, cooD, erow.size());
        }
        for (int f = 0; f < 6; ++f) {
            if (c->face_kind[f] != kind) continue;
            const int d = f / 2;
            const int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;
            cudaError_t e = launch_face_points(
                dp, f, 0, 0, c->ne[ta], c->ne[tb], nullptr, gx[ta], gw[ta], gx[tb], gw[tb],
                face_q0[f], lat ? c->lat64.p : c->bot64.p, Q, lat ? 1 : 0, dslot.p + face_e0[f],
                lat ? c->wlat_val.p : c->wbot_val.p, lat ? nullptr : cooR.p + face_e0[f],
                lat ? nullptr : cooD.p + face_e0[f], c->dperm.p, s);
            if (e != cudaSuccess) return sa_cuda_fail(c, e, "face points");
        }
        if (!lat && c->n_dir > 0) {
            // M_bot pattern: bottom-local dofs sharing a face element
            std::vector<std::vector<int>> nb(c->n_dir);
            for (int f = 0; f < 6; ++f) {
                if (c->face_kind[f] != kind) continue;
                const int d = f / 2;
                const int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;
                const int nfb = (c->p[ta] + 1) * (c->p[tb] + 1);
                const int npt = (c->p[ta] + 1) * (c->p[tb] + 1);
                const int nel = c->ne[ta] * c->ne[tb];
                for (int el = 0; el < nel; ++el) {
                    const int e0 = face_e0[f] + el * npt * nfb;   // first Gauss point
                    for (int a = 0; a < nfb; ++a)
                        for (int b = 0; b < nfb; ++b)
                            nb[erow[e0 + a] - c->n_free].push_back(erow[e0 + b] - c->n_free);
                }
            }
            std::vector<int> mptr(c->n_dir + 1, 0), mcol;
            for (int r = 0; r < c->n_dir; ++r) {
                std::sort(nb[r].begin(), nb[r].end());
                nb[r].erase(std::unique(nb[r].begin(), nb[r].end()), nb[r].end());
                mptr[r + 1] = mptr[r] + (int)nb[r].size();
                mcol.insert(mcol.end(), nb[r].begin(), nb[r].end());
            }
            c->nnz_mbot = (long long)mcol.size();
            SA_UPLOAD(c, c->mbot_ptr, mptr);
            SA_UPLOAD(c, c->mbot_col, mcol);
            SA_ALLOC(c, c->mbot_val, mcol.size());
            SA_ALLOC(c, c->mbot_dinv, c->n_dir);
            // face functions per point: same count on every Dirichlet face
            int nfb = -1;
            for (int f = 0; f < 6; ++f)
                if (c->face_kind[f] == kind) {
                    const int d = f / 2;
                    const int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;
                    const int v = (c->p[ta] + 1) * (c->p[tb] + 1);
                    if (nfb >= 0 && v != nfb)
                        return sa_fail(c, SA_ERR_ARG, "Dirichlet faces with different tangential degrees");
                    nfb = v;
                }
            cudaError_t e = launch_mbot_fill(c->n_dir, c->mbot_ptr.p, c->mbot_col.p, c->wbot_ptr.p,
                                             c->wbot_col.p, c->wbot_val.p, cooD.p, cooR.p, nfb,
                                             c->n_free, c->mbot_val.p, c->mbot_dinv.p, s);
            if (e != cudaSuccess) return sa_cuda_fail(c, e, "M_bot");
            {
                std::vector<long long> p64(mptr.begin(), mptr.end());
                std::vector<int> srcs(mcol.size()), dcol(c->n_dir);
                std::iota(srcs.begin(), srcs.end(), 0);
                std::iota(dcol.begin(), dcol.end(), 0);
                SellHost sh;
                build_sell(c->n_dir, p64, mcol, srcs, dcol, sh);
                SA_UPLOAD_SELL(c, c->mbot_s, sh);
                c->mbot_h = sh;
                SA_ALLOC(c, c->mbot_sval, sh.col.size());
                e = launch_sell_fill(c->mbot_s.n_stored, c->mbot_s.src.p, c->mbot_val.p, 1.0,
                                     nullptr, 0.0, c->mbot_sval.p, s);
                if (e == cudaSuccess && c->opt.precision == SA_MIXED) {
                    cudaError_t ea = c->mbot_sval32.alloc(sh.col.size());
                    if (ea != cudaSuccess) return sa_fail(c, SA_ERR_OOM, "allocation of M_bot FP32");
                    e = launch_to_f32(c->mbot_s.n_stored, c->mbot_sval.p, c->mbot_sval32.p, s);
                }
                if (e != cudaSuccess) return sa_cuda_fail(c, e, "M_bot SELL");
            }
            SA_CUDA(c, cudaStreamSynchronize(s));   // cooR/cooD freed on return
        }
        SA_CUDA(c, cudaStreamSynchronize(s));
    }
    SA_ALLOC(c, c->lat32, (size_t)6 * c->q_lat);
    SA_ALLOC(c, c->bot32, (size_t)3 * c->q_bot);
    {
        cudaError_t e = launch_points32(c->q_lat, c->q_bot, c->lat64.p, c->bot64.p, c->x_ref,
                                        c->y_ref, c->z_top, c->lat32.p, c->bot32.p, s);
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "points32");
    }
    {
        SA_CUDA(c, cudaStreamSynchronize(s));
        const sa_status st = sep_setup(c);
        if (st != SA_OK) return st;
    }

    // ---- CSR pattern of M and K (natural order) ---------------------------------
    std::vector<std::vector<int>> nbr1[3];
    for (int d = 0; d < 3; ++d) {
        nbr1[d].assign(c->n[d], {});
        for (int i = 0; i < c->n[d]; ++i)
            for (int j = 0; j < c->n[d]; ++j)
                if (std::max(c->elo[d][i], c->elo[d][j]) <= std::min(c->ehi[d][i], c->ehi[d][j]))
                    nbr1[d][i].push_back(j);
    }
    // control-point pattern (natural order)
    std::vector<long long> cptr(ndof + 1, 0);
    for (int k = 0; k < n2; ++k)
        for (int j = 0; j < n1; ++j)
            for (int i = 0; i < n0; ++i)
                cptr[nat(c, i, j, k) + 1] =
                    (long long)nbr1[0][i].size() * nbr1[1][j].size() * nbr1[2][k].size();
    for (int r = 0; r < ndof; ++r) cptr[r + 1] += cptr[r];
    const long long cnnz = cptr[ndof];
    std::vector<int> ccol(cnnz);
    for (int k = 0; k < n2; ++k)
        for (int j = 0; j < n1; ++j)
            for (int i = 0; i < n0; ++i) {
                long long s0 = cptr[nat(c, i, j, k)];
                for (int kk : nbr1[2][k])
                    for (int jj : nbr1[1][j])
                        for (int ii : nbr1[0][i]) ccol[s0++] = nat(c, ii, jj, kk);
            }
    // pattern over control variables: the same on an open patch; on a closed
    // one each entry lists the control-point entries summed into it
    std::vector<long long> mk_ptr, sptr;
    std::vector<int> mk_col, sidx;
    if (seam_dir < 0) {
        mk_ptr.swap(cptr);
        mk_col.swap(ccol);
    } else {
        std::vector<std::vector<int>> rows_of(nvar);
        for (int r = 0; r < ndof; ++r) rows_of[c->cmap[r]].push_back(r);
        mk_ptr.assign(nvar + 1, 0);
        sptr.assign(1, 0);
        std::vector<std::pair<int, int>> ent;   // (column, control-point slot)
        for (int R = 0; R < nvar; ++R) {
            ent.clear();
            for (int r : rows_of[R])
                for (long long t = cptr[r]; t < cptr[r + 1]; ++t) ent.push_back({c->cmap[ccol[t]], (int)t});
            std::sort(ent.begin(), ent.end());
            for (size_t a = 0; a < ent.size(); ++a) {
                if (a == 0 || ent[a].first != ent[a - 1].first) {
                    mk_col.push_back(ent[a].first);
                    sptr.push_back(sptr.back());
                }
                sidx.push_back(ent[a].second);
                sptr.back() += 1;
            }
            mk_ptr[R + 1] = (long long)mk_col.size();
        }
    }
    c->nnz = mk_ptr[nvar];
    SA_UPLOAD(c, c->mk_ptr, mk_ptr);
    SA_UPLOAD(c, c->mk_col, mk_col);
    SA_ALLOC(c, c->M, c->nnz);
    SA_ALLOC(c, c->K, c->nnz);

    // ---- element matrices (unit rho c_p and k) and their gather -------------------
    {
        for (int d = 0; d < 3; ++d) {
            SA_UPLOAD(c, c->d_elo[d], c->elo[d]);
            SA_UPLOAD(c, c->d_ehi[d], c->ehi[d]);
        }
        const int nloc = (c->p[0] + 1) * (c->p[1] + 1) * (c->p[2] + 1);
        DBuf<double> Mloc, Kloc;
        DBuf<int> bad;
        SA_ALLOC(c, Mloc, (size_t)c->n_elem * nloc * nloc);
        SA_ALLOC(c, Kloc, (size_t)c->n_elem * nloc * nloc);
        SA_ALLOC(c, bad, 1);
        SA_CUDA(c, cudaMemsetAsync(bad.p, 0, sizeof(int), s));
        double xg[3 * (SA_MAX_DEGREE + 1)], wg[3 * (SA_MAX_DEGREE + 1)];
        for (int d = 0; d < 3; ++d)
            for (int g = 0; g <= c->p[d]; ++g) {
                xg[d * (SA_MAX_DEGREE + 1) + g] = gx[d][g];
                wg[d * (SA_MAX_DEGREE + 1) + g] = gw[d][g];
            }
        cudaError_t e = launch_element_local(dp, 1.0, 1.0, xg, wg, Mloc.p, Kloc.p, bad.p, s);
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "element matrices");
        const int* elo[3] = {c->d_elo[0].p, c->d_elo[1].p, c->d_elo[2].p};
        const int* ehi[3] = {c->d_ehi[0].p, c->d_ehi[1].p, c->d_ehi[2].p};
        if (seam_dir < 0) {
            e = launch_mk_gather(dp, c->mk_ptr.p, c->mk_col.p, elo, ehi, Mloc.p, Kloc.p, c->M.p,
                                 c->K.p, s);
            if (e != cudaSuccess) return sa_cuda_fail(c, e, "gather M, K");
        } else {
            // control-point matrices, then P^T (.) P
            DBuf<long long> gptr, gsptr;
            DBuf<int> gcol, gsidx;
            DBuf<double> Mc, Kc;
            SA_UPLOAD(c, gptr, cptr);
            SA_UPLOAD(c, gcol, ccol);
            SA_UPLOAD(c, gsptr, sptr);
            SA_UPLOAD(c, gsidx, sidx);
            SA_ALLOC(c, Mc, cnnz);
            SA_ALLOC(c, Kc, cnnz);
            e = launch_mk_gather(dp, gptr.p, gcol.p, elo, ehi, Mloc.p, Kloc.p, Mc.p, Kc.p, s);
            if (e == cudaSuccess)
                e = launch_merge_csr(c->nnz, gsptr.p, gsidx.p, Mc.p, Kc.p, c->M.p, c->K.p, s);
            if (e != cudaSuccess) return sa_cuda_fail(c, e, "gather M, K");
            SA_CUDA(c, cudaStreamSynchronize(s));   // temporaries freed on return
        }
        int hbad = 0;
        SA_CUDA(c, cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        SA_CUDA(c, cudaStreamSynchronize(s));
        if (hbad) return sa_fail(c, SA_ERR_GEOMETRY, "det J <= 0 at a Gauss point (inverted or degenerate patch)");
    }

    // ---- free-free operator A and the free rows of M, K (SELL) ---------------
    {
        if (c->nnz > (long long)INT32_MAX)
            return sa_fail(c, SA_ERR_ARG, "operator too large for 32-bit slots");
        std::vector<long long> a_ptr(c->n_free + 1, 0), r_ptr(c->n_free + 1, 0);
        std::vector<int> a_col, a_src, r_col, r_src, dcol(c->n_free);
        a_col.reserve((size_t)c->nnz);
        a_src.reserve((size_t)c->nnz);
        r_col.reserve((size_t)c->nnz);
        r_src.reserve((size_t)c->nnz);
        for (int i = 0; i < c->n_free; ++i) {
            const int r = c->iperm[i];
            dcol[i] = i;
            for (long long t = mk_ptr[r]; t < mk_ptr[r + 1]; ++t) {
                const int j = c->perm[mk_col[t]];
                r_col.push_back(j);
                r_src.push_back((int)t);
                if (j < c->n_free) {
                    a_col.push_back(j);
                    a_src.push_back((int)t);
                }
            }
            a_ptr[i + 1] = (long long)a_col.size();
            r_ptr[i + 1] = (long long)r_col.size();
        }
        c->nnz_a = (long long)a_col.size();
        SellHost sa_h, sr_h;
        build_sell(c->n_free, a_ptr, a_col, a_src, dcol, sa_h);
        SA_UPLOAD_SELL(c, c->a_s, sa_h);
        SA_ALLOC(c, c->a_val, sa_h.col.size());
        SA_ALLOC(c, c->a_dinv, std::max(c->n_free, 1));
        build_sell(c->n_free, r_ptr, r_col, r_src, dcol, sr_h);
        SA_UPLOAD_SELL(c, c->r_s, sr_h);
        c->a_h = sa_h;
        c->r_h = sr_h;
        {
            const std::vector<unsigned char> hi = sell_hi_flags(sr_h);
            int lo = sr_h.n_slices, up = 0;
            for (int sl = 0; sl < sr_h.n_slices; ++sl)
                if (hi[sl]) {
                    lo = std::min(lo, sl);
                    up = sl + 1;
                }
            c->r_dir_sl0 = up > lo ? lo : 0;
            c->r_dir_sl1 = up > lo ? up : 0;
        }
        SA_ALLOC(c, c->r_M, sr_h.col.size());
        SA_ALLOC(c, c->r_K, sr_h.col.size());
        cudaError_t e = launch_sell_fill(c->r_s.n_stored, c->r_s.src.p, c->M.p, 1.0, nullptr, 0.0,
                                         c->r_M.p, s);
        if (e == cudaSuccess)
            e = launch_sell_fill(c->r_s.n_stored, c->r_s.src.p, c->K.p, 1.0, nullptr, 0.0, c->r_K.p, s);
        if (e == cudaSuccess && c->opt.precision == SA_MIXED) {
            SA_ALLOC(c, c->r_M32, sr_h.col.size());
            SA_ALLOC(c, c->r_K32, sr_h.col.size());
            SA_ALLOC(c, c->a_val32, sa_h.col.size());
            e = launch_to_f32(c->r_s.n_stored, c->r_M.p, c->r_M32.p, s);
            if (e == cudaSuccess) e = launch_to_f32(c->r_s.n_stored, c->r_K.p, c->r_K32.p, s);
        }
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "free-row SELL");
        if (c->opt.precision == SA_MIXED) {
            // the slices without Dirichlet columns stream 8 bytes a nonzero
            // instead of 12: FP32 K, bf16 M, 16-bit column offsets
            const std::vector<unsigned char> hi = sell_hi_flags(sr_h);
            std::vector<short> lo(sr_h.col.size(), 0);
            bool fits = sr_h.n > 0;
            for (int sl = 0; sl < sr_h.n_slices && fits; ++sl) {
                if (hi[sl]) continue;
                const long long w = (sr_h.sptr[sl + 1] - sr_h.sptr[sl]) / 32;
                for (int l = 0; l < 32 && fits; ++l) {
                    const int r = std::min(sl * 32 + l, sr_h.n - 1);
                    for (long long kk = 0; kk < w; ++kk) {
                        const long long ee = sr_h.sptr[sl] + 32 * kk + l;
                        const long long d = sl * 32 + l < sr_h.n ? (long long)sr_h.col[ee] - r : 0;
                        if (d < -32768 || d > 32767) {
                            fits = false;
                            break;
                        }
                        lo[ee] = (short)d;
                    }
                }
            }
            if (fits) {
                SA_UPLOAD(c, c->r_col16lo, lo);
                SA_ALLOC(c, c->r_M16, sr_h.col.size());
                e = launch_to_bf16(c->r_s.n_stored, c->r_M.p, c->r_M16.p, s);
                if (e != cudaSuccess) return sa_cuda_fail(c, e, "free-row M (bf16)");
            }
        }
    }

    // ---- state and work vectors ---------------------------------------------------
    const int nwork = std::max(std::max(c->n_free, c->n_dir), 1);
    SA_ALLOC(c, c->That, c->n_dof);
    SA_ALLOC(c, c->F0, c->n_dof);
    SA_ALLOC(c, c->F1, c->n_dof);
    SA_ALLOC(c, c->gnew, std::max(c->n_dir, 1));
    SA_ALLOC(c, c->bbot, std::max(c->n_dir, 1));
    SA_ALLOC(c, c->r0bot, std::max(c->n_dir, 1));
    SA_ALLOC(c, c->bsqbot, std::max(c->n_dir, 1));
    SA_ALLOC(c, c->rhs, nwork);
    SA_ALLOC(c, c->r0, nwork);
    SA_ALLOC(c, c->bsq, nwork);
    SA_ALLOC(c, c->dirv, 2 * (size_t)std::max(c->n_dir, 1));
    if (c->opt.initial_guess == SA_GUESS_EXTRAPOLATE) {
        SA_ALLOC(c, c->x_prev, c->n_dof);
        SA_ALLOC(c, c->dx_extrap, std::max(c->n_free, 1));
        SA_ALLOC(c, c->one, 1);
        const double one = 1.0;
        SA_CUDA(c, cudaMemcpy(c->one.p, &one, sizeof(double), cudaMemcpyHostToDevice));
    }
    c->nwork = nwork;
    SA_ALLOC(c, c->work64, (size_t)5 * nwork);
    {
        // halo of the padded SpMV vector: every column offset of A and M_bot
        int halo = 0;
        halo = std::max(halo, std::max(-c->a_s.dmin, c->a_s.dmax));
        halo = std::max(halo, std::max(-c->mbot_s.dmin, c->mbot_s.dmax));
        // a block's window reaches 32 s1 + dmax, up to 31 rows past n, and
        // starts up to 3 entries before 32 s0 + dmin (16-byte alignment)
        c->work_pad = (halo + 40 + 3) & ~3;
        const size_t vt = c->opt.precision == SA_MIXED ? sizeof(float) : sizeof(double);
        // two padded vectors (the pipelined PCG publishes into them alternately)
        SA_ALLOC(c, c->workpad, 2 * (nwork + 2 * (size_t)c->work_pad) * vt);
        SA_CUDA(c, cudaMemsetAsync(c->workpad.p, 0, 2 * (nwork + 2 * (size_t)c->work_pad) * vt, s));
    }
    SA_ALLOC(c, c->dev64, c->n_dof);
    SA_ALLOC(c, c->dev32, c->n_dof);
    if (c->opt.precision == SA_MIXED) {
        SA_ALLOC(c, c->a_dinv32, std::max(c->n_free, 1));
        SA_ALLOC(c, c->mbot_dinv32, std::max(c->n_dir, 1));
        if (c->n_dir > 0) {
            cudaError_t e = launch_to_f32(c->n_dir, c->mbot_dinv.p, c->mbot_dinv32.p, s);
            if (e != cudaSuccess) return sa_cuda_fail(c, e, "dinv FP32");
        }
    }
    SA_ALLOC(c, c->s_lat, std::max(c->q_lat, 1));
    SA_ALLOC(c, c->tt_bot, std::max(c->q_bot, 1));
    SA_CUDA(c, cudaMemsetAsync(c->F0.p, 0, sizeof(double) * c->n_dof, s));
    SA_CUDA(c, cudaMemsetAsync(c->F1.p, 0, sizeof(double) * c->n_dof, s));
    SA_CUDA(c, cudaMemsetAsync(c->s_lat.p, 0, sizeof(double) * std::max(c->q_lat, 1), s));
    SA_CUDA(c, cudaMemsetAsync(c->tt_bot.p, 0, sizeof(double) * std::max(c->q_bot, 1), s));
    SA_CUDA(c, cudaMemsetAsync(c->work64.p, 0, sizeof(double) * 5 * nwork, s));
    // PCG launch shape: co-resident blocks (cooperative launch)
    {
        int occ = 0;
        SA_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                       &occ, pcg_kernel_ptr(c->opt.precision), pcg_block_size(), 0));
        if (occ < 1) return sa_fail(c, SA_ERR_CUDA, "PCG kernel cannot be resident");
        c->pcg_block = pcg_block_size();
        c->pcg_grid = c->num_sms;   // one co-resident block of 1024 threads per SM
        SA_ALLOC(c, c->partials, (size_t)12 * c->pcg_grid);
        SA_ALLOC(c, c->npart, (size_t)2 * std::max(c->r_s.n_slices, 1));
        SA_ALLOC(c, c->npart_bot, (size_t)2 * std::max((8 * (long long)c->n_dir + 31) / 32, 1ll));
        if (c->opt.precond != SA_PRECOND_JACOBI) {
            sa_status fst = fd_setup(c);
            if (fst) return fst;
            if (c->opt.precond == SA_PRECOND_FD && !c->fdm.ok)
                return sa_fail(c, SA_ERR_ARG, "fast diagonalization needs the tensor grid of free "
                                              "control variables with at most 128 per direction");
            if (c->opt.precond == SA_PRECOND_FD && c->opt.pcg_variant == SA_PCG_GLOBAL)
                return sa_fail(c, SA_ERR_ARG, "fast diagonalization runs in the shared-memory PCG only");
        }
        if (c->opt.pcg_variant == SA_PCG_SHARED || c->opt.precond == SA_PRECOND_FD) {
            PcgLaunch L{};
            L.op = sell_view(c->a_s);
            L.pad = c->work_pad;
            L.grid = c->pcg_grid;
            L.fd = fd_view(c, c->fdm);
            if (!pcg_shared_fits(c->opt.precision, L))
                return sa_fail(c, SA_ERR_ARG,
                               "shared-memory PCG: %d rows per block do not fit in shared memory",
                               32 * ((c->a_s.n_slices + c->pcg_grid - 1) / c->pcg_grid));
        }
    }
    SA_CUDA(c, cudaStreamSynchronize(s));
    c->has_patch = true;
    c->n_step = 0;
    return SA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// stepping
// ---------------------------------------------------------------------------
namespace {

// Scan -> source positions (see sa_set_scan): tracks are maximal runs of
// laser-on segments; sources at arc lengths 0, v dt, 2 v dt, ... on each.
void discretize_scan(const sa_ctx* c, double dt, std::vector<double>& xy) {
    xy.clear();
    const int nv = (int)c->path.size() / 3;
    const double step = c->speed * dt;
    int s = 0;
    const int nseg = nv - 1;
    while (s < nseg) {
        if (!c->seg_on[s]) {
            ++s;
            continue;
        }
        int e = s;
        while (e < nseg && c->seg_on[e]) ++e;
        std::vector<double> cum(1, 0.0), len;
        for (int k = s; k < e; ++k) {
            const double* a = &c->path[3 * k];
            const double* b = &c->path[3 * (k + 1)];
            const double l = std::sqrt((b[0] - a[0]) * (b[0] - a[0]) + (b[1] - a[1]) * (b[1] - a[1]) +
                                       (b[2] - a[2]) * (b[2] - a[2]));
            len.push_back(l);
            cum.push_back(cum.back() + l);
        }
        const double L = cum.back();
        const long long count = (long long)std::floor(L / step + 1e-9) + 1;
        for (long long jj = 0; jj < count; ++jj) {
            const double arc = std::min(jj * step, L);
            int k = (int)(std::upper_bound(cum.begin(), cum.end(), arc) - cum.begin()) - 1;
            k = std::min(std::max(k, 0), (int)len.size() - 1);
            const double t = len[k] > 0 ? (arc - cum[k]) / len[k] : 0.0;
            const double* a = &c->path[3 * (s + k)];
            const double* b = &c->path[3 * (s + k + 1)];
            xy.push_back(a[0] + t * (b[0] - a[0]));
            xy.push_back(a[1] + t * (b[1] - a[1]));
        }
        s = e;
    }
}

sa_status ensure_sources(sa_ctx* c, double dt) {
    if (c->src_dt != 0.0) {
        if (dt != c->src_dt)
            return sa_fail(c, SA_ERR_ARG, "dt %g differs from the dt %g the scan was discretised with", dt, c->src_dt);
        return SA_OK;
    }
    std::vector<double> xy;
    discretize_scan(c, dt, xy);
    const int n = (int)(xy.size() / 2);
    std::vector<double2> pos(std::max(n, 1));
    for (int i = 0; i < n; ++i) pos[i] = make_double2(xy[2 * i] - c->x_ref, xy[2 * i + 1] - c->y_ref);
    SA_UPLOAD(c, c->src_pos, pos);
    const size_t m = std::max(n, 1);
    SA_ALLOC(c, c->src64T, m);
    SA_ALLOC(c, c->src64F, m);
    SA_ALLOC(c, c->src32T, m);
    SA_ALLOC(c, c->src32F, m);
    SA_ALLOC(c, c->evT, m);
    SA_ALLOC(c, c->evF, m);
    c->n_src = n;
    c->src_dt = dt;
    c->E = c->absorptivity * c->power * dt;
    return sep_alloc(c);
}

sa_status ensure_operator(sa_ctx* c, double theta, double dt) {
    if (c->op_dt == dt && c->op_theta == theta) return SA_OK;
    cudaError_t e = launch_sell_fill(c->a_s.n_stored, c->a_s.src.p, c->M.p, c->rho * c->cp / dt,
                                     c->K.p, theta * c->k, c->a_val.p, c->stream);
    if (e == cudaSuccess) e = launch_sell_dinv(c->n_free, c->a_s.diag.p, c->a_val.p, c->a_dinv.p, c->stream);
    if (e == cudaSuccess && c->opt.precision == SA_MIXED)
        e = launch_to_f32(c->a_s.n_stored, c->a_val.p, c->a_val32.p, c->stream);
    if (e == cudaSuccess && c->opt.precision == SA_MIXED)
        e = launch_to_f32(c->n_free, c->a_dinv.p, c->a_dinv32.p, c->stream);
    if (e == cudaSuccess) e = fd_prepare(c, theta, dt, c->stream);
    if (e != cudaSuccess) return sa_cuda_fail(c, e, "build A");
    c->op_dt = dt;
    c->op_theta = theta;
    drop_graphs(c);
    return SA_OK;
}

sa_status enqueue_step(sa_ctx* c, double theta, double dt) {
    cudaStream_t s = c->stream;
    const double alpha = c->k / (c->rho * c->cp);
    const bool timing = c->opt.stage_timing != 0;
#define SA_MARK(i)                                                        \
    do {                                                                  \
        if (timing) SA_CUDA(c, cudaEventRecord(c->ev[i], s));             \
    } while (0)
    cudaError_t e;
    SA_MARK(SA_STAGE_PROLOGUE);
    // the mixed separable sums form the source coefficients themselves
    const bool fused_coef = c->sep.ok && c->opt.precision == SA_MIXED;
    if (!fused_coef) {
        e = launch_prologue(c->st.p, 0, c->st.p, c->n_src, c->src_pos.p, dt, alpha,
                            c->spot_radius * c->spot_radius / (8.0 * alpha),
                            c->opt.half_space_factor * c->E / (c->rho * c->cp), c->opt.precision,
                            c->opt.precision == SA_FP64 ? c->src64T.p : nullptr,
                            c->opt.precision == SA_FP64 ? c->src64F.p : nullptr,
                            c->opt.precision == SA_MIXED ? c->src32T.p : nullptr,
                            c->opt.precision == SA_MIXED ? c->src32F.p : nullptr, s);
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "prologue");
    }
    // Two chains after the prologue: the bottom chain (history of the bottom
    // points, b_bot, the projection) on the second stream, beside the
    // lateral chain (history of the lateral points, F, the right-hand side of
    // the slices without Dirichlet columns); they join before the slices
    // with Dirichlet columns.  Stage timing keeps one stream.
    const bool overlap = !timing && c->aux != nullptr && c->n_dir > 0;
    cudaStream_t sb = overlap ? c->aux : s;
    if (overlap) {
        SA_CUDA(c, cudaEventRecord(c->ev_fork, s));
        SA_CUDA(c, cudaStreamWaitEvent(sb, c->ev_fork, 0));
    }
    SA_MARK(SA_STAGE_HISTORY);
    for (int part = overlap ? 2 : 0; part >= (overlap ? 1 : 0); --part) {
        if (c->sep.ok) {
            // the bottom chain is the longer one: its sums run first with the
            // whole GPU, the lateral sums after them (beside the bottom
            // gather and projection)
            e = launch_sep(c, part, dt, part == 2 ? sb : s);
            if (e == cudaSuccess && overlap && part == 2) e = cudaEventRecord(c->ev_hist, sb);
            if (e == cudaSuccess && overlap && part == 2) e = cudaStreamWaitEvent(s, c->ev_hist, 0);
        } else
            e = launch_history(c->opt.precision, c->hist_P, c->hist_W, c->st.p, c->q_lat,
                               c->q_bot, c->lat32.p, c->bot32.p, c->lat64.p, c->bot64.p,
                               c->x_ref, c->y_ref, c->z_top, c->src32F.p, c->src32T.p,
                               c->src64F.p, c->src64T.p, c->s_lat.p, c->tt_bot.p,
                               part == 2 ? sb : s, part);
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "history");
    }
    SA_MARK(SA_STAGE_GATHER);
    const bool extrap = c->opt.initial_guess == SA_GUESS_EXTRAPOLATE;
    if (extrap) {
        // proposals T^n - T^{n-1} (main solve) and 2 g^n - g^{n-1} (projection)
        e = launch_extrap(c->n_free, c->n_dir, c->That.p, c->x_prev.p, c->dx_extrap.p,
                          c->x_prev.p + c->n_free, c->gnew.p, sb);
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "extrapolated guess");
    } else if (c->n_dir > 0) {
        // x0 of the projection: g^n (the Dirichlet part of the state)
        e = cudaMemcpyAsync(c->gnew.p, c->That.p + c->n_free, sizeof(double) * c->n_dir,
                            cudaMemcpyDeviceToDevice, sb);
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "g0");
    }
    // the bottom rows also form the projection's initial residual
    BotResid br;
    br.mptr = c->mbot_ptr.p;
    br.mcol = c->mbot_col.p;
    br.mval = c->mbot_val.p;
    br.g0 = c->gnew.p;
    br.r0 = c->r0bot.p;
    br.bsq = c->bsqbot.p;
    // the projection's Z = S r0 and norms from the gather (2-D fast
    // diagonalization; no proposed start is tested in the projection)
    const FdView fdb_view = fd_view(c, c->fdb);
    const bool bot_pre = fdb_view.on && c->npart_bot.p && c->n_dir > 0;
    if (bot_pre) {
        br.fdS = fdb_view.S;
        br.fdZ = fdb_view.Z;
        br.f32 = c->opt.precision == SA_MIXED ? 1 : 0;
        br.npart = c->npart_bot.p;
    }
    for (int part = overlap ? 2 : 0; part >= (overlap ? 1 : 0); --part) {
        e = launch_gather(c->wlat_rows, c->wlat_rowdof.p, c->wlat_ptr.p, c->wlat_col.p,
                          c->wlat_val.p, c->s_lat.p, c->k, c->n_dir, c->wbot_ptr.p, c->wbot_col.p,
                          c->wbot_val.p, c->tt_bot.p, c->Tc, c->F1.p, c->bbot.p, c->n_dof,
                          c->That.p, c->dev64.p, c->dev32.p, part == 2 ? sb : s, part,
                          c->n_dir > 0 ? br : BotResid(), c->st.p);
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "gather");
    }
    const bool mixed = c->opt.precision == SA_MIXED;
    SA_MARK(SA_STAGE_BOTTOM);
    bool dir_ready = false;
    if (c->n_dir > 0) {
        PcgLaunch L;
        L.op = sell_view(c->mbot_s);
        L.val = mixed ? (const void*)c->mbot_sval32.p : (const void*)c->mbot_sval.p;
        L.val_hi = c->mbot_sval.p;
        L.dinv = c->mbot_dinv.p;
        L.dinvl = mixed ? (const void*)c->mbot_dinv32.p : (const void*)c->mbot_dinv.p;
        L.dx0 = nullptr;
        L.dx0_scale = nullptr;
        L.b = c->bbot.p;
        L.r0 = c->r0bot.p;       // r0 = b_bot - M_bot g0 from the gather (FP64)
        L.bsq = c->bsqbot.p;
        L.x = c->gnew.p;
        L.w64 = c->work64.p;
        L.vpad = c->workpad.p;
        L.pad = c->work_pad;
        L.stride = c->nwork;
        L.partials = c->partials.p;
        L.st = c->st.p;
        L.variant = c->opt.pcg_variant;
        L.fd = fdb_view;
        if (bot_pre) {
            L.npart = c->npart_bot.p;
            L.npart_n = (int)((8 * (long long)c->n_dir + 31) / 32);
        }
        L.which = 1;
        L.tol = c->opt.pcg_tol;
        L.max_iter = c->opt.pcg_max_iter;
        // small system: a few blocks of ~4 slices, so that most SMs stay
        // free for the lateral chain beside it; 512-thread blocks (half an
        // SM's registers), so that a block starts beside the lateral sums'
        // CTAs instead of waiting for an SM they have left
        L.grid = std::max(1, std::min(c->pcg_grid, 2 * ((c->mbot_s.n_slices + 7) / 8)));
        L.block = 512;
        L.ksplit = 0;
        // the shared-memory solve also writes g^{n+1} - g^n and g^{n+1} for
        // the right-hand side (no separate kernel after it)
        dir_ready = c->opt.pcg_variant != SA_PCG_GLOBAL && pcg_shared_fits(c->opt.precision, L);
        if (dir_ready) {
            L.dir_old = c->That.p + c->n_free;
            L.dir_out = c->dirv.p;
        }
        e = launch_pcg(c->opt.precision, L, sb);
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "bottom PCG");
    }
    SA_MARK(SA_STAGE_RHS);
    // the right-hand side kernel also writes the main solve's Z = S r0 and the
    // per-slice norms when the solve starts from T^n with the fast
    // diagonalization (no proposed start to test first)
    const FdView fdm_view = fd_view(c, c->fdm);
    const bool rhs_pre = fdm_view.on && !extrap && !c->ws_net && c->npart.p &&
                         c->npart.n >= (size_t)2 * c->r_s.n_slices;
    // Two launches when the chains overlap: the slices without Dirichlet
    // columns on the main stream after the lateral gather, the slices with
    // them on the second stream once the projection and the lateral gather
    // (F^{n+1} and the deviations T^n - T_c) are done, the two side by side;
    // the main solve waits for both.
    if (overlap) {
        SA_CUDA(c, cudaEventRecord(c->ev_lat, s));
        SA_CUDA(c, cudaStreamWaitEvent(sb, c->ev_lat, 0));
    }
    for (int only = overlap ? 2 : 0; only >= (overlap ? 1 : 0); --only) {
        e = launch_theta_rhs(c->opt.precision, sell_view(c->r_s),
                             mixed ? (const void*)c->r_K32.p : (const void*)c->r_K.p,
                             mixed ? (const void*)c->r_M32.p : (const void*)c->r_M.p,
                             mixed ? (const void*)c->dev32.p : (const void*)c->dev64.p, c->That.p,
                             c->gnew.p, c->F0.p, c->F1.p, c->rho * c->cp / dt, c->k, theta, c->Tc,
                             c->r0.p, c->bsq.p, c->n_dir, c->dirv.p, only == 2 ? sb : s, only, dir_ready,
                             rhs_pre ? fdm_view.S : nullptr, rhs_pre ? fdm_view.Z : nullptr,
                             rhs_pre ? c->npart.p : nullptr, mixed ? c->r_col16lo.p : nullptr,
                             mixed ? c->r_M16.p : nullptr, only == 2 ? c->r_dir_sl0 : 0,
                             only == 2 ? c->r_dir_sl1 : -1);
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "theta rhs");
    }
    if (overlap) {   // join
        SA_CUDA(c, cudaEventRecord(c->ev_join, sb));
        SA_CUDA(c, cudaStreamWaitEvent(s, c->ev_join, 0));
    }
    SA_MARK(SA_STAGE_PCG);
    const bool rec = c->rec_X != nullptr && c->rec_count < c->rec_cap;
    if (c->ws_net || rec) {
        e = launch_norm(c->n_free, c->r0.p, c->ws_part.p, c->ws_norm.p, s);
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "warm-start norm");
    }
    const float* dx0 = extrap ? c->dx_extrap.p : nullptr;
    const double* dx0_scale = extrap ? c->one.p : nullptr;
    if (c->ws_net) {
        e = launch_ws_input(c->ws_n_in, c->ws_idx.p, c->r0.p, c->ws_norm.p, c->ws_in.p, s);
        if (e == cudaSuccess) e = mlp_forward(c->ws_net, c->ws_in.p, 1, &dx0, s);
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "warm-start network");
    }
    if (rec) {
        e = launch_ws_input(c->rec_n_in, c->rec_idx.p, c->r0.p, c->ws_norm.p,
                            (unsigned char*)c->rec_X + (size_t)c->rec_count * c->rec_n_in * 2, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->ws_xold.p, c->That.p, sizeof(double) * c->n_free,
                                cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "recorder input");
    }
    bool fin_fused = false;
    {
        PcgLaunch L;
        L.dx0 = dx0;
        L.dx0_scale = c->ws_net ? c->ws_norm.p : dx0_scale;
        L.op = sell_view(c->a_s);
        L.val = mixed ? (const void*)c->a_val32.p : (const void*)c->a_val.p;
        L.val_hi = c->a_val.p;
        L.dinv = c->a_dinv.p;
        L.dinvl = mixed ? (const void*)c->a_dinv32.p : (const void*)c->a_dinv.p;
        L.b = nullptr;
        L.r0 = c->r0.p;
        L.bsq = c->bsq.p;
        L.x = c->That.p;
        L.w64 = c->work64.p;
        L.vpad = c->workpad.p;
        L.pad = c->work_pad;
        L.stride = c->nwork;
        L.partials = c->partials.p;
        L.st = c->st.p;
        L.variant = c->opt.pcg_variant;
        L.fd = fdm_view;
        if (rhs_pre) {
            L.npart = c->npart.p;
            L.npart_n = c->r_s.n_slices;
        }
        L.which = 0;
        L.tol = c->opt.pcg_tol;
        L.max_iter = c->opt.pcg_max_iter;
        L.grid = c->pcg_grid;
        L.ksplit = 0;
        // the step's finalize in the solve's tail when the shared-memory
        // solve runs and nothing reads the state between them (no recorder,
        // no stage timing)
        fin_fused = !rec && !timing && c->opt.pcg_variant != SA_PCG_GLOBAL &&
                    pcg_shared_fits(c->opt.precision, L);
        if (fin_fused) {
            L.fin_F1 = c->F1.p;
            L.fin_F0 = c->F0.p;
            L.fin_g = c->gnew.p;
            L.fin_That = c->That.p;
            L.fin_n_dof = c->n_dof;
            L.fin_n_dir = c->n_dir;
        }
        e = launch_pcg(c->opt.precision, L, s);
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "PCG");
    }
    if (rec) {
        e = launch_ws_target(c->n_free, c->That.p, c->ws_xold.p, c->ws_norm.p,
                             (unsigned char*)c->rec_Y + (size_t)c->rec_count * c->n_free * 2, s);
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "recorder target");
        c->rec_count += 1;
    }
    SA_MARK(SA_STAGE_FINALIZE);
    if (!fin_fused) {
        e = launch_finalize(c->n_dir, c->n_free, c->n_dof, c->gnew.p, c->That.p, c->F1.p, c->F0.p,
                            c->st.p, s);
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "finalize");
    }
    SA_MARK(SA_N_STAGES);
#undef SA_MARK
    if (timing) {
        SA_CUDA(c, cudaEventSynchronize(c->ev[SA_N_STAGES]));
        for (int i = 0; i < SA_N_STAGES; ++i) {
            float ms = 0.f;
            SA_CUDA(c, cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]));
            c->stage_ms[i] += ms;
        }
        c->stage_steps += 1;
    }
    return SA_OK;
}

sa_status init_state_if_needed(sa_ctx* c) {
    if (c->state_init) return SA_OK;
    std::vector<int> ipf(c->iperm.begin(), c->iperm.begin() + c->n_free);
    if (ipf.empty()) ipf.assign(1, 0);
    SA_UPLOAD(c, c->d_iperm_free, ipf);
    // T^(x, 0) = T_c (Section 2.1): constants are exact in the spline space
    std::vector<double> T0(c->n_dof, c->Tc);
    SA_CUDA(c, cudaMemcpy(c->That.p, T0.data(), sizeof(double) * c->n_dof, cudaMemcpyHostToDevice));
    if (c->x_prev.p)
        SA_CUDA(c, cudaMemcpy(c->x_prev.p, T0.data(), sizeof(double) * c->n_dof, cudaMemcpyHostToDevice));
    c->state_init = true;
    return SA_OK;
}

}  // namespace

// Sources, initial state and operator of (theta, dt), as the first sa_step
// would prepare them (used by sa_batch).
sa_status sa_prepare(sa_ctx* c, double theta, double dt) {
    sa_status st = check_usable(c);
    if (st) return st;
    if (!c->has_patch || !c->has_material || !c->has_scan)
        return sa_fail(c, SA_ERR_STATE, "instance needs patch, material and scan");
    if ((st = ensure_sources(c, dt))) return st;
    if ((st = init_state_if_needed(c))) return st;
    return ensure_operator(c, theta, dt);
}

extern "C" {

sa_status sa_step(sa_ctx* c, double theta, double dt, int n_steps, sa_step_stats* stats) {
    sa_status st = check_usable(c);
    if (st) return st;
    if (!c->has_patch || !c->has_material || !c->has_scan)
        return sa_fail(c, SA_ERR_STATE, "sa_step needs patch, material and scan");
    if (!(theta >= 0.0 && theta <= 1.0)) return sa_fail(c, SA_ERR_ARG, "theta %g not in [0, 1]", theta);
    if (!(dt > 0.0) || !is_fin(dt)) return sa_fail(c, SA_ERR_ARG, "dt %g must be > 0", dt);
    if (n_steps < 0) return sa_fail(c, SA_ERR_ARG, "n_steps < 0");
    if ((st = ensure_sources(c, dt))) return st;
    if ((st = init_state_if_needed(c))) return st;
    if ((st = ensure_operator(c, theta, dt))) return st;
    cudaStream_t s = c->stream;
    const bool graph = c->opt.use_graph && s != nullptr && !c->opt.stage_timing && c->rec_X == nullptr;
    // graphs of kGraphSteps steps while that many remain (no gap between the
    // steps inside one graph), then one-step graphs
    auto capture = [&](cudaGraphExec_t* exec, int steps) -> sa_status {
        cudaGraph_t g;
        SA_CUDA(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        sa_status es = SA_OK;
        for (int k = 0; k < steps && es == SA_OK; ++k) es = enqueue_step(c, theta, dt);
        cudaError_t ee = cudaStreamEndCapture(s, &g);
        if (es) return es;
        if (ee != cudaSuccess) return sa_cuda_fail(c, ee, "end capture");
        ee = cudaGraphInstantiate(exec, g, 0);
        cudaGraphDestroy(g);
        if (ee != cudaSuccess) return sa_cuda_fail(c, ee, "graph instantiate");
        return SA_OK;
    };
    for (int i = 0; i < n_steps;) {
        if (graph && n_steps - i >= kGraphSteps) {
            if (!c->graph_multi && (st = capture(&c->graph_multi, kGraphSteps))) return st;
            SA_CUDA(c, cudaGraphLaunch(c->graph_multi, s));
            i += kGraphSteps;
        } else if (graph) {
            if (!c->graph_exec && (st = capture(&c->graph_exec, 1))) return st;
            SA_CUDA(c, cudaGraphLaunch(c->graph_exec, s));
            ++i;
        } else {
            if ((st = enqueue_step(c, theta, dt))) return st;
            ++i;
        }
    }
    c->n_step += n_steps;
    if (stats) {
        // read the status, then (stream-ordered after the read) zero the
        // counters read here (not n, not the barrier words): the next stats
        // report covers the steps since this call; one synchronisation
        DevStatus h;
        static const DevStatus zero{};
        SA_CUDA(c, cudaMemcpyAsync(&h, c->st.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
        SA_CUDA(c, cudaMemcpyAsync(&c->st.p->err, &zero.err, offsetof(DevStatus, n), cudaMemcpyHostToDevice, s));
        SA_CUDA(c, cudaMemcpyAsync(&c->st.p->iters_total, &zero.iters_total,
                                   offsetof(DevStatus, pad) - offsetof(DevStatus, iters_total),
                                   cudaMemcpyHostToDevice, s));
        SA_CUDA(c, cudaStreamSynchronize(s));
        stats->steps_done = n_steps;
        stats->pcg_iters_last = h.pcg_iters;
        stats->pcg_iters_total = (int)h.iters_total;
        stats->pcg_iters_max = h.iters_max;
        stats->bot_iters_total = (int)h.bot_total;
        stats->hist_pairs_skipped = h.hist_skipped;
        stats->rel_res_last = h.rel_res;
        stats->n_active_sources = h.n_active;
        stats->step_index = h.n;
        stats->ws_used_last = h.ws_used;
        stats->ws_ratio_last = h.ws_ratio;
        if (h.err & SA_DEV_TIMEOUT) return sa_fail(c, SA_ERR_TIMEOUT, "a device-side wait timed out");
        if (h.err & SA_DEV_NAN) return sa_fail(c, SA_ERR_NAN, "non-finite value in the solve");
        if (h.err & (SA_DEV_NOT_CONVERGED | SA_DEV_BOT_NOT_CONVERGED))
            return sa_fail(c, SA_ERR_NOT_CONVERGED, "PCG did not converge (flags %d, rel res %g)", h.err, h.rel_res);
    }
    return SA_OK;
}

sa_status sa_set_warm_start(sa_ctx* c, sa_mlp* net, int n_in, const int* in_idx) {
    sa_status st = check_usable(c);
    if (st) return st;
    if (!c->has_patch) return sa_fail(c, SA_ERR_STATE, "no patch");
    drop_graphs(c);
    if (!net) {
        c->ws_net = nullptr;
        return SA_OK;
    }
    if (n_in <= 0 || !in_idx || mlp_n_in(net) != n_in || mlp_n_out(net) != c->n_free)
        return sa_fail(c, SA_ERR_ARG, "network sizes (%d in, %d out) do not match (%d, %d)",
                       mlp_n_in(net), mlp_n_out(net), n_in, c->n_free);
    for (int k = 0; k < n_in; ++k)
        if (in_idx[k] < 0 || in_idx[k] >= c->n_free) return sa_fail(c, SA_ERR_ARG, "in_idx[%d]", k);
    std::vector<int> idx(in_idx, in_idx + n_in);
    SA_UPLOAD(c, c->ws_idx, idx);
    SA_ALLOC(c, c->ws_in, (size_t)n_in * 2);
    if (!c->ws_norm.p) {
        SA_ALLOC(c, c->ws_norm, 1);
        SA_ALLOC(c, c->ws_part, 64);
    }
    if (mlp_prepare(net, 1) != 0) return sa_fail(c, SA_ERR_OOM, "network buffers");
    c->ws_net = net;
    c->ws_n_in = n_in;
    return SA_OK;
}

sa_status sa_set_recorder(sa_ctx* c, void* X, void* Y, int capacity, int n_in, const int* in_idx) {
    sa_status st = check_usable(c);
    if (st) return st;
    if (!c->has_patch) return sa_fail(c, SA_ERR_STATE, "no patch");
    if (!X) {
        c->rec_X = c->rec_Y = nullptr;
        c->rec_cap = c->rec_count = 0;
        return SA_OK;
    }
    if (!Y || capacity <= 0 || n_in <= 0 || !in_idx) return sa_fail(c, SA_ERR_ARG, "recorder arguments");
    for (int k = 0; k < n_in; ++k)
        if (in_idx[k] < 0 || in_idx[k] >= c->n_free) return sa_fail(c, SA_ERR_ARG, "in_idx[%d]", k);
    std::vector<int> idx(in_idx, in_idx + n_in);
    SA_UPLOAD(c, c->rec_idx, idx);
    if (!c->ws_norm.p) {
        SA_ALLOC(c, c->ws_norm, 1);
        SA_ALLOC(c, c->ws_part, 64);
    }
    if (c->ws_xold.n < (size_t)std::max(c->n_free, 1)) SA_ALLOC(c, c->ws_xold, std::max(c->n_free, 1));
    c->rec_X = X;
    c->rec_Y = Y;
    c->rec_cap = capacity;
    c->rec_count = 0;
    c->rec_n_in = n_in;
    return SA_OK;
}

sa_status sa_get_recorded(sa_ctx* c, int* count) {
    if (!c || !count) return SA_ERR_ARG;
    *count = c->rec_count;
    return SA_OK;
}

sa_status sa_get_stage_times(sa_ctx* c, double* ms, long long* steps) {
    if (!c || !ms || !steps) return SA_ERR_ARG;
    for (int i = 0; i < SA_N_STAGES; ++i) {
        ms[i] = c->stage_ms[i];
        c->stage_ms[i] = 0.0;
    }
    *steps = c->stage_steps;
    c->stage_steps = 0;
    return SA_OK;
}

sa_status sa_get_sizes(sa_ctx* c, sa_sizes* out) {
    if (!c || !out) return SA_ERR_ARG;
    if (!c->has_patch) return sa_fail(c, SA_ERR_STATE, "no patch");
    out->n_dof = c->n_dof;
    out->n_free = c->n_free;
    out->n_dir = c->n_dir;
    out->q_lat = c->q_lat;
    out->q_bot = c->q_bot;
    out->n_src = c->n_src;
    out->nnz_mk = c->nnz;
    out->nnz_a = c->nnz_a;
    out->step_index = c->n_step;
    out->n_elem = c->n_elem;
    out->hist_separable = c->sep.ok ? 1 : 0;
    out->sep_factors = c->sep.ok ? (long long)c->sep.n_tiles[0] * (64 + c->sep.tj[0]) +
                                       (long long)c->sep.n_tiles[1] * (64 + c->sep.tj[1])
                                 : 0;
    return SA_OK;
}

sa_status sa_get_field(sa_ctx* c, int field, double* out, long long count, int on_device) {
    sa_status st = check_usable(c);
    if (st) return st;
    if (!out) return sa_fail(c, SA_ERR_ARG, "out is NULL");
    if (!c->has_patch) return sa_fail(c, SA_ERR_STATE, "no patch");
    if (c->has_material) {
        if ((st = init_state_if_needed(c))) return st;
    }
    cudaStream_t s = c->stream;
    std::vector<double> h;
    long long need = 0;
    switch (field) {
        case SA_FIELD_THAT:
        case SA_FIELD_F: {
            need = c->n_dof;
            if (count < need) return sa_fail(c, SA_ERR_ARG, "count %lld < %lld", count, need);
            std::vector<double> in(c->n_dof);
            SA_CUDA(c, cudaMemcpyAsync(in.data(), field == SA_FIELD_THAT ? c->That.p : c->F0.p,
                                       sizeof(double) * c->n_dof, cudaMemcpyDeviceToHost, s));
            SA_CUDA(c, cudaStreamSynchronize(s));
            h.resize(c->n_dof);
            for (int i = 0; i < c->n_dof; ++i) h[i] = in[c->perm[i]];
            break;
        }
        case SA_FIELD_DTDN_LAT:
        case SA_FIELD_TT_BOT: {
            need = field == SA_FIELD_DTDN_LAT ? c->q_lat : c->q_bot;
            if (count < need) return sa_fail(c, SA_ERR_ARG, "count %lld < %lld", count, need);
            h.resize(need);
            if (need)
                SA_CUDA(c, cudaMemcpyAsync(h.data(), field == SA_FIELD_DTDN_LAT ? c->s_lat.p : c->tt_bot.p,
                                           sizeof(double) * need, cudaMemcpyDeviceToHost, s));
            SA_CUDA(c, cudaStreamSynchronize(s));
            break;
        }
        case SA_FIELD_LAT_X:
        case SA_FIELD_BOT_X: {
            const bool lat = field == SA_FIELD_LAT_X;
            const int Q = lat ? c->q_lat : c->q_bot;
            const int nc = lat ? 7 : 4;
            need = (long long)Q * nc;
            if (count < need) return sa_fail(c, SA_ERR_ARG, "count %lld < %lld", count, need);
            std::vector<double> soa(need);
            if (need)
                SA_CUDA(c, cudaMemcpyAsync(soa.data(), lat ? c->lat64.p : c->bot64.p,
                                           sizeof(double) * need, cudaMemcpyDeviceToHost, s));
            SA_CUDA(c, cudaStreamSynchronize(s));
            h.resize(need);
            for (int q = 0; q < Q; ++q)
                for (int k = 0; k < nc; ++k) h[(size_t)q * nc + k] = soa[(size_t)k * Q + q];
            break;
        }
        default:
            return sa_fail(c, SA_ERR_ARG, "unknown field %d", field);
    }
    if (on_device) {
        if (need) SA_CUDA(c, cudaMemcpy(out, h.data(), sizeof(double) * need, cudaMemcpyHostToDevice));
    } else {
        std::copy(h.begin(), h.end(), out);
    }
    return SA_OK;
}

sa_status sa_get_matrix_nnz(sa_ctx* c, long long* nnz) {
    if (!c || !nnz) return SA_ERR_ARG;
    if (!c->has_patch) return sa_fail(c, SA_ERR_STATE, "no patch");
    *nnz = c->nnz;
    return SA_OK;
}

sa_status sa_get_matrix(sa_ctx* c, int which, long long* rowptr, int* colind, double* vals) {
    sa_status st = check_usable(c);
    if (st) return st;
    if (!rowptr || !colind || !vals || (which != 0 && which != 1)) return sa_fail(c, SA_ERR_ARG, "bad argument");
    if (!c->has_patch || !c->has_material) return sa_fail(c, SA_ERR_STATE, "needs patch and material");
    SA_CUDA(c, cudaStreamSynchronize(c->stream));
    SA_CUDA(c, cudaMemcpy(rowptr, c->mk_ptr.p, sizeof(long long) * (c->n_dof + 1), cudaMemcpyDeviceToHost));
    SA_CUDA(c, cudaMemcpy(colind, c->mk_col.p, sizeof(int) * c->nnz, cudaMemcpyDeviceToHost));
    SA_CUDA(c, cudaMemcpy(vals, which == 0 ? c->M.p : c->K.p, sizeof(double) * c->nnz, cudaMemcpyDeviceToHost));
    const double f = which == 0 ? c->rho * c->cp : c->k;
    for (long long i = 0; i < c->nnz; ++i) vals[i] *= f;
    return SA_OK;
}

sa_status sa_get_state(sa_ctx* c, long long* n, double* T_hat, double* F) {
    sa_status st = check_usable(c);
    if (st) return st;
    if (!n || !T_hat || !F) return sa_fail(c, SA_ERR_ARG, "NULL argument");
    if (!c->has_patch || !c->has_material) return sa_fail(c, SA_ERR_STATE, "needs patch and material");
    if ((st = sa_get_field(c, SA_FIELD_THAT, T_hat, c->n_dof, 0))) return st;
    if ((st = sa_get_field(c, SA_FIELD_F, F, c->n_dof, 0))) return st;
    *n = c->n_step;
    return SA_OK;
}

sa_status sa_set_state(sa_ctx* c, long long n, const double* T_hat, const double* F) {
    sa_status st = check_usable(c);
    if (st) return st;
    if (!T_hat || !F || n < 0) return sa_fail(c, SA_ERR_ARG, "bad argument");
    if (!c->has_patch || !c->has_material) return sa_fail(c, SA_ERR_STATE, "needs patch and material");
    for (int i = 0; i < c->n_dof; ++i)
        if (!is_fin(T_hat[i]) || !is_fin(F[i])) return sa_fail(c, SA_ERR_NAN, "non-finite state");
    if ((st = init_state_if_needed(c))) return st;
    std::vector<double> Ti(c->n_dof), Fi(c->n_dof);
    for (int i = 0; i < c->n_dof; ++i) {
        Ti[c->perm[i]] = T_hat[i];
        Fi[c->perm[i]] = F[i];
    }
    cudaStream_t s = c->stream;
    SA_CUDA(c, cudaStreamSynchronize(s));
    SA_CUDA(c, cudaMemcpy(c->That.p, Ti.data(), sizeof(double) * c->n_dof, cudaMemcpyHostToDevice));
    SA_CUDA(c, cudaMemcpy(c->F0.p, Fi.data(), sizeof(double) * c->n_dof, cudaMemcpyHostToDevice));
    if (c->x_prev.p)   // the first step after a restore starts from T^n
        SA_CUDA(c, cudaMemcpy(c->x_prev.p, Ti.data(), sizeof(double) * c->n_dof, cudaMemcpyHostToDevice));
    SA_CUDA(c, cudaMemcpy(&c->st.p->n, &n, sizeof(long long), cudaMemcpyHostToDevice));
    // the cutoff's previous-step maxima belong to the old state: the first
    // step after a restore keeps the full sums
    if (c->sep.ref.p) SA_CUDA(c, cudaMemset(c->sep.ref.p, 0, sizeof(float) * c->sep.ref.n));
    c->n_step = n;
    return SA_OK;
}

// T (nrm null) or the heat-loss rates q~ (into out) and q^ (into out2) at
// n points.
static sa_status eval_points(sa_ctx* c, const double* pts, const double* nrm, int n, double* out,
                             double* out2, int on_device) {
    sa_status st = check_usable(c);
    if (st) return st;
    if (n < 0 || (n > 0 && (!pts || !out || (nrm && !out2))))
        return sa_fail(c, SA_ERR_ARG, "bad argument");
    if (!c->has_patch || !c->has_material) return sa_fail(c, SA_ERR_STATE, "needs patch and material");
    if (n == 0) return SA_OK;
    if ((st = init_state_if_needed(c))) return st;
    cudaStream_t s = c->stream;
    // mixed contexts: the centre search and the source sums in FP32 (the
    // source coefficients in the step's FP32 tables, which the next step
    // rewrites)
    const bool mixed = c->opt.precision == SA_MIXED;
    if (!c->ecent.p) {
        SA_ALLOC(c, c->ecent, (size_t)3 * c->n_elem);
        cudaError_t e = launch_elem_centers(c->dp, c->ecent.p, s);
        if (e == cudaSuccess && mixed) {
            SA_ALLOC(c, c->ecent32, (size_t)3 * c->n_elem);
            e = launch_to_f32((long long)3 * c->n_elem, c->ecent.p, c->ecent32.p, s);
        }
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "element centres");
    }
    int n_active = 0;
    if (c->has_scan && c->src_dt > 0.0 && c->n_step > 0 && c->n_src > 0) {
        const double alpha = c->k / (c->rho * c->cp);
        cudaError_t e = launch_prologue(nullptr, c->n_step, nullptr, c->n_src, c->src_pos.p, c->src_dt,
                                        alpha, c->spot_radius * c->spot_radius / (8.0 * alpha),
                                        c->opt.half_space_factor * c->E / (c->rho * c->cp),
                                        mixed ? SA_MIXED : SA_FP64, mixed ? nullptr : c->evT.p,
                                        mixed ? nullptr : c->evF.p, mixed ? c->src32T.p : nullptr,
                                        mixed ? c->src32F.p : nullptr, s);
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "eval prologue");
        n_active = (int)std::min<long long>(c->n_step, c->n_src);
    }
    const int nout = nrm ? 2 : 1;
    const double* dpts = pts;
    const double* dnrm = nrm;
    double* dout = out;
    double* dout2 = out2;
    if (!on_device) {
        if (c->eval_out.n < (size_t)nout * n || c->eval_pts.n < (size_t)6 * n) {
            // grown on demand, kept between calls
            SA_ALLOC(c, c->eval_pts, (size_t)6 * n);
            SA_ALLOC(c, c->eval_out, (size_t)2 * n);
        }
        SA_CUDA(c, cudaMemcpyAsync(c->eval_pts.p, pts, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
        dpts = c->eval_pts.p;
        if (nrm) {
            SA_CUDA(c, cudaMemcpyAsync(c->eval_pts.p + 3 * (size_t)n, nrm, sizeof(double) * 3 * n,
                                       cudaMemcpyHostToDevice, s));
            dnrm = c->eval_pts.p + 3 * (size_t)n;
        }
        dout = c->eval_out.p;
        dout2 = c->eval_out.p + n;
    }
    EvalFlux flux{dnrm, c->evF.p, mixed ? c->src32F.p : nullptr, c->k, dout2};
    cudaError_t e = launch_eval_points(c->dp, dpts, n, c->ecent.p, c->dperm.p, c->That.p,
                                       c->evT.p, n_active, c->x_ref, c->y_ref, c->z_top,
                                       c->length_scale, dout, s, mixed ? c->ecent32.p : nullptr,
                                       mixed ? c->src32T.p : nullptr, nrm ? &flux : nullptr);
    if (e != cudaSuccess) return sa_cuda_fail(c, e, "eval");
    if (!on_device) {
        SA_CUDA(c, cudaMemcpyAsync(out, dout, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        if (nrm)
            SA_CUDA(c, cudaMemcpyAsync(out2, dout2, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    }
    SA_CUDA(c, cudaStreamSynchronize(s));
    return SA_OK;
}

sa_status sa_eval_T(sa_ctx* c, const double* pts, int n, double* T_out, int on_device) {
    return eval_points(c, pts, nullptr, n, T_out, nullptr, on_device);
}

}  // extern "C"

namespace {
// acc += t - T_c: one more laser's temperature onto the superposed sum
__global__ void k_superpose(int n, const double* t, double* acc, double Tc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) acc[i] += t[i] - Tc;
}
}  // namespace

extern "C" {

sa_status sa_eval_T_superposed(sa_ctx* const* ctxs, int n_ctx, const double* pts, int n, double* T_out,
                               int on_device) {
    if (!ctxs || n_ctx < 1 || !ctxs[0]) return SA_ERR_ARG;
    sa_ctx* c0 = ctxs[0];
    sa_status st = check_usable(c0);
    if (st) return st;
    for (int l = 0; l < n_ctx; ++l) {
        sa_ctx* c = ctxs[l];
        if (!c) return sa_fail(c0, SA_ERR_ARG, "context %d is null", l);
        if ((st = check_usable(c))) return sa_fail(c0, st, "context %d is not usable", l);
        if (!c->has_patch || !c->has_material)
            return sa_fail(c0, SA_ERR_STATE, "context %d needs patch and material", l);
        if (c->n_dof != c0->n_dof || c->k != c0->k || c->rho != c0->rho || c->cp != c0->cp ||
            c->Tc != c0->Tc)
            return sa_fail(c0, SA_ERR_ARG, "context %d: another part or material than context 0", l);
        if (c->n_step != c0->n_step)
            return sa_fail(c0, SA_ERR_ARG, "context %d is at step %lld, context 0 at %lld", l,
                           c->n_step, c0->n_step);
    }
    if (n < 0 || (n > 0 && (!pts || !T_out))) return sa_fail(c0, SA_ERR_ARG, "bad argument");
    if (n == 0) return SA_OK;
    cudaStream_t s = c0->stream;
    if (c0->sup_acc.n < (size_t)n) {
        SA_ALLOC(c0, c0->sup_acc, (size_t)n);
        SA_ALLOC(c0, c0->sup_tmp, (size_t)n);
    }
    const double* dpts = pts;
    if (!on_device) {
        if (c0->sup_pts.n < (size_t)3 * n) SA_ALLOC(c0, c0->sup_pts, (size_t)3 * n);
        SA_CUDA(c0, cudaMemcpyAsync(c0->sup_pts.p, pts, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
        SA_CUDA(c0, cudaStreamSynchronize(s));   // the other contexts read the points on their streams
        dpts = c0->sup_pts.p;
    }
    // laser 0 into the sum, then each further laser's T - T_c onto it (each
    // evaluation is synchronous on its context's stream)
    if ((st = eval_points(c0, dpts, nullptr, n, c0->sup_acc.p, nullptr, 1))) return st;
    for (int l = 1; l < n_ctx; ++l) {
        if ((st = eval_points(ctxs[l], dpts, nullptr, n, c0->sup_tmp.p, nullptr, 1)))
            return sa_fail(c0, st, "context %d: %s", l, sa_last_error(ctxs[l]));
        k_superpose<<<(n + 255) / 256, 256, 0, s>>>(n, c0->sup_tmp.p, c0->sup_acc.p, c0->Tc);
        SA_CUDA(c0, cudaGetLastError());
        SA_CUDA(c0, cudaStreamSynchronize(s));   // sup_tmp is rewritten by the next laser
    }
    SA_CUDA(c0, cudaMemcpyAsync(T_out, c0->sup_acc.p, sizeof(double) * n,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    SA_CUDA(c0, cudaStreamSynchronize(s));
    return SA_OK;
}

sa_status sa_eval_flux(sa_ctx* c, const double* pts, const double* nrm, int n, double* q_tilde,
                       double* q_hat, int on_device) {
    if (!nrm && n > 0) return c ? sa_fail(c, SA_ERR_ARG, "nrm is NULL") : SA_ERR_ARG;
    return eval_points(c, pts, nrm, n, q_tilde, q_hat, on_device);
}

}  // extern "C"
