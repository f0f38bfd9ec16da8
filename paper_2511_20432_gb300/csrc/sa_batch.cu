// Batched stepping of many independent instances (patches of uneven size,
// different scans and powers) with one launch per stage.
//
// The instances' set-up is reused: their operators, boundary weights and
// points are concatenated into block-diagonal SELL operators and
// concatenated point / source tables.  Every instance's free rows and
// Dirichlet rows are padded to a multiple of 32 (one SELL slice never holds
// two instances) and its boundary points to a multiple of 128 (one
// history-sum tile never holds two instances).  The PCG runs per instance:
// dot products are summed per instance in fixed order (segmented
// reductions), each instance has its own alpha, beta and convergence test,
// and converged instances stop updating.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <type_traits>

#include "sa_async.cuh"
#include "sa_internal.h"

cudaError_t launch_prologue_batch(const DevStatus* st, int n_src_total, int n_inst,
                                  const int* src_inst, const int* src_off, const int* n_src,
                                  const double* coefE, const double* r2_8a, int* n_active,
                                  const double2* pos, double dt, double alpha, int precision,
                                  double4* s64T, double4* s64F, float4* s32T, float4* s32F,
                                  cudaStream_t s);
cudaError_t launch_history_batch(int precision, int P, int warps, DevStatus* st, int q_lat,
                                 int q_bot, const float* lat32, const float* bot32,
                                 const double* lat64, const double* bot64, const float4* s32F,
                                 const float4* s32T, const double4* s64F, const double4* s64T,
                                 double* s_lat, double* tt_bot, int n_inst, const int* qlat_off,
                                 const int* qbot_off, const int* src_off, const int* n_active,
                                 cudaStream_t s);

struct sa_batch {
    sa_options opt;
    std::string err;
    bool poisoned = false;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    std::vector<sa_ctx*> inst;
    int n_inst = 0;
    double k = 0, rho = 0, cp = 0, Tc = 0;
    double dt = 0, theta = -1;
    bool built = false;
    long long n_step = 0;
    // layout
    std::vector<int> free_off, dir_off, qlat_off, qbot_off, src_off, slice_off_a, slice_off_b;
    int n_free = 0, n_dir = 0, n_dof = 0, q_lat = 0, q_bot = 0, n_src = 0;
    int wlat_rows = 0;
    // device: geometry / data
    DBuf<double> lat64, bot64, s_lat, tt_bot;
    DBuf<float> lat32, bot32;
    DBuf<int> d_qlat_off, d_qbot_off, d_src_off, d_src_inst, d_n_src, d_n_active;
    DBuf<double> d_coefE, d_r2_8a;
    DBuf<double2> src_pos;
    DBuf<double4> s64T, s64F;
    DBuf<float4> s32T, s32F;
    DBuf<int> wlat_rowdof, wlat_ptr, wlat_col, wbot_ptr, wbot_col;
    DBuf<double> wlat_val, wbot_val;
    SellDev a_s, r_s, mbot_s;
    DBuf<double> a_val, r_K, r_M, mbot_val, a_dinv, mbot_dinv;
    DBuf<float> a_val32, r_K32, r_M32, mbot_val32;
    // mixed path, slices without Dirichlet columns: 16-bit column offsets and
    // M as bf16 (8 bytes a nonzero in the right-hand side; empty when an
    // offset does not fit)
    DBuf<short> r_col16lo;
    DBuf<unsigned short> r_M16;
    DBuf<int> slice_inst_a, slice_inst_b, d_slice_off_a, d_slice_off_b;
    // state and work
    DBuf<double> That, F0, F1, gnew, bbot, r0, bsq, dirv, wr, wz, wp0, wp1, wq, dev64, partials, inst_state;
    DBuf<float> dev32, wzl, wpl0, wpl1;
    DBuf<int> inst_iters;
    DBuf<unsigned> counters;
    DBuf<DevStatus> st;
    // fast diagonalization of every instance's main solve (when all have it)
    bool fd_on = false;
    int fd_mmax = 0;
    DBuf<unsigned char> fd_desc;   // BFd per instance
    DBuf<int> fd_loff;             // 3 x (n_inst + 1): line offsets per direction
    DBuf<unsigned char> fdS, fdZ;  // n_free x VT
    // the same for the bottom projections (2-D)
    bool fdb_on = false;
    DBuf<unsigned char> fdb_desc;
    DBuf<int> fdb_loff;
    DBuf<unsigned char> fdbS, fdbZ;   // n_dir x VT
    // separable history sums over all instances (every face a rectangle)
    SepPlan sep;
    int pcg_grid = 0;
    int hist_P = 4, hist_W = 8;
    cudaGraphExec_t graph_exec = nullptr;
};

namespace {

sa_status bfail(sa_batch* b, sa_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    return s;
}

sa_status bcuda(sa_batch* b, cudaError_t e, const char* where) {
    if (b) {
        b->poisoned = true;
        b->err = std::string(where) + ": " + cudaGetErrorString(e);
    }
    return SA_ERR_CUDA;
}

#define B_CUDA(b, call)                                                 \
    do {                                                                \
        cudaError_t e__ = (call);                                       \
        if (e__ != cudaSuccess) return bcuda(b, e__, #call);            \
    } while (0)

#define B_ALLOC(b, buf, count)                                          \
    do {                                                                \
        cudaError_t e__ = (buf).alloc(count);                           \
        if (e__ != cudaSuccess) {                                       \
            cudaGetLastError();                                         \
            return bfail(b, SA_ERR_OOM, "allocation of %s", #buf);      \
        }                                                               \
    } while (0)

template <class T>
sa_status bupload(sa_batch* b, DBuf<T>& d, const std::vector<T>& v, const char* what) {
    if (d.alloc(std::max<size_t>(v.size(), 1)) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, SA_ERR_OOM, "allocation of %s", what);
    }
    if (!v.empty() && cudaMemcpy(d.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return bcuda(b, cudaGetLastError(), what);
    return SA_OK;
}

int pad_to(int v, int m) { return (v + m - 1) / m * m; }

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// Copy one SoA component range with a shift: dst[i] = src[i] - shift.
__global__ void k_copy_shift(long long n, const double* src, double* dst, double shift) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i] - shift;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// grid barrier with a bounded wait (cooperative launch; count starts at zero)
__device__ __forceinline__ bool bgrid_barrier(unsigned* count, unsigned& nb, int* err) {
    return sa_dev::count_barrier(count, nb, err, SA_DEV_TIMEOUT);
}

// One instance's fast-diagonalization data (device pointers of its context).
struct BFd {
    int m[3];
    int row0;                 // first batch row of the instance
    const void* U[3];
    const void* Ut[3];
    const void* lamc[3];
    double cM;
};

// per-instance solver scalars (FP64), laid out [field][instance]
enum { IS_RZ = 0, IS_BB, IS_ALPHA, IS_BETA, IS_RR, IS_CONV, IS_NFIELDS };

template <typename VT>
struct BPcgArgs {
    int n, n_slices, n_inst;
    const long long* sptr;
    const int* col32;
    const short* col16;
    const VT* val;
    const double* val_hi;
    const int* slice_inst;
    const int* slice_off;     // n_inst + 1
    const double* dinv;
    const double* b;
    const double* r0;
    const double* bsq;        // with r0: b_i^2 per row (else b = r0 + A x by an SpMV)
    double* x;
    double* r;
    double* z;
    double* p0;
    double* p1;
    double* q;
    VT* zl;
    VT* pl0;
    VT* pl1;
    double* part;             // 3 * n_slices
    double* is;               // IS_NFIELDS * n_inst
    int* iters;               // n_inst
    unsigned* active;         // 2 counters
    DevStatus* st;
    int which;
    double tol;
    int max_iter;
    const BFd* fd;            // per-instance fast diagonalization, or null (Jacobi)
    int fd_nd;                // its dimension: 3 (main solves) or 2 (bottom projections)
    const int* fd_loff;       // 3 x (n_inst + 1)
    const VT* fdS;            // scaling per row
    VT* fdZ;                  // work vector
    int fd_mmax;              // line length the staged matrices hold (0: read through L1)
};

template <typename VT>
__device__ __forceinline__ int bcol(const BPcgArgs<VT>& a, long long e, int row) {
    return a.col16 ? row + (int)__ldg(a.col16 + e) : __ldg(a.col32 + e);
}

// Batched fast-diagonalization preconditioner z = S A_box^{-1} S r over
// every instance (independent grids): on entry fdZ = S r on all rows (grid
// barrier passed); 2 nd - 1 passes (3-D: U_0^T, U_1^T, U_2 D U_2^T, U_1, U_0;
// 2-D: U_0^T, U_1 D U_1^T, U_0) over the lines of all instances, one warp
// per line; the last pass writes z (FP64) and its operator-precision copy.
// Lines have at most 128 entries.  Inside the iteration loop the lines of
// instances that have converged are skipped (skip_converged): one straggler
// then costs its own lines, not every instance's.  A block takes a contiguous range of each
// pass's lines (instance-major), so it meets one or a few instances; for
// each it stages the instance's line matrix (and the middle pass's second
// one) in shared memory (Wsm: 2 m^2 entries), instead of reading it per
// line through L1, where a pass over hundreds of instances' matrices misses
// to L2 on every line.
template <typename VT>
__device__ bool bfd_apply(const BPcgArgs<VT>& a, VT* xs, VT* Wsm, double* z, VT* zl, unsigned* bc,
                          unsigned& bg, int* err, bool skip_converged) {
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    const int NI = a.n_inst;
    VT* Z = a.fdZ;
    const int nd = a.fd_nd, npass = 2 * nd - 1;
    for (int pass = 0; pass < npass; ++pass) {
        const int d = pass < nd ? pass : npass - 1 - pass;
        const bool mid = pass == nd - 1;
        const int* loff = a.fd_loff + d * (NI + 1);
        const int nlines = loff[NI];
        const int chunk = (nlines + (int)gridDim.x - 1) / (int)gridDim.x;
        const int l0 = min(nlines, (int)blockIdx.x * chunk), l1 = min(nlines, l0 + chunk);
        int inst = 0;                  // the instance of line l0: loff[inst] <= l0 < loff[inst + 1]
        {
            int lo = 0, hi = NI;
            while (hi - lo > 1) {
                const int md = (lo + hi) >> 1;
                if (loff[md] <= l0) lo = md;
                else hi = md;
            }
            inst = lo;
        }
        for (int s0 = l0; s0 < l1;) {
            while (inst + 1 < NI && loff[inst + 1] <= s0) ++inst;
            const int s1 = min(l1, loff[inst + 1]);
            if (skip_converged && ((volatile double*)a.is)[IS_CONV * NI + inst] != 0.0) {
                s0 = s1;               // a converged instance's z is not used again
                continue;
            }
            const BFd& f = a.fd[inst];
            const int m0 = f.m[0], m1 = f.m[1];
            const int m = f.m[d];
            const int stride = d == 0 ? 1 : (d == 1 ? m0 : m0 * m1);
            // this instance's matrices into shared memory (all copies of a
            // thread in flight at once); the previous segment is done with them
            __syncthreads();
            const VT* Wg = (const VT*)(pass < nd ? f.U[d] : f.Ut[d]);
            const VT* W2g = (const VT*)f.Ut[nd - 1];
            const bool staged = a.fd_mmax > 0;   // else (too large to stage) through L1
            if (staged) {
                for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
                    sa_dev::cp_async_ca<sizeof(VT)>(Wsm + t, Wg + t);
                    if (mid) sa_dev::cp_async_ca<sizeof(VT)>(Wsm + m * m + t, W2g + t);
                }
                sa_dev::cp_async_wait_all();
                __syncthreads();
            }
            const VT* W = staged ? Wsm : Wg;
            const VT* W2 = staged ? Wsm + m * m : W2g;
            for (int Lg = s0 + wib; Lg < s1; Lg += nwb) {
                const int L = Lg - loff[inst];
                const long long base = f.row0 + (d == 0 ? (long long)L * m0
                                                : (d == 1 ? (long long)(L / m0) * (m0 * m1) + (L % m0) : L));
                for (int q = lane; q < m; q += 32) xs[q] = __ldcg(Z + base + (long long)q * stride);
                __syncwarp();
                VT y[4] = {(VT)0, (VT)0, (VT)0, (VT)0};
#pragma unroll 4
                for (int q = 0; q < m; ++q) {
                    const VT xq = xs[q];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int o = lane + 32 * t;
                        if (o < m) y[t] = fma(W[q * m + o], xq, y[t]);
                    }
                }
                if (mid) {
                    const VT li = (VT)f.cM + ((const VT*)f.lamc[0])[L % m0] +
                                  (nd == 3 ? ((const VT*)f.lamc[1])[L / m0] : (VT)0);
                    const VT* l2 = (const VT*)f.lamc[nd - 1];
                    __syncwarp();
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int o = lane + 32 * t;
                        if (o < m) xs[o] = y[t] / (li + l2[o]);
                        y[t] = (VT)0;
                    }
                    __syncwarp();
#pragma unroll 4
                    for (int q = 0; q < m; ++q) {
                        const VT xq = xs[q];
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const int o = lane + 32 * t;
                            if (o < m) y[t] = fma(W2[q * m + o], xq, y[t]);
                        }
                    }
                }
                __syncwarp();
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int o = lane + 32 * t;
                    if (o < m) {
                        const long long idx = base + (long long)o * stride;
                        if (pass == npass - 1) {
                            const VT u = a.fdS[idx] * y[t];
                            z[idx] = (double)u;
                            zl[idx] = u;
                        } else {
                            Z[idx] = y[t];
                        }
                    }
                }
                __syncwarp();
            }
            s0 = s1;
        }
        if (!bgrid_barrier(bc, bg, err)) return false;
    }
    return true;
}

// dynamic shared memory of k_pcg_batch: two staged line matrices
template <typename VT>
size_t batch_pcg_smem(int mmax) { return (size_t)2 * mmax * mmax * sizeof(VT); }

// The line length to stage for: 0 (no staging, matrices read through L1)
// when two matrices would not fit beside the kernel's static scratch
// (32 x 128 entries) in a block's 227 KB.
template <typename VT>
int batch_pcg_stage_m(int mmax) {
    const size_t limit = (size_t)227 * 1024 - (size_t)32 * 128 * sizeof(VT) - 1024;
    return batch_pcg_smem<VT>(mmax) <= limit ? mmax : 0;
}

template <typename VT>
__global__ void __launch_bounds__(1024, 1) k_pcg_batch(BPcgArgs<VT> a) {
    constexpr bool LO = std::is_same<VT, float>::value;
    const int lane = threadIdx.x & 31;
    const int nwb = blockDim.x >> 5;
    const int gw = blockIdx.x * nwb + (threadIdx.x >> 5);
    const int nw = gridDim.x * nwb;
    unsigned* bc = &a.st->bar_count[2 + a.which];
    unsigned bg = 0;                       // barriers passed
    int* err = &a.st->err;
    const int S = a.n_slices, NI = a.n_inst;
    volatile double* is = a.is;
    __shared__ VT xsb[32][128];            // per-warp line scratch (fast diagonalization)
    VT* xs = xsb[threadIdx.x >> 5];
    extern __shared__ __align__(16) unsigned char bsm[];   // the staged line matrices
    VT* Wsm = (VT*)bsm;
    const bool fd = a.fd != nullptr;
    VT* const zlw = LO ? a.zl : (VT*)a.z;
    // ---- phase A: r = b - A x (FP64 values) or r = r0 (b = r0 + A x)
    for (int sl = gw; sl < S; sl += nw) {
        const long long base = a.sptr[sl];
        const int w = (int)((a.sptr[sl + 1] - base) >> 5);
        const int i = sl * 32 + lane;
        const int ir = min(i, a.n - 1);
        double acc = 0.0;
        if (a.r0 == nullptr) {
            for (int k = 0; k < w; ++k) {
                const long long e = base + 32ll * k + lane;
                acc = fma(__ldg(a.val_hi + e), a.x[bcol(a, e, ir)], acc);
            }
        } else if (a.bsq == nullptr) {
            VT s = 0;
            for (int k = 0; k < w; ++k) {
                const long long e = base + 32ll * k + lane;
                s = fma(__ldg(a.val + e), (VT)a.x[bcol(a, e, ir)], s);
            }
            acc = (double)s;
        }
        double ri = 0.0, bi = 0.0, zi = 0.0;
        if (i < a.n) {
            if (a.r0 == nullptr) {
                bi = a.b[i];
                ri = bi - acc;
            } else {
                ri = a.r0[i];
                // b_i^2 from the right-hand-side kernel when given (no SpMV;
                // only the square is used)
                bi = a.bsq ? 0.0 : ri + acc;
            }
            a.r[i] = ri;
            if (fd) {
                a.fdZ[i] = a.fdS[i] * (VT)ri;
            } else {
                zi = a.dinv[i] * ri;
                a.z[i] = zi;
                if (LO) a.zl[i] = (VT)zi;
            }
        }
        const double b2 = a.bsq ? (i < a.n ? a.bsq[i] : 0.0) : bi * bi;
        const double t0 = warp_sum(ri * zi), t1 = warp_sum(ri * ri), t2 = warp_sum(b2);
        if (lane == 0) {
            a.part[sl] = t0;
            a.part[S + sl] = t1;
            a.part[2 * S + sl] = t2;
        }
    }
    if (!bgrid_barrier(bc, bg, err)) return;
    if (fd) {
        // z = P^{-1} r, then (r, z) per slice
        if (!bfd_apply(a, xs, Wsm, a.z, zlw, bc, bg, err, false)) return;
        for (int sl = gw; sl < S; sl += nw) {
            const int i = sl * 32 + lane;
            const double t0 = warp_sum(i < a.n ? a.r[i] * a.z[i] : 0.0);
            if (lane == 0) a.part[sl] = t0;
        }
        if (!bgrid_barrier(bc, bg, err)) return;
    }
    // R0: per-instance rz, rr, bb; convergence; active count
    for (int i = gw; i < NI; i += nw) {
        const int s0 = a.slice_off[i], s1 = a.slice_off[i + 1];
        double t[3];
        for (int f = 0; f < 3; ++f) {
            const volatile double* pf = a.part + (long long)f * S;
            double v = 0.0;
            for (int s = s0 + lane; s < s1; s += 32) v += pf[s];
            t[f] = warp_sum(v);
        }
        if (lane == 0) {
            is[IS_RZ * NI + i] = t[0];
            is[IS_RR * NI + i] = t[1];
            is[IS_BB * NI + i] = t[2];
            is[IS_BETA * NI + i] = 0.0;
            const bool conv = t[1] <= a.tol * a.tol * t[2];
            is[IS_CONV * NI + i] = conv ? 1.0 : 0.0;
            a.iters[i] = 0;
            if (!conv) atomicAdd(&a.active[0], 1u);
        }
    }
    if (!bgrid_barrier(bc, bg, err)) return;
    int it = 0;
    unsigned n_active = *((volatile unsigned*)&a.active[0]);
    double* pc = a.p0;
    double* pn = a.p1;
    VT* plc = LO ? a.pl0 : (VT*)a.p0;
    VT* pln = LO ? a.pl1 : (VT*)a.p1;
    const VT* zl = LO ? a.zl : (const VT*)a.z;
    while (n_active > 0 && it < a.max_iter) {
        const bool first = (it == 0);
        // ---- B: p' = z + beta p ; q = A p' ; (p', q) per slice
        for (int sl = gw; sl < S; sl += nw) {
            const int inst = a.slice_inst[sl];
            const bool conv = is[IS_CONV * NI + inst] != 0.0;
            double pq = 0.0;
            if (!conv) {
                const double beta = is[IS_BETA * NI + inst];
                const VT bl = (VT)beta;
                const long long base = a.sptr[sl];
                const int w = (int)((a.sptr[sl + 1] - base) >> 5);
                const int i = sl * 32 + lane;
                const int ir = min(i, a.n - 1);
                VT acc = 0;
                constexpr int B = std::is_same<VT, float>::value ? 8 : 4;
                for (int k = 0; k < w; k += B) {
                    int jj[B];
                    VT vv[B], gg[B];
#pragma unroll
                    for (int u = 0; u < B; ++u) {
                        const bool ok = k + u < w;
                        const long long e = base + 32ll * (ok ? k + u : 0) + lane;
                        jj[u] = ok ? bcol(a, e, ir) : ir;
                        vv[u] = ok ? __ldg(a.val + e) : (VT)0;
                    }
#pragma unroll
                    for (int u = 0; u < B; ++u) gg[u] = first ? zl[jj[u]] : fma(bl, plc[jj[u]], zl[jj[u]]);
#pragma unroll
                    for (int u = 0; u < B; ++u) acc = fma(vv[u], gg[u], acc);
                }
                if (i < a.n) {
                    const double pi = first ? a.z[i] : fma(beta, pc[i], a.z[i]);
                    pn[i] = pi;
                    if (LO) pln[i] = (VT)pi;
                    a.q[i] = (double)acc;
                    pq = pi * (double)acc;
                }
            } else {
                // converged instance: keep its direction buffers consistent
                const int i = sl * 32 + lane;
                if (i < a.n) {
                    pn[i] = pc[i];
                    if (LO) pln[i] = plc[i];
                }
            }
            pq = warp_sum(pq);
            if (lane == 0) a.part[sl] = pq;
        }
        if (!bgrid_barrier(bc, bg, err)) return;
        // R1: alpha per instance; reset the next active counter
        if (gw == 0 && lane == 0) a.active[(it + 1) & 1] = 0u;
        for (int i = gw; i < NI; i += nw) {
            const int s0 = a.slice_off[i], s1 = a.slice_off[i + 1];
            double v = 0.0;
            for (int s = s0 + lane; s < s1; s += 32) v += ((volatile double*)a.part)[s];
            v = warp_sum(v);
            if (lane == 0) is[IS_ALPHA * NI + i] = (is[IS_CONV * NI + i] != 0.0) ? 0.0 : is[IS_RZ * NI + i] / v;
        }
        if (!bgrid_barrier(bc, bg, err)) return;
        // ---- C: x += alpha p' ; r -= alpha q ; z = D^{-1} r per slice
        for (int sl = gw; sl < S; sl += nw) {
            const int inst = a.slice_inst[sl];
            double rr = 0.0, rz = 0.0;
            if (is[IS_CONV * NI + inst] == 0.0) {
                const double alpha = is[IS_ALPHA * NI + inst];
                const int i = sl * 32 + lane;
                if (i < a.n) {
                    a.x[i] = fma(alpha, pn[i], a.x[i]);
                    const double ri = fma(-alpha, a.q[i], a.r[i]);
                    a.r[i] = ri;
                    rr = ri * ri;
                    if (fd) {
                        a.fdZ[i] = a.fdS[i] * (VT)ri;
                    } else {
                        const double zi = a.dinv[i] * ri;
                        a.z[i] = zi;
                        if (LO) a.zl[i] = (VT)zi;
                        rz = ri * zi;
                    }
                }
            }
            rr = warp_sum(rr);
            rz = warp_sum(rz);
            if (lane == 0) {
                a.part[S + sl] = rr;
                a.part[2 * S + sl] = rz;
            }
        }
        if (!bgrid_barrier(bc, bg, err)) return;
        if (fd) {
            // R2a: convergence from (r, r) before the preconditioner: an
            // instance that has converged needs no z, and when every one has
            // (the box preconditioner is the inverse: usually after the first
            // update) the application and its barriers are skipped
            for (int i = gw; i < NI; i += nw) {
                const int s0 = a.slice_off[i], s1 = a.slice_off[i + 1];
                const volatile double* pf = a.part + S;
                double v = 0.0;
                for (int s = s0 + lane; s < s1; s += 32) v += pf[s];
                const double rr = warp_sum(v);
                if (lane == 0 && is[IS_CONV * NI + i] == 0.0) {
                    is[IS_RR * NI + i] = rr;
                    a.iters[i] = it + 1;
                    const bool conv = rr <= a.tol * a.tol * is[IS_BB * NI + i];
                    if (!(rr == rr)) atomicOr(err, SA_DEV_NAN);
                    if (conv) is[IS_CONV * NI + i] = 1.0;
                    else atomicAdd(&a.active[(it + 1) & 1], 1u);
                }
            }
            if (!bgrid_barrier(bc, bg, err)) return;
            if (*((volatile unsigned*)&a.active[(it + 1) & 1]) > 0u) {
                // z = P^{-1} r (every row; converged instances ignore theirs), then (r, z)
                if (!bfd_apply(a, xs, Wsm, a.z, zlw, bc, bg, err, true)) return;
                for (int sl = gw; sl < S; sl += nw) {
                    const int inst = a.slice_inst[sl];
                    const int i = sl * 32 + lane;
                    double rz = 0.0;
                    if (is[IS_CONV * NI + inst] == 0.0 && i < a.n) rz = a.r[i] * a.z[i];
                    rz = warp_sum(rz);
                    if (lane == 0) a.part[2 * S + sl] = rz;
                }
                if (!bgrid_barrier(bc, bg, err)) return;
                // R2b: beta of the instances still running
                for (int i = gw; i < NI; i += nw) {
                    const int s0 = a.slice_off[i], s1 = a.slice_off[i + 1];
                    const volatile double* pf = a.part + 2 * S;
                    double v = 0.0;
                    for (int s = s0 + lane; s < s1; s += 32) v += pf[s];
                    const double rzn = warp_sum(v);
                    if (lane == 0 && is[IS_CONV * NI + i] == 0.0) {
                        is[IS_BETA * NI + i] = rzn / is[IS_RZ * NI + i];
                        is[IS_RZ * NI + i] = rzn;
                    }
                }
                if (!bgrid_barrier(bc, bg, err)) return;
            }
        } else {
            // R2: convergence, beta, active count
            for (int i = gw; i < NI; i += nw) {
                const int s0 = a.slice_off[i], s1 = a.slice_off[i + 1];
                double t[2];
                for (int f = 0; f < 2; ++f) {
                    const volatile double* pf = a.part + (long long)(1 + f) * S;
                    double v = 0.0;
                    for (int s = s0 + lane; s < s1; s += 32) v += pf[s];
                    t[f] = warp_sum(v);
                }
                if (lane == 0 && is[IS_CONV * NI + i] == 0.0) {
                    const double rr = t[0], rzn = t[1];
                    is[IS_RR * NI + i] = rr;
                    is[IS_BETA * NI + i] = rzn / is[IS_RZ * NI + i];
                    is[IS_RZ * NI + i] = rzn;
                    a.iters[i] = it + 1;
                    const bool conv = rr <= a.tol * a.tol * is[IS_BB * NI + i];
                    if (!(rr == rr)) atomicOr(err, SA_DEV_NAN);
                    if (conv) is[IS_CONV * NI + i] = 1.0;
                    else atomicAdd(&a.active[(it + 1) & 1], 1u);
                }
            }
            if (!bgrid_barrier(bc, bg, err)) return;
        }
        n_active = *((volatile unsigned*)&a.active[(it + 1) & 1]);
        ++it;
        double* t = pc;
        pc = pn;
        pn = t;
        VT* tl = plc;
        plc = pln;
        pln = tl;
        if (*((volatile int*)err) & SA_DEV_NAN) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int itmax = 0;
        for (int i = 0; i < NI; ++i) itmax = max(itmax, a.iters[i]);
        if (a.which == 0) {
            a.st->pcg_iters = itmax;
            if (n_active > 0) atomicOr(err, SA_DEV_NOT_CONVERGED);
        } else {
            a.st->bot_iters = itmax;
            if (n_active > 0) atomicOr(err, SA_DEV_BOT_NOT_CONVERGED);
        }
    }
}

template <typename VT>
cudaError_t launch_pcg_batch(sa_batch* b, int which, const SellDev& s, const void* val,
                             const double* val_hi, const int* slice_inst, const int* slice_off,
                             const double* dinv, const double* rhs, const double* r0, double* x,
                             cudaStream_t st) {
    BPcgArgs<VT> a;
    a.n = s.n;
    a.n_slices = s.n_slices;
    a.n_inst = b->n_inst;
    a.sptr = s.sptr.p;
    a.col16 = s.col16.p;
    a.col32 = s.col16.p ? nullptr : s.col.p;
    a.val = (const VT*)val;
    a.val_hi = val_hi;
    a.slice_inst = slice_inst;
    a.slice_off = slice_off;
    a.dinv = dinv;
    a.b = rhs;
    a.r0 = r0;
    a.bsq = (r0 != nullptr && which == 0) ? b->bsq.p : nullptr;
    a.x = x;
    a.r = b->wr.p;
    a.z = b->wz.p;
    a.p0 = b->wp0.p;
    a.p1 = b->wp1.p;
    a.q = b->wq.p;
    a.zl = (VT*)b->wzl.p;
    a.pl0 = (VT*)b->wpl0.p;
    a.pl1 = (VT*)b->wpl1.p;
    a.part = b->partials.p;
    a.is = b->inst_state.p;
    a.iters = b->inst_iters.p + which * b->n_inst;
    a.active = b->counters.p;
    a.st = b->st.p;
    a.which = which;
    a.tol = b->opt.pcg_tol;
    a.max_iter = b->opt.pcg_max_iter;
    const bool fd = which == 0 ? b->fd_on : b->fdb_on;
    a.fd = fd ? (const BFd*)(which == 0 ? b->fd_desc.p : b->fdb_desc.p) : nullptr;
    a.fd_nd = which == 0 ? 3 : 2;
    a.fd_loff = fd ? (which == 0 ? b->fd_loff.p : b->fdb_loff.p) : nullptr;
    a.fdS = fd ? (const VT*)(which == 0 ? b->fdS.p : b->fdbS.p) : nullptr;
    a.fdZ = fd ? (VT*)(which == 0 ? b->fdZ.p : b->fdbZ.p) : nullptr;
    a.fd_mmax = fd ? batch_pcg_stage_m<VT>(b->fd_mmax) : 0;
    cudaError_t e = cudaMemsetAsync(&b->st.p->bar_count[2 + which], 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->counters.p, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->pcg_grid);
    cfg.blockDim = dim3(1024);
    cfg.stream = st;
    cfg.dynamicSmemBytes = batch_pcg_smem<VT>(a.fd_mmax);
    e = cudaFuncSetAttribute(k_pcg_batch<VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cfg.dynamicSmemBytes);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_pcg_batch<VT>, a);
}

// ---------------------------------------------------------------------------
// concatenation of the instances (host patterns + device copies)
// ---------------------------------------------------------------------------
// Append instance SELL h (rows = its local rows, columns mapped by colmap)
// to the batch pattern out at row offset row0.  Slices are whole.
void append_sell(const SellHost& h, int row0, const std::vector<int>& colmap, SellHost& out,
                 bool keep16) {
    const long long base = out.sptr.empty() ? 0 : out.sptr.back();
    if (out.sptr.empty()) out.sptr.push_back(0);
    for (int s = 0; s < h.n_slices; ++s) out.sptr.push_back(base + h.sptr[s + 1]);
    for (size_t e = 0; e < h.col.size(); ++e) out.col.push_back(colmap.empty() ? h.col[e] + row0 : colmap[h.col[e]]);
    if (keep16) out.col16.insert(out.col16.end(), h.col16.begin(), h.col16.end());
    out.n_slices += h.n_slices;
    (void)row0;
}

cudaError_t d2d(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
}

sa_status build(sa_batch* b, double theta, double dt) {
    cudaStream_t s = b->stream;
    const int NI = b->n_inst;
    // every instance prepared for (theta, dt)
    for (int i = 0; i < NI; ++i) {
        sa_status st = sa_prepare(b->inst[i], theta, dt);
        if (st) return bfail(b, st, "instance %d: %s", i, sa_last_error(b->inst[i]));
        if (b->inst[i]->n_step != b->inst[0]->n_step)
            return bfail(b, SA_ERR_STATE, "instances are at different steps");
    }
    B_CUDA(b, cudaDeviceSynchronize());
    // ---- layout
    b->free_off.assign(NI + 1, 0);
    b->dir_off.assign(NI + 1, 0);
    b->qlat_off.assign(NI + 1, 0);
    b->qbot_off.assign(NI + 1, 0);
    b->src_off.assign(NI + 1, 0);
    for (int i = 0; i < NI; ++i) {
        const sa_ctx* c = b->inst[i];
        b->free_off[i + 1] = b->free_off[i] + pad_to(c->n_free, 32);
        b->dir_off[i + 1] = b->dir_off[i] + pad_to(c->n_dir, 32);
        b->qlat_off[i + 1] = b->qlat_off[i] + pad_to(c->q_lat, 128);
        b->qbot_off[i + 1] = b->qbot_off[i] + pad_to(c->q_bot, 128);
        b->src_off[i + 1] = b->src_off[i] + c->n_src;
    }
    b->n_free = b->free_off[NI];
    b->n_dir = b->dir_off[NI];
    b->n_dof = b->n_free + b->n_dir;
    b->q_lat = b->qlat_off[NI];
    b->q_bot = b->qbot_off[NI];
    b->n_src = b->src_off[NI];
    const bool mixed = b->opt.precision == SA_MIXED;

    // ---- points (FP64 shifted to each instance's reference, FP32 as is)
    B_ALLOC(b, b->lat64, (size_t)7 * std::max(b->q_lat, 1));
    B_ALLOC(b, b->bot64, (size_t)4 * std::max(b->q_bot, 1));
    B_ALLOC(b, b->lat32, (size_t)6 * std::max(b->q_lat, 1));
    B_ALLOC(b, b->bot32, (size_t)3 * std::max(b->q_bot, 1));
    B_CUDA(b, cudaMemsetAsync(b->lat64.p, 0, sizeof(double) * b->lat64.n, s));
    B_CUDA(b, cudaMemsetAsync(b->bot64.p, 0, sizeof(double) * b->bot64.n, s));
    B_CUDA(b, cudaMemsetAsync(b->lat32.p, 0, sizeof(float) * b->lat32.n, s));
    B_CUDA(b, cudaMemsetAsync(b->bot32.p, 0, sizeof(float) * b->bot32.n, s));
    for (int i = 0; i < NI; ++i) {
        const sa_ctx* c = b->inst[i];
        const double shift[7] = {c->x_ref, c->y_ref, c->z_top, 0, 0, 0, 0};
        for (int k = 0; k < 7 && c->q_lat; ++k) {
            const long long n = c->q_lat;
            k_copy_shift<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
                n, c->lat64.p + (size_t)k * c->q_lat, b->lat64.p + (size_t)k * b->q_lat + b->qlat_off[i],
                shift[k]);
        }
        const double shiftb[4] = {c->x_ref, c->y_ref, c->z_top, 0};
        for (int k = 0; k < 4 && c->q_bot; ++k) {
            const long long n = c->q_bot;
            k_copy_shift<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
                n, c->bot64.p + (size_t)k * c->q_bot, b->bot64.p + (size_t)k * b->q_bot + b->qbot_off[i],
                shiftb[k]);
        }
        for (int k = 0; k < 6; ++k)
            B_CUDA(b, d2d(b->lat32.p + (size_t)k * b->q_lat + b->qlat_off[i], c->lat32.p + (size_t)k * c->q_lat,
                          sizeof(float) * c->q_lat, s));
        for (int k = 0; k < 3; ++k)
            B_CUDA(b, d2d(b->bot32.p + (size_t)k * b->q_bot + b->qbot_off[i], c->bot32.p + (size_t)k * c->q_bot,
                          sizeof(float) * c->q_bot, s));
    }
    B_CUDA(b, cudaGetLastError());
    B_ALLOC(b, b->s_lat, std::max(b->q_lat, 1));
    B_ALLOC(b, b->tt_bot, std::max(b->q_bot, 1));

    // ---- sources
    {
        std::vector<int> src_inst(std::max(b->n_src, 1), 0), nsrc(NI);
        std::vector<double> coefE(NI), r2(NI);
        const double alpha = b->k / (b->rho * b->cp);
        for (int i = 0; i < NI; ++i) {
            const sa_ctx* c = b->inst[i];
            for (int g = b->src_off[i]; g < b->src_off[i + 1]; ++g) src_inst[g] = i;
            nsrc[i] = c->n_src;
            coefE[i] = c->opt.half_space_factor * c->E / (c->rho * c->cp);
            r2[i] = c->spot_radius * c->spot_radius / (8.0 * alpha);
        }
        sa_status st;
        if ((st = bupload(b, b->d_src_inst, src_inst, "src_inst"))) return st;
        if ((st = bupload(b, b->d_n_src, nsrc, "n_src"))) return st;
        if ((st = bupload(b, b->d_coefE, coefE, "coefE"))) return st;
        if ((st = bupload(b, b->d_r2_8a, r2, "r2_8a"))) return st;
        if ((st = bupload(b, b->d_src_off, b->src_off, "src_off"))) return st;
        if ((st = bupload(b, b->d_qlat_off, b->qlat_off, "qlat_off"))) return st;
        if ((st = bupload(b, b->d_qbot_off, b->qbot_off, "qbot_off"))) return st;
        B_ALLOC(b, b->d_n_active, std::max(NI, 1));
        B_ALLOC(b, b->src_pos, std::max(b->n_src, 1));
        for (int i = 0; i < NI; ++i)
            B_CUDA(b, d2d(b->src_pos.p + b->src_off[i], b->inst[i]->src_pos.p,
                          sizeof(double2) * b->inst[i]->n_src, s));
        const size_t m = std::max(b->n_src, 1);
        if (mixed) {
            B_ALLOC(b, b->s32T, m);
            B_ALLOC(b, b->s32F, m);
        } else {
            B_ALLOC(b, b->s64T, m);
            B_ALLOC(b, b->s64F, m);
        }
    }

    // ---- boundary weight matrices (rows and point columns remapped)
    {
        std::vector<int> rowdof, lptr(1, 0), lcol, bptr(1, 0), bcol;
        for (int i = 0; i < NI; ++i) {
            const sa_ctx* c = b->inst[i];
            for (size_t r = 0; r < c->wlat_rowdof_h.size(); ++r) {
                const int k = c->wlat_rowdof_h[r];
                rowdof.push_back(k < c->n_free ? b->free_off[i] + k : b->n_free + b->dir_off[i] + (k - c->n_free));
                for (int t = c->wlat_ptr_h[r]; t < c->wlat_ptr_h[r + 1]; ++t) lcol.push_back(c->wlat_col_h[t] + b->qlat_off[i]);
                lptr.push_back((int)lcol.size());
            }
            for (int r = 0; r < pad_to(c->n_dir, 32); ++r) {
                if (r < c->n_dir)
                    for (int t = c->wbot_ptr_h[r]; t < c->wbot_ptr_h[r + 1]; ++t) bcol.push_back(c->wbot_col_h[t] + b->qbot_off[i]);
                bptr.push_back((int)bcol.size());
            }
        }
        b->wlat_rows = (int)rowdof.size();
        sa_status st;
        if ((st = bupload(b, b->wlat_rowdof, rowdof, "wlat_rowdof"))) return st;
        if ((st = bupload(b, b->wlat_ptr, lptr, "wlat_ptr"))) return st;
        if ((st = bupload(b, b->wlat_col, lcol, "wlat_col"))) return st;
        if ((st = bupload(b, b->wbot_ptr, bptr, "wbot_ptr"))) return st;
        if ((st = bupload(b, b->wbot_col, bcol, "wbot_col"))) return st;
        B_ALLOC(b, b->wlat_val, std::max<size_t>(lcol.size(), 1));
        B_ALLOC(b, b->wbot_val, std::max<size_t>(bcol.size(), 1));
        size_t lo = 0, bo = 0;
        for (int i = 0; i < NI; ++i) {
            const sa_ctx* c = b->inst[i];
            const size_t nl = c->wlat_col_h.size(), nb = c->wbot_col_h.size();
            B_CUDA(b, d2d(b->wlat_val.p + lo, c->wlat_val.p, sizeof(double) * nl, s));
            B_CUDA(b, d2d(b->wbot_val.p + bo, c->wbot_val.p, sizeof(double) * nb, s));
            lo += nl;
            bo += nb;
        }
    }

    // ---- operators: A (free x free), R (free x all), M_bot (dir x dir)
    {
        bool a16 = true, m16 = true;
        for (int i = 0; i < NI; ++i) {
            a16 = a16 && !b->inst[i]->a_h.col16.empty();
            m16 = m16 && !b->inst[i]->mbot_h.col16.empty();
        }
        SellHost A, R, Mb;
        std::vector<int> slice_inst_a, slice_inst_b, so_a(1, 0), so_b(1, 0);
        for (int i = 0; i < NI; ++i) {
            const sa_ctx* c = b->inst[i];
            std::vector<int> rmap(c->n_dof);
            for (int k = 0; k < c->n_dof; ++k)
                rmap[k] = k < c->n_free ? b->free_off[i] + k : b->n_free + b->dir_off[i] + (k - c->n_free);
            append_sell(c->a_h, b->free_off[i], {}, A, a16);
            append_sell(c->r_h, b->free_off[i], rmap, R, false);
            append_sell(c->mbot_h, b->dir_off[i], {}, Mb, m16);
            for (int sl = 0; sl < c->a_h.n_slices; ++sl) slice_inst_a.push_back(i);
            for (int sl = 0; sl < c->mbot_h.n_slices; ++sl) slice_inst_b.push_back(i);
            so_a.push_back((int)slice_inst_a.size());
            so_b.push_back((int)slice_inst_b.size());
        }
        A.n = b->n_free;
        R.n = b->n_free;
        Mb.n = b->n_dir;
        if (A.n_slices * 32 != b->n_free || Mb.n_slices * 32 != b->n_dir)
            return bfail(b, SA_ERR_STATE, "internal: slice padding mismatch");
        auto up = [&](SellDev& d, SellHost& h, bool use16, const char* what) -> sa_status {
            d.n = h.n;
            d.n_slices = h.n_slices;
            d.n_stored = (long long)h.col.size();
            sa_status st;
            if ((st = bupload(b, d.sptr, h.sptr, what))) return st;
            if (use16) {
                if ((st = bupload(b, d.col16, h.col16, what))) return st;
            } else {
                if ((st = bupload(b, d.col, h.col, what))) return st;
            }
            if ((st = bupload(b, d.hi, sell_hi_flags(h), what))) return st;
            return SA_OK;
        };
        sa_status st;
        if ((st = up(b->a_s, A, a16, "A"))) return st;
        if ((st = up(b->r_s, R, false, "R"))) return st;
        if ((st = up(b->mbot_s, Mb, m16, "M_bot"))) return st;
        if ((st = bupload(b, b->slice_inst_a, slice_inst_a, "slice_inst_a"))) return st;
        if ((st = bupload(b, b->slice_inst_b, slice_inst_b, "slice_inst_b"))) return st;
        if ((st = bupload(b, b->d_slice_off_a, so_a, "slice_off_a"))) return st;
        if ((st = bupload(b, b->d_slice_off_b, so_b, "slice_off_b"))) return st;
        B_ALLOC(b, b->a_val, A.col.size());
        B_ALLOC(b, b->r_K, R.col.size());
        B_ALLOC(b, b->r_M, R.col.size());
        B_ALLOC(b, b->mbot_val, Mb.col.size());
        B_ALLOC(b, b->a_dinv, std::max(b->n_free, 1));
        B_ALLOC(b, b->mbot_dinv, std::max(b->n_dir, 1));
        B_CUDA(b, cudaMemsetAsync(b->a_dinv.p, 0, sizeof(double) * b->a_dinv.n, s));
        B_CUDA(b, cudaMemsetAsync(b->mbot_dinv.p, 0, sizeof(double) * b->mbot_dinv.n, s));
        long long ao = 0, ro = 0, mo = 0;
        for (int i = 0; i < NI; ++i) {
            const sa_ctx* c = b->inst[i];
            const size_t na = c->a_h.col.size(), nr = c->r_h.col.size(), nm = c->mbot_h.col.size();
            B_CUDA(b, d2d(b->a_val.p + ao, c->a_val.p, sizeof(double) * na, s));
            B_CUDA(b, d2d(b->r_K.p + ro, c->r_K.p, sizeof(double) * nr, s));
            B_CUDA(b, d2d(b->r_M.p + ro, c->r_M.p, sizeof(double) * nr, s));
            B_CUDA(b, d2d(b->mbot_val.p + mo, c->mbot_sval.p, sizeof(double) * nm, s));
            B_CUDA(b, d2d(b->a_dinv.p + b->free_off[i], c->a_dinv.p, sizeof(double) * c->n_free, s));
            B_CUDA(b, d2d(b->mbot_dinv.p + b->dir_off[i], c->mbot_dinv.p, sizeof(double) * c->n_dir, s));
            ao += na;
            ro += nr;
            mo += nm;
        }
        if (mixed) {
            B_ALLOC(b, b->a_val32, A.col.size());
            B_ALLOC(b, b->r_K32, R.col.size());
            B_ALLOC(b, b->r_M32, R.col.size());
            B_ALLOC(b, b->mbot_val32, Mb.col.size());
            cudaError_t e = launch_to_f32(b->a_s.n_stored, b->a_val.p, b->a_val32.p, s);
            if (e == cudaSuccess) e = launch_to_f32(b->r_s.n_stored, b->r_K.p, b->r_K32.p, s);
            if (e == cudaSuccess) e = launch_to_f32(b->r_s.n_stored, b->r_M.p, b->r_M32.p, s);
            if (e == cudaSuccess) e = launch_to_f32(b->mbot_s.n_stored, b->mbot_val.p, b->mbot_val32.p, s);
            if (e != cudaSuccess) return bcuda(b, e, "FP32 operators");
            const std::vector<unsigned char> hi = sell_hi_flags(R);
            std::vector<short> lo(R.col.size(), 0);
            bool fits = R.n > 0;
            for (int sl = 0; sl < R.n_slices && fits; ++sl) {
                if (hi[sl]) continue;
                const long long w = (R.sptr[sl + 1] - R.sptr[sl]) / 32;
                for (int l = 0; l < 32 && fits; ++l) {
                    const int r = std::min(sl * 32 + l, R.n - 1);
                    for (long long kk = 0; kk < w; ++kk) {
                        const long long ee = R.sptr[sl] + 32 * kk + l;
                        const long long d = sl * 32 + l < R.n ? (long long)R.col[ee] - r : 0;
                        if (d < -32768 || d > 32767) {
                            fits = false;
                            break;
                        }
                        lo[ee] = (short)d;
                    }
                }
            }
            if (fits) {
                sa_status st3;
                if ((st3 = bupload(b, b->r_col16lo, lo, "r_col16lo"))) return st3;
                B_ALLOC(b, b->r_M16, R.col.size());
                e = launch_to_bf16(b->r_s.n_stored, b->r_M.p, b->r_M16.p, s);
                if (e != cudaSuccess) return bcuda(b, e, "free-row M (bf16)");
            }
        }
    }

    // ---- state and work
    {
        const int nwork = std::max(std::max(b->n_free, b->n_dir), 1);
        B_ALLOC(b, b->That, std::max(b->n_dof, 1));
        B_ALLOC(b, b->F0, std::max(b->n_dof, 1));
        B_ALLOC(b, b->F1, std::max(b->n_dof, 1));
        B_ALLOC(b, b->gnew, std::max(b->n_dir, 1));
        B_ALLOC(b, b->bbot, std::max(b->n_dir, 1));
        B_ALLOC(b, b->r0, nwork);
        B_ALLOC(b, b->bsq, nwork);
        B_ALLOC(b, b->dirv, 2 * std::max(b->n_dir, 1));
        B_ALLOC(b, b->wr, nwork);
        B_ALLOC(b, b->wz, nwork);
        B_ALLOC(b, b->wp0, nwork);
        B_ALLOC(b, b->wp1, nwork);
        B_ALLOC(b, b->wq, nwork);
        B_ALLOC(b, b->dev64, std::max(b->n_dof, 1));
        B_ALLOC(b, b->dev32, std::max(b->n_dof, 1));
        B_ALLOC(b, b->wzl, nwork);
        B_ALLOC(b, b->wpl0, nwork);
        B_ALLOC(b, b->wpl1, nwork);
        const int smax = std::max(b->a_s.n_slices, b->mbot_s.n_slices);
        B_ALLOC(b, b->partials, (size_t)3 * std::max(smax, 1));
        // separable history sums when every instance's faces allow them
        if (b->opt.hist_mode != SA_HIST_PAIRWISE &&
            !sep_batch_plan(b->inst, b->qlat_off, b->qbot_off, b->opt.precision, b->sep) &&
            b->opt.hist_mode == SA_HIST_SEPARABLE)
            return bfail(b, SA_ERR_ARG, "separable history sums: an instance's faces are not rectangles");
        // fast diagonalization of the main solves: every instance has it, in
        // the batch's precision
        b->fd_on = b->opt.precond != SA_PRECOND_JACOBI;
        for (int i = 0; i < NI && b->fd_on; ++i)
            b->fd_on = b->inst[i]->fdm.ok && b->inst[i]->opt.precision == b->opt.precision;
        if (b->fd_on) {
            const size_t vt = mixed ? sizeof(float) : sizeof(double);
            std::vector<BFd> desc(NI);
            std::vector<int> loff(3 * (NI + 1), 0);
            for (int i = 0; i < NI; ++i) {
                const FdData& f = b->inst[i]->fdm;
                for (int d = 0; d < 3; ++d) {
                    b->fd_mmax = std::max(b->fd_mmax, f.m[d]);
                    desc[i].m[d] = f.m[d];
                    desc[i].U[d] = f.dU[d].p;
                    desc[i].Ut[d] = f.dUt[d].p;
                    desc[i].lamc[d] = f.dlamc[d].p;
                    loff[d * (NI + 1) + i + 1] = loff[d * (NI + 1) + i] + b->inst[i]->n_free / f.m[d];
                }
                desc[i].row0 = b->free_off[i];
                desc[i].cM = f.cM;
            }
            std::vector<unsigned char> raw(sizeof(BFd) * NI);
            std::memcpy(raw.data(), desc.data(), raw.size());
            sa_status st2;
            if ((st2 = bupload(b, b->fd_desc, raw, "fd_desc"))) return st2;
            if ((st2 = bupload(b, b->fd_loff, loff, "fd_loff"))) return st2;
            B_ALLOC(b, b->fdS, nwork * vt);
            B_ALLOC(b, b->fdZ, nwork * vt);
            B_CUDA(b, cudaMemsetAsync(b->fdS.p, 0, nwork * vt, s));
            for (int i = 0; i < NI; ++i)
                B_CUDA(b, d2d(b->fdS.p + (size_t)b->free_off[i] * vt, b->inst[i]->fdm.S.p,
                              (size_t)b->inst[i]->n_free * vt, s));
        }
        // the bottom projections' 2-D fast diagonalization, when every
        // instance has one
        b->fdb_on = b->opt.precond != SA_PRECOND_JACOBI && b->n_dir > 0;
        for (int i = 0; i < NI && b->fdb_on; ++i)
            b->fdb_on = b->inst[i]->fdb.ok && b->inst[i]->fdb.nd == 2 &&
                        b->inst[i]->opt.precision == b->opt.precision;
        if (b->fdb_on) {
            const size_t vt = mixed ? sizeof(float) : sizeof(double);
            std::vector<BFd> desc(NI);
            std::vector<int> loff(3 * (NI + 1), 0);
            for (int i = 0; i < NI; ++i) {
                const FdData& f = b->inst[i]->fdb;
                std::memset(&desc[i], 0, sizeof(BFd));
                for (int d = 0; d < 3; ++d) desc[i].m[d] = f.m[d];
                for (int d = 0; d < 2; ++d) {
                    b->fd_mmax = std::max(b->fd_mmax, f.m[d]);
                    desc[i].U[d] = f.dU[d].p;
                    desc[i].Ut[d] = f.dUt[d].p;
                    desc[i].lamc[d] = f.dlamc[d].p;
                    loff[d * (NI + 1) + i + 1] = loff[d * (NI + 1) + i] + b->inst[i]->n_dir / f.m[d];
                }
                desc[i].row0 = b->dir_off[i];
                desc[i].cM = f.cM;
            }
            std::vector<unsigned char> raw(sizeof(BFd) * NI);
            std::memcpy(raw.data(), desc.data(), raw.size());
            sa_status st2;
            if ((st2 = bupload(b, b->fdb_desc, raw, "fdb_desc"))) return st2;
            if ((st2 = bupload(b, b->fdb_loff, loff, "fdb_loff"))) return st2;
            const size_t ndw = (size_t)std::max(b->n_dir, 1);
            B_ALLOC(b, b->fdbS, ndw * vt);
            B_ALLOC(b, b->fdbZ, ndw * vt);
            B_CUDA(b, cudaMemsetAsync(b->fdbS.p, 0, ndw * vt, s));
            for (int i = 0; i < NI; ++i)
                B_CUDA(b, d2d(b->fdbS.p + (size_t)b->dir_off[i] * vt, b->inst[i]->fdb.S.p,
                              (size_t)b->inst[i]->n_dir * vt, s));
        }
        B_ALLOC(b, b->inst_state, (size_t)IS_NFIELDS * std::max(NI, 1));
        B_ALLOC(b, b->inst_iters, (size_t)2 * std::max(NI, 1));
        B_ALLOC(b, b->counters, 2);
        B_ALLOC(b, b->st, 1);
        B_CUDA(b, cudaMemsetAsync(b->st.p, 0, sizeof(DevStatus), s));
        B_CUDA(b, cudaMemsetAsync(b->inst_iters.p, 0, sizeof(int) * b->inst_iters.n, s));
        B_CUDA(b, cudaMemsetAsync(b->F0.p, 0, sizeof(double) * b->F0.n, s));
        B_CUDA(b, cudaMemsetAsync(b->F1.p, 0, sizeof(double) * b->F1.n, s));
        B_CUDA(b, cudaMemsetAsync(b->wp0.p, 0, sizeof(double) * nwork, s));
        B_CUDA(b, cudaMemsetAsync(b->wp1.p, 0, sizeof(double) * nwork, s));
        B_CUDA(b, cudaMemsetAsync(b->wpl0.p, 0, sizeof(float) * nwork, s));
        B_CUDA(b, cudaMemsetAsync(b->wpl1.p, 0, sizeof(float) * nwork, s));
        // padding rows hold T_c (dev = 0)
        std::vector<double> tc(b->n_dof, b->Tc);
        B_CUDA(b, cudaMemcpy(b->That.p, tc.data(), sizeof(double) * b->n_dof, cudaMemcpyHostToDevice));
        for (int i = 0; i < NI; ++i) {
            const sa_ctx* c = b->inst[i];
            B_CUDA(b, d2d(b->That.p + b->free_off[i], c->That.p, sizeof(double) * c->n_free, s));
            B_CUDA(b, d2d(b->That.p + b->n_free + b->dir_off[i], c->That.p + c->n_free, sizeof(double) * c->n_dir, s));
            B_CUDA(b, d2d(b->F0.p + b->free_off[i], c->F0.p, sizeof(double) * c->n_free, s));
            B_CUDA(b, d2d(b->F0.p + b->n_free + b->dir_off[i], c->F0.p + c->n_free, sizeof(double) * c->n_dir, s));
        }
        long long n0 = b->inst[0]->n_step;
        B_CUDA(b, cudaMemcpyAsync(&b->st.p->n, &n0, sizeof(long long), cudaMemcpyHostToDevice, s));
        b->n_step = n0;
        int occ = 0;
        const size_t pcg_smem = (b->fd_on || b->fdb_on)
                                    ? (mixed ? batch_pcg_smem<float>(batch_pcg_stage_m<float>(b->fd_mmax))
                                             : batch_pcg_smem<double>(batch_pcg_stage_m<double>(b->fd_mmax)))
                                    : 0;
        const void* pcg_fn = mixed ? (const void*)k_pcg_batch<float> : (const void*)k_pcg_batch<double>;
        B_CUDA(b, cudaFuncSetAttribute(pcg_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pcg_smem));
        B_CUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pcg_fn, 1024, pcg_smem));
        if (occ < 1) return bfail(b, SA_ERR_CUDA, "batched PCG kernel cannot be resident");
        b->pcg_grid = b->num_sms;
    }
    B_CUDA(b, cudaStreamSynchronize(s));
    b->dt = dt;
    b->theta = theta;
    b->built = true;
    return SA_OK;
}

sa_status enqueue_batch_step(sa_batch* b) {
    cudaStream_t s = b->stream;
    const bool mixed = b->opt.precision == SA_MIXED;
    const double alpha = b->k / (b->rho * b->cp);
    cudaError_t e = launch_prologue_batch(b->st.p, b->n_src, b->n_inst, b->d_src_inst.p, b->d_src_off.p,
                                          b->d_n_src.p, b->d_coefE.p, b->d_r2_8a.p, b->d_n_active.p,
                                          b->src_pos.p, b->dt, alpha, b->opt.precision, b->s64T.p,
                                          b->s64F.p, b->s32T.p, b->s32F.p, s);
    if (e != cudaSuccess) return bcuda(b, e, "batched prologue");
    if (b->sep.ok)
        e = launch_sep_batch(b->sep, b->opt.precision, b->st.p, b->d_n_active.p, b->d_src_off.p,
                             b->s32F.p, b->s32T.p, b->s64F.p, b->s64T.p, b->s_lat.p, b->tt_bot.p, s);
    else
        e = launch_history_batch(b->opt.precision, b->hist_P, b->hist_W, b->st.p, b->q_lat,
                                 b->q_bot, b->lat32.p, b->bot32.p, b->lat64.p, b->bot64.p,
                                 b->s32F.p, b->s32T.p, b->s64F.p, b->s64T.p, b->s_lat.p,
                                 b->tt_bot.p, b->n_inst, b->d_qlat_off.p, b->d_qbot_off.p,
                                 b->d_src_off.p, b->d_n_active.p, s);
    if (e != cudaSuccess) return bcuda(b, e, "batched history");
    e = launch_gather(b->wlat_rows, b->wlat_rowdof.p, b->wlat_ptr.p, b->wlat_col.p, b->wlat_val.p,
                      b->s_lat.p, b->k, b->n_dir, b->wbot_ptr.p, b->wbot_col.p, b->wbot_val.p,
                      b->tt_bot.p, b->Tc, b->F1.p, b->bbot.p, b->n_dof, b->That.p, b->dev64.p,
                      b->dev32.p, s);
    if (e != cudaSuccess) return bcuda(b, e, "batched gather");
    if (b->n_dir > 0) {
        e = cudaMemcpyAsync(b->gnew.p, b->That.p + b->n_free, sizeof(double) * b->n_dir,
                            cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) {
            if (mixed)
                e = launch_pcg_batch<float>(b, 1, b->mbot_s, b->mbot_val32.p, b->mbot_val.p,
                                            b->slice_inst_b.p, b->d_slice_off_b.p, b->mbot_dinv.p,
                                            b->bbot.p, nullptr, b->gnew.p, s);
            else
                e = launch_pcg_batch<double>(b, 1, b->mbot_s, b->mbot_val.p, b->mbot_val.p,
                                             b->slice_inst_b.p, b->d_slice_off_b.p, b->mbot_dinv.p,
                                             b->bbot.p, nullptr, b->gnew.p, s);
        }
        if (e != cudaSuccess) return bcuda(b, e, "batched bottom PCG");
    }
    e = launch_theta_rhs(b->opt.precision, sell_view(b->r_s),
                         mixed ? (const void*)b->r_K32.p : (const void*)b->r_K.p,
                         mixed ? (const void*)b->r_M32.p : (const void*)b->r_M.p,
                         mixed ? (const void*)b->dev32.p : (const void*)b->dev64.p, b->That.p,
                         b->gnew.p, b->F0.p, b->F1.p, b->rho * b->cp / b->dt, b->k, b->theta,
                         b->Tc, b->r0.p, b->bsq.p, b->n_dir, b->dirv.p, s, 0, false, nullptr, nullptr,
                         nullptr, mixed ? b->r_col16lo.p : nullptr, mixed ? b->r_M16.p : nullptr);
    if (e != cudaSuccess) return bcuda(b, e, "batched rhs");
    if (mixed)
        e = launch_pcg_batch<float>(b, 0, b->a_s, b->a_val32.p, b->a_val.p, b->slice_inst_a.p,
                                    b->d_slice_off_a.p, b->a_dinv.p, nullptr, b->r0.p, b->That.p, s);
    else
        e = launch_pcg_batch<double>(b, 0, b->a_s, b->a_val.p, b->a_val.p, b->slice_inst_a.p,
                                     b->d_slice_off_a.p, b->a_dinv.p, nullptr, b->r0.p, b->That.p, s);
    if (e != cudaSuccess) return bcuda(b, e, "batched PCG");
    e = launch_finalize(b->n_dir, b->n_free, b->n_dof, b->gnew.p, b->That.p, b->F1.p, b->F0.p, b->st.p, s);
    if (e != cudaSuccess) return bcuda(b, e, "batched finalize");
    return SA_OK;
}

}  // namespace

extern "C" {

sa_status sa_batch_create(sa_ctx* const* insts, int n_inst, const sa_options* o, sa_batch** out) {
    if (!out || !insts || n_inst <= 0) return SA_ERR_ARG;
    *out = nullptr;
    sa_batch* b = new sa_batch();
    if (o)
        b->opt = *o;
    else
        sa_options_default(&b->opt);
    if ((b->opt.precision != SA_FP64 && b->opt.precision != SA_MIXED) ||
        b->opt.hist_mode < SA_HIST_AUTO || b->opt.hist_mode > SA_HIST_SEPARABLE) {
        delete b;
        return SA_ERR_ARG;
    }
    b->stream = (cudaStream_t)b->opt.cuda_stream;
    b->hist_P = b->opt.hist_points_per_lane ? b->opt.hist_points_per_lane : 4;
    b->hist_W = b->opt.hist_warps ? b->opt.hist_warps : 8;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete b;
        return SA_ERR_CUDA;
    }
    for (int i = 0; i < n_inst; ++i) {
        sa_ctx* c = insts[i];
        if (!c || !c->has_patch || !c->has_material || !c->has_scan || c->poisoned) {
            delete b;
            return SA_ERR_STATE;
        }
        if (i == 0) {
            b->k = c->k;
            b->rho = c->rho;
            b->cp = c->cp;
            b->Tc = c->Tc;
        } else if (c->k != b->k || c->rho != b->rho || c->cp != b->cp || c->Tc != b->Tc) {
            delete b;
            return SA_ERR_ARG;   // one material per batch
        }
        b->inst.push_back(c);
    }
    b->n_inst = n_inst;
    *out = b;
    return SA_OK;
}

void sa_batch_destroy(sa_batch* b) {
    if (!b) return;
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    delete b;
}

const char* sa_batch_last_error(const sa_batch* b) { return b ? b->err.c_str() : "null batch"; }

sa_status sa_batch_step(sa_batch* b, double theta, double dt, int n_steps, sa_step_stats* stats) {
    if (!b) return SA_ERR_ARG;
    if (b->poisoned) return bfail(b, SA_ERR_STATE, "batch poisoned: %s", b->err.c_str());
    if (!(theta >= 0.0 && theta <= 1.0) || !(dt > 0.0) || n_steps < 0)
        return bfail(b, SA_ERR_ARG, "theta %g, dt %g, n_steps %d", theta, dt, n_steps);
    if (!b->built) {
        sa_status st = build(b, theta, dt);
        if (st) return st;
    } else if (theta != b->theta || dt != b->dt) {
        return bfail(b, SA_ERR_ARG, "a batch keeps the (theta, dt) of its first step");
    }
    cudaStream_t s = b->stream;
    const bool graph = b->opt.use_graph && s != nullptr;
    for (int i = 0; i < n_steps; ++i) {
        if (graph) {
            if (!b->graph_exec) {
                cudaGraph_t g;
                B_CUDA(b, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
                sa_status es = enqueue_batch_step(b);
                cudaError_t ee = cudaStreamEndCapture(s, &g);
                if (es) return es;
                if (ee != cudaSuccess) return bcuda(b, ee, "end capture");
                ee = cudaGraphInstantiate(&b->graph_exec, g, 0);
                cudaGraphDestroy(g);
                if (ee != cudaSuccess) return bcuda(b, ee, "graph instantiate");
            }
            B_CUDA(b, cudaGraphLaunch(b->graph_exec, s));
        } else {
            sa_status st = enqueue_batch_step(b);
            if (st) return st;
        }
    }
    b->n_step += n_steps;
    if (stats) {
        DevStatus h;
        B_CUDA(b, cudaMemcpyAsync(&h, b->st.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
        B_CUDA(b, cudaStreamSynchronize(s));
        std::memset(stats, 0, sizeof(*stats));
        stats->steps_done = n_steps;
        stats->pcg_iters_last = h.pcg_iters;
        stats->pcg_iters_total = (int)h.iters_total;
        stats->pcg_iters_max = h.iters_max;
        stats->bot_iters_total = (int)h.bot_total;
        stats->hist_pairs_skipped = h.hist_skipped;
        stats->step_index = h.n;
        DevStatus z;
        std::memset(&z, 0, sizeof(z));
        B_CUDA(b, cudaMemcpyAsync(&b->st.p->err, &z.err, offsetof(DevStatus, n), cudaMemcpyHostToDevice, s));
        B_CUDA(b, cudaMemcpyAsync(&b->st.p->iters_total, &z.iters_total,
                                  offsetof(DevStatus, pad) - offsetof(DevStatus, iters_total),
                                  cudaMemcpyHostToDevice, s));
        B_CUDA(b, cudaStreamSynchronize(s));
        if (h.err & SA_DEV_TIMEOUT) return bfail(b, SA_ERR_TIMEOUT, "a device-side wait timed out");
        if (h.err & SA_DEV_NAN) return bfail(b, SA_ERR_NAN, "non-finite value in a solve");
        if (h.err & (SA_DEV_NOT_CONVERGED | SA_DEV_BOT_NOT_CONVERGED))
            return bfail(b, SA_ERR_NOT_CONVERGED, "PCG did not converge for some instance");
    }
    return SA_OK;
}

sa_status sa_batch_get_field(sa_batch* b, int inst, int field, double* out, long long count) {
    if (!b || !out || inst < 0 || inst >= b->n_inst) return SA_ERR_ARG;
    if (!b->built) return bfail(b, SA_ERR_STATE, "batch has not stepped");
    sa_ctx* c = b->inst[inst];
    cudaStream_t s = b->stream;
    if (field == SA_FIELD_THAT || field == SA_FIELD_F) {
        if (count < c->n_dof) return bfail(b, SA_ERR_ARG, "count");
        const double* src = field == SA_FIELD_THAT ? b->That.p : b->F0.p;
        std::vector<double> in(c->n_dof);
        B_CUDA(b, cudaMemcpyAsync(in.data(), src + b->free_off[inst], sizeof(double) * c->n_free,
                                  cudaMemcpyDeviceToHost, s));
        B_CUDA(b, cudaMemcpyAsync(in.data() + c->n_free, src + b->n_free + b->dir_off[inst],
                                  sizeof(double) * c->n_dir, cudaMemcpyDeviceToHost, s));
        B_CUDA(b, cudaStreamSynchronize(s));
        for (int k = 0; k < c->n_dof; ++k) out[k] = in[c->perm[k]];
        return SA_OK;
    }
    if (field == SA_FIELD_DTDN_LAT || field == SA_FIELD_TT_BOT) {
        const bool lat = field == SA_FIELD_DTDN_LAT;
        const int Q = lat ? c->q_lat : c->q_bot;
        if (count < Q) return bfail(b, SA_ERR_ARG, "count");
        B_CUDA(b, cudaMemcpyAsync(out, (lat ? b->s_lat.p + b->qlat_off[inst] : b->tt_bot.p + b->qbot_off[inst]),
                                  sizeof(double) * Q, cudaMemcpyDeviceToHost, s));
        B_CUDA(b, cudaStreamSynchronize(s));
        return SA_OK;
    }
    return bfail(b, SA_ERR_ARG, "field %d not available from a batch", field);
}

sa_status sa_batch_get_iters(sa_batch* b, int* main_iters, int* bottom_iters) {
    if (!b || !main_iters || !bottom_iters) return SA_ERR_ARG;
    if (!b->built) return bfail(b, SA_ERR_STATE, "batch has not stepped");
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    B_CUDA(b, cudaMemcpy(main_iters, b->inst_iters.p, sizeof(int) * b->n_inst, cudaMemcpyDeviceToHost));
    B_CUDA(b, cudaMemcpy(bottom_iters, b->inst_iters.p + b->n_inst, sizeof(int) * b->n_inst,
                         cudaMemcpyDeviceToHost));
    return SA_OK;
}

// Tile autotuner for the batched history sum: times every (points per lane,
// warps) shape on the batch's own data at its current step (CUDA events on
// the batch stream, median of 5), keeps the fastest, and records the choice in
// a small JSON file keyed by the batch's sizes so later runs skip the timing.
sa_status sa_batch_autotune(sa_batch* b, const char* cache_path, int* P_out, int* NW_out,
                            double* best_ms_out) {
    if (!b || !P_out || !NW_out) return SA_ERR_ARG;
    if (!b->built) return bfail(b, SA_ERR_STATE, "step the batch once before tuning");
    char key[160];
    snprintf(key, sizeof(key), "hist:%d:%d:%d:%d:%d", b->n_inst, b->q_lat, b->q_bot, b->n_src,
             b->opt.precision);
    if (cache_path) {
        std::ifstream f(cache_path);
        std::string line;
        while (std::getline(f, line)) {
            const size_t k = line.find(key);
            if (k == std::string::npos) continue;
            int P = 0, W = 0;
            const size_t pp = line.find("\"P\":", k), ww = line.find("\"NW\":", k);
            if (pp != std::string::npos && ww != std::string::npos) {
                P = atoi(line.c_str() + pp + 4);
                W = atoi(line.c_str() + ww + 5);
            }
            if ((P == 1 || P == 2 || P == 4) && (W == 4 || W == 8)) {
                b->hist_P = P;
                b->hist_W = W;
                if (b->graph_exec) {
                    cudaGraphExecDestroy(b->graph_exec);
                    b->graph_exec = nullptr;
                }
                *P_out = P;
                *NW_out = W;
                if (best_ms_out) *best_ms_out = -1.0;
                return SA_OK;
            }
        }
    }
    cudaStream_t s = b->stream;
    const double alpha = b->k / (b->rho * b->cp);
    cudaError_t e = launch_prologue_batch(b->st.p, b->n_src, b->n_inst, b->d_src_inst.p, b->d_src_off.p,
                                          b->d_n_src.p, b->d_coefE.p, b->d_r2_8a.p, b->d_n_active.p,
                                          b->src_pos.p, b->dt, alpha, b->opt.precision, b->s64T.p,
                                          b->s64F.p, b->s32T.p, b->s32F.p, s);
    if (e != cudaSuccess) return bcuda(b, e, "autotune prologue");
    const int shapes[5][2] = {{1, 4}, {2, 4}, {2, 8}, {4, 4}, {4, 8}};
    cudaEvent_t e0, e1;
    B_CUDA(b, cudaEventCreate(&e0));
    B_CUDA(b, cudaEventCreate(&e1));
    double best = 1e300;
    int bp = b->hist_P, bw = b->hist_W;
    for (auto& sh : shapes) {
        std::vector<float> t;
        for (int rep = 0; rep < 6; ++rep) {
            B_CUDA(b, cudaEventRecord(e0, s));
            e = launch_history_batch(b->opt.precision, sh[0], sh[1], b->st.p, b->q_lat, b->q_bot,
                                     b->lat32.p, b->bot32.p, b->lat64.p, b->bot64.p, b->s32F.p,
                                     b->s32T.p, b->s64F.p, b->s64T.p, b->s_lat.p, b->tt_bot.p,
                                     b->n_inst, b->d_qlat_off.p, b->d_qbot_off.p, b->d_src_off.p,
                                     b->d_n_active.p, s);
            if (e != cudaSuccess) return bcuda(b, e, "autotune history");
            B_CUDA(b, cudaEventRecord(e1, s));
            B_CUDA(b, cudaEventSynchronize(e1));
            float ms = 0.f;
            B_CUDA(b, cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) t.push_back(ms);
        }
        std::sort(t.begin(), t.end());
        const double med = t[t.size() / 2];
        if (med < best) {
            best = med;
            bp = sh[0];
            bw = sh[1];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->hist_P = bp;
    b->hist_W = bw;
    if (b->graph_exec) {
        cudaGraphExecDestroy(b->graph_exec);
        b->graph_exec = nullptr;
    }
    if (cache_path) {
        std::ofstream f(cache_path, std::ios::app);
        f << "{\"key\": \"" << key << "\", \"P\": " << bp << ", \"NW\": " << bw << ", \"ms\": " << best
          << "}\n";
    }
    *P_out = bp;
    *NW_out = bw;
    if (best_ms_out) *best_ms_out = best;
    return SA_OK;
}


// Tuner of the launch shapes the batch runs with: the history sums (the
// separable product's tile widths per face kind and units per tile, or the
// pairwise tile when the faces are not rectangles) and the number of blocks
// of the batched solves.  History shapes are timed alone on the batch's data
// at its current step (their outputs are recomputed by every step); solve
// grids are timed over whole steps, with the batch's state (T^, F, step
// index) saved before and restored after, so tuning does not advance the
// simulation.  The choice is appended to the JSON-lines file cache_path
// (NULL: no cache) under a key of the batch's sizes and reused from there.
}  // extern "C"

namespace {

bool cache_lookup(const char* path, const char* key, sa_batch_shapes* sh) {
    if (!path) return false;
    std::ifstream f(path);
    std::string line;
    auto num = [&](const std::string& ln, const char* name, size_t from) -> int {
        const size_t k = ln.find(name, from);
        return k == std::string::npos ? -1 : atoi(ln.c_str() + k + strlen(name));
    };
    while (std::getline(f, line)) {
        const size_t k = line.find(std::string("\"") + key + "\"");
        if (k == std::string::npos) continue;
        sa_batch_shapes t{};
        t.hist_separable = num(line, "\"sep\": ", k);
        t.tj_lat = num(line, "\"tj_lat\": ", k);
        t.tj_bot = num(line, "\"tj_bot\": ", k);
        t.units_per_tile = num(line, "\"units\": ", k);
        t.hist_P = num(line, "\"P\": ", k);
        t.hist_NW = num(line, "\"NW\": ", k);
        t.pcg_grid = num(line, "\"grid\": ", k);
        const bool tj_ok = (t.tj_lat == 64 || t.tj_lat == 48 || t.tj_lat == 32) &&
                           (t.tj_bot == 64 || t.tj_bot == 48 || t.tj_bot == 32);
        const bool ok = t.pcg_grid >= 1 && (t.hist_P == 1 || t.hist_P == 2 || t.hist_P == 4) &&
                        (t.hist_NW == 4 || t.hist_NW == 8) &&
                        (t.hist_separable == 0 ||
                         (t.hist_separable == 1 && tj_ok && t.units_per_tile >= 1 && t.units_per_tile <= 8));
        if (!ok) continue;
        *sh = t;
        sh->step_ms = -1.0;
        return true;
    }
    return false;
}

void fill_shapes(const sa_batch* b, sa_batch_shapes* out, double ms) {
    out->hist_separable = b->sep.ok ? 1 : 0;
    out->tj_lat = b->sep.tj[0];
    out->tj_bot = b->sep.tj[1];
    out->units_per_tile = b->sep.ok ? b->sep.s_max : 0;
    out->hist_P = b->hist_P;
    out->hist_NW = b->hist_W;
    out->pcg_grid = b->pcg_grid;
    out->step_ms = ms;
}

}  // namespace

extern "C" {

sa_status sa_batch_get_shapes(sa_batch* b, sa_batch_shapes* out) {
    if (!b || !out) return SA_ERR_ARG;
    if (!b->built) return bfail(b, SA_ERR_STATE, "batch has not stepped");
    fill_shapes(b, out, 0.0);
    return SA_OK;
}

sa_status sa_batch_tune(sa_batch* b, const char* cache_path, long long at_step,
                        sa_batch_shapes* out) {
    if (!b || !out || at_step < 0) return SA_ERR_ARG;
    if (b->poisoned) return bfail(b, SA_ERR_STATE, "batch poisoned: %s", b->err.c_str());
    if (!b->built) return bfail(b, SA_ERR_STATE, "step the batch once before tuning");
    char key[200];
    const long long n_hist = at_step > 0 ? at_step : b->n_step + 1;
    snprintf(key, sizeof(key), "batch:%d:%d:%d:%d:%d:%d:%d:%lld", b->n_inst, b->q_lat, b->q_bot,
             b->n_src, b->n_dof, b->opt.precision, b->num_sms, n_hist);
    cudaStream_t s = b->stream;
    auto drop_graph = [&]() {
        if (b->graph_exec) {
            cudaGraphExecDestroy(b->graph_exec);
            b->graph_exec = nullptr;
        }
    };
    sa_batch_shapes c{};
    if (cache_lookup(cache_path, key, &c) && (c.hist_separable == 1) == b->sep.ok) {
        if (b->sep.ok && (c.tj_lat != b->sep.tj[0] || c.tj_bot != b->sep.tj[1] ||
                          c.units_per_tile != b->sep.s_max) &&
            !sep_batch_plan(b->inst, b->qlat_off, b->qbot_off, b->opt.precision, b->sep, c.tj_lat,
                            c.tj_bot, c.units_per_tile))
            return bfail(b, SA_ERR_OOM, "separable plan of the cached shapes");
        b->hist_P = c.hist_P;
        b->hist_W = c.hist_NW;
        b->pcg_grid = std::min(c.pcg_grid, b->num_sms);
        drop_graph();
        fill_shapes(b, out, -1.0);
        return SA_OK;
    }
    // the history shapes are timed with the sources active at step n_hist
    // (the prologue reads the step index from the status block, restored
    // below)
    const double alpha = b->k / (b->rho * b->cp);
    DevStatus st_keep;
    B_CUDA(b, cudaMemcpyAsync(&st_keep, b->st.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    B_CUDA(b, cudaStreamSynchronize(s));
    const long long n_pro = n_hist - 1;
    B_CUDA(b, cudaMemcpyAsync(&b->st.p->n, &n_pro, sizeof(long long), cudaMemcpyHostToDevice, s));
    cudaError_t e = launch_prologue_batch(b->st.p, b->n_src, b->n_inst, b->d_src_inst.p, b->d_src_off.p,
                                          b->d_n_src.p, b->d_coefE.p, b->d_r2_8a.p, b->d_n_active.p,
                                          b->src_pos.p, b->dt, alpha, b->opt.precision, b->s64T.p,
                                          b->s64F.p, b->s32T.p, b->s32F.p, s);
    if (e != cudaSuccess) return bcuda(b, e, "tuner prologue");
    cudaEvent_t e0, e1;
    B_CUDA(b, cudaEventCreate(&e0));
    B_CUDA(b, cudaEventCreate(&e1));
    // median of five timed repetitions (after one untimed) of enqueue()
    auto time_it = [&](auto enqueue, double* ms) -> sa_status {
        std::vector<float> t;
        for (int rep = 0; rep < 6; ++rep) {
            B_CUDA(b, cudaEventRecord(e0, s));
            cudaError_t ee = enqueue();
            if (ee != cudaSuccess) return bcuda(b, ee, "tuner launch");
            B_CUDA(b, cudaEventRecord(e1, s));
            B_CUDA(b, cudaEventSynchronize(e1));
            float v = 0.f;
            B_CUDA(b, cudaEventElapsedTime(&v, e0, e1));
            if (rep > 0) t.push_back(v);
        }
        std::sort(t.begin(), t.end());
        *ms = t[t.size() / 2];
        return SA_OK;
    };
    sa_status st = SA_OK;
    // ---- history shapes
    if (b->sep.ok) {
        double best = 1e300;
        int bl = b->sep.tj[0], bb = b->sep.tj[1], bu = b->sep.s_max;
        for (int units : {1, 2, 4})
            for (int tl : {64, 48, 32})
                for (int tb : {64, 48, 32}) {
                    if (st) break;
                    if (!sep_batch_plan(b->inst, b->qlat_off, b->qbot_off, b->opt.precision, b->sep, tl,
                                        tb, units)) {
                        st = bfail(b, SA_ERR_OOM, "separable plan (%d, %d, %d)", tl, tb, units);
                        break;
                    }
                    double ms = 0.0;
                    st = time_it([&]() {
                        return launch_sep_batch(b->sep, b->opt.precision, b->st.p, b->d_n_active.p,
                                                b->d_src_off.p, b->s32F.p, b->s32T.p, b->s64F.p,
                                                b->s64T.p, b->s_lat.p, b->tt_bot.p, s);
                    }, &ms);
                    if (st) break;
                    if (ms < best) {
                        best = ms;
                        bl = tl;
                        bb = tb;
                        bu = units;
                    }
                    if (st) break;
                }
        if (!st && !sep_batch_plan(b->inst, b->qlat_off, b->qbot_off, b->opt.precision, b->sep, bl, bb, bu))
            st = bfail(b, SA_ERR_OOM, "separable plan of the tuned shapes");
    } else {
        const int shapes[5][2] = {{1, 4}, {2, 4}, {2, 8}, {4, 4}, {4, 8}};
        double best = 1e300;
        int bp = b->hist_P, bw = b->hist_W;
        for (auto& sh : shapes) {
            double ms = 0.0;
            st = time_it([&]() {
                return launch_history_batch(b->opt.precision, sh[0], sh[1], b->st.p, b->q_lat, b->q_bot,
                                            b->lat32.p, b->bot32.p, b->lat64.p, b->bot64.p, b->s32F.p,
                                            b->s32T.p, b->s64F.p, b->s64T.p, b->s_lat.p, b->tt_bot.p,
                                            b->n_inst, b->d_qlat_off.p, b->d_qbot_off.p,
                                            b->d_src_off.p, b->d_n_active.p, s);
            }, &ms);
            if (st) break;
            if (ms < best) {
                best = ms;
                bp = sh[0];
                bw = sh[1];
            }
        }
        b->hist_P = bp;
        b->hist_W = bw;
    }
    B_CUDA(b, cudaMemcpyAsync(b->st.p, &st_keep, sizeof(DevStatus), cudaMemcpyHostToDevice, s));
    B_CUDA(b, cudaStreamSynchronize(s));
    drop_graph();
    // ---- grid of the batched solves, over whole steps from a saved state
    double best_step = 1e300;
    if (!st) {
        DBuf<double> T_save, F_save;
        DevStatus st_save;
        const long long n_save = b->n_step;
        if (T_save.alloc(b->That.n) != cudaSuccess || F_save.alloc(b->F0.n) != cudaSuccess) {
            cudaGetLastError();
            st = bfail(b, SA_ERR_OOM, "tuner state copy");
        }
        if (!st) {
            B_CUDA(b, cudaMemcpyAsync(T_save.p, b->That.p, sizeof(double) * b->That.n, cudaMemcpyDeviceToDevice, s));
            B_CUDA(b, cudaMemcpyAsync(F_save.p, b->F0.p, sizeof(double) * b->F0.n, cudaMemcpyDeviceToDevice, s));
            B_CUDA(b, cudaMemcpyAsync(&st_save, b->st.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
            B_CUDA(b, cudaStreamSynchronize(s));
        }
        auto restore = [&]() -> sa_status {
            B_CUDA(b, cudaMemcpyAsync(b->That.p, T_save.p, sizeof(double) * b->That.n, cudaMemcpyDeviceToDevice, s));
            B_CUDA(b, cudaMemcpyAsync(b->F0.p, F_save.p, sizeof(double) * b->F0.n, cudaMemcpyDeviceToDevice, s));
            B_CUDA(b, cudaMemcpyAsync(b->st.p, &st_save, sizeof(DevStatus), cudaMemcpyHostToDevice, s));
            B_CUDA(b, cudaStreamSynchronize(s));
            b->n_step = n_save;
            return SA_OK;
        };
        int best_grid = b->pcg_grid;
        const int G = b->num_sms;
        int grids[3] = {G, std::max(1, (3 * G) / 4), std::max(1, G / 2)};
        for (int gi = 0; gi < 3 && !st; ++gi) {
            if (gi > 0 && grids[gi] == grids[gi - 1]) continue;
            b->pcg_grid = grids[gi];
            drop_graph();
            st = sa_batch_step(b, b->theta, b->dt, 1, nullptr);        // capture, warm
            if (!st) {
                B_CUDA(b, cudaEventRecord(e0, s));
                st = sa_batch_step(b, b->theta, b->dt, 3, nullptr);
                B_CUDA(b, cudaEventRecord(e1, s));
                B_CUDA(b, cudaEventSynchronize(e1));
            }
            if (!st) {
                float v = 0.f;
                B_CUDA(b, cudaEventElapsedTime(&v, e0, e1));
                DevStatus h;
                B_CUDA(b, cudaMemcpy(&h, b->st.p, sizeof(DevStatus), cudaMemcpyDeviceToHost));
                // a shape whose solves gave up (device wait limit) is not chosen
                if (!(h.err & SA_DEV_TIMEOUT) && v / 3.0 < best_step) {
                    best_step = v / 3.0;
                    best_grid = grids[gi];
                }
            }
            if (!st) st = restore();
        }
        b->pcg_grid = best_grid;
        drop_graph();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    fill_shapes(b, out, best_step);
    if (cache_path) {
        std::ofstream f(cache_path, std::ios::app);
        f << "{\"key\": \"" << key << "\", \"sep\": " << out->hist_separable << ", \"tj_lat\": "
          << out->tj_lat << ", \"tj_bot\": " << out->tj_bot << ", \"units\": " << out->units_per_tile
          << ", \"P\": " << out->hist_P << ", \"NW\": " << out->hist_NW << ", \"grid\": "
          << out->pcg_grid << ", \"step_ms\": " << best_step << "}\n";
    }
    return SA_OK;
}

}  // extern "C"
