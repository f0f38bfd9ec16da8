// Per-step solver kernels: boundary integrals of the point-source data
// (Section 2.3, F_i = int_lat (-q_N) N_i dS; the bottom projection), the
// theta-scheme right-hand side (Eq. theta-method) and Jacobi-PCG.
//
// Precision: the plain path runs every stage in FP64.  The mixed path keeps
// FP64 for the state, the residuals, the dot products and the initial
// residual of each solve, and applies the operator in FP32 (FP32 values and
// FP32 copies of the gathered Krylov vectors).  Each solve works on the
// increment from its FP64 initial guess, so the FP32 operator perturbs the
// increment only (relative ~1e-7), far below the residual tolerance measured
// against the full right-hand side.
#include <type_traits>

#include "sa_internal.h"

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// F^{n+1} = W_lat (-k dT~/dn)  and  b_bot = W_bot (T_c - T~): one warp per
// row of the constant weight matrices, fixed order, no atomics.  The same
// launch writes dev = T^n - T_c (FP64 and FP32) for the right-hand side.
// ---------------------------------------------------------------------------
struct GatherArgs {
    int wlat_rows;
    const int* rowdof;
    const int* lptr;
    const int* lcol;
    const double* lval;
    const double* s_lat;
    double k;
    int n_dir;
    const int* bptr;
    const int* bcol;
    const double* bval;
    const double* tt_bot;
    double Tc;
    double* F1;
    double* bbot;
    int n_dof;
    const double* That;
    double* dev64;
    float* dev32;
};

__global__ void k_gather(GatherArgs a) {
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long row_threads = 32ll * (a.wlat_rows + a.n_dir);
    if (gt >= row_threads) {
        const long long i = gt - row_threads;
        if (i < a.n_dof) {
            const double d = a.That[i] - a.Tc;
            a.dev64[i] = d;
            a.dev32[i] = (float)d;
        }
        return;
    }
    const int row = (int)(gt >> 5);
    const int lane = threadIdx.x & 31;
    if (row < a.wlat_rows) {
        double acc = 0.0;
        for (int s = a.lptr[row] + lane; s < a.lptr[row + 1]; s += 32)
            acc += a.lval[s] * a.s_lat[a.lcol[s]];
        acc = warp_sum(acc);
        if (lane == 0) a.F1[a.rowdof[row]] = -a.k * acc;
    } else {
        const int r = row - a.wlat_rows;
        double acc = 0.0;
        for (int s = a.bptr[r] + lane; s < a.bptr[r + 1]; s += 32)
            acc += a.bval[s] * (a.Tc - a.tt_bot[a.bcol[s]]);
        acc = warp_sum(acc);
        if (lane == 0) a.bbot[r] = acc;
    }
}

// ---------------------------------------------------------------------------
// SELL operator access (slice height 32, lane = row)
// ---------------------------------------------------------------------------
template <typename VT>
struct Op {
    int n, n_slices;
    const long long* sptr;
    const int* col32;      // absolute column, or
    const short* col16;    // column - row (when every offset fits in 16 bits)
    const VT* val;
    __device__ __forceinline__ int col(long long e, int row) const {
        return col16 ? row + (int)__ldg(col16 + e) : __ldg(col32 + e);
    }
};

// ---------------------------------------------------------------------------
// theta right-hand side on the free rows, as the initial residual of the
// increment system (x0 = T^n):
//   r0 = b - A_ff T^n_f = theta F^{n+1} + (1-theta) F^n - [K (T^n - T_c)]_f
//        - A_fd (g^{n+1} - g^n)
// (B - A = -K and K 1 = 0).  No large terms cancel, so the FP32 operator of
// the mixed path keeps r0 accurate relative to the increment.  The M values
// are read only for Dirichlet columns.
// ---------------------------------------------------------------------------
template <typename VT>
struct RhsArgs {
    Op<VT> K;              // free rows of K (unit k), all columns (internal)
    const VT* Mval;        // free rows of M (unit rho c_p), same storage as K
    const VT* dev;         // T^n - T_c
    const double* That;
    const double* gnew;
    const double* F0;
    const double* F1;
    int n_free;
    double inv_dt_rhocp, k, theta;
    double* r0;
};

template <typename VT>
__global__ void __launch_bounds__(256) k_theta_rhs(RhsArgs<VT> a) {
    const int sl = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (sl >= a.K.n_slices) return;
    const int i = sl * 32 + lane;
    const int ir = min(i, a.n_free - 1);
    const long long base = a.K.sptr[sl];
    const int w = (int)((a.K.sptr[sl + 1] - base) >> 5);
    VT acc = 0;
    double accd = 0.0;
    for (int k = 0; k < w; k += 8) {
        int jj[8];
        VT kv[8], dv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const bool ok = k + u < w;
            const long long e = base + 32ll * (ok ? k + u : 0) + lane;
            jj[u] = ok ? a.K.col(e, ir) : ir;
            kv[u] = ok ? __ldg(a.K.val + e) : (VT)0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) dv[u] = a.dev[jj[u]];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            acc = fma(kv[u], dv[u], acc);
            const int j = jj[u];
            if (k + u < w && j >= a.n_free) {   // Dirichlet column: - A_ij (g^{n+1}_j - g^n_j)
                const long long e = base + 32ll * (k + u) + lane;
                const double Aij = (double)__ldg(a.Mval + e) * a.inv_dt_rhocp +
                                   a.theta * a.k * (double)kv[u];
                accd += Aij * (a.gnew[j - a.n_free] - a.That[j]);
            }
        }
    }
    if (i < a.n_free)
        a.r0[i] = a.theta * a.F1[i] + (1.0 - a.theta) * a.F0[i] - a.k * (double)acc - accd;
}

// ---------------------------------------------------------------------------
// synchronisation policies for the PCG body
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Deterministic block reduction of NV values per thread into out[] (visible
// to every thread on return): fixed xor tree in the warps, fixed warp order.
template <int NV>
__device__ void block_reduce(double (&v)[NV], double* out) {
    __shared__ double sred[NV][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sred[k][w] = v[k];
    __syncthreads();
    if (threadIdx.x < NV) {
        double t = 0.0;
        for (int ww = 0; ww < nw; ++ww) t += sred[threadIdx.x][ww];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

// Grid-wide: per-block partials, a bounded-wait barrier (co-residency from
// the cooperative launch; a wait over the limit flags SA_DEV_TIMEOUT and the
// kernel returns), then every block sums all partials in the same order.
struct GridSync {
    unsigned* count;
    unsigned* gen;
    int* err;
    double* part;
    __device__ bool barrier() const {
        __shared__ int ok;
        __syncthreads();
        if (threadIdx.x == 0) {
            ok = 1;
            volatile unsigned* vgen = gen;
            const unsigned my = *vgen;
            __threadfence();
            const unsigned arrived = atomicAdd(count, 1u) + 1u;
            if (arrived == gridDim.x) {
                atomicExch(count, 0u);
                __threadfence();
                atomicAdd(gen, 1u);
            } else {
                const unsigned long long t0 = global_ns();
                long long spins = 0;
                while (*vgen == my) {
                    if ((++spins & 255) == 0) {
                        if (global_ns() - t0 > 2000000000ull || spins > (1ll << 30)) {
                            atomicOr(err, SA_DEV_TIMEOUT);
                            ok = 0;
                            break;
                        }
                        if (*((volatile int*)err) & SA_DEV_TIMEOUT) {
                            ok = 0;
                            break;
                        }
                    }
                }
            }
            __threadfence();
        }
        __syncthreads();
        return ok != 0;
    }
    // slot: first of NV consecutive partial rows of length gridDim.x
    template <int NV>
    __device__ bool reduce(double (&v)[NV], int slot, double (&out)[NV]) const {
        __shared__ double bl[NV];
        __shared__ double res[NV];
        block_reduce<NV>(v, bl);
        const int G = gridDim.x;
        if (threadIdx.x < NV) part[(slot + threadIdx.x) * G + blockIdx.x] = bl[threadIdx.x];
        if (!barrier()) return false;
        if (threadIdx.x < 32) {
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const volatile double* pk = part + (slot + k) * G;
                double t = 0.0;
                for (int i = threadIdx.x; i < G; i += 32) t += pk[i];
                t = warp_sum(t);
                if (threadIdx.x == 0) res[k] = t;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = res[k];
        __syncthreads();
        return true;
    }
};

// One block: __syncthreads only.
struct BlockSync {
    template <int NV>
    __device__ bool reduce(double (&v)[NV], int, double (&out)[NV]) const {
        __shared__ double res[NV];
        block_reduce<NV>(v, res);
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = res[k];
        __syncthreads();
        return true;
    }
};

template <typename VT>
struct PcgArgs {
    Op<VT> A;
    const double* val_hi;  // FP64 values of A (mode 0 initial residual); may equal A.val
    const double* dinv;
    const VT* dinvl;       // dinv in the operator precision
    const double* b;       // mode 0: right-hand side (r0 = b - A x)
    const double* r0;      // mode 1: initial residual (x0 = x); b = r0 + A x for the norm
    double* x;
    double* p;
    double* r[2];
    double* w[2];
    double* s[2];
    VT* rl[2];             // operator-precision copies of r, w, s (gathered by the SpMV)
    VT* wl[2];
    VT* sl[2];
    double* part;
    DevStatus* st;
    int which;             // 0 main solve, 1 bottom projection
    double tol;
    int max_iter;
    int ksplit;            // warps per slice in the SpMV (divides the warps of a block)
    VT* sq;                // shared scratch for the split partial sums (set in-kernel)
};

// SpMV over the warp units of a phase: slice sl = u / KS, part h = u % KS of
// its k-range; the KS warps of a slice sit in one block and their partial
// sums are added in fixed order in shared memory.  f(j) gives the gathered
// vector entry; own(i, acc) consumes the row result (h == 0 warp only).
template <typename VT, class Gather, class Own>
__device__ __forceinline__ void spmv_units(const PcgArgs<VT>& a, int gw, int nw, Gather f,
                                           Own own) {
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int KS = a.ksplit;
    const int units = a.A.n_slices * KS;
    const int rounds = (units + nw - 1) / nw;
    const int n = a.A.n;
    for (int rd = 0; rd < rounds; ++rd) {
        const int u = rd * nw + gw;
        const int sl = u / KS, h = u % KS;
        VT acc = 0;
        if (sl < a.A.n_slices) {
            const long long base = a.A.sptr[sl];
            const int w = (int)((a.A.sptr[sl + 1] - base) >> 5);
            const int chunk = (w + KS - 1) / KS;
            const int k0 = h * chunk, k1 = min(w, k0 + chunk);
            const int ir = min(sl * 32 + lane, n - 1);
            // explicit batches of 8: all column/value loads, then all
            // gathers, then the FMAs, so each lane keeps many independent
            // memory requests in flight (a plain loop serialises on the
            // column -> gather dependency of every entry)
            constexpr int B = std::is_same<VT, float>::value ? 8 : 4;   // registers
            for (int k = k0; k < k1; k += B) {
                int jj[B];
                VT vv[B];
#pragma unroll
                for (int u = 0; u < B; ++u) {
                    const bool ok = k + u < k1;
                    const long long e = base + 32ll * (ok ? k + u : k0) + lane;
                    jj[u] = ok ? a.A.col(e, ir) : ir;
                    vv[u] = ok ? __ldg(a.A.val + e) : (VT)0;
                }
                VT gg[B];
#pragma unroll
                for (int u = 0; u < B; ++u) gg[u] = f(jj[u]);
#pragma unroll
                for (int u = 0; u < B; ++u) acc = fma(vv[u], gg[u], acc);
            }
        }
        if (KS > 1) {
            a.sq[wib * 32 + lane] = acc;
            __syncthreads();
        }
        if (h == 0 && sl < a.A.n_slices) {
            VT tot = acc;
            for (int hh = 1; hh < KS; ++hh) tot += a.sq[(wib + hh) * 32 + lane];
            const int i = sl * 32 + lane;
            if (i < n) own(i, tot);
        }
        if (KS > 1) __syncthreads();
    }
}

// Jacobi-preconditioned CG in the Chronopoulos-Gear form: one global
// reduction per iteration.  With u = D^{-1} r and w = A u:
//   p = u + beta p ; s = w + beta s ; x += alpha p ; r -= alpha s ;
//   u = D^{-1} r ; w = A u ; gamma = (r, u), delta = (w, u), (r, r) ;
//   beta' = gamma'/gamma ; alpha' = gamma' / (delta' - beta' gamma'/alpha).
// The SpMV of w needs u of the neighbouring rows after their update; each
// lane recomputes it from the neighbours' previous r, w, s (double-buffered),
// so one iteration is a single grid phase followed by one reduction.
template <typename VT, class Sync>
__device__ void pcg_body(const PcgArgs<VT>& a, const Sync& sync, int gw, int nw, int tid,
                         int nth) {
    constexpr bool LO = std::is_same<VT, float>::value;
    const int n = a.A.n;
    double bb;
    // ---- mode 0: r0 = b - A x (FP64 values), then a grid sync
    if (a.r0 == nullptr) {
        double v[1] = {0.0};
        // the FP64 residual: a plain FP64 pass over the rows (one warp per slice)
        const int lane = threadIdx.x & 31;
        for (int sl = gw; sl < a.A.n_slices; sl += nw) {
            const long long base = a.A.sptr[sl];
            const int w = (int)((a.A.sptr[sl + 1] - base) >> 5);
            const int i = sl * 32 + lane;
            const int ir = min(i, n - 1);
            double acc = 0.0;
#pragma unroll 4
            for (int k = 0; k < w; ++k) {
                const long long e = base + 32ll * k + lane;
                acc = fma(__ldg(a.val_hi + e), a.x[a.A.col(e, ir)], acc);
            }
            if (i < n) {
                const double ri = a.b[i] - acc;
                a.r[0][i] = ri;
                if (LO) a.rl[0][i] = (VT)ri;
                v[0] += a.b[i] * a.b[i];
            }
        }
        double o[1];
        if (!sync.template reduce<1>(v, 0, o)) return;
        bb = o[0];
    }
    // ---- w0 = A D^{-1} r0 ; gamma, delta, (r, r) [and (b, b) in mode 1]
    double gamma, delta, rr;
    {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        const bool m1 = a.r0 != nullptr;
        const double* rsrc = m1 ? a.r0 : a.r[0];
        if (m1) {
            // A x for the norm of b = r0 + A x
            spmv_units(
                a, gw, nw, [&](int j) { return (VT)a.x[j]; },
                [&](int i, VT ax) {
                    const double bi = a.r0[i] + (double)ax;
                    v[3] += bi * bi;
                });
        }
        spmv_units(
            a, gw, nw,
            [&](int j) {
                return LO ? a.dinvl[j] * (VT)rsrc[j] : (VT)(a.dinv[j] * rsrc[j]);
            },
            [&](int i, VT wacc) {
                const double ri = rsrc[i];
                const double ui = a.dinv[i] * ri;
                const double wi = (double)wacc;
                if (m1) {
                    a.r[0][i] = ri;
                    if (LO) a.rl[0][i] = (VT)ri;
                }
                a.w[0][i] = wi;
                if (LO) a.wl[0][i] = (VT)wi;
                v[0] += ri * ui;
                v[1] += wi * ui;
                v[2] += ri * ri;
            });
        double o[4];
        if (!sync.template reduce<4>(v, 1, o)) return;
        gamma = o[0];
        delta = o[1];
        rr = o[2];
        if (m1) bb = o[3];
    }
    const double stop2 = a.tol * a.tol * bb;
    int it = 0;
    bool conv = rr <= stop2;
    bool nan = !(rr == rr) || !(delta == delta);
    double alpha = gamma / delta, beta = 0.0;
    while (!conv && !nan && it < a.max_iter) {
        const int c = it & 1;
        const bool first = (it == 0);
        const VT al = (VT)alpha, bl = (VT)beta;
        // buffer selection by value (no dynamic indexing of the argument arrays)
        const double* rc = c ? a.r[1] : a.r[0];
        const double* wc = c ? a.w[1] : a.w[0];
        const double* sc = c ? a.s[1] : a.s[0];
        double* rn = c ? a.r[0] : a.r[1];
        double* wn = c ? a.w[0] : a.w[1];
        double* sn = c ? a.s[0] : a.s[1];
        VT* rln = c ? a.rl[0] : a.rl[1];
        VT* wln = c ? a.wl[0] : a.wl[1];
        VT* sln = c ? a.sl[0] : a.sl[1];
        const VT* rlc = LO ? (c ? a.rl[1] : a.rl[0]) : (const VT*)rc;
        const VT* wlc = LO ? (c ? a.wl[1] : a.wl[0]) : (const VT*)wc;
        const VT* slc = LO ? (c ? a.sl[1] : a.sl[0]) : (const VT*)sc;
        const VT* dl = LO ? a.dinvl : (const VT*)a.dinv;
        double v[3] = {0.0, 0.0, 0.0};
        spmv_units(
            a, gw, nw,
            [&](int j) {
                const VT sj = first ? wlc[j] : fma(bl, slc[j], wlc[j]);
                return dl[j] * fma(-al, sj, rlc[j]);
            },
            [&](int i, VT wacc) {
                const double ui_old = a.dinv[i] * rc[i];
                const double pi = first ? ui_old : fma(beta, a.p[i], ui_old);
                const double si = first ? wc[i] : fma(beta, sc[i], wc[i]);
                a.p[i] = pi;
                a.x[i] = fma(alpha, pi, a.x[i]);
                const double ri = fma(-alpha, si, rc[i]);
                const double ui = a.dinv[i] * ri;
                const double wi = (double)wacc;
                rn[i] = ri;
                sn[i] = si;
                wn[i] = wi;
                if (LO) {
                    rln[i] = (VT)ri;
                    sln[i] = (VT)si;
                    wln[i] = (VT)wi;
                }
                v[0] += ri * ui;
                v[1] += wi * ui;
                v[2] += ri * ri;
            });
        double o[3];
        // partial rows alternate between two slot sets: a block may write the
        // next iteration's partials while a slower one still reads these
        if (!sync.template reduce<3>(v, 5 + 3 * c, o)) return;
        const double gnew = o[0];
        delta = o[1];
        rr = o[2];
        ++it;
        beta = gnew / gamma;
        alpha = gnew / (delta - beta * gnew / alpha);
        gamma = gnew;
        nan = !(rr == rr) || !(alpha == alpha);
        conv = rr <= stop2;
    }
    (void)tid;
    (void)nth;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double rel = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
        int* err = &a.st->err;
        if (a.which == 0) {
            a.st->pcg_iters = it;
            a.st->rel_res = rel;
            if (!conv) atomicOr(err, SA_DEV_NOT_CONVERGED);
        } else {
            a.st->bot_iters = it;
            a.st->bot_rel_res = rel;
            if (!conv) atomicOr(err, SA_DEV_BOT_NOT_CONVERGED);
        }
        if (nan) atomicOr(err, SA_DEV_NAN);
    }
}

constexpr int kPcgBlock = 1024;

template <typename VT>
__global__ void __launch_bounds__(kPcgBlock, 1) k_pcg_grid(PcgArgs<VT> a) {
    __shared__ VT sq[kPcgBlock];
    a.sq = sq;
    GridSync sync{&a.st->bar_count[a.which], &a.st->bar_gen[a.which], &a.st->err, a.part};
    const int nwb = blockDim.x >> 5;
    pcg_body<VT, GridSync>(a, sync, blockIdx.x * nwb + (threadIdx.x >> 5), gridDim.x * nwb,
                           blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

template <typename VT>
__global__ void __launch_bounds__(kPcgBlock, 1) k_pcg_block(PcgArgs<VT> a) {
    __shared__ VT sq[kPcgBlock];
    a.sq = sq;
    BlockSync sync;
    pcg_body<VT, BlockSync>(a, sync, threadIdx.x >> 5, blockDim.x >> 5, threadIdx.x, blockDim.x);
}

__global__ void k_finalize(int n_dir, int n_free, int n_dof, const double* gnew, double* That,
                           const double* F1, double* F0, DevStatus* st) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_dir) That[n_free + i] = gnew[i];
    if (i < n_dof) F0[i] = F1[i];
    if (i == 0) {
        st->n += 1;
        st->iters_total += st->pcg_iters;
        st->bot_total += st->bot_iters;
        if (st->pcg_iters > st->iters_max) st->iters_max = st->pcg_iters;
    }
}

template <typename VT>
Op<VT> make_op(const SellView& s, const void* val) {
    Op<VT> o;
    o.n = s.n;
    o.n_slices = s.n_slices;
    o.sptr = s.sptr;
    o.col32 = s.col32;
    o.col16 = s.col16;
    o.val = (const VT*)val;
    return o;
}

template <typename VT>
cudaError_t launch_pcg_t(const PcgLaunch& L, cudaStream_t s) {
    PcgArgs<VT> a;
    a.A = make_op<VT>(L.op, L.val);
    a.val_hi = L.val_hi;
    a.dinv = L.dinv;
    a.dinvl = (const VT*)L.dinvl;
    a.b = L.b;
    a.r0 = L.r0;
    a.x = L.x;
    a.p = L.w64;
    for (int k = 0; k < 2; ++k) {
        a.r[k] = L.w64 + (size_t)(1 + k) * L.stride;
        a.w[k] = L.w64 + (size_t)(3 + k) * L.stride;
        a.s[k] = L.w64 + (size_t)(5 + k) * L.stride;
        a.rl[k] = (VT*)L.w32 + (size_t)(0 + k) * L.stride;
        a.wl[k] = (VT*)L.w32 + (size_t)(2 + k) * L.stride;
        a.sl[k] = (VT*)L.w32 + (size_t)(4 + k) * L.stride;
    }
    a.part = L.partials;
    a.st = L.st;
    a.which = L.which;
    a.tol = L.tol;
    a.max_iter = L.max_iter;
    a.ksplit = L.ksplit > 0 ? L.ksplit : 1;
    a.sq = nullptr;
    if (L.grid <= 1) {
        k_pcg_block<VT><<<1, kPcgBlock, 0, s>>>(a);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(&L.st->bar_count[L.which], 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(L.grid);
    cfg.blockDim = dim3(kPcgBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_pcg_grid<VT>, a);
}

}  // namespace

cudaError_t launch_gather(int wlat_rows, const int* wlat_rowdof, const int* wlat_ptr,
                          const int* wlat_col, const double* wlat_val, const double* s_lat,
                          double k, int n_dir, const int* wbot_ptr, const int* wbot_col,
                          const double* wbot_val, const double* tt_bot, double Tc, double* F1,
                          double* bbot, int n_dof, const double* That, double* dev64,
                          float* dev32, cudaStream_t s) {
    GatherArgs a{wlat_rows, wlat_rowdof, wlat_ptr, wlat_col, wlat_val, s_lat, k, n_dir,
                 wbot_ptr, wbot_col, wbot_val, tt_bot, Tc, F1, bbot, n_dof, That, dev64, dev32};
    const long long threads = 32ll * ((long long)wlat_rows + n_dir) + n_dof;
    if (threads == 0) return cudaSuccess;
    k_gather<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_theta_rhs(int precision, const SellView& op, const void* Kval,
                             const void* Mval, const void* dev, const double* That,
                             const double* gnew, const double* F0, const double* F1,
                             double inv_dt_rhocp, double k, double theta, double* r0,
                             cudaStream_t s) {
    if (op.n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)(((long long)op.n_slices * 32 + 255) / 256);
    if (precision == SA_MIXED) {
        RhsArgs<float> a{make_op<float>(op, Kval), (const float*)Mval, (const float*)dev, That,
                         gnew, F0, F1, op.n, inv_dt_rhocp, k, theta, r0};
        k_theta_rhs<float><<<blocks, 256, 0, s>>>(a);
    } else {
        RhsArgs<double> a{make_op<double>(op, Kval), (const double*)Mval, (const double*)dev,
                          That, gnew, F0, F1, op.n, inv_dt_rhocp, k, theta, r0};
        k_theta_rhs<double><<<blocks, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

int pcg_block_size() { return kPcgBlock; }
const void* pcg_kernel_ptr(int precision) {
    return precision == SA_MIXED ? (const void*)k_pcg_grid<float> : (const void*)k_pcg_grid<double>;
}

cudaError_t launch_pcg(int precision, const PcgLaunch& L, cudaStream_t s) {
    if (L.op.n == 0) return cudaSuccess;
    return precision == SA_MIXED ? launch_pcg_t<float>(L, s) : launch_pcg_t<double>(L, s);
}

cudaError_t launch_finalize(int n_dir, int n_free, int n_dof, const double* gnew, double* That,
                            const double* F1, double* F0, DevStatus* st, cudaStream_t s) {
    const int nmax = n_dof > 1 ? n_dof : 1;
    k_finalize<<<(nmax + 255) / 256, 256, 0, s>>>(n_dir, n_free, n_dof, gnew, That, F1, F0, st);
    return cudaGetLastError();
}
