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
#include <cuda_bf16.h>

#include <type_traits>

#include "sa_async.cuh"
#include "sa_internal.h"

namespace {
using namespace sa_dev;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// F^{n+1} = W_lat (-k dT~/dn)  and  b_bot = W_bot (T_c - T~): eight lanes
// per row of the constant weight matrices, fixed order, no atomics.  The same
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
    int part;              // 0: everything; 1: lateral rows and dev; 2: bottom rows
    BotResid br;           // br.mptr != null: also r0 = b_bot - M_bot g0 and b_bot^2
    DevStatus* st;         // non-null: zero the grid-barrier counter of the solve that
                           // follows on the same stream (part 1: main, 2: bottom, 0: both)
};

// Eight lanes per row (rows hold ~10-40 entries): four rows per warp.  The
// lateral and the bottom row ranges are each padded to whole warps, so every
// warp is in one range and all its lanes reach the shuffles.
constexpr int kRowLanes = 8;

__host__ __device__ inline long long gather_range(long long rows) {
    return (kRowLanes * rows + 31) / 32 * 32;
}

__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
    for (int o = kRowLanes / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void k_gather(GatherArgs a) {
    if (a.st && blockIdx.x == 0 && threadIdx.x == 0) {
        if (a.part != 2) a.st->bar_count[0] = 0u;
        if (a.part != 1) a.st->bar_count[1] = 0u;
    }
    long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    // thread space: [lateral rows | bottom rows | dev], parts skip a range
    const long long lat_threads = gather_range(a.wlat_rows);
    if (a.part == 2) gt += lat_threads;
    const long long row_threads = lat_threads + (a.part == 1 ? 0 : gather_range(a.n_dir));
    if (gt >= row_threads) {
        if (a.part == 2) return;
        const long long i = gt - row_threads;
        if (i < a.n_dof) {
            const double d = a.That[i] - a.Tc;
            a.dev64[i] = d;
            a.dev32[i] = (float)d;
        }
        return;
    }
    const int sub = (int)(gt & (kRowLanes - 1));
    if (gt < lat_threads) {
        const int row = (int)(gt / kRowLanes);
        const bool ok = row < a.wlat_rows;
        double acc = 0.0;
        if (ok)
            for (int s = a.lptr[row] + sub; s < a.lptr[row + 1]; s += kRowLanes)
                acc += a.lval[s] * a.s_lat[a.lcol[s]];
        acc = group_sum(acc);
        if (ok && sub == 0) a.F1[a.rowdof[row]] = -a.k * acc;
    } else {
        const int r = (int)((gt - lat_threads) / kRowLanes);
        const bool ok = r < a.n_dir;
        double acc = 0.0, mg = 0.0;
        if (ok) {
            for (int s = a.bptr[r] + sub; s < a.bptr[r + 1]; s += kRowLanes)
                acc += a.bval[s] * (a.Tc - a.tt_bot[a.bcol[s]]);
            if (a.br.mptr)
                for (int s = a.br.mptr[r] + sub; s < a.br.mptr[r + 1]; s += kRowLanes)
                    mg += a.br.mval[s] * a.br.g0[a.br.mcol[s]];
        }
        acc = group_sum(acc);
        mg = group_sum(mg);
        if (ok && sub == 0) {
            a.bbot[r] = acc;
            if (a.br.mptr) {
                a.br.r0[r] = acc - mg;
                a.br.bsq[r] = acc * acc;
                if (a.br.fdZ) {
                    if (a.br.f32)
                        ((float*)a.br.fdZ)[r] = ((const float*)a.br.fdS)[r] * (float)(acc - mg);
                    else
                        ((double*)a.br.fdZ)[r] = ((const double*)a.br.fdS)[r] * (acc - mg);
                }
            }
        }
        if (a.br.npart) {
            // the warp's rows (whole warps lie in the bottom range), FP32
            // sums as for the main solve
            float b2 = ok && sub == 0 ? (float)(acc * acc) : 0.f;
            float r2 = ok && sub == 0 ? (float)((acc - mg) * (acc - mg)) : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                b2 += __shfl_xor_sync(0xffffffffu, b2, o);
                r2 += __shfl_xor_sync(0xffffffffu, r2, o);
            }
            if ((threadIdx.x & 31) == 0) {
                const long long w = (gt - lat_threads) >> 5;
                a.br.npart[2 * w] = b2;
                a.br.npart[2 * w + 1] = r2;
            }
        }
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
    const unsigned char* hi;   // per slice: holds a column >= n (null: unknown)
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
// the mixed path keeps r0 accurate relative to the increment.
// ---------------------------------------------------------------------------
template <typename VT>
struct RhsArgs {
    Op<VT> K;              // free rows of K (unit k), all columns (internal)
    const VT* Mval;        // free rows of M (unit rho c_p), same storage as K
    const VT* dev;         // T^n - T_c
    const VT* dg;          // Dirichlet dofs: g^{n+1} - g^n
    const VT* g1;          // Dirichlet dofs: g^{n+1}
    const double* F0;
    const double* F1;
    int n_free;
    double inv_dt_rhocp, k, theta, Tc;
    double* r0;
    double* bsq;           // b_i^2, for the norm of the right-hand side
    int only;              // 0: every slice; 1: slices without Dirichlet columns; 2: with
    // for the solve that follows (null: off): Z = S r0 of its
    // fast-diagonalization preconditioner, and per slice the sums of b_i^2
    // and r0_i^2 over its rows ([slice][2])
    const VT* fdS;
    VT* fdZ;
    float* npart;
    // FP32 path, slices without Dirichlet columns (null: off): column
    // offsets from the row and M as bf16 bit patterns
    const short* col16lo;
    const unsigned short* M16;
    int sl0, sl1;          // the launch covers slices [sl0, sl1)
};

// g^{n+1} - g^n and g^{n+1} in the operator precision, so that the rows
// coupled to Dirichlet columns need no FP64 arithmetic per entry.
template <typename VT>
__global__ void k_dir_prep(int n_dir, int n_free, const double* That, const double* gnew,
                           VT* dg, VT* g1) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= n_dir) return;
    const double g = gnew[d];
    dg[d] = (VT)(g - That[n_free + d]);
    g1[d] = (VT)g;
}

// One slice (warp; lane = row): K dev, M dev and the row sum of M; with DIR,
// also the M and K products with (g^{n+1} - g^n) and g^{n+1} on the
// Dirichlet columns.  DIR is uniform over the warp (a flag per slice), so
// slices without Dirichlet columns carry none of that work.
template <bool DIR, typename VT>
__device__ __forceinline__ void rhs_slice(const RhsArgs<VT>& a, long long base, int k0, int k1,
                                          int lane, int ir, VT (&acc)[7]) {
    if (!DIR && sizeof(VT) == 4 && a.col16lo != nullptr) {
        // 8 bytes a nonzero: FP32 K, bf16 M (exact widening), 16-bit offsets.
        // Software-pipelined in batches of 8: the next batch's offsets and
        // values are in flight while this batch's gathers of T^n - T_c wait
        // (two dependent loads a batch otherwise leave HBM half idle).
        short cj[8];
        VT kv[8];
        unsigned short mb[8];
        auto load = [&](int k, short (&c)[8], VT (&kk)[8], unsigned short (&m)[8]) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const bool ok = k + u < k1;
                const long long e = base + 32ll * (ok ? k + u : 0) + lane;
                c[u] = ok ? __ldg(a.col16lo + e) : (short)0;
                kk[u] = ok ? __ldg(a.K.val + e) : (VT)0;
                m[u] = ok ? __ldg(a.M16 + e) : (unsigned short)0;
            }
        };
        if (k0 < k1) load(k0, cj, kv, mb);
        for (int k = k0; k < k1; k += 8) {
            VT dv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) dv[u] = a.dev[ir + (int)cj[u]];
            short cn[8];
            VT kn[8];
            unsigned short mn[8];
            if (k + 8 < k1) load(k + 8, cn, kn, mn);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const VT mv = (VT)__uint_as_float((unsigned)mb[u] << 16);
                acc[0] = fma(kv[u], dv[u], acc[0]);
                acc[1] = fma(mv, dv[u], acc[1]);
                acc[2] += mv;
            }
            if (k + 8 < k1) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    cj[u] = cn[u];
                    kv[u] = kn[u];
                    mb[u] = mn[u];
                }
            }
        }
        return;
    }
    for (int k = k0; k < k1; k += 8) {
        int jj[8];
        VT kv[8], mv[8], dv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {     // independent loads first
            const bool ok = k + u < k1;
            const long long e = base + 32ll * (ok ? k + u : 0) + lane;
            jj[u] = ok ? a.K.col(e, ir) : ir;
            kv[u] = ok ? __ldg(a.K.val + e) : (VT)0;
            mv[u] = ok ? __ldg(a.Mval + e) : (VT)0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) dv[u] = a.dev[jj[u]];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            acc[0] = fma(kv[u], dv[u], acc[0]);
            acc[1] = fma(mv[u], dv[u], acc[1]);
            acc[2] += mv[u];
        }
        if (DIR) {
            VT dg[8], g1[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int jd = jj[u] - a.n_free;
                dg[u] = jd >= 0 ? a.dg[jd] : (VT)0;
                g1[u] = jd >= 0 ? a.g1[jd] : (VT)0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                acc[3] = fma(mv[u], dg[u], acc[3]);
                acc[4] = fma(kv[u], dg[u], acc[4]);
                acc[5] = fma(mv[u], g1[u], acc[5]);
                acc[6] = fma(kv[u], g1[u], acc[6]);
            }
        }
    }
}

// Also forms b itself (only its squares are kept, for the PCG stopping test):
//   b = (rho c_p/dt) M T^n - (1-theta) k K T^n + theta F^{n+1} + (1-theta) F^n
//       - A_fd g^{n+1},   with M T^n = T_c (M 1) + M (T^n - T_c)
// and A_fd = (rho c_p/dt) M_fd + theta k K_fd.
// Warps sharing one slice's columns: 4 when every slice runs (two slices a
// block), 8 for the slices with Dirichlet columns alone (a short launch on
// the step's critical path: more warps in flight per SM).
template <int kRhsSplit, typename VT>
__global__ void __launch_bounds__(256) k_theta_rhs(RhsArgs<VT> a) {
    // 8 warps: 8 / kRhsSplit slices, each split over kRhsSplit warps by
    // columns (enough warps in flight to cover the memory latency); partial
    // sums combined in fixed order
    __shared__ VT part[8][7][32];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sl = a.sl0 + blockIdx.x * (8 / kRhsSplit) + wib / kRhsSplit;
    const int h = wib % kRhsSplit;
    VT acc[7] = {0, 0, 0, 0, 0, 0, 0};
    bool live = sl < a.sl1;
    if (live && a.only != 0) {
        const bool dir = a.K.hi == nullptr || a.K.hi[sl];
        live = (a.only == 2) == dir;
    }
    const int i = sl * 32 + lane;
    if (live) {
        const int ir = min(i, a.n_free - 1);
        const long long base = a.K.sptr[sl];
        const int w = (int)((a.K.sptr[sl + 1] - base) >> 5);
        const int chunk = (((w + kRhsSplit - 1) / kRhsSplit) + 7) & ~7;
        const int k0 = min(w, h * chunk), k1 = min(w, k0 + chunk);
        if (a.K.hi == nullptr || a.K.hi[sl])
            rhs_slice<true>(a, base, k0, k1, lane, ir, acc);
        else
            rhs_slice<false>(a, base, k0, k1, lane, ir, acc);
    }
#pragma unroll
    for (int v = 0; v < 7; ++v) part[wib][v][lane] = acc[v];
    __syncthreads();
    if (!live || h != 0) return;
#pragma unroll
    for (int v = 0; v < 7; ++v) {
        VT t = part[wib][v][lane];
        for (int hh = 1; hh < kRhsSplit; ++hh) t += part[wib + hh][v][lane];
        acc[v] = t;
    }
    double b2 = 0.0, r2 = 0.0;
    if (i < a.n_free) {
        const double tk = a.theta * a.k;
        const double accd = a.inv_dt_rhocp * (double)acc[3] + tk * (double)acc[4];
        const double accg = a.inv_dt_rhocp * (double)acc[5] + tk * (double)acc[6];
        const double f = a.theta * a.F1[i] + (1.0 - a.theta) * a.F0[i];
        const double r = f - a.k * (double)acc[0] - accd;
        a.r0[i] = r;
        const double b = a.inv_dt_rhocp * (a.Tc * (double)acc[2] + (double)acc[1]) -
                         (1.0 - a.theta) * a.k * (double)acc[0] + f - accg;
        a.bsq[i] = b * b;
        if (a.fdZ) a.fdZ[i] = a.fdS[i] * (VT)r;
        b2 = b * b;
        r2 = r * r;
    }
    if (a.npart) {
        // FP32 sums (a norm for the stopping test needs no more; the solve
        // falls back to its own FP64 norms if they overflow)
        float fb = (float)b2, fr = (float)r2;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            fb += __shfl_xor_sync(0xffffffffu, fb, o);
            fr += __shfl_xor_sync(0xffffffffu, fr, o);
        }
        if (lane == 0) {
            a.npart[2 * sl] = fb;
            a.npart[2 * sl + 1] = fr;
        }
    }
}

// ---------------------------------------------------------------------------
// synchronisation policies for the PCG body
// ---------------------------------------------------------------------------

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

// Memory-model primitives of the grid barrier (PTX acquire/release at GPU
// scope: no separate fences).
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(unsigned* p, unsigned v) {
    asm volatile("st.relaxed.gpu.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide: per-block partials, a bounded-wait barrier (co-residency from
// the cooperative launch; a wait over the limit flags SA_DEV_TIMEOUT and the
// kernel returns), then every block sums all partials in the same order.
// Barrier: thread 0 reads the generation, arrives with an acq_rel atomic
// (releasing the block's writes, ordered before it by the CTA barrier); the
// last arrival resets the count and publishes the next generation with a
// release store; the others poll the generation with acquire loads.
struct GridSync {
    unsigned* count;
    int* err;
    double* part;
    mutable unsigned nb = 0;   // barriers passed (every thread counts alike)
    __device__ bool barrier() const { return count_barrier(count, nb, err, SA_DEV_TIMEOUT); }
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
                const double* pk = part + (slot + k) * G;
                double t = 0.0;
                for (int i = threadIdx.x; i < G; i += 32) t += __ldcg(pk + i);   // L2, not L1
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

constexpr int kPcgBlock = 1024;

template <typename VT>
struct PcgArgs {
    Op<VT> A;
    int dmin, dmax;        // column - row offsets (window mode)
    bool window;           // gathers from a shared-memory window of u
    int wcap;              // window capacity (entries) per block
    const double* val_hi;  // FP64 values of A (mode 0 initial residual)
    const double* dinv;
    const double* b;       // mode 0: right-hand side (r0 = b - A x)
    const double* r0;      // mode 1: initial residual (x0 = x)
    const double* bsq;     // mode 1: b_i^2 per row (for the norm of b)
    double* x;
    double* p;
    double* r;
    double* w;
    double* s;
    double* u;
    VT* ul;                // u in the operator precision, padded: ul[-pad .. n + pad)
    double* part;
    DevStatus* st;
    int which;             // 0 main solve, 1 bottom projection
    double tol;
    int max_iter;
    int ksplit;            // warps per slice (divides the 32 warps of a block)
    const float* dx0;      // mode 1: proposed increment (scaled by *dx0_scale), or null
    const double* dx0_scale;
};

// Block b owns slices [s0, s1) (contiguous, balanced) and their rows.
__device__ __forceinline__ void block_slices(int S, int& s0, int& s1) {
    s0 = (int)(((long long)S * blockIdx.x) / gridDim.x);
    s1 = (int)(((long long)S * (blockIdx.x + 1)) / gridDim.x);
}

// What a block's SpMV needs of the operator and of the vector it gathers.
template <typename VT>
struct SpmvPlan {
    Op<VT> A;
    int dmin, dmax;        // column - row offsets (window mode)
    bool window;           // gathers from a shared-memory window of src
    int ksplit;            // warps per slice (divides the 32 warps of a block)
};

// Asynchronous window copy: an mbarrier in shared memory and the number of
// copies issued so far (every thread of the block counts the same calls).
struct WinAsync {
    unsigned long long* mbar;
    unsigned count;
    int* err;
};

// y = A src on the block's slices.  Window mode: the entries of src the
// block can touch, src[32 s0 + dmin .. 32 s1 + dmax), are first copied into
// shared memory, so every gather is a shared-memory read.  With wa, one
// thread issues that copy as one bulk asynchronous copy (TMA engine) and the
// warps load their first batch of matrix entries before waiting for it;
// otherwise the threads copy it (coalesced loads).  src is written by other
// blocks during the kernel, so it is read through L2 (ld.global.cg, or the
// bulk copy), never from a stale L1 line.  Each slice is split over KS
// consecutive warps (partial sums combined in fixed order).  own(i, y_i)
// runs once per row.
template <typename VT, class Own>
__device__ void spmv_block(const SpmvPlan<VT>& a, const VT* src, VT* win, VT* sq, Own own,
                           WinAsync* wa = nullptr) {
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int nwb = blockDim.x >> 5;
    const int n = a.A.n;
    int s0, s1;
    block_slices(a.A.n_slices, s0, s1);
    long long wlo = 0;
    bool pending = false;       // window copy issued, not yet waited for
    unsigned parity = 0;
    if (a.window) {
        wlo = ((long long)32 * s0 + a.dmin) & ~3ll;               // aligned start
        const long long whi = (long long)32 * s1 + a.dmax + 1;
        const int len = (int)(whi - wlo);
        if (wa != nullptr) {
            // 16-byte multiple (the padding of src covers the rounding)
            const unsigned bytes = (unsigned)((len * sizeof(VT) + 15) & ~(size_t)15);
            if (threadIdx.x == 0) {
                fence_proxy_async();
                bulk_load(win, src + wlo, bytes, wa->mbar);
            }
            parity = wa->count & 1u;
            wa->count += 1;
            pending = true;
        } else {
            // 8 independent loads in flight per thread, then the stores
            for (int t0 = threadIdx.x; t0 < len; t0 += 8 * blockDim.x) {
                VT tmp[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int t = t0 + u * blockDim.x;
                    tmp[u] = t < len ? __ldcg(src + wlo + t) : (VT)0;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int t = t0 + u * blockDim.x;
                    if (t < len) win[t] = tmp[u];
                }
            }
            __syncthreads();
        }
    }
    const int KS = a.ksplit;
    const int units = (s1 - s0) * KS;
    for (int base_u = 0; base_u < units; base_u += nwb) {
        const int u = base_u + wib;
        const int sl = s0 + u / KS, h = u % KS;
        VT acc = 0;
        if (u < units) {
            const long long base = a.A.sptr[sl];
            const int w = (int)((a.A.sptr[sl + 1] - base) >> 5);
            const int chunk = (w + KS - 1) / KS;
            const int k0 = h * chunk, k1 = min(w, k0 + chunk);
            const int ir = min(sl * 32 + lane, n - 1);
            if (a.window) {
                const VT* wv = win - wlo;
                // batches of 16: every column/value load of the batch is in
                // flight before the first (shared-memory) gather
                for (int k = k0; k < k1; k += 16) {
                    short dj[16];
                    VT vv[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const bool ok = k + u < k1;
                        const long long e = base + 32ll * (ok ? k + u : k0) + lane;
                        dj[u] = ok ? __ldg(a.A.col16 + e) : (short)0;
                        vv[u] = ok ? __ldg(a.A.val + e) : (VT)0;
                    }
                    if (pending) {
                        if (!mbar_wait_bounded(wa->mbar, parity)) atomicOr(wa->err, SA_DEV_TIMEOUT);
                        pending = false;
                    }
#pragma unroll
                    for (int u = 0; u < 16; ++u) acc = fma(vv[u], wv[ir + (int)dj[u]], acc);
                }
            } else {
#pragma unroll 8
                for (int k = k0; k < k1; ++k) {
                    const long long e = base + 32ll * k + lane;
                    acc = fma(__ldg(a.A.val + e), __ldcg(src + a.A.col(e, ir)), acc);
                }
            }
        }
        if (KS > 1) {
            sq[wib * 32 + lane] = acc;
            __syncthreads();
        }
        if (u < units && h == 0) {
            VT tot = acc;
            for (int hh = 1; hh < KS; ++hh) tot += sq[(wib + hh) * 32 + lane];
            const int i = sl * 32 + lane;
            if (i < n) own(i, tot);
        }
        if (KS > 1) __syncthreads();
    }
    // a thread without matrix work still observes the copy's completion, so
    // that no copy is in flight into the window when the block reuses it
    if (pending && !mbar_wait_bounded(wa->mbar, parity)) atomicOr(wa->err, SA_DEV_TIMEOUT);
}

template <typename VT>
__device__ __forceinline__ SpmvPlan<VT> plan_of(const PcgArgs<VT>& a) {
    return SpmvPlan<VT>{a.A, a.dmin, a.dmax, a.window, a.ksplit};
}

// Jacobi-preconditioned CG in the Chronopoulos-Gear form (u = D^{-1} r,
// w = A u, s = A p):
//   V: p = u + beta p ; s = w + beta s ; x += alpha p ; r -= alpha s ;
//      u = D^{-1} r                                   (own rows; grid sync)
//   S: w = A u ; gamma = (r, u), delta = (w, u), (r, r) (one reduction)
//   beta' = gamma'/gamma ; alpha' = gamma' / (delta' - beta' gamma'/alpha)
// Two grid syncs per iteration; the SpMV gathers only u, from shared memory.
template <typename VT>
__global__ void __launch_bounds__(1024, 1) k_pcg(PcgArgs<VT> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    VT* sq = (VT*)smem_raw;                 // 1024
    VT* win = sq + 1024;                    // window
    GridSync sync{&a.st->bar_count[a.which], &a.st->err, a.part};
    const int n = a.A.n;
    int s0, s1;
    block_slices(a.A.n_slices, s0, s1);
    const int row0 = 32 * s0, row1 = min(32 * s1, n);
    const int lane = threadIdx.x & 31;
    // ---- initial residual, u0, the norm of b
    double bb;
    {
        double v[1] = {0.0};
        if (a.r0 == nullptr) {   // mode 0: r = b - A x in FP64 (global gathers)
            const int wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
            for (int sl = s0 + wib; sl < s1; sl += nwb) {
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
                    const double bi = a.b[i], ri = bi - acc, ui = a.dinv[i] * ri;
                    a.r[i] = ri;
                    a.u[i] = ui;
                    a.ul[i] = (VT)ui;
                    v[0] += bi * bi;
                }
            }
        } else {                 // mode 1: r = r0 given
            bool warm = false;
            if (a.dx0) {
                // proposed start x0 + dx: its residual r0 - A dx, kept only if
                // smaller than r0 (otherwise the cold start x0 stays)
                const double sc = *a.dx0_scale;
                for (int i = row0 + threadIdx.x; i < row1; i += blockDim.x) a.ul[i] = (VT)(sc * a.dx0[i]);
                if (!sync.barrier()) return;
                double vw[2] = {0.0, 0.0};
                spmv_block(plan_of(a), a.ul, win, sq, [&](int i, VT t) {
                    const double rw = a.r0[i] - (double)t;
                    a.r[i] = rw;
                    vw[0] += rw * rw;
                    vw[1] += a.r0[i] * a.r0[i];
                });
                double ow[2];
                if (!sync.template reduce<2>(vw, 10, ow)) return;
                warm = ow[0] < ow[1];
                if (blockIdx.x == 0 && threadIdx.x == 0) {
                    a.st->ws_used = warm ? 1 : 0;
                    a.st->ws_ratio = ow[1] > 0.0 ? sqrt(ow[0] / ow[1]) : 0.0;
                }
                if (warm)
                    for (int i = row0 + threadIdx.x; i < row1; i += blockDim.x)
                        a.x[i] = fma(sc, (double)a.dx0[i], a.x[i]);
            }
            for (int i = row0 + threadIdx.x; i < row1; i += blockDim.x) {
                const double ri = warm ? a.r[i] : a.r0[i], ui = a.dinv[i] * ri;
                a.r[i] = ri;
                a.u[i] = ui;
                a.ul[i] = (VT)ui;
                v[0] += a.bsq[i];
            }
        }
        double o[1];
        if (!sync.template reduce<1>(v, 0, o)) return;
        bb = o[0];
    }
    double gamma, delta, rr;
    {
        double v[3] = {0.0, 0.0, 0.0};
        spmv_block(plan_of(a), a.ul, win, sq, [&](int i, VT wacc) {
            const double wi = (double)wacc, ui = a.u[i], ri = a.r[i];
            a.w[i] = wi;
            v[0] += ri * ui;
            v[1] += wi * ui;
            v[2] += ri * ri;
        });
        double o[3];
        if (!sync.template reduce<3>(v, 1, o)) return;
        gamma = o[0];
        delta = o[1];
        rr = o[2];
    }
    // scalar recurrences in one thread per block (FP64 division is slow on
    // this part: every other thread only reads the results)
    __shared__ double sc[4];   // alpha, beta, gamma, state (0 run, 1 converged, 2 nan)
    const double stop2 = a.tol * a.tol * bb;
    if (threadIdx.x == 0) {
        sc[0] = gamma / delta;
        sc[1] = 0.0;
        sc[2] = gamma;
        sc[3] = !(rr == rr) || !(delta == delta) ? 2.0 : (rr <= stop2 ? 1.0 : 0.0);
    }
    __syncthreads();
    int it = 0;
    double alpha = sc[0], beta = sc[1];
    bool conv = sc[3] == 1.0, nan = sc[3] == 2.0;
    __syncthreads();
    while (!conv && !nan && it < a.max_iter) {
        const bool first = (it == 0);
        // ---- V (own rows)
        for (int i = row0 + threadIdx.x; i < row1; i += blockDim.x) {
            const double ui = a.u[i], wi = a.w[i];
            const double pi = first ? ui : fma(beta, a.p[i], ui);
            const double si = first ? wi : fma(beta, a.s[i], wi);
            a.p[i] = pi;
            a.s[i] = si;
            a.x[i] = fma(alpha, pi, a.x[i]);
            const double ri = fma(-alpha, si, a.r[i]);
            const double un = a.dinv[i] * ri;
            a.r[i] = ri;
            a.u[i] = un;
            a.ul[i] = (VT)un;
        }
        if (!sync.barrier()) return;
        // ---- S
        double v[3] = {0.0, 0.0, 0.0};
        spmv_block(plan_of(a), a.ul, win, sq, [&](int i, VT wacc) {
            const double wi = (double)wacc, ui = a.u[i], ri = a.r[i];
            a.w[i] = wi;
            v[0] += ri * ui;
            v[1] += wi * ui;
            v[2] += ri * ri;
        });
        double o[3];
        // two slot sets: the next iteration's partials may be written while a
        // slower block still reads these
        if (!sync.template reduce<3>(v, 4 + 3 * (it & 1), o)) return;
        ++it;
        rr = o[2];
        if (threadIdx.x == 0) {
            const double gnew = o[0], dl = o[1];
            const double bt = gnew / sc[2];
            const double al = gnew / (dl - bt * gnew / sc[0]);
            sc[0] = al;
            sc[1] = bt;
            sc[2] = gnew;
            sc[3] = !(rr == rr) || !(al == al) ? 2.0 : (rr <= stop2 ? 1.0 : 0.0);
        }
        __syncthreads();
        alpha = sc[0];
        beta = sc[1];
        conv = sc[3] == 1.0;
        nan = sc[3] == 2.0;
        __syncthreads();
    }
    (void)gamma;
    (void)delta;
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

// ---------------------------------------------------------------------------
// Jacobi-PCG in the Chronopoulos-Gear form with every block's vectors in
// shared memory (FP64; u = D^{-1} r also published in the operator
// precision for the other blocks' gathers).  Per iteration:
//   V: p = u + beta p ; s = w + beta s ; d += alpha p ; r -= alpha s ;
//      u = D^{-1} r, published                         (grid barrier)
//   S: w = A u ; partial (r, u), (w, u), (r, r)         (grid reduction)
//   beta' = gamma'/gamma ; alpha' = gamma' / (delta' - beta' gamma'/alpha)
// d is the increment from the initial guess; x += d on exit.  Block partial
// sums are combined across blocks in a fixed order (deterministic).  The
// pipelined recurrences (one barrier per iteration) were tried and
// rejected: with the FP32 operator they stall near 1e-8 of ||b||.
// ---------------------------------------------------------------------------
constexpr int kSmemVecs = 7;   // d r u w s p dinv (FP64), then sigma r, sigma u in VT

template <typename VT>
struct SmemArgs {
    SpmvPlan<VT> plan;
    int rcap;              // rows per block (shared-memory vector length)
    const double* val_hi;  // FP64 values of A (mode 0 initial residual)
    const double* dinv;    // D^{-1}
    const double* b;       // mode 0: right-hand side (r0 = b - A x)
    const double* r0;      // mode 1: initial residual
    const double* bsq;     // mode 1: b_i^2 per row (for the norm of b)
    double* x;
    VT* ul;                // u published in VT, padded: ul[-pad .. n + pad)
    double* part;
    DevStatus* st;
    int which;
    double tol;
    int max_iter;
    const float* dx0;      // mode 1: proposed increment (scaled by *dx0_scale), or null
    const double* dx0_scale;
    const void* dinvl;     // D^{-1} in VT
    FdView fd;             // fast-diagonalization preconditioner (fd.on), else Jacobi
    const float* npart;    // with r0 and fd: the producer's per-slice (b^2, r0^2) sums and
    int npart_n;           // Z = S r0 already written (slices), else null
    // non-null fin_F1: the step's finalize at the end (see PcgLaunch)
    const double* fin_F1;
    double* fin_F0;
    const double* fin_g;
    double* fin_That;      // That + ... : the Dirichlet entries start at n (= n_free)
    int fin_n_dof, fin_n_dir;
    int fd_mmax;           // longest grid line (per-warp scratch entries)
    int plan_wcap;         // window entries reserved in shared memory
    const double* dir_old; // see PcgLaunch
    VT* dir_out;
    int fd_w2;             // 1: the region holds three m x m matrices (the fused
                           // pass's second one staged too), 0: two
    int fd_rows;           // > 0: plane form of the 3-D preconditioner with slabs
                           // of this many rows; 0: the line form
};

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sums of NV per-thread values (warp tree in AT, the 32 warp results
// in AT by warp 0, in fixed order) -> out[k] (shared, all threads).
template <int NV, typename AT>
__device__ void block_sum(AT (&v)[NV], AT* out) {
    __shared__ AT sb[NV][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum_t(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sb[k][w] = v[k];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            AT t = lane < nw ? sb[k][lane] : (AT)0;
            t = warp_sum_t(t);
            if (lane == 0) out[k] = t;
        }
    }
    __syncthreads();
}

// Block values bl[0..NV) -> partial slots (AT), grid barrier, the sum over
// all blocks in AT in a fixed order (identical in every block) -> res[k]
// (FP64, shared, all threads).
constexpr int kMaxGrid = 256;

template <int NV, typename AT>
__device__ bool grid_exchange(const GridSync& g, const AT* bl, int slot, double* res) {
    __shared__ AT gv[NV * kMaxGrid];
    const int G = gridDim.x;
    AT* part = (AT*)g.part;
    if (threadIdx.x < NV) part[(slot + threadIdx.x) * G + blockIdx.x] = bl[threadIdx.x];
    if (!g.barrier()) return false;
    // the NV rows of partials are contiguous: one load per thread, all in
    // flight together, then fixed-order sums from shared memory
    const AT* src = part + slot * G;
    const bool staged = G <= kMaxGrid;
    if (staged) {
        for (int t = threadIdx.x; t < NV * G; t += blockDim.x) gv[t] = __ldcg(src + t);
        __syncthreads();
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < NV) {
        AT t = (AT)0;
        for (int i = lane; i < G; i += 32) t += staged ? gv[w * G + i] : __ldcg(src + w * G + i);
        t = warp_sum_t(t);
        if (lane == 0) res[w] = (double)t;
    }
    __syncthreads();
    return true;
}

constexpr int kFdPerLane = 4;   // line entries per lane: lines of at most 128

// Fast-diagonalization preconditioner u = S A_box^{-1} S r over all rows.
// On entry Z = S r (every block wrote its rows, then a grid barrier).  Five
// passes over lines of the free grid (U_0^T, U_1^T, U_2 D U_2^T, U_1, U_0),
// one warp per line (in place: a line is read and written by one warp), a
// grid barrier between passes; the last pass writes S y into out.  Each
// block first copies the pass's m x m matrix into shared memory (wbuf, at
// least m^2 entries; the SpMV window is idle here).  Lines have at most 128
// entries (4 per lane).
template <typename VT>
__device__ __forceinline__ void fd_stage(VT* wbuf, const VT* W, int m) {
    const int mm = m * m;
    for (int t = threadIdx.x; t < mm; t += blockDim.x) wbuf[t] = __ldg(W + t);
}

template <typename VT>
__device__ __forceinline__ void fd_line_matvec(const VT* Wb, const VT* xs, int m, int lane, VT (&y)[kFdPerLane]) {
    // y[o] = sum_a Wb[a][o] xs[a], o = lane + 32 t
#pragma unroll
    for (int t = 0; t < kFdPerLane; ++t) y[t] = (VT)0;
#pragma unroll 4
    for (int a = 0; a < m; ++a) {
        const VT xa = xs[a];
        const VT* Wa = Wb + a * m;
#pragma unroll
        for (int t = 0; t < kFdPerLane; ++t) {
            const int o = lane + 32 * t;
            if (o < m) y[t] = fma(Wa[o], xa, y[t]);
        }
    }
}

template <typename VT>
__device__ bool fd_apply(const FdView& fd, const GridSync& sync, VT* wbuf, VT* xs, VT* out,
                         bool w2s) {
    const int lane = threadIdx.x & 31;
    // lines go to warp w of every block before warp w + 1 of any: spread over SMs
    const int gw = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int nd = fd.nd;                  // 3: passes 0 1 2f 1 0; 2: passes 0 1f 0
    const int npass = 2 * nd - 1;
    const int m0 = fd.m[0], m1 = fd.m[1], m2 = fd.m[2];
    const int mmax = max(m0, max(m1, m2));
    VT* Z = (VT*)fd.Z;
    const VT* S = (const VT*)fd.S;
    const VT* l0 = (const VT*)fd.lamc[0];
    const VT* l1 = (const VT*)fd.lamc[1];
    const VT* ll = (const VT*)fd.lamc[nd - 1];
    const VT cM = (VT)fd.cM;
    for (int pass = 0; pass < npass; ++pass) {
        const int d = pass < nd ? pass : npass - 1 - pass;
        const bool fused = pass == nd - 1;
        const int m = fd.m[d];
        const int stride = d == 0 ? 1 : (d == 1 ? m0 : m0 * m1);
        const int nlines = (m0 * m1 * m2) / m;
        // y[o] = sum_a W[a][o] x[a]: W = U_d (applies U_d^T) or U_d^T (applies
        // U_d), staged in wbuf + (pass & 1) mmax^2: the first by itself, the
        // next ones while the block waits at the grid barrier
        VT* Wb = wbuf + (pass & 1) * mmax * mmax;
        if (pass == 0) fd_stage(Wb, (const VT*)fd.U[0], m);
        __syncthreads();
        for (int L = gw; L < nlines; L += nw) {
            const int base = d == 0 ? L * m0 : (d == 1 ? (L / m0) * (m0 * m1) + (L % m0) : L);
            for (int a = lane; a < m; a += 32) xs[a] = __ldcg(Z + base + (long long)a * stride);
            __syncwarp();
            VT y[kFdPerLane];
            fd_line_matvec(Wb, xs, m, lane, y);
            if (fused) {
                // D = 1 / (c_M + sum_d c_d lambda_d), then U on the same line
                // (the last direction's U^T from global memory)
                const VT li = cM + l0[L % m0] + (nd == 3 ? l1[L / m0] : (VT)0);
                __syncwarp();
#pragma unroll
                for (int t = 0; t < kFdPerLane; ++t) {
                    const int o = lane + 32 * t;
                    if (o < m) xs[o] = y[t] / (li + ll[o]);
                }
                __syncwarp();
                if (w2s) {
                    fd_line_matvec(wbuf + 2 * mmax * mmax, xs, m, lane, y);
                } else {
                    const VT* W2 = (const VT*)fd.Ut[d];
#pragma unroll
                    for (int t = 0; t < kFdPerLane; ++t) y[t] = (VT)0;
#pragma unroll 4
                    for (int a = 0; a < m; ++a) {
                        const VT xa = xs[a];
                        const VT* Wa = W2 + a * m;
#pragma unroll
                        for (int t = 0; t < kFdPerLane; ++t) {
                            const int o = lane + 32 * t;
                            if (o < m) y[t] = fma(__ldg(Wa + o), xa, y[t]);
                        }
                    }
                }
            }
            __syncwarp();
#pragma unroll
            for (int t = 0; t < kFdPerLane; ++t) {
                const int o = lane + 32 * t;
                if (o < m) {
                    const long long idx = base + (long long)o * stride;
                    if (pass == npass - 1)
                        out[idx] = S[idx] * y[t];
                    else
                        Z[idx] = y[t];
                }
            }
            __syncwarp();
        }
        if (pass < npass - 1) {
            const int np = pass + 1;
            const int dn = np < nd ? np : npass - 1 - np;
            fd_stage(wbuf + (np & 1) * mmax * mmax, (const VT*)(np < nd ? fd.U[dn] : fd.Ut[dn]), fd.m[dn]);
            // the fused pass's second matrix (U_d^T) in the third buffer
            if (w2s && np == nd - 1) fd_stage(wbuf + 2 * mmax * mmax, (const VT*)fd.Ut[dn], fd.m[dn]);
            if (!sync.barrier()) return false;
        }
    }
    return true;
}

// Plane form of the 3-D preconditioner: u = S (U_2 (x) U_1 (x) U_0) D^{-1}
// (U_2 (x) U_1 (x) U_0)^T S r in three passes with two grid barriers
// (instead of five line passes and four):
//   A  every z-plane X (m1 x m0, x fastest) becomes U_1^T X U_0, Z -> Z2;
//   B  z-lines of Z2: U_2^T, the diagonal D, U_2, -> Z (the line pass of the
//      line form);
//   C  every plane becomes U_1 X U_0^T, times S, -> out.
// A plane is split into slabs of `rows` output rows over several blocks (the
// block count over the plane count), so that every SM works and no block
// transforms a whole plane alone; each block stages the plane, the m0 x m0
// matrix and its slab's columns of the m1 x m1 one in shared memory (wbuf:
// plane_slab_need entries) and forms its slab as two small products.
//
// The staging is asynchronous (cp.async): every copy of a thread is in flight
// at once, one L2 round trip for the whole stage instead of one per element
// that a load-then-store loop costs.  The plane is data other blocks wrote in
// this launch, so it goes in 16-byte chunks around L1 (.cg); the constant
// matrices go element by element through L1 (.ca).

// Shared-memory entries plane_slab stages for slabs of `rows` rows (16-byte
// alignment slack included).
__host__ __device__ inline long long plane_stage_entries(int m0, int m1, int rows) {
    return (long long)m0 * m1 + (long long)m0 * m0 + (long long)m1 * rows + (long long)rows * m0 +
           m0 + rows + 4;
}

template <typename VT>
__device__ void plane_slab(const VT* src, VT* dst, const VT* Sv, const VT* W1, const VT* W0,
                           int m0, int m1, int plane, int j0, int nrow, VT* wbuf,
                           const FdView* dg = nullptr) {
    // X (16-byte aligned) m1 x m0; A0 m0 x m0: W0[i][o]; A1 m1 x nrow:
    // W1[j][j0 + r]; Tm nrow x m0; 2-D: lambda_0 (m0), lambda_1 of the rows
    VT* X = (VT*)(((uintptr_t)wbuf + 15) & ~(uintptr_t)15);
    VT* A0 = X + m0 * m1;
    VT* A1 = A0 + m0 * m0;
    VT* Tm = A1 + m1 * nrow;
    VT* dl0 = Tm + nrow * m0;
    VT* dl1 = dl0 + m0;
    const long long base = (long long)plane * m0 * m1;
    const int nx = m0 * m1;
    __syncthreads();                    // wbuf free
    const VT* xsrc = src + base;
    if ((nx * (int)sizeof(VT)) % 16 == 0 && ((uintptr_t)xsrc & 15) == 0) {
        const int nc = nx * (int)sizeof(VT) / 16;
        for (int t = threadIdx.x; t < nc; t += blockDim.x)
            cp_async_cg16((char*)X + 16 * t, (const char*)xsrc + 16 * t);
    } else {
        for (int t = threadIdx.x; t < nx; t += blockDim.x) X[t] = __ldcg(xsrc + t);
    }
    for (int t = threadIdx.x; t < m0 * m0; t += blockDim.x) cp_async_ca<sizeof(VT)>(A0 + t, W0 + t);
    for (int t = threadIdx.x; t < m1 * nrow; t += blockDim.x) {
        const int j = t / nrow, r = t - j * nrow;
        cp_async_ca<sizeof(VT)>(A1 + t, W1 + j * m1 + j0 + r);
    }
    if (dg) {
        for (int t = threadIdx.x; t < m0 + nrow; t += blockDim.x) {
            if (t < m0) cp_async_ca<sizeof(VT)>(dl0 + t, (const VT*)dg->lamc[0] + t);
            else cp_async_ca<sizeof(VT)>(dl1 + (t - m0), (const VT*)dg->lamc[1] + j0 + (t - m0));
        }
    }
    cp_async_wait_all();
    __syncthreads();
    // T[r][i] = sum_j W1[j][j0 + r] X[j][i], one output a thread, the sum in
    // three interleaved partial sums (j mod 3: a third of the dependent chain)
    for (int t = threadIdx.x; t < nrow * m0; t += blockDim.x) {
        const int r = t / m0, i = t - r * m0;
        VT s0 = (VT)0, s1 = (VT)0, s2 = (VT)0;
        int j = 0;
#pragma unroll 2
        for (; j + 3 <= m1; j += 3) {
            s0 = fma(A1[j * nrow + r], X[j * m0 + i], s0);
            s1 = fma(A1[(j + 1) * nrow + r], X[(j + 1) * m0 + i], s1);
            s2 = fma(A1[(j + 2) * nrow + r], X[(j + 2) * m0 + i], s2);
        }
        for (; j < m1; ++j) s0 = fma(A1[j * nrow + r], X[j * m0 + i], s0);
        Tm[t] = (s0 + s1) + s2;
    }
    __syncthreads();
    // Y[r][o] = sum_i W0[i][o] T[r][i], the same way
    for (int t = threadIdx.x; t < nrow * m0; t += blockDim.x) {
        const int r = t / m0, o = t - r * m0;
        const VT* Tr = Tm + r * m0;
        VT s0 = (VT)0, s1 = (VT)0, s2 = (VT)0;
        int i = 0;
#pragma unroll 2
        for (; i + 3 <= m0; i += 3) {
            s0 = fma(A0[i * m0 + o], Tr[i], s0);
            s1 = fma(A0[(i + 1) * m0 + o], Tr[i + 1], s1);
            s2 = fma(A0[(i + 2) * m0 + o], Tr[i + 2], s2);
        }
        for (; i < m0; ++i) s0 = fma(A0[i * m0 + o], Tr[i], s0);
        VT v = (s0 + s1) + s2;
        const long long idx = base + (long long)(j0 + r) * m0 + o;
        if (dg)   // 2-D: the diagonal D = 1 / (c_M + c_0 lambda_0 + c_1 lambda_1)
            v = v / ((VT)dg->cM + dl0[o] + dl1[r]);
        dst[idx] = Sv ? Sv[idx] * v : v;
    }
}

template <typename VT>
__device__ bool fd_apply_planes(const FdView& fd, const GridSync& sync, VT* wbuf, VT* xs, VT* out,
                                int rows) {
    const int lane = threadIdx.x & 31;
    const int m0 = fd.m[0], m1 = fd.m[1], m2 = fd.m[2];
    VT* Z = (VT*)fd.Z;
    VT* Z2 = (VT*)fd.Z2;
    const VT* S = (const VT*)fd.S;
    const int nslab = (m1 + rows - 1) / rows;
    const int items = m2 * nslab;
    if (fd.nd == 2) {
        // one plane: A with the diagonal applied, then C (one grid barrier)
        for (int it = blockIdx.x; it < nslab; it += gridDim.x) {
            const int j0 = it * rows;
            plane_slab<VT>(Z, Z2, nullptr, (const VT*)fd.U[1], (const VT*)fd.U[0], m0, m1, 0, j0,
                           min(rows, m1 - j0), wbuf, &fd);
        }
        if (!sync.barrier()) return false;
        for (int it = blockIdx.x; it < nslab; it += gridDim.x) {
            const int j0 = it * rows;
            plane_slab<VT>(Z2, out, S, (const VT*)fd.Ut[1], (const VT*)fd.Ut[0], m0, m1, 0, j0,
                           min(rows, m1 - j0), wbuf);
        }
        return true;
    }
    // A: planes of Z -> Z2
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int p = it / nslab, j0 = (it - p * nslab) * rows;
        plane_slab<VT>(Z, Z2, nullptr, (const VT*)fd.U[1], (const VT*)fd.U[0], m0, m1, p, j0,
                       min(rows, m1 - j0), wbuf);
    }
    // stage U_2, U_2^T and the three lambda lists for B while waiting
    __syncthreads();
    VT* W2 = wbuf;
    VT* W2t = wbuf + m2 * m2;
    VT* l0 = W2t + m2 * m2;
    VT* l1 = l0 + m0;
    VT* l2 = l1 + m1;
    for (int t = threadIdx.x; t < m2 * m2; t += blockDim.x) {
        cp_async_ca<sizeof(VT)>(W2 + t, (const VT*)fd.U[2] + t);
        cp_async_ca<sizeof(VT)>(W2t + t, (const VT*)fd.Ut[2] + t);
    }
    for (int t = threadIdx.x; t < m0 + m1 + m2; t += blockDim.x) {
        const VT* from = t < m0 ? (const VT*)fd.lamc[0] + t
                                : (t < m0 + m1 ? (const VT*)fd.lamc[1] + (t - m0)
                                               : (const VT*)fd.lamc[2] + (t - m0 - m1));
        cp_async_ca<sizeof(VT)>(l0 + t, from);
    }
    cp_async_wait_all();
    if (!sync.barrier()) return false;
    // B: z-lines of Z2 -> Z (one warp a line, lines over all blocks' warps)
    const int gw = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const VT cM = (VT)fd.cM;
    const int plane = m0 * m1;
    for (int L = gw; L < plane; L += nw) {
        for (int k = lane; k < m2; k += 32) xs[k] = __ldcg(Z2 + L + (long long)k * plane);
        __syncwarp();
        VT y[kFdPerLane];
        fd_line_matvec(W2, xs, m2, lane, y);
        const VT li = cM + l0[L % m0] + l1[L / m0];
        __syncwarp();
#pragma unroll
        for (int t = 0; t < kFdPerLane; ++t) {
            const int o = lane + 32 * t;
            if (o < m2) xs[o] = y[t] / (li + l2[o]);
        }
        __syncwarp();
        fd_line_matvec(W2t, xs, m2, lane, y);
#pragma unroll
        for (int t = 0; t < kFdPerLane; ++t) {
            const int o = lane + 32 * t;
            if (o < m2) Z[L + (long long)o * plane] = y[t];
        }
        __syncwarp();
    }
    if (!sync.barrier()) return false;
    // C: planes of Z -> S (U_1 X U_0^T) into out
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int p = it / nslab, j0 = (it - p * nslab) * rows;
        plane_slab<VT>(Z, out, S, (const VT*)fd.Ut[1], (const VT*)fd.Ut[0], m0, m1, p, j0,
                       min(rows, m1 - j0), wbuf);
    }
    return true;
}

template <typename VT>
__global__ void __launch_bounds__(1024, 1) k_pcg_smem(SmemArgs<VT> a) {
    // AT: type of the dot products (the operator precision).  The mixed
    // path forms them in FP32 from copies of r and u scaled by 1/||b||
    // (range), with FP32 scalars; the vectors and their updates stay FP64.
    using AT = VT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* V = (double*)smem_raw;          // kSmemVecs x rcap (FP64)
    AT* R32 = (AT*)(V + kSmemVecs * a.rcap);   // sigma r
    AT* U32 = R32 + a.rcap;                 // sigma u
    VT* sq = (VT*)(U32 + a.rcap);           // 1024 (k-split partial sums)
    VT* win = sq + 1024;                    // SpMV window; the preconditioner's matrix
    VT* xsw = win + a.plan_wcap;            // per-warp line scratch (preconditioner)
    VT* xs = xsw + (threadIdx.x >> 5) * a.fd_mmax;
    const bool fd = a.fd.on;
    VT* const Zf = (VT*)a.fd.Z;
    const VT* const Sf = (const VT*)a.fd.S;
    double* const D = V;
    double* const R = V + a.rcap;
    double* const U = V + 2 * a.rcap;
    double* const W = V + 3 * a.rcap;
    double* const S = V + 4 * a.rcap;
    double* const P = V + 5 * a.rcap;
    double* const DI = V + 6 * a.rcap;
    __shared__ double bl64[4];
    __shared__ AT blt[8];
    __shared__ double res[8];
    __shared__ int shortcut;                // 1: the first update converged (estimate)
    __shared__ double sc[4];                // alpha, beta (applied), sigma
    __shared__ AT scl[4];                   // alpha, gamma (previous) in AT
    __shared__ int state;                   // 0 run, 1 converged, 2 nan, 3 iteration cap
    __shared__ unsigned long long wmbar;    // window copy completion
    GridSync sync{&a.st->bar_count[a.which], &a.st->err, a.part};
    if (threadIdx.x == 0) {
        mbar_init(&wmbar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    WinAsync wa{&wmbar, 0u, &a.st->err};
    const Op<VT>& A = a.plan.A;
    const int n = A.n;
    int s0, s1;
    block_slices(A.n_slices, s0, s1);
    const int row0 = 32 * s0, row1 = max(row0, min(32 * s1, n));
    const int nr = row1 - row0;
    const int lane = threadIdx.x & 31;
    // ---- initial residual and the norm of b
    // With the fast diagonalization the Jacobi scaling DI is unused: its
    // slot takes this block's rows of x, copied asynchronously now for the
    // update at the end (no load on the way out).
    double bbp = 0.0;
    for (int t = threadIdx.x; t < nr; t += blockDim.x) {
        if (fd) cp_async_ca<8>(DI + t, a.x + row0 + t);
        else DI[t] = a.dinv[row0 + t];
        D[t] = S[t] = P[t] = 0.0;
        if (a.r0 != nullptr) {
            R[t] = a.r0[row0 + t];
            bbp += a.bsq[row0 + t];
        }
    }
    if (a.r0 == nullptr) {      // mode 0: r = b - A x in FP64 (global gathers of x)
        const int wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
        for (int sl = s0 + wib; sl < s1; sl += nwb) {
            const long long base = A.sptr[sl];
            const int w = (int)((A.sptr[sl + 1] - base) >> 5);
            const int i = sl * 32 + lane;
            const int ir = min(i, n - 1);
            double acc = 0.0;
#pragma unroll 4
            for (int k = 0; k < w; ++k) {
                const long long e = base + 32ll * k + lane;
                acc = fma(__ldg(a.val_hi + e), a.x[A.col(e, ir)], acc);
            }
            if (i < n) {
                const double bi = a.b[i];
                R[i - row0] = bi - acc;
                bbp += bi * bi;
            }
        }
    }
    __syncthreads();
    // ---- optional proposed start: kept only if its residual is smaller
    if (a.dx0) {
        const double scx = *a.dx0_scale;
        for (int t = threadIdx.x; t < nr; t += blockDim.x) {
            const double d = scx * (double)a.dx0[row0 + t];
            D[t] = d;
            a.ul[row0 + t] = (VT)d;
        }
        if (!sync.barrier()) return;
        double vw[2] = {0.0, 0.0};
        spmv_block(a.plan, a.ul, win, sq, [&](int i, VT t) {
            const int l = i - row0;
            const double rw = R[l] - (double)t;
            W[l] = rw;
            vw[0] += rw * rw;
            vw[1] += R[l] * R[l];
        }, &wa);
        block_sum<2>(vw, bl64);
        if (!grid_exchange<2>(sync, bl64, 10, res)) return;
        const bool warm = res[0] < res[1];
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.st->ws_used = warm ? 1 : 0;
            a.st->ws_ratio = res[1] > 0.0 ? sqrt(res[0] / res[1]) : 0.0;
        }
        for (int t = threadIdx.x; t < nr; t += blockDim.x) {
            if (warm) R[t] = W[t];
            else D[t] = 0.0;
        }
        __syncthreads();
    }
    // ---- the norms of b and r0 -> sigma; convergence at the start.  With
    // the producer's per-slice sums (and its Z = S r0) every block adds them
    // in the same fixed order: no exchange, no barrier before the first
    // preconditioner pass.
    bool pre = a.npart != nullptr && fd && a.dx0 == nullptr && a.r0 != nullptr;
    double bb;
    int it = 0;
    __shared__ float nb2[2];
    if (pre) {
        // every thread adds a few slices, then an FP32 block sum in fixed
        // order (identical in every block, so every block takes the same
        // branch below)
        float v2[2] = {0.f, 0.f};
        const float2* np2 = (const float2*)a.npart;
        for (int q0 = 0; q0 < a.npart_n; q0 += 4 * (int)blockDim.x) {
            // four loads in flight, then the adds in the same order
            float2 pv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = q0 + u * blockDim.x + threadIdx.x;
                pv[u] = q < a.npart_n ? __ldcg(np2 + q) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                v2[0] += pv[u].x;
                v2[1] += pv[u].y;
            }
        }
        block_sum<2>(v2, nb2);
        pre = isfinite(nb2[0]) && isfinite(nb2[1]);   // else the FP64 norms below
    }
    if (fd && !pre)
        for (int t = threadIdx.x; t < nr; t += blockDim.x) Zf[row0 + t] = Sf[row0 + t] * (VT)R[t];
    if (pre) {
        // the sums are FP32: sigma and the relative norm in FP32 too (FP64
        // division and square root are slow on this part)
        bb = (double)nb2[0];
        if (threadIdx.x == 0) {
            const float b2 = nb2[0], r2 = nb2[1];
            sc[2] = b2 > 0.f ? (double)(1.f / sqrtf(b2)) : 1.0;
            const double rr0 = (double)(b2 > 0.f ? r2 / b2 : r2);
            sc[3] = rr0;
            state = !(rr0 == rr0) ? 2 : (rr0 <= a.tol * a.tol ? 1 : 0);
        }
        __syncthreads();
    } else {
        double rrp = 0.0;
        for (int t = threadIdx.x; t < nr; t += blockDim.x) rrp += R[t] * R[t];
        double v2[2] = {bbp, rrp};
        block_sum<2>(v2, bl64);
        if (!grid_exchange<2>(sync, bl64, 8, res)) return;
        bb = res[0];
        if (threadIdx.x == 0) {
            sc[2] = bb > 0.0 ? 1.0 / sqrt(bb) : 1.0;
            const double rr0 = bb > 0.0 ? res[1] / bb : res[1];
            sc[3] = rr0;
            state = !(rr0 == rr0) ? 2 : (rr0 <= a.tol * a.tol ? 1 : 0);
        }
        __syncthreads();
    }
    const AT sig = (AT)sc[2];
    const AT* DL = (const AT*)a.dinvl;
    // stop when (sigma r, sigma r) <= tol^2 (sigma^2 ||b||^2 = 1)
    const double stop2 = bb > 0.0 ? a.tol * a.tol : 0.0;
    for (int t = threadIdx.x; t < nr; t += blockDim.x) R32[t] = (AT)R[t] * sig;
    // u = P^{-1} r, published (Jacobi: local; fast diagonalization: passes)
    auto precondition = [&]() -> bool {
        if (fd) {
            if (a.fd_rows > 0) {
                if (!fd_apply_planes<VT>(a.fd, sync, win, xs, a.ul, a.fd_rows)) return false;
            } else if (!fd_apply<VT>(a.fd, sync, win, xs, a.ul, a.fd_w2 != 0)) {
                return false;
            }
            if (!sync.barrier()) return false;
            for (int t = threadIdx.x; t < nr; t += blockDim.x) {
                const VT u = __ldcg(a.ul + row0 + t);
                U[t] = (double)u;
                U32[t] = (AT)u * sig;
            }
        }
        return true;
    };
    if (!fd)
        for (int t = threadIdx.x; t < nr; t += blockDim.x) {
            const double u = DI[t] * R[t];
            U[t] = u;
            U32[t] = DL[row0 + t] * R32[t];
            a.ul[row0 + t] = (VT)u;
        }
    if (state == 0) {
        if (!fd && !sync.barrier()) return;
        if (!precondition()) return;
    }
    while (state == 0) {
        // ---- S: w = A u and (r, u), (w, u)
        // at the first iteration also (e, e), (e, w), (w, w) with e = r - w
        // (scaled like r): the residual after the first update is
        // r - al w = e + (1 - al) w, whose norm they give without
        // cancellation when the preconditioner is nearly the inverse (al
        // close to 1, e small), so a converged first update needs no
        // exchange of its own
        const bool first = it == 0;
        AT v[5] = {(AT)0, (AT)0, (AT)0, (AT)0, (AT)0};
        spmv_block(a.plan, a.ul, win, sq, [&](int i, VT wt) {
            const int l = i - row0;
            W[l] = (double)wt;
            const AT w32 = (AT)wt * sig;
            v[0] += R32[l] * U32[l];
            v[1] += w32 * U32[l];
            if (first) {
                const AT e32 = (AT)(R[l] - (double)wt) * sig;
                v[2] += e32 * e32;
                v[3] += e32 * w32;
                v[4] += w32 * w32;
            }
        }, &wa);
        // partial slots: warm start 10-11, norms 8-9, the first S 0-4, then
        // V 6 / 2 and S 4-5 / 0-1 alternating (a slot set is rewritten only
        // two barriers later)
        if (first) {
            block_sum<5>(v, blt);
            if (!grid_exchange<5>(sync, blt, 0, res)) return;
        } else {
            AT v2[2] = {v[0], v[1]};
            block_sum<2>(v2, blt);
            if (!grid_exchange<2>(sync, blt, 4 * (it & 1), res)) return;
        }
        if (threadIdx.x == 0) {
            const AT gamma = (AT)res[0], delta = (AT)res[1];
            AT be = (AT)0, al = gamma / delta;
            if (it > 0) {
                be = gamma / scl[1];
                al = gamma / (delta - be * gamma / scl[0]);
            }
            scl[0] = al;
            scl[1] = gamma;
            sc[0] = (double)al;
            sc[1] = (double)be;
            state = !(al == al) ? 2 : 0;
            shortcut = 0;
            if (first && state == 0) {
                // |(sigma r1, sigma r1) - est| <= bound: sums of one rounding
                // per product over a tree of depth ~24, with margin (the
                // Cauchy-Schwarz factor sqrt(ee) sqrt(ww) in FP32: each root
                // stays normal down to 1e-38, far below any stopping level;
                // FP64 square roots are slow on this part)
                const double om = 1.0 - (double)al;
                const double ee = res[2], ew = res[3], ww = res[4];
                const double est = ee + 2.0 * om * ew + om * om * ww;
                const double bound = 64.0 * (sizeof(AT) == 4 ? 5.9604644775390625e-8 : 1.1102230246251565e-16) *
                                     (ee + 2.0 * fabs(om) * (double)sqrtf((float)ee) *
                                               (double)sqrtf((float)ww) + om * om * ww);
                if (est + bound <= stop2) {
                    shortcut = 1;
                    sc[3] = est > 0.0 ? est : 0.0;
                }
            }
        }
        __syncthreads();
        if (state != 0) break;
        const double al = sc[0], be = sc[1];
        if (shortcut) {
            // converged by the estimate: only the step (p = u, beta = 0 at
            // the first update) goes on to x
            for (int t = threadIdx.x; t < nr; t += blockDim.x) D[t] = fma(al, U[t], D[t]);
            ++it;
            if (threadIdx.x == 0) state = 1;
            __syncthreads();
            break;
        }
        // ---- V: own rows; (r, r) of the update
        AT vr[1] = {(AT)0};
        for (int t = threadIdx.x; t < nr; t += blockDim.x) {
            const double p = fma(be, P[t], U[t]);
            const double s = fma(be, S[t], W[t]);
            P[t] = p;
            S[t] = s;
            D[t] = fma(al, p, D[t]);
            const double r = fma(-al, s, R[t]);
            const AT r32 = (AT)r * sig;
            R[t] = r;
            R32[t] = r32;
            vr[0] += r32 * r32;
            if (fd) {
                Zf[row0 + t] = Sf[row0 + t] * (VT)r;   // the next application's input
            } else {
                const double u = DI[t] * r;
                U[t] = u;
                U32[t] = DL[row0 + t] * r32;
                a.ul[row0 + t] = (VT)u;
            }
        }
        ++it;
        block_sum<1>(vr, blt);
        if (!grid_exchange<1>(sync, blt, 2 + 4 * (it & 1), res)) return;
        if (threadIdx.x == 0) {
            const double rr = res[0];
            sc[3] = rr;
            state = !(rr == rr) ? 2 : (rr <= stop2 ? 1 : (it >= a.max_iter ? 3 : 0));
        }
        __syncthreads();
        if (state != 0) break;
        if (!precondition()) return;
    }
    // the step's finalize inputs (one per thread when the grid covers them)
    // in flight together with the last reads of x
    const int fi = blockIdx.x * blockDim.x + threadIdx.x;
    double f1v = 0.0, gv = 0.0;
    if (a.fin_F1 && fi < a.fin_n_dof) {
        f1v = __ldcg(a.fin_F1 + fi);
        if (fi < a.fin_n_dir) gv = __ldcg(a.fin_g + fi);
    }
    if (fd) cp_async_wait_all();   // this thread's rows of x in DI
    for (int t = threadIdx.x; t < nr; t += blockDim.x) {
        const double xn = (fd ? DI[t] : a.x[row0 + t]) + D[t];
        a.x[row0 + t] = xn;
        if (a.dir_out) {
            a.dir_out[row0 + t] = (VT)(xn - a.dir_old[row0 + t]);
            a.dir_out[n + row0 + t] = (VT)xn;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double rel = sqrt(sc[3]);      // (sigma r, sigma r) = ||r||^2 / ||b||^2
        int* err = &a.st->err;
        if (a.which == 0) {
            a.st->pcg_iters = it;
            a.st->rel_res = rel;
            if (state != 1) atomicOr(err, SA_DEV_NOT_CONVERGED);
        } else {
            a.st->bot_iters = it;
            a.st->bot_rel_res = rel;
            if (state != 1) atomicOr(err, SA_DEV_BOT_NOT_CONVERGED);
        }
        if (state == 2) atomicOr(err, SA_DEV_NAN);
        if (a.fin_F1) {   // the step's counters (after this solve's own)
            a.st->n += 1;
            a.st->iters_total += a.st->pcg_iters;
            a.st->bot_total += a.st->bot_iters;
            if (a.st->pcg_iters > a.st->iters_max) a.st->iters_max = a.st->pcg_iters;
        }
    }
    if (a.fin_F1) {
        // the step's end (what k_finalize does otherwise): the Dirichlet
        // control variables take g^{n+1}, F^n <- F^{n+1}; no kernel of its own
        for (int i = fi; i < a.fin_n_dof; i += gridDim.x * blockDim.x) {
            a.fin_F0[i] = i == fi ? f1v : __ldcg(a.fin_F1 + i);
            if (i < a.fin_n_dir) a.fin_That[n + i] = i == fi ? gv : __ldcg(a.fin_g + i);
        }
    }
}

__global__ void k_extrap(int n_free, int n_dir, const double* That, double* Tprev, float* dx0,
                         double* gprev, double* g0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_free) {
        const double t = That[i];
        dx0[i] = (float)(t - Tprev[i]);
        Tprev[i] = t;
    } else if (i < n_free + n_dir) {
        const int d = i - n_free;
        const double g = That[i];
        g0[d] = 2.0 * g - gprev[d];
        gprev[d] = g;
    }
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
    o.hi = s.hi;
    o.val = (const VT*)val;
    return o;
}

// Launch shape shared by both variants: slices per block -> warps per slice
// (so the 32 warps of a block are busy), window length, shared memory.
template <typename VT>
struct PcgShape {
    int G, block, spb, ks, rcap, fd_mmax, fd_w2;
    long long wl, region;
    bool window;
    size_t smem;
    bool fits;             // (shared-memory variant) vectors + k-split scratch fit
};

constexpr size_t kSmemCap = 200 * 1024;

// Plane form of the preconditioner (3-D: planes over the blocks in slabs;
// 2-D: the one plane in slabs): rows per slab, and the shared entries it
// stages (a plane, the two m x m matrices, a slab); 0 rows: the line form.
inline int plane_slab_rows(const FdView& fd, int G) {
    if (!fd.on || fd.Z2 == nullptr || (fd.nd != 2 && fd.nd != 3)) return 0;
    const int m1 = fd.m[1], m2 = fd.nd == 3 ? fd.m[2] : 1;
    if (m2 > 32 * kFdPerLane) return 0;
    const int nslab = std::max(1, G / std::max(m2, 1));
    return (m1 + nslab - 1) / nslab;
}
inline long long plane_slab_need(const FdView& fd, int rows) {
    const long long m0 = fd.m[0], m1 = fd.m[1], m2 = fd.nd == 3 ? fd.m[2] : 1;
    // a slab's staging, or the z-line pass's (U_2, U_2^T, the three lambda lists)
    return std::max(plane_stage_entries((int)m0, (int)m1, rows), 2 * m2 * m2 + m0 + m1 + m2);
}

template <typename VT>
PcgShape<VT> pcg_shape(const PcgLaunch& L, bool pipelined) {
    PcgShape<VT> sh;
    sh.G = L.grid > 0 ? L.grid : 1;
    sh.block = L.block > 0 ? L.block : kPcgBlock;
    sh.spb = (L.op.n_slices + sh.G - 1) / sh.G;
    const int warps = sh.block / 32;
    int ks = 1;
    while (ks < 8 && ks * 2 <= warps && sh.spb * ks * 2 <= warps) ks *= 2;
    sh.ks = L.ksplit > 0 ? L.ksplit : ks;
    sh.rcap = 32 * std::max(sh.spb, 1);
    // window: 32 spb rows plus the halo, 4-entry alignment slack
    sh.wl = 32ll * sh.spb + (L.op.dmax - L.op.dmin) + 8;
    // the preconditioner's m x m matrix reuses the window region
    const int mmax = (pipelined && L.fd.on) ? std::max(L.fd.m[0], std::max(L.fd.m[1], L.fd.m[2])) : 0;
    long long fdw = 2ll * mmax * mmax;   // two staged matrices (three when they fit)
    sh.fd_mmax = mmax;
    const size_t fixed = 1024 * sizeof(VT) +
                         (pipelined ? (size_t)kSmemVecs * sh.rcap * sizeof(double) + 2 * sh.rcap * sizeof(VT) +
                                          (size_t)32 * mmax * sizeof(VT)
                                    : 0);
    sh.fits = fixed + fdw * sizeof(VT) <= kSmemCap;
    sh.fd_w2 = 0;
    if (mmax > 0 && fixed + 3ll * mmax * mmax * sizeof(VT) <= kSmemCap) {
        fdw = 3ll * mmax * mmax;
        sh.fd_w2 = 1;
    }
    // the plane form's staging, when it fits
    const int prows = pipelined ? plane_slab_rows(L.fd, sh.G) : 0;
    if (prows > 0) {
        const long long need = plane_slab_need(L.fd, prows);
        if (fixed + need * sizeof(VT) <= kSmemCap) fdw = std::max(fdw, need);
    }
    sh.window = L.op.col16 != nullptr && L.pad >= -L.op.dmin + 4 && L.pad >= L.op.dmax + 4 &&
                fixed + std::max(sh.wl, fdw) * sizeof(VT) <= kSmemCap;
    sh.region = sh.window ? std::max(sh.wl, fdw) : fdw;
    sh.smem = fixed + (size_t)sh.region * sizeof(VT);
    return sh;
}

template <typename VT>
int plane_rows(const PcgLaunch& L, const PcgShape<VT>& sh) {
    const int rows = plane_slab_rows(L.fd, sh.G);
    return rows > 0 && plane_slab_need(L.fd, rows) <= sh.region ? rows : 0;
}

cudaError_t launch_coop(const void* fn, int G, int block, size_t smem, void* args, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* params[1] = {args};
    return cudaLaunchCooperativeKernel(fn, dim3(G), dim3(block), params, smem, s);
}

template <typename VT>
cudaError_t launch_pcg_t(const PcgLaunch& L, cudaStream_t s) {
    const bool want_pipe = L.variant != SA_PCG_GLOBAL;
    if (want_pipe) {
        const PcgShape<VT> sh = pcg_shape<VT>(L, true);
        if (sh.fits) {
            SmemArgs<VT> a;
            a.plan = SpmvPlan<VT>{make_op<VT>(L.op, L.val), L.op.dmin, L.op.dmax, sh.window, sh.ks};
            a.rcap = sh.rcap;
            a.val_hi = L.val_hi;
            a.dinv = L.dinv;
            a.b = L.b;
            a.r0 = L.r0;
            a.bsq = L.bsq;
            a.x = L.x;
            a.ul = (VT*)L.vpad + L.pad;
            a.part = L.partials;
            a.st = L.st;
            a.which = L.which;
            a.tol = L.tol;
            a.max_iter = L.max_iter;
            a.dx0 = L.dx0;
            a.dx0_scale = L.dx0_scale;
            a.dinvl = L.dinvl;
            a.fd = L.fd;
            a.fd_mmax = sh.fd_mmax;
            a.plan_wcap = (int)sh.region;
            a.dir_old = L.dir_old;
            a.dir_out = (VT*)L.dir_out;
            a.fd_w2 = sh.fd_w2;
            a.npart = L.npart;
            a.npart_n = L.npart_n;
            a.fin_F1 = L.fin_F1;
            a.fin_F0 = L.fin_F0;
            a.fin_g = L.fin_g;
            a.fin_That = L.fin_That;
            a.fin_n_dof = L.fin_n_dof;
            a.fin_n_dir = L.fin_n_dir;
            // 3-D: the plane form when its staging fits the shared region
            a.fd_rows = plane_rows(L, sh);
            return launch_coop((const void*)k_pcg_smem<VT>, sh.G, sh.block, sh.smem, &a, s);
        }
        if (L.variant == SA_PCG_SHARED) return cudaErrorInvalidConfiguration;
    }
    const PcgShape<VT> sh = pcg_shape<VT>(L, false);
    PcgArgs<VT> a;
    a.A = make_op<VT>(L.op, L.val);
    a.dmin = L.op.dmin;
    a.dmax = L.op.dmax;
    a.val_hi = L.val_hi;
    a.dinv = L.dinv;
    a.b = L.b;
    a.r0 = L.r0;
    a.bsq = L.bsq;
    a.x = L.x;
    a.p = L.w64;
    a.r = L.w64 + L.stride;
    a.w = L.w64 + 2 * L.stride;
    a.s = L.w64 + 3 * L.stride;
    a.u = L.w64 + 4 * L.stride;
    a.ul = (VT*)L.vpad + L.pad;
    a.part = L.partials;
    a.st = L.st;
    a.which = L.which;
    a.tol = L.tol;
    a.max_iter = L.max_iter;
    a.dx0 = L.dx0;
    a.dx0_scale = L.dx0_scale;
    a.ksplit = sh.ks;
    a.window = sh.window;
    a.wcap = sh.window ? (int)sh.wl : 0;
    return launch_coop((const void*)k_pcg<VT>, sh.G, sh.block, sh.smem, &a, s);
}

// ---------------------------------------------------------------------------
// warm start / training-data recorder helpers
// ---------------------------------------------------------------------------
// ||r0||_2 over n entries: per-block partials then one block in fixed order.
__global__ void k_norm_part(int n, const double* r, double* part) {
    __shared__ double sh[256];
    double t = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        t += r[i] * r[i];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_norm_final(int nb, const double* part, double* norm) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double t = 0.0;
    for (int i = 0; i < nb; ++i) t += part[i];
    *norm = sqrt(t);
}

// x_in[k] = r0[idx[k]] / ||r0|| as BF16 (recorder: appended at row `slot`)
__global__ void k_ws_input(int n_in, const int* idx, const double* r0, const double* norm,
                           __nv_bfloat16* out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_in) return;
    const double nr = *norm;
    out[k] = __float2bfloat16(nr > 0.0 ? (float)(r0[idx[k]] / nr) : 0.f);
}

// y = (x_new - x_old) / ||r0|| as BF16
__global__ void k_ws_target(int n, const double* xnew, const double* xold, const double* norm,
                            __nv_bfloat16* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double nr = *norm;
    out[i] = __float2bfloat16(nr > 0.0 ? (float)((xnew[i] - xold[i]) / nr) : 0.f);
}

}  // namespace

cudaError_t launch_norm(int n, const double* r, double* part, double* norm, cudaStream_t s) {
    k_norm_part<<<64, 256, 0, s>>>(n, r, part);
    k_norm_final<<<1, 32, 0, s>>>(64, part, norm);
    return cudaGetLastError();
}

cudaError_t launch_ws_input(int n_in, const int* idx, const double* r0, const double* norm,
                            void* out, cudaStream_t s) {
    if (n_in == 0) return cudaSuccess;
    k_ws_input<<<(n_in + 255) / 256, 256, 0, s>>>(n_in, idx, r0, norm, (__nv_bfloat16*)out);
    return cudaGetLastError();
}

cudaError_t launch_ws_target(int n, const double* xnew, const double* xold, const double* norm,
                             void* out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_ws_target<<<(n + 255) / 256, 256, 0, s>>>(n, xnew, xold, norm, (__nv_bfloat16*)out);
    return cudaGetLastError();
}

cudaError_t launch_gather(int wlat_rows, const int* wlat_rowdof, const int* wlat_ptr,
                          const int* wlat_col, const double* wlat_val, const double* s_lat,
                          double k, int n_dir, const int* wbot_ptr, const int* wbot_col,
                          const double* wbot_val, const double* tt_bot, double Tc, double* F1,
                          double* bbot, int n_dof, const double* That, double* dev64,
                          float* dev32, cudaStream_t s, int part, const BotResid& br,
                          DevStatus* st) {
    GatherArgs a{wlat_rows, wlat_rowdof, wlat_ptr, wlat_col, wlat_val, s_lat, k, n_dir,
                 wbot_ptr, wbot_col, wbot_val, tt_bot, Tc, F1, bbot, n_dof, That, dev64, dev32,
                 part, br, st};
    const long long threads = part == 1   ? gather_range(wlat_rows) + n_dof
                              : part == 2 ? gather_range(n_dir)
                                          : gather_range(wlat_rows) + gather_range(n_dir) + n_dof;
    if (threads == 0) return cudaSuccess;
    k_gather<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_theta_rhs(int precision, const SellView& op, const void* Kval,
                             const void* Mval, const void* dev, const double* That,
                             const double* gnew, const double* F0, const double* F1,
                             double inv_dt_rhocp, double k, double theta, double Tc, double* r0,
                             double* bsq, int n_dir, void* dir_scratch, cudaStream_t s, int only,
                             bool dir_ready, const void* fdS, void* fdZ, float* npart,
                             const short* col16lo, const unsigned short* M16, int sl0, int sl1) {
    if (op.n == 0) return cudaSuccess;
    // Dirichlet increments for the flagged slices (unless the projection wrote them)
    const bool prep = only != 1 && n_dir > 0 && !dir_ready;
    // the Dirichlet-column slices alone: one slice a block, eight warps on it
    const int split = only == 2 ? 8 : 4;
    sl0 = std::max(0, sl0);
    sl1 = sl1 < 0 ? op.n_slices : std::min(sl1, op.n_slices);
    if (sl1 <= sl0) return cudaSuccess;
    const unsigned blocks = (unsigned)((sl1 - sl0 + (8 / split) - 1) / (8 / split));
    const unsigned pblocks = (unsigned)((n_dir + 255) / 256);
    if (precision == SA_MIXED) {
        float* dg = (float*)dir_scratch;
        float* g1 = dg + n_dir;
        if (prep) k_dir_prep<float><<<pblocks, 256, 0, s>>>(n_dir, op.n, That, gnew, dg, g1);
        RhsArgs<float> a{make_op<float>(op, Kval), (const float*)Mval, (const float*)dev, dg, g1,
                         F0, F1, op.n, inv_dt_rhocp, k, theta, Tc, r0, bsq, only,
                         (const float*)fdS, (float*)fdZ, npart, col16lo, M16, sl0, sl1};
        if (split == 8)
            k_theta_rhs<8, float><<<blocks, 256, 0, s>>>(a);
        else
            k_theta_rhs<4, float><<<blocks, 256, 0, s>>>(a);
    } else {
        double* dg = (double*)dir_scratch;
        double* g1 = dg + n_dir;
        if (prep) k_dir_prep<double><<<pblocks, 256, 0, s>>>(n_dir, op.n, That, gnew, dg, g1);
        RhsArgs<double> a{make_op<double>(op, Kval), (const double*)Mval, (const double*)dev, dg,
                          g1, F0, F1, op.n, inv_dt_rhocp, k, theta, Tc, r0, bsq, only,
                          (const double*)fdS, (double*)fdZ, npart, nullptr, nullptr, sl0, sl1};
        if (split == 8)
            k_theta_rhs<8, double><<<blocks, 256, 0, s>>>(a);
        else
            k_theta_rhs<4, double><<<blocks, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

int pcg_block_size() { return kPcgBlock; }
const void* pcg_kernel_ptr(int precision) {
    return precision == SA_MIXED ? (const void*)k_pcg<float> : (const void*)k_pcg<double>;
}

cudaError_t launch_pcg(int precision, const PcgLaunch& L, cudaStream_t s) {
    if (L.op.n == 0) return cudaSuccess;
    return precision == SA_MIXED ? launch_pcg_t<float>(L, s) : launch_pcg_t<double>(L, s);
}

cudaError_t launch_extrap(int n_free, int n_dir, const double* That, double* Tprev, float* dx0,
                          double* gprev, double* g0, cudaStream_t s) {
    const int n = n_free + n_dir;
    if (n == 0) return cudaSuccess;
    k_extrap<<<(n + 255) / 256, 256, 0, s>>>(n_free, n_dir, That, Tprev, dx0, gprev, g0);
    return cudaGetLastError();
}

bool pcg_shared_fits(int precision, const PcgLaunch& L) {
    return precision == SA_MIXED ? pcg_shape<float>(L, true).fits : pcg_shape<double>(L, true).fits;
}

cudaError_t launch_finalize(int n_dir, int n_free, int n_dof, const double* gnew, double* That,
                            const double* F1, double* F0, DevStatus* st, cudaStream_t s) {
    const int nmax = n_dof > 1 ? n_dof : 1;
    k_finalize<<<(nmax + 255) / 256, 256, 0, s>>>(n_dir, n_free, n_dof, gnew, That, F1, F0, st);
    return cudaGetLastError();
}
