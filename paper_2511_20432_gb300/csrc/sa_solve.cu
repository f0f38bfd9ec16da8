// Per-step solver kernels: boundary integrals of the point-source data
// (Section 2.3, F_i = int_lat (-q_N) N_i dS; the bottom projection), the
// theta-scheme right-hand side (Eq. theta-method) and a persistent
// cooperative Jacobi-PCG in FP64.
#include <cooperative_groups.h>

#include "sa_internal.h"

namespace {

// ---------------------------------------------------------------------------
// F^{n+1} = W_lat (-k dT~/dn)  and  b_bot = W_bot (T_c - T~): one warp per
// row of the constant weight matrices, fixed order, no atomics.
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
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void k_gather(GatherArgs a) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row < a.wlat_rows) {
        double acc = 0.0;
        for (int s = a.lptr[row] + lane; s < a.lptr[row + 1]; s += 32)
            acc += a.lval[s] * a.s_lat[a.lcol[s]];
        acc = warp_sum(acc);
        if (lane == 0) a.F1[a.rowdof[row]] = -a.k * acc;
    } else if (row < a.wlat_rows + a.n_dir) {
        const int r = row - a.wlat_rows;
        double acc = 0.0;
        for (int s = a.bptr[r] + lane; s < a.bptr[r + 1]; s += 32)
            acc += a.bval[s] * (a.Tc - a.tt_bot[a.bcol[s]]);
        acc = warp_sum(acc);
        if (lane == 0) a.bbot[r] = acc;
    }
}

// ---------------------------------------------------------------------------
// theta right-hand side on the free rows, with the Dirichlet values lifted:
//   b = (M/dt)(T^n - G) - K((1-theta) T^n + theta G) + theta F^{n+1}
//       + (1-theta) F^n,    G = g^{n+1} on Dirichlet columns, 0 elsewhere,
// which equals (M/dt - (1-theta)K) T^n + theta F^{n+1} + (1-theta) F^n
// - (M/dt + theta K)_{fd} g^{n+1}; and in the same pass the initial PCG
// residual r0 = b - A_ff T^n_f.  One warp per free row.
// ---------------------------------------------------------------------------
struct RhsArgs {
    int n_free;
    int n_slices;
    const long long* sptr;
    const int* col;            // internal column indices
    const double* M;           // unit rho c_p
    const double* K;           // unit k
    const double* That;
    const double* gnew;
    const double* F0;
    const double* F1;
    double inv_dt, kscale, theta;
    double* rhs;
    double* r0;
};

// One warp per 32-row slice, lane = free row (SELL storage).
__global__ void k_theta_rhs(RhsArgs a) {
    const int sl = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (sl >= a.n_slices) return;
    const int i = sl * 32 + lane;
    const long long base = a.sptr[sl];
    const int w = (int)((a.sptr[sl + 1] - base) >> 5);
    double accb = 0.0, acca = 0.0;
#pragma unroll 4
    for (int k = 0; k < w; ++k) {
        const long long e = base + 32ll * k + lane;
        const int j = __ldg(a.col + e);
        const double m = __ldg(a.M + e) * a.inv_dt, kk = __ldg(a.K + e) * a.kscale;
        const double T = a.That[j];
        if (j < a.n_free) {
            accb += m * T - kk * ((1.0 - a.theta) * T);
            acca += (m + a.theta * kk) * T;
        } else {
            const double G = a.gnew[j - a.n_free];
            accb += m * (T - G) - kk * ((1.0 - a.theta) * T + a.theta * G);
        }
    }
    if (i < a.n_free) {
        const double b = accb + a.theta * a.F1[i] + (1.0 - a.theta) * a.F0[i];
        a.rhs[i] = b;
        a.r0[i] = b - acca;
    }
}

// ---------------------------------------------------------------------------
// grid barrier with a bounded wait (co-residency is guaranteed by the
// cooperative launch; a wait that exceeds the limit flags SA_DEV_TIMEOUT and
// the kernel returns instead of hanging)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ bool grid_barrier(unsigned* count, unsigned* gen, int* err) {
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
                }
                if (*((volatile int*)err) & SA_DEV_TIMEOUT) {
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Deterministic block reduction of NV values per thread; thread 0 gets the
// sums in out[] (fixed xor-tree within warps, fixed warp order).
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
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = 0.0;
            for (int ww = 0; ww < nw; ++ww) t += sred[k][ww];
            out[k] = t;
        }
    __syncthreads();
}

// Sum of part[0..G) identical in every block (fixed order), broadcast to
// all threads of the block.
__device__ double grid_total(const double* part) {
    __shared__ double res;
    if (threadIdx.x < 32) {
        double t = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) t += ((volatile const double*)part)[i];
        t = warp_sum(t);
        if (threadIdx.x == 0) res = t;
    }
    __syncthreads();
    const double r = res;
    __syncthreads();
    return r;
}

struct PcgArgs {
    int n;
    int n_slices;
    const long long* sptr;     // SELL operator
    const int* col;
    const double* val;
    const double* dinv;
    const double* b;
    const double* r0;      // optional initial residual (x0 = x)
    double* x;
    double* r;
    double* z;
    double* p0;
    double* p1;
    double* q;
    double* part;          // 6 * gridDim.x
    DevStatus* st;
    int which;             // 0 main solve, 1 bottom projection
    double tol;
    int max_iter;
};

// Jacobi-preconditioned CG (Hestenes-Stiefel) in FP64.  The update of the
// search direction p = z + beta p is fused into the next SpMV (p double
// buffered), so one iteration is two grid phases:
//   B: p' = z + beta p ; q = A p' ; (p', q)
//   C: x += alpha p' ; r -= alpha q ; z = D^{-1} r ; (r, r), (r, z)
// SpMV: SELL-32, one warp per slice (lane = row), slices grid-strided over
// the warps; the k loop is unrolled so each lane keeps several independent
// coalesced loads in flight.
__global__ void __launch_bounds__(512) k_pcg(PcgArgs a) {
    const int n = a.n;
    const int G = gridDim.x;
    const int lane = threadIdx.x & 31;
    const int nwb = blockDim.x >> 5;
    const int gw = blockIdx.x * nwb + (threadIdx.x >> 5);
    const int nw = G * nwb;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = G * blockDim.x;
    unsigned* bc = &a.st->bar_count[a.which];
    unsigned* bg = &a.st->bar_gen[a.which];
    int* err = &a.st->err;
    __shared__ double red[3];

    // ---- phase A: r = b - A x (or given), z = D^{-1} r, (r,z), (r,r), (b,b)
    {
        double v[3] = {0.0, 0.0, 0.0};
        if (a.r0 == nullptr) {
            for (int sl = gw; sl < a.n_slices; sl += nw) {
                const long long base = a.sptr[sl];
                const int w = (int)((a.sptr[sl + 1] - base) >> 5);
                double acc = 0.0;
#pragma unroll 8
                for (int k = 0; k < w; ++k) {
                    const long long e = base + 32ll * k + lane;
                    acc = fma(__ldg(a.val + e), a.x[__ldg(a.col + e)], acc);
                }
                const int i = sl * 32 + lane;
                if (i < n) {
                    const double ri = a.b[i] - acc;
                    const double zi = a.dinv[i] * ri;
                    a.r[i] = ri;
                    a.z[i] = zi;
                    v[0] += ri * zi;
                    v[1] += ri * ri;
                    v[2] += a.b[i] * a.b[i];
                }
            }
        } else {
            for (int i = tid; i < n; i += nth) {
                const double ri = a.r0[i];
                const double zi = a.dinv[i] * ri;
                a.r[i] = ri;
                a.z[i] = zi;
                v[0] += ri * zi;
                v[1] += ri * ri;
                v[2] += a.b[i] * a.b[i];
            }
        }
        block_reduce<3>(v, red);
        if (threadIdx.x == 0) {
            a.part[0 * G + blockIdx.x] = red[0];
            a.part[1 * G + blockIdx.x] = red[1];
            a.part[2 * G + blockIdx.x] = red[2];
        }
    }
    if (!grid_barrier(bc, bg, err)) return;
    double rz = grid_total(a.part + 0 * G);
    double rr = grid_total(a.part + 1 * G);
    const double bb = grid_total(a.part + 2 * G);
    const double stop2 = a.tol * a.tol * bb;
    int it = 0;
    double beta = 0.0;
    bool conv = rr <= stop2;
    double* pc = a.p0;
    double* pn = a.p1;
    bool nan = !(rr == rr);
    while (!conv && !nan && it < a.max_iter) {
        // ---- phase B
        {
            double v[1] = {0.0};
            const bool first = (it == 0);
            for (int sl = gw; sl < a.n_slices; sl += nw) {
                const long long base = a.sptr[sl];
                const int w = (int)((a.sptr[sl + 1] - base) >> 5);
                double acc = 0.0;
                if (first) {
#pragma unroll 8
                    for (int k = 0; k < w; ++k) {
                        const long long e = base + 32ll * k + lane;
                        acc = fma(__ldg(a.val + e), a.z[__ldg(a.col + e)], acc);
                    }
                } else {
#pragma unroll 8
                    for (int k = 0; k < w; ++k) {
                        const long long e = base + 32ll * k + lane;
                        const int j = __ldg(a.col + e);
                        acc = fma(__ldg(a.val + e), fma(beta, pc[j], a.z[j]), acc);
                    }
                }
                const int i = sl * 32 + lane;
                if (i < n) {
                    const double pi = first ? a.z[i] : fma(beta, pc[i], a.z[i]);
                    pn[i] = pi;
                    a.q[i] = acc;
                    v[0] += pi * acc;
                }
            }
            block_reduce<1>(v, red);
            if (threadIdx.x == 0) a.part[3 * G + blockIdx.x] = red[0];
        }
        if (!grid_barrier(bc, bg, err)) return;
        const double pq = grid_total(a.part + 3 * G);
        const double alpha = rz / pq;
        // ---- phase C
        {
            double v[2] = {0.0, 0.0};
            for (int i = tid; i < n; i += nth) {
                a.x[i] += alpha * pn[i];
                const double ri = a.r[i] - alpha * a.q[i];
                const double zi = a.dinv[i] * ri;
                a.r[i] = ri;
                a.z[i] = zi;
                v[0] += ri * ri;
                v[1] += ri * zi;
            }
            block_reduce<2>(v, red);
            if (threadIdx.x == 0) {
                a.part[4 * G + blockIdx.x] = red[0];
                a.part[5 * G + blockIdx.x] = red[1];
            }
        }
        if (!grid_barrier(bc, bg, err)) return;
        rr = grid_total(a.part + 4 * G);
        const double rzn = grid_total(a.part + 5 * G);
        ++it;
        nan = !(rr == rr) || !(pq == pq);
        conv = rr <= stop2;
        beta = rzn / rz;
        rz = rzn;
        double* t = pc;
        pc = pn;
        pn = t;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double rel = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
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

}  // namespace

cudaError_t launch_gather(int wlat_rows, const int* wlat_rowdof, const int* wlat_ptr,
                          const int* wlat_col, const double* wlat_val, const double* s_lat,
                          double k, int n_dir, const int* wbot_ptr, const int* wbot_col,
                          const double* wbot_val, const double* tt_bot, double Tc, double* F1,
                          double* bbot, cudaStream_t s) {
    GatherArgs a{wlat_rows, wlat_rowdof, wlat_ptr, wlat_col, wlat_val, s_lat, k, n_dir,
                 wbot_ptr, wbot_col, wbot_val, tt_bot, Tc, F1, bbot};
    const long long rows = (long long)wlat_rows + n_dir;
    if (rows == 0) return cudaSuccess;
    k_gather<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_theta_rhs(int n_free, int n_slices, const long long* sptr, const int* col,
                             const double* M, const double* K, const double* That,
                             const double* gnew, const double* F0, const double* F1,
                             double inv_dt, double kscale, double theta, double* rhs,
                             double* r0, cudaStream_t s) {
    RhsArgs a{n_free, n_slices, sptr, col, M, K, That, gnew, F0, F1, inv_dt, kscale, theta, rhs,
              r0};
    if (n_free == 0) return cudaSuccess;
    k_theta_rhs<<<(unsigned)(((long long)n_slices * 32 + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

int pcg_block_size() { return 512; }
const void* pcg_kernel_ptr() { return (const void*)k_pcg; }

cudaError_t launch_pcg(int which, int n, int n_slices, const long long* sptr, const int* col,
                       const double* val, const double* dinv, const double* b,
                       const double* r0_or_null, double* x, double* r, double* z, double* p0,
                       double* p1, double* q, double* partials, DevStatus* st, double tol,
                       int max_iter, int grid, int block, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    PcgArgs a{n, n_slices, sptr, col, val, dinv, b, r0_or_null, x, r, z, p0, p1, q, partials, st,
              which, tol, max_iter};
    cudaError_t e = cudaMemsetAsync(&st->bar_count[which], 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_pcg, a);
}

cudaError_t launch_finalize(int n_dir, int n_free, int n_dof, const double* gnew, double* That,
                            const double* F1, double* F0, DevStatus* st, cudaStream_t s) {
    const int nmax = n_dof > 1 ? n_dof : 1;
    k_finalize<<<(nmax + 255) / 256, 256, 0, s>>>(n_dir, n_free, n_dof, gnew, That, F1, F0, st);
    return cudaGetLastError();
}
