// Per-step history sums of the analytical point-source field (Section 2.1,
// Eqs. sum-of-point-temp and semi-temperature) at the boundary quadrature
// points:
//   lateral points:  dT~/dn(x_q) = sum_I -g_I exp(-a_I R^2) (n_q . (x_q - x_I))
//   bottom points:   T~(x_q)     = sum_I  c_I exp(-a_I R^2)
// with, for source I at step n, age = (n - I) dt + r^2/(8 alpha),
// a_I = 1/(4 alpha age), c_I = s_img E / (rho c_p (4 pi alpha age)^{3/2}),
// g_I = 2 a_I c_I (the gradient of the Gaussian brings down
// -(x - x_I)/(2 alpha age) = -2 a_I (x - x_I)).
//
// The per-step prologue forms these coefficients once per source in FP64
// from the integer step difference.  The sum kernel is ALU-bound (FP32 FMA
// pipe + MUFU ex2 in the mixed path, the FP64 pipe in the plain path); it is
// not a contraction, so it does not use tensor cores.
//
// Work layout: one CTA owns a tile of 32*P points (P per lane, held in
// registers) and all of its NW warps split the active sources round-robin.
// Mixed path: the source table streams through shared memory in chunks of
// 512 (8 KB), double-buffered: one thread issues the bulk asynchronous copy
// (cp.async.bulk, TMA engine) of the next chunk, completion tracked by an
// mbarrier, while the CTA works on the current one; every source is then a
// broadcast shared-memory read.  Each lane accumulates an FP32 partial sum
// per chunk and adds it into a Neumaier-compensated FP32 pair; the NW warp
// results are added in FP64 in fixed order through shared memory.  FP64
// path: warp-uniform global loads (L1/L2-resident table).  Every output point
// is written by exactly one thread: deterministic, no atomics, no scratch
// memory.
#include <cmath>

#include "sa_async.cuh"
#include "sa_internal.h"

namespace {
using namespace sa_dev;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------------------
// prologue: source coefficients for step n1
// ---------------------------------------------------------------------------
struct PrologueArgs {
    const DevStatus* st_in;   // when non-null, n1 = st_in->n + 1; else n_explicit
    long long n_explicit;
    DevStatus* st_out;        // n_active written here when non-null
    int n_src;
    const double2* pos;
    double dt, alpha, r2_8a, coefE;
    float l2E;                // log2(coefE), for the FP32 coefficients
    int precision;
    double4* s64T;
    double4* s64F;
    float4* s32T;
    float4* s32F;
};

__global__ void k_prologue(PrologueArgs a) {
    const long long n1 = a.st_in ? a.st_in->n + 1 : a.n_explicit;
    const int K = (int)(n1 < (long long)a.n_src ? n1 : (long long)a.n_src);
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.st_out) a.st_out->n_active = K;
    const double kPi = 3.141592653589793;
    const double kLog2e = 1.4426950408889634;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x) {
        const long long I = i + 1;
        const double age = (double)(n1 - I) * a.dt + a.r2_8a;
        const double aI = 1.0 / (4.0 * a.alpha * age);
        const double base = 4.0 * kPi * a.alpha * age;
        const double cI = a.coefE / (base * sqrt(base));
        const double gI = 2.0 * aI * cI;
        const double2 p = a.pos[i];
        if (a.s64T) {
            a.s64T[i] = make_double4(p.x, p.y, aI, cI);
            if (a.s64F) a.s64F[i] = make_double4(p.x, p.y, aI, gI);
        }
        if (a.s32T) {
            const float sx = (float)p.x, sy = (float)p.y;
            const float na = (float)(-aI * kLog2e);
            a.s32T[i] = make_float4(sx, sy, na, (float)log2(cI));
            a.s32F[i] = make_float4(sx, sy, na, (float)log2(gI));
        }
    }
}

// Mixed path: the FP32 coefficients from FP32 arithmetic on the age (the
// FP64 transcendental functions run on GB300's narrow FP64 pipe; the FP32
// results are rounded to FP32 in either case):
//   log2 c = log2 E' - 1.5 log2(4 pi alpha age), log2 g = 1 - log2(4 alpha age) + log2 c.
__global__ void k_prologue32(PrologueArgs a) {
    const long long n1 = a.st_in ? a.st_in->n + 1 : a.n_explicit;
    const int K = (int)(n1 < (long long)a.n_src ? n1 : (long long)a.n_src);
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.st_out) a.st_out->n_active = K;
    const float kLog2e = 1.44269504f, kLog2Pi = 1.65149613f;
    const float four_alpha = (float)(4.0 * a.alpha);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x) {
        const long long I = i + 1;
        const float age = (float)((double)(n1 - I) * a.dt + a.r2_8a);
        const float fa = four_alpha * age;
        const float l4a = log2f(fa);
        const float na = -kLog2e / fa;
        const float l2c = a.l2E - 1.5f * (kLog2Pi + l4a);
        const double2 p = a.pos[i];
        const float sx = (float)p.x, sy = (float)p.y;
        a.s32T[i] = make_float4(sx, sy, na, l2c);
        a.s32F[i] = make_float4(sx, sy, na, 1.0f - l4a + l2c);
    }
}

// Batched prologue: every source of every instance; all instances share the
// step index n (lockstep), dt and the material; E, r and s_img enter through
// the per-instance coefE = s_img E / (rho c_p) and r2_8a = r^2 / (8 alpha).
struct PrologueBatchArgs {
    const DevStatus* st;
    int n_src_total, n_inst;
    const int* src_inst;
    const int* src_off;
    const int* n_src;
    const double* coefE;
    const double* r2_8a;
    int* n_active;
    const double2* pos;
    double dt, alpha;
    int precision;
    double4* s64T;
    double4* s64F;
    float4* s32T;
    float4* s32F;
};

__global__ void k_prologue_batch(PrologueBatchArgs a) {
    const long long n1 = a.st->n + 1;
    const double kPi = 3.141592653589793;
    const double kLog2e = 1.4426950408889634;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < a.n_inst) a.n_active[g] = (int)(n1 < (long long)a.n_src[g] ? n1 : (long long)a.n_src[g]);
    if (g >= a.n_src_total) return;
    const int inst = a.src_inst[g];
    const int l = g - a.src_off[inst];
    const long long K = n1 < (long long)a.n_src[inst] ? n1 : (long long)a.n_src[inst];
    if (l >= K) return;
    const long long I = l + 1;
    const double2 p = a.pos[g];
    if (a.precision != SA_MIXED) {
        const double age = (double)(n1 - I) * a.dt + a.r2_8a[inst];
        const double aI = 1.0 / (4.0 * a.alpha * age);
        const double base = 4.0 * kPi * a.alpha * age;
        const double cI = a.coefE[inst] / (base * sqrt(base));
        const double gI = 2.0 * aI * cI;
        a.s64T[g] = make_double4(p.x, p.y, aI, cI);
        a.s64F[g] = make_double4(p.x, p.y, aI, gI);
    } else {
        // FP32 arithmetic on the age, as in k_prologue32
        const float age = (float)((double)(n1 - I) * a.dt + a.r2_8a[inst]);
        const float fa = (float)(4.0 * a.alpha) * age;
        const float l4a = log2f(fa);
        const float l2c = log2f((float)a.coefE[inst]) - 1.5f * (1.65149613f + l4a);
        const float sx = (float)p.x, sy = (float)p.y;
        const float na = -(float)kLog2e / fa;
        a.s32T[g] = make_float4(sx, sy, na, l2c);
        a.s32F[g] = make_float4(sx, sy, na, 1.0f - l4a + l2c);
    }
}

// ---------------------------------------------------------------------------
// history sum
// ---------------------------------------------------------------------------
struct HistArgs {
    DevStatus* st;
    int q_lat, q_bot;
    int b_lat;                 // CTAs on lateral tiles; the rest on bottom tiles
    int blk0;                  // tile of block 0 (a launch can cover only the bottom tiles)
    const float* lat32;
    const float* bot32;
    const double* lat64;
    const double* bot64;
    double x_ref, y_ref, z_top;
    const float4* s32F;
    const float4* s32T;
    const double4* s64F;
    const double4* s64T;
    double* s_lat;
    double* tt_bot;
    // batched mode (n_inst > 0): the points of instance i are
    // [qlat_off[i], qlat_off[i+1]) / [qbot_off[i], qbot_off[i+1]) (multiples of
    // 128, so a tile never straddles two instances); its sources start at
    // src_off[i] and n_active[i] of them are in the sum
    int n_inst;
    const int* qlat_off;
    const int* qbot_off;
    const int* src_off;
    const int* n_active;
};

// Instance of a tile (batched mode) and its active source count / offset.
__device__ __forceinline__ void tile_sources(const HistArgs& a, bool flux, int q0, int& K,
                                             int& off) {
    if (a.n_inst == 0) {
        K = a.st->n_active;
        off = 0;
        return;
    }
    const int* qo = flux ? a.qlat_off : a.qbot_off;
    int lo = 0, hi = a.n_inst;   // qo[lo] <= q0 < qo[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (qo[mid] <= q0)
            lo = mid;
        else
            hi = mid;
    }
    K = a.n_active[lo];
    off = a.src_off[lo];
}

// Neumaier compensated addition of x into (s, c).
__device__ __forceinline__ void neumaier(float& s, float& c, float x) {
    const float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
}

// ---------------------------------------------------------------------------
// shared-memory staging of the source table: one thread issues a bulk
// asynchronous copy (TMA engine) of the next chunk while the CTA computes on
// the current one; completion is tracked by an mbarrier.  Waits are bounded.
// ---------------------------------------------------------------------------
constexpr int kChunk = 512;   // sources per staged chunk (8 KB)

struct Stage {
    float4 buf[2][kChunk];
    unsigned long long mbar[2];
    int abort_flag;
};

template <bool FLUX, int P, int NW>
__device__ void tile_mixed(const HistArgs& a, int tile, double* red, Stage& sg) {
    float4 (*sbuf)[kChunk] = sg.buf;
    unsigned long long* mbar = sg.mbar;
    int& abort_flag = sg.abort_flag;
    const int Q = FLUX ? a.q_lat : a.q_bot;
    const float* pts = FLUX ? a.lat32 : a.bot32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int q0 = tile * 32 * P;
    int K, soff;
    tile_sources(a, FLUX, q0, K, soff);
    const float4* src = (FLUX ? a.s32F : a.s32T) + soff;
    float px[P], py[P], dz2[P], nzdz[P], nx[P], ny[P];
    float s[P], c[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int q = q0 + lane + 32 * p;
        const bool ok = q < Q;
        px[p] = ok ? pts[0 * Q + q] : 0.f;
        py[p] = ok ? pts[1 * Q + q] : 0.f;
        dz2[p] = ok ? pts[2 * Q + q] : 0.f;
        if (FLUX) {
            nzdz[p] = ok ? pts[3 * Q + q] : 0.f;
            nx[p] = ok ? pts[4 * Q + q] : 0.f;
            ny[p] = ok ? pts[5 * Q + q] : 0.f;
        }
        s[p] = 0.f;
        c[p] = 0.f;
    }
    const int n_chunks = (K + kChunk - 1) / kChunk;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_fence_init();
        if (n_chunks > 0) bulk_load(sbuf[0], src, (unsigned)(min(K, kChunk) * sizeof(float4)), &mbar[0]);
    }
    __syncthreads();
    for (int ch = 0; ch < n_chunks; ++ch) {
        const int b = ch & 1;
        if (threadIdx.x == 0 && ch + 1 < n_chunks) {
            const int off = (ch + 1) * kChunk;
            bulk_load(sbuf[b ^ 1], src + off, (unsigned)(min(K - off, kChunk) * sizeof(float4)),
                      &mbar[b ^ 1]);
        }
        if (!mbar_wait_bounded(&mbar[b], (ch >> 1) & 1)) abort_flag = 1;
        __syncthreads();
        if (abort_flag) break;
        const int len = min(K - ch * kChunk, kChunk);
        float acc[P];
#pragma unroll
        for (int p = 0; p < P; ++p) acc[p] = 0.f;
#pragma unroll 4
        for (int j = w; j < len; j += NW) {
            const float4 sv = sbuf[b][j];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float dx = px[p] - sv.x;
                const float dy = py[p] - sv.y;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz2[p]));
                const float e = ex2_approx(fmaf(sv.z, r2, sv.w));
                if (FLUX) {
                    const float nd = fmaf(nx[p], dx, fmaf(ny[p], dy, nzdz[p]));
                    acc[p] = fmaf(e, nd, acc[p]);
                } else {
                    acc[p] += e;
                }
            }
        }
#pragma unroll
        for (int p = 0; p < P; ++p) neumaier(s[p], c[p], acc[p]);
        __syncthreads();   // every warp is done with buffer b before it is refilled
    }
    if (abort_flag) {
        // a chunk never arrived: flag it, let the copies in flight land
        // (bounded), write nothing
        if (threadIdx.x == 0) {
            atomicOr((int*)&a.st->err, SA_DEV_TIMEOUT);
            mbar_wait_bounded(&mbar[0], 0);
            mbar_wait_bounded(&mbar[1], 0);
        }
        __syncthreads();
        return;
    }
#pragma unroll
    for (int p = 0; p < P; ++p) red[w * 32 * P + lane + 32 * p] = (double)s[p] + (double)c[p];
    __syncthreads();
    for (int t = threadIdx.x; t < 32 * P; t += 32 * NW) {
        double tot = 0.0;
        for (int ww = 0; ww < NW; ++ww) tot += red[ww * 32 * P + t];
        const int q = q0 + t;
        if (q < Q) {
            if (FLUX)
                a.s_lat[q] = -tot;
            else
                a.tt_bot[q] = tot;
        }
    }
}

template <bool FLUX, int P, int NW>
__device__ void tile_fp64(const HistArgs& a, int tile, double* red) {
    const int Q = FLUX ? a.q_lat : a.q_bot;
    const double* pts = FLUX ? a.lat64 : a.bot64;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int q0 = tile * 32 * P;
    int K, soff;
    tile_sources(a, FLUX, q0, K, soff);
    const double4* src = (FLUX ? a.s64F : a.s64T) + soff;
    double px[P], py[P], dz[P], nx[P], ny[P], nz[P], acc[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int q = q0 + lane + 32 * p;
        const bool ok = q < Q;
        px[p] = ok ? pts[0 * Q + q] - a.x_ref : 0.0;
        py[p] = ok ? pts[1 * Q + q] - a.y_ref : 0.0;
        dz[p] = ok ? pts[2 * Q + q] - a.z_top : 0.0;
        if (FLUX) {
            nx[p] = ok ? pts[3 * Q + q] : 0.0;
            ny[p] = ok ? pts[4 * Q + q] : 0.0;
            nz[p] = ok ? pts[5 * Q + q] : 0.0;
        }
        acc[p] = 0.0;
    }
    for (int j = w; j < K; j += NW) {
        const double4 sv = src[j];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const double dx = px[p] - sv.x;
            const double dy = py[p] - sv.y;
            const double r2 = dx * dx + dy * dy + dz[p] * dz[p];
            const double e = sv.w * exp(-sv.z * r2);
            if (FLUX)
                acc[p] += e * (nx[p] * dx + ny[p] * dy + nz[p] * dz[p]);
            else
                acc[p] += e;
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) red[w * 32 * P + lane + 32 * p] = acc[p];
    __syncthreads();
    for (int t = threadIdx.x; t < 32 * P; t += 32 * NW) {
        double tot = 0.0;
        for (int ww = 0; ww < NW; ++ww) tot += red[ww * 32 * P + t];
        const int q = q0 + t;
        if (q < Q) {
            if (FLUX)
                a.s_lat[q] = -tot;
            else
                a.tt_bot[q] = tot;
        }
    }
}

template <int P, int NW>
__global__ void __launch_bounds__(32 * NW) k_history_mixed(HistArgs a) {
    __shared__ double red[NW * 32 * P];
    __shared__ __align__(128) Stage sg;
    const int b = (int)blockIdx.x + a.blk0;
    if (b < a.b_lat)
        tile_mixed<true, P, NW>(a, b, red, sg);
    else
        tile_mixed<false, P, NW>(a, b - a.b_lat, red, sg);
}

template <int P, int NW>
__global__ void __launch_bounds__(32 * NW) k_history_fp64(HistArgs a) {
    __shared__ double red[NW * 32 * P];
    const int b = (int)blockIdx.x + a.blk0;
    if (b < a.b_lat)
        tile_fp64<true, P, NW>(a, b, red);
    else
        tile_fp64<false, P, NW>(a, b - a.b_lat, red);
}

template <int P, int NW>
cudaError_t launch_hist_t(int precision, const HistArgs& a0, cudaStream_t s, int part = 0) {
    HistArgs a = a0;
    const int tile = 32 * P;
    a.b_lat = (a.q_lat + tile - 1) / tile;
    const int b_bot = (a.q_bot + tile - 1) / tile;
    // part 0: every tile; 1: lateral tiles; 2: bottom tiles
    a.blk0 = part == 2 ? a.b_lat : 0;
    const int grid = part == 1 ? a.b_lat : (part == 2 ? b_bot : a.b_lat + b_bot);
    if (grid == 0) return cudaSuccess;
    if (precision == SA_MIXED)
        k_history_mixed<P, NW><<<grid, 32 * NW, 0, s>>>(a);
    else
        k_history_fp64<P, NW><<<grid, 32 * NW, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_prologue(const DevStatus* st_in, long long n_explicit, DevStatus* st_out,
                            int n_src, const double2* pos, double dt, double alpha,
                            double r2_8a, double coefE, int precision, double4* s64T,
                            double4* s64F, float4* s32T, float4* s32F, cudaStream_t s) {
    PrologueArgs a;
    a.st_in = st_in;
    a.n_explicit = n_explicit;
    a.st_out = st_out;
    a.n_src = n_src;
    a.pos = pos;
    a.dt = dt;
    a.alpha = alpha;
    a.r2_8a = r2_8a;
    a.coefE = coefE;
    a.precision = precision;
    a.s64T = s64T;
    a.s64F = s64F;
    a.s32T = s32T;
    a.s32F = s32F;
    a.l2E = (float)std::log2(coefE);
    int blocks = (n_src + 127) / 128;
    if (blocks < 1) blocks = 1;
    if (s32T && !s64T)
        k_prologue32<<<blocks, 128, 0, s>>>(a);
    else
        k_prologue<<<blocks, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_history(int precision, int P, int warps, DevStatus* st, int q_lat,
                           int q_bot, const float* lat32, const float* bot32,
                           const double* lat64, const double* bot64, double x_ref,
                           double y_ref, double z_top, const float4* s32F,
                           const float4* s32T, const double4* s64F, const double4* s64T,
                           double* s_lat, double* tt_bot, cudaStream_t s, int part) {
    HistArgs a;
    a.st = st;
    a.q_lat = q_lat;
    a.q_bot = q_bot;
    a.b_lat = 0;
    a.blk0 = 0;
    a.lat32 = lat32;
    a.bot32 = bot32;
    a.lat64 = lat64;
    a.bot64 = bot64;
    a.x_ref = x_ref;
    a.y_ref = y_ref;
    a.z_top = z_top;
    a.s32F = s32F;
    a.s32T = s32T;
    a.s64F = s64F;
    a.s64T = s64T;
    a.s_lat = s_lat;
    a.tt_bot = tt_bot;
    a.n_inst = 0;
    a.qlat_off = a.qbot_off = a.src_off = a.n_active = nullptr;
    if (warps == 4) {
        if (P == 1) return launch_hist_t<1, 4>(precision, a, s, part);
        if (P == 2) return launch_hist_t<2, 4>(precision, a, s, part);
        return launch_hist_t<4, 4>(precision, a, s, part);
    }
    if (P == 1) return launch_hist_t<1, 8>(precision, a, s, part);
    if (P == 2) return launch_hist_t<2, 8>(precision, a, s, part);
    return launch_hist_t<4, 8>(precision, a, s, part);
}

cudaError_t launch_prologue_batch(const DevStatus* st, int n_src_total, int n_inst,
                                  const int* src_inst, const int* src_off, const int* n_src,
                                  const double* coefE, const double* r2_8a, int* n_active,
                                  const double2* pos, double dt, double alpha, int precision,
                                  double4* s64T, double4* s64F, float4* s32T, float4* s32F,
                                  cudaStream_t s) {
    PrologueBatchArgs a{st, n_src_total, n_inst, src_inst, src_off, n_src, coefE, r2_8a,
                        n_active, pos, dt, alpha, precision, s64T, s64F, s32T, s32F};
    const int n = n_src_total > n_inst ? n_src_total : n_inst;
    k_prologue_batch<<<(n + 255) / 256 > 0 ? (n + 255) / 256 : 1, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_history_batch(int precision, int P, int warps, DevStatus* st, int q_lat,
                                 int q_bot, const float* lat32, const float* bot32,
                                 const double* lat64, const double* bot64, const float4* s32F,
                                 const float4* s32T, const double4* s64F, const double4* s64T,
                                 double* s_lat, double* tt_bot, int n_inst, const int* qlat_off,
                                 const int* qbot_off, const int* src_off, const int* n_active,
                                 cudaStream_t s) {
    HistArgs a;
    a.st = st;
    a.q_lat = q_lat;
    a.q_bot = q_bot;
    a.b_lat = 0;
    a.blk0 = 0;
    a.lat32 = lat32;
    a.bot32 = bot32;
    a.lat64 = lat64;
    a.bot64 = bot64;
    a.x_ref = a.y_ref = a.z_top = 0.0;   // batched points carry z - z_top in z (see sa_batch)
    a.s32F = s32F;
    a.s32T = s32T;
    a.s64F = s64F;
    a.s64T = s64T;
    a.s_lat = s_lat;
    a.tt_bot = tt_bot;
    a.n_inst = n_inst;
    a.qlat_off = qlat_off;
    a.qbot_off = qbot_off;
    a.src_off = src_off;
    a.n_active = n_active;
    if (warps == 4) {
        if (P == 1) return launch_hist_t<1, 4>(precision, a, s);
        if (P == 2) return launch_hist_t<2, 4>(precision, a, s);
        return launch_hist_t<4, 4>(precision, a, s);
    }
    if (P == 1) return launch_hist_t<1, 8>(precision, a, s);
    if (P == 2) return launch_hist_t<2, 8>(precision, a, s);
    return launch_hist_t<4, 8>(precision, a, s);
}
