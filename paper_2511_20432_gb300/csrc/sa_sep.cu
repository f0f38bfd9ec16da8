// Separable evaluation of the history sums of the analytical point-source
// field (Section 2.1, Eqs. sum-of-point-temp and semi-temperature) on faces
// that are axis-aligned rectangles with tensor-grid quadrature.
//
// On such a face every quadrature point is x = (a_i, b_j, d) in the face's
// axes (A and B tangential, D along the normal), i over the A list (the Gauss
// points of the first tangential direction, element-major) and j over the B
// list.  The Gaussian of source I factorises exactly,
//   exp(-a_I |x - x_I|^2) = exp(-a_I (a_i - s_A)^2) exp(-a_I (b_j - s_B)^2)
//                           exp(-a_I (d - s_D)^2),
// so the face's sum is a matrix product over the active sources,
//   S[i][j] = sum_I FA[I][i] FB[I][j],
//   FA[I][i] = exp(-a_I (a_i - s_A)^2),
//   FB[I][j] = w_I exp(-a_I ((b_j - s_B)^2 + (d - s_D)^2)) m_I,
// with w_I = c_I, m_I = 1 for T~ at the bottom points and w_I = g_I,
// m_I = n_D (d - s_D) for the normal derivative at the lateral points
// (n . (x - x_I) = n_D (d - s_D) when n = n_D e_D).  A (point, source) pair
// costs one FMA instead of an exponential; the factors cost (TI + TJ)
// exponentials per source and tile.
//
// Work layout: CTA (tile, unit) multiplies the 64 x TJ output tile over one
// unit of consecutive sources: the active sources split evenly over a fixed
// number of units (about six CTAs per multiprocessor), so the grid is static
// while the active count grows and every CTA has work; a unit is staged in
// rounds of at most 512 sources (256 in FP64).  Per chunk of 32 sources the
// CTA writes FA and FB into shared memory (double-buffered), then each thread
// accumulates a 4 x 4 register tile (small, so that many warps hide the
// shared-memory latency).  Mixed path: FP32 factors and products, each chunk
// summed into fresh registers and then added to the unit's sum (the rounding
// error grows with the chunk length plus the number of chunks, not with the
// unit); FP64 path: FP64 throughout.  The unit sums go to a partial buffer;
// a second kernel adds the active units of every point in a fixed order and
// writes the point's value: deterministic, no atomics.  Batched instances
// share one plan: each face records its instance, whose active count and
// first source the kernels look up.
//
// This is not the paper's evaluation (it sums pairwise); it is the same sum
// reordered by the distributive law, and applies only where the faces are
// such rectangles.  Host set-up detects them from the computed points.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "sa_internal.h"

namespace {

constexpr int kTI = 64;            // tile rows (A list)
constexpr int kPStride = 64 * 64;  // partial-buffer entries per (tile, unit)
// sources per chunk and per staging round (static shared memory under 48 KB)
template <typename T>
__host__ __device__ constexpr int chunk_of() { return sizeof(T) == 4 ? 32 : 16; }
template <typename T>
__host__ __device__ constexpr int max_unit_of() { return sizeof(T) == 4 ? 512 : 256; }

// Sources per unit at active count K: the K sources split evenly over the
// s_max units, in whole chunks (the last units may be short or empty).
__host__ __device__ inline int unit_len(int K, int s_max, int kc) {
    const int per = (K + s_max - 1) / s_max;
    return per > 0 ? (per + kc - 1) / kc * kc : kc;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct SepArgs {
    const SepFace* faces;
    const int4* tiles;
    int tile0;                // first tile of this launch
    int n_tiles;              // tiles of this launch
    int unit, s_max;
    DevStatus* st;
    // coef = 1 (mixed path): the source coefficients are formed here from the
    // positions and the step index, as the FP32 prologue forms them (no
    // prologue launch; the reduction records the active count)
    int coef;
    int n_src;
    const double2* pos;
    double dt, r2_8a, four_alpha;
    float l2E;
    // batched instances: active sources and first source of each instance
    // (null for one context)
    const int* inst_K;
    const int* inst_src;
    const float* c32;
    const double* c64;
    const float4* s32F;
    const float4* s32T;
    const double4* s64F;
    const double4* s64T;
    float* p32;
    double* p64;
    double* s_lat;
    double* tt_bot;
    // opt-in cutoff (ref null: off): eta, and the largest |sum| of each face
    // kind at the last two steps ([kind][step parity], non-negative FP32
    // bit patterns); kind of this launch's tiles (0 lateral, 1 Dirichlet)
    float cutoff;
    float* ref;
    int kind;
};

template <typename T>
struct SrcOf;
template <>
struct SrcOf<float> {
    using V = float4;
};
template <>
struct SrcOf<double> {
    using V = double4;
};

// Active sources at this step: min(n + 1, n_src) (the prologue's count).
__device__ __forceinline__ int active_sources(const SepArgs& a, int inst) {
    if (a.inst_K) return a.inst_K[inst];
    if (!a.coef) return a.st->n_active;
    const long long n1 = a.st->n + 1;
    return (int)(n1 < (long long)a.n_src ? n1 : (long long)a.n_src);
}

template <typename T, int TJ>
__global__ void __launch_bounds__(4 * TJ, (sizeof(T) == 4 ? 1024 : 512) / (4 * TJ)) k_sep_gemm(SepArgs a) {
    constexpr int NT = 4 * TJ;           // (64 / 4) x (TJ / 4) threads, 4 x 4 outputs each
    constexpr int NCOL = kTI + TJ;       // factor columns: FA then FB
    constexpr bool kMixed = sizeof(T) == 4;
    using V = typename SrcOf<T>::V;
    using T4 = typename std::conditional<kMixed, float4, double4>::type;
    constexpr int kKC = chunk_of<T>();
    constexpr int kMaxUnit = max_unit_of<T>();
    __shared__ __align__(16) T fab[2][kKC][NCOL];   // per source: FA (64) then FB (TJ)
    __shared__ T xs[NCOL];               // A list then B list of the tile
    __shared__ T4 prm[kMaxUnit];         // per source: s_A, s_B, exponent scale, offset
    __shared__ T mul[kMaxUnit];
    const int tile = a.tile0 + (int)blockIdx.x;
    const int4 td = a.tiles[tile];
    const SepFace f = a.faces[td.x];
    // cutoff: this step's maximum starts at zero (the reduction kernel that
    // follows this launch fills it); the previous step's sets the threshold
    const long long n1 = a.st->n + 1;
    if (a.ref && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
        a.ref[a.kind * 2 + (int)(n1 & 1)] = 0.f;
    const int K = active_sources(a, f.inst);
    const int u = unit_len(K, a.s_max, kKC);
    const int k0 = (int)blockIdx.y * u;
    if (k0 >= K) return;                 // no sources for this unit (uniform per CTA)
    const int n = min(K - k0, u);
    const int so = a.inst_src ? a.inst_src[f.inst] : 0;   // the instance's first source
    const T* coord = kMixed ? (const T*)a.c32 : (const T*)a.c64;
    for (int t = threadIdx.x; t < NCOL; t += NT) {
        if (t < kTI) {
            const int i = td.y + t;
            xs[t] = i < f.La ? coord[f.a_off + i] : T(0);
        } else {
            const int j = td.z + t - kTI;
            xs[t] = j < f.Lb ? coord[f.b_off + j] : T(0);
        }
    }
    __syncthreads();   // xs written
    // cutoff: the tile's box along A and B, the unit's threshold
    __shared__ T box[4];                 // A min, A max, B min, B max
    __shared__ T bsum[NT / 32];
    __shared__ int skip;
    const int ni = min(kTI, f.La - td.y), nj = min(TJ, f.Lb - td.z);
    T thr = T(0);
    if (a.ref) {
        thr = (T)(a.cutoff * a.ref[a.kind * 2 + (int)((n1 - 1) & 1)]) / (T)a.s_max;
        if (threadIdx.x == 0) {
            T lo = xs[0], hi = xs[0];
            for (int t = 1; t < ni; ++t) {
                lo = min(lo, xs[t]);
                hi = max(hi, xs[t]);
            }
            box[0] = lo;
            box[1] = hi;
            lo = hi = xs[kTI];
            for (int t = 1; t < nj; ++t) {
                lo = min(lo, xs[kTI + t]);
                hi = max(hi, xs[kTI + t]);
            }
            box[2] = lo;
            box[3] = hi;
        }
        __syncthreads();
    }
    // factors of chunk c into buffer c & 1 (log2 units; FP64: natural ones
    // with w folded into m):
    //   FA = 2^(sc (x - s_A)^2)        thread t: column t % 64, sources
    //                                  t / 64, + NT / 64, ...
    //   FB = 2^(sc (x - s_B)^2 + off) m   thread t: column t % TJ, sources
    //                                  t / TJ, + 4, ...
    constexpr int GA = NT / kTI, GB = NT / TJ;
    const int ca = threadIdx.x % kTI, ga = threadIdx.x / kTI;
    const int cb = threadIdx.x % TJ, gb = threadIdx.x / TJ;
    const T xa = xs[ca], xb = xs[kTI + cb];
    auto gen = [&](int c) {
        const int b = c & 1, s0 = c * kKC;
#pragma unroll 4
        for (int kk = ga; kk < kKC; kk += GA) {
            const T4 p4 = prm[s0 + kk];
            const T d = xa - p4.x;
            const T e = p4.z * (d * d);
            fab[b][kk][ca] = kMixed ? (T)ex2_approx((float)e) : (T)exp((double)e);
        }
#pragma unroll 4
        for (int kk = gb; kk < kKC; kk += GB) {
            const T4 p4 = prm[s0 + kk];
            const T d = xb - p4.y;
            const T e = fma(p4.z, d * d, p4.w);
            fab[b][kk][kTI + cb] =
                (kMixed ? (T)ex2_approx((float)e) : (T)exp((double)e)) * mul[s0 + kk];
        }
    };
    // warp w: rows (w & 1) 32 + 4 (lane & 7) .. + 3, columns (w >> 1) 16 +
    // 4 (lane >> 3) .. + 3: a warp reads 128 contiguous bytes of FA and 64 of
    // FB per source
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int r0 = (wi & 1) * 32 + (lane & 7) * 4;
    const int c0 = (wi >> 1) * 16 + (lane >> 3) * 4;
    T acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) acc[r][cc] = T(0);
    // the unit in rounds of at most kMaxUnit sources: their parameters staged
    // once per round (chunk padding: FB = 0)
    for (int rb = 0; rb < n; rb += kMaxUnit) {
        const int nr = min(kMaxUnit, n - rb);
        __syncthreads();   // the previous round's parameters and factors are consumed
        {
            const V* src = kMixed ? (const V*)(f.flux ? (const void*)a.s32F : (const void*)a.s32T)
                                  : (const V*)(f.flux ? (const void*)a.s64F : (const void*)a.s64T);
            const T dd = (T)f.dd, nsgn = (T)f.nsgn;
            const int npad = (nr + kKC - 1) / kKC * kKC;
            T bnd = T(0);        // cutoff: this thread's share of the unit's bound
            for (int t = threadIdx.x; t < npad; t += NT) {
                T sa = 0, sb = 0, sc = 0, off = 0, m = 0;
                if (t < nr) {
                    V sv;
                    if (kMixed && a.coef) {
                        // (sx, sy, -a log2 e, log2 w) from the age, in FP32:
                        // log2 c = log2 E' - 1.5 log2(4 pi alpha age),
                        // log2 g = 1 - log2(4 alpha age) + log2 c
                        const long long I = k0 + rb + t + 1;
                        const float age = (float)((double)(a.st->n + 1 - I) * a.dt + a.r2_8a);
                        const float fa = (float)a.four_alpha * age;
                        const float l4a = log2f(fa);
                        const float l2c = a.l2E - 1.5f * (1.65149613f + l4a);
                        const double2 p = a.pos[k0 + rb + t];
                        sv.x = (float)p.x;
                        sv.y = (float)p.y;
                        sv.z = -1.44269504f / fa;
                        sv.w = f.flux ? 1.0f - l4a + l2c : l2c;
                    } else {
                        sv = src[so + k0 + rb + t];
                    }
                    // sources lie on the top plane (relative z = 0)
                    auto sc3 = [&](int ax) { return ax == 0 ? (T)sv.x : (ax == 1 ? (T)sv.y : T(0)); };
                    sa = sc3(f.axa);
                    sb = sc3(f.axb);
                    const T dsd = dd - sc3(f.axd);
                    if (kMixed) {
                        // log2 units: sv.z = -a log2 e, sv.w = log2 w
                        sc = (T)sv.z;
                        off = fma(sc, dsd * dsd, (T)sv.w);
                        m = f.flux ? nsgn * dsd : T(1);
                    } else {
                        // sv.z = a, sv.w = w
                        sc = -(T)sv.z;
                        off = sc * dsd * dsd;
                        m = (T)sv.w * (f.flux ? nsgn * dsd : T(1));
                    }
                }
                T4 p4;
                p4.x = sa;
                p4.y = sb;
                p4.z = sc;
                p4.w = off;
                prm[t] = p4;
                mul[t] = m;
                if (a.ref && t < nr) {
                    // the source's largest term over the tile: at the box
                    // point nearest to it (|n . d| is the same over a face)
                    const T dA = max(T(0), max(box[0] - sa, sa - box[1]));
                    const T dB = max(T(0), max(box[2] - sb, sb - box[3]));
                    const T e = fma(sc, fma(dA, dA, dB * dB), off);
                    bnd += (kMixed ? (T)ex2_approx((float)e) : (T)exp((double)e)) * (m < T(0) ? -m : m);
                }
            }
            if (a.ref) {
                // the round's bound, summed in a fixed order (deterministic)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) bnd += __shfl_xor_sync(0xffffffffu, bnd, o);
                if ((threadIdx.x & 31) == 0) bsum[threadIdx.x >> 5] = bnd;
            }
        }
        __syncthreads();
        if (a.ref) {
            if (threadIdx.x == 0) {
                T tot = T(0);
                for (int w = 0; w < NT / 32; ++w) tot += bsum[w];
                skip = tot <= thr * (T)nr / (T)n;
                if (skip)
                    atomicAdd((unsigned long long*)&a.st->hist_skipped,
                              (unsigned long long)nr * (unsigned long long)(ni * nj));
            }
            __syncthreads();
            if (skip) continue;
        }
        const int nch = (nr + kKC - 1) / kKC;
        gen(0);
        __syncthreads();
        for (int c = 0; c < nch; ++c) {
            if (c + 1 < nch) gen(c + 1);     // the other buffer
            const int b = c & 1;
            T cs[4][4];
    #pragma unroll
            for (int r = 0; r < 4; ++r)
    #pragma unroll
                for (int cc = 0; cc < 4; ++cc) cs[r][cc] = kMixed ? T(0) : acc[r][cc];
    #pragma unroll 8
            for (int kk = 0; kk < kKC; ++kk) {
                T av[4], bv[4];
    #pragma unroll
                for (int r = 0; r < 4; ++r) {
                    av[r] = fab[b][kk][r0 + r];
                    bv[r] = fab[b][kk][kTI + c0 + r];
                }
    #pragma unroll
                for (int r = 0; r < 4; ++r)
    #pragma unroll
                    for (int cc = 0; cc < 4; ++cc) cs[r][cc] = fma(av[r], bv[cc], cs[r][cc]);
            }
    #pragma unroll
            for (int r = 0; r < 4; ++r)
    #pragma unroll
                for (int cc = 0; cc < 4; ++cc) acc[r][cc] = kMixed ? acc[r][cc] + cs[r][cc] : cs[r][cc];
            __syncthreads();   // buffer b is consumed and the other one is written
        }
    }
    // unit sums: entry (jj, ii) of the tile at jj * 64 + ii
    T* part = (kMixed ? (T*)a.p32 : (T*)a.p64) +
              ((size_t)tile * a.s_max + blockIdx.y) * kPStride;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        T* col = part + (c0 + cc) * kTI + r0;
#pragma unroll
        for (int r = 0; r < 4; ++r) col[r] = acc[r][cc];
    }
}

// Sum of the active units of every point of the launch's tiles; writes
// s_lat = -sum (flux faces) or tt_bot = sum.
// Four lanes per point: lane g adds units g, g + 4, ... in order; the four
// sums are combined by the same butterfly on every lane.  The sum runs in the
// partials' precision (FP64 arithmetic is slow on this part; at most a few
// dozen unit sums of one sign per point in the mixed path).
template <typename T, int TJ>
__global__ void __launch_bounds__(256) k_sep_reduce(SepArgs a) {
    constexpr int kKC = chunk_of<T>();
    const int per = kTI * TJ;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int o = g >> 2, lane4 = g & 3;
    bool ok = o < a.n_tiles * per;
    const int tl = ok ? o / per : 0, e = o - tl * per;
    const int tile = a.tile0 + tl;
    const int4 td = ok ? a.tiles[tile] : make_int4(0, 0, 0, 0);
    const SepFace& f = a.faces[td.x];
    const int jj = e / kTI, ii = e - jj * kTI;
    const int i = td.y + ii, j = td.z + jj;
    ok = ok && i < f.La && j < f.Lb;
    const int K = active_sources(a, f.inst);
    if (a.coef && g == 0) a.st->n_active = K;
    const int u = unit_len(K, a.s_max, kKC);
    const int ns = K > 0 ? (K + u - 1) / u : 0;
    T tot = T(0);
    if (ok) {
        const T* p = (sizeof(T) == 4 ? (const T*)a.p32 : (const T*)a.p64) +
                     (size_t)tile * a.s_max * kPStride + e;
#pragma unroll 4
        for (int s = lane4; s < ns; s += 4) tot += p[(size_t)s * kPStride];
    }
    tot += __shfl_xor_sync(0xffffffffu, tot, 1);
    tot += __shfl_xor_sync(0xffffffffu, tot, 2);
    if (a.ref) {
        // cutoff: this step's largest |sum| of the face kind (non-negative
        // FP32 values order as their bit patterns)
        float v = ok ? fabsf((float)tot) : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if ((threadIdx.x & 31) == 0 && v > 0.f)
            atomicMax((int*)&a.ref[a.kind * 2 + (int)((a.st->n + 1) & 1)], __float_as_int(v));
    }
    if (!ok || lane4 != 0) return;
    const int ea = i / f.nga, ga = i - ea * f.nga;
    const int eb = j / f.ngb, gb = j - eb * f.ngb;
    const int q = f.q0 + ((eb * f.nea + ea) * f.ngb + gb) * f.nga + ga;
    if (f.flux)
        a.s_lat[q] = -(double)tot;
    else
        a.tt_bot[q] = (double)tot;
}

template <typename T, int TJ>
cudaError_t launch_sep_t(const SepArgs& a, cudaStream_t s) {
    if (a.n_tiles == 0) return cudaSuccess;
    k_sep_gemm<T, TJ><<<dim3(a.n_tiles, a.s_max), 4 * TJ, 0, s>>>(a);
    const int n = 4 * a.n_tiles * kTI * TJ;
    k_sep_reduce<T, TJ><<<(n + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sep_tj(int tj, const SepArgs& a, cudaStream_t s) {
    if (tj == 32) return launch_sep_t<T, 32>(a, s);
    if (tj == 48) return launch_sep_t<T, 48>(a, s);
    return launch_sep_t<T, 64>(a, s);
}

// point (i, j) of a face in the canonical order
inline int face_point(const SepFace& f, int i, int j) {
    const int ea = i / f.nga, ga = i - ea * f.nga;
    const int eb = j / f.ngb, gb = j - eb * f.ngb;
    return f.q0 + ((eb * f.nea + ea) * f.ngb + gb) * f.nga + ga;
}

template <class T>
sa_status put(sa_ctx* c, DBuf<T>& b, const std::vector<T>& v, const char* what) {
    cudaError_t e = b.alloc(v.size());
    if (e == cudaSuccess && !v.empty())
        e = cudaMemcpy(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) return SA_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? sa_fail(c, SA_ERR_OOM, "allocation of %s failed", what)
                                          : sa_cuda_fail(c, e, what);
}

}  // namespace

// Detect the separable faces from the computed quadrature points and build
// the plan (every lateral and Dirichlet face must qualify).
sa_status sep_setup(sa_ctx* c) {
    SepPlan& P = c->sep;
    P.ok = false;
    P.faces_h.clear();
    P.tiles_h.clear();
    P.coord_h.clear();
    P.n_tiles[0] = P.n_tiles[1] = 0;
    if (c->opt.hist_mode == SA_HIST_PAIRWISE) return SA_OK;
    std::vector<double> lat((size_t)7 * c->q_lat), bot((size_t)4 * c->q_bot);
    if (c->q_lat > 0)
        SA_CUDA(c, cudaMemcpy(lat.data(), c->lat64.p, sizeof(double) * lat.size(),
                              cudaMemcpyDeviceToHost));
    if (c->q_bot > 0)
        SA_CUDA(c, cudaMemcpy(bot.data(), c->bot64.p, sizeof(double) * bot.size(),
                              cudaMemcpyDeviceToHost));
    // tolerance: 1e-12 of the extent of the boundary points
    double lo[3] = {HUGE_VAL, HUGE_VAL, HUGE_VAL}, hi[3] = {-HUGE_VAL, -HUGE_VAL, -HUGE_VAL};
    for (int kind = 0; kind < 2; ++kind) {
        const std::vector<double>& X = kind == 0 ? lat : bot;
        const int Q = kind == 0 ? c->q_lat : c->q_bot;
        for (int ax = 0; ax < 3; ++ax)
            for (int q = 0; q < Q; ++q) {
                lo[ax] = std::min(lo[ax], X[(size_t)ax * Q + q]);
                hi[ax] = std::max(hi[ax], X[(size_t)ax * Q + q]);
            }
    }
    double ext = 0.0;
    for (int ax = 0; ax < 3; ++ax)
        if (hi[ax] >= lo[ax]) ext = std::max(ext, hi[ax] - lo[ax]);
    const double tol = 1e-12 * ext;
    const double ref[3] = {c->x_ref, c->y_ref, c->z_top};
    const char* why = nullptr;
    for (int kind = 0; kind < 2 && !why; ++kind) {
        const std::vector<double>& X = kind == 0 ? lat : bot;
        const int Q = kind == 0 ? c->q_lat : c->q_bot;
        const int want = kind == 0 ? SA_FACE_NEUMANN : SA_FACE_DIRICHLET;
        std::vector<int> mine;
        for (int f = 0; f < 6 && !why; ++f) {
            if (c->face_kind[f] != want) continue;
            const int d = f / 2;
            const int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;
            SepFace F{};
            F.q0 = c->face_q0[kind][f];
            F.nga = c->p[ta] + 1;
            F.nea = c->ne[ta];
            F.ngb = c->p[tb] + 1;
            F.La = F.nea * F.nga;
            F.Lb = c->ne[tb] * F.ngb;
            F.flux = kind == 0;
            auto x = [&](int ax, int i, int j) { return X[(size_t)ax * Q + face_point(F, i, j)]; };
            // the fixed axis: constant over the face
            int axd = -1;
            for (int ax = 0; ax < 3 && axd < 0; ++ax) {
                double mn = HUGE_VAL, mx = -HUGE_VAL;
                for (int j = 0; j < F.Lb; ++j)
                    for (int i = 0; i < F.La; ++i) {
                        mn = std::min(mn, x(ax, i, j));
                        mx = std::max(mx, x(ax, i, j));
                    }
                if (mx - mn <= tol) axd = ax;
            }
            if (axd < 0) {
                why = "a face is not planar and axis-aligned";
                break;
            }
            int u = axd == 0 ? 1 : 0, v = axd == 2 ? 1 : 2;
            auto only_i = [&](int ax) {
                for (int j = 0; j < F.Lb; ++j)
                    for (int i = 0; i < F.La; ++i)
                        if (std::fabs(x(ax, i, j) - x(ax, i, 0)) > tol) return false;
                return true;
            };
            auto only_j = [&](int ax) {
                for (int j = 0; j < F.Lb; ++j)
                    for (int i = 0; i < F.La; ++i)
                        if (std::fabs(x(ax, i, j) - x(ax, 0, j)) > tol) return false;
                return true;
            };
            if (only_i(u) && only_j(v)) {
                F.axa = u;
                F.axb = v;
            } else if (only_i(v) && only_j(u)) {
                F.axa = v;
                F.axb = u;
            } else {
                why = "a face's quadrature points are not a tensor grid along the axes";
                break;
            }
            F.axd = axd;
            F.nsgn = 1.0;
            if (F.flux) {
                // normal along axd, the same sign everywhere
                const double s0 = x(3 + axd, 0, 0) > 0 ? 1.0 : -1.0;
                for (int j = 0; j < F.Lb && !why; ++j)
                    for (int i = 0; i < F.La; ++i) {
                        const double nd = x(3 + axd, i, j);
                        const double no = std::fabs(x(3 + F.axa, i, j)) + std::fabs(x(3 + F.axb, i, j));
                        if (std::fabs(nd - s0) > 1e-12 || no > 1e-12) {
                            why = "a lateral face's normal is not a coordinate axis";
                            break;
                        }
                    }
                F.nsgn = s0;
            }
            F.dd = x(axd, 0, 0) - ref[axd];
            F.a_off = (int)P.coord_h.size();
            for (int i = 0; i < F.La; ++i) P.coord_h.push_back(x(F.axa, i, 0) - ref[F.axa]);
            F.b_off = (int)P.coord_h.size();
            for (int j = 0; j < F.Lb; ++j) P.coord_h.push_back(x(F.axb, 0, j) - ref[F.axb]);
            mine.push_back((int)P.faces_h.size());
            P.faces_h.push_back(F);
        }
        if (why) break;
        // tile width: the least padded area, ties to the wider tile
        long long best = -1;
        for (int tj : {64, 48, 32}) {
            long long area = 0;
            for (int fi : mine) {
                const SepFace& F = P.faces_h[fi];
                area += (long long)((F.La + kTI - 1) / kTI) * kTI * ((F.Lb + tj - 1) / tj) * tj;
            }
            if (best < 0 || area < best) {
                best = area;
                P.tj[kind] = tj;
            }
        }
        for (int fi : mine) {
            const SepFace& F = P.faces_h[fi];
            for (int i0 = 0; i0 < F.La; i0 += kTI)
                for (int j0 = 0; j0 < F.Lb; j0 += P.tj[kind]) {
                    P.tiles_h.push_back(make_int4(fi, i0, j0, 0));
                    ++P.n_tiles[kind];
                }
        }
    }
    if (why) {
        if (c->opt.hist_mode == SA_HIST_SEPARABLE)
            return sa_fail(c, SA_ERR_ARG, "separable history sums: %s", why);
        P.faces_h.clear();
        P.tiles_h.clear();
        P.coord_h.clear();
        P.n_tiles[0] = P.n_tiles[1] = 0;
        return SA_OK;
    }
    const std::vector<float> c32(P.coord_h.begin(), P.coord_h.end());
    sa_status st = put(c, P.faces, P.faces_h, "separable faces");
    if (!st) st = put(c, P.tiles, P.tiles_h, "separable tiles");
    if (!st) st = put(c, P.coord64, P.coord_h, "separable coordinates");
    if (!st) st = put(c, P.coord32, c32, "separable coordinates FP32");
    if (st) return st;
    P.ok = true;
    return SA_OK;
}

// Units and partial buffers for the context's source count.
sa_status sep_alloc(sa_ctx* c) {
    SepPlan& P = c->sep;
    if (!P.ok) return SA_OK;
    // about six CTAs a multiprocessor over the two launches (they run one
    // after the other: ~2.6 and ~3.5 a multiprocessor each; measured against
    // four, eight and twelve), and no unit longer than the shared-memory
    // staging holds at the full scan
    const int n = std::max(c->n_src, 1);
    const bool f32 = c->opt.precision == SA_MIXED;
    const int kc = f32 ? chunk_of<float>() : chunk_of<double>();
    const int umax = f32 ? max_unit_of<float>() : max_unit_of<double>();
    const int tiles = std::max(1, P.n_tiles[0] + P.n_tiles[1]);
    int s_max = std::max(1, (6 * c->num_sms + tiles - 1) / tiles);
    s_max = std::max(s_max, (n + umax - 1) / umax);
    // with K = n: unit_len <= umax (a whole number of chunks)
    while (unit_len(n, s_max, kc) > umax) ++s_max;
    P.s_max = s_max;
    P.unit = unit_len(n, s_max, kc);
    const size_t len = (size_t)(P.n_tiles[0] + P.n_tiles[1]) * P.s_max * kPStride;
    if (c->opt.precision == SA_MIXED) {
        SA_ALLOC(c, P.part32, len);
    } else {
        SA_ALLOC(c, P.part64, len);
    }
    if (c->opt.hist_cutoff > 0.0) {
        SA_ALLOC(c, P.ref, 4);
        SA_CUDA(c, cudaMemset(P.ref.p, 0, 4 * sizeof(float)));
    }
    return SA_OK;
}

// part 0: every face; 1: lateral faces; 2: Dirichlet faces.  Mixed path:
// the source coefficients of step n + 1 are formed in the product kernels
// (no prologue launch before them).
cudaError_t launch_sep(sa_ctx* c, int part, double dt, cudaStream_t s) {
    const SepPlan& P = c->sep;
    for (int kind = 0; kind < 2; ++kind) {
        if (part == 1 && kind == 1) continue;
        if (part == 2 && kind == 0) continue;
        SepArgs a;
        a.faces = P.faces.p;
        a.tiles = P.tiles.p;
        a.tile0 = kind == 0 ? 0 : P.n_tiles[0];
        a.n_tiles = P.n_tiles[kind];
        a.unit = P.unit;
        a.s_max = P.s_max;
        a.st = c->st.p;
        const double alpha = c->k / (c->rho * c->cp);
        a.coef = c->opt.precision == SA_MIXED ? 1 : 0;
        a.n_src = c->n_src;
        a.pos = c->src_pos.p;
        a.dt = dt;
        a.r2_8a = c->spot_radius * c->spot_radius / (8.0 * alpha);
        a.four_alpha = 4.0 * alpha;
        a.l2E = (float)std::log2(c->opt.half_space_factor * c->E / (c->rho * c->cp));
        a.inst_K = nullptr;
        a.inst_src = nullptr;
        a.c32 = P.coord32.p;
        a.c64 = P.coord64.p;
        a.s32F = c->src32F.p;
        a.s32T = c->src32T.p;
        a.s64F = c->src64F.p;
        a.s64T = c->src64T.p;
        a.p32 = P.part32.p;
        a.p64 = P.part64.p;
        a.s_lat = c->s_lat.p;
        a.tt_bot = c->tt_bot.p;
        a.cutoff = (float)c->opt.hist_cutoff;
        a.ref = c->opt.hist_cutoff > 0.0 ? P.ref.p : nullptr;
        a.kind = kind;
        const cudaError_t e = c->opt.precision == SA_MIXED ? launch_sep_tj<float>(P.tj[kind], a, s)
                                                           : launch_sep_tj<double>(P.tj[kind], a, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One plan over batched instances: every instance's faces with their output
// offsets moved to the batch's point ranges, their coordinate lists
// concatenated, tiles rebuilt with one tile width per kind (given, or the
// least padded); s_max units per tile (1: the unit runs in staging rounds
// and its sums are the tile's sums).
bool sep_batch_plan(const std::vector<sa_ctx*>& insts, const std::vector<int>& qlat_off,
                    const std::vector<int>& qbot_off, int precision, SepPlan& P, int tj_lat,
                    int tj_bot, int s_max) {
    P.ok = false;
    P.faces_h.clear();
    P.tiles_h.clear();
    P.coord_h.clear();
    P.n_tiles[0] = P.n_tiles[1] = 0;
    for (const sa_ctx* c : insts)
        if (!c->sep.ok) return false;
    std::vector<int> coff(insts.size());
    for (size_t i = 0; i < insts.size(); ++i) {
        coff[i] = (int)P.coord_h.size();
        P.coord_h.insert(P.coord_h.end(), insts[i]->sep.coord_h.begin(), insts[i]->sep.coord_h.end());
    }
    for (int kind = 0; kind < 2; ++kind) {
        std::vector<int> mine;
        for (size_t i = 0; i < insts.size(); ++i)
            for (SepFace F : insts[i]->sep.faces_h) {
                if (F.flux != (kind == 0)) continue;
                F.q0 += kind == 0 ? qlat_off[i] : qbot_off[i];
                F.a_off += coff[i];
                F.b_off += coff[i];
                F.inst = (int)i;
                mine.push_back((int)P.faces_h.size());
                P.faces_h.push_back(F);
            }
        // tile width: as given (the autotuner), else the least padded area
        const int forced = kind == 0 ? tj_lat : tj_bot;
        long long best = -1;
        for (int tj : {64, 48, 32}) {
            long long area = 0;
            for (int fi : mine) {
                const SepFace& F = P.faces_h[fi];
                area += (long long)((F.La + kTI - 1) / kTI) * kTI * ((F.Lb + tj - 1) / tj) * tj;
            }
            if (forced == tj || (forced == 0 && (best < 0 || area < best))) {
                best = area;
                P.tj[kind] = tj;
            }
        }
        for (int fi : mine) {
            const SepFace& F = P.faces_h[fi];
            for (int i0 = 0; i0 < F.La; i0 += kTI)
                for (int j0 = 0; j0 < F.Lb; j0 += P.tj[kind]) {
                    P.tiles_h.push_back(make_int4(fi, i0, j0, 0));
                    ++P.n_tiles[kind];
                }
        }
    }
    // units per tile: each instance's active sources split over s_max units
    // (the kernels derive the unit length from the instance's count)
    P.s_max = std::max(1, s_max);
    P.unit = 0;
    const std::vector<float> c32(P.coord_h.begin(), P.coord_h.end());
    const size_t len = (size_t)std::max(1, P.n_tiles[0] + P.n_tiles[1]) * P.s_max * kPStride;
    bool ok = P.faces.alloc(P.faces_h.size()) == cudaSuccess &&
              P.tiles.alloc(P.tiles_h.size()) == cudaSuccess &&
              P.coord64.alloc(P.coord_h.size()) == cudaSuccess &&
              P.coord32.alloc(c32.size()) == cudaSuccess &&
              (precision == SA_MIXED ? P.part32.alloc(len) : P.part64.alloc(len)) == cudaSuccess;
    ok = ok && cudaMemcpy(P.faces.p, P.faces_h.data(), sizeof(SepFace) * P.faces_h.size(),
                          cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(P.tiles.p, P.tiles_h.data(), sizeof(int4) * P.tiles_h.size(),
                          cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(P.coord64.p, P.coord_h.data(), sizeof(double) * P.coord_h.size(),
                          cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(P.coord32.p, c32.data(), sizeof(float) * c32.size(),
                          cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return false;
    }
    P.ok = true;
    return true;
}

cudaError_t launch_sep_batch(const SepPlan& P, int precision, DevStatus* st, const int* n_active,
                             const int* src_off, const float4* s32F, const float4* s32T,
                             const double4* s64F, const double4* s64T, double* s_lat,
                             double* tt_bot, cudaStream_t s) {
    for (int kind = 0; kind < 2; ++kind) {
        SepArgs a{};
        a.faces = P.faces.p;
        a.tiles = P.tiles.p;
        a.tile0 = kind == 0 ? 0 : P.n_tiles[0];
        a.n_tiles = P.n_tiles[kind];
        a.unit = 0;
        a.s_max = P.s_max;
        a.st = st;
        a.coef = 0;
        a.inst_K = n_active;
        a.inst_src = src_off;
        a.c32 = P.coord32.p;
        a.c64 = P.coord64.p;
        a.s32F = s32F;
        a.s32T = s32T;
        a.s64F = s64F;
        a.s64T = s64T;
        a.p32 = P.part32.p;
        a.p64 = P.part64.p;
        a.s_lat = s_lat;
        a.tt_bot = tt_bot;
        a.cutoff = 0.f;          // batches keep the full sums
        a.ref = nullptr;
        a.kind = kind;
        const cudaError_t e = precision == SA_MIXED ? launch_sep_tj<float>(P.tj[kind], a, s)
                                                    : launch_sep_tj<double>(P.tj[kind], a, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
