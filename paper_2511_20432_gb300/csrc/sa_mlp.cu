// Learned warm start: a 4-layer perceptron (width H, BF16 weights, FP32
// accumulation) that proposes the increment of the theta-step solve from
// the solve's initial residual.  The paper has no learned component; the
// network only changes the PCG initial guess, and PCG still runs to the same
// residual tolerance (with the cold start x0 = T^n as fallback).
//
//   x -> silu(W1 x + b1) -> silu(W2 h + b2) -> silu(W3 h + b3) -> W4 h + b4
//
// Dense layers of a batch run on the tensor cores (mma.sync m16n8k16, BF16
// inputs, FP32 accumulators); one sample (the warm start inside a step) runs
// as four memory-bound GEMVs; bias, activation, loss and Adam are
// elementwise kernels.  Training: mean squared error, Adam on FP32 master weights with
// BF16 copies for the GEMMs.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "sa_internal.h"

typedef __nv_bfloat16 bf16;

namespace {

// ---------------------------------------------------------------------------
// GEMM on the tensor cores: C[m][n] = sum_k A(m, k) B(k, n) (+ beta C)
//   A(m, k) = A[m * sam + k * sak],  B(k, n) = B[k * sbk + n * sbn]  (BF16)
//   C FP32 row-major (ldc).  Block tile 64 x 64 x 32, 4 warps (2 x 2), each
//   warp 32 x 32 = 2 x 4 mma tiles of m16n8k16.
// ---------------------------------------------------------------------------
constexpr int BM = 64, BN = 64, BK = 32, PADK = 8;

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4],
                                         const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, const bf16* A, long long sam,
                                              long long sak, const bf16* B, long long sbk,
                                              long long sbn, float* C, long long ldc, float beta) {
    __shared__ __align__(16) bf16 As[BM][BK + PADK];
    __shared__ __align__(16) bf16 Bs[BN][BK + PADK];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int g = lane >> 2, t = lane & 3;
    const long long m0 = (long long)blockIdx.y * BM, n0 = (long long)blockIdx.x * BN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    const bf16 zero = __float2bfloat16(0.f);
    for (long long k0 = 0; k0 < K; k0 += BK) {
        // tiles into shared memory (consecutive threads along the contiguous
        // dimension of each operand)
#pragma unroll
        for (int i = 0; i < (BM * BK) / 128; ++i) {
            const int idx = tid + 128 * i;
            int mm, kk;
            if (sak == 1) {
                mm = idx / BK;
                kk = idx % BK;
            } else {
                mm = idx % BM;
                kk = idx / BM;
            }
            const long long gm = m0 + mm, gk = k0 + kk;
            As[mm][kk] = (gm < M && gk < K) ? A[gm * sam + gk * sak] : zero;
        }
#pragma unroll
        for (int i = 0; i < (BN * BK) / 128; ++i) {
            const int idx = tid + 128 * i;
            int nn, kk;
            if (sbk == 1) {
                nn = idx / BK;
                kk = idx % BK;
            } else {
                nn = idx % BN;
                kk = idx / BN;
            }
            const long long gn = n0 + nn, gk = k0 + kk;
            Bs[nn][kk] = (gn < N && gk < K) ? B[gk * sbk + gn * sbn] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            unsigned af[2][4], bfr[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int r = wm * 32 + mi * 16 + g;
                af[mi][0] = *(const unsigned*)&As[r][ks + 2 * t];
                af[mi][1] = *(const unsigned*)&As[r + 8][ks + 2 * t];
                af[mi][2] = *(const unsigned*)&As[r][ks + 2 * t + 8];
                af[mi][3] = *(const unsigned*)&As[r + 8][ks + 2 * t + 8];
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int cidx = wn * 32 + ni * 8 + g;
                bfr[ni][0] = *(const unsigned*)&Bs[cidx][ks + 2 * t];
                bfr[ni][1] = *(const unsigned*)&Bs[cidx][ks + 2 * t + 8];
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bfr[ni]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const long long gm = m0 + wm * 32 + mi * 16 + g + (r >= 2 ? 8 : 0);
                const long long gn = n0 + wn * 32 + ni * 8 + 2 * t + (r & 1);
                if (gm < M && gn < N) {
                    float* cp = C + gm * ldc + gn;
                    *cp = acc[mi][ni][r] + (beta != 0.f ? beta * *cp : 0.f);
                }
            }
}

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

// Z += b (per column); H = silu(Z) (hidden layers) as BF16.
__global__ void k_bias_act(long long rows, int cols, float* Z, const float* b, bf16* H, int act) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const float z = Z[i] + b[i % cols];
    Z[i] = z;
    if (H) H[i] = __float2bfloat16(act ? silu(z) : z);
}

// Batch-1 forward (the warm start inside a theta-step): each layer is a
// matrix-vector product whose time is the read of its BF16 weights (21 M
// parameters, ~43 MB for the block's network), so it runs as a GEMV on the
// CUDA cores, not as a 64-row tensor-core tile of which 63 rows would be
// padding.  ROWS output rows per warp; each lane reads 4 weights (8 bytes)
// per load along the row, FP32 products and sums, a warp butterfly; then the
// bias and, on hidden layers, SiLU rounded to BF16 as the batched path
// stores it.  Z gets the pre-activation (FP32).
template <int ROWS>
__global__ void __launch_bounds__(256) k_gemv(int out, int in, const bf16* __restrict__ W,
                                              const float* __restrict__ bias,
                                              const bf16* __restrict__ x, float* __restrict__ Z,
                                              bf16* __restrict__ H) {
    const int lane = threadIdx.x & 31;
    const long long r0 = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * ROWS;
    if (r0 >= out) return;
    float acc[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) acc[r] = 0.f;
    if ((in & 3) == 0) {
        const int n4 = in >> 2;
        const uint2* xv = reinterpret_cast<const uint2*>(x);
        for (int k = lane; k < n4; k += 32) {
            const uint2 xu = __ldg(xv + k);
            const float2 x01 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&xu.x));
            const float2 x23 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&xu.y));
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                if (r0 + r >= out) break;
                const uint2 wu = __ldg(reinterpret_cast<const uint2*>(W + (r0 + r) * (long long)in) + k);
                const float2 w01 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&wu.x));
                const float2 w23 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&wu.y));
                acc[r] = fmaf(w01.x, x01.x, acc[r]);
                acc[r] = fmaf(w01.y, x01.y, acc[r]);
                acc[r] = fmaf(w23.x, x23.x, acc[r]);
                acc[r] = fmaf(w23.y, x23.y, acc[r]);
            }
        }
    } else {
        for (int k = lane; k < in; k += 32) {
            const float xk = __bfloat162float(x[k]);
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                if (r0 + r >= out) break;
                acc[r] = fmaf(__bfloat162float(W[(r0 + r) * (long long)in + k]), xk, acc[r]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    if (lane != 0) return;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        if (r0 + r >= out) break;
        const float z = acc[r] + bias[r0 + r];
        Z[r0 + r] = z;
        if (H) H[r0 + r] = __float2bfloat16(silu(z));
    }
}

// dZ = dH * silu'(Z) (in place on the FP32 gradient), BF16 copy for the GEMMs.
__global__ void k_act_bwd(long long n, float* G, const float* Z, bf16* Gb) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float d = G[i] * dsilu(Z[i]);
    G[i] = d;
    Gb[i] = __float2bfloat16(d);
}

// Output layer: dZ = (Z - Y) / rows ; per-block partial sums of (Z - Y)^2.
__global__ void k_mse(long long n, int rows, const float* Z, const bf16* Y, float* G, bf16* Gb,
                      double* part) {
    __shared__ double sh[256];
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double e2 = 0.0;
    if (i < n) {
        const float d = Z[i] - __bfloat162float(Y[i]);
        const float gi = d / (float)rows;
        G[i] = gi;
        Gb[i] = __float2bfloat16(gi);
        e2 = (double)d * d;
    }
    sh[threadIdx.x] = e2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// db[c] = sum over rows of G[r][c] (fixed order).
__global__ void k_colsum(int rows, int cols, const float* G, float* db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += G[(long long)r * cols + c];
    db[c] = s;
}

// Adam on FP32 master parameters, BF16 copy refreshed.
__global__ void k_adam(long long n, float* p, const float* g, float* m, float* v, bf16* pb,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (pb) pb[i] = __float2bfloat16(pi);
}

__global__ void k_to_bf16(long long n, const float* in, bf16* out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16(in[i]);
}

// Counter-based initialisation (splitmix64 of the parameter index): weights
// uniform in [-s, s] with s = sqrt(6 / fan_in), biases 0.
__global__ void k_init(long long n, float* p, unsigned long long seed, float scale) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    p[i] = (float)((2.0 * u - 1.0) * scale);
}

unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

struct sa_mlp {
    int n_in = 0, hidden = 0, n_out = 0;
    int dims[5];
    // per layer l (0..3): W (dims[l+1] x dims[l]), b (dims[l+1])
    DBuf<float> W[4], b[4], gW[4], gb[4], mW[4], vW[4], mb[4], vb[4];
    DBuf<bf16> Wb[4];
    // activations for the current batch capacity
    int cap = 0;
    DBuf<float> Z[4], G[4];
    DBuf<bf16> H[4], Gb[4];
    DBuf<double> part;
    long long step = 0;
    std::string err;
};

namespace {

cudaError_t ensure_batch(sa_mlp* m, int rows) {
    if (rows <= m->cap) return cudaSuccess;
    for (int l = 0; l < 4; ++l) {
        const size_t n = (size_t)rows * m->dims[l + 1];
        cudaError_t e;
        if ((e = m->Z[l].alloc(n)) != cudaSuccess) return e;
        if ((e = m->G[l].alloc(n)) != cudaSuccess) return e;
        if ((e = m->H[l].alloc(n)) != cudaSuccess) return e;
        if ((e = m->Gb[l].alloc(n)) != cudaSuccess) return e;
    }
    const size_t np = blocks_for((long long)rows * m->dims[4], 256);
    cudaError_t e = m->part.alloc(np);
    if (e != cudaSuccess) return e;
    m->cap = rows;
    return cudaSuccess;
}

cudaError_t gemm(int M, int N, int K, const bf16* A, long long sam, long long sak, const bf16* B,
                 long long sbk, long long sbn, float* C, long long ldc, float beta, cudaStream_t s) {
    dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM));
    k_gemm<<<grid, 128, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, beta);
    return cudaGetLastError();
}

// forward pass of `rows` samples X (rows x n_in, BF16); output Z[3] (FP32)
cudaError_t forward(sa_mlp* m, const bf16* X, int rows, cudaStream_t s) {
    const bf16* h = X;
    if (rows == 1) {            // one sample: four GEMVs
        for (int l = 0; l < 4; ++l) {
            const int in = m->dims[l], out = m->dims[l + 1];
            bf16* H = l < 3 ? m->H[l].p : nullptr;
            if (l == 0) {       // a long input row: one row per warp
                k_gemv<1><<<blocks_for(out, 8), 256, 0, s>>>(out, in, m->Wb[l].p, m->b[l].p, h,
                                                              m->Z[l].p, H);
            } else {            // four rows per warp: four loads in flight per lane
                k_gemv<4><<<blocks_for(out, 32), 256, 0, s>>>(out, in, m->Wb[l].p, m->b[l].p, h,
                                                               m->Z[l].p, H);
            }
            h = H;
        }
        return cudaGetLastError();
    }
    for (int l = 0; l < 4; ++l) {
        const int in = m->dims[l], out = m->dims[l + 1];
        cudaError_t e = gemm(rows, out, in, h, in, 1, m->Wb[l].p, 1, in, m->Z[l].p, out, 0.f, s);
        if (e != cudaSuccess) return e;
        const long long n = (long long)rows * out;
        k_bias_act<<<blocks_for(n, 256), 256, 0, s>>>(rows, out, m->Z[l].p, m->b[l].p,
                                                       l < 3 ? m->H[l].p : nullptr, l < 3 ? 1 : 0);
        h = m->H[l].p;
    }
    return cudaGetLastError();
}

// gradients of the mean squared error over the batch into gW, gb; loss
// partials in part
cudaError_t backward(sa_mlp* m, const bf16* X, const bf16* Y, int rows, cudaStream_t s) {
    const long long nout = (long long)rows * m->dims[4];
    k_mse<<<blocks_for(nout, 256), 256, 0, s>>>(nout, rows, m->Z[3].p, Y, m->G[3].p, m->Gb[3].p,
                                                m->part.p);
    for (int l = 3; l >= 0; --l) {
        const int in = m->dims[l], out = m->dims[l + 1];
        const bf16* hin = l > 0 ? m->H[l - 1].p : X;
        // gW = dZ^T H_in : M = out, N = in, K = rows
        cudaError_t e = gemm(out, in, rows, m->Gb[l].p, 1, out, hin, in, 1, m->gW[l].p, in, 0.f, s);
        if (e != cudaSuccess) return e;
        k_colsum<<<blocks_for(out, 256), 256, 0, s>>>(rows, out, m->G[l].p, m->gb[l].p);
        if (l > 0) {
            // dH_in = dZ W : M = rows, N = in, K = out ; then through silu'
            e = gemm(rows, in, out, m->Gb[l].p, out, 1, m->Wb[l].p, in, 1, m->G[l - 1].p, in, 0.f, s);
            if (e != cudaSuccess) return e;
            const long long n = (long long)rows * in;
            k_act_bwd<<<blocks_for(n, 256), 256, 0, s>>>(n, m->G[l - 1].p, m->Z[l - 1].p, m->Gb[l - 1].p);
        }
    }
    return cudaGetLastError();
}

sa_status mfail(sa_mlp* m, sa_status st, const char* what) {
    if (m) m->err = what;
    return st;
}

}  // namespace

// entry points used by sa_api.cu for the warm start
cudaError_t mlp_forward(sa_mlp* m, const void* X, int rows, const float** out, cudaStream_t s) {
    cudaError_t e = ensure_batch(m, rows);
    if (e != cudaSuccess) return e;
    e = forward(m, (const bf16*)X, rows, s);
    *out = m->Z[3].p;
    return e;
}
int mlp_n_in(const sa_mlp* m) { return m->n_in; }
int mlp_prepare(sa_mlp* m, int rows) { return ensure_batch(m, rows) == cudaSuccess ? 0 : 1; }
int mlp_n_out(const sa_mlp* m) { return m->n_out; }

extern "C" {

sa_status sa_mlp_create(int n_in, int hidden, int n_out, unsigned long long seed, sa_mlp** out) {
    if (!out || n_in <= 0 || hidden <= 0 || n_out <= 0) return SA_ERR_ARG;
    *out = nullptr;
    sa_mlp* m = new sa_mlp();
    m->n_in = n_in;
    m->hidden = hidden;
    m->n_out = n_out;
    const int d[5] = {n_in, hidden, hidden, hidden, n_out};
    std::memcpy(m->dims, d, sizeof(d));
    for (int l = 0; l < 4; ++l) {
        const size_t nw = (size_t)d[l + 1] * d[l], nb = d[l + 1];
        if (m->W[l].alloc(nw) || m->Wb[l].alloc(nw) || m->gW[l].alloc(nw) || m->mW[l].alloc(nw) ||
            m->vW[l].alloc(nw) || m->b[l].alloc(nb) || m->gb[l].alloc(nb) || m->mb[l].alloc(nb) ||
            m->vb[l].alloc(nb)) {
            cudaGetLastError();
            delete m;
            return SA_ERR_OOM;
        }
        k_init<<<blocks_for((long long)nw, 256), 256>>>((long long)nw, m->W[l].p,
                                                        seed * 4 + l, (float)std::sqrt(6.0 / d[l]));
        k_to_bf16<<<blocks_for((long long)nw, 256), 256>>>((long long)nw, m->W[l].p, m->Wb[l].p);
        cudaMemset(m->b[l].p, 0, nb * sizeof(float));
        cudaMemset(m->mW[l].p, 0, nw * sizeof(float));
        cudaMemset(m->vW[l].p, 0, nw * sizeof(float));
        cudaMemset(m->mb[l].p, 0, nb * sizeof(float));
        cudaMemset(m->vb[l].p, 0, nb * sizeof(float));
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        delete m;
        return SA_ERR_CUDA;
    }
    *out = m;
    return SA_OK;
}

void sa_mlp_destroy(sa_mlp* m) { delete m; }

long long sa_mlp_n_params(const sa_mlp* m) {
    if (!m) return 0;
    long long n = 0;
    for (int l = 0; l < 4; ++l) n += (long long)m->dims[l + 1] * m->dims[l] + m->dims[l + 1];
    return n;
}

// Parameters as one FP32 host array: for l = 0..3, W_l (row-major) then b_l.
sa_status sa_mlp_get_params(sa_mlp* m, float* host) {
    if (!m || !host) return SA_ERR_ARG;
    size_t o = 0;
    for (int l = 0; l < 4; ++l) {
        const size_t nw = (size_t)m->dims[l + 1] * m->dims[l], nb = m->dims[l + 1];
        if (cudaMemcpy(host + o, m->W[l].p, nw * 4, cudaMemcpyDeviceToHost)) return SA_ERR_CUDA;
        o += nw;
        if (cudaMemcpy(host + o, m->b[l].p, nb * 4, cudaMemcpyDeviceToHost)) return SA_ERR_CUDA;
        o += nb;
    }
    return SA_OK;
}

sa_status sa_mlp_set_params(sa_mlp* m, const float* host) {
    if (!m || !host) return SA_ERR_ARG;
    size_t o = 0;
    for (int l = 0; l < 4; ++l) {
        const size_t nw = (size_t)m->dims[l + 1] * m->dims[l], nb = m->dims[l + 1];
        if (cudaMemcpy(m->W[l].p, host + o, nw * 4, cudaMemcpyHostToDevice)) return SA_ERR_CUDA;
        o += nw;
        if (cudaMemcpy(m->b[l].p, host + o, nb * 4, cudaMemcpyHostToDevice)) return SA_ERR_CUDA;
        o += nb;
        k_to_bf16<<<blocks_for((long long)nw, 256), 256>>>((long long)nw, m->W[l].p, m->Wb[l].p);
    }
    return cudaDeviceSynchronize() == cudaSuccess ? SA_OK : SA_ERR_CUDA;
}

// Forward pass: X (rows x n_in, BF16, device) -> Y (rows x n_out, FP32, device).
sa_status sa_mlp_forward(sa_mlp* m, const void* X, int rows, float* Y, void* stream) {
    if (!m || !X || !Y || rows <= 0) return SA_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const float* out = nullptr;
    if (mlp_forward(m, X, rows, &out, s) != cudaSuccess) return mfail(m, SA_ERR_CUDA, "forward");
    if (cudaMemcpyAsync(Y, out, sizeof(float) * rows * m->n_out, cudaMemcpyDeviceToDevice, s))
        return mfail(m, SA_ERR_CUDA, "copy");
    return cudaStreamSynchronize(s) == cudaSuccess ? SA_OK : SA_ERR_CUDA;
}

// Loss 1/(2 rows) sum ||f(x) - y||^2 and its gradients (host, FP32, same
// layout as sa_mlp_get_params).  X, Y: device BF16.
sa_status sa_mlp_gradients(sa_mlp* m, const void* X, const void* Y, int rows, float* host_grads,
                           double* loss, void* stream) {
    if (!m || !X || !Y || rows <= 0) return SA_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const float* out = nullptr;
    if (mlp_forward(m, X, rows, &out, s) != cudaSuccess) return mfail(m, SA_ERR_CUDA, "forward");
    if (backward(m, (const bf16*)X, (const bf16*)Y, rows, s) != cudaSuccess)
        return mfail(m, SA_ERR_CUDA, "backward");
    if (cudaStreamSynchronize(s) != cudaSuccess) return SA_ERR_CUDA;
    if (loss) {
        const size_t np = blocks_for((long long)rows * m->n_out, 256);
        std::vector<double> p(np);
        cudaMemcpy(p.data(), m->part.p, np * 8, cudaMemcpyDeviceToHost);
        double t = 0.0;
        for (double v : p) t += v;
        *loss = 0.5 * t / rows;
    }
    if (host_grads) {
        size_t o = 0;
        for (int l = 0; l < 4; ++l) {
            const size_t nw = (size_t)m->dims[l + 1] * m->dims[l], nb = m->dims[l + 1];
            cudaMemcpy(host_grads + o, m->gW[l].p, nw * 4, cudaMemcpyDeviceToHost);
            o += nw;
            cudaMemcpy(host_grads + o, m->gb[l].p, nb * 4, cudaMemcpyDeviceToHost);
            o += nb;
        }
    }
    return SA_OK;
}

// One Adam step on a minibatch (X, Y device BF16); returns the loss.
sa_status sa_mlp_train_step(sa_mlp* m, const void* X, const void* Y, int rows, float lr,
                            double* loss, void* stream) {
    if (!m || !X || !Y || rows <= 0 || !(lr > 0.f)) return SA_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const float* out = nullptr;
    if (mlp_forward(m, X, rows, &out, s) != cudaSuccess) return mfail(m, SA_ERR_CUDA, "forward");
    if (backward(m, (const bf16*)X, (const bf16*)Y, rows, s) != cudaSuccess)
        return mfail(m, SA_ERR_CUDA, "backward");
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
    for (int l = 0; l < 4; ++l) {
        const long long nw = (long long)m->dims[l + 1] * m->dims[l], nb = m->dims[l + 1];
        k_adam<<<blocks_for(nw, 256), 256, 0, s>>>(nw, m->W[l].p, m->gW[l].p, m->mW[l].p, m->vW[l].p,
                                                    m->Wb[l].p, lr, b1, b2, eps, c1, c2);
        k_adam<<<blocks_for(nb, 256), 256, 0, s>>>(nb, m->b[l].p, m->gb[l].p, m->mb[l].p, m->vb[l].p,
                                                    nullptr, lr, b1, b2, eps, c1, c2);
    }
    if (cudaGetLastError() != cudaSuccess) return mfail(m, SA_ERR_CUDA, "adam");
    if (loss) {
        if (cudaStreamSynchronize(s) != cudaSuccess) return SA_ERR_CUDA;
        const size_t np = blocks_for((long long)rows * m->n_out, 256);
        std::vector<double> p(np);
        cudaMemcpy(p.data(), m->part.p, np * 8, cudaMemcpyDeviceToHost);
        double t = 0.0;
        for (double v : p) t += v;
        *loss = 0.5 * t / rows;
    }
    return SA_OK;
}

}  // extern "C"
