// Fast-diagonalization preconditioner of the theta-step operator
// A_ff = M/dt + theta K (free control variables of one tensor-product patch).
//
// The patch is replaced by the box with the same parametrisation and mean
// lengths L_d along its three parametric directions.  On that box M and K
// are Kronecker sums of one-dimensional B-spline matrices on the patch's
// own knot vectors (M^_d = int N_a N_b, K^_d = int N_a' N_b' over [0, 1]):
//   A_box = c_M M^_0 x M^_1 x M^_2 + c_0 K^_0 x M^_1 x M^_2
//         + c_1 M^_0 x K^_1 x M^_2 + c_2 M^_0 x M^_1 x K^_2,
//   c_M = rho c_p L_0 L_1 L_2 / dt,  c_d = theta k L_0 L_1 L_2 / L_d^2.
// With the generalised eigenpairs K^_d U_d = M^_d U_d Lambda_d
// (U_d^T M^_d U_d = I), A_box^{-1} = (U_0 x U_1 x U_2) D (U_0 x U_1 x U_2)^T
// with D = 1 / (c_M + c_0 lambda_0 + c_1 lambda_1 + c_2 lambda_2)
// (Lynch, Rice and Thomas, 1964; used as an isogeometric preconditioner by
// Sangalli and Tani, 2016).  For a box A_ff = A_box exactly.  For a curved
// patch the preconditioner is S A_box^{-1} S with S = diag(A_box)^{1/2}
// diag(A_ff)^{-1/2}, so that it matches A_ff on the diagonal.
//
// Dirichlet layers drop the end index of their direction; a closed (seam)
// direction folds its last index into the first (P^T M^ P).  The device
// applies it in five passes over lines of the grid (U_0^T, U_1^T,
// U_2 D U_2^T, U_1, U_0), inside the PCG kernel.
#include <cmath>
#include <vector>

#include "sa_internal.h"

namespace {

// Cox-de Boor values and first derivatives of the p+1 B-splines non-zero on
// span s of knot vector U at x (the local functions s-p .. s).
void bspline_ders_1d(const std::vector<double>& U, int p, int s, double x, double* N,
                     double* dN) {
    double left[SA_MAX_DEGREE + 2], right[SA_MAX_DEGREE + 2];
    double ndu[SA_MAX_DEGREE + 1][SA_MAX_DEGREE + 1];
    ndu[0][0] = 1.0;
    for (int j = 1; j <= p; ++j) {
        left[j] = x - U[s + 1 - j];
        right[j] = U[s + j] - x;
        double saved = 0.0;
        for (int r = 0; r < j; ++r) {
            ndu[j][r] = right[r + 1] + left[j - r];     // knot differences (lower triangle)
            const double t = ndu[r][j - 1] / ndu[j][r];
            ndu[r][j] = saved + right[r + 1] * t;
            saved = left[j - r] * t;
        }
        ndu[j][j] = saved;
    }
    for (int r = 0; r <= p; ++r) N[r] = ndu[r][p];
    // first derivative: p (N_{r,p-1} / (U_{s+r} - U_{s+r-p}) - N_{r+1,p-1} / (...))
    for (int r = 0; r <= p; ++r) {
        double d = 0.0;
        if (p > 0) {
            if (r >= 1) d += ndu[r - 1][p - 1] / ndu[p][r - 1];
            if (r <= p - 1) d -= ndu[r][p - 1] / ndu[p][r];
            d *= p;
        }
        dN[r] = d;
    }
}

// One-dimensional mass and stiffness matrices (dense, n x n) on [U_0, U_end]
// with (p+1) Gauss points per non-empty span.
void matrices_1d(const std::vector<double>& U, int p, int n, std::vector<double>& M,
                 std::vector<double>& K) {
    M.assign((size_t)n * n, 0.0);
    K.assign((size_t)n * n, 0.0);
    double gx[SA_MAX_DEGREE + 1], gw[SA_MAX_DEGREE + 1];
    gauss_legendre(p + 1, gx, gw);
    for (int s = p; s < n; ++s) {
        const double a = U[s], b = U[s + 1];
        if (!(b > a)) continue;
        for (int g = 0; g <= p; ++g) {
            const double x = a + 0.5 * (b - a) * (gx[g] + 1.0);
            const double w = 0.5 * (b - a) * gw[g];
            double N[SA_MAX_DEGREE + 1], dN[SA_MAX_DEGREE + 1];
            bspline_ders_1d(U, p, s, x, N, dN);
            for (int r = 0; r <= p; ++r)
                for (int q = 0; q <= p; ++q) {
                    M[(size_t)(s - p + r) * n + (s - p + q)] += w * N[r] * N[q];
                    K[(size_t)(s - p + r) * n + (s - p + q)] += w * dN[r] * dN[q];
                }
        }
    }
}

// Generalised symmetric-definite eigenproblem K u = lambda M u (dense, n x n,
// row-major): Cholesky M = L L^T, C = L^{-1} K L^{-T}, cyclic Jacobi rotations
// on C, U = L^{-T} V (so U^T M U = I, U^T K U = diag(lambda)).  Returns false
// if M is not positive definite.
bool gen_eig(int n, std::vector<double> M, const std::vector<double>& K, std::vector<double>& U,
             std::vector<double>& lam) {
    auto at = [n](std::vector<double>& A, int i, int j) -> double& { return A[(size_t)i * n + j]; };
    // Cholesky (lower) in place
    for (int j = 0; j < n; ++j) {
        double d = at(M, j, j);
        for (int k = 0; k < j; ++k) d -= at(M, j, k) * at(M, j, k);
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        at(M, j, j) = d;
        for (int i = j + 1; i < n; ++i) {
            double v = at(M, i, j);
            for (int k = 0; k < j; ++k) v -= at(M, i, k) * at(M, j, k);
            at(M, i, j) = v / d;
        }
        for (int i = 0; i < j; ++i) at(M, i, j) = 0.0;
    }
    // C = L^{-1} K L^{-T}: first B = L^{-1} K (forward substitution per column)
    std::vector<double> B(K), C((size_t)n * n);
    for (int c = 0; c < n; ++c)
        for (int i = 0; i < n; ++i) {
            double v = B[(size_t)i * n + c];
            for (int k = 0; k < i; ++k) v -= at(M, i, k) * B[(size_t)k * n + c];
            B[(size_t)i * n + c] = v / at(M, i, i);
        }
    // C^T = L^{-1} B^T, C symmetric: C[i][c] from rows of B
    for (int r = 0; r < n; ++r)
        for (int i = 0; i < n; ++i) {
            double v = B[(size_t)r * n + i];
            for (int k = 0; k < i; ++k) v -= at(M, i, k) * C[(size_t)r * n + k];
            C[(size_t)r * n + i] = v / at(M, i, i);
        }
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            const double s = 0.5 * (C[(size_t)i * n + j] + C[(size_t)j * n + i]);
            C[(size_t)i * n + j] = C[(size_t)j * n + i] = s;
        }
    // cyclic Jacobi
    std::vector<double> V((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    double fro = 0.0;
    for (double x : C) fro += x * x;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += C[(size_t)i * n + j] * C[(size_t)i * n + j];
        if (off <= 1e-30 * fro) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = C[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = C[(size_t)p * n + p], aqq = C[(size_t)q * n + q];
                const double tau = (aqq - app) / (2.0 * apq);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
                for (int k = 0; k < n; ++k) {          // columns p, q
                    const double ckp = C[(size_t)k * n + p], ckq = C[(size_t)k * n + q];
                    C[(size_t)k * n + p] = cs * ckp - sn * ckq;
                    C[(size_t)k * n + q] = sn * ckp + cs * ckq;
                }
                for (int k = 0; k < n; ++k) {          // rows p, q
                    const double cpk = C[(size_t)p * n + k], cqk = C[(size_t)q * n + k];
                    C[(size_t)p * n + k] = cs * cpk - sn * cqk;
                    C[(size_t)q * n + k] = sn * cpk + cs * cqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = cs * vkp - sn * vkq;
                    V[(size_t)k * n + q] = sn * vkp + cs * vkq;
                }
            }
    }
    lam.resize(n);
    for (int i = 0; i < n; ++i) lam[i] = C[(size_t)i * n + i];
    // U = L^{-T} V (back substitution per column)
    U.assign((size_t)n * n, 0.0);
    for (int c = 0; c < n; ++c)
        for (int i = n - 1; i >= 0; --i) {
            double v = V[(size_t)i * n + c];
            for (int k = i + 1; k < n; ++k) v -= at(M, k, i) * U[(size_t)k * n + c];
            U[(size_t)i * n + c] = v / at(M, i, i);
        }
    return true;
}

__global__ void k_fd_scale(int n, int m0, int m1, const double* md0, const double* kd0,
                           const double* md1, const double* kd1, const double* md2,
                           const double* kd2, double cM, double c0, double c1, double c2,
                           const double* dinv, void* S, int f32) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    const int i = f % m0, j = (f / m0) % m1, k = f / (m0 * m1);
    const double mz = md2 ? md2[k] : 1.0, kz = kd2 ? kd2[k] : 0.0;
    const double d = cM * md0[i] * md1[j] * mz + c0 * kd0[i] * md1[j] * mz +
                     c1 * md0[i] * kd1[j] * mz + c2 * md0[i] * md1[j] * kz;
    const double sc = sqrt(d * dinv[f]);
    if (f32)
        ((float*)S)[f] = (float)sc;
    else
        ((double*)S)[f] = sc;
}

template <typename T>
cudaError_t upload_as(DBuf<unsigned char>& buf, const std::vector<double>& v) {
    std::vector<T> h(v.begin(), v.end());
    cudaError_t e = buf.alloc(std::max<size_t>(h.size(), 1) * sizeof(T));
    if (e != cudaSuccess || h.empty()) return e;
    return cudaMemcpy(buf.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// 1-D data of parametric direction d: matrices on the knot vector, the seam
// folded, the end layers dropped (drop_lo / drop_hi), eigenpairs; the mean
// control-polygon length.  False when not usable.
bool direction_data(const sa_ctx* c, int d, bool drop_lo, bool drop_hi, FdData& f, int slot) {
    const int n = c->n[d], p = c->p[d];
    std::vector<double> M, K;
    matrices_1d(c->U[d], p, n, M, K);
    int nd = n;
    if (c->seam == d) {   // fold index n-1 into 0
        nd = n - 1;
        std::vector<double> Mf((size_t)nd * nd, 0.0), Kf((size_t)nd * nd, 0.0);
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) {
                Mf[(size_t)(a % nd) * nd + (b % nd)] += M[(size_t)a * n + b];
                Kf[(size_t)(a % nd) * nd + (b % nd)] += K[(size_t)a * n + b];
            }
        M.swap(Mf);
        K.swap(Kf);
    }
    const int lo = drop_lo ? 1 : 0, hi = nd - (drop_hi ? 1 : 0);
    const int m = hi - lo;
    if (m <= 0 || m > 128) return false;   // the device passes hold 4 entries per lane
    std::vector<double> Mr((size_t)m * m), Kr((size_t)m * m);
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) {
            Mr[(size_t)a * m + b] = M[(size_t)(a + lo) * nd + (b + lo)];
            Kr[(size_t)a * m + b] = K[(size_t)(a + lo) * nd + (b + lo)];
        }
    std::vector<double> U, lam;
    if (!gen_eig(m, Mr, Kr, U, lam)) return false;
    f.m[slot] = m;
    f.U[slot] = U;
    f.lam[slot] = lam;
    f.md[slot].resize(m);
    f.kd[slot].resize(m);
    for (int a = 0; a < m; ++a) {
        f.md[slot][a] = Mr[(size_t)a * m + a];
        f.kd[slot][a] = Kr[(size_t)a * m + a];
    }
    const int n0 = c->n[0], n1 = c->n[1];
    const int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;
    double sum = 0.0;
    int lines = 0;
    for (int ib = 0; ib < c->n[tb]; ++ib)
        for (int ia = 0; ia < c->n[ta]; ++ia) {
            double len = 0.0;
            for (int a = 0; a + 1 < n; ++a) {
                int i0[3], i1[3];
                i0[d] = a;
                i1[d] = a + 1;
                i0[ta] = i1[ta] = ia;
                i0[tb] = i1[tb] = ib;
                const double* P0 = &c->ctrl[3 * ((i0[2] * n1 + i0[1]) * n0 + i0[0])];
                const double* P1 = &c->ctrl[3 * ((i1[2] * n1 + i1[1]) * n0 + i1[0])];
                len += std::sqrt((P1[0] - P0[0]) * (P1[0] - P0[0]) + (P1[1] - P0[1]) * (P1[1] - P0[1]) +
                                 (P1[2] - P0[2]) * (P1[2] - P0[2]));
            }
            sum += len;
            ++lines;
        }
    f.L[slot] = sum / std::max(lines, 1);
    return f.L[slot] > 0.0;
}

sa_status upload_fd(sa_ctx* c, FdData& f, int n_rows) {
    const bool f32 = c->opt.precision == SA_MIXED;
    for (int d = 0; d < f.nd; ++d) {
        const int m = f.m[d];
        std::vector<double> Ut((size_t)m * m);
        for (int a = 0; a < m; ++a)
            for (int o = 0; o < m; ++o) Ut[(size_t)a * m + o] = f.U[d][(size_t)o * m + a];
        cudaError_t e = f32 ? upload_as<float>(f.dU[d], f.U[d]) : upload_as<double>(f.dU[d], f.U[d]);
        if (e == cudaSuccess) e = f32 ? upload_as<float>(f.dUt[d], Ut) : upload_as<double>(f.dUt[d], Ut);
        if (e == cudaSuccess) e = f.dlamc[d].alloc((size_t)m * (f32 ? 4 : 8));
        if (e == cudaSuccess) e = upload_as<double>(f.dmd[d], f.md[d]);
        if (e == cudaSuccess) e = upload_as<double>(f.dkd[d], f.kd[d]);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return sa_fail(c, SA_ERR_OOM, "fast-diagonalization data");
        }
    }
    cudaError_t e = f.S.alloc((size_t)std::max(n_rows, 1) * (f32 ? 4 : 8));
    if (e == cudaSuccess) e = f.Z.alloc((size_t)std::max(n_rows, 1) * (f32 ? 4 : 8));
    if (e == cudaSuccess) e = f.Z2.alloc((size_t)std::max(n_rows, 1) * (f32 ? 4 : 8));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return sa_fail(c, SA_ERR_OOM, "fast-diagonalization vectors");
    }
    f.ok = true;
    return SA_OK;
}

}  // namespace

// Geometry part (once per patch): 1-D matrices, eigenpairs, mean lengths,
// for the free control variables (3-D) and for the bottom Dirichlet layer
// (2-D, the projection's mass matrix) when that layer is the whole
// Dirichlet set.
sa_status fd_setup(sa_ctx* c) {
    c->fdm.ok = c->fdb.ok = false;
    bool dir[6];
    for (int f = 0; f < 6; ++f) dir[f] = c->face_kind[f] == SA_FACE_DIRICHLET;
    {
        FdData& f = c->fdm;
        f.nd = 3;
        bool ok = true;
        long long prod = 1;
        for (int d = 0; d < 3 && ok; ++d) {
            ok = direction_data(c, d, dir[2 * d], dir[2 * d + 1], f, d);
            prod *= f.m[d];
        }
        if (ok && prod == c->n_free) {
            sa_status st = upload_fd(c, f, c->n_free);
            if (st) return st;
        }
    }
    const bool bottom_only = dir[4] && !dir[0] && !dir[1] && !dir[2] && !dir[3] && !dir[5];
    if (bottom_only && c->seam != 2) {
        FdData& f = c->fdb;
        f.nd = 2;
        f.m[2] = 1;
        f.L[2] = 1.0;
        const bool ok = direction_data(c, 0, false, false, f, 0) && direction_data(c, 1, false, false, f, 1);
        if (ok && (long long)f.m[0] * f.m[1] == c->n_dir) {
            f.md[2].assign(1, 1.0);
            f.kd[2].assign(1, 0.0);
            sa_status st = upload_fd(c, f, c->n_dir);
            if (st) return st;
        }
    }
    return SA_OK;
}

// Operator part (per theta, dt): the scalings and S.  Main solve:
// c_M = rho c_p L0 L1 L2 / dt, c_d = theta k L0 L1 L2 / L_d^2.  Bottom
// projection (the face mass matrix): c_M = L0 L1, no stiffness.
cudaError_t fd_prepare(sa_ctx* c, double theta, double dt, cudaStream_t s) {
    const bool f32 = c->opt.precision == SA_MIXED;
    for (int which = 0; which < 2; ++which) {
        FdData& f = which == 0 ? c->fdm : c->fdb;
        if (!f.ok) continue;
        const int n = which == 0 ? c->n_free : c->n_dir;
        if (which == 0) {
            const double vol = f.L[0] * f.L[1] * f.L[2];
            f.cM = c->rho * c->cp * vol / dt;
            for (int d = 0; d < 3; ++d) f.c[d] = theta * c->k * vol / (f.L[d] * f.L[d]);
        } else {
            f.cM = f.L[0] * f.L[1];
            f.c[0] = f.c[1] = f.c[2] = 0.0;
        }
        for (int d = 0; d < f.nd; ++d) {
            std::vector<double> lc(f.lam[d]);
            for (double& x : lc) x *= f.c[d];
            cudaError_t e;
            if (f32) {
                std::vector<float> h(lc.begin(), lc.end());
                e = cudaMemcpy(f.dlamc[d].p, h.data(), h.size() * 4, cudaMemcpyHostToDevice);
            } else {
                e = cudaMemcpy(f.dlamc[d].p, lc.data(), lc.size() * 8, cudaMemcpyHostToDevice);
            }
            if (e != cudaSuccess) return e;
        }
        if (n == 0) continue;
        const double* md2 = f.nd == 3 ? (const double*)f.dmd[2].p : nullptr;
        const double* kd2 = f.nd == 3 ? (const double*)f.dkd[2].p : nullptr;
        k_fd_scale<<<(n + 255) / 256, 256, 0, s>>>(
            n, f.m[0], f.m[1], (const double*)f.dmd[0].p, (const double*)f.dkd[0].p,
            (const double*)f.dmd[1].p, (const double*)f.dkd[1].p, md2, kd2, f.cM, f.c[0], f.c[1],
            f.c[2], which == 0 ? c->a_dinv.p : c->mbot_dinv.p, f.S.p, f32 ? 1 : 0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

FdView fd_view(const sa_ctx* c, const FdData& f) {
    FdView v{};
    v.on = f.ok && c->opt.precond != SA_PRECOND_JACOBI;
    v.nd = f.nd;
    for (int d = 0; d < 3; ++d) {
        v.m[d] = f.m[d];
        v.U[d] = f.dU[d].p;
        v.Ut[d] = f.dUt[d].p;
        v.lamc[d] = f.dlamc[d].p;
    }
    v.cM = f.cM;
    v.S = f.S.p;
    v.Z = f.Z.p;
    v.Z2 = f.Z2.p;
    return v;
}
