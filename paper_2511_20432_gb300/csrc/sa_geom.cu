// One-time set-up kernels: NURBS basis by Cox-de Boor, boundary quadrature
// points with normals and weights, element matrices and their deterministic
// gather into CSR (Section 2.3: the map Phi, grad_x N = J^{-T} grad_xi N,
// dV = det J dxi, and the integrals M_ij, K_ij, F_i).
#include <cuda_bf16.h>

#include "sa_internal.h"

namespace {

// Non-zero B-spline values N[0..p] = N_{s-p..s, p}(u) and their first
// derivatives on the knot span s (U[s] <= u < U[s+1], or u = U[s+1] at the
// right end), by the triangular Cox-de Boor recursion: degree q is built
// from degree q-1, N_{i,q} = (u-U_i)/(U_{i+q}-U_i) N_{i,q-1}
// + (U_{i+q+1}-u)/(U_{i+q+1}-U_{i+1}) N_{i+1,q-1}; the derivative of degree
// p uses the degree p-1 values.  No denominator vanishes on a non-empty span.
__device__ void bspline_1d(const double* U, int p, int s, double u, double* N, double* dN) {
    double cur[SA_MAX_DEGREE + 1], prev[SA_MAX_DEGREE + 1];
    cur[0] = 1.0;
    for (int q = 1; q <= p; ++q) {
        for (int r = 0; r < q; ++r) prev[r] = cur[r];
        for (int r = 0; r <= q; ++r) {
            const int i = s - q + r;
            double v = 0.0;
            if (r > 0) v += (u - U[i]) / (U[i + q] - U[i]) * prev[r - 1];
            if (r < q) v += (U[i + q + 1] - u) / (U[i + q + 1] - U[i + 1]) * prev[r];
            cur[r] = v;
        }
    }
    // here prev holds degree p-1 (if p >= 1)
    for (int r = 0; r <= p; ++r) {
        N[r] = cur[r];
        if (p == 0) {
            dN[r] = 0.0;
            continue;
        }
        const int i = s - p + r;
        double d = 0.0;
        if (r > 0) d += p / (U[i + p] - U[i]) * prev[r - 1];
        if (r < p) d -= p / (U[i + p + 1] - U[i + 1]) * prev[r];
        dN[r] = d;
    }
}

struct Basis1D {
    double N[3][SA_MAX_DEGREE + 1];
    double dN[3][SA_MAX_DEGREE + 1];
    int s[3];
};

__device__ inline int nat_index(const DevPatch& dp, int i, int j, int k) {
    return (k * dp.n[1] + j) * dp.n[0] + i;
}

// NURBS geometry at one parametric point: first pass (weights W, dW and the
// Jacobian J[c][d] = d x_c / d xi_d through the quotient rule).
__device__ void nurbs_point(const DevPatch& dp, const Basis1D& b, double x[3], double J[3][3],
                            double& Wsum, double dW[3]) {
    Wsum = 0.0;
    dW[0] = dW[1] = dW[2] = 0.0;
    double xw[3] = {0, 0, 0};
    double dxw[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a2 = 0; a2 <= dp.p[2]; ++a2)
        for (int a1 = 0; a1 <= dp.p[1]; ++a1)
            for (int a0 = 0; a0 <= dp.p[0]; ++a0) {
                const int gi = b.s[0] - dp.p[0] + a0, gj = b.s[1] - dp.p[1] + a1,
                          gk = b.s[2] - dp.p[2] + a2;
                const double4 c = dp.cw[nat_index(dp, gi, gj, gk)];
                const double Nv = b.N[0][a0] * b.N[1][a1] * b.N[2][a2];
                const double d0 = b.dN[0][a0] * b.N[1][a1] * b.N[2][a2];
                const double d1 = b.N[0][a0] * b.dN[1][a1] * b.N[2][a2];
                const double d2 = b.N[0][a0] * b.N[1][a1] * b.dN[2][a2];
                const double wN = c.w * Nv;
                Wsum += wN;
                dW[0] += c.w * d0;
                dW[1] += c.w * d1;
                dW[2] += c.w * d2;
                const double P[3] = {c.x, c.y, c.z};
                for (int cc = 0; cc < 3; ++cc) {
                    xw[cc] += wN * P[cc];
                    dxw[cc][0] += c.w * d0 * P[cc];
                    dxw[cc][1] += c.w * d1 * P[cc];
                    dxw[cc][2] += c.w * d2 * P[cc];
                }
            }
    // x = xw / W ;  dx/dxi = (dxw W - xw dW) / W^2
    for (int cc = 0; cc < 3; ++cc) {
        x[cc] = xw[cc] / Wsum;
        for (int d = 0; d < 3; ++d) J[cc][d] = (dxw[cc][d] - x[cc] * dW[d]) / Wsum;
    }
}

__device__ inline double det3(const double J[3][3]) {
    return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

// ---------------------------------------------------------------------------
// boundary quadrature points of one face
// ---------------------------------------------------------------------------
struct FaceArgs {
    DevPatch dp;
    int d, side, ta, tb;       // fixed direction, side, tangential directions
    int nea, neb, nga, ngb;
    double xg_a[SA_MAX_DEGREE + 1], wg_a[SA_MAX_DEGREE + 1];
    double xg_b[SA_MAX_DEGREE + 1], wg_b[SA_MAX_DEGREE + 1];
    int q_offset, q_stride, with_normal;
    double* pts64;             // SoA with stride q_stride
    const int* slot;           // (face point, face function) -> CSR slot of W
    double* w_val;
    double* coo_R;             // optional: per point, face-function values
    int* coo_dof;              // optional: per point, internal dof of face functions
    const int* perm;
};

__global__ void k_face_points(FaceArgs a) {
    const int nq = a.nea * a.neb * a.nga * a.ngb;
    const int qf = blockIdx.x * blockDim.x + threadIdx.x;
    if (qf >= nq) return;
    const DevPatch& dp = a.dp;
    int t = qf;
    const int ga = t % a.nga; t /= a.nga;
    const int gb = t % a.ngb; t /= a.ngb;
    const int ea = t % a.nea; t /= a.nea;
    const int eb = t;
    Basis1D b;
    double xi[3];
    const int sa = dp.espan[a.ta][ea], sb = dp.espan[a.tb][eb];
    {
        const double lo = dp.U[a.ta][sa], hi = dp.U[a.ta][sa + 1];
        xi[a.ta] = lo + 0.5 * (hi - lo) * (a.xg_a[ga] + 1.0);
    }
    {
        const double lo = dp.U[a.tb][sb], hi = dp.U[a.tb][sb + 1];
        xi[a.tb] = lo + 0.5 * (hi - lo) * (a.xg_b[gb] + 1.0);
    }
    const int nd = dp.n[a.d], pd = dp.p[a.d];
    const int sd = a.side == 0 ? pd : nd - 1;
    xi[a.d] = a.side == 0 ? dp.U[a.d][pd] : dp.U[a.d][nd];
    b.s[a.ta] = sa;
    b.s[a.tb] = sb;
    b.s[a.d] = sd;
    for (int d = 0; d < 3; ++d) bspline_1d(dp.U[d], dp.p[d], b.s[d], xi[d], b.N[d], b.dN[d]);
    double x[3], J[3][3], W, dW[3];
    nurbs_point(dp, b, x, J, W, dW);
    const double ha = dp.U[a.ta][sa + 1] - dp.U[a.ta][sa];
    const double hb = dp.U[a.tb][sb + 1] - dp.U[a.tb][sb];
    const double wt = 0.25 * ha * hb * a.wg_a[ga] * a.wg_b[gb];
    // x_u x x_v, oriented outward: on the side-0 face the normal points to
    // decreasing xi_d, i.e. n . (dx/dxi_d) < 0, and > 0 on the side-1 face.
    const double xu[3] = {J[0][a.ta], J[1][a.ta], J[2][a.ta]};
    const double xv[3] = {J[0][a.tb], J[1][a.tb], J[2][a.tb]};
    double c[3] = {xu[1] * xv[2] - xu[2] * xv[1], xu[2] * xv[0] - xu[0] * xv[2],
                   xu[0] * xv[1] - xu[1] * xv[0]};
    const double area = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    const double dotd = c[0] * J[0][a.d] + c[1] * J[1][a.d] + c[2] * J[2][a.d];
    const double want = a.side == 0 ? -1.0 : 1.0;
    const double sgn = (dotd * want >= 0.0) ? 1.0 : -1.0;
    const double wdS = wt * area;
    const int q = a.q_offset + qf;
    double* P = a.pts64;
    P[0 * a.q_stride + q] = x[0];
    P[1 * a.q_stride + q] = x[1];
    P[2 * a.q_stride + q] = x[2];
    if (a.with_normal) {
        P[3 * a.q_stride + q] = sgn * c[0] / area;
        P[4 * a.q_stride + q] = sgn * c[1] / area;
        P[5 * a.q_stride + q] = sgn * c[2] / area;
        P[6 * a.q_stride + q] = wdS;
    } else {
        P[3 * a.q_stride + q] = wdS;
    }
    // face functions: the layer of the fixed direction that is non-zero on
    // the face (open knots: the first or last), tangential local indices
    const int ld = a.side == 0 ? 0 : pd;
    const int pa = dp.p[a.ta], pb = dp.p[a.tb];
    const int nfb = (pa + 1) * (pb + 1);
    for (int lb = 0; lb <= pb; ++lb)
        for (int la = 0; la <= pa; ++la) {
            int loc[3];
            loc[a.d] = ld;
            loc[a.ta] = la;
            loc[a.tb] = lb;
            int g3[3];
            for (int d = 0; d < 3; ++d) g3[d] = b.s[d] - dp.p[d] + loc[d];
            const int nat = nat_index(dp, g3[0], g3[1], g3[2]);
            const double Nv = b.N[0][loc[0]] * b.N[1][loc[1]] * b.N[2][loc[2]];
            const double R = dp.cw[nat].w * Nv / W;
            const int e = qf * nfb + lb * (pa + 1) + la;
            a.w_val[a.slot[e]] = wdS * R;
            if (a.coo_R) {
                a.coo_R[e] = R;
                a.coo_dof[e] = a.perm[nat];
            }
        }
}

// ---------------------------------------------------------------------------
// element matrices: one block per element
// ---------------------------------------------------------------------------
struct ElemArgs {
    DevPatch dp;
    double rho_cp, k;
    double xg[3][SA_MAX_DEGREE + 1], wg[3][SA_MAX_DEGREE + 1];
    double* Mloc;
    double* Kloc;
    int* bad_jac;
};

__global__ void k_element_local(ElemArgs a) {
    extern __shared__ double sm[];
    const DevPatch& dp = a.dp;
    const int nl0 = dp.p[0] + 1, nl1 = dp.p[1] + 1, nl2 = dp.p[2] + 1;
    const int nloc = nl0 * nl1 * nl2;
    const int nqp = nloc;                       // (p+1) Gauss points per direction
    double* sR = sm;                            // [nqp][nloc]
    double* sG = sR + nqp * nloc;               // [nqp][nloc][3]
    double* sw = sG + 3 * nqp * nloc;           // [nqp]
    const int e = blockIdx.x;
    const int e0 = e % dp.ne[0], e1 = (e / dp.ne[0]) % dp.ne[1], e2 = e / (dp.ne[0] * dp.ne[1]);
    const int es[3] = {e0, e1, e2};
    for (int qp = threadIdx.x; qp < nqp; qp += blockDim.x) {
        const int g0 = qp % nl0, g1 = (qp / nl0) % nl1, g2 = qp / (nl0 * nl1);
        const int gs[3] = {g0, g1, g2};
        Basis1D b;
        double wt = 1.0;
        for (int d = 0; d < 3; ++d) {
            const int s = dp.espan[d][es[d]];
            const double lo = dp.U[d][s], hi = dp.U[d][s + 1];
            const double u = lo + 0.5 * (hi - lo) * (a.xg[d][gs[d]] + 1.0);
            wt *= 0.5 * (hi - lo) * a.wg[d][gs[d]];
            b.s[d] = s;
            bspline_1d(dp.U[d], dp.p[d], s, u, b.N[d], b.dN[d]);
        }
        double x[3], J[3][3], W, dW[3];
        nurbs_point(dp, b, x, J, W, dW);
        const double det = det3(J);
        if (!(det > 0.0)) atomicOr(a.bad_jac, 1);
        // inverse transpose: grad_x R = J^{-T} grad_xi R
        double inv[3][3];
        inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
        inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
        inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
        inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
        sw[qp] = wt * det;
        for (int a2 = 0; a2 < nl2; ++a2)
            for (int a1 = 0; a1 < nl1; ++a1)
                for (int a0 = 0; a0 < nl0; ++a0) {
                    const int la = (a2 * nl1 + a1) * nl0 + a0;
                    const int gi = b.s[0] - dp.p[0] + a0, gj = b.s[1] - dp.p[1] + a1,
                              gk = b.s[2] - dp.p[2] + a2;
                    const double w = dp.cw[nat_index(dp, gi, gj, gk)].w;
                    const double Nv = b.N[0][a0] * b.N[1][a1] * b.N[2][a2];
                    const double dNv[3] = {b.dN[0][a0] * b.N[1][a1] * b.N[2][a2],
                                           b.N[0][a0] * b.dN[1][a1] * b.N[2][a2],
                                           b.N[0][a0] * b.N[1][a1] * b.dN[2][a2]};
                    const double R = w * Nv / W;
                    double dR[3];
                    for (int d = 0; d < 3; ++d) dR[d] = (w * dNv[d] - R * dW[d]) / W;
                    sR[qp * nloc + la] = R;
                    for (int c = 0; c < 3; ++c)
                        sG[(qp * nloc + la) * 3 + c] =
                            inv[0][c] * dR[0] + inv[1][c] * dR[1] + inv[2][c] * dR[2];
                }
    }
    __syncthreads();
    const size_t base = (size_t)e * nloc * nloc;
    for (int pr = threadIdx.x; pr < nloc * nloc; pr += blockDim.x) {
        const int ia = pr / nloc, ib = pr % nloc;
        double m = 0.0, kk = 0.0;
        for (int qp = 0; qp < nqp; ++qp) {
            const double w = sw[qp];
            m += w * sR[qp * nloc + ia] * sR[qp * nloc + ib];
            const double* ga = &sG[(qp * nloc + ia) * 3];
            const double* gb = &sG[(qp * nloc + ib) * 3];
            kk += w * (ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2]);
        }
        a.Mloc[base + pr] = a.rho_cp * m;
        a.Kloc[base + pr] = a.k * kk;
    }
}

// ---------------------------------------------------------------------------
// CSR gather: M_ij = sum over the elements supporting both i and j of the
// local entries, in a fixed element order (e2, e1, e0 ascending): one warp
// per row, deterministic, no atomics.
// ---------------------------------------------------------------------------
struct GatherArgs {
    DevPatch dp;
    const long long* ptr;
    const int* col;
    const int* elo[3];
    const int* ehi[3];
    const double* Mloc;
    const double* Kloc;
    double* M;
    double* K;
};

__global__ void k_mk_gather(GatherArgs a) {
    const DevPatch& dp = a.dp;
    const int n_dof = dp.n[0] * dp.n[1] * dp.n[2];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_dof) return;
    const int i = warp;
    const int ii[3] = {i % dp.n[0], (i / dp.n[0]) % dp.n[1], i / (dp.n[0] * dp.n[1])};
    const int nl0 = dp.p[0] + 1, nl1 = dp.p[1] + 1, nl2 = dp.p[2] + 1;
    const int nloc = nl0 * nl1 * nl2;
    for (long long s = a.ptr[i] + lane; s < a.ptr[i + 1]; s += 32) {
        const int j = a.col[s];
        const int jj[3] = {j % dp.n[0], (j / dp.n[0]) % dp.n[1], j / (dp.n[0] * dp.n[1])};
        int lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
            lo[d] = max(a.elo[d][ii[d]], a.elo[d][jj[d]]);
            hi[d] = min(a.ehi[d][ii[d]], a.ehi[d][jj[d]]);
        }
        double m = 0.0, kk = 0.0;
        for (int e2 = lo[2]; e2 <= hi[2]; ++e2)
            for (int e1 = lo[1]; e1 <= hi[1]; ++e1)
                for (int e0 = lo[0]; e0 <= hi[0]; ++e0) {
                    const int es[3] = {e0, e1, e2};
                    int la[3], lb[3];
                    for (int d = 0; d < 3; ++d) {
                        const int first = dp.espan[d][es[d]] - dp.p[d];
                        la[d] = ii[d] - first;
                        lb[d] = jj[d] - first;
                    }
                    const int ia = (la[2] * nl1 + la[1]) * nl0 + la[0];
                    const int ib = (lb[2] * nl1 + lb[1]) * nl0 + lb[0];
                    const size_t e = ((size_t)e2 * dp.ne[1] + e1) * dp.ne[0] + e0;
                    const size_t off = e * nloc * nloc + (size_t)ia * nloc + ib;
                    m += a.Mloc[off];
                    kk += a.Kloc[off];
                }
        a.M[s] = m;
        a.K[s] = kk;
    }
}

// M_bot[r][c] = sum_q wdS_q R_r(x_q) R_c(x_q): thread per CSR entry, the
// points of row r from W_bot (value wdS R_r), R_c from the point's list.
__global__ void k_mbot_fill(int n_rows, const int* mptr, const int* mcol, const int* wptr,
                            const int* wcol, const double* wval, const int* coo_dof,
                            const double* coo_R, int nfb, int n_free, double* mval,
                            double* dinv) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    for (int s = mptr[r]; s < mptr[r + 1]; ++s) {
        const int c = mcol[s];
        double acc = 0.0;
        for (int t = wptr[r]; t < wptr[r + 1]; ++t) {
            const int q = wcol[t];
            for (int f = 0; f < nfb; ++f)
                if (coo_dof[q * nfb + f] - n_free == c) acc += wval[t] * coo_R[q * nfb + f];
        }
        mval[s] = acc;
        if (c == r) dinv[r] = 1.0 / acc;
    }
}

// SELL values from a CSR source: out[e] = s1 in1[src[e]] + s2 in2[src[e]]
// (0 on padding).
__global__ void k_sell_fill(long long n_stored, const int* src, const double* in1, double s1,
                            const double* in2, double s2, double* out) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= n_stored) return;
    const int t = src[e];
    double v = 0.0;
    if (t >= 0) {
        v = s1 * in1[t];
        if (in2) v += s2 * in2[t];
    }
    out[e] = v;
}

__global__ void k_to_f32(long long n, const double* in, float* out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

// bf16 bit patterns (round to nearest even) of FP64 values
__global__ void k_to_bf16(long long n, const double* in, unsigned short* out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = __bfloat16_as_ushort(__float2bfloat16_rn((float)in[i]));
}

__global__ void k_sell_dinv(int n, const int* diag, const double* val, double* dinv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dinv[i] = 1.0 / val[diag[i]];
}

__global__ void k_points32(int q_lat, int q_bot, const double* lat64, const double* bot64,
                           double x_ref, double y_ref, double z_top, float* lat32,
                           float* bot32) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < q_lat) {
        const double dz = lat64[2 * q_lat + q] - z_top;
        lat32[0 * q_lat + q] = (float)(lat64[0 * q_lat + q] - x_ref);
        lat32[1 * q_lat + q] = (float)(lat64[1 * q_lat + q] - y_ref);
        lat32[2 * q_lat + q] = (float)(dz * dz);
        lat32[3 * q_lat + q] = (float)(lat64[5 * q_lat + q] * dz);
        lat32[4 * q_lat + q] = (float)lat64[3 * q_lat + q];
        lat32[5 * q_lat + q] = (float)lat64[4 * q_lat + q];
    }
    if (q < q_bot) {
        const double dz = bot64[2 * q_bot + q] - z_top;
        bot32[0 * q_bot + q] = (float)(bot64[0 * q_bot + q] - x_ref);
        bot32[1 * q_bot + q] = (float)(bot64[1 * q_bot + q] - y_ref);
        bot32[2 * q_bot + q] = (float)(dz * dz);
    }
}


// ---------------------------------------------------------------------------
// reconstruction T = T~ + T^ at physical points (Section 2.4)
// ---------------------------------------------------------------------------
__device__ int find_span(const double* U, int p, int n, double u) {
    if (u >= U[n]) {
        int s = n - 1;
        while (s > p && U[s] == U[s + 1]) --s;
        return s;
    }
    if (u <= U[p]) return p;
    int lo = p, hi = n;                 // U[lo] <= u < U[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (U[mid] <= u)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__device__ void eval_at(const DevPatch& dp, const double xi[3], Basis1D& b, double x[3],
                        double J[3][3], double& W) {
    for (int d = 0; d < 3; ++d) {
        b.s[d] = find_span(dp.U[d], dp.p[d], dp.n[d], xi[d]);
        bspline_1d(dp.U[d], dp.p[d], b.s[d], xi[d], b.N[d], b.dN[d]);
    }
    double dW[3];
    nurbs_point(dp, b, x, J, W, dW);
}

// eval_at by one warp: every lane evaluates the 1-D bases, the lanes share
// the (p0+1)(p1+1)(p2+1) tensor-product terms, and the sums (W, dW, x W,
// d(x W)) are formed by an xor butterfly (the same value on every lane).
__device__ void eval_at_warp(const DevPatch& dp, const double xi[3], Basis1D& b, double x[3],
                             double J[3][3], double& Wsum) {
    const int lane = threadIdx.x & 31;
    for (int d = 0; d < 3; ++d) {
        b.s[d] = find_span(dp.U[d], dp.p[d], dp.n[d], xi[d]);
        bspline_1d(dp.U[d], dp.p[d], b.s[d], xi[d], b.N[d], b.dN[d]);
    }
    const int n0 = dp.p[0] + 1, n1 = dp.p[1] + 1, nb = n0 * n1 * (dp.p[2] + 1);
    double v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = 0.0;
    for (int l = lane; l < nb; l += 32) {
        const int a0 = l % n0, a1 = (l / n0) % n1, a2 = l / (n0 * n1);
        const double4 c = dp.cw[nat_index(dp, b.s[0] - dp.p[0] + a0, b.s[1] - dp.p[1] + a1,
                                          b.s[2] - dp.p[2] + a2)];
        const double Nv = b.N[0][a0] * b.N[1][a1] * b.N[2][a2];
        const double dd[3] = {b.dN[0][a0] * b.N[1][a1] * b.N[2][a2],
                              b.N[0][a0] * b.dN[1][a1] * b.N[2][a2],
                              b.N[0][a0] * b.N[1][a1] * b.dN[2][a2]};
        const double wN = c.w * Nv;
        const double P[3] = {c.x, c.y, c.z};
        v[0] += wN;
#pragma unroll
        for (int d = 0; d < 3; ++d) v[1 + d] += c.w * dd[d];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            v[4 + cc] += wN * P[cc];
#pragma unroll
            for (int d = 0; d < 3; ++d) v[7 + 3 * cc + d] += c.w * dd[d] * P[cc];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    Wsum = v[0];
    for (int cc = 0; cc < 3; ++cc) {
        x[cc] = v[4 + cc] / Wsum;
        for (int d = 0; d < 3; ++d) J[cc][d] = (v[7 + 3 * cc + d] - x[cc] * v[1 + d]) / Wsum;
    }
}

// FP32 counterparts for the first Newton phase of the point inversion (FP64
// arithmetic is slow on this part): knots staged as FP32 in shared memory,
// control points relative to the patch's reference point.
constexpr int kEvalKnots = 512;   // knots per direction that the staging holds

struct BasisF {
    float N[3][SA_MAX_DEGREE + 1];
    float dN[3][SA_MAX_DEGREE + 1];
    int s[3];
};

__device__ int find_span_f(const float* U, int p, int n, float u) {
    if (u >= U[n]) {
        int s = n - 1;
        while (s > p && U[s] == U[s + 1]) --s;
        return s;
    }
    if (u <= U[p]) return p;
    int lo = p, hi = n;                 // U[lo] <= u < U[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (U[mid] <= u)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// The recursion of bspline_1d in FP32 (the span is non-empty in FP32, so no
// denominator vanishes).
__device__ void bspline_1d_f(const float* U, int p, int s, float u, float* N, float* dN) {
    float cur[SA_MAX_DEGREE + 1], prev[SA_MAX_DEGREE + 1];
    cur[0] = 1.0f;
    for (int q = 1; q <= p; ++q) {
        for (int r = 0; r < q; ++r) prev[r] = cur[r];
        for (int r = 0; r <= q; ++r) {
            const int i = s - q + r;
            float v = 0.0f;
            if (r > 0) v += (u - U[i]) / (U[i + q] - U[i]) * prev[r - 1];
            if (r < q) v += (U[i + q + 1] - u) / (U[i + q + 1] - U[i + 1]) * prev[r];
            cur[r] = v;
        }
    }
    for (int r = 0; r <= p; ++r) {
        N[r] = cur[r];
        if (p == 0) {
            dN[r] = 0.0f;
            continue;
        }
        const int i = s - p + r;
        float d = 0.0f;
        if (r > 0) d += p / (U[i + p] - U[i]) * prev[r - 1];
        if (r < p) d -= p / (U[i + p + 1] - U[i + 1]) * prev[r];
        dN[r] = d;
    }
}

__device__ inline float det3f(const float J[3][3]) {
    return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

// eval_at_warp in FP32: x relative to ref; sU holds the three knot vectors
// at stride kEvalKnots.
__device__ void eval_at_warp_f(const DevPatch& dp, const float* sU, const double ref[3],
                               const float xi[3], BasisF& b, float x[3], float J[3][3],
                               float& Wsum) {
    const int lane = threadIdx.x & 31;
    for (int d = 0; d < 3; ++d) {
        b.s[d] = find_span_f(sU + d * kEvalKnots, dp.p[d], dp.n[d], xi[d]);
        bspline_1d_f(sU + d * kEvalKnots, dp.p[d], b.s[d], xi[d], b.N[d], b.dN[d]);
    }
    const int n0 = dp.p[0] + 1, n1 = dp.p[1] + 1, nb = n0 * n1 * (dp.p[2] + 1);
    float v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = 0.0f;
    for (int l = lane; l < nb; l += 32) {
        const int a0 = l % n0, a1 = (l / n0) % n1, a2 = l / (n0 * n1);
        const double4 c = dp.cw[nat_index(dp, b.s[0] - dp.p[0] + a0, b.s[1] - dp.p[1] + a1,
                                          b.s[2] - dp.p[2] + a2)];
        const float cw = (float)c.w;
        const float P[3] = {(float)(c.x - ref[0]), (float)(c.y - ref[1]), (float)(c.z - ref[2])};
        const float Nv = b.N[0][a0] * b.N[1][a1] * b.N[2][a2];
        const float dd[3] = {b.dN[0][a0] * b.N[1][a1] * b.N[2][a2],
                             b.N[0][a0] * b.dN[1][a1] * b.N[2][a2],
                             b.N[0][a0] * b.N[1][a1] * b.dN[2][a2]};
        const float wN = cw * Nv;
        v[0] += wN;
#pragma unroll
        for (int d = 0; d < 3; ++d) v[1 + d] += cw * dd[d];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            v[4 + cc] += wN * P[cc];
#pragma unroll
            for (int d = 0; d < 3; ++d) v[7 + 3 * cc + d] += cw * dd[d] * P[cc];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    Wsum = v[0];
    const float iW = 1.0f / Wsum;
    for (int cc = 0; cc < 3; ++cc) {
        x[cc] = v[4 + cc] * iW;
        for (int d = 0; d < 3; ++d) J[cc][d] = (v[7 + 3 * cc + d] - x[cc] * v[1 + d]) * iW;
    }
}

__global__ void k_elem_centers(DevPatch dp, double* ecent) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int nel = dp.ne[0] * dp.ne[1] * dp.ne[2];
    if (e >= nel) return;
    const int es[3] = {e % dp.ne[0], (e / dp.ne[0]) % dp.ne[1], e / (dp.ne[0] * dp.ne[1])};
    double xi[3];
    for (int d = 0; d < 3; ++d) {
        const int s = dp.espan[d][es[d]];
        xi[d] = 0.5 * (dp.U[d][s] + dp.U[d][s + 1]);
    }
    Basis1D b;
    double x[3], J[3][3], W;
    eval_at(dp, xi, b, x, J, W);
    ecent[3 * e + 0] = x[0];
    ecent[3 * e + 1] = x[1];
    ecent[3 * e + 2] = x[2];
}

struct EvalArgs {
    DevPatch dp;
    const double* pts;
    int n;
    const double* ecent;
    const float* ecent32;      // FP32 copy of the centres (search only), or null
    const int* perm;
    const double* That;
    const double4* s64T;       // FP64 coefficients (sx, sy, a, c), or
    const float4* s32T;        // FP32 ones (sx, sy, -a log2 e, log2 c): mixed contexts
    int n_active;
    double x_ref, y_ref, z_top, scale;
    double* T_out;
    // heat-loss rates instead of T (nrm non-null): q~ = -k n . grad T~ into
    // T_out, q^ = -k n . grad T^ into q_hat; the sources' (.., g) tables
    const double* nrm;
    const double4* s64F;
    const float4* s32F;
    double k;
    double* q_hat;
};

constexpr int kEvalThreads = 512;   // the element search dominates a point's latency
constexpr int kEvalStride = 4;      // coarse search: every 4th element per direction
constexpr int kEvalFine = 8;        // then the elements within 8 of the best, per direction
constexpr int kEvalCoarseMin = 4096;   // elements above which the search is coarse to fine

__device__ __forceinline__ float eval_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Block-wide nearest element centre to xs among the elements (i, j, k) with
// lo[d] <= . <= hi[d], every st[d]-th (FP32 when a copy of the centres is
// given: the centre only seeds Newton).  Ties go to the lowest element
// index.  Every thread of the block calls it; the result is also left in
// *s_best.
__device__ int nearest_centre(const EvalArgs& a, const double xs[3], const int lo[3],
                              const int hi[3], const int st[3], double* s_d, int* s_e,
                              int* s_best) {
    const DevPatch& dp = a.dp;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int m0 = (hi[0] - lo[0]) / st[0] + 1, m1 = (hi[1] - lo[1]) / st[1] + 1;
    const int nc = m0 * m1 * ((hi[2] - lo[2]) / st[2] + 1);
    auto elem = [&](int c) {
        const int i = lo[0] + (c % m0) * st[0], j = lo[1] + ((c / m0) % m1) * st[1],
                  k = lo[2] + (c / (m0 * m1)) * st[2];
        return (k * dp.ne[1] + j) * dp.ne[0] + i;
    };
    int best = 0x7fffffff;
    double bd = 1e300;
    if (a.ecent32) {
        const float x0 = (float)xs[0], x1 = (float)xs[1], x2 = (float)xs[2];
        float bf = 3.0e38f;
        for (int c = threadIdx.x; c < nc; c += kEvalThreads) {
            const int e = elem(c);
            const float dx = a.ecent32[3 * e] - x0, dy = a.ecent32[3 * e + 1] - x1,
                        dz = a.ecent32[3 * e + 2] - x2;
            const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (d2 < bf) {
                bf = d2;
                best = e;
            }
        }
        bd = bf;
    } else {
        for (int c = threadIdx.x; c < nc; c += kEvalThreads) {
            const int e = elem(c);
            const double dx = a.ecent[3 * e] - xs[0], dy = a.ecent[3 * e + 1] - xs[1],
                         dz = a.ecent[3 * e + 2] - xs[2];
            const double d2 = dx * dx + dy * dy + dz * dz;
            if (d2 < bd) {
                bd = d2;
                best = e;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double od = __shfl_xor_sync(0xffffffffu, bd, o);
        const int ob = __shfl_xor_sync(0xffffffffu, best, o);
        if (od < bd || (od == bd && ob < best)) {
            bd = od;
            best = ob;
        }
    }
    if (lane == 0) {
        s_d[w] = bd;
        s_e[w] = best;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kEvalThreads / 32; ++k)
            if (s_d[k] < bd || (s_d[k] == bd && s_e[k] < best)) {
                bd = s_d[k];
                best = s_e[k];
            }
        *s_best = best;
    }
    __syncthreads();
    return *s_best;
}

// One block per query point: the threads search the element centres (in
// FP32 when a copy is given: the centre only seeds Newton) and sum the
// sources; warp 0 runs the Newton iteration (the basis terms over its
// lanes), first in FP32 to 1e-6 of the patch size, then in FP64 to 1e-13 of
// it.  With FP32 source tables (mixed contexts) and no flux the FP32 point
// and its FP32 basis give T^; a point the FP32 phase does not settle goes
// the FP64 way from the element centre.  Reductions in a fixed order (ties
// of the search: lowest element index).
__global__ void __maxnreg__(96) k_eval(EvalArgs a) {
    const int t = blockIdx.x;
    if (t >= a.n) return;
    __shared__ double s_d[kEvalThreads / 32];
    __shared__ int s_e[kEvalThreads / 32];
    __shared__ double s_T[kEvalThreads / 32];
    __shared__ int s_best;
    __shared__ double s_That;
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const DevPatch& dp = a.dp;
    const double xs[3] = {a.pts[3 * t], a.pts[3 * t + 1], a.pts[3 * t + 2]};
    // FP32 copies of the knot vectors (read after the search's barriers)
    __shared__ float sU[3 * kEvalKnots];
    const bool use32 = dp.n[0] + dp.p[0] + 1 <= kEvalKnots && dp.n[1] + dp.p[1] + 1 <= kEvalKnots &&
                       dp.n[2] + dp.p[2] + 1 <= kEvalKnots;
    if (use32)
        for (int d = 0; d < 3; ++d)
            for (int i = threadIdx.x; i < dp.n[d] + dp.p[d] + 1; i += kEvalThreads)
                sU[d * kEvalKnots + i] = (float)dp.U[d][i];
    // initial guess: parametric centre of the element with the nearest
    // physical centre.  Large patches: coarse to fine (every kEvalStride-th
    // element per direction, then the elements within kEvalFine of the best
    // of them); a point whose Newton iteration fails from that seed is
    // searched again over every element.
    const int nel = dp.ne[0] * dp.ne[1] * dp.ne[2];
    const bool coarse = nel > kEvalCoarseMin;
    for (int attempt = 0; attempt < 2; ++attempt) {
        int blo[3], bhi[3], bst[3];   // the element box searched
        for (int d = 0; d < 3; ++d) {
            blo[d] = 0;
            bhi[d] = dp.ne[d] - 1;
            bst[d] = 1;
        }
        if (attempt == 0 && coarse) {
            for (int d = 0; d < 3; ++d) {
                bst[d] = kEvalStride;
                blo[d] = min(kEvalStride / 2, dp.ne[d] - 1);
            }
            const int ec = nearest_centre(a, xs, blo, bhi, bst, s_d, s_e, &s_best);
            const int ic[3] = {ec % dp.ne[0], (ec / dp.ne[0]) % dp.ne[1], ec / (dp.ne[0] * dp.ne[1])};
            for (int d = 0; d < 3; ++d) {
                blo[d] = max(0, ic[d] - kEvalFine);
                bhi[d] = min(dp.ne[d] - 1, ic[d] + kEvalFine);
                bst[d] = 1;
            }
        }
        nearest_centre(a, xs, blo, bhi, bst, s_d, s_e, &s_best);
        if (w == 0) {
            // Newton on x(xi) = x*, clamped to the parametric box, by warp 0
            const int best = s_best;
            const int es[3] = {best % dp.ne[0], (best / dp.ne[0]) % dp.ne[1],
                               best / (dp.ne[0] * dp.ne[1])};
            double xi[3], lo[3], hi[3];
            for (int d = 0; d < 3; ++d) {
                const int s = dp.espan[d][es[d]];
                xi[d] = 0.5 * (dp.U[d][s] + dp.U[d][s + 1]);
                lo[d] = dp.U[d][dp.p[d]];
                hi[d] = dp.U[d][dp.n[d]];
            }
            bool ok32 = false;
            BasisF bf;
            float Wf = 1.0f, xf[3];
            if (use32) {
                const double ref[3] = {a.x_ref, a.y_ref, a.z_top};
                const float xr[3] = {(float)(xs[0] - ref[0]), (float)(xs[1] - ref[1]),
                                     (float)(xs[2] - ref[2])};
                float lof[3], hif[3];
                for (int d = 0; d < 3; ++d) {
                    xf[d] = (float)xi[d];
                    lof[d] = sU[d * kEvalKnots + dp.p[d]];
                    hif[d] = sU[d * kEvalKnots + dp.n[d]];
                }
                const float tol32 = 1e-6f * (float)a.scale;
                for (int it = 0; it < 30; ++it) {
                    float x32[3], J32[3][3];
                    eval_at_warp_f(dp, sU, ref, xf, bf, x32, J32, Wf);
                    const float f[3] = {xr[0] - x32[0], xr[1] - x32[1], xr[2] - x32[2]};
                    if (sqrtf(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]) <= tol32) {
                        ok32 = true;
                        break;
                    }
                    const float det = det3f(J32);
                    if (!(fabsf(det) > 0.0f)) break;
                    float dxi[3];
                    for (int c = 0; c < 3; ++c) {
                        float Jc[3][3];
                        for (int r = 0; r < 3; ++r)
                            for (int k = 0; k < 3; ++k) Jc[r][k] = (k == c) ? f[r] : J32[r][k];
                        dxi[c] = det3f(Jc) / det;
                    }
                    for (int d = 0; d < 3; ++d) xf[d] = fminf(hif[d], fmaxf(lof[d], xf[d] + dxi[d]));
                }
            }
            const bool done32 = ok32 && a.s32T && !a.nrm;
            if (done32) {
                // T^ = sum_a R_a T^_a with the FP32 basis, the terms over the lanes
                const int n0 = dp.p[0] + 1, n1 = dp.p[1] + 1, nb = n0 * n1 * (dp.p[2] + 1);
                const float iW = 1.0f / Wf;
                double part = 0.0;
                for (int l = lane; l < nb; l += 32) {
                    const int a0 = l % n0, a1 = (l / n0) % n1, a2 = l / (n0 * n1);
                    const int nat = nat_index(dp, bf.s[0] - dp.p[0] + a0, bf.s[1] - dp.p[1] + a1,
                                              bf.s[2] - dp.p[2] + a2);
                    const float R = (float)dp.cw[nat].w * bf.N[0][a0] * bf.N[1][a1] * bf.N[2][a2] * iW;
                    part += (double)R * a.That[a.perm[nat]];
                }
    #pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                if (lane == 0) {
                    s_That = part;
                    s_ok = 1;
                }
            }
            if (ok32)
                for (int d = 0; d < 3; ++d) xi[d] = (double)xf[d];
            Basis1D b;
            double x[3], J[3][3], W;
            double res = 1e300;
            for (int it = 0; it < 60 && !done32; ++it) {
                eval_at_warp(dp, xi, b, x, J, W);
                const double f[3] = {xs[0] - x[0], xs[1] - x[1], xs[2] - x[2]};
                res = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
                if (res <= 1e-13 * a.scale) break;
                const double det = det3(J);
                if (!(fabs(det) > 0.0)) break;
                double dxi[3];
                for (int c = 0; c < 3; ++c) {
                    double Jc[3][3];
                    for (int r = 0; r < 3; ++r)
                        for (int k = 0; k < 3; ++k) Jc[r][k] = (k == c) ? f[r] : J[r][k];
                    dxi[c] = det3(Jc) / det;
                }
                for (int d = 0; d < 3; ++d) xi[d] = fmin(hi[d], fmax(lo[d], xi[d] + dxi[d]));
            }
            if (lane == 0 && !done32) {
                const int ok = res <= 1e-9 * a.scale;
                const double iW = 1.0 / W;
                double That = 0.0;
                if (ok)
                    for (int a2 = 0; a2 <= dp.p[2]; ++a2)
                        for (int a1 = 0; a1 <= dp.p[1]; ++a1)
                            for (int a0 = 0; a0 <= dp.p[0]; ++a0) {
                                const int nat = nat_index(dp, b.s[0] - dp.p[0] + a0,
                                                          b.s[1] - dp.p[1] + a1, b.s[2] - dp.p[2] + a2);
                                const double R = dp.cw[nat].w * b.N[0][a0] * b.N[1][a1] * b.N[2][a2] * iW;
                                That += R * a.That[a.perm[nat]];
                            }
                s_That = That;
                s_ok = ok;
                if (ok && a.nrm) {
                    // grad T^ = J^{-T} sum_a T^_a grad_xi R_a (quotient rule)
                    double Wv = 0.0, dW[3] = {0.0, 0.0, 0.0};
                    for (int a2 = 0; a2 <= dp.p[2]; ++a2)
                        for (int a1 = 0; a1 <= dp.p[1]; ++a1)
                            for (int a0 = 0; a0 <= dp.p[0]; ++a0) {
                                const double w = dp.cw[nat_index(dp, b.s[0] - dp.p[0] + a0,
                                                                 b.s[1] - dp.p[1] + a1,
                                                                 b.s[2] - dp.p[2] + a2)].w;
                                Wv += w * b.N[0][a0] * b.N[1][a1] * b.N[2][a2];
                                dW[0] += w * b.dN[0][a0] * b.N[1][a1] * b.N[2][a2];
                                dW[1] += w * b.N[0][a0] * b.dN[1][a1] * b.N[2][a2];
                                dW[2] += w * b.N[0][a0] * b.N[1][a1] * b.dN[2][a2];
                            }
                    double gxi[3] = {0.0, 0.0, 0.0};
                    for (int a2 = 0; a2 <= dp.p[2]; ++a2)
                        for (int a1 = 0; a1 <= dp.p[1]; ++a1)
                            for (int a0 = 0; a0 <= dp.p[0]; ++a0) {
                                const int nat = nat_index(dp, b.s[0] - dp.p[0] + a0,
                                                          b.s[1] - dp.p[1] + a1, b.s[2] - dp.p[2] + a2);
                                const double w = dp.cw[nat].w;
                                const double Rv = w * b.N[0][a0] * b.N[1][a1] * b.N[2][a2] / Wv;
                                const double dd[3] = {w * b.dN[0][a0] * b.N[1][a1] * b.N[2][a2],
                                                      w * b.N[0][a0] * b.dN[1][a1] * b.N[2][a2],
                                                      w * b.N[0][a0] * b.N[1][a1] * b.dN[2][a2]};
                                const double Ta = a.That[a.perm[nat]];
                                for (int d = 0; d < 3; ++d) gxi[d] += Ta * (dd[d] - Rv * dW[d]) / Wv;
                            }
                    // J^T g = gxi (Cramer)
                    double JT[3][3];
                    for (int r = 0; r < 3; ++r)
                        for (int c = 0; c < 3; ++c) JT[r][c] = J[c][r];
                    const double det = det3(JT);
                    double g[3];
                    for (int c = 0; c < 3; ++c) {
                        double Jc[3][3];
                        for (int r = 0; r < 3; ++r)
                            for (int k = 0; k < 3; ++k) Jc[r][k] = (k == c) ? gxi[r] : JT[r][k];
                        g[c] = det3(Jc) / det;
                    }
                    const double* nv = a.nrm + 3 * t;
                    s_That = -a.k * (nv[0] * g[0] + nv[1] * g[1] + nv[2] * g[2]);
                }
            }
        }
        __syncthreads();   // s_ok written
        if (s_ok || attempt == 1 || !coarse) break;
    }
    if (a.nrm) {
        // q~ = -k dT~/dn, dT~/dn = sum -g exp(-a R^2) n . (x - x_I)
        const double* nv = a.nrm + 3 * t;
        const double px = xs[0] - a.x_ref, py = xs[1] - a.y_ref, dz = xs[2] - a.z_top;
        double Tt = 0.0;
        if (a.s32F) {
            const float fx = (float)px, fy = (float)py, fz2 = (float)(dz * dz);
            const float nx = (float)nv[0], ny = (float)nv[1], nzdz = (float)(nv[2] * dz);
            float acc = 0.0f;
            for (int j = threadIdx.x; j < a.n_active; j += kEvalThreads) {
                const float4 sv = a.s32F[j];
                const float dx = fx - sv.x, dy = fy - sv.y;
                const float e = eval_ex2(fmaf(sv.z, fmaf(dx, dx, fmaf(dy, dy, fz2)), sv.w));
                acc = fmaf(e, fmaf(nx, dx, fmaf(ny, dy, nzdz)), acc);
            }
            Tt = (double)acc;
        } else {
            for (int j = threadIdx.x; j < a.n_active; j += kEvalThreads) {
                const double4 sv = a.s64F[j];
                const double dx = px - sv.x, dy = py - sv.y;
                Tt += sv.w * exp(-sv.z * (dx * dx + dy * dy + dz * dz)) *
                      (nv[0] * dx + nv[1] * dy + nv[2] * dz);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) Tt += __shfl_xor_sync(0xffffffffu, Tt, o);
        if (lane == 0) s_T[w] = Tt;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int k = 0; k < kEvalThreads / 32; ++k) tot += s_T[k];
            a.T_out[t] = s_ok ? a.k * tot : nan("");      // -k * (-sum)
            a.q_hat[t] = s_ok ? s_That : nan("");
        }
        return;
    }
    // the sources: FP32 terms (each thread sums its ~n / 128 in FP32) or FP64
    const double px = xs[0] - a.x_ref, py = xs[1] - a.y_ref, dz = xs[2] - a.z_top;
    double Tt = 0.0;
    if (a.s32T) {
        const float fx = (float)px, fy = (float)py, fz2 = (float)(dz * dz);
        float acc = 0.0f;
        for (int j = threadIdx.x; j < a.n_active; j += kEvalThreads) {
            const float4 sv = a.s32T[j];
            const float dx = fx - sv.x, dy = fy - sv.y;
            acc += eval_ex2(fmaf(sv.z, fmaf(dx, dx, fmaf(dy, dy, fz2)), sv.w));
        }
        Tt = (double)acc;
    } else {
        for (int j = threadIdx.x; j < a.n_active; j += kEvalThreads) {
            const double4 sv = a.s64T[j];
            const double dx = px - sv.x, dy = py - sv.y;
            Tt += sv.w * exp(-sv.z * (dx * dx + dy * dy + dz * dz));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) Tt += __shfl_xor_sync(0xffffffffu, Tt, o);
    if (lane == 0) s_T[w] = Tt;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int k = 0; k < kEvalThreads / 32; ++k) tot += s_T[k];
        a.T_out[t] = s_ok ? tot + s_That : nan("");
    }
}
// Closed patches: every entry of the matrices over control variables is the
// sum of the control-point entries that map to it (P^T M P), in the fixed
// order of the source list.
__global__ void k_merge_csr(long long n, const long long* sptr, const int* sidx, const double* Mc,
                            const double* Kc, double* M, double* K) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= n) return;
    double m = 0.0, k = 0.0;
    for (long long t = sptr[e]; t < sptr[e + 1]; ++t) {
        m += Mc[sidx[t]];
        k += Kc[sidx[t]];
    }
    M[e] = m;
    K[e] = k;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_face_points(const DevPatch& dp, int face, int pa_unused, int pb_unused, int nea,
                               int neb, const int*, const double* xg_a, const double* wg_a,
                               const double* xg_b, const double* wg_b, int q_offset,
                               double* pts64, int q_stride, int with_normal,
                               const int* slot_of_entry, double* w_val, double* coo_R,
                               int* coo_dof, const int* perm, cudaStream_t s) {
    (void)pa_unused;
    (void)pb_unused;
    FaceArgs a;
    a.dp = dp;
    a.d = face / 2;
    a.side = face % 2;
    a.ta = a.d == 0 ? 1 : 0;
    a.tb = a.d == 2 ? 1 : 2;
    a.nea = nea;
    a.neb = neb;
    a.nga = dp.p[a.ta] + 1;
    a.ngb = dp.p[a.tb] + 1;
    for (int g = 0; g < a.nga; ++g) {
        a.xg_a[g] = xg_a[g];
        a.wg_a[g] = wg_a[g];
    }
    for (int g = 0; g < a.ngb; ++g) {
        a.xg_b[g] = xg_b[g];
        a.wg_b[g] = wg_b[g];
    }
    a.q_offset = q_offset;
    a.q_stride = q_stride;
    a.with_normal = with_normal;
    a.pts64 = pts64;
    a.slot = slot_of_entry;
    a.w_val = w_val;
    a.coo_R = coo_R;
    a.coo_dof = coo_dof;
    a.perm = perm;
    const int nq = nea * neb * a.nga * a.ngb;
    if (nq == 0) return cudaSuccess;
    k_face_points<<<(nq + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_element_local(const DevPatch& dp, double rho_cp, double k, const double* xg,
                                 const double* wg, double* Mloc, double* Kloc, int* bad_jac,
                                 cudaStream_t s) {
    ElemArgs a;
    a.dp = dp;
    a.rho_cp = rho_cp;
    a.k = k;
    for (int d = 0; d < 3; ++d)
        for (int g = 0; g <= dp.p[d]; ++g) {
            a.xg[d][g] = xg[d * (SA_MAX_DEGREE + 1) + g];
            a.wg[d][g] = wg[d * (SA_MAX_DEGREE + 1) + g];
        }
    a.Mloc = Mloc;
    a.Kloc = Kloc;
    a.bad_jac = bad_jac;
    const int nloc = (dp.p[0] + 1) * (dp.p[1] + 1) * (dp.p[2] + 1);
    const size_t smem = (size_t)nloc * nloc * 4 * sizeof(double) + nloc * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_element_local,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nel = dp.ne[0] * dp.ne[1] * dp.ne[2];
    k_element_local<<<nel, 128, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_merge_csr(long long n, const long long* sptr, const int* sidx, const double* Mc,
                             const double* Kc, double* M, double* K, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_merge_csr<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, sptr, sidx, Mc, Kc, M, K);
    return cudaGetLastError();
}

cudaError_t launch_mk_gather(const DevPatch& dp, const long long* ptr, const int* col,
                             const int* const* elo, const int* const* ehi, const double* Mloc,
                             const double* Kloc, double* M, double* K, cudaStream_t s) {
    GatherArgs a;
    a.dp = dp;
    a.ptr = ptr;
    a.col = col;
    for (int d = 0; d < 3; ++d) {
        a.elo[d] = elo[d];
        a.ehi[d] = ehi[d];
    }
    a.Mloc = Mloc;
    a.Kloc = Kloc;
    a.M = M;
    a.K = K;
    const int n_dof = dp.n[0] * dp.n[1] * dp.n[2];
    const long long threads = (long long)n_dof * 32;
    k_mk_gather<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mbot_fill(int n_rows, const int* mptr, const int* mcol, const int* wptr,
                             const int* wcol, const double* wval, const int* coo_dof,
                             const double* coo_R, int nfb, int n_free, double* mval,
                             double* dinv, cudaStream_t s) {
    if (n_rows == 0) return cudaSuccess;
    k_mbot_fill<<<(n_rows + 127) / 128, 128, 0, s>>>(n_rows, mptr, mcol, wptr, wcol, wval,
                                                     coo_dof, coo_R, nfb, n_free, mval, dinv);
    return cudaGetLastError();
}

cudaError_t launch_sell_fill(long long n_stored, const int* src, const double* in1, double s1,
                            const double* in2, double s2, double* out, cudaStream_t s) {
    if (n_stored == 0) return cudaSuccess;
    k_sell_fill<<<(unsigned)((n_stored + 255) / 256), 256, 0, s>>>(n_stored, src, in1, s1, in2, s2,
                                                                  out);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(long long n, const double* in, unsigned short* out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, in, out);
    return cudaGetLastError();
}

cudaError_t launch_to_f32(long long n, const double* in, float* out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, in, out);
    return cudaGetLastError();
}

cudaError_t launch_sell_dinv(int n, const int* diag, const double* val, double* dinv,
                             cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_sell_dinv<<<(n + 255) / 256, 256, 0, s>>>(n, diag, val, dinv);
    return cudaGetLastError();
}

cudaError_t launch_points32(int q_lat, int q_bot, const double* lat64, const double* bot64,
                            double x_ref, double y_ref, double z_top, float* lat32,
                            float* bot32, cudaStream_t s) {
    const int q = q_lat > q_bot ? q_lat : q_bot;
    if (q == 0) return cudaSuccess;
    k_points32<<<(q + 255) / 256, 256, 0, s>>>(q_lat, q_bot, lat64, bot64, x_ref, y_ref, z_top,
                                               lat32, bot32);
    return cudaGetLastError();
}

cudaError_t launch_elem_centers(const DevPatch& dp, double* ecent, cudaStream_t s) {
    const int nel = dp.ne[0] * dp.ne[1] * dp.ne[2];
    k_elem_centers<<<(nel + 127) / 128, 128, 0, s>>>(dp, ecent);
    return cudaGetLastError();
}

cudaError_t launch_eval_points(const DevPatch& dp, const double* pts, int n, const double* ecent,
                               const int* perm, const double* That, const double4* s64T,
                               int n_active, double x_ref, double y_ref, double z_top,
                               double scale, double* T_out, cudaStream_t s, const float* ecent32,
                               const float4* s32T, const EvalFlux* flux) {
    if (n == 0) return cudaSuccess;
    EvalArgs a{dp, pts, n, ecent, ecent32, perm, That, s64T, s32T, n_active, x_ref, y_ref,
               z_top, scale, T_out,
               flux ? flux->nrm : nullptr, flux ? flux->s64F : nullptr,
               flux ? flux->s32F : nullptr, flux ? flux->k : 0.0, flux ? flux->q_hat : nullptr};
    k_eval<<<(unsigned)n, kEvalThreads, 0, s>>>(a);
    return cudaGetLastError();
}
