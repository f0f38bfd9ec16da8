"""Correction-field time stepping (Sections 2.1-2.4).

Per step n -> n+1, in the paper's order:

1. T~ and dT~/dn at the boundary quadrature points from all sources active
   at t_{n+1} (Eqs. sum-of-point-temp, semi-temperature).
2. Neumann data q_N = k dT~/dn on the lateral faces (Eq. that-bc-n) and
   F_i^{n+1} = int_lat (-q_N) N_i dS (Section 2.3).
3. Dirichlet data T_c - T~ on the bottom face (Eq. that-bc-d), imposed on the
   bottom control variables as its L2 projection (reading R5).
4. Theta-scheme (Eq. theta-method):
       (M/dt + theta K) T^{n+1} = (M/dt - (1-theta) K) T^n
                                  + theta F^{n+1} + (1-theta) F^n
   with the Dirichlet control variables eliminated (lifting), solved by a
   sparse LU factorisation of the free block (a library direct solver,
   factored once per (dt, theta)).
5. T^{n+1} = T~^{n+1} + T^^{n+1} at requested points (Section 2.4).

Initial state: T^(x, 0) = T_c (Section 2.1), hence T^^0 = T_c at every control
variable (constants are reproduced exactly by the basis), F^0 = 0.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import assembly, pointsource, sources
from .geometry import PatchGeom

FACE_NEUMANN = 1
FACE_DIRICHLET = 2


class ThetaSolver:
    """theta-scheme for M dT/dt + K T = F with T fixed on ``dir_mask``."""

    def __init__(self, M, K, dir_mask, dt, theta, direct=True, cg_tol=1e-14):
        self.dt, self.theta = dt, theta
        self.A = (M / dt + theta * K).tocsr()
        self.B = (M / dt - (1.0 - theta) * K).tocsr()
        self.dir = np.asarray(dir_mask, bool)
        self.free = ~self.dir
        self.A_ff = self.A[self.free][:, self.free].tocsc()
        self.A_fd = self.A[self.free][:, self.dir].tocsr()
        self.direct = direct
        self.cg_tol = cg_tol
        self.lu = spla.splu(self.A_ff) if direct else None

    def rhs(self, T_n, F_n, F_np1, g_np1):
        """Right-hand side of the free block."""
        r = self.B @ T_n + self.theta * F_np1 + (1.0 - self.theta) * F_n
        return r[self.free] - self.A_fd @ g_np1

    def step(self, T_n, F_n, F_np1, g_np1):
        b = self.rhs(T_n, F_n, F_np1, g_np1)
        if self.direct:
            x_f = self.lu.solve(b)
        else:
            x_f, info = spla.cg(self.A_ff, b, x0=T_n[self.free], rtol=self.cg_tol, atol=0.0,
                                maxiter=10000)
            assert info == 0
        T = np.empty_like(T_n)
        T[self.free] = x_f
        T[self.dir] = g_np1
        return T


class Model:
    """The whole method on one patch, FP64, step by step."""

    def __init__(self, workload, s_img=2.0, direct=True, build_solver=True):
        self.wl = workload
        self.mat = workload.material
        self.scan = workload.scan
        self.dt = workload.dt
        self.theta = workload.theta
        self.s_img = s_img
        self.geom = g = PatchGeom(workload.patch)
        rho_cp = self.mat.rho * self.mat.cp
        self.M, self.K = assembly.assemble_MK(g, rho_cp, self.mat.k)
        self.lat = assembly.boundary_points(g, FACE_NEUMANN)
        self.bot = assembly.boundary_points(g, FACE_DIRICHLET)
        self.W_lat = assembly.weight_matrix(g, self.lat) if self.lat is not None else None
        self.W_bot = assembly.weight_matrix(g, self.bot) if self.bot is not None else None
        self.dir = g.dirichlet_dofs()
        self.M_bot_lu = None
        if self.bot is not None:
            Mb = assembly.boundary_mass(g, self.bot)
            self.M_bot = Mb[self.dir][:, self.dir].tocsc()
            self.M_bot_lu = spla.splu(self.M_bot)
        self.xs = sources.discretize(self.scan, self.dt)
        self.E = sources.energy(self.scan, self.dt)
        self.z_top = g.top_z()
        self.solver = ThetaSolver(self.M, self.K, self.dir, self.dt, self.theta,
                                  direct=direct) if build_solver else None
        self.reset()

    # ---- state -------------------------------------------------------------
    def reset(self):
        n = self.geom.n_dof
        self.n = 0
        self.T_hat = np.full(n, self.mat.T_c)
        self.F = np.zeros(n)
        self.last = {}

    def n_active(self, n):
        return min(n, len(self.xs))

    def source_ages(self, n):
        K = self.n_active(n)
        return pointsource.ages(n, K, self.dt, self.mat, self.scan.spot_radius)

    # ---- boundary data (steps 1-3) ----------------------------------------
    def flux_normal_derivative(self, n):
        """dT~/dn at the lateral points at step n."""
        K = self.n_active(n)
        if K == 0 or self.lat is None:
            return np.zeros(0 if self.lat is None else len(self.lat["x"]))
        return pointsource.dTdn_tilde(self.lat["x"], self.lat["n"], self.xs[:K],
                                      self.source_ages(n), self.E, self.mat, self.s_img)

    def T_tilde_at(self, x, n):
        K = self.n_active(n)
        if K == 0:
            return np.zeros(len(x))
        return pointsource.T_tilde(x, self.xs[:K], self.source_ages(n), self.E, self.mat,
                                   self.s_img)

    def neumann_F(self, s_lat):
        """F_i = int_lat (-q_N) N_i dS with q_N = k dT~/dn."""
        if self.W_lat is None:
            return np.zeros(self.geom.n_dof)
        return self.W_lat @ (-self.mat.k * s_lat)

    def dirichlet_g(self, T_tilde_bot):
        """L2 projection of T_c - T~ onto the bottom control variables."""
        if self.M_bot_lu is None:
            return np.zeros(0)
        b = (self.W_bot @ (self.mat.T_c - T_tilde_bot))[self.dir]
        return self.M_bot_lu.solve(b)

    # ---- one theta step (step 4) ------------------------------------------
    def step(self):
        n1 = self.n + 1
        s_lat = self.flux_normal_derivative(n1)
        F1 = self.neumann_F(s_lat)
        Tt_bot = self.T_tilde_at(self.bot["x"], n1) if self.bot is not None else np.zeros(0)
        g1 = self.dirichlet_g(Tt_bot)
        T1 = self.solver.step(self.T_hat, self.F, F1, g1)
        self.last = dict(s_lat=s_lat, F=F1, Tt_bot=Tt_bot, g=g1)
        self.T_hat, self.F, self.n = T1, F1, n1
        return T1

    def run(self, n_steps):
        for _ in range(n_steps):
            self.step()
        return self.T_hat

    # ---- reconstruction (step 5) --------------------------------------------
    def eval_T(self, xi_pts):
        """T = T~ + T^ at parametric points xi (P,3) at the current step."""
        xi_pts = np.atleast_2d(xi_pts)
        x = np.array([self.geom.point(xi) for xi in xi_pts])
        That = np.array([np.dot(self.geom.local_eval(xi)[1],
                                self.T_hat[self.geom.local_eval(xi)[0]]) for xi in xi_pts])
        return x, self.T_tilde_at(x, self.n) + That

    def eval_flux(self, xi_pts, nrm):
        """Heat-loss rates at parametric points xi (P,3) with unit normals nrm
        (P,3), current step (Section 3.1): q~ = -k n . grad T~ and
        q^ = -k n . grad T^, grad T^ = sum_a T^_a grad_x R_a with
        grad_x R_a = J^{-T} grad_xi R_a.  Returns x, q~, q^."""
        xi_pts = np.atleast_2d(xi_pts)
        nrm = np.atleast_2d(nrm)
        x, qh = [], []
        for xi, nv in zip(xi_pts, nrm):
            dofs, R, dR, xp, J = self.geom.local_eval(xi)
            gradR = np.linalg.solve(J.T, dR.T).T
            qh.append(-self.mat.k * np.dot(nv, gradR.T @ self.T_hat[dofs]))
            x.append(xp)
        x = np.array(x)
        K = self.n_active(self.n)
        if K == 0:
            qt = np.zeros(len(x))
        else:
            qt = -self.mat.k * pointsource.dTdn_tilde(x, nrm, self.xs[:K], self.source_ages(self.n),
                                                       self.E, self.mat, self.s_img)
        return x, qt, np.array(qh)


class MultiLaserModel(Model):
    """Several lasers on one patch, all switched on at t = 0 with the same
    time step (reading R22): every laser's discretised sources (its own path,
    speed and power; source j of laser l active from step j on) enter the
    same history sums, i.e. T~ and dT~/dn are Eq. sum-of-point-temp summed
    over the lasers, and ONE correction field T^ takes the combined boundary
    data through the theta-scheme.  ``workload`` gives the patch, material,
    dt and theta (its own scan is not used)."""

    def __init__(self, workload, scans, s_img=2.0, direct=True):
        super().__init__(workload, s_img, direct)
        self.lasers = [(sources.discretize(sc, self.dt), sources.energy(sc, self.dt), sc.spot_radius)
                       for sc in scans]

    def _laser_terms(self, n):
        """(positions, ages, E) of the sources of each laser active at step n."""
        out = []
        for xs, E, r in self.lasers:
            K = min(n, len(xs))
            if K > 0:
                out.append((xs[:K], pointsource.ages(n, K, self.dt, self.mat, r), E))
        return out

    def flux_normal_derivative(self, n):
        if self.lat is None:
            return np.zeros(0)
        s = np.zeros(len(self.lat["x"]))
        for xs, age, E in self._laser_terms(n):
            s += pointsource.dTdn_tilde(self.lat["x"], self.lat["n"], xs, age, E, self.mat, self.s_img)
        return s

    def T_tilde_at(self, x, n):
        t = np.zeros(len(x))
        for xs, age, E in self._laser_terms(n):
            t += pointsource.T_tilde(x, xs, age, E, self.mat, self.s_img)
        return t

    def eval_flux(self, xi_pts, nrm):
        """As Model.eval_flux, q~ summed over the lasers."""
        x, _, qh = Model.eval_flux(self, xi_pts, nrm)
        qt = np.zeros(len(x))
        for xs, age, E in self._laser_terms(self.n):
            qt += -self.mat.k * pointsource.dTdn_tilde(x, np.atleast_2d(nrm), xs, age, E, self.mat, self.s_img)
        return x, qt, qh
