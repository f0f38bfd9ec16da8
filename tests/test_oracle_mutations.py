"""Planted mistakes in the oracle, on the CPU: each replaces one oracle
function for the duration of one test by a plausible wrong restatement of
the method (a dropped term, a wrong sign or index, a transposed operand, a
swapped weight), and at least one of the pins named beside it must then
fail.  Nothing here touches the GPU path."""
import numpy as np
import pytest

import tests.test_oracle_pins as pins
from oracle import assembly, bspline, geometry, pointsource, solver, sources


def _caught(calls):
    """True when one of the pin calls fails (an assertion, or arithmetic the
    mistake makes impossible)."""
    for fn, args in calls:
        try:
            fn(*args)
        except (AssertionError, ArithmeticError, np.linalg.LinAlgError):
            return True
    return False


# ---- the planted mistakes ---------------------------------------------------
def _ages_without_tau_shift(n, n_active, dt, mat, spot_radius):
    I = np.arange(1, n_active + 1, dtype=np.float64)
    return (n - I) * dt + 1e-12


def _T_point_wrong_power(x, xs, age, E, mat, s_img=2.0):
    alpha = pointsource.diffusivity(mat)
    d = x[:, None, :] - xs[None, :, :]
    R2 = np.einsum("qkc,qkc->qk", d, d)
    pref = s_img * E / (mat.rho * mat.cp * (4.0 * np.pi * alpha * age) ** 1.0)
    return pref[None, :] * np.exp(-R2 / (4.0 * alpha * age[None, :]))


_T_point = pointsource.T_point


def _gradT_wrong_sign(x, xs, age, E, mat, s_img=2.0):
    alpha = pointsource.diffusivity(mat)
    d = x[:, None, :] - xs[None, :, :]
    return d / (2.0 * alpha * age[None, :, None]) * _T_point(x, xs, age, E, mat, s_img)[:, :, None]


def _energy_without_absorptivity(scan, dt):
    return scan.power * dt


def _neumann_F_wrong_sign(self, s_lat):
    if self.W_lat is None:
        return np.zeros(self.geom.n_dof)
    return self.W_lat @ (self.mat.k * s_lat)


def _rhs_swapped_theta(self, T_n, F_n, F_np1, g_np1):
    r = self.B @ T_n + (1.0 - self.theta) * F_np1 + self.theta * F_n
    return r[self.free] - self.A_fd @ g_np1


def _dirichlet_g_without_mass_solve(self, T_tilde_bot):
    if self.M_bot_lu is None:
        return np.zeros(0)
    return (self.W_bot @ (self.mat.T_c - T_tilde_bot))[self.dir]


def _element_matrices_J_not_transposed(geom, elem, rho_cp, k):
    Me = Ke = dofs = None
    for xi, wt in geom.element_quadrature(elem):
        dofs, R, dR, x, J = geom.local_eval(xi, [elem[d][2] for d in range(3)])
        wq = wt * np.linalg.det(J)
        gradR = np.linalg.solve(J, dR.T).T
        m = rho_cp * wq * np.outer(R, R)
        kk = k * wq * (gradR @ gradR.T)
        Me = m if Me is None else Me + m
        Ke = kk if Ke is None else Ke + kk
    return dofs, Me, Ke


_span_index = bspline.span_index


def _span_one_left(U, p, u):
    s = _span_index(U, p, u)
    return max(p, s - 1) if U[p] < u < U[len(U) - p - 1] else s


_local_eval = geometry.PatchGeom.local_eval


def _local_eval_without_weights(self, xi, spans=None):
    w = self.w
    self.w = np.ones_like(w)
    try:
        return _local_eval(self, xi, spans)
    finally:
        self.w = w


_eval_flux = solver.Model.eval_flux


def _eval_flux_wrong_q_tilde_sign(self, xi_pts, nrm):
    x, qt, qh = _eval_flux(self, xi_pts, nrm)
    return x, -qt, qh


_model_init = solver.Model.__init__


def _model_full_space(self, workload, s_img=2.0, direct=True, build_solver=True):
    _model_init(self, workload, s_img=1.0, direct=direct, build_solver=build_solver)


_ages = pointsource.ages


def _ages_one_step_old(n, n_active, dt, mat, spot_radius):
    return _ages(n + 1, n_active, dt, mat, spot_radius)


_discretize = sources.discretize


def _sources_one_step_late(scan, dt):
    return _discretize(scan, dt)[1:]


def _dirichlet_g_wrong_sign(self, T_tilde_bot):
    if self.M_bot_lu is None:
        return np.zeros(0)
    return self.M_bot_lu.solve((self.W_bot @ (self.mat.T_c + T_tilde_bot))[self.dir])


def _element_matrices_without_detJ(geom, elem, rho_cp, k):
    Me = Ke = dofs = None
    for xi, wt in geom.element_quadrature(elem):
        dofs, R, dR, x, J = geom.local_eval(xi, [elem[d][2] for d in range(3)])
        gradR = np.linalg.solve(J.T, dR.T).T
        m = rho_cp * wt * np.outer(R, R)
        kk = k * wt * (gradR @ gradR.T)
        Me = m if Me is None else Me + m
        Ke = kk if Ke is None else Ke + kk
    return dofs, Me, Ke


def _eval_flux_J_not_transposed(self, xi_pts, nrm):
    xi_pts = np.atleast_2d(xi_pts)
    nrm = np.atleast_2d(nrm)
    x, qh = [], []
    for xi, nv in zip(xi_pts, nrm):
        dofs, R, dR, xp, J = self.geom.local_eval(xi)
        gradR = np.linalg.solve(J, dR.T).T
        qh.append(-self.mat.k * np.dot(nv, gradR.T @ self.T_hat[dofs]))
        x.append(xp)
    x = np.array(x)
    _, qt, _ = _eval_flux(self, xi_pts, nrm)
    return x, qt, np.array(qh)


_boundary_points = assembly.boundary_points


def _boundary_normals_inward(geom, kind):
    pts = _boundary_points(geom, kind)
    if pts is not None:
        pts = dict(pts)
        pts["n"] = -pts["n"]
    return pts


def _laser_terms_last_laser_dropped(self, n):
    out = []
    for xs, E, r in self.lasers[:-1]:
        K = min(n, len(xs))
        if K > 0:
            out.append((xs[:K], pointsource.ages(n, K, self.dt, self.mat, r), E))
    return out


def _laser_terms_first_laser_energy(self, n):
    out = []
    E0 = self.lasers[0][1]
    for xs, E, r in self.lasers:
        K = min(n, len(xs))
        if K > 0:
            out.append((xs[:K], pointsource.ages(n, K, self.dt, self.mat, r), E0))
    return out


MUTATIONS = {
    "ages one step too old": (
        (pointsource, "ages", _ages_one_step_old),
        [(pins.test_table3_integrated_analytical_heat_loss, ())]),
    "first source one step late on each track": (
        (sources, "discretize", _sources_one_step_late),
        [(pins.test_R1_source_discretisation_counts_and_spacing, ())]),
    "Dirichlet data T_c + T~": (
        (solver.Model, "dirichlet_g", _dirichlet_g_wrong_sign),
        [(pins.test_R5_dirichlet_projection_reproduces_face_space_functions, ())]),
    "det J dropped from the volume quadrature": (
        (assembly, "element_matrices", _element_matrices_without_detJ),
        [(pins.test_P6_symmetry_constants_and_volume_on_curved_nurbs, ())]),
    "grad T^ with J^-1 instead of J^-T": (
        (solver.Model, "eval_flux", _eval_flux_J_not_transposed),
        [(pins.test_heat_loss_rate_is_minus_k_times_the_normal_derivative, ())]),
    "boundary normals pointing inward": (
        (assembly, "boundary_points", _boundary_normals_inward),
        [(pins.test_P9_energy_balance_all_neumann, (1.0,))]),
    "tau shift dropped from the ages": (
        (pointsource, "ages", _ages_without_tau_shift),
        [(pins.test_P4_sum_converges_to_rosenthal, ())]),
    "prefactor (4 pi alpha t)^1 instead of ^1.5": (
        (pointsource, "T_point", _T_point_wrong_power),
        [(pins.test_P1_point_source_equals_heat_kernel_convolution, (3e-5,))]),
    "gradient of T~ with the wrong sign": (
        (pointsource, "gradT_point", _gradT_wrong_sign),
        [(pins.test_P2_heat_equation_and_gradient_by_finite_differences, ())]),
    "absorptivity dropped from E": (
        (sources, "energy", _energy_without_absorptivity),
        [(pins.test_P3_energy_per_source_matches_paper, ())]),
    "Neumann load with the wrong sign": (
        (solver.Model, "neumann_F", _neumann_F_wrong_sign),
        [(pins.test_P9_energy_balance_all_neumann, (1.0,))]),
    "theta weights of F swapped": (
        (solver.ThetaSolver, "rhs", _rhs_swapped_theta),
        [(pins.test_P9_energy_balance_all_neumann, (1.0,))]),
    "bottom projection without the mass-matrix solve": (
        (solver.Model, "dirichlet_g", _dirichlet_g_without_mass_solve),
        [(pins.test_R5_dirichlet_projection_reproduces_face_space_functions, ())]),
    "grad_x R = J^-1 grad_xi R (J not transposed)": (
        (assembly, "element_matrices", _element_matrices_J_not_transposed),
        [(pins.test_P6_patch_test_linear_field_is_reproduced, ())]),
    "knot span one to the left": (
        (bspline, "span_index", _span_one_left),
        [(pins.test_P5_partition_of_unity_and_library_bspline, ())]),
    "NURBS weights dropped": (
        (geometry.PatchGeom, "local_eval", _local_eval_without_weights),
        [(pins.test_P5_table2_arc_is_exact_circle, ())]),
    "q~ with the wrong sign": (
        (solver.Model, "eval_flux", _eval_flux_wrong_q_tilde_sign),
        [(pins.test_heat_loss_rate_is_minus_k_times_the_normal_derivative, ())]),
    "several lasers: the last laser dropped": (
        (solver.MultiLaserModel, "_laser_terms", _laser_terms_last_laser_dropped),
        [(pins.test_R22_multi_laser_superposition_of_single_laser_solves, ())]),
    "several lasers: every laser with the first one's power": (
        (solver.MultiLaserModel, "_laser_terms", _laser_terms_first_laser_energy),
        [(pins.test_R22_multi_laser_superposition_of_single_laser_solves, ())]),
    "full-space kernel (s_img = 1) in the model": (
        (solver.Model, "__init__", _model_full_space),
        [(pins.test_table3_integrated_analytical_heat_loss, ())]),
}


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_planted_mistake_fails_a_pin(name, monkeypatch):
    (target, attr, wrong), calls = MUTATIONS[name]
    # (the same pins pass on the oracle as it stands: test_oracle_pins.py)
    monkeypatch.setattr(target, attr, wrong)
    assert _caught(calls), name
