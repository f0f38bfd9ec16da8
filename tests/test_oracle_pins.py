"""Pins of the FP64 oracle against what the paper and mathematics fix.

None of these compares the oracle with itself: each check uses an
independent route (numerical quadrature of the heat kernel, a library
B-spline routine, Kronecker products of 1-D matrices, textbook closed forms,
conservation identities, convergence rates, values printed in the paper).
"""
import os

import numpy as np
import scipy.sparse.linalg as spla
import pytest
import scipy.integrate as si
import scipy.sparse as sp
from scipy.interpolate import BSpline

import workloads as W
from oracle import assembly, bspline, pointsource, sources
from oracle.geometry import PatchGeom
from oracle.solver import Model, ThetaSolver

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MAT = W.MAT_DEFAULT
MAT_TI = W.MAT_TI64
ALPHA = MAT.k / (MAT.rho * MAT.cp)


def _gh(n):
    return np.polynomial.hermite.hermgauss(n)


# ---------------------------------------------------------------------------
# P1: the tau-shifted point source is a Gaussian spot (1/e^2 radius r,
#     variance r^2/4 per axis) carried forward by the heat kernel
#     (Section 2.1, Eq. semi-temperature and the definition of tau).
# ---------------------------------------------------------------------------
def _conv_1d(xd, s, sigma0, n=80):
    """int G1(xd - y, s) phi1(y) dy by Gauss-Hermite with the narrower of the
    two Gaussians as weight.  G1 = heat kernel of diffusivity ALPHA, phi1 the
    spot profile of variance sigma0^2."""
    u, w = _gh(n)
    var_g = 2.0 * ALPHA * s
    if s == 0.0:
        return np.exp(-xd ** 2 / (2 * sigma0 ** 2)) / np.sqrt(2 * np.pi * sigma0 ** 2)
    if var_g < sigma0 ** 2:
        y = xd + np.sqrt(2 * var_g) * u              # weight: heat kernel around xd
        f = np.exp(-y ** 2 / (2 * sigma0 ** 2)) / np.sqrt(2 * np.pi * sigma0 ** 2)
    else:
        y = np.sqrt(2 * sigma0 ** 2) * u             # weight: spot profile
        f = np.exp(-(xd - y) ** 2 / (4 * ALPHA * s)) / np.sqrt(4 * np.pi * ALPHA * s)
    return np.dot(w, f) / np.sqrt(np.pi)


@pytest.mark.parametrize("t_since", [0.0, 2e-6, 3e-5, 4e-4])
def test_P1_point_source_equals_heat_kernel_convolution(t_since):
    r = 20e-6
    E = 1e-3
    age = np.array([t_since + r * r / (8 * ALPHA)])
    xs = np.zeros((1, 3))
    pts = np.array([[0, 0, 0], [15e-6, -10e-6, -5e-6], [40e-6, 20e-6, -30e-6],
                    [-70e-6, 5e-6, -60e-6]])
    got = pointsource.T_point(pts, xs, age, E, MAT, s_img=1.0)[:, 0]
    sigma0 = r / 2.0
    for q, x in enumerate(pts):
        ref = E / (MAT.rho * MAT.cp)
        for d in range(3):
            ref *= _conv_1d(x[d], t_since, sigma0)
        assert abs(got[q] - ref) <= 1e-11 * abs(ref) + 1e-300, (q, got[q], ref)


# ---------------------------------------------------------------------------
# P2: T~ solves the heat equation; the gradient is its derivative; the normal
#     derivative vanishes on the top plane (Section 2.1).
# ---------------------------------------------------------------------------
def test_P2_heat_equation_and_gradient_by_finite_differences():
    E = 5e-4
    xs = np.array([[0.1e-3, -0.05e-3, 0.0]])
    x0 = np.array([[0.13e-3, -0.02e-3, -0.04e-3]])
    age = np.array([3e-5])
    T = lambda x, a: pointsource.T_point(x, xs, np.array([a]), E, MAT)[0, 0]
    g = pointsource.gradT_point(x0, xs, age, E, MAT)[0, 0]
    h = 1e-8
    lap = 0.0
    for d in range(3):
        e = np.zeros((1, 3))
        e[0, d] = h
        fd = (T(x0 + e, age[0]) - T(x0 - e, age[0])) / (2 * h)
        assert abs(fd - g[d]) < 1e-6 * np.abs(g).max()
        lap += (T(x0 + e, age[0]) - 2 * T(x0, age[0]) + T(x0 - e, age[0])) / h ** 2
    ht = 1e-9
    dTdt = (T(x0, age[0] + ht) - T(x0, age[0] - ht)) / (2 * ht)
    assert abs(dTdt - ALPHA * lap) < 1e-4 * abs(dTdt)
    # normal derivative on the top plane z = z_source vanishes
    xt = np.array([[0.3e-3, 0.1e-3, 0.0]])
    gt = pointsource.gradT_point(xt, xs, age, E, MAT)[0, 0]
    assert gt[2] == 0.0


# ---------------------------------------------------------------------------
# P3: E = A P dt printed in Section 3.1; the half-space integral carries E
#     for s_img = 2 (reading R2) and E/2 for the printed s_img = 1.
# ---------------------------------------------------------------------------
def _golden_kv(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split()[:2]
        out[k] = float(v)
    return out


def test_P3_energy_per_source_matches_paper():
    g = _golden_kv("paper_energy.txt")
    scan = W.straight_track((0, 0, 0), (1e-3, 0, 0), power=g["power_W"],
                            absorptivity=g["absorptivity"], speed=0.5)
    E = sources.energy(scan, g["dt_s"])
    assert round(E, 7) == pytest.approx(g["E_J"], abs=0.005e-4)


@pytest.mark.parametrize("s_img", [1.0, 2.0])
def test_P3_half_space_energy(s_img):
    E = 6.35e-4
    age = np.array([4e-5])
    xs = np.zeros((1, 3))
    u, w = _gh(60)
    sig = np.sqrt(4 * ALPHA * age[0])
    X, Y = np.meshgrid(sig * u, sig * u, indexing="ij")
    WW = np.outer(w, w) * sig * sig * np.exp(np.outer(u * u, np.ones_like(u)) +
                                             np.outer(np.ones_like(u), u * u))

    def fz(z):
        pts = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], axis=1)
        return np.dot(WW.ravel(), pointsource.T_point(pts, xs, age, E, MAT, s_img)[:, 0])

    val, _ = si.quad(fz, -12.0 * sig, 0.0, epsabs=0, epsrel=1e-12, limit=200)
    energy = MAT.rho * MAT.cp * val
    assert energy == pytest.approx(s_img * E / 2.0, rel=1e-9)


# ---------------------------------------------------------------------------
# P4: a long straight track of s_img = 2 sources converges to Rosenthal's
#     quasi-steady moving point-source solution (textbook closed form).
# ---------------------------------------------------------------------------
def test_P4_sum_converges_to_rosenthal():
    """Every tau-shifted source is a point source released r^2/(8 alpha)
    before its activation, so the equivalent continuous laser sits v r^2/(8
    alpha) ahead of the last source.  With that position the sum of equally
    spaced sources reproduces Rosenthal's solution to rounding (the rectangle
    rule is spectrally accurate for this smooth, decaying integrand)."""
    P, A, v, dt = 200.0, 0.4, 1.0, 2e-6
    n_src = 15000                      # 30 mm of track, 30 ms
    L = (n_src - 1) * v * dt
    scan = W.straight_track((0, 0, 0), (L, 0, 0), P, A, v)
    xs = sources.discretize(scan, dt)
    assert len(xs) == n_src
    E = sources.energy(scan, dt)
    age = pointsource.ages(n_src, n_src, dt, MAT, scan.spot_radius)
    x_laser = xs[-1, 0] + v * scan.spot_radius ** 2 / (8 * ALPHA)
    rel = np.array([[-300e-6, 120e-6, -50e-6], [0.0, 250e-6, 0.0], [150e-6, 200e-6, -100e-6],
                    [-600e-6, 0.0, -200e-6], [-250e-6, -250e-6, 0.0], [-100e-6, 60e-6, -60e-6]])
    pts = rel + np.array([xs[-1, 0], 0, 0])
    got = pointsource.T_tilde(pts, xs, age, E, MAT, s_img=2.0)
    d = pts - np.array([x_laser, 0, 0])
    R = np.linalg.norm(d, axis=1)
    ros = A * P / (2 * np.pi * MAT.k * R) * np.exp(-v * (R + d[:, 0]) / (2 * ALPHA))
    np.testing.assert_allclose(got, ros, rtol=1e-10)
    # the printed full-space kernel (s_img = 1) carries half of it
    got1 = pointsource.T_tilde(pts, xs, age, E, MAT, s_img=1.0)
    np.testing.assert_allclose(got1, 0.5 * ros, rtol=1e-10)


def test_R1_source_discretisation_counts_and_spacing():
    wl = W.block_meander(n_tracks=3)
    xs = sources.discretize(wl.scan, wl.dt)
    assert len(xs) == 3 * 584                         # 3.5 mm / 6 um -> 584 per track
    d = np.linalg.norm(np.diff(xs[:584], axis=0), axis=1)
    np.testing.assert_allclose(d, 1.2 * 5e-6, rtol=1e-9)
    # second track runs back, starting at its own start point
    np.testing.assert_allclose(xs[584], [3.75e-3, 1.15e-3, 1e-3], atol=1e-15)
    # contour: arc length continues across vertices of one track
    sc = W.Scan(path=np.array([[0, 0, 0], [1e-4, 0, 0], [1e-4, 1e-4, 0]]),
                seg_on=np.array([1, 1], np.uint8), power=1, absorptivity=1, speed=1.0)
    xc = sources.discretize(sc, 3e-5)
    np.testing.assert_allclose(xc[4], [1e-4, 2e-5, 0], atol=1e-15)
    assert len(xc) == 7


# ---------------------------------------------------------------------------
# P5: basis functions.
# ---------------------------------------------------------------------------
def test_P5_partition_of_unity_and_library_bspline():
    U = np.array([0, 0, 0, 0.2, 0.2, 0.5, 0.7, 1, 1, 1], float)
    p = 2
    n = len(U) - p - 1
    for u in np.linspace(0, 1, 57):
        N, dN = bspline.basis_all_ders(U, p, u)
        assert abs(N.sum() - 1) < 1e-15
        assert abs(dN.sum()) < 1e-12
        for i in range(n):
            c = np.zeros(n)
            c[i] = 1
            spl = BSpline(U, c, p, extrapolate=False)
            ref = spl(u) if u < 1 else BSpline(U, c, p)(u)
            dref = spl.derivative()(u) if u < 1 else BSpline(U, c, p).derivative()(u)
            if u in (0.2,):  # C0 knot: derivative one-sided (right limit) in both
                continue
            assert abs(N[i] - ref) < 1e-14
            assert abs(dN[i] - dref) < 1e-11


def test_P5_bernstein_on_one_element():
    U = np.array([0, 0, 0, 0, 1, 1, 1, 1], float)
    for u in np.linspace(0, 1, 11):
        N, dN = bspline.basis_all_ders(U, 3, u)
        B = [(1 - u) ** 3, 3 * u * (1 - u) ** 2, 3 * u ** 2 * (1 - u), u ** 3]
        dB = [-3 * (1 - u) ** 2, 3 * (1 - u) ** 2 - 6 * u * (1 - u), 6 * u * (1 - u) - 3 * u ** 2,
              3 * u ** 2]
        np.testing.assert_allclose(N, B, atol=1e-15)
        np.testing.assert_allclose(dN, dB, atol=1e-13)


def _table2_patch():
    """Quarter-cylinder part of Table 2 extruded from z = 0 to the printed
    top surface z = 2 mm (unit: m)."""
    rows = []
    kn = {}
    for line in open(os.path.join(GOLDEN, "table2_control_net.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        if f[0].startswith("knots"):
            kn[f[0]] = np.array([float(v) for v in f[1:]])
            continue
        ev = lambda s: float(eval(s, {"sqrt": np.sqrt}))
        rows.append(([ev(v) for v in f[1:4]], [ev(v) for v in f[4:7]]))
    n0 = len(rows)
    ctrl = np.zeros((2, 2, n0, 3))
    for i, (b1, b2) in enumerate(rows):
        for k, z in enumerate((0.0, 2.0)):
            ctrl[k, 0, i] = [b1[0], b1[1], z]
            ctrl[k, 1, i] = [b2[0], b2[1], z]
    wmid = np.cos(np.pi / 8)
    w1 = np.array([1, wmid, 1, wmid, 1.0])
    weights = np.broadcast_to(w1, (2, 2, n0)).copy()
    patch = W.Patch(degree=(2, 1, 1), knots=[kn["knots_xi"], kn["knots_eta"], kn["knots_zeta"]],
                    ctrl=ctrl * 1e-3, weights=weights)
    return patch


def test_P5_table2_arc_is_exact_circle():
    g = PatchGeom(_table2_patch())
    for u in np.linspace(0, 1, 41):
        x = g.point([u, 0.0, 1.0])
        assert abs(np.hypot(x[0] - 2e-3, x[1]) - 1e-3) < 1e-17
        assert abs(x[2] - 2e-3) < 1e-18
        # the ruled surface stays inside the square [0, 2] x [0, 2] mm
        y = g.point([u, 0.5, 0.5])
        assert -1e-15 <= y[0] <= 2e-3 + 1e-15 and -1e-15 <= y[1] <= 2e-3 + 1e-15
    # without the weights the arc is not a circle (the pin can fail)
    p = _table2_patch()
    p.weights = None
    g2 = PatchGeom(p)
    x = g2.point([0.25, 0.0, 1.0])
    assert abs(np.hypot(x[0] - 2e-3, x[1]) - 1e-3) > 1e-6


# ---------------------------------------------------------------------------
# P6: assembly.
# ---------------------------------------------------------------------------
def _bspline_1d_matrices(U, p, L, nq=12):
    """1-D mass and stiffness of B-splines via scipy's BSpline (independent
    of the oracle's Cox-de Boor) and a high-order Gauss rule on each span."""
    n = len(U) - p - 1
    xg, wg = np.polynomial.legendre.leggauss(nq)
    Mx = np.zeros((n, n))
    Sx = np.zeros((n, n))
    spl = []
    for i in range(n):
        c = np.zeros(n)
        c[i] = 1
        b = BSpline(U, c, p)
        spl.append((b, b.derivative()))
    for a, bnd in zip(U[:-1], U[1:]):
        if bnd <= a:
            continue
        u = a + (bnd - a) * (xg + 1) / 2
        w = wg * (bnd - a) / 2
        V = np.array([s[0](u) for s in spl])
        D = np.array([s[1](u) for s in spl])
        Mx += (V * w) @ V.T
        Sx += (D * w) @ D.T
    return Mx * L, Sx / L


def test_P6_cuboid_matrices_are_kronecker_products():
    size = (0.9e-3, 0.7e-3, 0.4e-3)
    n_el = (4, 3, 2)
    patch = W.cuboid_patch(size, n_el, 2)
    g = PatchGeom(patch)
    rho_cp = MAT.rho * MAT.cp
    M, K = assembly.assemble_MK(g, rho_cp, MAT.k)
    m1 = [_bspline_1d_matrices(patch.knots[d], 2, size[d]) for d in range(3)]
    Mk = rho_cp * np.kron(m1[2][0], np.kron(m1[1][0], m1[0][0]))
    Kk = MAT.k * (np.kron(m1[2][1], np.kron(m1[1][0], m1[0][0])) +
                  np.kron(m1[2][0], np.kron(m1[1][1], m1[0][0])) +
                  np.kron(m1[2][0], np.kron(m1[1][0], m1[0][1])))
    np.testing.assert_allclose(M.toarray(), Mk, rtol=0, atol=1e-12 * np.abs(Mk).max())
    np.testing.assert_allclose(K.toarray(), Kk, rtol=0, atol=1e-12 * np.abs(Kk).max())
    assert M.sum() == pytest.approx(rho_cp * np.prod(size), rel=1e-13)


def _distorted_patch(weights=False, seed=3):
    rng = np.random.default_rng(seed)
    patch = W.cuboid_patch((1e-3, 0.8e-3, 0.5e-3), (3, 3, 2), 2)
    c = patch.ctrl.copy()
    inner = c[1:-1, 1:-1, 1:-1]
    inner += rng.uniform(-0.04e-3, 0.04e-3, inner.shape)
    # bend the side faces too (keep the top plane flat)
    c[:-1, :, 0, 0] += rng.uniform(-0.03e-3, 0.03e-3, c[:-1, :, 0, 0].shape)
    c[:-1, 0, :, 1] += rng.uniform(-0.03e-3, 0.03e-3, c[:-1, 0, :, 1].shape)
    patch.ctrl = c
    if weights:
        patch.weights = rng.uniform(0.8, 1.2, c.shape[:3])
    return patch


def test_P6_symmetry_constants_and_volume_on_curved_nurbs():
    patch = _distorted_patch(weights=True)
    g = PatchGeom(patch)
    M, K = assembly.assemble_MK(g, 1.0, 1.0)
    assert abs(M - M.T).max() < 1e-14 * abs(M).max()
    assert abs(K - K.T).max() < 1e-14 * abs(K).max()
    assert np.abs(K @ np.ones(g.n_dof)).max() < 1e-12 * abs(K).max()
    # volume by the divergence theorem on the faces: V = (1/3) int x . n dS
    V = 0.0
    for f in range(6):
        fp = g.face_points(f)
        V += np.sum(fp["wdS"] * np.einsum("qc,qc->q", fp["x"], fp["n"])) / 3.0
    assert M.sum() == pytest.approx(V, rel=1e-6)


def test_P6_patch_test_linear_field_is_reproduced():
    """Steady conduction with flux data of a linear field on every face but
    the Dirichlet bottom: the Galerkin solution is the linear field itself
    (isoparametric; 3-point Gauss is exact for this B-spline patch)."""
    patch = _distorted_patch(weights=False)
    patch.faces = (1, 1, 1, 1, 2, 1)
    g = PatchGeom(patch)
    M, K = assembly.assemble_MK(g, 1.0, MAT.k)
    a, b = 300.0, np.array([2.0e4, -1.5e4, 3.0e4])
    ctrl = patch.ctrl.reshape(-1, 3)
    T_exact = a + ctrl @ b
    pts = assembly.boundary_points(g, 1)
    F = assembly.weight_matrix(g, pts) @ (MAT.k * pts["n"] @ b)
    d = g.dirichlet_dofs()
    f = ~d
    Kff = K[f][:, f].toarray()
    rhs = F[f] - K[f][:, d] @ T_exact[d]
    T_f = np.linalg.solve(Kff, rhs)
    np.testing.assert_allclose(T_f, T_exact[f], rtol=0, atol=1e-9 * a)


# ---------------------------------------------------------------------------
# P7: space and time convergence on a manufactured heat solution.
# ---------------------------------------------------------------------------
def _manufactured(n_el, dt, n_steps, theta, p=2):
    Lx, Ly, Lz = 1e-3, 1e-3, 0.5e-3
    kap = np.array([np.pi / Lx, 0.7 * np.pi / Ly, 0.5 * np.pi / Lz])
    phi = 0.3
    amp = 5.0
    lam = ALPHA * kap @ kap

    def T_ex(x, t):
        return MAT.T_c + amp * np.exp(-lam * t) * np.cos(x @ kap + phi)

    def grad_ex(x, t):
        return -amp * np.exp(-lam * t) * np.sin(x @ kap + phi)[:, None] * kap[None, :]

    patch = W.cuboid_patch((Lx, Ly, Lz), (n_el, n_el, max(1, n_el // 2)), p)
    patch.faces = (1, 1, 1, 1, 2, 1)
    g = PatchGeom(patch)
    rho_cp = MAT.rho * MAT.cp
    M, K = assembly.assemble_MK(g, rho_cp, MAT.k)
    nb = assembly.boundary_points(g, 1)
    Wn = assembly.weight_matrix(g, nb)
    bot = assembly.boundary_points(g, 2)
    Wb = assembly.weight_matrix(g, bot)
    d = g.dirichlet_dofs()
    Mb = assembly.boundary_mass(g, bot)[d][:, d].toarray()

    def F_at(t):
        return Wn @ (MAT.k * np.einsum("qc,qc->q", grad_ex(nb["x"], t), nb["n"]))

    def g_at(t):
        return np.linalg.solve(Mb, (Wb @ T_ex(bot["x"], t))[d])

    # initial coefficients: L2 projection of T_ex(., 0)
    elems = g.element_list()
    rows = []
    for e in elems:
        for xi, wt in g.element_quadrature(e):
            dofs, R, dR, x, J = g.local_eval(xi, [e[k][2] for k in range(3)])
            rows.append((dofs, R, x, wt * np.linalg.det(J)))
    n = g.n_dof
    Mp = np.zeros((n, n))
    bp = np.zeros(n)
    for dofs, R, x, w in rows:
        Mp[np.ix_(dofs, dofs)] += w * np.outer(R, R)
        bp[dofs] += w * R * T_ex(x[None, :], 0.0)[0]
    T = np.linalg.solve(Mp, bp)
    solver = ThetaSolver(M, K, d, dt, theta)
    F0 = F_at(0.0)
    for s in range(n_steps):
        t1 = (s + 1) * dt
        F1 = F_at(t1)
        T = solver.step(T, F0, F1, g_at(t1))
        F0 = F1
    err2 = 0.0
    for dofs, R, x, w in rows:
        err2 += w * (R @ T[dofs] - T_ex(x[None, :], n_steps * dt)[0]) ** 2
    return np.sqrt(err2), T


def test_P7_spatial_convergence_rate():
    dt, nst = 2e-4, 10
    errs = [_manufactured(n, dt, nst, 0.5)[0] for n in (2, 4, 8)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > 2.6, (errs, rates)          # O(h^{p+1}) = O(h^3) for p = 2


def _ramped_run(dt, n_steps, theta):
    """Start at T_c (exact in the space, compatible with the data at t = 0)
    and drive the lateral/top flux and the bottom temperature by a smooth
    ramp s(t) = sin^2(pi t / (2 T)) that starts with zero slope, so that the
    semi-discrete solution is smooth in time and the step order shows."""
    patch = W.cuboid_patch((1e-3, 1e-3, 0.5e-3), (3, 3, 2), 2)
    patch.faces = (1, 1, 1, 1, 2, 1)
    g = PatchGeom(patch)
    M, K = assembly.assemble_MK(g, MAT.rho * MAT.cp, MAT.k)
    nb = assembly.boundary_points(g, 1)
    q_prof = assembly.weight_matrix(g, nb) @ (2e5 * np.cos(3e3 * nb["x"][:, 0]) * nb["n"][:, 1])
    d = g.dirichlet_dofs()
    g_prof = 4.0 * np.sin(2e3 * patch.ctrl.reshape(-1, 3)[d, 0])
    T_tot = 4e-3
    ramp = lambda t: np.sin(0.5 * np.pi * t / T_tot) ** 2
    solver = ThetaSolver(M, K, d, dt, theta)
    T = np.full(g.n_dof, MAT.T_c)
    F0 = ramp(0.0) * q_prof
    for s_ in range(n_steps):
        t1 = (s_ + 1) * dt
        F1 = ramp(t1) * q_prof
        T = solver.step(T, F0, F1, MAT.T_c + ramp(t1) * g_prof)
        F0 = F1
    return T


@pytest.mark.parametrize("theta,order", [(0.5, 2), (1.0, 1)])
def test_P7_temporal_convergence_rate(theta, order):
    T_end = 4e-3
    sols = [_ramped_run(T_end / nst, nst, theta) for nst in (8, 16, 32, 512)]
    ref = sols[-1]
    e = [np.abs(s - ref).max() for s in sols[:-1]]
    rates = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert np.all(np.abs(rates - order) < 0.25), (e, rates)


# ---------------------------------------------------------------------------
# P9: conservation.  All faces but the top carry the T~ flux (no Dirichlet):
#     (a) algebraic: 1^T M (T^{n+1} - T^n) = dt 1^T (theta F^{n+1} + (1-theta) F^n);
#     (b) physical: box integral of rho c (T~ + T^ - T_c) equals the absorbed
#         energy n E, with the box integral of T~ in closed form (erf).
# ---------------------------------------------------------------------------
def _box_T_tilde_integral(lo, hi, xs, age, E, s_img=2.0):
    from scipy.special import erf
    sig = np.sqrt(2 * ALPHA * age)
    tot = np.full(len(age), s_img * E / (MAT.rho * MAT.cp))
    for d in range(3):
        a = (lo[d] - xs[:, d]) / (np.sqrt(2) * sig)
        b = (hi[d] - xs[:, d]) / (np.sqrt(2) * sig)
        tot *= 0.5 * (erf(b) - erf(a))
    return MAT.rho * MAT.cp * tot.sum()


@pytest.mark.parametrize("theta", [0.5, 1.0])
def test_P9_energy_balance_all_neumann(theta):
    size = (0.8e-3, 0.5e-3, 0.3e-3)
    patch = W.cuboid_patch(size, (16, 10, 6), 2, faces=(1, 1, 1, 1, 1, 0))
    scan = W.straight_track((0.1e-3, 0.08e-3, 0.3e-3), (0.7e-3, 0.08e-3, 0.3e-3),
                            power=100.0, absorptivity=0.5, speed=1.0)
    wl = W.Workload("p9", patch, MAT, scan, dt=10e-6, theta=theta, n_steps=60)
    m = Model(wl)
    ones = np.ones(m.geom.n_dof)
    roundoff = 1e-13 * (ones @ (m.M @ ones)) * MAT.T_c      # rounding of 1^T M T
    leak = 0.0
    for _ in range(wl.n_steps):
        T0, F0 = m.T_hat.copy(), m.F.copy()
        m.step()
        lhs = ones @ (m.M @ (m.T_hat - T0))
        rhs = wl.dt * ones @ (theta * m.last["F"] + (1 - theta) * F0)
        assert abs(lhs - rhs) <= 1e-9 * abs(rhs) + roundoff
        leak += rhs
    n = m.n
    age = m.source_ages(n)
    inside = _box_T_tilde_integral((0, 0, 0), size, m.xs[:n], age, m.E)
    total = inside + ones @ (m.M @ (m.T_hat - MAT.T_c))
    assert (n * m.E - inside) > 0.05 * n * m.E       # a real share leaves through the walls
    assert total == pytest.approx(n * m.E, rel=0.02)


def test_P10_far_field_correction_vanishes():
    patch = W.cuboid_patch((2e-3, 2e-3, 1e-3), (8, 8, 4), 2)
    scan = W.straight_track((1e-3, 1e-3, 1e-3), (1.02e-3, 1e-3, 1e-3), 100.0, 0.5, 1.0)
    wl = W.Workload("p10", patch, MAT, scan, dt=5e-6, theta=0.5, n_steps=5)
    m = Model(wl)
    m.run(5)
    assert np.abs(m.T_hat - MAT.T_c).max() < 1e-9


def test_R5_dirichlet_projection_reproduces_face_space_functions():
    """The L2 projection returns the coefficients of any function of the
    bottom-face spline space; linear fields are in it (x = sum R_i P_i)."""
    wl = W.small_block(n_el=(4, 3, 2))
    m = Model(wl, build_solver=False)
    ctrl = wl.patch.ctrl.reshape(-1, 3)
    f = lambda x: 2.0 + 3e3 * x[:, 0] - 5e3 * x[:, 1]
    # T~ chosen so that T_c - T~ = f on the bottom face
    g = m.dirichlet_g(wl.material.T_c - f(m.bot["x"]))
    np.testing.assert_allclose(g, f(ctrl[m.dir]), rtol=0, atol=1e-12)


def test_mlp_oracle_gradients_by_finite_differences():
    """The FP64 warm-start network reference: every analytic gradient entry
    checked against central differences of the loss."""
    from oracle import mlp
    rng = np.random.default_rng(0)
    sizes = [7, 5, 5, 5, 6]
    params = [(rng.normal(0, 0.5, (o, i)), rng.normal(0, 0.1, o)) for i, o in zip(sizes[:-1], sizes[1:])]
    X = rng.normal(size=(4, sizes[0]))
    Y = rng.normal(size=(4, sizes[-1]))
    loss, grads = mlp.loss_and_grads(params, X, Y)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for arr, g in ((W, grads[li][0]), (b, grads[li][1])):
            flat = arr.reshape(-1)
            gf = g.reshape(-1)
            for k in range(0, flat.size, max(1, flat.size // 7)):
                old = flat[k]
                flat[k] = old + h
                lp, _ = mlp.loss_and_grads(params, X, Y)
                flat[k] = old - h
                lm, _ = mlp.loss_and_grads(params, X, Y)
                flat[k] = old
                assert abs((lp - lm) / (2 * h) - gf[k]) < 1e-7 * max(1.0, abs(gf[k]))


# ---------------------------------------------------------------------------
# P12: the closed (seam) patch of the plate with a hole.
# ---------------------------------------------------------------------------
def _coarse_plate():
    return W.plate_with_hole_patch(n_el=(8, 4, 2))


def test_P12_plate_faces_lie_on_the_circle_and_the_square():
    """The hole face is the exact circle of radius R (rational quadratic
    arcs, elevated and refined exactly) and the outer face the square."""
    g = PatchGeom(_coarse_plate())
    hole = g.face_points(3)
    outer = g.face_points(2)
    r = np.hypot(hole["x"][:, 0], hole["x"][:, 1])
    np.testing.assert_allclose(r, 0.75e-3, rtol=1e-14, atol=0)
    # outward normal of the plate on the hole face points towards the axis
    radial = hole["x"][:, :2] / r[:, None]
    np.testing.assert_allclose(np.einsum("qc,qc->q", hole["n"][:, :2], radial), -1.0, atol=1e-12)
    m = np.max(np.abs(outer["x"][:, :2]), axis=1)
    np.testing.assert_allclose(m, 1.5e-3, rtol=1e-14, atol=0)


def test_P12_seam_merge_is_PtMP_of_the_open_patch():
    """Assembling on the merged control variables equals P^T M P of the same
    patch assembled with both seam layers kept (P: 0/1 control point ->
    control variable)."""
    plate = _coarse_plate()
    g = PatchGeom(plate)
    M, K = assembly.assemble_MK(g, 1.0, 1.0)
    open_patch = W.Patch(plate.degree, plate.knots, plate.ctrl, plate.weights,
                         faces=plate.faces, seam=-1)
    go = PatchGeom(open_patch)
    Mo, Ko = assembly.assemble_MK(go, 1.0, 1.0)
    n0, n1, n2 = go.n
    K3, J3, I3 = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    to = g.dof(I3.ravel(), J3.ravel(), K3.ravel())
    P = np.zeros((go.n_dof, g.n_dof))
    P[np.arange(go.n_dof), to] = 1.0
    np.testing.assert_allclose(M.toarray(), P.T @ Mo.toarray() @ P, rtol=0,
                               atol=1e-13 * abs(M).max())
    np.testing.assert_allclose(K.toarray(), P.T @ Ko.toarray() @ P, rtol=0,
                               atol=1e-13 * abs(K).max())
    assert g.n_dof == go.n_dof - n1 * n2


def test_P12_plate_volume_symmetry_and_constants():
    g = PatchGeom(_coarse_plate())
    M, K = assembly.assemble_MK(g, 1.0, 1.0)
    assert abs(M - M.T).max() < 1e-14 * abs(M).max()
    assert abs(K - K.T).max() < 1e-14 * abs(K).max()
    assert np.abs(K @ np.ones(g.n_dof)).max() < 1e-12 * abs(K).max()
    V = (4 * 1.5e-3 ** 2 - np.pi * 0.75e-3 ** 2) * 0.5e-3      # closed form
    assert M.sum() == pytest.approx(V, rel=1e-7)


def _plate_patch_test_error(n_el):
    plate = W.plate_with_hole_patch(n_el=n_el)
    plate.faces = (0, 0, 1, 1, 2, 1)
    g = PatchGeom(plate)
    M, K = assembly.assemble_MK(g, 1.0, MAT.k)
    a, b = 300.0, np.array([2.0e4, -1.5e4, 3.0e4])
    T_exact = np.empty(g.n_dof)
    for dof in range(g.n_dof):
        i, j, k = g.ctrl_points_of(dof)[0]
        T_exact[dof] = a + plate.ctrl[k, j, i] @ b
    pts = assembly.boundary_points(g, 1)
    F = assembly.weight_matrix(g, pts) @ (MAT.k * pts["n"] @ b)
    d = g.dirichlet_dofs()
    f = ~d
    rhs = F[f] - K[f][:, d] @ T_exact[d]
    T_f = spla.spsolve(K[f][:, f].tocsc(), rhs)
    return np.abs(T_f - T_exact[f]).max()


def test_P12_patch_test_on_the_closed_plate():
    """Linear field (45 K across the plate) with its flux on the hole, outer
    and top faces and its values on the bottom: the space contains it
    (isoparametric, merged seam), so the Galerkin solution reproduces it up
    to the quadrature error of the rational map, which falls at the rate of
    the (p+1)-point Gauss rule (h^8 for p = 3) when the angular and radial
    spans are halved.  A wrong seam merge or flux sign leaves an O(1 K)
    error that does not fall."""
    e8 = _plate_patch_test_error((8, 4, 2))
    e16 = _plate_patch_test_error((16, 8, 2))
    assert e16 <= 1e-5, (e8, e16)
    assert e8 / e16 >= 64.0, (e8, e16)


# ---------------------------------------------------------------------------
# R12: on a face that is an axis-aligned rectangle the quadrature points are
#      a tensor grid, and the history sums factorise along the face's axes
#      (Eq. sum-of-point-temp summed in another order): a matrix product over
#      the sources equals the oracle's pairwise sums.
# ---------------------------------------------------------------------------
def test_R12_separable_sums_equal_pairwise_on_box_faces():
    patch = W.cuboid_patch((0.9e-3, 0.7e-3, 0.4e-3), (5, 4, 3), (2, 3, 2))
    geom = PatchGeom(patch)
    z = geom.top_z()
    rng = np.random.default_rng(12)
    K = 40
    xs = np.column_stack([rng.uniform(0.1e-3, 0.8e-3, K), rng.uniform(0.1e-3, 0.6e-3, K),
                          np.full(K, z)])
    age = pointsource.ages(K + 5, K, 5e-6, MAT, 20e-6)
    E = 1e-3
    a = 1.0 / (4.0 * ALPHA * age)
    c = 2.0 * E / (MAT.rho * MAT.cp * (4.0 * np.pi * ALPHA * age) ** 1.5)
    g = 2.0 * a * c
    checked = 0
    for face, kind in enumerate(geom.faces):
        if kind == 0:
            continue
        pts = geom.face_points(face)
        x, nrm = pts["x"], pts["n"]
        d = int(np.argmax(np.abs(nrm[0])))                  # the normal's axis
        u, v = [ax for ax in range(3) if ax != d]
        # distinct coordinates up to rounding (1e-12 of the extent)
        key_u, key_v = np.round(x[:, u] / 1e-3, 9), np.round(x[:, v] / 1e-3, 9)
        ku, iu = np.unique(key_u, return_index=True)
        kv, iv = np.unique(key_v, return_index=True)
        A, B = x[iu, u], x[iv, v]
        assert len(A) * len(B) == len(x)                    # a full tensor grid
        i, j = np.searchsorted(ku, key_u), np.searchsorted(kv, key_v)
        assert np.abs(A[i] - x[:, u]).max() <= 1e-15 and np.abs(B[j] - x[:, v]).max() <= 1e-15
        dd = x[0, d]
        assert np.allclose(x[:, d], dd, rtol=0, atol=1e-15)
        FA = np.exp(-a[:, None] * (A[None, :] - xs[:, u, None]) ** 2)            # (K, |A|)
        ed = np.exp(-a * (dd - xs[:, d]) ** 2)
        if kind == 1:   # dT~/dn = sum -g n_d (d - s_d) exp(-a R^2)
            w = -g * nrm[0, d] * (dd - xs[:, d]) * ed
            ref = pointsource.dTdn_tilde(x, nrm, xs, age, E, MAT)
        else:           # T~ = sum c exp(-a R^2)
            w = c * ed
            ref = pointsource.T_tilde(x, xs, age, E, MAT)
        FB = w[:, None] * np.exp(-a[:, None] * (B[None, :] - xs[:, v, None]) ** 2)
        S = FA.T @ FB                                                           # (|A|, |B|)
        assert np.abs(S[i, j] - ref).max() <= 1e-13 * np.abs(ref).max(), face
        checked += 1
    assert checked == 5


# ---------------------------------------------------------------------------
# Heat-loss rates (Section 3.1, q~ + q^ = -k dT/dn): the oracle's q~ + q^
# equals -k times the central difference of its own T = T~ + T^ along the
# normal (points found by a Newton inversion with a finite-difference
# Jacobian, independent of the oracle's J).
# ---------------------------------------------------------------------------
def _invert_map(geom, x, xi0):
    xi = np.array(xi0, dtype=np.float64)
    for _ in range(60):
        f = geom.point(xi) - x
        if np.linalg.norm(f) < 1e-17:
            break
        J = np.empty((3, 3))
        for d in range(3):
            e = np.zeros(3)
            e[d] = 1e-7
            J[:, d] = (geom.point(xi + e) - geom.point(xi - e)) / 2e-7
        xi = np.clip(xi - np.linalg.solve(J, f), 1e-6, 1 - 1e-6)   # interior points only
    assert np.linalg.norm(geom.point(xi) - x) < 1e-14
    return xi


def _xi_near(geom, x, n=13):
    """Parametric point of x (inside the patch): the nearest of an n^3 grid
    of interior points, then Newton."""
    u = np.linspace(0.02, 0.98, n)
    best, bd = None, np.inf
    for a in u:
        for b in u:
            for c in u:
                d = np.linalg.norm(geom.point(np.array([a, b, c])) - x)
                if d < bd:
                    best, bd = np.array([a, b, c]), d
    return _invert_map(geom, x, best)


def test_heat_loss_rate_is_minus_k_times_the_normal_derivative():
    wl = W.quarter_cylinder_single_source((4, 2, 2), n_steps=6)
    m = Model(wl)
    for _ in range(6):
        m.step()
    rng = np.random.default_rng(31)
    # far from the source (q^ dominates) ...
    xi = np.column_stack([rng.choice([rng.uniform(0.1, 0.4), rng.uniform(0.6, 0.9)], 6),
                          rng.uniform(0.15, 0.85, 6), rng.uniform(0.5, 0.95, 6)])
    # ... and within ~70 um of it, below the top face (q~ dominates)
    near = m.xs[0] + np.array([[30e-6, 20e-6, -40e-6], [-50e-6, 10e-6, -20e-6],
                               [0.0, -40e-6, -60e-6]])
    xi = np.vstack([xi, [_xi_near(m.geom, x) for x in near]])
    nrm = rng.normal(size=(len(xi), 3))
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    x, qt, qh = m.eval_flux(xi, nrm)
    h = 1e-7
    q_fd = []
    for k in range(len(x)):
        xp = _invert_map(m.geom, x[k] + h * nrm[k], xi[k])
        xm = _invert_map(m.geom, x[k] - h * nrm[k], xi[k])
        Tp, Tm = m.eval_T(xp)[1][0], m.eval_T(xm)[1][0]
        q_fd.append(-MAT_TI.k * (Tp - Tm) / (2 * h))
    q_fd = np.array(q_fd)
    # each point against its own rate; both parts are a real share of it
    assert np.all(np.abs(qt + qh - q_fd) <= 1e-5 * np.abs(q_fd) + 1e-9 * np.abs(q_fd).max()), \
        (qt + qh, q_fd)
    assert np.abs(qt[6:]).min() > 0.5 * np.abs(q_fd[6:]).min()
    assert np.abs(qh[:6]).max() > 0.5 * np.abs(q_fd[:6]).max()


# ---------------------------------------------------------------------------
# Table 3: q~ on the top arc depends on the point sources alone (position,
# energy, ages at t = 1.9e-4 s, image factor), so every column of the table
# fixes int |q~| ds = net / ratio to within the rounding of its printed
# figures.  The oracle's int |q~| ds must lie in all five intervals.
# ---------------------------------------------------------------------------
def _half_unit(s):
    mant, _, ex = s.lower().partition("e")
    dec = len(mant.split(".")[1]) if "." in mant else 0
    return 0.5 * 10.0 ** (-dec) * 10.0 ** int(ex or 0)


def test_table3_integrated_analytical_heat_loss():
    lo, hi = 0.0, np.inf
    for line in open(os.path.join(GOLDEN, "table3_heat_loss.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        _, _, net_s, pct_s = line.split()
        net, dn = float(net_s), _half_unit(net_s)
        r, dr = float(pct_s) / 100, _half_unit(pct_s) / 100
        lo, hi = max(lo, (net - dn) / (r + dr)), min(hi, (net + dn) / (r - dr))
    assert lo < hi
    wl = W.quarter_cylinder_single_source((4, 2, 2), n_steps=19)
    m = Model(wl, build_solver=False)
    n = 19
    K = m.n_active(n)
    _, pts, nrm, ds = W.quarter_cylinder_arc_points(2001)
    qt = -wl.material.k * pointsource.dTdn_tilde(pts, nrm, m.xs[:K], m.source_ages(n), m.E,
                                                  wl.material, m.s_img)
    ana = float(np.sum(np.abs(qt) * ds))
    assert lo <= ana <= hi, (lo, ana, hi)


# ---------------------------------------------------------------------------
# Table 4: the same argument for the contour scan at t = 2e-3 s and 3e-3 s
# (both columns at one time fix int |q~| ds).  It separates the readings of
# the scan path: the arc part of the 100 um offset contour passes at both
# times; the whole 1.1 mm quarter circle started at the x2 face does not
# (0.35 % low at 2e-3 s).
# ---------------------------------------------------------------------------
def test_table4_integrated_analytical_heat_loss():
    win = {}
    for line in open(os.path.join(GOLDEN, "table4_heat_loss.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        t_s, _, _, net_s, pct_s = line.split()
        net, dn = float(net_s), _half_unit(net_s)
        r, dr = float(pct_s) / 100, _half_unit(pct_s) / 100
        lo, hi = win.get(t_s, (0.0, np.inf))
        win[t_s] = (max(lo, (net - dn) / (r + dr)), min(hi, (net + dn) / (r - dr)))
    assert len(win) == 2
    wl = W.quarter_cylinder_contour((4, 2, 2), n_steps=300)
    m = Model(wl, build_solver=False)
    _, pts, nrm, ds = W.quarter_cylinder_arc_points(4001)
    for t_s, (lo, hi) in win.items():
        assert lo < hi
        n = int(round(float(t_s) / wl.dt))
        K = m.n_active(n)
        qt = -wl.material.k * pointsource.dTdn_tilde(pts, nrm, m.xs[:K], m.source_ages(n),
                                                      m.E, wl.material, m.s_img)
        ana = float(np.sum(np.abs(qt) * ds))
        assert lo <= ana <= hi, (t_s, lo, ana, hi)


# ---------------------------------------------------------------------------
# C1: the bound of the opt-in history cutoff (not part of the paper's method)
# ---------------------------------------------------------------------------
def test_pin_C1_cutoff_bound_by_brute_force():
    """unit_bound is an upper bound of every term over a box (brute force on
    a 21 x 21 grid of each face box), is attained when the box is one point,
    and the sum over any dropped subset of sources is at most the sum of
    their bounds at every point of the box."""
    from oracle import pointsource as ps
    mat = W.MAT_DEFAULT
    rng = np.random.default_rng(17)
    E = 4e-4
    for trial in range(6):
        K = 40
        xs = np.column_stack([rng.uniform(0, 1e-3, K), rng.uniform(0, 1e-3, K), np.full(K, 0.5e-3)])
        age = rng.uniform(1e-6, 4e-4, K)
        ax = trial % 3                                 # face normal along x, y or z
        lo = rng.uniform(0, 0.6e-3, 3)
        hi = lo + rng.uniform(0.05e-3, 0.4e-3, 3)
        lo[ax] = hi[ax] = rng.uniform(0, 0.5e-3)
        nrm = np.eye(3)[ax] * (1 if trial % 2 else -1)
        t = [np.linspace(lo[k], hi[k], 21) if k != ax else np.array([lo[k]]) for k in range(3)]
        pts = np.array(np.meshgrid(*t, indexing="ij")).reshape(3, -1).T
        for normal in (None, nrm):
            bnd = ps.unit_bound(lo, hi, xs, age, E, mat, normal=normal)
            T = ps.T_point(pts, xs, age, E, mat)                      # (Q, K)
            terms = T if normal is None else np.abs(
                np.einsum("qkc,c->qk", ps.gradT_point(pts, xs, age, E, mat), normal))
            assert np.all(terms <= bnd[None, :] * (1 + 1e-12) + 1e-300)
            drop = rng.uniform(size=K) < 0.5
            assert np.all(terms[:, drop].sum(1) <= bnd[drop].sum() * (1 + 1e-12) + 1e-300)
            # one-point box: the bound is the term itself
            p = pts[len(pts) // 3]
            b1 = ps.unit_bound(p, p, xs, age, E, mat, normal=normal)
            t1 = T[len(pts) // 3] if normal is None else terms[len(pts) // 3]
            assert np.allclose(b1, t1, rtol=1e-12, atol=0)


# ---------------------------------------------------------------------------
# R22: several lasers.  The multi-laser model sums every laser's sources in
#      the history sums and runs ONE theta-scheme; the pins check it against
#      routes that do not share that sum: single-laser models (the problem
#      is linear, so one solve of the combined data must equal the sum of
#      single-laser solves, sum_l T_l - (L - 1) T_c), a one-laser list
#      (the plain model), and mirror symmetry of two mirrored lasers.
# ---------------------------------------------------------------------------
def _single(wl, scan):
    m = Model(W.Workload("laser", wl.patch, wl.material, scan, dt=wl.dt, theta=wl.theta,
                         n_steps=wl.n_steps))
    m.run(wl.n_steps)
    return m


def test_R22_multi_laser_one_laser_is_the_plain_model():
    from oracle.solver import MultiLaserModel
    wl, scans = W.two_lasers_cuboid(n_steps=12)
    m = MultiLaserModel(wl, scans[:1])
    m.run(12)
    ref = _single(wl, scans[0])
    assert np.abs(m.T_hat - ref.T_hat).max() <= 1e-12 * np.abs(ref.T_hat).max()
    assert np.abs(m.F - ref.F).max() <= 1e-12 * max(np.abs(ref.F).max(), 1e-300)


def test_R22_multi_laser_superposition_of_single_laser_solves():
    from oracle.solver import MultiLaserModel
    wl, scans = W.two_lasers_cuboid(n_steps=30)
    m = MultiLaserModel(wl, scans)
    m.run(30)
    singles = [_single(wl, sc) for sc in scans]
    Tc = wl.material.T_c
    sup = sum(s.T_hat for s in singles) - (len(singles) - 1) * Tc
    assert np.abs(m.T_hat - sup).max() <= 1e-9 * np.abs(sup).max()
    # F (linear in the sources, no T_c offset) and T at points on and under the tracks
    assert np.abs(m.F - sum(s.F for s in singles)).max() <= 1e-10 * np.abs(m.F).max()
    xi = np.array([[0.30, 0.30, 1.0], [0.50, 0.50, 0.9], [0.60, 0.70, 1.0], [0.10, 0.90, 0.5],
                   [0.80, 0.20, 0.2]])
    _, T = m.eval_T(xi)
    Ts = sum(s.eval_T(xi)[1] for s in singles) - (len(singles) - 1) * Tc
    assert np.abs(T - Ts).max() <= 1e-9 * np.abs(Ts).max()
    # both lasers matter: each single-laser field differs from the combined one
    for s in singles:
        assert np.abs(s.T_hat - m.T_hat).max() > 1e-3


def test_R22_mirrored_lasers_give_a_mirror_symmetric_field():
    from oracle.solver import MultiLaserModel
    wl, scans = W.two_lasers_cuboid(powers=(180.0, 180.0), ys=(0.3e-3, 0.7e-3), n_steps=20)
    m = MultiLaserModel(wl, scans)
    m.run(20)
    # near the tracks (laser front at x ~ 0.45 mm after 20 steps) and away from them
    xi = np.array([[0.20, 0.30, 1.0], [0.18, 0.25, 0.95], [0.45, 0.35, 0.8], [0.70, 0.10, 0.4],
                   [0.55, 0.45, 1.0]])
    mirror = xi.copy()
    mirror[:, 1] = 1.0 - mirror[:, 1]
    _, T = m.eval_T(xi)
    _, Tm = m.eval_T(mirror)
    assert np.abs(T - Tm).max() <= 1e-9 * np.abs(T).max()
    assert np.abs(T - wl.material.T_c).max() > 1e-3
