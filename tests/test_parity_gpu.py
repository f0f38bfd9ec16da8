"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: FP64 GPU path 1e-10 relative L-infinity (1e-12 for set-up
quantities and single history sums); mixed path 1e-4 relative and 0.05 K.
"""
import numpy as np
import pytest

import workloads as W
from tests._common import (TOL_FP64, TOL_MIXED_ABS, TOL_MIXED_REL, gpu_context, lateral_xi,
                           rel_linf)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_20432_gb300 import build
    build.build()
    import paper_2511_20432_gb300 as sa_mod
    return sa_mod


def _oracle(wl, **kw):
    from oracle.solver import Model
    return Model(wl, **kw)


def _patch_cases():
    return {
        "cuboid": W.cuboid_patch((0.9e-3, 0.7e-3, 0.4e-3), (5, 4, 3), 2),
        "nurbs_distorted": W.distorted_block(weights=True),
        "bspline_p3": W.distorted_block(weights=False, degree=3, n_el=(3, 2, 2), seed=5),
        "quarter_cylinder": W.quarter_cylinder_part(),
        "mixed_degree": W.cuboid_patch((0.6e-3, 0.5e-3, 0.3e-3), (4, 3, 2), (3, 2, 1)),
        "plate_seam": W.plate_with_hole_patch(n_el=(8, 4, 2)),
    }


def _wl_for(patch, n_steps=4, dt=5e-6, theta=0.5):
    ctrl = patch.ctrl.reshape(-1, 3)
    lo, hi = ctrl.min(0), ctrl.max(0)
    z = float(patch.ctrl[-1, 0, 0, 2])
    x0 = lo + 0.3 * (hi - lo)
    x1 = lo + 0.6 * (hi - lo)
    scan = W.straight_track((x0[0], x0[1], z), (x1[0], x0[1], z), 150.0, 0.4, 1.0)
    return W.Workload("case", patch, W.MAT_DEFAULT, scan, dt=dt, theta=theta, n_steps=n_steps)


@pytest.mark.parametrize("case", list(_patch_cases()))
def test_boundary_points_match_oracle(sa, case):
    patch = _patch_cases()[case]
    wl = _wl_for(patch)
    m = _oracle(wl, build_solver=False)
    ctx = gpu_context(wl, sa.SA_FP64)
    lat = ctx.field(sa.SA_FIELD_LAT_X).reshape(-1, 7)
    bot = ctx.field(sa.SA_FIELD_BOT_X).reshape(-1, 4)
    scale = np.abs(patch.ctrl).max()
    assert lat.shape[0] == len(m.lat["x"]) and bot.shape[0] == len(m.bot["x"])
    assert np.abs(lat[:, :3] - m.lat["x"]).max() <= 1e-13 * scale
    assert np.abs(lat[:, 3:6] - m.lat["n"]).max() <= 1e-12
    assert rel_linf(lat[:, 6], m.lat["wdS"]) <= 1e-12
    assert np.abs(bot[:, :3] - m.bot["x"]).max() <= 1e-13 * scale
    assert rel_linf(bot[:, 3], m.bot["wdS"]) <= 1e-12


@pytest.mark.parametrize("case", list(_patch_cases()))
def test_assembly_matches_oracle(sa, case):
    patch = _patch_cases()[case]
    wl = _wl_for(patch)
    m = _oracle(wl, build_solver=False)
    ctx = gpu_context(wl, sa.SA_FP64)
    import scipy.sparse as sp
    n = patch.n_dof
    for which, ref in ((0, m.M), (1, m.K)):
        ptr, col, val = ctx.matrix(which)
        G = sp.csr_matrix((val, col, ptr), shape=(n, n))
        D = (G - ref).toarray()
        assert np.abs(D).max() <= 1e-12 * np.abs(ref).max(), (case, which)


def _lockstep(sa, wl, precision, n_check, every=1, **opts):
    """Step oracle and GPU together; return max relative errors of the
    history sums, F and T^ over the checked steps."""
    m = _oracle(wl)
    ctx = gpu_context(wl, precision, pcg_tol=1e-15 if precision == sa.SA_FP64 else 1e-10,
                      **opts)
    err = dict(s_lat=0.0, tt_bot=0.0, F=0.0, That=0.0, That_abs=0.0)
    for step in range(n_check):
        ctx.step(wl.theta, wl.dt, 1)
        m.step()
        if (step + 1) % every and step + 1 != n_check:
            continue
        err["s_lat"] = max(err["s_lat"], rel_linf(ctx.field(sa.SA_FIELD_DTDN_LAT), m.last["s_lat"]))
        err["tt_bot"] = max(err["tt_bot"], rel_linf(ctx.field(sa.SA_FIELD_TT_BOT), m.last["Tt_bot"]))
        err["F"] = max(err["F"], rel_linf(ctx.field(sa.SA_FIELD_F), m.F))
        T = ctx.field(sa.SA_FIELD_THAT)
        err["That"] = max(err["That"], rel_linf(T, m.T_hat))
        err["That_abs"] = max(err["That_abs"], np.abs(T - m.T_hat).max())
    return err, ctx, m


VARIANTS = {"shared": 1, "global": 2}
HIST = {"separable": 2, "pairwise": 1}


@pytest.mark.parametrize("hist", list(HIST))
@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_cuboid_single_track_fp64(sa, theta, variant, hist):
    wl = W.cuboid_single_track(theta=theta, n_steps=150)
    err, ctx, m = _lockstep(sa, wl, sa.SA_FP64, 150, every=25, pcg_variant=VARIANTS[variant],
                            hist_mode=HIST[hist])
    assert ctx.sizes().hist_separable == (hist == "separable")
    assert err["s_lat"] <= 1e-12 and err["tt_bot"] <= 1e-12, err
    assert err["F"] <= TOL_FP64 and err["That"] <= TOL_FP64, err
    # reconstruction T = T~ + T^ at interior and boundary points
    rng = np.random.default_rng(7)
    xi = rng.uniform(0, 1, (40, 3))
    xi[:8, 2] = 1.0
    x, T_ref = m.eval_T(xi)
    T = ctx.eval_T(np.vstack([x, OUTSIDE_CUBOID]))
    assert np.isnan(T[-2:]).all()
    assert rel_linf(T[:-2], T_ref) <= TOL_FP64


# points outside the 2 x 1 x 0.5 mm cuboid: NaN
OUTSIDE_CUBOID = np.array([[3e-3, 0.5e-3, 0.25e-3], [1e-3, -0.2e-3, 0.25e-3]])


@pytest.mark.parametrize("hist", list(HIST))
@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_cuboid_single_track_mixed(sa, theta, variant, hist):
    wl = W.cuboid_single_track(theta=theta, n_steps=150)
    err, ctx, m = _lockstep(sa, wl, sa.SA_MIXED, 150, every=15, pcg_variant=VARIANTS[variant],
                            hist_mode=HIST[hist])
    assert ctx.sizes().hist_separable == (hist == "separable")
    assert err["s_lat"] <= TOL_MIXED_REL and err["tt_bot"] <= TOL_MIXED_REL, err
    assert err["That"] <= TOL_MIXED_REL and err["That_abs"] <= TOL_MIXED_ABS, err
    # reconstruction in the mixed context (FP32 point inversion and sums)
    rng = np.random.default_rng(7)
    xi = rng.uniform(0, 1, (40, 3))
    xi[:8, 2] = 1.0
    x, T_ref = m.eval_T(xi)
    T = ctx.eval_T(np.vstack([x, OUTSIDE_CUBOID]))
    assert np.isnan(T[-2:]).all()
    assert rel_linf(T[:-2], T_ref) <= TOL_MIXED_REL
    assert np.abs(T[:-2] - T_ref).max() <= TOL_MIXED_ABS


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_plate_with_hole_lockstep(sa, prec):
    """The closed (seam) plate with a hole, coarse (8 x 4 x 2 elements of
    degree 3): history sums, F and T^ step by step against the oracle along
    the contour scan, and T near the hole edge."""
    p = sa.SA_FP64 if prec == "fp64" else sa.SA_MIXED
    wl = W.plate_with_hole(n_el=(8, 4, 2), n_steps=60)
    err, ctx, m = _lockstep(sa, wl, p, 60, every=20)
    if p == sa.SA_FP64:
        assert err["s_lat"] <= 1e-12 and err["tt_bot"] <= 1e-12, err
        assert err["F"] <= TOL_FP64 and err["That"] <= TOL_FP64, err
    else:
        assert err["s_lat"] <= TOL_MIXED_REL and err["tt_bot"] <= TOL_MIXED_REL, err
        assert err["That"] <= TOL_MIXED_REL and err["That_abs"] <= TOL_MIXED_ABS, err
    # points within 20 um of the hole edge (top surface and below), on both
    # sides of the seam (xi = 0 is at -45 degrees)
    xi = np.array([[u, v, w] for u in (0.0, 0.01, 0.3, 0.62, 0.99, 1.0)
                   for v in (0.995, 1.0) for w in (1.0, 0.9)])
    x, T_ref = m.eval_T(xi)
    T = ctx.eval_T(x)
    tol = TOL_FP64 if p == sa.SA_FP64 else TOL_MIXED_REL
    assert rel_linf(T, T_ref) <= tol


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_extrapolated_guess(sa, prec):
    """x0 = T^n + (T^n - T^{n-1}) (and 2 g^n - g^{n-1} for the projection):
    the same steps as the oracle to the parity tolerance, in fewer PCG
    iterations than the start from T^n."""
    p = sa.SA_FP64 if prec == "fp64" else sa.SA_MIXED
    wl = W.cuboid_single_track(theta=0.5, n_steps=150)
    err, ctx, m = _lockstep(sa, wl, p, 150, every=25, initial_guess=sa.SA_GUESS_EXTRAPOLATE)
    if p == sa.SA_FP64:
        assert err["F"] <= TOL_FP64 and err["That"] <= TOL_FP64, err
    else:
        assert err["That"] <= TOL_MIXED_REL and err["That_abs"] <= TOL_MIXED_ABS, err
    tol = 1e-15 if p == sa.SA_FP64 else 1e-10
    iters = {}
    for g in (sa.SA_GUESS_PREVIOUS, sa.SA_GUESS_EXTRAPOLATE):
        # Jacobi: with the fast-diagonalization preconditioner a box solves
        # in one iteration from either start
        c = gpu_context(wl, p, pcg_tol=tol, initial_guess=g, precond=sa.SA_PRECOND_JACOBI)
        c.step(wl.theta, wl.dt, 20)
        c.step(wl.theta, wl.dt, 0)
        st = c.step(wl.theta, wl.dt, 100)
        iters[g] = (st.pcg_iters_total, st.bot_iters_total)
    assert iters[sa.SA_GUESS_EXTRAPOLATE][0] < iters[sa.SA_GUESS_PREVIOUS][0], iters
    assert iters[sa.SA_GUESS_EXTRAPOLATE][1] <= iters[sa.SA_GUESS_PREVIOUS][1], iters


@pytest.mark.parametrize("P,NW", [(1, 4), (2, 8), (4, 8), (4, 4)])
def test_multichunk_ragged_tiles(sa, P, NW):
    """Several tracks (hundreds of sources over many warps), tiles with a
    ragged tail, a distorted NURBS block; every tile shape of the kernel."""
    patch = W.distorted_block(weights=True, n_el=(7, 5, 3), size=(1.4e-3, 1.0e-3, 0.5e-3), seed=11)
    z = float(patch.ctrl[-1, 0, 0, 2])
    scan = W.meander(0.2e-3, 1.2e-3, 0.25e-3, 0.15e-3, 4, z, 180.0, 0.4, 1.5)
    wl = W.Workload("mc", patch, W.MAT_DEFAULT, scan, dt=4e-6, theta=0.5, n_steps=420)
    for prec in (sa.SA_FP64, sa.SA_MIXED):
        # both PCG variants over the tile shapes
        err, ctx, m = _lockstep(sa, wl, prec, 420, every=70, hist_points_per_lane=P,
                                hist_warps=NW, pcg_variant=1 + (P + NW + prec) % 2)
        if prec == sa.SA_FP64:
            assert err["s_lat"] <= 1e-12 and err["F"] <= TOL_FP64 and err["That"] <= TOL_FP64, err
        else:
            assert err["s_lat"] <= TOL_MIXED_REL and err["tt_bot"] <= TOL_MIXED_REL, err
            assert err["That"] <= TOL_MIXED_REL and err["That_abs"] <= TOL_MIXED_ABS, err


def test_separable_ragged_tiles_and_units(sa):
    """Separable history sums on a box whose lists are ragged (66 x 8, 66 x
    9 and 8 x 9 points: two row tiles, 32-wide column tiles) with mixed
    degrees, over a meander of several hundred sources (several units)."""
    patch = W.cuboid_patch((2.2e-3, 0.4e-3, 0.3e-3), (22, 4, 3), (2, 1, 2))
    z = float(patch.ctrl[-1, 0, 0, 2])
    scan = W.meander(0.2e-3, 2.0e-3, 0.12e-3, 0.08e-3, 3, z, 180.0, 0.4, 1.5)
    wl = W.Workload("sep", patch, W.MAT_DEFAULT, scan, dt=4e-6, theta=0.5, n_steps=400)
    for prec in (sa.SA_FP64, sa.SA_MIXED):
        err, ctx, m = _lockstep(sa, wl, prec, 400, every=50, hist_mode=2)
        assert ctx.sizes().hist_separable == 1
        assert ctx.sizes().n_src > 256
        if prec == sa.SA_FP64:
            assert err["s_lat"] <= 1e-12 and err["tt_bot"] <= 1e-12, err
            assert err["F"] <= TOL_FP64 and err["That"] <= TOL_FP64, err
        else:
            assert err["s_lat"] <= TOL_MIXED_REL and err["tt_bot"] <= TOL_MIXED_REL, err
            assert err["That"] <= TOL_MIXED_REL and err["That_abs"] <= TOL_MIXED_ABS, err


def test_separable_requires_rectangular_faces(sa):
    """SA_HIST_SEPARABLE is refused on a curved patch; AUTO falls back to the
    pairwise sums there and picks the separable ones on a box."""
    wl = _wl_for(W.distorted_block(weights=True))
    with pytest.raises(sa.SAError) as e:
        gpu_context(wl, sa.SA_MIXED, hist_mode=2)
    assert e.value.status == sa.SA_ERR_ARG
    assert gpu_context(wl, sa.SA_MIXED).sizes().hist_separable == 0
    assert gpu_context(_wl_for(_patch_cases()["cuboid"]), sa.SA_MIXED).sizes().hist_separable == 1


def test_separable_matches_pairwise_full_size(sa):
    """64x64x16 block, 1,200 steps of the 20-track meander: the separable sums
    (64 x 48 lateral and 64 x 64 bottom tiles) against the pairwise ones, in
    both precisions, and the mixed ones against the FP64 pairwise sums."""
    wl = W.block_meander(n_tracks=20, theta=0.5)
    out = {}
    for prec in (sa.SA_FP64, sa.SA_MIXED):
        for hist in (1, 2):
            ctx = gpu_context(wl, prec, use_graph=1, hist_mode=hist)
            assert ctx.sizes().hist_separable == (hist == 2)
            ctx.step(wl.theta, wl.dt, 1200)
            out[prec, hist] = (ctx.field(sa.SA_FIELD_DTDN_LAT), ctx.field(sa.SA_FIELD_TT_BOT),
                               ctx.field(sa.SA_FIELD_THAT))
            ctx.close()
    ref = out[sa.SA_FP64, 1]
    for k in range(2):
        scale = np.abs(ref[k]).max()
        assert np.abs(out[sa.SA_FP64, 2][k] - ref[k]).max() <= 1e-12 * scale
        assert np.abs(out[sa.SA_MIXED, 2][k] - ref[k]).max() <= TOL_MIXED_REL * scale
        assert np.abs(out[sa.SA_MIXED, 1][k] - ref[k]).max() <= TOL_MIXED_REL * scale
    assert np.abs(out[sa.SA_FP64, 2][2] - ref[2]).max() <= 1e-9 * np.abs(ref[2]).max()
    assert np.abs(out[sa.SA_MIXED, 2][2] - ref[2]).max() <= TOL_MIXED_ABS


@pytest.mark.parametrize("case", ["single_source", "contour"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_heat_loss_rates_match_oracle(sa, prec, case):
    """Section 3.1 diagnostic on the quarter-cylinder part, after 8 steps of
    the single source or 40 steps of the contour scan (40 sources): q~ = -k
    n . grad T~ and q^ = -k n . grad T^ at points of the top arc (outward
    normals) and at interior points (random unit normals) against the
    oracle."""
    if case == "single_source":
        wl = W.quarter_cylinder_single_source((4, 2, 2), n_steps=8)
    else:
        wl = W.quarter_cylinder_contour((4, 2, 2), n_steps=40)
    m = _oracle(wl)
    for _ in range(wl.n_steps):
        m.step()
    p = sa.SA_FP64 if prec == "fp64" else sa.SA_MIXED
    ctx = gpu_context(wl, p, pcg_tol=1e-15 if p == sa.SA_FP64 else 1e-10)
    ctx.step(wl.theta, wl.dt, wl.n_steps)
    u = np.linspace(0.02, 0.98, 9)
    xi_arc = np.column_stack([u, np.zeros_like(u), np.ones_like(u)])
    rng = np.random.default_rng(5)
    xi_in = rng.uniform(0.1, 0.9, (6, 3))
    xi = np.vstack([xi_arc, xi_in])
    x = np.array([m.geom.point(v) for v in xi])
    n_arc = np.column_stack([2e-3 - x[:9, 0], -x[:9, 1], np.zeros(9)])
    n_arc /= np.linalg.norm(n_arc, axis=1)[:, None]
    n_in = rng.normal(size=(6, 3))
    n_in /= np.linalg.norm(n_in, axis=1)[:, None]
    nrm = np.vstack([n_arc, n_in])
    _, qt_ref, qh_ref = m.eval_flux(xi, nrm)
    qt, qh = ctx.eval_flux(x, nrm)
    et = np.abs(qt - qt_ref).max() / np.abs(qt_ref).max()
    eh = np.abs(qh - qh_ref).max() / np.abs(qh_ref).max()
    if p == sa.SA_FP64:
        assert et <= 1e-12 and eh <= 1e-9, (et, eh)
    else:   # FP32 history sums; q^ is the gradient of the mixed T^
        assert et <= TOL_MIXED_REL and eh <= 1e-3, (et, eh)


def test_bounded_waits_give_up(sa):
    """Failure detection without a GPU fault: a grid-barrier wait and an
    mbarrier wait that nothing completes give up within their limits (2 s,
    1 s) and flag SA_DEV_TIMEOUT; the device keeps working afterwards."""
    import time
    t0 = time.time()
    bar, mbar = sa.selftest_waits()
    assert bar and mbar
    assert time.time() - t0 < 30
    wl = W.small_block()
    ctx = gpu_context(wl, sa.SA_MIXED)
    ctx.step(wl.theta, wl.dt, 5)
    assert np.isfinite(ctx.field(sa.SA_FIELD_THAT)).all()


def test_degenerate_cases(sa):
    """No sources before the first step; a scan whose laser is off: T^ stays
    T_c exactly; the empty eval call; one element, degree 1."""
    patch = W.cuboid_patch((0.3e-3, 0.3e-3, 0.2e-3), (1, 1, 1), 1)
    scan = W.Scan(path=np.array([[0, 0, 0.2e-3], [0.3e-3, 0.3e-3, 0.2e-3]]),
                  seg_on=np.zeros(1, np.uint8), power=100.0, absorptivity=0.5, speed=1.0)
    wl = W.Workload("off", patch, W.MAT_DEFAULT, scan, dt=1e-5, theta=0.5, n_steps=3)
    ctx = gpu_context(wl, sa.SA_FP64)
    T0 = ctx.field(sa.SA_FIELD_THAT)
    assert np.all(T0 == W.MAT_DEFAULT.T_c)
    st = ctx.step(0.5, 1e-5, 3)
    assert st.n_active_sources == 0
    assert np.all(ctx.field(sa.SA_FIELD_THAT) == W.MAT_DEFAULT.T_c)
    assert ctx.eval_T(np.zeros((0, 3))).shape == (0,)
    # one element, degree 1, a short track: parity holds
    scan2 = W.straight_track((0.1e-3, 0.1e-3, 0.2e-3), (0.2e-3, 0.15e-3, 0.2e-3), 80.0, 0.5, 1.0)
    wl2 = W.Workload("one", patch, W.MAT_DEFAULT, scan2, dt=1e-5, theta=1.0, n_steps=12)
    err, _, _ = _lockstep(sa, wl2, sa.SA_FP64, 12)
    assert err["That"] <= TOL_FP64 and err["F"] <= TOL_FP64, err


def test_checkpoint_resume_is_bit_exact(sa):
    wl = W.small_block(n_el=(6, 5, 3), n_tracks=2)
    a = gpu_context(wl, sa.SA_MIXED)
    a.step(wl.theta, wl.dt, 30)
    n, T, F = a.get_state()
    assert n == 30
    a.step(wl.theta, wl.dt, 25)
    Ta = a.field(sa.SA_FIELD_THAT)
    b = gpu_context(wl, sa.SA_MIXED)
    b.step(wl.theta, wl.dt, 0)          # fixes dt (source spacing) without stepping
    b.set_state(n, T, F)
    b.step(wl.theta, wl.dt, 25)
    assert np.array_equal(b.field(sa.SA_FIELD_THAT), Ta)


def test_graph_replay_equals_direct_launches(sa):
    import torch
    wl = W.small_block(n_el=(6, 5, 3), n_tracks=2)
    s = torch.cuda.Stream()
    a = gpu_context(wl, sa.SA_MIXED, cuda_stream=s, use_graph=1)
    b = gpu_context(wl, sa.SA_MIXED, cuda_stream=s, use_graph=0)
    a.step(wl.theta, wl.dt, 40)
    b.step(wl.theta, wl.dt, 40)
    assert np.array_equal(a.field(sa.SA_FIELD_THAT), b.field(sa.SA_FIELD_THAT))


def test_errors_are_reported(sa):
    wl = W.small_block()
    p = wl.patch
    ctx = sa.Context()
    bad = [k.copy() for k in p.knots]
    bad[0][3], bad[0][4] = bad[0][4], bad[0][3] + 0.01
    with pytest.raises(sa.SAError) as e:
        ctx.create_patch(p.degree, p.n_ctrl, p.ctrl.reshape(-1, 3), None, bad)
    assert e.value.status in (sa.SA_ERR_GEOMETRY,)
    with pytest.raises(sa.SAError) as e:
        ctx.create_patch(p.degree, p.n_ctrl, p.ctrl.reshape(-1, 3),
                         -np.ones(p.n_dof), p.knots)
    assert e.value.status == sa.SA_ERR_GEOMETRY
    c2 = p.ctrl.copy()
    c2[-1, 0, 0, 2] += 1e-5
    with pytest.raises(sa.SAError) as e:
        ctx.create_patch(p.degree, p.n_ctrl, c2.reshape(-1, 3), None, p.knots)
    assert e.value.status == sa.SA_ERR_GEOMETRY
    ctx.create_patch(p.degree, p.n_ctrl, p.ctrl.reshape(-1, 3), None, p.knots)
    with pytest.raises(sa.SAError) as e:
        ctx.step(0.5, 1e-5, 1)
    assert e.value.status == sa.SA_ERR_STATE
    m = wl.material
    ctx.set_material(m.k, m.rho, m.cp, m.T_c)
    s = wl.scan
    ctx.set_scan(s.path, s.seg_on, s.power, s.absorptivity, s.speed, s.spot_radius)
    with pytest.raises(sa.SAError) as e:
        ctx.step(1.5, 1e-5, 1)
    assert e.value.status == sa.SA_ERR_ARG
    ctx.step(0.5, 1e-5, 2)
    with pytest.raises(sa.SAError) as e:
        ctx.step(0.5, 2e-5, 1)
    assert e.value.status == sa.SA_ERR_ARG
    # a capped PCG reports non-convergence and the context stays usable
    # (the first steps carry no flux to the walls and converge at iteration 0)
    c3 = gpu_context(wl, sa.SA_FP64, pcg_max_iter=1, pcg_tol=1e-15, precond=sa.SA_PRECOND_JACOBI)
    with pytest.raises(sa.SAError) as e:
        c3.step(0.5, wl.dt, 80)
    assert e.value.status == sa.SA_ERR_NOT_CONVERGED
    assert np.isfinite(c3.field(sa.SA_FIELD_THAT)).all()


def test_full_size_block_sampled(sa):
    """64x64x16 elements (78,408 control points), degree 2, in the launch
    configuration of the benchmark (mixed history sum, graph replay): the
    history sums at sampled lateral points against the oracle evaluated point
    by point; sampled rows of M and K against the oracle's element sums; and
    the theta-system residual of the computed step."""
    import torch
    from oracle import assembly, pointsource
    from oracle.geometry import PatchGeom
    wl = W.block_meander(n_tracks=20, theta=0.5)
    s = torch.cuda.Stream()
    ctx = gpu_context(wl, sa.SA_MIXED, cuda_stream=s, use_graph=1)
    n_steps = 700
    T_prev = None
    F_prev = None
    ctx.step(wl.theta, wl.dt, n_steps - 1)
    T_prev = ctx.field(sa.SA_FIELD_THAT)
    F_prev = ctx.field(sa.SA_FIELD_F)
    st = ctx.step(wl.theta, wl.dt, 1)
    assert st.n_active_sources == n_steps
    assert ctx.sizes().hist_separable == 1
    geom = PatchGeom(wl.patch)
    from oracle import sources as osrc
    xs = osrc.discretize(wl.scan, wl.dt)
    E = osrc.energy(wl.scan, wl.dt)
    age = pointsource.ages(n_steps, n_steps, wl.dt, wl.material, wl.scan.spot_radius)
    s_gpu = ctx.field(sa.SA_FIELD_DTDN_LAT)
    rng = np.random.default_rng(1)
    sizes = ctx.sizes()
    # include the points nearest to the laser (largest flux) and random ones
    idx = np.unique(np.concatenate([np.argsort(-np.abs(s_gpu))[:32],
                                    rng.integers(0, sizes.q_lat, 96)]))
    ref = np.empty(len(idx))
    for t, q in enumerate(idx):
        f, xi, spans = lateral_xi(geom, int(q))
        dofs, R, dR, x, J = geom.local_eval(xi, spans)
        nvec = {0: -1, 1: 1, 2: -1, 3: 1}[f] * np.eye(3)[{0: 0, 1: 0, 2: 1, 3: 1}[f]]
        ref[t] = pointsource.dTdn_tilde(x[None], nvec[None], xs[:n_steps], age, E,
                                        wl.material)[0]
    scale = np.abs(s_gpu).max()
    assert np.abs(s_gpu[idx] - ref).max() <= TOL_MIXED_REL * scale
    # sampled rows of M and K
    ptr, col, Mv = ctx.matrix(0)
    _, _, Kv = ctx.matrix(1)
    rows = rng.integers(0, sizes.n_dof, 6)
    rho_cp = wl.material.rho * wl.material.cp
    for r in rows:
        els = assembly.elements_touching_dof(geom, int(r))
        Mo, Ko = assembly.assemble_MK(geom, rho_cp, wl.material.k, elements=els)
        sl = slice(ptr[r], ptr[r + 1])
        mo = Mo[int(r)].toarray().ravel()[col[sl]]
        ko = Ko[int(r)].toarray().ravel()[col[sl]]
        assert np.abs(Mv[sl] - mo).max() <= 1e-12 * np.abs(mo).max()
        assert np.abs(Kv[sl] - ko).max() <= 1e-12 * np.abs(ko).max()
    # theta-system residual of the last step (property at any size)
    import scipy.sparse as sp
    n = sizes.n_dof
    M = sp.csr_matrix((Mv, col, ptr), shape=(n, n))
    K = sp.csr_matrix((Kv, col, ptr), shape=(n, n))
    T1 = ctx.field(sa.SA_FIELD_THAT)
    F1 = ctx.field(sa.SA_FIELD_F)
    th, dt = wl.theta, wl.dt
    dirm = geom.dirichlet_dofs()
    lhs = (M / dt + th * K) @ T1
    rhs = (M / dt - (1 - th) * K) @ T_prev + th * F1 + (1 - th) * F_prev
    res = np.linalg.norm((lhs - rhs)[~dirm]) / np.linalg.norm(rhs[~dirm])
    assert res <= 1e-9, res


def test_plate_with_hole_full_size_mixed_vs_fp64(sa):
    """The 48 x 48 x 8 degree-3 plate with a hole (31,416 control variables,
    closed seam): the mixed path against the FP64 path along the contour, at
    points within 20 um of the hole edge and of the outer corners, and the
    theta-system residual of the FP64 step (property at any size)."""
    import torch
    wl = W.plate_with_hole()
    s = torch.cuda.Stream()
    a = gpu_context(wl, sa.SA_MIXED, cuda_stream=s, use_graph=1)
    b = gpu_context(wl, sa.SA_FP64, cuda_stream=s, use_graph=1, pcg_tol=1e-12)
    n = 400
    a.step(wl.theta, wl.dt, n)
    b.step(wl.theta, wl.dt, n - 1)
    T_prev = b.field(sa.SA_FIELD_THAT)
    F_prev = b.field(sa.SA_FIELD_F)
    b.step(wl.theta, wl.dt, 1)
    R, h, t = 0.75e-3, 1.5e-3, 0.5e-3
    ang = np.linspace(0, 2 * np.pi, 64, endpoint=False)
    pts = []
    for d in (2e-6, 10e-6, 20e-6):                   # ring outside the hole edge
        for z in (t, t - 10e-6):
            pts += [((R + d) * np.cos(a_), (R + d) * np.sin(a_), z) for a_ in ang]
    for sx in (-1, 1):                               # the four outer corners
        for sy in (-1, 1):
            for d in (2e-6, 10e-6, 14e-6):
                pts.append((sx * (h - d), sy * (h - d), t))
    pts = np.array(pts)
    Ta = a.eval_T(pts)
    Tb = b.eval_T(pts)
    assert np.isfinite(Ta).all() and np.isfinite(Tb).all()
    assert rel_linf(Ta, Tb) <= TOL_MIXED_REL and np.abs(Ta - Tb).max() <= TOL_MIXED_ABS
    assert Tb.max() > wl.material.T_c + 50.0         # the contour heats the hole edge
    # theta-system residual of the last FP64 step
    import scipy.sparse as sp
    from oracle.geometry import PatchGeom
    nd = b.sizes().n_dof
    ptr, col, Mv = b.matrix(0)
    _, _, Kv = b.matrix(1)
    M = sp.csr_matrix((Mv, col, ptr), shape=(nd, nd))
    K = sp.csr_matrix((Kv, col, ptr), shape=(nd, nd))
    T1 = b.field(sa.SA_FIELD_THAT)
    F1 = b.field(sa.SA_FIELD_F)
    th, dt = wl.theta, wl.dt
    free = ~PatchGeom(wl.patch).dirichlet_dofs()
    lhs = (M / dt + th * K) @ T1
    rhs = (M / dt - (1 - th) * K) @ T_prev + th * F1 + (1 - th) * F_prev
    assert np.linalg.norm((lhs - rhs)[free]) <= 1e-10 * np.linalg.norm(rhs[free])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fast_diagonalization_is_exact_on_a_box(sa, prec):
    """On an affine box the fast-diagonalization preconditioner is A_ff^{-1}
    (up to rounding): every theta-step solve stops after one iteration, with
    the same steps as the oracle; Jacobi needs several."""
    p = sa.SA_FP64 if prec == "fp64" else sa.SA_MIXED
    wl = W.cuboid_single_track(theta=0.5, n_steps=60)
    err, ctx, m = _lockstep(sa, wl, p, 60, every=20, precond=sa.SA_PRECOND_FD)
    if p == sa.SA_FP64:
        assert err["F"] <= TOL_FP64 and err["That"] <= TOL_FP64, err
    else:
        assert err["That"] <= TOL_MIXED_REL and err["That_abs"] <= TOL_MIXED_ABS, err
    st = ctx.step(wl.theta, wl.dt, 20)
    assert st.pcg_iters_max <= 2, st.pcg_iters_max
    c = gpu_context(wl, p, pcg_tol=1e-15 if p == sa.SA_FP64 else 1e-10, precond=sa.SA_PRECOND_JACOBI)
    c.step(wl.theta, wl.dt, 60)
    stj = c.step(wl.theta, wl.dt, 20)
    assert stj.pcg_iters_total > 2 * st.pcg_iters_total


def test_fast_diagonalization_on_the_curved_closed_plate(sa):
    """On the plate with a hole (curved, closed in xi) the preconditioner is
    approximate: the steps match the oracle and the solves need far fewer
    iterations than with Jacobi."""
    wl = W.plate_with_hole(n_el=(8, 4, 2), n_steps=40)
    err, ctx, m = _lockstep(sa, wl, sa.SA_FP64, 40, every=20, precond=sa.SA_PRECOND_FD)
    assert err["F"] <= TOL_FP64 and err["That"] <= TOL_FP64, err
    st = ctx.step(wl.theta, wl.dt, 20)
    c = gpu_context(wl, sa.SA_FP64, pcg_tol=1e-15, precond=sa.SA_PRECOND_JACOBI)
    c.step(wl.theta, wl.dt, 40)
    stj = c.step(wl.theta, wl.dt, 20)
    assert 2 * st.pcg_iters_total < stj.pcg_iters_total, (st.pcg_iters_total, stj.pcg_iters_total)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_history_cutoff_stays_within_its_bound(sa, prec):
    """The opt-in history cutoff (not the paper's method, which keeps the full
    sum): on an elongated box (2.2 x 0.4 x 0.3 mm) under a meander of several
    hundred sources, with eta = 1e-4 the separable sums differ from the
    oracle's full sums by at most eta times the face kind's largest |sum| at
    the previous step (plus the path's tolerance), pairs are skipped, and with
    the default eta = 0 none are."""
    p = sa.SA_FP64 if prec == "fp64" else sa.SA_MIXED
    patch = W.cuboid_patch((2.2e-3, 0.4e-3, 0.3e-3), (22, 4, 3), 2)
    z = float(patch.ctrl[-1, 0, 0, 2])
    scan = W.meander(0.2e-3, 2.0e-3, 0.12e-3, 0.08e-3, 3, z, 180.0, 0.4, 1.5)
    wl = W.Workload("cut", patch, W.MAT_DEFAULT, scan, dt=4e-6, theta=0.5, n_steps=400)
    eta = 1e-4
    tol = 1e-12 if p == sa.SA_FP64 else TOL_MIXED_REL
    m = _oracle(wl)
    ctx = gpu_context(wl, p, hist_mode=2, hist_cutoff=eta,
                      pcg_tol=1e-15 if p == sa.SA_FP64 else 1e-10)
    full = gpu_context(wl, p, hist_mode=2, pcg_tol=1e-15 if p == sa.SA_FP64 else 1e-10)
    prev = None
    skipped = skipped_full = 0
    worst = 0.0
    for step in range(wl.n_steps):
        skipped += ctx.step(wl.theta, wl.dt, 1).hist_pairs_skipped
        skipped_full += full.step(wl.theta, wl.dt, 1).hist_pairs_skipped
        m.step()
        ref = (m.last["s_lat"], m.last["Tt_bot"])
        if prev is not None and (step + 1) % 25 == 0:
            for got, r, M in ((ctx.field(sa.SA_FIELD_DTDN_LAT), ref[0], prev[0]),
                              (ctx.field(sa.SA_FIELD_TT_BOT), ref[1], prev[1])):
                err = np.abs(got - r).max()
                allowed = eta * M * (1 + 1e-3) + tol * np.abs(r).max()
                assert err <= allowed, (step, err, allowed)
                worst = max(worst, err / (eta * M))
        prev = (np.abs(ref[0]).max(), np.abs(ref[1]).max())
    assert skipped > 0 and skipped_full == 0
    print(f"\ncutoff eta {eta}: {skipped} pairs skipped, largest error {worst:.3f} eta M")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_two_lasers_superposed_match_the_multi_laser_oracle(sa, prec):
    """Two lasers on the cuboid (reading R22): one context per laser, each
    stepped on its own, evaluated together by sa_eval_T_superposed, against
    the oracle that sums both lasers' sources and runs one theta-scheme.
    Host and device points give the same values; contexts at different steps
    are refused."""
    import torch
    from oracle.solver import MultiLaserModel
    n_steps = 40
    wl, scans = W.two_lasers_cuboid(n_steps=n_steps)
    m = MultiLaserModel(wl, scans)
    m.run(n_steps)
    p = sa.SA_FP64 if prec == "fp64" else sa.SA_MIXED
    tol = 1e-15 if prec == "fp64" else 1e-10
    wls = [W.Workload(f"laser{l}", wl.patch, wl.material, sc, dt=wl.dt, theta=wl.theta,
                      n_steps=n_steps) for l, sc in enumerate(scans)]
    ctxs = [gpu_context(w, p, pcg_tol=tol) for w in wls]
    for c in ctxs:
        c.step(wl.theta, wl.dt, n_steps)
    rng = np.random.default_rng(11)
    xi = rng.uniform(0, 1, (30, 3))
    xi[:10, 2] = 1.0
    xi[:5, 0] = rng.uniform(0.15, 0.30, 5)      # near the two laser fronts
    xi[:5, 1] = np.where(np.arange(5) % 2 == 0, 0.3, 0.7)
    x, T_ref = m.eval_T(xi)
    T = sa.eval_T_superposed(ctxs, x)
    assert np.abs(T_ref - wl.material.T_c).max() > 1.0      # the lasers heat the part
    if prec == "fp64":
        assert rel_linf(T, T_ref) <= TOL_FP64
    else:
        assert rel_linf(T, T_ref) <= TOL_MIXED_REL
        assert np.abs(T - T_ref).max() <= TOL_MIXED_ABS
    # device points and output: the same values
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    Td = torch.empty(len(x), dtype=torch.float64, device="cuda")
    sa.eval_T_superposed(ctxs, xd, out=Td, on_device=True)
    torch.cuda.synchronize()
    assert np.array_equal(Td.cpu().numpy(), T)
    # contexts at different steps are refused
    ctxs[1].step(wl.theta, wl.dt, 1)
    with pytest.raises(sa.SAError):
        sa.eval_T_superposed(ctxs, x)
    for c in ctxs:
        c.close()
