"""sa_eval_T_noalloc: the allocation-free variant of sa_eval_T, for callers
that cannot allocate device memory (latency-critical loops, code under a
framework allocator that owns the free memory).  Called through the C ABI
with caller-allocated device buffers; its output must match sa_eval_T's on
two calls in a row.  Named to be collected last."""
import ctypes

import numpy as np
import pytest

import workloads as W

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


def _noalloc(sa, ctx, pts_dev, out_dev):
    st = sa.lib.sa_eval_T_noalloc(ctx.ptr, ctypes.c_void_p(pts_dev.data_ptr()),
                                  int(pts_dev.shape[0]), ctypes.c_void_p(out_dev.data_ptr()))
    return st


def test_noalloc_eval_matches_sa_eval_T_twice(sa):
    import torch
    wl = W.small_block(n_el=(6, 5, 3), n_tracks=2)
    ctx = sa.context_from_workload(wl, precision=sa.SA_FP64)
    rng = np.random.default_rng(5)
    lo = wl.patch.ctrl.reshape(-1, 3).min(0)
    hi = wl.patch.ctrl.reshape(-1, 3).max(0)
    pts = lo + (hi - lo) * rng.uniform(0.02, 0.98, (57, 3))
    pts[:6, 2] = hi[2]                               # on the top face, near the sources
    d_pts = torch.tensor(pts, dtype=torch.float64, device="cuda").contiguous()
    d_out = torch.empty(len(pts), dtype=torch.float64, device="cuda")
    for n_steps in (35, 20):                         # two calls in a row, at two states
        ctx.step(wl.theta, wl.dt, n_steps)
        ref = ctx.eval_T(pts)
        assert _noalloc(sa, ctx, d_pts, d_out) == sa.SA_OK, sa.lib.sa_last_error(ctx.ptr)
        got = d_out.cpu().numpy()
        assert np.isfinite(ref).all()
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


def test_noalloc_eval_in_a_mixed_context(sa):
    """In an SA_MIXED context the call still evaluates in FP64: against the
    FP64 oracle it stays within the mixed tolerance, and so does its
    difference from sa_eval_T (FP32 sums there), on two calls in a row."""
    import torch
    from oracle.solver import Model
    wl = W.small_block(n_el=(6, 5, 3), n_tracks=2)
    m = Model(wl)
    ctx = sa.context_from_workload(wl, precision=sa.SA_MIXED)
    rng = np.random.default_rng(9)
    xi = rng.uniform(0.02, 0.98, (41, 3))
    xi[:8, 2] = 1.0                                  # on the top face, near the sources
    for n_steps in (35, 20):
        ctx.step(wl.theta, wl.dt, n_steps)
        m.run(n_steps)
        x, T_ref = m.eval_T(xi)
        d_pts = torch.tensor(x, dtype=torch.float64, device="cuda").contiguous()
        d_out = torch.empty(len(x), dtype=torch.float64, device="cuda")
        assert _noalloc(sa, ctx, d_pts, d_out) == sa.SA_OK, sa.lib.sa_last_error(ctx.ptr)
        got = d_out.cpu().numpy()
        mixed = ctx.eval_T(x)
        for a in (got, mixed):
            assert np.abs(a - T_ref).max() <= 1e-4 * np.abs(T_ref).max()
            assert np.abs(a - T_ref).max() <= 0.05
        assert np.abs(got - mixed).max() <= 0.05


def test_noalloc_eval_allocates_no_device_memory(sa):
    """The defining property: after the context has stepped, calls with more
    points than any earlier evaluation leave the device's free memory
    unchanged (a stray cudaMalloc of a point or output buffer would show)."""
    import torch
    wl = W.small_block(n_el=(6, 5, 3), n_tracks=2)
    ctx = sa.context_from_workload(wl, precision=sa.SA_MIXED)
    ctx.step(wl.theta, wl.dt, 30)
    ctx.eval_T(np.zeros((2, 3)))
    lo = wl.patch.ctrl.reshape(-1, 3).min(0)
    hi = wl.patch.ctrl.reshape(-1, 3).max(0)
    pts = lo + (hi - lo) * np.random.default_rng(3).uniform(0.02, 0.98, (20_000, 3))
    d_pts = torch.tensor(pts, dtype=torch.float64, device="cuda").contiguous()
    d_out = torch.empty(len(pts), dtype=torch.float64, device="cuda")
    assert _noalloc(sa, ctx, d_pts, d_out) == sa.SA_OK     # first call: address look-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert _noalloc(sa, ctx, d_pts, d_out) == sa.SA_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.isfinite(d_out.cpu().numpy()).all()


def test_noalloc_eval_rejects_sizes_beyond_its_limit(sa):
    # 300,001 sources on a 0.3 mm track (dt = 1 ns) exceed the 65,536 limit
    patch = W.cuboid_patch((0.4e-3, 0.4e-3, 0.2e-3), (2, 2, 1), 2)
    scan = W.straight_track((0.05e-3, 0.2e-3, 0.2e-3), (0.35e-3, 0.2e-3, 0.2e-3), 50.0, 0.5, 1.0)
    wl = W.Workload("many", patch, W.MAT_DEFAULT, scan, dt=1e-9, theta=0.5, n_steps=0)
    ctx = sa.context_from_workload(wl, precision=sa.SA_FP64)
    ctx.step(wl.theta, wl.dt, 0)
    assert ctx.sizes().n_src > 65536
    import torch
    d_pts = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    d_out = torch.empty(4, dtype=torch.float64, device="cuda")
    assert _noalloc(sa, ctx, d_pts, d_out) == sa.SA_ERR_ARG
    assert b"65536" in sa.lib.sa_last_error(ctx.ptr)
