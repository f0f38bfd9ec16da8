"""The warm-start network: GPU forward/backward (tensor-core GEMMs) against
the FP64 oracle network, training, and its use as the PCG initial guess."""
import numpy as np
import pytest

import workloads as W
from tests._common import TOL_MIXED_ABS, TOL_MIXED_REL, gpu_context, rel_linf

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


def _bf16_round(a):
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _unpack(p, sizes):
    out, o = [], 0
    for i, j in zip(sizes[:-1], sizes[1:]):
        W = p[o:o + i * j].reshape(j, i)
        o += i * j
        b = p[o:o + j]
        o += j
        out.append((W.astype(np.float64), b.astype(np.float64)))
    return out


# Per-entry bound of the device's rounding: the device stores the hidden
# activations and the back-propagated gradients in BF16 (unit roundoff
# 2^-9 each) for its tensor-core products and sums in FP32; over four layers
# forward and back that is at most about eight BF16 roundings relative to the
# sum of the absolute values of the products that make up an entry.  A wrong
# row, sign or transposition moves an entry by the order of that sum.
KAPPA_BF16 = 8 * 2.0 ** -8


def test_mlp_gradients_match_oracle(sa):
    """Every entry of every weight and bias gradient, and of the output,
    against the FP64 oracle network on the same BF16 weights and inputs,
    within KAPPA_BF16 times the entry's absolute sum of products."""
    import torch
    from oracle import mlp as omlp
    n_in, H, n_out, B = 37, 48, 53, 19           # ragged against the 64-wide tiles
    net = sa.MLP(n_in, H, n_out, seed=7)
    rng = np.random.default_rng(3)
    X = _bf16_round(rng.normal(size=(B, n_in)))
    Y = _bf16_round(rng.normal(size=(B, n_out)))
    Xd = torch.tensor(X, dtype=torch.bfloat16, device="cuda")
    Yd = torch.tensor(Y, dtype=torch.bfloat16, device="cuda")
    loss, g = net.gradients(Xd, Yd)
    sizes = [n_in, H, H, H, n_out]
    p = net.params()
    params = [(_bf16_round(W).astype(np.float64), b) for W, b in _unpack(p, sizes)]
    ref_loss, ref_grads, deltas = omlp.loss_and_grads(params, X.astype(np.float64),
                                                      Y.astype(np.float64), with_deltas=True)
    assert abs(loss - ref_loss) <= KAPPA_BF16 * abs(ref_loss)
    gl = _unpack(g, sizes)
    for l, ((gW, gb), (rW, rb), (dl, hin)) in enumerate(zip(gl, ref_grads, deltas)):
        bound_W = KAPPA_BF16 * (np.abs(dl).T @ np.abs(hin)) + 1e-30
        bound_b = KAPPA_BF16 * np.abs(dl).sum(axis=0) + 1e-30
        assert np.all(np.abs(gW - rW) <= bound_W), (l, np.max(np.abs(gW - rW) / bound_W))
        assert np.all(np.abs(gb - rb) <= bound_b), (l, np.max(np.abs(gb - rb) / bound_b))
    # forward output, entry by entry
    out = torch.empty((B, n_out), dtype=torch.float32, device="cuda")
    net.forward(Xd, out)
    ref_out, cache = omlp.forward(params, X.astype(np.float64))
    W4, b4 = params[3]
    h3 = cache[3][0]
    bound = KAPPA_BF16 * (np.abs(h3) @ np.abs(W4).T + np.abs(b4)) + 1e-30
    assert np.all(np.abs(out.cpu().numpy() - ref_out) <= bound)


@pytest.mark.parametrize("n_in", [8516, 37])
def test_mlp_single_sample_forward(sa, n_in):
    """One sample runs as four GEMVs (the warm start inside a step): its
    output equals the oracle's entry by entry within the rounding bound, and
    the batched (tensor-core) forward of the same sample; n_in = 8516 is the
    block's input width (rows of 4-weight loads), 37 the scalar path."""
    import torch
    from oracle import mlp as omlp
    H, n_out = 256, 997
    net = sa.MLP(n_in, H, n_out, seed=11)
    rng = np.random.default_rng(4)
    X = _bf16_round(rng.normal(size=(2, n_in)))
    X[1] = X[0]
    Xd = torch.tensor(X, dtype=torch.bfloat16, device="cuda")
    one = torch.empty((1, n_out), dtype=torch.float32, device="cuda")
    two = torch.empty((2, n_out), dtype=torch.float32, device="cuda")
    net.forward(Xd[:1].contiguous(), one)
    net.forward(Xd, two)
    sizes = [n_in, H, H, H, n_out]
    params = [(_bf16_round(W).astype(np.float64), b) for W, b in _unpack(net.params(), sizes)]
    ref, cache = omlp.forward(params, X[:1].astype(np.float64))
    W4, b4 = params[3]
    bound = KAPPA_BF16 * (np.abs(cache[3][0]) @ np.abs(W4).T + np.abs(b4)) + 1e-30
    o1 = one.cpu().numpy()
    assert np.all(np.abs(o1 - ref) <= bound)
    assert np.all(np.abs(o1[0] - two.cpu().numpy()[0]) <= 2 * bound[0])


def test_mlp_training_fits_a_linear_map(sa):
    import torch
    rng = np.random.default_rng(5)
    n_in, n_out = 64, 96
    A = rng.normal(size=(n_out, n_in)) / np.sqrt(n_in)
    X = rng.normal(size=(1024, n_in))
    Y = X @ A.T
    Xd = torch.tensor(X, dtype=torch.bfloat16, device="cuda")
    Yd = torch.tensor(Y, dtype=torch.bfloat16, device="cuda")
    net = sa.MLP(n_in, 128, n_out, seed=1)
    first = net.train_step(Xd[:128], Yd[:128], 1e-3)
    for ep in range(40):
        for k in range(0, 1024, 128):
            last = net.train_step(Xd[k:k + 128], Yd[k:k + 128], 1e-3, want_loss=(k == 896))
    assert last < 0.2 * first, (first, last)


def _inputs_for(ctx, patch):
    """Free control variables on the lateral faces and the first free layer
    above the bottom (internal free order = natural order without the bottom
    layer)."""
    n0, n1, n2 = patch.n_ctrl
    idx = []
    for k in range(1, n2):
        for j in range(n1):
            for i in range(n0):
                if k == 1 or i in (0, n0 - 1) or j in (0, n1 - 1):
                    idx.append((k * n1 + j) * n0 + i - n0 * n1)
    return np.array(idx, dtype=np.int32)


def test_warm_start_keeps_the_solution_and_reports_iterations(sa):
    import torch
    wl = W.small_block(n_el=(10, 8, 4), n_tracks=3, size=(0.625e-3, 0.5e-3, 0.25e-3), speed=1.2,
                       power=180.0, dt=5e-6)
    n_free = gpu_context(wl, sa.SA_MIXED).sizes().n_free
    idx = _inputs_for(None, wl.patch)
    # training data from two other scans (different power / speed)
    X = torch.empty((400, len(idx)), dtype=torch.bfloat16, device="cuda")
    Y = torch.empty((400, n_free), dtype=torch.bfloat16, device="cuda")
    row = 0
    for P, v in ((140.0, 1.0), (220.0, 1.5)):
        wtr = W.small_block(n_el=(10, 8, 4), n_tracks=3, size=(0.625e-3, 0.5e-3, 0.25e-3), speed=v,
                            power=P, dt=5e-6)
        c = gpu_context(wtr, sa.SA_MIXED)
        c.set_recorder(X[row:], Y[row:], idx)
        c.step(0.5, 5e-6, 200)
        row += c.recorded()
        c.set_recorder(None, None, None)
    assert row == 400
    net = sa.MLP(len(idx), 256, n_free, seed=3)
    for ep in range(30):
        perm = torch.randperm(row, device="cuda")
        for k in range(0, row, 64):
            sel = perm[k:k + 64]
            net.train_step(X[sel].contiguous(), Y[sel].contiguous(), 1e-3, want_loss=False)
    cold = gpu_context(wl, sa.SA_MIXED)
    warm = gpu_context(wl, sa.SA_MIXED)
    warm.set_warm_start(net, idx)
    it_cold = it_warm = used = 0
    for s in range(150):
        a = cold.step(0.5, 5e-6, 1)
        b = warm.step(0.5, 5e-6, 1)
        it_cold += a.pcg_iters_last
        it_warm += b.pcg_iters_last
        used += b.ws_used_last
    Tc = cold.field(sa.SA_FIELD_THAT)
    Tw = warm.field(sa.SA_FIELD_THAT)
    assert rel_linf(Tw, Tc) <= TOL_MIXED_REL and np.abs(Tw - Tc).max() <= TOL_MIXED_ABS
    print(f"warm start: PCG iterations {it_warm} vs cold {it_cold}, learned guess used in {used}/150 steps")
    assert it_warm <= 1.05 * it_cold + 5
