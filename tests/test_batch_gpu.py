"""Batched stepping (one launch per stage for many uneven instances) against
the same instances stepped one by one, and against the oracle."""
import numpy as np
import pytest

import workloads as W
from tests._common import TOL_FP64, TOL_MIXED_ABS, TOL_MIXED_REL, gpu_context, rel_linf

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


def _instances():
    """Uneven patches, scans and powers; one material and dt."""
    out = []
    specs = [((5, 4, 2), 120.0, 1.0, 2), ((9, 6, 3), 200.0, 1.4, 3), ((3, 3, 2), 90.0, 0.7, 1),
             ((7, 7, 4), 260.0, 1.8, 2), ((4, 8, 3), 150.0, 1.1, 2)]
    for k, (n_el, P, v, nt) in enumerate(specs):
        size = tuple(62.5e-6 * np.array(n_el))
        wl = W.small_block(n_el=n_el, n_tracks=nt, size=size, speed=v, power=P, dt=5e-6)
        out.append(wl)
    return out


@pytest.mark.parametrize("hist", ["separable", "pairwise"])
@pytest.mark.parametrize("precond", ["fd", "jacobi"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_matches_single_contexts(sa, prec, precond, hist):
    import torch
    p = sa.SA_FP64 if prec == "fp64" else sa.SA_MIXED
    pc = sa.SA_PRECOND_AUTO if precond == "fd" else sa.SA_PRECOND_JACOBI
    hm = sa.SA_HIST_SEPARABLE if hist == "separable" else sa.SA_HIST_PAIRWISE
    wls = _instances()
    s = torch.cuda.Stream()
    tol = 1e-15 if p == sa.SA_FP64 else 1e-10
    ctxs = [gpu_context(wl, p, pcg_tol=tol, precond=pc, hist_mode=hm) for wl in wls]
    singles = [gpu_context(wl, p, pcg_tol=tol, precond=pc, hist_mode=hm) for wl in wls]
    batch = sa.Batch(ctxs, precision=p, pcg_tol=tol, cuda_stream=s, use_graph=1, precond=pc,
                     hist_mode=hm)
    n = 60
    batch.step(0.5, 5e-6, n)
    for c in singles:
        c.step(0.5, 5e-6, n)
    m_it, b_it = batch.iters()
    assert (m_it >= 0).all() and (b_it >= 0).all()
    if precond == "fd":   # boxes: the preconditioners are the inverses
        assert m_it.max() <= 2, m_it
        assert b_it.max() <= 3, b_it
    for i, c in enumerate(singles):
        Tb = batch.field(i, sa.SA_FIELD_THAT)
        Ts = c.field(sa.SA_FIELD_THAT)
        if p == sa.SA_FP64:
            assert rel_linf(Tb, Ts) <= 1e-11, i
        else:
            assert rel_linf(Tb, Ts) <= TOL_MIXED_REL and np.abs(Tb - Ts).max() <= TOL_MIXED_ABS, i
        # separable, mixed: the batch sums a tile's sources in one unit, the
        # context in several (other FP32 rounding, up to ~(32 + chunks) ulp)
        assert rel_linf(batch.field(i, sa.SA_FIELD_DTDN_LAT), c.field(sa.SA_FIELD_DTDN_LAT)) <= (
            1e-12 if p == sa.SA_FP64 else (1e-5 if hist == "separable" else 1e-6))


def test_batch_fp64_against_oracle(sa):
    from oracle.solver import Model
    wls = _instances()[:3]
    ctxs = [gpu_context(wl, sa.SA_FP64, pcg_tol=1e-15) for wl in wls]
    batch = sa.Batch(ctxs, precision=sa.SA_FP64, pcg_tol=1e-15)
    n = 40
    batch.step(0.5, 5e-6, n)
    for i, wl in enumerate(wls):
        m = Model(wl)
        m.run(n)
        assert rel_linf(batch.field(i, sa.SA_FIELD_THAT), m.T_hat) <= TOL_FP64, i
        assert rel_linf(batch.field(i, sa.SA_FIELD_F), m.F) <= TOL_FP64, i


def test_batch_autotune_and_cache(sa, tmp_path):
    wls = _instances()
    ctxs = [gpu_context(wl, sa.SA_MIXED) for wl in wls]
    batch = sa.Batch(ctxs, precision=sa.SA_MIXED)
    batch.step(0.5, 5e-6, 30)
    path = str(tmp_path / "tune.jsonl")
    P, NW, ms = batch.autotune(path)
    assert P in (1, 2, 4) and NW in (4, 8) and ms > 0
    P2, NW2, ms2 = batch.autotune(path)
    assert (P2, NW2) == (P, NW) and ms2 == -1.0
    batch.step(0.5, 5e-6, 10)
    assert np.isfinite(batch.field(0, sa.SA_FIELD_THAT)).all()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_tune_keeps_the_state_and_the_results(sa, prec, tmp_path):
    """sa_batch_tune times the separable tile shapes and the solve grid from
    a saved copy of the state: the batch does not advance, later steps equal
    those of an untuned batch (other tile shapes only reorder the sums), and
    the cached choice is applied without timing."""
    import torch
    p = sa.SA_FP64 if prec == "fp64" else sa.SA_MIXED
    tol = 1e-15 if p == sa.SA_FP64 else 1e-10
    wls = _instances()
    s = torch.cuda.Stream()
    tuned = sa.Batch([gpu_context(wl, p, pcg_tol=tol) for wl in wls], precision=p, pcg_tol=tol,
                     cuda_stream=s, use_graph=1)
    plain = sa.Batch([gpu_context(wl, p, pcg_tol=tol) for wl in wls], precision=p, pcg_tol=tol,
                     cuda_stream=s, use_graph=1)
    tuned.step(0.5, 5e-6, 30)
    plain.step(0.5, 5e-6, 30)
    T0 = tuned.field(0, sa.SA_FIELD_THAT)
    path = str(tmp_path / "shapes.jsonl")
    sh = tuned.tune(path, at_step=200)
    assert sh["hist_separable"] == 1 and sh["step_ms"] > 0
    assert sh["tj_lat"] in (64, 48, 32) and sh["tj_bot"] in (64, 48, 32)
    assert sh["units_per_tile"] in (1, 2, 4) and 1 <= sh["pcg_grid"]
    assert tuned.shapes()["pcg_grid"] == sh["pcg_grid"]
    assert np.array_equal(tuned.field(0, sa.SA_FIELD_THAT), T0)       # state restored
    st = tuned.step(0.5, 5e-6, 30)
    plain.step(0.5, 5e-6, 30)
    assert st.step_index == 60
    for i in range(len(wls)):
        a, b = tuned.field(i, sa.SA_FIELD_THAT), plain.field(i, sa.SA_FIELD_THAT)
        if p == sa.SA_FP64:
            assert rel_linf(a, b) <= 1e-11, i
        else:
            assert rel_linf(a, b) <= TOL_MIXED_REL and np.abs(a - b).max() <= TOL_MIXED_ABS, i
    again = sa.Batch([gpu_context(wl, p, pcg_tol=tol) for wl in wls], precision=p, pcg_tol=tol,
                     cuda_stream=s, use_graph=1)
    again.step(0.5, 5e-6, 30)
    sh2 = again.tune(path, at_step=200)
    assert sh2["step_ms"] == -1.0
    assert {k: v for k, v in sh2.items() if k != "step_ms"} == {k: v for k, v in sh.items() if k != "step_ms"}
