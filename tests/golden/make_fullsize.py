"""Write the full-size goldens ``tests/golden/fullsize_<case>.npz`` from the
FP64 oracle alone (``oracle/``) on the seeded inputs of ``workloads/``.

Each case steps the oracle's ``Model`` (Sections 2.1-2.4: history sums,
Neumann load, bottom L2 projection, theta-step by a sparse LU of the free
block) from step 0 to the case's last step and stores, at that step:

  T_hat   the correction field's control variables      (n_dof)
  F       the Neumann load F^{n}                          (n_dof)
  s_lat   dT~/dn at the lateral quadrature points         (q_lat)
  tt_bot  T~ at the bottom quadrature points              (q_bot)
  x, T    T = T~ + T^ at evaluation points                (n, 3), (n)
  meta    JSON: workload, steps, host timings (setup, factorisation,
          history sums, solves) and the worker count

The history sums of a step are split over a pool of worker processes by
quadrature point (each point's sum is still the oracle's own, over the
sources in order), and those of the next step run while the parent solves
the current one; everything else runs in the parent as written.

Usage: python tests/golden/make_fullsize.py CASE [CASE ...] [--procs N]
Cases: block (writes block600 and block10tracks), block600, block10tracks, plate, batch,
learned.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W                      # noqa: E402
from oracle import pointsource             # noqa: E402
from oracle.solver import Model            # noqa: E402

# config-3 instances whose goldens are stored (see batch_ids)
BATCH_IDS_FILE = os.path.join(HERE, "fullsize_batch_ids.txt")
LEARNED_HELDOUT = 1000          # learned_scan index of the held-out scan

_W = {}


def _init(lat_x, lat_n, bot_x, E, mat, s_img):
    _W.update(lat_x=lat_x, lat_n=lat_n, bot_x=bot_x, E=E, mat=mat, s_img=s_img)


def _part(args):
    kind, q0, q1, xs, age = args
    if kind == "lat":
        return pointsource.dTdn_tilde(_W["lat_x"][q0:q1], _W["lat_n"][q0:q1], xs, age, _W["E"],
                                      _W["mat"], _W["s_img"])
    return pointsource.T_tilde(_W["bot_x"][q0:q1], xs, age, _W["E"], _W["mat"], _W["s_img"])


class PooledModel(Model):
    """The oracle's model with the per-point history sums of a step spread
    over worker processes (same functions, same per-point order)."""

    def __init__(self, wl, procs):
        t0 = time.time()
        super().__init__(wl)
        self.t_setup = time.time() - t0
        self.procs = procs
        self.t_hist = 0.0
        self.t_solve = 0.0
        self.pending = {}
        self.pool = mp.get_context("spawn").Pool(
            procs, initializer=_init,
            initargs=(self.lat["x"], self.lat["n"], self.bot["x"], self.E, self.mat, self.s_img))

    def close(self):
        self.pool.close()
        self.pool.join()

    def _launch(self, kind, n):
        """Start the history sums of step n over the pool (asynchronous)."""
        n_pts = len((self.lat if kind == "lat" else self.bot)["x"])
        K = self.n_active(n)
        xs, age = self.xs[:K], self.source_ages(n)
        parts = max(1, min(4 * self.procs, n_pts // 256))
        cuts = np.linspace(0, n_pts, parts + 1).astype(int)
        self.pending[(kind, n)] = self.pool.map_async(
            _part, [(kind, int(a), int(b), xs, age) for a, b in zip(cuts[:-1], cuts[1:])])

    def _collect(self, kind, n):
        if (kind, n) not in self.pending:
            self._launch(kind, n)
        return np.concatenate(self.pending.pop((kind, n)).get())

    def flux_normal_derivative(self, n):
        if self.n_active(n) == 0 or self.lat is None:
            return super().flux_normal_derivative(n)
        t0 = time.time()
        out = self._collect("lat", n)
        self.t_hist += time.time() - t0
        return out

    def T_tilde_at(self, x, n):
        if self.n_active(n) == 0 or self.bot is None or x is not self.bot["x"]:
            return super().T_tilde_at(x, n)
        t0 = time.time()
        out = self._collect("bot", n)
        self.t_hist += time.time() - t0
        # the next step's sums run on the pool while this step's solve runs
        if self.n_active(n + 1) > 0:
            self._launch("lat", n + 1)
            self._launch("bot", n + 1)
        return out

    def step(self):
        t0 = time.time()
        h0 = self.t_hist
        out = super().step()
        self.t_solve += (time.time() - t0) - (self.t_hist - h0)
        return out


def _block_eval_xi(m, rng, n_rand=48, n_near=16):
    """Random interior and top-face points, plus top-face points within
    100 um of the last source (the hottest region)."""
    xi = rng.uniform(0.01, 0.99, (n_rand, 3))
    xi[: n_rand // 2, 2] = 1.0
    lo = m.wl.patch.ctrl.reshape(-1, 3).min(0)
    hi = m.wl.patch.ctrl.reshape(-1, 3).max(0)
    K = m.n_active(m.n)
    if K > 0:
        c = m.xs[K - 1]
        r = rng.uniform(0.0, 100e-6, n_near)
        a = rng.uniform(0.0, 2 * np.pi, n_near)
        near = np.column_stack([c[0] + r * np.cos(a), c[1] + r * np.sin(a), np.full(n_near, hi[2])])
        near = np.clip(near, lo + 1e-7, hi - 1e-7)
        near[:, 2] = hi[2]
        xi = np.vstack([xi, (near - lo) / (hi - lo)])
    return xi


def _plate_eval_xi():
    """Points within 20 um of the hole edge (eta near 0, on the top face and
    10 um below it) at 32 angles, and near the four outer corners (eta = 1
    at the C0 corners of the ring, u = 0, 1/4, 1/2, 3/4)."""
    xi = []
    for u in np.linspace(0.0, 1.0, 32, endpoint=False):
        for v in (0.0, 0.004, 0.012):
            for w in (1.0, 0.98):
                xi.append((u, v, w))
    for u in (0.0, 0.25, 0.5, 0.75):
        for v in (1.0, 0.995):
            for w in (1.0, 0.5):
                xi.append((u, v, w))
    return np.array(xi)


def run_case(name, wl, snapshots, procs, xi_fn, extra=None):
    """Step the oracle to the largest step of ``snapshots`` ({step: name})
    and write a golden at each of them."""
    n_steps = max(snapshots)
    print(f"[{name}] {wl.name}: {n_steps} steps", flush=True)
    t0 = time.time()
    m = PooledModel(wl, procs)
    t_fact = time.time() - t0 - m.t_setup
    print(f"[{name}] setup {m.t_setup:.1f} s, factorisation {t_fact:.1f} s, n_dof {m.geom.n_dof}",
          flush=True)
    t1 = time.time()
    for k in range(n_steps):
        m.step()
        if (k + 1) % 200 == 0:
            print(f"[{name}] step {k + 1}: history {m.t_hist:.0f} s, solve {m.t_solve:.0f} s",
                  flush=True)
        if k + 1 in snapshots:
            _write(snapshots[k + 1], m, wl, procs, xi_fn, t_fact, time.time() - t1, extra)
    m.close()


def _write(name, m, wl, procs, xi_fn, t_fact, t_run, extra):
    rng = np.random.default_rng(20251120)
    xi = xi_fn(m, rng)
    x, T = m.eval_T(xi)
    meta = dict(workload=wl.name, n_steps=int(m.n), theta=wl.theta, dt=wl.dt, s_img=m.s_img,
                n_dof=int(m.geom.n_dof), q_lat=int(len(m.lat["x"])), q_bot=int(len(m.bot["x"])),
                n_active=int(m.n_active(m.n)), procs=procs, host_cpu=_cpu(),
                setup_s=m.t_setup, factor_s=t_fact, run_s=t_run, history_s=m.t_hist,
                solve_s=m.t_solve)
    if extra:
        meta.update(extra)
    out = os.path.join(HERE, f"fullsize_{name}.npz")
    np.savez_compressed(out, T_hat=m.T_hat, F=m.F, s_lat=m.last["s_lat"],
                        tt_bot=m.last["Tt_bot"], x=x, T=T, meta=json.dumps(meta))
    print(f"[{name}] wrote {out}: {json.dumps(meta)}", flush=True)


def _cpu():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def batch_ids():
    """The stored config-3 instances (ids 0..255 of the sweep): the largest
    in-plane patch, the thickest one and the smallest one."""
    size = []
    for i in range(256):
        wl = W.batched_instance(i)
        n0, n1, n2 = wl.patch.n_ctrl
        size.append((i, n0 * n1, n2, n0 * n1 * n2))
    big = max(size, key=lambda t: (t[1], t[2]))[0]
    thick = max(size, key=lambda t: (t[2], t[1]))[0]
    small = min(size, key=lambda t: t[3])[0]
    ids = []
    for i in (big, thick, small):
        if i not in ids:
            ids.append(i)
    return ids


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cases", nargs="+")
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    for case in a.cases:
        if case == "block":
            # 600 steps, and the 10-track prefix (584 sources per track)
            wl = W.block_meander(n_tracks=20, theta=0.5)
            run_case(case, wl, {600: "block600", 10 * 584: "block10tracks"}, a.procs,
                     _block_eval_xi)
        elif case == "block10tracks":
            wl = W.block_meander(n_tracks=20, theta=0.5)
            run_case(case, wl, {10 * 584: "block10tracks"}, a.procs, _block_eval_xi)
        elif case == "block600":
            wl = W.block_meander(n_tracks=20, theta=0.5)
            run_case(case, wl, {600: "block600"}, a.procs, _block_eval_xi)
        elif case == "plate":
            wl = W.plate_with_hole()
            run_case(case, wl, {wl.n_steps: "plate"}, a.procs, lambda m, rng: _plate_eval_xi())
        elif case == "learned":
            base = W.block_meander(n_tracks=20, theta=0.5)
            wl = W.Workload(f"learned_heldout_{LEARNED_HELDOUT}", base.patch, base.material,
                            W.learned_scan(LEARNED_HELDOUT), dt=base.dt, theta=base.theta,
                            n_steps=400)
            run_case(case, wl, {400: "learned"}, a.procs, _block_eval_xi)
        elif case == "batch":
            ids = batch_ids()
            with open(BATCH_IDS_FILE, "w") as f:
                f.write("# config-3 instance ids with stored goldens (written by make_fullsize.py)\n")
                f.write(" ".join(str(i) for i in ids) + "\n")
            for i in ids:
                wl = W.batched_instance(i)
                run_case(f"batch{i}", wl, {wl.n_steps: f"batch{i}"}, a.procs, _block_eval_xi,
                         extra=dict(instance_id=i))
        else:
            raise SystemExit(f"unknown case {case}")


if __name__ == "__main__":
    main()
