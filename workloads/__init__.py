"""Seeded synthetic workloads: patches, scans, materials and step counts.

This module only builds INPUT data (control nets, knot vectors, scan
polylines, parameters drawn from a seeded generator).  It holds none of the
method's arithmetic: no basis functions, no point-source solution, no
quadrature and no solver.  Both the FP64 oracle (``oracle/``) and the GPU
library's tests and benchmark consume these descriptions.

Units are SI throughout (m, s, W, J, K).  A control net is stored as an array
of shape ``(n2, n1, n0, 3)``: the first parametric index (xi) runs fastest,
matching the C-ABI layout ``ctrl_xyz[((k*n1 + j)*n0 + i)*3 + c]``.

Face order used everywhere: 0 xi=0, 1 xi=1, 2 eta=0, 3 eta=1, 4 zeta=0,
5 zeta=1.  Face kinds: NONE (no boundary term; the top face, Section 2.1 of
the paper says its adiabatic condition is carried by the half-space solution),
NEUMANN (lateral faces, Eq. that-bc-n), DIRICHLET (bottom face, Eq. that-bc-d).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

FACE_NONE = 0
FACE_NEUMANN = 1
FACE_DIRICHLET = 2

# Lateral faces Neumann, bottom Dirichlet, top without a boundary term
# (Section 2, Eqs. neumann-bc-ori / dirichlet-bc-ori and Section 2.1).
DEFAULT_FACES = (FACE_NEUMANN, FACE_NEUMANN, FACE_NEUMANN, FACE_NEUMANN,
                 FACE_DIRICHLET, FACE_NONE)


@dataclass
class Patch:
    degree: tuple                    # (p0, p1, p2)
    knots: List[np.ndarray]          # three open knot vectors
    ctrl: np.ndarray                 # (n2, n1, n0, 3) control points [m]
    weights: Optional[np.ndarray] = None   # (n2, n1, n0) or None (B-spline)
    faces: tuple = DEFAULT_FACES

    @property
    def n_ctrl(self):
        n2, n1, n0, _ = self.ctrl.shape
        return (n0, n1, n2)

    @property
    def n_dof(self):
        n0, n1, n2 = self.n_ctrl
        return n0 * n1 * n2


@dataclass
class Material:
    k: float        # conductivity [W/(m K)]
    rho: float      # density [kg/m^3]
    cp: float       # specific heat [J/(kg K)]
    T_c: float      # platform / initial temperature [K]


@dataclass
class Scan:
    path: np.ndarray               # (nv, 3) polyline vertices on the top plane [m]
    seg_on: np.ndarray             # (nv-1,) uint8: 1 = laser on, 0 = jump (no time)
    power: float                   # P [W]
    absorptivity: float            # A [-]
    speed: float                   # v [m/s]
    spot_radius: float = 20e-6     # r [m]


@dataclass
class Workload:
    name: str
    patch: Patch
    material: Material
    scan: Scan
    dt: float
    theta: float
    n_steps: int
    meta: dict = field(default_factory=dict)


# --------------------------------------------------------------------------
# knot vectors and control nets
# --------------------------------------------------------------------------
def open_uniform_knots(p: int, n_el: int) -> np.ndarray:
    """Open knot vector on [0, 1] with n_el equal spans: p+1 repeated ends."""
    inner = np.linspace(0.0, 1.0, n_el + 1)
    return np.concatenate([np.zeros(p), inner, np.ones(p)])


def greville(knots: np.ndarray, p: int) -> np.ndarray:
    """Greville abscissae: the mean of p consecutive interior knots.

    Placing control points of a B-spline curve at L*greville gives the
    linear map x = L*xi exactly; this is how an affine cuboid is written as a
    spline patch (input construction, not part of the method).
    """
    n = len(knots) - p - 1
    return np.array([knots[i + 1:i + p + 1].mean() for i in range(n)])


def cuboid_patch(size, n_el, degree=2, origin=(0.0, 0.0, 0.0),
                 faces=DEFAULT_FACES) -> Patch:
    """Axis-aligned box [origin, origin+size] as one B-spline patch."""
    ps = (degree,) * 3 if np.isscalar(degree) else tuple(degree)
    knots = [open_uniform_knots(ps[d], n_el[d]) for d in range(3)]
    g = [origin[d] + size[d] * greville(knots[d], ps[d]) for d in range(3)]
    Z, Y, X = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    ctrl = np.stack([X, Y, Z], axis=-1).astype(np.float64)
    return Patch(degree=ps, knots=knots, ctrl=np.ascontiguousarray(ctrl),
                 weights=None, faces=tuple(faces))


# --------------------------------------------------------------------------
# scans
# --------------------------------------------------------------------------
def straight_track(p0, p1, power, absorptivity, speed, spot_radius=20e-6) -> Scan:
    path = np.array([p0, p1], dtype=np.float64)
    return Scan(path=path, seg_on=np.ones(1, np.uint8), power=power,
                absorptivity=absorptivity, speed=speed, spot_radius=spot_radius)


def meander(x_a, x_b, y0, hatch, n_tracks, z, power, absorptivity, speed,
            spot_radius=20e-6, angle=0.0, center=None) -> Scan:
    """Alternating-direction hatch: tracks x_a->x_b, x_b->x_a, ... at
    y = y0 + k*hatch.  Tracks are joined by laser-off jumps.  ``angle``
    rotates the whole pattern about ``center`` in the top plane."""
    verts = []
    on = []
    for k in range(n_tracks):
        y = y0 + k * hatch
        a, b = (x_a, x_b) if k % 2 == 0 else (x_b, x_a)
        if verts:
            on.append(0)
        verts.append((a, y, z))
        verts.append((b, y, z))
        on.append(1)
    path = np.array(verts, dtype=np.float64)
    if angle != 0.0:
        c = np.array(center if center is not None else path[:, :2].mean(0))
        R = np.array([[np.cos(angle), -np.sin(angle)], [np.sin(angle), np.cos(angle)]])
        path[:, :2] = (path[:, :2] - c) @ R.T + c
    return Scan(path=path, seg_on=np.array(on, np.uint8), power=power,
                absorptivity=absorptivity, speed=speed, spot_radius=spot_radius)


# --------------------------------------------------------------------------
# seeded generator (splitmix64, published by Steele, Lea and Flood, 2014)
# --------------------------------------------------------------------------
class SplitMix64:
    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self, lo=0.0, hi=1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] inclusive."""
        return lo + self.next_u64() % (hi - lo + 1)


SEED_BASE = 20251120

# material of the synthetic configurations (k, rho, c_p, T_0)
MAT_DEFAULT = Material(k=20.0, rho=4430.0, cp=560.0, T_c=300.0)
# Ti-6Al-4V, Table 1 of the paper
MAT_TI64 = Material(k=42.0, rho=4420.0, cp=990.0, T_c=20.0)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
def cuboid_single_track(theta=1.0, n_steps=150) -> Workload:
    """2.0 x 1.0 x 0.5 mm cuboid, degree 2, 16x8x4 elements (1080 control
    points); one 1.5 mm track along x at y = 0.5 mm, P = 200 W, A = 0.4,
    v = 1 m/s, dt = 10 us."""
    patch = cuboid_patch((2.0e-3, 1.0e-3, 0.5e-3), (16, 8, 4), 2)
    scan = straight_track((0.25e-3, 0.5e-3, 0.5e-3), (1.75e-3, 0.5e-3, 0.5e-3),
                          power=200.0, absorptivity=0.4, speed=1.0)
    return Workload("cuboid_2x1x0.5mm_p2_16x8x4_track1.5mm", patch, MAT_DEFAULT,
                    scan, dt=10e-6, theta=theta, n_steps=n_steps)


def block_meander(n_tracks=20, theta=0.5, n_steps=None, n_el=(64, 64, 16)) -> Workload:
    """4 x 4 x 1 mm block, degree 2, 64x64x16 elements (78,408 control
    points); meander of ``n_tracks`` 3.5 mm tracks (hatch 0.1 mm, alternating),
    P = 250 W, A = 0.4, v = 1.2 m/s, dt = 5 us, full history kept."""
    patch = cuboid_patch((4.0e-3, 4.0e-3, 1.0e-3), n_el, 2)
    scan = meander(0.25e-3, 3.75e-3, 1.05e-3, 0.1e-3, n_tracks, 1.0e-3,
                   power=250.0, absorptivity=0.4, speed=1.2)
    per_track = int(np.floor(3.5e-3 / (1.2 * 5e-6) + 1e-9)) + 1
    if n_steps is None:
        n_steps = per_track * n_tracks
    return Workload(f"block_4x4x1mm_p2_{n_el[0]}x{n_el[1]}x{n_el[2]}_meander{n_tracks}",
                    patch, MAT_DEFAULT, scan, dt=5e-6, theta=theta, n_steps=n_steps)


def small_block(n_el=(6, 5, 3), degree=2, n_tracks=3, n_steps=None, theta=0.5,
                dt=5e-6, size=(1.2e-3, 1.0e-3, 0.4e-3), speed=1.0, power=150.0) -> Workload:
    """Small parity case: a few elements, a short meander near the walls."""
    patch = cuboid_patch(size, n_el, degree)
    x_a, x_b = 0.15 * size[0], 0.85 * size[0]
    hatch = 0.6 * size[1] / max(n_tracks, 1)
    scan = meander(x_a, x_b, 0.2 * size[1], hatch, n_tracks, size[2],
                   power=power, absorptivity=0.4, speed=speed)
    if n_steps is None:
        L = (x_b - x_a)
        n_steps = (int(np.floor(L / (speed * dt) + 1e-9)) + 1) * n_tracks
    return Workload(f"small_block_{n_el[0]}x{n_el[1]}x{n_el[2]}_p{degree}", patch,
                    MAT_DEFAULT, scan, dt=dt, theta=theta, n_steps=n_steps)


def batched_instance(instance_id: int, n_steps=2000) -> Workload:
    """One seeded instance of the batched sweep: uneven cuboid patch
    (8-48 elements in-plane, 4-12 through the thickness, element size
    62.5 um, degree 2), P ~ U(100, 400) W, v ~ U(0.5, 2.0) m/s, 2-8 meander
    tracks along x with 0.1 mm hatch, dt = 5 us."""
    rng = SplitMix64(SEED_BASE + instance_id)
    h = 62.5e-6
    nx, ny, nz = rng.randint(8, 48), rng.randint(8, 48), rng.randint(4, 12)
    P = rng.uniform(100.0, 400.0)
    v = rng.uniform(0.5, 2.0)
    n_tr = rng.randint(2, 8)
    Lx, Ly, Lz = nx * h, ny * h, nz * h
    patch = cuboid_patch((Lx, Ly, Lz), (nx, ny, nz), 2)
    mx = max(0.1e-3, 0.1 * Lx)
    my = max(0.1e-3, 0.1 * Ly)
    hatch = 0.1e-3
    n_fit = max(1, int(np.floor((Ly - 2 * my) / hatch + 1e-9)) + 1)
    n_tr = min(n_tr, n_fit)
    scan = meander(mx, Lx - mx, my, hatch, n_tr, Lz, power=P, absorptivity=0.4, speed=v)
    return Workload(f"batched_{instance_id}", patch, MAT_DEFAULT, scan, dt=5e-6,
                    theta=0.5, n_steps=n_steps,
                    meta=dict(instance_id=instance_id, seed=SEED_BASE + instance_id))


def distorted_block(weights=False, seed=3, n_el=(3, 3, 2), size=(1e-3, 0.8e-3, 0.5e-3),
                    degree=2, jitter=0.04e-3, faces=DEFAULT_FACES) -> Patch:
    """A cuboid patch whose interior and side control points are moved by a
    seeded jitter (top plane kept flat); optional random weights in
    [0.8, 1.2] make it a genuine NURBS patch."""
    rng = np.random.default_rng(seed)
    patch = cuboid_patch(size, n_el, degree, faces=faces)
    c = patch.ctrl.copy()
    inner = c[1:-1, 1:-1, 1:-1]
    inner += rng.uniform(-jitter, jitter, inner.shape)
    c[:-1, :, 0, 0] += rng.uniform(-0.75 * jitter, 0.75 * jitter, c[:-1, :, 0, 0].shape)
    c[:-1, 0, :, 1] += rng.uniform(-0.75 * jitter, 0.75 * jitter, c[:-1, 0, :, 1].shape)
    patch.ctrl = c
    if weights:
        patch.weights = rng.uniform(0.8, 1.2, c.shape[:3])
    return patch


def quarter_cylinder_part(n_refine=1) -> Patch:
    """The quarter-cylinder part of Section 3.1 (Table 2 control net, knot
    vectors printed with it, middle arc weights cos(pi/8)), extruded from
    z = 0 to the printed top z = 2 mm; degree (2, 1, 1).  ``n_refine`` > 1 is
    not offered here (the printed net is used as is)."""
    r2 = np.sqrt(2.0)
    b1 = [(1, 0), (1, r2 - 1), (2 - r2 / 2, r2 / 2), (3 - r2, 1), (2, 1)]
    b2 = [(0, 0), (0, 1), (0, 2), (1, 2), (2, 2)]
    ctrl = np.zeros((2, 2, 5, 3))
    for i in range(5):
        for k, z in enumerate((0.0, 2.0)):
            ctrl[k, 0, i] = [b1[i][0], b1[i][1], z]
            ctrl[k, 1, i] = [b2[i][0], b2[i][1], z]
    wm = np.cos(np.pi / 8)
    w = np.broadcast_to(np.array([1, wm, 1, wm, 1.0]), (2, 2, 5)).copy()
    knots = [np.array([0, 0, 0, 0.5, 0.5, 1, 1, 1.0]), np.array([0, 0, 1, 1.0]),
             np.array([0, 0, 1, 1.0])]
    return Patch(degree=(2, 1, 1), knots=knots, ctrl=ctrl * 1e-3, weights=w)
