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
    seam: int = -1                   # parametric direction whose end layers coincide
                                     # (closed patch: merged into one layer), or -1

    @property
    def n_ctrl(self):
        n2, n1, n0, _ = self.ctrl.shape
        return (n0, n1, n2)

    @property
    def n_dof(self):
        n = list(self.n_ctrl)
        if self.seam >= 0:
            n[self.seam] -= 1
        return n[0] * n[1] * n[2]


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
# the plate with a hole (closed ring in xi): curve construction on control
# points only (Bezier degree elevation and Boehm knot insertion in
# homogeneous coordinates), no evaluation of basis functions
# --------------------------------------------------------------------------
def _elevate_quadratic_segments(Pw):
    """Rational quadratic Bezier segments (homogeneous points, consecutive
    segments sharing end points) -> the same curve as cubic segments:
    Q0 = P0, Q1 = (P0 + 2 P1)/3, Q2 = (2 P1 + P2)/3, Q3 = P2."""
    n_seg = (len(Pw) - 1) // 2
    out = [Pw[0]]
    for s in range(n_seg):
        P0, P1, P2 = Pw[2 * s], Pw[2 * s + 1], Pw[2 * s + 2]
        out += [(P0 + 2 * P1) / 3.0, (2 * P1 + P2) / 3.0, P2]
    return np.array(out)


def _insert_knot(U, Pw, p, u):
    """Boehm: insert u once into knot vector U of a degree-p curve with
    homogeneous control points Pw; returns the new knots and points."""
    k = int(np.searchsorted(U, u, side="right")) - 1       # U[k] <= u < U[k+1]
    Q = np.empty((len(Pw) + 1, Pw.shape[1]))
    for i in range(len(Q)):
        if i <= k - p:
            Q[i] = Pw[i]
        elif i >= k + 1:
            Q[i] = Pw[i - 1]
        else:
            a = (u - U[i]) / (U[i + p] - U[i])
            Q[i] = a * Pw[i] + (1.0 - a) * Pw[i - 1]
    return np.insert(U, k + 1, u), Q


def plate_with_hole_patch(n_el=(48, 48, 8), radius=0.75e-3, half=1.5e-3,
                          thickness=0.5e-3, degree=3) -> Patch:
    """Square plate [-half, half]^2 x [0, thickness] with a centred round
    hole, as ONE trivariate NURBS patch closed in xi (seam at angle -45 deg,
    a C0 corner).  xi: angle, four C0 sections of 90 deg (rational quadratic
    arcs with middle weight cos 45 deg, elevated to ``degree`` and refined to
    n_el[0]/4 spans each); eta: from the outer square (eta = 0) to the hole
    (eta = 1), straight lines between matching points of the square and of
    the circle; zeta: through the thickness.  Faces: xi ends are the seam
    (no boundary), eta = 0 and eta = 1 lateral (Neumann), zeta = 0 bottom
    (Dirichlet), zeta = 1 top."""
    assert degree == 3 and n_el[0] % 4 == 0
    c45 = np.cos(np.pi / 4)
    hole, square, wts = [], [], []
    for s in range(4):
        a0, am = np.pi / 2 * s - np.pi / 4, np.pi / 2 * s
        d0, dm = np.array([np.cos(a0), np.sin(a0)]), np.array([np.cos(am), np.sin(am)])
        hole += [radius * d0, radius / c45 * dm]
        square += [half / c45 * d0, half * dm]
        wts += [1.0, c45]
    hole.append(hole[0])
    square.append(square[0])
    wts.append(1.0)
    wts = np.array(wts)

    def ring(points):
        Pw = np.column_stack([np.array(points) * wts[:, None], wts])     # (9, 3)
        Pw = _elevate_quadratic_segments(Pw)                              # (13, 3)
        U = np.concatenate([[0.0] * 4, np.repeat([0.25, 0.5, 0.75], 3), [1.0] * 4])
        m = n_el[0] // 4
        for s in range(4):
            for t in range(1, m):
                U, Pw = _insert_knot(U, Pw, 3, (s + t / m) / 4.0)
        return U, Pw

    U0, Hw = ring(hole)
    _, Sw = ring(square)
    w0 = Hw[:, 2]
    assert np.allclose(w0, Sw[:, 2])
    H = Hw[:, :2] / w0[:, None]
    S = Sw[:, :2] / w0[:, None]
    U1 = open_uniform_knots(degree, n_el[1])
    U2 = open_uniform_knots(degree, n_el[2])
    t = greville(U1, degree)                     # eta: square (0) -> hole (1)
    z = thickness * greville(U2, degree)
    n0, n1, n2 = len(w0), len(t), len(z)
    ctrl = np.empty((n2, n1, n0, 3))
    for j in range(n1):
        ctrl[:, j, :, 0] = (1.0 - t[j]) * S[:, 0] + t[j] * H[:, 0]
        ctrl[:, j, :, 1] = (1.0 - t[j]) * S[:, 1] + t[j] * H[:, 1]
    ctrl[..., 2] = z[:, None, None]
    ctrl[:, :, -1, :] = ctrl[:, :, 0, :]         # the seam layers coincide exactly
    weights = np.broadcast_to(w0[None, None, :], (n2, n1, n0)).copy()
    faces = (FACE_NONE, FACE_NONE, FACE_NEUMANN, FACE_NEUMANN, FACE_DIRICHLET, FACE_NONE)
    return Patch(degree=(degree,) * 3, knots=[U0, U1, U2], ctrl=np.ascontiguousarray(ctrl),
                 weights=weights, faces=faces, seam=0)


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


def contour_and_radial_hatches(r_contour, r_in, half, margin, n_hatch, z, power,
                               absorptivity, speed, n_arc=720, spot_radius=20e-6) -> Scan:
    """One full counter-clockwise circle of radius r_contour about the origin
    (a polyline of n_arc chords, starting at angle pi/4), then n_hatch radial
    tracks at angles pi/4 + 2 pi k / n_hatch from radius r_in outwards to
    ``margin`` inside the square [-half, half]^2; laser-off jumps between
    tracks."""
    a0 = np.pi / 4
    ang = a0 + 2 * np.pi * np.arange(n_arc + 1) / n_arc
    verts = [(r_contour * np.cos(a), r_contour * np.sin(a), z) for a in ang]
    on = [1] * n_arc
    for k in range(n_hatch):
        a = a0 + 2 * np.pi * k / n_hatch
        d = np.array([np.cos(a), np.sin(a)])
        r_out = half / max(abs(d[0]), abs(d[1])) - margin
        on.append(0)
        verts.append((r_in * d[0], r_in * d[1], z))
        verts.append((r_out * d[0], r_out * d[1], z))
        on.append(1)
    return Scan(path=np.array(verts, dtype=np.float64), seg_on=np.array(on, np.uint8),
                power=power, absorptivity=absorptivity, speed=speed, spot_radius=spot_radius)


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


def two_lasers_cuboid(powers=(200.0, 150.0), ys=(0.3e-3, 0.7e-3), theta=0.5, n_steps=60):
    """The 2.0 x 1.0 x 0.5 mm cuboid (degree 2, 16x8x4 elements) with two
    lasers switched on together: straight 1.5 mm tracks along x at y = ys[0]
    and ys[1], powers ``powers``, A = 0.4, v = 1 m/s, dt = 10 us.  Returns the
    workload (patch, material, dt, theta; its scan is laser 0) and the list of
    the two scans."""
    patch = cuboid_patch((2.0e-3, 1.0e-3, 0.5e-3), (16, 8, 4), 2)
    scans = [straight_track((0.25e-3, y, 0.5e-3), (1.75e-3, y, 0.5e-3), power=p,
                            absorptivity=0.4, speed=1.0) for p, y in zip(powers, ys)]
    wl = Workload("cuboid_2x1x0.5mm_p2_16x8x4_two_lasers", patch, MAT_DEFAULT, scans[0],
                  dt=10e-6, theta=theta, n_steps=n_steps)
    return wl, scans


def block_meander(n_tracks=20, theta=0.5, n_steps=None, n_el=(64, 64, 16),
                  size=(4.0e-3, 4.0e-3, 1.0e-3)) -> Workload:
    """4 x 4 x 1 mm block, degree 2, 64x64x16 elements (78,408 control
    points); meander of ``n_tracks`` 3.5 mm tracks (hatch 0.1 mm, alternating),
    P = 250 W, A = 0.4, v = 1.2 m/s, dt = 5 us, full history kept.  ``size``
    gives a larger block with the same meander at the same place (near the
    corner x = y = 0)."""
    patch = cuboid_patch(size, n_el, 2)
    scan = meander(0.25e-3, 3.75e-3, 1.05e-3, 0.1e-3, n_tracks, 1.0e-3,
                   power=250.0, absorptivity=0.4, speed=1.2)
    per_track = int(np.floor(3.5e-3 / (1.2 * 5e-6) + 1e-9)) + 1
    if n_steps is None:
        n_steps = per_track * n_tracks
    tag = "4x4x1mm" if tuple(size) == (4.0e-3, 4.0e-3, 1.0e-3) else \
        "x".join(f"{v * 1e3:g}" for v in size) + "mm"
    return Workload(f"block_{tag}_p2_{n_el[0]}x{n_el[1]}x{n_el[2]}_meander{n_tracks}",
                    patch, MAT_DEFAULT, scan, dt=5e-6, theta=theta, n_steps=n_steps)


def plate_with_hole(n_el=(48, 48, 8), theta=0.5, n_steps=None) -> Workload:
    """3 x 3 x 0.5 mm plate with a centred hole of radius 0.75 mm, one
    degree-3 NURBS patch closed in xi (48 x 48 x 8 elements: 31,416 control
    variables after the seam merge); a contour at r = 0.85 mm (100 um from
    the hole edge) then 10 radial hatches from r = 0.95 mm to 0.1 mm inside
    the outer edge; P = 180 W, A = 0.4, v = 0.8 m/s, dt = 5 us."""
    patch = plate_with_hole_patch(n_el=n_el)
    scan = contour_and_radial_hatches(0.85e-3, 0.95e-3, 1.5e-3, 0.1e-3, 10, 0.5e-3,
                                      power=180.0, absorptivity=0.4, speed=0.8)
    if n_steps is None:
        n_steps = int(sum(np.floor(L / (0.8 * 5e-6) + 1e-9) + 1 for L in
                          _track_lengths(scan)))
    return Workload(f"plate_hole_3x3x0.5mm_p3_{n_el[0]}x{n_el[1]}x{n_el[2]}_contour_hatch10",
                    patch, MAT_DEFAULT, scan, dt=5e-6, theta=theta, n_steps=n_steps)


def learned_scan(k: int, z=1.0e-3, center=(2.0e-3, 2.0e-3)) -> Scan:
    """Scan k of the learned warm-start set (seed SEED_BASE + 4000 + k) on
    the 4 x 4 x 1 mm block: P ~ U(150, 350) W, v ~ U(0.6, 1.6) m/s, hatch
    spacing ~ U(0.08, 0.12) mm, 5-20 tracks of 2.4 mm centred on the top
    face, the whole pattern rotated by an angle ~ U(0, pi).  Even k: a
    meander (laser-off jumps between tracks); odd k: a zig-zag (the track
    ends joined by laser-on segments, so the laser never stops)."""
    rng = SplitMix64(SEED_BASE + 4000 + k)
    P, v = rng.uniform(150.0, 350.0), rng.uniform(0.6, 1.6)
    hatch, n_tr = rng.uniform(0.08e-3, 0.12e-3), rng.randint(5, 20)
    angle = rng.uniform(0.0, np.pi)
    y0 = center[1] - 0.5 * (n_tr - 1) * hatch
    sc = meander(center[0] - 1.2e-3, center[0] + 1.2e-3, y0, hatch, n_tr, z, P, 0.4, v,
                 angle=angle, center=center)
    if k % 2 == 1:
        sc.seg_on = np.ones_like(sc.seg_on)
    return sc


def warm_start_input_rows(patch) -> np.ndarray:
    """Rows of the theta-step residual that the learned warm start reads: the
    free control variables on the lateral faces and in the first free layer
    above the bottom, as indices into the free rows (the free rows are the
    control points in natural order without the bottom layer, which holds
    the Dirichlet control variables)."""
    n0, n1, n2 = patch.n_ctrl
    idx = [(k * n1 + j) * n0 + i - n0 * n1 for k in range(1, n2) for j in range(n1)
           for i in range(n0) if k == 1 or i in (0, n0 - 1) or j in (0, n1 - 1)]
    return np.array(idx, dtype=np.int32)


def _track_lengths(scan):
    """Lengths of the maximal runs of laser-on segments."""
    seg = np.linalg.norm(np.diff(scan.path, axis=0), axis=1)
    out, cur = [], 0.0
    for L, on in zip(seg, scan.seg_on):
        if on:
            cur += L
        elif cur > 0.0:
            out.append(cur)
            cur = 0.0
    if cur > 0.0:
        out.append(cur)
    return out


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


def _refine_direction(U, Pw, axis, p, new_knots):
    """Boehm insertion of new_knots along one parametric direction of a
    homogeneous control volume Pw (n2, n1, n0, 4); axis 0 = xi (last array
    axis 2), 1 = eta, 2 = zeta."""
    arr_axis = 2 - axis
    A = np.moveaxis(Pw, arr_axis, -2)            # (..., n_axis, 4)
    shp = A.shape
    lines = A.reshape(-1, shp[-2], 4)
    U_out = U
    out = []
    for line in lines:
        Uc, Q = U, line
        for u in new_knots:
            Uc, Q = _insert_knot(Uc, Q, p, u)
        out.append(Q)
        U_out = Uc
    A2 = np.array(out).reshape(shp[:-2] + (out[0].shape[0], 4))
    return U_out, np.moveaxis(A2, -2, arr_axis)


def _elevate_linear_direction(Pw, axis):
    """Degree 1 -> 2 along a direction with one span: (P0, P1) -> (P0, (P0 +
    P1)/2, P1) in homogeneous coordinates (the same map)."""
    arr_axis = 2 - axis
    A = np.moveaxis(Pw, arr_axis, 0)
    assert A.shape[0] == 2
    B = np.stack([A[0], 0.5 * (A[0] + A[1]), A[1]])
    return np.moveaxis(B, 0, arr_axis)


def quarter_cylinder_refined(n_el=(16, 8, 8)) -> Patch:
    """The quarter-cylinder part of Section 3.1 as degree 2 in every
    direction (the linear directions elevated) with n_el elements: the two
    xi spans split into n_el[0] / 2 each, eta and zeta into n_el[1] and
    n_el[2]; control-point operations only (the same geometry)."""
    base = quarter_cylinder_part()
    w = base.weights
    Pw = np.concatenate([base.ctrl * w[..., None], w[..., None]], axis=-1)   # (2, 2, 5, 4)
    Pw = _elevate_linear_direction(Pw, 1)
    Pw = _elevate_linear_direction(Pw, 2)
    U0 = base.knots[0]
    U12 = np.array([0, 0, 0, 1, 1, 1.0])
    assert n_el[0] % 2 == 0
    m0 = n_el[0] // 2
    ins0 = [(s + t / m0) / 2.0 for s in range(2) for t in range(1, m0)]
    U0, Pw = _refine_direction(U0, Pw, 0, 2, ins0)
    U1, Pw = _refine_direction(U12, Pw, 1, 2, [t / n_el[1] for t in range(1, n_el[1])])
    U2, Pw = _refine_direction(U12, Pw, 2, 2, [t / n_el[2] for t in range(1, n_el[2])])
    wts = Pw[..., 3]
    ctrl = Pw[..., :3] / wts[..., None]
    return Patch(degree=(2, 2, 2), knots=[U0, U1, U2], ctrl=np.ascontiguousarray(ctrl),
                 weights=np.ascontiguousarray(wts))


def quarter_cylinder_single_source(n_el=(16, 8, 8), n_steps=19, theta=0.5) -> Workload:
    """Section 3.1 single heat source: one pulse of dt = 1e-5 s, P = 82.5 W,
    A = 0.77 (E = 6.35e-4 J), r = 20 um, on the top surface 100 um from the
    arc where the line from the cylinder's axis makes pi/4 with the x2 axis
    (reading: the figure's origin is the cylinder's axis, x = 2 mm, y = 0 in
    the Table 2 coordinates); Ti-6Al-4V; observed at t = 1.9e-4 s (19
    steps)."""
    patch = quarter_cylinder_refined(n_el)
    rc = 1.1e-3
    c = np.array([2e-3, 0.0])
    xy = c + rc * np.array([-np.sin(np.pi / 4), np.cos(np.pi / 4)])
    p = (xy[0], xy[1], 2e-3)
    scan = Scan(path=np.array([p, p], dtype=np.float64), seg_on=np.array([1], dtype=np.uint8),
                power=82.5, absorptivity=0.77, speed=0.5, spot_radius=20e-6)
    return Workload("quarter_cylinder_single_source", patch, MAT_TI64, scan, dt=1e-5,
                    theta=theta, n_steps=n_steps, meta={"source_xy": tuple(xy)})


def quarter_cylinder_contour(n_el=(16, 8, 8), n_steps=300, theta=0.5, n_seg=2048) -> Workload:
    """Section 3.2 continuous scan on the quarter-cylinder part: P = 82.5 W,
    A = 0.77, v = 0.5 m/s, r = 20 um, dt = 1e-5 s, Ti-6Al-4V, the laser
    starting at t = 0 on the scan path offset 100 um into the part from the
    boundary.  Reading: the path is the arc part of that offset contour, the
    circle of radius 1.1 mm about the cylinder's axis between the points
    where it meets the offsets of the two flat faces (angles asin(0.1/1.1)
    and pi/2 - asin(0.1/1.1) from the x2 direction), scanned from the x2
    side as a polyline of n_seg chords; 1.53 mm long, so the laser is still
    on it at t = 3e-3 s (1.5 mm)."""
    patch = quarter_cylinder_refined(n_el)
    a0 = np.arcsin(0.1 / 1.1)
    th = np.linspace(a0, np.pi / 2 - a0, n_seg + 1)
    xy = np.array([2e-3, 0.0]) + 1.1e-3 * np.column_stack([-np.sin(th), np.cos(th)])
    path = np.column_stack([xy, np.full(n_seg + 1, 2e-3)])
    scan = Scan(path=np.ascontiguousarray(path), seg_on=np.ones(n_seg, np.uint8), power=82.5,
                absorptivity=0.77, speed=0.5, spot_radius=20e-6)
    return Workload("quarter_cylinder_contour", patch, MAT_TI64, scan, dt=1e-5, theta=theta,
                    n_steps=n_steps, meta={"arc_angles": (a0, np.pi / 2 - a0)})


def quarter_cylinder_arc_points(n, z=2e-3):
    """Points of the top arc (radius 1 mm about x = 2 mm, y = 0) from theta =
    0 (on the x2 direction) to pi/2, with the outward normal of the part (into
    the removed cylinder) and the arc-length weights of the trapezoid rule."""
    th = np.linspace(0.0, np.pi / 2, n)
    d = np.column_stack([-np.sin(th), np.cos(th)])      # from the axis to the arc
    xy = np.array([2e-3, 0.0]) + 1e-3 * d
    pts = np.column_stack([xy, np.full(n, z)])
    nrm = np.column_stack([-d, np.zeros(n)])            # out of the part: toward the axis
    ds = np.full(n, 1e-3 * (np.pi / 2) / (n - 1))
    ds[0] *= 0.5
    ds[-1] *= 0.5
    return th, pts, nrm, ds
