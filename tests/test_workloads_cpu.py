"""The quarter-cylinder inputs (Sections 3.1-3.2, Table 2) against the
paper's description: the refined patch is the same map as the Table 2 net,
the single source and the contour path sit where the text puts them, and
the arc points lie on the arc with the part's outward normal."""
import numpy as np

import workloads as W
from oracle.geometry import PatchGeom

AXIS = np.array([2e-3, 0.0])


def test_refined_part_is_the_table2_map():
    base = PatchGeom(W.quarter_cylinder_part())
    rng = np.random.default_rng(3)
    for n_el in ((4, 2, 2), (16, 8, 8)):
        fine = PatchGeom(W.quarter_cylinder_refined(n_el))
        for xi in rng.uniform(0.0, 1.0, (40, 3)):
            assert np.abs(fine.point(xi) - base.point(xi)).max() < 1e-17


def test_single_source_position():
    wl = W.quarter_cylinder_single_source((4, 2, 2))
    p = wl.scan.path[0]
    assert np.allclose(wl.scan.path[1], p)                 # one point: a pulse
    d = p[:2] - AXIS
    assert abs(np.hypot(*d) - 1.1e-3) < 1e-15              # 100 um from the R = 1 mm arc
    assert abs(np.arctan2(-d[0], d[1]) - np.pi / 4) < 1e-12  # pi/4 from the x2 direction
    assert p[2] == 2e-3                                    # on the top face
    assert wl.scan.power * wl.scan.absorptivity * wl.dt == np.float64(82.5 * 0.77 * 1e-5)


def test_contour_path_is_the_offset_arc():
    wl = W.quarter_cylinder_contour((4, 2, 2))
    P = wl.scan.path
    d = P[:, :2] - AXIS
    assert np.abs(np.hypot(d[:, 0], d[:, 1]) - 1.1e-3).max() < 1e-15
    assert np.all(P[:, 2] == 2e-3)
    # its ends are 100 um from the two flat faces x = 2 mm and y = 0
    assert abs(P[0, 0] - 1.9e-3) < 1e-15 and abs(P[-1, 1] - 0.1e-3) < 1e-15
    length = np.linalg.norm(np.diff(P, axis=0), axis=1).sum()
    arc = 1.1e-3 * (np.pi / 2 - 2 * np.arcsin(0.1 / 1.1))
    # 2,048 chords fall short of the arc by (dtheta)^2 / 24 of it, ~2e-8
    dth = (np.pi / 2 - 2 * np.arcsin(0.1 / 1.1)) / (len(P) - 1)
    assert abs(length - arc * (1 - dth ** 2 / 24)) < 1e-12 * arc
    assert wl.scan.speed * 3e-3 < length                   # still on it at t = 3e-3 s


def test_arc_points_normals_and_weights():
    th, pts, nrm, ds = W.quarter_cylinder_arc_points(181)
    d = pts[:, :2] - AXIS
    assert np.abs(np.hypot(d[:, 0], d[:, 1]) - 1e-3).max() < 1e-18
    assert np.allclose(np.linalg.norm(nrm, axis=1), 1.0)
    # outward from the part = toward the removed cylinder's axis
    assert np.allclose(nrm[:, :2], -d / 1e-3)
    assert abs(ds.sum() - 1e-3 * np.pi / 2) < 1e-18
    g = PatchGeom(W.quarter_cylinder_part())
    for u in np.linspace(0, 1, 9):                         # the patch's arc is this arc
        x = g.point([u, 0.0, 1.0])
        assert abs(np.hypot(x[0] - AXIS[0], x[1]) - 1e-3) < 1e-17
