import numpy as np

import workloads as W

TOL_FP64 = 1e-10          # relative L-infinity, FP64 GPU path vs oracle
TOL_MIXED_REL = 1e-4      # relative L-infinity, mixed path
TOL_MIXED_ABS = 0.05      # kelvin, mixed path


def rel_linf(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def gpu_context(wl, precision, **opts):
    import paper_2511_20432_gb300 as sa
    return sa.context_from_workload(wl, precision=precision, **opts)


def lateral_xi(geom, q):
    """Parametric coordinates of canonical lateral point q (faces of kind
    Neumann in increasing id, face elements tangential-a fastest, Gauss
    points tangential-a fastest)."""
    from oracle import bspline
    from oracle.geometry import FACE_DIR
    for f, kind in enumerate(geom.faces):
        if kind != 1:
            continue
        d, side = FACE_DIR[f]
        ta, tb = [t for t in range(3) if t != d]
        nga, ngb = geom.p[ta] + 1, geom.p[tb] + 1
        nea, neb = len(geom.elems[ta]), len(geom.elems[tb])
        nq = nea * neb * nga * ngb
        if q >= nq:
            q -= nq
            continue
        t = q
        ga = t % nga; t //= nga
        gb = t % ngb; t //= ngb
        ea = t % nea; eb = t // nea
        xa, _ = bspline.gauss_legendre(nga)
        xb, _ = bspline.gauss_legendre(ngb)
        A = geom.elems[ta][ea]
        B = geom.elems[tb][eb]
        xi = np.empty(3)
        xi[d] = 0.0 if side == 0 else 1.0
        xi[ta] = A[0] + 0.5 * (A[1] - A[0]) * (xa[ga] + 1)
        xi[tb] = B[0] + 0.5 * (B[1] - B[0]) * (xb[gb] + 1)
        spans = [0, 0, 0]
        spans[d] = bspline.span_index(geom.U[d], geom.p[d], xi[d])
        spans[ta], spans[tb] = A[2], B[2]
        return f, xi, spans
    raise IndexError(q)
