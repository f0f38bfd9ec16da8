"""NURBS geometry map and quadrature (Section 2.3).

x(xi) = sum_i R_i(xi) P_i with R_i = w_i N_i / sum_j w_j N_j (N_i the
tensor-product B-spline), J = dx/dxi, grad_x R = J^{-T} grad_xi R,
dV = det(J) dxi.  Faces: dS = |x_u x x_v| du dv with the outward unit normal.

Quadrature (reading R4): (p_d + 1) Gauss-Legendre points per direction on
every non-empty knot span, and on every face element.

Closed patches (a seam in direction d: the control layers i_d = 0 and
i_d = n_d - 1 coincide): the two layers are one set of control variables,
so the discrete space is the span of the merged basis functions R_0 + R_{n-1}
and every assembled quantity is P^T (.) P with P the 0/1 map from control
points to control variables.
"""
from __future__ import annotations

import numpy as np

from . import bspline

# face id -> (fixed parametric direction, fixed value side 0/1)
FACE_DIR = {0: (0, 0), 1: (0, 1), 2: (1, 0), 3: (1, 1), 4: (2, 0), 5: (2, 1)}


class PatchGeom:
    def __init__(self, patch):
        self.p = tuple(int(x) for x in patch.degree)
        self.U = [np.asarray(k, dtype=np.float64) for k in patch.knots]
        self.ctrl = np.asarray(patch.ctrl, dtype=np.float64)          # (n2,n1,n0,3)
        n2, n1, n0, _ = self.ctrl.shape
        self.n = (n0, n1, n2)
        w = patch.weights
        self.w = np.ones((n2, n1, n0)) if w is None else np.asarray(w, dtype=np.float64)
        self.faces = tuple(patch.faces)
        self.seam = int(getattr(patch, "seam", -1))
        nd = list(self.n)
        if self.seam >= 0:
            d = self.seam
            sl0 = [slice(None)] * 3
            sl1 = [slice(None)] * 3
            sl0[2 - d] = 0
            sl1[2 - d] = self.n[d] - 1
            assert np.allclose(self.ctrl[tuple(sl0)], self.ctrl[tuple(sl1)], rtol=0, atol=1e-15)
            assert np.allclose(self.w[tuple(sl0)], self.w[tuple(sl1)], rtol=0, atol=1e-15)
            assert self.faces[2 * d] == 0 and self.faces[2 * d + 1] == 0, "seam faces carry no boundary term"
            nd[d] -= 1
        self.nd = tuple(nd)                       # shape of the control-variable grid
        for d in range(3):
            assert bspline.n_basis(self.U[d], self.p[d]) == self.n[d]
        self.elems = [bspline.elements(self.U[d]) for d in range(3)]
        self._cache1d = {}

    # ---- indexing -------------------------------------------------------
    def dof(self, i, j, k):
        """Control variable of control point (i, j, k): natural order over the
        control-variable grid (the seam layer n_d - 1 is layer 0)."""
        idx = [np.asarray(i), np.asarray(j), np.asarray(k)]
        if self.seam >= 0:
            idx[self.seam] = idx[self.seam] % self.nd[self.seam]
        n0, n1, _ = self.nd
        return (idx[2] * n1 + idx[1]) * n0 + idx[0]

    def ctrl_points_of(self, dof):
        """Control-point index triples (i, j, k) of one control variable."""
        n0, n1, _ = self.nd
        base = [dof % n0, (dof // n0) % n1, dof // (n0 * n1)]
        out = [tuple(base)]
        if self.seam >= 0 and base[self.seam] == 0:
            other = list(base)
            other[self.seam] = self.n[self.seam] - 1
            out.append(tuple(other))
        return out

    @property
    def n_dof(self):
        return self.nd[0] * self.nd[1] * self.nd[2]

    # ---- evaluation at one parametric point -----------------------------
    def local_eval(self, xi, spans=None):
        """At parametric point xi (3,), on the element with knot-span indices
        ``spans`` (found from xi when None).  Returns

            dofs  (nloc,)   global indices of the (p0+1)(p1+1)(p2+1) functions
            R     (nloc,)   NURBS basis values
            dR    (nloc,3)  d R / d xi
            x     (3,)      physical point
            J     (3,3)     J[c, d] = d x_c / d xi_d
        """
        if spans is None:
            spans = [bspline.span_index(self.U[d], self.p[d], xi[d]) for d in range(3)]
        N1, dN1 = [], []
        for d in range(3):
            key = (d, int(spans[d]), float(xi[d]))
            if key not in self._cache1d:   # memo of the 1-D evaluation only
                self._cache1d[key] = bspline.local_ders_on_element(
                    self.U[d], self.p[d], spans[d], xi[d])
            a, b = self._cache1d[key]
            N1.append(a)
            dN1.append(b)
        p0, p1, p2 = self.p
        # tensor product, local ordering a = (a2*(p1+1) + a1)*(p0+1) + a0
        N = np.einsum("k,j,i->kji", N1[2], N1[1], N1[0]).ravel()
        dN = np.stack([
            np.einsum("k,j,i->kji", N1[2], N1[1], dN1[0]).ravel(),
            np.einsum("k,j,i->kji", N1[2], dN1[1], N1[0]).ravel(),
            np.einsum("k,j,i->kji", dN1[2], N1[1], N1[0]).ravel(),
        ], axis=1)
        i0 = spans[0] - p0
        j0 = spans[1] - p1
        k0 = spans[2] - p2
        kk, jj, ii = np.meshgrid(np.arange(k0, k0 + p2 + 1), np.arange(j0, j0 + p1 + 1),
                                 np.arange(i0, i0 + p0 + 1), indexing="ij")
        ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
        dofs = self.dof(ii, jj, kk)
        w = self.w[kk, jj, ii]
        P = self.ctrl[kk, jj, ii]                          # (nloc, 3)
        # rational basis (quotient rule)
        W = np.dot(w, N)
        dW = w @ dN                                        # (3,)
        R = w * N / W
        dR = (w[:, None] * dN * W - (w * N)[:, None] * dW[None, :]) / (W * W)
        x = R @ P
        J = P.T @ dR                                       # (3,3): [c, d]
        return dofs, R, dR, x, J

    def point(self, xi):
        return self.local_eval(np.asarray(xi, dtype=np.float64))[3]

    # ---- volume quadrature ------------------------------------------------
    def element_list(self):
        out = []
        for e2 in self.elems[2]:
            for e1 in self.elems[1]:
                for e0 in self.elems[0]:
                    out.append((e0, e1, e2))
        return out

    def element_quadrature(self, elem):
        """Gauss points of one element: list of (xi (3,), weight in xi-space)."""
        g = [bspline.gauss_legendre(self.p[d] + 1) for d in range(3)]
        pts = []
        for c2, w2 in zip(*g[2]):
            for c1, w1 in zip(*g[1]):
                for c0, w0 in zip(*g[0]):
                    xi = np.empty(3)
                    wt = 1.0
                    for d, (c, wq) in enumerate(((c0, w0), (c1, w1), (c2, w2))):
                        lo, hi, _ = elem[d]
                        xi[d] = lo + 0.5 * (hi - lo) * (c + 1.0)
                        wt *= 0.5 * (hi - lo) * wq
                    pts.append((xi, wt))
        return pts

    # ---- face quadrature --------------------------------------------------
    def face_points(self, face):
        """Quadrature points of one face, in the order: face elements with the
        lower tangential direction fastest, then Gauss points with the lower
        tangential direction fastest.

        Returns dict of arrays: xi (Q,3), x (Q,3), n (Q,3) outward unit normal,
        wdS (Q,) = Gauss weight * |x_u x x_v|, dofs (Q,nloc), R (Q,nloc).
        """
        d, side = FACE_DIR[face]
        ta, tb = [t for t in range(3) if t != d]           # tangential, ta < tb
        fixed = 0.0 if side == 0 else 1.0
        fixed_span = bspline.span_index(self.U[d], self.p[d], fixed)
        ga = bspline.gauss_legendre(self.p[ta] + 1)
        gb = bspline.gauss_legendre(self.p[tb] + 1)
        rec = {k: [] for k in ("xi", "x", "n", "wdS", "dofs", "R")}
        for eb in self.elems[tb]:
            for ea in self.elems[ta]:
                for cb, wb in zip(*gb):
                    for ca, wa in zip(*ga):
                        xi = np.empty(3)
                        xi[d] = fixed
                        xi[ta] = ea[0] + 0.5 * (ea[1] - ea[0]) * (ca + 1.0)
                        xi[tb] = eb[0] + 0.5 * (eb[1] - eb[0]) * (cb + 1.0)
                        wt = 0.25 * (ea[1] - ea[0]) * (eb[1] - eb[0]) * wa * wb
                        spans = [0, 0, 0]
                        spans[d] = fixed_span
                        spans[ta] = ea[2]
                        spans[tb] = eb[2]
                        dofs, R, dR, x, J = self.local_eval(xi, spans)
                        xu, xv, xd = J[:, ta], J[:, tb], J[:, d]
                        c = np.cross(xu, xv)
                        area = np.linalg.norm(c)
                        nrm = c / area
                        # outward: points toward decreasing xi_d on the side-0 face
                        want = -1.0 if side == 0 else 1.0
                        if np.sign(np.dot(nrm, xd)) != want:
                            nrm = -nrm
                        rec["xi"].append(xi)
                        rec["x"].append(x)
                        rec["n"].append(nrm)
                        rec["wdS"].append(wt * area)
                        rec["dofs"].append(dofs)
                        rec["R"].append(R)
        return {k: np.array(v) for k, v in rec.items()}

    def top_z(self):
        """z of the planar top face (reading R3: sources lie on it)."""
        zt = self.ctrl[-1, :, :, 2]
        assert np.allclose(zt, zt.flat[0], rtol=0, atol=1e-15), "top face is not planar z = const"
        return float(zt.flat[0])

    def dirichlet_dofs(self):
        """Control variables whose basis functions have support on the
        Dirichlet face(s): those non-zero at the face parameter."""
        mask = np.zeros(self.n_dof, dtype=bool)
        for face, kind in enumerate(self.faces):
            if kind != 2:
                continue
            d, side = FACE_DIR[face]
            fixed = 0.0 if side == 0 else 1.0
            Nd = bspline.basis_all(self.U[d], self.p[d], fixed)
            layers = np.nonzero(Nd != 0.0)[0]
            n0, n1, n2 = self.n
            K, J, I = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
            idx = [I, J, K]
            for L in layers:
                sel = idx[d] == L
                mask[self.dof(I[sel], J[sel], K[sel])] = True
        return mask
