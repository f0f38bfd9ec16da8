"""Assembly of the semi-discrete system (Section 2.3):

    M_ij = int rho c_p N_i N_j J dxi
    K_ij = int k (grad_x N_i) . (grad_x N_j) J dxi
    F_i  = int_{dV_lat} (-q_N) N_i dS

plus the boundary weight matrices used to form F and the Dirichlet data:

    W_lat[i, q] = wdS_q R_i(x_q)    over lateral (Neumann) face points
    W_bot[i, q] = wdS_q R_i(x_q)    over Dirichlet face points
    M_bot[i, j] = sum_q wdS_q R_i(x_q) R_j(x_q)   (L2 projection, reading R5)

Element by element with a dense local matrix, accumulated into a sparse
matrix by scipy's COO -> CSR conversion (duplicates summed).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .geometry import PatchGeom


def element_matrices(geom: PatchGeom, elem, rho_cp, k):
    """Local mass and conductivity matrices of one element."""
    Me = None
    Ke = None
    dofs = None
    for xi, wt in geom.element_quadrature(elem):
        spans = [elem[d][2] for d in range(3)]
        dofs, R, dR, x, J = geom.local_eval(xi, spans)
        detJ = np.linalg.det(J)
        gradR = np.linalg.solve(J.T, dR.T).T          # rows: grad_x R_a = J^{-T} grad_xi R_a
        wq = wt * detJ
        m = rho_cp * wq * np.outer(R, R)
        kk = k * wq * (gradR @ gradR.T)
        Me = m if Me is None else Me + m
        Ke = kk if Ke is None else Ke + kk
    return dofs, Me, Ke


def assemble_MK(geom: PatchGeom, rho_cp, k, elements=None):
    """Global M and K (CSR, n_dof x n_dof).  ``elements`` restricts the sum
    to a subset (used to build selected rows at large sizes)."""
    rows, cols, mv, kv = [], [], [], []
    for elem in (geom.element_list() if elements is None else elements):
        dofs, Me, Ke = element_matrices(geom, elem, rho_cp, k)
        r = np.repeat(dofs, len(dofs))
        c = np.tile(dofs, len(dofs))
        rows.append(r)
        cols.append(c)
        mv.append(Me.ravel())
        kv.append(Ke.ravel())
    n = geom.n_dof
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    M = sp.coo_matrix((np.concatenate(mv), (rows, cols)), shape=(n, n)).tocsr()
    K = sp.coo_matrix((np.concatenate(kv), (rows, cols)), shape=(n, n)).tocsr()
    M.sum_duplicates()
    K.sum_duplicates()
    return M, K


def elements_touching_dof(geom: PatchGeom, dof):
    """Elements on which the basis function(s) of control variable ``dof``
    can be non-zero."""
    out = []
    for idx in geom.ctrl_points_of(dof):
        lists = []
        for d in range(3):
            lists.append([e for e in geom.elems[d] if e[2] - geom.p[d] <= idx[d] <= e[2]])
        for e2 in lists[2]:
            for e1 in lists[1]:
                for e0 in lists[0]:
                    if (e0, e1, e2) not in out:
                        out.append((e0, e1, e2))
    return out


def boundary_points(geom: PatchGeom, kind):
    """Concatenated face points of all faces of the given kind, faces in
    increasing face id (canonical order shared with the GPU library)."""
    recs = [geom.face_points(f) for f, kf in enumerate(geom.faces) if kf == kind]
    if not recs:
        return None
    return {k: np.concatenate([r[k] for r in recs]) for k in recs[0]}


def weight_matrix(geom: PatchGeom, pts):
    """W[i, q] = wdS_q R_i(x_q) as CSR (n_dof x Q)."""
    Q, nloc = pts["R"].shape
    rows = pts["dofs"].ravel()
    cols = np.repeat(np.arange(Q), nloc)
    vals = (pts["wdS"][:, None] * pts["R"]).ravel()
    W = sp.coo_matrix((vals, (rows, cols)), shape=(geom.n_dof, Q)).tocsr()
    W.sum_duplicates()
    return W


def boundary_mass(geom: PatchGeom, pts):
    """M_bot[i, j] = sum_q wdS_q R_i R_j over the given face points."""
    rows, cols, vals = [], [], []
    for q in range(pts["R"].shape[0]):
        d = pts["dofs"][q]
        R = pts["R"][q]
        rows.append(np.repeat(d, len(d)))
        cols.append(np.tile(d, len(d)))
        vals.append(pts["wdS"][q] * np.outer(R, R).ravel())
    n = geom.n_dof
    Mb = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(n, n)).tocsr()
    Mb.sum_duplicates()
    return Mb
