"""B-spline basis by the Cox-de Boor recursion (Section 2.3: "B-spline or
NURBS basis functions of order p defined on the knot vectors").

Written directly from the recursive definition over ALL functions of the
knot vector, degree 0 up to p, so that every value can be checked by hand:

    N_{i,0}(u) = 1 if U_i <= u < U_{i+1} else 0
    N_{i,q}(u) = (u - U_i)/(U_{i+q} - U_i) N_{i,q-1}(u)
               + (U_{i+q+1} - u)/(U_{i+q+1} - U_{i+1}) N_{i+1,q-1}(u)
    d/du N_{i,q}(u) = q/(U_{i+q} - U_i) N_{i,q-1}(u)
                    - q/(U_{i+q+1} - U_{i+1}) N_{i+1,q-1}(u)

with 0/0 := 0.  At the right end u = U_last the last non-empty span is used
(so the basis is right-continuous there and sums to one).
"""
from __future__ import annotations

import numpy as np


def n_basis(U, p):
    return len(U) - p - 1


def span_index(U, p, u):
    """Largest s with U[s] <= u < U[s+1]; the last non-empty span at u = U[-1]."""
    U = np.asarray(U, dtype=np.float64)
    n = n_basis(U, p)
    if u >= U[n]:
        s = n - 1
        while U[s] == U[s + 1]:
            s -= 1
        return s
    s = int(np.searchsorted(U, u, side="right")) - 1
    return s


def _degree0(U, p, u):
    m = len(U) - 1
    N = np.zeros(m)
    N[span_index(U, p, u)] = 1.0
    return N


def basis_all(U, p, u):
    """All n values N_{i,p}(u), i = 0..n-1."""
    U = np.asarray(U, dtype=np.float64)
    N = _degree0(U, p, u)
    for q in range(1, p + 1):
        Nn = np.zeros(len(N) - 1)
        for i in range(len(Nn)):
            left = 0.0
            if U[i + q] != U[i]:
                left = (u - U[i]) / (U[i + q] - U[i]) * N[i]
            right = 0.0
            if U[i + q + 1] != U[i + 1]:
                right = (U[i + q + 1] - u) / (U[i + q + 1] - U[i + 1]) * N[i + 1]
            Nn[i] = left + right
        N = Nn
    return N


def basis_all_ders(U, p, u):
    """(N, dN): values and first derivatives of all n functions at u."""
    U = np.asarray(U, dtype=np.float64)
    if p == 0:
        N = basis_all(U, 0, u)
        return N, np.zeros_like(N)
    Nm = basis_all(U, p - 1, u)          # degree p-1, length n+1
    N = basis_all(U, p, u)
    dN = np.zeros(n_basis(U, p))
    for i in range(len(dN)):
        a = 0.0
        if U[i + p] != U[i]:
            a = p / (U[i + p] - U[i]) * Nm[i]
        b = 0.0
        if U[i + p + 1] != U[i + 1]:
            b = p / (U[i + p + 1] - U[i + 1]) * Nm[i + 1]
        dN[i] = a - b
    return N, dN


def elements(U):
    """Non-empty knot spans [U_s, U_{s+1}) as (lo, hi, s)."""
    U = np.asarray(U, dtype=np.float64)
    out = []
    for s in range(len(U) - 1):
        if U[s + 1] > U[s]:
            out.append((U[s], U[s + 1], s))
    return out


def local_ders_on_element(U, p, s, u):
    """Values and derivatives of the p+1 functions s-p..s that can be
    non-zero on span s, taken from the full evaluation above."""
    N, dN = basis_all_ders(U, p, u)
    return N[s - p:s + 1].copy(), dN[s - p:s + 1].copy()


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [-1, 1] (numpy's Golub-Welsch nodes)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w
