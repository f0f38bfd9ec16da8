"""Analytical point-source field (Section 2.1, Eqs. sum-of-point-temp and
semi-temperature):

    T~^(I)(x, t) = s_img E / (rho c_p [4 pi alpha (t - tau^(I))]^{3/2})
                   * exp(-|x - x^(I)|^2 / (4 alpha (t - tau^(I)))) H(t - tau^(I))
    tau^(I) = t^(I) - r^2 / (8 alpha)

and its gradient, obtained by differentiating the exponent:

    grad T~^(I) = -(x - x^(I)) / (2 alpha (t - tau^(I))) T~^(I).

Reading R1: a source enters the sum once t >= t^(I) (causal activation), so
its age t - tau^(I) is at least r^2/(8 alpha).  Reading R2: s_img = 2 by
default (the half-space with adiabatic top plane); the printed full-space
kernel is s_img = 1.

The age at step n of source I is computed as ((n - I) dt) + r^2/(8 alpha)
from the integer step difference, never as a difference of two large times.
"""
from __future__ import annotations

import numpy as np


def diffusivity(mat):
    """alpha = k / (rho c_p) (Eq. linear-heat)."""
    return mat.k / (mat.rho * mat.cp)


def ages(n, n_active, dt, mat, spot_radius):
    """Ages of sources I = 1..n_active at step n: (n - I) dt + r^2/(8 alpha)."""
    alpha = diffusivity(mat)
    I = np.arange(1, n_active + 1, dtype=np.float64)
    return (n - I) * dt + spot_radius ** 2 / (8.0 * alpha)


def T_point(x, xs, age, E, mat, s_img=2.0):
    """T~^(I) at points x (Q,3) from sources xs (K,3) of ages age (K,): (Q,K)."""
    alpha = diffusivity(mat)
    d = x[:, None, :] - xs[None, :, :]
    R2 = np.einsum("qkc,qkc->qk", d, d)
    pref = s_img * E / (mat.rho * mat.cp * (4.0 * np.pi * alpha * age) ** 1.5)
    return pref[None, :] * np.exp(-R2 / (4.0 * alpha * age[None, :]))


def gradT_point(x, xs, age, E, mat, s_img=2.0):
    """grad T~^(I) at x (Q,3): (Q,K,3)."""
    alpha = diffusivity(mat)
    d = x[:, None, :] - xs[None, :, :]
    T = T_point(x, xs, age, E, mat, s_img)
    return -d / (2.0 * alpha * age[None, :, None]) * T[:, :, None]


def T_tilde(x, xs, age, E, mat, s_img=2.0, chunk=256):
    """T~(x) = sum over the given sources, summed in source order."""
    out = np.zeros(len(x))
    for q0 in range(0, len(x), chunk):
        out[q0:q0 + chunk] = T_point(x[q0:q0 + chunk], xs, age, E, mat, s_img).sum(axis=1)
    return out


def dTdn_tilde(x, nrm, xs, age, E, mat, s_img=2.0, chunk=256):
    """dT~/dn(x) = n . grad T~(x), summed over the given sources."""
    out = np.zeros(len(x))
    for q0 in range(0, len(x), chunk):
        g = gradT_point(x[q0:q0 + chunk], xs, age, E, mat, s_img)   # (q,K,3)
        out[q0:q0 + chunk] = np.einsum("qkc,qc->q", g, nrm[q0:q0 + chunk])
    return out


def unit_bound(box_lo, box_hi, xs, age, E, mat, s_img=2.0, normal=None):
    """Upper bound, over the points x of the axis-aligned box [box_lo,
    box_hi], of sum_I |term_I(x)| for the given sources (the opt-in history
    cutoff, not part of the paper's method, which keeps every term).

    Each term decreases with the distance from its source, so it is largest
    at the box point nearest to the source, at distance d_I:
      T~ terms (normal None):    |T~^(I)(x)| <= c_I exp(-a_I d_I^2)
      normal-derivative terms on a face with unit normal n along a
      coordinate axis (box_lo = box_hi along it), where n . (x - x_I) is the
      same at every point:       |n . grad T~^(I)(x)| <= 2 a_I c_I |n . (x - x_I)| exp(-a_I d_I^2)
    with a_I = 1/(4 alpha age_I) and c_I the prefactor of Eq. semi-temperature.
    Returns the bound per source (K,)."""
    alpha = diffusivity(mat)
    lo = np.asarray(box_lo, float)
    hi = np.asarray(box_hi, float)
    a = 1.0 / (4.0 * alpha * age)
    c = s_img * E / (mat.rho * mat.cp * (4.0 * np.pi * alpha * age) ** 1.5)
    dv = np.maximum(0.0, np.maximum(lo[None, :] - xs, xs - hi[None, :]))
    d2 = np.einsum("kc,kc->k", dv, dv)
    b = c * np.exp(-a * d2)
    if normal is not None:
        b = 2.0 * a * b * np.abs((lo[None, :] - xs) @ np.asarray(normal, float))
    return b
