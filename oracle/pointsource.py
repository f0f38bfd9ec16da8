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
