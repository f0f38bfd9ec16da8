"""Scan -> discrete point sources (Section 2: source I+1 is activated dt after
source I, so successive sources are v*dt apart along the scan path; each
carries E = A*P*dt, Section 3.1).

Reading R1: a maximal run of consecutive laser-on segments is one track.  On
each track, sources sit at arc lengths 0, v*dt, 2*v*dt, ... up to the track
length.  Tracks follow one another without idle time (a laser-off segment is
a jump that takes no time and deposits nothing).  Numbering the sources
I = 1, 2, ... in scan order, source I activates at t^(I) = I*dt, i.e. it is
part of the sum from time step n = I on.
"""
from __future__ import annotations

import numpy as np


def energy(scan, dt):
    """E = A P dt (Section 3.1)."""
    return scan.absorptivity * scan.power * dt


def discretize(scan, dt):
    """Source positions (N, 3) in scan order."""
    path = np.asarray(scan.path, dtype=np.float64)
    on = np.asarray(scan.seg_on).astype(bool)
    step = scan.speed * dt
    out = []
    s = 0
    nseg = len(path) - 1
    while s < nseg:
        if not on[s]:
            s += 1
            continue
        e = s
        while e < nseg and on[e]:
            e += 1
        verts = path[s:e + 1]
        seg_len = np.linalg.norm(np.diff(verts, axis=0), axis=1)
        cum = np.concatenate([[0.0], np.cumsum(seg_len)])
        L = cum[-1]
        count = int(np.floor(L / step + 1e-9)) + 1
        for j in range(count):
            a = min(j * step, L)
            k = min(int(np.searchsorted(cum, a, side="right")) - 1, len(seg_len) - 1)
            t = (a - cum[k]) / seg_len[k] if seg_len[k] > 0 else 0.0
            out.append(verts[k] + t * (verts[k + 1] - verts[k]))
        s = e
    return np.array(out, dtype=np.float64).reshape(-1, 3)
