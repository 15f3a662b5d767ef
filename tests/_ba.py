"""Observation sets for the bundle-adjustment tests, built with the oracle's projection."""
import numpy as np

from oracle import ba as O


def observations(p, R, t, P, noise=True, tracks=False):
    """All (camera, point) pairs in front of the camera and inside the image (and, with tracks,
    inside the point's feature track), ordered by point then camera; points seen fewer than twice
    are dropped.  Returns (cams, pts, uv) as numpy arrays."""
    C = len(R)
    cams, pts, uvs = [], [], []
    for i in range(C):
        uv, Xc = O.project(R[i], t[i], P, p.K)
        ok = (Xc[:, 2] > 0.2) & (uv[:, 0] >= 0) & (uv[:, 0] < p.width) & (uv[:, 1] >= 0) & (uv[:, 1] < p.height)
        if tracks:
            ok &= (i - p.track_start) % C < p.track_len
        js = np.nonzero(ok)[0]
        cams.append(np.full(len(js), i))
        pts.append(js)
        uvs.append(uv[js] + (p.noise[i, js] if noise else 0.0))
    cams, pts, uvs = np.concatenate(cams), np.concatenate(pts), np.concatenate(uvs)
    keep = np.bincount(pts, minlength=len(P))[pts] >= 2   # a point needs two views
    order = np.lexsort((cams[keep], pts[keep]))
    return cams[keep][order], pts[keep][order], uvs[keep][order]
