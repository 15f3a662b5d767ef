"""CPU oracle of the bundle adjustment of the geometry prior (Sec. III-A, Eq. 2 objective, Eq. 3
reduced camera system) — TEST INFRASTRUCTURE ONLY (imported by the tests, never by the product
path).  Plain FP64 numpy, written from the definitions:

  camera i: world-to-camera rotation R_i and translation t_i; pinhole (fx, fy, cx, cy);
  pi(T_i, P_j) = (fx x / z + cx, fy y / z + cy) with (x, y, z) = R_i P_j + t_i;
  residual r_ij = pi(T_i, P_j) - p_ij, whitened by the observation sigma (W_ij = I / sigma^2);
  robust weight (Huber on the whitened residual norm e): w = 1 for e <= delta, delta / e beyond
  (the iteratively reweighted form of rho);
  local update of camera i: R_i <- exp([w]x) R_i, t_i <- t_i + v (rotation on the left, translation
  added), of point j: P_j <- P_j + d;
  gauge (Sec. III-A): camera 0 fixed; of camera 1's translation, the component on the axis where
  its initial baseline to camera 0, expressed in camera 1's frame, is largest is fixed;
  one Levenberg-Marquardt step: H = J^T W J and b = -J^T W r over the free parameters, damped as
  H + lam diag(H) (a parameter that no observation touches keeps a zero step), solved densely
  (numpy.linalg.solve) — the plain definition that the GPU's Schur complement (Eq. 3) reaches
  exactly up to rounding.

Parity status: analytic Jacobians pinned by central differences; a step from exact observations
at the solution is zero; Levenberg-Marquardt from perturbed poses and points on noise-free
observations drives the reprojection error to zero.
"""
from __future__ import annotations

import numpy as np


def skew(a):
    return np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])


def expso3(w):
    """Rodrigues' formula."""
    th = np.linalg.norm(w)
    if th < 1e-12:
        return np.eye(3) + skew(w)
    k = w / th
    K = skew(k)
    return np.eye(3) + np.sin(th) * K + (1.0 - np.cos(th)) * K @ K


def project(R, t, P, K):
    """pi for one camera (R [3][3], t [3]) and points P [n][3]; K = (fx, fy, cx, cy).
    Returns uv [n][2] and camera-frame points [n][3]."""
    Xc = P @ R.T + t
    fx, fy, cx, cy = K
    uv = np.stack([fx * Xc[:, 0] / Xc[:, 2] + cx, fy * Xc[:, 1] / Xc[:, 2] + cy], axis=1)
    return uv, Xc


def jacobians(R, t, P, K):
    """d pi / d(w, v) [n][2][6] and d pi / dP [n][2][3] at the current camera and points."""
    _, Xc = project(R, t, P, K)
    fx, fy = K[0], K[1]
    n = P.shape[0]
    Jc = np.zeros((n, 2, 6))
    Jp = np.zeros((n, 2, 3))
    for k in range(n):
        x, y, z = Xc[k]
        dpi = np.array([[fx / z, 0.0, -fx * x / (z * z)], [0.0, fy / z, -fy * y / (z * z)]])
        RP = R @ P[k]
        Jc[k, :, 0:3] = dpi @ (-skew(RP))   # d(exp([w]x) R P)/dw at w = 0
        Jc[k, :, 3:6] = dpi
        Jp[k] = dpi @ R
    return Jc, Jp


def gauge_axis(R, t):
    """The fixed translation component of camera 1: the largest component of its initial baseline
    to camera 0 in camera 1's frame (camera centres c = -R^T t)."""
    c0 = -R[0].T @ t[0]
    c1 = -R[1].T @ t[1]
    return int(np.argmax(np.abs(R[1] @ (c1 - c0))))


def free_layout(C, P, axis):
    """Index of every free parameter: cameras 1.. (camera 1 without translation `axis`), then
    points.  Returns (cam_index [C][6] with -1 for fixed, point offset)."""
    ci = -np.ones((C, 6), np.int64)
    k = 0
    for i in range(1, C):
        for d in range(6):
            if i == 1 and d == 3 + axis:
                continue
            ci[i, d] = k
            k += 1
    return ci, k


def cost_terms(R, t, P, obs, K, sigma, delta):
    """Per observation: residual r [m][2], whitened norm e, Huber weight w, robust cost rho."""
    cams, pts, uv = obs
    r = np.zeros((len(cams), 2))
    for i in np.unique(cams):
        sel = np.nonzero(cams == i)[0]
        pr, _ = project(R[i], t[i], P[pts[sel]], K)
        r[sel] = pr - uv[sel]
    e = np.linalg.norm(r, axis=1) / sigma
    w = np.where(e <= delta, 1.0, delta / np.maximum(e, 1e-300))
    rho = np.where(e <= delta, e * e, 2.0 * delta * e - delta * delta)
    return r, e, w, rho


def lm_step(R, t, P, obs, K, sigma, delta, lam, axis):
    """One damped Gauss-Newton step by the dense normal equations.  Returns (dcam [C][6] with zeros
    for fixed parameters, dP [n][3], cost before)."""
    cams, pts, uv = obs
    C, n = len(R), len(P)
    ci, nc = free_layout(C, n, axis)
    N = nc + 3 * n
    H = np.zeros((N, N))
    b = np.zeros(N)
    r, e, w, rho = cost_terms(R, t, P, obs, K, sigma, delta)
    for i in np.unique(cams):
        sel = np.nonzero(cams == i)[0]
        Jc, Jp = jacobians(R[i], t[i], P[pts[sel]], K)
        for q, m in enumerate(sel):
            J = np.zeros((2, N))
            for d in range(6):
                if ci[i, d] >= 0:
                    J[:, ci[i, d]] = Jc[q, :, d]
            j = pts[m]
            J[:, nc + 3 * j:nc + 3 * j + 3] = Jp[q]
            Wm = w[m] / (sigma * sigma)
            H += Wm * J.T @ J
            b -= Wm * J.T @ r[m]
    Hd = H + lam * np.diag(np.diag(H))
    unseen = np.diag(H) == 0.0  # a parameter no observation touches stays where it is
    Hd[unseen, unseen] = 1.0
    delta_x = np.linalg.solve(Hd, b)
    dcam = np.zeros((C, 6))
    for i in range(C):
        for d in range(6):
            if ci[i, d] >= 0:
                dcam[i, d] = delta_x[ci[i, d]]
    dP = delta_x[nc:].reshape(n, 3)
    return dcam, dP, float(rho.sum())


def apply(R, t, P, dcam, dP):
    R2 = np.array([expso3(dcam[i, 0:3]) @ R[i] for i in range(len(R))])
    t2 = t + dcam[:, 3:6]
    return R2, t2, P + dP


def solve(R, t, P, obs, K, sigma, delta, iters=20, lam=1e-4):
    """Levenberg-Marquardt: accept a step when the robust cost drops (lam / 10), else lam * 10."""
    axis = gauge_axis(R, t)
    costs = [float(cost_terms(R, t, P, obs, K, sigma, delta)[3].sum())]
    for _ in range(iters):
        dcam, dP, c0 = lm_step(R, t, P, obs, K, sigma, delta, lam, axis)
        R2, t2, P2 = apply(R, t, P, dcam, dP)
        c1 = float(cost_terms(R2, t2, P2, obs, K, sigma, delta)[3].sum())
        if c1 < c0:
            R, t, P, lam = R2, t2, P2, lam / 10.0
            costs.append(c1)
        else:
            lam *= 10.0
    return R, t, P, costs
