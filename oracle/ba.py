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

normal_residual evaluates the same normal equations matrix-free (a check of a proposed step that
runs at any problem size).

Parity status: analytic Jacobians pinned by central differences; a step from exact observations
at the solution is zero; Levenberg-Marquardt from perturbed poses and points on noise-free
observations drives the reprojection error to zero; the matrix-free residual vanishes at the dense
solution and equals H step - b of the dense equations for an arbitrary step.
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


def normal_equations(R, t, P, obs, K, sigma, delta, lam, axis):
    """The damped normal equations over the free parameters (cameras first, then points):
    (H + lam diag(H), b, H's diagonal, camera index [C][6], number of free camera parameters,
    robust cost).  Each observation adds its 2 x 9 Jacobian's block W J^T J at its parameters'
    indices (the same sum as over the full Jacobian, without its zero columns)."""
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
        free = [d for d in range(6) if ci[i, d] >= 0]
        for q, m in enumerate(sel):
            j = pts[m]
            idx = np.array([ci[i, d] for d in free] + [nc + 3 * j + c for c in range(3)])
            J = np.concatenate([Jc[q][:, free], Jp[q]], axis=1)
            Wm = w[m] / (sigma * sigma)
            H[np.ix_(idx, idx)] += Wm * J.T @ J
            b[idx] -= Wm * J.T @ r[m]
    diag = np.diag(H).copy()
    Hd = H + lam * np.diag(diag)
    return Hd, b, diag, ci, nc, float(rho.sum())


def lm_step(R, t, P, obs, K, sigma, delta, lam, axis):
    """One damped Gauss-Newton step by the dense normal equations.  Returns (dcam [C][6] with zeros
    for fixed parameters, dP [n][3], cost before)."""
    C, n = len(R), len(P)
    Hd, b, diag, ci, nc, cost = normal_equations(R, t, P, obs, K, sigma, delta, lam, axis)
    unseen = diag == 0.0  # a parameter no observation touches stays where it is
    Hd[unseen, unseen] = 1.0
    delta_x = np.linalg.solve(Hd, b)
    dcam = np.zeros((C, 6))
    for i in range(C):
        for d in range(6):
            if ci[i, d] >= 0:
                dcam[i, d] = delta_x[ci[i, d]]
    dP = delta_x[nc:].reshape(n, 3)
    return dcam, dP, cost


def normal_residual(R, t, P, obs, K, sigma, delta, lam, axis, dcam, dP):
    """For a proposed step (dcam, dP): the residual (H + lam diag H) step - b of the normal
    equations row by row, and per row the scale (|H| + lam diag H) |step| + |b| (|H| taken over
    the Jacobians' absolute values, an upper bound), without forming H, so it runs at any size.
    Returns (res_cam [C][6], scale_cam [C][6], res_pt [n][3], scale_pt [n][3]); fixed camera
    parameters get zeros."""
    cams, pts, uv = obs
    C, n = len(R), len(P)
    ci, _ = free_layout(C, n, axis)
    free = ci >= 0
    dc = np.where(free, dcam, 0.0)
    r, e, w, rho = cost_terms(R, t, P, obs, K, sigma, delta)
    Wm = w / (sigma * sigma)
    hc, sc, dgc, bc = (np.zeros((C, 6)) for _ in range(4))
    hp, sp, dgp, bpt = (np.zeros((n, 3)) for _ in range(4))
    for i in np.unique(cams):
        sel = np.nonzero(cams == i)[0]
        Jc, Jp = jacobians(R[i], t[i], P[pts[sel]], K)
        Jc = Jc * free[i][None, None, :]
        wq = Wm[sel][:, None]
        Jd = np.einsum("kad,d->ka", Jc, dc[i]) + np.einsum("kad,kd->ka", Jp, dP[pts[sel]])
        Ja = np.einsum("kad,d->ka", np.abs(Jc), np.abs(dc[i])) + np.einsum("kad,kd->ka", np.abs(Jp), np.abs(dP[pts[sel]]))
        hc[i] += np.einsum("kad,ka->d", Jc, wq * Jd)
        sc[i] += np.einsum("kad,ka->d", np.abs(Jc), wq * Ja)
        dgc[i] += np.einsum("kad,kad->d", Jc, Jc * wq[:, :, None])
        bc[i] -= np.einsum("kad,ka->d", Jc, wq * r[sel])
        np.add.at(hp, pts[sel], np.einsum("kad,ka->kd", Jp, wq * Jd))
        np.add.at(sp, pts[sel], np.einsum("kad,ka->kd", np.abs(Jp), wq * Ja))
        np.add.at(dgp, pts[sel], np.einsum("kad,kad->kd", Jp, Jp * wq[:, :, None]))
        np.add.at(bpt, pts[sel], -np.einsum("kad,ka->kd", Jp, wq * r[sel]))
    res_c = np.where(free, hc + lam * dgc * dc - bc, 0.0)
    scale_c = np.where(free, sc + lam * dgc * np.abs(dc) + np.abs(bc), 0.0)
    res_p = hp + lam * dgp * dP - bpt
    scale_p = sp + lam * dgp * np.abs(dP) + np.abs(bpt)
    return res_c, scale_c, res_p, scale_p


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
