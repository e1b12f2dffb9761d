"""FP64 oracle of the dense visual bundle-adjustment step of the tracker
(Sec. 3.2, "Vision Residual" Eq. 2 and "Frontend Tracking: Local Bundle
Adjustment" Eq. 4).

TEST INFRASTRUCTURE (see oracle/__init__.py).  Written from the definitions:

  keyframe k: world-to-camera pose T_k = (R_k, t_k); inverse-depth (disparity)
  map d_k on an h x w pixel grid u = (x, y) (pixel centres x + 0.5, y + 0.5);
  edge (i, j) of the frame graph: target correspondences u*_ij [h, w, 2] and
  confidence weights w_ij [h, w, 2] for the pixels of keyframe i.

  residual (Eq. 2): r = u*_ij - Pi(T_j T_i^-1 Pi^-1(u, d_i(u))), with
  Pi^-1(u, d) the point at inverse depth d along pixel u's ray and Pi the
  pinhole projection; the cost is sum w r^2 (Mahalanobis with diag(w)).

  variables: a left perturbation xi_k = (rho, phi) of every pose beyond the
  first n_fixed (T_k <- Exp(xi_k) T_k), and every inverse depth of every
  keyframe that is an edge source.

  one Levenberg-Marquardt step: H = J^T W J, g = J^T W r,
  (H + lambda diag(H) + eps I) delta = -g; the poses step by Exp(xi) (first
  order in the translation, as the renderer's pose tangent), the inverse
  depths by addition.

The oracle builds the full dense Jacobian and solves the full system (no
Schur complement), so it checks the GPU's block elimination of the diagonal
depth block C (Eq. 4) by the plain definition.

Parity status (tests/test_oracle_ba.py): Jacobian against central differences
of the residual; Gauss-Newton converging to the generating poses and depths on
exact synthetic correspondences; the solve against a least-squares routine.
"""
from __future__ import annotations

import numpy as np


def skew(v):
    v = np.asarray(v, np.float64)
    return np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])


def so3_exp(phi):
    phi = np.asarray(phi, np.float64)
    th = np.linalg.norm(phi)
    K = skew(phi)
    if th < 1e-12:
        return np.eye(3) + K
    return np.eye(3) + np.sin(th) / th * K + (1 - np.cos(th)) / th ** 2 * K @ K


def pixel_rays(intr, h, w):
    """Normalised rays (x', y', 1) of the pixel centres, [h, w, 3]."""
    fx, fy, cx, cy = intr
    ys, xs = np.mgrid[0:h, 0:w]
    return np.stack([(xs + 0.5 - cx) / fx, (ys + 0.5 - cy) / fy, np.ones((h, w))], -1)


def relative(R, t, i, j):
    """T_ij = T_j T_i^-1 (camera i -> camera j)."""
    Rij = R[j] @ R[i].T
    return Rij, t[j] - Rij @ t[i]


def residuals(R, t, disp, intr, edges, targets):
    """r [E, h, w, 2] = u* - Pi(T_ij Pi^-1(u, d))."""
    fx, fy, cx, cy = intr
    E = len(edges)
    h, w = disp.shape[1:]
    rays = pixel_rays(intr, h, w)
    out = np.zeros((E, h, w, 2))
    for e, (i, j) in enumerate(edges):
        Rij, tij = relative(R, t, i, j)
        p = rays @ Rij.T + disp[i][..., None] * tij          # the point times its inverse depth
        out[e, ..., 0] = targets[e, ..., 0] - (fx * p[..., 0] / p[..., 2] + cx)
        out[e, ..., 1] = targets[e, ..., 1] - (fy * p[..., 1] / p[..., 2] + cy)
    return out


def jacobian(R, t, disp, intr, edges, n_fixed):
    """Dense J [2 E h w, 6 (K - n_fixed) + K h w] of the residuals with respect
    to the pose perturbations (first order) and the inverse depths."""
    fx, fy, cx, cy = intr
    K = R.shape[0]
    h, w = disp.shape[1:]
    P = h * w
    nx = 6 * (K - n_fixed)
    rays = pixel_rays(intr, h, w).reshape(P, 3)
    J = np.zeros((2 * len(edges) * P, nx + K * P))
    for e, (i, j) in enumerate(edges):
        Rij, tij = relative(R, t, i, j)
        d = disp[i].reshape(P)
        for q in range(P):
            xb = rays[q]
            p = Rij @ xb + d[q] * tij
            iz = 1.0 / p[2]
            Jpi = np.array([[fx * iz, 0, -fx * p[0] * iz * iz], [0, fy * iz, -fy * p[1] * iz * iz]])
            rows = slice(2 * (e * P + q), 2 * (e * P + q) + 2)
            # T_j <- Exp(xi_j) T_j moves p by rho_j d + phi_j x p
            if j >= n_fixed:
                dp = np.hstack([d[q] * np.eye(3), -skew(p)])
                J[rows, 6 * (j - n_fixed):6 * (j - n_fixed) + 6] += -Jpi @ dp
            # T_i^-1 <- T_i^-1 Exp(-xi_i) moves the camera-i point by -(rho_i d + phi_i x xb)
            if i >= n_fixed:
                dp = np.hstack([-d[q] * Rij, Rij @ skew(xb)])
                J[rows, 6 * (i - n_fixed):6 * (i - n_fixed) + 6] += -Jpi @ dp
            J[rows, nx + i * P + q] = -Jpi @ tij
    return J


def lm_step(R, t, disp, intr, edges, targets, weights, n_fixed, lam=1e-4, eps=1e-4):
    """One damped Gauss-Newton step by the full dense solve.  Returns
    (dxi [K - n_fixed, 6], ddisp [K, h, w], H, g, cost)."""
    K = R.shape[0]
    h, w = disp.shape[1:]
    r = residuals(R, t, disp, intr, edges, targets).reshape(-1)
    W = np.asarray(weights, np.float64).reshape(-1)
    J = jacobian(R, t, disp, intr, edges, n_fixed)
    H = J.T @ (W[:, None] * J)
    g = J.T @ (W * r)
    A = H + lam * np.diag(np.diag(H)) + eps * np.eye(H.shape[0])
    delta = np.linalg.solve(A, -g)
    nx = 6 * (K - n_fixed)
    return delta[:nx].reshape(K - n_fixed, 6), delta[nx:].reshape(K, h, w), H, g, float(np.sum(W * r * r))


def apply_step(R, t, disp, dxi, ddisp, n_fixed):
    """T_k <- Exp(xi_k) T_k (translation to first order) for the free poses; d += dd."""
    R = R.copy(); t = t.copy()
    for k in range(n_fixed, R.shape[0]):
        rho, phi = dxi[k - n_fixed, :3], dxi[k - n_fixed, 3:]
        Rphi = so3_exp(phi)
        R[k] = Rphi @ R[k]
        t[k] = Rphi @ t[k] + rho
    return R, t, disp + ddisp
