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

Inertial factor (Eq. 3), between consecutive keyframes i, j = i + 1, on the
body-to-world rotation R_i = R_cw,i^T, position p_i = -R_i t_cw,i, velocity v_i
and IMU bias b_i = (b_g, b_a) (camera and body frames taken as one, as the
paper's equations do), with pre-integrated dR, dp, dv, Jacobians J_rot (3x3,
gyro bias), J_pos and J_vel (3x6, full bias), time step dt, gravity g and a
15 x 15 information matrix:
  r_rot  = Log((dR Exp(J_rot (b_g,i - bh_g,i)))^T R_i^T R_j)
  r_pos  = R_i^T (p_j - p_i - v_i dt - g dt^2 / 2) - (dp + J_pos (b_i - bh_i))
  r_vel  = R_i^T (v_j - v_i - g dt) - (dv + J_vel (b_i - bh_i))
  r_bias = b_j - b_i
(reading: the velocity term's bias correction uses the full bias, as the
position term's does; the printed equation writes the gyro part there).  The
variables of a keyframe become (rho, phi, v, b): 15; the inertial Jacobian is
taken by central differences of these residuals under the same perturbation
as the visual part (T_cw <- Exp(xi) T_cw; v, b additive), so it rests on the
residual's definition alone.

Parity status (tests/test_oracle_ba.py): as above, plus the inertial residual
vanishing on a consistent synthetic trajectory and Gauss-Newton over the
joint visual-inertial objective recovering it.

Parity status of the visual part (tests/test_oracle_ba.py): Jacobian against
central differences of the residual; Gauss-Newton converging to the generating
poses and depths on exact synthetic correspondences; the solve against a
least-squares routine.
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


# ------------------------------------------------------------------ inertial

IMU_FLOATS = 9 + 3 + 3 + 9 + 18 + 18 + 1 + 225     # one pair's record (see imu_record)


def so3_log(M):
    """Rotation vector of a rotation matrix."""
    M = np.asarray(M, np.float64)
    c = np.clip((np.trace(M) - 1.0) / 2.0, -1.0, 1.0)
    th = np.arccos(c)
    w = np.array([M[2, 1] - M[1, 2], M[0, 2] - M[2, 0], M[1, 0] - M[0, 1]]) / 2.0
    if th < 1e-8:
        return w
    return w * th / np.sin(th)


def body_states(R, t):
    """Body-to-world rotations R_i = R_cw^T and positions p_i = -R_i t_cw."""
    Rb = np.transpose(np.asarray(R, np.float64), (0, 2, 1))
    return Rb, -np.einsum("kab,kb->ka", Rb, np.asarray(t, np.float64))


def imu_record(dR, dp, dv, Jrot, Jpos, Jvel, dt, info):
    """One consecutive pair's pre-integration record in the library's layout."""
    return np.concatenate([np.asarray(dR, np.float64).reshape(9), dp, dv, np.asarray(Jrot).reshape(9),
                           np.asarray(Jpos).reshape(18), np.asarray(Jvel).reshape(18), [dt],
                           np.asarray(info).reshape(225)])


def _unpack(rec):
    rec = np.asarray(rec, np.float64)
    o = 0
    def take(k, shape):
        nonlocal o
        v = rec[o:o + k].reshape(shape); o += k
        return v
    dR = take(9, (3, 3)); dp = take(3, 3); dv = take(3, 3); Jrot = take(9, (3, 3))
    Jpos = take(18, (3, 6)); Jvel = take(18, (3, 6)); dt = take(1, 1)[0]; info = take(225, (15, 15))
    return dR, dp, dv, Jrot, Jpos, Jvel, dt, info


def inertial_residual(R, t, vel, bias, bias_hat, imu, gravity, i):
    """r (15) of the pair (i, i + 1), Eq. 3."""
    dR, dp, dv, Jrot, Jpos, Jvel, dt, _ = _unpack(imu[i])
    Rb, pb = body_states(R, t)
    j = i + 1
    g = np.asarray(gravity, np.float64)
    db = np.asarray(bias[i], np.float64) - np.asarray(bias_hat[i], np.float64)
    A = dR @ so3_exp(Jrot @ db[:3])
    r_rot = so3_log(A.T @ Rb[i].T @ Rb[j])
    r_pos = Rb[i].T @ (pb[j] - pb[i] - vel[i] * dt - 0.5 * g * dt * dt) - (dp + Jpos @ db)
    r_vel = Rb[i].T @ (vel[j] - vel[i] - g * dt) - (dv + Jvel @ db)
    r_bias = np.asarray(bias[j], np.float64) - np.asarray(bias[i], np.float64)
    return np.concatenate([r_rot, r_pos, r_vel, r_bias])


def apply_step_vi(R, t, disp, vel, bias, dx, ddisp, n_fixed):
    """dx [K - n_fixed, 15] = (rho, phi, dv, db) per free keyframe: poses by
    apply_step, velocities and biases additively."""
    dx = np.asarray(dx, np.float64)
    R2, t2, d2 = apply_step(R, t, disp, dx[:, :6], ddisp, n_fixed)
    v2 = np.array(vel, np.float64); b2 = np.array(bias, np.float64)
    v2[n_fixed:] += dx[:, 6:9]
    b2[n_fixed:] += dx[:, 9:15]
    return R2, t2, d2, v2, b2


def inertial_jacobian(R, t, vel, bias, bias_hat, imu, gravity, n_fixed, h=1e-6):
    """Dense J [15 (K - 1), 15 (K - n_fixed)] of all pairs' residuals by central
    differences over the free keyframes' (rho, phi, v, b)."""
    K = np.asarray(R).shape[0]
    nv = 15 * (K - n_fixed)
    disp0 = np.zeros((K, 1, 1))
    def all_res(dx):
        R2, t2, _, v2, b2 = apply_step_vi(R, t, disp0, vel, bias, dx.reshape(K - n_fixed, 15), 0.0, n_fixed)
        return np.concatenate([inertial_residual(R2, t2, v2, b2, bias_hat, imu, gravity, i) for i in range(K - 1)])
    J = np.zeros((15 * (K - 1), nv))
    for c in range(nv):
        e = np.zeros(nv); e[c] = h
        J[:, c] = (all_res(e) - all_res(-e)) / (2 * h)
    return J


def lm_step_vi(R, t, disp, vel, bias, bias_hat, intr, edges, targets, weights, imu, gravity, n_fixed,
               lam=1e-4, eps=1e-4):
    """One damped Gauss-Newton step of the joint visual (Eq. 2) + inertial
    (Eq. 3) objective by the full dense solve.  Returns (dx [K - n_fixed, 15],
    ddisp [K, h, w], cost)."""
    K = np.asarray(R).shape[0]
    h, w = disp.shape[1:]
    P = h * w
    nx6 = 6 * (K - n_fixed)
    # visual part, its pose columns spread into the 15-wide keyframe blocks
    rv = residuals(R, t, disp, intr, edges, targets).reshape(-1)
    Wv = np.asarray(weights, np.float64).reshape(-1)
    Jv6 = jacobian(R, t, disp, intr, edges, n_fixed)
    nx = 15 * (K - n_fixed)
    Jv = np.zeros((Jv6.shape[0], nx + K * P))
    for k in range(K - n_fixed):
        Jv[:, 15 * k:15 * k + 6] = Jv6[:, 6 * k:6 * k + 6]
    Jv[:, nx:] = Jv6[:, nx6:]
    # inertial part
    ri = np.concatenate([inertial_residual(R, t, vel, bias, bias_hat, imu, gravity, i) for i in range(K - 1)])
    Ji = np.zeros((15 * (K - 1), nx + K * P))
    Ji[:, :nx] = inertial_jacobian(R, t, vel, bias, bias_hat, imu, gravity, n_fixed)
    Wi = np.zeros((15 * (K - 1), 15 * (K - 1)))
    for i in range(K - 1):
        Wi[15 * i:15 * i + 15, 15 * i:15 * i + 15] = _unpack(imu[i])[7]
    H = Jv.T @ (Wv[:, None] * Jv) + Ji.T @ Wi @ Ji
    g = Jv.T @ (Wv * rv) + Ji.T @ Wi @ ri
    A = H + lam * np.diag(np.diag(H)) + eps * np.eye(H.shape[0])
    delta = np.linalg.solve(A, -g)
    cost = float(np.sum(Wv * rv * rv) + ri @ Wi @ ri)
    return delta[:nx].reshape(K - n_fixed, 15), delta[nx:].reshape(K, h, w), cost
