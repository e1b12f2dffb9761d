"""Pins of the dense bundle-adjustment oracle (oracle/ba.py, Eq. 2 / Eq. 4)."""
import numpy as np

from oracle import ba
from paper_2512_02293_gb300 import synth


def _exact_targets(R, t, disp, intr, edges):
    h, w = disp.shape[1:]
    zero = np.zeros((len(edges), h, w, 2))
    return -ba.residuals(R, t, disp, intr, edges, zero)        # u* = Pi(T_ij Pi^-1(u, d))


def test_jacobian_matches_central_differences():
    R, t, disp, intr, edges, wts = synth.ba_scene(1, K=4, h=4, w=5)
    rng = np.random.default_rng(2)
    targets = _exact_targets(R, t, disp, intr, edges) + rng.normal(0, 0.5, (len(edges), 4, 5, 2))
    n_fixed = 1
    J = ba.jacobian(R, t, disp, intr, edges, n_fixed)
    K, h, w = disp.shape
    nx = 6 * (K - n_fixed)
    hstep = 1e-6
    for col in list(range(nx)) + list(rng.choice(np.arange(nx, J.shape[1]), 12, replace=False)):
        def res(s):
            if col < nx:
                dxi = np.zeros((K - n_fixed, 6)); dxi.reshape(-1)[col] = s
                R2, t2, d2 = ba.apply_step(R, t, disp, dxi, np.zeros_like(disp), n_fixed)
            else:
                dd = np.zeros(K * h * w); dd[col - nx] = s
                R2, t2, d2 = R, t, disp + dd.reshape(K, h, w)
            return ba.residuals(R2, t2, d2, intr, edges, targets).reshape(-1)
        fd = (res(hstep) - res(-hstep)) / (2 * hstep)
        np.testing.assert_allclose(J[:, col], fd, rtol=1e-5, atol=1e-6, err_msg=str(col))


def test_gauss_newton_recovers_the_generating_window():
    R, t, disp, intr, edges, wts = synth.ba_scene(3, K=4, h=6, w=8)
    targets = _exact_targets(R, t, disp, intr, edges)
    rng = np.random.default_rng(4)
    n_fixed = 2                                     # fixes the gauge, scale included
    R0, t0 = R.copy(), t.copy()
    dxi = rng.normal(0, 0.01, (2, 6))
    R1, t1, d1 = ba.apply_step(R, t, disp, np.vstack([dxi]), rng.normal(0, 0.01, disp.shape), n_fixed)
    cost0 = None
    for it in range(15):
        dx, dd, H, g, cost = ba.lm_step(R1, t1, d1, intr, edges, targets, wts, n_fixed, lam=1e-6, eps=1e-9)
        cost0 = cost if cost0 is None else cost0
        R1, t1, d1 = ba.apply_step(R1, t1, d1, dx, dd, n_fixed)
    assert cost < 1e-12 * max(1.0, cost0)
    np.testing.assert_allclose(d1, disp, atol=1e-7)
    np.testing.assert_allclose(R1, R0, atol=1e-8)
    np.testing.assert_allclose(t1, t0, atol=1e-8)


def test_step_solves_the_damped_least_squares_problem():
    R, t, disp, intr, edges, wts = synth.ba_scene(5, K=3, h=4, w=5)
    rng = np.random.default_rng(6)
    targets = _exact_targets(R, t, disp, intr, edges) + rng.normal(0, 0.3, (len(edges), 4, 5, 2))
    lam, eps = 1e-2, 1e-3
    dx, dd, H, g, cost = ba.lm_step(R, t, disp, intr, edges, targets, wts, 1, lam=lam, eps=eps)
    r = ba.residuals(R, t, disp, intr, edges, targets).reshape(-1)
    J = ba.jacobian(R, t, disp, intr, edges, 1)
    sw = np.sqrt(np.asarray(wts).reshape(-1))
    D = np.sqrt(lam * np.diag(H) + eps)
    A = np.vstack([sw[:, None] * J, np.diag(D)])
    b = np.concatenate([-sw * r, np.zeros(J.shape[1])])
    delta = np.linalg.lstsq(A, b, rcond=None)[0]
    np.testing.assert_allclose(np.concatenate([dx.reshape(-1), dd.reshape(-1)]), delta, rtol=1e-7, atol=1e-10)


# ------------------------------------------------------------ inertial (Eq. 3)

def test_inertial_residual_vanishes_on_a_consistent_trajectory():
    R, t, disp, intr, edges, wts, vel, bias, bh, g, imu = synth.vi_scene(5, K=5)
    for i in range(4):
        np.testing.assert_allclose(ba.inertial_residual(R, t, vel, bias, bh, imu, g, i), 0.0, atol=1e-9)


def test_inertial_residual_terms():
    # each term moves with its own variable: a velocity offset moves r_pos by
    # -R_i^T dv dt and r_vel by -R_i^T dv; a common bias offset leaves r_bias at 0
    # and moves r_pos by -J_pos db and r_vel by -J_vel db; a rotation of keyframe j about its own frame
    # moves r_rot by that angle
    R, t, disp, intr, edges, wts, vel, bias, bh, g, imu = synth.vi_scene(6, K=3)
    Rb, _ = ba.body_states(R, t)
    dR, dp, dv, Jrot, Jpos, Jvel, dt, info = ba._unpack(imu[0])
    d = np.array([0.1, -0.2, 0.05])
    v2 = vel.copy(); v2[0] += d
    r = ba.inertial_residual(R, t, v2, bias, bh, imu, g, 0)
    np.testing.assert_allclose(r[3:6], -Rb[0].T @ d * dt, atol=1e-12)
    np.testing.assert_allclose(r[6:9], -Rb[0].T @ d, atol=1e-12)
    db = np.array([0, 0, 0, 0.02, -0.01, 0.03])
    b2 = bias + db
    r = ba.inertial_residual(R, t, vel, b2, bh, imu, g, 0)
    np.testing.assert_allclose(r[12:], 0.0, atol=1e-12)
    np.testing.assert_allclose(r[3:6], -Jpos @ db, atol=1e-12)
    # the velocity term's correction takes the accelerometer bias too (3 x 6 J_vel)
    np.testing.assert_allclose(r[6:9], -Jvel @ db, atol=1e-12)
    assert np.abs(Jvel[:, 3:] @ db[3:]).max() > 1e-3
    phi = np.array([0.01, -0.02, 0.015])
    R2 = R.copy(); R2[1] = (Rb[1] @ ba.so3_exp(phi)).T          # R_j <- R_j Exp(phi)
    r = ba.inertial_residual(R2, t - 0 * t, vel, bias, bh, imu, g, 0)
    np.testing.assert_allclose(r[:3], phi, atol=1e-9)


def test_visual_inertial_gauss_newton_recovers_the_window():
    R, t, disp, intr, edges, wts, vel, bias, bh, g, imu = synth.vi_scene(7, K=5, h=6, w=8)
    targets = _exact_targets(R, t, disp, intr, edges)
    rng = np.random.default_rng(8)
    n_fixed = 1
    dx0 = np.concatenate([rng.normal(0, 0.01, (4, 6)), rng.normal(0, 0.05, (4, 3)), rng.normal(0, 0.005, (4, 6))], 1)
    R1, t1, d1, v1, b1 = ba.apply_step_vi(R, t, disp, vel, bias, dx0, rng.normal(0, 0.01, disp.shape), n_fixed)
    costs = []
    for _ in range(8):
        dx, dd, cost = ba.lm_step_vi(R1, t1, d1, v1, b1, bh, intr, edges, targets, wts, imu, g, n_fixed,
                                     lam=1e-6, eps=1e-8)
        costs.append(cost)
        R1, t1, d1, v1, b1 = ba.apply_step_vi(R1, t1, d1, v1, b1, dx, dd, n_fixed)
    assert costs[-1] < 1e-10 * costs[0]
    np.testing.assert_allclose(d1, disp, atol=1e-7)
    np.testing.assert_allclose(t1, t, atol=1e-7)
    np.testing.assert_allclose(v1, vel, atol=1e-6)
    np.testing.assert_allclose(b1, bias, atol=1e-7)


def test_inertial_jacobian_closed_form_blocks():
    # blocks of the Eq. 3 Jacobian that are exact closed forms at any state, for
    # the pair (1, 2) of a perturbed 4-keyframe window with keyframe 0 fixed:
    # perturbation R_k <- R_k Exp(-phi), p_k <- p_k - R_k rho, v and b additive
    R, t, disp, intr, edges, wts, vel, bias, bh, g, imu = synth.vi_scene(8, K=4)
    rng = np.random.default_rng(9)
    dx0 = np.concatenate([rng.normal(0, 0.05, (3, 6)), rng.normal(0, 0.1, (3, 3)), rng.normal(0, 0.01, (3, 6))], 1)
    R, t, _, vel, bias = ba.apply_step_vi(R, t, disp, vel, bias, dx0, 0.0, 1)
    J = ba.inertial_jacobian(R, t, vel, bias, bh, imu, g, 1)
    Rb, _ = ba.body_states(R, t)
    _, _, _, _, Jpos, Jvel, dt, _ = ba._unpack(imu[1])
    rows = slice(15, 30)                       # residuals of pair (1, 2)
    Ji, Jj = J[rows, 0:15], J[rows, 15:30]     # columns of keyframes 1 and 2
    Ri, Rj = Rb[1], Rb[2]
    tol = dict(atol=1e-6)
    np.testing.assert_allclose(Ji[3:6, 0:3], np.eye(3), **tol)                 # d r_pos / d rho_i
    np.testing.assert_allclose(Jj[3:6, 0:3], -Ri.T @ Rj, **tol)                # d r_pos / d rho_j
    np.testing.assert_allclose(Ji[3:6, 6:9], -Ri.T * dt, **tol)                # d r_pos / d v_i
    np.testing.assert_allclose(Ji[6:9, 6:9], -Ri.T, **tol)                     # d r_vel / d v_i
    np.testing.assert_allclose(Jj[6:9, 6:9], Ri.T, **tol)                      # d r_vel / d v_j
    np.testing.assert_allclose(Ji[3:6, 9:15], -Jpos, **tol)                    # d r_pos / d b_i
    np.testing.assert_allclose(Ji[6:9, 9:15], -Jvel, **tol)                    # d r_vel / d b_i
    np.testing.assert_allclose(Ji[9:15, 9:15], -np.eye(6), **tol)              # d r_bias / d b_i
    np.testing.assert_allclose(Jj[9:15, 9:15], np.eye(6), **tol)               # d r_bias / d b_j
    for blk in (Ji[0:3, 0:3], Jj[0:3, 0:3], Ji[6:9, 0:3], Jj[6:9, 0:3], Ji[9:15, 0:9], Jj[9:15, 0:9],
                Jj[0:3, 6:15], Jj[3:9, 9:15]):
        np.testing.assert_allclose(blk, 0.0, **tol)                            # no dependence
