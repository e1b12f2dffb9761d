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
