"""Pins of the oracle's hand-derived backward pass (compositing, projection,
pose tangent, SH colour) by central finite differences of the oracle's own
forward, and of the loss / regulariser / optimiser by library routines
(torch in float64) and closed forms."""
import math
from types import SimpleNamespace

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import oracle
from paper_2512_02293_gb300 import synth

NAMES = oracle.PARAM_NAMES


def cam64(width, height, fx, fy, cx, cy, R_wc, t_wc):
    return SimpleNamespace(fx=fx, fy=fy, cx=cx, cy=cy, width=width, height=height,
                           R_wc=np.asarray(R_wc, np.float64), t_wc=np.asarray(t_wc, np.float64))


def small_problem(seed, n=10, sh_degree=0):
    g = synth.random_cloud(n, seed, box=((-0.6, 0.6), (-0.4, 0.4), (1.5, 2.5)), log_scale_mu=-2.2,
                           log_scale_sd=0.3, sh_degree=sh_degree).astype(np.float64)
    R = Rotation.from_rotvec([0.05, -0.08, 0.03]).as_matrix()
    cam = cam64(24, 16, 20.0, 21.0, 12.3, 7.8, R, [0.05, -0.02, 0.1])
    return g, cam


def objective(g, cam, prm, w, u):
    img = oracle.render_fwd(oracle.project(g, cam, prm), cam, prm)
    return float(np.sum(w * img["color"]) + np.sum(u * img["depth"]))


def analytic(g, cam, prm, w, u):
    pr = oracle.project(g, cam, prm)
    g2d = oracle.render_bwd(pr, cam, prm, w, u)
    return oracle.project_bwd(g, cam, prm, g2d)


def _with(g, name, idx, delta):
    arrs = {k: a.copy() for k, a in zip(NAMES, g.arrays())}
    arrs[name][idx] += delta
    return synth.GaussianMap(*(arrs[k] for k in NAMES))


def _pose_perturb(cam, xi):
    """Left perturbation of world-to-camera: T_cw <- (R(phi) R_cw, R(phi) t_cw + rho)."""
    Rcw = cam.R_wc.T; tcw = -cam.R_wc.T @ cam.t_wc
    Rphi = Rotation.from_rotvec(xi[3:]).as_matrix()
    Rcw2 = Rphi @ Rcw; tcw2 = Rphi @ tcw + xi[:3]
    return cam64(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, Rcw2.T, -Rcw2.T @ tcw2)


def _fd_check(g, cam, prm, h, rtol, n_entries=None, sh_degree=0):
    rng = np.random.default_rng(7)
    w = rng.standard_normal((3, cam.height, cam.width))
    u = rng.standard_normal((cam.height, cam.width))
    an = analytic(g, cam, prm, w, u)
    num, ana = [], []
    for name, arr in zip(NAMES, g.arrays()):
        for idx in np.ndindex(arr.shape):
            if n_entries is not None and idx[0] >= n_entries:
                continue
            fp = objective(_with(g, name, idx, h), cam, prm, w, u)
            fm = objective(_with(g, name, idx, -h), cam, prm, w, u)
            num.append((fp - fm) / (2 * h)); ana.append(an[name][idx])
    for k in range(6):
        xi = np.zeros(6); xi[k] = h
        fp = objective(g, _pose_perturb(cam, xi), prm, w, u)
        fm = objective(g, _pose_perturb(cam, -xi), prm, w, u)
        num.append((fp - fm) / (2 * h)); ana.append(an["pose"][k])
    num = np.array(num); ana = np.array(ana)
    err = np.linalg.norm(num - ana) / np.linalg.norm(num)
    assert err < rtol, err
    # per-component check on the large ones catches a wrong term that the norm hides
    big = np.abs(num) > 1e-3 * np.abs(num).max()
    np.testing.assert_allclose(ana[big], num[big], rtol=50 * rtol, atol=1e-6 * np.abs(num).max())
    return err


@pytest.mark.parametrize("seed", [11, 12])
def test_fd_smooth_mode_all_parameters_and_pose(seed):
    g, cam = small_problem(seed)
    _fd_check(g, cam, dict(smooth=True, tile=8, dilation=0.3), h=1e-6, rtol=1e-6)


def test_fd_method_mode_away_from_thresholds():
    # With every threshold decision far from its threshold the method-mode image
    # is smooth in a neighbourhood and the hand gradient must match FD there.
    g, cam = small_problem(21)
    prm = dict(tile=8, T_cut=1e-4, alpha_min=1 / 255, alpha_max=0.99)
    pr = oracle.project(g, cam, prm)
    img = oracle.render_fwd(pr, cam, prm)
    assert img["margin"].min() > 1e-5 and pr["margin"][pr["tiles"] > 0].min() > 1e-5
    _fd_check(g, cam, prm, h=1e-8, rtol=1e-4)


def test_fd_sh3_colour():
    g, cam = small_problem(31, n=6, sh_degree=3)
    _fd_check(g, cam, dict(smooth=True, tile=8, sh_degree=3), h=1e-6, rtol=1e-6)


def test_sh_basis_orthonormal():
    # Gauss-Legendre in cos(theta) x uniform phi integrates degree <= 6
    # polynomials on the sphere exactly.
    x, wx = np.polynomial.legendre.leggauss(8)
    phis = np.arange(16) * 2 * math.pi / 16
    G = np.zeros((16, 16))
    for ct, wt in zip(x, wx):
        st = math.sqrt(1 - ct * ct)
        for ph in phis:
            Y = oracle.sh_basis([st * math.cos(ph), st * math.sin(ph), ct])
            G += wt * (2 * math.pi / 16) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh3_degree0_band_reproduces_rgb():
    rng = np.random.default_rng(3)
    rgb = rng.random((5, 3))
    sh = synth.sh3_from_rgb(rgb, rng, sigma=0.0)
    g = synth.GaussianMap(rng.random((5, 3)) + [0, 0, 2], rng.standard_normal((5, 4)), np.full((5, 3), -3.0),
                          np.zeros(5), sh)
    cam = synth.identity_camera()
    pr = oracle.project(g, cam, dict(sh_degree=3))
    np.testing.assert_allclose(pr["rgb"], rgb, atol=1e-12)


# --------------------------------------------------------------------- losses

def test_l1_loss_matches_torch():
    rng = np.random.default_rng(0)
    H, W = 12, 9
    c = rng.random((3, H, W)); tc = rng.random((3, H, W)); tc[0, :3] = c[0, :3]   # some exact zeros
    d = rng.random((H, W)) * 4; td = rng.random((H, W)) * 4; td[rng.random((H, W)) < 0.3] = 0.0
    lc, ld = 0.9, 0.1
    terms, dc, dd = oracle.l1_loss(c, d, tc, td, lc, ld)
    C = torch.tensor(c, requires_grad=True); D = torch.tensor(d, requires_grad=True)
    valid = torch.tensor(td > 0)
    Lc = torch.nn.functional.l1_loss(C, torch.tensor(tc))
    Ld = torch.nn.functional.l1_loss(D[valid], torch.tensor(td)[valid])
    (lc * Lc + ld * Ld).backward()
    assert terms[0] == pytest.approx(Lc.item(), rel=1e-14)
    assert terms[1] == pytest.approx(Ld.item(), rel=1e-14)
    np.testing.assert_allclose(dc, C.grad.numpy(), atol=1e-16)
    np.testing.assert_allclose(dd, D.grad.numpy(), atol=1e-16)


def test_iso_loss_special_cases_and_fd():
    # isotropic scales: zero loss and zero gradient
    L, g = oracle.iso_loss(np.full((4, 3), -2.0), 10.0)
    assert L == 0.0 and np.all(g == 0)
    # one Gaussian with scales (1, 1, e): mean = (2 + e)/3, |1 - m|*2 + |e - m| = 4(e - 1)/3
    L, g = oracle.iso_loss(np.array([[0.0, 0.0, 1.0]]), 1.0)
    assert L == pytest.approx(4 * (math.e - 1) / 3)
    rng = np.random.default_rng(1)
    ls = rng.normal(-3, 0.5, (7, 3))
    L, g = oracle.iso_loss(ls, 2.5)
    h = 1e-7
    for idx in np.ndindex(ls.shape):
        a = ls.copy(); a[idx] += h; b = ls.copy(); b[idx] -= h
        fd = 2.5 * (oracle.iso_loss(a, 0)[0] - oracle.iso_loss(b, 0)[0]) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_adam_matches_torch():
    rng = np.random.default_rng(2)
    p0 = rng.standard_normal(50)
    p = p0.copy(); m = np.zeros(50); v = np.zeros(50)
    tp = torch.tensor(p0.copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-15)
    for step in range(1, 6):
        gr = rng.standard_normal(50)
        oracle.adam(p, gr, m, v, 1e-2, 0.9, 0.999, 1e-15, step)
        tp.grad = torch.tensor(gr)
        opt.step()
        np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_fd_sh3_room_subset_160x128():
    """The differentiation workload's own check: 4k Gaussians sub-sampled from
    the 1M-Gaussian degree-3 SH room, one of its keyframes scaled to 160x128,
    smooth mode, central differences with h = 1e-4.

    On a dense surface many Gaussians lie at nearly the same depth, and a step
    that swaps two of them in the depth order changes the blend by a jump: the
    rendered image is only piecewise smooth in anything that moves depths, and
    its gradient is the derivative at fixed order.  The h = 1e-4 directions
    therefore keep every Gaussian's camera depth: lateral moves of the means,
    all other parameters, the pose translations (all depths shift alike) and
    the rotation about the optical axis.  (The two tilts reorder depths; they
    are covered by the small-scene differences above and the rigid-motion
    invariant of the projection tests.)"""
    g_full, _, cams = synth.cfg4_problem()
    c = cams[5]
    cam = cam64(160, 128, c.fx / 8, c.fy / 8, c.cx / 8, c.cy / 8, c.R_wc, c.t_wc)
    prm = dict(smooth=True, tile=16, sh_degree=3)
    vis = np.nonzero(oracle.project(g_full, cam, dict(tile=16, sh_degree=3))["tiles"] > 0)[0]
    rng = np.random.default_rng(3)
    idx = np.sort(rng.choice(vis, 4000, replace=False))
    g = g_full.subset(idx).astype(np.float64)
    w = rng.standard_normal((3, cam.height, cam.width))
    u = rng.standard_normal((cam.height, cam.width))
    an = analytic(g, cam, prm, w, u)
    R_wc = np.asarray(cam.R_wc, np.float64)

    def along(d, dpose, h):
        gp = synth.GaussianMap(*(a + h * d[k] for k, a in zip(NAMES, g.arrays())))
        gm = synth.GaussianMap(*(a - h * d[k] for k, a in zip(NAMES, g.arrays())))
        fp = objective(gp, _pose_perturb(cam, h * dpose), prm, w, u)
        fm = objective(gm, _pose_perturb(cam, -h * dpose), prm, w, u)
        fd = (fp - fm) / (2 * h)
        dd = sum(float(np.sum(an[k] * d[k])) for k in NAMES) + float(np.dot(an["pose"], dpose))
        return fd, dd

    zero = {k: np.zeros_like(a) for k, a in zip(NAMES, g.arrays())}
    d = {k: rng.standard_normal(a.shape) for k, a in zip(NAMES, g.arrays())}
    lat = rng.standard_normal((g.n, 3)) * 0.1
    lat[:, 2] = 0.0
    d["mean"] = lat @ R_wc.T                                      # camera-frame lateral moves
    pose = np.zeros(6); pose[[0, 1, 2, 5]] = rng.standard_normal(4) * 0.01     # rho and phi_z
    sh = dict(zero); sh["color"] = rng.standard_normal(g.color.shape); sh["color"][:, 0] = 0.0
    dirs = [(d, pose, 1e-4),                                      # everything at once
            (sh, np.zeros(6), 1e-4),                              # higher SH orders only
            (zero, pose, 1e-4)]                                   # the pose alone
    for d, dp, h in dirs:
        fd, dd = along(d, dp, h)
        # central differences carry O(h^2) truncation: ~1e-5 relative at h = 1e-4
        tol = 1e-4 if h >= 1e-4 else 1e-5
        assert abs(fd - dd) < tol * max(1.0, abs(fd)), (fd, dd, h)
