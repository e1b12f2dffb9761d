"""Pins of the oracle's projection (EWA splatting of Sec. 3.3 "Preliminary")
against things other than itself: a closed form on the optical axis, scipy's
rotations, the Monte-Carlo covariance of the exact perspective map, rigid
motion invariance and brute-force tile rectangles."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2512_02293_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _single(mean, quat, log_scale, logit=0.0, color=(0.2, 0.4, 0.6)):
    f = lambda a: np.asarray(a, dtype=np.float32).reshape(1, -1)
    return synth.GaussianMap(f(mean), f(quat), f(log_scale), np.asarray([logit], np.float32), f(color))


def test_quaternion_matches_scipy():
    rng = np.random.default_rng(0)
    for _ in range(20):
        q = rng.standard_normal(4) * rng.uniform(0.2, 3.0)   # unnormalised, (w, x, y, z)
        R = oracle.quat_to_rot(q)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()   # scipy is scalar-last
        np.testing.assert_allclose(R, ref, atol=1e-12)


@pytest.mark.parametrize("dil", [0.0, 0.3])
def test_isotropic_on_axis_closed_form(dil):
    # A sphere of std s at depth z on the optical axis projects to a circle of
    # variance (f s / z)^2 + dilation centred on the principal point.
    cam = synth.identity_camera(64, 48, 60.0, 55.0, 32.0, 24.0)
    s, z = 0.05, 2.0
    g = _single([0, 0, z], [0.3, -0.5, 0.7, 0.1], [math.log(s)] * 3)
    pr = oracle.project(g, cam, dict(dilation=dil))
    a, b, c = pr["cov2"][0]
    assert a == pytest.approx((60.0 * s / z) ** 2 + dil, rel=1e-6)   # inputs are fp32
    assert c == pytest.approx((55.0 * s / z) ** 2 + dil, rel=1e-6)
    assert abs(b) < 1e-9
    np.testing.assert_allclose(pr["xy"][0], [32.0, 24.0], atol=1e-9)
    assert pr["depth"][0] == pytest.approx(z, rel=1e-7)
    np.testing.assert_allclose(pr["conic"][0], [1 / a, 0.0, 1 / c], rtol=1e-9, atol=1e-12)
    assert pr["opacity"][0] == pytest.approx(0.5)


def _mc_cov(mean, R_g, s, cam, n=400_000, seed=0):
    """Empirical mean/covariance of the exact pinhole projection of samples."""
    rng = np.random.default_rng(seed)
    X = mean + (rng.standard_normal((n, 3)) * s) @ R_g.T
    Rwc = cam.R_wc.astype(np.float64); t = cam.t_wc.astype(np.float64)
    Xc = (X - t) @ Rwc           # rows: R_wc^T (X - t)
    u = cam.fx * Xc[:, 0] / Xc[:, 2] + cam.cx
    v = cam.fy * Xc[:, 1] / Xc[:, 2] + cam.cy
    uv = np.stack([u, v], 1)
    return uv.mean(0), np.cov(uv.T)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_covariance_matches_monte_carlo_projection(seed):
    # EWA linearises the perspective map; for a small Gaussian the projected
    # sample covariance converges to J W Sigma W^T J^T.  Covariance built with
    # scipy, samples projected exactly.
    rng = np.random.default_rng(seed)
    R, eye = synth.look_at(rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3) + np.array([0, 0, 3.0]))
    cam = synth.Camera(400.0, 380.0, 160.0, 120.0, 320, 240, R, eye)
    fwd = R[:, 2].astype(np.float64)
    mean = eye + 2.5 * fwd + 0.4 * R[:, 0] - 0.3 * R[:, 1]
    q = rng.standard_normal(4); q /= np.linalg.norm(q)
    s = np.array([0.03, 0.012, 0.006])
    g = _single(mean, q, np.log(s))
    pr = oracle.project(g, cam, dict(dilation=0.0))
    Rg = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    s32 = np.exp(g.log_scale[0].astype(np.float64))
    m_emp, C_emp = _mc_cov(g.mean[0].astype(np.float64), Rg, s32, cam, seed=seed)
    a, b, c = pr["cov2"][0]
    C = np.array([[a, b], [b, c]])
    sd = np.sqrt(np.diag(C))
    # relative error in units of the projected std; MC noise ~ 2/sqrt(n)
    assert np.max(np.abs(C - C_emp) / np.outer(sd, sd)) < 0.02
    assert np.max(np.abs(pr["xy"][0] - m_emp) / sd) < 0.02


def test_rigid_motion_invariance():
    # Moving the camera and all Gaussians by the same rigid motion changes nothing.
    g, _, cam = synth.cfg1_problem(3)
    A = Rotation.from_rotvec([0.3, -0.7, 0.2]).as_matrix(); tA = np.array([0.5, -1.0, 2.0])
    qA = Rotation.from_matrix(A).as_quat()   # x, y, z, w
    qA = np.array([qA[3], qA[0], qA[1], qA[2]])
    def qmul(a, b):
        w1, x1, y1, z1 = a; w2, x2, y2, z2 = b.T
        return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                         w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], 1)
    g64 = g.astype(np.float64)
    g2 = synth.GaussianMap(g64.mean @ A.T + tA, qmul(qA, g64.quat), g64.log_scale, g64.opacity_logit, g64.color)
    cam2 = synth.Camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height, A @ cam.R_wc, A @ cam.t_wc + tA)
    p1 = oracle.project(g64, cam, {})
    p2 = oracle.project(g2, cam2, {})
    vis = p1["tiles"] > 0
    np.testing.assert_array_equal(vis, p2["tiles"] > 0)
    np.testing.assert_allclose(p1["xy"][vis], p2["xy"][vis], atol=1e-3)
    np.testing.assert_allclose(p1["conic"][vis], p2["conic"][vis], rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(p1["depth"][vis], p2["depth"][vis], rtol=1e-5)


def test_near_plane_cull():
    cam = synth.identity_camera()
    g = _single([0, 0, 0.15], [1, 0, 0, 0], [math.log(0.05)] * 3)
    pr = oracle.project(g, cam, dict(near=0.2))
    assert pr["tiles"][0] == 0 and pr["radius"][0] == 0
    pr = oracle.project(g, cam, dict(near=0.1))
    assert pr["tiles"][0] > 0


def test_radius_and_rect_brute_force():
    g, _, cam = synth.cfg1_problem(0)
    prm = dict(tile=16)
    pr = oracle.project(g, cam, prm)
    tx, ty = oracle.tiles_of(cam, prm)
    checked = 0
    for i in range(g.n):
        if pr["depth"][i] <= 0.2:
            continue
        a, b, c = pr["cov2"][i]
        mid = 0.5 * (a + c)
        disc = mid * mid - (a * c - b * b)
        lam = np.linalg.eigvalsh(np.array([[a, b], [b, c]])).max()
        if disc < 0.1:          # the discriminant floor of the radius rule
            lam = mid + math.sqrt(0.1)
        r = math.ceil(3 * math.sqrt(lam))
        mx, my = float(np.float32(pr["xy"][i, 0])), float(np.float32(pr["xy"][i, 1]))
        want = [(x, y) for y in range(ty) for x in range(tx)
                if x * 16 <= mx + r and (x + 1) * 16 > mx - r and y * 16 <= my + r and (y + 1) * 16 > my - r]
        if pr["tiles"][i] == 0:
            assert want == [], i
            continue
        assert pr["radius"][i] == r or pr["margin"][i] < 1e-6
        x0, y0, x1, y1 = pr["rect"][i]
        got = [(x, y) for y in range(y0, y1) for x in range(x0, x1)]
        assert sorted(got) == sorted(want), i
        assert pr["tiles"][i] == len(want)
        checked += 1
    assert checked > 100
