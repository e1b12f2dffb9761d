"""Pins of the keyframe-insertion oracle (oracle/keyframe.py)."""
import numpy as np
from scipy.spatial.transform import Rotation

import oracle
from oracle import keyframe as K
from paper_2512_02293_gb300 import synth


def _cam():
    R, e = synth.look_at([0.3, -0.2, 0.1], [1.0, 2.0, 3.5])
    return synth.Camera(50.0, 54.0, 20.0, 15.0, 40, 30, R, e)


def test_backprojected_mean_projects_to_the_pixel_centre():
    cam = _cam()
    rng = np.random.default_rng(0)
    depth = rng.uniform(1.0, 4.0, (cam.height, cam.width))
    color = rng.uniform(0, 1, (3, cam.height, cam.width))
    uv = np.stack([rng.integers(0, cam.width, 20), rng.integers(0, cam.height, 20)], 1)
    out = K.insert(color, depth, cam, uv, 2.5)
    g = synth.GaussianMap(out["mean"], out["quat"], out["log_scale"], out["logit"], out["color"])
    pr = oracle.project(g, cam, dict(oracle.DEFAULT_PARAMS))
    # the camera rotation is stored in float32, orthonormal to ~1e-7, so the round trip
    # through R and R^T carries ~1e-7 relative error (~2e-6 px here)
    np.testing.assert_allclose(pr["xy"], uv + 0.5, atol=1e-5)
    np.testing.assert_allclose(pr["depth"], depth[uv[:, 1], uv[:, 0]], rtol=1e-6)
    # isotropic footprint of one grid sample, identity rotation, opacity 0.5, pixel colour
    d = depth[uv[:, 1], uv[:, 0]]
    np.testing.assert_allclose(np.exp(out["log_scale"]), np.repeat((d * 2.5 / 52.0)[:, None], 3, 1), rtol=1e-12)
    assert np.all(out["quat"] == [1, 0, 0, 0]) and np.all(out["logit"] == 0)
    np.testing.assert_array_equal(out["color"], color[:, uv[:, 1], uv[:, 0]].T)


def test_sh_dc_coefficient_reproduces_the_pixel_colour():
    cam = _cam()
    color = np.full((3, cam.height, cam.width), 0.3); color[1] = 0.8
    depth = np.full((cam.height, cam.width), 2.0)
    out = K.insert(color, depth, cam, np.array([[5, 6]]), 2.0, sh_degree=3)
    rgb = oracle.sh_basis(np.array([0.0, 0.0, 1.0]))[0] * out["color"][0, :3] + 0.5
    np.testing.assert_allclose(rgb, [0.3, 0.8, 0.3], atol=1e-12)
    assert np.all(out["color"][0, 3:] == 0)


def test_learned_rotation_is_camera_rotation_times_predicted():
    cam = _cam()
    rng = np.random.default_rng(1)
    depth = np.full((cam.height, cam.width), 2.0)
    color = np.zeros((3, cam.height, cam.width))
    Y = rng.standard_normal((6, 8))
    uv = np.stack([np.arange(6), np.arange(6)], 1)
    out = K.insert(color, depth, cam, uv, 2.0, Y=Y)
    for k in range(6):
        qc = Y[k, 3:7] / np.linalg.norm(Y[k, 3:7])
        w, x, y, z = qc
        Rc = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                       [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                       [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        qw = out["quat"][k]
        Rw = Rotation.from_quat([qw[1], qw[2], qw[3], qw[0]]).as_matrix()
        np.testing.assert_allclose(Rw, np.asarray(cam.R_wc, np.float64) @ Rc, atol=1e-6)
        np.testing.assert_allclose(out["log_scale"][k], np.log(2.0 * 2.0 / 52.0) + Y[k, :3], rtol=1e-12)
        assert out["logit"][k] == Y[k, 7]


def test_patch_closed_forms():
    cam = _cam()
    H, W = cam.height, cam.width
    # constant colour, planar depth ramp along u: d = a + b u
    a, b = 2.0, 0.01
    depth = a + b * np.arange(W)[None, :].repeat(H, 0)
    color = np.empty((3, H, W)); color[0] = 0.25; color[1] = 0.5; color[2] = 0.75
    uv = np.array([[10, 12], [0, 0], [W - 1, H - 1]])
    X = K.extract_patches(color, depth, cam, uv, bf16=False)
    f = 52.0
    for k, (u, v) in enumerate(uv):
        dc = a + b * u
        for p in range(49):
            dx, dy = p % 7 - 3, p // 7 - 3
            assert tuple(X[k, 4 * p:4 * p + 3]) == (0.25, 0.5, 0.75)
            xu = min(max(u + dx, 0), W - 1)                   # clamped to the image
            want = np.log(dc) if p == 24 else (a + b * xu - dc) * f / (7 * dc)
            assert abs(X[k, 4 * p + 3] - want) < 1e-12
        assert X[k, 196] == 1.0 and np.all(X[k, 197:] == 0)
    # missing depth contributes 0
    depth2 = depth.copy(); depth2[12, 11] = 0.0
    X2 = K.extract_patches(color, depth2, cam, uv[:1], bf16=False)
    assert X2[0, 4 * 25 + 3] == 0.0
