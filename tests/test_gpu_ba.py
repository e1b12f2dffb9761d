"""Dense visual bundle adjustment on the GPU (gs_ba_step: Eq. 2 residuals, Eq. 4
Schur complement of the inverse-depth block) against the FP64 oracle's full
dense solve."""
import numpy as np
import pytest
import torch

from oracle import ba
from paper_2512_02293_gb300 import gs as G
from paper_2512_02293_gb300 import synth
from gpu_common import ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def _exact_targets(R, t, disp, intr, edges):
    h, w = disp.shape[1:]
    return -ba.residuals(R, t, disp, intr, edges, np.zeros((len(edges), h, w, 2)))


def _gpu_state(win):
    P = win.poses.cpu().numpy().astype(np.float64)
    return P[:, :9].reshape(-1, 3, 3), P[:, 9:], win.disp.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n_fixed", [1, 2])
def test_one_step_matches_dense_solve(n_fixed):
    R, t, disp, intr, edges, wts = synth.ba_scene(7, K=5, h=12, w=16)
    rng = np.random.default_rng(8)
    targets = _exact_targets(R, t, disp, intr, edges) + rng.normal(0, 0.3, (len(edges), 12, 16, 2))
    win = G.BAWindow(R, t, disp, intr, edges, targets, wts, n_fixed)
    lam, eps = 1e-3, 1e-3
    G.gs_ba_step(win, lam, eps)
    torch.cuda.synchronize()
    assert int(win.status[0].item()) == 0
    # the oracle on the same float32 inputs
    R32, t32, d32, T32, W32 = _f32(R), _f32(t), _f32(disp), _f32(targets), _f32(wts)
    intr32 = tuple(float(np.float32(x)) for x in intr)
    dx, dd, H, g, cost = ba.lm_step(R32, t32, d32, intr32, edges, T32, W32, n_fixed, lam=lam, eps=eps)
    Rr, tr, dr = ba.apply_step(R32, t32, d32, dx, dd, n_fixed)
    assert win.cost.item() == pytest.approx(cost, rel=1e-4)
    Rg, tg, dg = _gpu_state(win)
    step_d = np.abs(dd).max()
    np.testing.assert_allclose(dg, dr, atol=2e-3 * step_d + 1e-6)
    step_x = np.abs(dx).max()
    np.testing.assert_allclose(tg, tr, atol=2e-3 * step_x + 1e-6)
    np.testing.assert_allclose(Rg, Rr, atol=2e-3 * step_x + 1e-6)
    # the fixed poses did not move
    np.testing.assert_array_equal(win.poses.cpu().numpy()[:n_fixed], np.concatenate(
        [np.asarray(R, np.float32).reshape(-1, 9), np.asarray(t, np.float32)], 1)[:n_fixed])


def test_gauss_newton_recovers_the_window():
    R, t, disp, intr, edges, wts = synth.ba_scene(9, K=6, h=24, w=32)
    targets = _exact_targets(R, t, disp, intr, edges)
    rng = np.random.default_rng(10)
    n_fixed = 2
    R1, t1, d1 = ba.apply_step(R, t, disp, rng.normal(0, 0.01, (4, 6)), rng.normal(0, 0.01, disp.shape), n_fixed)
    win = G.BAWindow(R1, t1, d1, intr, edges, targets, wts, n_fixed)
    costs = []
    for _ in range(10):
        G.gs_ba_step(win, 1e-5, 1e-6)
        costs.append(win.cost.item())
    torch.cuda.synchronize()
    assert int(win.status[0].item()) == 0
    assert costs[-1] < 1e-6 * costs[0]
    Rg, tg, dg = _gpu_state(win)
    np.testing.assert_allclose(dg, disp, atol=2e-5)
    np.testing.assert_allclose(tg, t, atol=2e-5)
    np.testing.assert_allclose(Rg, R, atol=2e-5)


def test_bad_edge_is_reported():
    R, t, disp, intr, edges, wts = synth.ba_scene(11, K=3, h=4, w=4)
    targets = _exact_targets(R, t, disp, intr, edges)
    bad = list(edges) + [(1, 7)]
    win = G.BAWindow(R, t, disp, intr, bad, np.concatenate([targets, targets[:1]]),
                     np.concatenate([wts, wts[:1]]), 1)
    G.gs_ba_step(win)
    assert G.gs_read_device_status(win.status) == G.GS_ERR_INVALID_ARG


def test_too_many_edges_out_of_one_keyframe_is_reported():
    # 16 edges leave keyframe 0: above the 15 the Schur kernel stages per pixel
    R, t, disp, intr, _, _ = synth.ba_scene(12, K=17, h=4, w=4)
    edges = [(0, j) for j in range(1, 17)] + [(1, 0)]
    targets = _exact_targets(R, t, disp, intr, edges)
    wts = np.ones((len(edges), 4, 4, 2))
    win = G.BAWindow(R, t, disp, intr, edges, targets, wts, 1)
    G.gs_ba_step(win)
    assert G.gs_read_device_status(win.status) == G.GS_ERR_UNSUPPORTED
    # 15 edges out of keyframe 0 are within the limit
    edges = [(0, j) for j in range(1, 16)] + [(1, 0)]
    targets = _exact_targets(R, t, disp, intr, edges)
    win = G.BAWindow(R, t, disp, intr, edges, targets, np.ones((len(edges), 4, 4, 2)), 1)
    G.gs_ba_step(win)
    assert G.gs_read_device_status(win.status) == G.GS_OK


def test_largest_system_31_free_poses():
    # 32 keyframes with the first fixed: the reduced system is 186 x 186 (the
    # limit), solved in 139 KB of shared memory with 6 columns per lane
    R, t, disp, intr, edges, wts = synth.ba_scene(13, K=32, h=4, w=4, window=3)
    rng = np.random.default_rng(14)
    targets = _exact_targets(R, t, disp, intr, edges) + rng.normal(0, 0.3, (len(edges), 4, 4, 2))
    win = G.BAWindow(R, t, disp, intr, edges, targets, wts, 1)
    lam, eps = 1e-3, 1e-3
    G.gs_ba_step(win, lam, eps)
    torch.cuda.synchronize()
    assert int(win.status[0].item()) == 0
    R32, t32, d32, T32, W32 = _f32(R), _f32(t), _f32(disp), _f32(targets), _f32(wts)
    intr32 = tuple(float(np.float32(x)) for x in intr)
    dx, dd, H, g, cost = ba.lm_step(R32, t32, d32, intr32, edges, T32, W32, 1, lam=lam, eps=eps)
    Rr, tr, dr = ba.apply_step(R32, t32, d32, dx, dd, 1)
    assert win.cost.item() == pytest.approx(cost, rel=1e-4)
    Rg, tg, dg = _gpu_state(win)
    np.testing.assert_allclose(dg, dr, atol=2e-3 * np.abs(dd).max() + 1e-6)
    np.testing.assert_allclose(tg, tr, atol=2e-3 * np.abs(dx).max() + 1e-6)
    np.testing.assert_allclose(Rg, Rr, atol=2e-3 * np.abs(dx).max() + 1e-6)
    # one more free pose is refused on the host
    win33 = G.BAWindow(*synth.ba_scene(13, K=33, h=4, w=4, window=3)[:3], intr,
                       [(i, j) for i in range(33) for j in range(33) if i != j and abs(i - j) <= 1],
                       np.zeros((2 * 32, 4, 4, 2)), np.ones((2 * 32, 4, 4, 2)), 1)
    with pytest.raises(G.GsError):
        G.gs_ba_step(win33)


# ---------------------------------------------- visual-inertial (Eq. 2 + Eq. 3)

def _vi_window(seed, K, h, w, n_fixed, noise=0.3, dv=0.05, db=0.004, window=2):
    """A perturbed visual-inertial window and the float32 copy of its inputs the
    oracle sees."""
    R, t, disp, intr, edges, wts, vel, bias, bh, g, imu = synth.vi_scene(seed, K=K, h=h, w=w, window=window)
    rng = np.random.default_rng(seed + 1)
    targets = _exact_targets(R, t, disp, intr, edges) + rng.normal(0, noise, (len(edges), h, w, 2))
    vel = vel + rng.normal(0, dv, vel.shape)
    bias = bias + rng.normal(0, db, bias.shape)
    win = G.BAWindow(R, t, disp, intr, edges, targets, wts, n_fixed, imu=imu, vel=vel, bias=bias, bias_hat=bh,
                     gravity=g)
    f32 = dict(R=_f32(R), t=_f32(t), disp=_f32(disp), vel=_f32(vel), bias=_f32(bias), bias_hat=_f32(bh),
               intr=tuple(float(np.float32(x)) for x in intr), edges=edges, targets=_f32(targets),
               weights=_f32(wts), imu=_f32(imu), gravity=_f32(g))
    return win, f32


def _check_vi_step(win, o, n_fixed, lam, eps, rtol=2e-3):
    dx, dd, cost = ba.lm_step_vi(o["R"], o["t"], o["disp"], o["vel"], o["bias"], o["bias_hat"], o["intr"],
                                 o["edges"], o["targets"], o["weights"], o["imu"], o["gravity"], n_fixed,
                                 lam=lam, eps=eps)
    Rr, tr, dr, vr, br = ba.apply_step_vi(o["R"], o["t"], o["disp"], o["vel"], o["bias"], dx, dd, n_fixed)
    assert win.cost.item() == pytest.approx(cost, rel=1e-4)
    Rg, tg, dg = _gpu_state(win)
    sx, sd = np.abs(dx).max(), np.abs(dd).max()
    np.testing.assert_allclose(dg, dr, atol=rtol * sd + 1e-6)
    np.testing.assert_allclose(tg, tr, atol=rtol * sx + 1e-6)
    np.testing.assert_allclose(Rg, Rr, atol=rtol * sx + 1e-6)
    np.testing.assert_allclose(win.vel.cpu().numpy(), vr, atol=rtol * sx + 1e-6)
    np.testing.assert_allclose(win.bias.cpu().numpy(), br, atol=rtol * sx + 1e-6)
    # the fixed keyframes' velocities and biases did not move
    np.testing.assert_array_equal(win.vel.cpu().numpy()[:n_fixed], np.float32(o["vel"][:n_fixed]))
    np.testing.assert_array_equal(win.bias.cpu().numpy()[:n_fixed], np.float32(o["bias"][:n_fixed]))


@pytest.mark.parametrize("n_fixed", [1, 2])
def test_vi_one_step_matches_dense_solve(n_fixed):
    win, o = _vi_window(21, K=5, h=12, w=16, n_fixed=n_fixed)
    lam, eps = 1e-3, 1e-3
    G.gs_ba_step(win, lam, eps)
    torch.cuda.synchronize()
    assert int(win.status[0].item()) == 0
    _check_vi_step(win, o, n_fixed, lam, eps)


def test_vi_inertial_factor_alone():
    # no edges: only Eq. 3 constrains the free keyframes; the inverse depths keep their values
    win, o = _vi_window(22, K=4, h=4, w=4, n_fixed=1)
    win2 = G.BAWindow(o["R"], o["t"], o["disp"], o["intr"], [], np.zeros((0, 4, 4, 2)), np.zeros((0, 4, 4, 2)), 1,
                      imu=o["imu"], vel=o["vel"], bias=o["bias"], bias_hat=o["bias_hat"], gravity=o["gravity"])
    G.gs_ba_step(win2, 1e-3, 1e-3)
    torch.cuda.synchronize()
    assert int(win2.status[0].item()) == 0
    o = dict(o, edges=[], targets=np.zeros((0, 4, 4, 2)), weights=np.zeros((0, 4, 4, 2)))
    _check_vi_step(win2, o, 1, 1e-3, 1e-3)
    np.testing.assert_array_equal(win2.disp.cpu().numpy(), np.float32(o["disp"]))


def test_vi_gauss_newton_recovers_the_window():
    R, t, disp, intr, edges, wts, vel, bias, bh, g, imu = synth.vi_scene(23, K=6, h=24, w=32)
    targets = _exact_targets(R, t, disp, intr, edges)
    rng = np.random.default_rng(24)
    n_fixed = 1
    dx = np.concatenate([rng.normal(0, 0.01, (5, 6)), rng.normal(0, 0.02, (5, 3)), rng.normal(0, 0.002, (5, 6))], 1)
    R1, t1, d1, v1, b1 = ba.apply_step_vi(R, t, disp, vel, bias, dx, rng.normal(0, 0.01, disp.shape), n_fixed)
    win = G.BAWindow(R1, t1, d1, intr, edges, targets, wts, n_fixed, imu=imu, vel=v1, bias=b1, bias_hat=bh,
                     gravity=g)
    costs = []
    for _ in range(12):
        G.gs_ba_step(win, 1e-5, 1e-6)
        costs.append(win.cost.item())
    torch.cuda.synchronize()
    assert int(win.status[0].item()) == 0
    assert costs[-1] < 1e-5 * costs[0]
    Rg, tg, dg = _gpu_state(win)
    np.testing.assert_allclose(dg, disp, atol=5e-5)
    np.testing.assert_allclose(tg, t, atol=5e-5)
    np.testing.assert_allclose(Rg, R, atol=5e-5)
    np.testing.assert_allclose(win.vel.cpu().numpy(), vel, atol=2e-4)
    np.testing.assert_allclose(win.bias.cpu().numpy(), bias, atol=2e-4)


def test_vi_largest_system_15_free_keyframes():
    # 16 keyframes with the first fixed: 225 unknowns, padded to 228 in the solve
    win, o = _vi_window(25, K=16, h=4, w=4, n_fixed=1, window=3)
    lam, eps = 1e-3, 1e-3
    G.gs_ba_step(win, lam, eps)
    torch.cuda.synchronize()
    assert int(win.status[0].item()) == 0
    _check_vi_step(win, o, 1, lam, eps)
    # one more free keyframe is refused on the host
    win17, _ = _vi_window(25, K=17, h=4, w=4, n_fixed=1, window=3)
    with pytest.raises(G.GsError):
        G.gs_ba_step(win17)
    # as are inertial records without velocities
    with pytest.raises(ValueError):
        G.BAWindow(o["R"], o["t"], o["disp"], o["intr"], o["edges"], o["targets"], o["weights"], 1, imu=o["imu"])


def test_vi_convergence_at_the_benchmark_size():
    # the benchmark's window (16 keyframes at 60 x 80, edges up to 3 apart, one
    # keyframe fixed, the inertial factor between consecutive keyframes): from a
    # perturbed state of an exactly consistent window, damped Gauss-Newton steps
    # drive the joint cost down by more than four orders of magnitude (the state
    # itself settles within ~1e-3 of the generating one along a weakly observable
    # direction, so it is not compared here; the small windows above compare it)
    R, t, disp, intr, edges, wts, vel, bias, bh, g, imu = synth.vi_scene(31, K=16, h=60, w=80, f=70.0, window=3)
    targets = _exact_targets(R, t, disp, intr, edges)
    rng = np.random.default_rng(32)
    dx = np.concatenate([rng.normal(0, 0.005, (15, 6)), rng.normal(0, 0.01, (15, 3)),
                         rng.normal(0, 0.001, (15, 6))], 1)
    R1, t1, d1, v1, b1 = ba.apply_step_vi(R, t, disp, vel, bias, dx, rng.normal(0, 0.005, disp.shape), 1)
    win = G.BAWindow(R1, t1, d1, intr, edges, targets, wts, 1, imu=imu, vel=v1, bias=b1, bias_hat=bh, gravity=g)
    costs = []
    for _ in range(15):
        G.gs_ba_step(win, 1e-5, 1e-6)
        costs.append(win.cost.item())
    torch.cuda.synchronize()
    assert int(win.status[0].item()) == 0
    assert costs[-1] < 1e-4 * costs[0]
