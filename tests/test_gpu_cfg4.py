"""The differentiation workload at full size, through the autograd binding:
16 keyframes at 1280x1024 over 1M Gaussians with degree-3 SH colour (48
coefficients), gradients to every parameter and every keyframe's 6-DoF pose
tangent, from the per-pixel (T_final, n_contrib) checkpoint.

- colour / depth / T_final, and n_contrib bit-exact, on tile-aligned windows of
  two views against the FP64 oracle;
- every parameter gradient (incl. all SH coefficients) and the pose gradient of
  a loss that lives in one view's window; the 15 other poses get exactly 0;
- on the 4k-Gaussian, 160x128 sub-sample the oracle's differences pin
  (tests/test_oracle_grads.py), the GPU gradient against the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_02293_gb300 import gs as G
from paper_2512_02293_gb300 import synth
from paper_2512_02293_gb300.autograd import Rasterizer, render
from gpu_common import (COLOR_TOL, GRAD_RTOL, ensure_lib, excused_pixels, f32, margin_excuse, prm_dict, rel_l2)

pytestmark = pytest.mark.gpu


def _leaf(g):
    return [torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda().requires_grad_(True) for a in g.arrays()]


@pytest.fixture(scope="module")
def full():
    ensure_lib()
    g, _, cams = synth.cfg4_problem()
    params = G.RenderParams(sh_degree=3, tile=16)
    rast = Rasterizer(cams, g.n, params)
    leaves = _leaf(g)
    xi = torch.zeros(len(cams), 6, device="cuda", requires_grad=True)
    col, dep = render(*leaves, xi, rast)
    torch.cuda.synchronize()
    return g, cams, params, rast, leaves, xi, col, dep


def _crop(cam, x0, y0, w, h):
    return synth.Camera(cam.fx, cam.fy, cam.cx - x0, cam.cy - y0, w, h, cam.R_wc, cam.t_wc)


def _view(cams, v, flat, channels):
    base = sum(c.n_pixels for c in cams[:v])
    W, H = cams[v].width, cams[v].height
    return flat[channels * base:channels * (base + W * H)].view(channels, H, W) if channels > 1 else \
        flat[base:base + W * H].view(H, W)


@pytest.mark.parametrize("v,win", [(3, (640, 512, 64, 64)), (12, (96, 928, 64, 64))])
def test_forward_windows(full, v, win):
    g, cams, params, rast, leaves, xi, col, dep = full
    x0, y0, w, h = win
    crop = _crop(cams[v], x0, y0, w, h)
    prm = prm_dict(params)
    pr = oracle.project(g, crop, prm)
    img = oracle.render_fwd(pr, crop, prm)
    n = g.n
    ex, _ = excused_pixels(win, rast.proj.rect[v * n:(v + 1) * n].cpu().numpy(), pr["rect"], img["margin"], 16,
                           margin_excuse(cams[v]))
    ok = ~ex
    assert ok.mean() > 0.95
    c = _view(cams, v, col.detach(), 3).cpu().numpy()[:, y0:y0 + h, x0:x0 + w]
    d = _view(cams, v, dep.detach(), 1).cpu().numpy()[y0:y0 + h, x0:x0 + w]
    Tf = _view(cams, v, rast.img.T_final, 1).cpu().numpy()[y0:y0 + h, x0:x0 + w]
    nc = _view(cams, v, rast.img.n_contrib, 1).cpu().numpy().view(np.uint32)[y0:y0 + h, x0:x0 + w]
    np.testing.assert_allclose(c[:, ok], img["color"][:, ok], atol=COLOR_TOL)
    np.testing.assert_allclose(d[ok], img["depth"][ok], atol=COLOR_TOL)
    np.testing.assert_allclose(Tf[ok], img["T_final"][ok], atol=1e-5)
    np.testing.assert_array_equal(nc[ok], img["n_contrib"][ok])


def test_backward_window_all_parameters_and_poses(full):
    g, cams, params, rast, leaves, xi, col, dep = full
    v, (x0, y0, w, h) = 3, (640, 512, 64, 64)
    crop = _crop(cams[v], x0, y0, w, h)
    prm = prm_dict(params)
    pr = oracle.project(g, crop, prm)
    img = oracle.render_fwd(pr, crop, prm)
    n = g.n
    ex, _ = excused_pixels((x0, y0, w, h), rast.proj.rect[v * n:(v + 1) * n].cpu().numpy(), pr["rect"],
                           img["margin"], 16, margin_excuse(cams[v]))
    ok = ~ex
    rng = np.random.default_rng(4)
    wc = f32(rng.standard_normal((3, h, w)) * ok[None])
    ud = f32(rng.standard_normal((h, w)) * ok)
    Wc = torch.zeros_like(col); Ud = torch.zeros_like(dep)
    _view(cams, v, Wc, 3)[:, y0:y0 + h, x0:x0 + w] = torch.from_numpy(wc.astype(np.float32)).cuda()
    _view(cams, v, Ud, 1)[y0:y0 + h, x0:x0 + w] = torch.from_numpy(ud.astype(np.float32)).cuda()
    for t in leaves:
        t.grad = None
    xi.grad = None
    ((Wc * col).sum() + (Ud * dep).sum()).backward(retain_graph=True)
    ref = oracle.project_bwd(g, crop, prm, oracle.render_bwd(pr, crop, prm, wc, ud))
    for k, leaf in zip(oracle.PARAM_NAMES, leaves):
        assert rel_l2(leaf.grad.cpu().numpy(), ref[k]) < GRAD_RTOL, k
    # the higher SH orders on their own (not swamped by the DC band)
    assert rel_l2(leaves[4].grad[:, 1:].cpu().numpy(), ref["color"][:, 1:]) < GRAD_RTOL
    pg = xi.grad.cpu().numpy()
    assert rel_l2(pg[v], ref["pose"]) < GRAD_RTOL
    assert np.all(np.delete(pg, v, axis=0) == 0.0)


def test_subset_160x128_gradients_match_oracle():
    ensure_lib()
    g_full, _, cams = synth.cfg4_problem()
    c = cams[5]
    cam = synth.Camera(c.fx / 8, c.fy / 8, c.cx / 8, c.cy / 8, 160, 128, c.R_wc, c.t_wc)
    prm = dict(tile=16, sh_degree=3)
    vis = np.nonzero(oracle.project(g_full, cam, prm)["tiles"] > 0)[0]
    idx = np.sort(np.random.default_rng(3).choice(vis, 4000, replace=False))
    g = g_full.subset(idx)
    params = G.RenderParams(sh_degree=3, tile=16)
    rast = Rasterizer([cam], g.n, params)
    leaves = _leaf(g)
    xi = torch.zeros(1, 6, device="cuda", requires_grad=True)
    col, dep = render(*leaves, xi, rast)
    pr = oracle.project(g, cam, prm)
    img = oracle.render_fwd(pr, cam, prm)
    ok = img["margin"] >= margin_excuse(cam)
    rng = np.random.default_rng(5)
    wc = f32(rng.standard_normal((3, 128, 160)) * ok[None])
    ud = f32(rng.standard_normal((128, 160)) * ok)
    ((torch.from_numpy(wc.reshape(-1).astype(np.float32)).cuda() * col).sum() +
     (torch.from_numpy(ud.reshape(-1).astype(np.float32)).cuda() * dep).sum()).backward()
    ref = oracle.project_bwd(g, cam, prm, oracle.render_bwd(pr, cam, prm, wc, ud))
    for k, leaf in zip(oracle.PARAM_NAMES, leaves):
        assert rel_l2(leaf.grad.cpu().numpy(), ref[k]) < GRAD_RTOL, k
    assert rel_l2(xi.grad[0].cpu().numpy(), ref["pose"]) < GRAD_RTOL
