"""The batched mapping window at full size: 8 keyframes of uneven size
(4x 640x480, 2x 752x480, 2x 1280x1024) over a 500k-Gaussian room, every stage
one launch over all views, tile 16 (the shapes bench.py's window line times).

- each view of the batched render equals the same view rendered alone,
  bit for bit (identical per-tile lists and arithmetic);
- colour / depth / T_final, and n_contrib bit-exact, on tile-aligned windows of
  two views against the FP64 oracle;
- every parameter gradient and all eight pose gradients for a loss whose image
  gradient lives in a window of one view (the other poses get exactly zero), for
  one view of each of the three resolutions.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_02293_gb300 import gs as G
from paper_2512_02293_gb300 import synth
from paper_2512_02293_gb300.mapping import MapParams, MappingStep
from gpu_common import (COLOR_TOL, GRAD_RTOL, ensure_lib, excused_pixels, f32, grads_to_numpy, margin_excuse,
                        prm_dict, rel_l2)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def window():
    ensure_lib()
    g, gt, cams = synth.cfg3_problem()
    params = G.RenderParams(tile=16)
    P = G.gs_total_pixels(cams)
    step = MappingStep(G.Gaussians.from_numpy(g), cams, torch.zeros(3 * P, device="cuda"),
                       torch.zeros(P, device="cuda"), params, MapParams(1.0, 1.0, 0.0))
    step.render()
    torch.cuda.synchronize()
    assert step.check() == 0
    return g, cams, params, step


def _crop(cam, x0, y0, w, h):
    return synth.Camera(cam.fx, cam.fy, cam.cx - x0, cam.cy - y0, w, h, cam.R_wc, cam.t_wc)


def test_batched_view_equals_single_view(window):
    g, cams, params, step = window
    for v in (4, 6):
        P = cams[v].n_pixels
        one = MappingStep(step.g, [cams[v]], torch.zeros(3 * P, device="cuda"), torch.zeros(P, device="cuda"),
                          params, MapParams())
        one.render()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(one.color_image(0).cpu().numpy(), step.color_image(v).cpu().numpy())
        np.testing.assert_array_equal(one.depth_image(0).cpu().numpy(), step.depth_image(v).cpu().numpy())


@pytest.mark.parametrize("v,win", [(0, (320, 224, 64, 64)), (6, (608, 480, 64, 64)), (6, (1216, 960, 64, 64))])
def test_window_views_forward(window, v, win):
    g, cams, params, step = window
    x0, y0, w, h = win
    crop = _crop(cams[v], x0, y0, w, h)
    prm = prm_dict(params)
    pr = oracle.project(g, crop, prm)
    img = oracle.render_fwd(pr, crop, prm)
    n = g.n
    ex, _ = excused_pixels(win, step.proj.rect[v * n:(v + 1) * n].cpu().numpy(), pr["rect"], img["margin"], 16,
                           margin_excuse(cams[v]))
    ok = ~ex
    col = step.color_image(v).cpu().numpy()[:, y0:y0 + h, x0:x0 + w]
    dep = step.depth_image(v).cpu().numpy()[y0:y0 + h, x0:x0 + w]
    base = sum(c.n_pixels for c in cams[:v])
    W, H = cams[v].width, cams[v].height
    Tf = step.img.T_final[base:base + W * H].cpu().numpy().reshape(H, W)[y0:y0 + h, x0:x0 + w]
    nc = step.img.n_contrib[base:base + W * H].cpu().numpy().view(np.uint32).reshape(H, W)[y0:y0 + h, x0:x0 + w]
    assert ok.mean() > 0.95
    np.testing.assert_allclose(col[:, ok], img["color"][:, ok], atol=COLOR_TOL)
    np.testing.assert_allclose(dep[ok], img["depth"][ok], atol=COLOR_TOL)
    np.testing.assert_allclose(Tf[ok], img["T_final"][ok], atol=1e-5)
    np.testing.assert_array_equal(nc[ok], img["n_contrib"][ok])


@pytest.mark.parametrize("v,win", [(0, (320, 224, 64, 64)), (4, (352, 224, 64, 64)), (6, (608, 480, 64, 64))])
def test_window_backward_one_view(window, v, win):
    """One view of each resolution (640x480, 752x480, 1280x1024)."""
    g, cams, params, step = window
    x0, y0, w, h = win
    crop = _crop(cams[v], x0, y0, w, h)
    prm = prm_dict(params)
    pr = oracle.project(g, crop, prm)
    img = oracle.render_fwd(pr, crop, prm)
    n = g.n
    ex, _ = excused_pixels((x0, y0, w, h), step.proj.rect[v * n:(v + 1) * n].cpu().numpy(), pr["rect"],
                           img["margin"], 16, margin_excuse(cams[v]))
    ok = ~ex
    rng = np.random.default_rng(3)
    dcw = f32(rng.standard_normal((3, h, w)) * 1e-3 * ok[None])
    ddw = f32(rng.standard_normal((h, w)) * 1e-3 * ok)
    dc = torch.zeros_like(step.img.color); dd = torch.zeros_like(step.img.depth)
    base = sum(c.n_pixels for c in cams[:v])
    W, H = cams[v].width, cams[v].height
    dcv = np.zeros((3, H, W), np.float32); ddv = np.zeros((H, W), np.float32)
    dcv[:, y0:y0 + h, x0:x0 + w] = dcw; ddv[y0:y0 + h, x0:x0 + w] = ddw
    dc[3 * base:3 * (base + H * W)] = torch.from_numpy(dcv.reshape(-1)).cuda()
    dd[base:base + H * W] = torch.from_numpy(ddv.reshape(-1)).cuda()
    G.gs_render_bwd(step.g, step.proj, step.bins, step.img, dc, dd, step.cams, params, 0.0, step.grads, step.iso,
                    step.ws)
    torch.cuda.synchronize()
    ref = oracle.project_bwd(g, crop, prm, oracle.render_bwd(pr, crop, prm, dcw, ddw))
    got = grads_to_numpy(step.grads)
    for k in oracle.PARAM_NAMES:
        assert rel_l2(got[k], ref[k]) < GRAD_RTOL, k
    assert rel_l2(got["pose"][v], ref["pose"]) < GRAD_RTOL
    others = np.delete(got["pose"], v, axis=0)
    assert np.all(others == 0.0)
