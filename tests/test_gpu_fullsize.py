"""Parity at the benchmark's full size (640x480, 200k Gaussians, tile 16; the
kernels and launch shapes bench.py times), on outputs the oracle can compute
piecewise:

- projection of every Gaussian, element by element;
- keys / order / ranges bit-exact on the oracle's fp32-rounded projection;
- colour / depth / checkpoint (T_final, and n_contrib bit-exact) on
  tile-aligned windows (the oracle renders the window as its own camera, cx
  and cy shifted by the window offset);
- every parameter gradient and the pose gradient for a loss whose image
  gradient lives inside a window;
- properties of the GPU's own keys that hold at any size.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_02293_gb300 import gs as G
from paper_2512_02293_gb300 import synth
from paper_2512_02293_gb300.mapping import MapParams, MappingStep
from gpu_common import (COLOR_TOL, GRAD_RTOL, bins_to_numpy, ensure_lib, excused_pixels, f32, grads_to_numpy,
                        margin_excuse, oracle_bins, prm_dict, projected_to_device, rel_l2, round_projection,
                        run_bin_sort)

pytestmark = pytest.mark.gpu

WINDOWS = [(256, 192, 64, 64), (0, 0, 48, 32), (592, 448, 48, 32)]   # x0, y0, w, h (tile-aligned)


@pytest.fixture(scope="module")
def setup():
    ensure_lib()
    g, gt, cam = synth.cfg2_problem()
    params = G.RenderParams(tile=16)
    P = cam.n_pixels
    step = MappingStep(G.Gaussians.from_numpy(g), [cam], torch.zeros(3 * P, device="cuda"),
                       torch.zeros(P, device="cuda"), params, MapParams(1.0, 1.0, 0.0))
    step.render()
    torch.cuda.synchronize()
    assert step.check() == 0
    return g, cam, params, step


def _crop(cam, x0, y0, w, h):
    return synth.Camera(cam.fx, cam.fy, cam.cx - x0, cam.cy - y0, w, h, cam.R_wc, cam.t_wc)


def test_projection_all_entries(setup):
    g, cam, params, step = setup
    pr = oracle.project(g, cam, prm_dict(params))
    tt = step.proj.tiles_touched.cpu().numpy()
    vis = pr["tiles"] > 0
    boundary = pr["margin"] < 1e-3          # within 1e-3 px of a rounding boundary (reported, not compared)
    assert boundary[vis].mean() < 1e-2
    np.testing.assert_array_equal((tt > 0)[~boundary], vis[~boundary])
    ok = vis & (tt > 0) & ~boundary
    np.testing.assert_allclose(step.proj.xy.cpu().numpy()[ok], pr["xy"][ok], atol=5e-4)
    co = step.proj.conic_o.cpu().numpy()
    np.testing.assert_allclose(co[ok, :3], pr["conic"][ok], rtol=5e-4, atol=1e-6)
    np.testing.assert_allclose(step.proj.rgbd.cpu().numpy()[ok, 3], pr["depth"][ok], rtol=1e-6)
    np.testing.assert_array_equal(step.proj.rect.cpu().numpy()[ok], pr["rect"][ok])


def test_bin_sort_bit_exact_full_size(setup):
    g, cam, params, step = setup
    prs = [round_projection(oracle.project(g, cam, prm_dict(params)))]
    proj = projected_to_device(prs)
    keys_o, vals_o, ranges_o = oracle_bins(prs, [cam], 16)
    assert len(keys_o) > 200_000
    bins, _ = run_bin_sort(proj, g.n, [cam], params, capacity=int(len(keys_o) * 1.1))
    keys, vals, ranges = bins_to_numpy(bins)
    np.testing.assert_array_equal(keys, keys_o)
    np.testing.assert_array_equal(vals, vals_o)
    np.testing.assert_array_equal(ranges, ranges_o)


def test_gpu_keys_properties(setup):
    g, cam, params, step = setup
    keys, vals, ranges = bins_to_numpy(step.bins)
    tt = step.proj.tiles_touched.cpu().numpy().astype(np.int64)
    assert len(keys) == tt.sum()
    assert np.all(np.diff(keys.astype(np.uint64)) >= 0) if len(keys) > 1 else True
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    np.testing.assert_array_equal(np.bincount(vals, minlength=g.n), tt)       # one key per covered tile
    rect = step.proj.rect.cpu().numpy()
    tx = (cam.width + 15) // 16
    x, y = tiles % tx, tiles // tx
    r = rect[vals]
    assert np.all((x >= r[:, 0]) & (x < r[:, 2]) & (y >= r[:, 1]) & (y < r[:, 3]))
    z = step.proj.rgbd.cpu().numpy()[vals, 3]
    np.testing.assert_array_equal((keys & np.uint64(0xFFFFFFFF)).astype(np.uint32), z.view(np.uint32))
    same = np.diff(keys) == 0
    assert np.all(np.diff(vals.astype(np.int64))[same] > 0)                  # ties in index order
    for t in range(len(ranges)):
        s, e = ranges[t]
        if e > s:
            assert np.all(tiles[s:e] == t)


def _excused(cam, crop_xywh, pr_gpu_rect, pr_or, img_or):
    return excused_pixels(crop_xywh, pr_gpu_rect, pr_or["rect"], img_or["margin"], 16, margin_excuse(cam))


@pytest.mark.parametrize("win", WINDOWS)
def test_window_forward_and_backward(setup, win):
    g, cam, params, step = setup
    x0, y0, w, h = win
    crop = _crop(cam, x0, y0, w, h)
    prm = prm_dict(params)
    pr = oracle.project(g, crop, prm)
    img = oracle.render_fwd(pr, crop, prm)
    ex, n_rect = _excused(cam, win, step.proj.rect.cpu().numpy(), pr, img)
    assert ex.mean() < 0.05, (ex.mean(), n_rect)
    col = step.color_image(0).cpu().numpy()[:, y0:y0 + h, x0:x0 + w]
    dep = step.depth_image(0).cpu().numpy()[y0:y0 + h, x0:x0 + w]
    P = cam.n_pixels
    Tf = step.img.T_final.cpu().numpy().reshape(cam.height, cam.width)[y0:y0 + h, x0:x0 + w]
    nc = step.img.n_contrib.cpu().numpy().view(np.uint32).reshape(cam.height, cam.width)[y0:y0 + h, x0:x0 + w]
    ok = ~ex
    np.testing.assert_allclose(col[:, ok], img["color"][:, ok], atol=COLOR_TOL)
    np.testing.assert_allclose(dep[ok], img["depth"][ok], atol=COLOR_TOL)
    np.testing.assert_allclose(Tf[ok], img["T_final"][ok], atol=1e-5)
    # the checkpoint's integer half: the list position of each pixel's last blended splat
    np.testing.assert_array_equal(nc[ok], img["n_contrib"][ok])
    # backward for an image gradient supported on the window's non-excused pixels
    rng = np.random.default_rng(x0 + y0)
    dcw = rng.standard_normal((3, h, w)) * 1e-3 * ok[None]
    ddw = rng.standard_normal((h, w)) * 1e-3 * ok
    dcw = f32(dcw); ddw = f32(ddw)
    dc = np.zeros((3, cam.height, cam.width), np.float32); dd = np.zeros((cam.height, cam.width), np.float32)
    dc[:, y0:y0 + h, x0:x0 + w] = dcw; dd[y0:y0 + h, x0:x0 + w] = ddw
    dct = torch.from_numpy(dc.reshape(-1)).cuda(); ddt = torch.from_numpy(dd.reshape(-1)).cuda()
    G.gs_render_bwd(step.g, step.proj, step.bins, step.img, dct, ddt, step.cams, params, 0.0, step.grads, step.iso,
                    step.ws)
    torch.cuda.synchronize()
    ref2d = oracle.render_bwd(pr, crop, prm, dcw, ddw)
    ref = oracle.project_bwd(g, crop, prm, ref2d)
    got = grads_to_numpy(step.grads)
    for k in oracle.PARAM_NAMES:
        assert rel_l2(got[k], ref[k]) < GRAD_RTOL, k
    assert rel_l2(got["pose"][0], ref["pose"]) < GRAD_RTOL


def test_graph_replay_equals_eager(setup):
    g, cam, params, _ = setup
    P = cam.n_pixels
    tgt_c = torch.rand(3 * P, device="cuda"); tgt_d = torch.rand(P, device="cuda") * 4
    a = MappingStep(G.Gaussians.from_numpy(g), [cam], tgt_c, tgt_d, params, MapParams())
    b = MappingStep(G.Gaussians.from_numpy(g), [cam], tgt_c, tgt_d, params, MapParams(),
                    key_capacity=a.bins.capacity)
    a.step()
    b.capture(warmup=0)
    b.step()
    torch.cuda.synchronize()
    # one iteration: same arithmetic, same order except float atomics in the backward
    for ga, gb in zip(a.grads.tensors(), b.grads.tensors()):
        assert rel_l2(gb.cpu().numpy(), ga.cpu().numpy()) < 1e-5
    for _ in range(2):
        a.step()
        b.step()
    torch.cuda.synchronize()
    assert a.check() == 0 and b.check() == 0
    assert int(a.d_step[0].item()) == 3 and int(b.d_step[0].item()) == 3
    # Adam divides by sqrt(v): a near-zero gradient whose atomic summation order
    # differs may change the sign of its step; allow a handful such elements,
    # each off by at most the three steps' lr
    lrs = MapParams().lr
    for ta, tb, lr in zip(a.g.tensors(), b.g.tensors(), lrs):
        d = np.abs(tb.cpu().numpy() - ta.cpu().numpy())
        off = d > 1e-6 + 1e-4 * np.abs(ta.cpu().numpy())
        assert off.mean() < 1e-4 and (d[off].max() if off.any() else 0.0) <= 6 * lr + 1e-6


def test_mapping_iterations_reduce_the_loss(setup):
    g, cam, params, _ = setup
    gt = synth.perturb_map(g, 99)
    P = cam.n_pixels
    ts = MappingStep(G.Gaussians.from_numpy(gt), [cam], torch.zeros(3 * P, device="cuda"),
                     torch.zeros(P, device="cuda"), params)
    ts.render()
    torch.cuda.synchronize()
    step = MappingStep(G.Gaussians.from_numpy(g), [cam], ts.img.color.clone(), ts.img.depth.clone(), params,
                       MapParams(lambda_iso=0.0))
    losses = []
    for it in range(30):
        step.step()
        losses.append(float(step.loss().item()))
        if it == 0:
            assert not step.ensure_capacity()
    assert losses[-1] < 0.8 * losses[0], losses


def test_ordered_forward_on_the_deepest_blocks_matches_oracle(setup):
    """After one fused forward and backward, the next fused forward takes its
    8 x 4 blocks deepest first (the backward's order), the first ones handed to
    the first warps of different CTAs.  A 64x64 window around the deepest pixel
    is compared with the oracle, n_contrib bit-exact, and the whole image with
    the same step's first (natural-order) forward: bit for bit, since the order
    changes only which warp takes which block."""
    g, cam, params, _ = setup
    P = cam.n_pixels
    step = MappingStep(G.Gaussians.from_numpy(g), [cam], torch.zeros(3 * P, device="cuda"),
                       torch.zeros(P, device="cuda"), params, MapParams(1.0, 1.0, 0.0))
    step.render()
    step.loss_and_backward()                 # the backward writes the deepest-first order
    torch.cuda.synchronize()
    col0 = step.img.color.clone(); nc0 = step.img.n_contrib.clone()
    step.render()                            # ordered: deepest blocks first
    torch.cuda.synchronize()
    assert step.check() == 0
    nc = step.img.n_contrib.cpu().numpy().view(np.uint32).reshape(cam.height, cam.width)
    assert nc.max() > 768                    # a deep list (the long serial walk)
    yd, xd = np.unravel_index(np.argmax(nc), nc.shape)
    x0 = int(min(max(xd // 16 * 16 - 16, 0), cam.width - 64))
    y0 = int(min(max(yd // 16 * 16 - 16, 0), cam.height - 64))
    w = h = 64
    crop = _crop(cam, x0, y0, w, h)
    prm = prm_dict(params)
    pr = oracle.project(g, crop, prm)
    img = oracle.render_fwd(pr, crop, prm)
    ex, _ = _excused(cam, (x0, y0, w, h), step.proj.rect.cpu().numpy(), pr, img)
    ok = ~ex
    assert ok.mean() > 0.9
    col = step.color_image(0).cpu().numpy()[:, y0:y0 + h, x0:x0 + w]
    dep = step.depth_image(0).cpu().numpy()[y0:y0 + h, x0:x0 + w]
    Tf = step.img.T_final.cpu().numpy().reshape(cam.height, cam.width)[y0:y0 + h, x0:x0 + w]
    np.testing.assert_allclose(col[:, ok], img["color"][:, ok], atol=COLOR_TOL)
    np.testing.assert_allclose(dep[ok], img["depth"][ok], atol=COLOR_TOL)
    np.testing.assert_allclose(Tf[ok], img["T_final"][ok], atol=1e-5)
    np.testing.assert_array_equal(nc[y0:y0 + h, x0:x0 + w][ok], img["n_contrib"][ok])
    # against the natural-order forward of the same map
    assert torch.equal(step.img.color, col0) and torch.equal(step.img.n_contrib, nc0)
