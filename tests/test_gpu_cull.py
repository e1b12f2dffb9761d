"""Tile culling in the binning (gs_render_params.cull_tiles = 1): the lists keep
only the (entry, tile) pairs whose splat can reach 0.99 alpha_min somewhere in
the tile's box of pixel centres.

- The culled list is the plain one (every tile of the rectangle, compared
  bit-exactly with the oracle elsewhere) with entries removed, in the same order.
- Every removed pair is one whose FP64 weight stays below 0.99 alpha_min over
  the whole tile box, so it can never blend there. Every kept pair reaches
  within the kernel's rounding margin of it.
- Rendering from the culled lists gives bit-identical colour, depth and
  T_final. n_contrib names the same last blended splat, as a position in the
  shorter list. The loss and the gradients agree with the plain lists' up to
  the order of the float sums and atomics."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_02293_gb300 import gs as G
from paper_2512_02293_gb300 import synth
from gpu_common import (bins_to_numpy, ensure_lib, grads_to_numpy, oracle_bins, pack_images, prm_dict,
                        projected_to_device, rel_l2, round_projection, run_bin_sort)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _box_max_power(A, B, C, mx, my, x0, y0, w):
    """FP64 maximum over the box [x0, x0 + w] x [y0, y0 + w] of the power
    -(A dx^2 + 2 B dx dy + C dy^2) / 2 (A, C > 0, AC > B^2): a concave function,
    so its maximum over a box that does not hold the mean lies on the box edges
    that face the mean, each maximised at its clamped stationary point."""
    dx0, dy0 = x0 - mx, y0 - my
    dx1, dy1 = dx0 + w, dy0 + w
    vx = np.minimum(np.maximum(0.0, dx0), dx1)
    vy = np.minimum(np.maximum(0.0, dy0), dy1)
    sy = np.minimum(np.maximum(-B * vx / C, dy0), dy1)       # stationary dy on the line dx = vx
    sx = np.minimum(np.maximum(-B * vy / A, dx0), dx1)       # stationary dx on the line dy = vy
    pv = -0.5 * (A * vx * vx + 2 * B * vx * sy + C * sy * sy)
    ph = -0.5 * (A * sx * sx + 2 * B * sx * vy + C * vy * vy)
    return np.maximum(pv, ph)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_cull_tiles_drops_only_unreachable_tiles(tile):
    g, _, cam = synth.cfg1_problem(1)
    params = G.RenderParams(tile=tile, cull_tiles=1)
    pr = round_projection(oracle.project(g, cam, prm_dict(params)))
    proj = projected_to_device([pr])
    keys_o, vals_o, ranges_o = oracle_bins([pr], [cam], tile)
    bins, _ = run_bin_sort(proj, g.n, [cam], params, capacity=len(keys_o) + 17)
    assert G.gs_read_device_status(bins.status) == 0
    keys, vals, ranges = bins_to_numpy(bins)
    M = len(keys)
    assert int(bins.num_keys.item()) == M
    # a subsequence of the plain list, and the ranges are its tiles' segments
    where = {(int(k), int(v)): i for i, (k, v) in enumerate(zip(keys_o, vals_o))}
    idx = np.array([where[(int(k), int(v))] for k, v in zip(keys, vals)])
    assert np.all(np.diff(idx) > 0)
    t = (keys >> np.uint64(32)).astype(np.int64)
    counts = np.bincount(t, minlength=len(ranges))
    np.testing.assert_array_equal(ranges[:, 1].astype(np.int64) - ranges[:, 0], counts)
    nonempty = counts > 0
    np.testing.assert_array_equal(ranges[nonempty, 0].astype(np.int64), (np.cumsum(counts) - counts)[nonempty])
    # the decision of every pair of the plain list against the FP64 maximum over the tile box
    kept = np.zeros(len(keys_o), bool)
    kept[idx] = True
    tx = (cam.width + tile - 1) // tile
    to = (keys_o >> np.uint64(32)).astype(np.int64)
    e = vals_o.astype(np.int64)
    A, B, C = (pr["conic"][e, k].astype(np.float64) for k in range(3))
    o = pr["opacity"][e].astype(np.float64)
    mx, my = pr["xy"][e, 0].astype(np.float64), pr["xy"][e, 1].astype(np.float64)
    x0 = (to % tx) * tile + 0.5
    y0 = (to // tx) * tile + 0.5
    pmax = _box_max_power(A, B, C, mx, my, x0, y0, tile - 1.0)
    # the closed form is the maximum: no point of a dense grid over the box exceeds it
    gx = np.linspace(0.0, tile - 1.0, 33)
    dx = x0[:, None, None] + gx[None, None, :] - mx[:, None, None]
    dy = y0[:, None, None] + gx[None, :, None] - my[:, None, None]
    pg = (-0.5 * (A[:, None, None] * dx * dx + 2 * B[:, None, None] * dx * dy + C[:, None, None] * dy * dy)).max(
        axis=(1, 2))
    assert np.all(pg <= pmax + 1e-9)
    wmax = o * np.exp(pmax)
    thr = 0.99 * params.alpha_min
    assert np.all(wmax[~kept] < thr * (1 + 1e-4)), "a dropped pair can reach 0.99 alpha_min"
    assert np.all(wmax[kept] >= thr * 2 ** -0.004 * (1 - 1e-4)), "a kept pair stays below the margin"
    assert (~kept).sum() > 0 and kept.sum() > 0


def _render(g, cams, params, capacity):
    prs = [round_projection(oracle.project(g, c, prm_dict(params))) for c in cams]
    proj = projected_to_device(prs)
    bins, _ = run_bin_sort(proj, g.n, cams, params, capacity)
    img = G.Image.empty(G.gs_total_pixels(cams))
    G.gs_render_fwd(proj, bins, cams, params, img)
    torch.cuda.synchronize()
    return bins, img


@pytest.mark.parametrize("case", ["64x48", "640x480"])
def test_render_from_culled_lists_is_identical(case):
    if case == "64x48":
        g, _, cam = synth.cfg1_problem(0)
    else:
        g, _, cam = synth.cfg2_problem()
    cams = [cam]
    base = G.RenderParams(tile=16)
    m = sum(int(round_projection(oracle.project(g, c, prm_dict(base)))["tiles"].sum()) for c in cams) + 1
    b0, i0 = _render(g, cams, base, m)
    b1, i1 = _render(g, cams, G.RenderParams(tile=16, cull_tiles=1), m)
    assert int(b1.num_keys.item()) < int(b0.num_keys.item())
    for f in ("color", "depth", "T_final"):
        assert torch.equal(getattr(i0, f), getattr(i1, f)), f
    # n_contrib: the same last blended splat, at its position in each list
    tile = 16
    W, H = cam.width, cam.height
    tx = (W + tile - 1) // tile
    py, px = np.mgrid[0:H, 0:W]
    t = ((py // tile) * tx + px // tile).ravel()
    k0, v0, r0 = bins_to_numpy(b0)
    k1, v1, r1 = bins_to_numpy(b1)
    n0 = i0.n_contrib.cpu().numpy().astype(np.int64)
    n1 = i1.n_contrib.cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(n0 == 0, n1 == 0)
    nz = n0 > 0
    last0 = r0[t[nz], 0].astype(np.int64) + n0[nz] - 1
    last1 = r1[t[nz], 0].astype(np.int64) + n1[nz] - 1
    np.testing.assert_array_equal(k0[last0], k1[last1])
    np.testing.assert_array_equal(v0[last0], v1[last1])
    assert np.all(n1 <= n0)


def test_mapping_step_with_culled_lists_matches_plain_lists():
    from paper_2512_02293_gb300.mapping import MapParams, MappingStep
    g, gt, cam = synth.cfg1_problem(0)
    cams = [cam]
    params = G.RenderParams()
    prm = prm_dict(params)
    timgs = [oracle.render_fwd(oracle.project(gt, c, prm), c, prm) for c in cams]
    tc, td = pack_images([np.float32(t["color"]) for t in timgs], [np.float32(t["depth"]) for t in timgs])
    mp = MapParams(lambda_c=0.9, lambda_d=0.1, lambda_iso=10.0)
    out = []
    for cull in (0, 1):
        p = G.RenderParams(block_masks=1, cull_tiles=cull)
        step = MappingStep(G.Gaussians.from_numpy(g), cams, tc, td, p, mp)
        step.render()
        step.loss_and_backward()
        torch.cuda.synchronize()
        out.append((step.img.color.clone(), step.loss_terms.clone(), grads_to_numpy(step.grads)))
    assert torch.equal(out[0][0], out[1][0])
    # the loss sums: per-CTA partials of a dynamically scheduled launch, so equal up to their order
    np.testing.assert_allclose(out[1][1].cpu().numpy(), out[0][1].cpu().numpy(), rtol=1e-5)
    for k in oracle.PARAM_NAMES:
        assert rel_l2(out[1][2][k], out[0][2][k]) < 1e-5, k
    assert rel_l2(out[1][2]["pose"][0], out[0][2]["pose"][0]) < 1e-5
