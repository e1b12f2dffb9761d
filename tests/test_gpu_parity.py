"""GPU (libgs, through the C ABI) against the FP64 oracle, stage by stage and
end to end, on the 64x48 / 256-Gaussian case, ragged images, other tile
sizes, several views and the degenerate cases.

Tolerances: tile keys, order and ranges bit-exact; rendered colour and depth
within 1e-4 absolute; gradients within 1e-3 relative L2.  Pixels whose
threshold decisions (alpha_min, T_cut) lie within 1e-5 relative of the
threshold may legitimately differ between fp32 and fp64; the oracle reports
that margin and such pixels are counted (expected: none here)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_02293_gb300 import gs as G
from paper_2512_02293_gb300 import synth
from gpu_common import (COLOR_TOL, GRAD_RTOL, MARGIN_EXCUSE, bins_to_numpy, ensure_lib, f32, grads_to_numpy,
                        image_views, oracle_bins, pack_images, prm_dict, projected_to_device, rel_l2,
                        round_projection, run_bin_sort)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _problem(trial=0):
    g, gt, cam = synth.cfg1_problem(trial)
    return g, gt, cam


def _stage_inputs(g, cams, params):
    """Oracle projection of every view, rounded to fp32."""
    prm = prm_dict(params)
    return [round_projection(oracle.project(g, c, prm)) for c in cams]


# ------------------------------------------------------------------ projection

@pytest.mark.parametrize("trial", [0, 1])
def test_project_matches_oracle(trial):
    g, _, cam = _problem(trial)
    params = G.RenderParams()
    gd = G.Gaussians.from_numpy(g)
    out = G.Projected.empty(g.n)
    G.gs_project(gd, [cam], params, out)
    torch.cuda.synchronize()
    pr = oracle.project(g, cam, prm_dict(params))
    tt = out.tiles_touched.cpu().numpy()
    vis = pr["tiles"] > 0
    boundary = pr["margin"] < 1e-3
    np.testing.assert_array_equal((tt > 0)[~boundary], vis[~boundary])
    both = vis & (tt > 0)
    np.testing.assert_allclose(out.xy.cpu().numpy()[both], pr["xy"][both], atol=2e-4)
    co = out.conic_o.cpu().numpy()
    np.testing.assert_allclose(co[both, :3], pr["conic"][both], rtol=2e-4, atol=1e-6)
    np.testing.assert_allclose(co[both, 3], pr["opacity"][both], rtol=1e-6)
    cd = out.rgbd.cpu().numpy()
    np.testing.assert_allclose(cd[both, :3], pr["rgb"][both], rtol=1e-7)
    np.testing.assert_allclose(cd[both, 3], pr["depth"][both], rtol=1e-6)
    ok = both & ~boundary
    np.testing.assert_array_equal(out.radius.cpu().numpy()[ok], pr["radius"][ok])
    np.testing.assert_array_equal(out.rect.cpu().numpy()[ok], pr["rect"][ok])
    np.testing.assert_array_equal(tt[ok], pr["tiles"][ok])
    assert boundary[vis].sum() == 0   # no rounding-boundary case in this workload


# ------------------------------------------------------------------ binning

@pytest.mark.parametrize("tile", [8, 16, 32])
def test_bin_sort_bit_exact(tile):
    g, _, cam = _problem(0)
    params = G.RenderParams(tile=tile)
    prs = _stage_inputs(g, [cam], params)
    proj = projected_to_device(prs)
    keys_o, vals_o, ranges_o = oracle_bins(prs, [cam], tile)
    bins, _ = run_bin_sort(proj, g.n, [cam], params, capacity=len(keys_o) + 17)
    keys, vals, ranges = bins_to_numpy(bins)
    assert int(bins.status[0].item()) == 0
    np.testing.assert_array_equal(keys, keys_o)
    np.testing.assert_array_equal(vals, vals_o)
    np.testing.assert_array_equal(ranges, ranges_o)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_bin_sort_block_masks_are_conservative(tile):
    """gs_bins.masks, bit b of a key: the splat can reach pixel block b of its tile
    (8 x 4 blocks, row-major).  At every pixel centre of a block where the
    splat's weight o exp(power), in FP64 from the same projected values, reaches
    alpha_min, the block's bit must be set, so the rasterisers' culling drops
    nothing that blends; and the masks do cull (some bits are clear)."""
    g, _, cam = _problem(0)
    params = G.RenderParams(tile=tile)
    prs = _stage_inputs(g, [cam], params)
    proj = projected_to_device(prs)
    keys_o, vals_o, ranges_o = oracle_bins(prs, [cam], tile)
    bins, _ = run_bin_sort(proj, g.n, [cam], params, capacity=len(keys_o) + 17)
    keys, vals, _ = bins_to_numpy(bins)
    M = len(keys_o)
    masks = bins.masks[:M].cpu().numpy().view(np.uint32).astype(np.int64)
    pr = prs[0]
    t = (keys.astype(np.uint64) >> np.uint64(32)).astype(np.int64)
    e = vals.astype(np.int64)
    tiles_x = (cam.width + tile - 1) // tile
    tx, ty = t % tiles_x, t // tiles_x
    mx, my = pr["xy"][e, 0].astype(np.float64), pr["xy"][e, 1].astype(np.float64)
    A, B, C = (pr["conic"][e, k].astype(np.float64) for k in range(3))
    o = pr["opacity"][e].astype(np.float64)
    bw, nb = tile // 8, (tile // 8) * (tile // 4)
    cleared = 0
    for b in range(nb):
        px = (tx * tile + (b % bw) * 8)[:, None] + np.arange(8)[None, :] + 0.5      # [M, 8]
        py = (ty * tile + (b // bw) * 4)[:, None] + np.arange(4)[None, :] + 0.5     # [M, 4]
        dx = px[:, None, :] - mx[:, None, None]
        dy = py[:, :, None] - my[:, None, None]
        power = -0.5 * (A[:, None, None] * dx * dx + 2 * B[:, None, None] * dx * dy + C[:, None, None] * dy * dy)
        reach = (o[:, None, None] * np.exp(power) >= params.alpha_min).any(axis=(1, 2))
        bit = (masks >> b) & 1
        assert np.all(bit[reach] == 1), (b, int((bit[reach] == 0).sum()))
        cleared += int((bit == 0).sum())
    assert (masks >> nb).max() == 0            # no bits past the tile's blocks
    assert cleared > 0


def test_bin_sort_bit_exact_many_keys_ties_and_views():
    # Synthetic projected entries over three views of uneven size: ~300k keys,
    # many equal depths (ties broken by entry index), several sort blocks.
    rng = np.random.default_rng(7)
    cams = [synth.identity_camera(640, 480), synth.identity_camera(752, 480), synth.identity_camera(1280, 1024)]
    params = G.RenderParams(tile=16)
    n = 20000
    prs = []
    for c in cams:
        tx, ty = (c.width + 15) // 16, (c.height + 15) // 16
        x0 = rng.integers(0, tx, n); y0 = rng.integers(0, ty, n)
        rect = np.stack([x0, y0, np.minimum(x0 + rng.integers(1, 5, n), tx), np.minimum(y0 + rng.integers(1, 4, n), ty)], 1)
        culled = rng.random(n) < 0.2
        rect[culled] = 0
        depth = rng.choice(np.linspace(0.3, 8.0, 500), n)     # heavy ties
        tiles = (rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1])
        prs.append(dict(xy=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n), rgb=np.zeros((n, 3)),
                        depth=f32(depth), rect=rect.astype(np.int32), radius=np.ones(n, np.int32), tiles=tiles))
    proj = projected_to_device(prs)
    keys_o, vals_o, ranges_o = oracle_bins(prs, cams, 16)
    bins, _ = run_bin_sort(proj, n, cams, params, capacity=len(keys_o))
    keys, vals, ranges = bins_to_numpy(bins)
    assert len(keys_o) > 100_000
    np.testing.assert_array_equal(keys, keys_o)
    np.testing.assert_array_equal(vals, vals_o)
    np.testing.assert_array_equal(ranges, ranges_o)


@pytest.mark.parametrize("deep", [4096, 4097, 20000])
def test_bin_sort_bit_exact_deep_tiles(deep):
    # Tiles whose lists exceed what one CTA sorts in shared memory (4096 keys)
    # take the CTA-wide radix path; `deep` entries cover one tile, half of them
    # also its right neighbour (a list just below, at and far above the limit),
    # scattered through the entry order among shallow random entries, with
    # heavy depth ties (ties broken by entry index).
    rng = np.random.default_rng(deep)
    cam = synth.identity_camera(256, 128)                  # 16 x 8 tiles of 16 px
    params = G.RenderParams(tile=16)
    tx, ty = 16, 8
    n = deep + 3000
    x0 = rng.integers(0, tx, n); y0 = rng.integers(0, ty, n)
    rect = np.stack([x0, y0, np.minimum(x0 + rng.integers(1, 4, n), tx),
                     np.minimum(y0 + rng.integers(1, 3, n), ty)], 1)
    pile = rng.permutation(n)[:deep]
    rect[pile] = [5, 3, 6, 4]
    rect[pile[::2], 2] = 7
    culled = rng.random(n) < 0.1
    culled[pile] = False
    rect[culled] = 0
    depth = rng.choice(np.linspace(0.3, 8.0, 300), n)
    tiles = (rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1])
    prs = [dict(xy=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n), rgb=np.zeros((n, 3)),
                depth=f32(depth), rect=rect.astype(np.int32), radius=np.ones(n, np.int32), tiles=tiles)]
    proj = projected_to_device(prs)
    keys_o, vals_o, ranges_o = oracle_bins(prs, [cam], 16)
    r = ranges_o.reshape(-1, 2)
    assert r[3 * tx + 5, 1] - r[3 * tx + 5, 0] >= deep
    bins, _ = run_bin_sort(proj, n, [cam], params, capacity=len(keys_o) + 5)
    keys, vals, ranges = bins_to_numpy(bins)
    assert int(bins.status[0].item()) == 0
    np.testing.assert_array_equal(keys, keys_o)
    np.testing.assert_array_equal(vals, vals_o)
    np.testing.assert_array_equal(ranges, ranges_o)


def test_capacity_overflow_is_reported_not_faulted():
    g, _, cam = _problem(0)
    params = G.RenderParams()
    prs = _stage_inputs(g, [cam], params)
    proj = projected_to_device(prs)
    keys_o, _, _ = oracle_bins(prs, [cam], 16)
    bins, _ = run_bin_sort(proj, g.n, [cam], params, capacity=len(keys_o) // 3)
    assert G.gs_read_device_status(bins.status) == G.GS_ERR_CAPACITY
    assert int(bins.num_keys.item()) == len(keys_o)
    bins2, _ = run_bin_sort(proj, g.n, [cam], params, capacity=len(keys_o))
    assert G.gs_read_device_status(bins2.status) == 0
    np.testing.assert_array_equal(bins_to_numpy(bins2)[0], keys_o)


# ------------------------------------------------------------------ forward

def _gpu_forward(proj, n, cams, params, capacity):
    bins, ws = run_bin_sort(proj, n, cams, params, capacity)
    img = G.Image.empty(G.gs_total_pixels(cams))
    G.gs_render_fwd(proj, bins, cams, params, img)
    torch.cuda.synchronize()
    return bins, ws, img


def _compare_images(gpu, ref, what=""):
    excused = ref["margin"] < MARGIN_EXCUSE
    n_exc = int(excused.sum())
    ok = ~excused
    np.testing.assert_allclose(gpu["color"][:, ok], ref["color"][:, ok], atol=COLOR_TOL, err_msg=what)
    np.testing.assert_allclose(gpu["depth"][ok], ref["depth"][ok], atol=COLOR_TOL, err_msg=what)
    np.testing.assert_allclose(gpu["T_final"][ok], ref["T_final"][ok], atol=1e-5, err_msg=what)
    np.testing.assert_array_equal(gpu["n_contrib"][ok], ref["n_contrib"][ok], err_msg=what)
    return n_exc


@pytest.mark.parametrize("masks", [1, 0])
@pytest.mark.parametrize("tile,bg", [(16, (0.0, 0.0, 0.0)), (8, (0.2, 0.3, 0.4)), (32, (0.0, 0.0, 0.0))])
def test_render_fwd_matches_oracle(tile, bg, masks):
    """masks: the binning's pixel-block masks (1) or the rasteriser's own test (0)."""
    g, _, cam = _problem(1)
    params = G.RenderParams(tile=tile, bg=bg, block_masks=masks)
    prs = _stage_inputs(g, [cam], params)
    proj = projected_to_device(prs)
    m = int(sum(p["tiles"].sum() for p in prs))
    _, _, img = _gpu_forward(proj, g.n, [cam], params, m + 1)
    ref = oracle.render_fwd(prs[0], cam, prm_dict(params))
    assert _compare_images(image_views(img, [cam])[0], ref) == 0


def test_render_fwd_ragged_and_multiview():
    # Image sizes that are not multiples of the tile, several views in one call;
    # every view must equal its own oracle render.
    g, _, _ = _problem(2)
    R, e = synth.look_at([0.2, -0.1, -0.3], [0.0, 0.1, 2.0])
    cams = [synth.Camera(55.0, 57.0, 35.3, 22.1, 70, 45),
            synth.Camera(40.0, 40.0, 16.5, 13.0, 33, 26, R, e),
            synth.Camera(62.0, 62.0, 31.0, 24.0, 64, 48)]
    for tile in (8, 16):
        params = G.RenderParams(tile=tile)
        prs = _stage_inputs(g, cams, params)
        proj = projected_to_device(prs)
        m = int(sum(p["tiles"].sum() for p in prs))
        _, _, img = _gpu_forward(proj, g.n, cams, params, m)
        for v, (c, p) in enumerate(zip(cams, prs)):
            ref = oracle.render_fwd(p, c, prm_dict(params))
            assert _compare_images(image_views(img, cams)[v], ref, f"view {v} tile {tile}") == 0


def test_thirty_two_views_the_maximum():
    # GS_MAX_VIEWS views of different sizes and poses in one call: keys bit-exact,
    # every view equal to its own oracle render, the 33rd view refused on the host
    g, _, _ = _problem(3)
    rng = np.random.default_rng(32)
    cams = []
    for v in range(G.GS_MAX_VIEWS):
        R, e = synth.look_at(rng.normal(0, 0.15, 3) + [0.0, 0.0, -0.2], [0.0, 0.0, 2.0])
        W, H = int(rng.integers(20, 70)), int(rng.integers(16, 50))
        cams.append(synth.Camera(50.0, 50.0, W / 2, H / 2, W, H, R, e))
    params = G.RenderParams(tile=8)
    prs = _stage_inputs(g, cams, params)
    proj = projected_to_device(prs)
    m = int(sum(p["tiles"].sum() for p in prs))
    bins, _, img = _gpu_forward(proj, g.n, cams, params, m)
    keys, vals, ranges = bins_to_numpy(bins)
    ok_, ov, orr = oracle_bins(prs, cams, 8)
    np.testing.assert_array_equal(keys, ok_)
    np.testing.assert_array_equal(vals, ov)
    np.testing.assert_array_equal(ranges, orr)
    views = image_views(img, cams)
    excused = 0
    for v, (c, p) in enumerate(zip(cams, prs)):
        excused += _compare_images(views[v], oracle.render_fwd(p, c, prm_dict(params)), f"view {v}")
    assert excused <= 5          # near-threshold pixels over 32 views (each compared elsewhere exactly)
    with pytest.raises(G.GsError):
        G.gs_project(G.Gaussians.from_numpy(g), cams + cams[:1], params, G.Projected.empty(g.n * 33))


def test_splats_covering_every_tile():
    # Gaussians a few centimetres in front of the camera: their radius spans the
    # whole grid (and, for the nearest, exceeds any image), so every one of them
    # is keyed to every tile; bins and images still equal the oracle's.
    g, _, cam = _problem(4)
    big = synth.random_cloud(12, 5, box=((-0.05, 0.05), (-0.05, 0.05), (0.25, 0.4)), log_scale_mu=-1.0,
                             log_scale_sd=0.2)
    both = synth.GaussianMap(*(np.concatenate([a, b]) for a, b in zip(g.arrays(), big.arrays())))
    params = G.RenderParams(tile=16)
    prs = _stage_inputs(both, [cam], params)
    tiles = prs[0]["tiles"]
    total = G.gs_total_tiles([cam], 16)
    assert np.sum(tiles[g.n:] == total) >= 6
    proj = projected_to_device(prs)
    bins, _, img = _gpu_forward(proj, both.n, [cam], params, int(tiles.sum()))
    keys, vals, ranges = bins_to_numpy(bins)
    ok_, ov, orr = oracle_bins(prs, [cam], 16)
    np.testing.assert_array_equal(keys, ok_)
    np.testing.assert_array_equal(vals, ov)
    np.testing.assert_array_equal(ranges, orr)
    assert _compare_images(image_views(img, [cam])[0], oracle.render_fwd(prs[0], cam, prm_dict(params))) < 20


def test_degenerate_inputs():
    params = G.RenderParams()
    cam = synth.identity_camera()
    # no Gaussians at all
    g0 = synth.random_cloud(0, 1)
    gd = G.Gaussians.from_numpy(g0)
    proj = G.Projected.empty(0)
    G.gs_project(gd, [cam], params, proj)
    bins, ws = run_bin_sort(proj, 0, [cam], params, 1024)
    img = G.Image.empty(cam.n_pixels)
    G.gs_render_fwd(proj, bins, [cam], params, img)
    torch.cuda.synchronize()
    assert int(bins.num_keys.item()) == 0
    v = image_views(img, [cam])[0]
    assert np.all(v["color"] == 0) and np.all(v["T_final"] == 1) and np.all(v["n_contrib"] == 0)
    # every Gaussian behind the camera: all culled
    g = synth.random_cloud(64, 3, box=((-1, 1), (-1, 1), (-3, -1)))
    gd = G.Gaussians.from_numpy(g)
    proj = G.Projected.empty(g.n)
    G.gs_project(gd, [cam], params, proj)
    torch.cuda.synchronize()
    assert int(proj.tiles_touched.sum().item()) == 0
    bins, ws = run_bin_sort(proj, g.n, [cam], params, 1024)
    G.gs_render_fwd(proj, bins, [cam], params, img)
    torch.cuda.synchronize()
    assert int(bins.num_keys.item()) == 0
    assert np.all(image_views(img, [cam])[0]["T_final"] == 1)


# ------------------------------------------------------------------ loss

def test_loss_matches_oracle():
    rng = np.random.default_rng(4)
    cams = [synth.identity_camera(64, 48), synth.identity_camera(70, 45)]
    colors = [rng.random((3, c.height, c.width)) for c in cams]
    depths = [rng.random((c.height, c.width)) * 3 for c in cams]
    tcol = [np.where(rng.random(a.shape) < 0.1, f32(a), rng.random(a.shape)) for a in colors]
    tdep = [np.where(rng.random(a.shape) < 0.3, 0.0, rng.random(a.shape) * 3) for a in depths]
    c_d, d_d = pack_images(colors, depths)
    tc_d, td_d = pack_images(tcol, tdep)
    P = sum(c.n_pixels for c in cams)
    img = G.Image(c_d, d_d, torch.ones(P, device="cuda"), torch.zeros(P, device="cuda", dtype=torch.int32))
    dc = torch.empty_like(c_d); dd = torch.empty_like(d_d)
    terms = torch.empty(len(cams), 2, device="cuda")
    ws = torch.empty(1024, device="cuda")
    G.gs_loss(img, tc_d, td_d, cams, 0.9, 0.1, dc, dd, terms, ws)
    torch.cuda.synchronize()
    base = 0
    for v, c in enumerate(cams):
        t, gdc, gdd = oracle.l1_loss(f32(colors[v]), f32(depths[v]), f32(tcol[v]), f32(tdep[v]), 0.9, 0.1)
        HW = c.n_pixels
        np.testing.assert_allclose(terms[v].cpu().numpy(), t, rtol=1e-5)
        np.testing.assert_allclose(dc[3 * base:3 * (base + HW)].cpu().numpy(), gdc.reshape(-1), rtol=1e-6, atol=1e-12)
        np.testing.assert_allclose(dd[base:base + HW].cpu().numpy(), gdd.reshape(-1), rtol=1e-6, atol=1e-12)
        base += HW


# ------------------------------------------------------------------ backward

def _oracle_targets(gt, cams, params):
    prm = prm_dict(params)
    out = []
    for c in cams:
        img = oracle.render_fwd(oracle.project(gt, c, prm), c, prm)
        out.append((f32(img["color"]), f32(img["depth"])))
    return out


@pytest.mark.parametrize("sh", [0, 3])
def test_render_bwd_stagewise_matches_oracle(sh):
    g, gt, cam = _problem(3)
    if sh:
        rng = np.random.default_rng(5)
        g = synth.GaussianMap(g.mean, g.quat, g.log_scale, g.opacity_logit,
                              synth.sh3_from_rgb(g.color.astype(np.float64), rng).astype(np.float32))
    params = G.RenderParams(sh_degree=sh)
    prm = prm_dict(params)
    cams = [cam]
    prs = _stage_inputs(g, cams, params)
    proj = projected_to_device(prs)
    m = int(sum(p["tiles"].sum() for p in prs))
    bins, ws, img = _gpu_forward(proj, g.n, cams, params, m)
    rng = np.random.default_rng(9)
    # image gradients of a generic linear functional (no L1 kinks)
    dcol = [rng.standard_normal((3, c.height, c.width)) * 1e-3 for c in cams]
    ddep = [rng.standard_normal((c.height, c.width)) * 1e-3 for c in cams]
    dc, dd = pack_images(dcol, ddep)
    gd = G.Gaussians.from_numpy(g)
    grads = G.Grads.empty_like(gd, len(cams))
    iso = torch.zeros(1, device="cuda")
    G.gs_render_bwd(gd, proj, bins, img, dc, dd, cams, params, 0.0, grads, iso, ws)
    torch.cuda.synchronize()
    g2d_gpu = ws[: g.n * len(cams) * 12].view(-1, 12).cpu().numpy().astype(np.float64)
    ref2d = oracle.render_bwd(prs[0], cam, prm, f32(dcol[0]), f32(ddep[0]))
    # diagnostic: per-entry 2D gradients before the projection chain rule
    assert rel_l2(g2d_gpu[:, 0:2], ref2d["xy"]) < GRAD_RTOL
    assert rel_l2(g2d_gpu[:, 2:5], ref2d["conic"]) < GRAD_RTOL
    assert rel_l2(g2d_gpu[:, 5], ref2d["opacity"]) < GRAD_RTOL
    assert rel_l2(g2d_gpu[:, 6], ref2d["depth"]) < GRAD_RTOL
    assert rel_l2(g2d_gpu[:, 8:11], ref2d["rgb"]) < GRAD_RTOL
    ref = oracle.project_bwd(g, cam, prm, ref2d)
    got = grads_to_numpy(grads)
    for k in oracle.PARAM_NAMES:
        assert rel_l2(got[k], ref[k]) < GRAD_RTOL, k
    assert rel_l2(got["pose"][0], ref["pose"]) < GRAD_RTOL


@pytest.mark.parametrize("masks", [1, 0])
@pytest.mark.parametrize("tile", [8, 16, 32])
def test_render_bwd_deep_lists(tile, masks):
    # Thousands of faint, wide splats over the 64x48 case: front-to-back lists
    # of more than 2048 blending splats per pixel (the transmittance reaches its
    # cutoff only after thousands of splats; many batches of the backward's walk
    # per pixel block, each with every lane blending); colour, depth and the
    # gradients still equal the oracle's.
    g, _, cam = _problem(2)
    faint = synth.random_cloud(3000, 21, box=((-0.8, 0.8), (-0.6, 0.6), (1.5, 3.0)), log_scale_mu=-0.8,
                               log_scale_sd=0.2)
    faint = synth.GaussianMap(faint.mean, faint.quat, faint.log_scale,
                              np.full(faint.n, -6.0, np.float32), faint.color)
    both = synth.GaussianMap(*(np.concatenate([b, a]) for a, b in zip(g.arrays(), faint.arrays())))
    params = G.RenderParams(tile=tile, block_masks=masks)
    prm = prm_dict(params)
    prs = _stage_inputs(both, [cam], params)
    proj = projected_to_device(prs)
    bins, ws, img = _gpu_forward(proj, both.n, [cam], params, int(prs[0]["tiles"].sum()))
    ref_img = oracle.render_fwd(prs[0], cam, prm)
    assert _compare_images(image_views(img, [cam])[0], ref_img) < 20
    assert int(img.n_contrib.max()) > 2048
    rng = np.random.default_rng(17)
    dcol = rng.standard_normal((3, cam.height, cam.width)) * 1e-3
    ddep = rng.standard_normal((cam.height, cam.width)) * 1e-3
    dc, dd = pack_images([dcol], [ddep])
    gd = G.Gaussians.from_numpy(both)
    grads = G.Grads.empty_like(gd, 1)
    iso = torch.zeros(1, device="cuda")
    G.gs_render_bwd(gd, proj, bins, img, dc, dd, [cam], params, 0.0, grads, iso, ws)
    torch.cuda.synchronize()
    g2d_gpu = ws[: both.n * 12].view(-1, 12).cpu().numpy().astype(np.float64)
    ref2d = oracle.render_bwd(prs[0], cam, prm, f32(dcol), f32(ddep))
    assert rel_l2(g2d_gpu[:, 0:2], ref2d["xy"]) < GRAD_RTOL
    assert rel_l2(g2d_gpu[:, 2:5], ref2d["conic"]) < GRAD_RTOL
    assert rel_l2(g2d_gpu[:, 5], ref2d["opacity"]) < GRAD_RTOL
    assert rel_l2(g2d_gpu[:, 6], ref2d["depth"]) < GRAD_RTOL
    assert rel_l2(g2d_gpu[:, 8:11], ref2d["rgb"]) < GRAD_RTOL
    ref = oracle.project_bwd(both, cam, prm, ref2d)
    got = grads_to_numpy(grads)
    for k in oracle.PARAM_NAMES:
        assert rel_l2(got[k], ref[k]) < GRAD_RTOL, k
    assert rel_l2(got["pose"][0], ref["pose"]) < GRAD_RTOL


@pytest.mark.parametrize("masks", [1, 0])
@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("lambdas", [(1.0, 1.0, 0.0), (0.9, 0.1, 10.0)])
def test_full_iteration_end_to_end_matches_oracle(lambdas, fused, masks):
    from paper_2512_02293_gb300.mapping import MapParams, MappingStep
    g, gt, cam = _problem(0)
    params = G.RenderParams(block_masks=masks)
    cams = [cam]
    targets = _oracle_targets(gt, cams, params)
    tc, td = pack_images([t[0] for t in targets], [t[1] for t in targets])
    mp = MapParams(lambda_c=lambdas[0], lambda_d=lambdas[1], lambda_iso=lambdas[2])
    step = MappingStep(G.Gaussians.from_numpy(g), cams, tc, td, params, mp, fused_loss=fused)
    step.render()
    step.loss_and_backward()
    torch.cuda.synchronize()
    ref = oracle.mapping_loss_and_grads(g, cams, targets, prm_dict(params), lambdas)
    assert _compare_images(image_views(step.img, cams)[0], ref.images[0]) == 0
    np.testing.assert_allclose(step.loss_terms.cpu().numpy()[0], ref.loss_terms[0], rtol=1e-5)
    if lambdas[2]:
        assert step.iso.item() == pytest.approx(ref.iso, rel=1e-5)
    got = grads_to_numpy(step.grads)
    for k in oracle.PARAM_NAMES:
        assert rel_l2(got[k], ref.grads[k]) < GRAD_RTOL, k
    assert rel_l2(got["pose"][0], ref.pose_grads[0]) < GRAD_RTOL


def test_fused_loss_matches_separate_calls():
    # gs_render_fwd_loss + gs_render_bwd_raster_loss against gs_render_fwd +
    # gs_loss + gs_render_bwd_raster on two views whose depth targets are partly
    # invalid (D <= 0): identical images, loss terms to fp32 summation order,
    # gradients to atomic accumulation order
    from paper_2512_02293_gb300.mapping import MapParams, MappingStep
    g, gt, _ = _problem(4)
    R, e = synth.look_at([0.3, 0.2, -0.2], [0.0, 0.0, 2.0])
    cams = [synth.Camera(60.0, 60.0, 32.0, 24.0, 64, 48), synth.Camera(45.0, 45.0, 20.0, 15.0, 40, 30, R, e)]
    params = G.RenderParams()
    targets = _oracle_targets(gt, cams, params)
    tds = []
    for k, (_, d) in enumerate(targets):
        d = np.array(d, copy=True)
        d.reshape(-1)[k::3] = 0.0                  # a third of the depth targets invalid
        tds.append(d)
    tc, td = pack_images([t[0] for t in targets], tds)
    mp = MapParams(0.9, 0.1, 10.0)
    steps = [MappingStep(G.Gaussians.from_numpy(g), cams, tc, td, params, mp, fused_loss=f) for f in (True, False)]
    for st in steps:
        st.render()
        st.loss_and_backward()
    torch.cuda.synchronize()
    a, b = steps
    assert torch.equal(a.img.color, b.img.color) and torch.equal(a.img.n_contrib, b.img.n_contrib)
    assert int(a.bins.status[3].item()) == 0                      # the fused forward's ticket is back at zero
    np.testing.assert_allclose(a.loss_terms.cpu().numpy(), b.loss_terms.cpu().numpy(), rtol=2e-6)
    ga, gb = grads_to_numpy(a.grads), grads_to_numpy(b.grads)
    for k in oracle.PARAM_NAMES:
        assert rel_l2(ga[k], gb[k]) < 1e-5, k
    for v in range(2):
        assert rel_l2(ga["pose"][v], gb["pose"][v]) < 1e-5
    ref = oracle.mapping_loss_and_grads(g, cams, [(t[0], d) for t, d in zip(targets, tds)], prm_dict(params),
                                        (0.9, 0.1, 10.0))
    np.testing.assert_allclose(a.loss_terms.cpu().numpy(), np.asarray(ref.loss_terms), rtol=1e-5)
    for k in oracle.PARAM_NAMES:
        assert rel_l2(ga[k], ref.grads[k]) < GRAD_RTOL, k


def test_native_mapping_step_matches_the_six_calls():
    # gs_mapping_step (one C call, the eager MappingStep.step) against its six
    # calls issued one by one on an identical map
    from paper_2512_02293_gb300.mapping import MapParams, MappingStep
    g, gt, cam = _problem(3)
    params = G.RenderParams()
    targets = _oracle_targets(gt, [cam], params)
    tc, td = pack_images([targets[0][0]], [targets[0][1]])
    mp = MapParams(0.9, 0.1, 10.0)
    a, b = (MappingStep(G.Gaussians.from_numpy(g), [cam], tc, td, params, mp) for _ in range(2))
    assert [c.name for c in a._bound_calls()] == ["gs_mapping_step"]
    a.step()
    b.render(); b.loss_and_backward(); b.optimizer_step()
    torch.cuda.synchronize()
    assert a.check() == 0 and b.check() == 0
    assert torch.equal(a.img.color, b.img.color) and torch.equal(a.img.n_contrib, b.img.n_contrib)
    np.testing.assert_allclose(a.loss_terms.cpu().numpy(), b.loss_terms.cpu().numpy(), rtol=2e-6)
    ga, gb = grads_to_numpy(a.grads), grads_to_numpy(b.grads)
    for k in oracle.PARAM_NAMES:
        assert rel_l2(ga[k], gb[k]) < 1e-5, k
    assert int(a.d_step[0].item()) == 1 and int(b.d_step[0].item()) == 1


def test_repeated_launches_leave_work_counters_zero():
    # the persistent rasterisers' work counters are returned to zero by the last
    # warp of each launch (no reset on the stream): eager calls and graph replays
    # of the step reproduce the first result bit for bit and leave them zero
    from paper_2512_02293_gb300.mapping import MapParams, MappingStep
    g, gt, cam = _problem(1)
    params = G.RenderParams()
    targets = _oracle_targets(gt, [cam], params)
    tc, td = pack_images([targets[0][0]], [targets[0][1]])
    # zero learning rates: the graph's Adam step leaves the map as it is
    mp = MapParams(0.9, 0.1, 10.0, lr=(0.0,) * 5)
    step = MappingStep(G.Gaussians.from_numpy(g), [cam], tc, td, params, mp)
    outs = []
    for k in range(4):
        if k == 2:
            step.capture(warmup=0)
        if k >= 2:
            step.step()                      # graph replay: project ... Adam
        else:
            step.render()
            step.loss_and_backward()
        torch.cuda.synchronize()
        assert step.bins.status[1:].cpu().tolist() == [0, 0, 0]
        outs.append((step.img.color.clone(), step.img.n_contrib.clone(), step.grads.mean.clone()))
    for c, n, gm in outs[1:]:
        assert torch.equal(c, outs[0][0]) and torch.equal(n, outs[0][1])
    # gradient accumulation order is not fixed (atomics): equal to fp32 rounding
    for _, _, gm in outs[1:]:
        assert rel_l2(gm.cpu().numpy(), outs[0][2].cpu().numpy()) < 1e-5


def test_capture_with_host_copies():
    # MappingStep.capture(host_io=...): each replay copies the pinned host targets
    # in and the loss terms out, inside the graph
    from paper_2512_02293_gb300.mapping import MapParams, MappingStep
    g, gt, cam = _problem(2)
    params = G.RenderParams()
    targets = _oracle_targets(gt, [cam], params)
    tc, td = pack_images([targets[0][0]], [targets[0][1]])
    step = MappingStep(G.Gaussians.from_numpy(g), [cam], torch.zeros_like(tc), torch.zeros_like(td), params,
                       MapParams(0.9, 0.1, 10.0, lr=(0.0,) * 5))
    h = (tc.cpu().pin_memory(), td.cpu().pin_memory(), torch.empty(1, 2).pin_memory(), torch.empty(1).pin_memory())
    step.capture(warmup=0, host_io=h)
    step.step()
    torch.cuda.synchronize()
    assert torch.equal(step.target_color.cpu(), h[0]) and torch.equal(step.target_depth.cpu(), h[1])
    assert torch.equal(h[2], step.loss_terms.cpu()) and torch.equal(h[3], step.iso.cpu())
    first = h[2].clone()
    ref = oracle.mapping_loss_and_grads(g, [cam], targets, prm_dict(params), (0.9, 0.1, 10.0))
    np.testing.assert_allclose(first.numpy()[0], ref.loss_terms[0], rtol=1e-5)
    h[0].mul_(0.5)                           # a new target in the host buffer reaches the next replay
    step.step()
    torch.cuda.synchronize()
    assert torch.equal(step.target_color.cpu(), h[0])
    assert torch.equal(h[2], step.loss_terms.cpu()) and h[2][0, 0] != first[0, 0]
    with pytest.raises(ValueError):
        step.capture(warmup=0, host_io=(tc, h[1], h[2], h[3]))       # not pinned host memory


def test_multiview_gradients_are_the_sum_of_single_views():
    from paper_2512_02293_gb300.mapping import MapParams, MappingStep
    g, gt, _ = _problem(4)
    R, e = synth.look_at([0.3, 0.2, -0.2], [0.0, 0.0, 2.0])
    cams = [synth.Camera(60.0, 60.0, 32.0, 24.0, 64, 48), synth.Camera(45.0, 45.0, 20.0, 15.0, 40, 30, R, e)]
    params = G.RenderParams()
    targets = _oracle_targets(gt, cams, params)
    tc, td = pack_images([t[0] for t in targets], [t[1] for t in targets])
    mp = MapParams(1.0, 1.0, 0.0)
    step = MappingStep(G.Gaussians.from_numpy(g), cams, tc, td, params, mp)
    step.render(); step.loss_and_backward()
    torch.cuda.synchronize()
    ref = oracle.mapping_loss_and_grads(g, cams, targets, prm_dict(params), (1.0, 1.0, 0.0))
    got = grads_to_numpy(step.grads)
    for k in oracle.PARAM_NAMES:
        assert rel_l2(got[k], ref.grads[k]) < GRAD_RTOL, k
    for v in range(2):
        assert rel_l2(got["pose"][v], ref.pose_grads[v]) < GRAD_RTOL
        assert _compare_images(image_views(step.img, cams)[v], ref.images[v]) == 0


# ------------------------------------------------------------------ Adam

def test_adam_matches_oracle():
    rng = np.random.default_rng(1)
    sizes = [1000, 37, 4003]            # includes non-multiple-of-4 tails
    lrs = [1e-3, 5e-2, 2e-3]
    b1, b2, eps = np.float32(0.9), np.float32(0.999), np.float32(1e-15)
    ps = [rng.standard_normal(s).astype(np.float32) for s in sizes]
    dev = [[torch.from_numpy(p.copy()).cuda(), None, torch.zeros(s, device="cuda"), torch.zeros(s, device="cuda"), lr]
           for p, s, lr in zip(ps, sizes, lrs)]
    ref = [[p.astype(np.float64), np.zeros(s), np.zeros(s)] for p, s in zip(ps, sizes)]
    d_step = torch.zeros(2, device="cuda", dtype=torch.int32)
    for step in range(1, 6):
        grads = [rng.standard_normal(s).astype(np.float32) * 10 ** rng.uniform(-6, 0) for s in sizes]
        for d, gr in zip(dev, grads):
            d[1] = torch.from_numpy(gr).cuda()
        G.gs_adam_step([tuple(d) for d in dev], b1, b2, eps, d_step)
        for r, gr, lr in zip(ref, grads, lrs):
            oracle.adam(r[0], gr, r[1], r[2], lr, float(b1), float(b2), float(eps), step)
        torch.cuda.synchronize()
        assert int(d_step[0].item()) == step and int(d_step[1].item()) == 0
        for d, r in zip(dev, ref):
            # fp32 moments: errors relative to the largest moment (m can cancel to ~0)
            np.testing.assert_allclose(d[0].cpu().numpy(), r[0], rtol=1e-6, atol=1e-7)
            np.testing.assert_allclose(d[2].cpu().numpy(), r[1], rtol=1e-5, atol=1e-6 * np.abs(r[1]).max())
            np.testing.assert_allclose(d[3].cpu().numpy(), r[2], rtol=1e-5, atol=1e-6 * np.abs(r[2]).max())


def test_l2_read_probe_reads_every_element_reps_times():
    """gs_l2_read_probe (the L2 roofline's denominator) reads the whole buffer
    `reps` times: the sum it adds is exactly reps * sum(buf) (0 / 1 values, every
    partial sum an integer below 2^24), for a length that runs the four-load
    loop and leaves a ragged tail in every CTA's share."""
    n = 152 * 8 * 256 * 4 * 4 + 44
    vals = (np.arange(n) % 2).astype(np.float32)
    buf = torch.from_numpy(vals).cuda()
    out = torch.zeros(1, device="cuda")
    G.gs_l2_read_probe(buf, 3, out)
    torch.cuda.synchronize()
    assert out.item() == 3.0 * float(vals.sum())
