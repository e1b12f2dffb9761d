"""Helpers shared by the GPU parity tests: marshal oracle results into the
library's device layouts and run the C-ABI calls.  Nothing here computes any
part of the method."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2512_02293_gb300 import build as B
from paper_2512_02293_gb300 import gs as G

COLOR_TOL = 1e-4       # absolute, rendered colour and depth
GRAD_RTOL = 1e-3       # relative L2, gradients
MARGIN_EXCUSE = 1e-5   # relative distance of a threshold decision that may flip between fp32 and fp64


def margin_excuse(cam) -> float:
    """Relative threshold margin within which fp32 may decide differently from
    fp64, for a view of this size: the projected mean carries ~1 ulp of its
    pixel coordinate (1.2e-7 x coordinate), and a splat's log-weight moves by up
    to ~2 per pixel of mean shift at its alpha_min contour, so the relative
    weight error reaches ~2.4e-7 x the largest coordinate (1e-5 floor)."""
    return max(MARGIN_EXCUSE, 2.4e-7 * max(int(cam.width), int(cam.height)))


def ensure_lib():
    B.build()
    return G.load_library()


def prm_dict(p: G.RenderParams) -> dict:
    return dict(tile=p.tile, near=p.near_plane, alpha_min=p.alpha_min, alpha_max=p.alpha_max, T_cut=p.T_cut,
                dilation=p.dilation, radius_sigma=p.radius_sigma, bg=tuple(p.bg), sh_degree=p.sh_degree)


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def round_projection(pr: dict) -> dict:
    """The oracle's projection rounded to fp32 (what the GPU stages consume)."""
    out = dict(pr)
    for k in ("xy", "conic", "depth", "opacity", "rgb"):
        out[k] = f32(pr[k])
    return out


def projected_to_device(prs: list[dict], device="cuda") -> G.Projected:
    """Concatenate per-view oracle projections (entry e = v * n + i) into a
    device gs_projected."""
    xy = np.concatenate([p["xy"] for p in prs]).astype(np.float32)
    co = np.concatenate([np.concatenate([p["conic"], p["opacity"][:, None]], 1) for p in prs]).astype(np.float32)
    cd = np.concatenate([np.concatenate([p["rgb"], p["depth"][:, None]], 1) for p in prs]).astype(np.float32)
    rect = np.concatenate([p["rect"] for p in prs]).astype(np.int32)
    rad = np.concatenate([p["radius"] for p in prs]).astype(np.int32)
    tt = np.concatenate([p["tiles"] for p in prs]).astype(np.int32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    return G.Projected(t(xy), t(co), t(cd), t(rect), t(rad), t(tt))


def view_layout(cams, tile):
    tiles_x = [(c.width + tile - 1) // tile for c in cams]
    tiles_y = [(c.height + tile - 1) // tile for c in cams]
    tile_base = np.cumsum([0] + [a * b for a, b in zip(tiles_x, tiles_y)])
    return np.array(tiles_x, np.int32), np.array(tile_base[:-1], np.int32), int(tile_base[-1])


def oracle_bins(prs: list[dict], cams, tile):
    tiles_x, tile_base, total = view_layout(cams, tile)
    n = prs[0]["xy"].shape[0]
    depth = np.concatenate([p["depth"] for p in prs]).astype(np.float32)
    rect = np.concatenate([p["rect"] for p in prs]).astype(np.int32)
    view_of = np.repeat(np.arange(len(prs), dtype=np.int32), n)
    return oracle.bin_sort(depth, rect, view_of, tile_base, tiles_x, total)


def run_bin_sort(proj: G.Projected, n, cams, params, capacity):
    total = G.gs_total_tiles(cams, params.tile)
    bins = G.Bins.empty(capacity, total)
    ws = torch.empty(G.gs_workspace_size(n, cams, params, capacity) // 4 + 64, device="cuda", dtype=torch.float32)
    G.gs_bin_sort(proj, n, cams, params, bins, ws)
    torch.cuda.synchronize()
    return bins, ws


def bins_to_numpy(bins: G.Bins):
    m = int(bins.num_keys.item()) & 0xFFFFFFFF
    keys = bins.keys[:m].cpu().numpy().view(np.uint64)
    vals = bins.vals[:m].cpu().numpy().view(np.uint32)
    ranges = bins.ranges.cpu().numpy().view(np.uint32)
    return keys, vals, ranges


def image_views(img: G.Image, cams):
    """Split the packed device image into per-view numpy dicts."""
    col = img.color.cpu().numpy(); dep = img.depth.cpu().numpy(); T = img.T_final.cpu().numpy()
    nc = img.n_contrib.cpu().numpy().view(np.uint32)
    out, base = [], 0
    for c in cams:
        W, H = c.width, c.height
        out.append(dict(color=col[3 * base:3 * (base + W * H)].reshape(3, H, W), depth=dep[base:base + W * H].reshape(H, W),
                        T_final=T[base:base + W * H].reshape(H, W), n_contrib=nc[base:base + W * H].reshape(H, W)))
        base += W * H
    return out


def pack_images(imgs_color, imgs_depth):
    c = np.concatenate([np.asarray(a, np.float32).reshape(-1) for a in imgs_color])
    d = np.concatenate([np.asarray(a, np.float32).reshape(-1) for a in imgs_depth])
    return torch.from_numpy(c).cuda(), torch.from_numpy(d).cuda()


def rel_l2(a, b):
    a = np.asarray(a, np.float64).reshape(-1); b = np.asarray(b, np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def grads_to_numpy(gr: G.Grads):
    d = {k: t.cpu().numpy().astype(np.float64) for k, t in zip(oracle.PARAM_NAMES, gr.tensors())}
    d["pose"] = gr.pose.cpu().numpy().astype(np.float64) if gr.pose is not None else None
    return d


def excused_pixels(crop_xywh, gpu_rect, oracle_rect, oracle_margin, tile, excuse=MARGIN_EXCUSE):
    """Pixels of a tile-aligned window that fp32 / fp64 rounding may
    legitimately change: threshold decisions within MARGIN_EXCUSE of their
    threshold, and every pixel of a tile where an entry's GPU and oracle tile
    rectangles differ (rounding-boundary radius or centre).  gpu_rect is the
    full view's [n, 4]; oracle_rect is relative to the window.  Returns the
    boolean mask [h, w] and the number of differing rectangles."""
    x0, y0, w, h = crop_xywh
    ex = oracle_margin < excuse
    tx0, ty0 = x0 // tile, y0 // tile
    tw, th = (w + tile - 1) // tile, (h + tile - 1) // tile
    g_rect = np.array(gpu_rect, copy=True)
    g_rect[:, [0, 2]] = np.clip(g_rect[:, [0, 2]] - tx0, 0, tw)
    g_rect[:, [1, 3]] = np.clip(g_rect[:, [1, 3]] - ty0, 0, th)
    g_rect[(g_rect[:, 2] <= g_rect[:, 0]) | (g_rect[:, 3] <= g_rect[:, 1])] = 0
    diff = np.nonzero(np.any(g_rect != oracle_rect, axis=1))[0]
    for i in diff:
        for rr in (g_rect[i], oracle_rect[i]):
            ex[rr[1] * tile:rr[3] * tile, rr[0] * tile:rr[2] * tile] = True
    return ex, len(diff)
