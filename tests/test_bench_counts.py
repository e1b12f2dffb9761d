"""bench.py's count of the (pixel, splat) pairs the rasterisers evaluate
(`evaluated_pairs`), on CPU tensors built from the oracle's projection, bins
and forward pass of a small view.  It is checked against a brute force over a
fine grid of each pixel block's box of pixel centres: the exact test (the
maximum of the concave power over the box) keeps every pair the grid keeps,
and nothing the grid with a slightly lower threshold rejects."""
import os
import sys
import types

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_2512_02293_gb300 import synth  # noqa: E402


def _fake_step(tile):
    g, _, cam = synth.cfg1_problem(0)
    prm = dict(tile=tile)
    pr = oracle.project(g, cam, prm)
    img = oracle.render_fwd(pr, cam, prm)
    tx, ty = (cam.width + tile - 1) // tile, (cam.height + tile - 1) // tile
    keys, vals, ranges = oracle.bin_sort(pr["depth"].astype(np.float32), pr["rect"], np.zeros(g.n, np.int32),
                                         np.array([0], np.int32), np.array([tx], np.int32), tx * ty)
    st = types.SimpleNamespace(device=torch.device("cpu"), cams=[cam])
    st.params = types.SimpleNamespace(tile=tile, alpha_min=1.0 / 255.0)
    st.bins = types.SimpleNamespace(keys=torch.from_numpy(keys.view(np.int64).copy()),
                                    vals=torch.from_numpy(vals.view(np.int32).copy()),
                                    ranges=torch.from_numpy(ranges.view(np.int32).copy()), capacity=len(keys))
    st.num_keys = lambda: len(keys)
    co = np.concatenate([pr["conic"], pr["opacity"][:, None]], 1)
    st.proj = types.SimpleNamespace(xy=torch.from_numpy(pr["xy"].astype(np.float32)),
                                    conic_o=torch.from_numpy(co.astype(np.float32)))
    nc = img["n_contrib"].reshape(-1).astype(np.int32)
    st.img = types.SimpleNamespace(n_contrib=torch.from_numpy(nc))
    return st, keys, vals, ranges, st.proj.xy.double().numpy(), st.proj.conic_o.double().numpy(), \
        img["n_contrib"], tx


def _grid_count(tile, keys, vals, ranges, xy, co, nc, tx, amin, factor):
    """Pairs kept by a 57 x 25 grid over every block's box (threshold factor * amin)."""
    H, W = nc.shape
    bw = tile // 8
    nb = bw * (tile // 4)
    gx = np.linspace(0.0, 7.0, 57)
    gy = np.linspace(0.0, 3.0, 25)
    count = 0
    t_of = (keys >> np.uint64(32)).astype(np.int64)
    for k in range(len(keys)):
        t = int(t_of[k])
        pos = k - int(ranges[t, 0])
        e = int(vals[k])
        A, B, C, o = co[e]
        for b in range(nb):
            x0 = (t % tx) * tile + (b % bw) * 8
            y0 = (t // tx) * tile + (b // bw) * 4
            blk = nc[y0:min(y0 + 4, H), x0:min(x0 + 8, W)]
            if blk.size == 0 or pos >= blk.max():
                continue
            dx = x0 + 0.5 + gx[None, :] - xy[e, 0]
            dy = y0 + 0.5 + gy[:, None] - xy[e, 1]
            p = -0.5 * (A * dx * dx + 2 * B * dx * dy + C * dy * dy)
            if (o * np.exp(p)).max() >= factor * 0.99 * amin:
                count += 1
    return 32 * count


def test_evaluated_pairs_matches_a_grid_over_the_blocks():
    for tile in (8, 16):
        st, keys, vals, ranges, xy, co, nc, tx = _fake_step(tile)
        e = bench.evaluated_pairs(st)
        lo = _grid_count(tile, keys, vals, ranges, xy, co, nc, tx, 1.0 / 255.0, 1.0)
        hi = _grid_count(tile, keys, vals, ranges, xy, co, nc, tx, 1.0 / 255.0, 0.98)
        assert lo <= e <= hi, (tile, lo, e, hi)
        assert 0 < e < 32 * int(nc.sum())           # the culling keeps some pairs, not all
