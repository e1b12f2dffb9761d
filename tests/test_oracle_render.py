"""Pins of the oracle's binning and compositing (Sec. 3.3: pixel colour by
alpha blending of the visible Gaussians; colour and depth rendered per
keyframe).  The references here are closed forms, invariants, a library sort
and an independent numpy per-pixel renderer with no tiles or key machinery."""
import math

import numpy as np
import pytest

import oracle
from paper_2512_02293_gb300 import synth


def _single(mean, log_s, logit, color, quat=(1, 0, 0, 0)):
    f = lambda a: np.asarray(a, dtype=np.float32).reshape(len(mean), -1)
    return synth.GaussianMap(f(mean), f([quat] * len(mean)), f(log_s), np.asarray(logit, np.float32).reshape(-1), f(color))


# ------------------------------------------------------------------ binning

def test_bin_sort_matches_enumeration_and_library_sort():
    rng = np.random.default_rng(5)
    views = [(5, 3), (4, 4), (7, 2)]            # tiles_x, tiles_y per view
    tile_base = np.cumsum([0] + [a * b for a, b in views])[:-1].astype(np.int32)
    total = int(sum(a * b for a, b in views))
    E = 300
    view_of = rng.integers(0, 3, E).astype(np.int32)
    depth = rng.uniform(0.3, 5.0, E).astype(np.float32)
    depth[::7] = depth[3]                        # ties broken by entry index
    rect = np.zeros((E, 4), np.int32)
    for e in range(E):
        tx, ty = views[view_of[e]]
        if rng.random() < 0.1:
            continue                             # culled entry: empty rectangle
        x0 = rng.integers(0, tx); y0 = rng.integers(0, ty)
        rect[e] = [x0, y0, rng.integers(x0 + 1, tx + 1), rng.integers(y0 + 1, ty + 1)]
    keys, vals, ranges = oracle.bin_sort(depth, rect, view_of, tile_base, [v[0] for v in views], total)
    pairs = []
    for e in range(E):
        v = view_of[e]
        for y in range(rect[e, 1], rect[e, 3]):
            for x in range(rect[e, 0], rect[e, 2]):
                g = int(tile_base[v]) + y * views[v][0] + x
                pairs.append((g, float(depth[e]), e))
    pairs.sort()                                   # (tile, depth, entry) -- library sort
    assert len(keys) == len(pairs)
    np.testing.assert_array_equal(vals, [p[2] for p in pairs])
    zb = depth.view(np.uint32)
    np.testing.assert_array_equal(keys, [(np.uint64(p[0]) << np.uint64(32)) | np.uint64(zb[p[2]]) for p in pairs])
    for g in range(total):
        idx = [k for k, p in enumerate(pairs) if p[0] == g]
        if idx:
            assert tuple(ranges[g]) == (idx[0], idx[-1] + 1)
        else:
            assert tuple(ranges[g]) == (0, 0)


def test_depth_bits_are_monotone():
    z = np.sort(np.random.default_rng(1).uniform(0.2, 100.0, 10000).astype(np.float32))
    assert np.all(np.diff(z.view(np.uint32).astype(np.int64)) >= 0)


# ------------------------------------------------------- compositing: closed forms

def test_single_isotropic_splat_closed_form():
    # One isotropic Gaussian on the optical axis; the principal point sits on a
    # pixel sample, so the centre pixel reads c * min(o, alpha_max) and the
    # footprint is c * o * exp(-r^2 / (2 sigma^2)), sigma^2 = (f s / z)^2 + dilation.
    cam = synth.identity_camera(64, 48, 60.0, 60.0, 32.5, 24.5)
    s, z, dil = 0.06, 2.0, 0.3
    for o, logit in ((0.7, math.log(0.7 / 0.3)), (0.995, math.log(0.995 / 0.005))):
        g = _single([[0, 0, z]], [[math.log(s)] * 3], [logit], [[0.2, 0.5, 0.9]])
        prm = dict(dilation=dil)
        img = oracle.render_fwd(oracle.project(g, cam, prm), cam, prm)
        o32 = 1 / (1 + math.exp(-float(np.float32(logit))))
        sig2 = (60.0 * math.exp(float(np.float32(math.log(s)))) / z) ** 2 + dil
        a0 = min(o32, 0.99)
        np.testing.assert_allclose(img["color"][:, 24, 32], np.array([0.2, 0.5, 0.9], np.float32) * a0, rtol=1e-6)
        assert img["depth"][24, 32] == pytest.approx(z * a0, rel=1e-6)
        for dx, dy in ((1, 0), (2, 1), (-3, 2), (0, -4)):
            a = o32 * math.exp(-(dx * dx + dy * dy) / (2 * sig2))
            a = min(a, 0.99)
            want = a if a >= 1 / 255 else 0.0
            assert img["color"][1, 24 + dy, 32 + dx] == pytest.approx(np.float32(0.5) * want, rel=1e-6, abs=1e-15)
            assert img["T_final"][24 + dy, 32 + dx] == pytest.approx(1 - want, rel=1e-9)


def test_transmittance_cutoff_semantics():
    # Stack of identical opaque splats at one pixel: alpha = 0.95 each, so
    # T = 0.05^k.  With T_cut = 1e-4 the 4th splat would take T to 6.25e-6 and
    # is not blended: n_contrib = 3, T_final = 0.05^3.
    cam = synth.identity_camera(16, 16, 60.0, 60.0, 8.5, 8.5)
    logit = math.log(0.95 / 0.05)
    k = 6
    g = _single([[0, 0, 1.0 + 0.1 * i] for i in range(k)], [[math.log(0.2)] * 3] * k, [logit] * k,
                [[1.0, 0.5, 0.25]] * k)
    prm = dict(T_cut=1e-4, alpha_max=0.999)
    pr = oracle.project(g, cam, prm)
    img = oracle.render_fwd(pr, cam, prm)
    o = 1 / (1 + math.exp(-float(np.float32(logit))))
    assert img["n_contrib"][8, 8] == 3
    assert img["T_final"][8, 8] == pytest.approx((1 - o) ** 3, rel=1e-12)
    want_c = sum(o * (1 - o) ** j for j in range(3))
    assert img["color"][0, 8, 8] == pytest.approx(want_c, rel=1e-12)
    want_d = sum(float(np.float32(1.0 + 0.1 * j)) * o * (1 - o) ** j for j in range(3))
    assert img["depth"][8, 8] == pytest.approx(want_d, rel=1e-6)


def test_partition_of_unity_and_constant_colour():
    g, _, cam = synth.cfg1_problem(1)
    g.color[:] = 0.6
    for bg in ((0.0, 0.0, 0.0), (0.6, 0.6, 0.6)):
        prm = dict(bg=bg)
        img = oracle.render_fwd(oracle.project(g, cam, prm), cam, prm)
        c = float(np.float32(0.6))
        T = img["T_final"][None]
        want = c * (1 - T) + bg[0] * T         # sum_i alpha_i T_i = 1 - T_final
        np.testing.assert_allclose(img["color"], np.broadcast_to(want, img["color"].shape), atol=1e-12)


def test_order_invariance_and_index_tie_break():
    g, _, cam = synth.cfg1_problem(2)
    prm = {}
    base = oracle.render_fwd(oracle.project(g, cam, prm), cam, prm)
    perm = np.random.default_rng(0).permutation(g.n)
    img = oracle.render_fwd(oracle.project(g.subset(perm), cam, prm), cam, prm)
    for k in ("color", "depth", "T_final"):
        np.testing.assert_allclose(img[k], base[k], atol=1e-12)
    np.testing.assert_array_equal(img["n_contrib"], base["n_contrib"])
    # Two splats at equal depth: the lower index is in front.
    cam1 = synth.identity_camera(16, 16, 60.0, 60.0, 8.5, 8.5)
    two = _single([[0, 0, 1.0], [0, 0, 1.0]], [[math.log(0.1)] * 3] * 2, [0.5, 0.5], [[1, 0, 0], [0, 1, 0]])
    a = oracle.render_fwd(oracle.project(two, cam1, prm), cam1, prm)
    b = oracle.render_fwd(oracle.project(two.subset([1, 0]), cam1, prm), cam1, prm)
    assert a["color"][0, 8, 8] > a["color"][1, 8, 8]     # red (index 0) in front
    assert b["color"][1, 8, 8] > b["color"][0, 8, 8]     # green now index 0


# ------------------------------------- compositing: an independent brute force

def _numpy_render(pr, cam, prm):
    """Per-pixel composite over ALL Gaussians sorted by (depth, index), with the
    same thresholds, a Gaussian counting for a pixel iff the pixel's tile lies
    in its rectangle.  No tile lists, no keys."""
    p = dict(oracle.DEFAULT_PARAMS, **prm)
    H, W, t = cam.height, cam.width, p["tile"]
    order = np.lexsort((np.arange(len(pr["depth"])), pr["depth"]))
    col = np.zeros((3, H, W)); dep = np.zeros((H, W)); Tf = np.ones((H, W)); nc = np.zeros((H, W), int)
    for py in range(H):
        for px in range(W):
            tx, ty = px // t, py // t
            T = 1.0; c = np.zeros(3); d = 0.0; last = -1; k = -1
            for i in order:
                x0, y0, x1, y1 = pr["rect"][i]
                if not (x0 <= tx < x1 and y0 <= ty < y1):
                    continue
                k += 1
                dx = px + 0.5 - pr["xy"][i, 0]; dy = py + 0.5 - pr["xy"][i, 1]
                A, B, C = pr["conic"][i]
                power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy
                if power > 0:
                    continue
                a = min(p["alpha_max"], pr["opacity"][i] * math.exp(power))
                if a < p["alpha_min"]:
                    continue
                if T * (1 - a) < p["T_cut"]:
                    break
                c += pr["rgb"][i] * a * T; d += pr["depth"][i] * a * T
                T *= 1 - a; last = k
            col[:, py, px] = c + T * np.asarray(p["bg"]); dep[py, px] = d; Tf[py, px] = T; nc[py, px] = last + 1
    return col, dep, Tf, nc


@pytest.mark.parametrize("trial", [0, 1])
def test_matches_numpy_brute_force(trial):
    g, _, _ = synth.cfg1_problem(trial)
    g = g.subset(np.arange(48))
    cam = synth.identity_camera(40, 24, 30.0, 30.0, 20.0, 12.0)
    prm = dict(tile=8, bg=(0.1, 0.2, 0.3))
    pr = oracle.project(g, cam, prm)
    img = oracle.render_fwd(pr, cam, prm)
    col, dep, Tf, nc = _numpy_render(pr, cam, prm)
    np.testing.assert_allclose(img["color"], col, atol=1e-12)
    np.testing.assert_allclose(img["depth"], dep, atol=1e-12)
    np.testing.assert_allclose(img["T_final"], Tf, atol=1e-12)
    np.testing.assert_array_equal(img["n_contrib"], nc)
    # transmittance product over the blended splats
    assert np.all(img["T_final"] > 0) and np.all(img["T_final"] <= 1)


def test_tile_list_equals_sorted_key_range():
    # The oracle's per-tile lists are the key ranges of its own bin_sort.
    g, _, cam = synth.cfg1_problem(4)
    prm = {}
    pr = oracle.project(g, cam, prm)
    tx, ty = oracle.tiles_of(cam, prm)
    keys, vals, ranges = oracle.bin_sort(pr["depth"].astype(np.float32), pr["rect"], np.zeros(g.n, np.int32),
                                         [0], [tx], tx * ty)
    for gt in range(tx * ty):
        x, y = gt % tx, gt // tx
        members = [i for i in range(g.n) if pr["rect"][i, 0] <= x < pr["rect"][i, 2] and pr["rect"][i, 1] <= y < pr["rect"][i, 3]]
        members.sort(key=lambda i: (np.float32(pr["depth"][i]), i))
        s, e = ranges[gt]
        assert list(vals[s:e]) == members
