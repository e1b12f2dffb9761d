"""The oracle's host-thread loops (OpenMP) change nothing: a mapping iteration
run on one thread and on several gives bit-identical images, gradients, pose
gradients and Adam updates.  The parallel loops write disjoint outputs or add
their recorded contributions back in the serial order, so equality is exact."""
import numpy as np
import pytest

import oracle
from paper_2512_02293_gb300 import synth


def _iteration(g, cams, targets, prm, threads):
    prev = oracle.set_threads(threads)
    try:
        st = oracle.adam_state(g)
        res = oracle.mapping_iteration(g, cams, targets, prm, (0.9, 0.1, 10.0), (1e-3, 1e-3, 5e-3, 5e-2, 2.5e-3), st)
    finally:
        oracle.set_threads(prev)
    return res, st


def _targets(gt, cams, prm):
    out = []
    for c in cams:
        img = oracle.render_fwd(oracle.project(gt, c, prm), c, prm)
        out.append((img["color"], img["depth"]))
    return out


def _assert_identical(a, b):
    (ra, sa), (rb, sb) = a, b
    for k in oracle.PARAM_NAMES:
        np.testing.assert_array_equal(ra.grads[k], rb.grads[k], err_msg=k)
        np.testing.assert_array_equal(sa["params"][k], sb["params"][k], err_msg=k)
        np.testing.assert_array_equal(sa["m"][k], sb["m"][k])
        np.testing.assert_array_equal(sa["v"][k], sb["v"][k])
    np.testing.assert_array_equal(ra.pose_grads, rb.pose_grads)
    for ia, ib in zip(ra.images, rb.images):
        for key in ("color", "depth", "T_final", "n_contrib", "margin"):
            np.testing.assert_array_equal(ia[key], ib[key], err_msg=key)


@pytest.mark.parametrize("threads", [2, 5])
def test_threads_bit_identical_64x48(threads):
    g, gt, cam = synth.cfg1_problem(0)
    prm = dict(tile=16)
    tg = _targets(gt, [cam], prm)
    _assert_identical(_iteration(g, [cam], tg, prm, 1), _iteration(g, [cam], tg, prm, threads))


def test_threads_bit_identical_sh3_two_views_and_room_crop():
    # degree-3 SH colour on a 4k sub-sample of the 1M room, two 160x128 views
    g_full, _, cams = synth.cfg4_problem()
    cs = [synth.Camera(c.fx / 8, c.fy / 8, c.cx / 8, c.cy / 8, 160, 128, c.R_wc, c.t_wc) for c in cams[4:6]]
    prm = dict(tile=16, sh_degree=3)
    idx = np.sort(np.random.default_rng(3).choice(g_full.n, 4000, replace=False))
    g = g_full.subset(idx)
    gt = synth.perturb_map(g, 7)
    tg = _targets(gt, cs, prm)
    _assert_identical(_iteration(g, cs, tg, prm, 1), _iteration(g, cs, tg, prm, 3))
    # a 96x64 window of the 200k-Gaussian room at 640x480 (deep tile lists)
    g2, gt2, cam = synth.cfg2_problem()
    crop = synth.Camera(cam.fx, cam.fy, cam.cx - 288, cam.cy - 208, 96, 64, cam.R_wc, cam.t_wc)
    prm2 = dict(tile=16)
    tg2 = _targets(gt2, [crop], prm2)
    _assert_identical(_iteration(g2, [crop], tg2, prm2, 1), _iteration(g2, [crop], tg2, prm2, 4))
