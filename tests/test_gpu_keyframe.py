"""Keyframe insertion kernels (gs_extract_patches, gs_insert_gaussians) against
the FP64 keyframe oracle."""
import numpy as np
import pytest
import torch

from oracle import keyframe as K
from paper_2512_02293_gb300 import gs as G
from paper_2512_02293_gb300 import synth
from gpu_common import ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _keyframe(seed=0, W=64, H=48):
    R, e = synth.look_at([0.2, -0.1, 0.3], [1.0, 1.5, 4.0])
    cam = synth.Camera(60.0, 58.0, W / 2, H / 2, W, H, R, e)
    rng = np.random.default_rng(seed)
    color = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    yy, xx = np.mgrid[0:H, 0:W]
    depth = (2.0 + 0.02 * xx - 0.01 * yy + 0.05 * rng.standard_normal((H, W))).astype(np.float32)
    depth[5, 7] = 0.0                                   # a pixel without depth
    uv = np.stack([rng.integers(0, W, 300), rng.integers(0, H, 300)], 1).astype(np.int32)
    uv[:4] = [[0, 0], [W - 1, H - 1], [7, 5], [8, 5]]   # corners, the hole, next to the hole
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return cam, color, depth, uv, dev(color.reshape(-1)), dev(depth.reshape(-1)), dev(uv)


def test_patches_match_oracle():
    cam, color, depth, uv, c, d, u = _keyframe()
    X = torch.empty(uv.shape[0], 208, device="cuda", dtype=torch.bfloat16)
    st = torch.zeros(4, device="cuda", dtype=torch.int32)
    G.gs_extract_patches(c, d, cam, u, X, status=st)
    torch.cuda.synchronize()
    assert int(st[0].item()) == 0
    got = X.float().cpu().numpy()
    ref = K.extract_patches(color, depth, cam, uv)
    rgb = np.zeros(208, bool); rgb[np.arange(196)[np.arange(196) % 4 != 3]] = True
    np.testing.assert_array_equal(got[:, rgb], ref[:, rgb])              # colour: exact BF16 conversions
    np.testing.assert_array_equal(got[:, 196:], ref[:, 196:])
    dz = ~rgb; dz[196:] = False
    diff = got[:, dz] != ref[:, dz]                                       # depth features: FP32 vs FP64
    assert diff.mean() < 0.01
    np.testing.assert_allclose(got[:, dz], ref[:, dz], rtol=2 ** -7, atol=1e-6)


@pytest.mark.parametrize("learned", [False, True])
@pytest.mark.parametrize("sh", [0, 3])
def test_insertion_matches_oracle(learned, sh):
    cam, color, depth, uv, c, d, u = _keyframe(1)
    n = uv.shape[0]
    off = 17
    cap = n + off + 5
    ncol = 48 if sh == 3 else 3
    g = G.Gaussians(torch.full((cap, 3), 9.0, device="cuda"), torch.full((cap, 4), 9.0, device="cuda"),
                    torch.full((cap, 3), 9.0, device="cuda"), torch.full((cap,), 9.0, device="cuda"),
                    torch.full((cap, ncol), 9.0, device="cuda"))
    Y = np.random.default_rng(2).standard_normal((n, 8)).astype(np.float32) if learned else None
    G.gs_insert_gaussians(c, d, cam, u, 2.5, g, off, Y=torch.from_numpy(Y).cuda() if learned else None,
                          sh_degree=sh)
    torch.cuda.synchronize()
    ref = K.insert(color, depth, cam, uv, 2.5, Y=Y, sh_degree=sh)
    rows = slice(off, off + n)
    np.testing.assert_allclose(g.mean[rows].cpu().numpy(), ref["mean"], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(g.log_scale[rows].cpu().numpy(), ref["log_scale"], rtol=1e-5, atol=1e-5)
    q = g.quat[rows].cpu().numpy().astype(np.float64)
    sign = np.sign(np.sum(q * ref["quat"], 1))[:, None]                  # q and -q are one rotation
    np.testing.assert_allclose(q * sign, ref["quat"], atol=2e-6)
    np.testing.assert_array_equal(g.opacity_logit[rows].cpu().numpy(), ref["logit"].astype(np.float32))
    np.testing.assert_allclose(g.color[rows].cpu().numpy(), ref["color"], rtol=1e-6, atol=1e-6)
    # rows outside [off, off + n) untouched
    assert torch.all(g.mean[:off] == 9.0) and torch.all(g.mean[off + n:] == 9.0)


def test_out_of_image_samples_are_reported():
    cam, color, depth, uv, c, d, u = _keyframe(3)
    bad = torch.tensor([[cam.width, 0], [0, -1]], dtype=torch.int32, device="cuda")
    X = torch.empty(2, 208, device="cuda", dtype=torch.bfloat16)
    st = torch.zeros(4, device="cuda", dtype=torch.int32)
    G.gs_extract_patches(c, d, cam, bad, X, status=st)
    assert G.gs_read_device_status(st) == G.GS_ERR_INVALID_ARG
    assert torch.all(X.float() == 0)
