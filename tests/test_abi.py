"""The C-ABI library builds, loads and exports every entry point include/gs.h
declares; host-side argument checks answer without a GPU (no compute call is
made here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2512_02293_gb300 import build as B
from paper_2512_02293_gb300 import gs as G
from paper_2512_02293_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return G.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "gs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(gs_[a-z_0-9]+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12, names
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(names) == sorted(G.EXPORTS)


def test_abi_version_and_status_strings(lib):
    assert lib.gs_abi_version() == 6
    assert lib.gs_status_string(0) == b"GS_OK"
    assert lib.gs_status_string(2) == b"GS_ERR_CAPACITY"
    assert lib.gs_status_string(99) == b"GS_ERR_UNKNOWN"


def test_struct_sizes_match_header_layout():
    assert ctypes.sizeof(G.gs_camera) == 4 * 4 + 2 * 4 + 9 * 4 + 3 * 4
    assert ctypes.sizeof(G.gs_render_params) == 4 * 14
    assert ctypes.sizeof(G.gs_gaussians) == 6 * 8
    assert ctypes.sizeof(G.gs_bins) == 7 * 8
    assert ctypes.sizeof(G.gs_adam_group) == 4 * 8 + 8 + 8
    # 11 pointers, (ws, bytes), (loss_ws, bytes), 2 pointers, 2 int32, 6 floats
    assert ctypes.sizeof(G.gs_mapping_step_args) == 11 * 8 + 2 * 16 + 2 * 8 + 2 * 4 + 6 * 4


def test_tiles_pixels_workspace_host_only(lib):
    cams = [synth.identity_camera(64, 48), synth.identity_camera(70, 45)]
    assert G.gs_total_tiles(cams, 16) == 4 * 3 + 5 * 3
    assert G.gs_total_tiles(cams, 8) == 8 * 6 + 9 * 6
    assert G.gs_total_pixels(cams) == 64 * 48 + 70 * 45
    ws = G.gs_workspace_size(256, cams, G.RenderParams(), 4096)
    assert ws >= max(4096 * 8, 2 * 256 * 48) and ws % 256 == 0   # segment keys; backward scratch
    with pytest.raises(G.GsError):
        G.gs_total_tiles(cams, 12)          # unsupported tile size
    with pytest.raises(G.GsError):
        G.gs_workspace_size(-1, cams, G.RenderParams(), 10)


def test_invalid_arguments_are_rejected_before_any_launch(lib):
    # NULL pointers and bad parameters come back as GS_ERR_INVALID_ARG without
    # touching the device.
    cams = G.camera_array([synth.identity_camera()])
    p = G.RenderParams().struct()
    g = G.gs_gaussians(None, None, None, None, None, 10)
    out = G.gs_projected()
    assert lib.gs_project(ctypes.byref(g), cams, 1, ctypes.byref(p), ctypes.byref(out), None) == 1
    bad = G.RenderParams(tile=12).struct()
    g0 = G.gs_gaussians(None, None, None, None, None, 0)
    assert lib.gs_project(ctypes.byref(g0), cams, 1, ctypes.byref(bad), ctypes.byref(out), None) == 1
    assert lib.gs_project(ctypes.byref(g0), cams, 0, ctypes.byref(p), ctypes.byref(out), None) == 1
    assert lib.gs_project(ctypes.byref(g0), cams, 33, ctypes.byref(p), ctypes.byref(out), None) == 1
    assert lib.gs_adam_step(None, 1, 0.9, 0.999, 1e-15, None, None) == 1
    grp = (G.gs_adam_group * 1)()
    assert lib.gs_adam_step(grp, 9, 0.9, 0.999, 1e-15, ctypes.c_void_p(16), None) == 1
    assert lib.gs_read_device_status(None, None, None) == 1
    bins = G.gs_bins()
    assert lib.gs_bin_sort(None, 0, cams, 1, ctypes.byref(p), ctypes.byref(bins), None, 0, None) == 1
    nan_cam = G.camera_array([synth.Camera(float("nan"), 60.0, 32.0, 24.0, 64, 48)])
    assert lib.gs_total_tiles(nan_cam, 1, 16) == -1


def test_mlp_entry_points_reject_bad_arguments(lib):
    # host checks of the learned-initialiser calls; nothing reaches the device
    V = ctypes.c_void_p
    q = G.gs_mlp_packed(V(256), V(512), V(768), V(1024), V(2048), V(4096))
    qbad = G.gs_mlp_packed(V(256), V(512), V(770), V(1024), V(2048), V(4096))   # misaligned W3a
    assert lib.gs_mlp_pack(None, ctypes.byref(q), None) == 1
    assert lib.gs_mlp_fwd(None, V(256), 4, None, None, None, None, None, None, 0.0, None, None) == 1
    assert lib.gs_mlp_fwd(ctypes.byref(qbad), V(256), 4, None, None, None, None, None, None, 0.0, None, None) == 1
    assert lib.gs_mlp_fwd(ctypes.byref(q), V(256), -1, None, None, None, None, None, None, 0.0, None, None) == 1
    assert lib.gs_mlp_fwd(ctypes.byref(q), None, 4, None, None, None, None, None, None, 0.0, None, None) == 1
    assert lib.gs_mlp_fwd(ctypes.byref(q), V(256), 4, None, V(256), None, None, None, None, 0.0, None, None) == 1
    assert lib.gs_mlp_fwd(ctypes.byref(q), V(256), 4, None, None, None, V(256), None, None, 0.0, None, None) == 1
    assert lib.gs_mlp_fwd(ctypes.byref(q), V(258), 4, None, None, None, None, None, None, 0.0, None, None) == 1
    g = G.gs_mlp_grads(V(256), V(256), V(256), V(256), V(256), None)
    assert lib.gs_mlp_bwd(ctypes.byref(q), V(256), V(256), V(256), V(256), 4, ctypes.byref(g), None, None) == 1
    assert lib.gs_mlp_bwd(ctypes.byref(q), V(256), V(256), V(256), V(256), 4, None, None, None) == 1


def test_fused_loss_and_inertial_arguments_rejected_on_the_host(lib):
    # the fused-loss calls and the inertial factor of gs_ba_step check their
    # arguments before any launch
    V = ctypes.c_void_p
    assert lib.gs_fused_loss_workspace_size(0) == 0
    assert lib.gs_fused_loss_workspace_size(G.GS_MAX_VIEWS + 1) == 0
    one, two = lib.gs_fused_loss_workspace_size(1), lib.gs_fused_loss_workspace_size(2)
    assert 0 < one < two
    cams = G.camera_array([synth.identity_camera()])
    p = G.RenderParams().struct()
    assert lib.gs_render_fwd_loss(None, None, cams, 1, ctypes.byref(p), None, V(256), V(256), V(256), V(256),
                                  one, None) == 1
    assert lib.gs_render_bwd_raster_loss(None, None, None, V(256), V(256), 0.9, 0.1, V(256), one, cams, 1,
                                         ctypes.byref(p), 10, V(256), None) == 1
    # inertial factor: records without velocities, and 16 free keyframes
    pr = G.gs_ba_problem(V(256), V(256), V(256), V(256), V(256), V(256), 17, 0, 4, 4, 1, 20.0, 20.0, 2.0, 2.0,
                         V(256))
    pr.imu = V(256)
    assert lib.gs_ba_step(ctypes.byref(pr), 1e-3, 1e-3, V(256), V(256), 1 << 30, None) == 1
    pr.vel, pr.bias, pr.bias_hat = V(256), V(256), V(256)
    assert lib.gs_ba_step(ctypes.byref(pr), 1e-3, 1e-3, V(256), V(256), 1 << 30, None) == 6   # unsupported
    pr.gravity[2] = float("nan")
    assert lib.gs_ba_step(ctypes.byref(pr), 1e-3, 1e-3, V(256), V(256), 1 << 30, None) == 1
    # workspace sizes grow with the inertial unknowns (15 instead of 6 per free keyframe)
    assert lib.gs_ba_workspace_size(8, 10, 4, 4, 1, 1) > lib.gs_ba_workspace_size(8, 10, 4, 4, 1, 0)


def test_mapping_step_rejects_missing_arguments(lib):
    assert lib.gs_mapping_step(None, None) == 1
    a = G.gs_mapping_step_args()
    assert lib.gs_mapping_step(ctypes.byref(a), None) == 1          # no Gaussians, bins or workspace
    g = G.gs_gaussians(None, None, None, None, None, 10)
    bins = G.gs_bins()
    a.gaussians = ctypes.addressof(g)
    a.bins = ctypes.addressof(bins)
    a.ws = 256
    assert lib.gs_mapping_step(ctypes.byref(a), None) == 1          # the projection's checks reject NULL arrays


def test_mapping_step_rejects_a_workspace_smaller_than_gs_workspace_size(lib):
    # The whole-iteration call reuses its workspace as the backward's 2D-gradient
    # scratch (48 B per entry), which can be larger than what the sort alone
    # needs; a buffer of exactly the sort's size must be refused before any launch.
    V = ctypes.c_void_p
    cam = synth.identity_camera(64, 48)
    cams = G.camera_array([cam])
    p = G.RenderParams().struct()
    n, cap = 4096, 1024                               # few keys per entry: the scratch dominates
    need = lib.gs_workspace_size(n, 1, cams, ctypes.byref(p), cap)
    sort_only = lib.gs_workspace_size(0, 1, cams, ctypes.byref(p), cap)
    assert need >= 12 * 4 * n > sort_only
    g = G.gs_gaussians(V(256), V(256), V(256), V(256), V(256), n)
    bins = G.gs_bins(V(256), V(256), cap, V(256), V(256), V(256), V(256))
    a = G.gs_mapping_step_args()
    a.gaussians = ctypes.addressof(g)
    a.cams = ctypes.addressof(cams)
    a.params = ctypes.addressof(p)
    a.bins = ctypes.addressof(bins)
    a.n_views = 1
    a.ws = 256
    for size in (sort_only, need - 256):
        a.ws_bytes = size
        assert lib.gs_mapping_step(ctypes.byref(a), None) == G.GS_ERR_INVALID_ARG, size
    a.ws, a.ws_bytes = 257, need                      # misaligned
    assert lib.gs_mapping_step(ctypes.byref(a), None) == G.GS_ERR_INVALID_ARG


def test_noalloc_loss_view_limit_is_checked_on_the_host(lib):
    V = ctypes.c_void_p
    n = G.GS_NOALLOC_LOSS_MAX_VIEWS + 1
    cams = G.camera_array([synth.identity_camera(8, 8)] * n)
    im = G.gs_image(V(256), V(256), V(256), V(256))
    assert lib.gs_loss_noalloc(ctypes.byref(im), V(256), V(256), cams, n, 1.0, 1.0, V(256), V(256), V(256),
                               None) == G.GS_ERR_INVALID_ARG


def test_mlp_wait_poll_limit_is_set_and_restored(lib):
    prev = G.gs_mlp_set_wait_polls(0)
    try:
        assert prev == G.MLP_WAIT_POLLS_DEFAULT
        assert G.gs_mlp_set_wait_polls(7) == 0
        assert lib.gs_mlp_set_wait_polls(1 << 33) == -1          # out of range: unchanged
        assert G.gs_mlp_set_wait_polls(-1) == 7                  # negative: back to the default
        assert G.gs_mlp_set_wait_polls(-1) == G.MLP_WAIT_POLLS_DEFAULT
    finally:
        G.gs_mlp_set_wait_polls(-1)


def test_splat_stages_parameter_is_checked(lib):
    # 0 (the library's choice), 2 or 3 batches of 32 splats per forward warp; anything else is refused
    cams = G.camera_array([synth.identity_camera()])
    g0 = G.gs_gaussians(None, None, None, None, None, 0)
    out = G.gs_projected()
    for st, want in ((0, 0), (2, 0), (3, 0), (1, 1), (4, 1), (-1, 1)):
        p = G.RenderParams(splat_stages=st).struct()
        assert lib.gs_project(ctypes.byref(g0), cams, 1, ctypes.byref(p), ctypes.byref(out), None) == want, st


def test_l2_read_probe_rejects_bad_arguments(lib):
    """The L2 bandwidth probe checks its arguments on the host (no launch)."""
    buf = ctypes.c_void_p(16)
    out = ctypes.c_void_p(32)
    assert lib.gs_l2_read_probe(None, 4, 1, out, None) == G.GS_ERR_INVALID_ARG
    assert lib.gs_l2_read_probe(buf, 4, 1, None, None) == G.GS_ERR_INVALID_ARG
    assert lib.gs_l2_read_probe(buf, 6, 1, out, None) == G.GS_ERR_INVALID_ARG      # not a multiple of 4
    assert lib.gs_l2_read_probe(buf, 0, 1, out, None) == G.GS_ERR_INVALID_ARG
    assert lib.gs_l2_read_probe(buf, 4, 0, out, None) == G.GS_ERR_INVALID_ARG
    assert lib.gs_l2_read_probe(ctypes.c_void_p(20), 4, 1, out, None) == G.GS_ERR_INVALID_ARG   # misaligned


def test_block_masks_parameter_is_checked(lib):
    # 1 (binning writes the pixel-block masks the rasterisers read) or 0 (they test); anything else is refused
    cams = G.camera_array([synth.identity_camera()])
    g0 = G.gs_gaussians(None, None, None, None, None, 0)
    out = G.gs_projected()
    for bm, want in ((0, 0), (1, 0), (2, 1), (-1, 1)):
        p = G.RenderParams(block_masks=bm).struct()
        assert lib.gs_project(ctypes.byref(g0), cams, 1, ctypes.byref(p), ctypes.byref(out), None) == want, bm


def test_cull_tiles_parameter_is_checked(lib):
    # 1 (binning drops the tiles a splat cannot reach at 0.99 alpha_min) or 0 (every tile of the rectangle)
    cams = G.camera_array([synth.identity_camera()])
    g0 = G.gs_gaussians(None, None, None, None, None, 0)
    out = G.gs_projected()
    for ct, want in ((0, 0), (1, 0), (2, 1), (-1, 1)):
        p = G.RenderParams(cull_tiles=ct).struct()
        assert lib.gs_project(ctypes.byref(g0), cams, 1, ctypes.byref(p), ctypes.byref(out), None) == want, ct
