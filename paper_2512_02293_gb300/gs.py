"""Thin Python binding of libgs (include/gs.h): ctypes structs with the same
layout as the C ones and one function per entry point, with the same names.

Arguments are torch CUDA tensors (device memory) plus host-side cameras and
parameters; every function only converts them to pointers and calls the
library on the current torch stream.  There is no fallback: if libgs.so is
missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgs.so")
GS_MAX_VIEWS = 32
GS_NOALLOC_LOSS_MAX_VIEWS = 32     # views gs_loss_noalloc's static scratch array holds
_lib = None

STATUS = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_CAPACITY", 3: "GS_ERR_CUDA", 4: "GS_ERR_TIMEOUT",
          5: "GS_ERR_NUMERIC", 6: "GS_ERR_UNSUPPORTED"}
GS_OK, GS_ERR_INVALID_ARG, GS_ERR_CAPACITY, GS_ERR_CUDA = 0, 1, 2, 3
GS_ERR_TIMEOUT, GS_ERR_NUMERIC, GS_ERR_UNSUPPORTED = 4, 5, 6


class GsError(RuntimeError):
    def __init__(self, status, where):
        super().__init__(f"{where}: {STATUS.get(status, status)}")
        self.status = status


# ----------------------------------------------------------------- C structs

c_float_p = ctypes.POINTER(ctypes.c_float)


class gs_camera(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("R_wc", ctypes.c_float * 9),
                ("t_wc", ctypes.c_float * 3)]


class gs_render_params(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("near_plane", ctypes.c_float), ("alpha_min", ctypes.c_float),
                ("alpha_max", ctypes.c_float), ("T_cut", ctypes.c_float), ("dilation", ctypes.c_float),
                ("radius_sigma", ctypes.c_float), ("bg", ctypes.c_float * 3), ("sh_degree", ctypes.c_int32),
                ("splat_stages", ctypes.c_int32), ("block_masks", ctypes.c_int32), ("cull_tiles", ctypes.c_int32)]


class gs_gaussians(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_void_p), ("quat", ctypes.c_void_p), ("log_scale", ctypes.c_void_p),
                ("opacity_logit", ctypes.c_void_p), ("color", ctypes.c_void_p), ("n", ctypes.c_int64)]


class gs_projected(ctypes.Structure):
    _fields_ = [("xy", ctypes.c_void_p), ("conic_o", ctypes.c_void_p), ("rgbd", ctypes.c_void_p),
                ("rect", ctypes.c_void_p), ("radius", ctypes.c_void_p), ("tiles_touched", ctypes.c_void_p)]


class gs_bins(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("key_capacity", ctypes.c_int64),
                ("ranges", ctypes.c_void_p), ("num_keys", ctypes.c_void_p), ("status", ctypes.c_void_p),
                ("masks", ctypes.c_void_p)]


class gs_image(ctypes.Structure):
    _fields_ = [("color", ctypes.c_void_p), ("depth", ctypes.c_void_p), ("T_final", ctypes.c_void_p),
                ("n_contrib", ctypes.c_void_p)]


class gs_grads(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_void_p), ("quat", ctypes.c_void_p), ("log_scale", ctypes.c_void_p),
                ("opacity_logit", ctypes.c_void_p), ("color", ctypes.c_void_p), ("pose", ctypes.c_void_p)]


class gs_adam_group(ctypes.Structure):
    _fields_ = [("param", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("m", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("n", ctypes.c_int64), ("lr", ctypes.c_float), ("reserved", ctypes.c_int32)]


class gs_map_slots(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_void_p), ("quat", ctypes.c_void_p), ("log_scale", ctypes.c_void_p),
                ("opacity_logit", ctypes.c_void_p), ("color", ctypes.c_void_p), ("capacity", ctypes.c_int64)]


class gs_ba_problem(ctypes.Structure):
    _fields_ = [("poses", ctypes.c_void_p), ("disp", ctypes.c_void_p), ("targets", ctypes.c_void_p),
                ("weights", ctypes.c_void_p), ("ii", ctypes.c_void_p), ("jj", ctypes.c_void_p),
                ("n_keyframes", ctypes.c_int32), ("n_edges", ctypes.c_int32), ("height", ctypes.c_int32),
                ("width", ctypes.c_int32), ("n_fixed", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("status", ctypes.c_void_p),
                ("imu", ctypes.c_void_p), ("vel", ctypes.c_void_p), ("bias", ctypes.c_void_p),
                ("bias_hat", ctypes.c_void_p), ("gravity", ctypes.c_float * 3)]


GS_BA_IMU_FLOATS = 286


class gs_mapping_step_args(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("gaussians", "cams", "params", "proj", "bins", "img", "grads",
                                                "target_color", "target_depth", "loss_terms", "iso_loss")] + \
               [("ws", ctypes.c_void_p), ("ws_bytes", ctypes.c_size_t), ("loss_ws", ctypes.c_void_p),
                ("loss_ws_bytes", ctypes.c_size_t), ("adam_groups", ctypes.c_void_p), ("d_step", ctypes.c_void_p),
                ("n_views", ctypes.c_int32), ("n_adam_groups", ctypes.c_int32)] + \
               [(k, ctypes.c_float) for k in ("lambda_c", "lambda_d", "lambda_iso", "beta1", "beta2", "adam_eps")]


class gs_mlp_params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]


class gs_mlp_packed(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("W1a", "W2a", "W3a", "W2t", "gelu_tab", "dgelu_tab")]


class gs_mlp_grads(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]


EXPORTS = ["gs_abi_version", "gs_status_string", "gs_total_tiles", "gs_total_pixels", "gs_workspace_size",
           "gs_project", "gs_bin_sort", "gs_render_fwd", "gs_loss", "gs_loss_noalloc", "gs_render_bwd",
           "gs_render_bwd_raster",
           "gs_project_bwd", "gs_adam_step", "gs_read_device_status", "gs_mlp_pack", "gs_mlp_fwd", "gs_mlp_bwd",
           "gs_extract_patches", "gs_insert_gaussians", "gs_loop_closure_update", "gs_ba_workspace_size",
           "gs_ba_step", "gs_fused_loss_workspace_size", "gs_render_fwd_loss", "gs_render_bwd_raster_loss",
           "gs_mapping_step", "gs_mlp_set_wait_polls", "gs_project_perturbed", "gs_project_bwd_perturbed",
           "gs_l2_read_probe"]


def load_library(path: str | None = None):
    """Load libgs.so (no GPU needed to load it)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libgs.so is not built ({p}); run __graft_entry__.build() or "
                           "python paper_2512_02293_gb300/build.py")
    lib = ctypes.CDLL(p)
    V = ctypes.c_void_p
    lib.gs_abi_version.restype = ctypes.c_int32
    lib.gs_status_string.restype = ctypes.c_char_p
    lib.gs_status_string.argtypes = [ctypes.c_int32]
    lib.gs_total_tiles.restype = ctypes.c_int64
    lib.gs_total_tiles.argtypes = [V, ctypes.c_int32, ctypes.c_int32]
    lib.gs_total_pixels.restype = ctypes.c_int64
    lib.gs_total_pixels.argtypes = [V, ctypes.c_int32]
    lib.gs_workspace_size.restype = ctypes.c_size_t
    lib.gs_workspace_size.argtypes = [ctypes.c_int64, ctypes.c_int32, V, V, ctypes.c_int64]
    lib.gs_project.restype = ctypes.c_int32
    lib.gs_project.argtypes = [V, V, ctypes.c_int32, V, V, V]
    lib.gs_bin_sort.restype = ctypes.c_int32
    lib.gs_bin_sort.argtypes = [V, ctypes.c_int64, V, ctypes.c_int32, V, V, V, ctypes.c_size_t, V]
    lib.gs_render_fwd.restype = ctypes.c_int32
    lib.gs_render_fwd.argtypes = [V, V, V, ctypes.c_int32, V, V, V]
    lib.gs_loss.restype = ctypes.c_int32
    lib.gs_loss.argtypes = [V, V, V, V, ctypes.c_int32, ctypes.c_float, ctypes.c_float, V, V, V, V,
                            ctypes.c_size_t, V]
    lib.gs_loss_noalloc.restype = ctypes.c_int32
    lib.gs_loss_noalloc.argtypes = [V, V, V, V, ctypes.c_int32, ctypes.c_float, ctypes.c_float, V, V, V, V]
    lib.gs_render_bwd.restype = ctypes.c_int32
    lib.gs_render_bwd.argtypes = [V, V, V, V, V, V, V, ctypes.c_int32, V, ctypes.c_float, V, V, V, ctypes.c_size_t, V]
    lib.gs_render_bwd_raster.restype = ctypes.c_int32
    lib.gs_render_bwd_raster.argtypes = [V, V, V, V, V, V, ctypes.c_int32, V, ctypes.c_int64, V, V]
    lib.gs_project_bwd.restype = ctypes.c_int32
    lib.gs_project_bwd.argtypes = [V, V, ctypes.c_int32, V, V, ctypes.c_float, V, V, V]
    lib.gs_adam_step.restype = ctypes.c_int32
    lib.gs_adam_step.argtypes = [V, ctypes.c_int32, ctypes.c_float, ctypes.c_float, ctypes.c_float, V, V]
    lib.gs_l2_read_probe.restype = ctypes.c_int32
    lib.gs_l2_read_probe.argtypes = [V, ctypes.c_int64, ctypes.c_int32, V, V]
    lib.gs_read_device_status.restype = ctypes.c_int32
    lib.gs_read_device_status.argtypes = [V, V, V]
    lib.gs_mlp_pack.restype = ctypes.c_int32
    lib.gs_mlp_pack.argtypes = [V, V, V]
    lib.gs_mlp_fwd.restype = ctypes.c_int32
    lib.gs_mlp_fwd.argtypes = [V, V, ctypes.c_int64, V, V, V, V, V, V, ctypes.c_float, V, V]
    lib.gs_mlp_bwd.restype = ctypes.c_int32
    lib.gs_mlp_bwd.argtypes = [V, V, V, V, V, ctypes.c_int64, V, V, V]
    lib.gs_extract_patches.restype = ctypes.c_int32
    lib.gs_extract_patches.argtypes = [V, V, V, V, ctypes.c_int64, V, V, V]
    lib.gs_ba_workspace_size.restype = ctypes.c_size_t
    lib.gs_ba_workspace_size.argtypes = [ctypes.c_int32] * 6
    lib.gs_ba_step.restype = ctypes.c_int32
    lib.gs_ba_step.argtypes = [V, ctypes.c_float, ctypes.c_float, V, V, ctypes.c_size_t, V]
    lib.gs_loop_closure_update.restype = ctypes.c_int32
    lib.gs_loop_closure_update.argtypes = [V, V, V, V, V, ctypes.c_int32, V, V]
    lib.gs_insert_gaussians.restype = ctypes.c_int32
    lib.gs_insert_gaussians.argtypes = [V, V, V, V, ctypes.c_int64, ctypes.c_float, V, V, ctypes.c_int64,
                                        ctypes.c_int32, V, V]
    lib.gs_fused_loss_workspace_size.restype = ctypes.c_size_t
    lib.gs_fused_loss_workspace_size.argtypes = [ctypes.c_int32]
    lib.gs_render_fwd_loss.restype = ctypes.c_int32
    lib.gs_render_fwd_loss.argtypes = [V, V, V, ctypes.c_int32, V, V, V, V, V, V, ctypes.c_size_t, V]
    lib.gs_render_bwd_raster_loss.restype = ctypes.c_int32
    lib.gs_render_bwd_raster_loss.argtypes = [V, V, V, V, V, ctypes.c_float, ctypes.c_float, V, ctypes.c_size_t, V,
                                              ctypes.c_int32, V, ctypes.c_int64, V, V]
    lib.gs_mapping_step.restype = ctypes.c_int32
    lib.gs_mapping_step.argtypes = [V, V]
    lib.gs_mlp_set_wait_polls.restype = ctypes.c_int64
    lib.gs_mlp_set_wait_polls.argtypes = [ctypes.c_int64]
    lib.gs_project_perturbed.restype = ctypes.c_int32
    lib.gs_project_perturbed.argtypes = [V, V, ctypes.c_int32, V, V, V, V]
    lib.gs_project_bwd_perturbed.restype = ctypes.c_int32
    lib.gs_project_bwd_perturbed.argtypes = [V, V, ctypes.c_int32, V, V, V, ctypes.c_float, V, V, V]
    if lib.gs_abi_version() != 6:
        raise RuntimeError("libgs ABI version mismatch")
    if path is None:
        _lib = lib
    return lib


# --------------------------------------------------------- host-side values

@dataclass
class RenderParams:
    tile: int = 16
    near_plane: float = 0.2
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    T_cut: float = 1e-4
    dilation: float = 0.3
    radius_sigma: float = 3.0
    bg: tuple = (0.0, 0.0, 0.0)
    sh_degree: int = 0
    splat_stages: int = 0      # 0: the library chooses; 2 or 3 batches of 32 splats per forward warp
    block_masks: int = 1       # 1: binning writes per-key pixel-block masks the rasterisers read
    cull_tiles: int = 0        # 1: binning drops the tiles a splat cannot reach at 0.99 alpha_min

    def struct(self) -> gs_render_params:
        return gs_render_params(int(self.tile), self.near_plane, self.alpha_min, self.alpha_max, self.T_cut,
                                self.dilation, self.radius_sigma, (ctypes.c_float * 3)(*self.bg),
                                int(self.sh_degree), int(self.splat_stages), int(self.block_masks),
                                int(self.cull_tiles))


def camera_array(cams) -> ctypes.Array:
    """Array of gs_camera from objects with fx, fy, cx, cy, width, height, R_wc, t_wc."""
    arr = (gs_camera * len(cams))()
    for k, c in enumerate(cams):
        R = np.asarray(c.R_wc, dtype=np.float32).reshape(9)
        t = np.asarray(c.t_wc, dtype=np.float32).reshape(3)
        arr[k] = gs_camera(float(c.fx), float(c.fy), float(c.cx), float(c.cy), int(c.width), int(c.height),
                           (ctypes.c_float * 9)(*R), (ctypes.c_float * 3)(*t))
    return arr


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libgs takes device tensors")
    if not t.is_contiguous():
        raise ValueError("libgs takes contiguous tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _check(status, where):
    if status != GS_OK:
        raise GsError(status, where)


# ------------------------------------------------------- device containers

@dataclass
class Gaussians:
    mean: "torch.Tensor"
    quat: "torch.Tensor"
    log_scale: "torch.Tensor"
    opacity_logit: "torch.Tensor"
    color: "torch.Tensor"

    @property
    def n(self):
        return int(self.mean.shape[0])

    @staticmethod
    def from_numpy(g, device="cuda"):
        import torch
        return Gaussians(*(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(device) for a in g.arrays()))

    def tensors(self):
        return [self.mean, self.quat, self.log_scale, self.opacity_logit, self.color]

    def struct(self) -> gs_gaussians:
        for t in self.tensors():
            if t.dtype.itemsize != 4:
                raise ValueError("Gaussian parameters are float32")
        return gs_gaussians(*(_ptr(t) for t in self.tensors()), self.n)


@dataclass
class Projected:
    xy: "torch.Tensor"
    conic_o: "torch.Tensor"
    rgbd: "torch.Tensor"
    rect: "torch.Tensor"
    radius: "torch.Tensor"
    tiles_touched: "torch.Tensor"

    @staticmethod
    def empty(n_entries, device="cuda"):
        import torch
        f = dict(device=device, dtype=torch.float32)
        i = dict(device=device, dtype=torch.int32)
        return Projected(torch.empty(n_entries, 2, **f), torch.empty(n_entries, 4, **f), torch.empty(n_entries, 4, **f),
                         torch.empty(n_entries, 4, **i), torch.empty(n_entries, **i), torch.empty(n_entries, **i))

    def struct(self) -> gs_projected:
        return gs_projected(*(_ptr(getattr(self, f.name)) for f in fields(self)))


@dataclass
class Bins:
    keys: "torch.Tensor"       # int64 storage of uint64 keys
    vals: "torch.Tensor"       # int32 storage of uint32 values
    ranges: "torch.Tensor"     # int32 [total_tiles, 2]
    num_keys: "torch.Tensor"   # int32 [1]
    status: "torch.Tensor"     # int32 [4]: status word + raster work counters
    masks: "torch.Tensor"      # int32 storage of uint32 per-key pixel-block masks

    @staticmethod
    def empty(capacity, total_tiles, device="cuda"):
        import torch
        i = dict(device=device, dtype=torch.int32)
        return Bins(torch.empty(max(capacity, 1), device=device, dtype=torch.int64), torch.empty(max(capacity, 1), **i),
                    torch.zeros(total_tiles, 2, **i), torch.zeros(1, **i), torch.zeros(4, **i),
                    torch.empty(max(capacity, 1), **i))

    @property
    def capacity(self):
        return int(self.keys.shape[0])

    def struct(self) -> gs_bins:
        return gs_bins(_ptr(self.keys), _ptr(self.vals), self.capacity, _ptr(self.ranges), _ptr(self.num_keys),
                       _ptr(self.status), _ptr(self.masks))


@dataclass
class Image:
    color: "torch.Tensor"      # [3 * P]
    depth: "torch.Tensor"      # [P]
    T_final: "torch.Tensor"    # [P]
    n_contrib: "torch.Tensor"  # [P] int32 storage of uint32

    @staticmethod
    def empty(total_pixels, device="cuda"):
        import torch
        f = dict(device=device, dtype=torch.float32)
        return Image(torch.empty(3 * total_pixels, **f), torch.empty(total_pixels, **f), torch.empty(total_pixels, **f),
                     torch.empty(total_pixels, device=device, dtype=torch.int32))

    def struct(self) -> gs_image:
        return gs_image(_ptr(self.color), _ptr(self.depth), _ptr(self.T_final), _ptr(self.n_contrib))


@dataclass
class Grads:
    mean: "torch.Tensor"
    quat: "torch.Tensor"
    log_scale: "torch.Tensor"
    opacity_logit: "torch.Tensor"
    color: "torch.Tensor"
    pose: "torch.Tensor | None" = None

    @staticmethod
    def empty_like(g: Gaussians, n_views: int | None = None):
        import torch
        pose = None if n_views is None else torch.zeros(n_views, 6, device=g.mean.device, dtype=torch.float32)
        return Grads(*(torch.empty_like(t) for t in g.tensors()), pose)

    def tensors(self):
        return [self.mean, self.quat, self.log_scale, self.opacity_logit, self.color]

    def struct(self) -> gs_grads:
        return gs_grads(*(_ptr(t) for t in self.tensors()), _ptr(self.pose))


# ------------------------------------------------------------- entry points

def gs_total_tiles(cams, tile: int) -> int:
    arr = camera_array(cams)
    r = load_library().gs_total_tiles(arr, len(cams), tile)
    if r < 0:
        raise GsError(GS_ERR_INVALID_ARG, "gs_total_tiles")
    return int(r)


def gs_total_pixels(cams) -> int:
    arr = camera_array(cams)
    r = load_library().gs_total_pixels(arr, len(cams))
    if r < 0:
        raise GsError(GS_ERR_INVALID_ARG, "gs_total_pixels")
    return int(r)


def gs_workspace_size(n: int, cams, params: RenderParams, key_capacity: int) -> int:
    arr = camera_array(cams)
    p = params.struct()
    r = load_library().gs_workspace_size(n, len(cams), arr, ctypes.byref(p), key_capacity)
    if r == 0:
        raise GsError(GS_ERR_INVALID_ARG, "gs_workspace_size")
    return int(r)


def gs_project(g: Gaussians, cams, params: RenderParams, out: Projected, stream=None, xi=None):
    """xi: optional device float32 [n_views, 6] pose tangents applied on the device
    (gs_project_perturbed)."""
    arr = camera_array(cams); p = params.struct(); gg = g.struct(); o = out.struct()
    if xi is None:
        _check(load_library().gs_project(ctypes.byref(gg), arr, len(cams), ctypes.byref(p), ctypes.byref(o),
                                         _stream(stream)), "gs_project")
    else:
        _check(load_library().gs_project_perturbed(ctypes.byref(gg), arr, len(cams), ctypes.byref(p), _ptr(xi),
                                                   ctypes.byref(o), _stream(stream)), "gs_project_perturbed")


def gs_bin_sort(proj: Projected, n: int, cams, params: RenderParams, bins: Bins, ws, stream=None):
    arr = camera_array(cams); p = params.struct(); pr = proj.struct(); b = bins.struct()
    _check(load_library().gs_bin_sort(ctypes.byref(pr), n, arr, len(cams), ctypes.byref(p), ctypes.byref(b),
                                      _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)), "gs_bin_sort")


def gs_render_fwd(proj: Projected, bins: Bins, cams, params: RenderParams, img: Image, stream=None):
    arr = camera_array(cams); p = params.struct(); pr = proj.struct(); b = bins.struct(); im = img.struct()
    _check(load_library().gs_render_fwd(ctypes.byref(pr), ctypes.byref(b), arr, len(cams), ctypes.byref(p),
                                        ctypes.byref(im), _stream(stream)), "gs_render_fwd")


def gs_loss(img: Image, target_color, target_depth, cams, lambda_c: float, lambda_d: float, dL_dcolor, dL_ddepth,
            loss_terms, ws, stream=None):
    arr = camera_array(cams); im = img.struct()
    _check(load_library().gs_loss(ctypes.byref(im), _ptr(target_color), _ptr(target_depth), arr, len(cams),
                                  float(lambda_c), float(lambda_d), _ptr(dL_dcolor), _ptr(dL_ddepth), _ptr(loss_terms),
                                  _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)), "gs_loss")


def gs_loss_noalloc(img: Image, target_color, target_depth, cams, lambda_c: float, lambda_d: float, dL_dcolor,
                    dL_ddepth, loss_terms, stream=None):
    """gs_loss without a workspace (for callers that cannot allocate one); see gs.h."""
    arr = camera_array(cams); im = img.struct()
    _check(load_library().gs_loss_noalloc(ctypes.byref(im), _ptr(target_color), _ptr(target_depth), arr, len(cams),
                                          float(lambda_c), float(lambda_d), _ptr(dL_dcolor), _ptr(dL_ddepth),
                                          _ptr(loss_terms), _stream(stream)), "gs_loss_noalloc")


def gs_render_bwd(g: Gaussians, proj: Projected, bins: Bins, img: Image, dL_dcolor, dL_ddepth, cams,
                  params: RenderParams, lambda_iso: float, grads: Grads, iso_loss, ws, stream=None):
    arr = camera_array(cams); p = params.struct(); gg = g.struct(); pr = proj.struct(); b = bins.struct()
    im = img.struct(); gr = grads.struct()
    _check(load_library().gs_render_bwd(ctypes.byref(gg), ctypes.byref(pr), ctypes.byref(b), ctypes.byref(im),
                                        _ptr(dL_dcolor), _ptr(dL_ddepth), arr, len(cams), ctypes.byref(p),
                                        float(lambda_iso), ctypes.byref(gr), _ptr(iso_loss), _ptr(ws),
                                        ws.numel() * ws.element_size(), _stream(stream)), "gs_render_bwd")


def gs_render_bwd_raster(proj: Projected, bins: Bins, img: Image, dL_dcolor, dL_ddepth, cams, params: RenderParams,
                         n: int, grad2d, stream=None):
    arr = camera_array(cams); p = params.struct(); pr = proj.struct(); b = bins.struct(); im = img.struct()
    _check(load_library().gs_render_bwd_raster(ctypes.byref(pr), ctypes.byref(b), ctypes.byref(im), _ptr(dL_dcolor),
                                               _ptr(dL_ddepth), arr, len(cams), ctypes.byref(p), n, _ptr(grad2d),
                                               _stream(stream)), "gs_render_bwd_raster")


def gs_fused_loss_workspace_size(n_views: int) -> int:
    return int(load_library().gs_fused_loss_workspace_size(n_views))


def gs_render_fwd_loss(proj: Projected, bins: Bins, cams, params: RenderParams, img: Image, target_color,
                       target_depth, loss_terms, loss_ws, stream=None):
    """gs_render_fwd with the Eq. 6 colour/depth L1 sums fused in (see gs.h)."""
    arr = camera_array(cams); p = params.struct(); pr = proj.struct(); b = bins.struct(); im = img.struct()
    _check(load_library().gs_render_fwd_loss(ctypes.byref(pr), ctypes.byref(b), arr, len(cams), ctypes.byref(p),
                                             ctypes.byref(im), _ptr(target_color), _ptr(target_depth),
                                             _ptr(loss_terms), _ptr(loss_ws), loss_ws.numel() * loss_ws.element_size(),
                                             _stream(stream)), "gs_render_fwd_loss")


def gs_render_bwd_raster_loss(proj: Projected, bins: Bins, img: Image, target_color, target_depth, lambda_c: float,
                              lambda_d: float, loss_ws, cams, params: RenderParams, n: int, grad2d, stream=None):
    """gs_render_bwd_raster with the image gradients of the fused loss formed per pixel (see gs.h)."""
    arr = camera_array(cams); p = params.struct(); pr = proj.struct(); b = bins.struct(); im = img.struct()
    _check(load_library().gs_render_bwd_raster_loss(ctypes.byref(pr), ctypes.byref(b), ctypes.byref(im),
                                                    _ptr(target_color), _ptr(target_depth), float(lambda_c),
                                                    float(lambda_d), _ptr(loss_ws),
                                                    loss_ws.numel() * loss_ws.element_size(), arr, len(cams),
                                                    ctypes.byref(p), n, _ptr(grad2d), _stream(stream)),
           "gs_render_bwd_raster_loss")


def gs_project_bwd(g: Gaussians, cams, params: RenderParams, grad2d, lambda_iso: float, grads: Grads, iso_loss,
                   stream=None, xi=None):
    """xi: optional device float32 [n_views, 6] pose tangents (gs_project_bwd_perturbed)."""
    arr = camera_array(cams); p = params.struct(); gg = g.struct(); gr = grads.struct()
    if xi is None:
        _check(load_library().gs_project_bwd(ctypes.byref(gg), arr, len(cams), ctypes.byref(p), _ptr(grad2d),
                                             float(lambda_iso), ctypes.byref(gr), _ptr(iso_loss), _stream(stream)),
               "gs_project_bwd")
    else:
        _check(load_library().gs_project_bwd_perturbed(ctypes.byref(gg), arr, len(cams), ctypes.byref(p), _ptr(xi),
                                                       _ptr(grad2d), float(lambda_iso), ctypes.byref(gr),
                                                       _ptr(iso_loss), _stream(stream)), "gs_project_bwd_perturbed")


def gs_adam_step(groups, beta1: float, beta2: float, eps: float, d_step, stream=None):
    """groups: list of (param, grad, m, v, lr) tensors/floats."""
    arr = (gs_adam_group * len(groups))()
    for k, (p, gr, m, v, lr) in enumerate(groups):
        arr[k] = gs_adam_group(_ptr(p), _ptr(gr), _ptr(m), _ptr(v), p.numel(), float(lr), 0)
    _check(load_library().gs_adam_step(arr, len(groups), float(beta1), float(beta2), float(eps), _ptr(d_step),
                                       _stream(stream)), "gs_adam_step")


class BoundCall:
    """One C-ABI call with every argument but the stream marshalled once.  The
    tensors it points at must stay allocated and keep their storage; the
    ctypes structures the arguments refer to are held here."""
    __slots__ = ("fn", "args", "name", "keep")

    def __init__(self, name: str, args: tuple, keep: tuple = ()):
        self.fn = getattr(load_library(), name)
        self.args = args
        self.name = name
        self.keep = keep

    def __call__(self, stream=None):
        _check(self.fn(*self.args, _stream(stream)), self.name)


def bind_mapping_step(g: Gaussians, proj: Projected, bins: Bins, img: Image, cams, params: RenderParams,
                      target_color, target_depth, lambda_c: float, lambda_d: float, dL_dcolor, dL_ddepth,
                      loss_terms, lambda_iso: float, grads: Grads, iso_loss, ws, adam_groups,
                      beta1: float, beta2: float, eps: float, d_step, loss_ws=None, one_call: bool = True):
    """The calls of one mapping iteration as BoundCall objects, in order: with
    loss_ws (a fused-loss workspace) the single native gs_mapping_step (or, with
    one_call=False, its six calls gs_project, gs_bin_sort, gs_render_fwd_loss,
    gs_render_bwd_raster_loss, gs_project_bwd, gs_adam_step), else the seven with
    gs_render_fwd, gs_loss and gs_render_bwd_raster.  ws doubles as grad2d, as
    in the staged iteration."""
    arr = camera_array(cams); V = len(cams); p = params.struct()
    gg = g.struct(); pr = proj.struct(); b = bins.struct(); im = img.struct(); gr = grads.struct()
    wsb = ws.numel() * ws.element_size()
    groups = (gs_adam_group * len(adam_groups))()
    for k, (pp, gd, m, v, lr) in enumerate(adam_groups):
        groups[k] = gs_adam_group(_ptr(pp), _ptr(gd), _ptr(m), _ptr(v), pp.numel(), float(lr), 0)
    keep = (arr, p, gg, pr, b, im, gr, groups)
    by = ctypes.byref
    if loss_ws is not None and one_call:
        # the whole fused iteration as one native call (gs_mapping_step)
        lwb = loss_ws.numel() * loss_ws.element_size()
        ad = ctypes.addressof
        args = gs_mapping_step_args(ad(gg), ad(arr), ad(p), ad(pr), ad(b), ad(im), ad(gr), _ptr(target_color),
                                    _ptr(target_depth), _ptr(loss_terms), _ptr(iso_loss), _ptr(ws), wsb,
                                    _ptr(loss_ws), lwb, ad(groups), _ptr(d_step), V, len(adam_groups),
                                    float(lambda_c), float(lambda_d), float(lambda_iso), float(beta1), float(beta2),
                                    float(eps))
        return [BoundCall("gs_mapping_step", (ctypes.byref(args),), keep + (args,))]
    if loss_ws is not None:
        lwb = loss_ws.numel() * loss_ws.element_size()
        return [
            BoundCall("gs_project", (by(gg), arr, V, by(p), by(pr)), keep),
            BoundCall("gs_bin_sort", (by(pr), g.n, arr, V, by(p), by(b), _ptr(ws), wsb), keep),
            BoundCall("gs_render_fwd_loss", (by(pr), by(b), arr, V, by(p), by(im), _ptr(target_color),
                                             _ptr(target_depth), _ptr(loss_terms), _ptr(loss_ws), lwb), keep),
            BoundCall("gs_render_bwd_raster_loss", (by(pr), by(b), by(im), _ptr(target_color), _ptr(target_depth),
                                                    float(lambda_c), float(lambda_d), _ptr(loss_ws), lwb, arr, V,
                                                    by(p), g.n, _ptr(ws)), keep),
            BoundCall("gs_project_bwd", (by(gg), arr, V, by(p), _ptr(ws), float(lambda_iso), by(gr),
                                         _ptr(iso_loss)), keep),
            BoundCall("gs_adam_step", (groups, len(adam_groups), float(beta1), float(beta2), float(eps),
                                       _ptr(d_step)), keep),
        ]
    return [
        BoundCall("gs_project", (by(gg), arr, V, by(p), by(pr)), keep),
        BoundCall("gs_bin_sort", (by(pr), g.n, arr, V, by(p), by(b), _ptr(ws), wsb), keep),
        BoundCall("gs_render_fwd", (by(pr), by(b), arr, V, by(p), by(im)), keep),
        BoundCall("gs_loss", (by(im), _ptr(target_color), _ptr(target_depth), arr, V, float(lambda_c),
                              float(lambda_d), _ptr(dL_dcolor), _ptr(dL_ddepth), _ptr(loss_terms), _ptr(ws), wsb),
                  keep),
        BoundCall("gs_render_bwd_raster", (by(pr), by(b), by(im), _ptr(dL_dcolor), _ptr(dL_ddepth), arr, V, by(p),
                                           g.n, _ptr(ws)), keep),
        BoundCall("gs_project_bwd", (by(gg), arr, V, by(p), _ptr(ws), float(lambda_iso), by(gr), _ptr(iso_loss)),
                  keep),
        BoundCall("gs_adam_step", (groups, len(adam_groups), float(beta1), float(beta2), float(eps), _ptr(d_step)),
                  keep),
    ]


def gs_l2_read_probe(buf, reps: int, out, stream=None):
    """Read buf (FP32, length a multiple of 4) reps times over in one launch,
    adding the sum to out[0] (see gs.h: the L2 bandwidth probe)."""
    _check(load_library().gs_l2_read_probe(_ptr(buf), buf.numel(), int(reps), _ptr(out), _stream(stream)),
           "gs_l2_read_probe")


def gs_read_device_status(d_status, stream=None) -> int:
    out = ctypes.c_int32(0)
    _check(load_library().gs_read_device_status(_ptr(d_status), _stream(stream), ctypes.byref(out)),
           "gs_read_device_status")
    return int(out.value)


# ------------------------------------------------------ learned initialiser

MLP_IN, MLP_IN_STRIDE, MLP_HIDDEN, MLP_OUT = 196, 208, 128, 8
MLP_PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")
MLP_PARAM_SHAPES = {"W1": (128, 196), "b1": (128,), "W2": (128, 128), "b2": (128,), "W3": (8, 128), "b3": (8,)}


class MlpPacked:
    """BF16 GEMM operands (W1a [128,208], W2a [128,144], W3a [16,144], W2t [128,128]) and the
    activation tables over all BF16 inputs (gelu_tab BF16, dgelu_tab FP32, 65536 each)."""

    def __init__(self, device="cuda"):
        import torch
        bf = torch.bfloat16
        self.W1a = torch.zeros(128, 208, device=device, dtype=bf)
        self.W2a = torch.zeros(128, 144, device=device, dtype=bf)
        self.W3a = torch.zeros(16, 144, device=device, dtype=bf)
        self.W2t = torch.zeros(128, 128, device=device, dtype=bf)
        self.gelu_tab = torch.zeros(65536, device=device, dtype=bf)
        self.dgelu_tab = torch.zeros(65536, device=device, dtype=torch.float32)

    def struct(self):
        return gs_mlp_packed(_ptr(self.W1a), _ptr(self.W2a), _ptr(self.W3a), _ptr(self.W2t), _ptr(self.gelu_tab),
                             _ptr(self.dgelu_tab))


def gs_mlp_pack(params: dict, packed: MlpPacked, stream=None):
    """params: dict of FP32 device tensors W1, b1, W2, b2, W3, b3."""
    p = gs_mlp_params(*[_ptr(params[k]) for k in MLP_PARAM_NAMES])
    q = packed.struct()
    _check(load_library().gs_mlp_pack(ctypes.byref(p), ctypes.byref(q), _stream(stream)), "gs_mlp_pack")


def gs_mlp_fwd(packed: MlpPacked, X, Y=None, Z1=None, Z2=None, T=None, dY=None, loss=None, loss_scale: float = 0.0,
               status=None, stream=None):
    """X: bfloat16 [n, 208]; Y, dY, T float32 [n, 8]; Z1, Z2 bfloat16 [n, 128]."""
    q = packed.struct()
    _check(load_library().gs_mlp_fwd(ctypes.byref(q), _ptr(X), X.shape[0], _ptr(Y), _ptr(Z1), _ptr(Z2), _ptr(T),
                                     _ptr(dY), _ptr(loss), float(loss_scale), _ptr(status), _stream(stream)),
           "gs_mlp_fwd")


def gs_mlp_bwd(packed: MlpPacked, X, Z1, Z2, dY, grads: dict, status=None, stream=None):
    """grads: dict of FP32 device tensors shaped like the parameters (overwritten)."""
    q = packed.struct()
    g = gs_mlp_grads(*[_ptr(grads[k]) for k in MLP_PARAM_NAMES])
    _check(load_library().gs_mlp_bwd(ctypes.byref(q), _ptr(X), _ptr(Z1), _ptr(Z2), _ptr(dY), X.shape[0],
                                     ctypes.byref(g), _ptr(status), _stream(stream)), "gs_mlp_bwd")


MLP_WAIT_POLLS_DEFAULT = 1 << 26


def gs_mlp_set_wait_polls(polls: int) -> int:
    """Poll limit of the MLP kernels' mbarrier waits for later launches (a test
    hook of the timeout path; negative = the default); returns the previous one."""
    prev = int(load_library().gs_mlp_set_wait_polls(int(polls)))
    if prev < 0:
        raise GsError(GS_ERR_INVALID_ARG, "gs_mlp_set_wait_polls")
    return prev


# ------------------------------------------------------- keyframe insertion

def gs_extract_patches(color, depth, cam, uv, X, status=None, stream=None):
    """color [3*H*W] / [3,H,W], depth [H*W] float32; uv int32 [n, 2]; X bfloat16 [n, 208] (written)."""
    cams = camera_array([cam])
    _check(load_library().gs_extract_patches(_ptr(color), _ptr(depth), cams, _ptr(uv), uv.shape[0], _ptr(X),
                                             _ptr(status), _stream(stream)), "gs_extract_patches")


def gs_insert_gaussians(color, depth, cam, uv, stride: float, dst: "Gaussians", offset: int, Y=None,
                        sh_degree: int = 0, status=None, stream=None):
    """Write the Gaussians of the samples uv into rows offset.. of the map dst."""
    cams = camera_array([cam])
    slots = gs_map_slots(_ptr(dst.mean), _ptr(dst.quat), _ptr(dst.log_scale), _ptr(dst.opacity_logit),
                         _ptr(dst.color), dst.n)
    _check(load_library().gs_insert_gaussians(_ptr(color), _ptr(depth), cams, _ptr(uv), uv.shape[0], float(stride),
                                              _ptr(Y), ctypes.byref(slots), int(offset), int(sh_degree),
                                              _ptr(status), _stream(stream)), "gs_insert_gaussians")


# ------------------------------------------------------ loop-closure update

def gs_loop_closure_update(g: "Gaussians", anchor, pose_before, pose_after, scale_change, status=None,
                           stream=None):
    """In-place Eq. 7 / Eq. 8 update of g.  anchor int32 [n]; poses float32
    [K, 12] (R_wc row-major, t_wc); scale_change float32 [K]."""
    slots = gs_map_slots(_ptr(g.mean), _ptr(g.quat), _ptr(g.log_scale), _ptr(g.opacity_logit), _ptr(g.color), g.n)
    _check(load_library().gs_loop_closure_update(ctypes.byref(slots), _ptr(anchor), _ptr(pose_before),
                                                 _ptr(pose_after), _ptr(scale_change), int(pose_before.shape[0]),
                                                 _ptr(status), _stream(stream)), "gs_loop_closure_update")


# ------------------------------------------------------- bundle adjustment

class BAWindow:
    """Device state of a bundle-adjustment window (see gs_ba_step): poses
    [K, 12] (world-to-camera R row-major, t), inverse depths [K, h, w], targets
    and weights [E, h, w, 2], edges ii / jj [E], intrinsics of the grid.  With
    `imu` ([K - 1, GS_BA_IMU_FLOATS] pre-integration records) the window also
    holds velocities [K, 3], biases [K, 6] (b_g, b_a), the linearisation biases
    [K, 6] and gravity, and each step includes the inertial factor of Eq. 3."""

    def __init__(self, R, t, disp, intr, edges, targets, weights, n_fixed, device="cuda", imu=None, vel=None,
                 bias=None, bias_hat=None, gravity=None):
        import torch
        f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device)
        K, h, w = np.asarray(disp).shape
        self.K, self.h, self.w, self.E = K, h, w, len(edges)
        self.poses = f(np.concatenate([np.asarray(R).reshape(K, 9), np.asarray(t).reshape(K, 3)], 1))
        self.disp = f(disp)
        self.targets = f(targets)
        self.weights = f(weights)
        e = np.asarray(edges, np.int32).reshape(-1, 2)
        self.ii = torch.from_numpy(np.ascontiguousarray(e[:, 0])).to(device)
        self.jj = torch.from_numpy(np.ascontiguousarray(e[:, 1])).to(device)
        self.intr = tuple(float(x) for x in intr)
        self.n_fixed = int(n_fixed)
        self.status = torch.zeros(4, device=device, dtype=torch.int32)
        self.cost = torch.zeros(1, device=device)
        self.imu = None
        if imu is not None:
            if vel is None or bias is None or bias_hat is None or gravity is None:
                raise ValueError("the inertial factor needs velocities, biases, linearisation biases and gravity")
            self.imu = f(np.asarray(imu).reshape(K - 1, GS_BA_IMU_FLOATS))
            self.vel = f(np.asarray(vel).reshape(K, 3))
            self.bias = f(np.asarray(bias).reshape(K, 6))
            self.bias_hat = f(np.asarray(bias_hat).reshape(K, 6))
            self.gravity = tuple(float(x) for x in np.asarray(gravity).reshape(3))
        nbytes = gs_ba_workspace_size(K, self.E, h, w, n_fixed, self.imu is not None)
        self.ws = torch.empty((nbytes + 255) // 256 * 64 + 64, device=device, dtype=torch.float32)

    def struct(self):
        fx, fy, cx, cy = self.intr
        pr = gs_ba_problem(_ptr(self.poses), _ptr(self.disp), _ptr(self.targets), _ptr(self.weights), _ptr(self.ii),
                           _ptr(self.jj), self.K, self.E, self.h, self.w, self.n_fixed, fx, fy, cx, cy,
                           _ptr(self.status))
        if self.imu is not None:
            pr.imu, pr.vel, pr.bias, pr.bias_hat = (_ptr(self.imu), _ptr(self.vel), _ptr(self.bias),
                                                    _ptr(self.bias_hat))
            pr.gravity[:] = self.gravity
        return pr


def gs_ba_workspace_size(K: int, E: int, h: int, w: int, n_fixed: int, inertial: bool = False) -> int:
    return int(load_library().gs_ba_workspace_size(K, E, h, w, n_fixed, int(bool(inertial))))


def gs_ba_step(win: BAWindow, lam: float = 1e-4, eps: float = 1e-4, stream=None):
    """One Levenberg-Marquardt step in place; win.cost gets the cost before the step."""
    pr = win.struct()
    _check(load_library().gs_ba_step(ctypes.byref(pr), float(lam), float(eps), _ptr(win.cost), _ptr(win.ws),
                                     win.ws.numel() * 4, _stream(stream)), "gs_ba_step")
