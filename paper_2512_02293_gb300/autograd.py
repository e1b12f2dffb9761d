"""torch.autograd binding of the differentiable renderer.

``render(gaussians..., pose_xi, rasterizer)`` renders colour and depth of every
view through the C ABI (gs_project_perturbed -> gs_bin_sort -> gs_render_fwd)
and, in backward, runs the hand-written backward kernels
(gs_render_bwd_raster -> gs_project_bwd_perturbed), which start from the
per-pixel checkpoint (T_final, n_contrib) the forward wrote and return the
gradients of every Gaussian parameter and of each view's 6-DoF pose tangent
xi = (rho, phi) (left perturbation T_cw <- Exp(xi) T_cw), the gradient a
tracker needs.

Pose convention: the cameras given to the Rasterizer are the base poses;
``pose_xi`` (device [n_views, 6]) is applied on the device, view v rendered from
Exp(xi_v) T_cw, and the returned pose gradient is the left-perturbation
gradient at the rendered pose, i.e. d L / d xi exactly at xi = 0.  A tracker
keeps xi at zero, steps along -grad, and folds the step into the base pose.

No host synchronisation in forward or backward, so an iteration can be
captured in a CUDA graph: the key buffers are sized once (the first forward
measures the key count, or the caller passes a capacity), an overflow sets the
device status word, and the caller checks it outside the graph with
``Rasterizer.check()`` / ``ensure_capacity()`` (grow and redo), as
mapping.MappingStep does.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import gs as G


def so3_exp(phi) -> np.ndarray:
    """Rotation matrix of the rotation vector phi (Rodrigues)."""
    phi = np.asarray(phi, dtype=np.float64)
    th = float(np.linalg.norm(phi))
    K = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    if th < 1e-12:
        return np.eye(3) + K
    return np.eye(3) + math.sin(th) / th * K + (1 - math.cos(th)) / (th * th) * K @ K


def se3_left_update(cam, xi):
    """Camera with world-to-camera pose Exp(xi) T_cw (xi = (rho, phi); the
    translation uses the first-order V = I, exact in the limit xi -> 0)."""
    from .synth import Camera
    R_wc = np.asarray(cam.R_wc, np.float64); t_wc = np.asarray(cam.t_wc, np.float64)
    Rcw = R_wc.T; tcw = -R_wc.T @ t_wc
    Rphi = so3_exp(xi[3:])
    Rcw2 = Rphi @ Rcw
    tcw2 = Rphi @ tcw + np.asarray(xi[:3], np.float64)
    return Camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height, Rcw2.T, -Rcw2.T @ tcw2)


class Rasterizer:
    """Device buffers for rendering n Gaussians into a fixed set of views."""

    def __init__(self, cams, n: int, params: G.RenderParams | None = None, device="cuda", headroom=1.3,
                 key_capacity: int | None = None):
        self.cams = list(cams)
        self.params = params or G.RenderParams()
        self.n = int(n)
        self.V = len(self.cams)
        self.device = torch.device(device)
        self.total_tiles = G.gs_total_tiles(self.cams, self.params.tile)
        self.total_pixels = G.gs_total_pixels(self.cams)
        self.proj = G.Projected.empty(self.n * self.V, self.device)
        self.img = G.Image.empty(self.total_pixels, self.device)
        self.headroom = headroom
        self.bins = None
        self.ws = None
        if key_capacity is not None:
            self._alloc(key_capacity)

    def _alloc(self, capacity):
        capacity = max(int(capacity), 1024)
        self.bins = G.Bins.empty(capacity, self.total_tiles, self.device)
        ws = G.gs_workspace_size(self.n, self.cams, self.params, capacity)
        self.ws = torch.empty((ws + 255) // 256 * 64, device=self.device, dtype=torch.float32)

    def check(self) -> int:
        """Device status word of the last passes (0 = fine); synchronises."""
        return 0 if self.bins is None else G.gs_read_device_status(self.bins.status)

    def ensure_capacity(self) -> bool:
        """Grow the key buffers if a pass overflowed them (outside any graph);
        True if they were grown, in which case the iteration must be redone."""
        st = self.check()
        m = int(self.bins.num_keys.item()) & 0xFFFFFFFF if self.bins is not None else 0
        if st == G.GS_ERR_CAPACITY or (self.bins is not None and m > self.bins.capacity):
            self._alloc(int(m * self.headroom) + 1024)
            return True
        if st != 0:
            raise G.GsError(st, "device status")
        return False

    def forward(self, g: G.Gaussians, xi):
        G.gs_project(g, self.cams, self.params, self.proj, xi=xi)
        if self.bins is None:       # first call without a given capacity: measure (a host read, before any capture)
            self._alloc(int(self.proj.tiles_touched.to(torch.int64).sum().item() * self.headroom) + 1024)
        G.gs_bin_sort(self.proj, self.n, self.cams, self.params, self.bins, self.ws)
        G.gs_render_fwd(self.proj, self.bins, self.cams, self.params, self.img)


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mean, quat, log_scale, opacity_logit, color, pose_xi, rast: Rasterizer):
        g = G.Gaussians(mean.detach().contiguous(), quat.detach().contiguous(), log_scale.detach().contiguous(),
                        opacity_logit.detach().contiguous(), color.detach().contiguous())
        xi = pose_xi.detach().reshape(rast.V, 6).contiguous().float()
        rast.forward(g, xi)
        ctx.rast = rast
        ctx.g = g
        ctx.xi = xi
        # the checkpoint lives in rast.img; the outputs are copies so that a later
        # render into the same buffers cannot change them
        return rast.img.color.clone(), rast.img.depth.clone()

    @staticmethod
    def backward(ctx, dcolor, ddepth):
        rast = ctx.rast
        g = ctx.g
        grads = G.Grads.empty_like(g, rast.V)
        iso = torch.zeros(1, device=rast.device)
        dcolor = dcolor.contiguous().float() if dcolor is not None else torch.zeros_like(rast.img.color)
        ddepth = ddepth.contiguous().float() if ddepth is not None else torch.zeros_like(rast.img.depth)
        G.gs_render_bwd_raster(rast.proj, rast.bins, rast.img, dcolor, ddepth, rast.cams, rast.params, g.n, rast.ws)
        G.gs_project_bwd(g, rast.cams, rast.params, rast.ws, 0.0, grads, iso, xi=ctx.xi)
        return grads.mean, grads.quat, grads.log_scale, grads.opacity_logit, grads.color, grads.pose, None


def render(mean, quat, log_scale, opacity_logit, color, pose_xi, rast: Rasterizer):
    """Differentiable render of every view: returns (colour [3 P], depth [P]),
    views packed back to back as in gs.h."""
    return _Render.apply(mean, quat, log_scale, opacity_logit, color, pose_xi, rast)
