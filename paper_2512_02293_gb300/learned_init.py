"""Learned initialisation of the Gaussians a new keyframe inserts.

When a keyframe joins the map (Sec. 3.3 "Map Management"), its pixels are
back-projected with their depth into new Gaussians whose opacity starts at 0.5;
their size and orientation are left to the mapper.  Here a small network reads
the 7 x 7 RGB-D patch around each inserted pixel and predicts, in the camera
frame, the Gaussian the mapper would have converged to: log-scale offsets from
the footprint heuristic, a rotation and an opacity logit.  The heuristic
(isotropic footprint scale, identity rotation, opacity 0.5) stays the fallback.

Everything numeric runs in libgs: patches (gs_extract_patches), insertion
(gs_insert_gaussians), the network's forward / backward on the tensor cores
(gs_mlp_fwd / gs_mlp_bwd), Adam (gs_adam_step) and the mapper that produces the
training targets (MappingStep); the evaluation metrics (PSNR, depth L1) are
plain torch reductions.  The host only canonicalises targets (numpy): the
three axes are ordered by increasing scale, the rotation's columns follow, the
axes' signs are fixed (smallest axis towards the camera, middle axis with
non-negative camera-x, right-handed), and the quaternion's sign by w >= 0, so
that every Gaussian has one target.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import gs as G
from . import synth
from .mapping import MapParams, MappingStep


@dataclass
class InitConfig:
    stride: float = 2.5          # sample spacing in pixels: ~49k samples per 640x480 keyframe
    map_iters: int = 100         # mapper iterations behind a training target
    n_views: int = 3             # keyframe + neighbours the mapper fits
    baseline: float = 0.15       # metres between neighbouring views (sideways, same orientation)
    room_gaussians: int = 100_000
    width: int = 640
    height: int = 480
    focal: float = 525.0


def grid_samples(cam, stride: float, device="cuda"):
    """Pixels (u, v) of a regular grid with `stride` px spacing (int32 [n, 2])."""
    import torch
    us = np.floor((np.arange(int(cam.width / stride)) + 0.5) * stride).astype(np.int32)
    vs = np.floor((np.arange(int(cam.height / stride)) + 0.5) * stride).astype(np.int32)
    us = us[us < cam.width]; vs = vs[vs < cam.height]
    uu, vv = np.meshgrid(us, vs)
    uv = np.stack([uu.reshape(-1), vv.reshape(-1)], 1).astype(np.int32)
    return torch.from_numpy(np.ascontiguousarray(uv)).to(device)


def _quat_to_rot(q):
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                     np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                     np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)


def canonical_targets(log_scale, quat, logit, R_wc, s0):
    """Targets [n, 8] = (log-scale offsets from s0, ascending; camera-frame
    quaternion (w, x, y, z), w >= 0, of the axes in that order with fixed signs;
    opacity logit)."""
    from scipy.spatial.transform import Rotation
    R_cam = np.asarray(R_wc, np.float64).T[None] @ _quat_to_rot(np.asarray(quat, np.float64))
    order = np.argsort(log_scale, axis=1)
    ls = np.take_along_axis(np.asarray(log_scale, np.float64), order, 1)
    Rp = np.take_along_axis(R_cam, order[:, None, :].repeat(3, 1), 2)
    # an axis and its negation describe the same Gaussian: the smallest axis (a
    # surface's normal) points towards the camera, the middle one has a
    # non-negative camera-x component, the largest completes a right-handed frame
    a0 = Rp[:, :, 0] * np.where(Rp[:, 2, 0] > 0, -1.0, 1.0)[:, None]
    a1 = Rp[:, :, 1] * np.where(Rp[:, 0, 1] < 0, -1.0, 1.0)[:, None]
    Rp = np.stack([a0, a1, np.cross(a0, a1)], 2)
    xyzw = Rotation.from_matrix(Rp).as_quat()
    q = np.stack([xyzw[:, 3], xyzw[:, 0], xyzw[:, 1], xyzw[:, 2]], 1)
    q[q[:, 0] < 0] *= -1.0
    return np.concatenate([ls - np.asarray(s0, np.float64)[:, None], q, np.asarray(logit, np.float64)[:, None]],
                          1).astype(np.float32)


class LearnedInit:
    """The initialiser network: FP32 master weights, BF16 operands, Adam."""

    def __init__(self, seed: int = 0, device="cuda"):
        import torch
        self.device = device
        self.params = {k: torch.from_numpy(v).to(device) for k, v in synth.mlp_params(seed, bias_sd=0.0).items()}
        self.m = {k: torch.zeros_like(v) for k, v in self.params.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.params.items()}
        self.grads = {k: torch.empty_like(v) for k, v in self.params.items()}
        self.d_step = torch.zeros(2, device=device, dtype=torch.int32)
        self.packed = G.MlpPacked(device)
        self.status = torch.zeros(4, device=device, dtype=torch.int32)
        G.gs_mlp_pack(self.params, self.packed)

    def predict(self, X):
        import torch
        Y = torch.empty(X.shape[0], G.MLP_OUT, device=self.device)
        G.gs_mlp_fwd(self.packed, X, Y=Y, status=self.status)
        return Y

    def train(self, X, T, epochs: int, batch: int = 16384, lr: float = 1e-3):
        """Mini-batch Adam on the mean squared error; X, T in a fixed shuffled
        order.  Returns the mean training loss of every epoch."""
        import torch
        n = X.shape[0]
        Z1 = torch.empty(batch, G.MLP_HIDDEN, device=self.device, dtype=torch.bfloat16)
        Z2 = torch.empty_like(Z1)
        dY = torch.empty(batch, G.MLP_OUT, device=self.device)
        loss = torch.zeros(1, device=self.device)
        out = []
        for _ in range(epochs):
            loss.zero_()
            for b0 in range(0, n, batch):
                b1 = min(n, b0 + batch)
                m = b1 - b0
                x, t = X[b0:b1], T[b0:b1]
                G.gs_mlp_pack(self.params, self.packed)
                G.gs_mlp_fwd(self.packed, x, Z1=Z1[:m], Z2=Z2[:m], T=t, dY=dY[:m], loss=loss,
                             loss_scale=1.0 / (G.MLP_OUT * m), status=self.status)
                G.gs_mlp_bwd(self.packed, x, Z1[:m], Z2[:m], dY[:m], self.grads, status=self.status)
                G.gs_adam_step([(self.params[k], self.grads[k], self.m[k], self.v[k], lr) for k in G.MLP_PARAM_NAMES],
                               0.9, 0.999, 1e-8, self.d_step)
            out.append(loss.item() * batch / n)
        G.gs_mlp_pack(self.params, self.packed)
        if G.gs_read_device_status(self.status) != 0:
            raise G.GsError(G.gs_read_device_status(self.status), "learned init training")
        return out


# ------------------------------------------------------------- one keyframe

def keyframe_window(seed: int, cfg: InitConfig):
    """The keyframe (a seeded pose inside the room) and n_views - 1 neighbours
    displaced sideways by multiples of cfg.baseline with the same orientation,
    so that the views overlap like consecutive keyframes of a slow sweep."""
    (c0,), _ = synth.trajectory_cameras(seed, [(cfg.width, cfg.height, cfg.focal)])
    R = np.asarray(c0.R_wc, np.float64)
    cams = [c0]
    for k in range(1, cfg.n_views):
        off = (k + 1) // 2 * cfg.baseline * (1 if k % 2 else -1)
        t = np.asarray(c0.t_wc, np.float64) + R @ np.array([off, 0.0, 0.0])
        cams.append(synth.Camera(c0.fx, c0.fy, c0.cx, c0.cy, c0.width, c0.height, c0.R_wc, t.astype(np.float32)))
    return cams


class Keyframe:
    """A synthetic room seen by n_views nearby cameras; view 0 is the keyframe
    whose pixels are inserted.  The ground-truth map is rendered once
    (colour and depth) and serves as the mapper's target."""

    def __init__(self, seed: int, cfg: InitConfig, device="cuda"):
        import torch
        self.cfg = cfg
        self.cams = keyframe_window(seed, cfg)
        g = synth.room_scene(cfg.room_gaussians, seed, keep_out=[c.t_wc for c in self.cams])
        P = G.gs_total_pixels(self.cams)
        r = MappingStep(G.Gaussians.from_numpy(g, device), self.cams, torch.zeros(3 * P, device=device),
                        torch.zeros(P, device=device), G.RenderParams(tile=16), MapParams())
        r.render()
        self.color = r.img.color.clone()
        self.depth = r.img.depth.clone()
        c0 = self.cams[0]
        self.color0 = self.color[:3 * c0.n_pixels]
        self.depth0 = self.depth[:c0.n_pixels]
        self.uv = grid_samples(c0, cfg.stride, device)
        self.n = self.uv.shape[0]
        self.X = torch.empty(self.n, G.MLP_IN_STRIDE, device=device, dtype=torch.bfloat16)
        G.gs_extract_patches(self.color0, self.depth0, c0, self.uv, self.X)
        uvh = self.uv.cpu().numpy()
        d = self.depth0.cpu().numpy().reshape(c0.height, c0.width)[uvh[:, 1], uvh[:, 0]]
        self.valid = d > 0
        self.s0 = np.log(np.maximum(d, 1e-6) * cfg.stride / (0.5 * (c0.fx + c0.fy)))

    def new_map(self, Y=None, device="cuda"):
        """The inserted Gaussians alone: heuristic (Y None) or learned."""
        import torch
        n = self.n
        g = G.Gaussians(torch.empty(n, 3, device=device), torch.empty(n, 4, device=device),
                        torch.empty(n, 3, device=device), torch.empty(n, device=device),
                        torch.empty(n, 3, device=device))
        G.gs_insert_gaussians(self.color0, self.depth0, self.cams[0], self.uv, self.cfg.stride, g, 0, Y=Y)
        return g

    def mapper(self, g, mparams: MapParams | None = None):
        return MappingStep(g, self.cams, self.color, self.depth, G.RenderParams(tile=16), mparams or MapParams())

    def psnr(self, step: MappingStep) -> float:
        """PSNR (dB) of the mapper's last render of the keyframe (view 0, whose
        pixels the inserted Gaussians came from) against its ground truth."""
        P = self.cams[0].n_pixels
        diff = (step.img.color[:3 * P] - self.color0).double()
        mse = float((diff * diff).mean().item())
        return -10.0 * math.log10(max(mse, 1e-20))

    def depth_l1(self, step: MappingStep) -> float:
        """Mean absolute depth error (m) of the keyframe's last render."""
        P = self.cams[0].n_pixels
        return float((step.img.depth[:P] - self.depth0).abs().mean().item())


def training_pairs(seed: int, cfg: InitConfig, device="cuda"):
    """(X, T) of one room: patches of the keyframe's samples and the canonical
    form of the Gaussians the mapper reaches from the heuristic insertion."""
    import torch
    kf = Keyframe(seed, cfg, device)
    g = kf.new_map()
    step = kf.mapper(g)
    for _ in range(cfg.map_iters):
        step.step()
    if step.ensure_capacity():
        raise RuntimeError("key capacity grew during target generation")
    T = canonical_targets(g.log_scale.cpu().numpy(), g.quat.cpu().numpy(), g.opacity_logit.cpu().numpy(),
                          kf.cams[0].R_wc, kf.s0)
    keep = np.nonzero(kf.valid & np.all(np.isfinite(T), 1))[0]
    idx = torch.from_numpy(keep).to(device)
    return kf.X.index_select(0, idx), torch.from_numpy(T[keep]).to(device)


def mapping_curve(kf: Keyframe, Y, iters: int):
    """PSNR after every mapper iteration from the heuristic (Y None) or learned
    insertion; the map is rendered before each iteration's update."""
    g = kf.new_map(Y)
    step = kf.mapper(g)
    curve = []
    for _ in range(iters):
        step.step()
        curve.append(kf.psnr(step))
    step.render()
    curve.append(kf.psnr(step))
    return np.array(curve[1:]), kf.depth_l1(step)


def iterations_to_reach(curve, target: float) -> int | None:
    """1-based index of the first iteration whose PSNR reaches `target`."""
    hit = np.nonzero(curve >= target)[0]
    return int(hit[0]) + 1 if hit.size else None
