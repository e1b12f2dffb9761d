"""Pose refinement through the re-rendering loss.

The paper's tracker estimates poses by visual-inertial bundle adjustment and
names, as a limitation, that the Gaussian map does not feed back into
tracking (Sec. 4, "Limitations").  The differentiable renderer's pose tangent
gradient closes that loop: with the map held fixed, a keyframe's pose is
driven by the gradient of the same colour + depth loss the mapper minimises
(Eq. 6).  Each iteration renders the keyframe (gs_project -> gs_bin_sort ->
gs_render_fwd), takes the loss and its image gradient (gs_loss), runs the
backward (gs_render_bwd) for the pose tangent xi = (rho, phi) of the left
perturbation T_cw <- Exp(xi) T_cw, and folds an Adam step on xi into the pose.
The camera is a host value of the C ABI, so each iteration reads the six
gradient components back (24 bytes).

TrajectoryTracker runs the refinement over a sequence of keyframes: each
keyframe starts from the previous keyframe's estimate carried along the
sequence's relative motion (a motion prior), plus fresh noise, and the error
over the sequence is reported as the absolute trajectory error (RMSE of the
camera centres; the estimates live in the map's frame, so no alignment).
"""
from __future__ import annotations

import math

import numpy as np

from . import gs as G
from .autograd import se3_left_update
from .mapping import MapParams, MappingStep


def pose_error(cam, cam_ref):
    """(translation error in m, rotation error in rad) between two camera-to-world poses."""
    Ra = np.asarray(cam.R_wc, np.float64); Rb = np.asarray(cam_ref.R_wc, np.float64)
    dt = float(np.linalg.norm(np.asarray(cam.t_wc, np.float64) - np.asarray(cam_ref.t_wc, np.float64)))
    # angle from both the symmetric and the skew part of Ra^T Rb (stable at small
    # angles, where the trace alone loses half the digits)
    M = Ra.T @ Rb
    s = 0.5 * np.linalg.norm([M[2, 1] - M[1, 2], M[0, 2] - M[2, 0], M[1, 0] - M[0, 1]])
    c = (np.trace(M) - 1.0) / 2.0
    return dt, float(math.atan2(s, c))


class PoseAdam:
    """Adam on the 6-vector pose tangent, folded into the pose after every step
    (T_cw <- Exp(-step) T_cw), with the learning rate decayed exponentially from
    lr to lr_final over `iters` steps.  Host arithmetic in float64."""

    def __init__(self, lr: float = 5e-3, lr_final: float = 5e-5, iters: int = 250, beta1: float = 0.9,
                 beta2: float = 0.999, eps: float = 1e-12):
        self.lr, self.lr_final, self.iters = lr, lr_final, iters
        self.b1, self.b2, self.eps = beta1, beta2, eps
        self.m = np.zeros(6); self.v = np.zeros(6); self.t = 0

    def step(self, cam, grad):
        """The camera after one Adam step along the pose gradient `grad` (6)."""
        g = np.asarray(grad, np.float64)
        self.t += 1
        frac = min(1.0, (self.t - 1) / max(1, self.iters - 1))
        lr = self.lr * (self.lr_final / self.lr) ** frac          # exponential decay over the run
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t); vh = self.v / (1 - self.b2 ** self.t)
        return se3_left_update(cam, -lr * mh / (np.sqrt(vh) + self.eps))


class PoseTracker:
    """Refines one keyframe's pose against target colour and depth images with
    the map fixed."""

    def __init__(self, gaussians: G.Gaussians, cam, target_color, target_depth, params: G.RenderParams | None = None,
                 lambda_c: float = 0.9, lambda_d: float = 0.1, lr: float = 5e-3, lr_final: float = 5e-5,
                 iters: int = 250, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-12):
        self.cam = cam
        self.step = MappingStep(gaussians, [cam], target_color, target_depth, params or G.RenderParams(),
                                MapParams(lambda_c, lambda_d, 0.0))
        self.iters = iters
        self.adam = PoseAdam(lr, lr_final, iters, beta1, beta2, eps)

    def gradient(self):
        """(loss, pose gradient) at the current pose."""
        self.step.cams[0] = self.cam
        self.step.render()
        self.step.loss_and_backward()
        if self.step.ensure_capacity():                 # more keys than buffered: redo with grown buffers
            self.step.render()
            self.step.loss_and_backward()
        return float(self.step.loss().item()), self.step.grads.pose[0].cpu().numpy().astype(np.float64)

    def iterate(self) -> float:
        """One refinement step; returns the loss at the pose before the step."""
        loss, g = self.gradient()
        self.cam = self.adam.step(self.cam, g)
        return loss

    def run(self, iters: int | None = None):
        """Run the refinement; returns the loss of every iteration."""
        return [self.iterate() for _ in range(iters or self.iters)]


def world_to_camera(cam) -> np.ndarray:
    """4 x 4 world-to-camera transform of a camera-to-world pose."""
    R = np.asarray(cam.R_wc, np.float64); t = np.asarray(cam.t_wc, np.float64)
    T = np.eye(4)
    T[:3, :3] = R.T
    T[:3, 3] = -R.T @ t
    return T


def with_world_to_camera(cam, T):
    """`cam` with its pose replaced by the world-to-camera transform T."""
    from .synth import Camera
    R = T[:3, :3].T
    return Camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height, R, -R @ T[:3, 3])


class TrajectoryTracker:
    """Pose refinement over a sequence of keyframes with the map fixed.  Keyframe
    k starts from Exp(noise_k) E_{k-1} T_cw(k), where E_{k-1} = T_est T_true^-1 is
    the previous keyframe's remaining error (the relative motion between the
    keyframes is taken as known, as a motion prior would give it) and noise_k a
    fresh perturbation of up to `noise_m` metres and `noise_rad` radians per
    axis.  `targets` are the colour / depth images of each keyframe."""

    def __init__(self, gaussians: G.Gaussians, cams, targets, params: G.RenderParams | None = None,
                 iters: int = 250, noise_m: float = 0.03, noise_rad: float = 0.02, seed: int = 0):
        self.g = gaussians
        self.cams = list(cams)
        self.targets = list(targets)
        self.params = params or G.RenderParams()
        self.iters = iters
        self.noise_m, self.noise_rad = noise_m, noise_rad
        self.rng = np.random.default_rng(seed)

    def run(self) -> dict:
        E = np.eye(4)
        starts, estimates, losses = [], [], []
        for cam, (tc, td) in zip(self.cams, self.targets):
            noise = np.concatenate([self.rng.uniform(-1, 1, 3) * self.noise_m, self.rng.uniform(-1, 1, 3) * self.noise_rad])
            start = se3_left_update(with_world_to_camera(cam, E @ world_to_camera(cam)), noise)
            tr = PoseTracker(self.g, start, tc, td, self.params, iters=self.iters)
            losses.append(tr.run())
            starts.append(start)
            estimates.append(tr.cam)
            E = world_to_camera(tr.cam) @ np.linalg.inv(world_to_camera(cam))
        err_start = np.array([pose_error(s, c) for s, c in zip(starts, self.cams)])
        err = np.array([pose_error(e, c) for e, c in zip(estimates, self.cams)])
        return {"estimates": estimates, "starts": starts, "losses": losses,
                "ate_rmse_m": float(np.sqrt(np.mean(err[:, 0] ** 2))),
                "rot_rmse_rad": float(np.sqrt(np.mean(err[:, 1] ** 2))),
                "start_ate_rmse_m": float(np.sqrt(np.mean(err_start[:, 0] ** 2))),
                "start_rot_rmse_rad": float(np.sqrt(np.mean(err_start[:, 1] ** 2))),
                "per_keyframe_err_m_rad": err.tolist()}
