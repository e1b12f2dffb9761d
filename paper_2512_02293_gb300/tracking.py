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


class PoseTracker:
    """Refines one keyframe's pose against target colour and depth images with
    the map fixed."""

    def __init__(self, gaussians: G.Gaussians, cam, target_color, target_depth, params: G.RenderParams | None = None,
                 lambda_c: float = 0.9, lambda_d: float = 0.1, lr: float = 5e-3, lr_final: float = 5e-5,
                 iters: int = 250, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-12):
        self.cam = cam
        self.step = MappingStep(gaussians, [cam], target_color, target_depth, params or G.RenderParams(),
                                MapParams(lambda_c, lambda_d, 0.0))
        self.lr, self.lr_final, self.iters = lr, lr_final, iters
        self.b1, self.b2, self.eps = beta1, beta2, eps
        self.m = np.zeros(6); self.v = np.zeros(6); self.t = 0

    def iterate(self) -> float:
        """One refinement step; returns the loss at the pose before the step."""
        self.step.cams[0] = self.cam
        self.step.render()
        self.step.loss_and_backward()
        if self.step.ensure_capacity():                 # more keys than buffered: redo with grown buffers
            self.step.render()
            self.step.loss_and_backward()
        g = self.step.grads.pose[0].cpu().numpy().astype(np.float64)
        loss = float(self.step.loss().item())
        self.t += 1
        frac = min(1.0, (self.t - 1) / max(1, self.iters - 1))
        lr = self.lr * (self.lr_final / self.lr) ** frac          # exponential decay over the run
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t); vh = self.v / (1 - self.b2 ** self.t)
        self.cam = se3_left_update(self.cam, -lr * mh / (np.sqrt(vh) + self.eps))
        return loss

    def run(self, iters: int | None = None):
        """Run the refinement; returns the loss of every iteration."""
        return [self.iterate() for _ in range(iters or self.iters)]
