"""Final colour refinement of the Gaussian map (Sec. 3.3 "Final Color
Refinement"): after the run, every iteration draws one keyframe uniformly at
random from the whole keyframe list and takes one mapping step on the map for
that keyframe alone: the colour + depth L1 loss of Eq. 6 with the isotropic
regulariser, its backward, and Adam.

The loop runs on the mapping kernels.  One MappingStep holds the map, the Adam
state and the buffers for every keyframe: the keyframes share the camera
resolution, so one view's image, key and workspace buffers serve all of them.
The targets of all keyframes stay resident on the device.  One CUDA graph per
keyframe is captured with that keyframe's camera and targets. An iteration
replays the graph of the drawn keyframe, with no host marshalling and no copy of
targets. The key buffers are sized for the keyframe with the most keys. The
device status word is read every `check_every` iterations; an overflow regrows
the buffers and recaptures the graphs.
"""
from __future__ import annotations

import numpy as np
import torch

from . import gs as G
from .mapping import MapParams, MappingStep


class ColourRefiner:
    def __init__(self, gaussians: G.Gaussians, cams, target_colors, target_depths,
                 params: G.RenderParams | None = None, mparams: MapParams | None = None, seed: int = 0,
                 headroom: float = 1.3):
        self.cams = list(cams)
        if not self.cams:
            raise ValueError("no keyframes")
        w, h = self.cams[0].width, self.cams[0].height
        if any((c.width, c.height) != (w, h) for c in self.cams):
            raise ValueError("the keyframes must share the camera resolution")
        if len(target_colors) != len(self.cams) or len(target_depths) != len(self.cams):
            raise ValueError("one target colour and depth image per keyframe")
        self.colors = [t.contiguous() for t in target_colors]
        self.depths = [t.contiguous() for t in target_depths]
        self.g = gaussians
        self.params = params or G.RenderParams()
        self.headroom = headroom
        self.rng = np.random.default_rng(seed)
        proj = G.Projected.empty(gaussians.n, gaussians.mean.device)
        self.step = MappingStep(gaussians, [self.cams[0]], self.colors[0], self.depths[0], self.params, mparams,
                                key_capacity=self._max_keys(proj), headroom=headroom)
        self.graphs = []
        self._capture_all()
        self.iterations = 0
        self.draws = np.zeros(len(self.cams), dtype=np.int64)

    def _max_keys(self, proj) -> int:
        """Keys of the keyframe with the most (host read; outside any graph)."""
        m = 0
        for c in self.cams:
            G.gs_project(self.g, [c], self.params, proj)
            m = max(m, int(proj.tiles_touched.to(torch.int64).sum().item()))
        return int(m * self.headroom) + 1024

    def _capture_all(self):
        s = self.step
        self.graphs = []
        for c, tc, td in zip(self.cams, self.colors, self.depths):
            s.cams = [c]
            s.target_color, s.target_depth = tc, td
            s.graph = None
            self.graphs.append(s.capture(warmup=0))
        s.graph = None

    def check(self) -> bool:
        """Read the device status word; regrow the key buffers and recapture if
        a step overflowed them.  Returns True if it did."""
        st = self.step.check()
        if st == G.GS_ERR_CAPACITY or self.step.num_keys() > self.step.bins.capacity:
            proj = G.Projected.empty(self.g.n, self.g.mean.device)
            self.step._alloc_bins(self._max_keys(proj))
            self.step.bins.status.zero_()
            self._capture_all()
            return True
        if st != 0:
            raise G.GsError(st, "device status")
        return False

    def run(self, iters: int, check_every: int = 50):
        """`iters` refinement iterations; returns the keyframe index drawn for each."""
        drawn = self.rng.integers(0, len(self.cams), size=iters)
        for i, k in enumerate(drawn):
            self.graphs[k].replay()
            if (i + 1) % check_every == 0 and self.check():
                # the last check_every steps may have run with overflowed keys:
                # nothing is undone, later steps run with the grown buffers
                pass
        self.iterations += iters
        np.add.at(self.draws, drawn, 1)
        return drawn

    def render_psnr(self, k: int) -> float:
        """PSNR (dB) of keyframe k's render against its target colour (eager
        render; leaves the step's buffers holding keyframe k)."""
        s = self.step
        s.cams = [self.cams[k]]
        s.render()
        diff = (s.img.color - self.colors[k]).double()
        mse = float((diff * diff).mean().item())
        return -10.0 * np.log10(max(mse, 1e-20))

    def mean_psnr(self) -> float:
        return float(np.mean([self.render_psnr(k) for k in range(len(self.cams))]))
