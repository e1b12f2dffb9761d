"""One mapping iteration of Sec. 3.3 "Map Management" on the GPU:

    render colour and depth of every view -> Eq. 6 loss -> backward -> Adam

driven through the C ABI (gs_project, gs_bin_sort, gs_render_fwd, gs_loss,
gs_render_bwd, gs_adam_step).  All buffers are allocated once, up front, by
torch; the iteration itself allocates nothing and reads nothing back, so it
can be captured into a CUDA graph and replayed (``capture()`` / ``replay()``).

The number of (tile, Gaussian) keys depends on the map and the poses.  The key
buffers get a capacity with headroom from a first, uncaptured pass; every call
checks the device status word only when asked (``check()``), so an overflow
during replay is detected after the fact and ``ensure_capacity`` grows the
buffers.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import gs as G

PARAM_NAMES = ("mean", "quat", "log_scale", "opacity_logit", "color")


@dataclass
class MapParams:
    lambda_c: float = 0.9
    lambda_d: float = 0.1
    lambda_iso: float = 10.0
    lr: tuple = (1e-3, 1e-3, 5e-3, 5e-2, 2.5e-3)   # mean, quat, log_scale, logit, colour
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15


class MappingStep:
    def __init__(self, gaussians: G.Gaussians, cams, target_color: torch.Tensor, target_depth: torch.Tensor,
                 params: G.RenderParams | None = None, mparams: MapParams | None = None,
                 key_capacity: int | None = None, headroom: float = 1.3, fused_loss: bool = True):
        self.g = gaussians
        self.fused_loss = bool(fused_loss)
        self.cams = list(cams)
        self.params = params or G.RenderParams()
        self.mp = mparams or MapParams()
        dev = gaussians.mean.device
        self.device = dev
        self.n = gaussians.n
        self.V = len(self.cams)
        self.E = self.n * self.V
        self.total_tiles = G.gs_total_tiles(self.cams, self.params.tile)
        self.total_pixels = G.gs_total_pixels(self.cams)
        assert target_color.numel() == 3 * self.total_pixels and target_depth.numel() == self.total_pixels
        self.target_color = target_color.contiguous()
        self.target_depth = target_depth.contiguous()
        self.proj = G.Projected.empty(self.E, dev)
        self.img = G.Image.empty(self.total_pixels, dev)
        self.dL_dcolor = torch.empty(3 * self.total_pixels, device=dev, dtype=torch.float32)
        self.dL_ddepth = torch.empty(self.total_pixels, device=dev, dtype=torch.float32)
        self.loss_terms = torch.zeros(self.V, 2, device=dev, dtype=torch.float32)
        self.iso = torch.zeros(1, device=dev, dtype=torch.float32)
        self.grads = G.Grads.empty_like(gaussians, self.V)
        self.m = [torch.zeros_like(t) for t in gaussians.tensors()]
        self.v = [torch.zeros_like(t) for t in gaussians.tensors()]
        self.d_step = torch.zeros(2, device=dev, dtype=torch.int32)
        # fused loss: per-view totals carried from the forward to the backward call
        self.loss_ws = (torch.zeros((G.gs_fused_loss_workspace_size(self.V) + 3) // 4, device=dev,
                                    dtype=torch.float32) if self.fused_loss else None)
        self.stages = self.FUSED_STAGES if self.fused_loss else self.STAGES
        self.headroom = headroom
        self.graph = None
        self._io_stream = None
        self._bound = None          # the calls marshalled once (eager step); rebuilt when stale
        self._bound_key = None
        self._alloc_bins(key_capacity if key_capacity is not None else self._measure_keys())

    # -------------------------------------------------------------- buffers
    def _alloc_bins(self, capacity: int):
        capacity = max(int(capacity), 1024)
        self.bins = G.Bins.empty(capacity, self.total_tiles, self.device)
        ws = G.gs_workspace_size(self.n, self.cams, self.params, capacity)
        self.ws = torch.empty((ws + 255) // 256 * 64, device=self.device, dtype=torch.float32)
        self.graph = None
        self._bound = None

    def _measure_keys(self) -> int:
        """Project once and count the keys (host read; outside any graph)."""
        G.gs_project(self.g, self.cams, self.params, self.proj)
        m = int(self.proj.tiles_touched.to(torch.int64).sum().item())
        return int(m * self.headroom) + 1024

    def num_keys(self) -> int:
        return int(self.bins.num_keys.item()) & 0xFFFFFFFF

    def check(self) -> int:
        """Device status word (0 = fine); synchronises the stream."""
        return G.gs_read_device_status(self.bins.status)

    def ensure_capacity(self) -> bool:
        """Grow the key buffers if the last pass overflowed.  Returns True if grown."""
        st = self.check()
        if st == G.GS_ERR_CAPACITY or self.num_keys() > self.bins.capacity:
            self._alloc_bins(int(self.num_keys() * self.headroom) + 1024)
            return True
        if st != 0:
            raise G.GsError(st, "device status")
        return False

    # ------------------------------------------------------------ iteration
    def render(self):
        """Projection, binning and the forward pass (with the fused loss, also the
        loss terms against the current targets)."""
        G.gs_project(self.g, self.cams, self.params, self.proj)
        G.gs_bin_sort(self.proj, self.n, self.cams, self.params, self.bins, self.ws)
        if self.fused_loss:
            G.gs_render_fwd_loss(self.proj, self.bins, self.cams, self.params, self.img, self.target_color,
                                 self.target_depth, self.loss_terms, self.loss_ws)
        else:
            G.gs_render_fwd(self.proj, self.bins, self.cams, self.params, self.img)

    def loss_and_backward(self):
        """Eq. 6 loss and the gradients of every parameter and pose tangent (after render())."""
        if self.fused_loss:
            G.gs_render_bwd_raster_loss(self.proj, self.bins, self.img, self.target_color, self.target_depth,
                                        self.mp.lambda_c, self.mp.lambda_d, self.loss_ws, self.cams, self.params,
                                        self.n, self.ws)
            G.gs_project_bwd(self.g, self.cams, self.params, self.ws, self.mp.lambda_iso, self.grads, self.iso)
            return
        G.gs_loss(self.img, self.target_color, self.target_depth, self.cams, self.mp.lambda_c, self.mp.lambda_d,
                  self.dL_dcolor, self.dL_ddepth, self.loss_terms, self.ws)
        G.gs_render_bwd(self.g, self.proj, self.bins, self.img, self.dL_dcolor, self.dL_ddepth, self.cams,
                        self.params, self.mp.lambda_iso, self.grads, self.iso, self.ws)

    def optimizer_step(self):
        groups = [(p, gr, m, v, lr) for p, gr, m, v, lr in
                  zip(self.g.tensors(), self.grads.tensors(), self.m, self.v, self.mp.lr)]
        G.gs_adam_step(groups, self.mp.beta1, self.mp.beta2, self.mp.eps, self.d_step)

    def _bound_calls(self):
        """The iteration's C-ABI calls with their arguments marshalled once;
        rebuilt when the cameras, the buffers or the mapping parameters change."""
        mp = self.mp
        key = (tuple(id(c) for c in self.cams), id(self.bins), id(self.ws), id(self.target_color),
               id(self.target_depth), mp.lambda_c, mp.lambda_d, mp.lambda_iso, tuple(mp.lr), mp.beta1, mp.beta2,
               mp.eps, self.g.n)
        if self._bound is None or self._bound_key != key:
            groups = list(zip(self.g.tensors(), self.grads.tensors(), self.m, self.v, mp.lr))
            self._bound = G.bind_mapping_step(self.g, self.proj, self.bins, self.img, self.cams, self.params,
                                              self.target_color, self.target_depth, mp.lambda_c, mp.lambda_d,
                                              self.dL_dcolor, self.dL_ddepth, self.loss_terms, mp.lambda_iso,
                                              self.grads, self.iso, self.ws, groups, mp.beta1, mp.beta2, mp.eps,
                                              self.d_step, loss_ws=self.loss_ws)
            self._bound_key = key
        return self._bound

    def step(self):
        """One full mapping iteration (no host synchronisation): the captured graph
        if capture() was called, else the C-ABI calls (arguments marshalled once
        and reused)."""
        if self.graph is not None:
            self.graph.replay()
            return
        for call in self._bound_calls():
            call()

    STAGES = ("gs_project", "gs_bin_sort", "gs_render_fwd", "gs_loss", "gs_render_bwd_raster", "gs_project_bwd",
              "gs_adam_step")
    FUSED_STAGES = ("gs_project", "gs_bin_sort", "gs_render_fwd_loss", "gs_render_bwd_raster_loss", "gs_project_bwd",
                    "gs_adam_step")

    def _staged(self, events=None, host_io=None):
        """The iteration as its C-ABI calls (the names in self.stages); if
        `events` (len(self.stages) + 1) is given, events[k] is recorded before
        call k and the last one after the last call.  With `host_io` = (color,
        depth, loss_terms, iso) pinned host tensors, the targets are first copied
        in from the first two and the loss terms and the iso term copied out to
        the last two."""
        rec = (lambda k: events[k].record()) if events is not None else (lambda k: None)
        grad2d = self.ws
        main = torch.cuda.current_stream()
        if host_io is not None:
            # the targets are first read by the loss (fused: the forward pass); their
            # upload runs on a side branch beside projection and binning
            if self._io_stream is None:
                self._io_stream = torch.cuda.Stream()
            side = self._io_stream
            side.wait_stream(main)
            with torch.cuda.stream(side):
                self.target_color.copy_(host_io[0], non_blocking=True)
                self.target_depth.copy_(host_io[1], non_blocking=True)
        k = 0
        rec(k)
        G.gs_project(self.g, self.cams, self.params, self.proj)
        k += 1; rec(k)
        G.gs_bin_sort(self.proj, self.n, self.cams, self.params, self.bins, self.ws)
        if self.fused_loss:
            if host_io is not None:
                main.wait_stream(side)
            k += 1; rec(k)
            G.gs_render_fwd_loss(self.proj, self.bins, self.cams, self.params, self.img, self.target_color,
                                 self.target_depth, self.loss_terms, self.loss_ws)
            k += 1; rec(k)
            G.gs_render_bwd_raster_loss(self.proj, self.bins, self.img, self.target_color, self.target_depth,
                                        self.mp.lambda_c, self.mp.lambda_d, self.loss_ws, self.cams, self.params,
                                        self.n, grad2d)
        else:
            k += 1; rec(k)
            G.gs_render_fwd(self.proj, self.bins, self.cams, self.params, self.img)
            if host_io is not None:
                main.wait_stream(side)
            k += 1; rec(k)
            G.gs_loss(self.img, self.target_color, self.target_depth, self.cams, self.mp.lambda_c,
                      self.mp.lambda_d, self.dL_dcolor, self.dL_ddepth, self.loss_terms, self.ws)
            k += 1; rec(k)
            G.gs_render_bwd_raster(self.proj, self.bins, self.img, self.dL_dcolor, self.dL_ddepth, self.cams,
                                   self.params, self.n, grad2d)
        k += 1; rec(k)
        G.gs_project_bwd(self.g, self.cams, self.params, grad2d, self.mp.lambda_iso, self.grads, self.iso)
        if host_io is not None:
            # the loss terms and the iso term are final: read back beside Adam
            side.wait_stream(main)
            with torch.cuda.stream(side):
                host_io[2].copy_(self.loss_terms, non_blocking=True)
                host_io[3].copy_(self.iso, non_blocking=True)
        k += 1; rec(k)
        self.optimizer_step()
        k += 1; rec(k)
        if host_io is not None:
            main.wait_stream(side)

    def capture(self, warmup: int = 1, events=None, host_io=None):
        """Capture the iteration into a CUDA graph (replayed by step()).  With
        `events` (len(self.stages) + 1 torch.cuda.Event created with
        external=True) the graph also records them around each call, for
        per-stage timing.  With
        `host_io` = (color, depth, loss_terms, iso), pinned host tensors shaped
        like target_color, target_depth, loss_terms and iso, every replay also
        copies that step's targets in and its loss out (memcpy nodes of the same
        graph); the host values are valid after the stream is synchronised."""
        if host_io is not None:
            want = (self.target_color, self.target_depth, self.loss_terms, self.iso)
            for h, d in zip(host_io, want):
                if not h.is_pinned() or h.shape != d.shape or h.dtype != d.dtype:
                    raise ValueError("host_io needs pinned host tensors shaped like the targets, loss terms and iso")
        self.graph = None
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.step()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._staged(events, host_io)
        self.graph = g
        return g

    def loss(self) -> torch.Tensor:
        """Total Eq. 6 loss of the last pass (device tensor)."""
        t = self.loss_terms
        return (self.mp.lambda_c * t[:, 0] + self.mp.lambda_d * t[:, 1]).sum() + self.mp.lambda_iso * self.iso[0]

    # ------------------------------------------------------------- views
    def view_slices(self):
        """(pixel offset, W, H) of every view in the packed image buffers."""
        out, base = [], 0
        for c in self.cams:
            out.append((base, int(c.width), int(c.height)))
            base += int(c.width) * int(c.height)
        return out

    def color_image(self, v: int) -> torch.Tensor:
        base, W, H = self.view_slices()[v]
        return self.img.color[3 * base:3 * (base + W * H)].view(3, H, W)

    def depth_image(self, v: int) -> torch.Tensor:
        base, W, H = self.view_slices()[v]
        return self.img.depth[base:base + W * H].view(H, W)


def autotune_tile(gaussians: G.Gaussians, cams, target_color, target_depth, params: G.RenderParams | None = None,
                  mparams: MapParams | None = None, candidates=(8, 16, 32), iters: int = 10, stages=(2, 3),
                  masks=(1, 0)):
    """Pick the tile size, the forward rasteriser's splat staging (batches of
    32 splats a warp holds at once: 2 or 3) and whether the binning writes the
    pixel-block masks the rasterisers read and drops the tiles a splat cannot
    reach (1) or keeps every tile of the rectangle and the rasterisers test
    every list entry (0), by the fastest graph-replayed mapping iteration for
    this map and these views.  Every trial starts from the same map and the map is restored
    afterwards.  Returns (best RenderParams, {"tile/stages/masks": ms})."""
    import dataclasses
    base = params or G.RenderParams()
    saved = [t.clone() for t in gaussians.tensors()]
    times = {}
    for tile, st, bm in [(t, s, m) for t in candidates for s in stages for m in masks]:
        p = dataclasses.replace(base, tile=tile, splat_stages=st, block_masks=bm, cull_tiles=bm)
        step = MappingStep(gaussians, cams, target_color, target_depth, p, mparams)
        step.step()
        step.ensure_capacity()
        step.capture(warmup=1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ms = []
        for _ in range(iters):
            for t, s0 in zip(gaussians.tensors(), saved):
                t.copy_(s0)
            ev[0].record()
            step.step()
            ev[1].record()
            torch.cuda.synchronize()
            ms.append(ev[0].elapsed_time(ev[1]))
        ms.sort()
        times[f"{tile}/{st}/{bm}"] = ms[len(ms) // 2]
        del step
    for t, s0 in zip(gaussians.tensors(), saved):
        t.copy_(s0)
    best = min(times, key=times.get)
    tile, st, bm = (int(x) for x in best.split("/"))
    return dataclasses.replace(base, tile=tile, splat_stages=st, block_masks=bm, cull_tiles=bm), times
