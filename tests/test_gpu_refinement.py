"""Final colour refinement (Sec. 3.3 "Final Color Refinement"): random keyframe
draws over the whole keyframe list, one mapping step each, one captured graph
per keyframe."""
import numpy as np
import pytest
import torch

from paper_2512_02293_gb300 import gs as G
from paper_2512_02293_gb300 import synth
from paper_2512_02293_gb300.mapping import MapParams, MappingStep
from paper_2512_02293_gb300.refinement import ColourRefiner
from gpu_common import ensure_lib

pytestmark = pytest.mark.gpu


def _targets(gt, cams):
    """Colour and depth renders of the target map, one per keyframe."""
    tc, td = [], []
    P = cams[0].n_pixels
    for c in cams:
        r = MappingStep(G.Gaussians.from_numpy(gt), [c], torch.zeros(3 * P, device="cuda"),
                        torch.zeros(P, device="cuda"), G.RenderParams(tile=16))
        r.render()
        tc.append(r.img.color.clone()); td.append(r.img.depth.clone())
    return tc, td


@pytest.fixture(scope="module")
def problem():
    ensure_lib()
    g, gt, cams = synth.refinement_problem(0, n=60_000, views=6)
    tc, td = _targets(gt, cams)
    return g, cams, tc, td


def test_one_draw_equals_a_mapping_step_on_that_keyframe(problem):
    g, cams, tc, td = problem
    k = 3
    a = G.Gaussians.from_numpy(g)
    ref = ColourRefiner(a, cams, tc, td, G.RenderParams(tile=16), seed=0)
    ref.graphs[k].replay()
    b = G.Gaussians.from_numpy(g)
    step = MappingStep(b, [cams[k]], tc[k], td[k], G.RenderParams(tile=16), MapParams())
    step.step()
    torch.cuda.synchronize()
    assert ref.step.check() == 0 and step.check() == 0
    lr_max = max(MapParams().lr)
    for x, y in zip(a.tensors(), b.tensors()):
        # the same step; only the order of the gradient atomics differs.  Adam's
        # first step moves a parameter by lr sign(g), so a gradient within rounding
        # of 0 may move it the other way: allowed for 1 in 1000 elements
        x, y = x.cpu().numpy().ravel(), y.cpu().numpy().ravel()
        close = np.isclose(x, y, rtol=1e-4, atol=1e-6)
        assert close.mean() > 0.999
        assert np.abs(x - y).max() <= 2 * lr_max + 1e-6


def test_refinement_raises_the_psnr_of_every_keyframe(problem):
    g, cams, tc, td = problem
    gd = G.Gaussians.from_numpy(g)
    ref = ColourRefiner(gd, cams, tc, td, G.RenderParams(tile=16), seed=1)
    before = [ref.render_psnr(k) for k in range(len(cams))]
    drawn = ref.run(300)
    torch.cuda.synchronize()
    after = [ref.render_psnr(k) for k in range(len(cams))]
    assert ref.step.check() == 0
    assert set(drawn.tolist()) == set(range(len(cams)))          # every keyframe drawn
    assert min(a - b for a, b in zip(after, before)) > 2.0, (before, after)


def test_keyframes_of_different_resolution_are_refused(problem):
    g, cams, tc, td = problem
    small = synth.Camera(cams[1].fx / 2, cams[1].fy / 2, cams[1].cx / 2, cams[1].cy / 2, 320, 240,
                         cams[1].R_wc, cams[1].t_wc)
    with pytest.raises(ValueError):
        ColourRefiner(G.Gaussians.from_numpy(g), [cams[0], small], tc[:2], td[:2])
