"""Pose refinement through the re-rendering loss: a keyframe pose perturbed by a
few centimetres and degrees is recovered from the pose-tangent gradient of the
rendering loss alone, with the map fixed."""
import numpy as np
import pytest
import torch

from paper_2512_02293_gb300 import gs as G
from paper_2512_02293_gb300 import synth
from paper_2512_02293_gb300.autograd import se3_left_update
from paper_2512_02293_gb300.mapping import MapParams, MappingStep
from paper_2512_02293_gb300.tracking import PoseTracker, pose_error
from gpu_common import ensure_lib


def test_pose_error_metric():
    cam = synth.identity_camera()
    for ang in (0.02, 1e-5):
        xi = np.array([0.01, 0.0, 0.0, 0.0, 0.0, ang])
        dt, dr = pose_error(se3_left_update(cam, xi), cam)
        assert dr == pytest.approx(ang, rel=1e-4)
    assert pose_error(cam, cam) == (0.0, 0.0)


@pytest.mark.gpu
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_perturbed_pose_is_recovered(seed):
    ensure_lib()
    g, _, cam = synth.cfg2_problem()
    gd = G.Gaussians.from_numpy(g)
    P = cam.n_pixels
    r = MappingStep(gd, [cam], torch.zeros(3 * P, device="cuda"), torch.zeros(P, device="cuda"),
                    G.RenderParams(tile=16), MapParams())
    r.render()
    tc, td = r.img.color.clone(), r.img.depth.clone()
    rng = np.random.default_rng(seed)
    xi0 = np.concatenate([rng.uniform(-1, 1, 3) * 0.03, rng.uniform(-1, 1, 3) * 0.02])   # 3 cm, ~1.1 deg
    start = se3_left_update(cam, xi0)
    dt0, dr0 = pose_error(start, cam)
    tr = PoseTracker(gd, start, tc, td, G.RenderParams(tile=16))
    losses = tr.run()
    dt, dr = pose_error(tr.cam, cam)
    assert losses[-1] < 0.05 * losses[0]
    assert dt < 1e-3 and dr < 5e-4, (dt0, dr0, dt, dr)     # 1 mm, 0.03 deg from 3 cm, ~1.1 deg
