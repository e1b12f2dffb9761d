"""Pose refinement through the re-rendering loss, driven by the FP64 oracle's
pose gradient: the tracker's Adam (tracking.PoseAdam) for three iterations on
the 64x48 case.  Pins: at the true pose the loss and the pose gradient are
exactly zero (the target is the map's own render there, and the L1
subgradient at zero residual is 0); from a perturbed pose, three steps lower
the loss and move the pose toward the truth.  tests/test_gpu_tracking.py runs
the same three steps on the GPU and compares the poses."""
import numpy as np

import oracle
from paper_2512_02293_gb300 import synth
from paper_2512_02293_gb300.autograd import se3_left_update
from paper_2512_02293_gb300.tracking import PoseAdam, pose_error

PRM = dict(tile=16)
LAMBDAS = (0.9, 0.1, 0.0)
XI0 = np.array([0.02, -0.015, 0.01, 0.012, -0.008, 0.01])      # ~2.7 cm, ~0.9 deg


def tracking_problem():
    g, _, cam = synth.cfg1_problem(0)
    img = oracle.render_fwd(oracle.project(g, cam, PRM), cam, PRM)
    return g, cam, (img["color"], img["depth"])


def oracle_track(g, start, target, iters=3):
    """Poses and losses of `iters` tracker steps with the oracle's pose gradient."""
    adam = PoseAdam()
    cam, poses, losses = start, [], []
    for _ in range(iters):
        r = oracle.mapping_loss_and_grads(g, [cam], [target], PRM, LAMBDAS)
        losses.append(r.loss)
        cam = adam.step(cam, r.pose_grads[0])
        poses.append(cam)
    return poses, losses


def test_zero_loss_and_gradient_at_the_true_pose():
    g, cam, target = tracking_problem()
    r = oracle.mapping_loss_and_grads(g, [cam], [target], PRM, LAMBDAS)
    assert r.loss == 0.0
    np.testing.assert_array_equal(r.pose_grads[0], np.zeros(6))


def test_three_oracle_driven_steps_move_toward_the_truth():
    g, cam, target = tracking_problem()
    start = se3_left_update(cam, XI0)
    poses, losses = oracle_track(g, start, target)
    e0 = pose_error(start, cam)
    e3 = pose_error(poses[-1], cam)
    assert e3[0] < e0[0] and e3[1] < e0[1], (e0, e3)
    final = oracle.mapping_loss_and_grads(g, [poses[-1]], [target], PRM, LAMBDAS).loss
    assert final < losses[0]
