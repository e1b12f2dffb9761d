"""The torch.autograd binding: gradients of every Gaussian parameter and of the
6-DoF pose tangent, checked against the FP64 oracle and against central
finite differences of the GPU's own forward."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_02293_gb300 import gs as G
from paper_2512_02293_gb300 import synth
from paper_2512_02293_gb300.autograd import Rasterizer, render, se3_left_update
from gpu_common import GRAD_RTOL, ensure_lib, f32, prm_dict, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _leaf(g):
    return [torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda().requires_grad_(True) for a in g.arrays()]


def test_autograd_matches_oracle_including_pose():
    g, _, cam = synth.cfg1_problem(5)
    R, e = synth.look_at([0.1, -0.2, -0.1], [0.05, 0.0, 2.0])
    cams = [synth.Camera(60.0, 60.0, 32.0, 24.0, 64, 48, R, e), synth.Camera(50.0, 50.0, 24.0, 20.0, 48, 40)]
    params = G.RenderParams()
    rast = Rasterizer(cams, g.n, params)
    leaves = _leaf(g)
    xi = torch.zeros(2, 6, device="cuda", requires_grad=True)
    col, dep = render(*leaves, xi, rast)
    rng = np.random.default_rng(0)
    w = torch.from_numpy(rng.standard_normal(col.numel()).astype(np.float32)).cuda()
    u = torch.from_numpy(rng.standard_normal(dep.numel()).astype(np.float32)).cuda()
    loss = (w * col).sum() + (u * dep).sum()
    loss.backward()
    prm = prm_dict(params)
    ref = {k: 0.0 for k in oracle.PARAM_NAMES}
    base = 0
    for v, c in enumerate(cams):
        P = c.n_pixels
        wc = f32(w[3 * base:3 * (base + P)].cpu().numpy().reshape(3, c.height, c.width))
        ud = f32(u[base:base + P].cpu().numpy().reshape(c.height, c.width))
        pr = oracle.project(g, c, prm)
        gp = oracle.project_bwd(g, c, prm, oracle.render_bwd(pr, c, prm, wc, ud))
        for k in oracle.PARAM_NAMES:
            ref[k] = ref[k] + gp[k]
        assert rel_l2(xi.grad[v].cpu().numpy(), gp["pose"]) < GRAD_RTOL
        base += P
    for k, leaf in zip(oracle.PARAM_NAMES, leaves):
        assert rel_l2(leaf.grad.cpu().numpy(), ref[k]) < GRAD_RTOL, k


def test_autograd_pose_and_params_match_gpu_finite_differences():
    # Threshold-free settings (alpha_min = 0, T_cut = 0, wide splat support) make
    # the render smooth, so central differences of the GPU forward apply.
    g, _, cam = synth.cfg1_problem(6)
    params = G.RenderParams(alpha_min=0.0, T_cut=0.0, radius_sigma=8.0)
    rast = Rasterizer([cam], g.n, params)
    leaves = _leaf(g)
    xi = torch.zeros(1, 6, device="cuda", requires_grad=True)
    rng = np.random.default_rng(1)
    w = torch.from_numpy(rng.standard_normal(3 * cam.n_pixels).astype(np.float32)).cuda()
    u = torch.from_numpy(rng.standard_normal(cam.n_pixels).astype(np.float32)).cuda()

    def L(leaves_, xi_):
        with torch.no_grad():
            c, d = render(*leaves_, xi_, rast)
            return float((w.double() * c.double()).sum() + (u.double() * d.double()).sum())

    col, dep = render(*leaves, xi, rast)
    ((w * col).sum() + (u * dep).sum()).backward()
    h = 1e-3
    for k in range(6):
        e = torch.zeros(1, 6, device="cuda"); e[0, k] = h
        fd = (L(leaves, e) - L(leaves, -e)) / (2 * h)
        assert xi.grad[0, k].item() == pytest.approx(fd, rel=2e-2, abs=1e-2), k
    base = [t.detach().clone() for t in leaves]
    vis = np.nonzero(oracle.project(g, cam, prm_dict(params))["tiles"] > 0)[0][:6]
    for pi, name in enumerate(oracle.PARAM_NAMES):
        for i in vis[:3]:
            for comp in range(min(2, base[pi].shape[1] if base[pi].dim() > 1 else 1)):
                idx = (int(i), comp) if base[pi].dim() > 1 else (int(i),)
                hp = 1e-3
                plus = [t.clone() for t in base]; minus = [t.clone() for t in base]
                plus[pi][idx] += hp; minus[pi][idx] -= hp
                fd = (L(plus, torch.zeros(1, 6, device="cuda")) - L(minus, torch.zeros(1, 6, device="cuda"))) / (2 * hp)
                got = leaves[pi].grad[idx].item()
                assert got == pytest.approx(fd, rel=3e-2, abs=2e-2), (name, idx, got, fd)


def test_se3_left_update_first_order():
    cam = synth.identity_camera()
    xi = np.array([0.01, -0.02, 0.03, 0.001, 0.002, -0.003])
    c2 = se3_left_update(cam, xi)
    # world-to-camera of the updated camera maps a point p to ~ p + rho + phi x p
    p = np.array([0.3, -0.2, 2.0])
    pc = c2.R_wc.T.astype(np.float64) @ (p - c2.t_wc.astype(np.float64))
    want = p + xi[:3] + np.cross(xi[3:], p)
    np.testing.assert_allclose(pc, want, atol=1e-5)


def test_autograd_iteration_captures_in_a_graph():
    """Forward, loss and backward through the binding, captured once in a CUDA
    graph (nothing in them synchronises with the host) and replayed: the
    replays reproduce the eager iteration's gradients, including a non-zero
    pose tangent applied on the device."""
    g, gt, cam = synth.cfg1_problem(7)
    params = G.RenderParams()
    rast = Rasterizer([cam], g.n, params)
    leaves = _leaf(g)
    xi = torch.tensor([[0.004, -0.003, 0.002, 0.003, 0.002, -0.001]], device="cuda", requires_grad=True)
    with torch.no_grad():
        tcol, tdep = render(*_leaf(gt), torch.zeros(1, 6, device="cuda"), rast)
        tcol, tdep = tcol.clone(), tdep.clone()

    def one():
        for t in leaves + [xi]:
            t.grad = None
        col, dep = render(*leaves, xi, rast)
        loss = (col - tcol).abs().mean() + (dep - tdep).abs().mean()
        loss.backward()

    one()
    torch.cuda.synchronize()
    assert rast.check() == 0
    ref = [t.grad.clone() for t in leaves + [xi]]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        one()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        col, dep = render(*leaves, xi, rast)
        loss = (col - tcol).abs().mean() + (dep - tdep).abs().mean()
        grads = torch.autograd.grad(loss, leaves + [xi])
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        assert rast.check() == 0
        for got, want in zip(grads, ref):
            assert rel_l2(got.cpu().numpy(), want.cpu().numpy()) < 1e-5
