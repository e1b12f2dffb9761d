"""Pins of the FP64 oracle of the learned initialiser network (oracle/mlp.py)
against what mathematics and independent libraries fix."""
import math

import numpy as np
import pytest
import torch

from oracle import mlp as M
from paper_2512_02293_gb300 import synth


def test_bf16_round_ties_to_even_and_exact_values():
    one = 1.0
    cases = {
        one: one,
        one + 2.0 ** -8: one,                                  # tie between 1 and 1 + 2^-7 -> even (1)
        one + 3 * 2.0 ** -8: one + 2.0 ** -6,                  # tie between 1 + 2^-7 (odd) and 1 + 2^-6
        one + 2.0 ** -8 + 2.0 ** -20: one + 2.0 ** -7,         # above the tie
        -(one + 3 * 2.0 ** -8): -(one + 2.0 ** -6),
        3.140625: 3.140625,                                    # exactly representable (1.1001001b x 2)
        1e-3: 0.00099945068359375,                             # nearest bf16 of 1e-3
        0.0: 0.0,
    }
    for x, want in cases.items():
        assert M.bf16_round(np.array([x]))[0] == want, x


def test_gelu_values_from_the_normal_cdf():
    # Phi(1) and Phi(-1), Phi(2) from the error function (math.erf, an independent routine)
    Phi = lambda x: 0.5 * (1.0 + math.erf(x / math.sqrt(2.0)))
    for x in (-3.0, -1.0, -0.25, 0.0, 0.5, 1.0, 2.0):
        assert abs(M.gelu(np.array([x]))[0] - x * Phi(x)) < 1e-15
    assert abs(M.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15
    assert M.gelu_grad(np.array([0.0]))[0] == 0.5
    # gelu'(x) by central differences of gelu
    x = np.linspace(-4, 4, 41)
    h = 1e-6
    fd = (M.gelu(x + h) - M.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(M.gelu_grad(x), fd, atol=1e-9)


def test_permutation_network_closed_form():
    """W1 sends input k to hidden unit pi(k), W2 permutes hidden units by sigma,
    W3 reads unit j into output o: the output is gelu(gelu(x_k) + b) exactly (no
    rounding), which fixes the orientation of every weight matrix."""
    rng = np.random.default_rng(0)
    pi = rng.permutation(M.N_HID)                  # input k (< 128) -> hidden pi[k]
    sigma = rng.permutation(M.N_HID)               # hidden a -> hidden sigma[a]
    W1 = np.zeros((M.N_HID, M.N_IN)); W1[pi, np.arange(M.N_HID)] = 1.0
    W2 = np.zeros((M.N_HID, M.N_HID)); W2[sigma, np.arange(M.N_HID)] = 1.0
    W3 = np.zeros((M.N_OUT, M.N_HID))
    src = [3, 17, 64, 100, 0, 127, 45, 88]         # output o reads the chain of input src[o]
    for o, k in enumerate(src):
        W3[o, sigma[pi[k]]] = 1.0
    b1 = rng.standard_normal(M.N_HID) * 0.1
    b2 = rng.standard_normal(M.N_HID) * 0.1
    b3 = rng.standard_normal(M.N_OUT) * 0.1
    p = dict(W1=W1, b1=b1, W2=W2, b2=b2, W3=W3, b3=b3)
    X = rng.uniform(-1, 1, (5, M.N_IN))
    Y = M.forward(X, p, bf16=False)["Y"]
    g = lambda v: v * 0.5 * (1.0 + math.erf(v / math.sqrt(2.0)))
    for n in range(5):
        for o, k in enumerate(src):
            want = g(g(X[n, k] + b1[pi[k]]) + b2[sigma[pi[k]]]) + b3[o]
            assert abs(Y[n, o] - want) < 1e-13


def _torch_net(p, X):
    t = {k: torch.tensor(np.asarray(v, np.float64), requires_grad=True) for k, v in p.items()}
    x = torch.tensor(np.asarray(X, np.float64))
    gelu = lambda z: torch.nn.functional.gelu(z)          # exact (erf) form
    y = gelu(gelu(x @ t["W1"].T + t["b1"]) @ t["W2"].T + t["b2"]) @ t["W3"].T + t["b3"]
    return t, y


def test_backward_matches_torch_autograd_float64():
    p = synth.mlp_params(1)
    X, T = synth.mlp_batch(2, 37)
    cache = M.forward(X, p, bf16=False)
    L, dY = M.mse(cache["Y"], T)
    g = M.backward(cache, dY, bf16=False)
    t, y = _torch_net(p, X)
    lt = torch.nn.functional.mse_loss(y, torch.tensor(np.asarray(T, np.float64)))
    lt.backward()
    assert abs(L - lt.item()) < 1e-12 * max(1.0, abs(L))
    np.testing.assert_allclose(cache["Y"], y.detach().numpy(), rtol=1e-12, atol=1e-12)
    for k in M.PARAM_NAMES:
        np.testing.assert_allclose(g[k], t[k].grad.numpy(), rtol=1e-10, atol=1e-13, err_msg=k)


def test_backward_matches_central_differences():
    p = {k: v.astype(np.float64) for k, v in synth.mlp_params(3).items()}
    X, T = synth.mlp_batch(4, 9)

    def loss(pp):
        return M.mse(M.forward(X, pp, bf16=False)["Y"], T)[0]

    cache = M.forward(X, p, bf16=False)
    g = M.backward(cache, M.mse(cache["Y"], T)[1], bf16=False)
    rng = np.random.default_rng(5)
    h = 1e-6
    for k in M.PARAM_NAMES:
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in p[k].shape)
            pp = {kk: vv.copy() for kk, vv in p.items()}
            pp[k][idx] += h
            lp = loss(pp)
            pp[k][idx] -= 2 * h
            lm = loss(pp)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k][idx]) < 1e-7 + 1e-6 * abs(fd), (k, idx)
    # one random direction through all parameters at once
    d = {k: rng.standard_normal(v.shape) for k, v in p.items()}
    pp = {k: p[k] + h * d[k] for k in p}; lp = loss(pp)
    pm = {k: p[k] - h * d[k] for k in p}; lm = loss(pm)
    dd = sum(float((g[k] * d[k]).sum()) for k in p)
    assert abs((lp - lm) / (2 * h) - dd) < 1e-6 * max(1.0, abs(dd))


def test_bf16_mode_rounds_exactly_at_the_stated_points():
    p = synth.mlp_params(6)
    X, T = synth.mlp_batch(7, 16)
    c = M.forward(X, p, bf16=True)
    for k in ("X", "Z1", "H1", "Z2", "H2"):
        np.testing.assert_array_equal(M.bf16_round(c[k]), c[k], err_msg=k)
    np.testing.assert_array_equal(c["H1"], M.bf16_round(M.gelu(c["Z1"])))
    np.testing.assert_array_equal(c["H2"], M.bf16_round(M.gelu(c["Z2"])))
    # the rounded network stays within BF16-level error of the exact one
    ce = M.forward(X, p, bf16=False)
    assert np.max(np.abs(c["Y"] - ce["Y"])) < 0.05 * np.max(np.abs(ce["Y"]))
    dY = M.mse(c["Y"], T)[1]
    g = M.backward(c, dY, bf16=True)
    ge = M.backward(ce, dY, bf16=False)
    for k in M.PARAM_NAMES:
        assert np.linalg.norm(g[k] - ge[k]) < 0.05 * np.linalg.norm(ge[k]), k


def test_mse_matches_torch():
    Y = np.random.default_rng(8).standard_normal((11, 8))
    T = np.random.default_rng(9).standard_normal((11, 8))
    L, dY = M.mse(Y, T)
    yt = torch.tensor(Y, requires_grad=True)
    lt = torch.nn.functional.mse_loss(yt, torch.tensor(T))
    lt.backward()
    assert abs(L - lt.item()) < 1e-14
    np.testing.assert_allclose(dY, yt.grad.numpy(), rtol=1e-13)


@pytest.mark.parametrize("mistake", ["W2_transposed", "gelu_grad_dropped_term", "dZ1_skips_W2"])
def test_planted_mistakes_are_caught(mistake, monkeypatch):
    """Each plausible slip in the backward fails the autograd comparison."""
    orig_backward, orig_gg = M.backward, M.gelu_grad

    def bad_backward(cache, dY, bf16=True):
        W = dict(cache["W"])
        if mistake == "W2_transposed":
            W["W2"] = W["W2"].T
        c2 = dict(cache, W=W)
        if mistake == "dZ1_skips_W2":
            W["W2"] = np.eye(W["W2"].shape[0])
        return orig_backward(c2, dY, bf16)

    if mistake == "gelu_grad_dropped_term":
        monkeypatch.setattr(M, "gelu_grad", lambda z: 0.5 * (1.0 + np.vectorize(math.erf)(np.asarray(z) / math.sqrt(2.0))))
        bb = M.backward
    else:
        bb = bad_backward
    p = synth.mlp_params(10)
    X, T = synth.mlp_batch(11, 13)
    cache = M.forward(X, p, bf16=False)
    g = bb(cache, M.mse(cache["Y"], T)[1], bf16=False)
    t, y = _torch_net(p, X)
    torch.nn.functional.mse_loss(y, torch.tensor(np.asarray(T, np.float64))).backward()
    worst = max(np.linalg.norm(g[k] - t[k].grad.numpy()) / np.linalg.norm(t[k].grad.numpy()) for k in M.PARAM_NAMES)
    assert worst > 1e-3
    monkeypatch.setattr(M, "gelu_grad", orig_gg)
