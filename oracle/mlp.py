"""FP64 oracle of the learned Gaussian initialiser: a 196 -> 128 -> 128 -> 8
perceptron with GELU, trained by mean-squared error.

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may use it.

The network and its precision are part of the method as specified: weights,
inputs and the activations handed from layer to layer are BF16, products are
accumulated in (here: better than) FP32.  With ``bf16=True`` the oracle rounds
to BF16 (round to nearest, ties to even) at exactly these points and does all
arithmetic in float64 otherwise:

    X, W, b      given as BF16 values
    Z1 = bf16(W1 X + b1)          H1 = bf16(gelu(Z1))
    Z2 = bf16(W2 H1 + b2)         H2 = bf16(gelu(Z2))
    Y  = W3 H2 + b3               (not rounded)
    backward:  dZ2 = bf16((W3^T dY) * gelu'(Z2)),  dZ1 = bf16((W2^T dZ2) * gelu'(Z1))
               dW3 = dY H2^T, dW2 = dZ2 H1^T, dW1 = dZ1 X^T, db = row sums

GELU is the exact form x * Phi(x) (Phi the standard normal CDF).

Parity status (tests/test_oracle_mlp.py): pinned by GELU values from the normal
CDF, BF16 tie cases, closed-form outputs of permutation networks (which fix the
orientation of every weight matrix), torch float64 autograd of the same network
and central finite differences (bf16=False), and torch's mse_loss.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

N_IN, N_HID, N_OUT = 196, 128, 8
PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")
PARAM_SHAPES = {"W1": (N_HID, N_IN), "b1": (N_HID,), "W2": (N_HID, N_HID), "b2": (N_HID,),
                "W3": (N_OUT, N_HID), "b3": (N_OUT,)}


def bf16_round(x) -> np.ndarray:
    """Nearest BF16 value (ties to even) of each element, returned as float64.
    The value is first rounded to float32 (the type the GPU converts from)."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    z = np.asarray(z, np.float64)
    return z * 0.5 * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    z = np.asarray(z, np.float64)
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def _r(x, on):
    return bf16_round(x) if on else np.asarray(x, np.float64)


def forward(X, p: dict, bf16: bool = True) -> dict:
    """X [n, 196]; p holds W1 [128,196], b1, W2 [128,128], b2, W3 [8,128], b3.
    Returns the cache {X, Z1, H1, Z2, H2, Y} (rows = samples)."""
    W = {k: _r(p[k], bf16) for k in PARAM_NAMES}
    X = _r(X, bf16)
    Z1 = _r(X @ W["W1"].T + W["b1"], bf16)
    H1 = _r(gelu(Z1), bf16)
    Z2 = _r(H1 @ W["W2"].T + W["b2"], bf16)
    H2 = _r(gelu(Z2), bf16)
    Y = H2 @ W["W3"].T + W["b3"]
    return dict(X=X, Z1=Z1, H1=H1, Z2=Z2, H2=H2, Y=Y, W=W)


def backward(cache: dict, dY, bf16: bool = True) -> dict:
    """Gradients of sum(dY * Y) with respect to every parameter, through the
    rounding points listed in the module docstring."""
    W = cache["W"]
    dY = np.asarray(dY, np.float64)
    dH2 = dY @ W["W3"]
    dZ2 = _r(dH2 * gelu_grad(cache["Z2"]), bf16)
    dH1 = dZ2 @ W["W2"]
    dZ1 = _r(dH1 * gelu_grad(cache["Z1"]), bf16)
    return dict(W3=dY.T @ cache["H2"], b3=dY.sum(0), W2=dZ2.T @ cache["H1"], b2=dZ2.sum(0),
                W1=dZ1.T @ cache["X"], b1=dZ1.sum(0))


def mse(Y, T):
    """Mean over samples and the 8 outputs of (Y - T)^2, and its gradient."""
    Y = np.asarray(Y, np.float64); T = np.asarray(T, np.float64)
    d = Y - T
    return float(np.mean(d * d)), 2.0 * d / d.size
