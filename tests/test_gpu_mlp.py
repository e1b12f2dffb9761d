"""The learned initialiser's tensor-core kernels (gs_mlp_pack / gs_mlp_fwd /
gs_mlp_bwd) against the FP64 oracle with BF16 rounding at the same points.

Tolerances: the GPU accumulates in FP32 where the oracle uses FP64, so a BF16
rounding of an activation can land on the other side of a rounding boundary.
That happens for roughly (FP32 accumulation error) / (BF16 spacing) ~ 1e-6 /
4e-3 of the elements and moves each by one BF16 unit (2^-8 relative).  Hence:
Z1 equal except for < 0.5 % of elements, which differ by one unit; Z2 likewise,
plus the absolute change an H1 flip carries through W2; outputs within 1e-4 for
> 99 % of entries (5e-3 worst); gradients within the 1e-3 relative L2 of the
parity bar (1e-4 when the backward is fed the oracle's own activations).
"""
import numpy as np
import pytest
import torch

from oracle import mlp as M
from paper_2512_02293_gb300 import gs as G
from paper_2512_02293_gb300 import synth
from gpu_common import GRAD_RTOL, ensure_lib, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _device_params(p):
    return {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda() for k, v in p.items()}


def _device_x(X):
    """[n, 196] float32 -> bfloat16 [n, 208]; columns 196.. hold garbage the kernels must ignore."""
    n = X.shape[0]
    full = np.full((n, 208), 7.0, np.float32)
    full[:, :196] = X
    return torch.from_numpy(full).to(torch.bfloat16).cuda()


def _bf16_bits(t):
    return t.cpu().view(torch.int16).numpy().astype(np.int64) & 0xFFFF


def _oracle_bits(x):
    return (np.asarray(x, np.float32).view(np.uint32) >> 16).astype(np.int64)


def _run_fwd(p, X, T=None):
    n = X.shape[0]
    packed = G.MlpPacked()
    G.gs_mlp_pack(_device_params(p), packed)
    Xd = _device_x(X)
    Y = torch.empty(n, 8, device="cuda")
    Z1 = torch.empty(n, 128, device="cuda", dtype=torch.bfloat16)
    Z2 = torch.empty_like(Z1)
    st = torch.zeros(4, device="cuda", dtype=torch.int32)
    kw = {}
    if T is not None:
        kw = dict(T=torch.from_numpy(T).cuda(), dY=torch.empty(n, 8, device="cuda"),
                  loss=torch.zeros(1, device="cuda"), loss_scale=1.0 / (8 * n))
    G.gs_mlp_fwd(packed, Xd, Y=Y, Z1=Z1, Z2=Z2, status=st, **kw)
    torch.cuda.synchronize()
    assert int(st[0].item()) == 0
    return packed, Xd, Y, Z1, Z2, kw


@pytest.mark.parametrize("n", [1, 1000, 152 * 128 * 3 + 77])
def test_forward_matches_oracle(n):
    """n = 1000: one tile per CTA; 58445: 457 tiles, so one CTA takes four (two
    pairs of tensor-memory slots) and the others three (the last pair with one
    tile), the last tile ragged."""
    p = synth.mlp_params(21)
    X, _ = synth.mlp_batch(22, n)
    packed, _, Y, Z1, Z2, _ = _run_fwd(p, X)
    ref = M.forward(X, p, bf16=True)
    # Z1: a flip moves a value by at most one BF16 unit of the value plus the
    # error of its FP32 accumulation (197 products and the bias; bounded by
    # 2 (K + 3) 2^-24 sum |terms|, allowing directed rounding in the tensor
    # core), which exceeds a unit only near cancellation
    gb, ob = _bf16_bits(Z1), _oracle_bits(ref["Z1"])
    diff = gb != ob
    assert diff.mean() < 5e-3
    W = ref["W"]
    acc = 2.0 * (196 + 4) * 2.0 ** -24 * (np.abs(ref["X"]) @ np.abs(W["W1"]).T + np.abs(W["b1"]))
    unit = 2.0 ** (np.floor(np.log2(np.maximum(np.abs(ref["Z1"]), 2.0 ** -126))) - 7)
    z1 = Z1.float().cpu().numpy().astype(np.float64)
    assert np.all(np.abs(z1 - ref["Z1"]) <= unit + acc)
    # Z2: one BF16 unit of the value, its FP32 accumulation bound, and what W2
    # carries of the H1 values that differ from the oracle's (H1 on the GPU is
    # the packed activation table at the GPU's own Z1)
    tab = packed.gelu_tab.float().cpu().numpy().astype(np.float64)
    dh1 = np.abs(tab[gb] - ref["H1"])
    z2 = Z2.float().cpu().numpy().astype(np.float64)
    d2 = np.abs(z2 - ref["Z2"])
    assert (d2 > 0).mean() < 5e-3
    acc2 = 2.0 * (128 + 4) * 2.0 ** -24 * (np.abs(ref["H1"]) @ np.abs(W["W2"]).T + np.abs(W["b2"]))
    unit2 = 2.0 ** (np.floor(np.log2(np.maximum(np.abs(ref["Z2"]), 2.0 ** -126))) - 7)
    assert np.all(d2 <= unit2 + acc2 + dh1 @ np.abs(W["W2"]).T)
    err = np.abs(Y.cpu().numpy() - ref["Y"])
    assert (err > 1e-4).mean() < 0.01
    assert err.max() < 5e-3


def test_loss_and_output_gradient():
    n = 777
    p = synth.mlp_params(23)
    X, T = synth.mlp_batch(24, n)
    _, _, Y, _, _, kw = _run_fwd(p, X, T)
    y = Y.cpu().numpy().astype(np.float64)
    L, dY = M.mse(y, T)                                  # oracle loss of the GPU's own outputs
    assert abs(kw["loss"].item() - L) < 1e-5 * max(1.0, L)
    np.testing.assert_allclose(kw["dY"].cpu().numpy(), dY, rtol=1e-5, atol=1e-9)
    Lo, _ = M.mse(M.forward(X, p, bf16=True)["Y"], T)
    assert abs(kw["loss"].item() - Lo) < 1e-3 * Lo


def _grads_dev():
    return {k: torch.empty(G.MLP_PARAM_SHAPES[k], device="cuda") for k in G.MLP_PARAM_NAMES}


@pytest.mark.parametrize("n", [1, 300, 2048])
def test_backward_stagewise_from_oracle_activations(n):
    """The GPU backward fed the oracle's own Z1, Z2 and dY."""
    p = synth.mlp_params(25)
    X, T = synth.mlp_batch(26, n)
    ref = M.forward(X, p, bf16=True)
    _, dY = M.mse(ref["Y"], T)
    gref = M.backward(ref, dY, bf16=True)
    packed = G.MlpPacked()
    G.gs_mlp_pack(_device_params(p), packed)
    to_bf = lambda a: torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).cuda()
    grads = _grads_dev()
    st = torch.zeros(4, device="cuda", dtype=torch.int32)
    G.gs_mlp_bwd(packed, _device_x(X), to_bf(ref["Z1"]), to_bf(ref["Z2"]),
                 torch.from_numpy(dY.astype(np.float32)).cuda(), grads, status=st)
    torch.cuda.synchronize()
    assert int(st[0].item()) == 0
    for k in M.PARAM_NAMES:
        assert rel_l2(grads[k].cpu().numpy(), gref[k]) < 1e-4, k


@pytest.mark.parametrize("n", [1500, 40000])
def test_backward_end_to_end(n):
    p = synth.mlp_params(27)
    X, T = synth.mlp_batch(28, n)
    packed, Xd, _, Z1, Z2, kw = _run_fwd(p, X, T)
    grads = _grads_dev()
    G.gs_mlp_bwd(packed, Xd, Z1, Z2, kw["dY"], grads)
    torch.cuda.synchronize()
    ref = M.forward(X, p, bf16=True)
    gref = M.backward(ref, M.mse(ref["Y"], T)[1], bf16=True)
    for k in M.PARAM_NAMES:
        assert rel_l2(grads[k].cpu().numpy(), gref[k]) < GRAD_RTOL, k


def test_adam_training_reduces_the_loss():
    n = 4096
    p = synth.mlp_params(29)
    X, _ = synth.mlp_batch(30, n)
    T = M.forward(X, synth.mlp_params(31), bf16=False)["Y"].astype(np.float32)    # a reachable target
    params = _device_params(p)
    packed = G.MlpPacked()
    Xd = _device_x(X)
    Td = torch.from_numpy(T).cuda()
    Z1 = torch.empty(n, 128, device="cuda", dtype=torch.bfloat16); Z2 = torch.empty_like(Z1)
    dY = torch.empty(n, 8, device="cuda"); loss = torch.zeros(1, device="cuda")
    grads = _grads_dev()
    m = {k: torch.zeros_like(v) for k, v in params.items()}
    v = {k: torch.zeros_like(t) for k, t in params.items()}
    d_step = torch.zeros(2, device="cuda", dtype=torch.int32)
    losses = []
    for it in range(60):
        G.gs_mlp_pack(params, packed)
        loss.zero_()
        G.gs_mlp_fwd(packed, Xd, Z1=Z1, Z2=Z2, T=Td, dY=dY, loss=loss, loss_scale=1.0 / (8 * n))
        G.gs_mlp_bwd(packed, Xd, Z1, Z2, dY, grads)
        G.gs_adam_step([(params[k], grads[k], m[k], v[k], 3e-3) for k in G.MLP_PARAM_NAMES], 0.9, 0.999, 1e-8, d_step)
        losses.append(loss.item())
    assert losses[-1] < 0.3 * losses[0]


def test_bounded_waits_run_out_report_timeout_and_leave_the_gpu_usable():
    """With the poll limit set to 0 the first mbarrier wait of each kernel gives
    up at once: the kernel waits (bounded) for its MMAs and copies in flight,
    records GS_ERR_TIMEOUT, frees its tensor memory and returns.  The host reads
    the status through gs_read_device_status; afterwards the same context runs
    the kernels normally and matches the oracle."""
    n = 640
    p = synth.mlp_params(33)
    X, T = synth.mlp_batch(34, n)
    packed = G.MlpPacked()
    G.gs_mlp_pack(_device_params(p), packed)
    Xd = _device_x(X)
    Y = torch.empty(n, 8, device="cuda")
    Z1 = torch.zeros(n, 128, device="cuda", dtype=torch.bfloat16); Z2 = torch.zeros_like(Z1)
    dY = torch.zeros(n, 8, device="cuda")
    grads = _grads_dev()
    st_f = torch.zeros(1, device="cuda", dtype=torch.int32)
    st_b = torch.zeros(1, device="cuda", dtype=torch.int32)
    prev = G.gs_mlp_set_wait_polls(0)
    try:
        G.gs_mlp_fwd(packed, Xd, Y=Y, Z1=Z1, Z2=Z2, status=st_f)
        G.gs_mlp_bwd(packed, Xd, Z1, Z2, dY, grads, status=st_b)
    finally:
        G.gs_mlp_set_wait_polls(prev)
    assert G.gs_read_device_status(st_f) == G.GS_ERR_TIMEOUT
    assert G.gs_read_device_status(st_b) == G.GS_ERR_TIMEOUT
    # the default limit again: normal results on the same GPU context
    _, _, Y2, _, _, _ = _run_fwd(p, X)
    ref = M.forward(X, p, bf16=True)
    err = np.abs(Y2.cpu().numpy() - ref["Y"])
    assert (err > 1e-4).mean() < 0.01 and err.max() < 5e-3
