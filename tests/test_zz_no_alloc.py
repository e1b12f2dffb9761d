"""gs_loss_noalloc: the loss entry point for callers that cannot allocate a
device workspace (for example a tracker held to a fixed device-memory budget,
or a plugin whose host application owns the device allocator).  Its scratch
is a static device array inside the library, so the caller passes only
inputs and outputs.

Checked through the C ABI against gs_loss (the workspace version) on two calls
in a row with different inputs, so a result left in the shared scratch by the
first call would show up in the second.  This file is collected last on
purpose; it also passes when run on its own in a fresh process."""
import numpy as np
import pytest
import torch

from paper_2512_02293_gb300 import build as B
from paper_2512_02293_gb300 import gs as G
from paper_2512_02293_gb300 import synth

pytestmark = pytest.mark.gpu


def _inputs(seed, cams):
    rng = np.random.default_rng(seed)
    P = sum(c.n_pixels for c in cams)
    col = torch.from_numpy(rng.random(3 * P).astype(np.float32)).cuda()
    dep = torch.from_numpy((rng.random(P) * 4).astype(np.float32)).cuda()
    tcol = torch.from_numpy(rng.random(3 * P).astype(np.float32)).cuda()
    tdep_np = (rng.random(P) * 4).astype(np.float32)
    tdep_np[rng.random(P) < 0.25] = 0.0                   # pixels without target depth
    tdep = torch.from_numpy(tdep_np).cuda()
    img = G.Image(col, dep, torch.ones(P, device="cuda"), torch.zeros(P, device="cuda", dtype=torch.int32))
    return img, tcol, tdep


def test_noalloc_loss_matches_workspace_loss_twice():
    B.build()
    G.load_library()
    cams = [synth.identity_camera(64, 48), synth.identity_camera(70, 45), synth.identity_camera(33, 26)]
    P = sum(c.n_pixels for c in cams)
    for call, (seed, lc, ld) in enumerate([(11, 0.9, 0.1), (12, 1.0, 1.0)]):
        img, tcol, tdep = _inputs(seed, cams)
        ws = torch.empty(1024, device="cuda")
        ref_dc = torch.empty(3 * P, device="cuda"); ref_dd = torch.empty(P, device="cuda")
        ref_terms = torch.empty(len(cams), 2, device="cuda")
        G.gs_loss(img, tcol, tdep, cams, lc, ld, ref_dc, ref_dd, ref_terms, ws)
        dc = torch.full((3 * P,), 7.0, device="cuda"); dd = torch.full((P,), 7.0, device="cuda")
        terms = torch.full((len(cams), 2), 7.0, device="cuda")
        G.gs_loss_noalloc(img, tcol, tdep, cams, lc, ld, dc, dd, terms)
        torch.cuda.synchronize()
        np.testing.assert_allclose(terms.cpu().numpy(), ref_terms.cpu().numpy(), rtol=1e-5, err_msg=f"call {call}")
        np.testing.assert_allclose(dc.cpu().numpy(), ref_dc.cpu().numpy(), rtol=1e-5, atol=1e-12)
        np.testing.assert_allclose(dd.cpu().numpy(), ref_dd.cpu().numpy(), rtol=1e-5, atol=1e-12)


def test_noalloc_loss_rejects_too_many_views():
    B.build()
    G.load_library()
    n = G.GS_NOALLOC_LOSS_MAX_VIEWS + 1          # one view more than the scratch array holds
    cams = [synth.identity_camera(8, 8)] * n
    P = 64 * n
    buf = torch.zeros(3 * P, device="cuda")
    img = G.Image(buf, buf[:P], buf[:P], torch.zeros(P, device="cuda", dtype=torch.int32))
    with pytest.raises(G.GsError) as err:
        G.gs_loss_noalloc(img, buf, buf[:P], cams, 1.0, 1.0, buf.clone(), buf[:P].clone(),
                          torch.zeros(n, 2, device="cuda"))
    assert err.value.status == G.GS_ERR_INVALID_ARG
