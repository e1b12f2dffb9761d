"""What the learned initialiser gains over the heuristic insertion: trained on
mapper-produced pairs from seeded rooms, evaluated on held-out rooms by the
mapper's PSNR on the keyframe and its depth error."""
import numpy as np
import pytest
import torch

from paper_2512_02293_gb300 import learned_init as L
from gpu_common import ensure_lib


def test_canonical_targets_are_unique_per_gaussian():
    # permuted axes, axis pairs negated and negated quaternions describe one Gaussian
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(0)
    n = 64
    ls = rng.normal(-3, 0.5, (n, 3))
    q = rng.standard_normal((n, 4))
    R = Rotation.random(random_state=3).as_matrix()
    T = L.canonical_targets(ls, q, np.zeros(n), R, np.zeros(n))
    for trial in range(4):
        perm = rng.permutation(3)
        Rq = L._quat_to_rot(q)[:, :, perm]
        flips = np.array([[1, 1, 1], [-1, -1, 1], [-1, 1, -1], [1, -1, -1]])[rng.integers(0, 4, n)]
        Rq = Rq * flips[:, None, :]
        Rq[np.linalg.det(Rq) < 0, :, 0] *= -1.0          # odd permutations: restore a rotation
        xyzw = Rotation.from_matrix(Rq).as_quat()
        q2 = -np.stack([xyzw[:, 3], xyzw[:, 0], xyzw[:, 1], xyzw[:, 2]], 1)
        T2 = L.canonical_targets(ls[:, perm], q2, np.zeros(n), R, np.zeros(n))
        np.testing.assert_allclose(T, T2, atol=1e-5)
    assert np.all(np.diff(T[:, :3], axis=1) >= 0) and np.all(T[:, 3] >= 0)
    # the target rotation reproduces the covariance in the camera frame
    Rc = R.T[None] @ L._quat_to_rot(q)
    S = np.exp(2 * ls)
    cov = np.einsum("nij,nj,nkj->nik", Rc, S, Rc)
    Rt = L._quat_to_rot(T[:, 3:7].astype(np.float64))
    St = np.exp(2 * T[:, :3].astype(np.float64))
    np.testing.assert_allclose(np.einsum("nij,nj,nkj->nik", Rt, St, Rt), cov, rtol=1e-4, atol=1e-9)


@pytest.mark.gpu
def test_learned_init_beats_heuristic_on_held_out_rooms():
    ensure_lib()
    cfg = L.InitConfig()
    Xs, Ts = [], []
    for r in range(12):
        X, T = L.training_pairs(100 + r, cfg)
        Xs.append(X); Ts.append(T)
    X = torch.cat(Xs); T = torch.cat(Ts)
    perm = torch.from_numpy(np.random.default_rng(0).permutation(X.shape[0])).cuda()
    X = X.index_select(0, perm).contiguous(); T = T.index_select(0, perm).contiguous()
    net = L.LearnedInit(0)
    losses = net.train(X, T, epochs=30, batch=8192, lr=1e-3)
    Tn = T.cpu().numpy()
    assert losses[-1] < 0.7 * float(((Tn - Tn.mean(0)) ** 2).mean())      # better than the mean target
    for seed in (900, 901):
        kf = L.Keyframe(seed, cfg)
        heur, dh = L.mapping_curve(kf, None, 100)
        lrn, dl = L.mapping_curve(kf, net.predict(kf.X), 100)
        assert lrn[0] > heur[0] + 2.0                                     # dB after one iteration
        assert lrn[-1] > heur[-1]
        it = L.iterations_to_reach(lrn, heur[-1])
        assert it is not None and it <= 90
        assert dl < dh
