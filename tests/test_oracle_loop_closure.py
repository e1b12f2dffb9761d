"""Pins of the loop-closure Gaussian update oracle (Eq. 7, Eq. 8)."""
import numpy as np
from scipy.spatial.transform import Rotation

from oracle import loop_closure as LC


def _setup(seed, n=40, K=3):
    rng = np.random.default_rng(seed)
    mean = rng.uniform(-3, 3, (n, 3))
    quat = rng.standard_normal((n, 4))
    ls = rng.normal(-3, 0.5, (n, 3))
    anchor = rng.integers(0, K, n)
    Rb = Rotation.random(K, random_state=seed).as_matrix()
    Ra = Rotation.random(K, random_state=seed + 1).as_matrix()
    tb = rng.standard_normal((K, 3)); ta = rng.standard_normal((K, 3))
    ds = rng.uniform(0.7, 1.4, K)
    return mean, quat, ls, anchor, Rb, tb, Ra, ta, ds


def test_identity_update_changes_nothing():
    mean, quat, ls, anchor, Rb, tb, _, _, _ = _setup(0)
    m2, c2 = LC.update(mean, quat, ls, anchor, Rb, tb, Rb, tb, np.ones(3))
    np.testing.assert_allclose(m2, mean, atol=1e-12)
    np.testing.assert_allclose(c2, LC.covariance(quat, ls), rtol=1e-12, atol=1e-18)


def test_covariance_eigenvalues_scale_by_ds_squared():
    mean, quat, ls, anchor, Rb, tb, Ra, ta, ds = _setup(1)
    _, c2 = LC.update(mean, quat, ls, anchor, Rb, tb, Ra, ta, ds)
    ev_old = np.sort(np.exp(2 * ls), 1)
    ev_new = np.linalg.eigvalsh(c2)
    np.testing.assert_allclose(ev_new, ev_old * (ds[anchor] ** 2)[:, None], rtol=1e-10)


def test_camera_centre_and_rigid_frame_are_carried():
    mean, quat, ls, anchor, Rb, tb, Ra, ta, ds = _setup(2)
    # a Gaussian at keyframe k's old centre lands at its new centre
    m = tb[anchor]
    m2, _ = LC.update(m, quat, ls, anchor, Rb, tb, Ra, ta, ds)
    np.testing.assert_allclose(m2, ta[anchor], atol=1e-12)
    # camera-frame coordinates scale by ds: |mu+ - t+| = ds |mu- - t-|
    m3, _ = LC.update(mean, quat, ls, anchor, Rb, tb, Ra, ta, ds)
    np.testing.assert_allclose(np.linalg.norm(m3 - ta[anchor], axis=1),
                               ds[anchor] * np.linalg.norm(mean - tb[anchor], axis=1), rtol=1e-12)
    # the displacement seen in the keyframe's own frame is scaled, not rotated
    loc_old = np.einsum("nji,nj->ni", Rb[anchor], mean - tb[anchor])
    loc_new = np.einsum("nji,nj->ni", Ra[anchor], m3 - ta[anchor])
    np.testing.assert_allclose(loc_new, ds[anchor][:, None] * loc_old, atol=1e-12)
