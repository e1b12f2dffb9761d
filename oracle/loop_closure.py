"""FP64 oracle of the loop-closure Gaussian update (Sec. 3.3 "Loop Closure
Gaussian Update", Eq. 7 and Eq. 8).

TEST INFRASTRUCTURE (see oracle/__init__.py).  After pose-graph bundle
adjustment moves keyframe k from (R_k^-, t_k^-) to (R_k^+, t_k^+) and rescales
it by ds_k, every Gaussian anchored to k is carried along: its mean goes into
the old camera frame, is scaled, and comes out of the new one (Eq. 7); its
covariance is rotated and scaled the same way (Eq. 8); opacity and colour are
unchanged.  The oracle states both equations literally, on the covariance
matrix Sigma = R(q) diag(s^2) R(q)^T.

Parity status (tests/test_oracle_loop_closure.py): the identity update, the
eigenvalues scaling by ds^2, the old camera centre mapping to the new one, and
(on the GPU) the re-rendering invariant.
"""
from __future__ import annotations

import numpy as np


def quat_to_rot(q):
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                     np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                     np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def covariance(quat, log_scale):
    """Sigma = R(q) diag(exp(2 log s)) R(q)^T, [n, 3, 3]."""
    R = quat_to_rot(quat)
    s2 = np.exp(2.0 * np.asarray(log_scale, np.float64))
    return np.einsum("nij,nj,nkj->nik", R, s2, R)


def update(mean, quat, log_scale, anchor, R_before, t_before, R_after, t_after, ds):
    """Eq. 7 and Eq. 8 for every Gaussian.  R_* [K, 3, 3], t_* [K, 3], ds [K];
    anchor [n] in [0, K).  Returns (mean+ [n, 3], Sigma+ [n, 3, 3])."""
    a = np.asarray(anchor, np.int64)
    Rm, tm = np.asarray(R_before, np.float64)[a], np.asarray(t_before, np.float64)[a]
    Rp, tp = np.asarray(R_after, np.float64)[a], np.asarray(t_after, np.float64)[a]
    s = np.asarray(ds, np.float64)[a]
    x_loc = np.einsum("nji,nj->ni", Rm, np.asarray(mean, np.float64) - tm)       # (R^-)^T (mu^- - t^-)
    x_new = s[:, None] * x_loc
    mean_p = np.einsum("nij,nj->ni", Rp, x_new) + tp
    S = covariance(quat, log_scale)
    inner = (s * s)[:, None, None] * np.einsum("nji,njk,nkl->nil", Rm, S, Rm)     # ds^2 (R^-)^T Sigma R^-
    cov_p = np.einsum("nij,njk,nlk->nil", Rp, inner, Rp)                          # R^+ (...) (R^+)^T
    return mean_p, cov_p
