"""FP64 oracle of keyframe insertion (Sec. 3.3 "Map Management": back-project a
new keyframe's pixels with their depth into new Gaussians, opacity 0.5) and of
the 7 x 7 RGB-D patch the learned initialiser reads.

TEST INFRASTRUCTURE (see oracle/__init__.py).  Written from the definitions in
include/gs.h (gs_extract_patches, gs_insert_gaussians); the rotation of a
learned insertion is composed as a matrix product and converted to a
quaternion with scipy.

Parity status (tests/test_oracle_keyframe.py): back-projection pinned by the
projection oracle (the new mean projects to the pixel centre at depth d);
patches pinned by closed forms (constant image, planar depth ramp, border
clamping); the composed rotation pinned by its matrix.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial.transform import Rotation

from .mlp import bf16_round

SH0 = 0.28209479177387814        # Y_0^0 = 1 / (2 sqrt(pi))


def _cam(cam):
    return (float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy), int(cam.width), int(cam.height),
            np.asarray(cam.R_wc, np.float64).reshape(3, 3), np.asarray(cam.t_wc, np.float64).reshape(3))


def extract_patches(color, depth, cam, uv, bf16: bool = True) -> np.ndarray:
    """color [3, H, W], depth [H, W], uv [n, 2] (column, row) -> X [n, 208]."""
    fx, fy, cx, cy, W, H, R, t = _cam(cam)
    color = np.asarray(color, np.float64); depth = np.asarray(depth, np.float64)
    uv = np.asarray(uv, np.int64)
    f = 0.5 * (fx + fy)
    X = np.zeros((uv.shape[0], 208))
    for k, (u, v) in enumerate(uv):
        dc = depth[v, u]
        for p in range(49):
            dx, dy = p % 7 - 3, p // 7 - 3
            x = min(max(u + dx, 0), W - 1); y = min(max(v + dy, 0), H - 1)
            X[k, 4 * p:4 * p + 3] = color[:, y, x]
            d = depth[y, x]
            if p == 24:
                X[k, 4 * p + 3] = np.log(dc) if dc > 0 else 0.0
            else:
                X[k, 4 * p + 3] = (d - dc) * f / (7.0 * dc) if (d > 0 and dc > 0) else 0.0
        X[k, 196] = 1.0
    return bf16_round(X) if bf16 else X


def insert(color, depth, cam, uv, stride: float, Y=None, sh_degree: int = 0) -> dict:
    """The Gaussians inserted at the samples (see gs_insert_gaussians)."""
    fx, fy, cx, cy, W, H, R, t = _cam(cam)
    color = np.asarray(color, np.float64); depth = np.asarray(depth, np.float64)
    uv = np.asarray(uv, np.int64)
    n = uv.shape[0]
    ncol = 48 if sh_degree == 3 else 3
    out = dict(mean=np.zeros((n, 3)), quat=np.zeros((n, 4)), log_scale=np.zeros((n, 3)), logit=np.zeros(n),
               color=np.zeros((n, ncol)))
    f = 0.5 * (fx + fy)
    for k, (u, v) in enumerate(uv):
        d = depth[v, u]
        if not d > 0:
            out["mean"][k] = t; out["log_scale"][k] = -10.0; out["quat"][k] = (1, 0, 0, 0); out["logit"][k] = -30.0
            continue
        pc = np.array([(u + 0.5 - cx) / fx * d, (v + 0.5 - cy) / fy * d, d])
        out["mean"][k] = R @ pc + t
        s0 = np.log(d * stride / f)
        rgb = color[:, v, u]
        out["color"][k, :3] = (rgb - 0.5) / SH0 if sh_degree == 3 else rgb
        if Y is None:
            out["log_scale"][k] = s0; out["quat"][k] = (1, 0, 0, 0); out["logit"][k] = 0.0
        else:
            y = np.asarray(Y[k], np.float64)
            out["log_scale"][k] = s0 + y[:3]
            qc = y[3:7]
            nq = np.linalg.norm(qc)
            if nq > 1e-12:
                Rc = Rotation.from_quat([qc[1], qc[2], qc[3], qc[0]]).as_matrix()   # scipy order x, y, z, w
                xyzw = Rotation.from_matrix(R @ Rc).as_quat()
                out["quat"][k] = (xyzw[3], xyzw[0], xyzw[1], xyzw[2])
            else:
                out["quat"][k] = (1, 0, 0, 0)
            out["logit"][k] = y[7]
    return out
