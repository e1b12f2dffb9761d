"""Seeded synthetic inputs for the Gaussian-splatting mapping step.

This module only draws inputs: Gaussian maps, pinhole cameras, trajectories and
procedural textures.  It holds none of the rendering arithmetic (no projection,
no compositing, no gradients), so both the CUDA path and the FP64 oracle can
consume its output without sharing any of the method's code.

The paper's datasets (EuRoC, RPNG AR Table, UTMM, FAST-LIVO2; Sec. 4
"Datasets", Tab. 8) are not available; indoor-like synthetic rooms at the
paper's resolutions (640x480, 752x480, 1280x1024) stand in for them.  The map
parameterisation follows Sec. 3.3 "Preliminary": per Gaussian a mean, a
rotation (unit quaternion, (w, x, y, z)), per-axis log-scales, an opacity
logit (o = sigmoid) and a direct RGB colour.

Every array is float32, C-contiguous.  Cameras are camera-to-world
(R_wc, t_wc) with OpenCV axes (x right, y down, z forward); pixel (u, v) is
sampled at (u + 0.5, v + 0.5).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Camera", "GaussianMap", "random_cloud", "room_scene", "perturb_map",
    "look_at", "identity_camera", "trajectory_cameras", "sh3_from_rgb",
    "cfg1_problem", "cfg2_problem", "cfg3_problem", "cfg4_problem",
]


@dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    R_wc: np.ndarray = field(default_factory=lambda: np.eye(3, dtype=np.float32))
    t_wc: np.ndarray = field(default_factory=lambda: np.zeros(3, dtype=np.float32))

    def __post_init__(self):
        self.R_wc = np.ascontiguousarray(self.R_wc, dtype=np.float32).reshape(3, 3)
        self.t_wc = np.ascontiguousarray(self.t_wc, dtype=np.float32).reshape(3)

    @property
    def n_pixels(self) -> int:
        return int(self.width) * int(self.height)


@dataclass
class GaussianMap:
    mean: np.ndarray           # [n, 3]
    quat: np.ndarray           # [n, 4]  (w, x, y, z), not necessarily unit
    log_scale: np.ndarray      # [n, 3]
    opacity_logit: np.ndarray  # [n]
    color: np.ndarray          # [n, 3] RGB, or [n, 16, 3] degree-3 SH coefficients

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def arrays(self):
        return (self.mean, self.quat, self.log_scale, self.opacity_logit, self.color)

    def subset(self, idx) -> "GaussianMap":
        return GaussianMap(*(np.ascontiguousarray(a[idx]) for a in self.arrays()))

    def astype(self, dtype) -> "GaussianMap":
        return GaussianMap(*(np.ascontiguousarray(a, dtype=dtype) for a in self.arrays()))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _logit(p):
    return np.log(p) - np.log1p(-p)


def identity_camera(width=64, height=48, fx=60.0, fy=60.0, cx=None, cy=None) -> Camera:
    cx = width / 2.0 if cx is None else cx
    cy = height / 2.0 if cy is None else cy
    return Camera(fx, fy, cx, cy, width, height)


def look_at(eye, target, up=(0.0, 0.0, 1.0)):
    """Camera-to-world rotation whose +z axis points from eye to target, y down."""
    eye = np.asarray(eye, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    up = np.asarray(up, dtype=np.float64)
    right = np.cross(fwd, up)
    if np.linalg.norm(right) < 1e-9:
        right = np.cross(fwd, np.array([1.0, 0.0, 0.0]))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], axis=1)  # columns: camera x, y, z in world
    return R.astype(np.float32), eye.astype(np.float32)


def random_cloud(n: int, seed: int, box=((-1.0, 1.0), (-1.0, 1.0), (1.0, 3.0)),
                 log_scale_mu=-3.0, log_scale_sd=0.3, sh_degree=0) -> GaussianMap:
    """Gaussians with means uniform in `box`, log-scales N(mu, sd), random unit
    quaternions, logit ~ N(0, 1) and RGB ~ U[0, 1] (the 64x48 / 256-Gaussian case)."""
    rng = np.random.default_rng(seed)
    lo = np.array([b[0] for b in box]); hi = np.array([b[1] for b in box])
    mean = lo + (hi - lo) * rng.random((n, 3))
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    log_scale = log_scale_mu + log_scale_sd * rng.standard_normal((n, 3))
    logit = rng.standard_normal(n)
    rgb = rng.random((n, 3))
    color = rgb if sh_degree == 0 else sh3_from_rgb(rgb, rng)
    return GaussianMap(_f32(mean), _f32(q), _f32(log_scale), _f32(logit), _f32(color))


def sh3_from_rgb(rgb, rng, sigma=0.05):
    """Degree-3 SH coefficients [n, 16, 3]: DC chosen so that the l=0 band alone
    reproduces `rgb` under the convention colour = SH(dir) + 0.5, higher orders
    N(0, sigma)."""
    n = rgb.shape[0]
    c0 = 0.28209479177387814  # Y_0^0 = 1 / (2 sqrt(pi))
    sh = sigma * rng.standard_normal((n, 16, 3))
    sh[:, 0, :] = (rgb - 0.5) / c0
    return sh


def _quat_from_matrices(R):
    """(w, x, y, z) of a stack of proper rotation matrices [n, 3, 3] (Shepperd's method)."""
    R = np.asarray(R, dtype=np.float64)
    n = R.shape[0]
    q = np.zeros((n, 4))
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    d = np.stack([tr, R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]], axis=1)
    k = np.argmax(d, axis=1)
    for case in range(4):
        sel = k == case
        if not np.any(sel):
            continue
        M = R[sel]
        if case == 0:
            s = np.sqrt(tr[sel] + 1.0) * 2
            q[sel] = np.stack([0.25 * s, (M[:, 2, 1] - M[:, 1, 2]) / s, (M[:, 0, 2] - M[:, 2, 0]) / s, (M[:, 1, 0] - M[:, 0, 1]) / s], 1)
        elif case == 1:
            s = np.sqrt(1.0 + M[:, 0, 0] - M[:, 1, 1] - M[:, 2, 2]) * 2
            q[sel] = np.stack([(M[:, 2, 1] - M[:, 1, 2]) / s, 0.25 * s, (M[:, 0, 1] + M[:, 1, 0]) / s, (M[:, 0, 2] + M[:, 2, 0]) / s], 1)
        elif case == 2:
            s = np.sqrt(1.0 + M[:, 1, 1] - M[:, 0, 0] - M[:, 2, 2]) * 2
            q[sel] = np.stack([(M[:, 0, 2] - M[:, 2, 0]) / s, (M[:, 0, 1] + M[:, 1, 0]) / s, 0.25 * s, (M[:, 1, 2] + M[:, 2, 1]) / s], 1)
        else:
            s = np.sqrt(1.0 + M[:, 2, 2] - M[:, 0, 0] - M[:, 1, 1]) * 2
            q[sel] = np.stack([(M[:, 1, 0] - M[:, 0, 1]) / s, (M[:, 0, 2] + M[:, 2, 0]) / s, (M[:, 1, 2] + M[:, 2, 1]) / s, 0.25 * s], 1)
    return q / np.linalg.norm(q, axis=1, keepdims=True)


# Axis-aligned surface patches of the room: (normal axis, sign, fixed coordinate,
# extents of the two tangent axes).
def _room_planes(size):
    sx, sy, sz = size
    planes = []
    # interior faces of the room box [-sx/2, sx/2] x [-sy/2, sy/2] x [0, sz]; normals point inward
    planes.append((0, +1, -sx / 2, (-sy / 2, sy / 2), (0.0, sz)))
    planes.append((0, -1, +sx / 2, (-sy / 2, sy / 2), (0.0, sz)))
    planes.append((1, +1, -sy / 2, (-sx / 2, sx / 2), (0.0, sz)))
    planes.append((1, -1, +sy / 2, (-sx / 2, sx / 2), (0.0, sz)))
    planes.append((2, +1, 0.0, (-sx / 2, sx / 2), (-sy / 2, sy / 2)))
    planes.append((2, -1, sz, (-sx / 2, sx / 2), (-sy / 2, sy / 2)))
    return planes


def _box_planes(center, half):
    cx, cy, cz = center; hx, hy, hz = half
    out = []
    for ax in range(3):
        t = [a for a in range(3) if a != ax]
        c = (cx, cy, cz); h = (hx, hy, hz)
        for sgn in (-1, +1):
            fixed = c[ax] + sgn * h[ax]
            e0 = (c[t[0]] - h[t[0]], c[t[0]] + h[t[0]])
            e1 = (c[t[1]] - h[t[1]], c[t[1]] + h[t[1]])
            out.append((ax, sgn, fixed, e0, e1))
    return out


def _texture(plane_id, u, v):
    """Procedural RGB texture: a checker times a per-plane sinusoid, in [0.05, 0.95]."""
    rng = np.random.default_rng(1234 + plane_id)
    base = 0.25 + 0.5 * rng.random(3)
    f = 2.0 + 4.0 * rng.random(2)
    checker = ((np.floor(u * 2.5) + np.floor(v * 2.5)) % 2)[:, None]
    wave = 0.5 + 0.5 * np.sin(2 * math.pi * (f[0] * u + f[1] * v))[:, None]
    col = base[None, :] * (0.55 + 0.45 * checker) * (0.6 + 0.4 * wave)
    return np.clip(col, 0.05, 0.95)


def room_scene(n: int, seed: int, size=(6.0, 5.0, 3.0), n_boxes=20, keep_out=None,
               tangential_log_scale=math.log(0.02), log_scale_sd=0.3, normal_ratio=0.1,
               surface_noise=0.01, sh_degree=0) -> GaussianMap:
    """An indoor-like room: the six inner faces of a size[0] x size[1] x size[2] m
    box plus `n_boxes` axis-aligned boxes (0.2-1 m) on the floor.  Means are drawn
    area-proportionally on all faces with N(0, surface_noise) offsets along the
    normal; scales are flat along the normal (normal = normal_ratio x tangential),
    opacity ~ U(0.1, 1), colour from a procedural texture."""
    rng = np.random.default_rng(seed)
    sx, sy, sz = size
    planes = _room_planes(size)
    keep_out = [] if keep_out is None else [np.asarray(k, dtype=np.float64) for k in keep_out]
    boxes = 0
    tries = 0
    while boxes < n_boxes and tries < 10000:
        tries += 1
        half = 0.5 * (0.2 + 0.8 * rng.random(3))
        c = np.array([(rng.random() - 0.5) * (sx - 2 * half[0]), (rng.random() - 0.5) * (sy - 2 * half[1]), half[2]])
        if any(np.all(np.abs(k[:2] - c[:2]) < half[:2] + 0.6) for k in keep_out):
            continue
        planes += _box_planes(c, half)
        boxes += 1
    areas = np.array([(p[3][1] - p[3][0]) * (p[4][1] - p[4][0]) for p in planes])
    pid = rng.choice(len(planes), size=n, p=areas / areas.sum())
    u01 = rng.random((n, 2))
    mean = np.zeros((n, 3))
    normal = np.zeros((n, 3))
    tex_u = np.zeros(n); tex_v = np.zeros(n)
    for k, (ax, sgn, fixed, e0, e1) in enumerate(planes):
        sel = pid == k
        if not np.any(sel):
            continue
        t = [a for a in range(3) if a != ax]
        a = e0[0] + (e0[1] - e0[0]) * u01[sel, 0]
        b = e1[0] + (e1[1] - e1[0]) * u01[sel, 1]
        mean[sel, ax] = fixed
        mean[sel, t[0]] = a
        mean[sel, t[1]] = b
        normal[sel, ax] = sgn
        tex_u[sel] = a; tex_v[sel] = b
    mean += normal * (surface_noise * rng.standard_normal(n))[:, None]
    color = np.zeros((n, 3))
    for k in range(len(planes)):
        sel = pid == k
        if np.any(sel):
            color[sel] = _texture(k, tex_u[sel], tex_v[sel])
    # Rotation: local z (scale axis 2) onto the normal, random spin about it.
    spin = 2 * math.pi * rng.random(n)
    ref = np.where((np.abs(normal[:, 0]) < 0.9)[:, None], np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0]))
    ex = np.cross(ref, normal); ex /= np.linalg.norm(ex, axis=1, keepdims=True)
    ey = np.cross(normal, ex)
    c, s = np.cos(spin)[:, None], np.sin(spin)[:, None]
    R = np.stack([c * ex + s * ey, -s * ex + c * ey, normal], axis=2)
    quat = _quat_from_matrices(R)
    log_t = tangential_log_scale + log_scale_sd * rng.standard_normal((n, 2))
    log_scale = np.concatenate([log_t, (np.log(normal_ratio) + log_t.mean(axis=1))[:, None]], axis=1)
    opacity = 0.1 + 0.9 * rng.random(n)
    logit = _logit(np.clip(opacity, 1e-6, 1 - 1e-6))
    if sh_degree == 0:
        col = color
    else:
        col = sh3_from_rgb(color, rng)
    return GaussianMap(_f32(mean), _f32(quat), _f32(log_scale), _f32(logit), _f32(col))


def perturb_map(g: GaussianMap, seed: int, pos_sd=0.01, color_sd=0.05, logit_sd=0.2) -> GaussianMap:
    """A perturbed copy of a map (used to make a different target image)."""
    rng = np.random.default_rng(seed)
    mean = g.mean + pos_sd * rng.standard_normal(g.mean.shape)
    color = g.color + color_sd * rng.standard_normal(g.color.shape)
    if g.color.ndim == 2:
        color = np.clip(color, 0.0, 1.0)
    logit = g.opacity_logit + logit_sd * rng.standard_normal(g.opacity_logit.shape)
    return GaussianMap(_f32(mean), g.quat.copy(), g.log_scale.copy(), _f32(logit), _f32(color))


def _catmull_rom(p0, p1, p2, p3, t):
    t2, t3 = t * t, t * t * t
    return 0.5 * ((2 * p1) + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t2 + (-p0 + 3 * p1 - 3 * p2 + p3) * t3)


def trajectory_cameras(seed: int, sizes, length=5.0, height=1.4, jitter=0.15, room=(6.0, 5.0, 3.0)):
    """Cameras along a smooth Catmull-Rom path of about `length` metres inside the
    room, one per entry of `sizes` = [(width, height, fx), ...], looking at the
    room's far side with seeded look-at jitter."""
    rng = np.random.default_rng(seed)
    sx, sy, _ = room
    ctrl = np.array([[-length / 2 + length * k / 3.0, 0.6 * (rng.random() - 0.5) * sy * 0.5, height] for k in range(4)])
    ctrl = np.concatenate([ctrl[:1] - (ctrl[1] - ctrl[0]), ctrl, ctrl[-1:] + (ctrl[-1] - ctrl[-2])])
    cams = []
    V = len(sizes)
    for k, (w, h, f) in enumerate(sizes):
        s = (k + 0.5) / V * 3.0
        seg = min(int(s), 2); t = s - seg
        eye = _catmull_rom(ctrl[seg], ctrl[seg + 1], ctrl[seg + 2], ctrl[seg + 3], t)
        yaw = 2 * math.pi * k / V + rng.uniform(-0.3, 0.3)
        target = eye + np.array([math.cos(yaw), math.sin(yaw), 0.0]) * 2.0
        target = target + jitter * rng.standard_normal(3)
        R, e = look_at(eye, target)
        cams.append(Camera(float(f), float(f), w / 2.0, h / 2.0, int(w), int(h), R, e))
    return cams, ctrl[1:-1]


# ---------------------------------------------------------------------------
# The workloads (sizes stated in each docstring)
# ---------------------------------------------------------------------------

def cfg1_problem(trial: int = 0):
    """64x48 image, 256 Gaussians uniform in [-1,1]x[-1,1]x[1,3] in front of an
    identity camera (fx=fy=60, cx=32, cy=24); the target map is the seed+1 cloud."""
    seed = 1000 + trial
    cam = identity_camera(64, 48, 60.0, 60.0, 32.0, 24.0)
    return random_cloud(256, seed), random_cloud(256, seed + 1), cam


_ROOM_EYE = (-2.2, 0.3, 1.4)


def room_camera(width=640, height=480, f=525.0, eye=_ROOM_EYE, target=(2.5, -0.2, 1.1)) -> Camera:
    R, e = look_at(eye, target)
    return Camera(f, f, width / 2.0, height / 2.0, width, height, R, e)


def cfg2_problem(trial: int = 0, n=200_000):
    """640x480 (fx=fy=525) inside a 6x5x3 m room of n Gaussians (6 planes + 20
    boxes, 1 cm surface noise); target map = perturbed copy (seed+1)."""
    seed = 2000 + trial
    g = room_scene(n, seed, keep_out=[_ROOM_EYE])
    return g, perturb_map(g, seed + 1), room_camera()


def cfg3_problem(trial: int = 0, n=500_000):
    """8 keyframes (4x 640x480 fx=525, 2x 752x480 fx=458, 2x 1280x1024 fx=880)
    along a 5 m path inside a 500k-Gaussian room; target = perturbed copy."""
    seed = 3000 + trial
    sizes = [(640, 480, 525.0)] * 4 + [(752, 480, 458.0)] * 2 + [(1280, 1024, 880.0)] * 2
    cams, ctrl = trajectory_cameras(seed, sizes)
    g = room_scene(n, seed, keep_out=[c.t_wc for c in cams])
    return g, perturb_map(g, seed + 1), cams


def cfg4_problem(trial: int = 0, n=1_000_000, views=16, width=1280, height=1024, f=880.0):
    """16 keyframes at 1280x1024 over a 1M-Gaussian room with degree-3 SH colour."""
    seed = 4000 + trial
    sizes = [(width, height, f)] * views
    cams, ctrl = trajectory_cameras(seed, sizes)
    g = room_scene(n, seed, keep_out=[c.t_wc for c in cams], sh_degree=3)
    return g, perturb_map(g, seed + 1), cams


def vi_scene(seed: int, K: int = 4, h: int = 12, w: int = 16, f: float = 20.0, window: int = 2, dt: float = 0.5):
    """ba_scene plus the inertial quantities of Eq. 3 for consecutive keyframes:
    velocities [K, 3], IMU biases [K, 6] (constant along the window, so the bias
    term vanishes), the biases the pre-integration was linearised at [K, 6]
    (a small offset, so the bias corrections are exercised), gravity [3], and
    one pre-integration record per pair [K - 1, 286] (dR, dp, dv, J_rot, J_pos,
    J_vel, dt, 15 x 15 information; see oracle.ba.imu_record) built so that
    every inertial residual is zero at this state.  The pre-integration's own
    Jacobians and information are seeded random values of plausible size (the
    factor is exact for any of them)."""
    R, t, disp, intr, edges, weights = ba_scene(seed, K=K, h=h, w=w, f=f, window=window)
    rng = np.random.default_rng(seed + 17)
    Rb = np.transpose(R, (0, 2, 1))
    pb = -np.einsum("kab,kb->ka", Rb, t)
    vel = rng.normal(0.0, 0.3, (K, 3))
    b = np.concatenate([rng.normal(0, 0.01, 3), rng.normal(0, 0.05, 3)])
    bias = np.tile(b, (K, 1))
    bias_hat = bias + np.concatenate([rng.normal(0, 0.003, (K, 3)), rng.normal(0, 0.01, (K, 3))], 1)
    gravity = np.array([0.0, 0.0, -9.81])

    def exp3(phi):
        th = np.linalg.norm(phi)
        Kx = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
        if th < 1e-12:
            return np.eye(3) + Kx
        return np.eye(3) + np.sin(th) / th * Kx + (1 - np.cos(th)) / th ** 2 * Kx @ Kx

    recs = []
    for i in range(K - 1):
        j = i + 1
        Jrot = -dt * np.eye(3) + rng.normal(0, 0.02, (3, 3))
        Jpos = np.concatenate([rng.normal(0, 0.05, (3, 3)), -0.5 * dt * dt * np.eye(3)], 1)
        Jvel = np.concatenate([rng.normal(0, 0.1, (3, 3)), -dt * np.eye(3)], 1)
        db = bias[i] - bias_hat[i]
        dR = Rb[i].T @ Rb[j] @ exp3(Jrot @ db[:3]).T
        dp = Rb[i].T @ (pb[j] - pb[i] - vel[i] * dt - 0.5 * gravity * dt * dt) - Jpos @ db
        dv = Rb[i].T @ (vel[j] - vel[i] - gravity * dt) - Jvel @ db
        Lm = rng.normal(0, 0.3, (15, 15))
        info = Lm @ Lm.T + np.diag(np.concatenate([np.full(3, 400.0), np.full(3, 100.0), np.full(3, 100.0),
                                                   np.full(6, 1000.0)]))
        recs.append(np.concatenate([dR.reshape(9), dp, dv, Jrot.reshape(9), Jpos.reshape(18), Jvel.reshape(18),
                                    [dt], info.reshape(225)]))
    return R, t, disp, intr, edges, weights, vel, bias, bias_hat, gravity, np.stack(recs)


def refinement_problem(trial: int = 0, n=200_000, views=16, width=640, height=480, f=525.0):
    """A keyframe list for the final colour refinement: `views` keyframes of one
    resolution along a 5 m path inside an n-Gaussian room; the map to refine and
    the perturbed copy whose renders are the targets."""
    seed = 6000 + trial
    cams, ctrl = trajectory_cameras(seed, [(width, height, f)] * views)
    g = room_scene(n, seed, keep_out=[c.t_wc for c in cams])
    return g, perturb_map(g, seed + 1), cams


def mlp_params(seed: int, n_in: int = 196, n_hid: int = 128, n_out: int = 8, bias_sd: float = 0.1) -> dict:
    """Seeded float32 weights of the 196 -> 128 -> 128 -> 8 initialiser network:
    W ~ N(0, 1 / fan_in), biases ~ N(0, bias_sd^2)."""
    rng = np.random.default_rng(seed)
    f = lambda *shape, sd: (rng.standard_normal(shape) * sd).astype(np.float32)
    return {"W1": f(n_hid, n_in, sd=1.0 / np.sqrt(n_in)), "b1": f(n_hid, sd=bias_sd),
            "W2": f(n_hid, n_hid, sd=1.0 / np.sqrt(n_hid)), "b2": f(n_hid, sd=bias_sd),
            "W3": f(n_out, n_hid, sd=1.0 / np.sqrt(n_hid)), "b3": f(n_out, sd=bias_sd)}


def mlp_batch(seed: int, n: int, n_in: int = 196, n_out: int = 8):
    """Seeded float32 inputs X [n, n_in] ~ U(-1, 1) and targets T [n, n_out] ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    return (rng.uniform(-1.0, 1.0, (n, n_in)).astype(np.float32),
            rng.standard_normal((n, n_out)).astype(np.float32))


def ba_scene(seed: int, K: int = 4, h: int = 12, w: int = 16, f: float = 20.0, window: int = 2):
    """A bundle-adjustment window: K keyframes (world-to-camera R [K,3,3], t
    [K,3]) on a short sideways path looking at a smooth surface 2-4 m away,
    each with its inverse-depth map [K, h, w] of that surface seen along the
    pixel rays; edges (i, j) for 0 < |i - j| <= window; positive confidence
    weights [E, h, w, 2]; pinhole intrinsics (fx, fy, cx, cy) of the h x w grid."""
    rng = np.random.default_rng(seed)
    intr = (f, f * (1.0 + 0.05 * rng.uniform(-1, 1)), w / 2.0 + rng.uniform(-0.5, 0.5), h / 2.0 + rng.uniform(-0.5, 0.5))
    R = np.zeros((K, 3, 3)); t = np.zeros((K, 3))
    for k in range(K):
        ang = rng.normal(0.0, 0.02, 3) + np.array([0.0, 0.03 * k, 0.0])
        th = np.linalg.norm(ang)
        Kx = np.array([[0, -ang[2], ang[1]], [ang[2], 0, -ang[0]], [-ang[1], ang[0], 0]])
        Rk = np.eye(3) + np.sin(th) / th * Kx + (1 - np.cos(th)) / th ** 2 * Kx @ Kx if th > 0 else np.eye(3)
        c = np.array([0.15 * k, rng.normal(0, 0.02), rng.normal(0, 0.02)])        # camera centre
        R[k] = Rk; t[k] = -Rk @ c
    ys, xs = np.mgrid[0:h, 0:w]
    a = rng.uniform(-0.5, 0.5, 3)
    disp = np.zeros((K, h, w))
    for k in range(K):
        u = (xs + 0.5 - intr[2]) / intr[0]; v = (ys + 0.5 - intr[3]) / intr[1]
        depth = 3.0 + a[0] * u + a[1] * v + 0.3 * np.sin(2.0 * u + a[2]) * np.cos(1.5 * v)
        disp[k] = 1.0 / depth
    edges = [(i, j) for i in range(K) for j in range(K) if i != j and abs(i - j) <= window]
    weights = rng.uniform(0.5, 2.0, (len(edges), h, w, 2))
    return R, t, disp, intr, edges, weights
