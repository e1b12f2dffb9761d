"""FP64 CPU oracle of the Gaussian-splatting mapping step (VIGS-SLAM Sec. 3.3, Eq. 6).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the product path never
does.  The arithmetic lives in ``gs_oracle.c`` (plain C, double precision,
compiled here with gcc on first use); this module only marshals numpy arrays.

Parity status of each function (what pins it, see ``tests/test_oracle_*.py``):
  project       closed form on the optical axis, Monte-Carlo covariance of the
                exact perspective map, scipy rotations, rigid-motion invariance
  bin_sort      brute-force Python enumeration + ``sorted`` (library sort)
  render_fwd    closed-form single splat, partition of unity, transmittance
                product, order invariance, a numpy per-pixel sum without tiles
  render_bwd /  central finite differences of the oracle forward (smooth and
  project_bwd   method mode), pose tangent included
  l1_loss       torch.nn.functional.l1_loss and its autograd gradient
  iso_loss      finite differences + a hand-checked special case
  adam          torch.optim.Adam in float64
  sh basis      orthonormality on the sphere by quadrature
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

DEFAULT_PARAMS = dict(tile=16, near=0.2, alpha_min=1.0 / 255.0, alpha_max=0.99, T_cut=1e-4,
                      dilation=0.3, radius_sigma=3.0, bg=(0.0, 0.0, 0.0), smooth=False, sh_degree=0)


def build(force: bool = False) -> str:
    """Compile gs_oracle.c into _build/liboracle.so (gcc, -O2, no FMA contraction,
    OpenMP for the optional host threads; without OpenMP the loops run serially)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except (subprocess.CalledProcessError, OSError):
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.or_bin_count.restype = ctypes.c_long
        _lib.or_bin_sort.restype = ctypes.c_long
        _lib.or_iso_loss.restype = ctypes.c_double
        _lib.or_tile_rect.restype = ctypes.c_int
        _lib.or_set_threads.restype = ctypes.c_int
        _lib.or_set_threads.argtypes = [ctypes.c_int]
        _lib.or_num_procs.restype = ctypes.c_int
    return _lib


def set_threads(n: int) -> int:
    """Host threads of the oracle's parallel loops (results are bit-identical
    for every count); returns the previous count."""
    return int(_load().or_set_threads(int(n)))


def num_procs() -> int:
    """Processors the parallel loops can use (1 if built without OpenMP)."""
    return int(_load().or_num_procs())


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def cam_array(cam) -> np.ndarray:
    return np.array([cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height,
                     *np.asarray(cam.R_wc, dtype=np.float64).reshape(9),
                     *np.asarray(cam.t_wc, dtype=np.float64).reshape(3)], dtype=np.float64)


def prm_array(prm: dict) -> np.ndarray:
    p = dict(DEFAULT_PARAMS); p.update(prm)
    return np.array([p["tile"], p["near"], p["alpha_min"], p["alpha_max"], p["T_cut"], p["dilation"],
                     p["radius_sigma"], *p["bg"], 1.0 if p["smooth"] else 0.0, p["sh_degree"]], dtype=np.float64)


def tiles_of(cam, prm) -> tuple[int, int]:
    t = dict(DEFAULT_PARAMS, **prm)["tile"]
    return (int(cam.width) + t - 1) // t, (int(cam.height) + t - 1) // t


# ----------------------------------------------------------------- projection

def project(g, cam, prm: dict) -> dict:
    """Per-Gaussian projection into one view: xy, cov2 (a, b, c), conic (A, B, C),
    depth (camera z), opacity, rgb, radius, rect (x0, y0, x1, y1), tiles, margin."""
    lib = _load()
    n = g.n
    mean, quat, ls, logit, col = (_d(a) for a in g.arrays())
    out = dict(xy=np.zeros((n, 2)), cov2=np.zeros((n, 3)), conic=np.zeros((n, 3)), depth=np.zeros(n),
               opacity=np.zeros(n), rgb=np.zeros((n, 3)), radius=np.zeros(n, np.int32),
               rect=np.zeros((n, 4), np.int32), tiles=np.zeros(n, np.int32), margin=np.zeros(n))
    c = cam_array(cam); pr = prm_array(prm)
    lib.or_project(ctypes.c_long(n), _p(mean), _p(quat), _p(ls), _p(logit), _p(col), _p(c), _p(pr),
                   _p(out["xy"]), _p(out["cov2"]), _p(out["conic"]), _p(out["depth"]), _p(out["opacity"]),
                   _p(out["rgb"]), _p(out["radius"]), _p(out["rect"]), _p(out["tiles"]), _p(out["margin"]))
    return out


def quat_to_rot(q) -> np.ndarray:
    lib = _load()
    q = _d(q); R = np.zeros(9)
    lib.or_quat_to_rot(_p(q), _p(R))
    return R.reshape(3, 3)


def sh_basis(d) -> np.ndarray:
    lib = _load()
    d = _d(d); Y = np.zeros(16)
    lib.or_sh_basis(_p(d), _p(Y))
    return Y


def tile_rect(mx, my, r, tile, tx, ty):
    lib = _load()
    rect = np.zeros(4, np.int32)
    k = lib.or_tile_rect(ctypes.c_double(mx), ctypes.c_double(my), ctypes.c_int(r), ctypes.c_int(tile),
                         ctypes.c_int(tx), ctypes.c_int(ty), _p(rect))
    return rect, k


# -------------------------------------------------------------------- binning

def bin_sort(depth_f32, rect, view_of, tile_base, tiles_x, total_tiles):
    """Keys (uint64), values (uint32) and per-tile ranges [total_tiles, 2]."""
    lib = _load()
    depth_f32 = np.ascontiguousarray(depth_f32, dtype=np.float32)
    rect = np.ascontiguousarray(rect, dtype=np.int32)
    view_of = np.ascontiguousarray(view_of, dtype=np.int32)
    tile_base = np.ascontiguousarray(tile_base, dtype=np.int32)
    tiles_x = np.ascontiguousarray(tiles_x, dtype=np.int32)
    E = depth_f32.shape[0]
    m = lib.or_bin_count(ctypes.c_long(E), _p(rect))
    keys = np.zeros(max(m, 1), np.uint64); vals = np.zeros(max(m, 1), np.uint32)
    ranges = np.zeros((total_tiles, 2), np.uint32)
    lib.or_bin_sort(ctypes.c_long(E), _p(depth_f32), _p(rect), _p(view_of), _p(tile_base), _p(tiles_x),
                    ctypes.c_long(total_tiles), _p(keys), _p(vals), _p(ranges))
    return keys[:m], vals[:m], ranges


# ---------------------------------------------------------------- compositing

def _proj_arrays(pr):
    return (_d(pr["xy"]), _d(pr["conic"]), _d(pr["opacity"]), _d(pr["rgb"]), _d(pr["depth"]),
            np.ascontiguousarray(pr["rect"], dtype=np.int32))


def render_fwd(pr: dict, cam, prm: dict) -> dict:
    """Colour [3, H, W], depth, T_final, n_contrib [H, W] and threshold margins."""
    lib = _load()
    xy, conic, op, rgb, depth, rect = _proj_arrays(pr)
    n = xy.shape[0]
    H, W = int(cam.height), int(cam.width)
    out = dict(color=np.zeros((3, H, W)), depth=np.zeros((H, W)), T_final=np.zeros((H, W)),
               n_contrib=np.zeros((H, W), np.int32), margin=np.zeros((H, W)))
    lib.or_render_fwd(ctypes.c_long(n), _p(xy), _p(conic), _p(op), _p(rgb), _p(depth), _p(rect),
                      _p(cam_array(cam)), _p(prm_array(prm)), _p(out["color"]), _p(out["depth"]),
                      _p(out["T_final"]), _p(out["n_contrib"]), _p(out["margin"]))
    return out


def render_bwd(pr: dict, cam, prm: dict, dcolor, ddepth) -> dict:
    """Gradients of <dcolor, colour> + <ddepth, depth> w.r.t. the projected
    quantities: xy [n,2], conic [n,3], opacity [n], rgb [n,3], depth [n]."""
    lib = _load()
    xy, conic, op, rgb, depth, rect = _proj_arrays(pr)
    n = xy.shape[0]
    dcolor = _d(dcolor); ddepth = _d(ddepth)
    out = dict(xy=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n), rgb=np.zeros((n, 3)),
               depth=np.zeros(n))
    lib.or_render_bwd(ctypes.c_long(n), _p(xy), _p(conic), _p(op), _p(rgb), _p(depth), _p(rect),
                      _p(cam_array(cam)), _p(prm_array(prm)), _p(dcolor), _p(ddepth),
                      _p(out["xy"]), _p(out["conic"]), _p(out["opacity"]), _p(out["rgb"]), _p(out["depth"]))
    return out


def project_bwd(g, cam, prm: dict, g2d: dict) -> dict:
    """Chain rule from projected-quantity gradients to the parameters and the
    pose tangent (rho, phi) of T_cw <- Exp(xi) T_cw."""
    lib = _load()
    n = g.n
    mean, quat, ls, logit, col = (_d(a) for a in g.arrays())
    out = dict(mean=np.zeros((n, 3)), quat=np.zeros((n, 4)), log_scale=np.zeros((n, 3)),
               opacity_logit=np.zeros(n), color=np.zeros(col.shape), pose=np.zeros(6))
    lib.or_project_bwd(ctypes.c_long(n), _p(mean), _p(quat), _p(ls), _p(logit), _p(col),
                       _p(cam_array(cam)), _p(prm_array(prm)),
                       _p(_d(g2d["xy"])), _p(_d(g2d["conic"])), _p(_d(g2d["opacity"])), _p(_d(g2d["rgb"])),
                       _p(_d(g2d["depth"])), _p(out["mean"]), _p(out["quat"]), _p(out["log_scale"]),
                       _p(out["opacity_logit"]), _p(out["color"]), _p(out["pose"]))
    return out


# --------------------------------------------------------------------- losses

def l1_loss(color, depth, tcolor, tdepth, lambda_c, lambda_d):
    """(L_c, L_d), dL/dcolour, dL/ddepth for one view (Eq. 6 colour and depth terms)."""
    lib = _load()
    color = _d(color); depth = _d(depth); tcolor = _d(tcolor); tdepth = _d(tdepth)
    HW = depth.size
    terms = np.zeros(2); dc = np.zeros_like(color); dd = np.zeros_like(depth)
    lib.or_l1_loss(ctypes.c_long(HW), _p(color), _p(depth), _p(tcolor), _p(tdepth), ctypes.c_double(lambda_c),
                   ctypes.c_double(lambda_d), _p(terms), _p(dc), _p(dd))
    return terms, dc, dd


def iso_loss(log_scale, lam):
    """L_iso and lam * dL_iso/dlog_scale."""
    lib = _load()
    ls = _d(log_scale); g = np.zeros_like(ls)
    L = lib.or_iso_loss(ctypes.c_long(ls.shape[0]), _p(ls), ctypes.c_double(lam), _p(g))
    return L, g


def adam(param, grad, m, v, lr, beta1=0.9, beta2=0.999, eps=1e-15, step=1):
    """In-place Adam step on float64 arrays."""
    lib = _load()
    for a in (param, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    grad = _d(grad)
    lib.or_adam(ctypes.c_long(param.size), _p(param), _p(grad), _p(m), _p(v), ctypes.c_double(lr),
                ctypes.c_double(beta1), ctypes.c_double(beta2), ctypes.c_double(eps), ctypes.c_int(step))


# ------------------------------------------------------------ whole iteration

@dataclass
class StepResult:
    images: list
    proj: list
    loss_terms: list
    iso: float
    loss: float
    grads: dict
    pose_grads: np.ndarray
    g2d: list = field(default_factory=list)


PARAM_NAMES = ("mean", "quat", "log_scale", "opacity_logit", "color")


def mapping_loss_and_grads(g, cams, targets, prm: dict, lambdas=(1.0, 1.0, 0.0)) -> StepResult:
    """Render every view, take the Eq. 6 loss against (target colour, target
    depth) per view summed over views, and back-propagate to every parameter
    and every view's pose tangent."""
    lam_c, lam_d, lam_iso = lambdas
    grads = {k: np.zeros(np.shape(a), dtype=np.float64) for k, a in zip(PARAM_NAMES, g.arrays())}
    pose = np.zeros((len(cams), 6))
    images, projs, terms, g2ds = [], [], [], []
    total = 0.0
    for v, (cam, (tc, td)) in enumerate(zip(cams, targets)):
        pr = project(g, cam, prm)
        img = render_fwd(pr, cam, prm)
        t, dc, dd = l1_loss(img["color"], img["depth"], tc, td, lam_c, lam_d)
        g2d = render_bwd(pr, cam, prm, dc, dd)
        gp = project_bwd(g, cam, prm, g2d)
        for k in PARAM_NAMES:
            grads[k] += gp[k]
        pose[v] = gp["pose"]
        total += lam_c * t[0] + lam_d * t[1]
        images.append(img); projs.append(pr); terms.append(t); g2ds.append(g2d)
    iso = 0.0
    if lam_iso != 0.0:
        iso, gi = iso_loss(g.log_scale, lam_iso)
        grads["log_scale"] += gi
        total += lam_iso * iso
    return StepResult(images, projs, terms, iso, total, grads, pose, g2ds)


def mapping_iteration(g, cams, targets, prm: dict, lambdas, lrs, state: dict, beta1=0.9, beta2=0.999,
                      eps=1e-15) -> StepResult:
    """One whole mapping iteration (Sec. 3.3 "Map Management"): the loss and
    gradients of mapping_loss_and_grads, then one Adam step of every parameter
    group with its learning rate (lrs in PARAM_NAMES order).  state holds the
    float64 parameters ("params": dict by name), the moments ("m", "v") and the
    step count ("step"); all are updated in place."""
    res = mapping_loss_and_grads(g, cams, targets, prm, lambdas)
    state["step"] += 1
    for k, lr in zip(PARAM_NAMES, lrs):
        adam(state["params"][k], res.grads[k], state["m"][k], state["v"][k], lr, beta1, beta2, eps, state["step"])
    return res


def adam_state(g) -> dict:
    """float64 copies of the map's parameters and zero Adam moments."""
    params = {k: np.array(a, dtype=np.float64, copy=True) for k, a in zip(PARAM_NAMES, g.arrays())}
    return {"params": params, "m": {k: np.zeros_like(a) for k, a in params.items()},
            "v": {k: np.zeros_like(a) for k, a in params.items()}, "step": 0}
