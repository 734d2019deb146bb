"""Python driver of the FP64 C oracle for the splatting path (test infrastructure).

The C source ``render_oracle.c`` is compiled on first use into
``oracle/_build/liboracle.so`` with gcc and OpenMP.  Everything here works on
numpy arrays; scenes are dicts of structure-of-arrays float32 planes as produced
by the seeded input generators:

    means[3][n], log_scales[3][n], quats[4][n] (w,x,y,z), logits[n], rgb[3][n]

Cameras are dicts with width, height, fx, fy, cx, cy, world_to_cam (3x4) and
znear (OpenCV axes, pixel centres at integer coordinates).

The rasteriser constants below are not in the paper (it gives only eq1); they
are the standard values of the Gaussian-splatting rasteriser it cites (Sec. III).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "render_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

# near plane (camera carries it), 2D dilation (px^2), alpha clamp, alpha skip,
# transmittance stop, Jacobian clamp factor, support in sigmas
DILATION = 0.3
ALPHA_MAX = 0.99
ALPHA_MIN = 1.0 / 255.0
T_MIN = 1e-4
JAC_CLAMP = 1.3
SUPPORT_SIGMA = 3.0
KCONST = np.array([0.2, DILATION, ALPHA_MAX, ALPHA_MIN, T_MIN, JAC_CLAMP, SUPPORT_SIGMA],
                  dtype=np.float64)
# decision bands: relative band on alpha vs its thresholds, relative band on T vs
# T_MIN, absolute band on power vs 0.  A float32 evaluation of the same decision
# can land on the other side only inside these bands: on the same float32 splat
# values alpha's relative error is ~1e-6 (rounded power, exp2 approximation) and
# T's ~1e-5 after ~100 rounded products; the bands keep a factor ~5 above that.
BAND = np.array([5e-6, 5e-5, 1e-6], dtype=np.float64)

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc -O2 -fopenmp); returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        # no contraction into fused multiply-adds: the float32 decisions must round
        # every operation separately (aarch64 GCC fuses by default)
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            L.or_project.argtypes = [i64, P, P, P, P, P, P, ctypes.c_int, ctypes.c_int, P, P, P, P, P, P, P]
            L.or_count_pairs.argtypes = [i32, i64, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.or_count_pairs.restype = i64
            L.or_bin_sort.argtypes = [i32, i64, P, P, P, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P]
            L.or_bin_sort.restype = i64
            L.or_render_fwd.argtypes = [i64, P, P, P, P, P, P, P, P, ctypes.c_int, ctypes.c_int, P, P,
                                        i32, P, P, P, P, P, P]
            L.or_render_brute.argtypes = [i64, P, P, P, P, P, P, P, P, P, P, ctypes.c_int,
                                          ctypes.c_int, P, P, P]
            L.or_trace_pixel.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P, P, P, P, ctypes.c_int,
                                         ctypes.c_int, P, P, i32, P, i64]
            L.or_trace_pixel.restype = i64
            L.or_render_bwd.argtypes = [i64, P, P, P, P, P, P, P, ctypes.c_int, ctypes.c_int, P, P, i32,
                                        P, P, P, P, P]
            L.or_project_bwd.argtypes = [i64, P, P, P, P, P, P, P, P, P, P, P]
            L.or_loss.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P, f64, f64, f64, P, P]
            L.or_loss.restype = f64
            L.or_scale_reg.argtypes = [i64, P, f64, P]
            L.or_scale_reg.restype = f64
            L.or_adam.argtypes = [i64, P, P, P, P, f64, f64, f64, f64, i32]
            L.or_num_threads.restype = ctypes.c_int
            L.or_set_num_threads.argtypes = [ctypes.c_int]
            L.or_set_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_num_threads(n: int) -> int:
    """Threads of the oracle's OpenMP regions; returns the previous count."""
    return int(lib().or_set_num_threads(int(n)))


# ----------------------------------------------------------------------------------
# scene / camera conversion (structure-of-arrays float32 -> AoS float64)

def aos(scene: dict) -> dict:
    """Scene planes -> contiguous float64 arrays [n][k]."""
    return {
        "means": np.ascontiguousarray(np.asarray(scene["means"], np.float64).T),
        "log_scales": np.ascontiguousarray(np.asarray(scene["log_scales"], np.float64).T),
        "quats": np.ascontiguousarray(np.asarray(scene["quats"], np.float64).T),
        "logits": np.ascontiguousarray(np.asarray(scene["logits"], np.float64)),
        "rgb": np.ascontiguousarray(np.asarray(scene["rgb"], np.float64).T),
    }


def cam_vec(cam: dict) -> np.ndarray:
    w2c = np.asarray(cam["world_to_cam"], np.float64).reshape(3, 4)
    return np.concatenate([[cam["width"], cam["height"], cam["fx"], cam["fy"], cam["cx"], cam["cy"]],
                           w2c[:, :3].reshape(-1), w2c[:, 3], [cam["znear"]]]).astype(np.float64)


def tiles_of(cam: dict, tile_w: int, tile_h: int):
    return (cam["width"] + tile_w - 1) // tile_w, (cam["height"] + tile_h - 1) // tile_h


# ----------------------------------------------------------------------------------

def project(scene_aos: dict, cam: dict, tile_w: int = 16, tile_h: int = 16) -> dict:
    """EWA projection of every Gaussian into one view (Sec. III, C = R S S^T R^T).

    Returns mean2d[n][2], conic[n][3] (inverse of the dilated 2D covariance),
    depth[n] (camera z), opacity[n] (sigmoid of the logit), radius[n] (0 = culled),
    rect[n][4] (inclusive tile bounds of the 3-sigma box; x0 > x1 = none) and
    thr[n] (support threshold 2 ln(255 o) + margin; tiles where the splat's
    Mahalanobis form exceeds it everywhere cannot reach alpha 1/255)."""
    n = scene_aos["means"].shape[0]
    out = {
        "mean2d": np.zeros((n, 2)), "conic": np.zeros((n, 3)), "depth": np.zeros(n),
        "opacity": np.zeros(n), "radius": np.zeros(n, np.int32), "rect": np.zeros((n, 4), np.int32),
        "thr": np.zeros(n),
    }
    cv = cam_vec(cam)
    lib().or_project(n, _p(scene_aos["means"]), _p(scene_aos["log_scales"]), _p(scene_aos["quats"]),
                     _p(scene_aos["logits"]), _p(cv), _p(KCONST), tile_w, tile_h, _p(out["mean2d"]),
                     _p(out["conic"]), _p(out["depth"]), _p(out["opacity"]), _p(out["radius"]),
                     _p(out["rect"]), _p(out["thr"]))
    return out


def support_f64(splats: dict) -> np.ndarray:
    """[n][6] double (mx, my, a, b, c, thr) of one view's FP64 splats."""
    return np.ascontiguousarray(np.concatenate([splats["mean2d"], splats["conic"], splats["thr"][:, None]], 1))


def bin_sort(cams: list, tile_w: int, tile_h: int, depth_f32: np.ndarray, radius: np.ndarray,
             rect: np.ndarray, supp: np.ndarray | None = None):
    """Sorted (tile, Gaussian) lists of a view set.

    depth_f32[v][n] float32, radius[v][n], rect[v][n][4], supp[v][n][6] (mx, my, a,
    b, c, thr; float32 -> the support test in float32, float64 -> in double; None:
    the whole rect).  Order: global tile, float32 depth bits, id.  Returns
    (tile[P] uint32, id[P] int32, ranges[T][2])."""
    V = len(cams)
    n = depth_f32.shape[1]
    tx = np.array([tiles_of(c, tile_w, tile_h)[0] for c in cams], np.int32)
    ty = np.array([tiles_of(c, tile_w, tile_h)[1] for c in cams], np.int32)
    depth_f32 = np.ascontiguousarray(depth_f32, np.float32)
    radius = np.ascontiguousarray(radius, np.int32)
    rect = np.ascontiguousarray(rect, np.int32)
    sp, f32 = None, 0
    if supp is not None:
        f32 = 1 if supp.dtype == np.float32 else 0
        supp = np.ascontiguousarray(supp, np.float32 if f32 else np.float64)
        sp = _p(supp)
    P = lib().or_count_pairs(V, n, _p(radius), _p(rect), sp, f32, tile_w, tile_h)
    tiles = np.zeros(max(P, 1), np.uint32)
    ids = np.zeros(max(P, 1), np.int32)
    ranges = np.zeros((int((tx * ty).sum()), 2), np.int32)
    P2 = lib().or_bin_sort(V, n, _p(tx), _p(ty), _p(depth_f32), _p(radius), _p(rect), sp, f32, tile_w, tile_h,
                           _p(tiles), _p(ids), _p(ranges))
    assert P2 == P
    return tiles[:P], ids[:P], ranges


def _splat_arrays(splats: dict):
    return (np.ascontiguousarray(splats["mean2d"], np.float64), np.ascontiguousarray(splats["conic"], np.float64),
            np.ascontiguousarray(splats["depth"], np.float64), np.ascontiguousarray(splats["opacity"], np.float64))


def render_fwd(splats: dict, rgb: np.ndarray, cam: dict, ids: np.ndarray, ranges: np.ndarray,
               tile_base: int = 0, tile_w: int = 16, tile_h: int = 16) -> dict:
    """Tile-binned eq1 for one view (colour gamma = c, depth gamma = z, opacity
    gamma = 1).  splats: mean2d[n][2], conic[n][3], depth[n], opacity[n] of this
    view; rgb[n][3].  Returns color[3][H][W], depth, alpha, t_final [H][W],
    n_contrib and flag (1 where a decision was inside the float32 band)."""
    W, H = cam["width"], cam["height"]
    m2, cn, dp, op = _splat_arrays(splats)
    rgb = np.ascontiguousarray(rgb, np.float64)
    ids = np.ascontiguousarray(ids, np.int32)
    ranges = np.ascontiguousarray(ranges, np.int32)
    out = {"color": np.zeros((3, H, W)), "depth": np.zeros((H, W)), "alpha": np.zeros((H, W)),
           "t_final": np.zeros((H, W)), "n_contrib": np.zeros((H, W), np.int32),
           "flag": np.zeros((H, W), np.uint8)}
    lib().or_render_fwd(m2.shape[0], _p(m2), _p(cn), _p(dp), _p(op), _p(rgb), _p(cam_vec(cam)), _p(KCONST),
                        _p(BAND), tile_w, tile_h, _p(ids), _p(ranges), tile_base, _p(out["color"]),
                        _p(out["depth"]), _p(out["alpha"]), _p(out["t_final"]), _p(out["n_contrib"]),
                        _p(out["flag"]))
    return out


def render_brute(splats: dict, rgb: np.ndarray, cam: dict, depth_f32: np.ndarray, radius: np.ndarray,
                 rect: np.ndarray, tile_w: int = 16, tile_h: int = 16) -> dict:
    """Brute-force eq1: all Gaussians whose rect holds the pixel's tile, ordered
    per pixel by an insertion sort on (float32 depth bits, id)."""
    W, H = cam["width"], cam["height"]
    m2, cn, dp, op = _splat_arrays(splats)
    rgb = np.ascontiguousarray(rgb, np.float64)
    out = {"color": np.zeros((3, H, W)), "depth": np.zeros((H, W)), "alpha": np.zeros((H, W))}
    lib().or_render_brute(m2.shape[0], _p(m2), _p(cn), _p(dp), _p(op), _p(rgb),
                          _p(np.ascontiguousarray(depth_f32, np.float32)),
                          _p(np.ascontiguousarray(radius, np.int32)), _p(np.ascontiguousarray(rect, np.int32)),
                          _p(cam_vec(cam)), _p(KCONST), tile_w, tile_h, _p(out["color"]), _p(out["depth"]),
                          _p(out["alpha"]))
    return out


def trace_pixel(x: int, y: int, splats: dict, rgb: np.ndarray, cam: dict, ids, ranges, tile_base=0,
                tile_w=16, tile_h=16, max_len=4096) -> np.ndarray:
    """Transmittance before each blended Gaussian of pixel (x, y), then T_final."""
    m2, cn, dp, op = _splat_arrays(splats)
    rgb = np.ascontiguousarray(rgb, np.float64)
    tr = np.zeros(max_len)
    m = lib().or_trace_pixel(x, y, _p(m2), _p(cn), _p(dp), _p(op), _p(rgb), _p(cam_vec(cam)), _p(KCONST),
                             tile_w, tile_h, _p(np.ascontiguousarray(ids, np.int32)),
                             _p(np.ascontiguousarray(ranges, np.int32)), tile_base, _p(tr), max_len)
    return tr[:m]


def render_bwd(splats: dict, rgb: np.ndarray, cam: dict, ids, ranges, dC, dD=None, dA=None,
               tile_base: int = 0, tile_w: int = 16, tile_h: int = 16):
    """Adjoint of eq1 for one view.  Returns grad2d[n][7] (mean2d x, y, conic a, b,
    c, opacity, depth) and grad_rgb[n][3]."""
    m2, cn, dp, op = _splat_arrays(splats)
    n = m2.shape[0]
    rgb = np.ascontiguousarray(rgb, np.float64)
    g2 = np.zeros((n, 7))
    grgb = np.zeros((n, 3))
    dC = np.ascontiguousarray(dC, np.float64)
    keep = [np.ascontiguousarray(dD, np.float64) if dD is not None else None,
            np.ascontiguousarray(dA, np.float64) if dA is not None else None]
    dDp = _p(keep[0]) if keep[0] is not None else None
    dAp = _p(keep[1]) if keep[1] is not None else None
    lib().or_render_bwd(n, _p(m2), _p(cn), _p(dp), _p(op), _p(rgb), _p(cam_vec(cam)), _p(KCONST), tile_w,
                        tile_h, _p(np.ascontiguousarray(ids, np.int32)), _p(np.ascontiguousarray(ranges, np.int32)),
                        tile_base, _p(dC), dDp, dAp, _p(g2), _p(grgb))
    return g2, grgb


def project_bwd(scene_aos: dict, cam: dict, grad2d: np.ndarray, grads: dict | None = None) -> dict:
    """Chain rule of :func:`project` for one view; accumulates into (and returns)
    grads = dict(means[n][3], log_scales[n][3], quats[n][4], logits[n])."""
    n = scene_aos["means"].shape[0]
    if grads is None:
        grads = {"means": np.zeros((n, 3)), "log_scales": np.zeros((n, 3)), "quats": np.zeros((n, 4)),
                 "logits": np.zeros(n), "rgb": np.zeros((n, 3))}
    lib().or_project_bwd(n, _p(scene_aos["means"]), _p(scene_aos["log_scales"]), _p(scene_aos["quats"]),
                         _p(scene_aos["logits"]), _p(cam_vec(cam)), _p(KCONST),
                         _p(np.ascontiguousarray(grad2d, np.float64)), _p(grads["means"]),
                         _p(grads["log_scales"]), _p(grads["quats"]), _p(grads["logits"]))
    return grads


def loss(color, depth, color_gt, depth_gt, w_c=0.9, w_d=0.1, w_s=0.1):
    """eq16 (without the eq15 term) for one view; returns (L, dL/dC, dL/dD)."""
    C = np.ascontiguousarray(color, np.float64)
    H, W = C.shape[1], C.shape[2]
    dC = np.zeros_like(C)
    dD = np.zeros((H, W))
    L = lib().or_loss(W, H, _p(C), _p(np.ascontiguousarray(depth, np.float64)),
                      _p(np.ascontiguousarray(color_gt, np.float64)), _p(np.ascontiguousarray(depth_gt, np.float64)),
                      w_c, w_d, w_s, _p(dC), _p(dD))
    return L, dC, dD


def scale_reg(log_scales_aos: np.ndarray, weight: float):
    """eq15 times weight; returns (value, dL/dlog_scales[n][3])."""
    ls = np.ascontiguousarray(log_scales_aos, np.float64)
    g = np.zeros_like(ls)
    val = lib().or_scale_reg(ls.shape[0], _p(ls), weight, _p(g))
    return val, g


def adam(p, g, m, v, lr, b1=0.9, b2=0.999, eps=1e-15, t=1):
    """Bias-corrected Adam, in place on float64 arrays."""
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    lib().or_adam(p.size, _p(p), _p(g), _p(m), _p(v), lr, b1, b2, eps, t)


# ----------------------------------------------------------------------------------
# whole views and mapping steps

def splats_from_gpu(splat: np.ndarray, radius: np.ndarray, rect: np.ndarray) -> dict:
    """Teacher forcing: a view's float32 splat records [n][8] (mean2d, conic,
    opacity, depth, support threshold) and integer support, widened to float64."""
    s = np.asarray(splat, np.float64)
    return {"mean2d": np.ascontiguousarray(s[:, 0:2]), "conic": np.ascontiguousarray(s[:, 2:5]),
            "opacity": np.ascontiguousarray(s[:, 5]), "depth": np.ascontiguousarray(s[:, 6]),
            "thr": np.ascontiguousarray(s[:, 7]), "radius": np.asarray(radius, np.int32),
            "rect": np.asarray(rect, np.int32)}


def support_f32(splat: np.ndarray) -> np.ndarray:
    """[n][6] float32 (mx, my, a, b, c, thr) straight from a view's GPU records."""
    s = np.asarray(splat, np.float32)
    return np.ascontiguousarray(s[:, [0, 1, 2, 3, 4, 7]])


def render_views(scene: dict, cams: list, tile_w=16, tile_h=16) -> dict:
    """Project, bin and blend a view set from the FP64 scene.  Keys use the
    float32 rounding of the FP64 depth.  Returns per-view lists of outputs plus
    the splats and lists needed by :func:`backward_views`."""
    sa = aos(scene)
    projs, depth32, radius, rect = [], [], [], []
    for cam in cams:
        pr = project(sa, cam, tile_w, tile_h)
        projs.append(pr)
        depth32.append(pr["depth"].astype(np.float32))
        radius.append(pr["radius"])
        rect.append(pr["rect"])
    tiles, ids, ranges = bin_sort(cams, tile_w, tile_h, np.stack(depth32), np.stack(radius), np.stack(rect),
                                  np.stack([support_f64(p) for p in projs]))
    outs, base = [], 0
    for cam, pr in zip(cams, projs):
        outs.append(render_fwd(pr, sa["rgb"], cam, ids, ranges, base, tile_w, tile_h))
        tx, ty = tiles_of(cam, tile_w, tile_h)
        base += tx * ty
    return {"scene_aos": sa, "proj": projs, "tiles": tiles, "ids": ids, "ranges": ranges, "out": outs,
            "tile_w": tile_w, "tile_h": tile_h}


def backward_views(state: dict, cams: list, dCs: list, dDs: list, dAs: list | None = None) -> dict:
    """Gradients of every Gaussian parameter given per-view dL/d(C, D, A)."""
    sa = state["scene_aos"]
    n = sa["means"].shape[0]
    grads = {"means": np.zeros((n, 3)), "log_scales": np.zeros((n, 3)), "quats": np.zeros((n, 4)),
             "logits": np.zeros(n), "rgb": np.zeros((n, 3))}
    base = 0
    for v, cam in enumerate(cams):
        g2, grgb = render_bwd(state["proj"][v], sa["rgb"], cam, state["ids"], state["ranges"], dCs[v], dDs[v],
                              None if dAs is None else dAs[v], base, state["tile_w"], state["tile_h"])
        grads["rgb"] += grgb
        project_bwd(sa, cam, g2, grads)
        tx, ty = tiles_of(cam, state["tile_w"], state["tile_h"])
        base += tx * ty
    return grads


def grads_to_planes(grads: dict) -> dict:
    """AoS gradient dict -> structure-of-arrays planes like the scene."""
    return {"means": grads["means"].T.copy(), "log_scales": grads["log_scales"].T.copy(),
            "quats": grads["quats"].T.copy(), "logits": grads["logits"].copy(), "rgb": grads["rgb"].T.copy()}
