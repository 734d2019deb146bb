"""Thin ctypes binding of libfgs.so (the C ABI in include/fgs.h).

Every ``fgs_*`` function here marshals torch tensors into the C structs and
calls the entry point of the same name; all computation runs in the library's
CUDA kernels on the current torch stream.  There is no fallback: a missing or
unloadable library raises.

Besides the raw calls, :class:`GaussianMap` keeps the structure-of-arrays
Gaussian planes (``[14][capacity]`` float32: means 3, log-scales 3, quaternion 4,
opacity logit 1, rgb 3) and :class:`Frame` the per-view render buffers.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfgs.so")

c_void_p, c_int32, c_int64, c_float, c_size_t = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float,
                                                 ctypes.c_size_t)

FGS_DEV_PAIR_OVERFLOW, FGS_DEV_TIMEOUT, FGS_DEV_NONFINITE, FGS_DEV_MAP_FULL, FGS_DEV_WORK_OVERFLOW = 1, 2, 4, 8, 16
MAX_VIEWS = 16
PRIOR_IN, PRIOR_HID, PRIOR_OUT = 272, 128, 4


class Camera(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("fx", c_float), ("fy", c_float), ("cx", c_float),
                ("cy", c_float), ("world_to_cam", c_float * 12), ("znear", c_float)]


class Gaussians(ctypes.Structure):
    _fields_ = [("n", c_int64), ("capacity", c_int64), ("d_n", c_void_p), ("means", c_void_p),
                ("log_scales", c_void_p), ("quats", c_void_p), ("opacity_logits", c_void_p), ("rgb", c_void_p)]


class Projected(ctypes.Structure):
    _fields_ = [("stride", c_int64), ("splat", c_void_p), ("radius", c_void_p), ("rect", c_void_p)]


class Tiling(ctypes.Structure):
    _fields_ = [("tile_w", c_int32), ("tile_h", c_int32), ("batch_depth", c_int32)]


class LossParams(ctypes.Structure):
    _fields_ = [("w_l1_color", c_float), ("w_l1_depth", c_float), ("w_ssim", c_float)]


class AdamParams(ctypes.Structure):
    _fields_ = [("lr", c_float * 5), ("beta1", c_float), ("beta2", c_float), ("eps", c_float), ("step", c_int32)]


class Grid(ctypes.Structure):
    _fields_ = [("origin", c_float * 3), ("cell", c_float), ("dims", c_int32 * 3)]


class GicpParams(ctypes.Structure):
    _fields_ = [("iterations", c_int32), ("max_dist", c_float), ("overlap_dist", c_float)]


def grid(origin, cell: float, dims) -> Grid:
    g = Grid()
    for k in range(3):
        g.origin[k] = float(origin[k])
        g.dims[k] = int(dims[k])
    g.cell = float(cell)
    return g


def grid_cells(g: Grid) -> int:
    return int(g.dims[0]) * int(g.dims[1]) * int(g.dims[2])


class PruneParams(ctypes.Structure):
    _fields_ = [("min_logit", c_float), ("max_log_scale", c_float)]


class SeedParams(ctypes.Structure):
    _fields_ = [("d0", c_float), ("m", c_int32), ("n", c_int32), ("alpha_h", c_float), ("alpha_l", c_float),
                ("tau_alpha", c_float), ("tau_depth_rel", c_float), ("tau_color", c_float), ("max_new", c_int32),
                ("init_logit", c_float), ("prior_max_dev", c_float)]


class MLP(ctypes.Structure):
    _fields_ = [("w1", c_void_p), ("b1", c_void_p), ("w2", c_void_p), ("b2", c_void_p), ("w3", c_void_p),
                ("b3", c_void_p)]


class MLPMaster(ctypes.Structure):
    _fields_ = [("w1", c_void_p), ("b1", c_void_p), ("w2", c_void_p), ("b2", c_void_p), ("w3", c_void_p),
                ("b3", c_void_p), ("m", c_void_p), ("v", c_void_p)]


class TrainParams(ctypes.Structure):
    _fields_ = [("lr", c_float), ("beta1", c_float), ("beta2", c_float), ("eps", c_float), ("step", c_int32)]


_lock = threading.Lock()
_lib = None

_SIGS = {
    "fgs_project": ([c_void_p, c_void_p, c_int32, Tiling, c_void_p, c_void_p, c_void_p], c_int32),
    "fgs_num_tiles": ([c_void_p, c_int32, Tiling], c_int64),
    "fgs_bin_sort": ([c_void_p, c_int64, c_void_p, c_void_p, c_int32, Tiling, c_void_p, c_size_t, c_void_p, c_void_p,
                      c_int64, c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "fgs_bin_sort_workspace_size": ([c_void_p, c_int32, Tiling, c_int64, c_int64], c_size_t),
    "fgs_render_fwd": ([c_void_p, c_void_p, c_void_p, c_int32, Tiling, c_void_p, c_void_p, c_void_p, c_void_p,
                        c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "fgs_render_fwd_sampled": ([c_void_p, c_void_p, c_void_p, c_int32, Tiling, c_void_p, c_void_p, c_void_p,
                                c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p],
                               c_int32),
    "fgs_tile_order": ([c_void_p, c_int32, Tiling, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p], c_int32),
    "fgs_tile_order_workspace_size": ([c_void_p, c_int32, Tiling], c_size_t),
    "fgs_render_bwd": ([c_void_p, c_void_p, c_void_p, c_int32, Tiling, c_void_p, c_void_p, c_void_p, c_void_p,
                        c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "fgs_render_bwd_splats": ([c_void_p, c_void_p, c_void_p, c_int32, Tiling, c_void_p, c_void_p, c_void_p,
                               c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                               c_void_p], c_int32),
    "fgs_project_bwd": ([c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_void_p], c_int32),
    "fgs_loss": ([c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                  c_void_p, c_size_t, c_void_p], c_int32),
    "fgs_loss_workspace_size": ([c_void_p, c_int32], c_size_t),
    "fgs_scale_reg": ([c_void_p, c_float, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p], c_int32),
    "fgs_scale_reg_workspace_size": ([c_int64], c_size_t),
    "fgs_adam": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "fgs_prune": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p, c_void_p], c_int32),
    "fgs_prune_workspace_size": ([c_int64], c_size_t),
    "fgs_covisibility": ([c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p], c_int32),
    "fgs_select_keyframes": ([c_void_p, c_void_p, c_void_p, c_int32, c_float, c_float, c_void_p, c_void_p,
                              c_void_p], c_int32),
    "fgs_depth_points": ([c_void_p, c_void_p, ctypes.c_uint8, c_void_p, c_int32, c_void_p, c_int64, c_void_p,
                          c_void_p, c_size_t, c_void_p, c_void_p], c_int32),
    "fgs_depth_points_workspace_size": ([c_int32, c_int32, c_int32], c_size_t),
    "fgs_transform_points": ([c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "fgs_voxel_downsample": ([c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_size_t, c_void_p, c_int64, c_void_p,
                              c_void_p, c_void_p], c_int32),
    "fgs_voxel_workspace_size": ([c_void_p, c_int64], c_size_t),
    "fgs_grid_build": ([c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p],
                       c_int32),
    "fgs_grid_workspace_size": ([c_void_p, c_int64], c_size_t),
    "fgs_point_covariances": ([c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_int32, c_float, c_void_p,
                               c_void_p], c_int32),
    "fgs_gicp": ([c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                  c_void_p, c_void_p, c_void_p, c_size_t, c_void_p], c_int32),
    "fgs_gicp_workspace_size": ([c_int64], c_size_t),
    "fgs_project_bwd_adam": ([c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_float, c_void_p, c_void_p,
                              c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p], c_int32),
    "fgs_project_bwd_adam_workspace_size": ([c_int64], c_size_t),
    "fgs_last_error": ([], ctypes.c_char_p),
    "fgs_version": ([], c_int32),
    "fgs_launch_count": ([], c_int64),
    "fgs_memset_async": ([c_void_p, c_int32, c_size_t, c_void_p], c_int32),
    "fgs_memcpy_async": ([c_void_p, c_void_p, c_size_t, c_void_p], c_int32),
    "fgs_num_sms": ([], c_int32),
    "fgs_peak_probe": ([c_int32, c_int32, c_int64, c_void_p, ctypes.POINTER(c_int64), c_void_p], c_int32),
}
_OPTIONAL = {
    "fgs_fourier_seed": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                          c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p, c_void_p],
                         c_int32),
    "fgs_fourier_seed_workspace_size": ([c_int32, c_int32, c_int32], c_size_t),
    "fgs_fourier_energy": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p], c_int32),
    "fgs_fourier_seed_from_energy": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                      c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                                      c_void_p, c_void_p], c_int32),
    "fgs_prior_features": ([c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_int64, c_void_p, c_void_p], c_int32),
    "fgs_prior_infer": ([c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p], c_int32),
    "fgs_prior_train": ([c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_size_t,
                         c_void_p], c_int32),
    "fgs_prior_train_workspace_size": ([c_int64], c_size_t),
    "fgs_prior_num_params": ([], c_int64),
    "fgs_render_window": ([c_void_p, c_void_p, c_void_p, c_int32, Tiling, c_void_p, c_void_p, c_void_p, c_void_p,
                           c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                           c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p, c_void_p], c_int32),
    "fgs_render_window_workspace_size": ([c_void_p, c_int32], c_size_t),
    "fgs_loss_noalloc": ([c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                          c_void_p, c_void_p], c_int32),
    "fgs_lookback_probe": ([c_int32, c_int32, c_int64, c_void_p, c_size_t, c_void_p, c_void_p, c_void_p], c_int32),
    "fgs_lookback_probe_workspace_size": ([c_int32], c_size_t),
    "fgs_grid_barrier_probe": ([c_int32, c_int32, c_int64, c_void_p, c_size_t, c_void_p, c_void_p, c_void_p],
                               c_int32),
    "fgs_autotune": ([c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_void_p,
                      c_size_t, c_void_p, c_void_p, c_void_p], c_int32),
    "fgs_autotune_workspace_size": ([c_void_p, c_void_p, c_int32, c_int64], c_size_t),
}


def lib():
    """Loads libfgs.so (raises when it is missing: there is no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libfgs.so is not built ({LIB_PATH}); run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                f = getattr(L, name)
                f.argtypes, f.restype = args, res
            for name, (args, res) in _OPTIONAL.items():
                if hasattr(L, name):
                    f = getattr(L, name)
                    f.argtypes, f.restype = args, res
            _lib = L
    return _lib


class FGSError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise FGSError(f"{what} failed with status {rc}: {lib().fgs_last_error().decode()}")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def launch_count() -> int:
    return int(lib().fgs_launch_count())


# ----------------------------------------------------------------------------------
# host structs

def camera_struct(cam: dict) -> Camera:
    c = Camera()
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.fx, c.fy, c.cx, c.cy = float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"])
    w2c = np.asarray(cam["world_to_cam"], np.float32).reshape(-1)
    for k in range(12):
        c.world_to_cam[k] = float(w2c[k])
    c.znear = float(cam.get("znear", 0.2))
    return c


def camera_array(cams: list):
    arr = (Camera * len(cams))()
    for i, cam in enumerate(cams):
        arr[i] = camera_struct(cam)
    return arr


def tiling(tile_w=16, tile_h=16, batch_depth=128) -> Tiling:
    return Tiling(int(tile_w), int(tile_h), int(batch_depth))


def num_tiles(cams: list, til: Tiling) -> int:
    t = lib().fgs_num_tiles(camera_array(cams), len(cams), til)
    if t < 0:
        raise FGSError("bad cameras or tiling")
    return int(t)


# ----------------------------------------------------------------------------------
# device containers

PLANES = {"means": (0, 3), "log_scales": (3, 6), "quats": (6, 10), "logits": (10, 11), "rgb": (11, 14)}


class GaussianMap:
    """Structure-of-arrays Gaussian planes [14][capacity] on one device buffer."""

    def __init__(self, capacity: int, device="cuda", n: int = 0):
        self.capacity = int(capacity)
        self.buf = torch.zeros(14, self.capacity, dtype=torch.float32, device=device)
        self.n = int(n)
        self.d_n = torch.zeros(1, dtype=torch.int64, device=device)

    @classmethod
    def from_scene(cls, scene: dict, capacity: int | None = None, device="cuda") -> "GaussianMap":
        n = scene["means"].shape[-1]
        g = cls(capacity or n, device, n)
        for k, (a, b) in PLANES.items():
            g.buf[a:b, :n] = torch.as_tensor(np.asarray(scene[k], np.float32).reshape(b - a, n), device=device)
        g.d_n.fill_(n)
        return g

    def zeros_like(self) -> "GaussianMap":
        g = GaussianMap(self.capacity, self.buf.device, self.n)
        g.d_n.copy_(self.d_n)
        return g

    def plane(self, name):
        a, b = PLANES[name]
        return self.buf[a:b]

    def struct(self, use_device_count: bool = False, n: int | None = None) -> Gaussians:
        s = Gaussians()
        # with the device count, n is only an upper bound: the whole capacity
        s.n = (self.capacity if use_device_count else self.n) if n is None else int(n)
        s.capacity = self.capacity
        s.d_n = self.d_n.data_ptr() if use_device_count else None
        base = self.buf.data_ptr()
        row = 4 * self.capacity
        s.means, s.log_scales, s.quats = base, base + 3 * row, base + 6 * row
        s.opacity_logits, s.rgb = base + 10 * row, base + 11 * row
        return s

    def to_scene(self, n: int | None = None) -> dict:
        n = self.n if n is None else n
        out = {}
        for k, (a, b) in PLANES.items():
            v = self.buf[a:b, :n].detach().cpu().numpy()
            out[k] = v[0].copy() if b - a == 1 else v.copy()
        return out


class Projection:
    """Per-view splat records of a map: splat [V][stride][8], radius, rect."""

    def __init__(self, n_views: int, stride: int, device="cuda"):
        self.n_views, self.stride = n_views, int(stride)
        self.splat = torch.zeros(n_views, self.stride, 8, dtype=torch.float32, device=device)
        self.radius = torch.zeros(n_views, self.stride, dtype=torch.int32, device=device)
        self.rect = torch.zeros(n_views, self.stride, 4, dtype=torch.int16, device=device)

    def struct(self) -> Projected:
        return Projected(self.stride, self.splat.data_ptr(), self.radius.data_ptr(), self.rect.data_ptr())


def image_sizes(cams: list):
    return [int(c["width"]) * int(c["height"]) for c in cams]


class Frame:
    """Render outputs / upstream gradients of a view set (concatenated per view)."""

    def __init__(self, cams: list, device="cuda"):
        P = sum(image_sizes(cams))
        self.cams = cams
        self.total_pix = P
        self.color = torch.zeros(3 * P, dtype=torch.float32, device=device)
        self.depth = torch.zeros(P, dtype=torch.float32, device=device)
        self.alpha = torch.zeros(P, dtype=torch.float32, device=device)
        self.t_final = torch.zeros(P, dtype=torch.float32, device=device)
        self.n_contrib = torch.zeros(P, dtype=torch.int32, device=device)

    def view(self, v: int) -> dict:
        sizes = image_sizes(self.cams)
        o = sum(sizes[:v])
        H, W = self.cams[v]["height"], self.cams[v]["width"]
        return {"color": self.color[3 * o:3 * o + 3 * H * W].view(3, H, W), "depth": self.depth[o:o + H * W].view(H, W),
                "alpha": self.alpha[o:o + H * W].view(H, W), "t_final": self.t_final[o:o + H * W].view(H, W),
                "n_contrib": self.n_contrib[o:o + H * W].view(H, W)}


def pack_images(cams: list, colors: list, depths: list, device="cuda"):
    """Concatenates per-view colour [3][H][W] and depth [H][W] arrays."""
    c = torch.cat([torch.as_tensor(np.asarray(x, np.float32)).reshape(-1) for x in colors]).to(device)
    d = torch.cat([torch.as_tensor(np.asarray(x, np.float32)).reshape(-1) for x in depths]).to(device)
    return c, d


# ----------------------------------------------------------------------------------
# entry points (same names as the C ABI)

def fgs_project(g: GaussianMap, cams: list, til: Tiling, proj: Projection, status: torch.Tensor | None = None,
                use_device_count: bool = False):
    gs = g.struct(use_device_count)
    ps = proj.struct()
    _check(lib().fgs_project(ctypes.byref(gs), camera_array(cams), len(cams), til, ctypes.byref(ps), _ptr(status),
                             _stream()), "fgs_project")


def fgs_bin_sort_workspace_size(cams: list, til: Tiling, n_records: int, pair_capacity: int) -> int:
    return int(lib().fgs_bin_sort_workspace_size(camera_array(cams), len(cams), til, int(n_records),
                                                 int(pair_capacity)))


def fgs_bin_sort(proj: Projection, n: int, cams: list, til: Tiling, ws: torch.Tensor, tile_keys: torch.Tensor,
                 ids: torch.Tensor, tile_ranges: torch.Tensor, num_pairs: torch.Tensor, status: torch.Tensor | None,
                 d_n: torch.Tensor | None = None):
    """d_n: the map's device live count (int64), bounding the slots binned."""
    ps = proj.struct()
    _check(lib().fgs_bin_sort(ctypes.byref(ps), int(n), _ptr(d_n), camera_array(cams), len(cams), til, _ptr(ws),
                              ws.numel() * ws.element_size(), _ptr(tile_keys), _ptr(ids), ids.numel(),
                              _ptr(tile_ranges), _ptr(num_pairs), _ptr(status), _stream()), "fgs_bin_sort")


def fgs_render_fwd(proj: Projection, g: GaussianMap, cams: list, til: Tiling, ids, tile_ranges, frame: Frame,
                   status=None, tile_order=None):
    ps = proj.struct()
    gs = g.struct()
    _check(lib().fgs_render_fwd(ctypes.byref(ps), ctypes.byref(gs), camera_array(cams), len(cams), til, _ptr(ids),
                                _ptr(tile_ranges), _ptr(tile_order), _ptr(frame.color), _ptr(frame.depth),
                                _ptr(frame.alpha), _ptr(frame.t_final), _ptr(frame.n_contrib), _ptr(status),
                                _stream()), "fgs_render_fwd")


def fgs_render_fwd_sampled(proj: Projection, g: GaussianMap, cams: list, til: Tiling, ids, tile_ranges,
                           frame: Frame, sample_stride: int = 2, status=None, tile_order=None):
    ps = proj.struct()
    gs = g.struct()
    _check(lib().fgs_render_fwd_sampled(ctypes.byref(ps), ctypes.byref(gs), camera_array(cams), len(cams), til,
                                        _ptr(ids), _ptr(tile_ranges), _ptr(tile_order), int(sample_stride),
                                        _ptr(frame.color), _ptr(frame.depth), _ptr(frame.alpha),
                                        _ptr(frame.t_final), _ptr(frame.n_contrib), _ptr(status), _stream()),
           "fgs_render_fwd_sampled")


def fgs_tile_order_workspace_size(cams: list, til: Tiling) -> int:
    return int(lib().fgs_tile_order_workspace_size(camera_array(cams), len(cams), til))


def fgs_tile_order(cams: list, til: Tiling, n_contrib, tile_order, ws):
    """Heaviest-first launch order of the view set's tiles from a render's n_contrib."""
    _check(lib().fgs_tile_order(camera_array(cams), len(cams), til, _ptr(n_contrib), _ptr(tile_order), _ptr(ws),
                                ws.numel() * ws.element_size(), _stream()), "fgs_tile_order")


def fgs_render_bwd(g: GaussianMap, proj: Projection, cams: list, til: Tiling, ids, tile_ranges, frame: Frame,
                   dC, dD, dA, grad2d, grads: GaussianMap, status=None, use_device_count: bool = False,
                   tile_order=None):
    gs = g.struct(use_device_count)
    ps = proj.struct()
    gr = grads.struct(use_device_count)
    _check(lib().fgs_render_bwd(ctypes.byref(gs), ctypes.byref(ps), camera_array(cams), len(cams), til, _ptr(ids),
                                _ptr(tile_ranges), _ptr(tile_order), _ptr(frame.t_final), _ptr(frame.n_contrib),
                                _ptr(dC), _ptr(dD), _ptr(dA), _ptr(grad2d), ctypes.byref(gr), _ptr(status),
                                _stream()), "fgs_render_bwd")


def fgs_render_bwd_splats(g: GaussianMap, proj: Projection, cams: list, til: Tiling, ids, tile_ranges, frame: Frame,
                          dC, dD, dA, grad2d, grads: GaussianMap, status=None, use_device_count: bool = False,
                          tile_order=None):
    gs, ps, gr = g.struct(use_device_count), proj.struct(), grads.struct(use_device_count)
    _check(lib().fgs_render_bwd_splats(ctypes.byref(gs), ctypes.byref(ps), camera_array(cams), len(cams), til,
                                       _ptr(ids), _ptr(tile_ranges), _ptr(tile_order), _ptr(frame.t_final),
                                       _ptr(frame.n_contrib), _ptr(dC), _ptr(dD), _ptr(dA), _ptr(grad2d),
                                       ctypes.byref(gr), _ptr(status), _stream()), "fgs_render_bwd_splats")


def fgs_project_bwd(g: GaussianMap, proj: Projection, cams: list, grad2d, grads: GaussianMap,
                    use_device_count: bool = False):
    gs, ps, gr = g.struct(use_device_count), proj.struct(), grads.struct(use_device_count)
    _check(lib().fgs_project_bwd(ctypes.byref(gs), ctypes.byref(ps), camera_array(cams), len(cams), _ptr(grad2d),
                                 ctypes.byref(gr), _stream()), "fgs_project_bwd")


def fgs_loss_workspace_size(cams: list) -> int:
    return int(lib().fgs_loss_workspace_size(camera_array(cams), len(cams)))


def fgs_loss(cams: list, color, depth, color_gt, depth_gt, w_c, w_d, w_s, dC, dD, loss_acc, ws):
    p = LossParams(float(w_c), float(w_d), float(w_s))
    _check(lib().fgs_loss(camera_array(cams), len(cams), _ptr(color), _ptr(depth), _ptr(color_gt), _ptr(depth_gt),
                          ctypes.byref(p), _ptr(dC), _ptr(dD), _ptr(loss_acc), _ptr(ws),
                          ws.numel() * ws.element_size(), _stream()), "fgs_loss")


def fgs_loss_noalloc(cams: list, color, depth, color_gt, depth_gt, w_c, w_d, w_s, dC, dD, loss_acc):
    """fgs_loss with its scratch in a fixed array inside the library (no workspace)."""
    p = LossParams(float(w_c), float(w_d), float(w_s))
    _check(lib().fgs_loss_noalloc(camera_array(cams), len(cams), _ptr(color), _ptr(depth), _ptr(color_gt),
                                  _ptr(depth_gt), ctypes.byref(p), _ptr(dC), _ptr(dD), _ptr(loss_acc), _stream()),
           "fgs_loss_noalloc")


def fgs_lookback_probe(n_tiles: int, skip_first: bool, timeout_ns: int, ws, sums, status):
    _check(lib().fgs_lookback_probe(int(n_tiles), 1 if skip_first else 0, int(timeout_ns), _ptr(ws),
                                    ws.numel() * ws.element_size(), _ptr(sums), _ptr(status), _stream()),
           "fgs_lookback_probe")


def fgs_lookback_probe_workspace_size(n_tiles: int) -> int:
    return int(lib().fgs_lookback_probe_workspace_size(int(n_tiles)))


def fgs_grid_barrier_probe(n_blocks: int, n_expected: int, timeout_ns: int, ws, passed, status):
    """Self-test of the window's bounded grid barrier (see include/fgs.h)."""
    _check(lib().fgs_grid_barrier_probe(int(n_blocks), int(n_expected), int(timeout_ns), _ptr(ws),
                                        ws.numel() * ws.element_size(), _ptr(passed), _ptr(status), _stream()),
           "fgs_grid_barrier_probe")


def fgs_scale_reg_workspace_size(n: int) -> int:
    return int(lib().fgs_scale_reg_workspace_size(int(n)))


def fgs_scale_reg(g: GaussianMap, weight: float, grads: GaussianMap, loss_acc, ws, use_device_count=False):
    gs, gr = g.struct(use_device_count), grads.struct(use_device_count)
    _check(lib().fgs_scale_reg(ctypes.byref(gs), float(weight), ctypes.byref(gr), _ptr(loss_acc), _ptr(ws),
                               ws.numel() * ws.element_size(), _stream()), "fgs_scale_reg")


DEFAULT_LR = (1e-3, 5e-3, 1e-3, 5e-2, 2.5e-3)


def fgs_adam(g: GaussianMap, grads: GaussianMap, m: GaussianMap, v: GaussianMap, lr=DEFAULT_LR, beta1=0.9,
             beta2=0.999, eps=1e-15, step: int = 1, d_step=None, use_device_count=False):
    hp = AdamParams()
    for k in range(5):
        hp.lr[k] = float(lr[k])
    hp.beta1, hp.beta2, hp.eps, hp.step = beta1, beta2, eps, int(step)
    gs, gr, ms, vs = (x.struct(use_device_count) for x in (g, grads, m, v))
    _check(lib().fgs_adam(ctypes.byref(gs), ctypes.byref(gr), ctypes.byref(ms), ctypes.byref(vs), ctypes.byref(hp),
                          _ptr(d_step), _stream()), "fgs_adam")


def prune_params(min_opacity: float = 0.005, max_scale: float = 0.5) -> PruneParams:
    """Thresholds in the decision domain: opacity below min_opacity <=> logit below
    logit(min_opacity); a scale above max_scale <=> a log-scale above log(max_scale)
    (both rounded once to float32, the precision of the parameters)."""
    p = float(np.float32(min_opacity))
    return PruneParams(float(np.float32(math.log(p / (1.0 - p)))), float(np.float32(math.log(max_scale))))


def fgs_prune_workspace_size(capacity: int) -> int:
    return int(lib().fgs_prune_workspace_size(int(capacity)))


def fgs_prune(g: GaussianMap, m: GaussianMap | None, v: GaussianMap | None, params: PruneParams, ws: torch.Tensor,
              num_kept: torch.Tensor, use_device_count: bool = False):
    gs = g.struct(use_device_count)
    ms = m.struct(use_device_count) if m is not None else None
    vs = v.struct(use_device_count) if v is not None else None
    _check(lib().fgs_prune(ctypes.byref(gs), ctypes.byref(ms) if ms is not None else None,
                           ctypes.byref(vs) if vs is not None else None, ctypes.byref(params), _ptr(ws),
                           ws.numel() * ws.element_size(), _ptr(num_kept), _stream()), "fgs_prune")


def fgs_covisibility(depth: torch.Tensor, cam: dict, keyframes: list, step: int, inside: torch.Tensor,
                     valid: torch.Tensor):
    _check(lib().fgs_covisibility(_ptr(depth), camera_array([cam]), camera_array(keyframes), len(keyframes),
                                  int(step), _ptr(inside), _ptr(valid), _stream()), "fgs_covisibility")


def fgs_select_keyframes(inside: torch.Tensor, valid: torch.Tensor, u: torch.Tensor, threshold: float, frac: float,
                         kind: torch.Tensor, count: torch.Tensor):
    _check(lib().fgs_select_keyframes(_ptr(inside), _ptr(valid), _ptr(u), inside.numel(), float(threshold),
                                      float(frac), _ptr(kind), _ptr(count), _stream()), "fgs_select_keyframes")


def fgs_depth_points(depth: torch.Tensor, mask: torch.Tensor | None, mask_bits: int, cam: dict, step: int,
                     xyz: torch.Tensor, n: torch.Tensor, ws: torch.Tensor, status: torch.Tensor | None = None):
    _check(lib().fgs_depth_points(_ptr(depth), _ptr(mask), int(mask_bits), camera_array([cam]), int(step), _ptr(xyz),
                                  xyz.shape[0], _ptr(n), _ptr(ws), ws.numel() * ws.element_size(), _ptr(status),
                                  _stream()), "fgs_depth_points")


def fgs_depth_points_workspace_size(width: int, height: int, step: int) -> int:
    return int(lib().fgs_depth_points_workspace_size(int(width), int(height), int(step)))


def fgs_transform_points(xyz_in, cov_in, n: torch.Tensor, pose: torch.Tensor, xyz_out, cov_out=None):
    _check(lib().fgs_transform_points(_ptr(xyz_in), _ptr(cov_in), _ptr(n), xyz_in.shape[0], _ptr(pose), _ptr(xyz_out),
                                      _ptr(cov_out), _stream()), "fgs_transform_points")


def fgs_voxel_workspace_size(g: Grid, n_max: int) -> int:
    return int(lib().fgs_voxel_workspace_size(ctypes.byref(g), int(n_max)))


def fgs_voxel_downsample(xyz, n: torch.Tensor, g: Grid, ws, out_xyz, n_out: torch.Tensor, status=None):
    _check(lib().fgs_voxel_downsample(_ptr(xyz), _ptr(n), xyz.shape[0], ctypes.byref(g), _ptr(ws),
                                      ws.numel() * ws.element_size(), _ptr(out_xyz), out_xyz.shape[0], _ptr(n_out),
                                      _ptr(status), _stream()), "fgs_voxel_downsample")


def fgs_grid_workspace_size(g: Grid, n_max: int) -> int:
    return int(lib().fgs_grid_workspace_size(ctypes.byref(g), int(n_max)))


def fgs_grid_build(xyz, n: torch.Tensor, g: Grid, cell_start, order, ws):
    _check(lib().fgs_grid_build(_ptr(xyz), _ptr(n), xyz.shape[0], ctypes.byref(g), _ptr(cell_start), _ptr(order),
                                _ptr(ws), ws.numel() * ws.element_size(), _stream()), "fgs_grid_build")


def fgs_point_covariances(xyz, n: torch.Tensor, g: Grid, cell_start, order, k: int, eps: float, cov):
    _check(lib().fgs_point_covariances(_ptr(xyz), _ptr(n), xyz.shape[0], ctypes.byref(g), _ptr(cell_start),
                                       _ptr(order), int(k), float(eps), _ptr(cov), _stream()), "fgs_point_covariances")


def fgs_gicp_workspace_size(n_src_max: int) -> int:
    return int(lib().fgs_gicp_workspace_size(int(n_src_max)))


def fgs_gicp(src, src_cov, n_src: torch.Tensor, tgt, tgt_cov, g: Grid, cell_start, order, params: GicpParams,
             pose: torch.Tensor, stats: torch.Tensor, ws):
    _check(lib().fgs_gicp(_ptr(src), _ptr(src_cov), _ptr(n_src), src.shape[0], _ptr(tgt), _ptr(tgt_cov),
                          ctypes.byref(g), _ptr(cell_start), _ptr(order), ctypes.byref(params), _ptr(pose),
                          _ptr(stats), _ptr(ws), ws.numel() * ws.element_size(), _stream()), "fgs_gicp")


def fgs_project_bwd_adam_workspace_size(n: int) -> int:
    return int(lib().fgs_project_bwd_adam_workspace_size(int(n)))


def fgs_project_bwd_adam(g: GaussianMap, proj: Projection, cams: list, grad2d, grads: GaussianMap, reg_weight: float,
                         d_loss, m: GaussianMap, v: GaussianMap, lr=DEFAULT_LR, beta1=0.9, beta2=0.999, eps=1e-15,
                         step: int = 1, d_step=None, ws=None, use_device_count=False):
    hp = AdamParams()
    for k in range(5):
        hp.lr[k] = float(lr[k])
    hp.beta1, hp.beta2, hp.eps, hp.step = beta1, beta2, eps, int(step)
    gs, gr, ms, vs = (x.struct(use_device_count) for x in (g, grads, m, v))
    ps = proj.struct()
    _check(lib().fgs_project_bwd_adam(ctypes.byref(gs), ctypes.byref(ps), camera_array(cams), len(cams), _ptr(grad2d),
                                      ctypes.byref(gr), float(reg_weight), _ptr(d_loss), ctypes.byref(ms),
                                      ctypes.byref(vs), ctypes.byref(hp), _ptr(d_step), _ptr(ws),
                                      ws.numel() * ws.element_size(), _stream()), "fgs_project_bwd_adam")


def fgs_memset_async(t: torch.Tensor, value: int = 0):
    _check(lib().fgs_memset_async(_ptr(t), int(value), t.numel() * t.element_size(), _stream()), "fgs_memset_async")


def fgs_memcpy_async(dst: torch.Tensor, src: torch.Tensor):
    n = min(dst.numel() * dst.element_size(), src.numel() * src.element_size())
    _check(lib().fgs_memcpy_async(_ptr(dst), _ptr(src), n, _stream()), "fgs_memcpy_async")


FGS_PEAK_FFMA, FGS_PEAK_EX2, FGS_PEAK_LDS = 0, 1, 2


def fgs_num_sms() -> int:
    return int(lib().fgs_num_sms())


def fgs_peak_probe(kind: int, blocks_per_sm: int, iters: int, sink: torch.Tensor) -> int:
    """Launches one peak microbenchmark on the current stream; returns its operation count."""
    ops = c_int64(0)
    _check(lib().fgs_peak_probe(int(kind), int(blocks_per_sm), int(iters), _ptr(sink), ctypes.byref(ops), _stream()),
           "fgs_peak_probe")
    return int(ops.value)


def measure_peaks(target_ms: float = 20.0, reps: int = 3) -> dict:
    """Measured on-chip rates of the current device: FP32 FMA (TFLOP/s), MUFU ex2
    (G evaluations/s) and shared-memory loads (TB/s), each the best of `reps`
    launches timed with CUDA events and sized to about target_ms."""
    sink = torch.zeros(fgs_num_sms() * 32, dtype=torch.float32, device="cuda")
    out = {"sms": fgs_num_sms()}
    names = {FGS_PEAK_FFMA: ("fp32_fma_tflops", 1e12), FGS_PEAK_EX2: ("mufu_ex2_gops", 1e9),
             FGS_PEAK_LDS: ("smem_load_tbs", 1e12)}
    for kind, (name, unit) in names.items():
        iters, best = 1024, 0.0
        for _ in range(12):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            rates = []
            for _ in range(reps):
                e0.record()
                ops = fgs_peak_probe(kind, 8, iters, sink)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                rates.append(ops / (ms / 1e3))
            best = max(rates)
            if ms >= target_ms or iters >= (1 << 31):
                break
            iters = min(1 << 31, int(iters * max(2.0, target_ms / max(ms, 1e-3))))
        out[name] = best / unit
    return out


def ws_tensor(nbytes: int, device="cuda") -> torch.Tensor:
    """Workspace of at least nbytes, 256-byte aligned (torch allocations are)."""
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# ----------------------------------------------------------------------------------
# Fourier seeding and the learned prior

def seed_params(d0=0.25, m=2, n=8, alpha_h=1.0, alpha_l=4.0, tau_alpha=0.5, tau_depth_rel=0.05, tau_color=0.1,
                max_new=50000, init_logit=0.0, prior_max_dev=math.log(4.0)) -> SeedParams:
    """Defaults are the readings of Sec. III-A's unstated constants (see the header)."""
    return SeedParams(float(d0), int(m), int(n), float(alpha_h), float(alpha_l), float(tau_alpha),
                      float(tau_depth_rel), float(tau_color), int(max_new), float(init_logit), float(prior_max_dev))


def fgs_fourier_seed_workspace_size(width: int, height: int, max_new: int) -> int:
    return int(lib().fgs_fourier_seed_workspace_size(int(width), int(height), int(max_new)))


def fgs_fourier_seed(rgb_gt, depth_gt, r_color, r_depth, r_alpha, cam: dict, params: SeedParams, prior, mask,
                     energy, g: GaussianMap, num_new, threshold, ws, status=None, use_device_count: bool = True,
                     seed_xy=None, from_energy: bool = False):
    """fgs_fourier_seed, or with from_energy its second half
    (fgs_fourier_seed_from_energy) after an fgs_fourier_energy call on `ws`."""
    gs = g.struct(use_device_count)
    cs = camera_struct(cam)
    name = "fgs_fourier_seed_from_energy" if from_energy else "fgs_fourier_seed"
    _check(getattr(lib(), name)(_ptr(rgb_gt), _ptr(depth_gt), _ptr(r_color), _ptr(r_depth), _ptr(r_alpha),
                                ctypes.byref(cs), ctypes.byref(params),
                                None if prior is None else ctypes.byref(prior), _ptr(mask), _ptr(energy),
                                ctypes.byref(gs), _ptr(num_new), _ptr(threshold), _ptr(seed_xy), _ptr(ws),
                                ws.numel() * ws.element_size(), _ptr(status), _stream()), name)


def fgs_fourier_energy(rgb_gt, cam: dict, params: SeedParams, energy, threshold, ws):
    cs = camera_struct(cam)
    _check(lib().fgs_fourier_energy(_ptr(rgb_gt), ctypes.byref(cs), ctypes.byref(params), _ptr(energy),
                                    _ptr(threshold), _ptr(ws), ws.numel() * ws.element_size(), _stream()),
           "fgs_fourier_energy")


def fgs_prior_features(rgb, depth, width: int, height: int, seed_xy, n: int, features):
    _check(lib().fgs_prior_features(_ptr(rgb), _ptr(depth), int(width), int(height), _ptr(seed_xy), int(n),
                                    _ptr(features), _stream()), "fgs_prior_features")


def fgs_prior_infer(mlp: MLP, features, n: int, out, status=None):
    _check(lib().fgs_prior_infer(ctypes.byref(mlp), _ptr(features), int(n), _ptr(out), _ptr(status), _stream()),
           "fgs_prior_infer")


def fgs_prior_train(mlp: MLP, master: MLPMaster, features, targets, n: int, hp: TrainParams, loss_acc, ws):
    _check(lib().fgs_prior_train(ctypes.byref(mlp), ctypes.byref(master), _ptr(features), _ptr(targets), int(n),
                                 ctypes.byref(hp), _ptr(loss_acc), _ptr(ws), ws.numel() * ws.element_size(),
                                 _stream()), "fgs_prior_train")


def fgs_prior_train_workspace_size(n: int) -> int:
    return int(lib().fgs_prior_train_workspace_size(int(n)))


def fgs_prior_num_params() -> int:
    return int(lib().fgs_prior_num_params())


# ----------------------------------------------------------------------------------
# persistent keyframe window

def fgs_render_window_workspace_size(cams: list) -> int:
    return int(lib().fgs_render_window_workspace_size(camera_array(cams), len(cams)))


def fgs_render_window(g: GaussianMap, proj: Projection, cams: list, til: Tiling, ids, tile_ranges, color_gt, depth_gt,
                      w_c, w_d, w_s, frame: Frame, dC, dD, grad2d, grads: GaussianMap, loss_acc, ws, status,
                      use_device_count: bool = True, tile_order=None):
    gs, ps, gr = g.struct(use_device_count), proj.struct(), grads.struct(use_device_count)
    lp = LossParams(float(w_c), float(w_d), float(w_s))
    _check(lib().fgs_render_window(ctypes.byref(gs), ctypes.byref(ps), camera_array(cams), len(cams), til, _ptr(ids),
                                   _ptr(tile_ranges), _ptr(tile_order), _ptr(color_gt), _ptr(depth_gt), ctypes.byref(lp),
                                   _ptr(frame.color), _ptr(frame.depth), _ptr(frame.alpha), _ptr(frame.t_final),
                                   _ptr(frame.n_contrib), _ptr(dC), _ptr(dD), _ptr(grad2d), ctypes.byref(gr),
                                   _ptr(loss_acc), _ptr(ws), ws.numel() * ws.element_size(), _ptr(status),
                                   _stream()), "fgs_render_window")


AUTOTUNE_CONFIGS = 12
AUTOTUNE_ORDER = [((tw, th), bd) for (tw, th) in ((8, 8), (16, 16), (16, 32)) for bd in (32, 64, 128, 256)]


def fgs_autotune_workspace_size(g: GaussianMap, cams: list, pair_capacity: int, use_device_count: bool = True) -> int:
    gs = g.struct(use_device_count)
    return int(lib().fgs_autotune_workspace_size(ctypes.byref(gs), camera_array(cams), len(cams),
                                                 int(pair_capacity)))


def fgs_autotune(g: GaussianMap, cams: list, color_gt, depth_gt, w_c, w_d, w_s, pair_capacity: int, reps: int, ws,
                 use_device_count: bool = True):
    """Returns (best Tiling, [ms per tiling in AUTOTUNE_ORDER]); synchronises the stream."""
    gs = g.struct(use_device_count)
    lp = LossParams(float(w_c), float(w_d), float(w_s))
    best = Tiling()
    ms = (c_float * AUTOTUNE_CONFIGS)()
    _check(lib().fgs_autotune(ctypes.byref(gs), camera_array(cams), len(cams), _ptr(color_gt), _ptr(depth_gt),
                              ctypes.byref(lp), int(pair_capacity), int(reps), _ptr(ws), ws.numel() * ws.element_size(),
                              ctypes.byref(best), ms, _stream()), "fgs_autotune")
    return best, [float(x) for x in ms]
