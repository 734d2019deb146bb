"""FP64 oracle of the Fourier seeding of Sec. III-A (test infrastructure only).

Follows the paper's steps in its order and notation, with plain numpy:

1. gray frame I(x, y) (BT.601 luma of the RGB frame; the paper says only
   "image frame I(x,y)");
2. eq2, the W x H DFT, as products with explicit DFT matrices;
3. eq3, centring, read as the standard shift of the spectrum that puts the zero
   frequency at (W//2, H//2) (eq3 literally multiplies F by (-1)^(u+v), which
   shifts the image, not the spectrum);
4. eq5 / eq7, the Gaussian high-pass H = 1 - exp(-D^2 / (2 D0^2)) with D measured
   from the centre in Nyquist units (D = 1 at the Nyquist frequency on each axis);
5. eq8, the inverse DFT of the un-centred filtered spectrum, divided by H W (the
   printed eq8 sums over x, y with swapped limits; read as the standard inverse);
6. E = |I_h| and its 256-bin histogram over [0, max E] (a frame whose max E is
   at most 1e-5 of its peak gray has no high-frequency region: E is 0 in exact
   arithmetic and only rounding noise otherwise);
7. the triangle threshold between the histogram's peak and its far end;
8. M_h = bin > t, M_l = not M_h; eq9's missing region; eq10's intersections;
   equidistant sampling with spacings m < n; eq11's radius r = alpha d / f.

Where float32 decides an integer (a histogram bin, a mask bit), the
``*_f32`` helpers take that decision in float32 with the operation order the
kernels use, so both sides agree bit for bit on the same float32 inputs.
"""
from __future__ import annotations

import math

import numpy as np


def gray(rgb: np.ndarray) -> np.ndarray:
    """BT.601 luma of an RGB frame [3][H][W] in [0, 1] (reading of "I(x, y)")."""
    rgb = np.asarray(rgb, np.float64)
    return 0.299 * rgb[0] + 0.587 * rgb[1] + 0.114 * rgb[2]


def dft_matrix(N: int, inverse: bool = False) -> np.ndarray:
    """W[k, n] = exp(-+ j 2 pi k n / N), phase reduced exactly (k n mod N)."""
    k = np.arange(N)
    ph = (np.outer(k, k) % N).astype(np.float64) / N
    sign = 1.0 if inverse else -1.0
    return np.exp(sign * 2j * math.pi * ph)


def dft2(img: np.ndarray) -> np.ndarray:
    """eq2: F(u, v) = sum_x sum_y I(x, y) exp(-j 2 pi (u x / W + v y / H)).
    Array index [v, u] (row = vertical frequency)."""
    H, W = img.shape
    return dft_matrix(H) @ np.asarray(img, np.complex128) @ dft_matrix(W).T


def idft2(F: np.ndarray) -> np.ndarray:
    """eq8 read as the standard inverse: (1/(H W)) sum_u sum_v F(u,v) exp(+j 2 pi (u x/W + v y/H))."""
    H, W = F.shape
    return dft_matrix(H, True) @ F @ dft_matrix(W, True).T / (H * W)


def centre(F: np.ndarray) -> np.ndarray:
    """eq3 (reading): zero frequency moved to index (H//2, W//2)."""
    H, W = F.shape
    v = (np.arange(H) - H // 2) % H
    u = (np.arange(W) - W // 2) % W
    return F[np.ix_(v, u)]


def uncentre(Fc: np.ndarray) -> np.ndarray:
    """Inverse of :func:`centre`."""
    H, W = Fc.shape
    v = (np.arange(H) + H // 2) % H
    u = (np.arange(W) + W // 2) % W
    return Fc[np.ix_(v, u)]


def highpass(W: int, H: int, d0: float) -> np.ndarray:
    """eq5 on the centred grid: H(u, v) = 1 - exp(-D^2 / (2 D0^2)),
    D^2 = ((u - W//2) / (W/2))^2 + ((v - H//2) / (H/2))^2."""
    du = (np.arange(W) - W // 2) / (W / 2.0)
    dv = (np.arange(H) - H // 2) / (H / 2.0)
    D2 = dv[:, None] ** 2 + du[None, :] ** 2
    return 1.0 - np.exp(-D2 / (2.0 * d0 * d0))


def high_frequency_energy(rgb: np.ndarray, d0: float = 0.25) -> np.ndarray:
    """Steps 1-6: E(x, y) = |I_h(x, y)| of the high-pass filtered frame."""
    I = gray(rgb)
    H, W = I.shape
    F = dft2(I)                       # eq2
    Fc = centre(F)                    # eq3
    Fh = Fc * highpass(W, H, d0)      # eq5, eq7
    Ih = idft2(uncentre(Fh))          # eq8
    return np.abs(Ih)


NOISE_FLOOR = 1e-5   # max E at or below this fraction of the peak gray is rounding noise


def bins_f32(E32: np.ndarray, gray_max32=None) -> np.ndarray:
    """Histogram bin of each pixel, decided in float32:
    bin = min(255, floor((256 * e) / max E)); all zero when max E is not above
    NOISE_FLOOR * max |gray| (a frame without high-frequency content: in exact
    arithmetic E is then 0, any float rounding leaves only noise)."""
    E32 = np.asarray(E32, np.float32)
    mx = np.float32(E32.max()) if E32.size else np.float32(0)
    floor = np.float32(0) if gray_max32 is None else np.float32(NOISE_FLOOR) * np.float32(gray_max32)
    if not mx > floor:
        return np.zeros(E32.shape, np.int32)
    q = (np.float32(256.0) * E32) / mx          # both float32, IEEE round to nearest
    return np.minimum(np.floor(q), 255).astype(np.int32)


def bins_f64(E: np.ndarray, gray_max=None) -> np.ndarray:
    E = np.asarray(E, np.float64)
    mx = E.max()
    floor = 0.0 if gray_max is None else NOISE_FLOOR * gray_max
    if not mx > floor:
        return np.zeros(E.shape, np.int32)
    return np.minimum(np.floor(256.0 * E / mx), 255).astype(np.int32)


def histogram(bins: np.ndarray) -> np.ndarray:
    return np.bincount(np.asarray(bins).ravel(), minlength=256).astype(np.int64)


def triangle_threshold(hist) -> int:
    """Triangle method (Zack et al., 1977) as the paper describes it: a line from
    the histogram's highest peak to its far end, threshold at the bin farthest
    from that line.

    Readings: peak p = first argmax; the far end e is the last non-empty bin on
    the side of p with more bins (ties: the high side); the distance of (i, h_i)
    to the line is proportional to |(e - p)(h_i - h_p) - (i - p)(h_e - h_p)|,
    compared as exact integers; t = the first bin from p towards e with the
    largest distance.  Pixels with bin > t are high frequency."""
    h = [int(x) for x in hist]
    nz = [i for i, c in enumerate(h) if c > 0]
    if not nz:
        return 255
    p = max(range(len(h)), key=lambda i: (h[i], -i))
    lo, hi = nz[0], nz[-1]
    e = hi if (hi - p) >= (p - lo) else lo
    if e == p:
        return p
    step = 1 if e > p else -1
    best_t, best_d = p, -1
    for i in range(p, e + step, step):
        d = abs((e - p) * (h[i] - h[p]) - (i - p) * (h[e] - h[p]))
        if d > best_d:
            best_d, best_t = d, i
    return best_t


def missing_mask_f32(r_color, r_depth, r_alpha, color_gt, depth_gt, tau_alpha=0.5, tau_depth_rel=0.05,
                     tau_color=0.1) -> np.ndarray:
    """eq9, M_m = M_i | M_d | M_c, decided in float32:
    M_i: A < tau_alpha (opacity render of eq1 below the threshold);
    M_d: D_gt > 0, A > 0 and (D / A) - D_gt > tau_depth_rel * D_gt (the map's
         depth lies abnormally far behind the frame's: a foreground object);
    M_c: (|dR| + |dG|) + |dB| > 3 tau_color (significant colour difference)."""
    f = np.float32
    A = np.asarray(r_alpha, f)
    D = np.asarray(r_depth, f)
    C = np.asarray(r_color, f)
    Cg = np.asarray(color_gt, f)
    Dg = np.asarray(depth_gt, f)
    Mi = A < f(tau_alpha)
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.where(A > 0, D / np.where(A > 0, A, f(1)), f(0)).astype(f)
    diff = (q - Dg).astype(f)
    thr = (f(tau_depth_rel) * Dg).astype(f)
    Md = (Dg > 0) & (A > 0) & (diff > thr)
    s = ((np.abs(C[0] - Cg[0]) + np.abs(C[1] - Cg[1])).astype(f) + np.abs(C[2] - Cg[2])).astype(f)
    Mc = s > (f(3.0) * f(tau_color))
    return Mi | Md | Mc


def select_seeds(Mh: np.ndarray, Mm: np.ndarray, depth_gt: np.ndarray, m: int = 2, n: int = 8,
                 max_new: int = 50000):
    """eq10 and the equidistant sampling: high-frequency seeds (M_h & M_m) on the
    m-grid, then low-frequency seeds (M_l & M_m) on the n-grid, valid depth only,
    each in row-major order, truncated to max_new.  Returns (xy[k][2], is_high[k])."""
    H, W = Mh.shape
    ys, xs = np.mgrid[0:H, 0:W]
    valid = np.asarray(depth_gt) > 0
    hi = Mh & Mm & valid & (xs % m == 0) & (ys % m == 0)
    lo = (~Mh) & Mm & valid & (xs % n == 0) & (ys % n == 0)
    hy, hx = np.nonzero(hi)
    ly, lx = np.nonzero(lo)
    xy = np.concatenate([np.stack([hx, hy], 1), np.stack([lx, ly], 1)]).astype(np.int32)
    is_high = np.concatenate([np.ones(hx.size, bool), np.zeros(lx.size, bool)])
    return xy[:max_new], is_high[:max_new]


def new_gaussians(xy: np.ndarray, is_high: np.ndarray, rgb_gt: np.ndarray, depth_gt: np.ndarray, cam: dict,
                  alpha_h: float = 1.0, alpha_l: float = 4.0, init_logit: float = 0.0) -> dict:
    """eq11: back-project each seed pixel with the frame's depth d and give it the
    radius r = alpha_{h|l} d / f (f = (fx + fy)/2) on every axis as log-scale,
    identity rotation, the frame's colour and opacity logit init_logit."""
    x = xy[:, 0].astype(np.float64)
    y = xy[:, 1].astype(np.float64)
    d = np.asarray(depth_gt, np.float64)[xy[:, 1], xy[:, 0]]
    pc = np.stack([(x - cam["cx"]) * d / cam["fx"], (y - cam["cy"]) * d / cam["fy"], d])
    w2c = np.asarray(cam["world_to_cam"], np.float64).reshape(3, 4)
    pw = np.linalg.solve(w2c[:, :3], pc - w2c[:, 3:4])   # inverse of the world-to-camera map
    f = 0.5 * (cam["fx"] + cam["fy"])
    alpha = np.where(is_high, alpha_h, alpha_l)
    ls = np.log(alpha * d / f)
    k = xy.shape[0]
    rgb = np.asarray(rgb_gt, np.float64)[:, xy[:, 1], xy[:, 0]]
    return {"means": pw, "log_scales": np.stack([ls, ls, ls]),
            "quats": np.concatenate([np.ones((1, k)), np.zeros((3, k))]),
            "logits": np.full(k, init_logit), "rgb": rgb}


def seed_frame(rgb_gt, depth_gt, cam, r_color=None, r_depth=None, r_alpha=None, d0=0.25, m=2, n=8,
               alpha_h=1.0, alpha_l=4.0, tau_alpha=0.5, tau_depth_rel=0.05, tau_color=0.1, max_new=50000,
               init_logit=0.0, energy32=None) -> dict:
    """Sec. III-A end to end for one frame.  With energy32 given (teacher
    forcing), the histogram, threshold and masks start from that float32 E."""
    E = high_frequency_energy(rgb_gt, d0)
    gmax = float(np.abs(gray(rgb_gt)).max())
    if energy32 is not None:
        r = np.asarray(rgb_gt, np.float32)
        g32 = (np.float32(0.299) * r[0] + np.float32(0.587) * r[1] + np.float32(0.114) * r[2]).astype(np.float32)
        bins = bins_f32(energy32, np.abs(g32).max())
    else:
        bins = bins_f64(E, gmax)
    hist = histogram(bins)
    t = triangle_threshold(hist)
    Mh = bins > t
    H, W = Mh.shape
    if r_alpha is None:
        Mm = np.ones((H, W), bool)
    else:
        Mm = missing_mask_f32(r_color, r_depth, r_alpha, rgb_gt, depth_gt, tau_alpha, tau_depth_rel, tau_color)
    xy, is_high = select_seeds(Mh, Mm, depth_gt, m, n, max_new)
    g = new_gaussians(xy, is_high, rgb_gt, depth_gt, cam, alpha_h, alpha_l, init_logit)
    mask = (Mh.astype(np.uint8) | ((~Mh).astype(np.uint8) << 1) | (Mm.astype(np.uint8) << 2))
    seeded = np.zeros((H, W), bool)
    seeded[xy[:, 1], xy[:, 0]] = True
    mask |= seeded.astype(np.uint8) << 3
    return {"E": E, "bins": bins, "hist": hist, "threshold": t, "mask": mask, "xy": xy, "is_high": is_high,
            "gaussians": g}
