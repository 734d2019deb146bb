"""The C-ABI library loads without a GPU and exports every entry point that
include/fgs.h declares; the host-side argument checks answer without launching."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fgs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(fgs_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_01109_gb300 import build
    build.build()
    return ctypes.CDLL(build.OUT)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_string(lib):
    lib.fgs_version.restype = ctypes.c_int32
    assert lib.fgs_version() == 100
    lib.fgs_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.fgs_last_error(), bytes)


def test_host_checks_need_no_gpu(lib):
    from paper_2503_01109_gb300 import fgs, synthetic as syn
    L = fgs.lib()
    cams = fgs.camera_array([syn.pinhole(64, 48, 60.0)])
    assert L.fgs_num_tiles(cams, 1, fgs.tiling(16, 16, 128)) == 12
    assert L.fgs_num_tiles(cams, 1, fgs.tiling(16, 32, 64)) == 8
    assert L.fgs_num_tiles(cams, 1, fgs.tiling(12, 12, 64)) == -1
    assert L.fgs_num_tiles(cams, 0, fgs.tiling(16, 16, 64)) == -1
    assert L.fgs_bin_sort_workspace_size(cams, 1, fgs.tiling(16, 16, 128), 1000, 5000) > 0
    assert L.fgs_bin_sort_workspace_size(cams, 1, fgs.tiling(12, 12, 128), 1000, 5000) == 0
    # an argument error returns before any CUDA call
    g = fgs.Gaussians()
    g.n, g.capacity = 5, 2
    rc = L.fgs_project(ctypes.byref(g), cams, 1, fgs.tiling(16, 16, 128), None, None, None)
    assert rc == 1 and b"capacity" in L.fgs_last_error()


def test_barrier_probe_argument_checks(lib):
    """fgs_grid_barrier_probe refuses unusable grids before any CUDA call."""
    from paper_2503_01109_gb300 import fgs
    L = fgs.lib()
    ws = ctypes.create_string_buffer(64)
    word = ctypes.c_int32(0)
    ok_ptr = ctypes.cast(ws, ctypes.c_void_p)
    p = ctypes.cast(ctypes.byref(word), ctypes.c_void_p)
    for n_blocks, n_expected, timeout_ns in ((0, 1, 10**6), (8, 7, 10**6), (4, 4, 10), (4, 4, 6 * 10**9),
                                             (100000, 100000, 10**6)):
        rc = L.fgs_grid_barrier_probe(n_blocks, n_expected, timeout_ns, ok_ptr, 64, p, p, None)
        assert rc == 1, (n_blocks, n_expected, timeout_ns)
    rc = L.fgs_grid_barrier_probe(4, 4, 10**6, None, 64, p, p, None)
    assert rc == 1 and b"NULL" in L.fgs_last_error()


def test_lookback_probe_argument_checks(lib):
    """fgs_lookback_probe refuses bad tile counts, limits, NULLs and small
    workspaces before any CUDA call."""
    from paper_2503_01109_gb300 import fgs
    L = fgs.lib()
    assert L.fgs_lookback_probe_workspace_size(0) == 0
    need = L.fgs_lookback_probe_workspace_size(10)
    assert need >= 10 * 256 * 4
    word = ctypes.c_int32(0)
    p = ctypes.cast(ctypes.byref(word), ctypes.c_void_p)
    fake_ws = ctypes.c_void_p(1 << 20)  # never dereferenced: every case fails its checks first
    for n, timeout_ns, ws_bytes in ((0, 10**6, need), (5000, 10**6, need), (10, 10, need), (10, 6 * 10**9, need),
                                    (10, 10**6, need - 1)):
        rc = L.fgs_lookback_probe(n, 0, timeout_ns, fake_ws, ws_bytes, p, p, None)
        assert rc == 1, (n, timeout_ns, ws_bytes)
    rc = L.fgs_lookback_probe(10, 0, 10**6, fake_ws, need, None, p, None)
    assert rc == 1 and b"NULL" in L.fgs_last_error()


def test_kernel_timer_selects_spans():
    """The bench's timer records only the spans it was enabled for (no events are
    created for the others, so nothing here needs a GPU)."""
    from paper_2503_01109_gb300.frames import KernelTimer
    t = KernelTimer()
    assert not t.active("render_bwd")
    t.enable(("render_fwd", "render_bwd"))
    assert t.active("render_bwd") and t.active("render_fwd") and not t.active("loss")
    with t.span("loss"):
        pass
    assert t.events == {}
    t.enable()
    assert t.active("loss")
    t.disable()
    assert not t.active("render_bwd")


def test_fused_tail_argument_checks(lib):
    """fgs_project_bwd_adam answers argument errors before any CUDA call: a short
    workspace, a missing step number, grads that do not cover the parameters."""
    from paper_2503_01109_gb300 import fgs, synthetic as syn
    L = fgs.lib()
    cams = fgs.camera_array([syn.pinhole(64, 48, 60.0)])

    def gaussians(n, cap):
        g = fgs.Gaussians()
        g.n, g.capacity, g.d_n = n, cap, None
        base = 1 << 20                     # never dereferenced: every call below fails its checks first
        g.means, g.log_scales, g.quats = base, base + 12 * cap, base + 24 * cap
        g.opacity_logits, g.rgb = base + 40 * cap, base + 44 * cap
        return g

    p, gr, m, v = (gaussians(1000, 1024) for _ in range(4))
    proj = fgs.Projected(1024, 1 << 20, 1 << 21, 1 << 22)
    hp = fgs.AdamParams()
    hp.step = 1
    need = L.fgs_project_bwd_adam_workspace_size(1000)
    assert need >= 8 * 4
    args = lambda grads, hp_, ws_bytes: (ctypes.byref(p), ctypes.byref(proj), cams, 1, ctypes.c_void_p(1 << 23),
                                         ctypes.byref(grads), 0.01, ctypes.c_void_p(1 << 24), ctypes.byref(m),
                                         ctypes.byref(v), ctypes.byref(hp_), None, ctypes.c_void_p(1 << 25),
                                         ws_bytes, None)
    assert L.fgs_project_bwd_adam(*args(gr, hp, need - 1)) == 1 and b"workspace" in L.fgs_last_error()
    hp0 = fgs.AdamParams()
    hp0.step = 0
    assert L.fgs_project_bwd_adam(*args(gr, hp0, need)) == 1 and b"step" in L.fgs_last_error()
    short = gaussians(500, 1024)
    assert L.fgs_project_bwd_adam(*args(short, hp, need)) == 1 and b"cover" in L.fgs_last_error()


def test_peak_probe_argument_checks(lib):
    """fgs_peak_probe refuses an unknown kind or an empty launch before any CUDA call."""
    from paper_2503_01109_gb300 import fgs
    L = fgs.lib()
    ops = ctypes.c_int64(0)
    sink = ctypes.c_void_p(16)
    assert L.fgs_peak_probe(7, 1, 10, sink, ctypes.byref(ops), None) == 1
    assert b"unknown kind" in L.fgs_last_error()
    assert L.fgs_peak_probe(0, 0, 10, sink, ctypes.byref(ops), None) == 1
    assert L.fgs_peak_probe(0, 1, 0, sink, ctypes.byref(ops), None) == 1


def test_autotune_argument_checks(lib):
    """fgs_autotune refuses a missing workspace or bad repetitions before any CUDA call,
    and its workspace size answers on the host."""
    from paper_2503_01109_gb300 import fgs, synthetic as syn
    L = fgs.lib()
    cams = fgs.camera_array([syn.pinhole(64, 48, 60.0), syn.pinhole(40, 30, 40.0)])
    g = fgs.Gaussians()
    g.n, g.capacity = 100, 128
    for k in ("means", "log_scales", "quats", "opacity_logits", "rgb"):
        setattr(g, k, 256)
    need = L.fgs_autotune_workspace_size(ctypes.byref(g), cams, 2, 1 << 16)
    assert need > 2 * (1 << 16) * 4
    assert L.fgs_autotune_workspace_size(ctypes.byref(g), cams, 0, 1 << 16) == 0
    lp = fgs.LossParams(0.9, 0.1, 0.1)
    best = fgs.Tiling()
    dummy = ctypes.c_void_p(256)
    rc = L.fgs_autotune(ctypes.byref(g), cams, 2, dummy, dummy, ctypes.byref(lp), 1 << 16, 3, dummy, need - 1,
                        ctypes.byref(best), None, None)
    assert rc == 1 and b"workspace" in L.fgs_last_error()
    rc = L.fgs_autotune(ctypes.byref(g), cams, 2, dummy, dummy, ctypes.byref(lp), 1 << 16, 0, dummy, need,
                        ctypes.byref(best), None, None)
    assert rc == 1 and b"reps" in L.fgs_last_error()


def test_tile_order_argument_checks(lib):
    """fgs_tile_order refuses bad tilings, NULLs and small workspaces before any CUDA
    call; its workspace holds one int32 per tile of the view set."""
    from paper_2503_01109_gb300 import fgs, synthetic as syn
    L = fgs.lib()
    L.fgs_tile_order_workspace_size.restype = ctypes.c_size_t
    cams = fgs.camera_array([syn.pinhole(64, 48, 60.0), syn.pinhole(40, 30, 40.0)])
    til = fgs.tiling(16, 16, 128)
    tiles = L.fgs_num_tiles(cams, 2, til)
    need = L.fgs_tile_order_workspace_size(cams, 2, til)
    assert tiles == 12 + 6 and need >= 4 * tiles and need % 256 == 0
    assert L.fgs_tile_order_workspace_size(cams, 2, fgs.tiling(12, 12, 128)) == 0
    assert L.fgs_tile_order_workspace_size(cams, 0, til) == 0
    dummy = ctypes.c_void_p(256)  # never dereferenced: every case fails its checks first
    rc = L.fgs_tile_order(cams, 2, fgs.tiling(12, 12, 128), dummy, dummy, dummy, need, None)
    assert rc == 1 and b"tiling" in L.fgs_last_error()
    rc = L.fgs_tile_order(cams, 2, til, None, dummy, dummy, need, None)
    assert rc == 1 and b"NULL" in L.fgs_last_error()
    rc = L.fgs_tile_order(cams, 2, til, dummy, dummy, dummy, 4 * tiles - 1, None)
    assert rc == 1 and b"workspace" in L.fgs_last_error()


def test_fourier_halves_argument_checks(lib):
    """fgs_fourier_energy and fgs_fourier_seed_from_energy refuse NULLs, sizes the
    FFT does not cover and small workspaces before any CUDA call, with their own
    names in the message."""
    from paper_2503_01109_gb300 import fgs, synthetic as syn
    L = fgs.lib()
    prm = fgs.seed_params(max_new=1000)
    need = L.fgs_fourier_seed_workspace_size(64, 48, 1000)
    dummy = ctypes.c_void_p(256)  # never dereferenced: every case fails its checks first
    cam = fgs.camera_struct(syn.pinhole(64, 48, 60.0))
    rc = L.fgs_fourier_energy(None, ctypes.byref(cam), ctypes.byref(prm), None, dummy, dummy, need, None)
    assert rc == 1 and b"fgs_fourier_energy" in L.fgs_last_error()
    rc = L.fgs_fourier_energy(dummy, ctypes.byref(cam), ctypes.byref(prm), None, dummy, dummy, need - 1, None)
    assert rc == 1 and b"workspace" in L.fgs_last_error()
    odd = fgs.camera_struct(syn.pinhole(64 * 19, 48, 60.0))   # a prime factor of 19
    rc = L.fgs_fourier_energy(dummy, ctypes.byref(odd), ctypes.byref(prm), None, dummy, dummy, 1 << 30, None)
    assert rc == 5 and b"prime factor" in L.fgs_last_error()
    g = fgs.Gaussians()
    g.n, g.capacity = 0, 1000
    for k in ("means", "log_scales", "quats", "opacity_logits", "rgb"):
        setattr(g, k, 256)
    rc = L.fgs_fourier_seed_from_energy(dummy, None, None, None, None, ctypes.byref(cam), ctypes.byref(prm), None,
                                        dummy, None, ctypes.byref(g), dummy, dummy, None, dummy, need, None, None)
    assert rc == 1 and b"fgs_fourier_seed_from_energy" in L.fgs_last_error()
