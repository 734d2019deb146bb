// api.cu -- error state, version, launch counter and shared host helpers.
#include <cstdarg>
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace fgs {

static thread_local char g_err[512] = "";
static std::atomic<int64_t> g_launches{0};

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cached[dev] = v;
  }
  return cached[dev];
}

bool make_views(const fgs_camera *cams, int32_t n_views, int tile_w, int tile_h, DevViews *out) {
  if (cams == nullptr || n_views < 1 || n_views > FGS_MAX_VIEWS) {
    set_error("n_views must be 1..%d with a camera array", FGS_MAX_VIEWS);
    return false;
  }
  memset(out, 0, sizeof(*out));
  out->n = n_views;
  int64_t tiles = 0, pix = 0;
  for (int v = 0; v < n_views; ++v) {
    const fgs_camera &c = cams[v];
    if (c.width <= 0 || c.height <= 0 || c.width > 16384 || c.height > 16384 || !(c.fx > 0) ||
        !(c.fy > 0)) {
      set_error("camera %d: bad size or focal length", v);
      return false;
    }
    DevCam &d = out->cam[v];
    d.W = c.width;
    d.H = c.height;
    d.fx = c.fx;
    d.fy = c.fy;
    d.cx = c.cx;
    d.cy = c.cy;
    for (int r = 0; r < 3; ++r) {
      for (int k = 0; k < 3; ++k) d.R[3 * r + k] = c.world_to_cam[4 * r + k];
      d.t[r] = c.world_to_cam[4 * r + 3];
    }
    d.znear = c.znear;
    d.tiles_x = (c.width + tile_w - 1) / tile_w;
    d.tiles_y = (c.height + tile_h - 1) / tile_h;
    d.tile_base = (int)tiles;
    d.pix_base = pix;
    tiles += (int64_t)d.tiles_x * d.tiles_y;
    pix += (int64_t)c.width * c.height;
  }
  if (tiles > (1 << 24)) {
    set_error("too many tiles (%lld)", (long long)tiles);
    return false;
  }
  out->total_tiles = (int)tiles;
  out->total_pix = pix;
  return true;
}

bool gaussians_ok(const fgs_gaussians *g, const char *name) {
  if (g == nullptr) {
    set_error("%s is NULL", name);
    return false;
  }
  if (g->n < 0 || g->capacity < g->n || g->capacity > (int64_t(1) << 31) - 1) {
    set_error("%s: need 0 <= n <= capacity < 2^31", name);
    return false;
  }
  if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->rgb)) {
    set_error("%s: NULL parameter plane", name);
    return false;
  }
  return true;
}

}  // namespace fgs

extern "C" {

const char *fgs_last_error(void) { return fgs::g_err; }
int32_t fgs_version(void) { return FGS_VERSION; }
int64_t fgs_launch_count(void) { return fgs::g_launches.load(); }

fgs_status fgs_memset_async(void *dst, int32_t value, size_t bytes, void *stream) {
  if (bytes == 0) return FGS_OK;
  if (dst == nullptr) {
    fgs::set_error("fgs_memset_async: NULL destination");
    return FGS_ERR_INVALID_ARGUMENT;
  }
  FGS_CUDA(cudaMemsetAsync(dst, value, bytes, fgs::as_stream(stream)), "fgs_memset_async");
  return FGS_OK;
}

fgs_status fgs_memcpy_async(void *dst, const void *src, size_t bytes, void *stream) {
  if (bytes == 0) return FGS_OK;
  if (dst == nullptr || src == nullptr) {
    fgs::set_error("fgs_memcpy_async: NULL pointer");
    return FGS_ERR_INVALID_ARGUMENT;
  }
  FGS_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, fgs::as_stream(stream)), "fgs_memcpy_async");
  return FGS_OK;
}

int64_t fgs_num_tiles(const fgs_camera *cams, int32_t n_views, fgs_tiling tiling) {
  if (!fgs::tiling_ok(tiling)) return -1;
  fgs::DevViews vs;
  if (!fgs::make_views(cams, n_views, tiling.tile_w, tiling.tile_h, &vs)) return -1;
  return vs.total_tiles;
}

}  // extern "C"
