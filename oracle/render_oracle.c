/*
 * render_oracle.c -- FP64 CPU oracle of the splatting half of the mapping path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this file's library.  It shares no code, header or
 * constant table with the CUDA library.
 *
 * Plain, slow, direct code in double precision.  Every function cites the part
 * of the paper it follows (FGS-SLAM, arXiv 2503.01109; equations by LaTeX label):
 *   - Sec. III: Gaussians G{mu, S, R, alpha, c}, covariance C = R S S^T R^T, and
 *     their 2D projection; eq1 alpha blending with gamma = colour / depth / 1.
 *   - Sec. III-D: scale regulariser eq15 and mapping loss eq16.
 * The constants the paper does not state (near plane 0.2, dilation 0.3 px^2,
 * alpha clamp 0.99, skip below 1/255, stop when T < 1e-4, 3-sigma support,
 * Jacobian clamp 1.3 tan(half FOV)) are the standard Gaussian-splatting values
 * the paper cites; they are passed in from Python so that nothing is shared.
 *
 * Layouts (chosen for readability, array-of-structures):
 *   means[n][3], log_scales[n][3], quats[n][4] (w,x,y,z), logits[n], rgb[n][3]
 *   camera: double cam[19] = w, h, fx, fy, cx, cy, R[9] row-major, t[3], znear
 *   splats of one view: mean2d[n][2], conic[n][3], depth[n], opacity[n],
 *   radius[n] (0 = culled), rect[n][4] = tile x0, y0, x1, y1 (x0 > x1: none),
 *   thr[n] (support threshold, see or_project)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  double near_z, dilation, alpha_max, alpha_min, t_min, jac_clamp, support_sigma;
} OConst;

static void unpack_const(const double *k, OConst *c) {
  c->near_z = k[0];        /* unused when the camera carries znear */
  c->dilation = k[1];
  c->alpha_max = k[2];
  c->alpha_min = k[3];
  c->t_min = k[4];
  c->jac_clamp = k[5];
  c->support_sigma = k[6];
}

/* Rotation matrix of a unit quaternion (w, x, y, z). */
static void quat_to_rot(const double q[4], double R[9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Intermediate quantities of one Gaussian's projection (kept for the adjoint). */
typedef struct {
  int visible;
  double p[3];          /* camera-space mean */
  double qn[4], qlen;   /* normalised quaternion and the raw length */
  double s[3];          /* linear scales */
  double Rq[9];         /* rotation of the Gaussian */
  double Sigma[9];      /* 3D covariance (world) */
  double u, v, uc, vc;  /* x/z, y/z and their clamped values */
  int clamp_u, clamp_v; /* 1 when the clamp is active */
  double Jm[6];         /* 2x3 perspective Jacobian */
  double T[6];          /* J R_cam */
  double a, b, c;       /* Sigma' (dilated) */
  double det;
  double conic[3];
  double mean2d[2];
  double opacity;
} OProj;

/* Sec. III: covariance C = R S S^T R^T of a Gaussian and its EWA projection. */
static void project_one(const double *mu, const double *ls, const double *q, double logit,
                        const double *cam, const OConst *k, OProj *o) {
  const double W = cam[0], H = cam[1], fx = cam[2], fy = cam[3], cx = cam[4], cy = cam[5];
  const double *Rc = cam + 6, *tc = cam + 15, znear = cam[18];
  memset(o, 0, sizeof(*o));
  for (int r = 0; r < 3; ++r)
    o->p[r] = Rc[3 * r] * mu[0] + Rc[3 * r + 1] * mu[1] + Rc[3 * r + 2] * mu[2] + tc[r];
  o->opacity = 1.0 / (1.0 + exp(-logit));
  if (!(o->p[2] >= znear)) return;
  o->qlen = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int i = 0; i < 4; ++i) o->qn[i] = q[i] / o->qlen;
  quat_to_rot(o->qn, o->Rq);
  for (int i = 0; i < 3; ++i) o->s[i] = exp(ls[i]);
  /* Sigma = Rq diag(s^2) Rq^T */
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int l = 0; l < 3; ++l) acc += o->Rq[3 * i + l] * o->s[l] * o->s[l] * o->Rq[3 * j + l];
      o->Sigma[3 * i + j] = acc;
    }
  const double z = o->p[2];
  const double limx = k->jac_clamp * (0.5 * W / fx), limy = k->jac_clamp * (0.5 * H / fy);
  o->u = o->p[0] / z;
  o->v = o->p[1] / z;
  o->uc = clampd(o->u, -limx, limx);
  o->vc = clampd(o->v, -limy, limy);
  o->clamp_u = (o->uc != o->u);
  o->clamp_v = (o->vc != o->v);
  o->Jm[0] = fx / z; o->Jm[1] = 0;      o->Jm[2] = -fx * o->uc / z;
  o->Jm[3] = 0;      o->Jm[4] = fy / z; o->Jm[5] = -fy * o->vc / z;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int l = 0; l < 3; ++l) acc += o->Jm[3 * i + l] * Rc[3 * l + j];
      o->T[3 * i + j] = acc;
    }
  double S2[4] = {0, 0, 0, 0}; /* T Sigma T^T */
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      double acc = 0;
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) acc += o->T[3 * i + l] * o->Sigma[3 * l + m] * o->T[3 * j + m];
      S2[2 * i + j] = acc;
    }
  o->a = S2[0] + k->dilation;
  o->b = 0.5 * (S2[1] + S2[2]);
  o->c = S2[3] + k->dilation;
  o->det = o->a * o->c - o->b * o->b;
  if (!(o->det > 0)) return;
  o->conic[0] = o->c / o->det;
  o->conic[1] = -o->b / o->det;
  o->conic[2] = o->a / o->det;
  o->mean2d[0] = fx * o->u + cx;
  o->mean2d[1] = fy * o->v + cy;
  o->visible = 1;
}

/* Support threshold of a splat: alpha = o exp(-q/2) reaches 1/255 only where
 * q <= 2 ln(255 o); plus a margin above any float32 rounding of that test.  A
 * splat with 255 o <= 1 blends nowhere (-1). */
#define SUPPORT_MARGIN 0.01

/* Projection of n Gaussians into one view; rect uses tile_w x tile_h tiles. */
void or_project(int64_t n, const double *means, const double *log_scales, const double *quats,
                const double *logits, const double *cam, const double *kconst, int tile_w,
                int tile_h, double *mean2d, double *conic, double *depth, double *opacity,
                int32_t *radius, int32_t *rect, double *thr) {
  OConst k;
  unpack_const(kconst, &k);
  const int W = (int)cam[0], H = (int)cam[1];
  const int tiles_x = (W + tile_w - 1) / tile_w, tiles_y = (H + tile_h - 1) / tile_h;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    OProj o;
    project_one(means + 3 * i, log_scales + 3 * i, quats + 4 * i, logits[i], cam, &k, &o);
    mean2d[2 * i] = o.mean2d[0];
    mean2d[2 * i + 1] = o.mean2d[1];
    conic[3 * i] = o.conic[0];
    conic[3 * i + 1] = o.conic[1];
    conic[3 * i + 2] = o.conic[2];
    depth[i] = o.p[2];
    opacity[i] = o.opacity;
    int32_t *rc = rect + 4 * i;
    rc[0] = 1; rc[1] = 1; rc[2] = 0; rc[3] = 0;
    radius[i] = 0;
    thr[i] = 255.0 * o.opacity > 1.0 ? 2.0 * log(255.0 * o.opacity) + SUPPORT_MARGIN : -1.0;
    if (!o.visible) continue;
    double mid = 0.5 * (o.a + o.c);
    double lam = mid + sqrt(fmax(0.0, mid * mid - o.det));
    radius[i] = (int32_t)ceil(k.support_sigma * sqrt(lam));
    /* tiles whose pixel-centre box [tx*TW, tx*TW+TW-1] meets the 3-sigma box cut
     * to the bounding box of the support ellipse {q <= thr}: half-widths
     * sqrt(thr a), sqrt(thr c) with (a, c) the diagonal of the 2D covariance */
    double kk = fmin(k.support_sigma, sqrt(fmax(thr[i], 0.0)));
    double ex = kk * sqrt(o.a), ey = kk * sqrt(o.c);
    double x0 = ceil((o.mean2d[0] - ex - (tile_w - 1)) / tile_w);
    double x1 = floor((o.mean2d[0] + ex) / tile_w);
    double y0 = ceil((o.mean2d[1] - ey - (tile_h - 1)) / tile_h);
    double y1 = floor((o.mean2d[1] + ey) / tile_h);
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > tiles_x - 1) x1 = tiles_x - 1;
    if (y1 > tiles_y - 1) y1 = tiles_y - 1;
    if (x0 <= x1 && y0 <= y1 && thr[i] >= 0) {
      rc[0] = (int32_t)x0; rc[1] = (int32_t)y0; rc[2] = (int32_t)x1; rc[3] = (int32_t)y1;
    }
  }
}

/* ---------------------------------------------------------------------------------
 * Opacity-aware support of a splat on a row of tiles.  The splat can reach
 * alpha >= 1/255 only inside the ellipse E = {q(d) <= thr}, q(d) = a dx^2 +
 * 2 b dx dy + c dy^2 (d = pixel - mean2d).  A tile of tile row ty spans the row's
 * pixel-centre rows y0 <= dy <= y1, so it meets E iff its pixel-centre columns
 * meet [xl, xr], the x-extent of E within that strip.  E is convex and its left
 * boundary x(dy) = (-b dy - sqrt(thr a - det dy^2)) / a (det = a c - b^2) is convex
 * in dy with its minimum -sqrt(thr c / det) at dy = b sqrt(thr c / det) / c; over
 * the strip cut to E's y-range [-sqrt(thr a / det), +sqrt(thr a / det)] the
 * leftmost point lies at that dy clamped into the range (the right boundary
 * mirrors it).  Tile tx is kept iff tx tw + tw - 1 >= mx + xl and
 * tx tw <= mx + xr, i.e. for tx in [ceil((mx + xl - (tw - 1)) / tw),
 * floor((mx + xr) / tw)] cut to the rect's columns.
 * strip_f32 takes every step in float32 in this order (parity with the kernels);
 * strip_f64 is the same in double.  Both return 0 when the strip misses E. */
static int strip_f32(float mx, float my, float a, float b, float c, float thr, int ty, int tw, int th, float *xl,
                     float *xr) {
  const float y0 = (float)(ty * th) - my, y1 = (float)(ty * th + th - 1) - my;
  const float det = a * c - b * b;
  if (!(det > 0.f) || !(thr >= 0.f)) return 0;
  const float ta = thr * a;
  const float ys = sqrtf(ta / det), xs = sqrtf((thr * c) / det);
  const float lo = fmaxf(y0, -ys), hi = fminf(y1, ys);
  if (lo > hi) return 0;
  const float dl = (b * xs) / c;
  const float yl = fminf(fmaxf(dl, lo), hi), yr = fminf(fmaxf(-dl, lo), hi);
  const float rl = sqrtf(fmaxf(ta - det * (yl * yl), 0.f)), rr = sqrtf(fmaxf(ta - det * (yr * yr), 0.f));
  *xl = (-(b * yl) - rl) / a;
  *xr = (-(b * yr) + rr) / a;
  return 1;
}

static int strip_f64(double mx, double my, double a, double b, double c, double thr, int ty, int tw, int th,
                     double *xl, double *xr) {
  const double y0 = (double)(ty * th) - my, y1 = (double)(ty * th + th - 1) - my;
  const double det = a * c - b * b;
  if (!(det > 0.0) || !(thr >= 0.0)) return 0;
  const double ta = thr * a;
  const double ys = sqrt(ta / det), xs = sqrt((thr * c) / det);
  const double lo = fmax(y0, -ys), hi = fmin(y1, ys);
  if (lo > hi) return 0;
  const double dl = (b * xs) / c;
  const double yl = fmin(fmax(dl, lo), hi), yr = fmin(fmax(-dl, lo), hi);
  const double rl = sqrt(fmax(ta - det * (yl * yl), 0.0)), rr = sqrt(fmax(ta - det * (yr * yr), 0.0));
  *xl = (-(b * yl) - rl) / a;
  *xr = (-(b * yr) + rr) / a;
  return 1;
}

/* The tiles of rect row ty (rect columns [x0, x1]) that a splat keeps, as above;
 * supp: per record mx, my, a, b, c, thr -- float32 [v][n][6] (supp_f32 = 1) or
 * double (supp_f32 = 0); NULL = the whole rect row.  Returns 0 (and leaves
 * *first > *last) when no tile is kept. */
static int row_interval(const void *supp, int supp_f32, int64_t rec, int ty, int x0, int x1, int tw, int th,
                        int *first, int *last) {
  *first = 1;
  *last = 0;
  int a = x0, b = x1;
  if (supp && supp_f32) {
    const float *s = (const float *)supp + 6 * rec;
    float xl, xr;
    if (!strip_f32(s[0], s[1], s[2], s[3], s[4], s[5], ty, tw, th, &xl, &xr)) return 0;
    /* the tile bounds, clamped in float to [x0 - 1, x1 + 1] before the conversion */
    const float fa = fminf(fmaxf(ceilf(((s[0] + xl) - (float)(tw - 1)) / (float)tw), (float)x0), (float)x1 + 1.f);
    const float fb = fminf(fmaxf(floorf((s[0] + xr) / (float)tw), (float)x0 - 1.f), (float)x1);
    a = (int)fa;
    b = (int)fb;
  } else if (supp) {
    const double *s = (const double *)supp + 6 * rec;
    double xl, xr;
    if (!strip_f64(s[0], s[1], s[2], s[3], s[4], s[5], ty, tw, th, &xl, &xr)) return 0;
    const double fa = fmin(fmax(ceil(((s[0] + xl) - (double)(tw - 1)) / (double)tw), (double)x0), (double)x1 + 1.0);
    const double fb = fmin(fmax(floor((s[0] + xr) / (double)tw), (double)x0 - 1.0), (double)x1);
    a = (int)fa;
    b = (int)fb;
  }
  if (a > b) return 0;
  *first = a;
  *last = b;
  return 1;
}

/* ---------------------------------------------------------------------------------
 * Binning: every (tile, Gaussian) pair whose tile lies in the Gaussian's rect and
 * in the kept interval of its row (row_interval),
 * ordered by (global tile, float32 depth bits, id).  Depth order is the
 * front-to-back order eq1's product runs over.  depth_f32 is the float32 depth
 * the kernels key on; it is given, so the order is a pure integer question. */
typedef struct {
  uint32_t tile;
  uint32_t dbits;
  int32_t id;
} OPair;

static int pair_cmp(const void *pa, const void *pb) {
  const OPair *a = (const OPair *)pa, *b = (const OPair *)pb;
  if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
  if (a->dbits != b->dbits) return a->dbits < b->dbits ? -1 : 1;
  if (a->id != b->id) return a->id < b->id ? -1 : 1;
  return 0;
}

/* Counts the pairs of a view set.  rect[v][n][4], radius[v][n]. */
int64_t or_count_pairs(int32_t n_views, int64_t n, const int32_t *radius, const int32_t *rect,
                       const void *supp, int supp_f32, int tile_w, int tile_h) {
  int64_t total = 0;
  for (int32_t v = 0; v < n_views; ++v)
    for (int64_t i = 0; i < n; ++i) {
      const int32_t *r = rect + 4 * (v * n + i);
      if (radius[v * n + i] <= 0 || r[0] > r[2] || r[1] > r[3]) continue;
      for (int32_t ty = r[1]; ty <= r[3]; ++ty) {
        int a, b;
        if (row_interval(supp, supp_f32, v * n + i, ty, r[0], r[2], tile_w, tile_h, &a, &b)) total += b - a + 1;
      }
    }
  return total;
}

/* tiles_x[v], tiles_y[v] per view; outputs sorted tile/id lists and ranges
 * (ranges[2*t], ranges[2*t+1]).  Returns the pair count. */
int64_t or_bin_sort(int32_t n_views, int64_t n, const int32_t *tiles_x, const int32_t *tiles_y,
                    const float *depth_f32, const int32_t *radius, const int32_t *rect,
                    const void *supp, int supp_f32, int tile_w, int tile_h,
                    uint32_t *out_tile, int32_t *out_id, int32_t *ranges) {
  int64_t P = or_count_pairs(n_views, n, radius, rect, supp, supp_f32, tile_w, tile_h);
  OPair *pairs = (OPair *)malloc(sizeof(OPair) * (size_t)(P > 0 ? P : 1));
  int64_t k = 0;
  uint32_t tile_base = 0;
  for (int32_t v = 0; v < n_views; ++v) {
    for (int64_t i = 0; i < n; ++i) {
      const int32_t *r = rect + 4 * (v * n + i);
      if (radius[v * n + i] <= 0 || r[0] > r[2] || r[1] > r[3]) continue;
      uint32_t dbits;
      memcpy(&dbits, &depth_f32[v * n + i], 4);
      for (int32_t ty = r[1]; ty <= r[3]; ++ty) {
        int a, b;
        if (!row_interval(supp, supp_f32, v * n + i, ty, r[0], r[2], tile_w, tile_h, &a, &b)) continue;
        for (int32_t tx = a; tx <= b; ++tx) {
          pairs[k].tile = tile_base + (uint32_t)(ty * tiles_x[v] + tx);
          pairs[k].dbits = dbits;
          pairs[k].id = (int32_t)i;
          ++k;
        }
      }
    }
    tile_base += (uint32_t)(tiles_x[v] * tiles_y[v]);
  }
  qsort(pairs, (size_t)P, sizeof(OPair), pair_cmp);
  for (uint32_t t = 0; t < tile_base; ++t) ranges[2 * t] = ranges[2 * t + 1] = 0;
  for (int64_t j = 0; j < P; ++j) {
    out_tile[j] = pairs[j].tile;
    out_id[j] = pairs[j].id;
    if (j == 0 || pairs[j].tile != pairs[j - 1].tile) ranges[2 * pairs[j].tile] = (int32_t)j;
    if (j == P - 1 || pairs[j].tile != pairs[j + 1].tile) ranges[2 * pairs[j].tile + 1] = (int32_t)(j + 1);
  }
  free(pairs);
  return P;
}

/* ---------------------------------------------------------------------------------
 * eq1 front to back for one pixel over a given ordered list of Gaussians.
 * Records every blended Gaussian (for the adjoint) when rec != NULL.
 * Returns a decision-band flag: 1 when a threshold decision lay within the band
 * where a float32 evaluation could take the other branch. */
typedef struct {
  int32_t id;
  double alpha, T, G, dx, dy;
  int clamped;
} OContrib;

typedef struct {
  double band_alpha, band_t, band_power;
} OBand;

static int blend_pixel(double px, double py, const int32_t *list, int64_t len,
                       const double *mean2d, const double *conic, const double *depth,
                       const double *opacity, const double *rgb, const OConst *k,
                       const OBand *band, double out[5], double *t_final, int32_t *n_contrib,
                       OContrib *rec, int64_t *n_rec) {
  double T = 1.0, C[3] = {0, 0, 0}, D = 0, A = 0;
  int flag = 0;
  int32_t last = 0;
  int64_t nr = 0;
  for (int64_t j = 0; j < len; ++j) {
    int32_t g = list[j];
    double dx = mean2d[2 * g] - px, dy = mean2d[2 * g + 1] - py;
    double power = -0.5 * (conic[3 * g] * dx * dx + conic[3 * g + 2] * dy * dy) - conic[3 * g + 1] * dx * dy;
    if (band && fabs(power) <= band->band_power) flag = 1;
    if (power > 0) continue;
    double G = exp(power);
    double raw = opacity[g] * G;
    double alpha = raw < k->alpha_max ? raw : k->alpha_max;
    if (band && (fabs(raw - k->alpha_min) <= band->band_alpha * k->alpha_min ||
                 fabs(raw - k->alpha_max) <= band->band_alpha * k->alpha_max))
      flag = 1;
    if (alpha < k->alpha_min) continue;
    double Tn = T * (1 - alpha);
    if (band && fabs(Tn - k->t_min) <= band->band_t * k->t_min) flag = 1;
    if (Tn < k->t_min) break;
    for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * g + ch] * alpha * T;
    D += depth[g] * alpha * T;
    A += alpha * T;
    if (rec) {
      rec[nr].id = g;
      rec[nr].alpha = alpha;
      rec[nr].T = T;
      rec[nr].G = G;
      rec[nr].dx = dx;
      rec[nr].dy = dy;
      rec[nr].clamped = raw >= k->alpha_max;
      ++nr;
    }
    T = Tn;
    last = (int32_t)(j + 1);
  }
  out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = D; out[4] = A;
  if (t_final) *t_final = T;
  if (n_contrib) *n_contrib = last;
  if (n_rec) *n_rec = nr;
  return flag;
}

/* Tile-binned renderer of one view (eq1): per pixel, the list of its tile.
 * ids/ranges: sorted lists; tile_base: first global tile of this view.
 * Outputs color[3][H][W], depth, alpha, t_final [H][W], n_contrib, flag. */
void or_render_fwd(int64_t n, const double *mean2d, const double *conic, const double *depth,
                   const double *opacity, const double *rgb, const double *cam,
                   const double *kconst, const double *bandv, int tile_w, int tile_h,
                   const int32_t *ids, const int32_t *ranges, int32_t tile_base, double *color,
                   double *odepth, double *oalpha, double *t_final, int32_t *n_contrib,
                   uint8_t *flag) {
  (void)n;
  OConst k;
  unpack_const(kconst, &k);
  OBand band = {bandv[0], bandv[1], bandv[2]};
  const int W = (int)cam[0], H = (int)cam[1];
  const int tiles_x = (W + tile_w - 1) / tile_w;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t pix = 0; pix < (int64_t)W * H; ++pix) {
    int x = (int)(pix % W), y = (int)(pix / W);
    int t = tile_base + (y / tile_h) * tiles_x + (x / tile_w);
    int32_t s = ranges[2 * t], e = ranges[2 * t + 1];
    double out[5];
    flag[pix] = (uint8_t)blend_pixel(x, y, ids + s, e - s, mean2d, conic, depth, opacity, rgb, &k,
                                     &band, out, &t_final[pix], &n_contrib[pix], NULL, NULL);
    for (int ch = 0; ch < 3; ++ch) color[(int64_t)ch * W * H + pix] = out[ch];
    odepth[pix] = out[3];
    oalpha[pix] = out[4];
  }
}

/* Brute-force renderer of one view: for every pixel, every Gaussian whose rect
 * holds the pixel's tile, put in (float32 depth bits, id) order by a plain
 * insertion sort, then eq1.  No binning, no shared lists. */
void or_render_brute(int64_t n, const double *mean2d, const double *conic, const double *depth,
                     const double *opacity, const double *rgb, const float *depth_f32,
                     const int32_t *radius, const int32_t *rect, const double *cam,
                     const double *kconst, int tile_w, int tile_h, double *color,
                     double *odepth, double *oalpha) {
  OConst k;
  unpack_const(kconst, &k);
  const int W = (int)cam[0], H = (int)cam[1];
#pragma omp parallel
  {
    int32_t *list = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 16)
    for (int64_t pix = 0; pix < (int64_t)W * H; ++pix) {
      int x = (int)(pix % W), y = (int)(pix / W);
      int tx = x / tile_w, ty = y / tile_h;
      int64_t len = 0;
      for (int64_t i = 0; i < n; ++i) {
        const int32_t *r = rect + 4 * i;
        if (radius[i] <= 0 || tx < r[0] || tx > r[2] || ty < r[1] || ty > r[3]) continue;
        /* insertion by (depth bits, id) */
        uint32_t di;
        memcpy(&di, &depth_f32[i], 4);
        int64_t j = len;
        while (j > 0) {
          uint32_t dj;
          memcpy(&dj, &depth_f32[list[j - 1]], 4);
          if (dj < di || (dj == di && list[j - 1] < (int32_t)i)) break;
          list[j] = list[j - 1];
          --j;
        }
        list[j] = (int32_t)i;
        ++len;
      }
      double out[5];
      blend_pixel(x, y, list, len, mean2d, conic, depth, opacity, rgb, &k, NULL, out, NULL, NULL,
                  NULL, NULL);
      for (int ch = 0; ch < 3; ++ch) color[(int64_t)ch * W * H + pix] = out[ch];
      odepth[pix] = out[3];
      oalpha[pix] = out[4];
    }
    free(list);
  }
}

/* Per-pixel transmittance trace for the invariant test: T before each blended
 * Gaussian of pixel (x, y), written to trace (at most max_len); returns count. */
int64_t or_trace_pixel(int x, int y, const double *mean2d, const double *conic,
                       const double *depth, const double *opacity, const double *rgb,
                       const double *cam, const double *kconst, int tile_w, int tile_h,
                       const int32_t *ids, const int32_t *ranges, int32_t tile_base,
                       double *trace, int64_t max_len) {
  OConst k;
  unpack_const(kconst, &k);
  const int W = (int)cam[0];
  const int tiles_x = (W + tile_w - 1) / tile_w;
  int t = tile_base + (y / tile_h) * tiles_x + (x / tile_w);
  int32_t s = ranges[2 * t], e = ranges[2 * t + 1];
  OContrib *rec = (OContrib *)malloc(sizeof(OContrib) * (size_t)(e - s + 1));
  double out[5], tf;
  int64_t nr = 0;
  blend_pixel(x, y, ids + s, e - s, mean2d, conic, depth, opacity, rgb, &k, NULL, out, &tf, NULL,
              rec, &nr);
  int64_t m = 0;
  for (int64_t j = 0; j < nr && m < max_len; ++j) trace[m++] = rec[j].T;
  if (m < max_len) trace[m++] = tf;
  free(rec);
  return m;
}

/* ---------------------------------------------------------------------------------
 * Adjoint of eq1 for one view.  F = sum_i gamma_i alpha_i T_i with
 * T_i = prod_{j<i}(1 - alpha_j) gives
 *   dF/dalpha_i = gamma_i T_i - (sum_{j>i} gamma_j alpha_j T_j) / (1 - alpha_i),
 * written here with the suffix sums of a stored forward walk.  Then
 *   alpha = o G (unclamped), G = exp(power), power = -(a dx^2 + c dy^2)/2 - b dx dy,
 * d = mean2d - pixel.  Accumulates into grad2d[n][7] = (mean2d x, y, conic a, b, c,
 * opacity, depth) and grad_rgb[n][3].  dA may be NULL. */
void or_render_bwd(int64_t n, const double *mean2d, const double *conic, const double *depth,
                   const double *opacity, const double *rgb, const double *cam,
                   const double *kconst, int tile_w, int tile_h, const int32_t *ids,
                   const int32_t *ranges, int32_t tile_base, const double *dC, const double *dD,
                   const double *dA, double *grad2d, double *grad_rgb) {
  (void)n;
  OConst k;
  unpack_const(kconst, &k);
  const int W = (int)cam[0], H = (int)cam[1];
  const int tiles_x = (W + tile_w - 1) / tile_w;
  const int64_t HW = (int64_t)W * H;
#pragma omp parallel
  {
    int64_t cap = 1024;
    OContrib *rec = (OContrib *)malloc(sizeof(OContrib) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
    for (int64_t pix = 0; pix < HW; ++pix) {
      int x = (int)(pix % W), y = (int)(pix / W);
      int t = tile_base + (y / tile_h) * tiles_x + (x / tile_w);
      int32_t s = ranges[2 * t], e = ranges[2 * t + 1];
      if (e - s + 1 > cap) {
        cap = e - s + 1;
        rec = (OContrib *)realloc(rec, sizeof(OContrib) * (size_t)cap);
      }
      double out[5];
      int64_t nr = 0;
      blend_pixel(x, y, ids + s, e - s, mean2d, conic, depth, opacity, rgb, &k, NULL, out, NULL,
                  NULL, rec, &nr);
      double g[5] = {dC[pix], dC[HW + pix], dC[2 * HW + pix], dD ? dD[pix] : 0.0,
                     dA ? dA[pix] : 0.0};
      /* suffix sums S_i = sum_{j>i} gamma_j alpha_j T_j for the 5 channels */
      double S[5] = {0, 0, 0, 0, 0};
      for (int64_t j = nr - 1; j >= 0; --j) {
        const OContrib *c = &rec[j];
        int32_t id = c->id;
        double gam[5] = {rgb[3 * id], rgb[3 * id + 1], rgb[3 * id + 2], depth[id], 1.0};
        double dalpha = 0;
        for (int ch = 0; ch < 5; ++ch) dalpha += g[ch] * (gam[ch] * c->T - S[ch] / (1 - c->alpha));
        double w = c->alpha * c->T;
        double gr[3] = {g[0] * w, g[1] * w, g[2] * w};
        double gz = g[3] * w;
        double gm[2] = {0, 0}, gc[3] = {0, 0, 0}, go = 0;
        if (!c->clamped) {
          double dpower = dalpha * c->alpha; /* d alpha / d power = o G = alpha */
          const double *cn = conic + 3 * id;
          /* d power / d mean2d = -(a dx + b dy, b dx + c dy) since d = mean2d - pixel */
          gm[0] = dpower * (-(cn[0] * c->dx + cn[1] * c->dy));
          gm[1] = dpower * (-(cn[1] * c->dx + cn[2] * c->dy));
          gc[0] = dpower * (-0.5 * c->dx * c->dx);
          gc[1] = dpower * (-c->dx * c->dy);
          gc[2] = dpower * (-0.5 * c->dy * c->dy);
          go = dalpha * c->G;
        }
        double *gg = grad2d + 7 * (int64_t)id;
#pragma omp atomic
        gg[0] += gm[0];
#pragma omp atomic
        gg[1] += gm[1];
#pragma omp atomic
        gg[2] += gc[0];
#pragma omp atomic
        gg[3] += gc[1];
#pragma omp atomic
        gg[4] += gc[2];
#pragma omp atomic
        gg[5] += go;
#pragma omp atomic
        gg[6] += gz;
        for (int ch = 0; ch < 3; ++ch) {
#pragma omp atomic
          grad_rgb[3 * (int64_t)id + ch] += gr[ch];
        }
        for (int ch = 0; ch < 5; ++ch) S[ch] += gam[ch] * w;
      }
    }
    free(rec);
  }
}

/* ---------------------------------------------------------------------------------
 * Adjoint of the projection (chain rule of project_one), one view, accumulated
 * into g_means[n][3], g_log_scales[n][3], g_quats[n][4], g_logits[n].
 * grad2d[n][7] as produced by or_render_bwd. */
void or_project_bwd(int64_t n, const double *means, const double *log_scales,
                    const double *quats, const double *logits, const double *cam,
                    const double *kconst, const double *grad2d, double *g_means,
                    double *g_log_scales, double *g_quats, double *g_logits) {
  OConst k;
  unpack_const(kconst, &k);
  const double fx = cam[2], fy = cam[3];
  const double *Rc = cam + 6;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    OProj o;
    project_one(means + 3 * i, log_scales + 3 * i, quats + 4 * i, logits[i], cam, &k, &o);
    const double *gg = grad2d + 7 * i;
    /* opacity = sigmoid(logit) */
    g_logits[i] += gg[5] * o.opacity * (1 - o.opacity);
    if (!o.visible) continue;
    const double z = o.p[2], x = o.p[0], y = o.p[1];
    /* conic = inverse of [[a, b], [b, c]] */
    double det2 = o.det * o.det;
    double gA = gg[2], gB = gg[3], gC = gg[4];
    double ga = gA * (-o.c * o.c / det2) + gB * (o.b * o.c / det2) + gC * (-o.b * o.b / det2);
    double gb = gA * (2 * o.b * o.c / det2) + gB * (-(o.a * o.c + o.b * o.b) / det2) +
                gC * (2 * o.a * o.b / det2);
    double gc = gA * (-o.b * o.b / det2) + gB * (o.a * o.b / det2) + gC * (-o.a * o.a / det2);
    /* Sigma'' = T Sigma T^T (b is the shared off-diagonal entry) */
    double Gp[4] = {ga, 0.5 * gb, 0.5 * gb, gc};
    /* dL/dSigma = T^T G' T */
    double GS[9];
    for (int r = 0; r < 3; ++r)
      for (int c2 = 0; c2 < 3; ++c2) {
        double acc = 0;
        for (int l = 0; l < 2; ++l)
          for (int m = 0; m < 2; ++m) acc += o.T[3 * l + r] * Gp[2 * l + m] * o.T[3 * m + c2];
        GS[3 * r + c2] = acc;
      }
    /* dL/dT = 2 G' T Sigma */
    double GT[6];
    for (int r = 0; r < 2; ++r)
      for (int c2 = 0; c2 < 3; ++c2) {
        double acc = 0;
        for (int l = 0; l < 2; ++l)
          for (int m = 0; m < 3; ++m) acc += 2 * Gp[2 * r + l] * o.T[3 * l + m] * o.Sigma[3 * m + c2];
        GT[3 * r + c2] = acc;
      }
    /* T = J R_cam -> dL/dJ = dL/dT R_cam^T */
    double GJ[6];
    for (int r = 0; r < 2; ++r)
      for (int c2 = 0; c2 < 3; ++c2) {
        double acc = 0;
        for (int m = 0; m < 3; ++m) acc += GT[3 * r + m] * Rc[3 * c2 + m];
        GJ[3 * r + c2] = acc;
      }
    /* J entries as functions of p = (x, y, z) */
    double gp[3] = {0, 0, 0};
    gp[2] += GJ[0] * (-fx / (z * z));
    gp[2] += GJ[4] * (-fy / (z * z));
    if (o.clamp_u) {
      gp[2] += GJ[2] * (fx * o.uc / (z * z));
    } else { /* J02 = -fx x / z^2 */
      gp[0] += GJ[2] * (-fx / (z * z));
      gp[2] += GJ[2] * (2 * fx * x / (z * z * z));
    }
    if (o.clamp_v) {
      gp[2] += GJ[5] * (fy * o.vc / (z * z));
    } else {
      gp[1] += GJ[5] * (-fy / (z * z));
      gp[2] += GJ[5] * (2 * fy * y / (z * z * z));
    }
    /* mean2d = (fx x/z + cx, fy y/z + cy) */
    gp[0] += gg[0] * fx / z;
    gp[1] += gg[1] * fy / z;
    gp[2] += gg[0] * (-fx * x / (z * z)) + gg[1] * (-fy * y / (z * z));
    /* depth gamma = z */
    gp[2] += gg[6];
    /* p = R_cam mu + t */
    for (int c2 = 0; c2 < 3; ++c2)
      g_means[3 * i + c2] += Rc[c2] * gp[0] + Rc[3 + c2] * gp[1] + Rc[6 + c2] * gp[2];
    /* Sigma = M M^T, M = Rq diag(s): dL/dM = 2 GS M (GS symmetric) */
    double M[9], GM[9];
    for (int r = 0; r < 3; ++r)
      for (int c2 = 0; c2 < 3; ++c2) M[3 * r + c2] = o.Rq[3 * r + c2] * o.s[c2];
    for (int r = 0; r < 3; ++r)
      for (int c2 = 0; c2 < 3; ++c2) {
        double acc = 0;
        for (int m = 0; m < 3; ++m) acc += (GS[3 * r + m] + GS[3 * m + r]) * M[3 * m + c2];
        GM[3 * r + c2] = acc;
      }
    double gR[9];
    for (int c2 = 0; c2 < 3; ++c2) {
      double gs = 0;
      for (int r = 0; r < 3; ++r) {
        gs += GM[3 * r + c2] * o.Rq[3 * r + c2];
        gR[3 * r + c2] = GM[3 * r + c2] * o.s[c2];
      }
      g_log_scales[3 * i + c2] += gs * o.s[c2];
    }
    /* rotation entries as functions of the unit quaternion */
    double w = o.qn[0], qx = o.qn[1], qy = o.qn[2], qz = o.qn[3];
    double gq[4];
    gq[0] = gR[1] * (-2 * qz) + gR[2] * (2 * qy) + gR[3] * (2 * qz) + gR[5] * (-2 * qx) +
            gR[6] * (-2 * qy) + gR[7] * (2 * qx);
    gq[1] = gR[1] * (2 * qy) + gR[2] * (2 * qz) + gR[3] * (2 * qy) + gR[4] * (-4 * qx) +
            gR[5] * (-2 * w) + gR[6] * (2 * qz) + gR[7] * (2 * w) + gR[8] * (-4 * qx);
    gq[2] = gR[0] * (-4 * qy) + gR[1] * (2 * qx) + gR[2] * (2 * w) + gR[3] * (2 * qx) +
            gR[5] * (2 * qz) + gR[6] * (-2 * w) + gR[7] * (2 * qz) + gR[8] * (-4 * qy);
    gq[3] = gR[0] * (-4 * qz) + gR[1] * (-2 * w) + gR[2] * (2 * qx) + gR[3] * (2 * w) +
            gR[4] * (-4 * qz) + gR[5] * (2 * qy) + gR[6] * (2 * qx) + gR[7] * (2 * qy);
    /* q_hat = q / |q| */
    double dot = w * gq[0] + qx * gq[1] + qy * gq[2] + qz * gq[3];
    for (int c2 = 0; c2 < 4; ++c2) g_quats[4 * i + c2] += (gq[c2] - o.qn[c2] * dot) / o.qlen;
  }
}

/* ---------------------------------------------------------------------------------
 * eq16 per view: w_c mean|C - C*| + w_d mean_px([D* > 0] |D - D*|)
 * + w_s (1 - mean SSIM(C, C*)); SSIM with an 11x11 Gaussian window (sigma 1.5),
 * C1 = 0.01^2, C2 = 0.03^2, zero padding, mean over the 3 H W samples.
 * Direct (non-separable) window sums.  Returns the loss; writes dC, dD. */
double or_loss(int W, int H, const double *C, const double *D, const double *Cg,
               const double *Dg, double w_c, double w_d, double w_s, double *dC, double *dD) {
  const int64_t HW = (int64_t)W * H;
  double loss = 0;
  double l1c = 0, l1d = 0;
  for (int64_t i = 0; i < 3 * HW; ++i) {
    double d = C[i] - Cg[i];
    l1c += fabs(d);
    dC[i] = w_c * (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / (3.0 * HW);
  }
  for (int64_t i = 0; i < HW; ++i) {
    double d = D[i] - Dg[i];
    int valid = Dg[i] > 0;
    if (valid) l1d += fabs(d);
    dD[i] = valid ? w_d * (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / (double)HW : 0.0;
  }
  loss += w_c * l1c / (3.0 * HW) + w_d * l1d / (double)HW;
  if (w_s != 0) {
    double g1[11], gs = 0;
    for (int i = 0; i < 11; ++i) {
      g1[i] = exp(-(double)((i - 5) * (i - 5)) / (2 * 1.5 * 1.5));
      gs += g1[i];
    }
    for (int i = 0; i < 11; ++i) g1[i] /= gs;
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    double *m1 = (double *)malloc(sizeof(double) * HW), *m2 = (double *)malloc(sizeof(double) * HW);
    double *s11 = (double *)malloc(sizeof(double) * HW), *s22 = (double *)malloc(sizeof(double) * HW);
    double *s12 = (double *)malloc(sizeof(double) * HW);
    double *dm1 = (double *)malloc(sizeof(double) * HW), *ds11 = (double *)malloc(sizeof(double) * HW);
    double *ds12 = (double *)malloc(sizeof(double) * HW);
    double ssim_sum = 0;
    const double dS = -w_s / (3.0 * HW); /* dL / dSSIM(q) */
    for (int ch = 0; ch < 3; ++ch) {
      const double *X = C + ch * HW, *Y = Cg + ch * HW;
#pragma omp parallel for schedule(static) reduction(+ : ssim_sum)
      for (int64_t q = 0; q < HW; ++q) {
        int qx = (int)(q % W), qy = (int)(q / W);
        double a1 = 0, a2 = 0, a11 = 0, a22 = 0, a12 = 0;
        for (int j = -5; j <= 5; ++j)
          for (int i = -5; i <= 5; ++i) {
            int xx = qx + i, yy = qy + j;
            if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
            double w = g1[i + 5] * g1[j + 5];
            double xv = X[(int64_t)yy * W + xx], yv = Y[(int64_t)yy * W + xx];
            a1 += w * xv; a2 += w * yv; a11 += w * xv * xv; a22 += w * yv * yv; a12 += w * xv * yv;
          }
        m1[q] = a1; m2[q] = a2; s11[q] = a11; s22[q] = a22; s12[q] = a12;
        double sx = a11 - a1 * a1, sy = a22 - a2 * a2, sxy = a12 - a1 * a2;
        double A1 = 2 * a1 * a2 + C1, A2 = 2 * sxy + C2;
        double B1 = a1 * a1 + a2 * a2 + C1, B2 = sx + sy + C2;
        double S = A1 * A2 / (B1 * B2);
        ssim_sum += S;
        /* partial derivatives of S w.r.t. the window sums of x (m1, s11, s12) */
        dm1[q] = dS * ((2 * a2 * A2 - 2 * a2 * A1) / (B1 * B2) - S * (2 * a1 / B1 - 2 * a1 / B2));
        ds11[q] = dS * (-S / B2);
        ds12[q] = dS * (2 * A1 / (B1 * B2));
      }
#pragma omp parallel for schedule(static)
      for (int64_t p = 0; p < HW; ++p) {
        int px = (int)(p % W), py = (int)(p / W);
        double acc = 0;
        double xv = X[p], yv = Y[p];
        for (int j = -5; j <= 5; ++j)
          for (int i = -5; i <= 5; ++i) {
            int xx = px + i, yy = py + j;
            if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
            int64_t q = (int64_t)yy * W + xx;
            double w = g1[i + 5] * g1[j + 5];
            acc += w * (dm1[q] + 2 * xv * ds11[q] + yv * ds12[q]);
          }
        dC[ch * HW + p] += acc;
      }
    }
    loss += w_s * (1 - ssim_sum / (3.0 * HW));
    free(m1); free(m2); free(s11); free(s22); free(s12); free(dm1); free(ds11); free(ds12);
  }
  return loss;
}

/* eq15 with the per-Gaussian reading: s = exp(log_scale),
 * L = (1/n) sum_i (|s_i1 - m_i| + |s_i2 - m_i|) + (1/n) sum_i |s_i3|, m_i = (s_i1 + s_i2)/2.
 * Adds weight * dL/dlog_scale to g_log_scales; returns weight * L. */
double or_scale_reg(int64_t n, const double *log_scales, double weight, double *g_log_scales) {
  if (n <= 0) return 0;
  double L = 0;
  for (int64_t i = 0; i < n; ++i) {
    double s1 = exp(log_scales[3 * i]), s2 = exp(log_scales[3 * i + 1]), s3 = exp(log_scales[3 * i + 2]);
    double m = 0.5 * (s1 + s2);
    L += fabs(s1 - m) + fabs(s2 - m) + fabs(s3);
    /* d/ds1 |s1 - m| + |s2 - m| = 0.5 sgn(s1 - m) - 0.5 sgn(s2 - m) */
    double sg1 = (s1 - m > 0) ? 1.0 : (s1 - m < 0 ? -1.0 : 0.0);
    double sg2 = (s2 - m > 0) ? 1.0 : (s2 - m < 0 ? -1.0 : 0.0);
    double d1 = 0.5 * sg1 - 0.5 * sg2;
    double d2 = 0.5 * sg2 - 0.5 * sg1;
    double d3 = s3 > 0 ? 1.0 : 0.0;
    g_log_scales[3 * i] += weight * d1 * s1 / (double)n;
    g_log_scales[3 * i + 1] += weight * d2 * s2 / (double)n;
    g_log_scales[3 * i + 2] += weight * d3 * s3 / (double)n;
  }
  return weight * L / (double)n;
}

/* Bias-corrected Adam on a flat parameter array (one learning rate). */
void or_adam(int64_t n, double *p, const double *g, double *m, double *v, double lr, double b1,
             double b2, double eps, int32_t t) {
  double c1 = 1 - pow(b1, t), c2 = 1 - pow(b2, t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1 - b1) * g[i];
    v[i] = b2 * v[i] + (1 - b2) * g[i] * g[i];
    double mh = m[i] / c1, vh = v[i] / c2;
    p[i] -= lr * mh / (sqrt(vh) + eps);
  }
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the OpenMP regions above (the timed baseline runs on all host cores
 * and on one); returns the previous setting. */
int or_set_num_threads(int n) {
#ifdef _OPENMP
  int old = omp_get_max_threads();
  if (n >= 1) omp_set_num_threads(n);
  return old;
#else
  (void)n;
  return 1;
#endif
}
