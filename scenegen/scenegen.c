/*
 * scenegen.c -- seeded synthetic scenes and range scans (input generation only).
 *
 * This file holds no arithmetic of the integration method: it builds procedural
 * scenes (inside-out rooms, axis-aligned boxes, spheres, a bilinear terrain
 * heightfield), casts sensor rays into them (pinhole depth camera or spherical
 * LiDAR), adds seeded noise and dropout, and evaluates the scene's analytic
 * signed distance.  The scans it writes are the inputs that both the CPU oracle
 * and the CUDA path consume, and the analytic distance is the ground truth for
 * the SDF RMSE metric.
 *
 * Randomness is counter based (splitmix64 finaliser of seed, scan and pixel
 * counters), so a scan is the same whatever the thread count or machine.
 * All geometry is FP64; output points are rounded once to float32.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { SG_ROOM = 0, SG_BOX = 1, SG_SPHERE = 2 };

typedef struct {
  int type;
  double p[6]; /* ROOM/BOX: min xyz, max xyz.  SPHERE: centre xyz, radius */
} sg_prim;

typedef struct {
  int n;
  sg_prim* prims;
  /* terrain: heights th[j*tnx + i] at (tx0 + i*tres, ty0 + j*tres) */
  int has_terrain, tnx, tny;
  double tx0, ty0, tres, tmaxh;
  double* th;
  /* uniform xy grid over the small primitives (boxes, spheres) */
  int gnx, gny;
  double gx0, gy0, gres, gzmin, gzmax;
  int* cell_start; /* gnx*gny + 1 */
  int* cell_items;
  int nbig;
  int* big; /* primitives traced for every ray (rooms, very large boxes) */
} sg_scene;

/* ------------------------------------------------------------------ RNG */
static inline uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static inline double u01(uint64_t seed, uint64_t a, uint64_t b, uint64_t c) {
  uint64_t h = mix64(seed ^ mix64(a ^ mix64(b ^ mix64(c))));
  return ((double)(h >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}
static inline double gauss(uint64_t seed, uint64_t a, uint64_t b) {
  double u1 = u01(seed, a, b, 11), u2 = u01(seed, a, b, 12);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* ---------------------------------------------------- primitive tracing */
/* slab test; returns entry/exit params in *tn, *tf; 0 if the line misses */
static int slab(const double* mn, const double* mx, const double* o, const double* d,
                double* tn, double* tf) {
  double t0 = -INFINITY, t1 = INFINITY;
  for (int k = 0; k < 3; ++k) {
    if (d[k] == 0.0) {
      if (o[k] < mn[k] || o[k] > mx[k]) return 0;
    } else {
      double inv = 1.0 / d[k];
      double a = (mn[k] - o[k]) * inv, b = (mx[k] - o[k]) * inv;
      if (a > b) { double t = a; a = b; b = t; }
      if (a > t0) t0 = a;
      if (b < t1) t1 = b;
    }
  }
  *tn = t0;
  *tf = t1;
  return t0 <= t1;
}

static double trace_prim(const sg_prim* q, const double* o, const double* d) {
  double tn, tf;
  if (q->type == SG_ROOM) {
    if (!slab(q->p, q->p + 3, o, d, &tn, &tf)) return INFINITY;
    return tf > 0 ? tf : INFINITY;
  } else if (q->type == SG_BOX) {
    if (!slab(q->p, q->p + 3, o, d, &tn, &tf)) return INFINITY;
    if (tf <= 0) return INFINITY;
    return tn > 0 ? tn : 0.0;
  } else {
    double oc[3] = {o[0] - q->p[0], o[1] - q->p[1], o[2] - q->p[2]};
    double b = oc[0] * d[0] + oc[1] * d[1] + oc[2] * d[2];
    double c = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - q->p[3] * q->p[3];
    double disc = b * b - c;
    if (disc < 0) return INFINITY;
    double s = sqrt(disc);
    double t = -b - s;
    if (t > 0) return t;
    t = -b + s;
    return t > 0 ? 0.0 : INFINITY;
  }
}

/* ------------------------------------------------------------- terrain */
static inline double th_at(const sg_scene* s, int i, int j) {
  if (i < 0) i = 0;
  if (j < 0) j = 0;
  if (i >= s->tnx) i = s->tnx - 1;
  if (j >= s->tny) j = s->tny - 1;
  return s->th[(size_t)j * s->tnx + i];
}

static double terrain_h(const sg_scene* s, double x, double y, double* gx, double* gy) {
  double fx = (x - s->tx0) / s->tres, fy = (y - s->ty0) / s->tres;
  int i = (int)floor(fx), j = (int)floor(fy);
  double a = fx - i, b = fy - j;
  if (i < 0) { i = 0; a = 0; }
  if (j < 0) { j = 0; b = 0; }
  if (i >= s->tnx - 1) { i = s->tnx - 2; a = 1; }
  if (j >= s->tny - 1) { j = s->tny - 2; b = 1; }
  double h00 = th_at(s, i, j), h10 = th_at(s, i + 1, j), h01 = th_at(s, i, j + 1),
         h11 = th_at(s, i + 1, j + 1);
  if (gx) *gx = ((h10 - h00) * (1 - b) + (h11 - h01) * b) / s->tres;
  if (gy) *gy = ((h01 - h00) * (1 - a) + (h11 - h10) * a) / s->tres;
  return h00 * (1 - a) * (1 - b) + h10 * a * (1 - b) + h01 * (1 - a) * b + h11 * a * b;
}

/* first terrain hit in [0, tbest); walks the heightfield cells along the ray
 * and solves the bilinear patch (quadratic in t) exactly in each cell */
static double trace_terrain(const sg_scene* s, const double* o, const double* d, double tbest) {
  double fx = (o[0] - s->tx0) / s->tres, fy = (o[1] - s->ty0) / s->tres;
  double dx = d[0] / s->tres, dy = d[1] / s->tres;
  int i = (int)floor(fx), j = (int)floor(fy);
  if (i < 0 || j < 0 || i >= s->tnx - 1 || j >= s->tny - 1) return INFINITY;
  int sx = dx > 0 ? 1 : (dx < 0 ? -1 : 0), sy = dy > 0 ? 1 : (dy < 0 ? -1 : 0);
  double tdx = sx ? fabs(1.0 / dx) : INFINITY, tdy = sy ? fabs(1.0 / dy) : INFINITY;
  double tmx = sx > 0 ? (i + 1 - fx) / dx : (sx < 0 ? (i - fx) / dx : INFINITY);
  double tmy = sy > 0 ? (j + 1 - fy) / dy : (sy < 0 ? (j - fy) / dy : INFINITY);
  double tin = 0.0;
  for (int it = 0; it < 100000; ++it) {
    double tout = tmx < tmy ? tmx : tmy;
    if (tout > tbest) tout = tbest;
    double zin = o[2] + d[2] * tin;
    if (zin > s->tmaxh && d[2] >= 0) return INFINITY;
    /* local patch coordinates at t=0 relative to this cell */
    double s0 = fx - i, r0 = fy - j;
    double h00 = th_at(s, i, j), h10 = th_at(s, i + 1, j), h01 = th_at(s, i, j + 1),
           h11 = th_at(s, i + 1, j + 1);
    double e1 = h10 - h00, e2 = h01 - h00, e3 = h00 - h10 - h01 + h11;
    double c0 = h00 + e1 * s0 + e2 * r0 + e3 * s0 * r0;
    double c1 = e1 * dx + e2 * dy + e3 * (s0 * dy + r0 * dx);
    double c2 = e3 * dx * dy;
    /* f(t) = o_z + d_z t - h(t) */
    double A = -c2, B = d[2] - c1, C = o[2] - c0;
    double fin = A * tin * tin + B * tin + C;
    if (fin <= 0) return tin;
    double best = INFINITY;
    if (fabs(A) < 1e-14) {
      if (B != 0) {
        double t = -C / B;
        if (t >= tin && t <= tout) best = t;
      }
    } else {
      double disc = B * B - 4 * A * C;
      if (disc >= 0) {
        double sq = sqrt(disc);
        double q = -0.5 * (B + (B >= 0 ? sq : -sq));
        double t1 = q / A, t2 = (q != 0) ? C / q : INFINITY;
        if (t1 >= tin && t1 <= tout && t1 < best) best = t1;
        if (t2 >= tin && t2 <= tout && t2 < best) best = t2;
      }
    }
    if (best < INFINITY) return best;
    if (tout >= tbest) return INFINITY;
    tin = tout;
    if (tmx < tmy) { i += sx; tmx += tdx; } else { j += sy; tmy += tdy; }
    if (i < 0 || j < 0 || i >= s->tnx - 1 || j >= s->tny - 1) return INFINITY;
  }
  return INFINITY;
}

/* ---------------------------------------------------------- scene build */
sg_scene* sg_scene_create(const int* types, const double* params, int n, const double* heights,
                          int tnx, int tny, double tx0, double ty0, double tres, double grid_res) {
  sg_scene* s = (sg_scene*)calloc(1, sizeof(sg_scene));
  s->n = n;
  s->prims = (sg_prim*)malloc(sizeof(sg_prim) * (n > 0 ? n : 1));
  for (int k = 0; k < n; ++k) {
    s->prims[k].type = types[k];
    memcpy(s->prims[k].p, params + 6 * k, 6 * sizeof(double));
  }
  if (heights && tnx >= 2 && tny >= 2) {
    s->has_terrain = 1;
    s->tnx = tnx; s->tny = tny; s->tx0 = tx0; s->ty0 = ty0; s->tres = tres;
    s->th = (double*)malloc(sizeof(double) * (size_t)tnx * tny);
    memcpy(s->th, heights, sizeof(double) * (size_t)tnx * tny);
    s->tmaxh = -INFINITY;
    for (size_t q = 0; q < (size_t)tnx * tny; ++q)
      if (s->th[q] > s->tmaxh) s->tmaxh = s->th[q];
  }
  /* grid over small primitives */
  double mn[2] = {INFINITY, INFINITY}, mx[2] = {-INFINITY, -INFINITY};
  s->gzmin = INFINITY; s->gzmax = -INFINITY;
  s->big = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  int nsmall = 0;
  for (int k = 0; k < n; ++k) {
    const sg_prim* q = &s->prims[k];
    double lo[3], hi[3];
    if (q->type == SG_SPHERE) {
      for (int a = 0; a < 3; ++a) { lo[a] = q->p[a] - q->p[3]; hi[a] = q->p[a] + q->p[3]; }
    } else {
      for (int a = 0; a < 3; ++a) { lo[a] = q->p[a]; hi[a] = q->p[3 + a]; }
    }
    int big = q->type == SG_ROOM || (hi[0] - lo[0]) > 8 * grid_res || (hi[1] - lo[1]) > 8 * grid_res;
    if (big) { s->big[s->nbig++] = k; continue; }
    ++nsmall;
    if (lo[0] < mn[0]) mn[0] = lo[0];
    if (lo[1] < mn[1]) mn[1] = lo[1];
    if (hi[0] > mx[0]) mx[0] = hi[0];
    if (hi[1] > mx[1]) mx[1] = hi[1];
    if (lo[2] < s->gzmin) s->gzmin = lo[2];
    if (hi[2] > s->gzmax) s->gzmax = hi[2];
  }
  s->gres = grid_res;
  if (nsmall == 0) {
    s->gnx = s->gny = 1; s->gx0 = s->gy0 = 0;
    s->cell_start = (int*)calloc(2, sizeof(int));
    s->cell_items = (int*)malloc(sizeof(int));
    return s;
  }
  s->gx0 = mn[0] - 1e-6; s->gy0 = mn[1] - 1e-6;
  s->gnx = (int)ceil((mx[0] - s->gx0) / grid_res) + 1;
  s->gny = (int)ceil((mx[1] - s->gy0) / grid_res) + 1;
  int ncell = s->gnx * s->gny;
  int* cnt = (int*)calloc((size_t)ncell + 1, sizeof(int));
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      s->cell_start = (int*)malloc(sizeof(int) * ((size_t)ncell + 1));
      s->cell_start[0] = 0;
      for (int c = 0; c < ncell; ++c) s->cell_start[c + 1] = s->cell_start[c] + cnt[c];
      s->cell_items = (int*)malloc(sizeof(int) * (s->cell_start[ncell] > 0 ? s->cell_start[ncell] : 1));
      memset(cnt, 0, sizeof(int) * ncell);
    }
    for (int k = 0; k < n; ++k) {
      const sg_prim* q = &s->prims[k];
      int isbig = 0;
      for (int b = 0; b < s->nbig; ++b) if (s->big[b] == k) { isbig = 1; break; }
      if (isbig) continue;
      double lo[2], hi[2];
      if (q->type == SG_SPHERE) {
        lo[0] = q->p[0] - q->p[3]; hi[0] = q->p[0] + q->p[3];
        lo[1] = q->p[1] - q->p[3]; hi[1] = q->p[1] + q->p[3];
      } else {
        lo[0] = q->p[0]; hi[0] = q->p[3]; lo[1] = q->p[1]; hi[1] = q->p[4];
      }
      int i0 = (int)floor((lo[0] - s->gx0) / grid_res), i1 = (int)floor((hi[0] - s->gx0) / grid_res);
      int j0 = (int)floor((lo[1] - s->gy0) / grid_res), j1 = (int)floor((hi[1] - s->gy0) / grid_res);
      for (int j = j0; j <= j1; ++j)
        for (int i = i0; i <= i1; ++i) {
          if (i < 0 || j < 0 || i >= s->gnx || j >= s->gny) continue;
          int c = j * s->gnx + i;
          if (pass == 1) s->cell_items[s->cell_start[c] + cnt[c]] = k;
          cnt[c]++;
        }
    }
  }
  free(cnt);
  return s;
}

void sg_scene_destroy(sg_scene* s) {
  if (!s) return;
  free(s->prims); free(s->th); free(s->cell_start); free(s->cell_items); free(s->big);
  free(s);
}

/* nearest hit along unit direction d within tmax; INFINITY if none */
static double trace(const sg_scene* s, const double* o, const double* d, double tmax) {
  double tbest = tmax;
  for (int b = 0; b < s->nbig; ++b) {
    double t = trace_prim(&s->prims[s->big[b]], o, d);
    if (t < tbest) tbest = t;
  }
  if (s->cell_start[s->gnx * s->gny] > 0) {
    /* clip to the grid's bounding box, then 2-D DDA over cells */
    double mn[3] = {s->gx0, s->gy0, s->gzmin}, mx[3] = {s->gx0 + s->gnx * s->gres,
                                                       s->gy0 + s->gny * s->gres, s->gzmax};
    double tn, tf;
    if (slab(mn, mx, o, d, &tn, &tf) && tf > 0 && tn < tbest) {
      double t0 = tn > 0 ? tn : 0;
      double px = o[0] + d[0] * t0, py = o[1] + d[1] * t0;
      double fx = (px - s->gx0) / s->gres, fy = (py - s->gy0) / s->gres;
      int i = (int)floor(fx), j = (int)floor(fy);
      if (i >= s->gnx) i = s->gnx - 1;
      if (j >= s->gny) j = s->gny - 1;
      if (i < 0) i = 0;
      if (j < 0) j = 0;
      double dx = d[0] / s->gres, dy = d[1] / s->gres;
      int sx = dx > 0 ? 1 : (dx < 0 ? -1 : 0), sy = dy > 0 ? 1 : (dy < 0 ? -1 : 0);
      double tdx = sx ? fabs(1.0 / dx) : INFINITY, tdy = sy ? fabs(1.0 / dy) : INFINITY;
      double tmx = sx > 0 ? t0 + (i + 1 - fx) / dx : (sx < 0 ? t0 + (i - fx) / dx : INFINITY);
      double tmy = sy > 0 ? t0 + (j + 1 - fy) / dy : (sy < 0 ? t0 + (j - fy) / dy : INFINITY);
      double tin = t0;
      while (tin < tbest && tin <= tf) {
        int c = j * s->gnx + i;
        for (int q = s->cell_start[c]; q < s->cell_start[c + 1]; ++q) {
          double t = trace_prim(&s->prims[s->cell_items[q]], o, d);
          if (t < tbest) tbest = t;
        }
        if (tmx < tmy) { tin = tmx; i += sx; tmx += tdx; }
        else { tin = tmy; j += sy; tmy += tdy; }
        if (i < 0 || j < 0 || i >= s->gnx || j >= s->gny) break;
        if (!sx && !sy) break;
      }
    }
  }
  if (s->has_terrain) {
    double t = trace_terrain(s, o, d, tbest);
    if (t < tbest) tbest = t;
  }
  return tbest;
}

/* ----------------------------------------------------------- SDF eval */
static double prim_sdf(const sg_prim* q, const double* x) {
  if (q->type == SG_SPHERE) {
    double a = x[0] - q->p[0], b = x[1] - q->p[1], c = x[2] - q->p[2];
    return sqrt(a * a + b * b + c * c) - q->p[3];
  }
  double c[3], h[3], e[3];
  for (int k = 0; k < 3; ++k) {
    c[k] = 0.5 * (q->p[k] + q->p[3 + k]);
    h[k] = 0.5 * (q->p[3 + k] - q->p[k]);
    e[k] = fabs(x[k] - c[k]) - h[k];
  }
  double out2 = 0, mx = -INFINITY;
  for (int k = 0; k < 3; ++k) {
    if (e[k] > 0) out2 += e[k] * e[k];
    if (e[k] > mx) mx = e[k];
  }
  double box = sqrt(out2) + (mx < 0 ? mx : 0); /* positive outside the box */
  return q->type == SG_ROOM ? -box : box;
}

/* scene signed distance (positive in free space), clamped to [-cap, cap] */
void sg_sdf(const sg_scene* s, const double* pts, int64_t n, double cap, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < n; ++q) {
    const double* x = pts + 3 * q;
    double best = cap;
    for (int b = 0; b < s->nbig; ++b) {
      double v = prim_sdf(&s->prims[s->big[b]], x);
      if (v < best) best = v;
    }
    if (s->cell_start[s->gnx * s->gny] > 0) {
      int i = (int)floor((x[0] - s->gx0) / s->gres), j = (int)floor((x[1] - s->gy0) / s->gres);
      int reach = (int)ceil(cap / s->gres) + 1;
      for (int jj = j - reach; jj <= j + reach; ++jj)
        for (int ii = i - reach; ii <= i + reach; ++ii) {
          if (ii < 0 || jj < 0 || ii >= s->gnx || jj >= s->gny) continue;
          int c = jj * s->gnx + ii;
          for (int k = s->cell_start[c]; k < s->cell_start[c + 1]; ++k) {
            double v = prim_sdf(&s->prims[s->cell_items[k]], x);
            if (v < best) best = v;
          }
        }
    }
    if (s->has_terrain) {
      double gx, gy;
      double h = terrain_h(s, x[0], x[1], &gx, &gy);
      double v = (x[2] - h) / sqrt(1.0 + gx * gx + gy * gy);
      if (v < best) best = v;
    }
    if (best < -cap) best = -cap;
    out[q] = best;
  }
}

/* ------------------------------------------------------------ sensors */
/* pinhole depth camera.  Sensor frame: z along the optical axis, x right, y down.
 * noise_kind 0: none, 1: Gaussian along the ray (sigma metres),
 * 2: axial Gaussian with sigma = noise_k * z^2.  Dropped or missing pixels are NaN.
 * T_ws: world <- sensor, 3x4 row-major (FP64).  Returns the number of valid pixels. */
int64_t sg_render_pinhole(const sg_scene* s, const double* T, int W, int H, double fx, double fy,
                          double cx, double cy, double max_depth, int noise_kind, double noise_k,
                          double dropout, uint64_t seed, uint64_t scan_id, float* out) {
  int64_t valid = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : valid)
  for (int v = 0; v < H; ++v) {
    for (int u = 0; u < W; ++u) {
      float* P = out + 3 * ((int64_t)v * W + u);
      double dc[3] = {(u - cx) / fx, (v - cy) / fy, 1.0};
      double nrm = sqrt(dc[0] * dc[0] + dc[1] * dc[1] + 1.0);
      double dw[3], o[3] = {T[3], T[7], T[11]};
      for (int k = 0; k < 3; ++k)
        dw[k] = (T[4 * k] * dc[0] + T[4 * k + 1] * dc[1] + T[4 * k + 2] * dc[2]) / nrm;
      double t = trace(s, o, dw, max_depth * nrm * 1.5);
      double z = t / nrm;
      uint64_t pix = (uint64_t)v * W + u;
      int ok = isfinite(t) && z <= max_depth && z > 0;
      if (ok && dropout > 0 && u01(seed, scan_id, pix, 3) < dropout) ok = 0;
      if (!ok) { P[0] = P[1] = P[2] = NAN; continue; }
      if (noise_kind == 1) z = (t + noise_k * gauss(seed, scan_id, pix)) / nrm;
      else if (noise_kind == 2) z = z + noise_k * z * z * gauss(seed, scan_id, pix);
      P[0] = (float)(dc[0] * z); P[1] = (float)(dc[1] * z); P[2] = (float)z;
      ++valid;
    }
  }
  return valid;
}

/* spherical LiDAR: rows span elevation el_max (row 0) .. el_min (last row),
 * columns azimuth 2*pi*c/cols.  Sensor frame: x forward, z up.  Gaussian noise
 * sigma along the ray; no return within max_range gives NaN. */
int64_t sg_render_lidar(const sg_scene* s, const double* T, int rows, int cols, double el_min,
                        double el_max, double max_range, double sigma, uint64_t seed,
                        uint64_t scan_id, float* out) {
  int64_t valid = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : valid)
  for (int r = 0; r < rows; ++r) {
    double el = rows > 1 ? el_max + (el_min - el_max) * r / (rows - 1) : 0.5 * (el_min + el_max);
    for (int c = 0; c < cols; ++c) {
      float* P = out + 3 * ((int64_t)r * cols + c);
      double az = 6.283185307179586 * c / cols;
      double ds[3] = {cos(el) * cos(az), cos(el) * sin(az), sin(el)};
      double dw[3], o[3] = {T[3], T[7], T[11]};
      for (int k = 0; k < 3; ++k) dw[k] = T[4 * k] * ds[0] + T[4 * k + 1] * ds[1] + T[4 * k + 2] * ds[2];
      double t = trace(s, o, dw, max_range);
      uint64_t pix = (uint64_t)r * cols + c;
      if (!(t < max_range) || t <= 0) { P[0] = P[1] = P[2] = NAN; continue; }
      if (sigma > 0) t += sigma * gauss(seed, scan_id, pix);
      P[0] = (float)(ds[0] * t); P[1] = (float)(ds[1] * t); P[2] = (float)(ds[2] * t);
      ++valid;
    }
  }
  return valid;
}

/* trace arbitrary world rays (used by trajectory planning and tests) */
void sg_trace_rays(const sg_scene* s, const double* o, const double* d, int64_t n, double tmax,
                   double* t_out) {
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < n; ++q) t_out[q] = trace(s, o + 3 * q, d + 3 * q, tmax);
}

double sg_terrain_height(const sg_scene* s, double x, double y) {
  return s->has_terrain ? terrain_h(s, x, y, 0, 0) : 0.0;
}
