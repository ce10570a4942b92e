/*
 * oracle.cpp -- TEST INFRASTRUCTURE ONLY.  A plain, slow, obviously correct CPU
 * statement of projective TSDF integration into block-hashed submaps.  Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg load it; the
 * product path never does.  It shares no code with the CUDA library.
 *
 * What it computes (coVoxSLAM, Sec. III-C "TSDF Representation" and Sec. III-D
 * "Point cloud Integration"):
 *   - every valid point of a scan is used (Sec. III-C, raycasting paragraph);
 *   - each point's ray is traversed over the band [-trunc, +trunc] around the
 *     point (raycasting from the optical centre, restricted to the truncation
 *     band), voxel by voxel with an Amanatides-Woo traversal; with carving,
 *     from the optical centre itself to trunc behind the point;
 *   - the voxels are grouped in 8^3 blocks indexed by their integer 3-D
 *     position (Sec. III-C, "indexed by their 3D position");
 *   - per scan, the weighted distances of all observations of a voxel are
 *     summed (the sums are commutative, Sec. III-D processing phase) and then
 *     merged into the stored voxel as D <- (D W + S_wd) / (W + S_w),
 *     W <- min(W + S_w, max_weight);
 *   - weights are constant, 1/z^2, or given per point, optionally with a
 *     behind-surface drop-off (Sec. III-C, weighting paragraph);
 *   - with colours given per point, every voxel also fuses an RGB colour with
 *     the same observation weights and the same merge rule,
 *     C <- (C W + S_wc) / (W + S_w) (the "TSDF + Color" integration timed in
 *     Sec. IV); a point with a non-finite colour channel is invalid, like one
 *     with an unusable per-point weight.
 *
 * Precision: distances, weights, sums and stored D/W are FP64.  The traversal
 * itself is FP32 with a fixed operation order (the same FP32 formula the CUDA
 * path uses, written here independently) so that touched voxel and block sets
 * can be compared bit-exactly.  Storage is a std::map keyed by the block's
 * integer coordinates: no hashing.  An optional FP16 storage mode rounds the
 * stored D / trunc and W to IEEE half (round to nearest even) after every merge.
 *
 * Build: g++ -O2 -std=c++17 -ffp-contract=off (never -ffast-math): the FP32
 * traversal must not be contracted into FMAs.
 */
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <map>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace {

constexpr int kBlock = 8;            // voxels per block edge (Sec. III-E: n = 8)
constexpr int kBlockVox = 512;       // 8^3
constexpr float kKeyLimit = 8388608.0f;  // 2^23 voxels = 2^20 blocks per axis

using Key = std::array<int32_t, 3>;

struct Block {
  double D[kBlockVox];
  double W[kBlockVox];
  double C[3][kBlockVox];   // fused RGB (zero unless scans carried colours)
};

struct Map {
  float vs, trunc, max_w;
  int fp16;
  std::map<Key, Block> blocks;
};

inline int32_t floor_div8(int32_t v) { return v >= 0 ? v / 8 : -((-v + 7) / 8); }
inline int32_t mod8(int32_t v) { return v - 8 * floor_div8(v); }

/* ---- FP32 point transform and band traversal (fixed operation order) ---- */
struct Ray {
  float p[3];      // point in the submap frame
  float o[3];      // sensor origin in the submap frame
  float len;       // |p - o|
  float u[3];      // unit direction
};

// p = R ps + t, each row summed left to right; r = p - o with o = t.
// A pinhole depth sensor only returns points in front of it (z > 0).
bool make_ray(const float* ps, const float* T, float min_range, float max_range, int sensor,
              Ray* ray) {
  if (!(std::isfinite(ps[0]) && std::isfinite(ps[1]) && std::isfinite(ps[2]))) return false;
  if (sensor == 0 && !(ps[2] > 0.0f)) return false;
  for (int k = 0; k < 3; ++k) {
    float a = T[4 * k + 0] * ps[0];
    float b = T[4 * k + 1] * ps[1];
    float c = T[4 * k + 2] * ps[2];
    float s = a + b;
    s = s + c;
    ray->p[k] = s + T[4 * k + 3];
    ray->o[k] = T[4 * k + 3];
  }
  float r[3];
  for (int k = 0; k < 3; ++k) r[k] = ray->p[k] - ray->o[k];
  float rr = r[0] * r[0];
  rr = rr + r[1] * r[1];
  rr = rr + r[2] * r[2];
  float len = std::sqrt(rr);
  ray->len = len;
  if (!(len >= min_range && len <= max_range)) return false;
  float inv_len = 1.0f / len;
  for (int k = 0; k < 3; ++k) ray->u[k] = r[k] * inv_len;
  return true;
}

// Amanatides-Woo traversal of the segment A -> B given in voxel units.
// Emits floor(A), then one 6-connected step per boundary crossing, ending at
// floor(B).  The axis to step is the one with the smallest tMax among the
// axes not yet at their end index; ties go to the lowest axis (x, y, z).
int traverse(const float* A, const float* B, std::vector<Key>* out) {
  int32_t i[3], i1[3], s[3];
  float tmax[3], tdelta[3];
  int n = 0;
  for (int k = 0; k < 3; ++k) {
    i[k] = (int32_t)std::floor(A[k]);
    i1[k] = (int32_t)std::floor(B[k]);
    float d = B[k] - A[k];
    if (d > 0.0f) {
      s[k] = 1;
      tdelta[k] = 1.0f / d;
      tmax[k] = ((float)(i[k] + 1) - A[k]) * tdelta[k];
    } else if (d < 0.0f) {
      s[k] = -1;
      tdelta[k] = 1.0f / (-d);
      tmax[k] = (A[k] - (float)i[k]) * tdelta[k];
    } else {
      s[k] = 0;
      tdelta[k] = std::numeric_limits<float>::infinity();
      tmax[k] = std::numeric_limits<float>::infinity();
    }
    n += std::abs(i1[k] - i[k]);
  }
  out->push_back({i[0], i[1], i[2]});
  for (int step = 0; step < n; ++step) {
    int best = -1;
    for (int k = 0; k < 3; ++k) {
      if (i[k] == i1[k]) continue;
      if (best < 0 || tmax[k] < tmax[best]) best = k;
    }
    i[best] += s[best];
    tmax[best] = tmax[best] + tdelta[best];
    out->push_back({i[0], i[1], i[2]});
  }
  return n + 1;
}

// Band endpoints a = p - trunc u, b = p + trunc u, scaled by 1/vs.  With
// free-space carving the segment starts at the sensor origin instead
// (a = o: the ray cast from the optical centre, Sec. III-C).
// Returns false if either endpoint leaves the +-2^23 voxel key range.
bool band_segment(const Ray& ray, float trunc, float vs, float* A, float* B, bool carve = false) {
  float inv_vs = 1.0f / vs;
  for (int k = 0; k < 3; ++k) {
    float tu = trunc * ray.u[k];
    float a = carve ? ray.o[k] : ray.p[k] - tu;
    float b = ray.p[k] + tu;
    A[k] = a * inv_vs;
    B[k] = b * inv_vs;
    if (!(A[k] >= -kKeyLimit && A[k] < kKeyLimit && B[k] >= -kKeyLimit && B[k] < kKeyLimit))
      return false;
  }
  return true;
}

/* ---- FP64 distance and weight of one observation ---- */
struct Obs {
  Key v;
  double d, w;
};

// Projective distance of voxel centre c_v to the point along the ray:
// d = (p - c_v) . u, positive on the sensor side, clamped to [-trunc, trunc].
double voxel_distance(const Ray& ray, const Key& v, float vs, float trunc) {
  double r[3], len2 = 0;
  for (int k = 0; k < 3; ++k) {
    r[k] = (double)ray.p[k] - (double)ray.o[k];
    len2 += r[k] * r[k];
  }
  double len = std::sqrt(len2), d = 0;
  for (int k = 0; k < 3; ++k) {
    double c = ((double)v[k] + 0.5) * (double)vs;
    d += ((double)ray.p[k] - c) * (r[k] / len);
  }
  double t = trunc;
  return d > t ? t : (d < -t ? -t : d);
}

// weight_mode: 0 constant 1, 1 quadratic 1/z^2 (z = optical-axis depth for a
// pinhole sensor, range for a spherical one), 2 per-point value.
// dropoff: behind the surface (d < -eps, eps = vs) the weight falls to zero at
// d = -trunc, linearly (1) or with the linear factor squared (2).
double obs_weight(double base, double d, float vs, float trunc, int dropoff) {
  double eps = vs;
  if (dropoff != 0 && d < -eps) {
    double f = ((double)trunc + d) / ((double)trunc - eps);
    if (f < 0) f = 0;
    return dropoff == 1 ? base * f : base * f * f;
  }
  return base;
}

// A per-point weight must be a finite, non-negative number; a point whose
// given weight is not is invalid like a point without a return (it is not
// integrated and allocates nothing).
bool point_weight_ok(const float* pw, int64_t i, int weight_mode) {
  if (weight_mode != 2) return true;
  const float w = pw[i];
  return std::isfinite(w) && w >= 0.0f;
}

// With colours, a point is usable only if all three channels are finite.
bool point_colour_ok(const float* rgb, int64_t i) {
  if (!rgb) return true;
  return std::isfinite(rgb[3 * i]) && std::isfinite(rgb[3 * i + 1]) && std::isfinite(rgb[3 * i + 2]);
}

double base_weight(const float* ps, const Ray& ray, const float* pw, int64_t i, int weight_mode,
                   int sensor) {
  if (weight_mode == 0) return 1.0;
  if (weight_mode == 2) return (double)pw[i];
  double z;
  if (sensor == 0) {
    z = (double)ps[2];
  } else {
    double r2 = 0;
    for (int k = 0; k < 3; ++k) {
      double r = (double)ray.p[k] - (double)ray.o[k];
      r2 += r * r;
    }
    z = std::sqrt(r2);
  }
  return 1.0 / (z * z);
}

inline Key block_of(const Key& v) { return {floor_div8(v[0]), floor_div8(v[1]), floor_div8(v[2])}; }
inline int local_of(const Key& v) { return mod8(v[0]) + 8 * mod8(v[1]) + 64 * mod8(v[2]); }

double round_half(double x) { return (double)(_Float16)x; }

struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = (uint64_t)(uint32_t)k[0] * 0x9E3779B97F4A7C15ull;
    h ^= (uint64_t)(uint32_t)k[1] * 0xC2B2AE3D27D4EB4Full + (h << 6) + (h >> 2);
    h ^= (uint64_t)(uint32_t)k[2] * 0x165667B19E3779F9ull + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};

// Per-frame sums of one voxel: weighted distance, weight, weighted colour.
struct VoxelSums {
  double swd = 0.0, sw = 0.0;
  double swc[3] = {0.0, 0.0, 0.0};
};

void merge_voxel(Map* m, Block& b, int l, const VoxelSums& vs_) {
  const double swd = vs_.swd, sw = vs_.sw;
  double W = b.W[l], D = b.D[l];
  double Wn = W + sw;
  if (!(Wn > 0)) return;
  for (int k = 0; k < 3; ++k) b.C[k][l] = (b.C[k][l] * W + vs_.swc[k]) / Wn;
  double Dn = (D * W + swd) / Wn;
  double Wc = Wn < (double)m->max_w ? Wn : (double)m->max_w;
  if (m->fp16) {
    Dn = round_half(Dn / (double)m->trunc) * (double)m->trunc;
    Wc = round_half(Wc);
  }
  b.D[l] = Dn;
  b.W[l] = Wc;
}

using FrameSums = std::map<Key, VoxelSums>;

struct FrameCounts {
  int64_t valid = 0, nobs = 0, bad = 0;
};

// Observations of points [i0, i1) of one scan, summed per voxel in point
// order into `frame` (weighted distance, weight, and with rgb -- [n,3]
// colours -- weighted colour).
void accumulate_points(const Map* m, const float* pts, int64_t i0, int64_t i1, const float* T,
                       const float* pw, int weight_mode, int dropoff, float min_range,
                       float max_range, int sensor, int carve, const float* rgb, FrameSums* frame,
                       FrameCounts* cnt) {
  std::vector<Key> vox;
  for (int64_t i = i0; i < i1; ++i) {
    const float* ps = pts + 3 * i;
    Ray ray;
    if (!make_ray(ps, T, min_range, max_range, sensor, &ray)) continue;
    if (!point_weight_ok(pw, i, weight_mode)) continue;
    if (!point_colour_ok(rgb, i)) continue;
    float A[3], B[3];
    if (!band_segment(ray, m->trunc, m->vs, A, B, carve != 0)) {
      ++cnt->bad;
      continue;
    }
    ++cnt->valid;
    vox.clear();
    traverse(A, B, &vox);
    double base = base_weight(ps, ray, pw, i, weight_mode, sensor);
    for (const Key& v : vox) {
      double d = voxel_distance(ray, v, m->vs, m->trunc);
      double w = obs_weight(base, d, m->vs, m->trunc, dropoff);
      auto& acc = (*frame)[v];
      acc.swd += w * d;
      acc.sw += w;
      if (rgb)
        for (int k = 0; k < 3; ++k) acc.swc[k] += w * (double)rgb[3 * i + k];
      ++cnt->nobs;
    }
  }
}

// End of a frame: allocate every block an observation fell in (even with zero
// weight), then, unless a point left the key range, merge each voxel's sums.
int apply_frame(Map* m, const FrameSums& frame, const FrameCounts& cnt, int64_t* stats) {
  std::map<Key, int> touched;
  int64_t newb = 0;
  for (auto& kv : frame) {
    Key b = block_of(kv.first);
    if (touched.emplace(b, 1).second && m->blocks.find(b) == m->blocks.end()) {
      Block& blk = m->blocks[b];
      std::memset(&blk, 0, sizeof(Block));
      ++newb;
    }
  }
  if (cnt.bad == 0) {
    for (auto& kv : frame) {
      Block& blk = m->blocks[block_of(kv.first)];
      merge_voxel(m, blk, local_of(kv.first), kv.second);
    }
  }
  if (stats) {
    stats[0] = cnt.valid;
    stats[1] = cnt.nobs;
    stats[2] = (int64_t)frame.size();
    stats[3] = (int64_t)touched.size();
    stats[4] = newb;
    stats[5] = cnt.bad;
  }
  return cnt.bad ? -4 : 0;
}

}  // namespace

extern "C" {

/* Create an empty submap.  fp16 != 0 selects the FP16 storage mode. */
void* orc_create(float voxel_size, float trunc, float max_weight, int fp16) {
  Map* m = new Map();
  m->vs = voxel_size;
  m->trunc = trunc;
  m->max_w = max_weight;
  m->fp16 = fp16;
  return m;
}

void orc_destroy(void* h) { delete (Map*)h; }

int64_t orc_num_blocks(void* h) { return (int64_t)((Map*)h)->blocks.size(); }

/* Traversal of one segment given in voxel units (test hook). Returns the
 * number of voxels, or -1 if cap is too small. */
int orc_traverse(const float* A, const float* B, int32_t* out, int cap) {
  std::vector<Key> v;
  traverse(A, B, &v);
  if ((int)v.size() > cap) return -1;
  for (size_t q = 0; q < v.size(); ++q)
    for (int k = 0; k < 3; ++k) out[3 * q + k] = v[q][k];
  return (int)v.size();
}

/* Observations of a single point (test hook): voxels, FP64 distance and weight.
 * Returns the count, 0 for an invalid point, -1 if cap is too small, -2 for a
 * key-range violation.  seg (optional, 6 floats) receives the band segment A, B. */
int orc_point_obs(const float* ps, const float* T, float vs, float trunc, float min_range,
                  float max_range, int weight_mode, int dropoff, int sensor, float point_weight,
                  int32_t* vox, double* d, double* w, int cap, float* seg) {
  Ray ray;
  if (!make_ray(ps, T, min_range, max_range, sensor, &ray)) return 0;
  if (!point_weight_ok(&point_weight, 0, weight_mode)) return 0;
  float A[3], B[3];
  if (!band_segment(ray, trunc, vs, A, B)) return -2;
  if (seg) {
    for (int k = 0; k < 3; ++k) { seg[k] = A[k]; seg[3 + k] = B[k]; }
  }
  std::vector<Key> v;
  traverse(A, B, &v);
  if ((int)v.size() > cap) return -1;
  double base = base_weight(ps, ray, &point_weight, 0, weight_mode, sensor);
  for (size_t q = 0; q < v.size(); ++q) {
    for (int k = 0; k < 3; ++k) vox[3 * q + k] = v[q][k];
    d[q] = voxel_distance(ray, v[q], vs, trunc);
    w[q] = obs_weight(base, d[q], vs, trunc, dropoff);
  }
  return (int)v.size();
}


/* Integrate one scan (one frame).  pts: [n,3] sensor frame; T: 3x4 row-major
 * submap <- sensor; pw: per-point weights (weight_mode 2) or NULL; rgb: per
 * point colours [n,3] or NULL.
 * stats (optional, 6 entries): valid points, observations, unique voxels,
 * touched blocks, new blocks, key-range rejects.  Returns 0, or -4 if any point
 * left the key range (those points are skipped and, as in the CUDA path, the
 * merge of that frame is skipped while newly seen blocks stay allocated). */
int orc_integrate(void* h, const float* pts, int64_t n, const float* T, const float* pw,
                  int weight_mode, int dropoff, float min_range, float max_range, int sensor,
                  int64_t* stats, int carve, const float* rgb) {
  Map* m = (Map*)h;
  FrameSums frame;   // frame sums keyed by voxel, accumulated in point-index order
  FrameCounts cnt;
  accumulate_points(m, pts, 0, n, T, pw, weight_mode, dropoff, min_range, max_range, sensor, carve,
                    rgb, &frame, &cnt);
  return apply_frame(m, frame, cnt, stats);
}

/* The same frame with its sums accumulated by `threads` OpenMP threads, each
 * over a contiguous chunk of the points into its own map; the chunk maps are
 * then added in chunk order.  The result differs from orc_integrate only by
 * the FP64 rounding of the sums' order.  The parallel CPU baseline. */
int orc_integrate_parallel(void* h, const float* pts, int64_t n, const float* T, const float* pw,
                           int weight_mode, int dropoff, float min_range, float max_range,
                           int sensor, int64_t* stats, int carve, int threads) {
  Map* m = (Map*)h;
  if (threads < 1) threads = 1;
  std::vector<FrameSums> part(threads);
  std::vector<FrameCounts> pc(threads);
#pragma omp parallel for num_threads(threads) schedule(static, 1)
  for (int t = 0; t < threads; ++t) {
    const int64_t i0 = n * t / threads, i1 = n * (t + 1) / threads;
    accumulate_points(m, pts, i0, i1, T, pw, weight_mode, dropoff, min_range, max_range, sensor,
                      carve, nullptr, &part[t], &pc[t]);
  }
  FrameSums frame = std::move(part[0]);
  FrameCounts cnt = pc[0];
  for (int t = 1; t < threads; ++t) {
    for (auto& kv : part[t]) {
      auto& acc = frame[kv.first];
      acc.swd += kv.second.swd;
      acc.sw += kv.second.sw;
    }
    cnt.valid += pc[t].valid;
    cnt.nobs += pc[t].nobs;
    cnt.bad += pc[t].bad;
  }
  return apply_frame(m, frame, cnt, stats);
}

/* Copy out all blocks in ascending key order: keys [nb,3], D and W [nb,512]
 * (local voxel index lx + 8 ly + 64 lz).  D is in metres in both modes. */
void orc_extract(void* h, int32_t* keys, double* D, double* W) {
  Map* m = (Map*)h;
  int64_t q = 0;
  for (auto& kv : m->blocks) {
    for (int k = 0; k < 3; ++k) keys[3 * q + k] = kv.first[k];
    std::memcpy(D + q * kBlockVox, kv.second.D, sizeof(double) * kBlockVox);
    std::memcpy(W + q * kBlockVox, kv.second.W, sizeof(double) * kBlockVox);
    ++q;
  }
}

/* Fused colours of all blocks in ascending key order: [nb, 3, 512]. */
void orc_extract_colors(void* h, double* C) {
  Map* m = (Map*)h;
  int64_t q = 0;
  for (auto& kv : m->blocks) {
    std::memcpy(C + q * 3 * kBlockVox, kv.second.C, sizeof(double) * 3 * kBlockVox);
    ++q;
  }
}

/* ---- large-workload helpers: the same definitions, restricted outputs ---- */

/* Set of blocks touched by a sequence of scans (no voxel values).  keys_out
 * receives the sorted keys when it is non-NULL and cap suffices; returns the
 * number of distinct blocks.  point_weights (optional, one array per scan):
 * per-point weights, whose invalid entries drop their points. */
int64_t orc_block_set(const float* const* scans, const int64_t* counts, const float* poses,
                      int nscans, float vs, float trunc, float min_range, float max_range,
                      const int* sensors, const float* const* point_weights, int32_t* keys_out,
                      int64_t cap) {
  std::unordered_set<Key, KeyHash> blocks;
  std::vector<Key> vox;
  for (int s = 0; s < nscans; ++s) {
    for (int64_t i = 0; i < counts[s]; ++i) {
      Ray ray;
      if (!make_ray(scans[s] + 3 * i, poses + 12 * s, min_range, max_range,
                    sensors ? sensors[s] : 0, &ray))
        continue;
      if (point_weights && !point_weight_ok(point_weights[s], i, 2)) continue;
      float A[3], B[3];
      if (!band_segment(ray, trunc, vs, A, B)) continue;
      vox.clear();
      traverse(A, B, &vox);
      for (const Key& v : vox) blocks.insert(block_of(v));
    }
  }
  if (keys_out && (int64_t)blocks.size() <= cap) {
    std::vector<Key> sorted(blocks.begin(), blocks.end());
    std::sort(sorted.begin(), sorted.end());
    for (size_t q = 0; q < sorted.size(); ++q)
      for (int k = 0; k < 3; ++k) keys_out[3 * q + k] = sorted[q][k];
  }
  return (int64_t)blocks.size();
}

/* Final D, W of a sample of voxels after integrating a sequence of scans, each
 * scan one frame: exactly the full integration restricted to the sample.
 * vox: [ns,3] voxel indices.  D, W: [ns] outputs (W = 0, D = 0 if never seen).
 * obs_out (optional): observations per sample voxel. */
void orc_sampled(const float* const* scans, const int64_t* counts, const float* poses,
                 const float* const* point_weights, int nscans, float vs, float trunc,
                 float max_weight, int fp16, int weight_mode, int dropoff, float min_range,
                 float max_range, const int* sensors, const int32_t* vox, int64_t ns, double* D,
                 double* W, int64_t* obs_out) {
  std::unordered_map<Key, int64_t, KeyHash> index;
  for (int64_t q = 0; q < ns; ++q) index[{vox[3 * q], vox[3 * q + 1], vox[3 * q + 2]}] = q;
  std::vector<double> swd(ns), sw(ns);
  std::vector<char> hit(ns);
  for (int64_t q = 0; q < ns; ++q) {
    D[q] = 0;
    W[q] = 0;
    if (obs_out) obs_out[q] = 0;
  }
  Map m;
  m.vs = vs;
  m.trunc = trunc;
  m.max_w = max_weight;
  m.fp16 = fp16;
  std::vector<Key> vv;
  for (int s = 0; s < nscans; ++s) {
    std::fill(swd.begin(), swd.end(), 0.0);
    std::fill(sw.begin(), sw.end(), 0.0);
    std::fill(hit.begin(), hit.end(), 0);
    const float* pw = point_weights ? point_weights[s] : nullptr;
    for (int64_t i = 0; i < counts[s]; ++i) {
      const float* ps = scans[s] + 3 * i;
      Ray ray;
      if (!make_ray(ps, poses + 12 * s, min_range, max_range, sensors ? sensors[s] : 0, &ray))
        continue;
      if (!point_weight_ok(pw, i, weight_mode)) continue;
      float A[3], B[3];
      if (!band_segment(ray, trunc, vs, A, B)) continue;
      vv.clear();
      traverse(A, B, &vv);
      double base = base_weight(ps, ray, pw, i, weight_mode, sensors ? sensors[s] : 0);
      for (const Key& v : vv) {
        auto it = index.find(v);
        if (it == index.end()) continue;
        double d = voxel_distance(ray, v, vs, trunc);
        double w = obs_weight(base, d, vs, trunc, dropoff);
        swd[it->second] += w * d;
        sw[it->second] += w;
        hit[it->second] = 1;
        if (obs_out) obs_out[it->second]++;
      }
    }
    for (int64_t q = 0; q < ns; ++q) {
      if (!hit[q]) continue;
      Block tmp;  // reuse the single-voxel merge on a scratch block slot 0
      tmp.D[0] = D[q];
      tmp.W[0] = W[q];
      VoxelSums vsum;
      vsum.swd = swd[q];
      vsum.sw = sw[q];
      merge_voxel(&m, tmp, 0, vsum);
      D[q] = tmp.D[0];
      W[q] = tmp.W[0];
    }
  }
}

/* IEEE half rounding used by the FP16 storage mode (test hook). */
void orc_round_half(const double* x, int64_t n, double* out) {
  for (int64_t q = 0; q < n; ++q) out[q] = round_half(x[q]);
}

}  // extern "C"
