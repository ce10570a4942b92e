// covox_dev.cuh -- device-side building blocks of the integration path:
// the block hash (coVoxSLAM Sec. III-B), the FP32 band traversal (Sec. III-C
// ray casting, Amanatides-Woo), the observation distance/weight, and the
// device views of a submap and of a scan.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace covox {

constexpr int kVoxPerBlock = 512;           // 8^3
constexpr uint64_t kEmptyKey = ~0ull;       // unreachable: packed keys use 63 bits
constexpr int kGroupsPerBlock = kVoxPerBlock / 4;   // 4-voxel groups: local index >> 2
constexpr float kKeyLimit = 8388608.0f;     // 2^23 voxels = 2^20 blocks per axis

enum : int32_t { kErrCapacity = 1, kErrKeyRange = 2, kErrTimeout = 4 };

// Device-resident bookkeeping of one submap.
struct State {
  int32_t n_blocks;     // block pool bump pointer (allocation phase, Sec. III-D)
  int32_t nb_closed0;   // batched pipelined waves: n_blocks when the tiles of the scan in
  int32_t frame_err;    //   per-scan set 0 (nb_closed0) or 1 (nb_closed1) had finished
  int32_t sticky_err;   // frame_err: error bits of the current scan; sticky_err: OR of all scans'
  uint32_t ticket;      // last-CTA detection of the merge pass
  int32_t nb_closed1;
  int32_t frame_err_b;  // second per-scan set of a pipelined submap
  int32_t parity;       // pipelined per-scan path: set the next scan accumulates into
  int32_t pending;      // pipelined per-scan path: set parity ^ 1 holds an unmerged scan
  uint32_t epoch;       // scans whose tiles have completed; the running scan's epoch is epoch + 1
  unsigned long long frames, valid_pts, obs, voxels_merged, blocks_touched;
  int32_t frame_err_c;  // per-scan sets 2 and 3 of a four-set submap
  int32_t frame_err_d;
};

// Everything a kernel needs to address one submap (passed by value).
struct SubmapDev {
  unsigned long long* keys;   // [slots] packed block keys, kEmptyKey when free
  int32_t* vals;              // [slots] pool index of the slot's block (-1: not yet published, -3: none)
  int32_t* block_keys;        // [max_blocks,3] integer block coordinates
  void* D;                    // [max_blocks,512] float or half (D / trunc)
  void* W;                    // [max_blocks,512] float or half
  float2* acc;                // [max_blocks,512] per-scan sums (sum w (d - trunc), sum w), zero between scans
  uint32_t* tepoch;           // [max_blocks] epoch of the last scan of this per-scan set that touched the
                              // block: the scan's touched blocks are those holding its epoch
  uint8_t* gep;               // [max_blocks,128] touch tag of each 4-voxel group (a run of 4 along x) by
                              // this per-scan set: group_tag() of the last scan that observed a voxel of
                              // it, so a merge reads the sums of touched groups only
  float4* cacc;               // colour submaps: [max_blocks,512] per-scan colour sums (sum w r, sum w g,
                              // sum w b, 0) of this set, zero between scans; nullptr otherwise
  float* C;                   // colour submaps: [max_blocks,3,512] fused RGB planes; nullptr otherwise
  State* st;
  int32_t* frame_err;         // error bits of this per-scan set (&st->frame_err or _b)
  uint32_t slot_mask;
  int32_t max_probe;
  int32_t max_blocks;
  float vs, inv_vs, trunc, max_w;
  int32_t storage;
};

// One scan (frame) as the kernels see it, with its tiling: an organised
// scan (height x width == n) is cut into tile_w x tile_h pixel tiles, an
// unorganised one into runs of tile_w * tile_h consecutive points.
struct ScanDev {
  const float* pts;      // [n,3] sensor frame
  const float* pw;       // [n] per-point weights or nullptr
  const float* rgb;      // [n,3] per-point colours (colour submaps) or nullptr
  long long n;
  float T[12];           // submap <- sensor, row-major 3x4
  float min_range, max_range;
  int32_t weight_mode, dropoff, sensor, organised;
  int32_t carve;         // traverse from the sensor origin (free-space carving)
  int32_t long_band;     // a band may cross more than 512 cells per axis (trunc > 250 voxels)
  uint32_t epoch_add;    // the scan's epoch is st->epoch + 1 + epoch_add (its rank in a batched launch)
  int32_t height, width, tile_w, tile_h, tiles_x, n_tiles;
};

// ------------------------------------------------------------------ hash
__device__ __forceinline__ unsigned long long pack_key(int bx, int by, int bz) {
  return ((unsigned long long)(uint32_t)(bx + (1 << 20)) << 42) |
         ((unsigned long long)(uint32_t)(by + (1 << 20)) << 21) |
         (unsigned long long)(uint32_t)(bz + (1 << 20));
}

__device__ __forceinline__ uint32_t hash_key(unsigned long long k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return (uint32_t)k;
}

// Lookup only (keys are not modified by the caller's kernel).
__device__ __forceinline__ int hash_find(const SubmapDev& m, unsigned long long key) {
  uint32_t s = hash_key(key) & m.slot_mask;
  for (int p = 0; p < m.max_probe; ++p) {
    unsigned long long cur = __ldg(m.keys + s);
    if (cur == key) return (int)s;
    if (cur == kEmptyKey) return -1;
    s = (s + 1) & m.slot_mask;
  }
  return -1;
}

// --------------------------------------------------------- ray and band
// Point transform p = R ps + t (row sums left to right), r = p - o with
// o = t, len = |r|, u = r / len.  FP32 with explicit round-to-nearest
// intrinsics so that nothing is contracted into an FMA: the traversal below
// must reproduce the same voxels bit for bit on any IEEE FP32 machine.
struct Ray {
  float p[3], o[3], u[3], len;
};

__device__ __forceinline__ bool make_ray(const ScanDev& sc, long long i, Ray& r) {
  const float x = __ldg(sc.pts + 3 * i), y = __ldg(sc.pts + 3 * i + 1), z = __ldg(sc.pts + 3 * i + 2);
  if (!(isfinite(x) && isfinite(y) && isfinite(z))) return false;
  if (sc.sensor == 0 && !(z > 0.0f)) return false;   // a depth camera sees only z > 0
  float rr[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float s = __fadd_rn(__fmul_rn(sc.T[4 * k], x), __fmul_rn(sc.T[4 * k + 1], y));
    s = __fadd_rn(s, __fmul_rn(sc.T[4 * k + 2], z));
    r.p[k] = __fadd_rn(s, sc.T[4 * k + 3]);
    r.o[k] = sc.T[4 * k + 3];
    rr[k] = __fsub_rn(r.p[k], r.o[k]);
  }
  float l2 = __fmul_rn(rr[0], rr[0]);
  l2 = __fadd_rn(l2, __fmul_rn(rr[1], rr[1]));
  l2 = __fadd_rn(l2, __fmul_rn(rr[2], rr[2]));
  r.len = __fsqrt_rn(l2);
  if (!(r.len >= sc.min_range && r.len <= sc.max_range)) return false;
  const float il = __frcp_rn(r.len);
#pragma unroll
  for (int k = 0; k < 3; ++k) r.u[k] = __fmul_rn(rr[k], il);
  return true;
}

// Band endpoints in voxel units: A = (p - trunc u) / vs, B = (p + trunc u) / vs
// (the division is a multiply by the FP32 reciprocal of vs); with carving,
// A = o / vs (the ray starts at the sensor origin).  False if an endpoint
// leaves the key range.
__device__ __forceinline__ bool band(const Ray& r, float trunc, float inv_vs, float A[3], float B[3],
                                     bool carve = false) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float tu = __fmul_rn(trunc, r.u[k]);
    A[k] = carve ? __fmul_rn(r.o[k], inv_vs) : __fmul_rn(__fsub_rn(r.p[k], tu), inv_vs);
    B[k] = __fmul_rn(__fadd_rn(r.p[k], tu), inv_vs);
    ok = ok && (A[k] >= -kKeyLimit) && (A[k] < kKeyLimit) && (B[k] >= -kKeyLimit) && (B[k] < kKeyLimit);
  }
  return ok;
}

// Amanatides-Woo traversal of A -> B.  The next axis is the one with the
// smallest tMax among axes not yet at their end cell; ties take the lowest
// axis.  tMax starts at the first boundary crossing times 1/|B - A| and grows
// by that reciprocal per step.
struct Dda {
  int v[3], e[3], s[3];
  float tm[3], td[3];
  int left;

  __device__ __forceinline__ void init(const float A[3], const float B[3]) {
    left = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      v[k] = (int)floorf(A[k]);
      e[k] = (int)floorf(B[k]);
      const float d = __fsub_rn(B[k], A[k]);
      if (d > 0.0f) {
        s[k] = 1;
        td[k] = __frcp_rn(d);
        tm[k] = __fmul_rn(__fsub_rn((float)(v[k] + 1), A[k]), td[k]);
      } else if (d < 0.0f) {
        s[k] = -1;
        td[k] = __frcp_rn(-d);
        tm[k] = __fmul_rn(__fsub_rn(A[k], (float)v[k]), td[k]);
      } else {
        s[k] = 0;
        td[k] = __int_as_float(0x7f800000);
        tm[k] = __int_as_float(0x7f800000);
      }
      left += abs(e[k] - v[k]);
    }
  }

  __device__ __forceinline__ void step() {
    int best = -1;
    float bt = 0.0f;
    if (v[0] != e[0]) { best = 0; bt = tm[0]; }
    if (v[1] != e[1] && (best < 0 || tm[1] < bt)) { best = 1; bt = tm[1]; }
    if (v[2] != e[2] && (best < 0 || tm[2] < bt)) { best = 2; }
    if (best == 0) { v[0] += s[0]; tm[0] = __fadd_rn(tm[0], td[0]); }
    else if (best == 1) { v[1] += s[1]; tm[1] = __fadd_rn(tm[1], td[1]); }
    else { v[2] += s[2]; tm[2] = __fadd_rn(tm[2], td[2]); }
    --left;
  }
};

// ---------------------------------------------------- distance and weight
// d = (p - c_v).u with c_v = (v + 1/2) vs.  Each component p - (v+1/2) vs is
// one FMA (v + 1/2 is exact for |v| < 2^23), so the residual carries a single
// rounding however far the submap origin is.
__device__ __forceinline__ float voxel_distance(const Ray& r, const int v[3], float vs, float trunc) {
  const float q0 = fmaf(-((float)v[0] + 0.5f), vs, r.p[0]);
  const float q1 = fmaf(-((float)v[1] + 0.5f), vs, r.p[1]);
  const float q2 = fmaf(-((float)v[2] + 0.5f), vs, r.p[2]);
  const float d = fmaf(q2, r.u[2], fmaf(q1, r.u[1], q0 * r.u[0]));
  return fminf(fmaxf(d, -trunc), trunc);
}

// Unclamped d of the same definition.
__device__ __forceinline__ float voxel_distance_raw(const Ray& r, const int v[3], float vs) {
  const float q0 = fmaf(-((float)v[0] + 0.5f), vs, r.p[0]);
  const float q1 = fmaf(-((float)v[1] + 0.5f), vs, r.p[1]);
  const float q2 = fmaf(-((float)v[2] + 0.5f), vs, r.p[2]);
  return fmaf(q2, r.u[2], fmaf(q1, r.u[1], q0 * r.u[0]));
}

__device__ __forceinline__ float base_weight(const ScanDev& sc, long long i, const Ray& r) {
  if (sc.weight_mode == 0) return 1.0f;
  if (sc.weight_mode == 2) return __ldg(sc.pw + i);
  const float z = sc.sensor == 0 ? __ldg(sc.pts + 3 * i + 2) : r.len;
  return 1.0f / (z * z);
}

// A given per-point weight must be finite and non-negative; otherwise the
// point is invalid (skipped like a point without a return).
__device__ __forceinline__ bool weight_ok(const ScanDev& sc, float w0) {
  return sc.weight_mode != 2 || (isfinite(w0) && w0 >= 0.0f);
}

// A given colour must be finite in all three channels; otherwise the point is
// invalid, as for a per-point weight.
__device__ __forceinline__ bool colour_ok(const ScanDev& sc, long long i, float c[3]) {
  if (!sc.rgb) return true;
  c[0] = __ldg(sc.rgb + 3 * i);
  c[1] = __ldg(sc.rgb + 3 * i + 1);
  c[2] = __ldg(sc.rgb + 3 * i + 2);
  return isfinite(c[0]) && isfinite(c[1]) && isfinite(c[2]);
}

__device__ __forceinline__ float dropoff_weight(float w, float d, float vs, float trunc, int mode) {
  if (mode != 0 && d < -vs) {
    float f = fmaxf((trunc + d) / (trunc - vs), 0.0f);
    return mode == 1 ? w * f : w * f * f;
  }
  return w;
}

__device__ __forceinline__ int floor_div8(int v) { return v >> 3; }   // arithmetic shift
__device__ __forceinline__ int local_index(const int v[3]) {
  return (v[0] & 7) | ((v[1] & 7) << 3) | ((v[2] & 7) << 6);
}

}  // namespace covox
