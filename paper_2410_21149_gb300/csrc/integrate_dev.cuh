// integrate_dev.cuh -- the two phases of integrating one scan, as device
// functions shared by the per-scan kernels and the persistent batched kernel.
//
//   integrate_tile : count + allocate + reduce for one tile of points
//                    (coVoxSLAM Sec. III-D): one band traversal per point,
//                    per-voxel sums of the tile's blocks in shared memory,
//                    then one activation per distinct block (Sec. III-B) and a
//                    vector-atomic flush into the blocks' per-scan sums.
//   merge_span     : the blocks of a span of pool indices that the scan
//                    touched (their touch epoch is the scan's: the stream
//                    compaction of the allocation pass, Sec. III-D), each
//                    D <- (D W + sum w d)/(W + sum w), W <- min(W + sum w,
//                    max_weight) for voxels with sum w > 0, with vectorised
//                    loads/stores; clears the sums.
#pragma once

#include "covox_dev.cuh"

namespace covox {

constexpr int kTileThreads = 256;
constexpr int kTileBlocks = 64;      // distinct blocks recorded per tile (power of two)
constexpr int kMapDead = -3;         // vals[] marker: block unusable (pool exhausted)
constexpr long long kSpinLimit = 1 << 20;   // polls of an unpublished slot (~1 s)

// Touch tag of scan epoch ep in the per-group tags (never 0, the cleared
// value).  Tags repeat every 255 scans: a stale tag equal to the current one
// only makes a merge read a group whose sums are zero.
__device__ __forceinline__ uint8_t group_tag(uint32_t ep) { return (uint8_t)(1u + ep % 255u); }

// Global activation of one block ("activate", Sec. III-B: insert-or-find,
// pool index by atomic bump for a new block), and its mark as touched by the
// scan: the block's touch epoch is set to the scan's epoch `ep` (a plain
// store; every toucher writes the same value).  Returns the pool index or -1
// (error recorded).
//
// A slot holds the packed key and the pool index; the probe loads both at
// once, so finding an existing block costs one L2 round trip and nothing
// waits on an atomic.  The inserter of a new block publishes its pool index
// after writing the block's key; a thread that finds the key before that
// waits for the publication (bounded).
__device__ inline int global_activate(const SubmapDev& m, unsigned long long key, uint32_t ep) {
  uint32_t s = hash_key(key) & m.slot_mask;
  for (int p = 0; p < m.max_probe; ++p) {
    const unsigned long long cur = *((volatile unsigned long long*)(m.keys + s));
    int pool = *((volatile int32_t*)(m.vals + s));
    bool found = cur == key;
    if (cur == kEmptyKey) {
      const unsigned long long old = atomicCAS(m.keys + s, kEmptyKey, key);
      if (old == kEmptyKey) {   // inserted: allocate, publish
        pool = atomicAdd(&m.st->n_blocks, 1);
        if (pool >= m.max_blocks) {
          atomicOr(m.frame_err, kErrCapacity);
          atomicExch(m.vals + s, kMapDead);
          return -1;
        }
        m.block_keys[3 * pool] = (int)((key >> 42) & 0x1fffff) - (1 << 20);
        m.block_keys[3 * pool + 1] = (int)((key >> 21) & 0x1fffff) - (1 << 20);
        m.block_keys[3 * pool + 2] = (int)(key & 0x1fffff) - (1 << 20);
        m.tepoch[pool] = ep;
        atomicExch(m.vals + s, pool);   // publish
        return pool;
      }
      found = old == key;
      pool = -1;   // read it once published
    }
    if (found) {
      for (long long it = 0; pool == -1 && it < kSpinLimit; ++it) {   // the inserter publishes shortly
        __nanosleep(64);
        pool = *((volatile int32_t*)(m.vals + s));
      }
      if (pool == -1) {
        atomicOr(m.frame_err, kErrTimeout);
        return -1;
      }
      if (pool < 0) return -1;   // block unusable (pool was exhausted)
      m.tepoch[pool] = ep;
      return pool;
    }
    s = (s + 1) & m.slot_mask;
  }
  atomicOr(m.frame_err, kErrCapacity);   // bounded probe found no room
  return -1;
}

// (a, b) added to a float2 in global memory by the L2, fire and forget: a
// vector reduction that returns nothing, so no warp waits on it.
__device__ __forceinline__ void red_add2(float2* addr, float a, float b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(a), "f"(b) : "memory");
}

__device__ __forceinline__ void red_add4(float4* addr, float a, float b, float c) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(0.0f)
               : "memory");
}

// Pool index of an already activated block (read-only probe), or -1.
__device__ __forceinline__ int find_pool(const SubmapDev& m, unsigned long long key) {
  const int s = hash_find(m, key);
  if (s < 0) return -1;
  const int p = __ldg(m.vals + s);
  return p >= 0 ? p : -1;
}

// Points of one tile: iteration k of this thread gives a point index or -1.
struct TilePoints {
  long long base, end;   // unorganised: [base, end)
  int x0, y0;            // organised: tile origin in pixels

  __device__ __forceinline__ TilePoints(const ScanDev& sc, int tile) {
    if (!sc.organised) {
      base = (long long)tile * sc.tile_w * sc.tile_h;
      end = min(base + (long long)sc.tile_w * sc.tile_h, sc.n);
      x0 = y0 = 0;
    } else {
      base = end = 0;
      x0 = (tile % sc.tiles_x) * sc.tile_w;
      y0 = (tile / sc.tiles_x) * sc.tile_h;
    }
  }

  __device__ __forceinline__ long long point(const ScanDev& sc, int k) const {
    const int t = threadIdx.x;
    if (!sc.organised) {
      const long long i = base + (long long)k * kTileThreads + t;
      return i < end ? i : -1;
    }
    int x, y;
    if (sc.tile_w == 32 && (sc.tile_h & 31) == 0) {
      // lanes of a warp on an 8 x 4 grid spaced 4 x 8 pixels over a 32 x 32 chunk:
      // neighbouring lanes rarely share a voxel, so shared atomics rarely collide
      const int l = t & 31, w = t >> 5;
      x = (l & 7) * 4 + (w & 3);
      y = (k >> 2) * 32 + (l >> 3) * 8 + (w >> 2) * 4 + (k & 3);
    } else if (sc.tile_w == 32) {   // lanes on an 8 x 4 grid of a 32 x 8 chunk
      const int l = t & 31, w = t >> 5;
      x = (l & 7) * 4 + (w & 3);
      y = k * 8 + (l >> 3) * 2 + (w >> 2);
    } else {
      const int p = k * kTileThreads + t;
      x = p % sc.tile_w;
      y = p / sc.tile_w;
    }
    const int gx = x0 + x, gy = y0 + y;
    if (gx >= sc.width || gy >= sc.height || y >= sc.tile_h) return -1;
    return (long long)gy * sc.width + gx;
  }
};

__device__ __forceinline__ int tile_iters(const ScanDev& sc) {
  return (sc.tile_w * sc.tile_h + kTileThreads - 1) / kTileThreads;
}

// ------------------------------------------------ count + allocate + process
// One pass per tile.  Each point's band is traversed once; at every block
// boundary the block key is looked up in a small shared-memory map whose
// position is the block's slot of per-voxel sums: a new key is claimed with a
// single CAS, so lookups never wait.  Observations add w*d and w to the slot
// with shared atomics.  After the pass the tile's distinct blocks (its count
// phase) are activated once each in the block hash (Sec. III-B "activate":
// insert-or-find, pool index by atomic bump, touch epoch: Sec. III-D
// allocation phase) and the slots are flushed with vector atomics
// into the blocks' per-scan accumulators.  A block that finds the map full is
// activated on the spot and accumulated straight into global memory.
__device__ __forceinline__ uint32_t slot_hash(unsigned long long key) {
  return ((uint32_t)key ^ (uint32_t)(key >> 29)) * 0x9E3779B1u;
}

constexpr int kCache = 256;         // block -> pool cache entries per CTA (power of two)
constexpr int kCachePending = -2;

// The per-scan sums of a voxel are (sum w (d - trunc), sum w): distances are
// summed relative to +trunc, so the many observations of free space (d
// clamped to +trunc) add exact zeros, and D is recovered as
// trunc + ((D - trunc) W + sum w (d - trunc)) / (W + sum w) -- the same value
// as (D W + sum w d) / (W + sum w).
// Shared per-voxel sums are exact 64-bit fixed point X = hi * 2^S + lo held
// in two 32-bit words (lo unsigned, < 2^S per observation; hi signed), so
// every update is two native 32-bit integer atomics, which the hardware
// merges when lanes collide (float shared atomics retry instead).
struct TileSmem {
  unsigned long long* mkey;   // [lb] block key of each slot, kEmptyKey if free
  int* pool;                  // [lb]
  unsigned* lo_wd;            // [lb * 512]
  int* hi_wd;                 // [lb * 512]
  unsigned* lo_w;             // [lb * 512]
  int* hi_w;                  // [lb * 512]
  float* wmax;                // [warps] per-warp maxima of the tile's weights
  unsigned long long* red;    // [2 * warps]
  unsigned long long* ckey;   // [kCache] block -> pool cache
  int* cpool;                 // [kCache]
  int* list;                  // [warps * kListPerWarp] each warp's compacted candidate points
};

constexpr int kGather = 8;                  // tile iterations gathered per compaction round
constexpr int kListPerWarp = kGather * 32;

__host__ __device__ inline size_t tile_smem_bytes(int lb) {
  return (size_t)lb * 8 + (size_t)lb * 4 + 2 * (kTileThreads / 32) * 8 + 16 + (size_t)lb * kVoxPerBlock * 16 +
         (size_t)kCache * 12 + 16 + (kTileThreads / 32) * 4 + 16 + (size_t)(kTileThreads / 32) * kListPerWarp * 4 +
         16;
}

__device__ inline TileSmem tile_smem(char* base, int lb) {
  TileSmem t;
  t.lo_wd = reinterpret_cast<unsigned*>(base);
  base += (size_t)lb * kVoxPerBlock * 4;
  t.hi_wd = reinterpret_cast<int*>(base);
  base += (size_t)lb * kVoxPerBlock * 4;
  t.lo_w = reinterpret_cast<unsigned*>(base);
  base += (size_t)lb * kVoxPerBlock * 4;
  t.hi_w = reinterpret_cast<int*>(base);
  base += (size_t)lb * kVoxPerBlock * 4;
  t.mkey = reinterpret_cast<unsigned long long*>(base);
  base += (size_t)lb * 8;
  t.red = reinterpret_cast<unsigned long long*>(base);
  base += 2 * (kTileThreads / 32) * 8;
  t.ckey = reinterpret_cast<unsigned long long*>(base);
  base += kCache * 8;
  t.cpool = reinterpret_cast<int*>(base);
  base += kCache * 4;
  t.wmax = reinterpret_cast<float*>(base);
  base += ((kTileThreads / 32) * 4 + 15) / 16 * 16;
  t.pool = reinterpret_cast<int*>(base);
  base += ((size_t)lb * 4 + 15) / 16 * 16;
  t.list = reinterpret_cast<int*>(base);
  return t;
}

// Fixed-point format of a tile: value = X * 2^-F, X = hi * 2^S + lo.  With
// n observations per voxel at most (a ray meets a voxel once, so n <= the
// tile's points) the lo words never overflow when n * 2^S <= 2^32, and the hi
// words never overflow when n * max|X| < 2^(31 + S); F is the largest scale
// with max|X| = 2 * wmax * max(trunc, 1) * 2^F inside that bound.
struct Fixed {
  int S;
  float scale, inv_scale;   // 2^F, 2^-F
};

__device__ __forceinline__ Fixed fixed_format(int tile_points, float wmax, float trunc) {
  const int bn = 32 - __clz(max(tile_points, 2) - 1);           // ceil(log2 n)
  Fixed f;
  f.S = 32 - bn;
  const float bound = 2.0f * fmaxf(wmax, 1e-30f) * fmaxf(trunc, 1.0f);
  int e;
  frexpf(bound, &e);                                             // bound < 2^e
  const int F = min(max(31 + f.S - bn - 1 - e, -120), 120);      // n * 2^(F+e) < 2^(31+S); 2^F a normal float
  f.scale = ldexpf(1.0f, F);
  f.inv_scale = ldexpf(1.0f, -F);
  return f;
}

__device__ __forceinline__ void fixed_add(unsigned* lo, int* hi, int S, long long X) {
  atomicAdd(lo, (unsigned)(X & ((1ll << S) - 1)));
  atomicAdd(hi, (int)(X >> S));
}

// X * 2^-F rounded once to FP32: the integer conversion rounds, the scaling
// by a power of two is exact (no FP64 anywhere on the GPU path).
__device__ __forceinline__ float fixed_value(unsigned lo, int hi, int S, float inv_scale) {
  const long long X = ((long long)hi << S) + (long long)lo;
  return __ll2float_rn(X) * inv_scale;
}

// Pool index of a block through the CTA's block -> pool cache.  The first
// thread to claim an entry looks the block up in the global hash and
// publishes the answer there; a thread that finds the entry still pending
// does not wait for it but looks the block up itself (a lookup of an existing
// block is one read of its hash slot and a store of the same touch epoch;
// two threads inserting one key are ordered by the key's CAS).
__device__ __forceinline__ int cached_pool(const SubmapDev& m, const TileSmem& t, unsigned long long key,
                                           uint32_t ep) {
  const uint32_t h = slot_hash(key) >> 24;
  for (int p = 0; p < 8; ++p) {
    const int q = (h + p) & (kCache - 1);
    unsigned long long cur = *((volatile unsigned long long*)(t.ckey + q));
    if (cur == kEmptyKey) {
      cur = atomicCAS(t.ckey + q, kEmptyKey, key);
      if (cur == kEmptyKey) {
        const int pool = global_activate(m, key, ep);
        atomicExch(t.cpool + q, pool);
        return pool;
      }
    }
    if (cur == key) {
      const int pool = *((volatile int*)(t.cpool + q));
      return pool != kCachePending ? pool : global_activate(m, key, ep);
    }
  }
  return global_activate(m, key, ep);
}

// Shared slot of a block in a map of lb (power of two) slots, or -1 if full.
__device__ __forceinline__ int local_slot(const TileSmem& t, int lb, unsigned long long key) {
  if (lb == 0) return -1;
  const uint32_t h = slot_hash(key) >> 16;
  for (int p = 0; p < lb; ++p) {
    const int q = (h + p) & (lb - 1);
    unsigned long long cur = *((volatile unsigned long long*)(t.mkey + q));
    if (cur == kEmptyKey) {
      cur = atomicCAS(t.mkey + q, kEmptyKey, key);
      if (cur == kEmptyKey) return q;
    }
    if (cur == key) return q;
  }
  return -1;
}

// Flush of a tile's shared sums (kLocal) into its blocks' per-scan sums:
// every voxel with a nonzero weight sum by one vector reduction, and the
// touch tag of each group holding one.
__device__ __forceinline__ void flush_slots(const SubmapDev& m, const TileSmem& t, int lb, const Fixed& fx,
                                            uint8_t tag) {
  const int tid = threadIdx.x, lane = tid & 31;
  for (int q = 0; q < lb; ++q) {
    const int pool = t.pool[q];
    if (pool < 0) continue;
    float2* dst = m.acc + (size_t)pool * kVoxPerBlock;
    for (int v = tid; v < kVoxPerBlock; v += kTileThreads) {
      const int e = q * kVoxPerBlock + v;
      bool nz = (t.lo_w[e] | (unsigned)t.hi_w[e]) != 0u;
      if (nz) {
        const float w = fixed_value(t.lo_w[e], t.hi_w[e], fx.S, fx.inv_scale);
        const float wd = fixed_value(t.lo_wd[e], t.hi_wd[e], fx.S, fx.inv_scale);
        nz = w != 0.0f;
        if (nz) red_add2(dst + v, wd, w);
      }
      // lanes 4j .. 4j + 3 hold the voxels of one group
      const unsigned bal = __ballot_sync(0xffffffffu, nz);
      if ((lane & 3) == 0 && ((bal >> lane) & 0xFu)) m.gep[(size_t)pool * kGroupsPerBlock + (v >> 2)] = tag;
    }
  }
}

// The general form of the tile phase, one point after another per thread:
// any band length, and free-space carving (rays from the sensor origin, with
// the distance recomputed exactly near the band).  Scans without carving and
// with bands of at most 512 cells per axis take integrate_tile_t below.
template <bool kLocal, int kDrop, bool kCarve = false>
__device__ inline void integrate_tile_legacy(const SubmapDev& m, const ScanDev& sc, int tile, char* smem,
                                             int lb) {
  const TileSmem t = tile_smem(smem, lb);
  const int tid = threadIdx.x;
  for (int q = tid; q < kCache; q += kTileThreads) {
    t.ckey[q] = kEmptyKey;
    t.cpool[q] = kCachePending;
  }
  const TilePoints tp(sc, tile);
  const int iters = tile_iters(sc);
  const uint32_t ep = *((volatile uint32_t*)&m.st->epoch) + 1u + sc.epoch_add;   // this scan's epoch
  Fixed fx;
  if (kLocal) {
    for (int q = tid; q < lb; q += kTileThreads) t.mkey[q] = kEmptyKey;
    uint4* z = reinterpret_cast<uint4*>(t.lo_wd);
    const int n4 = lb * kVoxPerBlock * 4 / 4;
    for (int q = tid; q < n4; q += kTileThreads) z[q] = make_uint4(0u, 0u, 0u, 0u);
    // the fixed-point scale bounds the tile's weights (a cheap pre-pass over
    // its points; the constant weight is 1)
    float wm = 1.0f;
    if (sc.weight_mode != 0) {
      wm = 0.0f;
      for (int k = 0; k < iters; ++k) {
        const long long i = tp.point(sc, k);
        if (i < 0) continue;
        float w0;
        if (sc.weight_mode == 2) {
          w0 = __ldg(sc.pw + i);
        } else {
          const float x = __ldg(sc.pts + 3 * i), y = __ldg(sc.pts + 3 * i + 1), z3 = __ldg(sc.pts + 3 * i + 2);
          const float zz = sc.sensor == 0 ? z3 * z3 : x * x + y * y + z3 * z3;
          w0 = 1.0f / zz;
        }
        if (isfinite(w0) && w0 >= 0.0f) wm = fmaxf(wm, w0);   // other per-point weights drop their point
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) wm = fmaxf(wm, __shfl_xor_sync(0xffffffffu, wm, o));
      if ((tid & 31) == 0) t.wmax[tid >> 5] = wm;
    }
    __syncthreads();
    if (sc.weight_mode != 0) {
      wm = 0.0f;
      for (int w = 0; w < kTileThreads / 32; ++w) wm = fmaxf(wm, t.wmax[w]);
    }
    fx = fixed_format(iters * kTileThreads, wm, m.trunc);
  }
  __syncthreads();

  const float inv_drop = 1.0f / (m.trunc - m.vs);
  const uint8_t tag = group_tag(ep);
  unsigned n_obs = 0, n_valid = 0;
  for (int k = 0; k < iters; ++k) {
    const long long i = tp.point(sc, k);
    if (i < 0) continue;
    Ray r;
    if (!make_ray(sc, i, r)) continue;
    const float w0 = base_weight(sc, i, r);
    if (!weight_ok(sc, w0)) continue;
    float col[3] = {0.0f, 0.0f, 0.0f};
    if (!colour_ok(sc, i, col)) continue;
    float A[3], B[3];
    if (!band(r, m.trunc, m.inv_vs, A, B, kCarve)) {
      atomicOr(m.frame_err, kErrKeyRange);
      continue;
    }
    ++n_valid;
    Dda d;
    d.init(A, B);
    n_obs += d.left + 1;
    // incremental state: distance (exact at the first voxel, then one add per
    // step), local voxel index and packed block key
    float dist = voxel_distance_raw(r, d.v, m.vs);
    const float dd0 = -(float)d.s[0] * m.vs * r.u[0];
    const float dd1 = -(float)d.s[1] * m.vs * r.u[1];
    const float dd2 = -(float)d.s[2] * m.vs * r.u[2];
    int l = local_index(d.v);
    unsigned long long key = pack_key(d.v[0] >> 3, d.v[1] >> 3, d.v[2] >> 3);
    int slot = kLocal ? local_slot(t, lb, key) : -1;
    int gpool = slot < 0 ? cached_pool(m, t, key, ep) : -1;
    // The band ends in the block of its last cell; most bands meet one or two
    // blocks, so the end block is looked up here, with every lane of the warp,
    // and only a block met in between is looked up inside the loop.
    const unsigned long long key_end = pack_key(d.e[0] >> 3, d.e[1] >> 3, d.e[2] >> 3);
    int slot_end = slot, gpool_end = gpool;
    if (key_end != key) {
      slot_end = kLocal ? local_slot(t, lb, key_end) : -1;
      gpool_end = slot_end < 0 ? cached_pool(m, t, key_end, ep) : -1;
    }
    int last_g = -1;   // group of the previous cell (the group changes at every block crossing)
    for (;;) {
      const float dc = fminf(fmaxf(dist, -m.trunc), m.trunc);
      float w = w0;
      if (kDrop != 0 && dc < -m.vs) {
        const float f = fmaxf((m.trunc + dc) * inv_drop, 0.0f);
        w = kDrop == 1 ? w * f : w * f * f;
      }
      if (kLocal && slot >= 0) {
        const int e = slot * kVoxPerBlock + l;
        fixed_add(t.lo_wd + e, t.hi_wd + e, fx.S, __float2ll_rn(w * (dc - m.trunc) * fx.scale));
        fixed_add(t.lo_w + e, t.hi_w + e, fx.S, __float2ll_rn(w * fx.scale));
      } else if (gpool >= 0) {
        red_add2(m.acc + (size_t)gpool * kVoxPerBlock + l, w * (dc - m.trunc), w);
        if (sc.rgb) red_add4(m.cacc + (size_t)gpool * kVoxPerBlock + l, w * col[0], w * col[1], w * col[2]);
        if ((l >> 2) != last_g) m.gep[(size_t)gpool * kGroupsPerBlock + (l >> 2)] = tag;
      }
      last_g = l >> 2;
      if (d.left == 0) break;
      // next axis: the traversal rule of Dda::step, as selects
      const bool a0 = d.v[0] != d.e[0], a1 = d.v[1] != d.e[1], a2 = d.v[2] != d.e[2];
      int best = a0 ? 0 : (a1 ? 1 : 2);
      float bt = a0 ? d.tm[0] : (a1 ? d.tm[1] : d.tm[2]);
      if (a1 && d.tm[1] < bt) { best = 1; bt = d.tm[1]; }
      if (a2 && d.tm[2] < bt) best = 2;
      --d.left;
      int sk, stride, shift;
      if (best == 0) {
        sk = d.s[0]; d.v[0] += sk; d.tm[0] = __fadd_rn(d.tm[0], d.td[0]); dist += dd0; stride = 1; shift = 42;
      } else if (best == 1) {
        sk = d.s[1]; d.v[1] += sk; d.tm[1] = __fadd_rn(d.tm[1], d.td[1]); dist += dd1; stride = 8; shift = 21;
      } else {
        sk = d.s[2]; d.v[2] += sk; d.tm[2] = __fadd_rn(d.tm[2], d.td[2]); dist += dd2; stride = 64; shift = 0;
      }
      // A carved ray reaches the band after many steps of free space, where
      // the clamp hides the drift of the running sum; near the band the
      // distance is recomputed exactly.
      if (kCarve && dist < m.trunc + 2.0f * m.vs) dist = voxel_distance_raw(r, d.v, m.vs);
      const int mask = 7 * stride;
      const int f = ((l & mask) + sk * stride) & mask;
      l = (l & ~mask) | f;
      if (f == (sk > 0 ? 0 : mask)) {   // crossed into the neighbouring block
        key += sk > 0 ? (1ull << shift) : (0ull - (1ull << shift));
        if (key == key_end) {
          slot = slot_end;
          gpool = gpool_end;
        } else {
          slot = kLocal ? local_slot(t, lb, key) : -1;
          gpool = slot < 0 ? cached_pool(m, t, key, ep) : -1;
        }
      }
    }
  }
  __syncthreads();
  if (kLocal) {
    // allocation: each distinct block of the tile's shared slots is activated once
    for (int q = tid; q < lb; q += kTileThreads) {
      const unsigned long long key = t.mkey[q];
      t.pool[q] = key == kEmptyKey ? -1 : cached_pool(m, t, key, ep);
    }
    __syncthreads();
    flush_slots(m, t, lb, fx, tag);   // the tile's sums into the per-scan accumulators
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n_obs += __shfl_xor_sync(0xffffffffu, n_obs, o);
    n_valid += __shfl_xor_sync(0xffffffffu, n_valid, o);
  }
  if ((tid & 31) == 0) {
    t.red[tid >> 5] = n_obs;
    t.red[kTileThreads / 32 + (tid >> 5)] = n_valid;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long a = 0, c = 0;
    for (int w = 0; w < kTileThreads / 32; ++w) {
      a += t.red[w];
      c += t.red[kTileThreads / 32 + w];
    }
    if (a) atomicAdd(&m.st->obs, a);
    if (c) atomicAdd(&m.st->valid_pts, c);
  }
  __syncthreads();   // shared memory is reused by the caller's next tile
}

// ------------------------------------------------- tile phase, warp-parallel
// A point survives the first test if its coordinates are finite, it lies in
// front of a pinhole sensor and its per-point weight (if any) is usable; the
// range gate, which needs the transformed ray, is make_ray's.
__device__ __forceinline__ bool point_candidate(const ScanDev& sc, long long i) {
  const float x = __ldg(sc.pts + 3 * i), y = __ldg(sc.pts + 3 * i + 1), z = __ldg(sc.pts + 3 * i + 2);
  if (!(isfinite(x) && isfinite(y) && isfinite(z))) return false;
  if (sc.sensor == 0 && !(z > 0.0f)) return false;
  if (sc.weight_mode == 2) {
    const float w = __ldg(sc.pw + i);
    if (!(isfinite(w) && w >= 0.0f)) return false;
  }
  return true;
}

// Band traversal state of one ray.  The tMax of an axis that has reached its
// end cell is +inf, so the axis to step is the plain argmin of the three tMax
// values with ties to the lowest axis: the rule of Dda::step (an axis with no
// crossing left can never be chosen, and an axis with crossings left never
// holds +inf: one whose 1/|B - A| overflowed holds the largest finite float).
// Per axis two counters sit in 10-bit fields of two words: the steps left on
// the axis, biased by 511 (the axis reaches its end cell when bit 9 of its
// field clears), and the steps left before the next block boundary, biased by
// 8 (the step crosses into the neighbouring block when bit 3 clears).  One
// subtraction steps the chosen axis in both words.
struct Walk {
  float tm0, tm1, tm2, td0, td1, td2;
  float dist, dd0, dd1, dd2;   // distance of the current cell; change per step on each axis
  int dl0, dl1, dl2;           // change of the local voxel index per step on each axis
  uint32_t nrem, cb;
  int l, left;
};

// The same initial values as Dda::init (operation for operation), then the
// packed counters.  v and e receive the start and end cells.  False if an
// axis needs more than 512 steps (not representable: the host sends such
// scans to integrate_tile_legacy).
__device__ __forceinline__ bool walk_init(const Ray& r, const float A[3], const float B[3], float vs, Walk& w,
                                          int v[3], int e[3]) {
  float tm[3], td[3];
  int s[3];
  w.left = 0;
  w.nrem = 0;
  w.cb = 0;
  bool ok = true;
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
    const int n = abs(e[k] - v[k]);
    w.left += n;
    ok = ok && n <= 512;
    if (n == 0) tm[k] = __int_as_float(0x7f800000);
    else if (isinf(tm[k])) tm[k] = 3.40282347e38f;
    const int c = v[k] & 7;
    w.nrem |= (uint32_t)(min(n, 512) + 511) << (10 * k);
    w.cb |= (uint32_t)((s[k] > 0 ? 7 - c : (s[k] < 0 ? c : 7)) + 8) << (10 * k);
  }
  w.tm0 = tm[0]; w.tm1 = tm[1]; w.tm2 = tm[2];
  w.td0 = td[0]; w.td1 = td[1]; w.td2 = td[2];
  w.dl0 = s[0]; w.dl1 = 8 * s[1]; w.dl2 = 64 * s[2];
  w.dist = voxel_distance_raw(r, v, vs);
  w.dd0 = -(float)s[0] * vs * r.u[0];
  w.dd1 = -(float)s[1] * vs * r.u[1];
  w.dd2 = -(float)s[2] * vs * r.u[2];
  w.l = local_index(v);
  return ok;
}

// Shared slot and pool index of the block `key` for the lanes of the warp in
// `act` (this lane takes part if `on`): lanes holding the same key elect the
// lowest as leader, which looks it up (shared slot, CTA cache, global hash);
// the others read the answer from it.  Lanes outside `act` return at once and
// keep their outputs.
template <bool kLocal>
__device__ __forceinline__ void warp_lookup(const SubmapDev& m, const TileSmem& t, int lb, uint32_t ep,
                                            unsigned act, bool on, unsigned long long key, int& slot, int& pool) {
  if (!on) return;
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(act, key);
  const int leader = __ffs(peers) - 1;
  int s = -1, p = -1;
  if (lane == leader) {
    s = kLocal ? local_slot(t, lb, key) : -1;
    if (s < 0) p = cached_pool(m, t, key, ep);
  }
  if (kLocal) s = __shfl_sync(act, s, leader);
  p = __shfl_sync(act, p, leader);
  slot = s;
  pool = p;
}

// Count + allocate + process for one tile (coVoxSLAM Sec. III-D), warp by
// warp.  Each warp first gathers its valid points (a ballot per iteration,
// so invalid points -- no return, out of range -- leave no idle lanes in the
// traversal), then takes them 32 at a time: ray set-up, one warp-aggregated
// lookup of each band's first and last block (Sec. III-B "activate"), and the band
// traversal with one observation per cell: w (d - trunc) and w added to the
// block's per-scan sums, in shared memory as exact fixed point (kLocal, slot
// found) or by an L2 vector reduction.  A block met between the first and the
// last is looked up by its lane alone.  (lookup: insert-or-find, pool index
// by atomic bump, the block's touch epoch set to this scan's.)
template <bool kLocal, int kDrop>
__device__ inline void integrate_tile_t(const SubmapDev& m, const ScanDev& sc, int tile, char* smem, int lb) {
  const TileSmem t = tile_smem(smem, lb);
  const int tid = threadIdx.x, lane = tid & 31;
  for (int q = tid; q < kCache; q += kTileThreads) {
    t.ckey[q] = kEmptyKey;
    t.cpool[q] = kCachePending;
  }
  const TilePoints tp(sc, tile);
  const int iters = tile_iters(sc);
  const uint32_t ep = *((volatile uint32_t*)&m.st->epoch) + 1u + sc.epoch_add;   // this scan's epoch
  Fixed fx;
  if (kLocal) {
    for (int q = tid; q < lb; q += kTileThreads) t.mkey[q] = kEmptyKey;
    uint4* z = reinterpret_cast<uint4*>(t.lo_wd);
    const int n4 = lb * kVoxPerBlock * 4 / 4;
    for (int q = tid; q < n4; q += kTileThreads) z[q] = make_uint4(0u, 0u, 0u, 0u);
    // the fixed-point scale bounds the tile's weights (a cheap pre-pass over
    // its points; the constant weight is 1)
    float wm = 1.0f;
    if (sc.weight_mode != 0) {
      wm = 0.0f;
      for (int k = 0; k < iters; ++k) {
        const long long i = tp.point(sc, k);
        if (i < 0) continue;
        float w0;
        if (sc.weight_mode == 2) {
          w0 = __ldg(sc.pw + i);
        } else {
          const float x = __ldg(sc.pts + 3 * i), y = __ldg(sc.pts + 3 * i + 1), z3 = __ldg(sc.pts + 3 * i + 2);
          const float zz = sc.sensor == 0 ? z3 * z3 : x * x + y * y + z3 * z3;
          w0 = 1.0f / zz;
        }
        if (isfinite(w0) && w0 >= 0.0f) wm = fmaxf(wm, w0);   // other per-point weights drop their point
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) wm = fmaxf(wm, __shfl_xor_sync(0xffffffffu, wm, o));
      if (lane == 0) t.wmax[tid >> 5] = wm;
    }
    __syncthreads();
    if (sc.weight_mode != 0) {
      wm = 0.0f;
      for (int w = 0; w < kTileThreads / 32; ++w) wm = fmaxf(wm, t.wmax[w]);
    }
    fx = fixed_format(iters * kTileThreads, wm, m.trunc);
  }
  __syncthreads();

  const float inv_drop = 1.0f / (m.trunc - m.vs);
  const float INF = __int_as_float(0x7f800000);
  const uint8_t tag = group_tag(ep);
  unsigned n_obs = 0, n_valid = 0;
  int* list = t.list + (tid >> 5) * kListPerWarp;
  for (int k0 = 0; k0 < iters; k0 += kGather) {
    // gather this warp's candidate points of up to kGather iterations
    int nl = 0;
    const int k1 = min(iters, k0 + kGather);
    for (int k = k0; k < k1; ++k) {
      const long long i = tp.point(sc, k);
      const bool ok = i >= 0 && point_candidate(sc, i);
      const unsigned bal = __ballot_sync(0xffffffffu, ok);
      if (ok) list[nl + __popc(bal & ((1u << lane) - 1u))] = (int)i;
      nl += __popc(bal);
    }
    __syncwarp();
    for (int r0 = 0; r0 < nl; r0 += 32) {
      // ray set-up
      const int q = r0 + lane;
      bool act = false;
      Ray r;
      float A[3], B[3], w0 = 0.0f;
      if (q < nl) {
        const long long i = list[q];
        if (make_ray(sc, i, r)) {
          w0 = base_weight(sc, i, r);
          if (band(r, m.trunc, m.inv_vs, A, B)) act = true;
          else atomicOr(m.frame_err, kErrKeyRange);
        }
      }
      Walk w;
      unsigned long long key = 0, key_end = 0;
      if (act) {
        int v[3], e[3];
        walk_init(r, A, B, m.vs, w, v, e);
        key = pack_key(v[0] >> 3, v[1] >> 3, v[2] >> 3);
        key_end = pack_key(e[0] >> 3, e[1] >> 3, e[2] >> 3);
        ++n_valid;
        n_obs += w.left + 1;
      }
      const unsigned actm = __ballot_sync(0xffffffffu, act);
      if (actm == 0) continue;
      // the band's first and last blocks, warp-aggregated
      int slot = -1, pool = -1;
      warp_lookup<kLocal>(m, t, lb, ep, actm, act, key, slot, pool);
      int slot_end = slot, pool_end = pool;
      const bool two = act && key_end != key;
      const unsigned twom = __ballot_sync(0xffffffffu, two);
      if (twom) warp_lookup<kLocal>(m, t, lb, ep, twom, two, key_end, slot_end, pool_end);
      if (!act) continue;
      // traversal: one observation per cell
      int last_g = -1;   // group of the previous cell (the group changes at every block crossing)
      for (;;) {
        const float dc = fminf(fmaxf(w.dist, -m.trunc), m.trunc);
        float wt = w0;
        if (kDrop != 0 && dc < -m.vs) {
          const float f = fmaxf((m.trunc + dc) * inv_drop, 0.0f);
          wt = kDrop == 1 ? wt * f : wt * f * f;
        }
        if (kLocal && slot >= 0) {
          const int e = slot * kVoxPerBlock + w.l;
          fixed_add(t.lo_wd + e, t.hi_wd + e, fx.S, __float2ll_rn(wt * (dc - m.trunc) * fx.scale));
          fixed_add(t.lo_w + e, t.hi_w + e, fx.S, __float2ll_rn(wt * fx.scale));
        } else if (pool >= 0) {
          red_add2(m.acc + (size_t)pool * kVoxPerBlock + w.l, wt * (dc - m.trunc), wt);
          if ((w.l >> 2) != last_g) m.gep[(size_t)pool * kGroupsPerBlock + (w.l >> 2)] = tag;
        }
        last_g = w.l >> 2;
        if (w.left == 0) break;
        --w.left;
        const bool p1 = w.tm1 < w.tm0;
        const float t01 = p1 ? w.tm1 : w.tm0;
        const bool p2 = w.tm2 < t01;
        const uint32_t inc = p2 ? (1u << 20) : (p1 ? (1u << 10) : 1u);
        w.nrem -= inc;
        w.cb -= inc;
        const float tdb = p2 ? w.td2 : (p1 ? w.td1 : w.td0);
        const float nt = (w.nrem & (inc << 9)) ? __fadd_rn(p2 ? w.tm2 : t01, tdb) : INF;
        w.tm0 = (p1 || p2) ? w.tm0 : nt;
        w.tm1 = (p1 && !p2) ? nt : w.tm1;
        w.tm2 = p2 ? nt : w.tm2;
        const int dlb = p2 ? w.dl2 : (p1 ? w.dl1 : w.dl0);
        w.dist += p2 ? w.dd2 : (p1 ? w.dd1 : w.dd0);
        w.l += dlb;
        if ((w.cb & (inc << 3)) == 0) {   // crossed into the neighbouring block
          w.cb += inc << 3;
          w.l -= 8 * dlb;
          const int shift = p2 ? 0 : (p1 ? 21 : 42);
          key += dlb > 0 ? (1ull << shift) : (0ull - (1ull << shift));
          if (key == key_end) {
            slot = slot_end;
            pool = pool_end;
          } else {
            slot = kLocal ? local_slot(t, lb, key) : -1;
            pool = slot < 0 ? cached_pool(m, t, key, ep) : -1;
          }
        }
      }
    }
    __syncwarp();   // the next gather rewrites the list
  }
  __syncthreads();
  if (kLocal) {
    // allocation: each distinct block of the tile's shared slots is activated once
    for (int q = tid; q < lb; q += kTileThreads) {
      const unsigned long long key = t.mkey[q];
      t.pool[q] = key == kEmptyKey ? -1 : cached_pool(m, t, key, ep);
    }
    __syncthreads();
    flush_slots(m, t, lb, fx, tag);   // the tile's sums into the per-scan accumulators
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n_obs += __shfl_xor_sync(0xffffffffu, n_obs, o);
    n_valid += __shfl_xor_sync(0xffffffffu, n_valid, o);
  }
  if (lane == 0) {
    t.red[tid >> 5] = n_obs;
    t.red[kTileThreads / 32 + (tid >> 5)] = n_valid;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long a = 0, c = 0;
    for (int w = 0; w < kTileThreads / 32; ++w) {
      a += t.red[w];
      c += t.red[kTileThreads / 32 + w];
    }
    if (a) atomicAdd(&m.st->obs, a);
    if (c) atomicAdd(&m.st->valid_pts, c);
  }
  __syncthreads();   // shared memory is reused by the caller's next tile
}

// lb > 0: per-voxel sums of up to lb blocks in shared memory, flushed once per
// tile; lb == 0: every observation is a vector atomic on the block's global
// per-scan sums (the L2 performs the float additions).  The accumulation and
// drop-off modes are compile-time variants.
template <bool kCarve>
__device__ inline void integrate_tile_c(const SubmapDev& m, const ScanDev& sc, int tile, char* smem, int lb) {
  if (lb > 0) {
    if (sc.dropoff == 0) integrate_tile_legacy<true, 0, kCarve>(m, sc, tile, smem, lb);
    else if (sc.dropoff == 1) integrate_tile_legacy<true, 1, kCarve>(m, sc, tile, smem, lb);
    else integrate_tile_legacy<true, 2, kCarve>(m, sc, tile, smem, lb);
  } else {
    if (sc.dropoff == 0) integrate_tile_legacy<false, 0, kCarve>(m, sc, tile, smem, lb);
    else if (sc.dropoff == 1) integrate_tile_legacy<false, 1, kCarve>(m, sc, tile, smem, lb);
    else integrate_tile_legacy<false, 2, kCarve>(m, sc, tile, smem, lb);
  }
}

template <bool kLocal>
__device__ inline void integrate_tile_d(const SubmapDev& m, const ScanDev& sc, int tile, char* smem, int lb) {
  if (sc.dropoff == 0) integrate_tile_t<kLocal, 0>(m, sc, tile, smem, lb);
  else if (sc.dropoff == 1) integrate_tile_t<kLocal, 1>(m, sc, tile, smem, lb);
  else integrate_tile_t<kLocal, 2>(m, sc, tile, smem, lb);
}

// Any scan: accumulation mode, drop-off and form chosen at run time (carved
// rays and very long bands take the general per-thread form, whose extra
// registers the plain variants need not hold).
// Colour scans (sc.rgb) take the general form in the L2 accumulation mode
// (their host descriptors carry lb == 0).
__device__ inline void integrate_tile(const SubmapDev& m, const ScanDev& sc, int tile, char* smem, int lb) {
  if (sc.carve) integrate_tile_c<true>(m, sc, tile, smem, lb);
  else if (sc.long_band || sc.rgb) integrate_tile_c<false>(m, sc, tile, smem, lb);
  else if (lb > 0) integrate_tile_d<true>(m, sc, tile, smem, lb);
  else integrate_tile_d<false>(m, sc, tile, smem, lb);
}

// Variant index of a scan: accumulation mode x drop-off (0..5), so a launch
// whose scans share one variant runs a kernel holding only that code.
// general: carving, bands longer than 512 cells per axis, or colours.
__host__ __device__ inline int tile_variant(int lb, int dropoff, int general) {
  return general ? -1 : (lb > 0 ? 3 : 0) + dropoff;   // -1: the run-time dispatching kernel
}

template <int kVariant>
__device__ __forceinline__ void integrate_tile_v(const SubmapDev& m, const ScanDev& sc, int tile, char* smem,
                                                 int lb) {
  if (kVariant < 0) integrate_tile(m, sc, tile, smem, lb);
  else integrate_tile_t<(kVariant >= 3), (kVariant % 3)>(m, sc, tile, smem, lb);
}

// ------------------------------------------------------------- merge
// Merge of one scan's sums into D and W, group by group.  A CTA of 256
// threads merges the blocks of eight spans of kSpanBlocks consecutive pool
// indices (one span per warp; the spans strided, so that touched blocks that
// cluster in pool order spread over the CTAs of a merge) in three steps,
// each one round of independent loads:
//   1. the spans' touch epochs: the blocks holding the scan's epoch `ep`
//      (the stream compaction of the allocation pass, Sec. III-D) are
//      compacted into a list;
//   2. the touch tags of those blocks' groups (16 per thread): the groups
//      holding the scan's tag are compacted into a list of (block, group)
//      items, at most 16 per thread;
//   3. the items, one per thread at a time: the group's sums, D and W
//      loaded together, D <- (D W + sum w d)/(W + sum w), W <- min(W + sum
//      w, max_weight) for its voxels with sum w > 0 (and the colour update
//      of colour submaps), stores, and the group's sums cleared.
// skip (the scan had a device error): the sums are only cleared.
constexpr int kSpanBlocks = 32;                  // blocks of one span (one warp's epochs)
constexpr int kSpansPerCall = kTileThreads / 32; // spans one merge_span call covers
constexpr int kCallBlocks = kSpanBlocks * kSpansPerCall;
constexpr int kTagChunks = kGroupsPerBlock / 16; // 16-byte chunks of a block's tags
constexpr int kMergeItems = 16 * kTileThreads;   // items of one round of tag chunks

struct MergeSmem {
  int* pool;              // [kCallBlocks] touched blocks of the spans
  unsigned short* item;   // [kMergeItems] (index into pool) << 7 | group
  int* wsum;              // [kTileThreads / 32] per-warp partial sums
};

struct MergeSmemStatic {
  int pool[kCallBlocks];
  unsigned short item[kMergeItems];
  int wsum[kTileThreads / 32];
  __device__ MergeSmem view() { return MergeSmem{pool, item, wsum}; }
};

// The merge's lists inside a tile CTA's dynamic shared memory (any lb): a
// CTA runs either a tile or a merge at a time.
__device__ inline MergeSmem merge_smem(char* smem) {
  const TileSmem t = tile_smem(smem, 0);
  static_assert(kCache * 8 >= kCallBlocks * 4, "touched-block list fits the block cache");
  static_assert((kTileThreads / 32) * kListPerWarp * 4 >= kMergeItems * 2, "item list fits the point lists");
  return MergeSmem{reinterpret_cast<int*>(t.ckey), reinterpret_cast<unsigned short*>(t.list),
                   reinterpret_cast<int*>(t.red)};
}

// Exclusive prefix sum of v over the CTA; *total gets the sum (every thread).
__device__ __forceinline__ int cta_exclusive_scan(int v, int* wsum, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  int off = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kTileThreads / 32; ++w) {
    const int t = wsum[w];
    off += w < warp ? t : 0;
    tot += t;
  }
  __syncthreads();   // wsum is reused by the next scan
  *total = tot;
  return off + x - v;
}

// Bits of the bytes of w equal to the byte in every lane of t4 (byte k -> bit k).
__device__ __forceinline__ uint32_t tag_bits4(uint32_t w, uint32_t t4) {
  return ((__vcmpeq4(w, t4) & 0x01010101u) * 0x01020408u) >> 24;
}

template <int kStore>
struct Vox4;

template <>
struct Vox4<0> {
  static __device__ __forceinline__ void load(const SubmapDev& m, size_t e, float D[4], float W[4]) {
    const float4 d = __ldcg(reinterpret_cast<const float4*>((const float*)m.D + e));
    const float4 w = __ldcg(reinterpret_cast<const float4*>((const float*)m.W + e));
    D[0] = d.x; D[1] = d.y; D[2] = d.z; D[3] = d.w;
    W[0] = w.x; W[1] = w.y; W[2] = w.z; W[3] = w.w;
  }
  static __device__ __forceinline__ void store(const SubmapDev& m, size_t e, const float D[4], const float W[4]) {
    *reinterpret_cast<float4*>((float*)m.D + e) = make_float4(D[0], D[1], D[2], D[3]);
    *reinterpret_cast<float4*>((float*)m.W + e) = make_float4(W[0], W[1], W[2], W[3]);
  }
};

template <>
struct Vox4<1> {   // FP16 storage: D / trunc and W as IEEE half, FP32 arithmetic
  static __device__ __forceinline__ void load(const SubmapDev& m, size_t e, float D[4], float W[4]) {
    const uint2 d = __ldcg(reinterpret_cast<const uint2*>((const __half*)m.D + e));
    const uint2 w = __ldcg(reinterpret_cast<const uint2*>((const __half*)m.W + e));
    const __half2* dh = reinterpret_cast<const __half2*>(&d);
    const __half2* wh = reinterpret_cast<const __half2*>(&w);
    const float2 d0 = __half22float2(dh[0]), d1 = __half22float2(dh[1]);
    const float2 w0 = __half22float2(wh[0]), w1 = __half22float2(wh[1]);
    D[0] = d0.x * m.trunc; D[1] = d0.y * m.trunc; D[2] = d1.x * m.trunc; D[3] = d1.y * m.trunc;
    W[0] = w0.x; W[1] = w0.y; W[2] = w1.x; W[3] = w1.y;
  }
  static __device__ __forceinline__ void store(const SubmapDev& m, size_t e, const float D[4], const float W[4]) {
    uint2 d, w;
    __half2* dh = reinterpret_cast<__half2*>(&d);
    __half2* wh = reinterpret_cast<__half2*>(&w);
    dh[0] = __halves2half2(__float2half_rn(D[0] / m.trunc), __float2half_rn(D[1] / m.trunc));
    dh[1] = __halves2half2(__float2half_rn(D[2] / m.trunc), __float2half_rn(D[3] / m.trunc));
    wh[0] = __halves2half2(__float2half_rn(W[0]), __float2half_rn(W[1]));
    wh[1] = __halves2half2(__float2half_rn(W[2]), __float2half_rn(W[3]));
    *reinterpret_cast<uint2*>((__half*)m.D + e) = d;
    *reinterpret_cast<uint2*>((__half*)m.W + e) = w;
  }
};

// One group's loaded values: its sums (sum w (d - trunc), sum w per voxel),
// and D, W.
struct GroupVals {
  float4 s0, s1;
  float D[4], W[4];
};

template <int kStore>
__device__ __forceinline__ void load_group(const SubmapDev& m, size_t e, bool skip, GroupVals& g) {
  const float4* a = reinterpret_cast<const float4*>(m.acc + e);
  g.s0 = __ldcg(a);
  g.s1 = __ldcg(a + 1);
  if (!skip) Vox4<kStore>::load(m, e, g.D, g.W);
}

// Colour update of one group (colour submaps), before its D/W merge: C <- (C W
// + S_wc) / (W + S_w) wherever S_w != 0, W being the stored weight before the
// merge (the same rule as D); the group's colour sums are cleared.
__device__ __forceinline__ void merge_colour_group(const SubmapDev& m, size_t e, const GroupVals& g, bool skip) {
  float4* cs = m.cacc + e;
  if (!skip) {
    const float sw[4] = {g.s0.y, g.s0.w, g.s1.y, g.s1.w};
    float4 c4[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) c4[q] = __ldcg(cs + q);
    const size_t pool = e / kVoxPerBlock, v = e % kVoxPerBlock;
    float* cp = m.C + pool * 3 * kVoxPerBlock + v;
    float4 c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = __ldcg(reinterpret_cast<const float4*>(cp + k * kVoxPerBlock));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (sw[q] == 0.f) continue;
      const float wn = g.W[q] + sw[q];
      float* r = reinterpret_cast<float*>(&c[0]) + q;
      float* gr = reinterpret_cast<float*>(&c[1]) + q;
      float* b = reinterpret_cast<float*>(&c[2]) + q;
      *r = (*r * g.W[q] + c4[q].x) / wn;
      *gr = (*gr * g.W[q] + c4[q].y) / wn;
      *b = (*b * g.W[q] + c4[q].z) / wn;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) *reinterpret_cast<float4*>(cp + k * kVoxPerBlock) = c[k];
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) cs[q] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Merge of one loaded group; returns its merged voxels.
template <int kStore, bool kColour>
__device__ __forceinline__ int merge_group(const SubmapDev& m, size_t e, GroupVals& g, bool skip) {
  const float sw[4] = {g.s0.x, g.s0.z, g.s1.x, g.s1.z}, w[4] = {g.s0.y, g.s0.w, g.s1.y, g.s1.w};
  if (w[0] == 0.f && w[1] == 0.f && w[2] == 0.f && w[3] == 0.f) return 0;   // weight-0 observations only
  if (kColour && m.C) merge_colour_group(m, e, g, skip);
  int merged = 0;
  if (!skip) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (w[q] != 0.0f) {
        const float wn = g.W[q] + w[q];
        g.D[q] = m.trunc + ((g.D[q] - m.trunc) * g.W[q] + sw[q]) / wn;
        g.W[q] = fminf(wn, m.max_w);
        ++merged;
      }
    Vox4<kStore>::store(m, e, g.D, g.W);
  }
  float4* a = reinterpret_cast<float4*>(m.acc + e);
  a[0] = make_float4(0.f, 0.f, 0.f, 0.f);
  a[1] = make_float4(0.f, 0.f, 0.f, 0.f);
  return merged;
}

// The listed items, one per thread at a time: the group's sums, D and W
// are loaded together.  (Two items in flight per thread cost spills in the
// tile code of the kernels that hold both phases.)
template <int kStore, bool kColour>
__device__ __forceinline__ int merge_items(const SubmapDev& m, const MergeSmem& ms, int n_items, bool skip) {
  int merged = 0;
  for (int i = threadIdx.x; i < n_items; i += kTileThreads) {
    const unsigned it = ms.item[i];
    const size_t e = (size_t)ms.pool[it >> 7] * kVoxPerBlock + 4 * (it & 127u);
    GroupVals g;
    load_group<kStore>(m, e, skip, g);
    merged += merge_group<kStore, kColour>(m, e, g, skip);
  }
  return merged;
}

// Merge of the spans span0 + w * step (w = 0 .. kSpansPerCall - 1, warp w
// takes span w) of a submap with nb allocated blocks.  Returns this thread's
// merged voxels; *touched (every thread) gets the spans' touched blocks.
// kColour: the colour update of colour submaps is compiled in (kernels whose
// scans include no colour scan, and so no colour submap, leave it out).
template <bool kColour = true>
__device__ __forceinline__ int merge_span(const SubmapDev& m, int span0, int step, int nb, uint32_t ep, bool skip,
                                          const MergeSmem& ms, int* touched) {
  const int tid = threadIdx.x;
  const long long p = (long long)(span0 + (tid >> 5) * step) * kSpanBlocks + (tid & 31);
  const bool t = p < nb && __ldcg(m.tepoch + p) == ep;
  int cnt = 0;
  const int o = cta_exclusive_scan(t ? 1 : 0, ms.wsum, &cnt);
  if (t) ms.pool[o] = (int)p;
  *touched = cnt;
  if (cnt == 0) return 0;   // uniform over the CTA
  __syncthreads();
  const uint8_t tag = group_tag(ep);
  const uint32_t t4 = 0x01010101u * tag;
  const int n_chunks = cnt * kTagChunks;
  const uint4* tags = reinterpret_cast<const uint4*>(m.gep);
  // the next round's tag chunk is loaded while the current round is merged
  uint4 next = make_uint4(0u, 0u, 0u, 0u);
  if (tid < n_chunks) next = __ldcg(tags + (size_t)ms.pool[tid / kTagChunks] * kTagChunks + tid % kTagChunks);
  int merged = 0;
  for (int c0 = 0; c0 < n_chunks; c0 += kTileThreads) {
    const int c = c0 + tid;
    const uint4 g = next;
    const int cn = c + kTileThreads;
    if (cn < n_chunks) next = __ldcg(tags + (size_t)ms.pool[cn / kTagChunks] * kTagChunks + cn % kTagChunks);
    uint32_t bits = 0;
    if (c < n_chunks)
      bits = tag_bits4(g.x, t4) | (tag_bits4(g.y, t4) << 4) | (tag_bits4(g.z, t4) << 8) | (tag_bits4(g.w, t4) << 12);
    int n_items = 0;
    int k = cta_exclusive_scan(__popc(bits), ms.wsum, &n_items);
    const unsigned base = (unsigned)(c / kTagChunks) << 7 | (unsigned)(c % kTagChunks) * 16u;
    while (bits) {
      const int b = __ffs(bits) - 1;
      bits &= bits - 1;
      ms.item[k++] = (unsigned short)(base + b);
    }
    __syncthreads();
    merged += m.storage == 0 ? merge_items<0, kColour>(m, ms, n_items, skip)
                             : merge_items<1, kColour>(m, ms, n_items, skip);
    __syncthreads();   // the item list is rewritten by the next round
  }
  return merged;
}

}  // namespace covox
