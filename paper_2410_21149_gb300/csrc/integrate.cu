// integrate.cu -- the integration kernels and the C ABI of one submap.
//
// Per scan (one frame), three kernels on the caller's stream implement the
// count / allocate / process sequence of coVoxSLAM Sec. III-D:
//   K1 alloc_kernel   : one thread per point; band traversal; the distinct
//                       blocks of the point are deduplicated across the warp
//                       (__match_any_sync) and the leader activates them in
//                       the block hash (insert-or-find, Sec. III-B), takes a
//                       pool index for new blocks by atomic bump (allocation
//                       phase) and gives the scan's first toucher of a block a
//                       per-scan slot j (stream compaction of touched blocks).
//   K2 accum_kernel   : one CTA per tile of points; the traversal again, each
//                       observation's w*d and w summed in a shared-memory table
//                       keyed by (j, voxel) and flushed once per tile with
//                       vector atomics into the per-scan accumulator
//                       (segmented reduction of commutative sums, Sec. III-D).
//   K3 merge_kernel   : one CTA per touched block; reads the block's sums,
//                       merges them into D and W with coalesced vector loads and
//                       stores, clears the sums, and the last CTA resets the
//                       per-scan state.  One owner per block: no write races.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/covox.h"
#include "covox_dev.cuh"
#include "prof.h"

using namespace covox;

namespace {

constexpr int kAllocThreads = 256;
constexpr int kAccThreads = 256;
constexpr int kTblLog2 = 11;                 // shared table: 2048 (key, sum w d, sum w)
constexpr int kTbl = 1 << kTblLog2;
constexpr int kTblProbe = 8;
constexpr int kMergeThreads = 128;           // 4 voxels per thread
constexpr int kMaxBlocksPerPoint = 8;        // warp-aggregated; more are activated one by one

// ------------------------------------------------------------------ K1
__device__ void activate_and_claim(const SubmapDev& m, unsigned long long key, int bx, int by, int bz) {
  bool inserted;
  const int s = hash_activate(m, key, &inserted);
  if (s < 0) {
    atomicOr(&m.st->frame_err, kErrCapacity);
    return;
  }
  if (inserted) {
    const int pool = atomicAdd(&m.st->n_blocks, 1);
    if (pool >= m.max_blocks) {
      atomicOr(&m.st->frame_err, kErrCapacity);
      m.vals[s] = -1;
    } else {
      m.vals[s] = pool;
      m.block_keys[3 * pool] = bx;
      m.block_keys[3 * pool + 1] = by;
      m.block_keys[3 * pool + 2] = bz;
    }
  }
  if (*((volatile int32_t*)(m.touch + s)) == -1 && atomicCAS(m.touch + s, -1, -2) == -1) {
    const int j = atomicAdd(&m.st->n_touched, 1);
    if (j < m.max_touched) {
      m.touched[j] = s;
      m.touch[s] = j;
    } else {
      atomicOr(&m.st->frame_err, kErrCapacity);
      m.touch[s] = -1;
    }
  }
}

__global__ void __launch_bounds__(kAllocThreads) alloc_kernel(SubmapDev m, ScanDev sc) {
  const int lane = threadIdx.x & 31;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long bk[kMaxBlocksPerPoint];
  int nb = 0;
  bool overflow = false;
  Ray r;
  float A[3], B[3];
  if (i < sc.n && make_ray(sc, i, r)) {
    if (!band(r, m.trunc, m.inv_vs, A, B)) {
      atomicOr(&m.st->frame_err, kErrKeyRange);
    } else {
      Dda t;
      t.init(A, B);
      int cb0 = t.v[0] >> 3, cb1 = t.v[1] >> 3, cb2 = t.v[2] >> 3;
      bk[0] = pack_key(cb0, cb1, cb2);
      nb = 1;
      while (t.left > 0) {
        t.step();
        const int b0 = t.v[0] >> 3, b1 = t.v[1] >> 3, b2 = t.v[2] >> 3;
        if (b0 != cb0 || b1 != cb1 || b2 != cb2) {
          cb0 = b0; cb1 = b1; cb2 = b2;
          const unsigned long long k = pack_key(b0, b1, b2);
#pragma unroll
          for (int q = 0; q < kMaxBlocksPerPoint; ++q)
            if (q == nb) bk[q] = k;
          if (nb < kMaxBlocksPerPoint) ++nb; else overflow = true;
        }
      }
    }
  }
  // Warp-aggregated activation: equal keys in a round are handled once.
#pragma unroll
  for (int q = 0; q < kMaxBlocksPerPoint; ++q) {
    const bool has = q < nb;
    if (__ballot_sync(0xffffffffu, has) == 0u) break;
    const unsigned long long key = has ? bk[q] : kEmptyKey;
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    if (has && lane == __ffs(grp) - 1) {
      const int bx = (int)((key >> 42) & 0x1fffff) - (1 << 20);
      const int by = (int)((key >> 21) & 0x1fffff) - (1 << 20);
      const int bz = (int)(key & 0x1fffff) - (1 << 20);
      activate_and_claim(m, key, bx, by, bz);
    }
  }
  if (overflow) {  // rare: more distinct blocks than the register list holds
    Dda t;
    t.init(A, B);
    int cb0 = t.v[0] >> 3, cb1 = t.v[1] >> 3, cb2 = t.v[2] >> 3, seen = 1;
    while (t.left > 0) {
      t.step();
      const int b0 = t.v[0] >> 3, b1 = t.v[1] >> 3, b2 = t.v[2] >> 3;
      if (b0 != cb0 || b1 != cb1 || b2 != cb2) {
        cb0 = b0; cb1 = b1; cb2 = b2;
        if (++seen > kMaxBlocksPerPoint) activate_and_claim(m, pack_key(b0, b1, b2), b0, b1, b2);
      }
    }
  }
}

// ------------------------------------------------------------------ K2
struct AccTable {
  int key[kTbl];
  float swd[kTbl];
  float sw[kTbl];
};

__device__ __forceinline__ void table_add(AccTable& t, const SubmapDev& m, int addr, float wd, float w) {
  uint32_t h = ((uint32_t)addr * 2654435761u) >> (32 - kTblLog2);
#pragma unroll 1
  for (int p = 0; p < kTblProbe; ++p) {
    const int q = (h + p) & (kTbl - 1);
    int k = *((volatile int*)&t.key[q]);
    if (k == -1) k = atomicCAS(&t.key[q], -1, addr), k = (k == -1) ? addr : k;
    if (k == addr) {
      atomicAdd(&t.swd[q], wd);
      atomicAdd(&t.sw[q], w);
      return;
    }
  }
  atomicAdd(m.acc + addr, make_float2(wd, w));
}

__global__ void __launch_bounds__(kAccThreads) accum_kernel(SubmapDev m, ScanDev sc, int pts_per_cta) {
  __shared__ AccTable tbl;
  __shared__ unsigned long long red_obs[kAccThreads / 32], red_valid[kAccThreads / 32];
  for (int q = threadIdx.x; q < kTbl; q += blockDim.x) {
    tbl.key[q] = -1;
    tbl.swd[q] = 0.0f;
    tbl.sw[q] = 0.0f;
  }
  __syncthreads();
  const long long base = (long long)blockIdx.x * pts_per_cta;
  const long long end = min(base + (long long)pts_per_cta, sc.n);
  unsigned long long n_obs = 0, n_valid = 0;
  for (long long i = base + threadIdx.x; i < end; i += blockDim.x) {
    Ray r;
    if (!make_ray(sc, i, r)) continue;
    float A[3], B[3];
    if (!band(r, m.trunc, m.inv_vs, A, B)) continue;
    ++n_valid;
    const float w0 = base_weight(sc, i, r);
    Dda t;
    t.init(A, B);
    int cb0 = 0x7fffffff, cb1 = 0, cb2 = 0, j = -1;
    for (;;) {
      const int b0 = t.v[0] >> 3, b1 = t.v[1] >> 3, b2 = t.v[2] >> 3;
      if (b0 != cb0 || b1 != cb1 || b2 != cb2) {
        cb0 = b0; cb1 = b1; cb2 = b2;
        const int s = hash_find(m, pack_key(b0, b1, b2));
        j = s >= 0 ? __ldg(m.touch + s) : -1;
      }
      if (j >= 0) {
        const float d = voxel_distance(r, t.v, m.vs, m.trunc);
        const float w = dropoff_weight(w0, d, m.vs, m.trunc, sc.dropoff);
        table_add(tbl, m, j * kVoxPerBlock + local_index(t.v), w * d, w);
      }
      ++n_obs;
      if (t.left == 0) break;
      t.step();
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < kTbl; q += blockDim.x) {
    const int k = tbl.key[q];
    if (k >= 0) atomicAdd(m.acc + k, make_float2(tbl.swd[q], tbl.sw[q]));
  }
  // per-CTA counters
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n_obs += __shfl_xor_sync(0xffffffffu, n_obs, o);
    n_valid += __shfl_xor_sync(0xffffffffu, n_valid, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red_obs[threadIdx.x >> 5] = n_obs;
    red_valid[threadIdx.x >> 5] = n_valid;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a = 0, b = 0;
    for (int w = 0; w < kAccThreads / 32; ++w) { a += red_obs[w]; b += red_valid[w]; }
    if (a) atomicAdd(&m.st->obs, a);
    if (b) atomicAdd(&m.st->valid_pts, b);
  }
}

// ------------------------------------------------------------------ K3
template <int kStore>
struct Vox4;

template <>
struct Vox4<CVX_STORE_F32> {
  static __device__ __forceinline__ void load(const SubmapDev& m, size_t e, float D[4], float W[4]) {
    const float4 d = *reinterpret_cast<const float4*>((const float*)m.D + e);
    const float4 w = *reinterpret_cast<const float4*>((const float*)m.W + e);
    D[0] = d.x; D[1] = d.y; D[2] = d.z; D[3] = d.w;
    W[0] = w.x; W[1] = w.y; W[2] = w.z; W[3] = w.w;
  }
  static __device__ __forceinline__ void store(const SubmapDev& m, size_t e, const float D[4], const float W[4]) {
    *reinterpret_cast<float4*>((float*)m.D + e) = make_float4(D[0], D[1], D[2], D[3]);
    *reinterpret_cast<float4*>((float*)m.W + e) = make_float4(W[0], W[1], W[2], W[3]);
  }
};

template <>
struct Vox4<CVX_STORE_F16> {
  static __device__ __forceinline__ void load(const SubmapDev& m, size_t e, float D[4], float W[4]) {
    const uint2 d = *reinterpret_cast<const uint2*>((const __half*)m.D + e);
    const uint2 w = *reinterpret_cast<const uint2*>((const __half*)m.W + e);
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

template <int kStore>
__global__ void __launch_bounds__(kMergeThreads) merge_kernel(SubmapDev m) {
  __shared__ unsigned long long red[kMergeThreads / 32];
  const int nt = min(*((volatile int32_t*)&m.st->n_touched), m.max_touched);
  const bool skip = *((volatile int32_t*)&m.st->frame_err) != 0;
  const int tid = threadIdx.x;
  unsigned long long merged = 0;
  for (int j = blockIdx.x; j < nt; j += gridDim.x) {
    const int s = m.touched[j];
    const int pool = m.vals[s];
    float4* a = reinterpret_cast<float4*>(m.acc + (size_t)j * kVoxPerBlock) + 2 * tid;
    const float4 a0 = a[0], a1 = a[1];
    const float swd[4] = {a0.x, a0.z, a1.x, a1.z};
    const float sw[4] = {a0.y, a0.w, a1.y, a1.w};
    const bool any = (sw[0] != 0.0f) | (sw[1] != 0.0f) | (sw[2] != 0.0f) | (sw[3] != 0.0f);
    if (any) {
      if (!skip && pool >= 0) {
        const size_t e = (size_t)pool * kVoxPerBlock + 4 * tid;
        float D[4], W[4];
        Vox4<kStore>::load(m, e, D, W);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (sw[q] != 0.0f) {
            const float wn = W[q] + sw[q];
            D[q] = (D[q] * W[q] + swd[q]) / wn;
            W[q] = fminf(wn, m.max_w);
            ++merged;
          }
        }
        Vox4<kStore>::store(m, e, D, W);
      }
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      a[0] = z;
      a[1] = z;
    }
    if (tid == 0) m.touch[s] = -1;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) merged += __shfl_xor_sync(0xffffffffu, merged, o);
  if ((tid & 31) == 0) red[tid >> 5] = merged;
  __syncthreads();
  if (tid == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kMergeThreads / 32; ++w) t += red[w];
    if (t) atomicAdd(&m.st->voxels_merged, t);
    __threadfence();
    const unsigned ticket = atomicAdd(&m.st->ticket, 1u);
    if (ticket == gridDim.x - 1) {  // last CTA: every CTA has finished reading
      __threadfence();
      State* st = m.st;
      st->blocks_touched += (unsigned long long)nt;
      st->frames += 1;
      st->sticky_err |= st->frame_err;
      st->frame_err = 0;
      st->n_touched = 0;
      st->ticket = 0;
    }
  }
}

// Zero the allocated part of the pool (reset).
__global__ void zero_pool_kernel(SubmapDev m, int bytes_per_block) {
  const long long nbytes = (long long)min(m.st->n_blocks, m.max_blocks) * bytes_per_block;
  const long long n16 = nbytes / 16;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n16; q += stride) {
    reinterpret_cast<uint4*>(m.D)[q] = make_uint4(0, 0, 0, 0);
    reinterpret_cast<uint4*>(m.W)[q] = make_uint4(0, 0, 0, 0);
  }
}

int g_num_sms = 0;
int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  }
  return g_num_sms;
}

}  // namespace

// ===================================================================== C ABI
struct cvx_submap {
  cvx_submap_params p;
  SubmapDev dev;
  size_t bytes_per_vox;
  cudaStream_t last_stream;
  struct Alloc { void* ptr; size_t bytes; } allocs[10];
  int n_allocs;
};

namespace {

void* sub_alloc(cvx_submap* m, size_t bytes) {
  void* ptr = nullptr;
  if (m->p.alloc) {
    ptr = m->p.alloc(bytes, m->p.stream, m->p.alloc_ctx);
  } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
  }
  if (ptr) m->allocs[m->n_allocs++] = {ptr, bytes};
  return ptr;
}

void sub_free_all(cvx_submap* m) {
  for (int q = m->n_allocs - 1; q >= 0; --q) {
    if (m->p.free) m->p.free(m->allocs[q].ptr, m->allocs[q].bytes, m->p.stream, m->p.alloc_ctx);
    else if (!m->p.alloc) cudaFree(m->allocs[q].ptr);
  }
  m->n_allocs = 0;
}

bool finite12(const float* T) {
  for (int q = 0; q < 12; ++q)
    if (!std::isfinite(T[q])) return false;
  return true;
}

cvx_status status_from_bits(int bits) {
  if (bits & kErrCapacity) return CVX_ERR_CAPACITY;
  if (bits & kErrKeyRange) return CVX_ERR_KEY_RANGE;
  if (bits & kErrTimeout) return CVX_ERR_TIMEOUT;
  return CVX_OK;
}

}  // namespace

extern "C" {

const char* cvx_version(void) { return "covox-gb300 0.1 (sm_103a)"; }

cvx_status cvx_create_submap(const cvx_submap_params* p, cvx_submap** out) {
  if (!p || !out) return CVX_ERR_INVALID_ARG;
  *out = nullptr;
  if (!(p->voxel_size > 0) || !(p->trunc > 0) || !(p->max_weight > 0) ||
      !std::isfinite(p->voxel_size) || !std::isfinite(p->trunc) || !std::isfinite(p->max_weight))
    return CVX_ERR_INVALID_ARG;
  if (p->storage != CVX_STORE_F32 && p->storage != CVX_STORE_F16) return CVX_ERR_INVALID_ARG;
  if (p->max_blocks <= 0 || p->max_blocks > (1ll << 30)) return CVX_ERR_INVALID_ARG;
  if (p->hash_slots < 2 || (p->hash_slots & (p->hash_slots - 1)) || p->hash_slots > (1ll << 31))
    return CVX_ERR_INVALID_ARG;
  if (p->max_touched < 0) return CVX_ERR_INVALID_ARG;
  if (p->storage == CVX_STORE_F16 && p->max_weight > 65504.0f) return CVX_ERR_INVALID_ARG;
  if ((p->alloc == nullptr) != (p->free == nullptr)) return CVX_ERR_INVALID_ARG;

  cvx_submap* m = new (std::nothrow) cvx_submap();
  if (!m) return CVX_ERR_OOM;
  m->p = *p;
  const int64_t max_touched = p->max_touched ? std::min<int64_t>(p->max_touched, p->max_blocks)
                                             : std::min<int64_t>(p->max_blocks, 65536);
  m->p.max_touched = max_touched;
  const size_t slots = (size_t)p->hash_slots, nb = (size_t)p->max_blocks;
  m->bytes_per_vox = p->storage == CVX_STORE_F32 ? 4 : 2;
  SubmapDev& d = m->dev;
  d.keys = (unsigned long long*)sub_alloc(m, slots * 8);
  d.vals = (int32_t*)sub_alloc(m, slots * 4);
  d.touch = (int32_t*)sub_alloc(m, slots * 4);
  d.block_keys = (int32_t*)sub_alloc(m, nb * 12);
  d.D = sub_alloc(m, nb * kVoxPerBlock * m->bytes_per_vox);
  d.W = sub_alloc(m, nb * kVoxPerBlock * m->bytes_per_vox);
  d.acc = (float2*)sub_alloc(m, (size_t)max_touched * kVoxPerBlock * sizeof(float2));
  d.touched = (int32_t*)sub_alloc(m, (size_t)max_touched * 4);
  d.st = (State*)sub_alloc(m, sizeof(State));
  if (m->n_allocs != 9) {
    sub_free_all(m);
    delete m;
    return CVX_ERR_OOM;
  }
  d.slot_mask = (uint32_t)(slots - 1);
  d.max_probe = (int)std::min<size_t>(slots, 4096);
  d.max_blocks = (int)nb;
  d.max_touched = (int)max_touched;
  d.vs = p->voxel_size;
  d.inv_vs = 1.0f / p->voxel_size;
  d.trunc = p->trunc;
  d.max_w = p->max_weight;
  cudaStream_t s = (cudaStream_t)p->stream;
  m->last_stream = s;
  cudaMemsetAsync(d.keys, 0xff, slots * 8, s);
  cudaMemsetAsync(d.vals, 0xff, slots * 4, s);
  cudaMemsetAsync(d.touch, 0xff, slots * 4, s);
  cudaMemsetAsync(d.D, 0, nb * kVoxPerBlock * m->bytes_per_vox, s);
  cudaMemsetAsync(d.W, 0, nb * kVoxPerBlock * m->bytes_per_vox, s);
  cudaMemsetAsync(d.acc, 0, (size_t)max_touched * kVoxPerBlock * sizeof(float2), s);
  cudaMemsetAsync(d.st, 0, sizeof(State), s);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    sub_free_all(m);
    delete m;
    return CVX_ERR_CUDA;
  }
  *out = m;
  return CVX_OK;
}

cvx_status cvx_integrate_scan(cvx_submap* map, const float* points_xyz, int64_t n,
                              const float T_sub_sensor[12], const float* point_weights,
                              const cvx_integrate_params* ip, void* stream) {
  if (!map || !ip || !T_sub_sensor || n < 0 || (n > 0 && !points_xyz)) return CVX_ERR_INVALID_ARG;
  if (!finite12(T_sub_sensor)) return CVX_ERR_INVALID_ARG;
  if (ip->weight_mode < 0 || ip->weight_mode > 2 || ip->dropoff < 0 || ip->dropoff > 2)
    return CVX_ERR_INVALID_ARG;
  if (ip->weight_mode == CVX_W_PER_POINT && n > 0 && !point_weights) return CVX_ERR_INVALID_ARG;
  if (ip->dropoff != CVX_DROP_NONE && !(map->p.trunc > map->p.voxel_size)) return CVX_ERR_INVALID_ARG;
  if (ip->sensor != 0 && ip->sensor != 1) return CVX_ERR_INVALID_ARG;
  if (!(ip->min_range >= 0) || !(ip->max_range >= ip->min_range)) return CVX_ERR_INVALID_ARG;
  if (ip->pts_per_cta < 0 || ip->pts_per_cta > (1 << 20)) return CVX_ERR_INVALID_ARG;
  if (n > (1ll << 31)) return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  map->last_stream = s;
  if (n == 0) return CVX_OK;
  ScanDev sc;
  sc.pts = points_xyz;
  sc.pw = point_weights;
  sc.n = n;
  std::memcpy(sc.T, T_sub_sensor, sizeof(sc.T));
  sc.min_range = ip->min_range;
  sc.max_range = ip->max_range;
  sc.weight_mode = ip->weight_mode;
  sc.dropoff = ip->dropoff;
  sc.sensor = ip->sensor;
  sc.pad = 0;
  const int ppc = ip->pts_per_cta > 0 ? ip->pts_per_cta : 512;
  COVOX_LAUNCH(kKAlloc, s,
               alloc_kernel<<<(unsigned)((n + kAllocThreads - 1) / kAllocThreads), kAllocThreads, 0, s>>>(
                   map->dev, sc));
  COVOX_LAUNCH(kKAccum, s, accum_kernel<<<(unsigned)((n + ppc - 1) / ppc), kAccThreads, 0, s>>>(map->dev, sc, ppc));
  const int grid = std::min<int>(map->dev.max_touched, num_sms() * 8);
  if (map->p.storage == CVX_STORE_F32)
    COVOX_LAUNCH(kKMerge, s, merge_kernel<CVX_STORE_F32><<<grid, kMergeThreads, 0, s>>>(map->dev));
  else
    COVOX_LAUNCH(kKMerge, s, merge_kernel<CVX_STORE_F16><<<grid, kMergeThreads, 0, s>>>(map->dev));
  return cudaGetLastError() == cudaSuccess ? CVX_OK : CVX_ERR_CUDA;
}

cvx_status cvx_extract_blocks(cvx_submap* map, int64_t capacity, int32_t* keys, void* dist,
                              void* weight, int64_t* n_out, void* stream) {
  if (!map || !n_out || capacity < 0) return CVX_ERR_INVALID_ARG;
  if (keys && capacity > 0 && (!dist || !weight)) return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t nb = 0;
  if (cudaMemcpyAsync(&nb, &map->dev.st->n_blocks, sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  nb = std::min<int32_t>(nb, map->dev.max_blocks);
  if (!keys) {
    *n_out = nb;
    return CVX_OK;
  }
  const int64_t n = std::min<int64_t>(nb, capacity);
  *n_out = n;
  if (n == 0) return CVX_OK;
  const size_t vb = (size_t)n * kVoxPerBlock * map->bytes_per_vox;
  if (cudaMemcpyAsync(keys, map->dev.block_keys, (size_t)n * 12, cudaMemcpyDefault, s) != cudaSuccess ||
      cudaMemcpyAsync(dist, map->dev.D, vb, cudaMemcpyDefault, s) != cudaSuccess ||
      cudaMemcpyAsync(weight, map->dev.W, vb, cudaMemcpyDefault, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  return CVX_OK;
}

cvx_status cvx_reset_submap(cvx_submap* map, void* stream) {
  if (!map) return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  map->last_stream = s;
  const int bpb = (int)(kVoxPerBlock * map->bytes_per_vox);
  COVOX_LAUNCH(kKZeroPool, s, zero_pool_kernel<<<num_sms() * 4, 256, 0, s>>>(map->dev, bpb));
  cudaMemsetAsync(map->dev.keys, 0xff, (size_t)map->p.hash_slots * 8, s);
  cudaMemsetAsync(map->dev.vals, 0xff, (size_t)map->p.hash_slots * 4, s);
  cudaMemsetAsync(map->dev.st, 0, sizeof(State), s);
  return cudaGetLastError() == cudaSuccess ? CVX_OK : CVX_ERR_CUDA;
}

cvx_status cvx_submap_counters(cvx_submap* map, cvx_counters* out) {
  if (!map || !out) return CVX_ERR_INVALID_ARG;
  State st;
  if (cudaMemcpyAsync(&st, map->dev.st, sizeof(State), cudaMemcpyDeviceToHost, map->last_stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(map->last_stream) != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  out->n_blocks = std::min<int64_t>(st.n_blocks, map->dev.max_blocks);
  out->frames = (int64_t)st.frames;
  out->valid_points = (int64_t)st.valid_pts;
  out->observations = (int64_t)st.obs;
  out->voxels_merged = (int64_t)st.voxels_merged;
  out->blocks_touched = (int64_t)st.blocks_touched;
  return CVX_OK;
}

cvx_status cvx_submap_status(cvx_submap* map) {
  if (!map) return CVX_ERR_INVALID_ARG;
  State st;
  if (cudaMemcpyAsync(&st, map->dev.st, sizeof(State), cudaMemcpyDeviceToHost, map->last_stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(map->last_stream) != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  return status_from_bits(st.sticky_err | st.frame_err);
}

void cvx_destroy(cvx_submap* map) {
  if (!map) return;
  cudaStreamSynchronize(map->last_stream);
  sub_free_all(map);
  delete map;
}

}  // extern "C"
