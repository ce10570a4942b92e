// esdf.cu -- Euclidean distance field of a submap (coVoxSLAM Sec. III-E),
// and the submap queries of the backend (registration points, bounds).
//
// For every voxel of every allocated block: the distance between its centre
// and the centre of the nearest site voxel (W > w_min and |D| <= site_band),
// capped at max_dist.  The paper updates its ESDF incrementally with
// per-block queues and Parallel Banding (PBA) sweeps; this library computes
// the same exact field from scratch for a whole submap:
//   esdf_bbox_kernel   the voxel box spanned by the allocated blocks;
//   esdf_sites_kernel  sites marked 0 in a dense int32 grid of the box (the
//                      rest stays "far");
//   esdf_first_pass_kernel  x lines: squared distance to the line's nearest
//                      site, one sweep each way;
//   esdf_pass_kernel   y then z lines, one thread per line: the lower
//                      envelope of the parabolas (q - p)^2 + f(p) of the
//                      line's finite entries, intersections compared as
//                      exact integer fractions, so each pass returns the
//                      exact minimum (squared distances in voxel units);
//   esdf_out_kernel    gather into the blocks' [n_blocks, 512] layout.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>

#include "../../include/covox.h"
#include "covox_dev.cuh"
#include "prof.h"
#include "submap.h"

using namespace covox;

namespace {

constexpr int32_t kFar = 0x7f7f7f7f;       // memset byte 0x7f: no site on the line (yet)
constexpr int kMaxAxis = 16384;            // voxels per box axis: 3 * 16383^2 + 16383^2 < kFar

__global__ void esdf_bbox_kernel(const int32_t* __restrict__ block_keys, int nb, int* box) {
  int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int k = block_keys[3 * b + c];
      mn[c] = min(mn[c], k);
      mx[c] = max(mx[c], k);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    mn[c] = __reduce_min_sync(0xffffffffu, mn[c]);
    mx[c] = __reduce_max_sync(0xffffffffu, mx[c]);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      atomicMin(box + c, mn[c]);
      atomicMax(box + 3 + c, mx[c]);
    }
  }
}

__global__ void esdf_box_init_kernel(int* box) {
  if (threadIdx.x < 3) {
    box[threadIdx.x] = INT_MAX;
    box[3 + threadIdx.x] = INT_MIN;
  }
}

struct Box {
  int lo[3];    // lowest voxel index
  int n[3];     // extents in voxels
};

__device__ __forceinline__ size_t grid_index(const Box& bx, int v0, int v1, int v2) {
  return (size_t)(v0 - bx.lo[0]) + (size_t)bx.n[0] * ((size_t)(v1 - bx.lo[1]) + (size_t)bx.n[1] * (v2 - bx.lo[2]));
}

__global__ void esdf_sites_kernel(SubmapDev m, int nb, Box bx, float site_band, float w_min,
                                  int32_t* __restrict__ grid) {
  const size_t total = (size_t)nb * kVoxPerBlock;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / kVoxPerBlock), l = (int)(e % kVoxPerBlock);
    float D, W;
    if (m.storage == CVX_STORE_F32) {
      D = ((const float*)m.D)[e];
      W = ((const float*)m.W)[e];
    } else {
      D = __half2float(((const __half*)m.D)[e]) * m.trunc;
      W = __half2float(((const __half*)m.W)[e]);
    }
    if (!(W > w_min && fabsf(D) <= site_band)) continue;
    const int v0 = m.block_keys[3 * b] * 8 + (l & 7);
    const int v1 = m.block_keys[3 * b + 1] * 8 + ((l >> 3) & 7);
    const int v2 = m.block_keys[3 * b + 2] * 8 + (l >> 6);
    grid[grid_index(bx, v0, v1, v2)] = 0;
  }
}

// Line L of a pass: start base + q * se for q < n; scratch element k of the
// line at k * lines + L (adjacent lines adjacent in memory).
struct Pass {
  int n, lines, c0;
  long long s0, s1, se;
};

__global__ void esdf_pass_kernel(int32_t* __restrict__ grid, Pass ps, int32_t* __restrict__ sv,
                                 int32_t* __restrict__ sf, long long* __restrict__ szn, int32_t* __restrict__ szd) {
  const int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= ps.lines) return;
  const size_t lines = (size_t)ps.lines;
  const long long base = (long long)(L % ps.c0) * ps.s0 + (long long)(L / ps.c0) * ps.s1;
  // envelope: vertices v[0..k], their values f, left interval bounds z = zn / zd (z[0] = -inf: zd = 0)
  int k = -1;
  for (int q = 0; q < ps.n; ++q) {
    const int32_t fq = grid[base + q * ps.se];
    if (fq >= kFar) continue;
    const long long Fq = (long long)fq + (long long)q * q;
    long long num = 0;
    int den = 0;
    while (k >= 0) {
      const size_t at = (size_t)k * lines + L;
      const int p = sv[at];
      num = Fq - ((long long)sf[at] + (long long)p * p);   // parabolas of p and q meet at num / den
      den = 2 * (q - p);
      const int zdk = szd[at];
      if (zdk == 0 || num * zdk > szn[at] * den) break;     // meets right of z[k]: keep p
      --k;
    }
    ++k;
    const size_t at = (size_t)k * lines + L;
    sv[at] = q;
    sf[at] = fq;
    szn[at] = k == 0 ? 0 : num;
    szd[at] = k == 0 ? 0 : den;
  }
  if (k < 0) return;   // no finite entry: the line stays far
  const int K = k;
  k = 0;
  for (int q = 0; q < ps.n; ++q) {
    while (k < K) {
      const size_t nx = (size_t)(k + 1) * lines + L;
      if (szn[nx] > (long long)q * szd[nx]) break;   // z[k+1] > q
      ++k;
    }
    const size_t at = (size_t)k * lines + L;
    const long long d = (long long)(q - sv[at]) * (q - sv[at]) + sf[at];
    grid[base + q * ps.se] = (int32_t)d;   // < kFar by the box limit
  }
}

// First pass (x lines, sites 0, the rest far): the squared distance to the
// nearest site of the line by one sweep each way; no envelope needed.
__global__ void esdf_first_pass_kernel(int32_t* __restrict__ grid, Pass ps) {
  const int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= ps.lines) return;
  const long long base = (long long)(L % ps.c0) * ps.s0 + (long long)(L / ps.c0) * ps.s1;
  int last = INT_MIN;
  for (int q = 0; q < ps.n; ++q) {
    int32_t* g = grid + base + q * ps.se;
    if (*g == 0) last = q;
    else if (last != INT_MIN) *g = (q - last) * (q - last);
  }
  int next = INT_MIN;
  for (int q = ps.n - 1; q >= 0; --q) {
    int32_t* g = grid + base + q * ps.se;
    if (*g == 0) {
      next = q;
    } else if (next != INT_MIN) {
      const int32_t d = (next - q) * (next - q);
      if (d < *g) *g = d;
    }
  }
}

__global__ void esdf_out_kernel(SubmapDev m, int nb, Box bx, const int32_t* __restrict__ grid, float vs,
                                float max_dist, float* __restrict__ out, int32_t* __restrict__ sq) {
  const size_t total = (size_t)nb * kVoxPerBlock;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / kVoxPerBlock), l = (int)(e % kVoxPerBlock);
    const int v0 = m.block_keys[3 * b] * 8 + (l & 7);
    const int v1 = m.block_keys[3 * b + 1] * 8 + ((l >> 3) & 7);
    const int v2 = m.block_keys[3 * b + 2] * 8 + (l >> 6);
    const int32_t g = grid[grid_index(bx, v0, v1, v2)];
    if (sq) sq[e] = g >= kFar ? -1 : g;
    out[e] = g >= kFar ? max_dist : fminf(__fsqrt_rn((float)g) * vs, max_dist);
  }
}

void* scratch_alloc(cvx_submap* map, size_t bytes, cudaStream_t s) {
  void* p = nullptr;
  if (map->p.alloc) return map->p.alloc(bytes, s, map->p.alloc_ctx);
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void scratch_free(cvx_submap* map, void* p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  if (map->p.free) map->p.free(p, bytes, s, map->p.alloc_ctx);
  else if (!map->p.alloc) cudaFree(p);
}

}  // namespace

extern "C" cvx_status cvx_compute_esdf(cvx_submap* map, float site_band, float w_min, float max_dist,
                                       float* out, int32_t* sq_dist, void* stream) {
  if (!map || !out) return CVX_ERR_INVALID_ARG;
  if (!(site_band >= 0) || !std::isfinite(site_band) || !(w_min >= 0) || !std::isfinite(w_min) ||
      !(max_dist > 0) || !std::isfinite(max_dist))
    return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  map->last_stream = s;
  if (flush_pending(map, s, false) != CVX_OK) return CVX_ERR_CUDA;
  int32_t nb32 = 0;
  if (cudaMemcpyAsync(&nb32, &map->dev.st->n_blocks, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  const int nb = std::min<int32_t>(nb32, map->dev.max_blocks);
  if (nb <= 0) return CVX_OK;
  const SubmapDev& m = map->dev;
  // block box (6 ints)
  int* box = (int*)scratch_alloc(map, 64, s);
  if (!box) return CVX_ERR_OOM;
  int hb[6];
  COVOX_LAUNCH(kKEsdf, s, esdf_box_init_kernel<<<1, 32, 0, s>>>(box));
  COVOX_LAUNCH(kKEsdf, s, esdf_bbox_kernel<<<std::min(num_sms() * 4, (nb + 255) / 256), 256, 0, s>>>(
                              m.block_keys, nb, box));
  const bool ok = cudaMemcpyAsync(hb, box, sizeof(hb), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
                  cudaStreamSynchronize(s) == cudaSuccess;
  scratch_free(map, box, 64, s);
  if (!ok) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  Box bx;
  size_t voxels = 1;
  for (int c = 0; c < 3; ++c) {
    bx.lo[c] = hb[c] * 8;
    const long long n = ((long long)hb[3 + c] - hb[c] + 1) * 8;
    if (n > kMaxAxis) return CVX_ERR_CAPACITY;   // beyond the exact int32 range of the passes
    bx.n[c] = (int)n;
    voxels *= (size_t)n;
  }
  // dense grid and per-line envelope scratch (20 B per grid voxel)
  const size_t grid_bytes = voxels * 4, scr_bytes = voxels * 20;
  char* mem = (char*)scratch_alloc(map, grid_bytes + scr_bytes, s);
  if (!mem) return CVX_ERR_OOM;
  int32_t* grid = (int32_t*)mem;
  long long* szn = (long long*)(mem + grid_bytes);
  int32_t* sv = (int32_t*)(mem + grid_bytes + voxels * 8);
  int32_t* sf = (int32_t*)(mem + grid_bytes + voxels * 12);
  int32_t* szd = (int32_t*)(mem + grid_bytes + voxels * 16);
  cudaMemsetAsync(grid, 0x7f, grid_bytes, s);
  const int g1 = num_sms() * 8;
  COVOX_LAUNCH(kKEsdf, s, esdf_sites_kernel<<<g1, 256, 0, s>>>(m, nb, bx, site_band, w_min, grid));
  const long long nx = bx.n[0], ny = bx.n[1], nz = bx.n[2];
  const Pass passes[3] = {
      {(int)nx, (int)(ny * nz), (int)ny, nx, nx * ny, 1},        // x lines: y + ny z
      {(int)ny, (int)(nx * nz), (int)nx, 1, nx * ny, nx},        // y lines: x + nx z
      {(int)nz, (int)(nx * ny), (int)nx, 1, nx, nx * ny},        // z lines: x + nx y
  };
  // x: sites only (two sweeps); y and z: envelopes (adjacent threads read adjacent voxels)
  COVOX_LAUNCH(kKEsdf, s, esdf_first_pass_kernel<<<(passes[0].lines + 127) / 128, 128, 0, s>>>(grid, passes[0]));
  for (int a = 1; a < 3; ++a)
    COVOX_LAUNCH(kKEsdf, s, esdf_pass_kernel<<<(passes[a].lines + 127) / 128, 128, 0, s>>>(grid, passes[a], sv, sf,
                                                                                            szn, szd));
  COVOX_LAUNCH(kKEsdf, s, esdf_out_kernel<<<g1, 256, 0, s>>>(m, nb, bx, grid, map->p.voxel_size, max_dist,
                                                              out, sq_dist));
  const bool launched = cudaGetLastError() == cudaSuccess;
  scratch_free(map, mem, grid_bytes + scr_bytes, s);
  return launched ? CVX_OK : CVX_ERR_CUDA;
}

// ------------------------------------------------ registration points, bounds
// The backend's ICP takes its points from each submap by their weights and
// finds overlapping submaps by axis-aligned boxes (Sec. III-F).  Library
// reading: the registration points are the centres of the allocated voxels
// with W >= w_min and |D| <= d_band, compacted with one atomic per warp.
namespace {

__global__ void regpoints_kernel(SubmapDev m, int nb, float w_min, float d_band, long long capacity,
                                 float* __restrict__ xyz, unsigned long long* __restrict__ count) {
  const int lane = threadIdx.x & 31;
  const size_t total = (size_t)nb * kVoxPerBlock;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e0 = (size_t)blockIdx.x * blockDim.x; e0 < total; e0 += stride) {   // warp-uniform
    const size_t e = e0 + threadIdx.x;
    bool take = false;
    if (e < total) {
      float D, W;
      if (m.storage == CVX_STORE_F32) {
        D = ((const float*)m.D)[e];
        W = ((const float*)m.W)[e];
      } else {
        D = __half2float(((const __half*)m.D)[e]) * m.trunc;
        W = __half2float(((const __half*)m.W)[e]);
      }
      take = W >= w_min && W > 0.0f && fabsf(D) <= d_band;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, take);
    unsigned long long base = 0;
    if (lane == 0 && bal) base = atomicAdd(count, (unsigned long long)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (take) {
      const unsigned long long at = base + __popc(bal & ((1u << lane) - 1u));
      if ((long long)at < capacity) {
        const int b = (int)(e / kVoxPerBlock), l = (int)(e % kVoxPerBlock);
        const int v0 = m.block_keys[3 * b] * 8 + (l & 7);
        const int v1 = m.block_keys[3 * b + 1] * 8 + ((l >> 3) & 7);
        const int v2 = m.block_keys[3 * b + 2] * 8 + (l >> 6);
        xyz[3 * at] = __fmul_rn((float)v0 + 0.5f, m.vs);
        xyz[3 * at + 1] = __fmul_rn((float)v1 + 0.5f, m.vs);
        xyz[3 * at + 2] = __fmul_rn((float)v2 + 0.5f, m.vs);
      }
    }
  }
}

// the submap's block count (synchronous); -1 on a CUDA error
int read_blocks(cvx_submap* map, cudaStream_t s) {
  int32_t nb32 = 0;
  if (cudaMemcpyAsync(&nb32, &map->dev.st->n_blocks, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return std::min<int32_t>(nb32, map->dev.max_blocks);
}

}  // namespace

extern "C" cvx_status cvx_registration_points(cvx_submap* map, float w_min, float d_band, int64_t capacity,
                                              float* xyz, int64_t* n_out, void* stream) {
  if (!map || !n_out || capacity < 0 || (capacity > 0 && !xyz) || !(d_band >= 0) || !std::isfinite(d_band) ||
      !std::isfinite(w_min))
    return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  map->last_stream = s;
  if (flush_pending(map, s, false) != CVX_OK) return CVX_ERR_CUDA;
  const int nb = read_blocks(map, s);
  if (nb < 0) return CVX_ERR_CUDA;
  *n_out = 0;
  if (nb == 0) return CVX_OK;
  unsigned long long* count = (unsigned long long*)scratch_alloc(map, 64, s);
  if (!count) return CVX_ERR_OOM;
  unsigned long long h = 0;
  cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
  COVOX_LAUNCH(kKEsdf, s, regpoints_kernel<<<num_sms() * 8, 256, 0, s>>>(map->dev, nb, w_min, d_band, capacity,
                                                                         xyz, count));
  const bool ok = cudaMemcpyAsync(&h, count, sizeof(h), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
                  cudaStreamSynchronize(s) == cudaSuccess;
  scratch_free(map, count, 64, s);
  if (!ok) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  *n_out = (int64_t)h;
  return CVX_OK;
}

extern "C" cvx_status cvx_submap_bounds(cvx_submap* map, float lo_hi[6], void* stream) {
  if (!map || !lo_hi) return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  map->last_stream = s;
  const int nb = read_blocks(map, s);
  if (nb < 0) return CVX_ERR_CUDA;
  if (nb == 0) {
    for (int c = 0; c < 3; ++c) {
      lo_hi[c] = 1.0f;
      lo_hi[3 + c] = 0.0f;
    }
    return CVX_OK;
  }
  int* box = (int*)scratch_alloc(map, 64, s);
  if (!box) return CVX_ERR_OOM;
  int hb[6];
  COVOX_LAUNCH(kKEsdf, s, esdf_box_init_kernel<<<1, 32, 0, s>>>(box));
  COVOX_LAUNCH(kKEsdf, s, esdf_bbox_kernel<<<std::min(num_sms() * 4, (nb + 255) / 256), 256, 0, s>>>(
                              map->dev.block_keys, nb, box));
  const bool ok = cudaMemcpyAsync(hb, box, sizeof(hb), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
                  cudaStreamSynchronize(s) == cudaSuccess;
  scratch_free(map, box, 64, s);
  if (!ok) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  const float bs = 8.0f * map->p.voxel_size;
  for (int c = 0; c < 3; ++c) {
    lo_hi[c] = (float)hb[c] * bs;
    lo_hi[3 + c] = (float)(hb[3 + c] + 1) * bs;
  }
  return CVX_OK;
}

// ------------------------------------------------------------- submap overlap
// World-frame boxes of two posed submaps and their intersection (the AABB
// overlap test of the backend, Sec. III-F): each submap's block-corner box
// (cvx_submap_bounds, submap frame) is carried to the world frame by its pose
// (world <- submap, 3x4 row-major), the axis-aligned box of its 8 corners
// taken, and the two boxes intersected.  One thread per ordered pair.
__device__ __forceinline__ void world_box(const float* b, const float* T, float lo[3], float hi[3]) {
  for (int k = 0; k < 3; ++k) {
    lo[k] = 3.40282347e38f;
    hi[k] = -3.40282347e38f;
  }
  for (int c = 0; c < 8; ++c) {
    const float x = (c & 1) ? b[3] : b[0], y = (c & 2) ? b[4] : b[1], z = (c & 4) ? b[5] : b[2];
    for (int k = 0; k < 3; ++k) {
      const float w = T[4 * k] * x + T[4 * k + 1] * y + T[4 * k + 2] * z + T[4 * k + 3];
      lo[k] = fminf(lo[k], w);
      hi[k] = fmaxf(hi[k], w);
    }
  }
}

__global__ void overlap_kernel(int n, const float* __restrict__ bounds, const float* __restrict__ poses,
                               float* __restrict__ volume, float* __restrict__ boxes) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)n * n) return;
  const int i = (int)(q / n), j = (int)(q % n);
  const float* bi = bounds + 6 * i;
  const float* bj = bounds + 6 * j;
  const bool empty = bi[0] > bi[3] || bi[1] > bi[4] || bi[2] > bi[5] || bj[0] > bj[3] || bj[1] > bj[4] || bj[2] > bj[5];
  float li[3], hi_[3], lj[3], hj[3], lo[3], hi[3];
  world_box(bi, poses + 12 * i, li, hi_);
  world_box(bj, poses + 12 * j, lj, hj);
  float v = empty ? 0.0f : 1.0f;
  for (int k = 0; k < 3; ++k) {
    lo[k] = fmaxf(li[k], lj[k]);
    hi[k] = fminf(hi_[k], hj[k]);
    v *= fmaxf(hi[k] - lo[k], 0.0f);
  }
  volume[q] = v;
  if (boxes)
    for (int k = 0; k < 3; ++k) {
      boxes[6 * q + k] = lo[k];
      boxes[6 * q + 3 + k] = hi[k];
    }
}

extern "C" cvx_status cvx_submap_overlaps(int32_t n, const float* bounds, const float* poses, float* volume,
                                          float* boxes, void* stream) {
  if (n <= 0 || n > 65536 || !bounds || !poses || !volume) return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const long long pairs = (long long)n * n;
  COVOX_LAUNCH(kKEsdf, s, overlap_kernel<<<(unsigned)((pairs + 255) / 256), 256, 0, s>>>(n, bounds, poses, volume,
                                                                                         boxes));
  return cudaGetLastError() == cudaSuccess ? CVX_OK : CVX_ERR_CUDA;
}

