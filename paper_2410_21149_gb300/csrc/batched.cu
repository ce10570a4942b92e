// batched.cu -- many submaps and scans of uneven size in one persistent launch.
//
// Scans of one submap are frames in the order given; scans of different
// submaps are independent (submaps are separate maps, coVoxSLAM Sec. III-C).
// The host groups the scans into waves (wave k = the k-th scan of every
// submap that has one) and one cooperative kernel walks the waves:
//   phase 1  every tile of every scan of the wave: integrate_tile (count,
//            allocate, per-voxel sums; Sec. III-D), tiles spread over all
//            CTAs so uneven scans share the GPU (workload equalisation);
//   phase 2  every touched block of every submap of the wave: merge_block;
//   phase 3  per-submap bookkeeping of the frame (counters, error words).
// Phases are separated by grid barriers whose spins are bounded: a barrier
// that gives up records CVX_ERR_TIMEOUT and every CTA leaves the kernel.
// The arithmetic is the per-scan path's device code, unchanged.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/covox.h"
#include "covox_dev.cuh"
#include "integrate_dev.cuh"
#include "prof.h"
#include "submap.h"

using namespace covox;

namespace {

struct BatchDev {
  const SubmapDev* maps;   // [n_maps] views, or [2 * n_maps] (parity views) when pipelined
  const ScanDev* scans;    // [n_scans] in wave order
  const int* scan_map;     // [n_scans] submap of each scan
  const int* scan_lb;      // [n_scans] shared block slots
  const int* tile_prefix;  // [n_scans + 1] tiles before each scan (wave order)
  const int* wave_begin;   // [n_waves + 1] first scan of each wave
  int n_waves;
  int pipelined;           // 1: wave w uses per-scan set w & 1 and merges overlap the next tiles
  unsigned* bar_count;
  unsigned* bar_gen;
  int* err;
  unsigned long long* phase_ns;   // [n_waves * 3 + 1] globaltimer stamps, or nullptr
};

__device__ __forceinline__ const SubmapDev& view(const BatchDev& b, int map, int wave) {
  return b.pipelined ? b.maps[2 * map + (wave & 1)] : b.maps[map];
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void stamp(const BatchDev& b, int slot) {
  if (b.phase_ns && blockIdx.x == 0 && threadIdx.x == 0) b.phase_ns[slot] = global_ns();
}

constexpr long long kBarrierSpin = 1ll << 24;   // ~1 s at the sleep below
constexpr int kMaxWaveScans = 1024;

__device__ bool grid_barrier(const BatchDev& b) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned g = *((volatile unsigned*)b.bar_gen);
    __threadfence();
    if (atomicAdd(b.bar_count, 1u) == gridDim.x - 1) {
      *((volatile unsigned*)b.bar_count) = 0;
      __threadfence();
      atomicAdd(b.bar_gen, 1u);
    } else {
      long long it = 0;
      while (*((volatile unsigned*)b.bar_gen) == g) {
        if (++it > kBarrierSpin || *((volatile int*)b.err) != 0) {
          atomicOr(b.err, kErrTimeout);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ int find_scan(const int* prefix, int lo, int hi, int g) {
  // largest s in [lo, hi) with prefix[s] <= g
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= g) lo = mid; else hi = mid;
  }
  return lo;
}

// Merge work of wave w: every touched block of every submap of the wave,
// taken in spans of kSpan consecutive blocks of the wave's concatenated
// touched lists.  A span's pool indices, scans and skip flags are gathered in
// one round of independent loads into shared memory; then each half CTA
// merges pairs of blocks (loads of both in flight), so a block costs the
// round trips of its sums and voxels only.  Spans first, first + step, ...
// (single: only the first).
constexpr int kSpan = 32;

struct SpanSmem {
  int pool[kSpan];
  int scan[kSpan];
  int skip[kSpan];
};

__device__ void merge_wave(const BatchDev& b, int w, const int* nt_prefix, int first, int step, bool single,
                           SpanSmem* sp) {
  const int tid = threadIdx.x;
  const int s0 = b.wave_begin[w], ns = b.wave_begin[w + 1] - s0;
  const int nt_total = nt_prefix[ns];
  const int half = tid >> 7, sub = tid & (kMergeThreads - 1);
  for (int span = first;; span += step) {
    const int g0 = span * kSpan;
    if (g0 >= nt_total) break;
    const int n = min(kSpan, nt_total - g0);
    if (tid < n) {
      const int q = find_scan(nt_prefix, 0, ns, g0 + tid);
      const SubmapDev& m = view(b, b.scan_map[s0 + q], w);
      sp->pool[tid] = m.touched[g0 + tid - nt_prefix[q]];
      sp->scan[tid] = q;
      sp->skip[tid] = *((volatile int32_t*)m.frame_err) != 0;
    }
    __syncthreads();
    for (int k = 2 * half; k < n; k += 4) {
      const int q = sp->scan[k];
      const SubmapDev& m = view(b, b.scan_map[s0 + q], w);
      const bool pair = k + 1 < n && sp->scan[k + 1] == q;   // a pair shares one submap
      int merged = m.storage == 0 ? merge_pools<0>(m, sp->pool[k], pair ? sp->pool[k + 1] : -1, sp->skip[k], sub)
                                  : merge_pools<1>(m, sp->pool[k], pair ? sp->pool[k + 1] : -1, sp->skip[k], sub);
      unsigned long long c = merged;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
      if ((tid & 31) == 0 && c) atomicAdd(&m.st->voxels_merged, c);
      if (!pair && k + 1 < n) {   // the next block starts the next submap
        const SubmapDev& m2 = view(b, b.scan_map[s0 + sp->scan[k + 1]], w);
        merged = m2.storage == 0 ? merge_pools<0>(m2, sp->pool[k + 1], -1, sp->skip[k + 1], sub)
                                 : merge_pools<1>(m2, sp->pool[k + 1], -1, sp->skip[k + 1], sub);
        c = merged;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if ((tid & 31) == 0 && c) atomicAdd(&m2.st->voxels_merged, c);
      }
    }
    __syncthreads();   // the span's shared arrays are rewritten next
    if (single) break;
  }
}

// touched-block counts of wave w's scans (thread 0), prefix sums in nt_prefix
__device__ void wave_touched(const BatchDev& b, int w, int* nt_prefix) {
  if (threadIdx.x == 0) {
    const int s0 = b.wave_begin[w], s1 = b.wave_begin[w + 1];
    int acc = 0;
    for (int s = s0; s < s1; ++s) {
      nt_prefix[s - s0] = acc;
      const SubmapDev& m = view(b, b.scan_map[s], w);
      acc += min(*((volatile int32_t*)m.n_touched), m.max_blocks);
    }
    nt_prefix[s1 - s0] = acc;
  }
  __syncthreads();
}

// per-submap bookkeeping of wave w's frames (CTA 0)
__device__ void wave_bookkeeping(const BatchDev& b, int w, const int* nt_prefix) {
  if (blockIdx.x != 0) return;
  const int s0 = b.wave_begin[w], s1 = b.wave_begin[w + 1];
  for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
    const SubmapDev& m = view(b, b.scan_map[s], w);
    State* st = m.st;
    st->blocks_touched += (unsigned long long)(nt_prefix[s - s0 + 1] - nt_prefix[s - s0]);
    st->frames += 1;
    st->sticky_err |= *m.frame_err;
    *m.frame_err = 0;
    *m.n_touched = 0;
    if (!b.pipelined) st->epoch += 1;   // the submap's next scan takes the next epoch
  }
}

// pipelined: the tiles of wave w are done, so their submaps' next scans take
// the next epoch (CTA 0, after the step's barrier)
__device__ void wave_epoch(const BatchDev& b, int w) {
  if (blockIdx.x != 0) return;
  for (int s = b.wave_begin[w] + threadIdx.x; s < b.wave_begin[w + 1]; s += blockDim.x)
    view(b, b.scan_map[s], w).st->epoch += 1;
}

template <int kVariant>
__global__ void __launch_bounds__(kTileThreads, 4) batched_kernel(BatchDev b) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int nt_prefix[kMaxWaveScans + 1];
  __shared__ SpanSmem span;
  stamp(b, 0);
  if (!b.pipelined) {
    for (int w = 0; w < b.n_waves; ++w) {
      const int s0 = b.wave_begin[w], s1 = b.wave_begin[w + 1];
      // phase 1: tiles of all scans of the wave
      const int t0 = b.tile_prefix[s0], total = b.tile_prefix[s1] - t0;
      for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int s = find_scan(b.tile_prefix, s0, s1, t0 + t);
        integrate_tile_v<kVariant>(view(b, b.scan_map[s], w), b.scans[s], t0 + t - b.tile_prefix[s], smem,
                                   b.scan_lb[s]);
      }
      if (!grid_barrier(b)) return;
      stamp(b, 3 * w + 1);
      // phase 2: merge every touched block of every submap of the wave
      wave_touched(b, w, nt_prefix);
      merge_wave(b, w, nt_prefix, blockIdx.x, gridDim.x, false, &span);
      if (!grid_barrier(b)) return;
      stamp(b, 3 * w + 2);
      // phase 3: per-submap bookkeeping of this frame
      wave_bookkeeping(b, w, nt_prefix);
      if (!grid_barrier(b)) return;
      stamp(b, 3 * w + 3);
    }
    return;
  }
  // pipelined: step w runs the tiles of wave w and the merges of wave w - 1
  // (different per-scan sets; tiles never read D or W), then the bookkeeping
  // of wave w - 1 frees its set for wave w + 1.
  for (int w = 0; w <= b.n_waves; ++w) {
    int n_tiles = 0, t0 = 0, s0 = 0, s1 = 0;
    if (w < b.n_waves) {
      s0 = b.wave_begin[w];
      s1 = b.wave_begin[w + 1];
      t0 = b.tile_prefix[s0];
      n_tiles = b.tile_prefix[s1] - t0;
    }
    int n_spans = 0;
    if (w > 0) {
      wave_touched(b, w - 1, nt_prefix);
      n_spans = (nt_prefix[b.wave_begin[w] - b.wave_begin[w - 1]] + kSpan - 1) / kSpan;   // merge spans
    }
    const int items = n_tiles + n_spans;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
      if (it < n_tiles) {
        const int s = find_scan(b.tile_prefix, s0, s1, t0 + it);
        integrate_tile_v<kVariant>(view(b, b.scan_map[s], w), b.scans[s], t0 + it - b.tile_prefix[s], smem,
                                   b.scan_lb[s]);
      } else {
        merge_wave(b, w - 1, nt_prefix, it - n_tiles, 1, true, &span);   // one item: a span
      }
    }
    if (!grid_barrier(b)) return;
    stamp(b, 3 * w + 1);
    if (w > 0) wave_bookkeeping(b, w - 1, nt_prefix);
    if (w < b.n_waves) wave_epoch(b, w);
    if (!grid_barrier(b)) return;
    stamp(b, 3 * w + 2);
    stamp(b, 3 * w + 3);
  }
}

using BatchedFn = void (*)(BatchDev);
const BatchedFn kBatched[7] = {batched_kernel<-1>, batched_kernel<0>, batched_kernel<1>, batched_kernel<2>,
                               batched_kernel<3>, batched_kernel<4>, batched_kernel<5>};

}  // namespace

struct cvx_batch {
  int max_maps, max_scans;
  void* dev;          // descriptor block on the device
  void* host;         // pinned staging of the same layout
  size_t bytes;
  unsigned* bar;      // count, gen, err (device)
  cudaEvent_t copied; // host staging reusable once the previous upload ran
  bool pending;
  int grid;           // persistent grid size (CTAs)
  int lb_max;
  unsigned long long* phase_ns;   // [3 * max_scans + 1] when phase timing is on
  bool timing;
  int last_waves;
  int wave_limit;     // most scans per wave (0: no limit)
};

namespace {

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

struct Layout {
  size_t maps, scans, scan_map, scan_lb, tile_prefix, wave_begin, total;
};

Layout layout(int max_maps, int max_scans) {
  Layout L;
  size_t o = 0;
  L.maps = o;
  o = align16(o + sizeof(SubmapDev) * 2 * max_maps);
  L.scans = o;
  o = align16(o + sizeof(ScanDev) * max_scans);
  L.scan_map = o;
  o = align16(o + sizeof(int) * max_scans);
  L.scan_lb = o;
  o = align16(o + sizeof(int) * max_scans);
  L.tile_prefix = o;
  o = align16(o + sizeof(int) * (max_scans + 1));
  L.wave_begin = o;
  o = align16(o + sizeof(int) * (max_scans + 1));
  L.total = o;
  return L;
}

}  // namespace

extern "C" {

cvx_status cvx_batch_create(int32_t max_submaps, int32_t max_scans, cvx_batch** out) {
  if (!out || max_submaps <= 0 || max_scans <= 0 || max_submaps > kMaxWaveScans || max_scans > (1 << 20))
    return CVX_ERR_INVALID_ARG;
  *out = nullptr;
  cvx_batch* b = new (std::nothrow) cvx_batch();
  if (!b) return CVX_ERR_OOM;
  b->max_maps = max_submaps;
  b->max_scans = max_scans;
  const Layout L = layout(max_submaps, max_scans);
  b->bytes = L.total;
  if (cudaMalloc(&b->dev, L.total) != cudaSuccess || cudaMallocHost(&b->host, L.total) != cudaSuccess ||
      cudaMalloc((void**)&b->bar, 16) != cudaSuccess || cudaMemset(b->bar, 0, 16) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (b->dev) cudaFree(b->dev);
    if (b->host) cudaFreeHost(b->host);
    if (b->bar) cudaFree(b->bar);
    delete b;
    return CVX_ERR_OOM;
  }
  b->lb_max = kMaxLocalBlocks;
  if (cudaMalloc((void**)&b->phase_ns, sizeof(unsigned long long) * (3 * (size_t)max_scans + 8)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(b->dev);
    cudaFreeHost(b->host);
    cudaFree(b->bar);
    delete b;
    return CVX_ERR_OOM;
  }
  for (int v = 0; v < 7; ++v)
    cudaFuncSetAttribute((const void*)kBatched[v], cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tile_smem_bytes(kMaxLocalBlocks));
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)kBatched[0], kTileThreads,
                                                    tile_smem_bytes(kDefaultLocalBlocks)) != cudaSuccess ||
      per_sm <= 0) {
    cudaGetLastError();
    per_sm = 1;
  }
  b->grid = per_sm * num_sms();
  *out = b;
  return CVX_OK;
}

void cvx_batch_destroy(cvx_batch* b) {
  if (!b) return;
  cudaEventSynchronize(b->copied);
  cudaFree(b->dev);
  cudaFreeHost(b->host);
  cudaFree(b->bar);
  cudaFree(b->phase_ns);
  cudaEventDestroy(b->copied);
  delete b;
}

cvx_status cvx_batch_wave_limit(cvx_batch* b, int32_t max_scans_per_wave) {
  if (!b || max_scans_per_wave < 0) return CVX_ERR_INVALID_ARG;
  b->wave_limit = max_scans_per_wave;
  return CVX_OK;
}

cvx_status cvx_batch_timing(cvx_batch* b, int32_t enable) {
  if (!b) return CVX_ERR_INVALID_ARG;
  b->timing = enable != 0;
  return CVX_OK;
}

int32_t cvx_batch_phase_times(cvx_batch* b, double* ms, int32_t max_waves) {
  if (!b || !ms || max_waves <= 0) return CVX_ERR_INVALID_ARG;
  const int nw = b->last_waves < max_waves ? b->last_waves : max_waves;
  if (nw <= 0) return 0;
  unsigned long long* t = new (std::nothrow) unsigned long long[3 * (size_t)nw + 1];
  if (!t) return CVX_ERR_OOM;
  if (cudaMemcpy(t, b->phase_ns, sizeof(unsigned long long) * (3 * (size_t)nw + 1), cudaMemcpyDeviceToHost) !=
      cudaSuccess) {
    cudaGetLastError();
    delete[] t;
    return CVX_ERR_CUDA;
  }
  for (int w = 0; w < nw; ++w)
    for (int p = 0; p < 3; ++p) ms[3 * w + p] = (double)(t[3 * w + p + 1] - t[3 * w + p]) * 1e-6;
  delete[] t;
  return nw;
}

cvx_status cvx_integrate_batch(cvx_batch* b, cvx_submap* const* maps, int32_t n_maps,
                               const cvx_scan_desc* scans, int32_t n_scans, void* stream) {
  if (!b || !maps || n_maps <= 0 || n_maps > b->max_maps || n_scans < 0 || n_scans > b->max_scans ||
      (n_scans > 0 && !scans))
    return CVX_ERR_INVALID_ARG;
  for (int q = 0; q < n_maps; ++q)
    for (int r = 0; r < q; ++r)
      if (!maps[q] || maps[q] == maps[r]) return CVX_ERR_INVALID_ARG;   // distinct submaps
  // validate and describe every scan; empty scans are no frames; group the
  // rest into waves (wave k = k-th non-empty scan of each submap)
  std::vector<ScanDev> sd(n_scans);
  std::vector<int> lbs(n_scans), rank(n_scans), per_map(n_maps, 0), order;
  int n_waves = 0, lb_max = 0;
  for (int s = 0; s < n_scans; ++s) {
    const cvx_scan_desc& d = scans[s];
    if (d.submap < 0 || d.submap >= n_maps) return CVX_ERR_INVALID_ARG;
    const cvx_status v =
        make_scan_dev(maps[d.submap], d.points_xyz, d.n, d.T_sub_sensor, d.point_weights, &d.params, &sd[s], &lbs[s]);
    if (v != CVX_OK) return v;
    if (d.n == 0) continue;
    rank[s] = per_map[d.submap]++;
    lb_max = std::max(lb_max, lbs[s]);
    order.push_back(s);
  }
  if (order.empty()) return CVX_OK;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return rank[a] < rank[c]; });
  const int n_run = (int)order.size();
  // waves: the k-th scans of all submaps, cut into chunks of at most
  // wave_limit scans (chunks of one rank are independent of each other)
  {
    int w = -1, prev = -1, in_wave = 0;
    for (int k = 0; k < n_run; ++k) {
      const int rk = rank[order[k]];
      if (rk != prev || (b->wave_limit > 0 && in_wave >= b->wave_limit)) {
        ++w;
        in_wave = 0;
        prev = rk;
      }
      rank[order[k]] = w;   // from here on: the wave index
      ++in_wave;
    }
    n_waves = w + 1;
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  // the staging buffer may still feed the previous upload
  if (b->pending && !capturing) {
    if (cudaEventSynchronize(b->copied) != cudaSuccess) {
      cudaGetLastError();
      return CVX_ERR_CUDA;
    }
    b->pending = false;
  }
  const Layout L = layout(b->max_maps, b->max_scans);
  char* h = (char*)b->host;
  SubmapDev* hm = (SubmapDev*)(h + L.maps);
  ScanDev* hs = (ScanDev*)(h + L.scans);
  int* hmap = (int*)(h + L.scan_map);
  int* hlb = (int*)(h + L.scan_lb);
  int* htp = (int*)(h + L.tile_prefix);
  int* hwb = (int*)(h + L.wave_begin);
  bool pipelined = true;
  for (int q = 0; q < n_maps; ++q) pipelined = pipelined && maps[q]->pipelined;
  for (int q = 0; q < n_maps; ++q) {
    if (pipelined) {
      hm[2 * q] = maps[q]->dev;
      hm[2 * q + 1] = maps[q]->dev_b;
    } else {
      hm[q] = maps[q]->dev;
    }
  }
  int tiles = 0, wave = -1;
  for (int k = 0; k < n_run; ++k) {
    const int s = order[k];
    while (wave < rank[s]) hwb[++wave] = k;
    hs[k] = sd[s];
    hmap[k] = scans[s].submap;
    hlb[k] = lbs[s];
    htp[k] = tiles;
    tiles += sd[s].n_tiles;
  }
  htp[n_run] = tiles;
  hwb[n_waves] = n_run;
  if (cudaMemcpyAsync(b->dev, b->host, L.total, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  if (!capturing) {
    if (cudaEventRecord(b->copied, st) != cudaSuccess) {
      cudaGetLastError();
      return CVX_ERR_CUDA;
    }
    b->pending = true;
  }
  for (int q = 0; q < n_maps; ++q) {
    maps[q]->last_stream = st;
    // a scan left pending by the pipelined per-scan path is merged first
    if (flush_pending(maps[q], st, false) != CVX_OK) return CVX_ERR_CUDA;
  }
  char* d = (char*)b->dev;
  BatchDev bd;
  bd.maps = (const SubmapDev*)(d + L.maps);
  bd.scans = (const ScanDev*)(d + L.scans);
  bd.scan_map = (const int*)(d + L.scan_map);
  bd.scan_lb = (const int*)(d + L.scan_lb);
  bd.tile_prefix = (const int*)(d + L.tile_prefix);
  bd.wave_begin = (const int*)(d + L.wave_begin);
  bd.n_waves = n_waves;
  bd.pipelined = pipelined ? 1 : 0;
  bd.bar_count = b->bar;
  bd.bar_gen = b->bar + 1;
  bd.err = (int*)(b->bar + 2);
  bd.phase_ns = b->timing ? b->phase_ns : nullptr;
  b->last_waves = pipelined ? n_waves + 1 : n_waves;   // pipelined: steps (tiles of w + merges of w - 1)
  if (cudaMemsetAsync(b->bar, 0, 16, st) != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  // one variant for every scan: a kernel holding only that code
  int variant = -2;
  for (int k = 0; k < n_run; ++k) {
    const int v = tile_variant(lbs[order[k]], sd[order[k]].dropoff, sd[order[k]].carve);
    variant = variant == -2 ? v : (variant == v ? v : -1);
  }
  const BatchedFn kern = kBatched[variant + 1];
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)kern, kTileThreads,
                                                    tile_smem_bytes(lb_max)) != cudaSuccess ||
      per_sm <= 0) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  const int grid = per_sm * num_sms();
  void* args[] = {&bd};
  cudaError_t e;
  COVOX_LAUNCH(kKBatched, st,
               e = cudaLaunchCooperativeKernel((void*)kern, dim3(grid), dim3(kTileThreads), args,
                                               tile_smem_bytes(lb_max), st));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  return CVX_OK;
}

int32_t cvx_batch_error(cvx_batch* b) {
  if (!b) return CVX_ERR_INVALID_ARG;
  unsigned v[3] = {0, 0, 0};
  if (cudaMemcpy(v, b->bar, 12, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  return (v[2] & kErrTimeout) ? CVX_ERR_TIMEOUT : CVX_OK;
}

}  // extern "C"
