// batched.cu -- many submaps and scans of uneven size in one persistent launch.
//
// Scans of one submap are frames in the order given; scans of different
// submaps are independent (submaps are separate maps, coVoxSLAM Sec. III-C).
// The host groups the scans into waves (wave k = the k-th scan of every
// submap that has one) and one cooperative kernel walks the waves:
//   phase 1  every tile of every scan of the wave: integrate_tile (count,
//            allocate, per-voxel sums; Sec. III-D), tiles spread over all
//            CTAs so uneven scans share the GPU (workload equalisation);
//   phase 2  every touched block of every submap of the wave: merge_span;
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
  long long barrier_polls;        // polls before a grid barrier gives up
  int missing_cta;                // test hook: this CTA leaves before its first arrival (-1: none)
};

__device__ __forceinline__ const SubmapDev& view(const BatchDev& b, int map, int wave) {
  return b.pipelined ? b.maps[2 * map + (wave & 1)] : b.maps[map];
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Sum of one value over the 256-thread CTA (thread 0 gets it).
__device__ __forceinline__ unsigned long long cta_sum_b(unsigned long long v, unsigned long long* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned long long t = 0;
  if (threadIdx.x == 0)
    for (int k = 0; k < kTileThreads / 32; ++k) t += red[k];
  __syncthreads();   // red is reused by the next call
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
        if (++it > b.barrier_polls || *((volatile int*)b.err) != 0) {
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

// Blocks a merge of wave w covers: the submap's allocated blocks -- with
// pipelined waves as they stood when the wave's tiles had finished (the next
// wave's tiles allocate meanwhile; every CTA must see the same count, since
// the spans of all the wave's submaps are numbered together).
__device__ __forceinline__ int wave_blocks(const BatchDev& b, const SubmapDev& m, int w) {
  const int nb = b.pipelined ? *((volatile int32_t*)((w & 1) ? &m.st->nb_closed1 : &m.st->nb_closed0))
                             : *((volatile int32_t*)&m.st->n_blocks);
  return min(nb, m.max_blocks);
}

// Merge work of wave w: the allocated blocks of every submap of the wave in
// spans of kSpanBlocks consecutive pool indices (a span never crosses
// submaps; span_prefix counts them per scan of the wave).  In each span the
// blocks stamped with the scan's epoch are compacted and merged (merge_span).
// Spans first, first + step, ... (single: only the first).
__device__ void merge_wave(const BatchDev& b, int w, const int* span_prefix, int first, int step, bool single,
                           SpanList* sl, unsigned long long* red) {
  const int s0 = b.wave_begin[w], ns = b.wave_begin[w + 1] - s0;
  const int total = span_prefix[ns];
  for (int span = first; span < total; span += step) {
    const int q = find_scan(span_prefix, 0, ns, span);
    const SubmapDev& m = view(b, b.scan_map[s0 + q], w);
    const int nb = wave_blocks(b, m, w);
    const int p0 = (span - span_prefix[q]) * kSpanBlocks;
    const bool skip = *((volatile int32_t*)m.frame_err) != 0;
    // the scan's epoch: its tiles ran with st->epoch + 1; pipelined waves have
    // advanced st->epoch past them before their merges
    const uint32_t ep = *((volatile uint32_t*)&m.st->epoch) + (b.pipelined ? 0u : 1u);
    int t = 0;
    const int merged = merge_span(m, p0, min(kSpanBlocks, nb - p0), ep, skip, sl, &t);
    const unsigned long long c = cta_sum_b(merged, red);
    if (threadIdx.x == 0) {
      if (c) atomicAdd(&m.st->voxels_merged, c);
      if (t) atomicAdd(&m.st->blocks_touched, (unsigned long long)t);
    }
    if (single) break;
  }
}

// spans of wave w's scans (thread 0), prefix sums in span_prefix
__device__ void wave_spans(const BatchDev& b, int w, int* span_prefix) {
  if (threadIdx.x == 0) {
    const int s0 = b.wave_begin[w], s1 = b.wave_begin[w + 1];
    int acc = 0;
    for (int s = s0; s < s1; ++s) {
      span_prefix[s - s0] = acc;
      const SubmapDev& m = view(b, b.scan_map[s], w);
      acc += (wave_blocks(b, m, w) + kSpanBlocks - 1) / kSpanBlocks;
    }
    span_prefix[s1 - s0] = acc;
  }
  __syncthreads();
}

// per-submap bookkeeping of wave w's frames (CTA 0)
__device__ void wave_bookkeeping(const BatchDev& b, int w) {
  if (blockIdx.x != 0) return;
  const int s0 = b.wave_begin[w], s1 = b.wave_begin[w + 1];
  for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
    const SubmapDev& m = view(b, b.scan_map[s], w);
    State* st = m.st;
    st->frames += 1;
    st->sticky_err |= *m.frame_err;
    *m.frame_err = 0;
    if (!b.pipelined) st->epoch += 1;   // the submap's next scan takes the next epoch
  }
}

// pipelined: the tiles of wave w are done, so their submaps' next scans take
// the next epoch (CTA 0, after the step's barrier)
__device__ void wave_epoch(const BatchDev& b, int w) {
  if (blockIdx.x != 0) return;
  for (int s = b.wave_begin[w] + threadIdx.x; s < b.wave_begin[w + 1]; s += blockDim.x) {
    State* st = view(b, b.scan_map[s], w).st;
    if (w & 1) st->nb_closed1 = st->n_blocks;
    else st->nb_closed0 = st->n_blocks;
    st->epoch += 1;
  }
}

template <int kVariant>
__global__ void __launch_bounds__(kTileThreads, 4) batched_kernel(BatchDev b) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int span_prefix[kMaxWaveScans + 1];
  __shared__ SpanList span;
  __shared__ unsigned long long red[kTileThreads / 32];
  if ((int)blockIdx.x == b.missing_cta) return;   // test hook: never arrives at a barrier
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
      wave_spans(b, w, span_prefix);
      merge_wave(b, w, span_prefix, blockIdx.x, gridDim.x, false, &span, red);
      if (!grid_barrier(b)) return;
      stamp(b, 3 * w + 2);
      // phase 3: per-submap bookkeeping of this frame
      wave_bookkeeping(b, w);
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
      wave_spans(b, w - 1, span_prefix);
      n_spans = span_prefix[b.wave_begin[w] - b.wave_begin[w - 1]];   // merge spans
    }
    const int items = n_tiles + n_spans;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
      if (it < n_tiles) {
        const int s = find_scan(b.tile_prefix, s0, s1, t0 + it);
        integrate_tile_v<kVariant>(view(b, b.scan_map[s], w), b.scans[s], t0 + it - b.tile_prefix[s], smem,
                                   b.scan_lb[s]);
      } else {
        merge_wave(b, w - 1, span_prefix, it - n_tiles, 1, true, &span, red);   // one item: a span
      }
    }
    if (!grid_barrier(b)) return;
    stamp(b, 3 * w + 1);
    if (w > 0) wave_bookkeeping(b, w - 1);
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
  int missing_cta;    // test hook (-1: off)
  long long barrier_polls;
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
  b->missing_cta = -1;
  b->barrier_polls = kBarrierSpin;
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

cvx_status cvx_batch_test_missing_cta(cvx_batch* b, int32_t missing_cta, int64_t barrier_polls) {
  if (!b) return CVX_ERR_INVALID_ARG;
  b->missing_cta = missing_cta < 0 ? -1 : missing_cta;
  b->barrier_polls = (missing_cta >= 0 && barrier_polls > 0) ? barrier_polls : kBarrierSpin;
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
  bd.barrier_polls = b->barrier_polls;
  bd.missing_cta = b->missing_cta;
  b->last_waves = pipelined ? n_waves + 1 : n_waves;   // pipelined: steps (tiles of w + merges of w - 1)
  if (cudaMemsetAsync(b->bar, 0, 16, st) != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  // one variant for every scan: a kernel holding only that code
  int variant = -2;
  for (int k = 0; k < n_run; ++k) {
    const int v = tile_variant(lbs[order[k]], sd[order[k]].dropoff, sd[order[k]].carve || sd[order[k]].long_band);
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
