// batched.cu -- many submaps and scans of uneven size in one persistent launch.
//
// Scans of one submap are frames in the order given; scans of different
// submaps are independent (submaps are separate maps, coVoxSLAM Sec. III-C).
// One persistent kernel works through a queue of items in dependency order,
// with no grid-wide barrier:
//   tile item   one tile of one scan: integrate_tile (count, allocate,
//               per-voxel sums; Sec. III-D) into the scan's per-scan set;
//   merge item  one of the scan's merge parts: every parts-th span of
//               the submap's allocated blocks, the
//               blocks stamped with the scan's epoch merged into D and W.
// An item waits (bounded) only for what it needs: a tile for the merge that
// last used its per-scan set (pipelined submaps have two or four sets, so a
// scan's tiles overlap the previous scans' merges), a merge part for all tiles of its
// scan and for the merge of the submap's previous scan (D and W in frame
// order).  Every item waits only on items earlier in the queue, which a
// running CTA has already taken (a CTA takes items only while it runs, and
// the items a wait needs all precede the waiting one), so the launch always
// progresses whether or not all its CTAs are resident at once -- an ordinary
// launch suffices; a wait that runs out records CVX_ERR_TIMEOUT, after which
// every CTA drains the queue and leaves.
// Load balance is dynamic (Sec. III-D workload equalisation): each CTA takes
// the next item as soon as it is free.  The arithmetic is the per-scan path's
// device code, unchanged.
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

constexpr int kMaxMergeParts = 256;              // merge items per scan, at most
constexpr long long kWaitPolls = 1ll << 21;      // about a second of polling at the sleep below
constexpr int kMaxBatchMaps = 1024;
constexpr int kErrIncomplete = 8;                // a scan was left unmerged (only after a timeout)

// Per scan of a launch, in queue order of its tiles.
struct ScanMeta {
  int view;       // index into BatchDev::views (4 * submap + per-scan set)
  int prev;       // previous scan of the same submap (its merge precedes this one's), or -1
  int prev_set;   // the scan whose merge frees this scan's per-scan set, or -1
  int n_tiles;
  int lb;         // shared block slots
  int epoch_end;  // > 0: the submap's last scan of the launch, st->epoch advances by this much
  int parts;      // merge items of the scan
  int rank;       // frame number of the scan within its submap in this launch
  int part_chain; // 1: the previous scan's merge has the same parts, so merge part p waits only for
                  // the previous merge's part p (the same spans, hence the same blocks)
};

struct BatchDev {
  const SubmapDev* views;   // [4 * n_maps]: per submap, its per-scan sets 0..3 (repeated when it has fewer)
  const ScanDev* scans;     // [n_scans]
  const ScanMeta* meta;     // [n_scans]
  const int* seg_first;     // [n_segs + 1] first item of each queue segment
  const int* seg_code;      // [n_segs] scan index, bit 30 set for a merge segment
  int n_segs;
  int n_scans;
  int* ctr;                 // head, err, exit count, scans closed, then per scan: tiles done, merge tickets, merged flag
  int* part_done;           // [submaps of the launch][kMaxMergeParts]: 1 + rank of the last merge whose part p is done
  unsigned long long* phase_ns;   // [1 + 2 * n_scans]: launch start, per scan tiles done / merged
  long long polls;          // polls before a wait gives up
  int missing_cta;          // test hook: this CTA takes one item and leaves without doing it (-1: none)
};

__device__ __forceinline__ int* tiles_done(const BatchDev& b, int s) { return b.ctr + 4 + 3 * s; }
__device__ __forceinline__ int* merge_ticket(const BatchDev& b, int s) { return b.ctr + 4 + 3 * s + 1; }
__device__ __forceinline__ int* merged_flag(const BatchDev& b, int s) { return b.ctr + 4 + 3 * s + 2; }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0 waits until *addr >= target (bounded; gives up at once when the
// launch has failed), then the CTA goes on.  The fence after the wait orders
// the CTA's later reads after the producer's writes, which it published with
// a fence before its counter update.
__device__ bool wait_at_least(const BatchDev& b, const int* addr, int target, int* ok_smem) {
  if (threadIdx.x == 0) {
    int ok = 1;
    long long it = 0;
    while (*((volatile const int*)addr) < target) {
      if (*((volatile int*)(b.ctr + 1)) != 0) {
        ok = 0;
        break;
      }
      if (++it > b.polls) {
        atomicOr(b.ctr + 1, kErrTimeout);
        ok = 0;
        break;
      }
      __nanosleep(100);
    }
    __threadfence();
    *ok_smem = ok;
  }
  __syncthreads();
  const int ok = *ok_smem;
  __syncthreads();
  return ok != 0;
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

// Merge part `part` of scan s: spans part, part + parts, ... of the
// submap's allocated blocks (blocks the submap's next scan allocates
// meanwhile carry other epochs, so any count read now covers this scan's).
template <bool kColour>
__device__ void merge_part(const BatchDev& b, int s, int part, const MergeSmem& ms, unsigned long long* red) {
  const SubmapDev& m = b.views[b.meta[s].view];
  // Thread 0 reads the block count, error bits and epoch once for the CTA:
  // the count grows while later scans' tiles allocate, and every thread must
  // run the same spans (each merge_span holds CTA barriers).
  __shared__ int head[3];
  if (threadIdx.x == 0) {
    head[0] = min(*((volatile int32_t*)&m.st->n_blocks), m.max_blocks);
    head[1] = *((volatile int32_t*)m.frame_err);
    head[2] = (int)(*((volatile uint32_t*)&m.st->epoch) + 1u + b.scans[s].epoch_add);
  }
  __syncthreads();
  const int nb = head[0];
  const bool skip = head[1] != 0;
  const uint32_t ep = (uint32_t)head[2];
  __syncthreads();   // head is rewritten by the CTA's next merge item
  unsigned long long merged = 0, touched = 0;
  const int parts = b.meta[s].parts;
  for (int span = part; span * kSpanBlocks < nb; span += kSpansPerCall * parts) {
    int t = 0;
    merged += merge_span<kColour>(m, span, parts, nb, ep, skip, ms, &t);
    touched += t;
  }
  const unsigned long long c = cta_sum_b(merged, red);
  if (threadIdx.x == 0) {
    if (c) atomicAdd(&m.st->voxels_merged, c);
    if (touched) atomicAdd(&m.st->blocks_touched, touched);
  }
}

// Frame bookkeeping of scan s, by the CTA finishing its last merge part.
__device__ void close_scan(const BatchDev& b, int s) {
  const ScanMeta& sm = b.meta[s];
  const SubmapDev& m = b.views[sm.view];
  State* st = m.st;
  // atomics: the close of the submap's next scan may run at the same time
  // (its merge parts wait only for this merge's parts, not for this close)
  atomicAdd(&st->frames, 1ull);
  atomicOr(&st->sticky_err, *((volatile int32_t*)m.frame_err));
  *m.frame_err = 0;
  if (sm.epoch_end > 0) st->epoch += (uint32_t)sm.epoch_end;   // after the submap's last scan of the launch
  atomicAdd(b.ctr + 3, 1);
}

// The queue segment holding item it (read-only descriptors: through the
// non-coherent cache).
__device__ __forceinline__ int find_segment(const BatchDev& b, int it) {
  int lo = 0, hi = b.n_segs;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(b.seg_first + mid) <= it) lo = mid; else hi = mid;
  }
  return lo;
}

// Resident CTAs per SM the register budget is cut for (a build-time knob).
#ifndef COVOX_BATCHED_MIN_CTAS
#define COVOX_BATCHED_MIN_CTAS 4
#endif

template <int kVariant>
__global__ void __launch_bounds__(kTileThreads, COVOX_BATCHED_MIN_CTAS) batched_kernel(BatchDev b) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int item_smem[3];
  __shared__ int ok_smem;
  __shared__ unsigned long long red[kTileThreads / 32];
  if (b.phase_ns && blockIdx.x == 0 && threadIdx.x == 0) b.phase_ns[0] = global_ns();
  const int n_items = __ldg(b.seg_first + b.n_segs);
  // dependencies this CTA has already seen satisfied (counters only grow)
  int seen_merged = -1, seen_tiles = -1;
  for (bool first = true;; first = false) {
    if (threadIdx.x == 0) {
      const int it = *((volatile int*)(b.ctr + 1)) != 0 ? n_items : atomicAdd(b.ctr, 1);
      item_smem[0] = it;
      item_smem[1] = it < n_items ? find_segment(b, it) : -1;
    }
    __syncthreads();
    const int it = item_smem[0], seg = item_smem[1];
    __syncthreads();
    if (it >= n_items) break;
    if (first && (int)blockIdx.x == b.missing_cta) break;   // test hook: the item is never done
    const int code = __ldg(b.seg_code + seg);
    const int s = code & 0x3fffffff;
    const int part = it - __ldg(b.seg_first + seg);
    const ScanMeta sm = b.meta[s];
    if (!(code & (1 << 30))) {   // tile item
      if (sm.prev_set >= 0 && sm.prev_set != seen_merged) {
        if (!wait_at_least(b, merged_flag(b, sm.prev_set), 1, &ok_smem)) continue;
        seen_merged = sm.prev_set;
      }
      integrate_tile_v<kVariant>(b.views[sm.view], b.scans[s], part, smem, sm.lb);
      if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(tiles_done(b, s), 1) == sm.n_tiles - 1 && b.phase_ns) b.phase_ns[1 + 2 * s] = global_ns();
      }
    } else {                     // merge item
      if (s != seen_tiles) {
        if (!wait_at_least(b, tiles_done(b, s), sm.n_tiles, &ok_smem)) continue;
        seen_tiles = s;
      }
      int* my_part = b.part_done + (size_t)(sm.view >> 2) * kMaxMergeParts + part;
      if (sm.prev >= 0) {   // D and W in frame order
        if (sm.part_chain) {
          if (!wait_at_least(b, my_part, sm.rank, &ok_smem)) continue;
        } else if (sm.prev != seen_merged) {
          if (!wait_at_least(b, merged_flag(b, sm.prev), 1, &ok_smem)) continue;
          seen_merged = sm.prev;
        }
      }
      merge_part<(kVariant < 0)>(b, s, part, merge_smem(smem), red);
      if (threadIdx.x == 0) {
        __threadfence();
        atomicExch(my_part, sm.rank + 1);   // this part's blocks are merged up to this scan
        if (atomicAdd(merge_ticket(b, s), 1) == sm.parts - 1) {
          close_scan(b, s);
          if (b.phase_ns) b.phase_ns[2 + 2 * s] = global_ns();
          __threadfence();
          atomicExch(merged_flag(b, s), 1);
        }
      }
      __syncthreads();
    }
  }
  // the last CTA to leave checks that every scan was merged (each CTA
  // fenced its closes before counting itself out)
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(b.ctr + 2, 1) == gridDim.x - 1 && *((volatile int*)(b.ctr + 3)) != b.n_scans)
      atomicOr(b.ctr + 1, kErrIncomplete);
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
  int* ctr;           // launch counters (device)
  cudaEvent_t copied; // host staging reusable once the previous upload ran
  bool pending;
  int lb_max;
  unsigned long long* phase_ns;   // [1 + 2 * max_scans] when timing is on
  bool timing;
  int last_scans;
  int wave_limit;     // most scans per round of the queue (0: no limit)
  int missing_cta;    // test hook (-1: off)
  long long polls;
  int merge_parts;    // merge items per scan (0: chosen per round of each launch)
  int* part_done;     // [max_maps][kMaxMergeParts] per-part merge progress (device)
  int submap_group;   // queue order by groups of this many submaps (0: all submaps in one group)
};

namespace {

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

struct Layout {
  size_t views, scans, meta, seg_first, seg_code, total;
};

Layout layout(int max_maps, int max_scans) {
  Layout L;
  size_t o = 0;
  L.views = o;
  o = align16(o + sizeof(SubmapDev) * 4 * max_maps);
  L.scans = o;
  o = align16(o + sizeof(ScanDev) * max_scans);
  L.meta = o;
  o = align16(o + sizeof(ScanMeta) * max_scans);
  L.seg_first = o;
  o = align16(o + sizeof(int) * (2 * (size_t)max_scans + 1));
  L.seg_code = o;
  o = align16(o + sizeof(int) * 2 * (size_t)max_scans);
  L.total = o;
  return L;
}

size_t counter_bytes(int n_scans) { return sizeof(int) * (4 + 3 * (size_t)n_scans); }

}  // namespace

extern "C" {

cvx_status cvx_batch_create(int32_t max_submaps, int32_t max_scans, cvx_batch** out) {
  if (!out || max_submaps <= 0 || max_scans <= 0 || max_submaps > kMaxBatchMaps || max_scans > (1 << 20))
    return CVX_ERR_INVALID_ARG;
  *out = nullptr;
  cvx_batch* b = new (std::nothrow) cvx_batch();
  if (!b) return CVX_ERR_OOM;
  b->max_maps = max_submaps;
  b->max_scans = max_scans;
  const Layout L = layout(max_submaps, max_scans);
  b->bytes = L.total;
  b->lb_max = kMaxLocalBlocks;
  b->missing_cta = -1;
  b->polls = kWaitPolls;
  if (cudaMalloc(&b->dev, L.total) != cudaSuccess || cudaMallocHost(&b->host, L.total) != cudaSuccess ||
      cudaMalloc((void**)&b->ctr, counter_bytes(max_scans)) != cudaSuccess ||
      cudaMalloc((void**)&b->part_done, sizeof(int) * (size_t)max_submaps * kMaxMergeParts) != cudaSuccess ||
      cudaMalloc((void**)&b->phase_ns, sizeof(unsigned long long) * (1 + 2 * (size_t)max_scans)) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (b->dev) cudaFree(b->dev);
    if (b->host) cudaFreeHost(b->host);
    if (b->ctr) cudaFree(b->ctr);
    if (b->part_done) cudaFree(b->part_done);
    if (b->phase_ns) cudaFree(b->phase_ns);
    delete b;
    return CVX_ERR_OOM;
  }
  if (cudaMemset(b->ctr, 0, counter_bytes(max_scans)) != cudaSuccess) {
    cudaGetLastError();
    cvx_batch_destroy(b);
    return CVX_ERR_CUDA;
  }
  for (int v = 0; v < 7; ++v)
    cudaFuncSetAttribute((const void*)kBatched[v], cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tile_smem_bytes(kMaxLocalBlocks));
  *out = b;
  return CVX_OK;
}

void cvx_batch_destroy(cvx_batch* b) {
  if (!b) return;
  cudaEventSynchronize(b->copied);
  cudaFree(b->dev);
  cudaFreeHost(b->host);
  cudaFree(b->ctr);
  cudaFree(b->part_done);
  cudaFree(b->phase_ns);
  cudaEventDestroy(b->copied);
  delete b;
}

cvx_status cvx_batch_wave_limit(cvx_batch* b, int32_t max_scans_per_wave) {
  if (!b || max_scans_per_wave < 0) return CVX_ERR_INVALID_ARG;
  b->wave_limit = max_scans_per_wave;
  return CVX_OK;
}

cvx_status cvx_batch_submap_group(cvx_batch* b, int32_t group) {
  if (!b || group < 0) return CVX_ERR_INVALID_ARG;
  b->submap_group = group;
  return CVX_OK;
}

cvx_status cvx_batch_merge_parts(cvx_batch* b, int32_t parts) {
  if (!b || parts < 0 || parts > kMaxMergeParts) return CVX_ERR_INVALID_ARG;
  b->merge_parts = parts;
  return CVX_OK;
}

cvx_status cvx_batch_test_missing_cta(cvx_batch* b, int32_t missing_cta, int64_t barrier_polls) {
  if (!b) return CVX_ERR_INVALID_ARG;
  b->missing_cta = missing_cta < 0 ? -1 : missing_cta;
  b->polls = (missing_cta >= 0 && barrier_polls > 0) ? barrier_polls : kWaitPolls;
  return CVX_OK;
}

cvx_status cvx_batch_timing(cvx_batch* b, int32_t enable) {
  if (!b) return CVX_ERR_INVALID_ARG;
  b->timing = enable != 0;
  return CVX_OK;
}

int32_t cvx_batch_phase_times(cvx_batch* b, double* ms, int32_t max_scans) {
  if (!b || !ms || max_scans <= 0) return CVX_ERR_INVALID_ARG;
  const int ns = b->last_scans < max_scans ? b->last_scans : max_scans;
  if (ns <= 0) return 0;
  std::vector<unsigned long long> t(1 + 2 * (size_t)ns);
  if (cudaMemcpy(t.data(), b->phase_ns, sizeof(unsigned long long) * t.size(), cudaMemcpyDeviceToHost) !=
      cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  for (int s = 0; s < ns; ++s) {
    ms[3 * s] = (double)(t[1 + 2 * s] - t[0]) * 1e-6;
    ms[3 * s + 1] = (double)(t[2 + 2 * s] - t[0]) * 1e-6;
    ms[3 * s + 2] = 0.0;
  }
  return ns;
}

cvx_status cvx_integrate_batch(cvx_batch* b, cvx_submap* const* maps, int32_t n_maps,
                               const cvx_scan_desc* scans, int32_t n_scans, void* stream) {
  if (!b || !maps || n_maps <= 0 || n_maps > b->max_maps || n_scans < 0 || n_scans > b->max_scans ||
      (n_scans > 0 && !scans))
    return CVX_ERR_INVALID_ARG;
  for (int q = 0; q < n_maps; ++q)
    for (int r = 0; r < q; ++r)
      if (!maps[q] || maps[q] == maps[r]) return CVX_ERR_INVALID_ARG;   // distinct submaps
  // validate and describe every scan; empty scans are no frames; the rank of
  // a scan is its frame number within its submap in this launch
  std::vector<ScanDev> sd(n_scans);
  std::vector<int> lbs(n_scans), rank(n_scans), per_map(n_maps, 0), order;
  int lb_max = 0;
  for (int s = 0; s < n_scans; ++s) {
    const cvx_scan_desc& d = scans[s];
    if (d.submap < 0 || d.submap >= n_maps) return CVX_ERR_INVALID_ARG;
    const cvx_status v =
        make_scan_dev(maps[d.submap], d.points_xyz, d.n, d.T_sub_sensor, d.point_weights, &d.params, &sd[s], &lbs[s],
                      d.colors_rgb);
    if (v != CVX_OK) return v;
    if (d.n == 0) continue;
    rank[s] = per_map[d.submap]++;
    lb_max = std::max(lb_max, lbs[s]);
    order.push_back(s);
  }
  if (order.empty()) return CVX_OK;
  // queue order: groups of submap_group submaps one after another (all of
  // them in one group by default), within a group rounds of scans of equal
  // rank (cut into chunks of at most wave_limit scans); the merges of a
  // round's scans follow in the next round
  auto group_of = [&](int s) { return b->submap_group > 0 ? scans[s].submap / b->submap_group : 0; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    return group_of(a) != group_of(c) ? group_of(a) < group_of(c) : rank[a] < rank[c];
  });
  const int n_run = (int)order.size();
  std::vector<int> round_of(n_run);
  int n_rounds = 0;
  {
    long long prev = -1;
    int in_round = 0;
    for (int k = 0; k < n_run; ++k) {
      const long long rk = ((long long)group_of(order[k]) << 32) | (long long)rank[order[k]];
      if (rk != prev || (b->wave_limit > 0 && in_round >= b->wave_limit)) {
        ++n_rounds;
        in_round = 0;
        prev = rk;
      }
      round_of[k] = n_rounds - 1;
      ++in_round;
    }
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
  SubmapDev* hv = (SubmapDev*)(h + L.views);
  ScanDev* hs = (ScanDev*)(h + L.scans);
  ScanMeta* hm = (ScanMeta*)(h + L.meta);
  int* hsf = (int*)(h + L.seg_first);
  int* hsc = (int*)(h + L.seg_code);
  for (int q = 0; q < n_maps; ++q)
    for (int k = 0; k < 4; ++k) hv[4 * q + k] = set_view(maps[q], k % maps[q]->n_sets);
  // per scan (in queue order): descriptor, set, dependencies (the scans of
  // each submap so far, in order: the set of scan k is k mod n_sets)
  std::vector<std::vector<int>> of_map(n_maps);
  for (int k = 0; k < n_run; ++k) {
    const int s = order[k];
    const int q = scans[s].submap;
    const int ns = maps[q]->n_sets;
    std::vector<int>& prior = of_map[q];
    hs[k] = sd[s];
    hs[k].epoch_add = (uint32_t)rank[s];
    ScanMeta& mt = hm[k];
    mt.view = 4 * q + rank[s] % ns;
    mt.prev = prior.empty() ? -1 : prior.back();
    mt.prev_set = (int)prior.size() >= ns ? prior[prior.size() - ns] : -1;
    mt.n_tiles = sd[s].n_tiles;
    mt.lb = lbs[s];
    mt.epoch_end = rank[s] == per_map[q] - 1 ? per_map[q] : 0;
    prior.push_back(k);
  }
  // one variant for every scan: a kernel holding only that code
  int variant = -2;
  for (int k = 0; k < n_run; ++k) {
    const int v = tile_variant(lbs[order[k]], sd[order[k]].dropoff, general_form(sd[order[k]]));
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
  const int ctas = per_sm * num_sms();
  // Merge items per scan, per round of the queue: a round of few scans (one
  // submap, or the last frames of the longest chains) is a few merges on the
  // critical path, each cut into many parts (short latency); a round of many
  // scans runs its merges side by side, where fewer, larger parts cost less
  // queue traffic.  About one merge item per resident CTA per round: the
  // largest power of two <= ctas / (scans of the round), within [8, 64].
  std::vector<int> round_size(n_rounds, 0);
  for (int k = 0; k < n_run; ++k) ++round_size[round_of[k]];
  auto parts_of_round = [&](int r) {
    if (b->merge_parts > 0) return b->merge_parts;
    int p = 8;
    while (p < 64 && 2 * p * round_size[r] <= ctas) p *= 2;
    return p;
  };
  for (int k = 0; k < n_run; ++k) hm[k].parts = parts_of_round(round_of[k]);
  for (int k = 0; k < n_run; ++k) {
    hm[k].rank = rank[order[k]];
    hm[k].part_chain = hm[k].prev >= 0 && hm[hm[k].prev].parts == hm[k].parts;
  }
  // queue segments, round by round: merges of the previous round's
  // single-set scans (their submaps' next tiles wait for them), this round's
  // tiles, then the merges of the previous round's two-set scans (the next
  // tiles of those submaps do not wait for them)
  int n_segs = 0, items = 0;
  auto add_seg = [&](int code, int n) {
    hsf[n_segs] = items;
    hsc[n_segs] = code;
    ++n_segs;
    items += n;
  };
  {
    int k0 = 0;
    int pk0 = 0, pk1 = 0;   // previous round's scans [pk0, pk1)
    for (int r = 0; r <= n_rounds; ++r) {
      int k1 = k0;
      while (k1 < n_run && round_of[k1] == r) ++k1;
      for (int k = pk0; k < pk1; ++k)
        if (!maps[scans[order[k]].submap]->pipelined) add_seg(k | (1 << 30), hm[k].parts);
      for (int k = k0; k < k1; ++k) add_seg(k, hm[k].n_tiles);
      for (int k = pk0; k < pk1; ++k)
        if (maps[scans[order[k]].submap]->pipelined) add_seg(k | (1 << 30), hm[k].parts);
      pk0 = k0;
      pk1 = k1;
      k0 = k1;
    }
  }
  hsf[n_segs] = items;
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
  if (cudaMemsetAsync(b->ctr, 0, counter_bytes(n_run), st) != cudaSuccess ||
      cudaMemsetAsync(b->part_done, 0, sizeof(int) * (size_t)n_maps * kMaxMergeParts, st) != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  char* d = (char*)b->dev;
  BatchDev bd;
  bd.views = (const SubmapDev*)(d + L.views);
  bd.scans = (const ScanDev*)(d + L.scans);
  bd.meta = (const ScanMeta*)(d + L.meta);
  bd.seg_first = (const int*)(d + L.seg_first);
  bd.seg_code = (const int*)(d + L.seg_code);
  bd.n_segs = n_segs;
  bd.n_scans = n_run;
  bd.ctr = b->ctr;
  bd.part_done = b->part_done;
  bd.phase_ns = b->timing ? b->phase_ns : nullptr;
  bd.polls = b->polls;
  bd.missing_cta = b->missing_cta;
  b->last_scans = n_run;
  const int grid = std::min(ctas, std::max(items, 1));   // one wave of resident CTAs
  COVOX_LAUNCH(kKBatched, st, kern<<<grid, kTileThreads, tile_smem_bytes(lb_max), st>>>(bd));
  return cudaGetLastError() == cudaSuccess ? CVX_OK : CVX_ERR_CUDA;
}

int32_t cvx_batch_error(cvx_batch* b) {
  if (!b) return CVX_ERR_INVALID_ARG;
  int v[2] = {0, 0};
  if (cudaMemcpy(v, b->ctr, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  return (v[1] & (kErrTimeout | kErrIncomplete)) ? CVX_ERR_TIMEOUT : CVX_OK;
}

}  // extern "C"
