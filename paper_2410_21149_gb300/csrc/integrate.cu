// integrate.cu -- the per-scan kernels and the C ABI of one submap.
//
// Per scan (one frame), two kernels on the caller's stream implement the
// count / allocate / process sequence of coVoxSLAM Sec. III-D:
//   integrate_kernel : one CTA per tile of points; band traversal of every
//                      point; blocks activated in the block hash through a
//                      CTA-local cache (Sec. III-B "activate"), pool indices
//                      claimed by atomic bump (allocation phase), each touched
//                      block stamped with the scan's epoch; observation sums
//                      reduced in shared memory or by L2 vector reductions
//                      (segmented reduction of commutative sums).
//   merge_kernel     : spans of 32 allocated blocks per CTA: the blocks stamped
//                      with the scan's epoch (the stream compaction) merged
//                      into D and W with coalesced vector loads and stores;
//                      the last CTA closes the frame.  One owner per block: no
//                      write races.
// A submap created with CVX_SUBMAP_PIPELINED runs one kernel per scan
// instead (integrate_pipelined_kernel): the merges of the previous scan share
// the launch with this scan's tiles, and flush_kernel merges the last scan
// before anything reads D and W.
// The device functions all kernels use live in integrate_dev.cuh so that the
// persistent batched kernel runs exactly the same arithmetic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "../../include/covox.h"
#include "covox_dev.cuh"
#include "integrate_dev.cuh"
#include "prof.h"
#include "submap.h"

using namespace covox;

namespace {

template <int kVariant>
__global__ void __launch_bounds__(kTileThreads) integrate_kernel(SubmapDev m, ScanDev sc, int lb) {
  extern __shared__ __align__(16) char smem[];
  integrate_tile_v<kVariant>(m, sc, blockIdx.x, smem, lb);
}

using IntegrateFn = void (*)(SubmapDev, ScanDev, int);
const IntegrateFn kIntegrate[7] = {integrate_kernel<-1>, integrate_kernel<0>, integrate_kernel<1>,
                                   integrate_kernel<2>,  integrate_kernel<3>, integrate_kernel<4>,
                                   integrate_kernel<5>};   // [variant + 1]

// Sum of one value over a 256-thread CTA (thread 0 gets it).
__device__ __forceinline__ unsigned long long cta_sum(unsigned long long v, unsigned long long* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned long long t = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kTileThreads / 32; ++w) t += red[w];
  return t;
}

// Merge of one scan: every allocated block's touch epoch checked, span by
// span.  Reads, by thread 0, the scan's block count, error bits and epoch, then
// takes a ticket (the fence orders the reads first; nothing is in flight
// yet).  The CTA drawing the last ticket knows every CTA has read them and
// closes the frame at once; the others merge from the values they read.
__global__ void __launch_bounds__(kTileThreads) merge_kernel(SubmapDev m) {
  __shared__ int head[3];
  __shared__ MergeSmemStatic sl;
  __shared__ unsigned long long red[kTileThreads / 32];
  if (threadIdx.x == 0) {
    const int nb = min(*((volatile int32_t*)&m.st->n_blocks), m.max_blocks);
    const int fe = *((volatile int32_t*)m.frame_err);
    const uint32_t ep = *((volatile uint32_t*)&m.st->epoch) + 1u;
    head[0] = nb;
    head[1] = fe;
    head[2] = (int)ep;
    __threadfence();
    if (atomicAdd(&m.st->ticket, 1u) == gridDim.x - 1) {
      State* st = m.st;
      st->frames += 1;
      st->sticky_err |= fe;
      st->epoch += 1;   // the next scan's tiles take the next epoch
      *m.frame_err = 0;
      st->ticket = 0;
    }
  }
  __syncthreads();
  const int nb = head[0];
  const bool skip = head[1] != 0;
  const uint32_t ep = (uint32_t)head[2];
  unsigned long long merged = 0, touched = 0;
  for (int span = blockIdx.x; span * kSpanBlocks < nb; span += kSpansPerCall * gridDim.x) {
    int t = 0;
    merged += merge_span(m, span, gridDim.x, nb, ep, skip, sl.view(), &t);
    touched += t;
  }
  const unsigned long long sum = cta_sum(merged, red);
  if (threadIdx.x == 0) {
    if (sum) atomicAdd(&m.st->voxels_merged, sum);
    if (touched) atomicAdd(&m.st->blocks_touched, touched);
  }
}

// Reset of up to kResetMaps submaps in two launches.  reset_pools_kernel:
// every hash slot emptied, the pool planes (D, W, colours) of the allocated
// blocks zeroed, every touch epoch and group tag cleared, and the per-scan sums a launch
// that gave up left unmerged cleared too: the blocks of a per-scan set
// stamped with an epoch after the last closed one (a batched launch numbers
// its scans st->epoch + 1, + 2, ... and closes them all at its end; a pending
// pipelined scan was dropped before this runs; merged blocks hold zero sums).
// Only blocks below min(n_blocks, max_blocks) ever receive an epoch.  The
// submaps' State words are read here and zeroed by reset_states_kernel
// afterwards.
constexpr int kResetMaps = 48;

struct ResetDesc {
  unsigned long long* keys;
  int32_t* vals;
  State* st;
  uint4 *D, *W, *C;              // pool planes; C: colour submaps, else nullptr
  float4* acc[4];                // per-scan sums of each set (float2 pairs)
  float4* cacc[4];               // per-scan colour sums of each set, or nullptr
  uint32_t* tepoch[4];
  uint32_t* gep[4];              // group tags of each set (32-bit words)
  long long slots;
  int32_t max_blocks, n_sets;
  int32_t plane16;               // 16-byte words of one block's D (or W) plane
};

struct ResetBatch {
  ResetDesc m[kResetMaps];
  int32_t n;
};

__global__ void __launch_bounds__(256) reset_pools_kernel(const __grid_constant__ ResetBatch rb) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthr = (long long)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const uint4 z = make_uint4(0u, 0u, 0u, 0u);
  for (int k = 0; k < rb.n; ++k) {
    const ResetDesc& d = rb.m[k];
    const int nb = min(d.st->n_blocks, d.max_blocks);
    const uint32_t e = d.st->epoch;
    for (long long q = tid; q < d.slots; q += nthr) {
      d.keys[q] = kEmptyKey;
      d.vals[q] = -1;
    }
    const long long n16 = (long long)nb * d.plane16;
    for (long long q = tid; q < n16; q += nthr) {
      d.D[q] = z;
      d.W[q] = z;
    }
    if (d.C)
      for (long long q = tid; q < 3 * (long long)nb * kVoxPerBlock / 4; q += nthr) d.C[q] = z;
    // one warp per (set, block): lane 0 reads and clears the epoch
    for (long long r = tid >> 5; r < (long long)d.n_sets * nb; r += nthr >> 5) {
      const int set = (int)(r / nb), p = (int)(r % nb);
      uint32_t t = 0;
      if (lane == 0) {
        t = d.tepoch[set][p];
        if (t) d.tepoch[set][p] = 0u;
      }
      t = __shfl_sync(0xffffffffu, t, 0);
      if (t == 0) continue;   // never touched by this set: its tags are clear
      d.gep[set][(size_t)p * (kGroupsPerBlock / 4) + lane] = 0u;
      if (t <= e) continue;
      float4* a = d.acc[set] + (size_t)p * (kVoxPerBlock / 2);
      for (int q = lane; q < kVoxPerBlock / 2; q += 32) a[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (d.cacc[set]) {
        float4* c = d.cacc[set] + (size_t)p * kVoxPerBlock;
        for (int q = lane; q < kVoxPerBlock; q += 32) c[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
}

__global__ void reset_states_kernel(const __grid_constant__ ResetBatch rb) {
  constexpr int kWords = (int)(sizeof(State) / 4);
  static_assert(sizeof(State) % 4 == 0, "State is a whole number of 32-bit words");
  for (int q = threadIdx.x; q < rb.n * kWords; q += blockDim.x)
    reinterpret_cast<uint32_t*>(rb.m[q / kWords].st)[q % kWords] = 0u;
}

// The per-scan set `which` of a pipelined submap: a describes set 0 (and
// everything the sets share), b the second set (a copy of a but for acc,
// cacc, tepoch, gep and frame_err).
__device__ __forceinline__ SubmapDev pick_set(const SubmapDev& a, const SubmapDev& b, int which) {
  SubmapDev m = a;
  if (which) {
    m.acc = b.acc;
    m.cacc = b.cacc;
    m.tepoch = b.tepoch;
    m.gep = b.gep;
    m.frame_err = b.frame_err;
  }
  return m;
}

// Merge the blocks of set m stamped with epoch ep among the first nb pool
// indices: spans first, first + step, ... (256-thread CTA).  Adds the merged
// voxels and touched blocks to the submap's counters.
template <bool kColour = true>
__device__ __noinline__ void merge_set(const SubmapDev& m, int nb, uint32_t ep, bool skip, int first, int step,
                                       const MergeSmem& ms, unsigned long long* red) {
  unsigned long long merged = 0, touched = 0;
  for (int span = first; span * kSpanBlocks < nb; span += kSpansPerCall * step) {
    int t = 0;
    merged += merge_span<kColour>(m, span, step, nb, ep, skip, ms, &t);
    touched += t;
  }
  const unsigned long long sum = cta_sum(merged, red);
  if (threadIdx.x == 0) {
    if (sum) atomicAdd(&m.st->voxels_merged, sum);
    if (touched) atomicAdd(&m.st->blocks_touched, touched);
  }
}

// Per-scan words of a pipelined submap as one launch sees them.  Thread 0 of
// every CTA reads them on entry and then takes a ticket (a fence orders the
// reads first; nothing of the CTA is in flight yet, so it costs little).  The
// CTA drawing the last ticket knows that every CTA has read, and at once
// closes the pending scan's frame (counters, sticky error, its set cleared
// for reuse; the merging CTAs work from the values they read), sets pending
// to `pend_after` and flips the parity when asked.  No CTA waits at its end.
struct PipeHead {
  int par;       // set this launch accumulates into
  int pending;   // set par ^ 1 holds a scan to merge
  int nb;        // allocated blocks
  int fe;        // the pending scan's error bits
  uint32_t ep;   // its epoch
};

__device__ __forceinline__ void pipe_head(const SubmapDev& a, const SubmapDev& b, int pend_after, bool flip,
                                          PipeHead* h) {
  if (threadIdx.x == 0) {
    State* st = a.st;
    const int par = *((volatile int32_t*)&st->parity);
    const int pend = *((volatile int32_t*)&st->pending);
    int32_t* fep = par ? a.frame_err : b.frame_err;   // the pending set is par ^ 1
    h->par = par;
    h->pending = pend;
    h->nb = min(*((volatile int32_t*)&st->n_blocks), a.max_blocks);
    h->fe = pend ? *((volatile int32_t*)fep) : 0;
    h->ep = *((volatile uint32_t*)&st->epoch);        // the pending scan closed its tiles with this epoch
    __threadfence();
    if (atomicAdd(&st->ticket, 1u) == gridDim.x - 1) {
      if (pend) {
        st->frames += 1;
        st->sticky_err |= h->fe;
        *fep = 0;
      }
      st->pending = pend_after;
      if (flip) st->parity = par ^ 1;
      st->ticket = 0;
    }
  }
  __syncthreads();
}

// Pipelined per-scan kernel.  The first sc.n_tiles CTAs integrate this
// scan's tiles into set parity; the n_merge CTAs after them merge the scan
// the previous call integrated (set parity ^ 1, if one is pending), filling
// the SMs the last tiles leave idle.  The tiles read neither D nor
// W, and the two sets share only the block hash and pool, so results equal
// merging each scan before the next one starts.  The per-scan words do not
// change during the launch: pipe_close_kernel, launched after it, closes the
// merged frame, makes this scan the pending one and flips the parity.
template <int kVariant>
__global__ void __launch_bounds__(kTileThreads, 5) integrate_pipelined_kernel(SubmapDev a, SubmapDev b, ScanDev sc,
                                                                           int lb, int n_merge) {
  extern __shared__ __align__(16) char smem[];
  __shared__ unsigned long long red[kTileThreads / 32];
  const int par = *((volatile int32_t*)&a.st->parity);
  if ((int)blockIdx.x < sc.n_tiles) {
    integrate_tile_v<kVariant>(pick_set(a, b, par), sc, (int)blockIdx.x, smem, lb);
    return;
  }
  if (*((volatile int32_t*)&a.st->pending) == 0) return;   // uniform over the merging CTAs
  const SubmapDev prev = pick_set(a, b, par ^ 1);
  // Blocks this scan's tiles allocate meanwhile carry other epochs, so any
  // count read here will do -- but one count for the whole CTA, read by
  // thread 0: every thread must run the same spans (CTA barriers inside).
  __shared__ int head[3];
  if (threadIdx.x == 0) {
    head[0] = min(*((volatile int32_t*)&a.st->n_blocks), a.max_blocks);
    head[1] = *((volatile int32_t*)prev.frame_err);
    head[2] = (int)*((volatile uint32_t*)&a.st->epoch);   // the previous scan's epoch
  }
  __syncthreads();
  merge_set<(kVariant < 0)>(prev, head[0], (uint32_t)head[2], head[1] != 0, (int)blockIdx.x - sc.n_tiles, n_merge,
                            merge_smem(smem), red);
}

// One thread, after integrate_pipelined_kernel: close the frame it merged
// (counters, sticky error, its set cleared for reuse), make the scan it
// accumulated the pending one and flip the parity.
__global__ void pipe_close_kernel(SubmapDev a, SubmapDev b) {
  State* st = a.st;
  const int par = st->parity;
  if (st->pending) {
    int32_t* fep = par ? a.frame_err : b.frame_err;   // the pending set is par ^ 1
    st->frames += 1;
    st->sticky_err |= *fep;
    *fep = 0;
  }
  st->pending = 1;
  st->parity = par ^ 1;
  st->epoch += 1;   // the next scan's tiles take the next epoch
}

using PipelinedFn = void (*)(SubmapDev, SubmapDev, ScanDev, int, int);
const PipelinedFn kPipelined[7] = {integrate_pipelined_kernel<-1>, integrate_pipelined_kernel<0>,
                                   integrate_pipelined_kernel<1>,  integrate_pipelined_kernel<2>,
                                   integrate_pipelined_kernel<3>,  integrate_pipelined_kernel<4>,
                                   integrate_pipelined_kernel<5>};   // [variant + 1]

// Merge the pending scan of a pipelined submap (no-op when none is pending).
// discard: clear its sums without touching D and W.
__global__ void __launch_bounds__(kTileThreads) flush_kernel(SubmapDev a, SubmapDev b, int discard) {
  __shared__ PipeHead h;
  __shared__ unsigned long long red[kTileThreads / 32];
  __shared__ MergeSmemStatic sl;
  pipe_head(a, b, 0, false, &h);
  if (!h.pending) return;   // uniform over the grid
  merge_set(pick_set(a, b, h.par ^ 1), h.nb, h.ep, discard || h.fe != 0, blockIdx.x, gridDim.x, sl.view(), red);
}

}  // namespace

namespace covox {

cvx_status flush_pending(cvx_submap* map, cudaStream_t s, bool discard) {
  if (!map->pipelined || !map->maybe_pending) return CVX_OK;
  COVOX_LAUNCH(kKFlush, s, flush_kernel<<<num_sms(), kTileThreads, 0, s>>>(map->dev, map->dev_b, discard ? 1 : 0));
  if (cudaGetLastError() != cudaSuccess) return CVX_ERR_CUDA;
  map->maybe_pending = false;
  return CVX_OK;
}

}  // namespace covox

// ===================================================================== C ABI
namespace {

// The per-scan kernels may use more than 48 KB of dynamic shared memory: the
// attribute is per device, so it is set once for each device, with that
// device current.
constexpr int kMaxDevices = 64;
std::mutex g_attr_mu;
bool g_attr_set[kMaxDevices];

cvx_status kernel_attributes() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (g_attr_set[dev]) return CVX_OK;
  const int bytes = (int)tile_smem_bytes(kMaxLocalBlocks);
  for (int v = 0; v < 7; ++v)
    if (cudaFuncSetAttribute((const void*)kIntegrate[v], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
            cudaSuccess ||
        cudaFuncSetAttribute((const void*)kPipelined[v], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
            cudaSuccess) {
      cudaGetLastError();
      return CVX_ERR_CUDA;
    }
  g_attr_set[dev] = true;
  return CVX_OK;
}

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
  if (p->max_blocks <= 0 || p->max_blocks > (1ll << 25)) return CVX_ERR_INVALID_ARG;
  if (p->hash_slots < 2 || (p->hash_slots & (p->hash_slots - 1)) || p->hash_slots > (1ll << 31))
    return CVX_ERR_INVALID_ARG;
  if (p->flags & ~(int64_t)(CVX_SUBMAP_PIPELINED | CVX_SUBMAP_FOUR_SETS | CVX_SUBMAP_COLOR))
    return CVX_ERR_INVALID_ARG;
  if (p->storage == CVX_STORE_F16 && p->max_weight > 65504.0f) return CVX_ERR_INVALID_ARG;
  if ((p->alloc == nullptr) != (p->free == nullptr)) return CVX_ERR_INVALID_ARG;

  cvx_submap* m = new (std::nothrow) cvx_submap();
  if (!m) return CVX_ERR_OOM;
  m->p = *p;
  const size_t slots = (size_t)p->hash_slots, nb = (size_t)p->max_blocks;
  m->bytes_per_vox = p->storage == CVX_STORE_F32 ? 4 : 2;
  SubmapDev& d = m->dev;
  d.keys = (unsigned long long*)sub_alloc(m, slots * 8);
  d.vals = (int32_t*)sub_alloc(m, slots * 4);
  d.block_keys = (int32_t*)sub_alloc(m, nb * 12);
  d.D = sub_alloc(m, nb * kVoxPerBlock * m->bytes_per_vox);
  d.W = sub_alloc(m, nb * kVoxPerBlock * m->bytes_per_vox);
  d.acc = (float2*)sub_alloc(m, nb * kVoxPerBlock * sizeof(float2));
  d.tepoch = (uint32_t*)sub_alloc(m, nb * 4);
  d.gep = (uint8_t*)sub_alloc(m, nb * kGroupsPerBlock);
  d.st = (State*)sub_alloc(m, sizeof(State));
  m->n_sets = (p->flags & CVX_SUBMAP_FOUR_SETS) ? 4 : ((p->flags & CVX_SUBMAP_PIPELINED) ? 2 : 1);
  m->pipelined = m->n_sets > 1;
  m->colour = (p->flags & CVX_SUBMAP_COLOR) != 0;
  const int expect = 9 + 3 * (m->n_sets - 1) + (m->colour ? 1 + m->n_sets : 0);
  float2* acc_x[3] = {nullptr, nullptr, nullptr};
  uint32_t* tep_x[3] = {nullptr, nullptr, nullptr};
  uint8_t* gep_x[3] = {nullptr, nullptr, nullptr};
  float4* cacc_x[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int k = 1; k < m->n_sets; ++k) {   // further per-scan sets: sums, touch epochs and group tags
    acc_x[k - 1] = (float2*)sub_alloc(m, nb * kVoxPerBlock * sizeof(float2));
    tep_x[k - 1] = (uint32_t*)sub_alloc(m, nb * 4);
    gep_x[k - 1] = (uint8_t*)sub_alloc(m, nb * kGroupsPerBlock);
  }
  if (m->colour) {   // RGB planes, and colour sums per per-scan set
    d.C = (float*)sub_alloc(m, nb * 3 * kVoxPerBlock * sizeof(float));
    for (int k = 0; k < m->n_sets; ++k) cacc_x[k] = (float4*)sub_alloc(m, nb * kVoxPerBlock * sizeof(float4));
    d.cacc = cacc_x[0];
  }
  if (m->n_allocs != expect) {
    sub_free_all(m);
    delete m;
    return CVX_ERR_OOM;
  }
  d.slot_mask = (uint32_t)(slots - 1);
  d.max_probe = (int)std::min<size_t>(slots, 4096);
  d.max_blocks = (int)nb;
  d.storage = p->storage;
  d.frame_err = &d.st->frame_err;
  d.vs = p->voxel_size;
  d.inv_vs = 1.0f / p->voxel_size;
  d.trunc = p->trunc;
  d.max_w = p->max_weight;
  int32_t* fe_x[3] = {&d.st->frame_err_b, &d.st->frame_err_c, &d.st->frame_err_d};
  for (int k = 1; k < m->n_sets; ++k) {
    SubmapDev& v = k == 1 ? m->dev_b : m->dev_cd[k - 2];
    v = d;
    v.acc = acc_x[k - 1];
    v.cacc = cacc_x[k];
    v.tepoch = tep_x[k - 1];
    v.gep = gep_x[k - 1];
    v.frame_err = fe_x[k - 1];
  }
  cudaStream_t s = (cudaStream_t)p->stream;
  m->last_stream = s;
  cudaMemsetAsync(d.keys, 0xff, slots * 8, s);
  cudaMemsetAsync(d.vals, 0xff, slots * 4, s);
  cudaMemsetAsync(d.tepoch, 0, nb * 4, s);
  cudaMemsetAsync(d.gep, 0, nb * kGroupsPerBlock, s);
  cudaMemsetAsync(d.D, 0, nb * kVoxPerBlock * m->bytes_per_vox, s);
  cudaMemsetAsync(d.W, 0, nb * kVoxPerBlock * m->bytes_per_vox, s);
  cudaMemsetAsync(d.acc, 0, nb * kVoxPerBlock * sizeof(float2), s);
  cudaMemsetAsync(d.st, 0, sizeof(State), s);
  for (int k = 1; k < m->n_sets; ++k) {
    cudaMemsetAsync(set_view(m, k).acc, 0, nb * kVoxPerBlock * sizeof(float2), s);
    cudaMemsetAsync(set_view(m, k).tepoch, 0, nb * 4, s);
    cudaMemsetAsync(set_view(m, k).gep, 0, nb * kGroupsPerBlock, s);
  }
  if (m->colour) {
    cudaMemsetAsync(d.C, 0, nb * 3 * kVoxPerBlock * sizeof(float), s);
    for (int k = 0; k < m->n_sets; ++k) cudaMemsetAsync(cacc_x[k], 0, nb * kVoxPerBlock * sizeof(float4), s);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    sub_free_all(m);
    delete m;
    return CVX_ERR_CUDA;
  }
  *out = m;
  return CVX_OK;
}

namespace {

cvx_status integrate_scan(cvx_submap* map, const float* points_xyz, int64_t n, const float T_sub_sensor[12],
                          const float* point_weights, const float* colors_rgb, const cvx_integrate_params* ip,
                          void* stream) {
  ScanDev sc;
  int lb = 0;
  const cvx_status v = make_scan_dev(map, points_xyz, n, T_sub_sensor, point_weights, ip, &sc, &lb, colors_rgb);
  if (v != CVX_OK) return v;
  cudaStream_t s = (cudaStream_t)stream;
  map->last_stream = s;
  if (n == 0) return CVX_OK;
  const size_t smem = tile_smem_bytes(lb);
  if (kernel_attributes() != CVX_OK) return CVX_ERR_CUDA;
  if (map->pipelined) {
    const int n_merge = num_sms();
    const PipelinedFn pf = kPipelined[tile_variant(lb, sc.dropoff, general_form(sc)) + 1];
    COVOX_LAUNCH(kKPipelined, s,
                 pf<<<n_merge + sc.n_tiles, kTileThreads, smem, s>>>(map->dev, map->dev_b, sc, lb, n_merge));
    COVOX_LAUNCH(kKPipeClose, s, pipe_close_kernel<<<1, 1, 0, s>>>(map->dev, map->dev_b));
    if (cudaGetLastError() != cudaSuccess) return CVX_ERR_CUDA;
    map->maybe_pending = true;
    return CVX_OK;
  }
  const IntegrateFn fn = kIntegrate[tile_variant(lb, sc.dropoff, general_form(sc)) + 1];
  COVOX_LAUNCH(kKAccum, s, fn<<<sc.n_tiles, kTileThreads, smem, s>>>(map->dev, sc, lb));
  const int grid = std::min<int>((map->dev.max_blocks + kCallBlocks - 1) / kCallBlocks, num_sms() * 2);
  COVOX_LAUNCH(kKMerge, s, merge_kernel<<<grid, kTileThreads, 0, s>>>(map->dev));
  return cudaGetLastError() == cudaSuccess ? CVX_OK : CVX_ERR_CUDA;
}

}  // namespace

cvx_status cvx_integrate_scan(cvx_submap* map, const float* points_xyz, int64_t n,
                              const float T_sub_sensor[12], const float* point_weights,
                              const cvx_integrate_params* ip, void* stream) {
  return integrate_scan(map, points_xyz, n, T_sub_sensor, point_weights, nullptr, ip, stream);
}

cvx_status cvx_integrate_scan_color(cvx_submap* map, const float* points_xyz, int64_t n,
                                    const float T_sub_sensor[12], const float* point_weights,
                                    const float* colors_rgb, const cvx_integrate_params* ip, void* stream) {
  return integrate_scan(map, points_xyz, n, T_sub_sensor, point_weights, colors_rgb, ip, stream);
}

cvx_status cvx_extract_colors(cvx_submap* map, int64_t capacity, float* rgb, int64_t* n_out, void* stream) {
  if (!map || !n_out || capacity < 0 || !map->colour) return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (flush_pending(map, s, false) != CVX_OK) return CVX_ERR_CUDA;
  int32_t nb = 0;
  if (cudaMemcpyAsync(&nb, &map->dev.st->n_blocks, sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  nb = std::min<int32_t>(nb, map->dev.max_blocks);
  if (!rgb) {
    *n_out = nb;
    return CVX_OK;
  }
  const int64_t n = std::min<int64_t>(nb, capacity);
  *n_out = n;
  if (n == 0) return CVX_OK;
  if (cudaMemcpyAsync(rgb, map->dev.C, (size_t)n * 3 * kVoxPerBlock * sizeof(float), cudaMemcpyDefault, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  return CVX_OK;
}

cvx_status cvx_extract_blocks(cvx_submap* map, int64_t capacity, int32_t* keys, void* dist,
                              void* weight, int64_t* n_out, void* stream) {
  if (!map || !n_out || capacity < 0) return CVX_ERR_INVALID_ARG;
  if (keys && capacity > 0 && (!dist || !weight)) return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (flush_pending(map, s, false) != CVX_OK) return CVX_ERR_CUDA;
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

cvx_status cvx_reset_submaps(cvx_submap* const* maps, int32_t n, void* stream) {
  if (n < 0 || (n > 0 && !maps)) return CVX_ERR_INVALID_ARG;
  for (int q = 0; q < n; ++q)
    if (!maps[q]) return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  for (int q0 = 0; q0 < n; q0 += kResetMaps) {
    ResetBatch rb;
    std::memset(&rb, 0, sizeof(rb));
    rb.n = std::min(kResetMaps, n - q0);
    long long work = 0;
    for (int k = 0; k < rb.n; ++k) {
      cvx_submap* map = maps[q0 + k];
      map->last_stream = s;
      if (flush_pending(map, s, true) != CVX_OK) return CVX_ERR_CUDA;
      ResetDesc& d = rb.m[k];
      d.keys = map->dev.keys;
      d.vals = map->dev.vals;
      d.st = map->dev.st;
      d.D = (uint4*)map->dev.D;
      d.W = (uint4*)map->dev.W;
      d.C = (uint4*)map->dev.C;
      for (int k2 = 0; k2 < map->n_sets; ++k2) {
        const SubmapDev& v = set_view(map, k2);
        d.acc[k2] = (float4*)v.acc;
        d.cacc[k2] = v.cacc;
        d.tepoch[k2] = v.tepoch;
        d.gep[k2] = (uint32_t*)v.gep;
      }
      d.slots = map->p.hash_slots;
      d.max_blocks = map->dev.max_blocks;
      d.n_sets = map->n_sets;
      d.plane16 = (int)(kVoxPerBlock * map->bytes_per_vox / 16);
      work += d.slots + (long long)d.max_blocks * d.plane16;
    }
    // enough CTAs for the largest possible reset, at most four per SM
    const int grid = (int)std::max<long long>(1, std::min<long long>(4ll * num_sms(), work / 4096 + 1));
    COVOX_LAUNCH(kKZeroPool, s, reset_pools_kernel<<<grid, 256, 0, s>>>(rb));
    COVOX_LAUNCH(kKDiscard, s, reset_states_kernel<<<1, 256, 0, s>>>(rb));
  }
  return cudaGetLastError() == cudaSuccess ? CVX_OK : CVX_ERR_CUDA;
}

cvx_status cvx_reset_submap(cvx_submap* map, void* stream) {
  if (!map) return CVX_ERR_INVALID_ARG;
  return cvx_reset_submaps(&map, 1, stream);
}

cvx_status cvx_submap_counters(cvx_submap* map, cvx_counters* out) {
  if (!map || !out) return CVX_ERR_INVALID_ARG;
  if (flush_pending(map, map->last_stream, false) != CVX_OK) return CVX_ERR_CUDA;
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
  return status_from_bits(st.sticky_err | st.frame_err | st.frame_err_b | st.frame_err_c | st.frame_err_d);
}

cvx_status cvx_flush_submap(cvx_submap* map, void* stream) {
  if (!map) return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  map->last_stream = s;
  return flush_pending(map, s, false);
}

void cvx_destroy(cvx_submap* map) {
  if (!map) return;
  cudaStreamSynchronize(map->last_stream);
  sub_free_all(map);
  delete map;
}

}  // extern "C"
