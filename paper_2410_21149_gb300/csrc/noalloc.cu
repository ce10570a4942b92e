// noalloc.cu -- integration of one scan without any device allocation.
//
// Some callers cannot call cudaMalloc: a real-time loop that must never
// allocate after start-up, a host whose memory manager owns all device memory
// and hands out fixed buffers, or a plugin that is not allowed to touch the
// process's allocator.  For them,
// cvx_integrate_scan_noalloc() integrates a scan into submap storage the
// caller already owns (a cvx_submap_view) and keeps its per-scan scratch (the
// per-voxel sums, the blocks' touch epochs and their groups' touch tags) in
// one file-scope device array
// of fixed size.  It runs the same device functions as cvx_integrate_scan.
//
// The scratch array is a host-side symbol in host code: its device address is
// obtained with cudaGetSymbolAddress once per device (with that device
// current) the first time the entry point runs there, and passed to the
// kernels.  Every GPU that loads this library holds the array until exit.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/covox.h"
#include "covox_dev.cuh"
#include "integrate_dev.cuh"
#include "prof.h"
#include "submap.h"

using namespace covox;

namespace {

constexpr size_t kAccBytes = (size_t)CVX_NOALLOC_MAX_BLOCKS * kVoxPerBlock * sizeof(float2);
constexpr size_t kEpochBytes = (size_t)CVX_NOALLOC_MAX_BLOCKS * sizeof(uint32_t);
constexpr size_t kTagBytes = (size_t)CVX_NOALLOC_MAX_BLOCKS * kGroupsPerBlock;
constexpr size_t kScratchBytes = kAccBytes + kEpochBytes + kTagBytes;

// per-scan sums | touch epochs of the blocks | touch tags of their groups
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

static_assert(sizeof(State) <= CVX_SUBMAP_STATE_BYTES, "state buffer too small");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices];

__global__ void __launch_bounds__(kTileThreads) integrate_static_kernel(SubmapDev m, ScanDev sc, int lb);

// Device address of the scratch array on the current device.  Set-up runs
// once per device, with that device current: the symbol address and the
// shared-memory limit of the variant kernel.
cvx_status scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return CVX_ERR_CUDA;
    }
    if (cudaFuncSetAttribute(integrate_static_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tile_smem_bytes(kMaxLocalBlocks)) != cudaSuccess) {
      cudaGetLastError();
      return CVX_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return CVX_OK;
}

__global__ void __launch_bounds__(kTileThreads) integrate_static_kernel(SubmapDev m, ScanDev sc, int lb) {
  extern __shared__ __align__(16) char smem[];
  integrate_tile(m, sc, blockIdx.x, smem, lb);
}

// The scan's epoch is 1: the touch epochs are cleared before every call.
__global__ void __launch_bounds__(kTileThreads) merge_static_kernel(SubmapDev m) {
  __shared__ unsigned long long red[kTileThreads / 32];
  __shared__ MergeSmemStatic sl;
  const int nb = min(*((volatile int32_t*)&m.st->n_blocks), m.max_blocks);
  const bool skip = *((volatile int32_t*)m.frame_err) != 0;
  unsigned long long merged = 0, touched = 0;
  for (int span = blockIdx.x; span * kSpanBlocks < nb; span += kSpansPerCall * gridDim.x) {
    int t = 0;
    merged += merge_span(m, span, gridDim.x, nb, 1u, skip, sl.view(), &t);
    touched += t;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) merged += __shfl_xor_sync(0xffffffffu, merged, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = merged;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kTileThreads / 32; ++w) t += red[w];
    if (t) atomicAdd(&m.st->voxels_merged, t);
    if (touched) atomicAdd(&m.st->blocks_touched, touched);
    __threadfence();
    if (atomicAdd(&m.st->ticket, 1u) == gridDim.x - 1) {
      __threadfence();
      State* st = m.st;
      st->frames += 1;
      st->sticky_err |= *m.frame_err;
      *m.frame_err = 0;
      st->ticket = 0;
    }
  }
}

}  // namespace

extern "C" cvx_status cvx_integrate_scan_noalloc(const cvx_submap_view* view, const float* points_xyz,
                                                 int64_t n, const float T_sub_sensor[12],
                                                 const float* point_weights,
                                                 const cvx_integrate_params* params, void* stream) {
  if (!view || !view->hash_keys || !view->hash_vals || !view->block_keys || !view->dist ||
      !view->weight || !view->state)
    return CVX_ERR_INVALID_ARG;
  if (view->hash_slots < 2 || (view->hash_slots & (view->hash_slots - 1)) ||
      view->hash_slots > (1ll << 31) || view->max_blocks <= 0)
    return CVX_ERR_INVALID_ARG;
  if (!(view->voxel_size > 0) || !(view->trunc > 0) || !(view->max_weight > 0))
    return CVX_ERR_INVALID_ARG;
  // Vector loads and stores of D and W (16 bytes), 64-bit atomics on the hash
  // keys and the state's counters: misaligned views are rejected here rather
  // than faulting on the GPU.
  const auto misaligned = [](const void* p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) != 0; };
  if (misaligned(view->dist, 16) || misaligned(view->weight, 16) || misaligned(view->hash_keys, 8) ||
      misaligned(view->state, 8) || misaligned(view->hash_vals, 4) || misaligned(view->block_keys, 4))
    return CVX_ERR_INVALID_ARG;
  if (view->max_blocks > CVX_NOALLOC_MAX_BLOCKS) return CVX_ERR_CAPACITY;   // beyond the scratch

  // A stack-only submap description for the shared argument checks.
  cvx_submap desc;
  std::memset(&desc, 0, sizeof(desc));
  desc.p.voxel_size = view->voxel_size;
  desc.p.trunc = view->trunc;
  desc.p.max_weight = view->max_weight;
  ScanDev sc;
  int lb = 0;
  const cvx_status v = make_scan_dev(&desc, points_xyz, n, T_sub_sensor, point_weights, params, &sc, &lb);
  if (v != CVX_OK) return v;

  void* scratch = nullptr;
  const cvx_status ss = scratch_address(&scratch);
  if (ss != CVX_OK) return ss;

  SubmapDev m;
  std::memset(&m, 0, sizeof(m));
  m.keys = view->hash_keys;
  m.vals = view->hash_vals;
  m.block_keys = view->block_keys;
  m.D = view->dist;
  m.W = view->weight;
  m.st = (State*)view->state;
  m.frame_err = &m.st->frame_err;
  unsigned char* base = (unsigned char*)scratch;
  m.acc = (float2*)base;
  m.tepoch = (uint32_t*)(base + kAccBytes);
  m.gep = base + kAccBytes + kEpochBytes;
  m.slot_mask = (uint32_t)(view->hash_slots - 1);
  m.max_probe = (int)(view->hash_slots < 4096 ? view->hash_slots : 4096);
  m.max_blocks = (int)view->max_blocks;
  m.vs = view->voxel_size;
  m.inv_vs = 1.0f / view->voxel_size;
  m.trunc = view->trunc;
  m.max_w = view->max_weight;
  m.storage = CVX_STORE_F32;

  cudaStream_t s = (cudaStream_t)stream;
  // The scratch keeps the previous call's contents: clear the sums, the
  // touch epochs, the group tags and this scan's fields of the caller's state (error bits,
  // merge ticket, epoch: the scan's epoch is 1).
  const size_t acc_bytes = (size_t)view->max_blocks * kVoxPerBlock * sizeof(float2);
  if (cudaMemsetAsync(m.acc, 0, acc_bytes, s) != cudaSuccess ||
      cudaMemsetAsync(m.tepoch, 0, (size_t)view->max_blocks * sizeof(uint32_t), s) != cudaSuccess ||
      cudaMemsetAsync(m.gep, 0, (size_t)view->max_blocks * kGroupsPerBlock, s) != cudaSuccess ||
      cudaMemsetAsync((char*)view->state + offsetof(State, frame_err), 0, sizeof(int32_t), s) != cudaSuccess ||
      cudaMemsetAsync((char*)view->state + offsetof(State, ticket), 0, sizeof(uint32_t), s) != cudaSuccess ||
      cudaMemsetAsync((char*)view->state + offsetof(State, epoch), 0, sizeof(uint32_t), s) != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  if (n == 0) return CVX_OK;
  COVOX_LAUNCH(kKAccum, s,
               integrate_static_kernel<<<sc.n_tiles, kTileThreads, tile_smem_bytes(lb), s>>>(m, sc, lb));
  const int spans = (m.max_blocks + kCallBlocks - 1) / kCallBlocks;
  const int grid = spans < num_sms() * 2 ? spans : num_sms() * 2;
  COVOX_LAUNCH(kKMerge, s, merge_static_kernel<<<grid, kTileThreads, 0, s>>>(m));
  return cudaGetLastError() == cudaSuccess ? CVX_OK : CVX_ERR_CUDA;
}
