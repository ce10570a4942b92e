// hash.cu -- the block hash on its own (coVoxSLAM Sec. III-B "activate";
// the paper's hash stress test inserts tens of millions of keys).
//
// Same table as a submap's (packed 3 x 21-bit block keys, open addressing
// with linear probing from a murmur-finalised hash, keys claimed by 64-bit
// CAS, pool index published after the claim) but driven by a batch of block
// coordinates instead of scans:
//   hash_insert_kernel  insert-or-find; the new keys of a warp take their
//                       pool indices with one atomic per warp (warp-
//                       aggregated allocation), publish them, and every
//                       lane returns its key's pool index;
//   hash_find_kernel    read-only lookup (-1: absent).
// Waits are bounded (publication of a pool index by another warp).
#include <cuda_runtime.h>

#include <algorithm>
#include <new>

#include "../../include/covox.h"
#include "covox_dev.cuh"
#include "prof.h"
#include "submap.h"

using namespace covox;

struct cvx_block_hash {
  unsigned long long* keys;
  int32_t* vals;
  int32_t* block_keys;
  State* st;
  int64_t slots, max_blocks;
  cudaStream_t last_stream;
};

namespace {

constexpr int32_t kHashDead = -3;          // slot claimed but the pool was full
constexpr long long kPublishSpin = 1 << 22;

struct HashDev {
  unsigned long long* keys;
  int32_t* vals;
  int32_t* block_keys;
  State* st;
  uint32_t slot_mask;
  int max_probe, max_blocks;
};

HashDev view(const cvx_block_hash* h) {
  HashDev d;
  d.keys = h->keys;
  d.vals = h->vals;
  d.block_keys = h->block_keys;
  d.st = h->st;
  d.slot_mask = (uint32_t)(h->slots - 1);
  d.max_probe = (int)std::min<int64_t>(h->slots, 4096);
  d.max_blocks = (int)h->max_blocks;
  return d;
}

__device__ __forceinline__ bool key_in_range(int x, int y, int z) {
  const int lim = 1 << 20;
  return x >= -lim && x < lim && y >= -lim && y < lim && z >= -lim && z < lim;
}

__global__ void hash_insert_kernel(HashDev h, const int32_t* __restrict__ coords, long long n,
                                   int32_t* __restrict__ pool_out) {
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i0 = (long long)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {   // warp-uniform
    const long long i = i0 + threadIdx.x;
    bool valid = i < n;
    int x = 0, y = 0, z = 0;
    if (valid) {
      x = coords[3 * i];
      y = coords[3 * i + 1];
      z = coords[3 * i + 2];
      if (!key_in_range(x, y, z)) {
        atomicOr(&h.st->frame_err, kErrKeyRange);
        pool_out[i] = -1;
        valid = false;
      }
    }
    // probe: claim the key's slot or find it
    int slot = -1;
    bool inserted = false;
    if (valid) {
      const unsigned long long key = pack_key(x, y, z);
      uint32_t s = hash_key(key) & h.slot_mask;
      for (int p = 0; p < h.max_probe; ++p) {
        unsigned long long cur = *((volatile unsigned long long*)(h.keys + s));
        if (cur == kEmptyKey) {
          cur = atomicCAS(h.keys + s, kEmptyKey, key);
          if (cur == kEmptyKey) {
            inserted = true;
            slot = (int)s;
            break;
          }
        }
        if (cur == key) {
          slot = (int)s;
          break;
        }
        s = (s + 1) & h.slot_mask;
      }
      if (slot < 0) {
        atomicOr(&h.st->frame_err, kErrCapacity);
        pool_out[i] = -1;
      }
    }
    // warp-aggregated pool allocation of the warp's new keys
    __syncwarp();
    const unsigned ins = __ballot_sync(0xffffffffu, inserted);
    int base = 0;
    if (lane == 0 && ins) base = atomicAdd(&h.st->n_blocks, __popc(ins));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (inserted) {
      const int pool = base + __popc(ins & ((1u << lane) - 1u));
      if (pool >= h.max_blocks) {
        atomicOr(&h.st->frame_err, kErrCapacity);
        atomicExch(h.vals + slot, kHashDead);
        pool_out[i] = -1;
      } else {
        h.block_keys[3 * pool] = x;
        h.block_keys[3 * pool + 1] = y;
        h.block_keys[3 * pool + 2] = z;
        atomicExch(h.vals + slot, pool);   // publish
        pool_out[i] = pool;
      }
    }
    __syncwarp();   // the warp's own new keys are published before its lanes wait for others
    if (!inserted && slot >= 0) {
      int pool = *((volatile int32_t*)(h.vals + slot));
      for (long long it = 0; pool == -1 && it < kPublishSpin; ++it) {   // published by its inserter shortly
        __nanosleep(64);
        pool = *((volatile int32_t*)(h.vals + slot));
      }
      if (pool == -1) atomicOr(&h.st->frame_err, kErrTimeout);
      pool_out[i] = pool >= 0 ? pool : -1;
    }
  }
}

__global__ void hash_find_kernel(HashDev h, const int32_t* __restrict__ coords, long long n,
                                 int32_t* __restrict__ pool_out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int x = coords[3 * i], y = coords[3 * i + 1], z = coords[3 * i + 2];
    int pool = -1;
    if (key_in_range(x, y, z)) {
      const unsigned long long key = pack_key(x, y, z);
      uint32_t s = hash_key(key) & h.slot_mask;
      for (int p = 0; p < h.max_probe; ++p) {
        const unsigned long long cur = __ldg(h.keys + s);
        if (cur == key) {
          const int v = __ldg(h.vals + s);
          pool = v >= 0 ? v : -1;
          break;
        }
        if (cur == kEmptyKey) break;
        s = (s + 1) & h.slot_mask;
      }
    }
    pool_out[i] = pool;
  }
}

int grid_for(long long n) {
  const long long want = (n + 255) / 256;
  return (int)std::max<long long>(1, std::min<long long>(want, (long long)num_sms() * 16));
}

}  // namespace

extern "C" {

cvx_status cvx_block_hash_create(int64_t slots, int64_t max_blocks, cvx_block_hash** out) {
  if (!out || slots < 2 || (slots & (slots - 1)) || slots > (1ll << 31) || max_blocks <= 0 ||
      max_blocks > (1ll << 31) - 1)
    return CVX_ERR_INVALID_ARG;
  *out = nullptr;
  cvx_block_hash* h = new (std::nothrow) cvx_block_hash();
  if (!h) return CVX_ERR_OOM;
  h->slots = slots;
  h->max_blocks = max_blocks;
  h->last_stream = nullptr;
  if (cudaMalloc((void**)&h->keys, (size_t)slots * 8) != cudaSuccess ||
      cudaMalloc((void**)&h->vals, (size_t)slots * 4) != cudaSuccess ||
      cudaMalloc((void**)&h->block_keys, (size_t)max_blocks * 12) != cudaSuccess ||
      cudaMalloc((void**)&h->st, sizeof(State)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(h->keys);
    cudaFree(h->vals);
    cudaFree(h->block_keys);
    cudaFree(h->st);
    delete h;
    return CVX_ERR_OOM;
  }
  if (cudaMemset(h->keys, 0xff, (size_t)slots * 8) != cudaSuccess ||
      cudaMemset(h->vals, 0xff, (size_t)slots * 4) != cudaSuccess ||
      cudaMemset(h->st, 0, sizeof(State)) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    cudaFree(h->keys);
    cudaFree(h->vals);
    cudaFree(h->block_keys);
    cudaFree(h->st);
    delete h;
    return CVX_ERR_CUDA;
  }
  *out = h;
  return CVX_OK;
}

cvx_status cvx_block_hash_insert(cvx_block_hash* h, const int32_t* coords, int64_t n, int32_t* pool,
                                 void* stream) {
  if (!h || n < 0 || (n > 0 && (!coords || !pool))) return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  if (n == 0) return CVX_OK;
  COVOX_LAUNCH(kKHash, s, hash_insert_kernel<<<grid_for(n), 256, 0, s>>>(view(h), coords, n, pool));
  return cudaGetLastError() == cudaSuccess ? CVX_OK : CVX_ERR_CUDA;
}

cvx_status cvx_block_hash_find(cvx_block_hash* h, const int32_t* coords, int64_t n, int32_t* pool, void* stream) {
  if (!h || n < 0 || (n > 0 && (!coords || !pool))) return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  if (n == 0) return CVX_OK;
  COVOX_LAUNCH(kKHash, s, hash_find_kernel<<<grid_for(n), 256, 0, s>>>(view(h), coords, n, pool));
  return cudaGetLastError() == cudaSuccess ? CVX_OK : CVX_ERR_CUDA;
}

cvx_status cvx_block_hash_info(cvx_block_hash* h, int64_t* n_blocks, int32_t* block_keys, int64_t capacity) {
  if (!h || !n_blocks) return CVX_ERR_INVALID_ARG;
  State st;
  if (cudaMemcpyAsync(&st, h->st, sizeof(State), cudaMemcpyDeviceToHost, h->last_stream) != cudaSuccess ||
      cudaStreamSynchronize(h->last_stream) != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  const int64_t nb = std::min<int64_t>(st.n_blocks, h->max_blocks);
  *n_blocks = nb;
  if (block_keys && capacity > 0) {
    const int64_t k = std::min<int64_t>(nb, capacity);
    if (cudaMemcpy(block_keys, h->block_keys, (size_t)k * 12, cudaMemcpyDefault) != cudaSuccess) {
      cudaGetLastError();
      return CVX_ERR_CUDA;
    }
  }
  if (st.frame_err & kErrCapacity) return CVX_ERR_CAPACITY;
  if (st.frame_err & kErrKeyRange) return CVX_ERR_KEY_RANGE;
  if (st.frame_err & kErrTimeout) return CVX_ERR_TIMEOUT;
  return CVX_OK;
}

void cvx_block_hash_destroy(cvx_block_hash* h) {
  if (!h) return;
  cudaStreamSynchronize(h->last_stream);
  cudaFree(h->keys);
  cudaFree(h->vals);
  cudaFree(h->block_keys);
  cudaFree(h->st);
  delete h;
}

}  // extern "C"
