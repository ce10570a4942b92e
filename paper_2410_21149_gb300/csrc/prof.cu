// prof.cu -- launch counter and per-kernel event timing (tracing subsystem).
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "../../include/covox.h"
#include "prof.h"

namespace {

const char* kNames[covox::kNumKinds] = {"alloc_kernel",    "integrate_kernel", "merge_kernel",
                                        "reset_pools_kernel", "batched_kernel", "features_kernel",
                                        "mlp_fwd_kernel",  "mlp_bwd_kernel", "adam_kernel",
                                        "targets_kernel", "integrate_pipelined_kernel", "flush_kernel",
                                        "pipe_close_kernel", "esdf_kernels",
                                        "hash_kernels", "reset_states_kernel", "point_weights_kernel"};

struct Rec {
  int kind;
  cudaEvent_t a, b;
};

long long g_launches[covox::kNumKinds];
bool g_on = false;
long long g_cap = 0;
std::vector<Rec> g_recs;        // recorded this session
std::vector<cudaEvent_t> g_pool;  // created events for reuse
Rec g_open;
bool g_open_valid = false;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

}  // namespace

namespace covox {

void prof_begin(int kind, cudaStream_t s) {
  g_launches[kind]++;
  g_open_valid = false;
  if (!g_on || (long long)g_recs.size() >= g_cap) return;
  cudaEvent_t a = get_event(), b = get_event();
  if (!a || !b) return;
  cudaEventRecord(a, s);
  g_open = {kind, a, b};
  g_open_valid = true;
}

void prof_end(int kind, cudaStream_t s) {
  if (!g_open_valid || g_open.kind != kind) return;
  cudaEventRecord(g_open.b, s);
  g_recs.push_back(g_open);
  g_open_valid = false;
}

}  // namespace covox

extern "C" {

cvx_status cvx_profile_start(int64_t max_launches) {
  if (max_launches < 0) return CVX_ERR_INVALID_ARG;
  g_cap = max_launches;
  g_on = true;
  return CVX_OK;
}

cvx_status cvx_profile_stop(void) {
  g_on = false;
  return CVX_OK;
}

int32_t cvx_profile_read(int32_t max_kinds, char* names, double* total_ms, int64_t* launches) {
  double tot[covox::kNumKinds] = {0};
  long long cnt[covox::kNumKinds] = {0};
  for (const Rec& r : g_recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      tot[r.kind] += ms;
      cnt[r.kind]++;
    } else {
      cudaGetLastError();
    }
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  const int n = max_kinds < covox::kNumKinds ? max_kinds : covox::kNumKinds;
  for (int k = 0; k < n; ++k) {
    if (names) {
      std::strncpy(names + 32 * k, kNames[k], 31);
      names[32 * k + 31] = 0;
    }
    if (total_ms) total_ms[k] = tot[k];
    if (launches) launches[k] = cnt[k];
  }
  return n;
}

int64_t cvx_launch_count(void) {
  long long t = 0;
  for (int k = 0; k < covox::kNumKinds; ++k) t += g_launches[k];
  return t;
}

}  // extern "C"
