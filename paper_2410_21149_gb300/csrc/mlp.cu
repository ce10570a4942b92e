// mlp.cu -- learned per-point integration weight: features, training targets,
// a 3-32-32-1 MLP (BF16 tensor-core GEMMs, FP32 accumulation), its backward
// pass with a deterministic gradient reduction, and Adam.
//
// coVoxSLAM Sec. III-C (weighting paragraph): the weight should follow the
// sensor's error curve, and ray casting lets every point carry its own
// weight.  Here a small network predicts that weight from the point's range,
// incidence angle and local depth variance; it is trained on residuals of
// noisy scans against the TSDF the plain integrator fuses from the same scans
// without noise (negative log likelihood w e2 - ln w, optimum w = 1 / e2).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <mma.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "../../include/covox.h"
#include "covox_dev.cuh"
#include "integrate_dev.cuh"
#include "prof.h"
#include "submap.h"
#include "weights_dev.cuh"

using namespace covox;
using namespace covox::wnet;
namespace wm = nvcuda::wmma;

namespace {

constexpr int kInPad = 16;            // K of the first GEMM
constexpr int kWarps = 4;
constexpr int kThreads = 32 * kWarps;
constexpr int kMaxGrid = 1024;

__global__ void __launch_bounds__(kFtThreads) features_kernel(const float* __restrict__ pts, int H, int W,
                                                               int sensor, float max_range,
                                                               float* __restrict__ out) {
  __shared__ FeatTile T;
  const int tiles_x = (W + kFtW - 1) / kFtW;
  const int x0 = (blockIdx.x % tiles_x) * kFtW - kHalo, y0 = (blockIdx.x / tiles_x) * kFtH - kHalo;
  stage_tile(T, pts, H, W, sensor, x0, y0);
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float f2[kFtRows];
  tile_variance_features(T, tx, ty, f2);
  const int u = x0 + kHalo + tx;
#pragma unroll
  for (int k = 0; k < kFtRows; ++k) {
    const int v = y0 + kHalo + kFtRows * ty + k;
    if (u >= W || v >= H) continue;
    float f[3];
    point_features(T, tx, ty, k, x0, y0, H, W, 1.0f / max_range, f2[k], f);
    const size_t idx = (size_t)v * W + u;
    out[3 * idx] = f[0];
    out[3 * idx + 1] = f[1];
    out[3 * idx + 2] = f[2];
  }
}

// ------------------------------------------------------- training targets
// e2 = mean over the point's band voxels with clean W > 0 of (d - D_clean)^2.
__global__ void targets_kernel(SubmapDev clean, ScanDev sc, float* __restrict__ e2, float* __restrict__ mask) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sc.n) return;
  float acc = 0.0f;
  int cnt = 0;
  Ray r;
  float A[3], B[3];
  if (make_ray(sc, i, r) && band(r, clean.trunc, clean.inv_vs, A, B)) {
    Dda d;
    d.init(A, B);
    int cb0 = 0x7fffffff, cb1 = 0, cb2 = 0, pool = -1;
    for (;;) {
      const int b0 = d.v[0] >> 3, b1 = d.v[1] >> 3, b2 = d.v[2] >> 3;
      if (b0 != cb0 || b1 != cb1 || b2 != cb2) {
        cb0 = b0; cb1 = b1; cb2 = b2;
        pool = find_pool(clean, pack_key(b0, b1, b2));
      }
      if (pool >= 0) {
        const size_t e = (size_t)pool * kVoxPerBlock + local_index(d.v);
        const float w = ((const float*)clean.W)[e];
        if (w > 0.0f) {
          const float diff = voxel_distance(r, d.v, clean.vs, clean.trunc) - ((const float*)clean.D)[e];
          acc += diff * diff;
          ++cnt;
        }
      }
      if (d.left == 0) break;
      d.step();
    }
  }
  e2[i] = cnt ? acc / cnt : 0.0f;
  mask[i] = cnt ? 1.0f : 0.0f;
}

// ------------------------------------------------------------------ MLP
struct alignas(128) WarpSmem {
  __nv_bfloat16 xb[16 * kInPad];   // [16 pts][16 in]
  __nv_bfloat16 h1b[16 * kH];      // [16 pts][32]
  __nv_bfloat16 h2b[16 * kH];
  __nv_bfloat16 g2b[16 * kH];      // dh2 rounded
  __nv_bfloat16 g1b[16 * kH];      // dh1 rounded
  float c[16 * kH];                // accumulator staging
  float h1[16 * kH];               // post-relu activations (relu masks)
  float h2[16 * kH];
  float dout[16];
};

struct alignas(128) MlpSmem {
  alignas(128) __nv_bfloat16 w1b[kH * kInPad];  // [32 out][16 in], zero padded
  __nv_bfloat16 w2b[kH * kH];      // [32 out][32 in]
  float b1[kH], b2[kH], w3[kH], b3;
  alignas(128) WarpSmem warp[kWarps];
  float red[kWarps][kP + 2];       // per-warp partial gradients (+ loss, count)
};

// mode 0: inference (writes w); mode 1: training (per-CTA partial gradient
// sums, loss sum and valid count in partial[blockIdx.x][kP + 2]).
template <int kMode>
__global__ void __launch_bounds__(kThreads) mlp_kernel(const float* __restrict__ params,
                                                        const float* __restrict__ x, const float* __restrict__ e2,
                                                        const float* __restrict__ mask, long long n,
                                                        float* __restrict__ wout, float* __restrict__ partial) {
  extern __shared__ __align__(128) char smem_raw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  WarpSmem& ws = S.warp[wid];
  for (int q = tid; q < kH * kInPad; q += kThreads) {
    const int o = q / kInPad, k = q % kInPad;
    S.w1b[q] = __float2bfloat16_rn(k < kIn ? params[kOW1 + o * kIn + k] : 0.0f);
  }
  for (int q = tid; q < kH * kH; q += kThreads) S.w2b[q] = __float2bfloat16_rn(params[kOW2 + q]);
  if (tid < kH) {
    S.b1[tid] = params[kOB1 + tid];
    S.b2[tid] = params[kOB2 + tid];
    S.w3[tid] = params[kOW3 + tid];
  }
  if (tid == 0) S.b3 = params[kOB3];
  __syncthreads();

  // per-lane gradient partials (lane = feature index)
  float g_b1 = 0.f, g_b2 = 0.f, g_w3 = 0.f, g_b3 = 0.f, g_loss = 0.f, g_cnt = 0.f;
  wm::fragment<wm::accumulator, 16, 16, 16, float> acc_w2[2][2], acc_w1[2];
  if (kMode == 1) {
    for (int a = 0; a < 2; ++a) {
      wm::fill_fragment(acc_w1[a], 0.0f);
      for (int b = 0; b < 2; ++b) wm::fill_fragment(acc_w2[a][b], 0.0f);
    }
  }
  const long long tiles = (n + 15) / 16;
  for (long long t = (long long)blockIdx.x * kWarps + wid; t < tiles; t += (long long)gridDim.x * kWarps) {
    const long long p0 = t * 16;
    // ---- inputs
    for (int q = lane; q < 16 * kInPad; q += 32) {
      const int pt = q / kInPad, k = q % kInPad;
      const long long i = p0 + pt;
      ws.xb[q] = __float2bfloat16_rn((k < kIn && i < n) ? x[3 * i + k] : 0.0f);
    }
    __syncwarp();
    // ---- layer 1: [16 x 16] . [16 x 32]
    {
      wm::fragment<wm::matrix_a, 16, 16, 16, __nv_bfloat16, wm::row_major> a;
      wm::load_matrix_sync(a, ws.xb, kInPad);
      for (int nt = 0; nt < 2; ++nt) {
        wm::fragment<wm::matrix_b, 16, 16, 16, __nv_bfloat16, wm::col_major> b;
        wm::fragment<wm::accumulator, 16, 16, 16, float> c;
        wm::fill_fragment(c, 0.0f);
        wm::load_matrix_sync(b, S.w1b + nt * 16 * kInPad, kInPad);
        wm::mma_sync(c, a, b, c);
        wm::store_matrix_sync(ws.c + nt * 16, c, kH, wm::mem_row_major);
      }
    }
    __syncwarp();
    for (int q = lane; q < 16 * kH; q += 32) {
      const float h = fmaxf(ws.c[q] + S.b1[q % kH], 0.0f);
      ws.h1[q] = h;
      ws.h1b[q] = __float2bfloat16_rn(h);
    }
    __syncwarp();
    // ---- layer 2: [16 x 32] . [32 x 32]
    for (int nt = 0; nt < 2; ++nt) {
      wm::fragment<wm::accumulator, 16, 16, 16, float> c;
      wm::fill_fragment(c, 0.0f);
      for (int kt = 0; kt < 2; ++kt) {
        wm::fragment<wm::matrix_a, 16, 16, 16, __nv_bfloat16, wm::row_major> a;
        wm::fragment<wm::matrix_b, 16, 16, 16, __nv_bfloat16, wm::col_major> b;
        wm::load_matrix_sync(a, ws.h1b + kt * 16, kH);
        wm::load_matrix_sync(b, S.w2b + nt * 16 * kH + kt * 16, kH);
        wm::mma_sync(c, a, b, c);
      }
      wm::store_matrix_sync(ws.c + nt * 16, c, kH, wm::mem_row_major);
    }
    __syncwarp();
    for (int q = lane; q < 16 * kH; q += 32) {
      const float h = fmaxf(ws.c[q] + S.b2[q % kH], 0.0f);
      ws.h2[q] = h;
      ws.h2b[q] = __float2bfloat16_rn(h);
    }
    __syncwarp();
    // ---- layer 3 (scalar) and the loss
    if (lane < 16) {
      const long long i = p0 + lane;
      float o = S.b3;
      for (int k = 0; k < kH; ++k) o += S.w3[k] * __bfloat162float(ws.h2b[lane * kH + k]);
      const float w = softplus_f(o);
      float dout = 0.0f;
      if (i < n) {
        if (kMode == 0) {
          wout[i] = w;
        } else {
          const float m = mask[i];
          const float e = e2[i];
          dout = m * (e - 1.0f / w) * sigmoid_f(o);
          g_loss += m * (w * e - logf(w));
          g_cnt += m;
        }
      }
      ws.dout[lane] = dout;
    }
    if (kMode == 0) {
      __syncwarp();
      continue;
    }
    __syncwarp();
    // ---- backward: output layer (lane = feature k)
    {
      float s = 0.0f, sb = 0.0f;
      for (int pt = 0; pt < 16; ++pt) {
        const float d = ws.dout[pt];
        s += d * __bfloat162float(ws.h2b[pt * kH + lane]);
        sb += d;
      }
      g_w3 += s;
      if (lane == 0) g_b3 += sb;
    }
    // dh2 = dout W3 * relu'(a2)
    {
      float sb2 = 0.0f;
      for (int pt = 0; pt < 16; ++pt) {
        const int q = pt * kH + lane;
        const float g = ws.h2[q] > 0.0f ? ws.dout[pt] * S.w3[lane] : 0.0f;
        sb2 += g;
        ws.g2b[q] = __float2bfloat16_rn(g);
      }
      g_b2 += sb2;
    }
    __syncwarp();
    // dW2 += dh2b^T h1b ; dh1 = dh2b W2b
    for (int mt = 0; mt < 2; ++mt) {
      wm::fragment<wm::matrix_a, 16, 16, 16, __nv_bfloat16, wm::col_major> a;   // dh2b^T
      wm::load_matrix_sync(a, ws.g2b + mt * 16, kH);
      for (int nt = 0; nt < 2; ++nt) {
        wm::fragment<wm::matrix_b, 16, 16, 16, __nv_bfloat16, wm::row_major> b;  // h1b
        wm::load_matrix_sync(b, ws.h1b + nt * 16, kH);
        wm::mma_sync(acc_w2[mt][nt], a, b, acc_w2[mt][nt]);
      }
    }
    for (int nt = 0; nt < 2; ++nt) {
      wm::fragment<wm::accumulator, 16, 16, 16, float> c;
      wm::fill_fragment(c, 0.0f);
      for (int kt = 0; kt < 2; ++kt) {
        wm::fragment<wm::matrix_a, 16, 16, 16, __nv_bfloat16, wm::row_major> a;   // dh2b
        wm::fragment<wm::matrix_b, 16, 16, 16, __nv_bfloat16, wm::row_major> b;   // W2b [out][in]
        wm::load_matrix_sync(a, ws.g2b + kt * 16, kH);
        wm::load_matrix_sync(b, S.w2b + kt * 16 * kH + nt * 16, kH);
        wm::mma_sync(c, a, b, c);
      }
      wm::store_matrix_sync(ws.c + nt * 16, c, kH, wm::mem_row_major);
    }
    __syncwarp();
    {
      float sb1 = 0.0f;
      for (int pt = 0; pt < 16; ++pt) {
        const int q = pt * kH + lane;
        const float g = ws.h1[q] > 0.0f ? ws.c[q] : 0.0f;
        sb1 += g;
        ws.g1b[q] = __float2bfloat16_rn(g);
      }
      g_b1 += sb1;
    }
    __syncwarp();
    // dW1 += dh1b^T xb
    for (int mt = 0; mt < 2; ++mt) {
      wm::fragment<wm::matrix_a, 16, 16, 16, __nv_bfloat16, wm::col_major> a;
      wm::fragment<wm::matrix_b, 16, 16, 16, __nv_bfloat16, wm::row_major> b;
      wm::load_matrix_sync(a, ws.g1b + mt * 16, kH);
      wm::load_matrix_sync(b, ws.xb, kInPad);
      wm::mma_sync(acc_w1[mt], a, b, acc_w1[mt]);
    }
    __syncwarp();
  }
  if (kMode == 0) return;
  // ---- per-warp partials to shared memory, then a fixed-order CTA sum
  float* r = S.red[wid];
  for (int mt = 0; mt < 2; ++mt)
    for (int nt = 0; nt < 2; ++nt) {
      wm::store_matrix_sync(ws.c, acc_w2[mt][nt], 16, wm::mem_row_major);
      __syncwarp();
      for (int q = lane; q < 256; q += 32) {
        const int o = mt * 16 + q / 16, i = nt * 16 + q % 16;
        r[kOW2 + o * kH + i] = ws.c[q];
      }
      __syncwarp();
    }
  for (int mt = 0; mt < 2; ++mt) {
    wm::store_matrix_sync(ws.c, acc_w1[mt], 16, wm::mem_row_major);
    __syncwarp();
    for (int q = lane; q < 16 * kIn; q += 32) {
      const int o = mt * 16 + q / kIn, i = q % kIn;
      r[kOW1 + o * kIn + i] = ws.c[(q / kIn) * 16 + i];
    }
    __syncwarp();
  }
  r[kOB1 + lane] = g_b1;
  r[kOB2 + lane] = g_b2;
  r[kOW3 + lane] = g_w3;
  float lsum = g_loss, csum = g_cnt, b3s = g_b3;
  for (int o = 16; o > 0; o >>= 1) {
    lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    csum += __shfl_xor_sync(0xffffffffu, csum, o);
  }
  if (lane == 0) {
    r[kOB3] = b3s;
    r[kP] = lsum;
    r[kP + 1] = csum;
  }
  __syncthreads();
  for (int q = tid; q < kP + 2; q += kThreads) {
    float s = 0.0f;
    for (int w = 0; w < kWarps; ++w) s += S.red[w][q];
    partial[(size_t)blockIdx.x * (kP + 2) + q] = s;
  }
}

// Inference only: 8 warps, each with the weight fragments of both GEMMs held
// in registers across its tiles of 16 points; small shared staging.
constexpr int kIWarps = 8;
struct alignas(128) InferWarp {
  __nv_bfloat16 xb[16 * kInPad];
  __nv_bfloat16 h1b[16 * kH];
  __nv_bfloat16 h2b[16 * kH];
  float c[16 * kH];
};
struct alignas(128) InferSmem {
  alignas(128) __nv_bfloat16 w1b[kH * kInPad];
  __nv_bfloat16 w2b[kH * kH];
  float b1[kH], b2[kH], w3[kH], b3;
  alignas(128) InferWarp warp[kIWarps];
};

__global__ void __launch_bounds__(32 * kIWarps) mlp_infer_kernel(const float* __restrict__ params,
                                                                  const float* __restrict__ x, long long n,
                                                                  float* __restrict__ wout) {
  __shared__ InferSmem S;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  InferWarp& ws = S.warp[wid];
  for (int q = tid; q < kH * kInPad; q += blockDim.x) {
    const int o = q / kInPad, k = q % kInPad;
    S.w1b[q] = __float2bfloat16_rn(k < kIn ? params[kOW1 + o * kIn + k] : 0.0f);
  }
  for (int q = tid; q < kH * kH; q += blockDim.x) S.w2b[q] = __float2bfloat16_rn(params[kOW2 + q]);
  if (tid < kH) {
    S.b1[tid] = params[kOB1 + tid];
    S.b2[tid] = params[kOB2 + tid];
    S.w3[tid] = params[kOW3 + tid];
  }
  if (tid == 0) S.b3 = params[kOB3];
  __syncthreads();
  wm::fragment<wm::matrix_b, 16, 16, 16, __nv_bfloat16, wm::col_major> B1[2], B2[2][2];
  for (int nt = 0; nt < 2; ++nt) {
    wm::load_matrix_sync(B1[nt], S.w1b + nt * 16 * kInPad, kInPad);
    for (int kt = 0; kt < 2; ++kt) wm::load_matrix_sync(B2[nt][kt], S.w2b + nt * 16 * kH + kt * 16, kH);
  }
  // padding columns of the input tile stay zero; each tile writes its 48 values
  for (int q = lane; q < 16 * kInPad; q += 32) ws.xb[q] = __float2bfloat16_rn(0.0f);
  __syncwarp();
  const long long tiles = (n + 15) / 16;
  long long t = (long long)blockIdx.x * kIWarps + wid;
  // the next tile's inputs are loaded (coalesced, 48 floats) while this one runs
  float nx0 = 0.f, nx1 = 0.f;
  auto load = [&](long long tt) {
    const long long b = tt * 48;
    nx0 = (tt < tiles && b + lane < 3 * n) ? __ldg(x + b + lane) : 0.0f;
    nx1 = (tt < tiles && lane < 16 && b + 32 + lane < 3 * n) ? __ldg(x + b + 32 + lane) : 0.0f;
  };
  load(t);
  for (; t < tiles; t += (long long)gridDim.x * kIWarps) {
    const long long p0 = t * 16;
    ws.xb[(lane / 3) * kInPad + lane % 3] = __float2bfloat16_rn(nx0);
    if (lane < 16) ws.xb[((32 + lane) / 3) * kInPad + (32 + lane) % 3] = __float2bfloat16_rn(nx1);
    load(t + (long long)gridDim.x * kIWarps);
    __syncwarp();
    {
      wm::fragment<wm::matrix_a, 16, 16, 16, __nv_bfloat16, wm::row_major> a;
      wm::load_matrix_sync(a, ws.xb, kInPad);
      for (int nt = 0; nt < 2; ++nt) {
        wm::fragment<wm::accumulator, 16, 16, 16, float> c;
        wm::fill_fragment(c, 0.0f);
        wm::mma_sync(c, a, B1[nt], c);
        wm::store_matrix_sync(ws.c + nt * 16, c, kH, wm::mem_row_major);
      }
    }
    __syncwarp();
    for (int q = lane; q < 16 * kH; q += 32) ws.h1b[q] = __float2bfloat16_rn(fmaxf(ws.c[q] + S.b1[q % kH], 0.0f));
    __syncwarp();
    for (int nt = 0; nt < 2; ++nt) {
      wm::fragment<wm::accumulator, 16, 16, 16, float> c;
      wm::fill_fragment(c, 0.0f);
      for (int kt = 0; kt < 2; ++kt) {
        wm::fragment<wm::matrix_a, 16, 16, 16, __nv_bfloat16, wm::row_major> a;
        wm::load_matrix_sync(a, ws.h1b + kt * 16, kH);
        wm::mma_sync(c, a, B2[nt][kt], c);
      }
      wm::store_matrix_sync(ws.c + nt * 16, c, kH, wm::mem_row_major);
    }
    __syncwarp();
    for (int q = lane; q < 16 * kH; q += 32) ws.h2b[q] = __float2bfloat16_rn(fmaxf(ws.c[q] + S.b2[q % kH], 0.0f));
    __syncwarp();
    // layer 3: two lanes per point, 16 features each
    {
      const int pt = lane >> 1, half = lane & 1;
      float o = 0.0f;
#pragma unroll
      for (int k = 0; k < 16; ++k) o += S.w3[half * 16 + k] * __bfloat162float(ws.h2b[pt * kH + half * 16 + k]);
      o += __shfl_xor_sync(0xffffffffu, o, 1);
      const long long i = p0 + pt;
      if (half == 0 && i < n) wout[i] = softplus_f(o + S.b3);
    }
    __syncwarp();
  }
}

// Resident CTAs per SM the register budget of point_weights_kernel is cut
// for (a build-time knob).
#ifndef COVOX_PW_MIN_CTAS
#define COVOX_PW_MIN_CTAS 2
#endif

// Features and network of n_frames organised scans [n_frames, H, W, 3] in one
// persistent launch: CTAs take (frame, 32 x 32 tile) items in frame-major
// order.  The GEMM operands stay in registers in fragment layout.
__global__ void __launch_bounds__(kFtThreads, COVOX_PW_MIN_CTAS) point_weights_kernel(
    const float* __restrict__ params, const float* __restrict__ pts, int n_frames, int H, int W, int sensor,
    float max_range, float* __restrict__ wout) {
  __shared__ FeatTile T;
  __shared__ float P[kP];
  for (int q = threadIdx.x; q < kP; q += blockDim.x) P[q] = params[q];
  __syncthreads();
  const WeightFrags F = build_fragments(P, threadIdx.x & 31);
  const float b3 = P[kOB3];
  const float inv_max_range = 1.0f / max_range;
  const int tiles_x = (W + kFtW - 1) / kFtW;
  const int n_tiles = tiles_x * ((H + kFtH - 1) / kFtH);
  const long long n_items = (long long)n_tiles * n_frames;
  for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int frame = (int)(item / n_tiles), tile = (int)(item % n_tiles);
    const int x0 = (tile % tiles_x) * kFtW - kHalo, y0 = (tile / tiles_x) * kFtH - kHalo;
    __syncthreads();   // the previous tile's staging is no longer read
    weights_tile(T, F, b3, pts + (size_t)frame * H * W * 3, H, W, sensor, inv_max_range, x0, y0,
                 wout + (size_t)frame * H * W);
  }
}

// Target normalisation: per-CTA partial sums of e2 * mask and mask over a
// fixed grid-stride partition, summed in CTA order by one thread (so the mean
// does not depend on scheduling), then every target divided by the mean.
constexpr int kNormCtas = 256;

// Compensated FP32 sum (Neumaier): s + c carries the exact sum to about one
// rounding of its value, so the mean needs no FP64.
struct CSum {
  float s, c;
};

__device__ __forceinline__ void csum_add(CSum& a, float x) {
  const float t = a.s + x;
  a.c += fabsf(a.s) >= fabsf(x) ? (a.s - t) + x : (x - t) + a.s;
  a.s = t;
}

__device__ __forceinline__ void csum_merge(CSum& a, const CSum& b) {
  csum_add(a, b.s);
  a.c += b.c;
}

__global__ void __launch_bounds__(256) target_sums_kernel(const float* __restrict__ e2,
                                                          const float* __restrict__ mask, long long n,
                                                          float4* __restrict__ partial) {
  __shared__ CSum se[256], sm[256];
  CSum a{0.0f, 0.0f}, c{0.0f, 0.0f};
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const float mk = mask[i];
    if (mk != 0.0f) {
      csum_add(a, e2[i] * mk);
      csum_add(c, mk);
    }
  }
  se[threadIdx.x] = a;
  sm[threadIdx.x] = c;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      csum_merge(se[threadIdx.x], se[threadIdx.x + o]);
      csum_merge(sm[threadIdx.x], sm[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = make_float4(se[0].s, se[0].c, sm[0].s, sm[0].c);
}

__global__ void target_scale_kernel(float* __restrict__ e2, long long n, const float4* __restrict__ partial,
                                    int nparts, float* __restrict__ mean_out) {
  __shared__ float inv;
  if (threadIdx.x == 0) {
    CSum a{0.0f, 0.0f}, c{0.0f, 0.0f};
    for (int p = 0; p < nparts; ++p) {
      const float4 q = partial[p];
      csum_merge(a, CSum{q.x, q.y});
      csum_merge(c, CSum{q.z, q.w});
    }
    const float cnt = c.s + c.c;
    const float mean = (a.s + a.c) / (cnt > 1.0f ? cnt : 1.0f);
    if (blockIdx.x == 0) *mean_out = mean;
    inv = mean > 0.0f ? 1.0f / mean : 1.0f;
  }
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    e2[i] *= inv;
}

// Fixed-order sum of the CTA partials, mean over valid points, Adam.
__global__ void adam_kernel(float* __restrict__ params, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ partial, int nparts, float lr, float b1, float b2,
                            float eps, int t, float* __restrict__ grad_out, float* __restrict__ loss_out) {
  __shared__ float count;
  if (threadIdx.x == 0) {
    float c = 0.0f;
    for (int p = 0; p < nparts; ++p) c += partial[(size_t)p * (kP + 2) + kP + 1];
    count = fmaxf(c, 1.0f);
  }
  __syncthreads();
  const float inv = 1.0f / count;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < kP + 1; j += gridDim.x * blockDim.x) {
    float g = 0.0f;
    for (int p = 0; p < nparts; ++p) g += partial[(size_t)p * (kP + 2) + j];
    g *= inv;
    if (j == kP) {
      if (loss_out) *loss_out = g;
      continue;
    }
    if (grad_out) grad_out[j] = g;
    if (lr > 0.0f) {
      const float mj = b1 * m[j] + (1.0f - b1) * g;
      const float vj = b2 * v[j] + (1.0f - b2) * g * g;
      m[j] = mj;
      v[j] = vj;
      const float mh = mj / (1.0f - powf(b1, (float)t));
      const float vh = vj / (1.0f - powf(b2, (float)t));
      params[j] -= lr * mh / (sqrtf(vh) + eps);
    }
  }
}

}  // namespace

struct cvx_weight_model {
  float* params;   // device [kP]
  float* m;
  float* v;
  float* partial;  // [kMaxGrid][kP + 2]
  float* grad;     // last gradient [kP]
  float* loss;     // last loss
  int t;
  int grid;
};

extern "C" {

cvx_status cvx_weight_model_create(const float* init_params, cvx_weight_model** out) {
  if (!out || !init_params) return CVX_ERR_INVALID_ARG;
  *out = nullptr;
  cvx_weight_model* w = new (std::nothrow) cvx_weight_model();
  if (!w) return CVX_ERR_OOM;
  if (cudaMalloc(&w->params, kP * 4) != cudaSuccess || cudaMalloc(&w->m, kP * 4) != cudaSuccess ||
      cudaMalloc(&w->v, kP * 4) != cudaSuccess ||
      cudaMalloc(&w->partial, (size_t)kMaxGrid * (kP + 2) * 4) != cudaSuccess ||
      cudaMalloc(&w->grad, kP * 4) != cudaSuccess || cudaMalloc(&w->loss, 4) != cudaSuccess ||
      cudaMemcpy(w->params, init_params, kP * 4, cudaMemcpyDefault) != cudaSuccess ||
      cudaMemset(w->m, 0, kP * 4) != cudaSuccess || cudaMemset(w->v, 0, kP * 4) != cudaSuccess ||
      cudaMemset(w->grad, 0, kP * 4) != cudaSuccess || cudaMemset(w->loss, 0, 4) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(w->params); cudaFree(w->m); cudaFree(w->v); cudaFree(w->partial); cudaFree(w->grad); cudaFree(w->loss);
    delete w;
    return CVX_ERR_OOM;
  }
  for (auto f : {(const void*)mlp_kernel<0>, (const void*)mlp_kernel<1>})
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpSmem));
  w->grid = std::min(kMaxGrid, num_sms() * 2);
  *out = w;
  return CVX_OK;
}

void cvx_weight_model_destroy(cvx_weight_model* w) {
  if (!w) return;
  cudaDeviceSynchronize();
  cudaFree(w->params); cudaFree(w->m); cudaFree(w->v); cudaFree(w->partial); cudaFree(w->grad); cudaFree(w->loss);
  delete w;
}

cvx_status cvx_weight_model_params(cvx_weight_model* w, const float* set, float* get, void* stream) {
  if (!w) return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (set && cudaMemcpyAsync(w->params, set, kP * 4, cudaMemcpyDefault, s) != cudaSuccess) goto fail;
  if (get && (cudaMemcpyAsync(get, w->params, kP * 4, cudaMemcpyDefault, s) != cudaSuccess ||
              cudaStreamSynchronize(s) != cudaSuccess))
    goto fail;
  return CVX_OK;
fail:
  cudaGetLastError();
  return CVX_ERR_CUDA;
}

cvx_status cvx_point_features(const float* points, int32_t height, int32_t width, int32_t sensor,
                              float max_range, float* features, void* stream) {
  if (!points || !features || height <= 0 || width <= 0 || (sensor != 0 && sensor != 1) || !(max_range > 0))
    return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int tiles = ((width + kFtW - 1) / kFtW) * ((height + kFtH - 1) / kFtH);
  COVOX_LAUNCH(kKFeatures, s,
               features_kernel<<<tiles, kFtThreads, 0, s>>>(points, height, width, sensor, max_range, features));
  return cudaGetLastError() == cudaSuccess ? CVX_OK : CVX_ERR_CUDA;
}

cvx_status cvx_weight_model_infer(cvx_weight_model* w, const float* features, int64_t n, float* weights,
                                  void* stream) {
  if (!w || n < 0 || (n > 0 && (!features || !weights))) return CVX_ERR_INVALID_ARG;
  if (n == 0) return CVX_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const long long tiles = (n + 15) / 16;
  const int grid = (int)std::min<long long>((tiles + kIWarps - 1) / kIWarps, (long long)num_sms() * 4);
  COVOX_LAUNCH(kKMlpFwd, s, mlp_infer_kernel<<<grid, 32 * kIWarps, 0, s>>>(w->params, features, n, weights));
  return cudaGetLastError() == cudaSuccess ? CVX_OK : CVX_ERR_CUDA;
}

cvx_status cvx_weight_model_point_weights_frames(cvx_weight_model* w, const float* points, int32_t n_frames,
                                                 int32_t height, int32_t width, int32_t sensor, float max_range,
                                                 float* weights, void* stream) {
  if (!w || !points || !weights || n_frames <= 0 || height <= 0 || width <= 0 || (sensor != 0 && sensor != 1) ||
      !(max_range > 0))
    return CVX_ERR_INVALID_ARG;
  if ((long long)n_frames * height * width > (1ll << 40)) return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const long long items = (long long)((width + kFtW - 1) / kFtW) * ((height + kFtH - 1) / kFtH) * n_frames;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)point_weights_kernel, kFtThreads, 0) !=
          cudaSuccess ||
      per_sm <= 0) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  const int grid = (int)std::min<long long>(items, (long long)num_sms() * per_sm);
  COVOX_LAUNCH(kKPointWeights, s,
               point_weights_kernel<<<grid, kFtThreads, 0, s>>>(w->params, points, n_frames, height, width, sensor,
                                                                  max_range, weights));
  return cudaGetLastError() == cudaSuccess ? CVX_OK : CVX_ERR_CUDA;
}

cvx_status cvx_weight_model_point_weights(cvx_weight_model* w, const float* points, int32_t height, int32_t width,
                                          int32_t sensor, float max_range, float* weights, void* stream) {
  return cvx_weight_model_point_weights_frames(w, points, 1, height, width, sensor, max_range, weights, stream);
}

cvx_status cvx_weight_model_train_step(cvx_weight_model* w, const float* features, const float* e2,
                                       const float* mask, int64_t n, float lr, void* stream) {
  if (!w || n <= 0 || !features || !e2 || !mask || !(lr >= 0)) return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const long long tiles = (n + 15) / 16;
  const int grid = (int)std::min<long long>((tiles + kWarps - 1) / kWarps, w->grid);
  COVOX_LAUNCH(kKMlpBwd, s,
               mlp_kernel<1><<<grid, kThreads, sizeof(MlpSmem), s>>>(w->params, features, e2, mask, n, nullptr,
                                                                     w->partial));
  if (lr > 0) w->t += 1;
  COVOX_LAUNCH(kKAdam, s,
               adam_kernel<<<(kP + 1 + 255) / 256, 256, 0, s>>>(w->params, w->m, w->v, w->partial, grid, lr, 0.9f,
                                                                0.999f, 1e-8f, w->t > 0 ? w->t : 1, w->grad,
                                                                w->loss));
  return cudaGetLastError() == cudaSuccess ? CVX_OK : CVX_ERR_CUDA;
}

cvx_status cvx_weight_model_last(cvx_weight_model* w, float* grad, float* loss, void* stream) {
  if (!w) return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if ((grad && cudaMemcpyAsync(grad, w->grad, kP * 4, cudaMemcpyDefault, s) != cudaSuccess) ||
      (loss && cudaMemcpyAsync(loss, w->loss, 4, cudaMemcpyDefault, s) != cudaSuccess) ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  return CVX_OK;
}

cvx_status cvx_normalise_targets(float* e2, const float* mask, int64_t n, float* mean_out, void* stream) {
  if (!e2 || !mask || !mean_out || n <= 0) return CVX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  float4* partial = nullptr;
  float* mean_dev = nullptr;
  // a small scratch of partials: stream-ordered allocation, freed on the stream
  if (cudaMallocAsync((void**)&partial, sizeof(float4) * kNormCtas + 16, s) != cudaSuccess) {
    cudaGetLastError();
    return CVX_ERR_OOM;
  }
  mean_dev = (float*)(partial + kNormCtas);
  COVOX_LAUNCH(kKTargets, s, target_sums_kernel<<<kNormCtas, 256, 0, s>>>(e2, mask, n, partial));
  const int grid = (int)std::min<long long>((n + 255) / 256, (long long)num_sms() * 8);
  COVOX_LAUNCH(kKTargets, s, target_scale_kernel<<<grid, 256, 0, s>>>(e2, n, partial, kNormCtas, mean_dev));
  float mean = 0.0f;
  const bool ok = cudaMemcpyAsync(&mean, mean_dev, sizeof(float), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
                  cudaFreeAsync(partial, s) == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return CVX_ERR_CUDA;
  }
  *mean_out = mean;
  return CVX_OK;
}

cvx_status cvx_training_targets(cvx_submap* clean, const float* points, int64_t n, const float T[12],
                                const cvx_integrate_params* ip, float* e2, float* mask, void* stream) {
  if (!clean || clean->p.storage != CVX_STORE_F32 || !e2 || !mask) return CVX_ERR_INVALID_ARG;
  ScanDev sc;
  int lb = 0;
  const cvx_status v = make_scan_dev(clean, points, n, T, nullptr, ip, &sc, &lb, nullptr, false);
  if (v != CVX_OK) return v;
  if (n == 0) return CVX_OK;
  cudaStream_t s = (cudaStream_t)stream;
  COVOX_LAUNCH(kKTargets, s,
               targets_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(clean->dev, sc, e2, mask));
  return cudaGetLastError() == cudaSuccess ? CVX_OK : CVX_ERR_CUDA;
}

}  // extern "C"
