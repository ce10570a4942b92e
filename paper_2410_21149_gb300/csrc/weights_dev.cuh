// weights_dev.cuh -- device code of the learned per-point weight shared by
// the stand-alone weight kernel and the weight items of the batched launch:
// the features of an organised scan (range, incidence angle, 5x5 depth
// variance) and the 3-32-32-1 network on mma.sync BF16 fragments.
//
// coVoxSLAM Sec. III-C (weighting paragraph): the weight should follow the
// sensor's error curve, and ray casting lets every point carry its own
// weight; the network predicts that weight from the point's features.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/covox.h"

namespace covox {
namespace wnet {

constexpr int kH = 32;                // hidden width
constexpr int kIn = 3;                // features
constexpr int kP = CVX_MLP_PARAMS;    // 1217
// offsets of the flat parameter vector: W1 [32,3], b1, W2 [32,32], b2, W3, b3
constexpr int kOW1 = 0, kOB1 = 96, kOW2 = 128, kOB2 = 1152, kOW3 = 1184, kOB3 = 1216;
static_assert(kOB3 + 1 == kP, "parameter layout");

__device__ __forceinline__ float softplus_f(float o) { return o > 20.0f ? o : log1pf(expf(o)); }

// softplus from the fast exp and log: ln(1 + x), x = e^o, by the series
// x - x^2/2 + x^3/3 for x < e^-5 (truncation below 1e-7 relative), else by
// __logf of 1 + x (result >= 6.7e-3, so __logf's ~1e-7 absolute error stays
// below 2e-5 relative); __expf's relative error is ~2e-6 at |o| = 20.
__device__ __forceinline__ float softplus_fast(float o) {
  if (o > 20.0f) return o;
  const float x = __expf(o);
  return o < -5.0f ? x * fmaf(x, fmaf(x, 1.0f / 3.0f, -0.5f), 1.0f) : __logf(1.0f + x);
}
__device__ __forceinline__ float sigmoid_f(float o) { return 1.0f / (1.0f + expf(-o)); }

// ------------------------------------------------------------- features
__device__ __forceinline__ bool pt_valid(const float* P, int sensor) {
  return isfinite(P[0]) && isfinite(P[1]) && isfinite(P[2]) && (sensor != 0 || P[2] > 0.0f);
}

// One CTA per 32 x 32 pixel tile, eight warps of four pixel rows each (warp
// w takes rows 4w .. 4w + 3, lane = column); the tile and its 2-pixel halo
// (36 x 36 points) are staged in shared memory once: each point's
// coordinates, and its depth (z for a pinhole, range for a spherical sensor)
// beside a validity weight of 1 or 0.
constexpr int kFtW = 32, kFtH = 32, kHalo = 2, kFtRows = 4;
constexpr int kFsW = kFtW + 2 * kHalo, kFsH = kFtH + 2 * kHalo;
constexpr int kFtThreads = kFtW * kFtH / kFtRows;   // 256
constexpr int kStageIters = (kFsW * kFsH + kFtThreads - 1) / kFtThreads;

struct FeatTile {
  float sp[kFsH][kFsW][3];
  float2 zm[kFsH][kFsW];   // (depth, 1) for a valid point, (0, 0) otherwise
};

__device__ __forceinline__ void stage_tile(FeatTile& T, const float* __restrict__ pts, int H, int W, int sensor,
                                           int x0, int y0) {
  // all loads of the thread first (independent), then the stores
  float P[kStageIters][3];
#pragma unroll
  for (int j = 0; j < kStageIters; ++j) {
    const int q = threadIdx.x + j * kFtThreads;
    const int ly = q / kFsW, lx = q - ly * kFsW, gx = x0 + lx, gy = y0 + ly;
    P[j][0] = P[j][1] = P[j][2] = NAN;
    if (q < kFsW * kFsH && gx >= 0 && gx < W && gy >= 0 && gy < H) {
      const float* src = pts + 3 * ((size_t)gy * W + gx);
      P[j][0] = __ldg(src);
      P[j][1] = __ldg(src + 1);
      P[j][2] = __ldg(src + 2);
    }
  }
#pragma unroll
  for (int j = 0; j < kStageIters; ++j) {
    const int q = threadIdx.x + j * kFtThreads;
    if (q >= kFsW * kFsH) break;
    const int ly = q / kFsW, lx = q - ly * kFsW;
    const bool ok = pt_valid(P[j], sensor);
    T.sp[ly][lx][0] = P[j][0];
    T.sp[ly][lx][1] = P[j][1];
    T.sp[ly][lx][2] = P[j][2];
    const float z = sensor == 0 ? P[j][2] : sqrtf(P[j][0] * P[j][0] + P[j][1] * P[j][1] + P[j][2] * P[j][2]);
    T.zm[ly][lx] = ok ? make_float2(z, 1.0f) : make_float2(0.0f, 0.0f);
  }
}

// Third feature of the thread's four points (rows 4 ty + k of the tile,
// column tx): ln(var + 1e-8) / 10 of the depths in the point's 5 x 5 window.
// The variance of each window is taken about the point's own depth zc: with
// s1 = sum (z - zc) and s2 = sum (z - zc)^2 over the window's valid points,
// var = (s2 - s1^2 / n) / n -- the variance of the definition, whose
// cancellation is bounded (zc is one of the window's points) -- and the
// thread's four windows share their loads.
__device__ __forceinline__ void tile_variance_features(const FeatTile& T, int tx, int ty, float f2[kFtRows]) {
  float zc[kFtRows], s1[kFtRows], s2[kFtRows], cnt[kFtRows];
#pragma unroll
  for (int k = 0; k < kFtRows; ++k) {
    zc[k] = T.zm[kFtRows * ty + k + kHalo][tx + kHalo].x;
    s1[k] = s2[k] = cnt[k] = 0.0f;
  }
#pragma unroll
  for (int dx = 0; dx < 2 * kHalo + 1; ++dx) {
    float2 c[kFtRows + 2 * kHalo];
#pragma unroll
    for (int r = 0; r < kFtRows + 2 * kHalo; ++r) c[r] = T.zm[kFtRows * ty + r][tx + dx];
#pragma unroll
    for (int k = 0; k < kFtRows; ++k)
#pragma unroll
      for (int r = k; r <= k + 2 * kHalo; ++r) {
        const float d = c[r].x - zc[k];
        const float dm = d * c[r].y;   // 0 for an invalid point
        s1[k] += dm;
        s2[k] = fmaf(dm, d, s2[k]);
        cnt[k] += c[r].y;
      }
  }
#pragma unroll
  for (int k = 0; k < kFtRows; ++k) {
    float var = 0.0f;
    if (cnt[k] >= 3.0f) {
      const float ic = __fdividef(1.0f, cnt[k]);
      var = fmaxf((s2[k] - s1[k] * s1[k] * ic) * ic, 0.0f);
    }
    f2[k] = __logf(var + 1e-8f) * 0.1f;   // absolute error ~1e-7 over the feature's range
  }
}

// Features of the point in row 4 ty + k, column tx of the tile (image pixel
// (x0 + 2 + tx, y0 + 2 + 4 ty + k)), its third feature given: r / max_range,
// the incidence angle / (pi / 2), and f2; all zero for an invalid point.
__device__ __forceinline__ void point_features(const FeatTile& T, int tx, int ty, int k, int x0, int y0, int H, int W,
                                               float inv_max_range, float f2, float f[3]) {
  const int cx = tx + kHalo, cy = kFtRows * ty + k + kHalo;
  const int u = x0 + cx, v = y0 + cy;
  f[0] = f[1] = f[2] = 0.0f;
  if (T.zm[cy][cx].y == 0.0f) return;
  const float* P = T.sp[cy][cx];
  const float r = sqrtf(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
  f[0] = r * inv_max_range;
  float th = 0.0f;
  if (u > 0 && u < W - 1 && v > 0 && v < H - 1 && T.zm[cy][cx - 1].y != 0.0f && T.zm[cy][cx + 1].y != 0.0f &&
      T.zm[cy - 1][cx].y != 0.0f && T.zm[cy + 1][cx].y != 0.0f) {
    const float* L = T.sp[cy][cx - 1];
    const float* R = T.sp[cy][cx + 1];
    const float* U = T.sp[cy - 1][cx];
    const float* Dn = T.sp[cy + 1][cx];
    const float a0 = R[0] - L[0], a1 = R[1] - L[1], a2 = R[2] - L[2];
    const float b0 = Dn[0] - U[0], b1 = Dn[1] - U[1], b2 = Dn[2] - U[2];
    const float n0 = a1 * b2 - a2 * b1, n1 = a2 * b0 - a0 * b2, n2 = a0 * b1 - a1 * b0;
    const float nn2 = n0 * n0 + n1 * n1 + n2 * n2;
    // cos = |n.P| / (|n| r); rsqrtf's relative error (a few 1e-7) moves the
    // angle by well under 1e-3 even where acos is steep
    if (nn2 > 0.0f) th = acosf(fminf(fabsf(n0 * P[0] + n1 * P[1] + n2 * P[2]) * rsqrtf(nn2) / r, 1.0f));
  }
  f[1] = th * 0.636619772367581343f;   // / (pi / 2)
  f[2] = f2;
}

// ------------------------------------------------ fused features + network
// Per-point weights of organised scans in one pass: each CTA stages a 32 x 32
// pixel tile (and halo) in shared memory, every thread computes the features
// of its four points (one per pixel row it owns), and each warp runs the
// network on one row of 32 points at a time (two 16-point row blocks) with
// mma.sync m16n8k16 BF16 fragments that stay in registers from layer to
// layer: the FP32 accumulator layout of a 16 x 8 output tile, two tiles side
// by side, is the A-operand layout of the next layer's 16-wide K slice.  Each
// accumulator starts at its layer's bias, and one cvt.rn.relu.bf16x2 applies
// ReLU and the BF16 rounding to two activations at once.  The output layer
// (32 -> 1) is a third GEMM whose two B columns hold W3 as a pair of BF16
// values, hi = bf16(W3) and lo = bf16(W3 - hi) (16 significant bits; the
// products are exact and accumulate in FP32), so o = b3 + hi.h + lo.h.
// Roundings: BF16 operands of every GEMM, FP32 accumulation, biases in FP32.
__device__ __forceinline__ void mma_bf16_16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// d = a b + c with the accumulator input c apart from the output d (a bias
// broadcast to both rows needs no copies).
__device__ __forceinline__ void mma_bf16_16816_c(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1, float c0,
                                                 float c1, float c2, float c3) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%10,%11,%12,%13};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c0), "f"(c1), "f"(c2), "f"(c3));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// (bf16(max(lo, 0)), bf16(max(hi, 0))) packed low / high, round to nearest even.
__device__ __forceinline__ uint32_t pack_relu_bf16(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// One lane's GEMM operands in mma.sync fragment layout (B[k][n] = W[n][k],
// col-major K x N): layer 1 B fragments of the four n-tiles; layer 2 B
// fragments of n-tile nt ((kt 0: b0, b1), (kt 1: b0, b1)); layer 3 B
// fragments ((kt 0: b0, b1), (kt 1: b0, b1)); and the biases of the lane's
// two accumulator columns of each n-tile, b1 and b2 (n-tiles 0-1, 2-3).
struct WeightFrags {
  uint4 w1, w3;
  uint4 w2[4];
  float4 c1[2], c2[2];
  __device__ __forceinline__ uint4 W1() const { return w1; }
  __device__ __forceinline__ uint4 W2(int nt) const { return w2[nt]; }
  __device__ __forceinline__ uint4 W3() const { return w3; }
  __device__ __forceinline__ float4 C1(int h) const { return c1[h]; }
  __device__ __forceinline__ float4 C2(int h) const { return c2[h]; }
};

// Every lane's operands in shared memory, one array per operand (each
// warp's 16-byte loads of them are conflict free).
struct alignas(16) WeightFragSmem {
  uint4 w1[32], w3[32];
  uint4 w2[4][32];
  float4 c1[2][32], c2[2][32];
  float b3;
};

struct WeightFragView {
  const WeightFragSmem* s;
  int lane;
  __device__ __forceinline__ uint4 W1() const { return s->w1[lane]; }
  __device__ __forceinline__ uint4 W2(int nt) const { return s->w2[nt][lane]; }
  __device__ __forceinline__ uint4 W3() const { return s->w3[lane]; }
  __device__ __forceinline__ float4 C1(int h) const { return s->c1[h][lane]; }
  __device__ __forceinline__ float4 C2(int h) const { return s->c2[h][lane]; }
};

// One lane's operands from the flat parameter vector P (device or shared
// memory).  The output layer's B columns: 0 holds bf16(W3), 1 the BF16
// remainder bf16(W3 - bf16(W3)); the other columns are zero.
__device__ __forceinline__ WeightFrags build_fragments(const float* P, int lane) {
  const int g = lane >> 2, tig = lane & 3;
  uint32_t b1[4], b2[4][4], b3[4];
  float c1[8], c2[8];
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int n = nt * 8 + g;
    const int k0 = tig * 2;
    b1[nt] = pack_bf16(k0 < kIn ? P[kOW1 + n * kIn + k0] : 0.0f, k0 + 1 < kIn ? P[kOW1 + n * kIn + k0 + 1] : 0.0f);
#pragma unroll
    for (int kt = 0; kt < 2; ++kt) {
      const int k = kt * 16 + tig * 2;
      b2[nt][2 * kt] = pack_bf16(P[kOW2 + n * kH + k], P[kOW2 + n * kH + k + 1]);
      b2[nt][2 * kt + 1] = pack_bf16(P[kOW2 + n * kH + k + 8], P[kOW2 + n * kH + k + 9]);
    }
    c1[2 * nt] = P[kOB1 + nt * 8 + tig * 2];
    c1[2 * nt + 1] = P[kOB1 + nt * 8 + tig * 2 + 1];
    c2[2 * nt] = P[kOB2 + nt * 8 + tig * 2];
    c2[2 * nt + 1] = P[kOB2 + nt * 8 + tig * 2 + 1];
  }
#pragma unroll
  for (int kt = 0; kt < 2; ++kt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float v[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const float w3 = P[kOW3 + kt * 16 + h * 8 + tig * 2 + j];
        const float hi = __bfloat162float(__float2bfloat16_rn(w3));
        v[j] = g == 0 ? hi : (g == 1 ? w3 - hi : 0.0f);
      }
      b3[2 * kt + h] = pack_bf16(v[0], v[1]);
    }
  WeightFrags F;
  F.w1 = make_uint4(b1[0], b1[1], b1[2], b1[3]);
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) F.w2[nt] = make_uint4(b2[nt][0], b2[nt][1], b2[nt][2], b2[nt][3]);
  F.w3 = make_uint4(b3[0], b3[1], b3[2], b3[3]);
  F.c1[0] = make_float4(c1[0], c1[1], c1[2], c1[3]);
  F.c1[1] = make_float4(c1[4], c1[5], c1[6], c1[7]);
  F.c2[0] = make_float4(c2[0], c2[1], c2[2], c2[3]);
  F.c2[1] = make_float4(c2[4], c2[5], c2[6], c2[7]);
  return F;
}

// Warp 0 of a CTA writes every lane's operands (and b3) into S.
__device__ __forceinline__ void store_fragments(const float* P, WeightFragSmem& S, int lane) {
  const WeightFrags F = build_fragments(P, lane);
  S.w1[lane] = F.w1;
  S.w3[lane] = F.w3;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) S.w2[nt][lane] = F.w2[nt];
  S.c1[0][lane] = F.c1[0];
  S.c1[1][lane] = F.c1[1];
  S.c2[0][lane] = F.c2[0];
  S.c2[1][lane] = F.c2[1];
  if (lane == 0) S.b3 = P[kOB3];
}

// Network output o (before the softplus) of 16 points, rows g and g + 8 of a
// row block: layer-1 A fragments A0 (row g) and A1 (row g + 8) hold the
// features (K padded to 16).  Lanes with tig == 0 receive o of rows g (og)
// and g + 8 (og8).  Frag: WeightFrags (registers) or WeightFragView.
template <class Frag>
__device__ __forceinline__ void network_rows(const Frag& F, int lane, uint32_t A0, uint32_t A1, float b3,
                                             float& og, float& og8) {
  const int tig = lane & 3;
  const uint32_t A[4] = {A0, A1, 0u, 0u};
  // layer 1: C = b1 + x W1^T
  float C[4][4];
  {
    const uint4 w1 = F.W1();
    const float4 p0 = F.C1(0), p1 = F.C1(1);
    const uint32_t b[4] = {w1.x, w1.y, w1.z, w1.w};
    const float c[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
      mma_bf16_16816_c(C[nt], A, b[nt], 0u, c[2 * nt], c[2 * nt + 1], c[2 * nt], c[2 * nt + 1]);
  }
  // h1 = bf16(relu(C)) in the A layout of layer 2: {row g, k..k+1},
  // {row g+8, k..}, {row g, k+8..}, {row g+8, k+8..} of each K slice
  uint32_t A2[2][4];
#pragma unroll
  for (int kt = 0; kt < 2; ++kt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      A2[kt][2 * h] = pack_relu_bf16(C[2 * kt + h][0], C[2 * kt + h][1]);
      A2[kt][2 * h + 1] = pack_relu_bf16(C[2 * kt + h][2], C[2 * kt + h][3]);
    }
  // layer 2: D = b2 + h1 W2^T
  float D[4][4];
  {
    const float4 p0 = F.C2(0), p1 = F.C2(1);
    const float c[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const uint4 w2 = F.W2(nt);
      mma_bf16_16816_c(D[nt], A2[0], w2.x, w2.y, c[2 * nt], c[2 * nt + 1], c[2 * nt], c[2 * nt + 1]);
      mma_bf16_16816(D[nt], A2[1], w2.z, w2.w);
    }
  }
  uint32_t A3[2][4];
#pragma unroll
  for (int kt = 0; kt < 2; ++kt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      A3[kt][2 * h] = pack_relu_bf16(D[2 * kt + h][0], D[2 * kt + h][1]);
      A3[kt][2 * h + 1] = pack_relu_bf16(D[2 * kt + h][2], D[2 * kt + h][3]);
    }
  // layer 3: E[., 0] = b3 + bf16(W3) h2, E[., 1] = remainder(W3) h2
  const uint4 w3 = F.W3();
  const float e0 = tig == 0 ? b3 : 0.0f;
  float E[4];
  mma_bf16_16816_c(E, A3[0], w3.x, w3.y, e0, 0.0f, e0, 0.0f);
  mma_bf16_16816(E, A3[1], w3.z, w3.w);
  og = E[0] + E[1];
  og8 = E[2] + E[3];
}

// Per-point weights of one 32 x 32 tile of an organised scan (pts: the
// scan's [H*W,3] points; x0, y0: the tile's origin minus the halo) by the
// CTA's 256 threads, written to fw ([H*W]).  Stages the tile into T and
// synchronises the CTA once; T must be free on entry (the caller
// synchronises between uses).  Each warp runs the network on one pixel row
// of 32 points at a time (two 16-point row blocks).
template <class Frag>
__device__ __forceinline__ void weights_tile(FeatTile& T, const Frag& F, float b3, const float* __restrict__ pts,
                                             int H, int W, int sensor, float inv_max_range, int x0, int y0,
                                             float* __restrict__ fw) {
  const int lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
  const int tx = lane, ty = threadIdx.x >> 5;
  stage_tile(T, pts, H, W, sensor, x0, y0);
  __syncthreads();
  float f2[kFtRows];
  tile_variance_features(T, tx, ty, f2);
#pragma unroll 1
  for (int k = 0; k < kFtRows; ++k) {
    float f[3];
    point_features(T, tx, ty, k, x0, y0, H, W, inv_max_range, f2[k], f);
    // network of this warp's row k: points (columns) 16 mt + g and 16 mt + g + 8
    float og[2], og8[2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int pa = mt * 16 + g, pb = pa + 8;
      const float fa0 = __shfl_sync(0xffffffffu, f[0], pa), fa1 = __shfl_sync(0xffffffffu, f[1], pa);
      const float fa2 = __shfl_sync(0xffffffffu, f[2], pa);
      const float fb0 = __shfl_sync(0xffffffffu, f[0], pb), fb1 = __shfl_sync(0xffffffffu, f[1], pb);
      const float fb2 = __shfl_sync(0xffffffffu, f[2], pb);
      const uint32_t A0 = tig == 0 ? pack_bf16(fa0, fa1) : (tig == 1 ? pack_bf16(fa2, 0.0f) : 0u);
      const uint32_t A1 = tig == 0 ? pack_bf16(fb0, fb1) : (tig == 1 ? pack_bf16(fb2, 0.0f) : 0u);
      network_rows(F, lane, A0, A1, b3, og[mt], og8[mt]);
    }
    // lane L takes the output of its own point (column L): row L & 15 of row
    // block L >> 4, held by lane 4 (L & 7)
    const int src = (lane & 7) * 4;
    const float v00 = __shfl_sync(0xffffffffu, og[0], src), v01 = __shfl_sync(0xffffffffu, og8[0], src);
    const float v10 = __shfl_sync(0xffffffffu, og[1], src), v11 = __shfl_sync(0xffffffffu, og8[1], src);
    const bool lo8 = (lane & 8) == 0;
    const float o = lane < 16 ? (lo8 ? v00 : v01) : (lo8 ? v10 : v11);
    const int u = x0 + kHalo + tx, v = y0 + kHalo + kFtRows * ty + k;
    if (u < W && v < H) fw[(size_t)v * W + u] = softplus_fast(o);
  }
}

}  // namespace wnet
}  // namespace covox
