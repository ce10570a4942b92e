// submap.h -- host-side definition of a submap handle and the scan
// validation / tiling shared by the per-scan and batched entry points.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "../../include/covox.h"
#include "covox_dev.cuh"
#include "integrate_dev.cuh"

struct cvx_submap {
  cvx_submap_params p;
  covox::SubmapDev dev;
  covox::SubmapDev dev_b;   // the second per-scan set of a pipelined submap
  covox::SubmapDev dev_cd[2];   // the third and fourth per-scan sets of a four-set submap
  int n_sets;               // per-scan sets: 1, 2 (pipelined) or 4
  bool colour;              // CVX_SUBMAP_COLOR: fused RGB planes and per-set colour sums
  bool pipelined;
  bool maybe_pending;       // a pipelined per-scan launch may have left a scan unmerged
  size_t bytes_per_vox;
  cudaStream_t last_stream;
  struct Alloc {
    void* ptr;
    size_t bytes;
  } allocs[32];
  int n_allocs;
};

namespace covox {

// The view of per-scan set k (0 .. n_sets - 1) of a submap.
inline const SubmapDev& set_view(const cvx_submap* m, int k) {
  return k == 0 ? m->dev : (k == 1 ? m->dev_b : m->dev_cd[k - 2]);
}

inline int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

// Merge the scan a pipelined submap's last per-scan launch left pending
// (discard: drop its sums instead).  No-op for other submaps.
cvx_status flush_pending(cvx_submap* map, cudaStream_t s, bool discard);

constexpr int kDefaultLocalBlocks = 8;
constexpr int kMaxLocalBlocks = 16;   // 8 KB of fixed-point sums each

// Validate one scan's arguments and fill its device descriptor (with the
// tile layout).  Returns CVX_OK or CVX_ERR_INVALID_ARG; *lb gets the number
// of shared-memory block slots per CTA.  rgb: per-point colours, required
// (n > 0) when integrating into a colour submap and refused by any other;
// colour scans accumulate in the L2 mode (*lb = 0).  integrating = false
// (a scan that is only read against the submap) lifts the requirement.
inline cvx_status make_scan_dev(const cvx_submap* map, const float* pts, int64_t n, const float* T,
                                const float* pw, const cvx_integrate_params* ip, ScanDev* sc, int* lb,
                                const float* rgb = nullptr, bool integrating = true) {
  if (!map || !ip || !T || n < 0 || (n > 0 && !pts)) return CVX_ERR_INVALID_ARG;
  if (rgb && (!map->colour || !integrating)) return CVX_ERR_INVALID_ARG;
  if (map->colour && integrating && n > 0 && !rgb) return CVX_ERR_INVALID_ARG;
  for (int q = 0; q < 12; ++q)
    if (!std::isfinite(T[q])) return CVX_ERR_INVALID_ARG;
  if (ip->weight_mode < 0 || ip->weight_mode > 2 || ip->dropoff < 0 || ip->dropoff > 2)
    return CVX_ERR_INVALID_ARG;
  if (ip->weight_mode == CVX_W_PER_POINT && n > 0 && !pw) return CVX_ERR_INVALID_ARG;
  if (ip->dropoff != CVX_DROP_NONE && !(map->p.trunc > map->p.voxel_size)) return CVX_ERR_INVALID_ARG;
  if (ip->sensor != 0 && ip->sensor != 1) return CVX_ERR_INVALID_ARG;
  if (!(ip->min_range >= 0) || !(ip->max_range >= ip->min_range)) return CVX_ERR_INVALID_ARG;
  if (ip->pts_per_cta < 0 || ip->pts_per_cta > (1 << 16)) return CVX_ERR_INVALID_ARG;
  if (ip->local_blocks < -1 || ip->local_blocks > kMaxLocalBlocks ||
      (ip->local_blocks > 0 && (ip->local_blocks & (ip->local_blocks - 1)) != 0))
    return CVX_ERR_INVALID_ARG;   // -1, 0 or a power of two
  if (ip->height < 0 || ip->width < 0) return CVX_ERR_INVALID_ARG;
  if (ip->flags & ~CVX_INTEGRATE_CARVE) return CVX_ERR_INVALID_ARG;
  if (n > (1ll << 31) - 1) return CVX_ERR_INVALID_ARG;
  std::memset(sc, 0, sizeof(*sc));
  sc->pts = pts;
  sc->pw = pw;
  sc->rgb = rgb;
  sc->n = n;
  std::memcpy(sc->T, T, sizeof(sc->T));
  sc->min_range = ip->min_range;
  sc->max_range = ip->max_range;
  sc->weight_mode = ip->weight_mode;
  sc->dropoff = ip->dropoff;
  sc->sensor = ip->sensor;
  sc->carve = (ip->flags & CVX_INTEGRATE_CARVE) ? 1 : 0;
  sc->long_band = (double)map->p.trunc / (double)map->p.voxel_size < 250.0 ? 0 : 1;
  sc->organised = (ip->height > 0 && ip->width >= 32 && (int64_t)ip->height * ip->width == n) ? 1 : 0;
  sc->height = ip->height;
  sc->width = ip->width;
  const int ppc = ip->pts_per_cta;
  if (sc->organised) {
    sc->tile_w = 32;
    int th = ppc > 0 ? ppc / 32 : 8;
    th = th < 8 ? 8 : (th / 8) * 8;
    sc->tile_h = th;
    sc->tiles_x = (ip->width + 31) / 32;
    sc->n_tiles = sc->tiles_x * ((ip->height + th - 1) / th);
  } else {
    int run = ppc > 0 ? ppc : 256;
    run = run < 256 ? 256 : (run / 256) * 256;
    sc->tile_w = run;
    sc->tile_h = 1;
    sc->tiles_x = 1;
    sc->n_tiles = (int)((n + run - 1) / run);
  }
  *lb = ip->local_blocks > 0 ? ip->local_blocks : (ip->local_blocks < 0 ? 0 : kDefaultLocalBlocks);
  if (rgb) *lb = 0;
  return CVX_OK;
}

// A scan the compile-time variants do not cover: carving, bands longer than
// 512 cells per axis, colours (the run-time dispatching kernel runs it).
inline int general_form(const ScanDev& sc) { return sc.carve || sc.long_band || sc.rgb != nullptr; }

}  // namespace covox
