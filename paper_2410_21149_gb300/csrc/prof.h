// prof.h -- launch accounting and optional per-kernel CUDA-event timing.
// Every kernel the library launches goes through COVOX_LAUNCH, which counts
// the launch and, while profiling is on, records an event pair around it on
// the launching stream.
#pragma once
#include <cuda_runtime.h>

namespace covox {

enum KernelKind : int {
  kKAlloc = 0,      // block activation / allocation pass
  kKAccum = 1,      // per-scan observation accumulation
  kKMerge = 2,      // per-block merge into D, W
  kKZeroPool = 3,   // reset: hash, block pool, touch epochs, unmerged sums
  kKBatched = 4,    // persistent batched integration
  kKFeatures = 5,   // per-point features of the weight model
  kKMlpFwd = 6,     // weight model forward
  kKMlpBwd = 7,     // weight model backward + reduction
  kKAdam = 8,       // weight model optimiser step
  kKTargets = 9,    // training targets
  kKPipelined = 10, // pipelined per-scan kernel (tiles + merges of the previous scan)
  kKFlush = 11,     // merge of a pipelined submap's pending scan
  kKPipeClose = 12, // pipelined per-scan bookkeeping after each scan
  kKEsdf = 13,      // distance field of a submap
  kKHash = 14,      // stand-alone block hash insert / find
  kKDiscard = 15,   // reset: the submaps' state words
  kKPointWeights = 16,   // fused features + weight network of organised scans
  kNumKinds = 17
};

void prof_begin(int kind, cudaStream_t s);
void prof_end(int kind, cudaStream_t s);

}  // namespace covox

#define COVOX_LAUNCH(kind, stream, ...)         \
  do {                                          \
    ::covox::prof_begin((kind), (stream));      \
    __VA_ARGS__;                                \
    ::covox::prof_end((kind), (stream));        \
  } while (0)
