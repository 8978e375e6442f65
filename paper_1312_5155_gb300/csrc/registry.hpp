// Registry of compiled kernel instantiations, keyed by what they compute.
// The table itself is generated by the build (one translation unit per
// instantiation, plus registry.cu listing them).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "job.hpp"
#include "launch.hpp"

namespace rsgb {

enum KernelFamily : int {
  kFamPoly = 0,        // PolyBody<W, M, OP>
  kFamMatRuntime = 1,  // MatRuntimeBody<W, M, OP, LAYOUT>
  kFamMatFixed = 2,    // MatFixedBody<W, K, M, KIND, OP>
  kFamPolyMixed = 3,   // MixedBody of PolyBody<W, M, enc/dec> for M in mset
};

struct KernelKey {
  int family = 0;
  int w = 0;
  int m = 0;       // M of the body (0 for mixed kernels)
  int op = 0;      // kOp* (-1 for mixed: both encode and decode)
  int layout = 0;
  int kind = 0;    // kKindVandermonde / kKindCauchy for kFamMatFixed
  int k = 0;       // data blocks for kFamMatFixed
  uint32_t mset = 0;  // kFamPolyMixed: bit M set for every M covered
  int wide = 0;       // 1: the two-column-group variant of the same kernel
};

using Launcher = cudaError_t (*)(const JobParams&, const LaunchShape&, cudaStream_t);

struct KernelEntry {
  KernelKey key;
  Launcher launch;
  int max_warps;
  int groups;  // 32-column groups per consumer lane (tile slice = warps * groups * segment)
  int producer_warps;  // 1, or 4: a producer warpgroup (consumer count a multiple of 4)
  const char* name;
};

extern const KernelEntry* const kKernelRegistryPtr;
extern const int kKernelRegistrySize;

inline bool same_key(const KernelKey& a, const KernelKey& b) {
  return a.family == b.family && a.w == b.w && a.m == b.m && a.op == b.op && a.layout == b.layout &&
         a.kind == b.kind && a.k == b.k && a.mset == b.mset && a.wide == b.wide;
}

inline const KernelEntry* find_kernel(const KernelKey& k) {
  for (int i = 0; i < kKernelRegistrySize; ++i)
    if (same_key(kKernelRegistryPtr[i].key, k)) return &kKernelRegistryPtr[i];
  return nullptr;
}

}  // namespace rsgb
