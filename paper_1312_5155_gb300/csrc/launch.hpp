// Host-side launch interface between the C ABI and the kernel units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "job.hpp"

namespace rsgb {

constexpr size_t kMaxDynamicSmem = 227u * 1024u;

struct LaunchShape {
  int grid = 0;        // CTAs
  int threads = 0;     // (consumer warps + 1) * 32
  size_t smem = 0;     // dynamic shared memory bytes
};

// Launch tuning knobs (chosen per code by the autotuner or the defaults).
struct TuneCfg {
  int consumer_warps = 8;  // NC
  int depth = 16;          // ring slots
  int ctas_per_sm = 1;
  int groups = 0;          // 32-column groups per thread: 0 = by block size, 1, or 2 where compiled
};

// Thread-local message behind rs_last_error (set on failure, cleared on
// success by every entry point).
void set_last_error(const std::string& msg);
void clear_last_error();

// Dynamic shared memory of a launch: mbarriers, one tile header per slot,
// the slots.
inline size_t ring_smem_bytes(uint32_t depth, uint32_t slice) {
  return ((2u * depth * 8u + 127u) & ~127u) + (size_t)depth * (kHeaderBytes + slice);
}


}  // namespace rsgb
