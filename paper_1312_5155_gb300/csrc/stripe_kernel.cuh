// Persistent, TMA-staged stripe kernel (sm_103a).
//
// CTA = NC consumer warps + 1 producer warp.  The producer's lane 0 walks the
// CTA's tiles (global tile t = blockIdx.x + i * gridDim.x) and, for every
// input block of the tile's stripe, issues one 1-D bulk copy of the tile's
// slice of that block into the next ring slot (full barrier counts the
// bytes).  Consumer warps walk the same tile sequence; each thread owns 32
// symbol columns of its warp's segment of the slice, loads them from the
// slot (16-byte LDS per chunk), runs the codec on bit-planes in registers
// and stores the output chunks straight to global memory.  Slots are
// released through the empty barriers (every consumer thread arrives).
//
// Symbol layout: warp segment = 32 lanes x 32 symbols; lane l owns the
// 16-byte chunks at l*16 + c*512 (c < W/4) of the segment, so each warp-wide
// load or store instruction covers 512 contiguous bytes.
#pragma once
#include <cuda_runtime.h>

#include <mutex>

#include "codec_poly.hpp"
#include "job.hpp"
#include "launch.hpp"
#include "pipeline.cuh"

namespace rsgb {

// Thread cap per instantiation: small register footprints get up to 16
// consumer warps, large ones (decode, or big M*W) up to 8.
RS_CHD constexpr int max_consumer_warps(int w, int m, int op) {
  return (op == kOpEncode && m * w <= 64) ? 16 : 8;
}
RS_CHD constexpr int max_threads(int w, int m, int op) { return (max_consumer_warps(w, m, op) + 1) * 32; }

struct Ring {
  uint64_t* full;
  uint64_t* empty;
  uint8_t* slots;
  uint32_t depth;
  uint32_t slice;
  uint32_t s = 0;    // next slot
  uint32_t par = 0;  // parity of the next slot's current round
  __device__ __forceinline__ void advance() {
    if (++s == depth) {
      s = 0;
      par ^= 1u;
    }
  }
};

__device__ __forceinline__ uint32_t find_stripe(const StripeDesc* st, uint32_t n, uint32_t tile) {
  uint32_t lo = 0, hi = n;  // last stripe with tile_begin <= tile
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (st[mid].tile_begin <= tile) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Consumer-side view of one tile in the symbol layout.
template <int W>
struct SymTile {
  Ring* ring;
  const uint64_t* ptrs;  // stripe pointers: inputs then outputs
  int n_in;
  uint64_t goff;   // byte offset of the tile within each block
  uint32_t len;    // valid bytes of this tile (<= slice)
  uint32_t seg;    // this warp's segment offset
  uint32_t lane;
  int* status;
  bool failed;

  __device__ __forceinline__ void load(int i, uint32_t* x) {
    Ring& r = *ring;
    const uint32_t s = r.s, par = r.par;
    r.advance();
    if (!failed && !mbar_wait(&r.full[s], par)) {
      failed = true;
      record_status(status, kDevErrTimeoutFull);
    }
    const uint8_t* slot = r.slots + (size_t)s * r.slice;
    const uint32_t len16 = len & ~15u;
#pragma unroll
    for (int c = 0; c < W / 4; ++c) {
      const uint32_t co = seg + (uint32_t)c * 512u + lane * 16u;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (!failed) {
        if (co + 16u <= len16) {
          v = *reinterpret_cast<const uint4*>(slot + co);
        } else if (co < len) {
          // ragged end of the block (< 16 bytes): read it from global memory
          const uint8_t* g = reinterpret_cast<const uint8_t*>(ptrs[i]) + goff + co;
          uint8_t b[16];
#pragma unroll
          for (int t = 0; t < 16; ++t) b[t] = (co + (uint32_t)t < len) ? g[t] : 0;
          v.x = b[0] | (b[1] << 8) | (b[2] << 16) | ((uint32_t)b[3] << 24);
          v.y = b[4] | (b[5] << 8) | (b[6] << 16) | ((uint32_t)b[7] << 24);
          v.z = b[8] | (b[9] << 8) | (b[10] << 16) | ((uint32_t)b[11] << 24);
          v.w = b[12] | (b[13] << 8) | (b[14] << 16) | ((uint32_t)b[15] << 24);
        }
      }
      x[4 * c + 0] = v.x;
      x[4 * c + 1] = v.y;
      x[4 * c + 2] = v.z;
      x[4 * c + 3] = v.w;
    }
    mbar_arrive(&r.empty[s]);
  }

  __device__ __forceinline__ void store(int t, const uint32_t* x) {
    if (failed) return;
    uint8_t* out = reinterpret_cast<uint8_t*>(ptrs[n_in + t]) + goff;
#pragma unroll
    for (int c = 0; c < W / 4; ++c) {
      const uint32_t co = seg + (uint32_t)c * 512u + lane * 16u;
      const uint4 v = make_uint4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
      if (co + 16u <= len) {
        *reinterpret_cast<uint4*>(out + co) = v;
      } else if (co < len) {
        const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
        for (uint32_t t2 = 0; co + t2 < len; ++t2) out[co + t2] = (uint8_t)(wv[t2 >> 2] >> (8 * (t2 & 3)));
      }
    }
  }
};

// Runtime matrix W[t][j] as masks, layout [t][j][c] with dims M x M x W.
template <int W, int M>
struct CoefMasks {
  const uint32_t* base;
  __device__ __forceinline__ uint32_t mask(int t, int j, int c) const {
    return base[(t * M + j) * W + c];
  }
};

__device__ __forceinline__ void producer_loop(const JobParams& p, const StripeDesc* stripes,
                                              const uint64_t* ptrs, Ring& ring) {
  uint32_t q = 0;
  bool ok = true;
  for (uint32_t tile = blockIdx.x; tile < p.total_tiles && ok; tile += gridDim.x) {
    const StripeDesc& d = stripes[find_stripe(stripes, p.n_stripes, tile)];
    const uint64_t goff = (uint64_t)(tile - d.tile_begin) * ring.slice;
    const uint64_t rem = d.bytes - goff;
    const uint32_t len = rem < ring.slice ? (uint32_t)rem : ring.slice;
    const uint32_t len16 = len & ~15u;
    const uint64_t* ip = ptrs + d.ptr_off;
    for (int i = 0; i < d.n_in; ++i) {
      const uint32_t s = ring.s, par = ring.par;
      if (q >= ring.depth && !mbar_wait(&ring.empty[s], par ^ 1u)) {
        record_status(p.status, kDevErrTimeoutEmpty);
        ok = false;
        break;
      }
      uint8_t* dst = ring.slots + (size_t)s * ring.slice;
      if (len16) {
        mbar_arrive_expect_tx(&ring.full[s], len16);
        tma_load_1d(dst, reinterpret_cast<const uint8_t*>(ip[i]) + goff, len16, &ring.full[s]);
      } else {
        mbar_arrive(&ring.full[s]);
      }
      ring.advance();
      ++q;
    }
  }
  // Drain: the CTA must not retire with bulk copies still writing its shared
  // memory, so wait for the last fills to land (they complete on their own).
  const uint32_t first = q > ring.depth ? q - ring.depth : 0;
  for (uint32_t f = first; f < q; ++f) {
    if (!mbar_wait(&ring.full[f % ring.depth], (f / ring.depth) & 1u)) {
      record_status(p.status, kDevErrTimeoutDrain);
      break;
    }
  }
}

template <int W, int M, int OP>
__global__ void __launch_bounds__(max_threads(W, M, OP), 1) rs_poly_kernel(const __grid_constant__ JobParams p) {
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t depth = p.depth;
  Ring ring;
  ring.full = reinterpret_cast<uint64_t*>(smem);
  ring.empty = ring.full + depth;
  ring.slots = smem + ((2u * depth * 8u + 127u) & ~127u);
  ring.depth = depth;
  ring.slice = p.slice_bytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nc = (int)(blockDim.x >> 5) - 1;
  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < depth; ++s) {
      mbar_init(&ring.full[s], 1);
      mbar_init(&ring.empty[s], (uint32_t)nc * 32u);
    }
    fence_barrier_init();
  }
  __syncthreads();
  const StripeDesc* stripes = p.stripes ? p.stripes : &p.inl_stripe;
  const uint64_t* ptrs = p.ptrs ? p.ptrs : p.inl_ptrs;
  const uint32_t* coef = p.coef ? p.coef : p.inl_coef;

  if (warp == nc) {
    if (lane == 0) producer_loop(p, stripes, ptrs, ring);
    return;
  }

  SymTile<W> tile;
  tile.ring = &ring;
  tile.lane = (uint32_t)lane;
  tile.seg = (uint32_t)warp * segment_bytes(W);
  tile.status = p.status;
  tile.failed = false;
  for (uint32_t t = blockIdx.x; t < p.total_tiles; t += gridDim.x) {
    const StripeDesc& d = stripes[find_stripe(stripes, p.n_stripes, t)];
    tile.goff = (uint64_t)(t - d.tile_begin) * ring.slice;
    const uint64_t rem = d.bytes - tile.goff;
    tile.len = rem < ring.slice ? (uint32_t)rem : ring.slice;
    tile.ptrs = ptrs + d.ptr_off;
    tile.n_in = d.n_in;
    if constexpr (OP == kOpEncode) {
      PolyEncode<W, M>::run((int)d.k, tile, tile);
    } else {
      CoefMasks<W, M> cm{coef + d.coef_off};
      PolyDecode<W, M>::run((int)d.n_pos, d.read_mask, (int)d.e, tile, tile, cm);
    }
    if (tile.failed) break;
  }
}

// Launch one instantiation (sets the shared-memory attribute once per device).
template <int W, int M, int OP>
cudaError_t launch_poly_instance(const JobParams& p, const LaunchShape& sh, cudaStream_t st) {
  constexpr int kMaxDevices = 64;
  static std::once_flag once[kMaxDevices];
  static cudaError_t attr_err[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (sh.threads > max_threads(W, M, OP)) return cudaErrorInvalidConfiguration;
  std::call_once(once[dev], [&] {
    attr_err[dev] = cudaFuncSetAttribute(rs_poly_kernel<W, M, OP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxDynamicSmem);
  });
  if (attr_err[dev] != cudaSuccess) return attr_err[dev];
  rs_poly_kernel<W, M, OP><<<sh.grid, sh.threads, sh.smem, st>>>(p);
  return cudaGetLastError();
}

#define RSGB_POLY_LAUNCHER_NAME(W, M, OP) launch_poly_w##W##_m##M##_op##OP
#define RSGB_DEFINE_POLY_LAUNCHER(W, M, OP)                                                        \
  cudaError_t RSGB_POLY_LAUNCHER_NAME(W, M, OP)(const JobParams& p, const LaunchShape& sh,         \
                                                cudaStream_t st) {                                 \
    return launch_poly_instance<W, M, OP>(p, sh, st);                                              \
  }

}  // namespace rsgb
