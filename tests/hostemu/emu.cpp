// Test harness: runs the library's codec templates (codec_poly.hpp,
// bitslice.hpp) and host planner (plan.cpp) on the CPU, with the same
// 32-symbol chunk layout as the GPU kernels (warp segment of 32 lanes, lane l
// owning the 16-byte chunks at l*16 + c*512).  It checks the bit-sliced
// arithmetic and the decode plans against the oracle without a GPU.  It is
// not a CPU fallback: nothing in the library calls it.
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "codec_poly.hpp"
#include "job.hpp"
#include "plan.hpp"

using namespace rsgb;

namespace {

template <int W>
struct HostTile {
  const uint8_t* const* in;  // inputs in consumption order
  uint8_t* const* out;
  size_t B;
  size_t seg;   // segment offset within the block
  int lane;
  void load(int i, uint32_t* x) {
    for (int c = 0; c < W / 4; ++c) {
      const size_t co = seg + (size_t)c * 512 + (size_t)lane * 16;
      uint8_t b[16] = {0};
      for (int t = 0; t < 16; ++t)
        if (co + t < B) b[t] = in[i][co + t];
      for (int q = 0; q < 4; ++q)
        x[4 * c + q] = b[4 * q] | (b[4 * q + 1] << 8) | (b[4 * q + 2] << 16) | ((uint32_t)b[4 * q + 3] << 24);
    }
  }
  void store(int t, const uint32_t* x) {
    for (int c = 0; c < W / 4; ++c) {
      const size_t co = seg + (size_t)c * 512 + (size_t)lane * 16;
      for (int q = 0; q < 16; ++q)
        if (co + q < B) out[t][co + q] = (uint8_t)(x[4 * c + q / 4] >> (8 * (q % 4)));
    }
  }
};

template <int W, int M>
struct HostCoef {
  const DecodePlan* pl;
  uint32_t mask(int t, int j, int c) const { return ((pl->W[t][j] >> c) & 1u) ? 0xFFFFFFFFu : 0u; }
};

template <int W, int M>
void run_encode(int k, uint8_t* blocks, size_t B) {
  std::vector<const uint8_t*> in(k);
  std::vector<uint8_t*> out(M);
  for (int i = 0; i < k; ++i) in[i] = blocks + (size_t)(k - 1 - i) * B;
  for (int j = 0; j < M; ++j) out[j] = blocks + (size_t)(k + j) * B;
  const size_t segb = segment_bytes(W);
  for (size_t seg = 0; seg < B; seg += segb)
    for (int lane = 0; lane < 32; ++lane) {
      HostTile<W> t{in.data(), out.data(), B, seg, lane};
      PolyEncode<W, M>::run(k, t, t);
    }
}

template <int W, int M>
void run_decode(const DecodePlan& pl, uint8_t* blocks, size_t B) {
  std::vector<const uint8_t*> in;
  std::vector<uint8_t*> out;
  for (int b : pl.in_blocks) in.push_back(blocks + (size_t)b * B);
  for (int b : pl.out_blocks) out.push_back(blocks + (size_t)b * B);
  const size_t segb = segment_bytes(W);
  HostCoef<W, M> cf{&pl};
  for (size_t seg = 0; seg < B; seg += segb)
    for (int lane = 0; lane < 32; ++lane) {
      HostTile<W> t{in.data(), out.data(), B, seg, lane};
      PolyDecode<W, M>::run(pl.n_pos, pl.read_mask, pl.e, t, t, cf);
    }
}

template <int W>
int encode_w(int k, int m, uint8_t* blocks, size_t B) {
  switch (m) {
    case 1: run_encode<W, 1>(k, blocks, B); return 0;
    case 2: run_encode<W, 2>(k, blocks, B); return 0;
    case 3: run_encode<W, 3>(k, blocks, B); return 0;
    case 4: run_encode<W, 4>(k, blocks, B); return 0;
    case 5: run_encode<W, 5>(k, blocks, B); return 0;
    case 6: run_encode<W, 6>(k, blocks, B); return 0;
    case 7: run_encode<W, 7>(k, blocks, B); return 0;
    case 8: run_encode<W, 8>(k, blocks, B); return 0;
  }
  return -1;
}

template <int W>
int decode_w(const DecodePlan& pl, uint8_t* blocks, size_t B) {
  switch (pl.M) {
    case 1: run_decode<W, 1>(pl, blocks, B); return 0;
    case 2: run_decode<W, 2>(pl, blocks, B); return 0;
    case 3: run_decode<W, 3>(pl, blocks, B); return 0;
    case 4: run_decode<W, 4>(pl, blocks, B); return 0;
    case 5: run_decode<W, 5>(pl, blocks, B); return 0;
    case 6: run_decode<W, 6>(pl, blocks, B); return 0;
    case 7: run_decode<W, 7>(pl, blocks, B); return 0;
    case 8: run_decode<W, 8>(pl, blocks, B); return 0;
  }
  return -1;
}

}  // namespace

extern "C" {

int emu_poly_encode(int w, int k, int m, uint8_t* blocks, size_t B) {
  return w == 8 ? encode_w<8>(k, m, blocks, B) : (w == 16 ? encode_w<16>(k, m, blocks, B) : -1);
}

int emu_poly_decode(int w, int k, int m, const int* er, int e, int read_all, uint8_t* blocks, size_t B) {
  DecodePlan pl;
  std::string err;
  if (!make_poly_decode_plan(k, m, w, er, e, read_all != 0, pl, err)) return -1;
  if (e == 0) return 0;
  return w == 8 ? decode_w<8>(pl, blocks, B) : decode_w<16>(pl, blocks, B);
}

// Plan introspection for tests: M, read mask, W rows.
int emu_poly_plan(int k, int m, int w, const int* er, int e, int read_all, int* M, uint64_t* read_mask,
                  uint32_t* Wout /* 8x8 */) {
  DecodePlan pl;
  std::string err;
  if (!make_poly_decode_plan(k, m, w, er, e, read_all != 0, pl, err)) return -1;
  *M = pl.M;
  *read_mask = pl.read_mask;
  for (int t = 0; t < 8; ++t)
    for (int j = 0; j < 8; ++j) Wout[t * 8 + j] = pl.W[t][j];
  return 0;
}

// The compile-time generator polynomial coefficients the kernels use.
int emu_genpoly(int w, int m, uint32_t* g) {
  const GenPoly gp = make_genpoly(w, m);
  for (int i = 0; i <= m; ++i) g[i] = gp.c[i];
  return 0;
}

// Transpose round trip and plane semantics for the tests.
int emu_transpose(int w, uint32_t* x) {
  if (w == 8) transpose<8>(x);
  else if (w == 16) transpose<16>(x);
  else return -1;
  return 0;
}

}  // extern "C"
