// GF(2^w) arithmetic for the library, usable at compile time (constexpr),
// in host code and in device code.
//
// Field: GF(2)[x] / p(x) with p = 0x11D for w = 8 and 0x1100B for w = 16;
// the primitive element is alpha = x = 2 (the paper's §3.1 example uses
// primitive root 2 over GF(2^8)).  Products are shift-and-add with reduction;
// they are only evaluated on the host (per code / per erasure pattern) or at
// compile time, never per symbol on the device: the device works on
// bit-sliced planes where a product by a constant is a GF(2) bit-matrix.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define RS_HD __host__ __device__ __forceinline__
#define RS_CHD __host__ __device__
#else
#define RS_HD inline
#define RS_CHD
#endif

namespace rsgb {

constexpr int kMaxM = 8;        // parity blocks handled by the device path
constexpr int kMaxBlocks = 64;  // k + m handled by the device path

// Words of an m x m decode matrix over GF(2^w) in selector form: per row,
// one nibble per (coefficient bit, chunk of four syndromes), eight a word.
RS_CHD constexpr int selector_words(int m, int w) { return m * ((w * ((m + 3) / 4) + 7) / 8); }

RS_CHD constexpr uint32_t prim_poly(int w) { return w == 8 ? 0x11Du : (w == 16 ? 0x1100Bu : 0u); }

RS_CHD constexpr uint32_t gf_mul(uint32_t a, uint32_t b, int w) {
  uint32_t r = 0;
  const uint32_t top = 1u << w, p = prim_poly(w);
  for (int i = 0; i < w; ++i) {
    if (b & 1u) r ^= a;
    b >>= 1;
    a <<= 1;
    if (a & top) a ^= p;
  }
  return r;
}

RS_CHD constexpr uint32_t gf_pow(uint32_t a, uint64_t e, int w) {
  uint32_t r = 1;
  while (e) {
    if (e & 1u) r = gf_mul(r, a, w);
    a = gf_mul(a, a, w);
    e >>= 1;
  }
  return r;
}

// alpha^e with alpha = 2; exponents taken modulo the group order 2^w - 1.
RS_CHD constexpr uint32_t gf_alpha_pow(uint64_t e, int w) {
  return gf_pow(2u, e % ((1ull << w) - 1ull), w);
}

// a^-1 = a^(2^w - 2) for a != 0.
RS_CHD constexpr uint32_t gf_inv(uint32_t a, int w) { return gf_pow(a, (1ull << w) - 2ull, w); }

// Generator polynomial of §3.1: g(x) = prod_{i<m} (x + alpha^i), monic,
// coefficient of x^i in c[i].
struct GenPoly {
  uint32_t c[kMaxM + 1];
};

RS_CHD constexpr GenPoly make_genpoly(int w, int m) {
  GenPoly g{};
  for (int i = 0; i <= kMaxM; ++i) g.c[i] = 0;
  g.c[0] = 1;
  for (int i = 0; i < m; ++i) {
    const uint32_t root = gf_alpha_pow((uint64_t)i, w);
    for (int j = i + 1; j >= 1; --j) g.c[j] = g.c[j - 1] ^ gf_mul(root, g.c[j], w);
    g.c[0] = gf_mul(root, g.c[0], w);
  }
  return g;
}

// Bit-matrix of "multiply by e" (§2.3's projection): column c is the bit
// vector of e * alpha^c; row r, as a w-bit mask over columns, is returned by
// bitmatrix_row.  Then bit r of e*x = parity(row_r & x).
RS_CHD constexpr uint32_t bitmatrix_row(uint32_t e, int r, int w) {
  uint32_t row = 0;
  uint32_t col = e;
  for (int c = 0; c < w; ++c) {
    if ((col >> r) & 1u) row |= (1u << c);
    col = gf_mul(col, 2u, w);
  }
  return row;
}

template <int W, uint32_t E>
struct BitMatrix {
  struct Rows {
    uint32_t r[W];
  };
  static constexpr Rows make() {
    Rows m{};
    for (int i = 0; i < W; ++i) m.r[i] = bitmatrix_row(E, i, W);
    return m;
  }
  static constexpr Rows value = make();
};

template <int W, int M>
struct GenPolyOf {
  static constexpr GenPoly value = make_genpoly(W, M);
};

}  // namespace rsgb
