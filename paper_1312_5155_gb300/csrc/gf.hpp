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

// Ones of the bit-matrix of e (§2.3 projection): the XOR count of a
// product by e in the bit-matrix codes.  Column c is e * alpha^c.
RS_CHD constexpr int bitmatrix_ones(uint32_t e, int w) {
  int n = 0;
  uint32_t col = e;
  for (int c = 0; c < w; ++c) {
    for (uint32_t v = col; v; v &= v - 1u) ++n;
    col = gf_mul(col, 2u, w);
  }
  return n;
}

// "Good" Cauchy matrix (§2.3: Cauchy matrices differ in XOR cost; GoodCRS
// of §5.1), in place on an m x k parity matrix (row stride k) holding the
// original Cauchy matrix.  Scaling a row or a column by a nonzero element
// keeps every square submatrix nonsingular (the code stays MDS), so: every
// column is divided by its row-0 entry (row 0 becomes all ones, w ones
// each), then every other row is divided by whichever of 1 and its own
// entries leaves the fewest ones (the first such on ties).  at(i, j)
// returns a reference to entry (i, j).
template <class At>
RS_CHD constexpr void good_cauchy_scale(At&& at, int k, int m, int w) {
  for (int j = 0; j < k; ++j) {
    const uint32_t d = gf_inv(at(0, j), w);
    for (int i = 0; i < m; ++i) at(i, j) = gf_mul(at(i, j), d, w);
  }
  for (int i = 1; i < m; ++i) {
    uint32_t best = 1;
    long best_ones = -1;
    for (int t = -1; t < k; ++t) {
      const uint32_t vi = gf_inv(t < 0 ? 1u : at(i, t), w);
      long n = 0;
      for (int j = 0; j < k; ++j) n += bitmatrix_ones(gf_mul(at(i, j), vi, w), w);
      if (best_ones < 0 || n < best_ones) {
        best_ones = n;
        best = vi;
      }
    }
    for (int j = 0; j < k; ++j) at(i, j) = gf_mul(at(i, j), best, w);
  }
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
