// Host-side planning: which blocks a decode reads, in which order, and the
// small runtime matrix the device applies.  One plan per (code, erasure
// pattern); the library caches them (Opt1/Opt3 of §4: coefficients and the
// inverted Vandermonde matrix are computed once, not per column).
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "gf.hpp"

namespace rsgb {

enum class Realization : int { Poly = 0, Vandermonde = 1, Cauchy = 2, PolyMatrix = 3, PolyBitMatrix = 4, GoodCauchy = 5 };

struct DecodePlan {
  int M = 0;                  // unknowns = syndromes evaluated
  int e = 0;                  // outputs written
  int n_pos = 0;              // codeword length n
  uint64_t read_mask = 0;     // bit p: position (poly) / block (matrix) p is read
  std::vector<int> in_blocks;   // block indices, in device consumption order
  std::vector<int> out_blocks;  // erased block indices, row order of W
  uint32_t W[kMaxM][kMaxM] = {};  // output t = sum_j W[t][j] * syndrome_j
};

// Position of block b in the codeword polynomial: d_i at x^(m+i), p_j at x^j
// (§3.2 Eq. 2 and its example, where d_0 multiplies x^m).
inline int poly_position(int k, int m, int b) { return b < k ? m + b : b - k; }

// Invert an n x n matrix over GF(2^w) (Gauss-Jordan).  false if singular.
bool gf_invert(int w, int n, const std::vector<uint32_t>& A, std::vector<uint32_t>& Ainv);

// Validates the erasure list (distinct, in [0, n), e <= m) and builds the
// plan for the polynomial realization.  read_all: read every survivor
// (§3.3's second remark) instead of the first k by block index.
bool make_poly_decode_plan(int k, int m, int w, const int* erasures, int e, bool read_all,
                           DecodePlan& plan, std::string& err);

// Matrix realizations decode through the parity-check matrix H = [P | I_m]
// (P = parity rows of the systematic generator, m x k): syndrome
// s_i = p_i + sum_j P[i][j] d_j over the read blocks equals the contribution
// of the unread/erased blocks, so the unknowns follow from the M x M system
// H_U.  Same runtime-matrix form as the polynomial decode.
bool make_matrix_decode_plan(int k, int m, int w, const std::vector<uint32_t>& P,
                             const int* erasures, int e, bool read_all, DecodePlan& plan,
                             std::string& err);

// Pack an R x Q matrix of w-bit field elements (row-major in `a`) into the
// bit layout of PackedBits<W, R, Q>: entry (r, q) at bits [(q*R + r)*w, +w).
std::vector<uint32_t> pack_bits(const uint32_t* a, int R, int Q, int w);

// Words of the runtime decode matrix W (e used rows of the M x M slot) in
// the device's selector form: for row t, coefficient bit c and chunk h of
// four syndromes, a nibble whose bit i is bit c of W[t][4h + i]; nibble
// n = c * ceil(M/4) + h of row t at bits 4 * (n % 8) of word
// t * ceil(w * ceil(M/4) / 8) + n / 8.
std::vector<uint32_t> pack_decode_selectors(const DecodePlan& pl, int w);

// Words of P's columns for the runtime-P kernels: column j (entries
// P[0..m-1][j]) occupies column_words(m, w) consecutive words.
inline int column_words(int m, int w) { return (m * w + 31) / 32; }
std::vector<uint32_t> pack_columns(const std::vector<uint32_t>& P, int k, int m, int w);

// Parity rows (m x k, row-major) of the systematic generators (§2.2, §2.3).
bool vandermonde_parity_matrix(int k, int m, int w, std::vector<uint32_t>& P);
void cauchy_parity_matrix(int k, int m, int w, std::vector<uint32_t>& P);
// The "good" Cauchy matrix (§2.3, GoodCRS of §5.1): good_cauchy_scale of the above.
void good_cauchy_parity_matrix(int k, int m, int w, std::vector<uint32_t>& P);
// Polynomial code as a generator matrix (§6): column i = x^(m+i) mod g(x).
void poly_parity_matrix(int k, int m, int w, std::vector<uint32_t>& P);

}  // namespace rsgb
