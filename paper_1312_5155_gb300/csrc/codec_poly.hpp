// Polynomial realization (§3), per group of 32 symbol columns held in
// bit-planes by one thread.  Host/device code; the caller supplies
//   src.load(i, x)   : W words of input i (consumption order), as stored
//   dst.store(t, x)  : W words of output t, as stored
//   coef.word(i)     : word i of the runtime matrix W as packed bits
//                      (PackedBits<W, M, M> layout, entry (t, j))
#pragma once
#include "bitslice.hpp"

namespace rsgb {

// ---------------------------------------------------------------- encode
// §3.2 Eq. 1: p(x) = x^m d(x) mod g(x).  Division by the monic g(x) as a
// linear-feedback shift register fed with the data symbols from the highest
// degree down (d_{k-1} first, since d_i sits at x^(m+i)):
//   f = d_i + r_{m-1};  r_j = r_{j-1} + g_j f (j = m-1..1);  r_0 = g_0 f.
// After the k data symbols, r_j is the coefficient of x^j of the remainder,
// i.e. parity p_j.  All g_j are compile-time constants (they depend on m
// only), so every product is a fixed XOR pattern over bit-planes.
template <int W, int M, int J>
struct LfsrShift {
  static RS_HD void run(uint32_t (*r)[W], const uint32_t* f) {
#pragma unroll
    for (int b = 0; b < W; ++b) r[J][b] = r[J - 1][b];
    mul_acc<W, GenPolyOf<W, M>::value.c[J]>(r[J], f);
    LfsrShift<W, M, J - 1>::run(r, f);
  }
};
template <int W, int M>
struct LfsrShift<W, M, 0> {
  static RS_HD void run(uint32_t (*r)[W], const uint32_t* f) {
    mul_set<W, GenPolyOf<W, M>::value.c[0]>(r[0], f);
  }
};

template <int W, int M>
struct PolyEncode {
  // inputs: k data blocks in the order d_{k-1}, ..., d_0; outputs p_0..p_{m-1}
  template <class Src, class Dst>
  static RS_HD void run(int k, Src& src, Dst& dst) {
    uint32_t r[M][W];
#pragma unroll
    for (int j = 0; j < M; ++j)
#pragma unroll
      for (int b = 0; b < W; ++b) r[j][b] = 0;
    for (int i = 0; i < k; ++i) {
      uint32_t x[W];
      src.load(i, x);
      transpose<W>(x);
      uint32_t f[W];
#pragma unroll
      for (int b = 0; b < W; ++b) f[b] = x[b] ^ r[M - 1][b];
      LfsrShift<W, M, M - 1>::run(r, f);
    }
#pragma unroll
    for (int j = 0; j < M; ++j) {
      transpose<W>(r[j]);
      dst.store(j, r[j]);
    }
  }
};

// ---------------------------------------------------------------- decode
// §3.3 Step 1 with Opt1/Opt2 of §4: the error-evaluator values
// D_j = c(alpha^j) over the read blocks (unread positions contribute 0),
// j = 0..M-1, evaluated by Horner's rule over the positions n-1..0:
//   S_j <- alpha^j S_j + c_pos.
// The multipliers alpha^j are compile-time constants.  Step 2 with Opt3:
// the host inverts the M x M Vandermonde system once per erasure pattern;
// output t is sum_j W[t][j] S_j with the runtime matrix W (rows of the
// inverse for the erased blocks).
template <int W, int M, int J>
struct HornerMul {
  static RS_HD void run(uint32_t (*S)[W]) {
    uint32_t t[W];
#pragma unroll
    for (int b = 0; b < W; ++b) t[b] = S[J][b];
    mul_set<W, gf_alpha_pow(J, W)>(S[J], t);
    HornerMul<W, M, J - 1>::run(S);
  }
};
template <int W, int M>
struct HornerMul<W, M, 0> {
  static RS_HD void run(uint32_t (*)[W]) {}  // alpha^0 = 1
};

// out[t] = sum_j W[t][j] S_j for t < e, with W as packed bits (entry (t, j)).
// For every syndrome j the chain alpha^c S_j (c = 0..W-1) is walked once and
// shared by all outputs; each chain term costs one AND-XOR per plane.  S is
// clobbered.
template <int W, int M>
RS_HD void apply_runtime_matrix(uint32_t (*out)[W], uint32_t (*S)[W], int e, const PackedBits<W, M, M>& wm) {
#pragma unroll
  for (int t = 0; t < M; ++t)
#pragma unroll
    for (int b = 0; b < W; ++b) out[t][b] = 0;
#pragma unroll
  for (int j = 0; j < M; ++j) {
#pragma unroll
    for (int c = 0; c < W; ++c) {
#pragma unroll
      for (int t = 0; t < M; ++t) {
        if (t < e) {
          const uint32_t mk = wm.mask(t, j, c);
#pragma unroll
          for (int b = 0; b < W; ++b) out[t][b] ^= S[j][b] & mk;
        }
      }
      if (c + 1 < W) mul_alpha<W>(S[j]);
    }
  }
}

template <int W, int M>
struct PolyDecode {
  // n_pos: codeword length n; read_mask bit p: position p was read, in which
  // case the next input (inputs ordered by descending position) holds it.
  template <class Src, class Dst, class Coef>
  static RS_HD void run(int n_pos, uint64_t read_mask, int e, Src& src, Dst& dst, Coef& coef) {
    PackedBits<W, M, M> wm;  // loaded first: its latency hides behind Step 1
    wm.load(coef);
    uint32_t S[M][W];
#pragma unroll
    for (int j = 0; j < M; ++j)
#pragma unroll
      for (int b = 0; b < W; ++b) S[j][b] = 0;
    int i = 0;
    for (int pos = n_pos - 1; pos >= 0; --pos) {
      HornerMul<W, M, M - 1>::run(S);
      if ((read_mask >> pos) & 1ull) {
        uint32_t x[W];
        src.load(i++, x);
        transpose<W>(x);
#pragma unroll
        for (int j = 0; j < M; ++j)
#pragma unroll
          for (int b = 0; b < W; ++b) S[j][b] ^= x[b];
      }
    }
    uint32_t out[M][W];
    apply_runtime_matrix<W, M>(out, S, e, wm);
#pragma unroll
    for (int t = 0; t < M; ++t) {
      if (t < e) {
        transpose<W>(out[t]);
        dst.store(t, out[t]);
      }
    }
  }
};

}  // namespace rsgb
