// Polynomial realization (§3), per group of 32 symbol columns held in
// bit-planes by one thread.  Host/device code; the caller supplies
//   src.load(i, x)   : W words of input i (consumption order), as stored
//   dst.store(t, x)  : W words of output t, as stored
//   dst.store(t, x)  : may be called with a runtime t
//   coef.word(i)     : word i of the runtime matrix W in selector form
//                      (Selectors<W, M> layout)
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
// One LFSR step with register renaming: after S steps (mod M) logical r_j
// lives in physical register (j - S) mod M.  Then every update is in place:
// new r_j = old r_{j-1} + g_j f lands in the register that held r_{j-1}, and
// new r_0 = g_0 f in the one that held r_{m-1} (already folded into f).  M
// consecutive steps return the mapping to the identity, so a runtime loop
// over groups of M steps needs no register moves.
template <int W, int M>
struct PolyEncode {
  static RS_CHD constexpr int phys(int j, int S) { return ((j - S) % M + M) % M; }

  template <int S>
  static RS_HD void step(uint32_t (*r)[W], const uint32_t* x) {
    constexpr int top = phys(M - 1, S);
    uint32_t f[W];
#pragma unroll
    for (int b = 0; b < W; ++b) f[b] = x[b] ^ r[top][b];
    StaticFor<1, M>::run([&](auto J) {
      constexpr int j = decltype(J)::value;
      mul_acc<W, GenPolyOf<W, M>::value.c[j]>(r[phys(j - 1, S)], f);
    });
    mul_set<W, GenPolyOf<W, M>::value.c[0]>(r[top], f);
  }

  template <int S, class Src>
  static RS_HD void load_step(int i, uint32_t (*r)[W], Src& src) {
    uint32_t x[W];
    src.load(i, x);
    transpose<W>(x);
    step<S>(r, x);
  }

  // Remaining R < M steps after the grouped loop, then the stores with the
  // mapping rotated by R.
  template <int R, class Src, class Dst>
  static RS_HD void finish(int i, int rem, uint32_t (*r)[W], Src& src, Dst& dst) {
    if constexpr (R < M) {
      if (rem == R) {
        StaticFor<0, R>::run([&](auto S) { load_step<decltype(S)::value>(i + decltype(S)::value, r, src); });
        StaticFor<0, M>::run([&](auto J) {
          constexpr int p = phys(decltype(J)::value, R);
          transpose<W>(r[p]);
          dst.store(decltype(J)::value, r[p]);
        });
        return;
      }
      finish<R + 1>(i, rem, r, src, dst);
    }
  }

  // §3.2 Eq. 1: p(x) = x^m d(x) mod g(x).  Division by the monic g(x) as a
  // linear-feedback shift register fed with the data symbols from the highest
  // degree down (d_{k-1} first, since d_i sits at x^(m+i)):
  //   f = d_i + r_{m-1};  r_j = r_{j-1} + g_j f (j = m-1..1);  r_0 = g_0 f.
  // After the k data symbols, r_j is the coefficient of x^j of the remainder,
  // i.e. parity p_j.  All g_j are compile-time constants (they depend on m
  // only), so every product is a fixed XOR pattern over bit-planes.
  // inputs: k data blocks in the order d_{k-1}, ..., d_0; outputs p_0..p_{m-1}
  template <class Src, class Dst>
  static RS_HD void run(int k, Src& src, Dst& dst) {
    uint32_t r[M][W];
#pragma unroll
    for (int j = 0; j < M; ++j)
#pragma unroll
      for (int b = 0; b < W; ++b) r[j][b] = 0;
    int i = 0;
    for (; i + M <= k; i += M) {
      StaticFor<0, M>::run([&](auto S) { load_step<decltype(S)::value>(i + decltype(S)::value, r, src); });
    }
    finish<0>(i, k - i, r, src, dst);
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
// Multiply by alpha in place under register renaming: logical plane b of
// the value lives in physical register (b - ROT) mod W.  The shift of the
// planes is the renaming itself (ROT grows by one); only the fold of the top
// plane through the primitive polynomial costs XORs.
template <int W, int ROT>
RS_HD void mul_alpha_renamed(uint32_t* x) {
  constexpr uint32_t low = prim_poly(W) & ((1u << W) - 1u);
  constexpr int np = ROT + 1;                       // rotation after the step
  constexpr int top = ((0 - np) % W + W) % W;       // new logical 0 = old logical W-1
#pragma unroll
  for (int r = 1; r < W; ++r) {
    if ((low >> r) & 1u) x[((r - np) % W + W) % W] ^= x[top];
  }
}

// Syndrome j multiplied by alpha^j at step s of a group: j renamed alpha
// steps, starting from rotation j*s.
template <int W, int M, int s>
RS_HD void horner_mul(uint32_t (*S)[W]) {
  StaticFor<1, M>::run([&](auto J) {
    constexpr int j = decltype(J)::value;
    StaticFor<0, j>::run([&](auto T) {
      mul_alpha_renamed<W, (j * s + decltype(T)::value) % W>(S[j]);
    });
  });
}

// One Horner step with an input: S_j = alpha^j S_j + x for every j.  The
// last alpha step of each syndrome is fused with the addition, so its fold
// of the top plane and the input's plane cost one 3-input XOR.
template <int W, int M, int s>
RS_HD void horner_mul_add(uint32_t (*S)[W], const uint32_t* x) {
  constexpr uint32_t low = prim_poly(W) & ((1u << W) - 1u);
#pragma unroll
  for (int b = 0; b < W; ++b) S[0][b] ^= x[b];
  StaticFor<1, M>::run([&](auto J) {
    constexpr int j = decltype(J)::value;
    StaticFor<0, j - 1>::run([&](auto T) {
      mul_alpha_renamed<W, (j * s + decltype(T)::value) % W>(S[j]);
    });
    constexpr int np = j * s + j;               // rotation after the fused step
    constexpr int top = ((0 - np) % W + W) % W;  // register of new logical plane 0
#pragma unroll
    for (int b = 1; b < W; ++b) {
      const int ph = ((b - np) % W + W) % W;
      if ((low >> b) & 1u)
        S[j][ph] ^= S[j][top] ^ x[b];
      else
        S[j][ph] ^= x[b];
    }
    S[j][top] ^= x[0];  // after the folds, which read the old top plane
  });
}

// One bit of the decode-matrix Horner rule, y <- alpha * y + Z (Z the
// subset of the syndromes the selector names), with y going from rotation
// ROT - 1 to ROT: on the GPU one jump-table dispatch whose cases merge the
// fold of alpha * y into the selected XORs; elsewhere the two steps.
template <int W, int ROT, int NS>
RS_HD void fold_and_select(uint32_t sel, uint32_t* y, const uint32_t (*S)[W], const uint32_t (*P)[W]) {
#if defined(__CUDA_ARCH__)
  if constexpr (W == 8) {
    fold_select_w8<ROT, NS>(sel, y, S, P);
    return;
  } else if constexpr (W == 16) {
    fold_select_w16<ROT, NS>(sel, y, S);
    return;
  }
#endif
  mul_alpha_renamed<W, ROT - 1>(y);
  xor_selected<W, ROT, NS>(sel, y, S, P);
}

// The same for two 32-column groups (y0 from A, y1 from B; no pair sums).
template <int W, int ROT, int NS>
RS_HD void fold_and_select2(uint32_t sel, uint32_t* y0, uint32_t* y1, const uint32_t (*A)[W], const uint32_t (*B)[W]) {
#if defined(__CUDA_ARCH__)
  if constexpr (W == 8) {
    fold_select2_w8<ROT, NS>(sel, y0, y1, A, B);
    return;
  } else if constexpr (W == 16) {
    fold_select2_w16<ROT, NS>(sel, y0, y1, A, B);
    return;
  }
#endif
  mul_alpha_renamed<W, ROT - 1>(y0);
  mul_alpha_renamed<W, ROT - 1>(y1);
  xor_selected2<W, ROT, NS>(sel, y0, y1, A, B);
}

// Two groups with the pair sums PA = (A0^A1, A2^A3), PB likewise.
template <int W, int ROT, int NS>
RS_HD void fold_and_select2p(uint32_t sel, uint32_t* y0, uint32_t* y1, const uint32_t (*A)[W], const uint32_t (*B)[W],
                             const uint32_t (*PA)[W], const uint32_t (*PB)[W]) {
#if defined(__CUDA_ARCH__)
  if constexpr (W == 8) {
    fold_select2p_w8<ROT, NS>(sel, y0, y1, A, B, PA, PB);
    return;
  }
#endif
  mul_alpha_renamed<W, ROT - 1>(y0);
  mul_alpha_renamed<W, ROT - 1>(y1);
  xor_selected<W, ROT, NS>(sel, y0, A, PA);
  xor_selected<W, ROT, NS>(sel, y1, B, PB);
}

// Steps per pass of the syndrome Horner and bits per pass of the
// decode-matrix Horner.  Fully unrolling the W-step renaming period makes
// the decode's loop body larger than the instruction cache serves well;
// shorter passes with one move of the planes back to rotation 0 at the end
// of each pass measured faster on GB300 (4 and 2 against W and W).
template <int W>
constexpr int kHornerSteps = 4;
template <int W>
constexpr int kApplySteps = 2;

// Erased outputs from the M syndromes: out_t = sum_j W[t][j] S_j for t < e,
// one output at a time.  Each output is Horner's rule in alpha over the bits
// of its row of W (top bit first): y = alpha * y + Z_{t,c}, where Z_{t,c} is
// the XOR of the syndromes that the warp-uniform selector of (t, c) names
// (at most two terms per chunk of four, using precomputed pair sums).
// The alpha steps are renamed within a pass, so an output costs W folds of
// the top plane plus one XOR per selected syndrome and plane (and a move of
// the planes per pass), instead of W * M masked XORs per plane.
template <int W, int M, bool kTranspose, class Dst>
RS_HD void apply_and_store(int e, const uint32_t (*S)[W], const Selectors<W, M>& sel, Dst& dst) {
  using Sel = Selectors<W, M>;
  // pair sums per chunk of four syndromes (entries a chunk lacks stay unused)
  uint32_t P[Sel::kChunks][2][W];
#pragma unroll
  for (int h = 0; h < Sel::kChunks; ++h)
#pragma unroll
    for (int b = 0; b < W; ++b) {
      if (4 * h + 1 < M) P[h][0][b] = S[4 * h][b] ^ S[4 * h + 1][b];
      if (4 * h + 3 < M) P[h][1][b] = S[4 * h + 2][b] ^ S[4 * h + 3][b];
    }
#pragma unroll 1
  for (int t = 0; t < e; ++t) {
    uint32_t row[Sel::kRowWords];
    sel.row(t, row);
    uint32_t y[W];
#pragma unroll
    for (int b = 0; b < W; ++b) y[b] = 0;
    // Horner over the coefficient bits, top bit first, kSteps bits per pass:
    // inside a pass the alpha steps are renamed; a pass that ends off
    // rotation 0 moves the planes back so every pass runs the same code.
    constexpr int kSteps = kApplySteps<W>;
#pragma unroll 1
    for (int c0 = W - 1; c0 >= 0; c0 -= kSteps) {
      StaticFor<0, kSteps>::run([&](auto Uu) {
        constexpr int u = decltype(Uu)::value;
        const int c = c0 - u;
        // alpha * y (alpha * 0 on the first bit: harmless) fused with the
        // first chunk's selected syndromes
        StaticFor<0, Sel::kChunks>::run([&](auto H) {
          constexpr int h = decltype(H)::value;
          constexpr int ns = (M - 4 * h < 4) ? M - 4 * h : 4;
          if constexpr (h == 0)
            fold_and_select<W, u + 1, ns>(Sel::nibble(row, c * Sel::kChunks), y, S, P[0]);
          else
            xor_selected<W, u + 1, ns>(Sel::nibble(row, c * Sel::kChunks + h), y, S + 4 * h, P[h]);
        });
      });
      if constexpr (kSteps % W != 0) {
        uint32_t r[W];
#pragma unroll
        for (int b = 0; b < W; ++b) r[b] = y[((b - kSteps) % W + W) % W];
#pragma unroll
        for (int b = 0; b < W; ++b) y[b] = r[b];
      }
    }
    if (kTranspose) transpose<W>(y);
    dst.store(t, y);
  }
}

template <int W, int M>
struct PolyDecode {
  // n_pos: codeword length n; read_mask bit p: position p was read, in which
  // case the next input (inputs ordered by descending position) holds it.
  template <class Src, class Dst, class Coef>
  static RS_HD void run(int n_pos, uint64_t read_mask, int e, Src& src, Dst& dst, Coef& coef) {
    Selectors<W, M> sel;  // loaded first: its latency hides behind Step 1
    sel.load(coef);
    uint32_t S[M][W];
#pragma unroll
    for (int j = 0; j < M; ++j)
#pragma unroll
      for (int b = 0; b < W; ++b) S[j][b] = 0;
    // Horner over positions in groups of W steps (the renaming period); the
    // count is padded at the top with positions that hold no data.  Step i
    // (from the top) handles position groups*W - 1 - i: bit i of `order` says
    // whether that position was read.  Until the first read position the
    // syndromes are zero, so those steps skip their multiply too.
    constexpr int U = kHornerSteps<W>;
    const int groups = (n_pos + U - 1) / U;
    const uint64_t order = bit_reverse64(read_mask) >> (64 - groups * U);
    const uint64_t live = ~((order & (~order + 1ull)) - 1ull);  // steps from the first read one on
    int i = 0;
#pragma unroll 1
    for (int g = 0; g < groups; ++g) {
      const uint32_t ob = (uint32_t)(order >> (g * U));
      const uint32_t lb = (uint32_t)(live >> (g * U));
      StaticFor<0, U>::run([&](auto St) {
        constexpr int st = decltype(St)::value;
        if ((ob >> st) & 1u) {
          uint32_t x[W];
          src.load(i++, x);
          transpose<W>(x);
          horner_mul_add<W, M, st>(S, x);
        } else if ((lb >> st) & 1u) {
          horner_mul<W, M, st>(S);
        }
      });
      if constexpr (U % W != 0) {
        // syndrome j is now in rotation j*U: move its planes back to rotation 0
        StaticFor<1, M>::run([&](auto J) {
          constexpr int rot = (decltype(J)::value * U) % W;
          if constexpr (rot != 0) {
            uint32_t r[W];
#pragma unroll
            for (int b = 0; b < W; ++b) r[b] = S[decltype(J)::value][((b - rot) % W + W) % W];
#pragma unroll
            for (int b = 0; b < W; ++b) S[decltype(J)::value][b] = r[b];
          }
        });
      }
    }
    apply_and_store<W, M, true>(e, S, sel, dst);
  }
};

// apply_and_store for two 32-column groups: output t of group 0 from the
// syndromes A, of group 1 from B, stored as one 2W-word output (group 0 in
// words 0..W-1; planes back to symbols with kTranspose).  Pair sums with
// kPairSums (M <= 4, one selector chunk); M = 5..8 take a second chunk per
// coefficient bit.
template <int W, int M, bool kTranspose = true, bool kPairSums = false, class Dst>
RS_HD void apply2_and_store(int e, const uint32_t (*A)[W], const uint32_t (*B)[W], const Selectors<W, M>& sel,
                            Dst& dst) {
  static_assert(M <= 8 && (M <= 4 || !kPairSums), "two selector chunks, pair sums with one");
  using Sel = Selectors<W, M>;
  // pair sums A0^A1, A2^A3 (and of B) when the kernel has registers for
  // them: a subset of four syndromes is then at most two terms per plane
  constexpr bool kPairs = kPairSums && M >= 2;
  uint32_t PA[2][W], PB[2][W];
  if constexpr (kPairs) {
#pragma unroll
    for (int b = 0; b < W; ++b) {
      PA[0][b] = A[0][b] ^ A[1][b];
      PB[0][b] = B[0][b] ^ B[1][b];
      if (M > 3) {
        PA[1][b] = A[2][b] ^ A[3][b];
        PB[1][b] = B[2][b] ^ B[3][b];
      }
    }
  }
#pragma unroll 1
  for (int t = 0; t < e; ++t) {
    uint32_t row[Sel::kRowWords];
    sel.row(t, row);
    uint32_t y[2 * W];
#pragma unroll
    for (int b = 0; b < 2 * W; ++b) y[b] = 0;
    constexpr int kSteps = kApplySteps<W>;
#pragma unroll 1
    for (int c0 = W - 1; c0 >= 0; c0 -= kSteps) {
      StaticFor<0, kSteps>::run([&](auto Uu) {
        constexpr int u = decltype(Uu)::value;
        const int c = c0 - u;
        constexpr int ns0 = M < 4 ? M : 4;
        if constexpr (kPairs)
          fold_and_select2p<W, u + 1, M>(Sel::nibble(row, c), y, y + W, A, B, PA, PB);
        else
          fold_and_select2<W, u + 1, ns0>(Sel::nibble(row, c * Sel::kChunks), y, y + W, A, B);
        if constexpr (Sel::kChunks > 1)
          xor_selected2<W, u + 1, M - 4>(Sel::nibble(row, c * Sel::kChunks + 1), y, y + W, A + 4, B + 4);
      });
      if constexpr (kSteps % W != 0) {
        uint32_t r[2 * W];
#pragma unroll
        for (int b = 0; b < W; ++b) {
          r[b] = y[((b - kSteps) % W + W) % W];
          r[W + b] = y[W + ((b - kSteps) % W + W) % W];
        }
#pragma unroll
        for (int b = 0; b < 2 * W; ++b) y[b] = r[b];
      }
    }
    if (kTranspose) {
      transpose<W>(y);
      transpose<W>(y + W);
    }
    dst.store(t, y);
  }
}

// Two 32-column groups per thread (G = 2): the same decode as PolyDecode on
// 2W words (group 0 = words 0..W-1, group 1 = W..2W-1 of every input and
// output).  Every warp-uniform decision -- the Horner presence test, the
// barrier waits, the selector dispatch -- then serves 64 columns, and the
// two groups' instruction streams are independent.  Pair sums in the
// decode-matrix step with kPairSums (they need the larger register budget
// of the split kernel; M <= 4); M = 5..8 without.
template <int W, int M, bool kPairSums = false>
struct PolyDecode2 {
  static_assert(M <= 8 && (M <= 4 || !kPairSums), "pair sums with one selector chunk");
  template <class Src, class Dst, class Coef>
  static RS_HD void run(int n_pos, uint64_t read_mask, int e, Src& src, Dst& dst, Coef& coef) {
    Selectors<W, M> sel;
    sel.load(coef);
    uint32_t A[M][W], B[M][W];
#pragma unroll
    for (int j = 0; j < M; ++j)
#pragma unroll
      for (int b = 0; b < W; ++b) A[j][b] = B[j][b] = 0;
    // a whole renaming period per pass: no rotation fix (measured 2-4 %
    // faster than 4-step passes with two groups)
    constexpr int U = W;
    const int groups = (n_pos + U - 1) / U;
    const uint64_t order = bit_reverse64(read_mask) >> (64 - groups * U);
    const uint64_t live = ~((order & (~order + 1ull)) - 1ull);
    int i = 0;
#pragma unroll 1
    for (int g = 0; g < groups; ++g) {
      const uint32_t ob = (uint32_t)(order >> (g * U));
      const uint32_t lb = (uint32_t)(live >> (g * U));
      StaticFor<0, U>::run([&](auto St) {
        constexpr int st = decltype(St)::value;
        if ((ob >> st) & 1u) {
          uint32_t x[2 * W];
          src.load(i++, x);
          transpose<W>(x);
          transpose<W>(x + W);
          horner_mul_add<W, M, st>(A, x);
          horner_mul_add<W, M, st>(B, x + W);
        } else if ((lb >> st) & 1u) {
          horner_mul<W, M, st>(A);
          horner_mul<W, M, st>(B);
        }
      });
      if constexpr (U % W != 0) {
        StaticFor<1, M>::run([&](auto J) {
          constexpr int j = decltype(J)::value;
          constexpr int rot = (j * U) % W;
          if constexpr (rot != 0) {
            uint32_t ra[W], rb[W];
#pragma unroll
            for (int b = 0; b < W; ++b) {
              ra[b] = A[j][((b - rot) % W + W) % W];
              rb[b] = B[j][((b - rot) % W + W) % W];
            }
#pragma unroll
            for (int b = 0; b < W; ++b) {
              A[j][b] = ra[b];
              B[j][b] = rb[b];
            }
          }
        });
      }
    }
    apply2_and_store<W, M, true, kPairSums>(e, A, B, sel, dst);
  }
};

}  // namespace rsgb
