// Bit-sliced GF(2^w) arithmetic on 32 symbols at a time.
//
// A thread holds 32 symbols of one block as W 32-bit words (W = w: 8 words
// = 32 bytes for GF(2^8), 16 words = 32 little-endian uint16 for GF(2^16)).
// transpose_w() turns those words into W bit-planes: plane b holds bit b of
// all 32 symbols.  In that form
//   - adding symbols is one XOR per plane,
//   - multiplying by a constant e is the GF(2) matrix of §2.3's bit-matrix
//     projection applied to the planes: plane r of e*x is the XOR of the
//     planes c with bit r of (e * alpha^c) set.
// When e is known at compile time only the XORs for the ones of its matrix
// are emitted; when it is a runtime value every (row, column) pair costs one
// AND-XOR with a 0/~0 mask.
//
// The symbol-to-plane transpose is three (w=8) or four (w=16) rounds of
// masked swaps between register pairs; each round exchanges one bit of the
// register index with one bit of the position inside the word, so the whole
// transpose is an involution and also converts planes back to symbols.
// Plane b ends up with bit b of symbol (word v, lane i) at position
// w*i + v (i = symbol within the 32-bit word).
#pragma once
#include "gf.hpp"

namespace rsgb {

// Compile-time loop: f(Int<I>{}) for I = I0 .. N-1.
template <int V>
struct Int {
  static constexpr int value = V;
};

template <int I, int N>
struct StaticFor {
  template <class F>
  static RS_HD void run(F&& f) {
    f(Int<I>{});
    StaticFor<I + 1, N>::run(f);
  }
};
template <int N>
struct StaticFor<N, N> {
  template <class F>
  static RS_HD void run(F&&) {}
};


// Bit i of x moved to bit 63 - i.
RS_HD uint64_t bit_reverse64(uint64_t x) {
#if defined(__CUDA_ARCH__)
  return __brevll(x);
#else
  uint64_t r = 0;
  for (int i = 0; i < 64; ++i) r |= ((x >> i) & 1ull) << (63 - i);
  return r;
#endif
}

// Shifts by a constant, written as multiplies so that on the GPU they run
// on the FMA pipe (IMAD / IMAD.HI) and leave the integer-logic pipe, which
// bounds these kernels, to the XORs.
template <int S>
RS_HD uint32_t shl_fma(uint32_t x) {
  return x * (1u << S);
}
template <int S>
RS_HD uint32_t shr_fma(uint32_t x) {
#if defined(__CUDA_ARCH__)
  return __umulhi(x, 1u << (32 - S));
#else
  return x >> S;
#endif
}

// (a & m) | (b & ~m) as one 3-input logic instruction (truth table 0xE4 over
// a = 0xF0, b = 0xCC, m = 0xAA); written out because the compiler otherwise
// splits it in two.
RS_HD uint32_t bit_select(uint32_t a, uint32_t b, uint32_t m) {
#if defined(__CUDA_ARCH__)
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, 0xE4;" : "=r"(d) : "r"(a), "r"(b), "r"(m));
  return d;
#else
  return (a & m) | (b & ~m);
#endif
}

// x[i], x[i+D] for all i with bit D clear: exchange the bits of x[i] above
// the mask with the bits of x[i+D] below it.
template <int N, int D, int S, uint32_t MASK>
RS_HD void swap_round(uint32_t* x) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if ((i & D) == 0) {
      const uint32_t lo = x[i], hi = x[i + D];
#if defined(__CUDA_ARCH__)
      if (S == 8) {
        // byte-granular round: one PRMT per output word
        x[i] = __byte_perm(lo, hi, 0x6240);
        x[i + D] = __byte_perm(lo, hi, 0x7351);
        continue;
      }
#endif
      x[i] = bit_select(lo, shl_fma<S>(hi), MASK);
      x[i + D] = bit_select(shr_fma<S>(lo), hi, MASK);
    }
  }
}

template <int W>
RS_HD void transpose(uint32_t* x);

template <>
RS_HD void transpose<8>(uint32_t* x) {
  swap_round<8, 4, 4, 0x0F0F0F0Fu>(x);
  swap_round<8, 2, 2, 0x33333333u>(x);
  swap_round<8, 1, 1, 0x55555555u>(x);
}

template <>
RS_HD void transpose<16>(uint32_t* x) {
  swap_round<16, 8, 8, 0x00FF00FFu>(x);
  swap_round<16, 4, 4, 0x0F0F0F0Fu>(x);
  swap_round<16, 2, 2, 0x33333333u>(x);
  swap_round<16, 1, 1, 0x55555555u>(x);
}

// acc ^= E * in   (E a compile-time field element); the compiler folds
// each row's XOR chain into 3-input logic instructions.
template <int W, uint32_t E>
RS_HD void mul_acc(uint32_t* acc, const uint32_t* in) {
  constexpr typename BitMatrix<W, E>::Rows M = BitMatrix<W, E>::value;
#pragma unroll
  for (int r = 0; r < W; ++r) {
#pragma unroll
    for (int c = 0; c < W; ++c) {
      if ((M.r[r] >> c) & 1u) acc[r] ^= in[c];
    }
  }
}

// out = E * in
template <int W, uint32_t E>
RS_HD void mul_set(uint32_t* out, const uint32_t* in) {
#pragma unroll
  for (int r = 0; r < W; ++r) out[r] = 0;
  mul_acc<W, E>(out, in);
}

// x = alpha * x in place: shift the planes up by one and fold the top plane
// back in through the low bits of the primitive polynomial.
template <int W>
RS_HD void mul_alpha(uint32_t* x) {
  constexpr uint32_t low = prim_poly(W) & ((1u << W) - 1u);
  const uint32_t top = x[W - 1];
#pragma unroll
  for (int r = W - 1; r >= 1; --r) x[r] = x[r - 1];
  x[0] = top;
#pragma unroll
  for (int r = 1; r < W; ++r) {
    if ((low >> r) & 1u) x[r] ^= top;
  }
}

// A runtime matrix of field elements held as packed bits in registers.
// Entry (r, q) of an R x Q matrix is bits [(q*R + r)*W, +W) of the bit
// string; mask(r, q, c) expands bit c of that entry to 0 / ~0 with two
// shifts, so the entries cost kWords registers instead of R*Q*W.
template <int W, int R, int Q>
struct PackedBits {
  static constexpr int kWords = (R * Q * W + 31) / 32;
  uint32_t w[kWords];
  RS_HD uint32_t mask(int r, int q, int c) const {
    const int p = (q * R + r) * W + c;
    return (uint32_t)((int32_t)(w[p >> 5] << (31 - (p & 31))) >> 31);
  }
  template <class Src>
  RS_HD void load(const Src& src) {
#pragma unroll
    for (int i = 0; i < kWords; ++i) w[i] = src.word(i);
  }
};

// A runtime M x M decode matrix W in selector form.  Output row t is
// evaluated as a polynomial in alpha over the bits of its entries,
//   out_t = sum_c alpha^c Z_{t,c},   Z_{t,c} = sum_j [bit c of W[t][j]] S_j,
// and Z_{t,c} is named by selector nibbles: nibble h of (t, c) holds in bit i
// the bit c of W[t][4h + i].  Row t occupies kRowWords words; nibble
// n = c * kChunks + h of the row sits at bits 4 * (n % 8) of word n / 8.
// Every lane of a warp works on the same stripe, so the selectors are
// warp-uniform and a branch on one never diverges.
template <int W, int M>
struct Selectors {
  static constexpr int kChunks = (M + 3) / 4;
  static constexpr int kRowWords = (W * kChunks + 7) / 8;
  static constexpr int kWords = M * kRowWords;
  static_assert(kWords == selector_words(M, W), "selector layout");
  uint32_t w[kWords];
  template <class Src>
  RS_HD void load(const Src& src) {
#pragma unroll
    for (int i = 0; i < kWords; ++i) w[i] = src.word(i);
  }
  // Nibble n of a row (runtime n; selects instead of indexing).
  static RS_HD uint32_t nibble(const uint32_t* r, int n) {
    uint32_t v = r[0];
#pragma unroll
    for (int q = 1; q < kRowWords; ++q) v = ((n >> 3) == q) ? r[q] : v;
    return (v >> ((n & 7) * 4)) & 15u;
  }
  // Words of row t (runtime t; selects instead of indexing so that w stays
  // in registers).
  RS_HD void row(int t, uint32_t* r) const {
#pragma unroll
    for (int q = 0; q < kRowWords; ++q) {
      uint32_t v = w[q];
#pragma unroll
      for (int u = 1; u < M; ++u) v = (t == u) ? w[u * kRowWords + q] : v;
      r[q] = v;
    }
  }
};

// y ^= sum of S[i] over the set bits i of V (V < 2^NS), with y in rotation
// ROT (logical plane b in register (b - ROT) mod W) and S in natural order.
// P holds the pair sums S[0]^S[1] and S[2]^S[3], so any subset of four is
// at most two terms and every plane costs one 3-input XOR.
template <int W, int ROT, int NS, int V>
RS_HD void xor_subset(uint32_t* y, const uint32_t (*S)[W], const uint32_t (*P)[W]) {
  constexpr int lo = V & 3, hi = (V >> 2) & 3;
#pragma unroll
  for (int b = 0; b < W; ++b) {
    uint32_t z = y[((b - ROT) % W + W) % W];
    if constexpr (lo == 1) z ^= S[0][b];
    if constexpr (lo == 2) z ^= S[1][b];
    if constexpr (lo == 3) z ^= P[0][b];
    if constexpr (hi == 1) z ^= S[2][b];
    if constexpr (hi == 2) z ^= S[3][b];
    if constexpr (hi == 3) z ^= P[1][b];
    y[((b - ROT) % W + W) % W] = z;
  }
}

RS_CHD constexpr int rotated(int b, int rot, int w) { return ((b - rot) % w + w) % w; }

#if defined(__CUDA_ARCH__)

// GF(2^8) form of xor_selected with a warp-uniform jump table (brx.idx.uni)
// over the 16 selector values; written out because the compiler lowers the
// switch to a tree of compares.  Operand order: y planes %0-%7 (logical,
// so the rotation is in the operand list), S0..S3 %8-%39, the pair sums
// %40-%55, sel %56.  Operands of syndromes beyond NS feed only unreachable
// cases and are bound to S0.
template <int ROT, int NS>
__device__ __forceinline__ void xor_selected_w8(uint32_t sel, uint32_t* y, const uint32_t (*S)[8],
                                                const uint32_t (*P)[8]) {
  const uint32_t* s0 = S[0];
  const uint32_t* s1 = NS > 1 ? S[1] : S[0];
  const uint32_t* s2 = NS > 2 ? S[2] : S[0];
  const uint32_t* s3 = NS > 3 ? S[3] : S[0];
  const uint32_t* p0 = NS > 1 ? P[0] : S[0];
  const uint32_t* p1 = NS > 3 ? P[1] : S[0];
  asm("{\n\t"
      "ts: .branchtargets L0, L1, L2, L3, L4, L5, L6, L7, L8, L9, L10, L11, L12, L13, L14, L15;\n\t"
      "brx.idx.uni %56, ts;\n"
      "L0: bra.uni END;\n"
      "L1: xor.b32 %0, %0, %8; xor.b32 %1, %1, %9; xor.b32 %2, %2, %10; xor.b32 %3, %3, %11; xor.b32 %4, %4, %12; xor.b32 %5, %5, %13; xor.b32 %6, %6, %14; xor.b32 %7, %7, %15; bra.uni END;\n"
      "L2: xor.b32 %0, %0, %16; xor.b32 %1, %1, %17; xor.b32 %2, %2, %18; xor.b32 %3, %3, %19; xor.b32 %4, %4, %20; xor.b32 %5, %5, %21; xor.b32 %6, %6, %22; xor.b32 %7, %7, %23; bra.uni END;\n"
      "L3: xor.b32 %0, %0, %40; xor.b32 %1, %1, %41; xor.b32 %2, %2, %42; xor.b32 %3, %3, %43; xor.b32 %4, %4, %44; xor.b32 %5, %5, %45; xor.b32 %6, %6, %46; xor.b32 %7, %7, %47; bra.uni END;\n"
      "L4: xor.b32 %0, %0, %24; xor.b32 %1, %1, %25; xor.b32 %2, %2, %26; xor.b32 %3, %3, %27; xor.b32 %4, %4, %28; xor.b32 %5, %5, %29; xor.b32 %6, %6, %30; xor.b32 %7, %7, %31; bra.uni END;\n"
      "L5: lop3.b32 %0, %0, %8, %24, 0x96; lop3.b32 %1, %1, %9, %25, 0x96; lop3.b32 %2, %2, %10, %26, 0x96; lop3.b32 %3, %3, %11, %27, 0x96; lop3.b32 %4, %4, %12, %28, 0x96; lop3.b32 %5, %5, %13, %29, 0x96; lop3.b32 %6, %6, %14, %30, 0x96; lop3.b32 %7, %7, %15, %31, 0x96; bra.uni END;\n"
      "L6: lop3.b32 %0, %0, %16, %24, 0x96; lop3.b32 %1, %1, %17, %25, 0x96; lop3.b32 %2, %2, %18, %26, 0x96; lop3.b32 %3, %3, %19, %27, 0x96; lop3.b32 %4, %4, %20, %28, 0x96; lop3.b32 %5, %5, %21, %29, 0x96; lop3.b32 %6, %6, %22, %30, 0x96; lop3.b32 %7, %7, %23, %31, 0x96; bra.uni END;\n"
      "L7: lop3.b32 %0, %0, %40, %24, 0x96; lop3.b32 %1, %1, %41, %25, 0x96; lop3.b32 %2, %2, %42, %26, 0x96; lop3.b32 %3, %3, %43, %27, 0x96; lop3.b32 %4, %4, %44, %28, 0x96; lop3.b32 %5, %5, %45, %29, 0x96; lop3.b32 %6, %6, %46, %30, 0x96; lop3.b32 %7, %7, %47, %31, 0x96; bra.uni END;\n"
      "L8: xor.b32 %0, %0, %32; xor.b32 %1, %1, %33; xor.b32 %2, %2, %34; xor.b32 %3, %3, %35; xor.b32 %4, %4, %36; xor.b32 %5, %5, %37; xor.b32 %6, %6, %38; xor.b32 %7, %7, %39; bra.uni END;\n"
      "L9: lop3.b32 %0, %0, %8, %32, 0x96; lop3.b32 %1, %1, %9, %33, 0x96; lop3.b32 %2, %2, %10, %34, 0x96; lop3.b32 %3, %3, %11, %35, 0x96; lop3.b32 %4, %4, %12, %36, 0x96; lop3.b32 %5, %5, %13, %37, 0x96; lop3.b32 %6, %6, %14, %38, 0x96; lop3.b32 %7, %7, %15, %39, 0x96; bra.uni END;\n"
      "L10: lop3.b32 %0, %0, %16, %32, 0x96; lop3.b32 %1, %1, %17, %33, 0x96; lop3.b32 %2, %2, %18, %34, 0x96; lop3.b32 %3, %3, %19, %35, 0x96; lop3.b32 %4, %4, %20, %36, 0x96; lop3.b32 %5, %5, %21, %37, 0x96; lop3.b32 %6, %6, %22, %38, 0x96; lop3.b32 %7, %7, %23, %39, 0x96; bra.uni END;\n"
      "L11: lop3.b32 %0, %0, %40, %32, 0x96; lop3.b32 %1, %1, %41, %33, 0x96; lop3.b32 %2, %2, %42, %34, 0x96; lop3.b32 %3, %3, %43, %35, 0x96; lop3.b32 %4, %4, %44, %36, 0x96; lop3.b32 %5, %5, %45, %37, 0x96; lop3.b32 %6, %6, %46, %38, 0x96; lop3.b32 %7, %7, %47, %39, 0x96; bra.uni END;\n"
      "L12: xor.b32 %0, %0, %48; xor.b32 %1, %1, %49; xor.b32 %2, %2, %50; xor.b32 %3, %3, %51; xor.b32 %4, %4, %52; xor.b32 %5, %5, %53; xor.b32 %6, %6, %54; xor.b32 %7, %7, %55; bra.uni END;\n"
      "L13: lop3.b32 %0, %0, %8, %48, 0x96; lop3.b32 %1, %1, %9, %49, 0x96; lop3.b32 %2, %2, %10, %50, 0x96; lop3.b32 %3, %3, %11, %51, 0x96; lop3.b32 %4, %4, %12, %52, 0x96; lop3.b32 %5, %5, %13, %53, 0x96; lop3.b32 %6, %6, %14, %54, 0x96; lop3.b32 %7, %7, %15, %55, 0x96; bra.uni END;\n"
      "L14: lop3.b32 %0, %0, %16, %48, 0x96; lop3.b32 %1, %1, %17, %49, 0x96; lop3.b32 %2, %2, %18, %50, 0x96; lop3.b32 %3, %3, %19, %51, 0x96; lop3.b32 %4, %4, %20, %52, 0x96; lop3.b32 %5, %5, %21, %53, 0x96; lop3.b32 %6, %6, %22, %54, 0x96; lop3.b32 %7, %7, %23, %55, 0x96; bra.uni END;\n"
      "L15: lop3.b32 %0, %0, %40, %48, 0x96; lop3.b32 %1, %1, %41, %49, 0x96; lop3.b32 %2, %2, %42, %50, 0x96; lop3.b32 %3, %3, %43, %51, 0x96; lop3.b32 %4, %4, %44, %52, 0x96; lop3.b32 %5, %5, %45, %53, 0x96; lop3.b32 %6, %6, %46, %54, 0x96; lop3.b32 %7, %7, %47, %55, 0x96;\n"
      "END:\n\t}"
      : "+r"(y[rotated(0, ROT, 8)]), "+r"(y[rotated(1, ROT, 8)]), "+r"(y[rotated(2, ROT, 8)]),
        "+r"(y[rotated(3, ROT, 8)]), "+r"(y[rotated(4, ROT, 8)]), "+r"(y[rotated(5, ROT, 8)]),
        "+r"(y[rotated(6, ROT, 8)]), "+r"(y[rotated(7, ROT, 8)])
      : "r"(s0[0]), "r"(s0[1]), "r"(s0[2]), "r"(s0[3]), "r"(s0[4]), "r"(s0[5]), "r"(s0[6]), "r"(s0[7]),
        "r"(s1[0]), "r"(s1[1]), "r"(s1[2]), "r"(s1[3]), "r"(s1[4]), "r"(s1[5]), "r"(s1[6]), "r"(s1[7]),
        "r"(s2[0]), "r"(s2[1]), "r"(s2[2]), "r"(s2[3]), "r"(s2[4]), "r"(s2[5]), "r"(s2[6]), "r"(s2[7]),
        "r"(s3[0]), "r"(s3[1]), "r"(s3[2]), "r"(s3[3]), "r"(s3[4]), "r"(s3[5]), "r"(s3[6]), "r"(s3[7]),
        "r"(p0[0]), "r"(p0[1]), "r"(p0[2]), "r"(p0[3]), "r"(p0[4]), "r"(p0[5]), "r"(p0[6]), "r"(p0[7]),
        "r"(p1[0]), "r"(p1[1]), "r"(p1[2]), "r"(p1[3]), "r"(p1[4]), "r"(p1[5]), "r"(p1[6]), "r"(p1[7]),
        "r"(sel));
}
// GF(2^16) form: 16 y planes %0-%15 (logical order), S0..S3 %16-%79, sel %80;
// no pair sums (registers), so three- and four-term cases take two
// instructions per plane.
template <int ROT, int NS>
__device__ __forceinline__ void xor_selected_w16(uint32_t sel, uint32_t* y, const uint32_t (*S)[16]) {
  const uint32_t* s0 = S[0];
  const uint32_t* s1 = NS > 1 ? S[1] : S[0];
  const uint32_t* s2 = NS > 2 ? S[2] : S[0];
  const uint32_t* s3 = NS > 3 ? S[3] : S[0];
  asm("{\n\t"
      "ts: .branchtargets L0, L1, L2, L3, L4, L5, L6, L7, L8, L9, L10, L11, L12, L13, L14, L15;\n\t"
      "brx.idx.uni %80, ts;\n"
      "L0: bra.uni END;\n"
      "L1: xor.b32 %0, %0, %16; xor.b32 %1, %1, %17; xor.b32 %2, %2, %18; xor.b32 %3, %3, %19; xor.b32 %4, %4, %20; xor.b32 %5, %5, %21; xor.b32 %6, %6, %22; xor.b32 %7, %7, %23; xor.b32 %8, %8, %24; xor.b32 %9, %9, %25; xor.b32 %10, %10, %26; xor.b32 %11, %11, %27; xor.b32 %12, %12, %28; xor.b32 %13, %13, %29; xor.b32 %14, %14, %30; xor.b32 %15, %15, %31; bra.uni END;\n"
      "L2: xor.b32 %0, %0, %32; xor.b32 %1, %1, %33; xor.b32 %2, %2, %34; xor.b32 %3, %3, %35; xor.b32 %4, %4, %36; xor.b32 %5, %5, %37; xor.b32 %6, %6, %38; xor.b32 %7, %7, %39; xor.b32 %8, %8, %40; xor.b32 %9, %9, %41; xor.b32 %10, %10, %42; xor.b32 %11, %11, %43; xor.b32 %12, %12, %44; xor.b32 %13, %13, %45; xor.b32 %14, %14, %46; xor.b32 %15, %15, %47; bra.uni END;\n"
      "L3: lop3.b32 %0, %0, %16, %32, 0x96; lop3.b32 %1, %1, %17, %33, 0x96; lop3.b32 %2, %2, %18, %34, 0x96; lop3.b32 %3, %3, %19, %35, 0x96; lop3.b32 %4, %4, %20, %36, 0x96; lop3.b32 %5, %5, %21, %37, 0x96; lop3.b32 %6, %6, %22, %38, 0x96; lop3.b32 %7, %7, %23, %39, 0x96; lop3.b32 %8, %8, %24, %40, 0x96; lop3.b32 %9, %9, %25, %41, 0x96; lop3.b32 %10, %10, %26, %42, 0x96; lop3.b32 %11, %11, %27, %43, 0x96; lop3.b32 %12, %12, %28, %44, 0x96; lop3.b32 %13, %13, %29, %45, 0x96; lop3.b32 %14, %14, %30, %46, 0x96; lop3.b32 %15, %15, %31, %47, 0x96; bra.uni END;\n"
      "L4: xor.b32 %0, %0, %48; xor.b32 %1, %1, %49; xor.b32 %2, %2, %50; xor.b32 %3, %3, %51; xor.b32 %4, %4, %52; xor.b32 %5, %5, %53; xor.b32 %6, %6, %54; xor.b32 %7, %7, %55; xor.b32 %8, %8, %56; xor.b32 %9, %9, %57; xor.b32 %10, %10, %58; xor.b32 %11, %11, %59; xor.b32 %12, %12, %60; xor.b32 %13, %13, %61; xor.b32 %14, %14, %62; xor.b32 %15, %15, %63; bra.uni END;\n"
      "L5: lop3.b32 %0, %0, %16, %48, 0x96; lop3.b32 %1, %1, %17, %49, 0x96; lop3.b32 %2, %2, %18, %50, 0x96; lop3.b32 %3, %3, %19, %51, 0x96; lop3.b32 %4, %4, %20, %52, 0x96; lop3.b32 %5, %5, %21, %53, 0x96; lop3.b32 %6, %6, %22, %54, 0x96; lop3.b32 %7, %7, %23, %55, 0x96; lop3.b32 %8, %8, %24, %56, 0x96; lop3.b32 %9, %9, %25, %57, 0x96; lop3.b32 %10, %10, %26, %58, 0x96; lop3.b32 %11, %11, %27, %59, 0x96; lop3.b32 %12, %12, %28, %60, 0x96; lop3.b32 %13, %13, %29, %61, 0x96; lop3.b32 %14, %14, %30, %62, 0x96; lop3.b32 %15, %15, %31, %63, 0x96; bra.uni END;\n"
      "L6: lop3.b32 %0, %0, %32, %48, 0x96; lop3.b32 %1, %1, %33, %49, 0x96; lop3.b32 %2, %2, %34, %50, 0x96; lop3.b32 %3, %3, %35, %51, 0x96; lop3.b32 %4, %4, %36, %52, 0x96; lop3.b32 %5, %5, %37, %53, 0x96; lop3.b32 %6, %6, %38, %54, 0x96; lop3.b32 %7, %7, %39, %55, 0x96; lop3.b32 %8, %8, %40, %56, 0x96; lop3.b32 %9, %9, %41, %57, 0x96; lop3.b32 %10, %10, %42, %58, 0x96; lop3.b32 %11, %11, %43, %59, 0x96; lop3.b32 %12, %12, %44, %60, 0x96; lop3.b32 %13, %13, %45, %61, 0x96; lop3.b32 %14, %14, %46, %62, 0x96; lop3.b32 %15, %15, %47, %63, 0x96; bra.uni END;\n"
      "L7: lop3.b32 %0, %0, %16, %32, 0x96; xor.b32 %0, %0, %48; lop3.b32 %1, %1, %17, %33, 0x96; xor.b32 %1, %1, %49; lop3.b32 %2, %2, %18, %34, 0x96; xor.b32 %2, %2, %50; lop3.b32 %3, %3, %19, %35, 0x96; xor.b32 %3, %3, %51; lop3.b32 %4, %4, %20, %36, 0x96; xor.b32 %4, %4, %52; lop3.b32 %5, %5, %21, %37, 0x96; xor.b32 %5, %5, %53; lop3.b32 %6, %6, %22, %38, 0x96; xor.b32 %6, %6, %54; lop3.b32 %7, %7, %23, %39, 0x96; xor.b32 %7, %7, %55; lop3.b32 %8, %8, %24, %40, 0x96; xor.b32 %8, %8, %56; lop3.b32 %9, %9, %25, %41, 0x96; xor.b32 %9, %9, %57; lop3.b32 %10, %10, %26, %42, 0x96; xor.b32 %10, %10, %58; lop3.b32 %11, %11, %27, %43, 0x96; xor.b32 %11, %11, %59; lop3.b32 %12, %12, %28, %44, 0x96; xor.b32 %12, %12, %60; lop3.b32 %13, %13, %29, %45, 0x96; xor.b32 %13, %13, %61; lop3.b32 %14, %14, %30, %46, 0x96; xor.b32 %14, %14, %62; lop3.b32 %15, %15, %31, %47, 0x96; xor.b32 %15, %15, %63; bra.uni END;\n"
      "L8: xor.b32 %0, %0, %64; xor.b32 %1, %1, %65; xor.b32 %2, %2, %66; xor.b32 %3, %3, %67; xor.b32 %4, %4, %68; xor.b32 %5, %5, %69; xor.b32 %6, %6, %70; xor.b32 %7, %7, %71; xor.b32 %8, %8, %72; xor.b32 %9, %9, %73; xor.b32 %10, %10, %74; xor.b32 %11, %11, %75; xor.b32 %12, %12, %76; xor.b32 %13, %13, %77; xor.b32 %14, %14, %78; xor.b32 %15, %15, %79; bra.uni END;\n"
      "L9: lop3.b32 %0, %0, %16, %64, 0x96; lop3.b32 %1, %1, %17, %65, 0x96; lop3.b32 %2, %2, %18, %66, 0x96; lop3.b32 %3, %3, %19, %67, 0x96; lop3.b32 %4, %4, %20, %68, 0x96; lop3.b32 %5, %5, %21, %69, 0x96; lop3.b32 %6, %6, %22, %70, 0x96; lop3.b32 %7, %7, %23, %71, 0x96; lop3.b32 %8, %8, %24, %72, 0x96; lop3.b32 %9, %9, %25, %73, 0x96; lop3.b32 %10, %10, %26, %74, 0x96; lop3.b32 %11, %11, %27, %75, 0x96; lop3.b32 %12, %12, %28, %76, 0x96; lop3.b32 %13, %13, %29, %77, 0x96; lop3.b32 %14, %14, %30, %78, 0x96; lop3.b32 %15, %15, %31, %79, 0x96; bra.uni END;\n"
      "L10: lop3.b32 %0, %0, %32, %64, 0x96; lop3.b32 %1, %1, %33, %65, 0x96; lop3.b32 %2, %2, %34, %66, 0x96; lop3.b32 %3, %3, %35, %67, 0x96; lop3.b32 %4, %4, %36, %68, 0x96; lop3.b32 %5, %5, %37, %69, 0x96; lop3.b32 %6, %6, %38, %70, 0x96; lop3.b32 %7, %7, %39, %71, 0x96; lop3.b32 %8, %8, %40, %72, 0x96; lop3.b32 %9, %9, %41, %73, 0x96; lop3.b32 %10, %10, %42, %74, 0x96; lop3.b32 %11, %11, %43, %75, 0x96; lop3.b32 %12, %12, %44, %76, 0x96; lop3.b32 %13, %13, %45, %77, 0x96; lop3.b32 %14, %14, %46, %78, 0x96; lop3.b32 %15, %15, %47, %79, 0x96; bra.uni END;\n"
      "L11: lop3.b32 %0, %0, %16, %32, 0x96; xor.b32 %0, %0, %64; lop3.b32 %1, %1, %17, %33, 0x96; xor.b32 %1, %1, %65; lop3.b32 %2, %2, %18, %34, 0x96; xor.b32 %2, %2, %66; lop3.b32 %3, %3, %19, %35, 0x96; xor.b32 %3, %3, %67; lop3.b32 %4, %4, %20, %36, 0x96; xor.b32 %4, %4, %68; lop3.b32 %5, %5, %21, %37, 0x96; xor.b32 %5, %5, %69; lop3.b32 %6, %6, %22, %38, 0x96; xor.b32 %6, %6, %70; lop3.b32 %7, %7, %23, %39, 0x96; xor.b32 %7, %7, %71; lop3.b32 %8, %8, %24, %40, 0x96; xor.b32 %8, %8, %72; lop3.b32 %9, %9, %25, %41, 0x96; xor.b32 %9, %9, %73; lop3.b32 %10, %10, %26, %42, 0x96; xor.b32 %10, %10, %74; lop3.b32 %11, %11, %27, %43, 0x96; xor.b32 %11, %11, %75; lop3.b32 %12, %12, %28, %44, 0x96; xor.b32 %12, %12, %76; lop3.b32 %13, %13, %29, %45, 0x96; xor.b32 %13, %13, %77; lop3.b32 %14, %14, %30, %46, 0x96; xor.b32 %14, %14, %78; lop3.b32 %15, %15, %31, %47, 0x96; xor.b32 %15, %15, %79; bra.uni END;\n"
      "L12: lop3.b32 %0, %0, %48, %64, 0x96; lop3.b32 %1, %1, %49, %65, 0x96; lop3.b32 %2, %2, %50, %66, 0x96; lop3.b32 %3, %3, %51, %67, 0x96; lop3.b32 %4, %4, %52, %68, 0x96; lop3.b32 %5, %5, %53, %69, 0x96; lop3.b32 %6, %6, %54, %70, 0x96; lop3.b32 %7, %7, %55, %71, 0x96; lop3.b32 %8, %8, %56, %72, 0x96; lop3.b32 %9, %9, %57, %73, 0x96; lop3.b32 %10, %10, %58, %74, 0x96; lop3.b32 %11, %11, %59, %75, 0x96; lop3.b32 %12, %12, %60, %76, 0x96; lop3.b32 %13, %13, %61, %77, 0x96; lop3.b32 %14, %14, %62, %78, 0x96; lop3.b32 %15, %15, %63, %79, 0x96; bra.uni END;\n"
      "L13: lop3.b32 %0, %0, %16, %48, 0x96; xor.b32 %0, %0, %64; lop3.b32 %1, %1, %17, %49, 0x96; xor.b32 %1, %1, %65; lop3.b32 %2, %2, %18, %50, 0x96; xor.b32 %2, %2, %66; lop3.b32 %3, %3, %19, %51, 0x96; xor.b32 %3, %3, %67; lop3.b32 %4, %4, %20, %52, 0x96; xor.b32 %4, %4, %68; lop3.b32 %5, %5, %21, %53, 0x96; xor.b32 %5, %5, %69; lop3.b32 %6, %6, %22, %54, 0x96; xor.b32 %6, %6, %70; lop3.b32 %7, %7, %23, %55, 0x96; xor.b32 %7, %7, %71; lop3.b32 %8, %8, %24, %56, 0x96; xor.b32 %8, %8, %72; lop3.b32 %9, %9, %25, %57, 0x96; xor.b32 %9, %9, %73; lop3.b32 %10, %10, %26, %58, 0x96; xor.b32 %10, %10, %74; lop3.b32 %11, %11, %27, %59, 0x96; xor.b32 %11, %11, %75; lop3.b32 %12, %12, %28, %60, 0x96; xor.b32 %12, %12, %76; lop3.b32 %13, %13, %29, %61, 0x96; xor.b32 %13, %13, %77; lop3.b32 %14, %14, %30, %62, 0x96; xor.b32 %14, %14, %78; lop3.b32 %15, %15, %31, %63, 0x96; xor.b32 %15, %15, %79; bra.uni END;\n"
      "L14: lop3.b32 %0, %0, %32, %48, 0x96; xor.b32 %0, %0, %64; lop3.b32 %1, %1, %33, %49, 0x96; xor.b32 %1, %1, %65; lop3.b32 %2, %2, %34, %50, 0x96; xor.b32 %2, %2, %66; lop3.b32 %3, %3, %35, %51, 0x96; xor.b32 %3, %3, %67; lop3.b32 %4, %4, %36, %52, 0x96; xor.b32 %4, %4, %68; lop3.b32 %5, %5, %37, %53, 0x96; xor.b32 %5, %5, %69; lop3.b32 %6, %6, %38, %54, 0x96; xor.b32 %6, %6, %70; lop3.b32 %7, %7, %39, %55, 0x96; xor.b32 %7, %7, %71; lop3.b32 %8, %8, %40, %56, 0x96; xor.b32 %8, %8, %72; lop3.b32 %9, %9, %41, %57, 0x96; xor.b32 %9, %9, %73; lop3.b32 %10, %10, %42, %58, 0x96; xor.b32 %10, %10, %74; lop3.b32 %11, %11, %43, %59, 0x96; xor.b32 %11, %11, %75; lop3.b32 %12, %12, %44, %60, 0x96; xor.b32 %12, %12, %76; lop3.b32 %13, %13, %45, %61, 0x96; xor.b32 %13, %13, %77; lop3.b32 %14, %14, %46, %62, 0x96; xor.b32 %14, %14, %78; lop3.b32 %15, %15, %47, %63, 0x96; xor.b32 %15, %15, %79; bra.uni END;\n"
      "L15: lop3.b32 %0, %0, %16, %32, 0x96; lop3.b32 %0, %0, %48, %64, 0x96; lop3.b32 %1, %1, %17, %33, 0x96; lop3.b32 %1, %1, %49, %65, 0x96; lop3.b32 %2, %2, %18, %34, 0x96; lop3.b32 %2, %2, %50, %66, 0x96; lop3.b32 %3, %3, %19, %35, 0x96; lop3.b32 %3, %3, %51, %67, 0x96; lop3.b32 %4, %4, %20, %36, 0x96; lop3.b32 %4, %4, %52, %68, 0x96; lop3.b32 %5, %5, %21, %37, 0x96; lop3.b32 %5, %5, %53, %69, 0x96; lop3.b32 %6, %6, %22, %38, 0x96; lop3.b32 %6, %6, %54, %70, 0x96; lop3.b32 %7, %7, %23, %39, 0x96; lop3.b32 %7, %7, %55, %71, 0x96; lop3.b32 %8, %8, %24, %40, 0x96; lop3.b32 %8, %8, %56, %72, 0x96; lop3.b32 %9, %9, %25, %41, 0x96; lop3.b32 %9, %9, %57, %73, 0x96; lop3.b32 %10, %10, %26, %42, 0x96; lop3.b32 %10, %10, %58, %74, 0x96; lop3.b32 %11, %11, %27, %43, 0x96; lop3.b32 %11, %11, %59, %75, 0x96; lop3.b32 %12, %12, %28, %44, 0x96; lop3.b32 %12, %12, %60, %76, 0x96; lop3.b32 %13, %13, %29, %45, 0x96; lop3.b32 %13, %13, %61, %77, 0x96; lop3.b32 %14, %14, %30, %46, 0x96; lop3.b32 %14, %14, %62, %78, 0x96; lop3.b32 %15, %15, %31, %47, 0x96; lop3.b32 %15, %15, %63, %79, 0x96;\n"
      "END:\n\t}"
      : "+r"(y[rotated(0, ROT, 16)]), "+r"(y[rotated(1, ROT, 16)]), "+r"(y[rotated(2, ROT, 16)]), "+r"(y[rotated(3, ROT, 16)]),
        "+r"(y[rotated(4, ROT, 16)]), "+r"(y[rotated(5, ROT, 16)]), "+r"(y[rotated(6, ROT, 16)]), "+r"(y[rotated(7, ROT, 16)]),
        "+r"(y[rotated(8, ROT, 16)]), "+r"(y[rotated(9, ROT, 16)]), "+r"(y[rotated(10, ROT, 16)]), "+r"(y[rotated(11, ROT, 16)]),
        "+r"(y[rotated(12, ROT, 16)]), "+r"(y[rotated(13, ROT, 16)]), "+r"(y[rotated(14, ROT, 16)]), "+r"(y[rotated(15, ROT, 16)])
      : "r"(s0[0]), "r"(s0[1]), "r"(s0[2]), "r"(s0[3]), "r"(s0[4]), "r"(s0[5]), "r"(s0[6]), "r"(s0[7]),
        "r"(s0[8]), "r"(s0[9]), "r"(s0[10]), "r"(s0[11]), "r"(s0[12]), "r"(s0[13]), "r"(s0[14]), "r"(s0[15]),
        "r"(s1[0]), "r"(s1[1]), "r"(s1[2]), "r"(s1[3]), "r"(s1[4]), "r"(s1[5]), "r"(s1[6]), "r"(s1[7]),
        "r"(s1[8]), "r"(s1[9]), "r"(s1[10]), "r"(s1[11]), "r"(s1[12]), "r"(s1[13]), "r"(s1[14]), "r"(s1[15]),
        "r"(s2[0]), "r"(s2[1]), "r"(s2[2]), "r"(s2[3]), "r"(s2[4]), "r"(s2[5]), "r"(s2[6]), "r"(s2[7]),
        "r"(s2[8]), "r"(s2[9]), "r"(s2[10]), "r"(s2[11]), "r"(s2[12]), "r"(s2[13]), "r"(s2[14]), "r"(s2[15]),
        "r"(s3[0]), "r"(s3[1]), "r"(s3[2]), "r"(s3[3]), "r"(s3[4]), "r"(s3[5]), "r"(s3[6]), "r"(s3[7]),
        "r"(s3[8]), "r"(s3[9]), "r"(s3[10]), "r"(s3[11]), "r"(s3[12]), "r"(s3[13]), "r"(s3[14]), "r"(s3[15]),
        "r"(sel));
}
#endif

#if defined(__CUDA_ARCH__)
// Two 32-column groups at once (GF(2^8), no pair sums): y0 %0-%7 and y1
// %8-%15 (logical planes), the four syndromes of group 0 %16-%47 and of
// group 1 %48-%79, sel %80.  Operands of syndromes beyond NS feed only
// unreachable cases and are bound to syndrome 0.
template <int ROT, int NS>
__device__ __forceinline__ void xor_selected2_w8(uint32_t sel, uint32_t* y0, uint32_t* y1, const uint32_t (*A)[8],
                                                 const uint32_t (*B)[8]) {
  const uint32_t *a0 = A[0], *a1 = NS > 1 ? A[1] : A[0], *a2 = NS > 2 ? A[2] : A[0], *a3 = NS > 3 ? A[3] : A[0];
  const uint32_t *b0 = B[0], *b1 = NS > 1 ? B[1] : B[0], *b2 = NS > 2 ? B[2] : B[0], *b3 = NS > 3 ? B[3] : B[0];
  asm("{\n\t"
      "ts: .branchtargets L0, L1, L2, L3, L4, L5, L6, L7, L8, L9, L10, L11, L12, L13, L14, L15;\n\t"
      "brx.idx.uni %80, ts;\n"
      "L0: bra.uni END;\n"
      "L1: xor.b32 %0, %0, %16; xor.b32 %1, %1, %17; xor.b32 %2, %2, %18; xor.b32 %3, %3, %19; xor.b32 %4, %4, %20; xor.b32 %5, %5, %21; xor.b32 %6, %6, %22; xor.b32 %7, %7, %23; xor.b32 %8, %8, %48; xor.b32 %9, %9, %49; xor.b32 %10, %10, %50; xor.b32 %11, %11, %51; xor.b32 %12, %12, %52; xor.b32 %13, %13, %53; xor.b32 %14, %14, %54; xor.b32 %15, %15, %55; bra.uni END;\n"
      "L2: xor.b32 %0, %0, %24; xor.b32 %1, %1, %25; xor.b32 %2, %2, %26; xor.b32 %3, %3, %27; xor.b32 %4, %4, %28; xor.b32 %5, %5, %29; xor.b32 %6, %6, %30; xor.b32 %7, %7, %31; xor.b32 %8, %8, %56; xor.b32 %9, %9, %57; xor.b32 %10, %10, %58; xor.b32 %11, %11, %59; xor.b32 %12, %12, %60; xor.b32 %13, %13, %61; xor.b32 %14, %14, %62; xor.b32 %15, %15, %63; bra.uni END;\n"
      "L3: lop3.b32 %0, %0, %16, %24, 0x96; lop3.b32 %1, %1, %17, %25, 0x96; lop3.b32 %2, %2, %18, %26, 0x96; lop3.b32 %3, %3, %19, %27, 0x96; lop3.b32 %4, %4, %20, %28, 0x96; lop3.b32 %5, %5, %21, %29, 0x96; lop3.b32 %6, %6, %22, %30, 0x96; lop3.b32 %7, %7, %23, %31, 0x96; lop3.b32 %8, %8, %48, %56, 0x96; lop3.b32 %9, %9, %49, %57, 0x96; lop3.b32 %10, %10, %50, %58, 0x96; lop3.b32 %11, %11, %51, %59, 0x96; lop3.b32 %12, %12, %52, %60, 0x96; lop3.b32 %13, %13, %53, %61, 0x96; lop3.b32 %14, %14, %54, %62, 0x96; lop3.b32 %15, %15, %55, %63, 0x96; bra.uni END;\n"
      "L4: xor.b32 %0, %0, %32; xor.b32 %1, %1, %33; xor.b32 %2, %2, %34; xor.b32 %3, %3, %35; xor.b32 %4, %4, %36; xor.b32 %5, %5, %37; xor.b32 %6, %6, %38; xor.b32 %7, %7, %39; xor.b32 %8, %8, %64; xor.b32 %9, %9, %65; xor.b32 %10, %10, %66; xor.b32 %11, %11, %67; xor.b32 %12, %12, %68; xor.b32 %13, %13, %69; xor.b32 %14, %14, %70; xor.b32 %15, %15, %71; bra.uni END;\n"
      "L5: lop3.b32 %0, %0, %16, %32, 0x96; lop3.b32 %1, %1, %17, %33, 0x96; lop3.b32 %2, %2, %18, %34, 0x96; lop3.b32 %3, %3, %19, %35, 0x96; lop3.b32 %4, %4, %20, %36, 0x96; lop3.b32 %5, %5, %21, %37, 0x96; lop3.b32 %6, %6, %22, %38, 0x96; lop3.b32 %7, %7, %23, %39, 0x96; lop3.b32 %8, %8, %48, %64, 0x96; lop3.b32 %9, %9, %49, %65, 0x96; lop3.b32 %10, %10, %50, %66, 0x96; lop3.b32 %11, %11, %51, %67, 0x96; lop3.b32 %12, %12, %52, %68, 0x96; lop3.b32 %13, %13, %53, %69, 0x96; lop3.b32 %14, %14, %54, %70, 0x96; lop3.b32 %15, %15, %55, %71, 0x96; bra.uni END;\n"
      "L6: lop3.b32 %0, %0, %24, %32, 0x96; lop3.b32 %1, %1, %25, %33, 0x96; lop3.b32 %2, %2, %26, %34, 0x96; lop3.b32 %3, %3, %27, %35, 0x96; lop3.b32 %4, %4, %28, %36, 0x96; lop3.b32 %5, %5, %29, %37, 0x96; lop3.b32 %6, %6, %30, %38, 0x96; lop3.b32 %7, %7, %31, %39, 0x96; lop3.b32 %8, %8, %56, %64, 0x96; lop3.b32 %9, %9, %57, %65, 0x96; lop3.b32 %10, %10, %58, %66, 0x96; lop3.b32 %11, %11, %59, %67, 0x96; lop3.b32 %12, %12, %60, %68, 0x96; lop3.b32 %13, %13, %61, %69, 0x96; lop3.b32 %14, %14, %62, %70, 0x96; lop3.b32 %15, %15, %63, %71, 0x96; bra.uni END;\n"
      "L7: lop3.b32 %0, %0, %16, %24, 0x96; xor.b32 %0, %0, %32; lop3.b32 %1, %1, %17, %25, 0x96; xor.b32 %1, %1, %33; lop3.b32 %2, %2, %18, %26, 0x96; xor.b32 %2, %2, %34; lop3.b32 %3, %3, %19, %27, 0x96; xor.b32 %3, %3, %35; lop3.b32 %4, %4, %20, %28, 0x96; xor.b32 %4, %4, %36; lop3.b32 %5, %5, %21, %29, 0x96; xor.b32 %5, %5, %37; lop3.b32 %6, %6, %22, %30, 0x96; xor.b32 %6, %6, %38; lop3.b32 %7, %7, %23, %31, 0x96; xor.b32 %7, %7, %39; lop3.b32 %8, %8, %48, %56, 0x96; xor.b32 %8, %8, %64; lop3.b32 %9, %9, %49, %57, 0x96; xor.b32 %9, %9, %65; lop3.b32 %10, %10, %50, %58, 0x96; xor.b32 %10, %10, %66; lop3.b32 %11, %11, %51, %59, 0x96; xor.b32 %11, %11, %67; lop3.b32 %12, %12, %52, %60, 0x96; xor.b32 %12, %12, %68; lop3.b32 %13, %13, %53, %61, 0x96; xor.b32 %13, %13, %69; lop3.b32 %14, %14, %54, %62, 0x96; xor.b32 %14, %14, %70; lop3.b32 %15, %15, %55, %63, 0x96; xor.b32 %15, %15, %71; bra.uni END;\n"
      "L8: xor.b32 %0, %0, %40; xor.b32 %1, %1, %41; xor.b32 %2, %2, %42; xor.b32 %3, %3, %43; xor.b32 %4, %4, %44; xor.b32 %5, %5, %45; xor.b32 %6, %6, %46; xor.b32 %7, %7, %47; xor.b32 %8, %8, %72; xor.b32 %9, %9, %73; xor.b32 %10, %10, %74; xor.b32 %11, %11, %75; xor.b32 %12, %12, %76; xor.b32 %13, %13, %77; xor.b32 %14, %14, %78; xor.b32 %15, %15, %79; bra.uni END;\n"
      "L9: lop3.b32 %0, %0, %16, %40, 0x96; lop3.b32 %1, %1, %17, %41, 0x96; lop3.b32 %2, %2, %18, %42, 0x96; lop3.b32 %3, %3, %19, %43, 0x96; lop3.b32 %4, %4, %20, %44, 0x96; lop3.b32 %5, %5, %21, %45, 0x96; lop3.b32 %6, %6, %22, %46, 0x96; lop3.b32 %7, %7, %23, %47, 0x96; lop3.b32 %8, %8, %48, %72, 0x96; lop3.b32 %9, %9, %49, %73, 0x96; lop3.b32 %10, %10, %50, %74, 0x96; lop3.b32 %11, %11, %51, %75, 0x96; lop3.b32 %12, %12, %52, %76, 0x96; lop3.b32 %13, %13, %53, %77, 0x96; lop3.b32 %14, %14, %54, %78, 0x96; lop3.b32 %15, %15, %55, %79, 0x96; bra.uni END;\n"
      "L10: lop3.b32 %0, %0, %24, %40, 0x96; lop3.b32 %1, %1, %25, %41, 0x96; lop3.b32 %2, %2, %26, %42, 0x96; lop3.b32 %3, %3, %27, %43, 0x96; lop3.b32 %4, %4, %28, %44, 0x96; lop3.b32 %5, %5, %29, %45, 0x96; lop3.b32 %6, %6, %30, %46, 0x96; lop3.b32 %7, %7, %31, %47, 0x96; lop3.b32 %8, %8, %56, %72, 0x96; lop3.b32 %9, %9, %57, %73, 0x96; lop3.b32 %10, %10, %58, %74, 0x96; lop3.b32 %11, %11, %59, %75, 0x96; lop3.b32 %12, %12, %60, %76, 0x96; lop3.b32 %13, %13, %61, %77, 0x96; lop3.b32 %14, %14, %62, %78, 0x96; lop3.b32 %15, %15, %63, %79, 0x96; bra.uni END;\n"
      "L11: lop3.b32 %0, %0, %16, %24, 0x96; xor.b32 %0, %0, %40; lop3.b32 %1, %1, %17, %25, 0x96; xor.b32 %1, %1, %41; lop3.b32 %2, %2, %18, %26, 0x96; xor.b32 %2, %2, %42; lop3.b32 %3, %3, %19, %27, 0x96; xor.b32 %3, %3, %43; lop3.b32 %4, %4, %20, %28, 0x96; xor.b32 %4, %4, %44; lop3.b32 %5, %5, %21, %29, 0x96; xor.b32 %5, %5, %45; lop3.b32 %6, %6, %22, %30, 0x96; xor.b32 %6, %6, %46; lop3.b32 %7, %7, %23, %31, 0x96; xor.b32 %7, %7, %47; lop3.b32 %8, %8, %48, %56, 0x96; xor.b32 %8, %8, %72; lop3.b32 %9, %9, %49, %57, 0x96; xor.b32 %9, %9, %73; lop3.b32 %10, %10, %50, %58, 0x96; xor.b32 %10, %10, %74; lop3.b32 %11, %11, %51, %59, 0x96; xor.b32 %11, %11, %75; lop3.b32 %12, %12, %52, %60, 0x96; xor.b32 %12, %12, %76; lop3.b32 %13, %13, %53, %61, 0x96; xor.b32 %13, %13, %77; lop3.b32 %14, %14, %54, %62, 0x96; xor.b32 %14, %14, %78; lop3.b32 %15, %15, %55, %63, 0x96; xor.b32 %15, %15, %79; bra.uni END;\n"
      "L12: lop3.b32 %0, %0, %32, %40, 0x96; lop3.b32 %1, %1, %33, %41, 0x96; lop3.b32 %2, %2, %34, %42, 0x96; lop3.b32 %3, %3, %35, %43, 0x96; lop3.b32 %4, %4, %36, %44, 0x96; lop3.b32 %5, %5, %37, %45, 0x96; lop3.b32 %6, %6, %38, %46, 0x96; lop3.b32 %7, %7, %39, %47, 0x96; lop3.b32 %8, %8, %64, %72, 0x96; lop3.b32 %9, %9, %65, %73, 0x96; lop3.b32 %10, %10, %66, %74, 0x96; lop3.b32 %11, %11, %67, %75, 0x96; lop3.b32 %12, %12, %68, %76, 0x96; lop3.b32 %13, %13, %69, %77, 0x96; lop3.b32 %14, %14, %70, %78, 0x96; lop3.b32 %15, %15, %71, %79, 0x96; bra.uni END;\n"
      "L13: lop3.b32 %0, %0, %16, %32, 0x96; xor.b32 %0, %0, %40; lop3.b32 %1, %1, %17, %33, 0x96; xor.b32 %1, %1, %41; lop3.b32 %2, %2, %18, %34, 0x96; xor.b32 %2, %2, %42; lop3.b32 %3, %3, %19, %35, 0x96; xor.b32 %3, %3, %43; lop3.b32 %4, %4, %20, %36, 0x96; xor.b32 %4, %4, %44; lop3.b32 %5, %5, %21, %37, 0x96; xor.b32 %5, %5, %45; lop3.b32 %6, %6, %22, %38, 0x96; xor.b32 %6, %6, %46; lop3.b32 %7, %7, %23, %39, 0x96; xor.b32 %7, %7, %47; lop3.b32 %8, %8, %48, %64, 0x96; xor.b32 %8, %8, %72; lop3.b32 %9, %9, %49, %65, 0x96; xor.b32 %9, %9, %73; lop3.b32 %10, %10, %50, %66, 0x96; xor.b32 %10, %10, %74; lop3.b32 %11, %11, %51, %67, 0x96; xor.b32 %11, %11, %75; lop3.b32 %12, %12, %52, %68, 0x96; xor.b32 %12, %12, %76; lop3.b32 %13, %13, %53, %69, 0x96; xor.b32 %13, %13, %77; lop3.b32 %14, %14, %54, %70, 0x96; xor.b32 %14, %14, %78; lop3.b32 %15, %15, %55, %71, 0x96; xor.b32 %15, %15, %79; bra.uni END;\n"
      "L14: lop3.b32 %0, %0, %24, %32, 0x96; xor.b32 %0, %0, %40; lop3.b32 %1, %1, %25, %33, 0x96; xor.b32 %1, %1, %41; lop3.b32 %2, %2, %26, %34, 0x96; xor.b32 %2, %2, %42; lop3.b32 %3, %3, %27, %35, 0x96; xor.b32 %3, %3, %43; lop3.b32 %4, %4, %28, %36, 0x96; xor.b32 %4, %4, %44; lop3.b32 %5, %5, %29, %37, 0x96; xor.b32 %5, %5, %45; lop3.b32 %6, %6, %30, %38, 0x96; xor.b32 %6, %6, %46; lop3.b32 %7, %7, %31, %39, 0x96; xor.b32 %7, %7, %47; lop3.b32 %8, %8, %56, %64, 0x96; xor.b32 %8, %8, %72; lop3.b32 %9, %9, %57, %65, 0x96; xor.b32 %9, %9, %73; lop3.b32 %10, %10, %58, %66, 0x96; xor.b32 %10, %10, %74; lop3.b32 %11, %11, %59, %67, 0x96; xor.b32 %11, %11, %75; lop3.b32 %12, %12, %60, %68, 0x96; xor.b32 %12, %12, %76; lop3.b32 %13, %13, %61, %69, 0x96; xor.b32 %13, %13, %77; lop3.b32 %14, %14, %62, %70, 0x96; xor.b32 %14, %14, %78; lop3.b32 %15, %15, %63, %71, 0x96; xor.b32 %15, %15, %79; bra.uni END;\n"
      "L15: lop3.b32 %0, %0, %16, %24, 0x96; lop3.b32 %0, %0, %32, %40, 0x96; lop3.b32 %1, %1, %17, %25, 0x96; lop3.b32 %1, %1, %33, %41, 0x96; lop3.b32 %2, %2, %18, %26, 0x96; lop3.b32 %2, %2, %34, %42, 0x96; lop3.b32 %3, %3, %19, %27, 0x96; lop3.b32 %3, %3, %35, %43, 0x96; lop3.b32 %4, %4, %20, %28, 0x96; lop3.b32 %4, %4, %36, %44, 0x96; lop3.b32 %5, %5, %21, %29, 0x96; lop3.b32 %5, %5, %37, %45, 0x96; lop3.b32 %6, %6, %22, %30, 0x96; lop3.b32 %6, %6, %38, %46, 0x96; lop3.b32 %7, %7, %23, %31, 0x96; lop3.b32 %7, %7, %39, %47, 0x96; lop3.b32 %8, %8, %48, %56, 0x96; lop3.b32 %8, %8, %64, %72, 0x96; lop3.b32 %9, %9, %49, %57, 0x96; lop3.b32 %9, %9, %65, %73, 0x96; lop3.b32 %10, %10, %50, %58, 0x96; lop3.b32 %10, %10, %66, %74, 0x96; lop3.b32 %11, %11, %51, %59, 0x96; lop3.b32 %11, %11, %67, %75, 0x96; lop3.b32 %12, %12, %52, %60, 0x96; lop3.b32 %12, %12, %68, %76, 0x96; lop3.b32 %13, %13, %53, %61, 0x96; lop3.b32 %13, %13, %69, %77, 0x96; lop3.b32 %14, %14, %54, %62, 0x96; lop3.b32 %14, %14, %70, %78, 0x96; lop3.b32 %15, %15, %55, %63, 0x96; lop3.b32 %15, %15, %71, %79, 0x96;\n"
      "END:\n\t}"
      : "+r"(y0[rotated(0, ROT, 8)]), "+r"(y0[rotated(1, ROT, 8)]), "+r"(y0[rotated(2, ROT, 8)]), "+r"(y0[rotated(3, ROT, 8)]), "+r"(y0[rotated(4, ROT, 8)]), "+r"(y0[rotated(5, ROT, 8)]), "+r"(y0[rotated(6, ROT, 8)]), "+r"(y0[rotated(7, ROT, 8)]),
        "+r"(y1[rotated(0, ROT, 8)]), "+r"(y1[rotated(1, ROT, 8)]), "+r"(y1[rotated(2, ROT, 8)]), "+r"(y1[rotated(3, ROT, 8)]), "+r"(y1[rotated(4, ROT, 8)]), "+r"(y1[rotated(5, ROT, 8)]), "+r"(y1[rotated(6, ROT, 8)]), "+r"(y1[rotated(7, ROT, 8)])
      : "r"(a0[0]), "r"(a0[1]), "r"(a0[2]), "r"(a0[3]), "r"(a0[4]), "r"(a0[5]), "r"(a0[6]), "r"(a0[7]),
        "r"(a1[0]), "r"(a1[1]), "r"(a1[2]), "r"(a1[3]), "r"(a1[4]), "r"(a1[5]), "r"(a1[6]), "r"(a1[7]),
        "r"(a2[0]), "r"(a2[1]), "r"(a2[2]), "r"(a2[3]), "r"(a2[4]), "r"(a2[5]), "r"(a2[6]), "r"(a2[7]),
        "r"(a3[0]), "r"(a3[1]), "r"(a3[2]), "r"(a3[3]), "r"(a3[4]), "r"(a3[5]), "r"(a3[6]), "r"(a3[7]),
        "r"(b0[0]), "r"(b0[1]), "r"(b0[2]), "r"(b0[3]), "r"(b0[4]), "r"(b0[5]), "r"(b0[6]), "r"(b0[7]),
        "r"(b1[0]), "r"(b1[1]), "r"(b1[2]), "r"(b1[3]), "r"(b1[4]), "r"(b1[5]), "r"(b1[6]), "r"(b1[7]),
        "r"(b2[0]), "r"(b2[1]), "r"(b2[2]), "r"(b2[3]), "r"(b2[4]), "r"(b2[5]), "r"(b2[6]), "r"(b2[7]),
        "r"(b3[0]), "r"(b3[1]), "r"(b3[2]), "r"(b3[3]), "r"(b3[4]), "r"(b3[5]), "r"(b3[6]), "r"(b3[7]),
        "r"(sel));
}
#endif

// y0 ^= subset of A, y1 ^= the same subset of B (two column groups), with
// y0 and y1 in rotation ROT; the subset is the 4-bit selector sel.
template <int W, int ROT, int NS>
RS_HD void xor_selected2(uint32_t sel, uint32_t* y0, uint32_t* y1, const uint32_t (*A)[W], const uint32_t (*B)[W]) {
#if defined(__CUDA_ARCH__)
  constexpr bool kTable = W == 8;
#else
  constexpr bool kTable = false;
#endif
  if constexpr (kTable) {
#if defined(__CUDA_ARCH__)
    xor_selected2_w8<ROT, NS>(sel, y0, y1, A, B);
#endif
  } else {
#pragma unroll
    for (int b = 0; b < W; ++b) {
      uint32_t z0 = 0, z1 = 0;
#pragma unroll
      for (int i = 0; i < NS; ++i)
        if ((sel >> i) & 1u) {
          z0 ^= A[i][b];
          z1 ^= B[i][b];
        }
      y0[((b - ROT) % W + W) % W] ^= z0;
      y1[((b - ROT) % W + W) % W] ^= z1;
    }
  }
}

// y ^= the subset of S[0..NS-1] named by the 4-bit selector sel.
template <int W, int ROT, int NS>
RS_HD void xor_selected(uint32_t sel, uint32_t* y, const uint32_t (*S)[W], const uint32_t (*P)[W]) {
#if defined(__CUDA_ARCH__)
  if constexpr (W == 8) {
    xor_selected_w8<ROT, NS>(sel, y, S, P);
    return;
  } else if constexpr (W == 16) {
    xor_selected_w16<ROT, NS>(sel, y, S);
    return;
  }
#endif
  switch (sel) {
#define RSGB_SELECT_CASE(v)                                           \
  case v:                                                             \
    if constexpr (v < (1 << NS)) xor_subset<W, ROT, NS, v>(y, S, P); \
    break;
    RSGB_SELECT_CASE(1)
    RSGB_SELECT_CASE(2)
    RSGB_SELECT_CASE(3)
    RSGB_SELECT_CASE(4)
    RSGB_SELECT_CASE(5)
    RSGB_SELECT_CASE(6)
    RSGB_SELECT_CASE(7)
    RSGB_SELECT_CASE(8)
    RSGB_SELECT_CASE(9)
    RSGB_SELECT_CASE(10)
    RSGB_SELECT_CASE(11)
    RSGB_SELECT_CASE(12)
    RSGB_SELECT_CASE(13)
    RSGB_SELECT_CASE(14)
    RSGB_SELECT_CASE(15)
#undef RSGB_SELECT_CASE
    default:
      break;
  }
}

}  // namespace rsgb

#include "select_gen.hpp"

namespace rsgb {

// acc[r] ^= sum_q M[r][q] * in_q ... for one input q: acc[r] ^= M[r][q] * x,
// as sum over c of mask(r, q, c) & (alpha^c x).  x is clobbered.
template <int W, int R, int Q>
RS_HD void mul_acc_packed_column(uint32_t (*acc)[W], uint32_t* x, const PackedBits<W, R, Q>& m, int q) {
#pragma unroll
  for (int c = 0; c < W; ++c) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t mk = m.mask(r, q, c);
#pragma unroll
      for (int b = 0; b < W; ++b) acc[r][b] ^= x[b] & mk;
    }
    if (c + 1 < W) mul_alpha<W>(x);
  }
}

}  // namespace rsgb
