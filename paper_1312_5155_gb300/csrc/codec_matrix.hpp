// Matrix realizations (§2), per group of 32 columns in bit-planes.
//
// Encode (§2.1): parity_i = sum_j P[i][j] d_j with P the parity rows of the
// systematic generator (Vandermonde §2.2 or Cauchy §2.3).  Inputs are the
// data blocks d_0..d_{k-1} in order.
//
// Decode: instead of inverting the k x k survivor matrix and multiplying it
// by k survivors per erased block (§2.1's four steps), the device evaluates
// the m syndromes of the parity-check matrix H = [P | I_m] over the read
// blocks,  s_i = sum_{read data j} P[i][j] d_j + (p_i if read),  which equal
// the contribution of the unknown blocks; the host inverts the small system
// once per erasure pattern and the device applies it (runtime matrix W).
// The bytes are the same as §2.1's procedure (the code is MDS, so the erased
// symbols are unique); the device work for the fixed part is the same XOR
// pattern as encoding.
//
// Two forms: compile-time P (a registered (k, m) code: every product is a
// fixed XOR pattern) and runtime P (any code: products as masked AND-XOR).
// `kTranspose` selects the symbol layout (bytes / 16-bit words, transposed
// to planes) or the packet layout (§2.3's bit-matrix layout: the W words a
// thread loads are already the planes).
#pragma once
#include "bitslice.hpp"
#include "codec_poly.hpp"
#include "job.hpp"

namespace rsgb {

// ------------------------------------------------ compile-time generators

template <int K, int M>
struct MatKM {
  uint32_t a[M][K];
};

// Entry (i, j) of a MatKM by reference (the accessor good_cauchy_scale takes).
template <int K, int M>
struct MatKMEntry {
  MatKM<K, M>& p;
  RS_CHD constexpr uint32_t& operator()(int i, int j) const { return p.a[i][j]; }
};

// Gauss-Jordan inverse over GF(2^w) of a K x K matrix, at compile time.
template <int K>
RS_CHD constexpr bool ct_invert(uint32_t (&A)[K][K], uint32_t (&R)[K][K], int w) {
  for (int i = 0; i < K; ++i)
    for (int j = 0; j < K; ++j) R[i][j] = (i == j) ? 1u : 0u;
  for (int col = 0; col < K; ++col) {
    int piv = -1;
    for (int r = col; r < K && piv < 0; ++r)
      if (A[r][col]) piv = r;
    if (piv < 0) return false;
    for (int c = 0; c < K; ++c) {
      uint32_t t = A[col][c]; A[col][c] = A[piv][c]; A[piv][c] = t;
      t = R[col][c]; R[col][c] = R[piv][c]; R[piv][c] = t;
    }
    const uint32_t iv = gf_inv(A[col][col], w);
    for (int c = 0; c < K; ++c) {
      A[col][c] = gf_mul(A[col][c], iv, w);
      R[col][c] = gf_mul(R[col][c], iv, w);
    }
    for (int r = 0; r < K; ++r) {
      if (r == col || !A[r][col]) continue;
      const uint32_t f = A[r][col];
      for (int c = 0; c < K; ++c) {
        A[r][c] ^= gf_mul(f, A[col][c], w);
        R[r][c] ^= gf_mul(f, R[col][c], w);
      }
    }
  }
  return true;
}

// Parity rows of the systematic generator.
//   Vandermonde (§2.2): G = V_full V_top^-1 with V_full[r][c] = r^c.
//   Cauchy (§2.3): C[i][j] = 1 / (i + (m + j)), X = {0..m-1}, Y = {m..m+k-1};
//   its "good" form: rows and columns scaled to fewer ones (good_cauchy_scale).
//   Polynomial code as a matrix (§6): column i = x^(m+i) mod g(x), since
//   x^m d(x) mod g = sum_i d_i (x^(m+i) mod g) (Eq. 1).
template <int W, int K, int M, int KIND>
struct ParityMatrix {
  static constexpr MatKM<K, M> make() {
    MatKM<K, M> P{};
    if (KIND == kKindPolyMatrix || KIND == kKindPolyBitMatrix) {
      const GenPoly g = make_genpoly(W, M);
      uint32_t r[M] = {};
      for (int j = 0; j < M; ++j) r[j] = g.c[j];  // x^m = sum_{j<m} g_j x^j (mod g, char 2)
      for (int i = 0; i < K; ++i) {
        for (int j = 0; j < M; ++j) P.a[j][i] = r[j];
        const uint32_t top = r[M - 1];  // multiply by x and reduce
        for (int j = M - 1; j >= 1; --j) r[j] = r[j - 1] ^ gf_mul(top, g.c[j], W);
        r[0] = gf_mul(top, g.c[0], W);
      }
    } else if (KIND == kKindCauchy || KIND == kKindGoodCauchy) {
      for (int i = 0; i < M; ++i)
        for (int j = 0; j < K; ++j) P.a[i][j] = gf_inv((uint32_t)i ^ (uint32_t)(M + j), W);
      if (KIND == kKindGoodCauchy)
        good_cauchy_scale(MatKMEntry<K, M>{P}, K, M, W);
    } else {
      uint32_t top[K][K] = {};
      uint32_t inv[K][K] = {};
      for (int r = 0; r < K; ++r) {
        uint32_t pw = 1;
        for (int c = 0; c < K; ++c) {
          top[r][c] = pw;
          pw = gf_mul(pw, (uint32_t)r, W);
        }
      }
      ct_invert<K>(top, inv, W);
      for (int i = 0; i < M; ++i) {
        uint32_t row[K] = {};
        uint32_t pw = 1;
        for (int c = 0; c < K; ++c) {
          row[c] = pw;
          pw = gf_mul(pw, (uint32_t)(K + i), W);
        }
        for (int c = 0; c < K; ++c) {
          uint32_t s = 0;
          for (int t = 0; t < K; ++t) s ^= gf_mul(row[t], inv[t][c], W);
          P.a[i][c] = s;
        }
      }
    }
    return P;
  }
  static constexpr MatKM<K, M> value = make();
};

// ------------------------------------------------ compile-time P: encode
template <int W, int K, int M, int KIND, bool kTranspose>
struct MatEncodeFixed {
  template <class Src, class Dst>
  static RS_HD void run(Src& src, Dst& dst) {
    uint32_t acc[M][W];
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
      for (int b = 0; b < W; ++b) acc[i][b] = 0;
    StaticFor<0, K>::run([&](auto J) {
      uint32_t x[W];
      src.load(decltype(J)::value, x);
      if (kTranspose) transpose<W>(x);
      StaticFor<0, M>::run([&](auto I) {
        mul_acc<W, ParityMatrix<W, K, M, KIND>::value.a[decltype(I)::value][decltype(J)::value]>(
            acc[decltype(I)::value], x);
      });
    });
#pragma unroll
    for (int i = 0; i < M; ++i) {
      if (kTranspose) transpose<W>(acc[i]);
      dst.store(i, acc[i]);
    }
  }
};

// Compile-time-P encode on two 32-column groups per thread (symbol layout,
// with transposes; packet layout without: group g is word g of the unit).
template <int W, int K, int M, int KIND, bool kTranspose = true>
struct MatEncodeFixed2 {
  template <class Src, class Dst>
  static RS_HD void run(Src& src, Dst& dst) {
    uint32_t a[M][W], b[M][W];
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
      for (int c = 0; c < W; ++c) a[i][c] = b[i][c] = 0;
    StaticFor<0, K>::run([&](auto J) {
      uint32_t x[2 * W];
      src.load(decltype(J)::value, x);
      if (kTranspose) {
        transpose<W>(x);
        transpose<W>(x + W);
      }
      StaticFor<0, M>::run([&](auto I) {
        constexpr uint32_t c = ParityMatrix<W, K, M, KIND>::value.a[decltype(I)::value][decltype(J)::value];
        mul_acc<W, c>(a[decltype(I)::value], x);
        mul_acc<W, c>(b[decltype(I)::value], x + W);
      });
    });
#pragma unroll
    for (int i = 0; i < M; ++i) {
      uint32_t y[2 * W];
#pragma unroll
      for (int c = 0; c < W; ++c) {
        y[c] = a[i][c];
        y[W + c] = b[i][c];
      }
      if (kTranspose) {
        transpose<W>(y);
        transpose<W>(y + W);
      }
      dst.store(i, y);
    }
  }
};

// ------------------------------------------------ compile-time P: decode
template <int W, int K, int M, int KIND, bool kTranspose>
struct MatDecodeFixed {
  template <class Src, class Dst, class Coef>
  static RS_HD void run(uint64_t read_mask, int e, Src& src, Dst& dst, Coef& coef) {
    Selectors<W, M> sel;
    sel.load(coef);
    uint32_t S[M][W];
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
      for (int b = 0; b < W; ++b) S[i][b] = 0;
    int in = 0;
    StaticFor<0, K>::run([&](auto J) {
      if ((read_mask >> decltype(J)::value) & 1ull) {
        uint32_t x[W];
        src.load(in++, x);
        if (kTranspose) transpose<W>(x);
        StaticFor<0, M>::run([&](auto I) {
          mul_acc<W, ParityMatrix<W, K, M, KIND>::value.a[decltype(I)::value][decltype(J)::value]>(
              S[decltype(I)::value], x);
        });
      }
    });
#pragma unroll
    for (int j = 0; j < M; ++j) {
      if ((read_mask >> (K + j)) & 1ull) {
        uint32_t x[W];
        src.load(in++, x);
        if (kTranspose) transpose<W>(x);
#pragma unroll
        for (int b = 0; b < W; ++b) S[j][b] ^= x[b];
      }
    }
    apply_and_store<W, M, kTranspose>(e, S, sel, dst);
  }
};

// Compile-time-P decode with two 32-column groups per thread (M <= 4): the
// syndromes of both groups, then apply2_and_store.
template <int W, int K, int M, int KIND, bool kTranspose = true, bool kPairSums = false>
struct MatDecodeFixed2 {
  template <class Src, class Dst, class Coef>
  static RS_HD void run(uint64_t read_mask, int e, Src& src, Dst& dst, Coef& coef) {
    Selectors<W, M> sel;
    sel.load(coef);
    uint32_t A[M][W], B[M][W];
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
      for (int b = 0; b < W; ++b) A[i][b] = B[i][b] = 0;
    int in = 0;
    StaticFor<0, K>::run([&](auto J) {
      if ((read_mask >> decltype(J)::value) & 1ull) {
        uint32_t x[2 * W];
        src.load(in++, x);
        if (kTranspose) {
          transpose<W>(x);
          transpose<W>(x + W);
        }
        StaticFor<0, M>::run([&](auto I) {
          constexpr uint32_t c = ParityMatrix<W, K, M, KIND>::value.a[decltype(I)::value][decltype(J)::value];
          mul_acc<W, c>(A[decltype(I)::value], x);
          mul_acc<W, c>(B[decltype(I)::value], x + W);
        });
      }
    });
#pragma unroll
    for (int j = 0; j < M; ++j) {
      if ((read_mask >> (K + j)) & 1ull) {
        uint32_t x[2 * W];
        src.load(in++, x);
        if (kTranspose) {
          transpose<W>(x);
          transpose<W>(x + W);
        }
#pragma unroll
        for (int b = 0; b < W; ++b) {
          A[j][b] ^= x[b];
          B[j][b] ^= x[W + b];
        }
      }
    }
    apply2_and_store<W, M, kTranspose, kPairSums>(e, A, B, sel, dst);
  }
};

// ------------------------------------------------ runtime P (any code)
// cols.column(j) returns a PackedBits<W, M, 1> source for data column j of P
// (entry (i, 0) = P[i][j]); the column's words are loaded before the input's
// transpose so their latency overlaps it.
template <int W, int M, bool kTranspose>
struct MatEncodeRuntime {
  template <class Src, class Dst, class Cols>
  static RS_HD void run(int k, Src& src, Dst& dst, const Cols& cols) {
    uint32_t acc[M][W];
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
      for (int b = 0; b < W; ++b) acc[i][b] = 0;
    for (int j = 0; j < k; ++j) {
      PackedBits<W, M, 1> col;
      col.load(cols.column(j));
      uint32_t x[W];
      src.load(j, x);
      if (kTranspose) transpose<W>(x);
      mul_acc_packed_column<W, M, 1>(acc, x, col, 0);
    }
#pragma unroll
    for (int i = 0; i < M; ++i) {
      if (kTranspose) transpose<W>(acc[i]);
      dst.store(i, acc[i]);
    }
  }
};

template <int W, int M, bool kTranspose>
struct MatDecodeRuntime {
  template <class Src, class Dst, class Cols, class Coef>
  static RS_HD void run(int k, uint64_t read_mask, int e, Src& src, Dst& dst, const Cols& cols, Coef& coef) {
    uint32_t S[M][W];
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
      for (int b = 0; b < W; ++b) S[i][b] = 0;
    int in = 0;
    Selectors<W, M> sel;
    sel.load(coef);
    for (int j = 0; j < k; ++j) {
      if (!((read_mask >> j) & 1ull)) continue;
      PackedBits<W, M, 1> col;
      col.load(cols.column(j));
      uint32_t x[W];
      src.load(in++, x);
      if (kTranspose) transpose<W>(x);
      mul_acc_packed_column<W, M, 1>(S, x, col, 0);
    }
#pragma unroll
    for (int j = 0; j < M; ++j) {
      if ((read_mask >> (k + j)) & 1ull) {
        uint32_t x[W];
        src.load(in++, x);
        if (kTranspose) transpose<W>(x);
#pragma unroll
        for (int b = 0; b < W; ++b) S[j][b] ^= x[b];
      }
    }
    apply_and_store<W, M, kTranspose>(e, S, sel, dst);
  }
};

}  // namespace rsgb
