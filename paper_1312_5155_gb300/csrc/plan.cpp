// Host-side decode planning and generator construction (see plan.hpp).
#include "plan.hpp"

#include <algorithm>

namespace rsgb {

bool gf_invert(int w, int n, const std::vector<uint32_t>& Ain, std::vector<uint32_t>& Ainv) {
  std::vector<uint32_t> A(Ain);
  Ainv.assign((size_t)n * n, 0);
  for (int i = 0; i < n; ++i) Ainv[(size_t)i * n + i] = 1;
  for (int col = 0; col < n; ++col) {
    int piv = -1;
    for (int r = col; r < n; ++r)
      if (A[(size_t)r * n + col]) { piv = r; break; }
    if (piv < 0) return false;
    if (piv != col)
      for (int c = 0; c < n; ++c) {
        std::swap(A[(size_t)col * n + c], A[(size_t)piv * n + c]);
        std::swap(Ainv[(size_t)col * n + c], Ainv[(size_t)piv * n + c]);
      }
    const uint32_t iv = gf_inv(A[(size_t)col * n + col], w);
    for (int c = 0; c < n; ++c) {
      A[(size_t)col * n + c] = gf_mul(A[(size_t)col * n + c], iv, w);
      Ainv[(size_t)col * n + c] = gf_mul(Ainv[(size_t)col * n + c], iv, w);
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const uint32_t f = A[(size_t)r * n + col];
      if (!f) continue;
      for (int c = 0; c < n; ++c) {
        A[(size_t)r * n + c] ^= gf_mul(f, A[(size_t)col * n + c], w);
        Ainv[(size_t)r * n + c] ^= gf_mul(f, Ainv[(size_t)col * n + c], w);
      }
    }
  }
  return true;
}

static bool check_erasures(int n, int m, const int* er, int e, std::string& err) {
  if (e < 0) { err = "negative erasure count"; return false; }
  if (e > m) { err = "more erasures than parity blocks"; return false; }
  for (int i = 0; i < e; ++i) {
    if (er[i] < 0 || er[i] >= n) { err = "erasure index out of range"; return false; }
    for (int j = 0; j < i; ++j)
      if (er[j] == er[i]) { err = "duplicate erasure index"; return false; }
  }
  return true;
}

// Read set: every survivor (read_all) or the first k survivors by block index.
static void choose_reads(int n, int k, const int* er, int e, bool read_all, std::vector<char>& read) {
  std::vector<char> erased(n, 0);
  for (int i = 0; i < e; ++i) erased[er[i]] = 1;
  read.assign(n, 0);
  int got = 0;
  for (int b = 0; b < n; ++b) {
    if (erased[b]) continue;
    if (!read_all && got == k) break;
    read[b] = 1;
    ++got;
  }
}

bool make_poly_decode_plan(int k, int m, int w, const int* er, int e, bool read_all,
                           DecodePlan& plan, std::string& err) {
  const int n = k + m;
  if (!check_erasures(n, m, er, e, err)) return false;
  plan = DecodePlan();
  plan.e = e;
  plan.n_pos = n;
  if (e == 0) return true;
  std::vector<char> read;
  choose_reads(n, k, er, e, read_all, read);
  // unknown positions: everything not read; the erased ones come first so
  // the rows of W follow the caller's erasure order
  std::vector<int> unknown(er, er + e);
  for (int b = 0; b < n; ++b) {
    if (read[b]) continue;
    if (std::find(unknown.begin(), unknown.end(), b) == unknown.end()) unknown.push_back(b);
  }
  const int M = (int)unknown.size();
  if (M > kMaxM) { err = "too many unknowns for the device path"; return false; }
  plan.M = M;
  // consumption order = descending codeword position (Horner from x^(n-1))
  std::vector<std::pair<int, int>> rp;
  for (int b = 0; b < n; ++b)
    if (read[b]) {
      const int p = poly_position(k, m, b);
      plan.read_mask |= 1ull << p;
      rp.push_back({p, b});
    }
  std::sort(rp.begin(), rp.end(), [](auto a, auto b) { return a.first > b.first; });
  for (auto& x : rp) plan.in_blocks.push_back(x.second);
  // V[j][u] = alpha^(j * pos_u), j < M: the Step-2 system of §3.3
  std::vector<uint32_t> V((size_t)M * M), Vi;
  for (int j = 0; j < M; ++j)
    for (int u = 0; u < M; ++u)
      V[(size_t)j * M + u] = gf_alpha_pow((uint64_t)j * (uint64_t)poly_position(k, m, unknown[u]), w);
  if (!gf_invert(w, M, V, Vi)) { err = "singular decode system"; return false; }
  for (int t = 0; t < e; ++t) {
    plan.out_blocks.push_back(unknown[t]);
    for (int j = 0; j < M; ++j) plan.W[t][j] = Vi[(size_t)t * M + j];
  }
  return true;
}

bool make_matrix_decode_plan(int k, int m, int w, const std::vector<uint32_t>& P, const int* er,
                             int e, bool read_all, DecodePlan& plan, std::string& err) {
  const int n = k + m;
  if (!check_erasures(n, m, er, e, err)) return false;
  plan = DecodePlan();
  plan.e = e;
  plan.n_pos = n;
  if (e == 0) return true;
  std::vector<char> read;
  choose_reads(n, k, er, e, read_all, read);
  std::vector<int> unknown(er, er + e);
  for (int b = 0; b < n; ++b) {
    if (read[b]) continue;
    if (std::find(unknown.begin(), unknown.end(), b) == unknown.end()) unknown.push_back(b);
  }
  const int U = (int)unknown.size();
  if (m > kMaxM || U > kMaxM) { err = "too many parity blocks for the device path"; return false; }
  // H = [P | I_m]: column b of H is P's column b for data, e_(b-k) for parity.
  auto Hcol = [&](int row, int b) -> uint32_t {
    return b < k ? P[(size_t)row * k + b] : (uint32_t)(b - k == row);
  };
  // U unknowns need U independent syndrome rows: all m rows when U = m
  // (min-read), otherwise the first row subset that gives an invertible
  // U x U system (the code is MDS, so one exists).
  std::vector<int> rows(U);
  for (int a = 0; a < U; ++a) rows[a] = a;
  std::vector<uint32_t> Hi;
  for (;;) {
    std::vector<uint32_t> H((size_t)U * U);
    for (int a = 0; a < U; ++a)
      for (int u = 0; u < U; ++u) H[(size_t)a * U + u] = Hcol(rows[a], unknown[u]);
    if (gf_invert(w, U, H, Hi)) break;
    // next combination of U rows out of m (lexicographic)
    int i = U - 1;
    while (i >= 0 && rows[i] == m - U + i) --i;
    if (i < 0) { err = "singular decode system"; return false; }
    ++rows[i];
    for (int j = i + 1; j < U; ++j) rows[j] = rows[j - 1] + 1;
  }
  // The device evaluates all m syndromes; W has zero columns for rows that
  // the chosen system does not use.
  plan.M = m;
  for (int b = 0; b < n; ++b)
    if (read[b]) {
      plan.read_mask |= 1ull << b;
      plan.in_blocks.push_back(b);  // data ascending, then parity ascending
    }
  for (int t = 0; t < e; ++t) {
    plan.out_blocks.push_back(unknown[t]);
    for (int a = 0; a < U; ++a) plan.W[t][rows[a]] = Hi[(size_t)t * U + a];
  }
  return true;
}

std::vector<uint32_t> pack_bits(const uint32_t* a, int R, int Q, int w) {
  std::vector<uint32_t> out(((size_t)R * Q * w + 31) / 32, 0u);
  for (int r = 0; r < R; ++r)
    for (int q = 0; q < Q; ++q)
      for (int c = 0; c < w; ++c)
        if ((a[(size_t)r * Q + q] >> c) & 1u) {
          const size_t pbit = ((size_t)q * R + r) * w + c;
          out[pbit >> 5] |= 1u << (pbit & 31);
        }
  return out;
}

std::vector<uint32_t> pack_decode_selectors(const DecodePlan& pl, int w) {
  const int M = pl.M;
  const int chunks = (M + 3) / 4;
  const int row_words = (w * chunks + 7) / 8;
  std::vector<uint32_t> out((size_t)selector_words(M, w), 0u);
  for (int t = 0; t < pl.e; ++t)
    for (int c = 0; c < w; ++c)
      for (int h = 0; h < chunks; ++h) {
        uint32_t nib = 0;
        for (int i = 0; i < 4 && 4 * h + i < M; ++i)
          if ((pl.W[t][4 * h + i] >> c) & 1u) nib |= 1u << i;
        const int n = c * chunks + h;
        out[(size_t)t * row_words + (n >> 3)] |= nib << ((n & 7) * 4);
      }
  return out;
}

std::vector<uint32_t> pack_columns(const std::vector<uint32_t>& P, int k, int m, int w) {
  const int cw = column_words(m, w);
  std::vector<uint32_t> out((size_t)k * cw, 0u);
  std::vector<uint32_t> col(m);
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i < m; ++i) col[i] = P[(size_t)i * k + j];
    const std::vector<uint32_t> words = pack_bits(col.data(), m, 1, w);
    for (int x = 0; x < cw; ++x) out[(size_t)j * cw + x] = words[x];
  }
  return out;
}

bool vandermonde_parity_matrix(int k, int m, int w, std::vector<uint32_t>& P) {
  // G = V_full * V_top^-1 with V_full[r][c] = r^c (0^0 = 1), §2.2.
  const int n = k + m;
  std::vector<uint32_t> V((size_t)n * k), top((size_t)k * k), ti;
  for (int r = 0; r < n; ++r) {
    uint32_t pw = 1;
    for (int c = 0; c < k; ++c) {
      V[(size_t)r * k + c] = pw;
      pw = gf_mul(pw, (uint32_t)r, w);
    }
  }
  std::copy(V.begin(), V.begin() + (size_t)k * k, top.begin());
  if (!gf_invert(w, k, top, ti)) return false;
  P.assign((size_t)m * k, 0);
  for (int i = 0; i < m; ++i)
    for (int c = 0; c < k; ++c) {
      uint32_t s = 0;
      for (int t = 0; t < k; ++t) s ^= gf_mul(V[(size_t)(k + i) * k + t], ti[(size_t)t * k + c], w);
      P[(size_t)i * k + c] = s;
    }
  return true;
}

void cauchy_parity_matrix(int k, int m, int w, std::vector<uint32_t>& P) {
  // C[i][j] = 1 / (x_i + y_j), X = {0..m-1}, Y = {m..m+k-1}  (§2.3)
  P.assign((size_t)m * k, 0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < k; ++j) P[(size_t)i * k + j] = gf_inv((uint32_t)i ^ (uint32_t)(m + j), w);
}

void good_cauchy_parity_matrix(int k, int m, int w, std::vector<uint32_t>& P) {
  cauchy_parity_matrix(k, m, w, P);
  good_cauchy_scale([&P, k](int i, int j) -> uint32_t& { return P[(size_t)i * k + j]; }, k, m, w);
}

void poly_parity_matrix(int k, int m, int w, std::vector<uint32_t>& P) {
  const GenPoly g = make_genpoly(w, m);
  P.assign((size_t)m * k, 0);
  std::vector<uint32_t> r(m);
  for (int j = 0; j < m; ++j) r[j] = g.c[j];
  for (int i = 0; i < k; ++i) {
    for (int j = 0; j < m; ++j) P[(size_t)j * k + i] = r[j];
    const uint32_t top = r[m - 1];
    for (int j = m - 1; j >= 1; --j) r[j] = r[j - 1] ^ gf_mul(top, g.c[j], w);
    r[0] = gf_mul(top, g.c[0], w);
  }
}

}  // namespace rsgb
