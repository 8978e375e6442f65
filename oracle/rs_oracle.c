/*
 * Reed-Solomon reference oracle: plain, slow, scalar C.
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference legs load this file (through oracle/oracle.py).
 * The product library never links, includes or calls it, and the two share
 * no code: not the field tables, not the code construction, not the layouts.
 *
 * What it computes follows "On the Effectiveness of Polynomial Realization
 * of Reed-Solomon Codes for Storage Systems" (Sheykh Esmaili and Datta):
 *   - GF(2^w) with precomputed multiplication / division tables (§5.1),
 *     primitive element alpha = 2 (§3.1 example);
 *   - generator polynomial g(x) = prod_{i<m} (x + alpha^i) (§3.1);
 *   - polynomial encode: p(x) = x^m d(x) mod g(x) by textbook long division
 *     (§3.2, Eq. 1 and Eq. 2), data d_i at x^(m+i), parity p_j at x^j;
 *   - polynomial decode: Step 1 evaluates D(x) at alpha^0..alpha^(e-1) over
 *     the survivors, Step 2 solves the e x e Vandermonde system by Gaussian
 *     elimination, separately for every column (§3.3);
 *   - matrix realization (§2.1): systematic Vandermonde generator (§2.2)
 *     and Cauchy generator with its bit-matrix projection (§2.3).
 *
 * Symbols: w = 4 stores one symbol per byte (low nibble), w = 8 one byte,
 * w = 16 one little-endian 16-bit word.  A block of B bytes holds B/s
 * symbols (s = symbol bytes); symbol t of every block forms one column,
 * an independent codeword.  Blocks 0..k-1 are data d_0..d_{k-1}, blocks
 * k..k+m-1 are parity p_0..p_{m-1}; all n blocks are passed as one
 * n x B byte array.
 *
 * Every function returns 0 on success and a negative value on bad input.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ field */
/* GF(2^w): exp[i] = alpha^i, log[exp[i]] = i, built by repeated
 * multiplication by alpha = 2 modulo the primitive polynomial
 * (0x13 for w=4, 0x11D for w=8, 0x1100B for w=16). */
typedef struct {
    int w;
    uint32_t prim;
    uint32_t q;        /* 2^w */
    uint32_t *exp;     /* q-1 entries */
    uint32_t *log;     /* q entries, log[0] unused */
} field_t;

static field_t g_fields[3];

static field_t *field_for(int w) {
    int slot;
    uint32_t prim;
    if (w == 4) { slot = 0; prim = 0x13; }
    else if (w == 8) { slot = 1; prim = 0x11D; }
    else if (w == 16) { slot = 2; prim = 0x1100B; }
    else return NULL;
    field_t *f = &g_fields[slot];
    if (f->exp) return f;
    uint32_t q = 1u << w;
    uint32_t *ex = (uint32_t *)malloc(sizeof(uint32_t) * (q - 1));
    uint32_t *lg = (uint32_t *)calloc(q, sizeof(uint32_t));
    if (!ex || !lg) { free(ex); free(lg); return NULL; }
    uint32_t x = 1;
    for (uint32_t i = 0; i < q - 1; i++) {
        ex[i] = x;
        lg[x] = i;
        x <<= 1;
        if (x & q) x ^= prim;
    }
    f->w = w; f->prim = prim; f->q = q; f->log = lg; f->exp = ex;
    return f;
}

/* Build all three fields up front (call before using the oracle from
 * several threads). */
int rso_init(void) {
    if (!field_for(4) || !field_for(8) || !field_for(16)) return -1;
    return 0;
}

static uint32_t gmul(const field_t *f, uint32_t a, uint32_t b) {
    if (a == 0 || b == 0) return 0;
    return f->exp[(f->log[a] + f->log[b]) % (f->q - 1)];
}

static uint32_t ginv(const field_t *f, uint32_t a) {
    /* a != 0 */
    return f->exp[(f->q - 1 - f->log[a]) % (f->q - 1)];
}

static uint32_t gpow_alpha(const field_t *f, uint64_t e) {
    return f->exp[e % (f->q - 1)];
}

/* element-wise helpers exported for the field tests */
int rso_gf_mul_array(int w, const uint32_t *a, const uint32_t *b, uint32_t *out, size_t cnt) {
    field_t *f = field_for(w);
    if (!f) return -1;
    for (size_t i = 0; i < cnt; i++) out[i] = gmul(f, a[i], b[i]);
    return 0;
}

int rso_gf_inv_array(int w, const uint32_t *a, uint32_t *out, size_t cnt) {
    field_t *f = field_for(w);
    if (!f) return -1;
    for (size_t i = 0; i < cnt; i++) {
        if (a[i] == 0) return -2;
        out[i] = ginv(f, a[i]);
    }
    return 0;
}

int rso_gf_exp_table(int w, uint32_t *out) {
    field_t *f = field_for(w);
    if (!f) return -1;
    memcpy(out, f->exp, sizeof(uint32_t) * (f->q - 1));
    return 0;
}

/* ---------------------------------------------------------------- symbols */
static int sym_bytes(int w) { return w == 16 ? 2 : 1; }

static uint32_t get_sym(const uint8_t *blk, size_t t, int w) {
    if (w == 16) return (uint32_t)blk[2 * t] | ((uint32_t)blk[2 * t + 1] << 8);
    if (w == 4) return blk[t] & 0xFu;
    return blk[t];
}

static void put_sym(uint8_t *blk, size_t t, int w, uint32_t v) {
    if (w == 16) { blk[2 * t] = (uint8_t)(v & 0xFF); blk[2 * t + 1] = (uint8_t)(v >> 8); }
    else blk[t] = (uint8_t)v;
}

static int check_code(int w, int k, int m, field_t **fo) {
    field_t *f = field_for(w);
    if (!f || k < 1 || m < 0) return -1;
    if ((uint32_t)(k + m) > f->q - 1) return -1;   /* distinct alpha^pos / field rows */
    *fo = f;
    return 0;
}

static int check_erasures(int n, int m, const int *er, int e) {
    if (e < 0 || e > m) return -1;
    for (int i = 0; i < e; i++) {
        if (er[i] < 0 || er[i] >= n) return -1;
        for (int j = 0; j < i; j++) if (er[j] == er[i]) return -1;
    }
    return 0;
}

/* position of block b in the codeword polynomial: d_i at x^(m+i), p_j at x^j
 * (§3.2 Eq. 2 and the §3.2 example, where d_0 = 48 multiplies x^3). */
static int poly_pos(int k, int m, int b) { return b < k ? m + b : b - k; }

/* ---------------------------------------------------- generator polynomial */
/* §3.1: g(x) = (x + alpha^0)(x + alpha^1)...(x + alpha^(m-1)), expanded by
 * multiplying in one factor at a time.  g[i] is the coefficient of x^i;
 * g[m] = 1. */
int rso_genpoly(int w, int m, uint32_t *g) {
    field_t *f = field_for(w);
    if (!f || m < 0) return -1;
    for (int i = 0; i <= m; i++) g[i] = 0;
    g[0] = 1;
    for (int i = 0; i < m; i++) {
        uint32_t root = gpow_alpha(f, (uint64_t)i);
        /* (x + root) * g(x): new[j] = g[j-1] + root*g[j] */
        for (int j = i + 1; j >= 1; j--) g[j] = g[j - 1] ^ gmul(f, root, g[j]);
        g[0] = gmul(f, root, g[0]);
    }
    return 0;
}

/* ------------------------------------------------------ polynomial encode */
/* §3.2 Eq. 1: parity = coefficients of the remainder of x^m d(x) divided by
 * g(x).  Long division over the whole degree-(n-1) polynomial: at each
 * degree from n-1 down to m, subtract (= add) lead * x^(deg-m) * g(x). */
int rso_poly_encode_column(int w, int k, int m, const uint32_t *d, uint32_t *p) {
    field_t *f;
    if (check_code(w, k, m, &f)) return -1;
    int n = k + m;
    uint32_t g[257];
    if (m > 256) return -1;
    rso_genpoly(w, m, g);
    uint32_t *c = (uint32_t *)calloc((size_t)n, sizeof(uint32_t));
    if (!c) return -3;
    for (int i = 0; i < k; i++) c[m + i] = d[i];
    for (int deg = n - 1; deg >= m; deg--) {
        uint32_t lead = c[deg];
        if (lead == 0) continue;
        for (int t = 0; t <= m; t++) c[deg - m + t] ^= gmul(f, lead, g[t]);
    }
    for (int j = 0; j < m; j++) p[j] = c[j];
    free(c);
    return 0;
}

int rso_poly_encode(int w, int k, int m, uint8_t *blocks, size_t block_bytes) {
    field_t *f;
    if (check_code(w, k, m, &f)) return -1;
    if (block_bytes % (size_t)sym_bytes(w)) return -1;
    size_t S = block_bytes / (size_t)sym_bytes(w);
    uint32_t d[256], p[256];
    if (k > 256 || m > 256) return -1;
    for (size_t t = 0; t < S; t++) {
        for (int i = 0; i < k; i++) d[i] = get_sym(blocks + (size_t)i * block_bytes, t, w);
        rso_poly_encode_column(w, k, m, d, p);
        for (int j = 0; j < m; j++) put_sym(blocks + (size_t)(k + j) * block_bytes, t, w, p[j]);
    }
    return 0;
}

/* ------------------------------------------------ Gaussian elimination */
/* Solve A x = b (A is e x e, row-major) in place over GF(2^w).
 * Returns -2 if A is singular. */
static int gauss_solve(const field_t *f, int e, uint32_t *A, uint32_t *b) {
    for (int col = 0; col < e; col++) {
        int piv = -1;
        for (int r = col; r < e; r++) if (A[r * e + col]) { piv = r; break; }
        if (piv < 0) return -2;
        if (piv != col) {
            for (int c = 0; c < e; c++) { uint32_t t = A[col * e + c]; A[col * e + c] = A[piv * e + c]; A[piv * e + c] = t; }
            uint32_t t = b[col]; b[col] = b[piv]; b[piv] = t;
        }
        uint32_t inv = ginv(f, A[col * e + col]);
        for (int c = 0; c < e; c++) A[col * e + c] = gmul(f, A[col * e + c], inv);
        b[col] = gmul(f, b[col], inv);
        for (int r = 0; r < e; r++) {
            if (r == col) continue;
            uint32_t fac = A[r * e + col];
            if (!fac) continue;
            for (int c = 0; c < e; c++) A[r * e + c] ^= gmul(f, fac, A[col * e + c]);
            b[r] ^= gmul(f, fac, b[col]);
        }
    }
    return 0;
}

/* Gauss-Jordan inverse of an n x n matrix; -2 if singular. */
static int gauss_invert(const field_t *f, int n, const uint32_t *Ain, uint32_t *Ainv) {
    uint32_t *A = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n * n);
    if (!A) return -3;
    memcpy(A, Ain, sizeof(uint32_t) * (size_t)n * n);
    for (int r = 0; r < n; r++) for (int c = 0; c < n; c++) Ainv[r * n + c] = (r == c);
    for (int col = 0; col < n; col++) {
        int piv = -1;
        for (int r = col; r < n; r++) if (A[r * n + col]) { piv = r; break; }
        if (piv < 0) { free(A); return -2; }
        if (piv != col) {
            for (int c = 0; c < n; c++) {
                uint32_t t = A[col * n + c]; A[col * n + c] = A[piv * n + c]; A[piv * n + c] = t;
                t = Ainv[col * n + c]; Ainv[col * n + c] = Ainv[piv * n + c]; Ainv[piv * n + c] = t;
            }
        }
        uint32_t inv = ginv(f, A[col * n + col]);
        for (int c = 0; c < n; c++) { A[col * n + c] = gmul(f, A[col * n + c], inv); Ainv[col * n + c] = gmul(f, Ainv[col * n + c], inv); }
        for (int r = 0; r < n; r++) {
            if (r == col) continue;
            uint32_t fac = A[r * n + col];
            if (!fac) continue;
            for (int c = 0; c < n; c++) {
                A[r * n + c] ^= gmul(f, fac, A[col * n + c]);
                Ainv[r * n + c] ^= gmul(f, fac, Ainv[col * n + c]);
            }
        }
    }
    free(A);
    return 0;
}

int rso_gf_invert_matrix(int w, int n, const uint32_t *A, uint32_t *Ainv) {
    field_t *f = field_for(w);
    if (!f || n < 1) return -1;
    return gauss_invert(f, n, A, Ainv);
}

/* ------------------------------------------------------ polynomial decode */
/* §3.3, one column.  c holds all n symbols (block order); erased entries are
 * ignored.  Step 1: D_j = sum over surviving blocks b of c_b alpha^(j pos(b))
 * for j = 0..e-1 (erased terms skipped, as Opt2 of §4 does).  Step 2: solve
 * D_j = sum_t alpha^(j pos(erased_t)) x_t for the erased symbols x.  D_out
 * and V_out (e x e, row j = power, column t = erasure) receive Step 1's
 * values and the system matrix when non-NULL.  The recovered symbols are
 * written into c at the erased indices. */
int rso_poly_decode_column(int w, int k, int m, const int *er, int e,
                           uint32_t *c, uint32_t *D_out, uint32_t *V_out) {
    field_t *f;
    if (check_code(w, k, m, &f)) return -1;
    int n = k + m;
    if (check_erasures(n, m, er, e)) return -1;
    if (e == 0) return 0;
    uint32_t D[256], V[256 * 256];
    if (e < 0 || e > 256) return -1;
    const size_t ue = (size_t)e;
    char erased[512];
    if (n > 512) return -1;
    memset(erased, 0, sizeof(erased));
    for (int t = 0; t < e; t++) erased[er[t]] = 1;
    for (int j = 0; j < e; j++) {
        uint32_t s = 0;
        for (int b = 0; b < n; b++) {
            if (erased[b]) continue;
            s ^= gmul(f, c[b], gpow_alpha(f, (uint64_t)j * (uint64_t)poly_pos(k, m, b)));
        }
        D[j] = s;
        for (int t = 0; t < e; t++)
            V[j * e + t] = gpow_alpha(f, (uint64_t)j * (uint64_t)poly_pos(k, m, er[t]));
    }
    if (D_out) memcpy(D_out, D, sizeof(uint32_t) * ue);
    if (V_out) memcpy(V_out, V, sizeof(uint32_t) * ue * ue);
    int rc = gauss_solve(f, e, V, D);
    if (rc) return rc;
    for (int t = 0; t < e; t++) c[er[t]] = D[t];
    return 0;
}

int rso_poly_decode(int w, int k, int m, const int *er, int e, uint8_t *blocks, size_t block_bytes) {
    field_t *f;
    if (check_code(w, k, m, &f)) return -1;
    int n = k + m;
    if (check_erasures(n, m, er, e)) return -1;
    if (block_bytes % (size_t)sym_bytes(w)) return -1;
    size_t S = block_bytes / (size_t)sym_bytes(w);
    uint32_t c[512];
    if (n > 512) return -1;
    for (size_t t = 0; t < S; t++) {
        for (int b = 0; b < n; b++) c[b] = get_sym(blocks + (size_t)b * block_bytes, t, w);
        int rc = rso_poly_decode_column(w, k, m, er, e, c, NULL, NULL);
        if (rc) return rc;
        for (int i = 0; i < e; i++) put_sym(blocks + (size_t)er[i] * block_bytes, t, w, c[er[i]]);
    }
    return 0;
}

/* --------------------------------------------- systematic Vandermonde (§2.2) */
/* V_full[r][c] = r^c (r taken as a field element, 0^0 = 1), n x k.  Any k
 * rows are a Vandermonde matrix on distinct points, hence invertible.  The
 * systematic form is G = V_full * (rows 0..k-1 of V_full)^-1: multiplying on
 * the right by that inverse is the column reduction that turns the top
 * block into I_k (§2.2 defers the transformation to Plank's tutorial).
 * G is n x k, row-major. */
int rso_vand_matrix(int w, int k, int m, uint32_t *G) {
    field_t *f;
    if (check_code(w, k, m, &f)) return -1;
    int n = k + m;
    uint32_t *V = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n * k);
    uint32_t *Ti = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)k * k);
    if (!V || !Ti) { free(V); free(Ti); return -3; }
    for (int r = 0; r < n; r++) {
        uint32_t pw = 1;
        for (int c = 0; c < k; c++) { V[r * k + c] = pw; pw = gmul(f, pw, (uint32_t)r); }
    }
    int rc = gauss_invert(f, k, V, Ti);    /* top k rows */
    if (rc) { free(V); free(Ti); return rc; }
    for (int r = 0; r < n; r++)
        for (int c = 0; c < k; c++) {
            uint32_t s = 0;
            for (int t = 0; t < k; t++) s ^= gmul(f, V[r * k + t], Ti[t * k + c]);
            G[r * k + c] = s;
        }
    free(V); free(Ti);
    return 0;
}

/* c = G d (§2.1): parity row i of the codeword is row k+i of G times d. */
static int matrix_encode(const field_t *f, int w, int k, int m, const uint32_t *G,
                         uint8_t *blocks, size_t block_bytes) {
    size_t S = block_bytes / (size_t)sym_bytes(w);
    for (size_t t = 0; t < S; t++) {
        for (int i = 0; i < m; i++) {
            uint32_t s = 0;
            for (int j = 0; j < k; j++)
                s ^= gmul(f, G[(size_t)(k + i) * k + j], get_sym(blocks + (size_t)j * block_bytes, t, w));
            put_sym(blocks + (size_t)(k + i) * block_bytes, t, w, s);
        }
    }
    return 0;
}

/* §2.1 decoding: drop the erased rows of G, keep k survivors (lowest block
 * indices first), invert that k x k matrix, multiply it by the surviving
 * symbols to get the data, then recompute erased parity from G. */
static int matrix_decode(const field_t *f, int w, int k, int m, const uint32_t *G,
                         const int *er, int e, uint8_t *blocks, size_t block_bytes) {
    int n = k + m;
    char erased[512];
    memset(erased, 0, sizeof(erased));
    for (int t = 0; t < e; t++) erased[er[t]] = 1;
    int surv[512], ns = 0;
    for (int b = 0; b < n && ns < k; b++) if (!erased[b]) surv[ns++] = b;
    uint32_t *Gs = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)k * k);
    uint32_t *Gi = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)k * k);
    uint32_t *cs = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)k);
    uint32_t *d = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)k);
    if (!Gs || !Gi || !cs || !d) { free(Gs); free(Gi); free(cs); free(d); return -3; }
    for (int r = 0; r < k; r++) memcpy(Gs + (size_t)r * k, G + (size_t)surv[r] * k, sizeof(uint32_t) * (size_t)k);
    int rc = gauss_invert(f, k, Gs, Gi);
    if (rc) { free(Gs); free(Gi); free(cs); free(d); return rc; }
    size_t S = block_bytes / (size_t)sym_bytes(w);
    for (size_t t = 0; t < S; t++) {
        for (int r = 0; r < k; r++) cs[r] = get_sym(blocks + (size_t)surv[r] * block_bytes, t, w);
        for (int j = 0; j < k; j++) {
            uint32_t s = 0;
            for (int r = 0; r < k; r++) s ^= gmul(f, Gi[(size_t)j * k + r], cs[r]);
            d[j] = s;
        }
        for (int x = 0; x < e; x++) {
            int b = er[x];
            uint32_t v;
            if (b < k) v = d[b];
            else {
                v = 0;
                for (int j = 0; j < k; j++) v ^= gmul(f, G[(size_t)b * k + j], d[j]);
            }
            put_sym(blocks + (size_t)b * block_bytes, t, w, v);
        }
    }
    free(Gs); free(Gi); free(cs); free(d);
    return 0;
}

int rso_vand_encode(int w, int k, int m, uint8_t *blocks, size_t block_bytes) {
    field_t *f;
    if (check_code(w, k, m, &f)) return -1;
    if (block_bytes % (size_t)sym_bytes(w)) return -1;
    int n = k + m;
    uint32_t *G = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n * k);
    if (!G) return -3;
    int rc = rso_vand_matrix(w, k, m, G);
    if (!rc) rc = matrix_encode(f, w, k, m, G, blocks, block_bytes);
    free(G);
    return rc;
}

int rso_vand_decode(int w, int k, int m, const int *er, int e, uint8_t *blocks, size_t block_bytes) {
    field_t *f;
    if (check_code(w, k, m, &f)) return -1;
    int n = k + m;
    if (check_erasures(n, m, er, e)) return -1;
    if (block_bytes % (size_t)sym_bytes(w)) return -1;
    if (e == 0) return 0;
    uint32_t *G = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n * k);
    if (!G) return -3;
    int rc = rso_vand_matrix(w, k, m, G);
    if (!rc) rc = matrix_decode(f, w, k, m, G, er, e, blocks, block_bytes);
    free(G);
    return rc;
}

/* ------------------------------------------------------------ Cauchy (§2.3) */
/* m x k Cauchy matrix C[i][j] = 1 / (x_i + y_j) with X = {0..m-1} and
 * Y = {m..m+k-1}: distinct field elements, X and Y disjoint. */
int rso_cauchy_matrix(int w, int k, int m, uint32_t *C) {
    field_t *f;
    if (check_code(w, k, m, &f)) return -1;
    if ((uint32_t)(k + m) > f->q) return -1;
    for (int i = 0; i < m; i++)
        for (int j = 0; j < k; j++) C[i * k + j] = ginv(f, (uint32_t)i ^ (uint32_t)(m + j));
    return 0;
}

/* §2.3 projection of an element e onto a w x w matrix over GF(2): column c
 * is the bit vector of e * alpha^c, row r holds bit r.  Then the bit vector
 * of e*x is M(e) times the bit vector of x.  M is row-major bytes (0/1). */
int rso_bitmatrix(int w, uint32_t e, uint8_t *M) {
    field_t *f = field_for(w);
    if (!f) return -1;
    for (int c = 0; c < w; c++) {
        uint32_t col = gmul(f, e, gpow_alpha(f, (uint64_t)c));
        for (int r = 0; r < w; r++) M[r * w + c] = (uint8_t)((col >> r) & 1u);
    }
    return 0;
}

/* Packet layout: a block is a sequence of super-packets of w*P bytes; packet
 * c (0..w-1) of a super-packet is bit-row c.  Bit b of packet c (byte b/8,
 * bit b%8) is bit c of symbol b of that super-packet. */
static const uint8_t *packet(const uint8_t *blocks, size_t B, int blk, size_t sp, int c, int w, size_t P) {
    return blocks + (size_t)blk * B + sp * (size_t)w * P + (size_t)c * P;
}

/* out (P bytes) ^= packet: one XOR of the bit-matrix schedule. */
static void xor_into(uint8_t *out, const uint8_t *in, size_t P) {
    for (size_t i = 0; i < P; i++) out[i] ^= in[i];
}

/* Parity block i, super-packet sp: packet r = XOR over data blocks j and
 * rows c with M(coef[j])[r][c] = 1 of data packet (j, c). */
static void bitmatrix_apply(const field_t *f, int w, int nin, const int *in_blocks,
                            const uint32_t *coef, uint8_t *blocks, size_t B, size_t P,
                            int out_block) {
    uint8_t M[16 * 16];
    size_t nsp = B / ((size_t)w * P);
    (void)f;
    for (size_t sp = 0; sp < nsp; sp++) {
        for (int r = 0; r < w; r++)
            memset((uint8_t *)packet(blocks, B, out_block, sp, r, w, P), 0, P);
        for (int j = 0; j < nin; j++) {
            rso_bitmatrix(w, coef[j], M);
            for (int r = 0; r < w; r++)
                for (int c = 0; c < w; c++)
                    if (M[r * w + c])
                        xor_into((uint8_t *)packet(blocks, B, out_block, sp, r, w, P),
                                 packet(blocks, B, in_blocks[j], sp, c, w, P), P);
        }
    }
}

static int cauchy_check(int w, int k, int m, size_t B, size_t P, field_t **f) {
    if (check_code(w, k, m, f)) return -1;
    if (w != 8 && w != 16 && w != 4) return -1;
    if (P == 0 || B % ((size_t)w * P)) return -1;
    return 0;
}

/* Encode with the bit-matrix projection of an m x k parity matrix C. */
static int bitmatrix_code_encode(const field_t *f, int w, int k, int m, const uint32_t *C, uint8_t *blocks,
                                 size_t B, size_t P) {
    int *ins = (int *)malloc(sizeof(int) * (size_t)k);
    if (!ins) return -3;
    for (int j = 0; j < k; j++) ins[j] = j;
    for (int i = 0; i < m; i++) bitmatrix_apply(f, w, k, ins, C + (size_t)i * k, blocks, B, P, k + i);
    free(ins);
    return 0;
}

int rso_cauchy_encode(int w, int k, int m, uint8_t *blocks, size_t B, size_t P) {
    field_t *f;
    if (cauchy_check(w, k, m, B, P, &f)) return -1;
    uint32_t *C = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)m * k);
    if (!C) return -3;
    rso_cauchy_matrix(w, k, m, C);
    int rc = bitmatrix_code_encode(f, w, k, m, C, blocks, B, P);
    free(C);
    return rc;
}

/* Decoding (§2.1 steps on the generator [I_k; C]): k survivors with the
 * lowest block indices, invert their k x k rows, project each needed row of
 * the inverse to bit-matrices and XOR the surviving packets; erased parity
 * is then re-encoded from the completed data. */
static int bitmatrix_code_decode(const field_t *f, int w, int k, int m, const uint32_t *Cin, const int *er,
                                 int e, uint8_t *blocks, size_t B, size_t P) {
    int n = k + m;
    if (e == 0) return 0;
    uint32_t *C = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)m * k);
    uint32_t *Gs = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)k * k);
    uint32_t *Gi = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)k * k);
    int *surv = (int *)malloc(sizeof(int) * (size_t)n);
    int *dat = (int *)malloc(sizeof(int) * (size_t)k);
    if (!C || !Gs || !Gi || !surv || !dat) { free(C); free(Gs); free(Gi); free(surv); free(dat); return -3; }
    memcpy(C, Cin, sizeof(uint32_t) * (size_t)m * k);
    char erased[512];
    memset(erased, 0, sizeof(erased));
    for (int t = 0; t < e; t++) erased[er[t]] = 1;
    int ns = 0;
    for (int b = 0; b < n && ns < k; b++) if (!erased[b]) surv[ns++] = b;
    for (int r = 0; r < k; r++) {
        int b = surv[r];
        for (int c = 0; c < k; c++)
            Gs[r * k + c] = b < k ? (uint32_t)(b == c) : C[(size_t)(b - k) * k + c];
    }
    int rc = gauss_invert(f, k, Gs, Gi);
    if (!rc) {
        for (int x = 0; x < e; x++)
            if (er[x] < k) bitmatrix_apply(f, w, k, surv, Gi + (size_t)er[x] * k, blocks, B, P, er[x]);
        for (int j = 0; j < k; j++) dat[j] = j;
        for (int x = 0; x < e; x++)
            if (er[x] >= k) bitmatrix_apply(f, w, k, dat, C + (size_t)(er[x] - k) * k, blocks, B, P, er[x]);
    }
    free(C); free(Gs); free(Gi); free(surv); free(dat);
    return rc;
}

int rso_cauchy_decode(int w, int k, int m, const int *er, int e, uint8_t *blocks, size_t B, size_t P) {
    field_t *f;
    if (cauchy_check(w, k, m, B, P, &f)) return -1;
    if (check_erasures(k + m, m, er, e)) return -1;
    uint32_t *C = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)m * k);
    if (!C) return -3;
    rso_cauchy_matrix(w, k, m, C);
    int rc = bitmatrix_code_decode(f, w, k, m, C, er, e, blocks, B, P);
    free(C);
    return rc;
}

/* ------------------------------------------- "good" Cauchy matrix (§2.3) */
/* §2.3 notes that Cauchy matrices differ in efficiency -- the XOR count of a
 * bit-matrix code is the number of ones of its projection -- and points to
 * work on choosing good ones without giving a construction.  Reading taken
 * here (the scaling heuristic of Plank and Xu's optimised Cauchy RS codes,
 * restated): scaling a row or a column of the parity matrix by a nonzero
 * element keeps every square submatrix nonsingular, so the code stays MDS;
 * start from the original X = {0..m-1}, Y = {m..m+k-1} matrix, (1) divide
 * every column by its row-0 entry (row 0 becomes all ones, the cheapest
 * element: w ones), (2) for every other row, among the divisors 1 and the
 * row's own entries take the one that leaves the fewest ones in the row
 * (the first such divisor on ties) and divide the row by it. */
static int ones_of(const field_t *f, int w, uint32_t e) {
    int n = 0;
    for (int c = 0; c < w; c++) {
        uint32_t col = gmul(f, e, gpow_alpha(f, (uint64_t)c));
        for (int r = 0; r < w; r++) n += (int)((col >> r) & 1u);
    }
    return n;
}

int rso_bitmatrix_ones(int w, uint32_t e) {
    field_t *f = field_for(w);
    if (!f) return -1;
    return ones_of(f, w, e);
}

int rso_goodcauchy_matrix(int w, int k, int m, uint32_t *C) {
    field_t *f;
    if (rso_cauchy_matrix(w, k, m, C)) return -1;
    f = field_for(w);
    for (int j = 0; j < k; j++) {
        uint32_t d = ginv(f, C[j]);
        for (int i = 0; i < m; i++) C[i * k + j] = gmul(f, C[i * k + j], d);
    }
    for (int i = 1; i < m; i++) {
        uint32_t best = 1;
        long best_ones = -1;
        for (int t = -1; t < k; t++) {
            uint32_t v = t < 0 ? 1u : C[i * k + t];
            uint32_t vi = ginv(f, v);
            long ones = 0;
            for (int j = 0; j < k; j++) ones += ones_of(f, w, gmul(f, C[i * k + j], vi));
            if (best_ones < 0 || ones < best_ones) {
                best_ones = ones;
                best = v;
            }
        }
        uint32_t bi = ginv(f, best);
        for (int j = 0; j < k; j++) C[i * k + j] = gmul(f, C[i * k + j], bi);
    }
    return 0;
}

int rso_goodcauchy_encode(int w, int k, int m, uint8_t *blocks, size_t B, size_t P) {
    field_t *f;
    if (cauchy_check(w, k, m, B, P, &f)) return -1;
    uint32_t *C = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)m * k);
    if (!C) return -3;
    rso_goodcauchy_matrix(w, k, m, C);
    int rc = bitmatrix_code_encode(f, w, k, m, C, blocks, B, P);
    free(C);
    return rc;
}

int rso_goodcauchy_decode(int w, int k, int m, const int *er, int e, uint8_t *blocks, size_t B, size_t P) {
    field_t *f;
    if (cauchy_check(w, k, m, B, P, &f)) return -1;
    if (check_erasures(k + m, m, er, e)) return -1;
    uint32_t *C = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)m * k);
    if (!C) return -3;
    rso_goodcauchy_matrix(w, k, m, C);
    int rc = bitmatrix_code_decode(f, w, k, m, C, er, e, blocks, B, P);
    free(C);
    return rc;
}

/* ------------------------------------ polynomial code as a generator matrix */
/* §6 (third direction): a generator polynomial can be turned into a
 * generator matrix.  Column i of the m x k parity matrix holds the
 * remainder of x^(m+i) divided by g(x): the parity of the unit data vector
 * e_i, obtained here by the same long division as the encoder (Eq. 1). */
int rso_polymat_matrix(int w, int k, int m, uint32_t *Pm) {
    field_t *f;
    if (check_code(w, k, m, &f)) return -1;
    uint32_t d[256], p[256];
    if (k > 256 || m > 256) return -1;
    for (int i = 0; i < k; i++) {
        for (int t = 0; t < k; t++) d[t] = (uint32_t)(t == i);
        rso_poly_encode_column(w, k, m, d, p);
        for (int j = 0; j < m; j++) Pm[(size_t)j * k + i] = p[j];
    }
    return 0;
}

/* §6 (first direction): the polynomial code's generator matrix in the
 * bit-matrix (packet) layout of §2.3. */
int rso_polybm_encode(int w, int k, int m, uint8_t *blocks, size_t B, size_t P) {
    field_t *f;
    if (cauchy_check(w, k, m, B, P, &f)) return -1;
    uint32_t *C = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)m * k);
    if (!C) return -3;
    rso_polymat_matrix(w, k, m, C);
    int rc = bitmatrix_code_encode(f, w, k, m, C, blocks, B, P);
    free(C);
    return rc;
}

int rso_polybm_decode(int w, int k, int m, const int *er, int e, uint8_t *blocks, size_t B, size_t P) {
    field_t *f;
    if (cauchy_check(w, k, m, B, P, &f)) return -1;
    if (check_erasures(k + m, m, er, e)) return -1;
    uint32_t *C = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)m * k);
    if (!C) return -3;
    rso_polymat_matrix(w, k, m, C);
    int rc = bitmatrix_code_decode(f, w, k, m, C, er, e, blocks, B, P);
    free(C);
    return rc;
}
