/*
 * oracle.c -- plain CPU reference for Montgomery multiplication, the NTT and
 * polynomial multiplication over word-size primes.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It shares no code
 * with the CUDA library.  Every function computes its result from the
 * definition with 64-bit `%` (Meng, Sec. 1-2: the naive modular multiply) and
 * never runs REDC, so it can serve as the check on the REDC-based kernels.
 * R = 2^32 throughout.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_R ((uint64_t)1 << 32)

uint32_t or_mulmod(uint32_t a, uint32_t b, uint32_t p)
{
    return (uint32_t)(((uint64_t)a * b) % p);
}

uint32_t or_powmod(uint32_t a, uint64_t e, uint32_t p)
{
    uint64_t result = 1 % p, base = a % p;
    while (e) {
        if (e & 1) result = (result * base) % p;
        base = (base * base) % p;
        e >>= 1;
    }
    return (uint32_t)result;
}

/* Extended Euclid: returns s with s*a == 1 (mod m), 0 <= s < m; 0 if no inverse. */
uint64_t or_invmod(uint64_t a, uint64_t m)
{
    int64_t old_r = (int64_t)(a % m), r = (int64_t)m;
    int64_t old_s = 1, s = 0;
    while (r != 0) {
        int64_t q = old_r / r, tmp;
        tmp = old_r - q * r; old_r = r; r = tmp;
        tmp = old_s - q * s; old_s = s; s = tmp;
    }
    if (old_r != 1) return 0;
    old_s %= (int64_t)m;
    if (old_s < 0) old_s += (int64_t)m;
    return (uint64_t)old_s;
}

/*
 * Montgomery constants (Sec. 3.1): R^-1 and P' are the integers with
 * 0 < R^-1 < P, 0 < P' < R and R R^-1 - P P' = 1.  R^-1 comes from the
 * extended Euclidean algorithm; P' then follows exactly from the identity.
 */
int or_setup(uint32_t p, or_ctx *out)
{
    if (!out || p < 3 || (p & 1u) == 0 || p >= 0x80000000u) return -1;
    uint64_t r_inv = or_invmod(OR_R % p, p);
    if (r_inv == 0) return -1;
    uint64_t rr = OR_R * r_inv - 1;          /* < 2^63 since r_inv < 2^31 */
    if (rr % p != 0) return -1;
    out->p = p;
    out->r_inv = (uint32_t)r_inv;
    out->p_prime = (uint32_t)(rr / p);
    out->r_mod_p = (uint32_t)(OR_R % p);
    out->r2_mod_p = or_mulmod(out->r_mod_p, out->r_mod_p, p);
    return 0;
}

/* i-bar = i R mod P (Sec. 3.1) */
uint32_t or_to_mont(const or_ctx *c, uint32_t a)
{
    return (uint32_t)(((uint64_t)a << 32) % c->p);
}

uint32_t or_from_mont(const or_ctx *c, uint32_t x)
{
    return or_mulmod(x, c->r_inv, c->p);
}

/* What REDC(x, y) returns (Alg. 2): x y R^-1 mod P, fully reduced. */
uint32_t or_mont_mul(const or_ctx *c, uint32_t x, uint32_t y)
{
    return or_mulmod(or_mulmod(x, y, c->p), c->r_inv, c->p);
}

uint32_t or_mont_fma(const or_ctx *c, uint32_t x, uint32_t y, uint32_t z)
{
    return (uint32_t)(((uint64_t)or_mont_mul(c, x, y) + z) % c->p);
}

void or_to_mont_vec(const or_ctx *c, const uint32_t *in, uint32_t *out, size_t n)
{
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < n; i++) out[i] = or_to_mont(c, in[i]);
}

void or_from_mont_vec(const or_ctx *c, const uint32_t *in, uint32_t *out, size_t n)
{
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < n; i++) out[i] = or_from_mont(c, in[i]);
}

void or_mont_mul_vec(const or_ctx *c, const uint32_t *x, const uint32_t *y, uint32_t *out, size_t n)
{
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < n; i++) out[i] = or_mont_mul(c, x[i], y[i]);
}

void or_mont_fma_vec(const or_ctx *c, const uint32_t *x, const uint32_t *y, const uint32_t *z,
                     uint32_t *out, size_t n)
{
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < n; i++) out[i] = or_mont_fma(c, x[i], y[i], z[i]);
}

void or_mulmod_vec(uint32_t p, const uint32_t *x, const uint32_t *y, uint32_t *out, size_t n)
{
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < n; i++) out[i] = or_mulmod(x[i], y[i], p);
}

/* Smallest g whose order is P - 1: g^((P-1)/q) != 1 for every prime q | P - 1. */
uint32_t or_primitive_root(uint32_t p)
{
    uint32_t factors[32];
    int nf = 0;
    uint32_t m = p - 1;
    for (uint32_t q = 2; (uint64_t)q * q <= m; q++) {
        if (m % q == 0) {
            factors[nf++] = q;
            while (m % q == 0) m /= q;
        }
    }
    if (m > 1) factors[nf++] = m;
    for (uint32_t g = 2; g < p; g++) {
        int ok = 1;
        for (int i = 0; i < nf && ok; i++)
            if (or_powmod(g, (p - 1) / factors[i], p) == 1) ok = 0;
        if (ok) return g;
    }
    return 0;
}

uint32_t or_root_of_unity(uint32_t p, uint64_t n, int inverse)
{
    if (n == 0 || (p - 1) % n != 0) return 0;
    uint32_t w = or_powmod(or_primitive_root(p), (p - 1) / n, p);
    return inverse ? (uint32_t)or_invmod(w, p) : w;
}

/* X_k = sum_j x_j w^(jk); inverse: w -> w^-1 and a final factor N^-1. */
int or_dft(uint32_t p, const uint32_t *x, uint32_t *out, size_t n, int inverse)
{
    if (n == 0) return 0;
    uint32_t w = or_root_of_unity(p, n, inverse);
    if (w == 0) return -1;
    uint32_t *wpow = (uint32_t *)malloc(n * sizeof(uint32_t));
    if (!wpow) return -1;
    wpow[0] = 1 % p;
    for (size_t k = 1; k < n; k++) wpow[k] = or_mulmod(wpow[k - 1], w, p);
    uint32_t ninv = inverse ? (uint32_t)or_invmod(n % p, p) : 1;
#pragma omp parallel for schedule(static)
    for (size_t k = 0; k < n; k++) {
        uint64_t acc = 0;
        for (size_t j = 0; j < n; j++)
            acc = (acc + or_mulmod(x[j], wpow[(uint64_t)j * k % n], p)) % p;
        out[k] = inverse ? or_mulmod((uint32_t)acc, ninv, p) : (uint32_t)acc;
    }
    free(wpow);
    return 0;
}

/*
 * Textbook recursive radix-2 NTT: split into even- and odd-indexed halves,
 * transform each with w^2, then X_k = E_k + w^k O_k, X_{k+n/2} = E_k - w^k O_k.
 */
static void ntt_rec(uint32_t p, const uint32_t *x, size_t stride, size_t n, uint32_t w, uint32_t *out)
{
    if (n == 1) {
        out[0] = x[0];
        return;
    }
    size_t half = n / 2;
    uint32_t w2 = or_mulmod(w, w, p);
    ntt_rec(p, x, 2 * stride, half, w2, out);
    ntt_rec(p, x + stride, 2 * stride, half, w2, out + half);
    uint32_t wk = 1 % p;
    for (size_t k = 0; k < half; k++) {
        uint32_t e = out[k], o = or_mulmod(out[k + half], wk, p);
        out[k] = (uint32_t)(((uint64_t)e + o) % p);
        out[k + half] = (uint32_t)(((uint64_t)e + p - o) % p);
        wk = or_mulmod(wk, w, p);
    }
}

int or_ntt(uint32_t p, const uint32_t *x, uint32_t *out, size_t n, int inverse)
{
    if (n == 0) return 0;
    if (n & (n - 1)) return -1;
    uint32_t w = or_root_of_unity(p, n, inverse);
    if (w == 0) return -1;
    ntt_rec(p, x, 1, n, w, out);
    if (inverse) {
        uint32_t ninv = (uint32_t)or_invmod(n % p, p);
        for (size_t k = 0; k < n; k++) out[k] = or_mulmod(out[k], ninv, p);
    }
    return 0;
}

void or_polymul_schoolbook(uint32_t p, const uint32_t *a, size_t la, const uint32_t *b, size_t lb,
                           uint32_t *c)
{
    if (la == 0 || lb == 0) return;
    size_t lc = la + lb - 1;
    for (size_t k = 0; k < lc; k++) c[k] = 0;
    for (size_t i = 0; i < la; i++)
        for (size_t j = 0; j < lb; j++)
            c[i + j] = (uint32_t)(((uint64_t)c[i + j] + or_mulmod(a[i], b[j], p)) % p);
}

int or_polymul_ntt(uint32_t p, const uint32_t *a, size_t la, const uint32_t *b, size_t lb, uint32_t *c)
{
    if (la == 0 || lb == 0) return -1;
    size_t lc = la + lb - 1, n = 1;
    while (n < lc) n <<= 1;
    if ((p - 1) % n != 0) return -1;
    uint32_t *buf = (uint32_t *)calloc(4 * n, sizeof(uint32_t));
    if (!buf) return -1;
    uint32_t *pa = buf, *pb = buf + n, *fa = buf + 2 * n, *fb = buf + 3 * n;
    memcpy(pa, a, la * sizeof(uint32_t));
    memcpy(pb, b, lb * sizeof(uint32_t));
    or_ntt(p, pa, fa, n, 0);
    or_ntt(p, pb, fb, n, 0);
    for (size_t k = 0; k < n; k++) fa[k] = or_mulmod(fa[k], fb[k], p);
    or_ntt(p, fa, pa, n, 1);
    memcpy(c, pa, lc * sizeof(uint32_t));
    free(buf);
    return 0;
}

/*
 * Truncated Fourier transform (J. van der Hoeven, "The truncated Fourier
 * transform and applications", ISSAC 2004; the paper cites TFT-based
 * polynomial libraries in Sec. 1).  The size-N = 2^K transform is taken in
 * its in-place Cooley-Tukey form: level s = 0 .. K-1 splits the array into
 * 2^s blocks of 2h = N / 2^s entries, and block i pairs (j, j + h) with the
 * twiddle r = w^(brev_s(i) h):  (x, y) -> (x + r y, x - r y).  After level
 * K-1, position q holds X_{brev_K(q)}.  The TFT of x (l entries, zero beyond)
 * is the first l positions of that output; it computes, at each level, only
 * the entries that the remaining levels need to produce them.  Arithmetic by
 * 64-bit `%`, as everywhere in this file.
 */
static uint64_t brev_bits(uint64_t i, int bits)
{
    uint64_t r = 0;
    for (int b = 0; b < bits; b++) r |= ((i >> b) & 1u) << (bits - 1 - b);
    return r;
}

static uint32_t addmod(uint32_t a, uint32_t b, uint32_t p)
{
    return (uint32_t)(((uint64_t)a + b) % p);
}

static uint32_t submod(uint32_t a, uint32_t b, uint32_t p)
{
    return (uint32_t)(((uint64_t)a + p - b) % p);
}

int or_tft(uint32_t p, const uint32_t *x, size_t l, int log2n, uint32_t *out)
{
    if (log2n < 0 || log2n > 30) return -1;
    const size_t n = (size_t)1 << log2n;
    if (l == 0 || l > n) return -1;
    const uint32_t w = or_root_of_unity(p, n, 0);
    if (w == 0) return -1;
    uint32_t *a = (uint32_t *)calloc(n, sizeof(uint32_t));
    if (!a) return -1;
    memcpy(a, x, l * sizeof(uint32_t));
    for (int s = 0; s < log2n; s++) {
        const size_t h = n >> (s + 1);
        const size_t need = (l + h - 1) / h * h;   /* entries later levels read */
        for (size_t b = 0; b < need; b += 2 * h) {
            const uint32_t r = or_powmod(w, brev_bits(b / (2 * h), s) * h, p);
            for (size_t j = b; j < b + h; j++) {
                const uint32_t u = a[j], v = or_mulmod(a[j + h], r, p);
                a[j] = addmod(u, v, p);
                if (j + h < need) a[j + h] = submod(u, v, p);
            }
        }
    }
    memcpy(out, a, l * sizeof(uint32_t));
    free(a);
    return 0;
}

/*
 * Inverse TFT (van der Hoeven's recursion).  Node: block i of level s,
 * `size` = N / 2^s entries at a[0 .. size).  On entry a[0 .. l) holds the
 * node's transform outputs and a[l .. size) its (known) level-s inputs; on
 * return a[0 .. size) holds all of its level-s inputs.  With h = size / 2
 * and r the node's twiddle, the level-s butterfly gives the left child
 * u_j = x_j + r x_{j+h} and the right child v_j = x_j - r x_{j+h}:
 *  - l >= h: the left child's outputs are all known, so its inputs u follow
 *    by recursion; for j >= l - h the right child's input is known too,
 *    v_j = u_j - 2 r x_{j+h}; recursion on the right child gives the other
 *    v_j; then x_j = (u_j + v_j) / 2, x_{j+h} = (u_j - v_j) / (2r).
 *  - l < h: for j >= l the left child's input u_j = x_j + r x_{j+h} is
 *    known; recursion on the left child gives u_j for j < l, and then
 *    x_j = u_j - r x_{j+h}.
 */
static void itft_node(uint32_t p, uint32_t *a, size_t size, int s, uint64_t i, size_t l, uint32_t w, int log2n,
                      uint32_t inv2)
{
    if (size == 1 || l == 0) return;
    const size_t h = size / 2;
    const uint32_t r = or_powmod(w, brev_bits(i, s) * ((uint64_t)1 << (log2n - s - 1)), p);
    if (l >= h) {
        itft_node(p, a, h, s + 1, 2 * i, h, w, log2n, inv2);
        for (size_t j = l - h; j < h; j++) a[h + j] = submod(a[j], or_mulmod(2 % p, or_mulmod(r, a[h + j], p), p), p);
        itft_node(p, a + h, h, s + 1, 2 * i + 1, l - h, w, log2n, inv2);
        const uint32_t inv2r = or_mulmod(inv2, (uint32_t)or_invmod(r, p), p);
        for (size_t j = 0; j < h; j++) {
            const uint32_t u = a[j], v = a[h + j];
            a[j] = or_mulmod(addmod(u, v, p), inv2, p);
            a[h + j] = or_mulmod(submod(u, v, p), inv2r, p);
        }
    } else {
        for (size_t j = l; j < h; j++) a[j] = addmod(a[j], or_mulmod(r, a[h + j], p), p);
        itft_node(p, a, h, s + 1, 2 * i, l, w, log2n, inv2);
        for (size_t j = 0; j < h; j++) a[j] = submod(a[j], or_mulmod(r, a[h + j], p), p);
    }
}

int or_itft(uint32_t p, const uint32_t *y, size_t l, int log2n, uint32_t *out)
{
    if (log2n < 0 || log2n > 30) return -1;
    const size_t n = (size_t)1 << log2n;
    if (l == 0 || l > n) return -1;
    const uint32_t w = or_root_of_unity(p, n, 0);
    if (w == 0) return -1;
    uint32_t *a = (uint32_t *)calloc(n, sizeof(uint32_t));   /* inputs beyond l are zero */
    if (!a) return -1;
    memcpy(a, y, l * sizeof(uint32_t));
    itft_node(p, a, n, 0, 0, l, w, log2n, (uint32_t)((p + 1u) / 2u));
    memcpy(out, a, l * sizeof(uint32_t));
    free(a);
    return 0;
}

/* c = a * b through TFTs of length l = la + lb - 1 in the transform of size
 * 2^ceil(log2 l): the first l outputs of both operands, their pointwise
 * products (the TFT of c, whose degree is below l) and the inverse TFT. */
int or_polymul_tft(uint32_t p, const uint32_t *a, size_t la, const uint32_t *b, size_t lb, uint32_t *c)
{
    if (la == 0 || lb == 0) return -1;
    const size_t l = la + lb - 1;
    int k = 0;
    while (((size_t)1 << k) < l) k++;
    uint32_t *buf = (uint32_t *)calloc(3 * l, sizeof(uint32_t));
    if (!buf) return -1;
    uint32_t *pa = buf, *pb = buf + l, *t = buf + 2 * l;
    memcpy(t, a, la * sizeof(uint32_t));
    int rc = or_tft(p, t, l, k, pa);
    memset(t, 0, l * sizeof(uint32_t));
    memcpy(t, b, lb * sizeof(uint32_t));
    if (rc == 0) rc = or_tft(p, t, l, k, pb);
    for (size_t q = 0; q < l && rc == 0; q++) pa[q] = or_mulmod(pa[q], pb[q], p);
    if (rc == 0) rc = or_itft(p, pa, l, k, c);
    free(buf);
    return rc;
}

int or_polymul_batch(const uint32_t *ps, const uint32_t *a, const uint64_t *a_off, const uint64_t *la,
                     const uint32_t *b, const uint64_t *b_off, const uint64_t *lb, uint32_t *c,
                     const uint64_t *c_off, size_t count, int use_ntt)
{
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(|| : bad)
    for (size_t i = 0; i < count; i++) {
        if (use_ntt) {
            if (or_polymul_ntt(ps[i], a + a_off[i], la[i], b + b_off[i], lb[i], c + c_off[i]) != 0)
                bad = 1;
        } else {
            or_polymul_schoolbook(ps[i], a + a_off[i], la[i], b + b_off[i], lb[i], c + c_off[i]);
        }
    }
    return bad ? -1 : 0;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
