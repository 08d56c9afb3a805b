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
