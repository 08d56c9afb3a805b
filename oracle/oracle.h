/*
 * oracle.h -- plain, slow, obviously-correct CPU reference for the Montgomery
 * multiplication / NTT / polynomial-multiplication path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA product path
 * shares no code, header, table or constant generator with it.
 *
 * Every value here is computed from its definition with 64-bit integer
 * arithmetic and the `%` operator (the "naive" modular multiply of Meng,
 * "Automatic Generation of Vectorized Montgomery Algorithm", Sec. 1 and 2),
 * never with REDC itself:
 *   mulmod(a, b)       = (uint64)a * b % P
 *   to_mont(a)         = a * R mod P                       (Sec. 3.1, residue i-bar = iR mod P)
 *   from_mont(x)       = x * R^-1 mod P
 *   mont_mul(x, y)     = x * y * R^-1 mod P                (Sec. 3.1, what REDC returns, Alg. 2)
 *   mont_fma(x, y, z)  = (x * y * R^-1 + z) mod P
 *   R^-1, P'           : 0 < R^-1 < P, 0 < P' < R, R R^-1 - P P' = 1 (Sec. 3.1),
 *                        from the extended Euclidean algorithm.
 *   DFT_N(x)_k         = sum_j x_j w^(jk) mod P, w = g^((P-1)/N), g the smallest
 *                        primitive root of P; the inverse includes N^-1.
 *   polymul            = schoolbook convolution c_k = sum_{i+j=k} a_i b_j mod P.
 * R = 2^32 throughout.  P must be odd with 3 <= P < 2^31.
 */
#ifndef MONT_ORACLE_H
#define MONT_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    uint32_t p;        /* modulus P                                  */
    uint32_t p_prime;  /* P' with R R^-1 - P P' = 1, 0 < P' < R       */
    uint32_t r_inv;    /* R^-1 mod P, 0 < R^-1 < P                    */
    uint32_t r_mod_p;  /* R mod P                                     */
    uint32_t r2_mod_p; /* R^2 mod P                                   */
} or_ctx;

/* 0 on success, -1 if P is even, < 3 or >= 2^31. */
int or_setup(uint32_t p, or_ctx *out);

uint32_t or_mulmod(uint32_t a, uint32_t b, uint32_t p);
uint32_t or_powmod(uint32_t a, uint64_t e, uint32_t p);
/* Multiplicative inverse of a modulo m (gcd(a, m) = 1), by extended Euclid. */
uint64_t or_invmod(uint64_t a, uint64_t m);

/* Scalar forms of the Montgomery-domain operations (definitions above). */
uint32_t or_to_mont(const or_ctx *c, uint32_t a);
uint32_t or_from_mont(const or_ctx *c, uint32_t x);
uint32_t or_mont_mul(const or_ctx *c, uint32_t x, uint32_t y);
uint32_t or_mont_fma(const or_ctx *c, uint32_t x, uint32_t y, uint32_t z);

/* Vector forms: one independent scalar call per element (OpenMP over elements). */
void or_to_mont_vec(const or_ctx *c, const uint32_t *in, uint32_t *out, size_t n);
void or_from_mont_vec(const or_ctx *c, const uint32_t *in, uint32_t *out, size_t n);
void or_mont_mul_vec(const or_ctx *c, const uint32_t *x, const uint32_t *y, uint32_t *out, size_t n);
void or_mont_fma_vec(const or_ctx *c, const uint32_t *x, const uint32_t *y, const uint32_t *z,
                     uint32_t *out, size_t n);
void or_mulmod_vec(uint32_t p, const uint32_t *x, const uint32_t *y, uint32_t *out, size_t n);

/* Smallest primitive root of prime P (trial factorisation of P - 1). */
uint32_t or_primitive_root(uint32_t p);
/* Principal N-th root of unity w_N = g^((P-1)/N) (its inverse if inverse != 0);
 * 0 if N does not divide P - 1. */
uint32_t or_root_of_unity(uint32_t p, uint64_t n, int inverse);

/* Direct O(N^2) DFT over Z_P (natural order in and out).  inverse != 0 uses
 * w^-1 and multiplies by N^-1.  Returns -1 if N does not divide P - 1. */
int or_dft(uint32_t p, const uint32_t *x, uint32_t *out, size_t n, int inverse);
/* Textbook recursive radix-2 (even/odd split) NTT, same result as or_dft.
 * N must be a power of two dividing P - 1. */
int or_ntt(uint32_t p, const uint32_t *x, uint32_t *out, size_t n, int inverse);

/* Schoolbook product c[0 .. la+lb-2] = a * b mod P. */
void or_polymul_schoolbook(uint32_t p, const uint32_t *a, size_t la, const uint32_t *b, size_t lb,
                           uint32_t *c);
/* Same product through or_ntt (zero padding to the next power of two >= la+lb-1). */
int or_polymul_ntt(uint32_t p, const uint32_t *a, size_t la, const uint32_t *b, size_t lb,
                   uint32_t *c);

/* Batches of independent products (OpenMP over products).  Product i uses
 * prime ps[i], operands at a + a_off[i] (length la[i]), b + b_off[i] (lb[i]),
 * result at c + c_off[i] (la[i] + lb[i] - 1).  use_ntt selects or_polymul_ntt. */
int or_polymul_batch(const uint32_t *ps, const uint32_t *a, const uint64_t *a_off, const uint64_t *la,
                     const uint32_t *b, const uint64_t *b_off, const uint64_t *lb, uint32_t *c,
                     const uint64_t *c_off, size_t count, int use_ntt);

/* Threads an OpenMP region of this library uses. */
/* Truncated Fourier transform (van der Hoeven 2004) of x (l entries, zero
 * beyond) in the transform of size N = 2^log2n >= l: out[q] = X_{brev(q)}
 * for q < l, X the DFT of the zero-padded x (the in-place Cooley-Tukey
 * output order).  -1 for l == 0, l > N or no N-th root of unity mod p. */
int or_tft(uint32_t p, const uint32_t *x, size_t l, int log2n, uint32_t *out);
/* Inverse: the x (l entries, zero beyond) whose TFT is y. */
int or_itft(uint32_t p, const uint32_t *y, size_t l, int log2n, uint32_t *out);
/* c = a * b (la + lb - 1 entries) through TFTs of length la + lb - 1. */
int or_polymul_tft(uint32_t p, const uint32_t *a, size_t la, const uint32_t *b, size_t lb, uint32_t *c);
int or_num_threads(void);
/* Threads of the OpenMP loops from now on (n > 0); timing only. */
void or_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
