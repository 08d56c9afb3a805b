// mont_arith.cuh -- device arithmetic for 32-bit Montgomery residues, R = 2^32.
//
// Montgomery reduction after Meng, Sec. 3.1 (Alg. 2, REDC).  On sm_103a one
// thread is one SIMD lane of the paper's Sec. 3.2, so the 64-bit product T
// arrives in one register pair (its mul.lo / mul.hi halves) and no lane
// gather is needed:
//
//   T = a b             -> mul.wide.u32: both 32-bit halves of the product
//   m = (T mod R) P'    -> mul.lo(lo(T), P')     the "short product" (Sec. 3.1/3.2)
//   t = (T + m P) / R   -> mad.wide.u32 m, P, T and keep the high word: the
//                          64-bit sum is exact (T + mP < 2RP < 2^64) and its
//                          low word is 0, so the carry out of the low words
//                          is folded into the one multiply-add
//   t >= P ? t - P : t  -> min(t, t - P) as unsigned (t - P wraps above t when t < P)
//
// Requirements (Alg. 2): 0 <= a b < R P.  With P < 2^31 this holds whenever
// one operand is < 2P and the other < P, and then t < 2P < R.
#pragma once
#include <cstdint>

namespace mont {

// Conditional subtract: [0, 2P) -> [0, P).
__device__ __forceinline__ uint32_t csub(uint32_t t, uint32_t p)
{
    return min(t, t - p);
}

// REDC of T = a b without the final subtract: returns t in [0, 2P).
__device__ __forceinline__ uint32_t redc_lazy(uint32_t a, uint32_t b, uint32_t p, uint32_t p_prime)
{
    const uint64_t T = static_cast<uint64_t>(a) * b;
    const uint32_t m = static_cast<uint32_t>(T) * p_prime;
    return static_cast<uint32_t>((static_cast<uint64_t>(m) * p + T) >> 32);
}

// Full REDC (Alg. 2): a b R^-1 mod P in [0, P).
__device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b, uint32_t p, uint32_t p_prime)
{
    return csub(redc_lazy(a, b, p, p_prime), p);
}

// Alg. 3 (Montgomery over the Fourier prime P = c 2^n + 1, R = 2^32, 2n >= 32):
// q1 = ab / R, r1 = ab mod R, (q2, r2) = (c 2^n r1) / R, mod R,
// q3 = (c 2^n r2) / R, t = q1 - q2 + q3 in (-(P-1), 2(P-1)), then the
// sign-mask corrections.  The 31-bit sign tests need 2(P-1) < 2^31, i.e.
// P < 2^30.  w = c 2^n = P - 1.  Result: ab R^-1 mod P in [0, P), as REDC.
// One operand may be lazy (< 2P): q1 < 2P^2 / R < P / 2 keeps t in the same
// interval.
__device__ __forceinline__ uint32_t fourier_redc(uint32_t a, uint32_t b, uint32_t p, uint32_t w)
{
    const uint64_t T = static_cast<uint64_t>(a) * b;
    const uint32_t q1 = static_cast<uint32_t>(T >> 32), r1 = static_cast<uint32_t>(T);
    const uint64_t U = static_cast<uint64_t>(r1) * w;
    const uint32_t q2 = static_cast<uint32_t>(U >> 32), r2 = static_cast<uint32_t>(U);
    const uint32_t q3 = __umulhi(r2, w);
    int32_t t = static_cast<int32_t>(q1 - q2 + q3);
    t += (t >> 31) & static_cast<int32_t>(p);
    t -= static_cast<int32_t>(p);
    t += (t >> 31) & static_cast<int32_t>(p);
    return static_cast<uint32_t>(t);
}

// (x + y) mod P for x, y in [0, P).
__device__ __forceinline__ uint32_t add_mod(uint32_t x, uint32_t y, uint32_t p)
{
    return csub(x + y, p);
}

// (x - y) mod P for x, y in [0, P).
__device__ __forceinline__ uint32_t sub_mod(uint32_t x, uint32_t y, uint32_t p)
{
    const uint32_t d = x - y;
    return min(d, d + p);
}

}  // namespace mont
