// mont_arith.cuh -- device arithmetic for 32-bit Montgomery residues, R = 2^32.
//
// Montgomery reduction after Meng, Sec. 3.1 (Alg. 2, REDC).  On sm_103a one
// thread is one SIMD lane of the paper's Sec. 3.2, so the 64-bit product T
// arrives directly as its two halves (mul.lo / mul.hi) and no lane gather is
// needed:
//
//   T = a b             -> (lo, hi) = (mul.lo(a, b), mul.hi(a, b))
//   m = (T mod R) P'    -> mul.lo(lo, P')        the "short product" (Sec. 3.1/3.2)
//   t = (T + m P) / R   -> hi + mul.hi(m, P) + carry, where
//                          lo + mul.lo(m, P) == 0 (mod R), so the low words
//                          carry 1 exactly when lo != 0
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
    const uint32_t lo = a * b;
    const uint32_t hi = __umulhi(a, b);
    const uint32_t m = lo * p_prime;
    const uint32_t mh = __umulhi(m, p);
    return hi + mh + (lo != 0u ? 1u : 0u);
}

// Full REDC (Alg. 2): a b R^-1 mod P in [0, P).
__device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b, uint32_t p, uint32_t p_prime)
{
    return csub(redc_lazy(a, b, p, p_prime), p);
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
