// ntt_core.cuh -- shared-memory NTT passes with Montgomery twiddle multiplies.
//
// Transform (the modular FFT the paper's libraries compute, Sec. 1 and 5):
// X_k = sum_j x_j w^(jk) mod P, w = g^((P-1)/N), N = 2^K.
//
// Forward: Cooley-Tukey levels s = 0 .. K-1, natural order in, bit-reversed
// order out.  At level s the array splits into 2^s blocks of 2h elements
// (h = N / 2^(s+1)); block i pairs (j, j+h) and uses ONE twiddle
// r = tw[2^s + i] = w_(2^(s+1))^bitrev_s(i):   (x, y) -> (x + r y, x - r y).
// Inverse: Gentleman-Sande levels s = K-1 .. 0 with r^-1:
// (x, y) -> (x + y, (x - y) r^-1), which undoes a forward level up to a
// factor 2; the caller applies N^-1.
// Because w_(2^(s+1)) = g^((P-1)/2^(s+1)) does not depend on N, one table
// tw[1 .. 2^Kmax) serves every N <= 2^Kmax.
//
// Twiddles are stored in Montgomery form as pairs (r R mod P, (r R mod P) P'
// mod R), so REDC (Alg. 2) of y * rR needs no mul.lo for T: m = (T mod R) P'
// mod R = y ((rR) P' mod R) mod R is one mul.lo of y by the precomputed
// word (the short product of Sec. 3.1/3.2), and with y plain the result is
// y r mod P in plain form.
//
// Register passes: each thread holds a group of 2^E elements at stride
// HMIN = N / 2^(S0+E) and applies levels S0 .. S0+E-1 to it in registers
// (radix 2^E); passes exchange data through shared memory.  Shared-memory
// index j is stored at swz(j), an XOR swizzle of the low five bits that keeps
// the strided group accesses of every pass (nearly) free of bank conflicts
// and never leaves the aligned 32-word segment (identity for j < 16).
#pragma once
#include <cstdint>

#include "mont_arith.cuh"

namespace mont {

// Montgomery product y * w (w = (wR mod P, (wR mod P) P' mod R)) without the
// final subtract: y w mod P + {0, P}, in [0, 2P) for y < 2P.
__device__ __forceinline__ uint32_t redc_tw(uint32_t y, uint2 w, uint32_t p)
{
    const uint32_t hi = __umulhi(y, w.x);
    const uint32_t m = y * w.y;
    const uint32_t mh = __umulhi(m, p);
    // (T + mP) / R = hi + mh + carry: the low words T mod R and mP mod R sum to
    // 0 or R, carrying exactly when m != 0 (m = 0 iff T mod R = 0).
    uint32_t t;
    asm("{\n\t.reg .u32 d;\n\tadd.cc.u32 d, %1, 0xffffffff;\n\taddc.u32 %0, %2, %3;\n\t}"
        : "=r"(t)
        : "r"(m), "r"(hi), "r"(mh));
    return t;
}

// CT butterfly, all values in [0, P).
__device__ __forceinline__ void bfly_ct(uint32_t &x, uint32_t &y, uint2 w, uint32_t p)
{
    const uint32_t t = csub(redc_tw(y, w, p), p);
    const uint32_t s = x + t;
    const uint32_t d = x - t + p;
    x = csub(s, p);
    y = csub(d, p);
}

// CT butterfly with twiddle 1.
__device__ __forceinline__ void bfly_ct1(uint32_t &x, uint32_t &y, uint32_t p)
{
    const uint32_t s = x + y;
    const uint32_t d = x - y + p;
    x = csub(s, p);
    y = csub(d, p);
}

// GS butterfly, all values in [0, P).  x - y + P < 2P is a valid REDC operand
// (one factor < 2P, the other < P keeps T < RP), so it is not reduced first.
__device__ __forceinline__ void bfly_gs(uint32_t &x, uint32_t &y, uint2 w, uint32_t p)
{
    const uint32_t s = x + y;
    const uint32_t d = x - y + p;
    x = csub(s, p);
    y = csub(redc_tw(d, w, p), p);
}

__device__ __forceinline__ int swz(int j)
{
    return j ^ (((j >> 4) ^ (j >> 5)) & 31);
}

// CNT consecutive twiddle pairs starting at i0 (i0 a multiple of CNT).
template <int CNT>
__device__ __forceinline__ void load_tw(uint2 (&w)[CNT], const uint2 *__restrict__ tw, int i0)
{
    if constexpr (CNT == 1) {
        w[0] = __ldg(tw + i0);
    } else {
        const uint4 *v = reinterpret_cast<const uint4 *>(tw + i0);
#pragma unroll
        for (int k = 0; k < CNT / 2; k++) {
            const uint4 q = __ldg(v + k);
            w[2 * k] = make_uint2(q.x, q.y);
            w[2 * k + 1] = make_uint2(q.z, q.w);
        }
    }
}

// One forward level (local level L of a group of 2^E elements): 2^L local
// blocks, block lb uses twiddle index 2^(s_abs+L) + (blk << L) + lb.
// TRIVIAL: this is level 0 of the whole transform (twiddle 1).
template <int E, int L, int NARR, bool TRIVIAL>
__device__ __forceinline__ void ct_level(uint32_t (&x)[NARR][1 << E], const uint2 *__restrict__ tw,
                                         int s_abs, int blk, uint32_t p)
{
    constexpr int G = 1 << E, HALF = G >> (L + 1), NB = 1 << L;
    if constexpr (TRIVIAL) {
#pragma unroll
        for (int u = 0; u < G / 2; u++)
#pragma unroll
            for (int a = 0; a < NARR; a++) bfly_ct1(x[a][u], x[a][u + G / 2], p);
    } else {
        uint2 w[NB];
        load_tw<NB>(w, tw, (1 << (s_abs + L)) + (blk << L));
#pragma unroll
        for (int lb = 0; lb < NB; lb++)
#pragma unroll
            for (int u = 0; u < HALF; u++)
#pragma unroll
                for (int a = 0; a < NARR; a++)
                    bfly_ct(x[a][lb * 2 * HALF + u], x[a][lb * 2 * HALF + u + HALF], w[lb], p);
    }
}

template <int E, int L, int NARR, bool TRIVIAL>
__device__ __forceinline__ void gs_level(uint32_t (&x)[NARR][1 << E], const uint2 *__restrict__ itw,
                                         int s_abs, int blk, uint32_t p)
{
    constexpr int G = 1 << E, HALF = G >> (L + 1), NB = 1 << L;
    if constexpr (TRIVIAL) {
#pragma unroll
        for (int u = 0; u < G / 2; u++)
#pragma unroll
            for (int a = 0; a < NARR; a++) bfly_ct1(x[a][u], x[a][u + G / 2], p);
    } else {
        uint2 w[NB];
        load_tw<NB>(w, itw, (1 << (s_abs + L)) + (blk << L));
#pragma unroll
        for (int lb = 0; lb < NB; lb++)
#pragma unroll
            for (int u = 0; u < HALF; u++)
#pragma unroll
                for (int a = 0; a < NARR; a++)
                    bfly_gs(x[a][lb * 2 * HALF + u], x[a][lb * 2 * HALF + u + HALF], w[lb], p);
    }
}

// Forward levels s_abs .. s_abs+E-1 on NARR register groups of 2^E elements
// sharing block index `blk`.  TRIVIAL0: s_abs is level 0 of the transform.
template <int E, int NARR, bool TRIVIAL0, int L = 0>
__device__ __forceinline__ void ct_group(uint32_t (&x)[NARR][1 << E], const uint2 *__restrict__ tw,
                                         int s_abs, int blk, uint32_t p)
{
    if constexpr (L < E) {
        ct_level<E, L, NARR, TRIVIAL0 && L == 0>(x, tw, s_abs, blk, p);
        ct_group<E, NARR, TRIVIAL0, L + 1>(x, tw, s_abs, blk, p);
    }
}

// Inverse levels s_abs+E-1 .. s_abs (reverse order), same grouping.
template <int E, int NARR, bool TRIVIAL0, int L = E - 1>
__device__ __forceinline__ void gs_group(uint32_t (&x)[NARR][1 << E], const uint2 *__restrict__ itw,
                                         int s_abs, int blk, uint32_t p)
{
    if constexpr (L >= 0) {
        gs_level<E, L, NARR, TRIVIAL0 && L == 0>(x, itw, s_abs, blk, p);
        gs_group<E, NARR, TRIVIAL0, L - 1>(x, itw, s_abs, blk, p);
    }
}

// Pass schedule for a sub-transform of 2^LOGN elements: ceil(LOGN / 4)
// passes of (nearly) equal numbers of levels, at most 4 each.
template <int LOGN>
struct Sched {
    static constexpr int kPasses = LOGN <= 0 ? 0 : (LOGN + 3) / 4;
    static constexpr int levels(int i) { return LOGN / kPasses + (i < LOGN % kPasses ? 1 : 0); }
    static constexpr int start(int i) { return i == 0 ? 0 : start(i - 1) + levels(i - 1); }
};

// Geometry of pass I of a 2^LOGN sub-transform processed by NT threads, each
// holding EPT = 2^LOGN / NT elements per array (EPT / 2^E groups).
template <int LOGN, int NT, int I>
struct PassGeom {
    static constexpr int S0 = Sched<LOGN>::start(I);
    static constexpr int E = Sched<LOGN>::levels(I);
    static constexpr int G = 1 << E;
    static constexpr int LOG_HMIN = LOGN - S0 - E;
    static constexpr int HMIN = 1 << LOG_HMIN;
    static constexpr int GPT = (1 << LOGN) / G / NT;
    static_assert(GPT >= 1, "too many threads for this sub-transform");
    // element index of item t of group r handled by thread tid
    __device__ __forceinline__ static int blk(int tid, int r) { return (tid + NT * r) >> LOG_HMIN; }
    __device__ __forceinline__ static int base(int tid, int r)
    {
        const int q = tid + NT * r;
        return ((q >> LOG_HMIN) << (LOGN - S0)) + (q & (HMIN - 1));
    }
};

// ---------------------------------------------------------------- layouts
//
// A layout maps element j of a sub-transform to its shared-memory word.

// Whole transform in one buffer with the XOR swizzle.
struct SwzLayout {
    uint32_t *base;
    __device__ __forceinline__ uint32_t &operator[](int j) const { return base[swz(j)]; }
};

// Column c of a column tile: base = c * (N1 + PAD), XOR of the low five bits
// with XR = (c * MUL) & 31, optionally on top of swz.  Chosen per column size
// so that the coalesced tile loads and the strided pass accesses hit distinct
// banks.
template <bool SW>
struct ColLayout {
    uint32_t *base;
    int xr;
    __device__ __forceinline__ uint32_t &operator[](int j) const { return base[(SW ? swz(j) : j) ^ xr]; }
};

// ---------------------------------------------------------------- passes
//
// Pass I of a 2^LOGN sub-transform whose level s_loc is level s_base + s_loc
// of the whole transform and which is block b of 2^s_base blocks
// (twiddle index 2^(s_base+s_loc) + (b << s_loc) + local block).  BASE0:
// s_base is known to be 0, so local level 0 has twiddle 1.

template <int LOGN, int NT, int I, int NARR, bool BASE0, class L>
__device__ __forceinline__ void fwd_pass(const L (&lay)[NARR], int tid, const uint2 *__restrict__ tw, int s_base,
                                         int b, uint32_t p)
{
    using PG = PassGeom<LOGN, NT, I>;
#pragma unroll
    for (int r = 0; r < PG::GPT; r++) {
        const int base = PG::base(tid, r), blk = PG::blk(tid, r);
        uint32_t x[NARR][PG::G];
#pragma unroll
        for (int a = 0; a < NARR; a++)
#pragma unroll
            for (int t = 0; t < PG::G; t++) x[a][t] = lay[a][base + t * PG::HMIN];
        ct_group<PG::E, NARR, BASE0 && PG::S0 == 0>(x, tw, s_base + PG::S0, (b << PG::S0) + blk, p);
#pragma unroll
        for (int a = 0; a < NARR; a++)
#pragma unroll
            for (int t = 0; t < PG::G; t++) lay[a][base + t * PG::HMIN] = x[a][t];
    }
}

template <int LOGN, int NT, int I, bool BASE0, class L>
__device__ __forceinline__ void inv_pass(const L &lay, int tid, const uint2 *__restrict__ itw, int s_base, int b,
                                         uint32_t p)
{
    using PG = PassGeom<LOGN, NT, I>;
#pragma unroll
    for (int r = 0; r < PG::GPT; r++) {
        const int base = PG::base(tid, r), blk = PG::blk(tid, r);
        uint32_t x[1][PG::G];
#pragma unroll
        for (int t = 0; t < PG::G; t++) x[0][t] = lay[base + t * PG::HMIN];
        gs_group<PG::E, 1, BASE0 && PG::S0 == 0>(x, itw, s_base + PG::S0, (b << PG::S0) + blk, p);
#pragma unroll
        for (int t = 0; t < PG::G; t++) lay[base + t * PG::HMIN] = x[0][t];
    }
}

// Forward passes I .. LAST, each followed by a CTA barrier.
template <int LOGN, int NT, int NARR, bool BASE0, int I, int LAST, class L>
__device__ __forceinline__ void fwd_passes(const L (&lay)[NARR], int tid, const uint2 *__restrict__ tw, int s_base,
                                           int b, uint32_t p)
{
    if constexpr (I <= LAST) {
        fwd_pass<LOGN, NT, I, NARR, BASE0>(lay, tid, tw, s_base, b, p);
        __syncthreads();
        fwd_passes<LOGN, NT, NARR, BASE0, I + 1, LAST>(lay, tid, tw, s_base, b, p);
    }
}

// Inverse passes I, I-1, .. FIRST, each followed by a CTA barrier.
template <int LOGN, int NT, bool BASE0, int I, int FIRST, class L>
__device__ __forceinline__ void inv_passes(const L &lay, int tid, const uint2 *__restrict__ itw, int s_base, int b,
                                           uint32_t p)
{
    if constexpr (I >= FIRST) {
        inv_pass<LOGN, NT, I, BASE0>(lay, tid, itw, s_base, b, p);
        __syncthreads();
        inv_passes<LOGN, NT, BASE0, I - 1, FIRST>(lay, tid, itw, s_base, b, p);
    }
}

// Last forward pass of both operands, pointwise REDC product (A B~ R^-1),
// then the same levels of the inverse in reverse, result into lay[0].
template <int LOGN, int NT, bool BASE0, class L>
__device__ __forceinline__ void fused_middle_pass(const L (&lay)[2], int tid, const uint2 *__restrict__ tw,
                                                  const uint2 *__restrict__ itw, int s_base, int b, uint32_t p,
                                                  uint32_t pp)
{
    using PL = PassGeom<LOGN, NT, Sched<LOGN>::kPasses - 1>;
#pragma unroll
    for (int r = 0; r < PL::GPT; r++) {
        const int base = PL::base(tid, r), blk = (b << PL::S0) + PL::blk(tid, r);
        uint32_t x[2][PL::G];
#pragma unroll
        for (int t = 0; t < PL::G; t++) {
            x[0][t] = lay[0][base + t * PL::HMIN];
            x[1][t] = lay[1][base + t * PL::HMIN];
        }
        ct_group<PL::E, 2, BASE0 && PL::S0 == 0>(x, tw, s_base + PL::S0, blk, p);
        uint32_t y[1][PL::G];
#pragma unroll
        for (int t = 0; t < PL::G; t++) y[0][t] = mont_mul(x[0][t], x[1][t], p, pp);
        gs_group<PL::E, 1, BASE0 && PL::S0 == 0>(y, itw, s_base + PL::S0, blk, p);
#pragma unroll
        for (int t = 0; t < PL::G; t++) lay[0][base + t * PL::HMIN] = y[0][t];
    }
}

}  // namespace mont
