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
// tw[1 .. 2^Kmax) serves every N <= 2^Kmax.  Entry 2^s (block 0) is 1.
//
// Twiddles are stored in Montgomery form rR mod P.  REDC (Alg. 2) of
// y * rR with y a plain residue returns y r mod P in plain form, so the data
// never leave plain form.
//
// Register passes: each thread holds a group of 2^E elements at stride
// HMIN = N / 2^(S0+E) and applies levels S0 .. S0+E-1 to it in registers
// (radix 2^E, E <= 4, or 5 when a thread holds 32 or more elements); passes
// exchange data through shared memory.  A whole transform lives at word
// j + (j >> 5) (PadLayout: compile-time offsets within a group, at most
// 2-way bank conflicts); column tiles use an XOR layout per column
// (ColLayout, optionally on top of the swizzle swz).
//
// Reductions: REDC (Alg. 2) everywhere by default; FourierREDC (Alg. 3) as
// the RedAlg3 policy for the reduction comparison.  Forward values stay
// lazily in [0, 2P) (see below), inverse values in [0, P).
#pragma once
#include <cstdint>

#include "mont_arith.cuh"

namespace mont {

struct Mod {
    uint32_t p;    // modulus P
    uint32_t pp;   // P' = -P^-1 mod 2^32
};

// Reduction policies for the twiddle and pointwise multiplies: mul(a, b)
// returns a b R^-1 mod P in [0, P) for a < 2P, b < P.  RedAlg2 is REDC
// (Alg. 2) and serves every P < 2^31; RedAlg3 is FourierREDC (Alg. 3) for
// Fourier primes P = c 2^n + 1 < 2^30 with 2n >= 32.  Both give the same
// residue, so tables and results do not depend on the policy.
struct RedAlg2 {
    __device__ __forceinline__ static uint32_t mul(uint32_t a, uint32_t b, Mod m) { return mont_mul(a, b, m.p, m.pp); }
};

struct RedAlg3 {
    __device__ __forceinline__ static uint32_t mul(uint32_t a, uint32_t b, Mod m)
    {
        return fourier_redc(a, b, m.p, m.p - 1u);
    }
};

// Forward values are kept lazily in [0, 2P): with P < 2^31, 2P < R, so the
// sum of two reduced values fits 32 bits, and REDC of a lazy value by a
// reduced twiddle (T < 2P^2 < RP) is below 2P.  Each CT butterfly therefore
// reduces its inputs rather than its outputs (one conditional subtract fewer),
// and level 0, whose inputs are the transform's reduced input, reduces
// nothing.  Whoever consumes a forward result reduces it: the pointwise
// product reduces one factor (REDC of [0, P) x [0, 2P) is below 2P), the
// stand-alone forward transform reduces on store.  Inverse (GS) values stay
// in [0, P).

// CT butterfly: x, y in [0, 2P) -> x + r y, x - r y in [0, 2P).
template <class RED>
__device__ __forceinline__ void bfly_ct(uint32_t &x, uint32_t &y, uint32_t w, Mod m)
{
    const uint32_t t = RED::mul(y, w, m);
    const uint32_t u = csub(x, m.p);
    x = u + t;
    y = u - t + m.p;
}

// CT butterfly with twiddle 1, [0, 2P) in and out.
__device__ __forceinline__ void bfly_ct_one(uint32_t &x, uint32_t &y, Mod m)
{
    const uint32_t u = csub(x, m.p);
    const uint32_t v = csub(y, m.p);
    x = u + v;
    y = u - v + m.p;
}

// CT butterfly with twiddle 1 on reduced inputs (level 0): out in [0, 2P).
__device__ __forceinline__ void bfly_ct_first(uint32_t &x, uint32_t &y, Mod m)
{
    const uint32_t s = x + y;
    y = x - y + m.p;
    x = s;
}

// GS butterfly with twiddle 1, all values in [0, P).
__device__ __forceinline__ void bfly_gs_one(uint32_t &x, uint32_t &y, Mod m)
{
    const uint32_t s = x + y;
    const uint32_t d = x - y + m.p;
    x = csub(s, m.p);
    y = csub(d, m.p);
}

// GS butterfly, all values in [0, P).  x - y + P < 2P is a valid REDC operand
// (one factor < 2P, the other < P keeps T < RP), so it is not reduced first.
template <class RED>
__device__ __forceinline__ void bfly_gs(uint32_t &x, uint32_t &y, uint32_t w, Mod m)
{
    const uint32_t s = x + y;
    const uint32_t d = x - y + m.p;
    x = csub(s, m.p);
    y = RED::mul(d, w, m);
}

__device__ __forceinline__ int swz(int j)
{
    return j ^ (((j >> 4) ^ (j >> 5)) & 31);
}

// CNT consecutive twiddles starting at i0 (i0 a multiple of CNT).
template <int CNT>
__device__ __forceinline__ void load_tw(uint32_t (&w)[CNT], const uint32_t *__restrict__ tw, int i0)
{
    if constexpr (CNT == 1) {
        w[0] = __ldg(tw + i0);
    } else if constexpr (CNT == 2) {
        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(tw + i0));
        w[0] = q.x;
        w[1] = q.y;
    } else {
        const uint4 *v = reinterpret_cast<const uint4 *>(tw + i0);
#pragma unroll
        for (int k = 0; k < CNT / 4; k++) {
            const uint4 q = __ldg(v + k);
            w[4 * k] = q.x;
            w[4 * k + 1] = q.y;
            w[4 * k + 2] = q.z;
            w[4 * k + 3] = q.w;
        }
    }
}

// One forward level (local level L of a group of 2^E elements): 2^L local
// blocks, block lb uses twiddle index 2^(s_abs+L) + (blk << L) + lb.
// FIRST_BLOCK: the group lies in block 0 of the transform at every level
// (blk == 0 and s_abs == 0), so local block 0 has twiddle 1, and local
// level 0 is level 0 of the transform (reduced inputs).
template <int E, int L, int NARR, bool FIRST_BLOCK, class RED>
__device__ __forceinline__ void ct_level(uint32_t (&x)[NARR][1 << E], const uint32_t *__restrict__ tw, int s_abs,
                                         int blk, Mod m)
{
    constexpr int G = 1 << E, HALF = G >> (L + 1), NB = 1 << L;
    uint32_t w[NB];
    if constexpr (NB > 1 || !FIRST_BLOCK) load_tw<NB>(w, tw, (1 << (s_abs + L)) + (blk << L));
#pragma unroll
    for (int lb = 0; lb < NB; lb++)
#pragma unroll
        for (int u = 0; u < HALF; u++)
#pragma unroll
            for (int a = 0; a < NARR; a++) {
                uint32_t &x0 = x[a][lb * 2 * HALF + u];
                uint32_t &x1 = x[a][lb * 2 * HALF + u + HALF];
                if (FIRST_BLOCK && lb == 0) {
                    if constexpr (L == 0) bfly_ct_first(x0, x1, m);
                    else bfly_ct_one(x0, x1, m);
                } else {
                    bfly_ct<RED>(x0, x1, w[lb], m);
                }
            }
}

template <int E, int L, int NARR, bool FIRST_BLOCK, class RED>
__device__ __forceinline__ void gs_level(uint32_t (&x)[NARR][1 << E], const uint32_t *__restrict__ itw, int s_abs,
                                         int blk, Mod m)
{
    constexpr int G = 1 << E, HALF = G >> (L + 1), NB = 1 << L;
    uint32_t w[NB];
    if constexpr (NB > 1 || !FIRST_BLOCK) load_tw<NB>(w, itw, (1 << (s_abs + L)) + (blk << L));
#pragma unroll
    for (int lb = 0; lb < NB; lb++)
#pragma unroll
        for (int u = 0; u < HALF; u++)
#pragma unroll
            for (int a = 0; a < NARR; a++) {
                uint32_t &x0 = x[a][lb * 2 * HALF + u];
                uint32_t &x1 = x[a][lb * 2 * HALF + u + HALF];
                if (FIRST_BLOCK && lb == 0) bfly_gs_one(x0, x1, m);
                else bfly_gs<RED>(x0, x1, w[lb], m);
            }
}

// Forward levels s_abs .. s_abs+E-1 on NARR register groups of 2^E elements
// sharing block index `blk`.
template <int E, int NARR, bool FIRST_BLOCK, class RED = RedAlg2, int L = 0>
__device__ __forceinline__ void ct_group(uint32_t (&x)[NARR][1 << E], const uint32_t *__restrict__ tw, int s_abs,
                                         int blk, Mod m)
{
    if constexpr (L < E) {
        ct_level<E, L, NARR, FIRST_BLOCK, RED>(x, tw, s_abs, blk, m);
        ct_group<E, NARR, FIRST_BLOCK, RED, L + 1>(x, tw, s_abs, blk, m);
    }
}

// Inverse levels s_abs+E-1 .. s_abs (reverse order), same grouping.
template <int E, int NARR, bool FIRST_BLOCK, class RED = RedAlg2, int L = E - 1>
__device__ __forceinline__ void gs_group(uint32_t (&x)[NARR][1 << E], const uint32_t *__restrict__ itw, int s_abs,
                                         int blk, Mod m)
{
    if constexpr (L >= 0) {
        gs_level<E, L, NARR, FIRST_BLOCK, RED>(x, itw, s_abs, blk, m);
        gs_group<E, NARR, FIRST_BLOCK, RED, L - 1>(x, itw, s_abs, blk, m);
    }
}

// Pass schedule for a sub-transform of 2^LOGN elements: ceil(LOGN / EMAX)
// passes of (nearly) equal numbers of levels, at most EMAX each, larger
// passes first.
template <int LOGN, int EMAX = 4>
struct Sched {
    static constexpr int kPasses = LOGN <= 0 ? 0 : (LOGN + EMAX - 1) / EMAX;
    static constexpr int levels(int i) { return LOGN / kPasses + (i < LOGN % kPasses ? 1 : 0); }
    static constexpr int start(int i) { return i == 0 ? 0 : start(i - 1) + levels(i - 1); }
};

constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

// Schedule for NT threads: a pass covers up to 4 levels (radix-16 groups),
// 5 (radix-32) when each thread holds 32 or more elements per array, which
// saves a shared-memory round trip for 2^13 elements on 256 threads.
template <int LOGN, int NT>
using SchedFor = Sched<LOGN, (LOGN - ilog2(NT) >= 5 ? 5 : 4)>;

// Geometry of pass I of a 2^LOGN sub-transform processed by NT threads, each
// holding EPT = 2^LOGN / NT elements per array (EPT / 2^E groups).  Group q
// (of NT * GPT) starts at element ((q / HMIN) << (LOGN - S0)) + q % HMIN;
// thread tid takes groups grp(tid) + NT r.
//
// PADDED (the PadLayout, one padding word per 32): a warp whose lanes run
// over 32 / HMIN blocks of HMIN * G words sees block b's words shifted by
// b * HMIN * G / 32 banks, so with G = 16 and HMIN = 8 or 16 (the middle
// passes of 2^11 .. 2^13) consecutive blocks overlap: 2-way conflicts.
// grp then hands the warp's HMIN-lane segments blocks D = 32 / G apart,
// shifting each segment by HMIN banks, and the warp covers 32 banks.
template <int LOGN, int NT, int I, bool PADDED = false>
struct PassGeom {
    static constexpr int S0 = SchedFor<LOGN, NT>::start(I);
    static constexpr int E = SchedFor<LOGN, NT>::levels(I);
    static constexpr int G = 1 << E;
    static constexpr int LOG_HMIN = LOGN - S0 - E;
    static constexpr int HMIN = 1 << LOG_HMIN;
    static constexpr int GPT = (1 << LOGN) / G / NT;
    static_assert(GPT >= 1, "too many threads for this sub-transform");
    static constexpr int D = G < 32 ? 32 / G : 1;
    static constexpr bool REMAP =
        PADDED && HMIN >= 2 && HMIN < 32 && G < 32 && HMIN * G >= 32 && NT % (32 * D) == 0;
    __device__ __forceinline__ static int grp(int tid)
    {
        if constexpr (!REMAP) {
            return tid;
        } else {
            constexpr int NB = 32 / HMIN;   // blocks one warp touches
            const int w = tid >> 5, l = tid & 31;
            const int block = (w / D) * (D * NB) + (w % D) + (l / HMIN) * D;
            return block * HMIN + (l % HMIN);
        }
    }
    // block index (at level S0) and first element of group r of thread tid
    __device__ __forceinline__ static int blk(int tid, int r) { return (grp(tid) + NT * r) >> LOG_HMIN; }
    __device__ __forceinline__ static int base(int tid, int r)
    {
        const int q = grp(tid) + NT * r;
        return ((q >> LOG_HMIN) << (LOGN - S0)) + (q & (HMIN - 1));
    }
};

// ---------------------------------------------------------------- layouts
//
// A layout maps element j of a sub-transform to its shared-memory word.

// Whole transform in one buffer with the XOR swizzle.
struct SwzLayout {
    uint32_t *base;
    static constexpr bool kAdditive = false;
    __device__ __forceinline__ uint32_t &operator[](int j) const { return base[swz(j)]; }
};

// Whole transform in one buffer with one padding word after every 32:
// word(j) = j + (j >> 5).  For j = base + t*HMIN with base and t*HMIN on
// disjoint bits (true for every group of every pass), word(j) =
// word(base) + word(t*HMIN), so each element of a group is addressed as a
// per-group pointer plus a compile-time offset, with no index arithmetic.
// Banks: the strided group accesses are at most 2-way conflicted.
struct PadLayout {
    uint32_t *base;
    static constexpr bool kAdditive = true;
    static constexpr int words(int n) { return n + (n >> 5); }
    __host__ __device__ static constexpr int off(int j) { return j + (j >> 5); }
    __device__ __forceinline__ uint32_t &operator[](int j) const { return base[off(j)]; }
    __device__ __forceinline__ uint32_t *at(int j) const { return base + off(j); }
};

// Element base + k of a layout (k a compile-time offset after unrolling,
// on bits disjoint from base).
template <class L>
__device__ __forceinline__ uint32_t &elem(const L &lay, int base, int k)
{
    if constexpr (L::kAdditive) return lay.at(base)[L::off(k)];
    else return lay[base + k];
}

// Column c of a column tile: base = c * (N1 + PAD), XOR of the low five bits
// with XR = (c * MUL) & 31, optionally on top of swz.  Chosen per column size
// so that the coalesced tile loads and the strided pass accesses hit distinct
// banks.
template <bool SW>
struct ColLayout {
    uint32_t *base;
    int xr;
    static constexpr bool kAdditive = false;
    __device__ __forceinline__ uint32_t &operator[](int j) const { return base[(SW ? swz(j) : j) ^ xr]; }
};

// ---------------------------------------------------------------- passes
//
// Pass I of a 2^LOGN sub-transform whose level s_loc is level s_base + s_loc
// of the whole transform and which is block b of 2^s_base blocks
// (twiddle index 2^(s_base+s_loc) + (b << s_loc) + local block).  BASE0:
// s_base is known to be 0 (and b = 0), so pass 0 lies in block 0 of every
// level and its local block 0 has twiddle 1.

// The NARR arrays are transformed one after the other (the twiddles are
// reloaded from L1 for each), which keeps one group live at a time.
template <int LOGN, int NT, int I, int NARR, bool BASE0, class RED = RedAlg2, class L>
__device__ __forceinline__ void fwd_pass(const L (&lay)[NARR], int tid, const uint32_t *__restrict__ tw, int s_base,
                                         int b, Mod m)
{
    using PG = PassGeom<LOGN, NT, I, L::kAdditive>;
#pragma unroll
    for (int a = 0; a < NARR; a++)
#pragma unroll
        for (int r = 0; r < PG::GPT; r++) {
            const int base = PG::base(tid, r), blk = PG::blk(tid, r);
            uint32_t x[1][PG::G];
#pragma unroll
            for (int t = 0; t < PG::G; t++) x[0][t] = elem(lay[a], base, t * PG::HMIN);
            ct_group<PG::E, 1, BASE0 && PG::S0 == 0, RED>(x, tw, s_base + PG::S0, (b << PG::S0) + blk, m);
#pragma unroll
            for (int t = 0; t < PG::G; t++) elem(lay[a], base, t * PG::HMIN) = x[0][t];
        }
}

template <int LOGN, int NT, int I, bool BASE0, class RED = RedAlg2, class L>
__device__ __forceinline__ void inv_pass(const L &lay, int tid, const uint32_t *__restrict__ itw, int s_base, int b,
                                         Mod m)
{
    using PG = PassGeom<LOGN, NT, I, L::kAdditive>;
#pragma unroll
    for (int r = 0; r < PG::GPT; r++) {
        const int base = PG::base(tid, r), blk = PG::blk(tid, r);
        uint32_t x[1][PG::G];
#pragma unroll
        for (int t = 0; t < PG::G; t++) x[0][t] = elem(lay, base, t * PG::HMIN);
        gs_group<PG::E, 1, BASE0 && PG::S0 == 0, RED>(x, itw, s_base + PG::S0, (b << PG::S0) + blk, m);
#pragma unroll
        for (int t = 0; t < PG::G; t++) elem(lay, base, t * PG::HMIN) = x[0][t];
    }
}

// Forward passes I .. LAST, each followed by a CTA barrier.
template <int LOGN, int NT, int NARR, bool BASE0, int I, int LAST, class RED = RedAlg2, class L>
__device__ __forceinline__ void fwd_passes(const L (&lay)[NARR], int tid, const uint32_t *__restrict__ tw,
                                           int s_base, int b, Mod m)
{
    if constexpr (I <= LAST) {
        fwd_pass<LOGN, NT, I, NARR, BASE0, RED>(lay, tid, tw, s_base, b, m);
        __syncthreads();
        fwd_passes<LOGN, NT, NARR, BASE0, I + 1, LAST, RED>(lay, tid, tw, s_base, b, m);
    }
}

// Inverse passes I, I-1, .. FIRST, each followed by a CTA barrier.
template <int LOGN, int NT, bool BASE0, int I, int FIRST, class RED = RedAlg2, class L>
__device__ __forceinline__ void inv_passes(const L &lay, int tid, const uint32_t *__restrict__ itw, int s_base, int b,
                                           Mod m)
{
    if constexpr (I >= FIRST) {
        inv_pass<LOGN, NT, I, BASE0, RED>(lay, tid, itw, s_base, b, m);
        __syncthreads();
        inv_passes<LOGN, NT, BASE0, I - 1, FIRST, RED>(lay, tid, itw, s_base, b, m);
    }
}

// Last forward pass of both operands, pointwise REDC product (A B~ R^-1, one
// lazy factor reduced first),
// then the same levels of the inverse in reverse, result into lay[0].
template <int LOGN, int NT, bool BASE0, class RED = RedAlg2, class L>
__device__ __forceinline__ void fused_middle_pass(const L (&lay)[2], int tid, const uint32_t *__restrict__ tw,
                                                  const uint32_t *__restrict__ itw, int s_base, int b, Mod m)
{
    using PL = PassGeom<LOGN, NT, SchedFor<LOGN, NT>::kPasses - 1>;
#pragma unroll
    for (int r = 0; r < PL::GPT; r++) {
        const int base = PL::base(tid, r), blk = (b << PL::S0) + PL::blk(tid, r);
        uint32_t x[2][PL::G];
#pragma unroll
        for (int t = 0; t < PL::G; t++) {
            x[0][t] = elem(lay[0], base, t * PL::HMIN);
            x[1][t] = elem(lay[1], base, t * PL::HMIN);
        }
        ct_group<PL::E, 2, BASE0 && PL::S0 == 0, RED>(x, tw, s_base + PL::S0, blk, m);
        uint32_t y[1][PL::G];
#pragma unroll
        for (int t = 0; t < PL::G; t++) y[0][t] = RED::mul(csub(x[0][t], m.p), x[1][t], m);
        gs_group<PL::E, 1, BASE0 && PL::S0 == 0, RED>(y, itw, s_base + PL::S0, blk, m);
#pragma unroll
        for (int t = 0; t < PL::G; t++) elem(lay[0], base, t * PL::HMIN) = y[0][t];
    }
}

// ---------------------------------------------------------------- inverse TFT

// x / 2 mod P for x in [0, P): x >> 1, plus (P + 1) / 2 when x is odd.
__device__ __forceinline__ uint32_t half_mod(uint32_t x, uint32_t p)
{
    return (x >> 1) + ((x & 1u) ? (p >> 1) + 1u : 0u);
}

// Inverse truncated Fourier transform of one column (van der Hoeven's
// recursion) over node `block I of level S` of the column transform, SIZE
// entries at x[OFF ..): on entry x[OFF .. OFF + L) holds the node's outputs
// (bit-reversed order) and x[OFF + L .. OFF + SIZE) its level-S inputs; on
// return x[OFF .. OFF + SIZE) holds all of its level-S inputs.  The node's
// butterfly is (x, y) -> (x + r y, x - r y) with r = tw[2^S + I]:
//  - L >= SIZE/2: the left child's inputs u follow from its (all known)
//    outputs; the right child's inputs v_j = u_j - 2 r x_{j+h} are known for
//    j >= L - h, the rest follow from its L - h outputs; then
//    x_j = (u_j + v_j) / 2 and x_{j+h} = (u_j - v_j) / (2 r);
//  - L < SIZE/2: for j >= L the left child's input u_j = x_j + r x_{j+h} is
//    known, the others follow from its L outputs, then x_j = u_j - r x_{j+h}.
// All values in [0, P); every division is exact (no deferred scale factor).
// Used by the inverse column passes of truncated products (row-granular
// TFT): the column transforms are block 0 of levels 0 .. K1-1, so node
// (S, I) of a column is block I of level S of the whole transform.
template <int N1, int OFF, int SIZE, int L, int S, int I>
__device__ __forceinline__ void itft_node(uint32_t (&x)[N1], const uint32_t *__restrict__ tw,
                                          const uint32_t *__restrict__ itw, Mod m)
{
    if constexpr (SIZE > 1 && L > 0) {
        constexpr int H = SIZE / 2;
        const uint32_t r = __ldg(tw + (1 << S) + I);   // Montgomery form: REDC(y, r) = y w
        if constexpr (L >= H) {
            itft_node<N1, OFF, H, H, S + 1, 2 * I>(x, tw, itw, m);
            const uint32_t r2 = add_mod(r, r, m.p);
#pragma unroll
            for (int j = L - H; j < H; j++)
                x[OFF + H + j] = sub_mod(x[OFF + j], mont_mul(x[OFF + H + j], r2, m.p, m.pp), m.p);
            itft_node<N1, OFF + H, H, L - H, S + 1, 2 * I + 1>(x, tw, itw, m);
            const uint32_t ri = __ldg(itw + (1 << S) + I);
#pragma unroll
            for (int j = 0; j < H; j++) {
                const uint32_t u = x[OFF + j], v = x[OFF + H + j];
                x[OFF + j] = half_mod(add_mod(u, v, m.p), m.p);
                x[OFF + H + j] = half_mod(mont_mul(u - v + m.p, ri, m.p, m.pp), m.p);
            }
        } else {
#pragma unroll
            for (int j = L; j < H; j++) x[OFF + j] = add_mod(x[OFF + j], mont_mul(x[OFF + H + j], r, m.p, m.pp), m.p);
            itft_node<N1, OFF, H, L, S + 1, 2 * I>(x, tw, itw, m);
#pragma unroll
            for (int j = 0; j < H; j++) x[OFF + j] = sub_mod(x[OFF + j], mont_mul(x[OFF + H + j], r, m.p, m.pp), m.p);
        }
    }
}

}  // namespace mont
