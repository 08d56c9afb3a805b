// polymul_batch.cu -- many products of uneven sizes and mixed primes in one
// persistent kernel launch, or in the phased form's few kernels (either
// optionally replayed as a CUDA graph).
//
// The host turns the batch into a job list.  A product with N <= 2^13 is
// computed whole by one team of threads (SMALL job; a job covers as many
// products of one size as fit in a 256-thread CTA; 2^12 and 2^13 take the
// whole CTA).  A product with N = 2^K > 2^13 is split as in ntt_large.cu
// (K1 = K - 13 column levels, rows of 2^13): COLF jobs run the forward
// column levels of both operands on a block of columns, ROW jobs run one row
// (forward row levels, pointwise product, inverse row levels), COLI jobs run
// the inverse column levels of a block of columns and write c.  Columns of
// up to 2^4 elements are transformed in registers straight from and to
// global memory; longer ones go through shared-memory tiles.  Split products
// up to 2^15 run as one WHOLE job instead: one CTA runs their rows (column
// levels computed on load) and the output column pass in sequence (no
// waits; their scratch stays in L2).
// Scratch: 2N words per large product.
//
// CTAs of the persistent grid claim jobs in list order with one atomic
// counter (each CTA one job ahead of the one it runs).  A ROW job waits until every COLF tile of its product has
// finished, a COLI job until every ROW of its product has; both waits only
// depend on jobs earlier in the list, which were claimed by running CTAs,
// so the grid always makes progress.  Each wait is bounded (iterations and
// elapsed time); on expiry the CTA sets the error word, skips the job and
// the host reports MONT_ETIMEOUT.
//
// Truncated products (Prod::tft) compute only the rows of 2^13 their output
// reaches and invert each column with an inverse TFT (itft_node).  The
// phased form (further below) runs the same jobs as one kernel per job kind
// in stream order, with no waits.
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "batch_internal.cuh"

namespace mont {
namespace {

// Shared memory per CTA: one 2^13 product (both operands, padded layout).
constexpr int kSmemWords = team_smem_words<kSmallLog>();

// Column tile geometry for a 256-thread CTA: columns of N1 = 2^K1 at stride
// N1 + PAD, NT1 threads per column, C0 = 256 / NT1 columns per round and C
// columns per tile, so each thread runs ROUNDS = C / C0 columns one after
// the other.  Layouts as in ntt_large.cu: column c XORs its low five bits
// with (c * MUL) & 31, which makes the tile loads conflict-free and the pass
// accesses nearly so.  Where that pattern repeats every C0 columns (every
// round then sees the same banks), C is the most columns (a power of two, at
// most a row) whose two operands fit kSmemWords; otherwise C = C0.
constexpr int col_nt1(int k1) { return k1 <= 4 ? 1 : (1 << k1) / 16; }
constexpr int col_mul(int k1) { return k1 <= 4 ? 0 : ((k1 == 5 || k1 == 8) ? 17 : 9); }
constexpr int col_stride(int k1) { return (1 << k1) + (k1 <= 4 ? 1 : 0); }
constexpr int col_tile_cols(int k1)
{
    const int c0 = kThreads / col_nt1(k1);
    if ((c0 * col_mul(k1)) % 32 != 0) return c0;
    int c = 1 << kRowLog;
    while (c > c0 && 2 * c * col_stride(k1) > kSmemWords) c >>= 1;
    return c;
}

template <int K1>
struct ColTile {
    static constexpr int N1 = 1 << K1;
    static constexpr int NT1 = col_nt1(K1);
    static constexpr int C0 = kThreads / NT1;
    static constexpr int C = col_tile_cols(K1);
    static constexpr int ROUNDS = C / C0;
    static constexpr int MUL = col_mul(K1);
    static constexpr bool SW = K1 >= 8;
    static constexpr int STRIDE = col_stride(K1);
    static constexpr int WORDS = C * STRIDE;
    static_assert(ROUNDS >= 1 && C % C0 == 0 && (ROUNDS == 1 || (C0 * MUL) % 32 == 0), "column tile geometry");
    static_assert(2 * WORDS <= kSmemWords, "column tile does not fit");
};

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Coherent at GPU scope but without acquire ordering: polling with it does
// not invalidate the SM's L1 (which an acquire load does, for every CTA on
// the SM) on each poll.
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 only: wait until *ctr >= target, bounded by iterations and time.
// Gives up at once when another CTA has already recorded an expired wait, so
// a failed batch costs at most about one wait limit in total.
__device__ bool bounded_wait(const uint32_t *ctr, uint32_t target, const BatchArgs &A)
{
    const uint32_t *err = A.sync + 1;
    const unsigned long long t0 = globaltimer();
    for (uint32_t it = 0;; it++) {
        // Relaxed polls; once the count is reached, one acquire load (the
        // counter only grows, so it sees it too) orders the caller's reads of
        // the producers' data after their writes.
        if (ld_relaxed(ctr) >= target) return ld_acquire(ctr) >= target;
        if (ld_relaxed(err) != 0u || it >= A.wait_iters || globaltimer() - t0 > A.wait_ns) return false;
        __nanosleep(200);
    }
}

// A thread's share of a C x N1 column tile: PER elements, u = 0 .. PER-1, at
// column c0 + dc(u) and row t0 + dt(u), in the order of a CTA-wide sweep of
// the tile in row-major order (consecutive threads on consecutive columns,
// so global accesses are coalesced).  dc(u) is a multiple of 256 columns,
// under which the XOR pattern of ColLayout repeats, so a thread's XOR value
// is fixed; element u then sits at a compile-time offset from the thread's
// first element, in global memory as in shared memory.
template <class CF>
struct TileShare {
    static constexpr bool WIDE = CF::C >= kThreads;
    static constexpr int PER = CF::C * CF::N1 / kThreads;
    static constexpr int dc(int u) { return WIDE ? (u * kThreads) % CF::C : 0; }
    static constexpr int dt(int u) { return WIDE ? (u * kThreads) / CF::C : u * (kThreads / CF::C); }
    static constexpr int goff(int u) { return dc(u) + (dt(u) << kRowLog); }   // from the first element
    int c0, t0, xr;
    __device__ explicit TileShare(int tx)
        : c0(WIDE ? tx : tx % CF::C), t0(WIDE ? 0 : tx / CF::C), xr((c0 * CF::MUL) & 31)
    {
    }
    __device__ int rel0() const { return c0 + (t0 << kRowLog); }
    // Shared-memory word of element u relative to the thread's column base
    // (the same word ColLayout gives for that column and row).
    __device__ int soff(int u) const
    {
        const int t = t0 + dt(u);
        return dc(u) * CF::STRIDE + ((CF::SW ? swz(t) : t) ^ xr);
    }
};

// Elements of a product from the thread's first element (o0 + rel0) to the
// end of a length-len array, clamped to [-1, 2^30].
__device__ __forceinline__ int room_of(size_t len, size_t first)
{
    if (len <= first) return -1;
    const size_t r = len - first;
    return r > (size_t{1} << 30) ? (1 << 30) : static_cast<int>(r);
}

template <int K1, bool INV>
__device__ __forceinline__ void col_tile(uint32_t *smem, const Prod &P, const PrimeInfo &pr, uint32_t tile)
{
    using CF = ColTile<K1>;
    using TS = TileShare<CF>;
    constexpr int NP = SchedFor<K1, ColTile<K1>::NT1>::kPasses;
    constexpr int NARR = INV ? 1 : 2;
    const size_t n = size_t{1} << P.k;
    const size_t o0 = static_cast<size_t>(tile) * CF::C;
    const Mod md{pr.p, pr.pp};
    const TS ts(threadIdx.x);
    const size_t first = o0 + ts.rel0();
    auto col = [&](int a, int c) {
        return ColLayout<CF::SW>{smem + a * CF::WORDS + c * CF::STRIDE, (c * CF::MUL) & 31};
    };
    // Tile loads: one cp.async per element (zero-filled past the operand's
    // end), so all of a thread's loads are in flight together; then each
    // thread scales the b elements it copied (b N^-1 R^2 R^-1).
#pragma unroll
    for (int a = 0; a < NARR; a++) {
        const uint32_t *base = INV ? P.ws : (a ? P.b : P.a);
        const int room = room_of(INV ? n : (a ? P.lb : P.la), first);
        const uint32_t *src = base + first;
        uint32_t *sm = smem + a * CF::WORDS + ts.c0 * CF::STRIDE;
#pragma unroll 8
        for (int u = 0; u < TS::PER; u++) {
            const bool in = TS::goff(u) < room;
            cp_async4(sm + ts.soff(u), in ? src + TS::goff(u) : base, in ? 4u : 0u);
        }
    }
    cp_async_wait_all();
    if constexpr (!INV) {
        uint32_t *sm = smem + CF::WORDS + ts.c0 * CF::STRIDE;
#pragma unroll 8
        for (int u = 0; u < TS::PER; u++) sm[ts.soff(u)] = mont_mul(sm[ts.soff(u)], P.k_scale, pr.p, pr.pp);
    }
    __syncthreads();
    const int tid = threadIdx.x % CF::NT1;
#pragma unroll 1
    for (int r = 0; r < CF::ROUNDS; r++) {
        const int c = threadIdx.x / CF::NT1 + r * CF::C0;
        if constexpr (!INV) {
            const ColLayout<CF::SW> lay[2] = {col(0, c), col(1, c)};
            fwd_passes<K1, CF::NT1, 2, true, 0, NP - 1>(lay, tid, pr.tw, 0, 0, md);
        } else {
            inv_passes<K1, CF::NT1, true, NP - 1, 0>(col(0, c), tid, pr.itw, 0, 0, md);
        }
    }
#pragma unroll
    for (int a = 0; a < NARR; a++) {
        uint32_t *dst = (INV ? P.c : P.ws + a * n) + first;
        const int room = INV ? room_of(P.lc, first) : (1 << 30);
        const uint32_t *sm = smem + a * CF::WORDS + ts.c0 * CF::STRIDE;
#pragma unroll 8
        for (int u = 0; u < TS::PER; u++)
            if (TS::goff(u) < room) dst[TS::goff(u)] = sm[ts.soff(u)];
    }
}

// Hint that the 128-byte line holding p will be read soon: fetched into L2,
// no register written, nothing to wait for.
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Columns per job for the register column jobs: 2^14 elements per operand.
constexpr int reg_cols(int k1) { return (1 << 14) >> k1 < (1 << kRowLog) ? (1 << 14) >> k1 : (1 << kRowLog); }

// Column levels 0 .. K1-1 (K1 <= 4) of reg_cols(K1) consecutive columns of
// one product, in registers: thread tx takes columns o0 + tx + 256 m, G at a
// time (G x 2^K1 <= 16 elements per operand), element t of column c being
// word c + (t << kRowLog).  A warp's load or store of one (column, row) slot
// covers 32 consecutive words, and all of a thread's loads of a step are
// independent, so they are in flight together.  The columns of a step share
// their twiddles (levels 0 .. K1-1, block 0 of the transform), so they run
// as the NARR arrays of one register group.  A warp's slots of a step are
// NA x 2^K1 whole 128-byte lines; while a step loads, lane l asks L2 for
// line l of the warp's next step (one prefetch per thread), so the next
// step's loads find their lines in L2.
template <int K1, bool INV>
__device__ __forceinline__ void col_regs(const Prod &P, const PrimeInfo &pr, uint32_t tile)
{
    constexpr int N1 = 1 << K1, G = 16 / N1, STEPS = reg_cols(K1) / kThreads / G;
    constexpr int NA = INV ? G : 2 * G;
    static_assert(STEPS >= 1 && reg_cols(K1) % (kThreads * G) == 0, "register column job geometry");
    static_assert(NA * N1 <= 32, "one line per lane");
    const size_t n = size_t{1} << P.k;
    const Mod md{pr.p, pr.pp};
    const size_t c0 = static_cast<size_t>(tile) * reg_cols(K1) + threadIdx.x;
    const int lane = threadIdx.x & 31;
    auto prefetch_step = [&](int st) {
        if (st >= STEPS || lane >= NA * N1) return;
        const int arr = lane / N1, t = lane % N1;   // slot (array, row) of this lane's line
        const size_t j = c0 - lane + static_cast<size_t>(st) * G * kThreads + (arr % G) * kThreads +
                         (static_cast<size_t>(t) << kRowLog);
        if constexpr (!INV) {
            const bool opb = arr >= G;
            if (j < (opb ? P.lb : P.la)) prefetch_l2((opb ? P.b : P.a) + j);
        } else {
            prefetch_l2(P.ws + j);
        }
    };
#pragma unroll 1
    for (int st = 0; st < STEPS; st++) {
        const size_t cs = c0 + static_cast<size_t>(st) * G * kThreads;
        uint32_t x[NA][N1];
        prefetch_step(st + 1);
        if constexpr (!INV) {
#pragma unroll
            for (int a = 0; a < 2; a++) {
                const uint32_t *src = a ? P.b : P.a;
                const size_t len = a ? P.lb : P.la;
#pragma unroll
                for (int g = 0; g < G; g++)
#pragma unroll
                    for (int t = 0; t < N1; t++) {
                        const size_t j = cs + g * kThreads + (static_cast<size_t>(t) << kRowLog);
                        x[a * G + g][t] = j < len ? __ldg(src + j) : 0u;
                    }
            }
#pragma unroll
            for (int g = 0; g < G; g++)
#pragma unroll
                for (int t = 0; t < N1; t++) x[G + g][t] = mont_mul(x[G + g][t], P.k_scale, pr.p, pr.pp);
            ct_group<K1, NA, true>(x, pr.tw, 0, 0, md);
            // Row t of the column outputs goes to scratch row t; a truncated
            // product (tft) computes and reads only its first nrows rows.
#pragma unroll
            for (int a = 0; a < 2; a++)
#pragma unroll
                for (int g = 0; g < G; g++)
#pragma unroll
                    for (int t = 0; t < N1; t++)
                        if (static_cast<uint32_t>(t) < P.nrows)
                            P.ws[a * n + cs + g * kThreads + (static_cast<size_t>(t) << kRowLog)] = x[a * G + g][t];
        } else {
#pragma unroll
            for (int g = 0; g < G; g++)
#pragma unroll
                for (int t = 0; t < N1; t++)
                    x[g][t] = P.ws[cs + g * kThreads + (static_cast<size_t>(t) << kRowLog)];
            gs_group<K1, NA, true>(x, pr.itw, 0, 0, md);
#pragma unroll
            for (int g = 0; g < G; g++)
#pragma unroll
                for (int t = 0; t < N1; t++) {
                    const size_t j = cs + g * kThreads + (static_cast<size_t>(t) << kRowLog);
                    if (j < P.lc) P.c[j] = x[g][t];
                }
        }
    }
}

// Inverse column pass of a truncated split product (K1 <= 4 column levels,
// L = nrows rows computed): the columns of reg_cols(K1) consecutive columns,
// each an inverse TFT of its L known outputs (the rows) with its inputs
// beyond L known to be zero (c is zero from L x 2^13 on), written to c.
template <int K1, int L>
__device__ __forceinline__ void col_regs_itft(const Prod &P, const PrimeInfo &pr, uint32_t tile)
{
    constexpr int N1 = 1 << K1, G = 16 / N1, STEPS = reg_cols(K1) / kThreads / G;
    const Mod md{pr.p, pr.pp};
    const size_t c0 = static_cast<size_t>(tile) * reg_cols(K1) + threadIdx.x;
    const int lane = threadIdx.x & 31;
    auto prefetch_step = [&](int st) {               // line (g, t) of the warp's step st, as in col_regs
        if (st >= STEPS || lane >= G * L) return;
        prefetch_l2(P.ws + (c0 - lane + static_cast<size_t>(st) * G * kThreads) + (lane / L) * kThreads +
                    (static_cast<size_t>(lane % L) << kRowLog));
    };
#pragma unroll 1
    for (int st = 0; st < STEPS; st++) {
        const size_t cs = c0 + static_cast<size_t>(st) * G * kThreads;
        uint32_t x[G][N1];
        prefetch_step(st + 1);
#pragma unroll
        for (int g = 0; g < G; g++)
#pragma unroll
            for (int t = 0; t < N1; t++)
                x[g][t] = t < L ? P.ws[cs + g * kThreads + (static_cast<size_t>(t) << kRowLog)] : 0u;
#pragma unroll
        for (int g = 0; g < G; g++) itft_node<N1, 0, N1, L, 0, 0>(x[g], pr.tw, pr.itw, md);
#pragma unroll
        for (int g = 0; g < G; g++)
#pragma unroll
            for (int t = 0; t < L; t++) {
                const size_t j = cs + g * kThreads + (static_cast<size_t>(t) << kRowLog);
                if (j < P.lc) P.c[j] = x[g][t];
            }
    }
}

template <int K1>
__device__ __forceinline__ void col_itft_dispatch(const Prod &P, const PrimeInfo &pr, uint32_t tile)
{
    // nrows lies in (2^(K1-1), 2^K1): the product is longer than half of N.
    if constexpr (K1 == 2) {
        col_regs_itft<2, 3>(P, pr, tile);
    } else if constexpr (K1 == 3) {
        switch (P.nrows) {
        case 5: col_regs_itft<3, 5>(P, pr, tile); break;
        case 6: col_regs_itft<3, 6>(P, pr, tile); break;
        default: col_regs_itft<3, 7>(P, pr, tile); break;
        }
    } else if constexpr (K1 == 4) {
        switch (P.nrows) {
        case 9: col_regs_itft<4, 9>(P, pr, tile); break;
        case 10: col_regs_itft<4, 10>(P, pr, tile); break;
        case 11: col_regs_itft<4, 11>(P, pr, tile); break;
        case 12: col_regs_itft<4, 12>(P, pr, tile); break;
        case 13: col_regs_itft<4, 13>(P, pr, tile); break;
        case 14: col_regs_itft<4, 14>(P, pr, tile); break;
        default: col_regs_itft<4, 15>(P, pr, tile); break;
        }
    }
}

// Row r of a split product with K1 <= 2 column levels, the column levels
// computed as the row is loaded: element j of the row is element r of the
// forward column transform of the 2^K1 inputs at j + i 2^13 (levels
// 0 .. K1-1, block 0 of the transform: twiddles tw[1 .. 2^K1 - 1]); b's is
// then multiplied by k_scale (the transform is linear, so this equals
// scaling its inputs).  Inputs reduced, results below 2P (lazy forward
// values, as the row passes take them).
template <int K1>
struct ColFusedLoad {
    const uint32_t *a, *b;
    uint32_t la, lb, k_scale;
    Mod m;
    const uint32_t *tw;
    int r;
    __device__ __forceinline__ uint32_t operator()(int arr, int j) const
    {
        const uint32_t *g = arr ? b : a;
        const uint32_t len = arr ? lb : la;
        uint32_t x[1][1 << K1];
#pragma unroll
        for (int i = 0; i < (1 << K1); i++) {
            const uint32_t idx = static_cast<uint32_t>(j) + (static_cast<uint32_t>(i) << kRowLog);
            x[0][i] = idx < len ? __ldg(g + idx) : 0u;
        }
        ct_group<K1, 1, true>(x, tw, 0, 0, m);
        uint32_t v = x[0][0];
#pragma unroll
        for (int i = 1; i < (1 << K1); i++) v = r == i ? x[0][i] : v;
        return arr ? RedAlg2::mul(v, k_scale, m) : v;
    }
};

// Operand source reading a row already staged in shared memory (padded
// layout); pass 0 then transforms it in place.
struct StagedLoad {
    PadLayout lay[2];
    __device__ __forceinline__ uint32_t operator()(int arr, int j) const { return lay[arr][j]; }
};

// All jobs of one split product (K1 <= 2) by this CTA: each row stages its
// operands into shared memory with the column levels computed as they are
// loaded (no forward scratch round trip; the inputs are read 2^K1 times,
// from L2 after the first), runs the row levels, the pointwise product and
// the inverse row levels into scratch; then the inverse column pass writes
// c.  The barriers make the rows' scratch writes visible to the column
// pass's coherent loads.
template <int K1>
__device__ __forceinline__ void whole_job(uint32_t *smem, const Prod &P, const PrimeInfo &pr)
{
    static_assert(K1 <= 2, "whole jobs recompute at most two column levels per row");
    constexpr int N2 = 1 << kRowLog;
    const Mod md{pr.p, pr.pp};
    const StagedLoad staged{{{smem}, {smem + PadLayout::words(N2)}}};
    for (uint32_t r = 0; r < P.nrows; r++) {
        const ColFusedLoad<K1> ld{P.a, P.b, P.la, P.lb, P.k_scale, md, pr.tw, static_cast<int>(r)};
#pragma unroll 2
        for (int j = threadIdx.x; j < N2; j += kThreads) {
            staged.lay[0][j] = ld(0, j);
            staged.lay[1][j] = ld(1, j);
        }
        __syncthreads();
        uint32_t *row = P.ws + (static_cast<size_t>(r) << kRowLog);
        polymul_team_ld<kRowLog, false, kThreads, RedAlg2>(smem, threadIdx.x, staged, row, size_t{1} << kRowLog,
                                                           pr.tw, pr.itw, K1, static_cast<int>(r), md);
        __syncthreads();
    }
    if (P.tft) {
        if constexpr (K1 >= kMinTftColLog)
            for (uint32_t t = 0; t < P.ntiles; t++) col_itft_dispatch<K1>(P, pr, t);
    } else {
        for (uint32_t t = 0; t < P.ntiles; t++) col_regs<K1, true>(P, pr, t);
    }
}

__device__ __forceinline__ void whole_dispatch(uint32_t *smem, const Prod &P, const PrimeInfo &pr)
{
    static_assert(kWholeMaxLog - kRowLog <= 2, "extend the dispatch");
    switch (P.k - kRowLog) {
    case 1: whole_job<1>(smem, P, pr); break;
    case 2: whole_job<2>(smem, P, pr); break;
    default: break;
    }
}

template <bool INV>
__device__ __forceinline__ void col_job(uint32_t *smem, const Prod &P, const PrimeInfo &pr, uint32_t tile)
{
    if (INV && P.tft) {
        switch (P.k - kRowLog) {
        case 2: col_itft_dispatch<2>(P, pr, tile); break;
        case 3: col_itft_dispatch<3>(P, pr, tile); break;
        case 4: col_itft_dispatch<4>(P, pr, tile); break;
        default: break;
        }
        return;
    }
    switch (P.k - kRowLog) {
    case 1: col_regs<1, INV>(P, pr, tile); break;
    case 2: col_regs<2, INV>(P, pr, tile); break;
    case 3: col_regs<3, INV>(P, pr, tile); break;
    case 4: col_regs<4, INV>(P, pr, tile); break;
    case 5: col_tile<5, INV>(smem, P, pr, tile); break;
    case 6: col_tile<6, INV>(smem, P, pr, tile); break;
    case 7: col_tile<7, INV>(smem, P, pr, tile); break;
    case 8: col_tile<8, INV>(smem, P, pr, tile); break;
    default: break;
    }
}

template <int K>
__device__ __forceinline__ void small_job(uint32_t *smem, const BatchArgs &A, const Job &J)
{
    constexpr int NT = nt_of<K>() < kThreads ? nt_of<K>() : kThreads, T = kThreads / NT;
    const int team = threadIdx.x / NT, tid = threadIdx.x - team * NT;
    const bool valid = static_cast<uint32_t>(team) < J.idx;
    const Prod &P = A.prods[J.prod + (valid ? team : 0)];
    const PrimeInfo &pr = A.primes[P.prime];
    static_assert(T * team_smem_words<K>() <= kSmemWords, "small job does not fit");
    polymul_team<K, true, true, NT>(smem + team * team_smem_words<K>(), tid, P.a, valid ? P.la : 0, P.b, valid ? P.lb : 0, P.c,
                                valid ? P.lc : 0, pr.tw, pr.itw, 0, 0, pr.p, pr.pp, P.k_scale);
}

__device__ __forceinline__ void small_dispatch(uint32_t *smem, const BatchArgs &A, const Job &J)
{
    switch (J.k) {
    case 0: small_job<0>(smem, A, J); break;
    case 1: small_job<1>(smem, A, J); break;
    case 2: small_job<2>(smem, A, J); break;
    case 3: small_job<3>(smem, A, J); break;
    case 4: small_job<4>(smem, A, J); break;
    case 5: small_job<5>(smem, A, J); break;
    case 6: small_job<6>(smem, A, J); break;
    case 7: small_job<7>(smem, A, J); break;
    case 8: small_job<8>(smem, A, J); break;
    case 9: small_job<9>(smem, A, J); break;
    case 10: small_job<10>(smem, A, J); break;
    case 11: small_job<11>(smem, A, J); break;
    case 12: small_job<12>(smem, A, J); break;
    case 13: small_job<13>(smem, A, J); break;
    default: break;
    }
}

// MINB: CTAs per SM the registers are budgeted for (2: up to 128 registers;
// 3: up to 85, a few spills, more warps to hide memory latency).  The
// autotuner picks one.
template <int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_polymul_batch(BatchArgs A)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ uint32_t s_job;
    __shared__ int s_ok;
    uint32_t *err = A.sync + 1;
    // Thread 0 claims one job ahead: the claim of a CTA's next job is issued
    // when its current job starts, so the atomic's round trip overlaps the
    // work.  Progress still holds: every job waits only on earlier jobs, a
    // CTA finishes its current job before its next, so the earliest
    // unfinished job is always some CTA's current job and can run.
    uint32_t next = 0;
    if (threadIdx.x == 0) {
        s_job = atomicAdd(A.sync, 1u);
        next = atomicAdd(A.sync, 1u);
    }
    for (;;) {
        __syncthreads();
        const uint32_t jid = s_job;
        if (jid >= A.njobs) break;
        const Job J = A.jobs[jid];
        if (J.type == JOB_SMALL) {
            small_dispatch(smem, A, J);
        } else if (J.type == JOB_WHOLE) {
            const Prod &P = A.prods[J.prod];
            whole_dispatch(smem, P, A.primes[P.prime]);
        } else {
            const Prod &P = A.prods[J.prod];
            const PrimeInfo &pr = A.primes[P.prime];
            uint32_t *done = A.sync + 2 + 2 * static_cast<size_t>(J.prod);
            if (J.type != JOB_COLF && threadIdx.x == 0) {
                const bool ok = J.type == JOB_ROW ? bounded_wait(done, P.ntiles, A)
                                                  : bounded_wait(done + 1, P.nrows, A);
                if (!ok) atomicOr(err, 1u);
                s_ok = ok;
            }
            __syncthreads();
            const bool ok = J.type == JOB_COLF || s_ok;
            // Thread 0's acquire load of the counter, then the barrier, orders
            // every thread's reads of the producers' data after their writes.
            if (ok) {
                if (J.type == JOB_COLF) {
                    col_job<false>(smem, P, pr, J.idx);
                } else if (J.type == JOB_ROW) {
                    uint32_t *row = P.ws + (static_cast<size_t>(J.idx) << kRowLog);
                    const size_t n = size_t{1} << P.k;
                    polymul_team<kRowLog, false, false, kThreads>(smem, threadIdx.x, row, size_t{1} << kRowLog, row + n,
                                                        size_t{1} << kRowLog, row, size_t{1} << kRowLog, pr.tw,
                                                        pr.itw, static_cast<int>(P.k) - kRowLog,
                                                        static_cast<int>(J.idx), pr.p, pr.pp, 0u);
                } else {
                    col_job<true>(smem, P, pr, J.idx);
                }
            }
            __syncthreads();
            if (ok && threadIdx.x == 0 && J.type != JOB_COLI) {
                __threadfence();
                atomicAdd(J.type == JOB_COLF ? done : done + 1, 1u);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_job = next;
            next = atomicAdd(A.sync, 1u);
        }
    }
}

// ---------------------------------------------------------------- phased form
//
// The same products as separate kernels, one CTA per job (or per team of
// small products), ordered by stream dependencies instead of device-side
// waits: every kernel gets the register budget of its own job kind.  A
// batch runs as: small products (one kernel per size, N <= 2^13) on a side
// branch, and every larger product's forward column tiles, then its rows,
// then its output tiles on the main branch (products of 2^14 and 2^15 too:
// without waits to avoid, splitting them is 1 % faster for the uneven
// workload than one CTA per product recomputing its column levels row by
// row); the host joins the branches (polymul_batch_run / the graph of
// polymul_batch_run_graph).  No kernel waits on another's progress.

// Products prods[first .. first + count), all of size 2^K (K <= 13), one
// team each, teams_of<K>() per CTA.
template <int K>
__global__ void __launch_bounds__(teams_of<K>() * nt_of<K>(), min_ctas_of<K>())
k_phase_small(BatchArgs A, uint32_t first, uint32_t count)
{
    constexpr int NT = nt_of<K>(), TEAMS = teams_of<K>();
    extern __shared__ __align__(16) uint32_t smem[];
    const int team = threadIdx.x / NT, tid = threadIdx.x - team * NT;
    const uint32_t i = blockIdx.x * TEAMS + team;
    const bool valid = i < count;
    const Prod &P = A.prods[first + (valid ? i : 0)];
    const PrimeInfo &pr = A.primes[P.prime];
    polymul_team<K, true, true, NT>(smem + team * team_smem_words<K>(), tid, P.a, valid ? P.la : 0, P.b,
                                    valid ? P.lb : 0, P.c, valid ? P.lc : 0, pr.tw, pr.itw, 0, 0, pr.p, pr.pp,
                                    P.k_scale);
}

// Row jobs of split products, one CTA each (their column tiles are done).
__global__ void __launch_bounds__(kThreads, 3) k_phase_row(BatchArgs A)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const Job J = A.jobs[blockIdx.x];
    const Prod &P = A.prods[J.prod];
    const PrimeInfo &pr = A.primes[P.prime];
    uint32_t *row = P.ws + (static_cast<size_t>(J.idx) << kRowLog);
    const size_t n = size_t{1} << P.k;
    polymul_team<kRowLog, false, false, kThreads>(smem, threadIdx.x, row, size_t{1} << kRowLog, row + n,
                                                  size_t{1} << kRowLog, row, size_t{1} << kRowLog, pr.tw, pr.itw,
                                                  static_cast<int>(P.k) - kRowLog, static_cast<int>(J.idx), pr.p,
                                                  pr.pp, 0u);
}

// Column jobs with K1 <= 4 column levels (registers, no shared memory):
// forward (INV false) or inverse, the inverse of a truncated product as an
// inverse TFT per column.
template <bool INV>
__global__ void __launch_bounds__(kThreads, 4) k_phase_col_regs(BatchArgs A)
{
    const Job J = A.jobs[blockIdx.x];
    const Prod &P = A.prods[J.prod];
    const PrimeInfo &pr = A.primes[P.prime];
    if (INV && P.tft) {
        switch (P.k - kRowLog) {
        case 2: col_itft_dispatch<2>(P, pr, J.idx); break;
        case 3: col_itft_dispatch<3>(P, pr, J.idx); break;
        case 4: col_itft_dispatch<4>(P, pr, J.idx); break;
        default: break;
        }
        return;
    }
    switch (P.k - kRowLog) {
    case 1: col_regs<1, INV>(P, pr, J.idx); break;
    case 2: col_regs<2, INV>(P, pr, J.idx); break;
    case 3: col_regs<3, INV>(P, pr, J.idx); break;
    case 4: col_regs<4, INV>(P, pr, J.idx); break;
    default: break;
    }
}

// Column jobs with K1 >= 5 (shared-memory column tiles).
template <bool INV>
__global__ void __launch_bounds__(kThreads, 3) k_phase_col_tile(BatchArgs A)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const Job J = A.jobs[blockIdx.x];
    const Prod &P = A.prods[J.prod];
    const PrimeInfo &pr = A.primes[P.prime];
    switch (P.k - kRowLog) {
    case 5: col_tile<5, INV>(smem, P, pr, J.idx); break;
    case 6: col_tile<6, INV>(smem, P, pr, J.idx); break;
    case 7: col_tile<7, INV>(smem, P, pr, J.idx); break;
    case 8: col_tile<8, INV>(smem, P, pr, J.idx); break;
    default: break;
    }
}

int col_tiles(int k1)
{
    return (1 << kRowLog) / (k1 <= kMaxRegColLog ? reg_cols(k1) : col_tile_cols(k1));
}

int teams_for(int k)
{
    const int nt = k <= 4 ? 1 : (1 << (k - 4));
    return nt >= kThreads ? 1 : kThreads / nt;
}

}  // namespace

size_t batch_ws_words(size_t lc)
{
    const int k = ceil_log2(lc);
    return k > kSmallLog ? (size_t{2} << k) : 0;
}

int batch_build(const polymul_desc *descs, size_t count, BatchHost &out, std::vector<uint32_t> &prime_list,
                std::vector<int> &prime_log2, bool fixed_primes, bool tft)
{
    out.prods.clear();
    for (auto &j : out.jobs) j.clear();
    out.ws_words = 0;
    if (count && !descs) return MONT_EINVAL;
    std::vector<Prod> prods(count);
    std::vector<size_t> small, large;
    for (size_t i = 0; i < count; i++) {
        const polymul_desc &d = descs[i];
        if (!d.a || !d.b || !d.c || d.la == 0 || d.lb == 0 || d.reserved != 0) return MONT_EINVAL;
        if (d.la > (1u << 24) || d.lb > (1u << 24)) return MONT_ERANGE;
        const size_t lc = static_cast<size_t>(d.la) + d.lb - 1;
        const int k = ceil_log2(lc);
        if (k > kRowLog + kMaxColLog) return MONT_EUNSUPPORTED;
        if (any_overlap(d.c, lc * 4, d.a, size_t{d.la} * 4) || any_overlap(d.c, lc * 4, d.b, size_t{d.lb} * 4))
            return MONT_EINVAL;
        size_t pi = 0;
        while (pi < prime_list.size() && prime_list[pi] != d.p) pi++;
        if (pi == prime_list.size()) {
            if (fixed_primes) return MONT_EINVAL;
            if (pi == kMaxPrimes) return MONT_EUNSUPPORTED;
            if (d.p < 3 || d.p >= 0x80000000u || !(d.p & 1u)) return MONT_EINVAL;
            prime_list.push_back(d.p);
            prime_log2.push_back(0);
        }
        if (k > prime_log2[pi]) {
            if (fixed_primes) return MONT_ERANGE;
            prime_log2[pi] = k;
        }
        Prod &P = prods[i];
        P.a = d.a;
        P.b = d.b;
        P.c = d.c;
        P.ws = nullptr;
        P.la = d.la;
        P.lb = d.lb;
        P.lc = static_cast<uint32_t>(lc);
        P.k = static_cast<uint32_t>(k);
        P.prime = static_cast<uint16_t>(pi);
        P.tft = 0;
        P.ntiles = P.nrows = 0;
        int scale_log = k;   // b is scaled by (2^scale_log)^-1 R^2
        if (k > kSmallLog) {
            const int k1 = k - kRowLog;
            P.ntiles = static_cast<uint32_t>(col_tiles(k1));
            P.nrows = 1u << k1;
            const uint32_t need = static_cast<uint32_t>((lc + (size_t{1} << kRowLog) - 1) >> kRowLog);
            if (tft && k1 >= kMinTftColLog && k1 <= kMaxRegColLog && need < P.nrows) {
                P.tft = 1;
                P.nrows = need;
                scale_log = kRowLog;
            }
            P.ws = reinterpret_cast<uint32_t *>(out.ws_words);   // word offset until rebased
            out.ws_words += size_t{2} << k;
            large.push_back(i);
        } else {
            small.push_back(i);
        }
        const uint32_t n_mod = static_cast<uint32_t>((uint64_t{1} << scale_log) % d.p);
        P.k_scale = host_to_mont(host_to_mont(host_powmod(n_mod, d.p - 2, d.p), d.p), d.p);
    }
    std::stable_sort(small.begin(), small.end(), [&](size_t x, size_t y) { return prods[x].k < prods[y].k; });
    out.prods.reserve(count);
    for (size_t i : small) out.prods.push_back(prods[i]);
    for (size_t i : large) out.prods.push_back(prods[i]);
    const size_t nsmall = small.size();
    std::vector<Job> colf, sm, row, coli, whole;
    std::vector<size_t> piped;   // split products run as column / row / column jobs
    for (size_t i = nsmall; i < count; i++) {
        const Prod &P = out.prods[i];
        const uint32_t id = static_cast<uint32_t>(i);
        if (P.k <= static_cast<uint32_t>(kWholeMaxLog)) {
            whole.push_back(Job{JOB_WHOLE, P.k, id, 0});
            continue;
        }
        piped.push_back(i);
        for (uint32_t t = 0; t < P.ntiles; t++) colf.push_back(Job{JOB_COLF, P.k, id, t});
        for (uint32_t r = 0; r < P.nrows; r++) row.push_back(Job{JOB_ROW, P.k, id, r});
        for (uint32_t t = 0; t < P.ntiles; t++) coli.push_back(Job{JOB_COLI, P.k, id, t});
    }
    for (size_t s = 0; s < nsmall;) {
        const uint32_t k = out.prods[s].k;
        const size_t per = static_cast<size_t>(teams_for(static_cast<int>(k)));
        size_t e = s;
        while (e < nsmall && e - s < per && out.prods[e].k == k) e++;
        sm.push_back(Job{JOB_SMALL, k, static_cast<uint32_t>(s), static_cast<uint32_t>(e - s)});
        s = e;
    }
    // Whole jobs are the longest: largest first.
    std::stable_sort(whole.begin(), whole.end(), [](const Job &x, const Job &y) { return x.k > y.k; });
    // order 0: split products' column tiles first, whole and small products
    // fill the time until their rows can start; order 1: whole and small
    // products first.
    for (int order = 0; order < 2; order++) {
        std::vector<Job> &jobs = out.jobs[order];
        const std::vector<Job> *seq0[5] = {&colf, &whole, &sm, &row, &coli};
        const std::vector<Job> *seq1[5] = {&whole, &sm, &colf, &row, &coli};
        for (const std::vector<Job> *v : (order == 0 ? seq0 : seq1)) jobs.insert(jobs.end(), v->begin(), v->end());
    }
    // orders 2, 3: the whole jobs, then rounds r = 0, 1, ...: column tiles of
    // pipelined product r, rows of product r - D, output tiles of product
    // r - 2D, and an even share of the small products.  Every job waits only
    // on jobs of earlier rounds.
    const size_t nlarge = piped.size();
    std::vector<size_t> colf_at(nlarge + 1, 0), row_at(nlarge + 1, 0);
    for (size_t i = 0; i < nlarge; i++) {
        colf_at[i + 1] = colf_at[i] + out.prods[piped[i]].ntiles;
        row_at[i + 1] = row_at[i] + out.prods[piped[i]].nrows;
    }
    for (int order = 2; order < kJobOrders; order++) {
        const size_t D = order == 2 ? 32 : 64;
        std::vector<Job> &jobs = out.jobs[order];
        jobs.reserve(whole.size() + colf.size() + sm.size() + row.size() + coli.size());
        jobs.insert(jobs.end(), whole.begin(), whole.end());
        const size_t rounds = nlarge + 2 * D;
        size_t si = 0;
        for (size_t r = 0; r < rounds; r++) {
            if (r < nlarge) jobs.insert(jobs.end(), colf.begin() + colf_at[r], colf.begin() + colf_at[r + 1]);
            if (r >= D && r - D < nlarge)
                jobs.insert(jobs.end(), row.begin() + row_at[r - D], row.begin() + row_at[r - D + 1]);
            if (r >= 2 * D && r - 2 * D < nlarge)
                jobs.insert(jobs.end(), coli.begin() + colf_at[r - 2 * D], coli.begin() + colf_at[r - 2 * D + 1]);
            const size_t until = sm.size() * (r + 1) / rounds;
            for (; si < until; si++) jobs.push_back(sm[si]);
        }
        for (; si < sm.size(); si++) jobs.push_back(sm[si]);
    }
    for (const std::vector<Job> &jobs : out.jobs)
        if (jobs.size() > UINT32_MAX) return MONT_ERANGE;   // the kernel counts jobs in 32 bits
    return MONT_OK;
}

void batch_rebase(BatchHost &b, uint32_t *ws)
{
    for (Prod &P : b.prods)
        if (P.k > static_cast<uint32_t>(kSmallLog)) P.ws = ws + reinterpret_cast<size_t>(P.ws);
}

int batch_occupancy(int variant, int *per_sm)
{
    const void *k = variant ? reinterpret_cast<const void *>(k_polymul_batch<3>)
                            : reinterpret_cast<const void *>(k_polymul_batch<2>);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemWords * sizeof(uint32_t)) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, kThreads, kSmemWords * sizeof(uint32_t)) !=
            cudaSuccess) {
        cudaGetLastError();
        return MONT_ECUDA;
    }
    return *per_sm > 0 ? MONT_OK : MONT_ECUDA;
}

void phased_build(const BatchHost &b, PhasedHost &out)
{
    std::vector<Job> lists[PH_LISTS];
    for (const Job &J : b.jobs[0]) {
        const bool reg = J.k - kRowLog <= static_cast<uint32_t>(kMaxRegColLog);
        switch (J.type) {
        case JOB_WHOLE: {   // column / row / column jobs here (K1 = 1, 2: register columns)
            const Prod &P = b.prods[J.prod];
            for (uint32_t t = 0; t < P.ntiles; t++) lists[PH_COLF_REG].push_back(Job{JOB_COLF, P.k, J.prod, t});
            for (uint32_t r = 0; r < P.nrows; r++) lists[PH_ROW].push_back(Job{JOB_ROW, P.k, J.prod, r});
            for (uint32_t t = 0; t < P.ntiles; t++) lists[PH_COLI_REG].push_back(Job{JOB_COLI, P.k, J.prod, t});
            break;
        }
        case JOB_COLF: lists[reg ? PH_COLF_REG : PH_COLF_TILE].push_back(J); break;
        case JOB_ROW: lists[PH_ROW].push_back(J); break;
        case JOB_COLI: lists[reg ? PH_COLI_REG : PH_COLI_TILE].push_back(J); break;
        default: break;
        }
    }
    out.jobs.clear();
    for (int l = 0; l < PH_LISTS; l++) {
        out.off[l] = static_cast<uint32_t>(out.jobs.size());
        out.cnt[l] = static_cast<uint32_t>(lists[l].size());
        out.jobs.insert(out.jobs.end(), lists[l].begin(), lists[l].end());
    }
    out.small.clear();
    for (size_t i = 0; i < b.prods.size() && b.prods[i].k <= static_cast<uint32_t>(kSmallLog);) {
        size_t e = i;
        while (e < b.prods.size() && b.prods[e].k == b.prods[i].k) e++;
        out.small.insert(out.small.end(), {b.prods[i].k, static_cast<uint32_t>(i), static_cast<uint32_t>(e - i)});
        i = e;
    }
}

namespace {

template <int K>
int launch_phase_small(const BatchArgs &A, uint32_t first, uint32_t count, cudaStream_t s)
{
    constexpr int T = teams_of<K>(), NT = nt_of<K>();
    const size_t smem = static_cast<size_t>(T) * team_smem_words<K>() * sizeof(uint32_t);
    if (ensure_smem(k_phase_small<K>, smem) != MONT_OK) return MONT_ECUDA;
    k_phase_small<K><<<(count + T - 1) / T, T * NT, smem, s>>>(A, first, count);
    return launch_status();
}

int phase_small(int k, const BatchArgs &A, uint32_t first, uint32_t count, cudaStream_t s)
{
    switch (k) {
#define X(L) \
    case L: return launch_phase_small<L>(A, first, count, s);
        X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13)
#undef X
    default: return MONT_EUNSUPPORTED;
    }
}

template <typename K>
int phase_jobs(K kernel, BatchArgs A, const Job *jobs, uint32_t count, size_t smem, cudaStream_t s)
{
    if (count == 0) return MONT_OK;
    if (ensure_smem(kernel, smem) != MONT_OK) return MONT_ECUDA;
    A.jobs = jobs;
    A.njobs = count;
    kernel<<<count, kThreads, smem, s>>>(A);
    return launch_status();
}

}  // namespace

int batch_launch_phased(BatchArgs A, const PhasedHost &ph, const Job *d_jobs, size_t sync_words, cudaStream_t s,
                        cudaStream_t aux, cudaEvent_t fork, cudaEvent_t join)
{
    if (cudaMemsetAsync(A.sync, 0, sync_words * sizeof(uint32_t), s) != cudaSuccess) return MONT_ECUDA;
    const bool side = aux != nullptr && aux != s;   // else every kernel in order on s
    if (!side) aux = s;
    else if (cudaEventRecord(fork, s) != cudaSuccess || cudaStreamWaitEvent(aux, fork, 0) != cudaSuccess)
        return MONT_ECUDA;
    int rc = MONT_OK;
    for (size_t i = 0; i + 2 < ph.small.size() && rc == MONT_OK; i += 3)
        rc = phase_small(static_cast<int>(ph.small[i]), A, ph.small[i + 1], ph.small[i + 2], aux);
    const size_t smem = kSmemWords * sizeof(uint32_t);
    auto list = [&](int l) { return d_jobs + ph.off[l]; };
    if (rc == MONT_OK) rc = phase_jobs(k_phase_col_regs<false>, A, list(PH_COLF_REG), ph.cnt[PH_COLF_REG], 0, s);
    if (rc == MONT_OK) rc = phase_jobs(k_phase_col_tile<false>, A, list(PH_COLF_TILE), ph.cnt[PH_COLF_TILE], smem, s);
    if (rc == MONT_OK) rc = phase_jobs(k_phase_row, A, list(PH_ROW), ph.cnt[PH_ROW], smem, s);
    if (rc == MONT_OK) rc = phase_jobs(k_phase_col_regs<true>, A, list(PH_COLI_REG), ph.cnt[PH_COLI_REG], 0, s);
    if (rc == MONT_OK) rc = phase_jobs(k_phase_col_tile<true>, A, list(PH_COLI_TILE), ph.cnt[PH_COLI_TILE], smem, s);
    // Join the side branch back into s (also after a failed launch, so no
    // branch is left open in a capture).
    const bool joined = !side || (cudaEventRecord(join, aux) == cudaSuccess && cudaStreamWaitEvent(s, join, 0) == cudaSuccess);
    return rc != MONT_OK ? rc : (joined ? MONT_OK : MONT_ECUDA);
}

int batch_launch(BatchArgs A, const Job *jobs, uint32_t njobs, size_t sync_words, int grid, int variant,
                 cudaStream_t s)
{
    A.jobs = jobs;
    A.njobs = njobs;
    if (cudaMemsetAsync(A.sync, 0, sync_words * sizeof(uint32_t), s) != cudaSuccess) return MONT_ECUDA;
    if (njobs == 0) return MONT_OK;
    const unsigned g = static_cast<unsigned>(std::max(1, std::min<int>(grid, static_cast<int>(std::min<uint32_t>(njobs, 1u << 30)))));
    if (variant) k_polymul_batch<3><<<g, kThreads, kSmemWords * sizeof(uint32_t), s>>>(A);
    else k_polymul_batch<2><<<g, kThreads, kSmemWords * sizeof(uint32_t), s>>>(A);
    return launch_status();
}

}  // namespace mont

// host[v], d_jobs[v], d_prods[v]: the batch with row-granular truncated
// transforms (v = 0) and with every product padded to a full transform
// (v = 1, polymul_batch_config.full_transforms); both share counters and
// scratch (the same layout).
struct polymul_batch_plan {
    int device = 0;
    mont::BatchHost host[2];
    std::vector<uint32_t> prime_list;
    std::vector<int> prime_log2;
    mont::BatchArgs args{};
    mont::Job *d_jobs[2][mont::kJobOrders] = {};
    mont::Prod *d_prods[2] = {};
    mont::PhasedHost phased[2];              // the phased form's job lists (kernel 2)
    mont::Job *d_phased[2] = {};
    cudaStream_t aux = nullptr;              // the phased form's side stream (small products)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    uint32_t *d_sync = nullptr;
    size_t sync_words = 0;
    uint32_t *d_ws = nullptr;
    int occupancy = 1;       // CTAs per SM of the selected kernel variant
    int occ[2] = {1, 1};     // per variant
    int sms = 1;
    polymul_batch_config cfg{};
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    polymul_batch_config graph_cfg{};
};

namespace mont {
namespace {

std::mutex g_tune_mu;
std::map<std::string, polymul_batch_config> g_tune_cache;

std::string signature(const polymul_batch_plan *pl)
{
    std::map<uint32_t, size_t> hist;
    for (const Prod &P : pl->host[0].prods) hist[P.k]++;
    std::string s = std::to_string(pl->device) + ":";
    for (auto &kv : hist) s += std::to_string(kv.first) + "x" + std::to_string(kv.second) + ",";
    return s;
}

void free_plan(polymul_batch_plan *pl)
{
    if (pl->graph) cudaGraphExecDestroy(pl->graph);
    if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
    for (auto &v : pl->d_jobs)
        for (mont::Job *j : v) cudaFree(j);
    for (mont::Prod *d : pl->d_prods) cudaFree(d);
    for (mont::Job *j : pl->d_phased) cudaFree(j);
    if (pl->aux) cudaStreamDestroy(pl->aux);
    if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
    if (pl->ev_join) cudaEventDestroy(pl->ev_join);
    cudaFree(pl->d_sync);
    cudaFree(pl->d_ws);
}

int launch(polymul_batch_plan *pl, const polymul_batch_config &cfg, cudaStream_t s)
{
    const int order = (cfg.order >= 0 && cfg.order < kJobOrders) ? cfg.order : 0;
    const int variant = cfg.kernel == 1 ? 1 : 0;
    const int full = cfg.full_transforms ? 1 : 0;
    if (cfg.kernel == 2) {
        BatchArgs A = pl->args;
        A.prods = pl->d_prods[full];
        return batch_launch_phased(A, pl->phased[full], pl->d_phased[full], pl->sync_words, s, pl->aux, pl->ev_fork,
                                   pl->ev_join);
    }
    const int occ = pl->occ[variant];
    const int per_sm = std::max(1, std::min(cfg.ctas_per_sm > 0 ? cfg.ctas_per_sm : occ, occ));
    BatchArgs A = pl->args;
    A.prods = pl->d_prods[full];
    return batch_launch(A, pl->d_jobs[full][order], static_cast<uint32_t>(pl->host[full].jobs[order].size()),
                        pl->sync_words, pl->sms * per_sm, variant, s);
}

}  // namespace
}  // namespace mont

extern "C" int polymul_batch_describe(const polymul_desc *descs, size_t count, int order, int full_transforms,
                                      uint32_t *jobs, size_t cap, uint32_t *prods, size_t *njobs)
{
    using namespace mont;
    if (!njobs || (count && !descs) || order < 0 || order >= kJobOrders || (cap && !jobs) ||
        (full_transforms != 0 && full_transforms != 1))
        return MONT_EINVAL;
    if (count > (size_t{1} << 31)) return MONT_ERANGE;
    BatchHost host;
    std::vector<uint32_t> prime_list;
    std::vector<int> prime_log2;
    const int rc = batch_build(descs, count, host, prime_list, prime_log2, false, full_transforms == 0);
    if (rc != MONT_OK) return rc;
    const std::vector<Job> &list = host.jobs[order];
    *njobs = list.size();
    for (size_t i = 0; i < list.size() && i < cap; i++) {
        jobs[4 * i] = list[i].type;
        jobs[4 * i + 1] = list[i].k;
        jobs[4 * i + 2] = list[i].prod;
        jobs[4 * i + 3] = list[i].idx;
    }
    if (prods)
        for (size_t i = 0; i < host.prods.size(); i++) {
            prods[4 * i] = host.prods[i].k;
            prods[4 * i + 1] = host.prods[i].ntiles;
            prods[4 * i + 2] = host.prods[i].nrows;
            prods[4 * i + 3] = host.prods[i].tft;
        }
    return MONT_OK;
}

extern "C" int polymul_batch_plan_create(const polymul_desc *descs, size_t count, polymul_batch_plan **out)
{
    using namespace mont;
    if (!out || (count && !descs)) return MONT_EINVAL;
    *out = nullptr;
    if (count > (size_t{1} << 31)) return MONT_ERANGE;
    polymul_batch_plan *pl = new (std::nothrow) polymul_batch_plan();
    if (!pl) return MONT_ENOMEM;
    int rc = cudaGetDevice(&pl->device) == cudaSuccess ? MONT_OK : MONT_ECUDA;
    if (rc == MONT_OK) rc = batch_build(descs, count, pl->host[0], pl->prime_list, pl->prime_log2, false, true);
    if (rc == MONT_OK) rc = batch_build(descs, count, pl->host[1], pl->prime_list, pl->prime_log2, true, false);
    for (size_t pi = 0; pi < pl->prime_list.size() && rc == MONT_OK; pi++) {
        const TwTable *t = nullptr;
        rc = get_table(pl->prime_list[pi], std::max(pl->prime_log2[pi], kRowLog), &t);
        if (rc == MONT_OK) pl->args.primes[pi] = PrimeInfo{t->p, t->p_prime, t->fwd, t->inv};
    }
    if (rc != MONT_OK) {
        delete pl;
        return rc;
    }
    bool ok = true;
    pl->sync_words = 2 + 2 * count;
    ok = cudaMalloc(&pl->d_sync, pl->sync_words * sizeof(uint32_t)) == cudaSuccess &&
         cudaMemset(pl->d_sync, 0, pl->sync_words * sizeof(uint32_t)) == cudaSuccess;
    if (ok && pl->host[0].ws_words)
        ok = cudaMalloc(&pl->d_ws, pl->host[0].ws_words * sizeof(uint32_t)) == cudaSuccess;
    for (int v = 0; v < 2 && ok; v++) {
        BatchHost &h = pl->host[v];
        batch_rebase(h, pl->d_ws);
        phased_build(h, pl->phased[v]);
        const std::vector<Job> &pj = pl->phased[v].jobs;
        if (!pj.empty())
            ok = cudaMalloc(&pl->d_phased[v], pj.size() * sizeof(Job)) == cudaSuccess &&
                 cudaMemcpy(pl->d_phased[v], pj.data(), pj.size() * sizeof(Job), cudaMemcpyHostToDevice) == cudaSuccess;
        if (count)
            ok = cudaMalloc(&pl->d_prods[v], count * sizeof(Prod)) == cudaSuccess &&
                 cudaMemcpy(pl->d_prods[v], h.prods.data(), count * sizeof(Prod), cudaMemcpyHostToDevice) ==
                     cudaSuccess;
        for (int o = 0; o < kJobOrders && ok; o++)
            if (!h.jobs[o].empty())
                ok = cudaMalloc(&pl->d_jobs[v][o], h.jobs[o].size() * sizeof(Job)) == cudaSuccess &&
                     cudaMemcpy(pl->d_jobs[v][o], h.jobs[o].data(), h.jobs[o].size() * sizeof(Job),
                                cudaMemcpyHostToDevice) == cudaSuccess;
    }
    if (ok) ok = batch_occupancy(0, &pl->occ[0]) == MONT_OK && batch_occupancy(1, &pl->occ[1]) == MONT_OK;
    if (ok)
        ok = cudaStreamCreateWithFlags(&pl->aux, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    pl->occupancy = pl->occ[0];
    pl->sms = device_sm_count();
    if (!ok || pl->sms <= 0) {
        cudaGetLastError();
        free_plan(pl);
        delete pl;
        return MONT_ENOMEM;
    }
    pl->args.prods = pl->d_prods[0];
    pl->args.sync = pl->d_sync;
    pl->args.wait_iters = 1u << 22;
    pl->args.wait_ns = 2000000000ull;   // 2 s per wait
    pl->cfg.ctas_per_sm = pl->occ[0];
    pl->cfg.order = 0;
    pl->cfg.kernel = 0;
    pl->cfg.full_transforms = 0;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(signature(pl));
        if (it != g_tune_cache.end()) pl->cfg = it->second;
    }
    *out = pl;
    return MONT_OK;
}

extern "C" void polymul_batch_plan_destroy(polymul_batch_plan *plan)
{
    if (!plan) return;
    mont::free_plan(plan);
    delete plan;
}

extern "C" size_t polymul_batch_plan_workspace_bytes(const polymul_batch_plan *plan)
{
    return plan ? plan->host[0].ws_words * sizeof(uint32_t) : 0;
}

extern "C" int polymul_batch_plan_get_config(const polymul_batch_plan *plan, polymul_batch_config *cfg)
{
    if (!plan || !cfg) return MONT_EINVAL;
    *cfg = plan->cfg;
    return MONT_OK;
}

extern "C" int polymul_batch_plan_set_config(polymul_batch_plan *plan, const polymul_batch_config *cfg)
{
    if (!plan || !cfg || cfg->ctas_per_sm < 0 || cfg->order < 0 || cfg->order >= mont::kJobOrders || cfg->kernel < 0 ||
        cfg->kernel > 2 || cfg->full_transforms < 0 || cfg->full_transforms > 1)
        return MONT_EINVAL;
    plan->cfg = *cfg;
    return MONT_OK;
}

extern "C" int polymul_batch_plan_set_wait_limit(polymul_batch_plan *plan, uint32_t iterations, uint64_t nanoseconds)
{
    if (!plan || iterations == 0 || nanoseconds == 0) return MONT_EINVAL;
    plan->args.wait_iters = iterations;
    plan->args.wait_ns = nanoseconds;
    if (plan->graph) {
        cudaGraphExecDestroy(plan->graph);
        plan->graph = nullptr;
    }
    return MONT_OK;
}

extern "C" int polymul_batch_run(polymul_batch_plan *plan, cudaStream_t stream)
{
    if (!plan) return MONT_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return MONT_ECUDA;
    if (dev != plan->device) return MONT_EINVAL;
    return mont::launch(plan, plan->cfg, stream);
}

extern "C" int polymul_batch_run_graph(polymul_batch_plan *plan, cudaStream_t stream)
{
    if (!plan) return MONT_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return MONT_ECUDA;
    if (dev != plan->device) return MONT_EINVAL;
    if (plan->graph && (plan->graph_cfg.ctas_per_sm != plan->cfg.ctas_per_sm || plan->graph_cfg.order != plan->cfg.order ||
                        plan->graph_cfg.kernel != plan->cfg.kernel ||
                        plan->graph_cfg.full_transforms != plan->cfg.full_transforms)) {
        cudaGraphExecDestroy(plan->graph);
        plan->graph = nullptr;
    }
    if (!plan->graph) {
        if (!plan->cap_stream && cudaStreamCreateWithFlags(&plan->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
            return MONT_ECUDA;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(plan->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MONT_ECUDA;
        const int rc = mont::launch(plan, plan->cfg, plan->cap_stream);
        const cudaError_t ec = cudaStreamEndCapture(plan->cap_stream, &g);
        if (rc != MONT_OK || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return rc != MONT_OK ? rc : MONT_ECUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&plan->graph, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            plan->graph = nullptr;
            cudaGetLastError();
            return MONT_ECUDA;
        }
        plan->graph_cfg = plan->cfg;
    }
    return cudaGraphLaunch(plan->graph, stream) == cudaSuccess ? MONT_OK : MONT_ECUDA;
}

// Synchronous: waits for `stream`, then reads the device error word.
extern "C" int polymul_batch_status(polymul_batch_plan *plan, cudaStream_t stream)
{
    if (!plan) return MONT_EINVAL;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return MONT_ECUDA;
    uint32_t err = 0;
    if (cudaMemcpy(&err, plan->d_sync + 1, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess) return MONT_ECUDA;
    return err ? MONT_ETIMEOUT : MONT_OK;
}

// Autotuner: times every (kernel variant, CTAs per SM, job order) choice `trials` times
// with CUDA events on `stream` and keeps the fastest; the result is cached
// for batches with the same size histogram on this device.
extern "C" int polymul_batch_plan_tune(polymul_batch_plan *plan, cudaStream_t stream, int trials)
{
    if (!plan || trials <= 0) return MONT_EINVAL;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return MONT_ECUDA;
    polymul_batch_config best = plan->cfg;
    float best_ms = 1e30f;
    int rc = MONT_OK;
    for (int variant = 0; variant < 2 && rc == MONT_OK; variant++)
    for (int per = 1; per <= plan->occ[variant] && rc == MONT_OK; per++)
        for (int order = 0; order < mont::kJobOrders && rc == MONT_OK; order++) {
            polymul_batch_config c{};
            c.ctas_per_sm = per;
            c.order = order;
            c.kernel = variant;
            c.full_transforms = plan->cfg.full_transforms;
            rc = mont::launch(plan, c, stream);   // warm-up
            float total = 0.f;
            for (int t = 0; t < trials && rc == MONT_OK; t++) {
                cudaEventRecord(e0, stream);
                rc = mont::launch(plan, c, stream);
                cudaEventRecord(e1, stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) rc = MONT_ECUDA;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                total += ms;
            }
            if (rc == MONT_OK && total < best_ms) {
                best_ms = total;
                best = c;
            }
        }
    if (rc == MONT_OK) {   // the phased form: launch shape and job order do not apply
        polymul_batch_config c{};
        c.ctas_per_sm = 0;
        c.order = 0;
        c.kernel = 2;
        c.full_transforms = plan->cfg.full_transforms;
        rc = mont::launch(plan, c, stream);
        float total = 0.f;
        for (int t = 0; t < trials && rc == MONT_OK; t++) {
            cudaEventRecord(e0, stream);
            rc = mont::launch(plan, c, stream);
            cudaEventRecord(e1, stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = MONT_ECUDA;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            total += ms;
        }
        if (rc == MONT_OK && total < best_ms) {
            best_ms = total;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MONT_OK) return rc;
    plan->cfg = best;
    std::lock_guard<std::mutex> lock(mont::g_tune_mu);
    mont::g_tune_cache[mont::signature(plan)] = best;
    return polymul_batch_status(plan, stream);
}

// Test hook for failure detection: makes the first product that runs as
// column / row / column jobs (N > 2^15) expect one more column tile than
// exists, so its row jobs wait on a count that is never reached; the bounded
// waits expire and the batch reports MONT_ETIMEOUT.  Undone by recreating
// the plan.
extern "C" int polymul_batch_plan_inject_stall(polymul_batch_plan *plan)
{
    if (!plan) return MONT_EINVAL;
    for (size_t i = 0; i < plan->host[0].prods.size(); i++) {
        if (plan->host[0].prods[i].k <= static_cast<uint32_t>(mont::kWholeMaxLog)) continue;   // no cross-CTA waits
        for (int v = 0; v < 2; v++) {
            mont::Prod &P = plan->host[v].prods[i];
            P.ntiles += 1;
            if (cudaMemcpy(plan->d_prods[v] + i, &P, sizeof(mont::Prod), cudaMemcpyHostToDevice) != cudaSuccess)
                return MONT_ECUDA;
        }
        return MONT_OK;
    }
    return MONT_EINVAL;
}
