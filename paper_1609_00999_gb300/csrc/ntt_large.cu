// ntt_large.cu -- transforms and products with N = 2^K > 2^14 (up to 2^24).
//
// The K levels split into K1 column levels and K2 row levels (K2 = 12 up
// to K = 16, K - 4 for K = 17, 18, then max(13, K - 10)).  Viewing the N elements as a
// [2^K1][2^K2] row-major matrix, levels 0 .. K1-1 pair elements of the same
// column (stride 2^K2) and their twiddles depend only on the row index, so
// every column is an independent 2^K1-point transform with the table
// entries 1 .. 2^K1 - 1.  Levels K1 .. K-1 stay inside one row; row r is
// block r of level K1, so its twiddle for local level l and local block i
// is entry 2^(K1+l) + (r << l) + i.
//
// Column kernels: up to four levels in registers, straight from and to
// global memory (k_col_regs); five to eight levels as two register passes
// over a tile of 32 or more consecutive columns, the first loading from and
// the second storing to global memory, with one exchange through shared
// memory between them (k_col_direct); more levels through a shared-memory
// tile loaded with coalesced row segments, one team of threads per column
// (k_col).  Row kernel: one CTA per row, the same register passes as the
// single-CTA kernels, its first pass loading from (forward) or its last pass
// storing to (inverse) global memory.  Forward values between the
// column and row kernels are lazy ([0, 2P), as inside the passes); the row
// kernels take them as such and reduce what they finally store.
#include <algorithm>
#include <type_traits>

#include "ntt_kernels.cuh"

namespace mont {
namespace {

// Column tile geometry and shared-memory layout per column size 2^K1:
// C columns per CTA, NT1 threads per column (512 threads per CTA), column c
// at c * (N1 + PAD) with the low five bits XORed by (c * MUL) & 31 (on top
// of swz when SW).  These choices make the coalesced tile loads bank-conflict
// free and keep the pass accesses at most 1.5-way conflicted on average.
template <int K1>
struct ColCfg {
    static constexpr int N1 = 1 << K1;
    static constexpr int C = K1 <= 4 ? 512 : (K1 >= 10 ? 8 : (1 << (13 - K1)));
    static constexpr int NT1 = N1 <= 16 ? 1 : N1 / 16;
    static constexpr int THREADS = C * NT1;
    static constexpr int PAD = (K1 <= 4) ? 1 : (K1 == 8 ? 16 : 0);
    static constexpr int MUL = (K1 <= 4) ? 0 : (K1 == 5 || K1 == 9) ? 17 : (K1 == 8 ? 3 : 9);
    static constexpr bool SW = K1 >= 8;
    static constexpr int STRIDE = N1 + PAD;
    static constexpr size_t SMEM = static_cast<size_t>(C) * STRIDE * sizeof(uint32_t);
    static_assert(THREADS <= 1024, "column tile too large");
};

struct ColArgs {
    const uint32_t *src[2];
    size_t src_len[2];      // elements at index >= src_len read as zero
    size_t src_stride[2];   // per product (grid.z)
    uint32_t *dst[2];
    size_t dst_len;         // elements at index >= dst_len are not stored
    size_t dst_stride;
    int k2;
    const uint32_t *tw;
    const uint32_t *itw;    // inverse twiddles (the inverse TFT of truncated products)
    uint32_t p, pp;
    uint32_t scale[2];      // nonzero: REDC-multiply inputs by it on load
    uint32_t post;          // nonzero: REDC-multiply outputs by it on store
    uint32_t rows;          // register column passes store rows t < rows only (truncated products)
};

template <int K1, bool INVERSE>
__global__ void __launch_bounds__(ColCfg<K1>::THREADS)
k_col(ColArgs A, size_t prod0)
{
    using CF = ColCfg<K1>;
    constexpr int NP = SchedFor<K1, ColCfg<K1>::NT1>::kPasses;
    extern __shared__ __align__(16) uint32_t smem[];
    const bool op1 = blockIdx.y != 0;   // operand select without indexing the parameter arrays
    const size_t prod = prod0 + blockIdx.z;
    const uint32_t *src = (op1 ? A.src[1] : A.src[0]) + prod * (op1 ? A.src_stride[1] : A.src_stride[0]);
    const size_t slen = op1 ? A.src_len[1] : A.src_len[0];
    uint32_t *dst = (op1 ? A.dst[1] : A.dst[0]) + prod * A.dst_stride;
    const uint32_t scale = op1 ? A.scale[1] : A.scale[0];
    const size_t o0 = static_cast<size_t>(blockIdx.x) * CF::C;
    const uint32_t p = A.p, pp = A.pp;
    auto col = [&](int c) { return ColLayout<CF::SW>{smem + c * CF::STRIDE, (c * CF::MUL) & 31}; };

    // Tile sweep in row-major order, THREADS elements per step: this thread
    // always lands on column cT and rows t0 + u S (S = THREADS / C rows per
    // step), so its elements sit at fixed strides from one base, in global
    // memory and in its column of shared memory.
    static_assert(CF::THREADS % CF::C == 0, "tile sweep");
    constexpr int S = CF::THREADS / CF::C, PER = CF::N1 / S;
    const int cT = threadIdx.x % CF::C, t0 = threadIdx.x / CF::C;
    const ColLayout<CF::SW> mine = col(cT);
    const size_t first = o0 + cT + (static_cast<size_t>(t0) << A.k2), step = static_cast<size_t>(S) << A.k2;
    const long long room_in = static_cast<long long>(slen) - static_cast<long long>(first);
    {
        uint32_t v[PER];
#pragma unroll
        for (int u = 0; u < PER; u++) v[u] = static_cast<long long>(u * step) < room_in ? __ldg(src + first + u * step) : 0u;
#pragma unroll
        for (int u = 0; u < PER; u++) mine[t0 + u * S] = scale ? mont_mul(v[u], scale, p, pp) : v[u];
    }
    __syncthreads();
    const int c = threadIdx.x / CF::NT1, tid = threadIdx.x % CF::NT1;
    const ColLayout<CF::SW> lay[1] = {col(c)};
    if constexpr (!INVERSE) fwd_passes<K1, CF::NT1, 1, true, 0, NP - 1>(lay, tid, A.tw, 0, 0, Mod{p, pp});
    else inv_passes<K1, CF::NT1, true, NP - 1, 0>(lay[0], tid, A.tw, 0, 0, Mod{p, pp});
    const long long room_out = static_cast<long long>(A.dst_len) - static_cast<long long>(first);
#pragma unroll
    for (int u = 0; u < PER; u++) {
        uint32_t v = mine[t0 + u * S];
        if (A.post) v = mont_mul(v, A.post, p, pp);
        if (static_cast<long long>(u * step) < room_out) dst[first + u * step] = v;
    }
}

// Column tiles for K1 = 5 .. 8 (two passes of at most four levels, 16
// elements per thread, C >= 32 columns per CTA).  The pass that starts the
// transform loads its elements straight from global memory and the pass
// that ends it stores them straight back, so only the exchange between the
// two passes goes through shared memory.  Thread x takes column c = x % C
// and team position tid = x / C: every access of a warp is one row of 32
// consecutive columns, a 128-byte segment in global memory, and with column
// c at word c * (N1 + 1) thirty-two distinct banks in shared memory (each
// element a per-group pointer plus a compile-time offset).
template <int K1, bool INVERSE>
__global__ void __launch_bounds__(ColCfg<K1>::THREADS, 3)
k_col_direct(ColArgs A, size_t prod0)
{
    using CF = ColCfg<K1>;
    constexpr int NT = CF::NT1;
    static_assert(SchedFor<K1, NT>::kPasses == 2 && CF::C % 32 == 0, "two passes, whole-warp rows");
    using P0 = PassGeom<K1, NT, 0>;
    using P1 = PassGeom<K1, NT, 1>;
    using PIN = std::conditional_t<INVERSE, P1, P0>;    // the pass that reads global memory
    using POUT = std::conditional_t<INVERSE, P0, P1>;   // the pass that writes it
    extern __shared__ __align__(16) uint32_t smem[];
    const bool op1 = blockIdx.y != 0;
    const size_t prod = prod0 + blockIdx.z;
    const uint32_t *src = (op1 ? A.src[1] : A.src[0]) + prod * (op1 ? A.src_stride[1] : A.src_stride[0]);
    const size_t slen = op1 ? A.src_len[1] : A.src_len[0];
    uint32_t *dst = (op1 ? A.dst[1] : A.dst[0]) + prod * A.dst_stride;
    const uint32_t scale = op1 ? A.scale[1] : A.scale[0];
    const int c = threadIdx.x % CF::C, tid = threadIdx.x / CF::C;
    const size_t col = static_cast<size_t>(blockIdx.x) * CF::C + c;
    uint32_t *mine = smem + c * (CF::N1 + 1);
    const Mod m{A.p, A.pp};

    // Row j of this column is element col + j 2^k2 (< 2^24, so 32-bit
    // offsets); rows_below(len) counts the rows j with that index below len.
    const int k2 = A.k2;
    auto rows_below = [&](size_t len) -> int {
        if (len <= col) return 0;
        const size_t rows = (len - col + (size_t{1} << k2) - 1) >> k2;
        return rows < static_cast<size_t>(CF::N1) ? static_cast<int>(rows) : CF::N1;
    };
    uint32_t x[PIN::GPT][1][PIN::G];
    {
        const int rows_in = rows_below(slen);
        const uint32_t *sc = src + col;
        const uint32_t hs = static_cast<uint32_t>(PIN::HMIN) << k2;
#pragma unroll
        for (int r = 0; r < PIN::GPT; r++) {
            const int j0 = PIN::base(tid, r);
            const uint32_t e0 = static_cast<uint32_t>(j0) << k2;
#pragma unroll
            for (int t = 0; t < PIN::G; t++)
                x[r][0][t] = j0 + t * PIN::HMIN < rows_in ? __ldg(sc + (e0 + t * hs)) : 0u;
        }
    }
#pragma unroll
    for (int r = 0; r < PIN::GPT; r++) {
        if (scale) {
#pragma unroll
            for (int t = 0; t < PIN::G; t++) x[r][0][t] = mont_mul(x[r][0][t], scale, m.p, m.pp);
        }
        if constexpr (!INVERSE) ct_group<P0::E, 1, true>(x[r], A.tw, 0, 0, m);
        else gs_group<P1::E, 1, false>(x[r], A.tw, P1::S0, P1::blk(tid, r), m);
        uint32_t *g = mine + PIN::base(tid, r);
#pragma unroll
        for (int t = 0; t < PIN::G; t++) g[t * PIN::HMIN] = x[r][0][t];
    }
    __syncthreads();
    const int rows_out = rows_below(A.dst_len);
    uint32_t *dc = dst + col;
    const uint32_t hs_out = static_cast<uint32_t>(POUT::HMIN) << k2;
#pragma unroll
    for (int r = 0; r < POUT::GPT; r++) {
        uint32_t y[1][POUT::G];
        const uint32_t *g = mine + POUT::base(tid, r);
#pragma unroll
        for (int t = 0; t < POUT::G; t++) y[0][t] = g[t * POUT::HMIN];
        if constexpr (!INVERSE) ct_group<P1::E, 1, false>(y, A.tw, P1::S0, P1::blk(tid, r), m);
        else gs_group<P0::E, 1, true>(y, A.tw, 0, 0, m);
#pragma unroll
        for (int t = 0; t < POUT::G; t++) {
            uint32_t v = y[0][t];
            if (A.post) v = mont_mul(v, A.post, m.p, m.pp);
            const int j0 = POUT::base(tid, r);
            if (j0 + t * POUT::HMIN < rows_out) dc[(static_cast<uint32_t>(j0) << k2) + t * hs_out] = v;
        }
    }
}

// Column pass in registers for K1 <= 4: each of 128 threads takes G = 16 /
// 2^K1 consecutive-by-128 columns of one operand (16 elements), loads them
// straight from global memory (a warp reads 32 consecutive words of one row
// per load, all of a thread's loads in flight together), runs the column
// levels as the G arrays of one register group (they share twiddles:
// levels 0 .. K1-1, block 0) and stores them back: no shared memory, no
// barriers.
constexpr int kRegColThreads = 128;

template <int K1, bool INVERSE>
__global__ void __launch_bounds__(kRegColThreads) k_col_regs(ColArgs A, size_t prod0)
{
    constexpr int N1 = 1 << K1, G = 16 / N1;
    const bool op1 = blockIdx.y != 0;
    const size_t prod = prod0 + blockIdx.z;
    const uint32_t *src = (op1 ? A.src[1] : A.src[0]) + prod * (op1 ? A.src_stride[1] : A.src_stride[0]);
    const size_t slen = op1 ? A.src_len[1] : A.src_len[0];
    uint32_t *dst = (op1 ? A.dst[1] : A.dst[0]) + prod * A.dst_stride;
    const uint32_t scale = op1 ? A.scale[1] : A.scale[0];
    const uint32_t p = A.p, pp = A.pp;
    const size_t c0 = static_cast<size_t>(blockIdx.x) * (kRegColThreads * G) + threadIdx.x;
    uint32_t x[G][N1];
#pragma unroll
    for (int g = 0; g < G; g++)
#pragma unroll
        for (int t = 0; t < N1; t++) {
            const size_t j = c0 + g * kRegColThreads + (static_cast<size_t>(t) << A.k2);
            x[g][t] = j < slen ? __ldg(src + j) : 0u;
        }
    if (scale)
#pragma unroll
        for (int g = 0; g < G; g++)
#pragma unroll
            for (int t = 0; t < N1; t++) x[g][t] = mont_mul(x[g][t], scale, p, pp);
    if constexpr (!INVERSE) ct_group<K1, G, true>(x, A.tw, 0, 0, Mod{p, pp});
    else gs_group<K1, G, true>(x, A.tw, 0, 0, Mod{p, pp});
#pragma unroll
    for (int g = 0; g < G; g++)
#pragma unroll
        for (int t = 0; t < N1; t++) {
            const size_t j = c0 + g * kRegColThreads + (static_cast<size_t>(t) << A.k2);
            uint32_t v = x[g][t];
            if (A.post) v = mont_mul(v, A.post, p, pp);
            if (j < A.dst_len && static_cast<uint32_t>(t) < A.rows) dst[j] = v;
        }
}

// Inverse column pass of a truncated product (row-granular TFT): the
// product computed only rows t < L of the 2^K1 rows of 2^k2, so each column
// holds L known outputs of its column transform and has zero inputs from L
// on (c is zero from L 2^k2 on); an inverse TFT per column (itft_node)
// recovers its L inputs, exactly scaled, and writes those below dst_len.
template <int K1, int L>
__global__ void __launch_bounds__(kRegColThreads) k_col_regs_itft(ColArgs A, size_t prod0)
{
    constexpr int N1 = 1 << K1, G = 16 / N1;
    const size_t prod = prod0 + blockIdx.z;
    const uint32_t *src = A.src[0] + prod * A.src_stride[0];
    uint32_t *dst = A.dst[0] + prod * A.dst_stride;
    const Mod md{A.p, A.pp};
    const size_t c0 = static_cast<size_t>(blockIdx.x) * (kRegColThreads * G) + threadIdx.x;
    uint32_t x[G][N1];
#pragma unroll
    for (int g = 0; g < G; g++)
#pragma unroll
        for (int t = 0; t < N1; t++)
            x[g][t] = t < L ? __ldg(src + c0 + g * kRegColThreads + (static_cast<size_t>(t) << A.k2)) : 0u;
#pragma unroll
    for (int g = 0; g < G; g++) itft_node<N1, 0, N1, L, 0, 0>(x[g], A.tw, A.itw, md);
#pragma unroll
    for (int g = 0; g < G; g++)
#pragma unroll
        for (int t = 0; t < L; t++) {
            const size_t j = c0 + g * kRegColThreads + (static_cast<size_t>(t) << A.k2);
            if (j < A.dst_len) dst[j] = x[g][t];
        }
}

struct RowArgs {
    uint32_t *ws;       // product i: A' at ws + i * 2N, B' at + N; C' overwrites A'
    size_t n;
    int k1;
    const uint32_t *tw, *itw;
    uint32_t p, pp;
};

// Row r of a product: forward row levels of A' and B', pointwise product,
// inverse row levels, C' in place of A'.
template <int K2>
__global__ void __launch_bounds__(nt_of<K2>(), min_ctas_of<K2>())
k_row_polymul(RowArgs A, size_t prod0)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const size_t prod = prod0 + blockIdx.y;
    const int r = blockIdx.x;
    uint32_t *base = A.ws + prod * 2 * A.n + (static_cast<size_t>(r) << K2);
    polymul_team<K2, false, false>(smem, threadIdx.x, base, size_t{1} << K2, base + A.n, size_t{1} << K2, base,
                                   size_t{1} << K2, A.tw, A.itw, A.k1, r, A.p, A.pp, 0u);
}

struct RowNttArgs {
    uint32_t *data;
    size_t n;
    int k1;
    const uint32_t *tw;
    uint32_t p, pp;
};

// K1 >= 0: the column level count as a compile-time constant, so every
// twiddle index of the row levels folds; K1 = -1 takes A.k1.
template <int K2, int K1, bool INVERSE>
__global__ void __launch_bounds__(nt_of<K2>(), K2 <= 13 ? 4 : 1)
k_row_ntt(RowNttArgs A, size_t prod0)
{
    constexpr int N2 = 1 << K2, NT = nt_of<K2>(), NP = SchedFor<K2, NT>::kPasses;
    const int k1 = K1 >= 0 ? K1 : A.k1;
    extern __shared__ __align__(16) uint32_t smem[];
    const size_t prod = prod0 + blockIdx.y;
    const int r = blockIdx.x;
    uint32_t *g = A.data + prod * A.n + (static_cast<size_t>(r) << K2);
    const PadLayout lay[1] = {{smem}};
    const Mod md{A.p, A.pp};
    using P0 = PassGeom<K2, NT, 0>;
    static_assert(NP >= 2, "rows take at least two passes");
    if constexpr (!INVERSE) {
        // pass 0 straight from global memory (a warp reads consecutive words)
#pragma unroll
        for (int q = 0; q < P0::GPT; q++) {
            const int base = P0::base(threadIdx.x, q);
            uint32_t x[1][P0::G];
#pragma unroll
            for (int t = 0; t < P0::G; t++) x[0][t] = g[base + t * P0::HMIN];
            ct_group<P0::E, 1, false>(x, A.tw, k1, (r << P0::S0) + P0::blk(threadIdx.x, q), md);
#pragma unroll
            for (int t = 0; t < P0::G; t++) elem(lay[0], base, t * P0::HMIN) = x[0][t];
        }
        __syncthreads();
        fwd_passes<K2, NT, 1, false, 1, NP - 1>(lay, threadIdx.x, A.tw, k1, r, md);
        // word tid + NT i: tid < NT and NT i on disjoint bits, so its padded
        // position is this thread's pointer plus a compile-time offset
        const uint32_t *src = lay[0].at(threadIdx.x);
#pragma unroll
        for (int i = 0; i < N2 / NT; i++) g[threadIdx.x + i * NT] = csub(src[PadLayout::off(i * NT)], A.p);
    } else {
        {
            // every load of the thread in flight before its first store; the
            // padded positions as in the forward's output loop
            uint32_t v[N2 / NT];
#pragma unroll
            for (int i = 0; i < N2 / NT; i++) v[i] = g[threadIdx.x + i * NT];
            uint32_t *dst = lay[0].at(threadIdx.x);
#pragma unroll
            for (int i = 0; i < N2 / NT; i++) dst[PadLayout::off(i * NT)] = v[i];
        }
        __syncthreads();
        inv_passes<K2, NT, false, NP - 1, 1>(lay[0], threadIdx.x, A.tw, k1, r, md);
        // pass 0 straight to global memory
#pragma unroll
        for (int q = 0; q < P0::GPT; q++) {
            const int base = P0::base(threadIdx.x, q);
            uint32_t x[1][P0::G];
#pragma unroll
            for (int t = 0; t < P0::G; t++) x[0][t] = elem(lay[0], base, t * P0::HMIN);
            gs_group<P0::E, 1, false>(x, A.tw, k1, (r << P0::S0) + P0::blk(threadIdx.x, q), md);
#pragma unroll
            for (int t = 0; t < P0::G; t++) g[base + t * P0::HMIN] = x[0][t];
        }
    }
}

__device__ __forceinline__ int brev5(int x)
{
    return static_cast<int>(__brev(static_cast<unsigned>(x)) >> 27);
}

// In-place bit reversal of each row of 2^log2n elements (log2n >= 10) by
// 32 x 32 tiles.  Index i = (a, b, c): a the top 5 bits, c the bottom 5, b
// the log2n - 10 bits between; brev(i) = (brev5(c), brev(b), brev5(a)).  So
// tile b (32 rows a of 32 consecutive words c, rows 2^(log2n-5) apart) and
// tile brev(b) trade places with a transpose: one CTA per pair, both tiles
// read before either is written.  Loads and stores move 128-byte row
// segments; the padded shared-memory tiles make the transposed reads
// conflict-free.
__global__ void __launch_bounds__(256) k_bitrev_tiles(uint32_t *data, int log2n, size_t row0)
{
    __shared__ uint32_t t0[32][33], t1[32][33];
    const int mb = log2n - 10;
    const unsigned b = blockIdx.x;
    const unsigned bb = mb > 0 ? (__brev(b) >> (32 - mb)) : 0u;
    if (b > bb) return;                                  // the pair's other CTA does it
    uint32_t *g = data + (row0 + blockIdx.y) * (size_t{1} << log2n);
    const size_t rs = size_t{1} << (log2n - 5);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int a = ty + 8 * k;
        t0[a][tx] = g[a * rs + (static_cast<size_t>(b) << 5) + tx];
        t1[a][tx] = g[a * rs + (static_cast<size_t>(bb) << 5) + tx];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int r = ty + 8 * k;                        // output row brev5(c), column tx = brev5(a)
        g[r * rs + (static_cast<size_t>(bb) << 5) + tx] = t0[brev5(tx)][brev5(r)];
        if (b != bb) g[r * rs + (static_cast<size_t>(b) << 5) + tx] = t1[brev5(tx)][brev5(r)];
    }
}

constexpr unsigned kMaxGridZ = 65535;

template <int K1, bool INVERSE>
int launch_col(const ColArgs &A, size_t nops, size_t count, cudaStream_t s)
{
    using CF = ColCfg<K1>;
    constexpr bool kDirect = CF::C % 32 == 0 && SchedFor<K1, CF::NT1>::kPasses == 2;
    constexpr size_t smem = kDirect ? static_cast<size_t>(CF::C) * (CF::N1 + 1) * sizeof(uint32_t) : CF::SMEM;
    void (*kern)(ColArgs, size_t);
    if constexpr (kDirect) kern = k_col_direct<K1, INVERSE>;
    else kern = k_col<K1, INVERSE>;
    if (ensure_smem(kern, smem) != MONT_OK) return MONT_ECUDA;
    const size_t n2 = size_t{1} << A.k2;
    for (size_t first = 0; first < count; first += kMaxGridZ) {
        const unsigned z = static_cast<unsigned>(std::min<size_t>(kMaxGridZ, count - first));
        dim3 grid(static_cast<unsigned>(n2 / CF::C), static_cast<unsigned>(nops), z);
        kern<<<grid, CF::THREADS, smem, s>>>(A, first);
        if (cudaGetLastError() != cudaSuccess) return MONT_ECUDA;
    }
    return MONT_OK;
}

template <int K1, bool INVERSE>
int launch_col_regs(const ColArgs &A, size_t nops, size_t count, cudaStream_t s)
{
    constexpr int COLS = kRegColThreads * (16 >> K1);
    const size_t n2 = size_t{1} << A.k2;
    for (size_t first = 0; first < count; first += kMaxGridZ) {
        const unsigned z = static_cast<unsigned>(std::min<size_t>(kMaxGridZ, count - first));
        dim3 grid(static_cast<unsigned>(n2 / COLS), static_cast<unsigned>(nops), z);
        k_col_regs<K1, INVERSE><<<grid, kRegColThreads, 0, s>>>(A, first);
        if (cudaGetLastError() != cudaSuccess) return MONT_ECUDA;
    }
    return MONT_OK;
}

template <int K2>
int launch_row_polymul(const RowArgs &A, size_t count, cudaStream_t s, uint32_t rows)
{
    const size_t smem = team_smem_words<K2>() * sizeof(uint32_t);
    if (ensure_smem(k_row_polymul<K2>, smem) != MONT_OK) return MONT_ECUDA;
    for (size_t first = 0; first < count; first += kMaxGridZ) {
        const unsigned y = static_cast<unsigned>(std::min<size_t>(kMaxGridZ, count - first));
        k_row_polymul<K2><<<dim3(rows, y), nt_of<K2>(), smem, s>>>(A, first);
        if (cudaGetLastError() != cudaSuccess) return MONT_ECUDA;
    }
    return MONT_OK;
}

template <int K2, int K1, bool INVERSE>
int launch_row_ntt(const RowNttArgs &A, size_t count, cudaStream_t s)
{
    const size_t smem = PadLayout::words(1 << K2) * sizeof(uint32_t);
    if (ensure_smem(k_row_ntt<K2, K1, INVERSE>, smem) != MONT_OK) return MONT_ECUDA;
    const unsigned rows = static_cast<unsigned>(A.n >> K2);
    for (size_t first = 0; first < count; first += kMaxGridZ) {
        const unsigned y = static_cast<unsigned>(std::min<size_t>(kMaxGridZ, count - first));
        k_row_ntt<K2, K1, INVERSE><<<dim3(rows, y), nt_of<K2>(), smem, s>>>(A, first);
        if (cudaGetLastError() != cudaSuccess) return MONT_ECUDA;
    }
    return MONT_OK;
}

// Row levels K2: 2^12 rows up to N = 2^16; rows of 2^13 and 2^14 for
// N = 2^17 and 2^18, which keeps four column levels (register column
// passes); beyond, rows of 2^13 (measured against rows of 2^12 and 2^14 for
// N = 2^19, 2^20, 2^21: 1-6 % faster, the shared-memory column tiles then
// one level shorter) until K - 10 > 13.
int split_k2(int k)
{
    if (k <= 16) return 12;
    if (k <= 18) return k - 4;
    return std::max(13, k - 10);
}

// Products of N = 2^19 and 2^20 take rows of 2^12 (the fused 4096-point row
// product, four CTAs per SM, after seven or eight column levels): 18 % and
// 11 % faster than rows of 2^13, while 2^21 is faster with rows of 2^13 and
// the stand-alone transforms keep rows of 2^13.
int split_k2_polymul(int k)
{
    return (k == 19 || k == 20) ? 12 : split_k2(k);
}

#define MONT_K1_TILE_CASES(X) X(5) X(6) X(7) X(8) X(9) X(10)

template <bool INVERSE>
int dispatch_col(int k1, const ColArgs &A, size_t nops, size_t count, cudaStream_t s)
{
    switch (k1) {
    case 1: return launch_col_regs<1, INVERSE>(A, nops, count, s);
    case 2: return launch_col_regs<2, INVERSE>(A, nops, count, s);
    case 3: return launch_col_regs<3, INVERSE>(A, nops, count, s);
    case 4: return launch_col_regs<4, INVERSE>(A, nops, count, s);
#define X(K) \
    case K: return launch_col<K, INVERSE>(A, nops, count, s);
        MONT_K1_TILE_CASES(X)
#undef X
    default: return MONT_EUNSUPPORTED;
    }
}

int dispatch_row_polymul(int k2, const RowArgs &A, size_t count, cudaStream_t s, uint32_t rows)
{
    switch (k2) {
    case 12: return launch_row_polymul<12>(A, count, s, rows);
    case 13: return launch_row_polymul<13>(A, count, s, rows);
    case 14: return launch_row_polymul<14>(A, count, s, rows);
    default: return MONT_EUNSUPPORTED;
    }
}

// The (K2, K1) pairs split_k2 gives for N = 2^15 .. 2^24 have their own row
// kernels; any other pair runs the kernel that reads K1 from its arguments.
template <bool INVERSE>
int dispatch_row_ntt(int k2, const RowNttArgs &A, size_t count, cudaStream_t s)
{
    switch (k2 * 16 + A.k1) {
#define X(K2, K1) \
    case K2 * 16 + K1: return launch_row_ntt<K2, K1, INVERSE>(A, count, s);
        X(12, 3) X(12, 4) X(13, 4) X(14, 4) X(13, 6) X(13, 7) X(13, 8) X(13, 9) X(13, 10) X(14, 10)
#undef X
    default: break;
    }
    switch (k2) {
    case 12: return launch_row_ntt<12, -1, INVERSE>(A, count, s);
    case 13: return launch_row_ntt<13, -1, INVERSE>(A, count, s);
    case 14: return launch_row_ntt<14, -1, INVERSE>(A, count, s);
    default: return MONT_EUNSUPPORTED;
    }
}

template <int K1, int L>
int launch_col_itft(const ColArgs &A, size_t count, cudaStream_t s)
{
    constexpr int COLS = kRegColThreads * (16 >> K1);
    const size_t n2 = size_t{1} << A.k2;
    for (size_t first = 0; first < count; first += kMaxGridZ) {
        const unsigned z = static_cast<unsigned>(std::min<size_t>(kMaxGridZ, count - first));
        k_col_regs_itft<K1, L><<<dim3(static_cast<unsigned>(n2 / COLS), 1, z), kRegColThreads, 0, s>>>(A, first);
        if (cudaGetLastError() != cudaSuccess) return MONT_ECUDA;
    }
    return MONT_OK;
}

// Inverse TFT column pass for K1 column levels of which `rows` rows were
// computed, 2^(K1-1) < rows < 2^K1.
int dispatch_col_itft(int k1, uint32_t rows, const ColArgs &A, size_t count, cudaStream_t s)
{
    switch (k1 * 16 + static_cast<int>(rows)) {
    case 2 * 16 + 3: return launch_col_itft<2, 3>(A, count, s);
    case 3 * 16 + 5: return launch_col_itft<3, 5>(A, count, s);
    case 3 * 16 + 6: return launch_col_itft<3, 6>(A, count, s);
    case 3 * 16 + 7: return launch_col_itft<3, 7>(A, count, s);
    case 4 * 16 + 9: return launch_col_itft<4, 9>(A, count, s);
    case 4 * 16 + 10: return launch_col_itft<4, 10>(A, count, s);
    case 4 * 16 + 11: return launch_col_itft<4, 11>(A, count, s);
    case 4 * 16 + 12: return launch_col_itft<4, 12>(A, count, s);
    case 4 * 16 + 13: return launch_col_itft<4, 13>(A, count, s);
    case 4 * 16 + 14: return launch_col_itft<4, 14>(A, count, s);
    case 4 * 16 + 15: return launch_col_itft<4, 15>(A, count, s);
    default: return MONT_EUNSUPPORTED;
    }
}

int launch_bitrev(uint32_t *data, int log2n, size_t batch, cudaStream_t s)
{
    if (log2n < 10) return MONT_EUNSUPPORTED;
    const unsigned tiles = 1u << (log2n - 10);
    for (size_t first = 0; first < batch; first += kMaxGridZ) {
        const unsigned y = static_cast<unsigned>(std::min<size_t>(kMaxGridZ, batch - first));
        k_bitrev_tiles<<<dim3(tiles, y), 256, 0, s>>>(data, log2n, first);
        if (cudaGetLastError() != cudaSuccess) return MONT_ECUDA;
    }
    return MONT_OK;
}

}  // namespace

int polymul_large(const ntt_plan &plan, const uint32_t *a, size_t la, const uint32_t *b, size_t lb, uint32_t *c,
                  size_t count, uint32_t *ws, cudaStream_t s)
{
    const int k = plan.log2n, k2 = split_k2_polymul(k), k1 = k - k2;
    const size_t n = size_t{1} << k;
    // Row-granular truncated transform (as in the batches): with register
    // column passes (2 <= K1 <= 4), compute only the ceil(lc / 2^K2) rows the
    // output reaches, and invert each column with an inverse TFT; b is then
    // scaled by (2^K2)^-1 R^2, since the inverse column pass scales exactly.
    const size_t lc = la + lb - 1;
    const uint32_t rows_all = 1u << k1;
    const uint32_t need = static_cast<uint32_t>((lc + (size_t{1} << k2) - 1) >> k2);
    const bool tft = k1 >= 2 && k1 <= 4 && need < rows_all;
    uint32_t k_scale = plan.k_scale;
    if (tft) {
        const uint32_t m_mod = static_cast<uint32_t>((uint64_t{1} << k2) % plan.p);
        k_scale = host_to_mont(host_to_mont(host_powmod(m_mod, plan.p - 2, plan.p), plan.p), plan.p);
    }
    ColArgs F{};
    F.src[0] = a;
    F.src[1] = b;
    F.src_len[0] = la;
    F.src_len[1] = lb;
    F.src_stride[0] = la;
    F.src_stride[1] = lb;
    F.dst[0] = ws;
    F.dst[1] = ws + n;
    F.dst_len = n;
    F.dst_stride = 2 * n;
    F.k2 = k2;
    F.tw = plan.table->fwd;
    F.p = plan.p;
    F.pp = plan.p_prime;
    F.scale[0] = 0;
    F.scale[1] = k_scale;
    F.post = 0;
    F.rows = tft ? need : rows_all;
    int rc = dispatch_col<false>(k1, F, 2, count, s);
    if (rc != MONT_OK) return rc;
    RowArgs R{ws, n, k1, plan.table->fwd, plan.table->inv, plan.p, plan.p_prime};
    rc = dispatch_row_polymul(k2, R, count, s, tft ? need : rows_all);
    if (rc != MONT_OK) return rc;
    ColArgs I{};
    I.src[0] = I.src[1] = ws;
    I.src_len[0] = I.src_len[1] = n;
    I.src_stride[0] = I.src_stride[1] = 2 * n;
    I.dst[0] = I.dst[1] = c;
    I.dst_len = la + lb - 1;
    I.dst_stride = la + lb - 1;
    I.k2 = k2;
    I.tw = plan.table->inv;
    I.p = plan.p;
    I.pp = plan.p_prime;
    I.rows = rows_all;
    if (tft) {
        I.tw = plan.table->fwd;   // itft_node takes both tables
        I.itw = plan.table->inv;
        return dispatch_col_itft(k1, need, I, count, s);
    }
    return dispatch_col<true>(k1, I, 1, count, s);
}

int ntt_large(const ntt_plan *plan, uint32_t *data, size_t batch, int flags, bool inverse, cudaStream_t s)
{
    const int k = plan->log2n, k2 = split_k2(k), k1 = k - k2;
    const size_t n = size_t{1} << k;
    if (batch > SIZE_MAX / n / 4) return MONT_ERANGE;
    ColArgs C{};
    C.src[0] = C.src[1] = data;
    C.src_len[0] = C.src_len[1] = n;
    C.src_stride[0] = C.src_stride[1] = n;
    C.dst[0] = C.dst[1] = data;
    C.dst_len = n;
    C.dst_stride = n;
    C.k2 = k2;
    C.p = plan->p;
    C.pp = plan->p_prime;
    C.rows = 1u << k1;
    RowNttArgs R{data, n, k1, nullptr, plan->p, plan->p_prime};
    int rc;
    if (!inverse) {
        C.tw = R.tw = plan->table->fwd;
        if ((rc = dispatch_col<false>(k1, C, 1, batch, s)) != MONT_OK) return rc;
        if ((rc = dispatch_row_ntt<false>(k2, R, batch, s)) != MONT_OK) return rc;
        if (!(flags & NTT_BITREV)) return launch_bitrev(data, k, batch, s);
        return MONT_OK;
    }
    C.tw = R.tw = plan->table->inv;
    C.post = plan->ninv_mont;
    if (!(flags & NTT_BITREV) && (rc = launch_bitrev(data, k, batch, s)) != MONT_OK) return rc;
    if ((rc = dispatch_row_ntt<true>(k2, R, batch, s)) != MONT_OK) return rc;
    return dispatch_col<true>(k1, C, 1, batch, s);
}

}  // namespace mont
