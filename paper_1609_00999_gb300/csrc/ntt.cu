// ntt.cu -- NTT and fused polynomial-multiplication kernels, C-ABI entry points.
//
// Polymul of one product (c = a * b mod P, la + lb - 1 coefficients, cyclic
// convolution of size N = 2^K >= la + lb - 1), N <= 2^14, in one team of
// threads with both operands in shared memory:
//   pass 0       : load a, b from HBM (zero padding), scale b by N^-1 R^2 on
//                  load, forward levels of pass 0 in registers -> smem
//   passes 1..   : forward levels, smem -> registers -> smem
//   last pass    : forward levels of both operands, pointwise REDC
//                  C = A * B~ * R^-1 (= A B N^-1), then the same levels of the
//                  inverse in reverse, all in registers -> smem (one array)
//   back down    : inverse levels, smem -> registers -> smem
//   pass 0       : inverse levels -> c in HBM (only the la + lb - 1 outputs)
// One HBM read of a and b and one write of c per product.  The forward
// output stays in bit-reversed order and the inverse consumes it there, so
// no permutation is ever done.
//
// N > 2^14 splits the K levels into K1 column levels and K2 = K - K1 row
// levels (ntt_large.cu): a column kernel runs levels 0..K1-1 on strided
// columns of 2^K1 elements, the row kernel runs levels K1..K-1 of both
// operands on contiguous rows of 2^K2 elements (block r of the transform),
// the pointwise product and the inverse row levels, and a second column
// kernel runs the inverse column levels.  Three HBM round trips through a
// scratch buffer of 2N words per product.
#include <algorithm>

#include "ntt_internal.cuh"
#include "ntt_kernels.cuh"

namespace mont {
namespace {

template <int LOGN>
__device__ __forceinline__ int brev(int k)
{
    if constexpr (LOGN == 0) return 0;
    else return static_cast<int>(__brev(static_cast<unsigned>(k)) >> (32 - LOGN));
}

// The same for a compile-time k.
template <int LOGN>
constexpr int brev_c(int k)
{
    int r = 0;
    for (int b = 0; b < LOGN; b++) r |= ((k >> b) & 1) << (LOGN - 1 - b);
    return r;
}

// Natural-order I/O of a transform held in the padded layout at bit-reversed
// positions (word k of the natural order sits at brev(k)).  A warp that
// walks 32 consecutive k hits brev(k) at addresses whose low bits repeat,
// 2- to 16-way bank conflicts for N = 2^11 .. 2^14.  Instead, lane-step m
// covers the S consecutive words k = S m + r, r < S, with
// S = max(4, 2^(log2 N - 10)), and the lanes of a warp take consecutive m:
// for a fixed r the 32 lanes then differ in bits 5 .. 9 of brev(k) (bits
// 4 .. 8 for N = 2^11), which the padding word per 32 maps onto 32 distinct
// banks.  Each lane moves its S words of global memory as S / 4 uint4.
// S m and r < S have disjoint bits, so brev(S m + r) = brev(S m) | brev(r),
// and the padded layout adds over disjoint bits: word r of a lane-step is
// the step's pointer plus the compile-time offset of brev(r).
template <int LOGN, int NT>
struct BrevIO {
    static constexpr int N = 1 << LOGN;
    static constexpr int S = LOGN > 12 ? (1 << (LOGN - 10)) : 4;
    static constexpr int STEPS = N / S / NT;
    static constexpr bool kUse = LOGN >= 11 && STEPS >= 1 && N % (S * NT) == 0;
};

struct NttArgs {
    uint32_t *data;
    size_t batch;
    const uint32_t *tw;
    uint32_t p, pp, ninv_mont;
    int bitrev;
    int aligned16;   // data 16-byte aligned: rows move as uint4
};

// In-place forward NTT of [batch][N]; natural order in, natural (or, with
// bitrev, bit-reversed) order out.
template <int LOGN>
__global__ void __launch_bounds__(teams_of<LOGN>() * nt_of<LOGN>())
k_ntt_fwd(NttArgs A)
{
    constexpr int N = 1 << LOGN, NT = nt_of<LOGN>(), NP = SchedFor<LOGN, NT>::kPasses;
    extern __shared__ __align__(16) uint32_t smem[];
    const int team = threadIdx.x / NT, tid = threadIdx.x - team * NT;
    const size_t prod = static_cast<size_t>(blockIdx.x) * teams_of<LOGN>() + team;
    const bool valid = prod < A.batch;
    uint32_t *g = A.data + (valid ? prod * N : 0);
    const PadLayout lay[1] = {{smem + static_cast<size_t>(team) * PadLayout::words(N)}};
    const Mod md{A.p, A.pp};
    if constexpr (NP <= 1) {
        stage_in<N, NT>(lay[0], g, tid, valid, [](int k) { return k; });
        __syncthreads();
        fwd_passes<LOGN, NT, 1, true, 0, NP - 1>(lay, tid, A.tw, 0, 0, md);
    } else {
        // pass 0 straight from global memory (a warp reads consecutive words)
        using P0 = PassGeom<LOGN, NT, 0>;
#pragma unroll
        for (int r = 0; r < P0::GPT; r++) {
            const int base = P0::base(tid, r);
            uint32_t x[1][P0::G];
#pragma unroll
            for (int t = 0; t < P0::G; t++) x[0][t] = valid ? g[base + t * P0::HMIN] : 0u;
            ct_group<P0::E, 1, true>(x, A.tw, 0, 0, md);
#pragma unroll
            for (int t = 0; t < P0::G; t++) elem(lay[0], base, t * P0::HMIN) = x[0][t];
        }
        __syncthreads();
        fwd_passes<LOGN, NT, 1, true, 1, NP - 1>(lay, tid, A.tw, 0, 0, md);
    }
    if (!valid) return;
    if constexpr (BrevIO<LOGN, NT>::kUse) {
        using IO = BrevIO<LOGN, NT>;
        if (!A.bitrev && A.aligned16) {
#pragma unroll
            for (int i = 0; i < IO::STEPS; i++) {
                const int k0 = IO::S * (tid + NT * i);
                uint4 *dst = reinterpret_cast<uint4 *>(g + k0);
                const uint32_t *src = lay[0].at(brev<LOGN>(k0));
#pragma unroll
                for (int q = 0; q < IO::S / 4; q++) {
                    uint4 v;
                    v.x = csub(src[PadLayout::off(brev_c<LOGN>(4 * q))], A.p);
                    v.y = csub(src[PadLayout::off(brev_c<LOGN>(4 * q + 1))], A.p);
                    v.z = csub(src[PadLayout::off(brev_c<LOGN>(4 * q + 2))], A.p);
                    v.w = csub(src[PadLayout::off(brev_c<LOGN>(4 * q + 3))], A.p);
                    dst[q] = v;
                }
            }
            return;
        }
    }
    for (int k = tid; k < N; k += NT) g[k] = csub(lay[0][A.bitrev ? k : brev<LOGN>(k)], A.p);
}

// In-place inverse NTT (with the factor N^-1) of [batch][N]; natural (or,
// with bitrev, bit-reversed) order in, natural order out.
template <int LOGN>
__global__ void __launch_bounds__(teams_of<LOGN>() * nt_of<LOGN>())
k_ntt_inv(NttArgs A)
{
    constexpr int N = 1 << LOGN, NT = nt_of<LOGN>(), NP = SchedFor<LOGN, NT>::kPasses;
    extern __shared__ __align__(16) uint32_t smem[];
    const int team = threadIdx.x / NT, tid = threadIdx.x - team * NT;
    const size_t prod = static_cast<size_t>(blockIdx.x) * teams_of<LOGN>() + team;
    const bool valid = prod < A.batch;
    uint32_t *g = A.data + (valid ? prod * N : 0);
    const PadLayout lay = {smem + static_cast<size_t>(team) * PadLayout::words(N)};
    const Mod md{A.p, A.pp};
    const int bitrev = A.bitrev;
    bool staged = false;
    if constexpr (BrevIO<LOGN, NT>::kUse) {
        using IO = BrevIO<LOGN, NT>;
        if (!bitrev && A.aligned16) {
            // every uint4 load of the thread in flight before its first store
            uint4 v[IO::STEPS][IO::S / 4];
#pragma unroll
            for (int i = 0; i < IO::STEPS; i++)
#pragma unroll
                for (int q = 0; q < IO::S / 4; q++)
                    v[i][q] = valid ? reinterpret_cast<const uint4 *>(g + IO::S * (tid + NT * i))[q]
                                    : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int i = 0; i < IO::STEPS; i++) {
                uint32_t *dst = lay.at(brev<LOGN>(IO::S * (tid + NT * i)));
#pragma unroll
                for (int q = 0; q < IO::S / 4; q++) {
                    dst[PadLayout::off(brev_c<LOGN>(4 * q))] = v[i][q].x;
                    dst[PadLayout::off(brev_c<LOGN>(4 * q + 1))] = v[i][q].y;
                    dst[PadLayout::off(brev_c<LOGN>(4 * q + 2))] = v[i][q].z;
                    dst[PadLayout::off(brev_c<LOGN>(4 * q + 3))] = v[i][q].w;
                }
            }
            staged = true;
        }
    }
    if (!staged) stage_in<N, NT>(lay, g, tid, valid, [bitrev](int k) { return bitrev ? k : brev<LOGN>(k); });
    __syncthreads();
    if constexpr (NP <= 1) {
        inv_passes<LOGN, NT, true, NP - 1, 0>(lay, tid, A.tw, 0, 0, md);
        if (valid)
            for (int k = tid; k < N; k += NT) g[k] = mont_mul(lay[k], A.ninv_mont, A.p, A.pp);
    } else {
        inv_passes<LOGN, NT, true, NP - 1, 1>(lay, tid, A.tw, 0, 0, md);
        // pass 0 scaled by N^-1 and stored straight to global memory
        using P0 = PassGeom<LOGN, NT, 0>;
#pragma unroll
        for (int r = 0; r < P0::GPT; r++) {
            const int base = P0::base(tid, r);
            uint32_t y[1][P0::G];
#pragma unroll
            for (int t = 0; t < P0::G; t++) y[0][t] = elem(lay, base, t * P0::HMIN);
            gs_group<P0::E, 1, true>(y, A.tw, 0, 0, md);
            if (valid)
#pragma unroll
                for (int t = 0; t < P0::G; t++) g[base + t * P0::HMIN] = mont_mul(y[0][t], A.ninv_mont, A.p, A.pp);
        }
    }
}

template <int LOGN>
int launch_ntt_smem(const NttArgs &A, bool inverse, cudaStream_t s)
{
    constexpr int T = teams_of<LOGN>(), NT = nt_of<LOGN>();
    const size_t smem = static_cast<size_t>(T) * PadLayout::words(1 << LOGN) * sizeof(uint32_t);
    const size_t grid = (A.batch + T - 1) / T;
    if (grid > 0x7FFFFFFFu) return MONT_ERANGE;
    if (inverse) {
        if (ensure_smem(k_ntt_inv<LOGN>, smem) != MONT_OK) return MONT_ECUDA;
        k_ntt_inv<LOGN><<<static_cast<unsigned>(grid), T * NT, smem, s>>>(A);
    } else {
        if (ensure_smem(k_ntt_fwd<LOGN>, smem) != MONT_OK) return MONT_ECUDA;
        k_ntt_fwd<LOGN><<<static_cast<unsigned>(grid), T * NT, smem, s>>>(A);
    }
    return launch_status();
}

#define MONT_LOGN_CASES(X) \
    X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14)

int ntt_common(const ntt_plan *plan, uint32_t *data, size_t batch, int flags, bool inverse, cudaStream_t s)
{
    if (!plan || (flags & ~NTT_BITREV)) return MONT_EINVAL;
    if (batch == 0) return MONT_OK;
    if (!data) return MONT_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return MONT_ECUDA;
    if (dev != plan->device) return MONT_EINVAL;
    if (plan->log2n > kMaxSmemLog2N) return ntt_large(plan, data, batch, flags, inverse, s);
    NttArgs A;
    A.data = data;
    A.batch = batch;
    A.tw = inverse ? plan->table->inv : plan->table->fwd;
    A.p = plan->p;
    A.pp = plan->p_prime;
    A.ninv_mont = plan->ninv_mont;
    A.bitrev = (flags & NTT_BITREV) ? 1 : 0;
    A.aligned16 = (reinterpret_cast<uintptr_t>(data) & 15u) == 0;
    switch (plan->log2n) {
#define X(L) \
    case L: return launch_ntt_smem<L>(A, inverse, s);
        MONT_LOGN_CASES(X)
#undef X
    default: return MONT_EUNSUPPORTED;
    }
}

}  // namespace

int ceil_log2(size_t n)
{
    int k = 0;
    while ((size_t{1} << k) < n) k++;
    return k;
}

int dispatch_polymul_smem(int log2n, const PolyArgs &A, cudaStream_t s)
{
    switch (log2n) {
#define X(L) \
    case L: return launch_polymul_smem<L, RedAlg2>(A, s);
        MONT_LOGN_CASES(X)
#undef X
    default: return MONT_EUNSUPPORTED;
    }
}

// Checks shared by the polymul entry points; fills the plan for N.
int polymul_prepare(uint32_t p, const uint32_t *a, size_t la, const uint32_t *b, size_t lb, const uint32_t *c,
                    size_t count, ntt_plan *plan, int *log2n)
{
    if (!a || !b || !c || la == 0 || lb == 0) return MONT_EINVAL;
    if (la > (size_t{1} << 30) || lb > (size_t{1} << 30)) return MONT_ERANGE;
    const size_t lc = la + lb - 1;
    if (count > SIZE_MAX / 4 / (lc + la + lb)) return MONT_ERANGE;
    const size_t wa = count * la * 4, wb = count * lb * 4, wc = count * lc * 4;
    if (any_overlap(c, wc, a, wa) || any_overlap(c, wc, b, wb)) return MONT_EINVAL;
    *log2n = ceil_log2(lc);
    if (*log2n > kMaxLog2N) return MONT_ERANGE;
    return make_plan(p, *log2n, plan);
}

}  // namespace mont

extern "C" int ntt_fwd(const ntt_plan *plan, uint32_t *data, size_t batch, int flags, cudaStream_t stream)
{
    return mont::ntt_common(plan, data, batch, flags, false, stream);
}

extern "C" int ntt_inv(const ntt_plan *plan, uint32_t *data, size_t batch, int flags, cudaStream_t stream)
{
    return mont::ntt_common(plan, data, batch, flags, true, stream);
}

extern "C" size_t polymul_workspace_bytes(size_t la, size_t lb, size_t count)
{
    if (la == 0 || lb == 0 || count == 0) return 0;
    const int log2n = mont::ceil_log2(la + lb - 1);
    if (log2n <= mont::kMaxSmemLog2N) return 0;
    return count * 2 * (size_t{1} << log2n) * sizeof(uint32_t);
}

extern "C" int polymul_many_ws(uint32_t p, const uint32_t *a, size_t la, const uint32_t *b, size_t lb, uint32_t *c,
                               size_t count, void *workspace, size_t ws_bytes, cudaStream_t stream)
{
    if (count == 0) return MONT_OK;
    ntt_plan plan;
    int log2n = 0;
    int rc = mont::polymul_prepare(p, a, la, b, lb, c, count, &plan, &log2n);
    if (rc != MONT_OK) return rc;
    const size_t lc = la + lb - 1;
    if (log2n <= mont::kMaxSmemLog2N) {
        mont::PolyArgs A;
        A.a = a;
        A.b = b;
        A.c = c;
        A.la = la;
        A.lb = lb;
        A.lc = lc;
        A.count = count;
        A.tw = plan.table->fwd;
        A.itw = plan.table->inv;
        A.p = p;
        A.pp = plan.p_prime;
        A.k_scale = plan.k_scale;
        return mont::dispatch_polymul_smem(log2n, A, stream);
    }
    const size_t per = 2 * (size_t{1} << log2n) * sizeof(uint32_t);
    if (!workspace || ws_bytes < per) return MONT_EINVAL;
    if ((reinterpret_cast<uintptr_t>(workspace) & 15u) != 0) return MONT_EINVAL;
    const size_t chunk = ws_bytes / per;
    for (size_t first = 0; first < count; first += chunk) {
        const size_t n = std::min(chunk, count - first);
        rc = mont::polymul_large(plan, a + first * la, la, b + first * lb, lb, c + first * lc, n,
                                 static_cast<uint32_t *>(workspace), stream);
        if (rc != MONT_OK) return rc;
    }
    return MONT_OK;
}

extern "C" int polymul_many(uint32_t p, const uint32_t *a, size_t la, const uint32_t *b, size_t lb, uint32_t *c,
                            size_t count, cudaStream_t stream)
{
    if (count == 0) return MONT_OK;
    const size_t need = polymul_workspace_bytes(la, lb, count);
    if (need == 0) return polymul_many_ws(p, a, la, b, lb, c, count, nullptr, 0, stream);
    // Library-owned scratch, one buffer per (device, stream), at most 1 GiB:
    // larger batches run in chunks of products.
    const size_t per = polymul_workspace_bytes(la, lb, 1);
    const size_t cap = std::max(per, std::min(need, size_t{1} << 30) / per * per);
    void *ws = nullptr;
    int rc = mont::stream_workspace(stream, cap, &ws);
    if (rc != MONT_OK) return rc;
    return polymul_many_ws(p, a, la, b, lb, c, count, ws, cap, stream);
}

extern "C" int polymul(uint32_t p, const uint32_t *a, size_t la, const uint32_t *b, size_t lb, uint32_t *c,
                       cudaStream_t stream)
{
    return polymul_many(p, a, la, b, lb, c, 1, stream);
}
