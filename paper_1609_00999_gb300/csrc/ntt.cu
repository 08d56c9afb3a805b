// ntt.cu -- single-CTA NTT and fused polynomial-multiplication kernels (N <= 2^14)
// and the C-ABI entry points ntt_fwd, ntt_inv, polymul, polymul_many.
//
// Polymul of one product in one team of threads (c = a * b mod P,
// length la + lb - 1, cyclic convolution of size N = 2^K >= la + lb - 1):
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
#include <algorithm>

#include "ntt_core.cuh"
#include "ntt_internal.cuh"

namespace mont {
namespace {

template <int LOGN>
constexpr int nt_of()
{
    return LOGN <= 4 ? 1 : (1 << (LOGN - 4));
}

template <int LOGN>
constexpr int teams_of()
{
    return nt_of<LOGN>() >= 256 ? 1 : 256 / nt_of<LOGN>();
}

template <int LOGN>
__device__ __forceinline__ int brev(int k)
{
    if constexpr (LOGN == 0) return 0;
    else return static_cast<int>(__brev(static_cast<unsigned>(k)) >> (32 - LOGN));
}

// Forward pass I over NARR arrays held in smem (array a at sm + a * 2^LOGN).
template <int LOGN, int NT, int I, int NARR>
__device__ __forceinline__ void fwd_pass(uint32_t *sm, int tid, const uint2 *__restrict__ tw, uint32_t p)
{
    using PG = PassGeom<LOGN, NT, I>;
    constexpr int N = 1 << LOGN;
#pragma unroll
    for (int r = 0; r < PG::GPT; r++) {
        const int base = PG::base(tid, r);
        uint32_t x[NARR][PG::G];
#pragma unroll
        for (int a = 0; a < NARR; a++)
#pragma unroll
            for (int t = 0; t < PG::G; t++) x[a][t] = sm[a * N + swz(base + t * PG::HMIN)];
        ct_group<PG::E, NARR, PG::S0 == 0>(x, tw, PG::S0, PG::blk(tid, r), p);
#pragma unroll
        for (int a = 0; a < NARR; a++)
#pragma unroll
            for (int t = 0; t < PG::G; t++) sm[a * N + swz(base + t * PG::HMIN)] = x[a][t];
    }
}

template <int LOGN, int NT, int I>
__device__ __forceinline__ void inv_pass(uint32_t *sm, int tid, const uint2 *__restrict__ itw, uint32_t p)
{
    using PG = PassGeom<LOGN, NT, I>;
#pragma unroll
    for (int r = 0; r < PG::GPT; r++) {
        const int base = PG::base(tid, r);
        uint32_t x[1][PG::G];
#pragma unroll
        for (int t = 0; t < PG::G; t++) x[0][t] = sm[swz(base + t * PG::HMIN)];
        gs_group<PG::E, 1, PG::S0 == 0>(x, itw, PG::S0, PG::blk(tid, r), p);
#pragma unroll
        for (int t = 0; t < PG::G; t++) sm[swz(base + t * PG::HMIN)] = x[0][t];
    }
}

// Forward passes I .. LAST, each followed by a CTA barrier.
template <int LOGN, int NT, int NARR, int I, int LAST>
__device__ __forceinline__ void fwd_passes(uint32_t *sm, int tid, const uint2 *__restrict__ tw, uint32_t p)
{
    if constexpr (I <= LAST) {
        fwd_pass<LOGN, NT, I, NARR>(sm, tid, tw, p);
        __syncthreads();
        fwd_passes<LOGN, NT, NARR, I + 1, LAST>(sm, tid, tw, p);
    }
}

// Inverse passes I, I-1, .. FIRST, each followed by a CTA barrier.
template <int LOGN, int NT, int I, int FIRST>
__device__ __forceinline__ void inv_passes(uint32_t *sm, int tid, const uint2 *__restrict__ itw, uint32_t p)
{
    if constexpr (I >= FIRST) {
        inv_pass<LOGN, NT, I>(sm, tid, itw, p);
        __syncthreads();
        inv_passes<LOGN, NT, I - 1, FIRST>(sm, tid, itw, p);
    }
}

struct PolyArgs {
    const uint32_t *a, *b;
    uint32_t *c;
    size_t la, lb, lc, count;
    const uint2 *tw, *itw;
    uint32_t p, pp, k_scale;
};

// Pointwise product and the inverse levels of the last pass, on registers.
template <int G>
__device__ __forceinline__ void pointwise(uint32_t (&x)[2][G], uint32_t (&y)[1][G], uint32_t p, uint32_t pp)
{
#pragma unroll
    for (int t = 0; t < G; t++) y[0][t] = mont_mul(x[0][t], x[1][t], p, pp);
}

template <int LOGN>
__global__ void __launch_bounds__(teams_of<LOGN>() * nt_of<LOGN>())
k_polymul(PolyArgs A)
{
    constexpr int N = 1 << LOGN, NT = nt_of<LOGN>(), NP = Sched<LOGN>::kPasses;
    extern __shared__ __align__(16) uint32_t smem[];
    const int team = threadIdx.x / NT, tid = threadIdx.x - team * NT;
    const size_t prod = static_cast<size_t>(blockIdx.x) * teams_of<LOGN>() + team;
    const bool valid = prod < A.count;
    const uint32_t *ga = A.a + (valid ? prod * A.la : 0);
    const uint32_t *gb = A.b + (valid ? prod * A.lb : 0);
    uint32_t *gc = A.c + (valid ? prod * A.lc : 0);
    const int la = valid ? static_cast<int>(A.la) : 0;
    const int lb = valid ? static_cast<int>(A.lb) : 0;
    const int lc = valid ? static_cast<int>(A.lc) : 0;
    const uint32_t p = A.p, pp = A.pp;

    if constexpr (LOGN == 0) {
        if (valid) gc[0] = mont_mul(ga[0], mont_mul(gb[0], A.k_scale, p, pp), p, pp);
        return;
    } else {
        uint32_t *sm = smem + static_cast<size_t>(team) * 2 * N;
        using P0 = PassGeom<LOGN, NT, 0>;
#pragma unroll
        for (int r = 0; r < P0::GPT; r++) {
            const int base = P0::base(tid, r);
            uint32_t x[2][P0::G];
#pragma unroll
            for (int t = 0; t < P0::G; t++) {
                const int j = base + t * P0::HMIN;
                x[0][t] = j < la ? __ldg(ga + j) : 0u;
                x[1][t] = j < lb ? mont_mul(__ldg(gb + j), A.k_scale, p, pp) : 0u;
            }
            ct_group<P0::E, 2, true>(x, A.tw, 0, 0, p);
            if constexpr (NP == 1) {
                uint32_t y[1][P0::G];
                pointwise<P0::G>(x, y, p, pp);
                gs_group<P0::E, 1, true>(y, A.itw, 0, 0, p);
#pragma unroll
                for (int t = 0; t < P0::G; t++) {
                    const int j = base + t * P0::HMIN;
                    if (j < lc) gc[j] = y[0][t];
                }
            } else {
#pragma unroll
                for (int t = 0; t < P0::G; t++) {
                    sm[swz(base + t * P0::HMIN)] = x[0][t];
                    sm[N + swz(base + t * P0::HMIN)] = x[1][t];
                }
            }
        }
        if constexpr (NP > 1) {
            __syncthreads();
            fwd_passes<LOGN, NT, 2, 1, NP - 2>(sm, tid, A.tw, p);
            using PL = PassGeom<LOGN, NT, NP - 1>;
#pragma unroll
            for (int r = 0; r < PL::GPT; r++) {
                const int base = PL::base(tid, r), blk = PL::blk(tid, r);
                uint32_t x[2][PL::G];
#pragma unroll
                for (int t = 0; t < PL::G; t++) {
                    x[0][t] = sm[swz(base + t * PL::HMIN)];
                    x[1][t] = sm[N + swz(base + t * PL::HMIN)];
                }
                ct_group<PL::E, 2, false>(x, A.tw, PL::S0, blk, p);
                uint32_t y[1][PL::G];
                pointwise<PL::G>(x, y, p, pp);
                gs_group<PL::E, 1, false>(y, A.itw, PL::S0, blk, p);
#pragma unroll
                for (int t = 0; t < PL::G; t++) sm[swz(base + t * PL::HMIN)] = y[0][t];
            }
            __syncthreads();
            inv_passes<LOGN, NT, NP - 2, 1>(sm, tid, A.itw, p);
#pragma unroll
            for (int r = 0; r < P0::GPT; r++) {
                const int base = P0::base(tid, r);
                uint32_t y[1][P0::G];
#pragma unroll
                for (int t = 0; t < P0::G; t++) y[0][t] = sm[swz(base + t * P0::HMIN)];
                gs_group<P0::E, 1, true>(y, A.itw, 0, 0, p);
#pragma unroll
                for (int t = 0; t < P0::G; t++) {
                    const int j = base + t * P0::HMIN;
                    if (j < lc) gc[j] = y[0][t];
                }
            }
        }
    }
}

struct NttArgs {
    uint32_t *data;
    size_t batch;
    const uint2 *tw;
    uint32_t p, pp, ninv_mont;
    int bitrev;
};

// In-place forward NTT of [batch][N]; natural order in, natural (or, with
// bitrev, bit-reversed) order out.
template <int LOGN>
__global__ void __launch_bounds__(teams_of<LOGN>() * nt_of<LOGN>())
k_ntt_fwd(NttArgs A)
{
    constexpr int N = 1 << LOGN, NT = nt_of<LOGN>(), NP = Sched<LOGN>::kPasses;
    extern __shared__ __align__(16) uint32_t smem[];
    const int team = threadIdx.x / NT, tid = threadIdx.x - team * NT;
    const size_t prod = static_cast<size_t>(blockIdx.x) * teams_of<LOGN>() + team;
    const bool valid = prod < A.batch;
    uint32_t *g = A.data + (valid ? prod * N : 0);
    uint32_t *sm = smem + static_cast<size_t>(team) * N;
    for (int k = tid; k < N; k += NT) sm[swz(k)] = valid ? g[k] : 0u;
    __syncthreads();
    fwd_passes<LOGN, NT, 1, 0, NP - 1>(sm, tid, A.tw, A.p);
    if (valid)
        for (int k = tid; k < N; k += NT) g[k] = sm[swz(A.bitrev ? k : brev<LOGN>(k))];
}

// In-place inverse NTT (with the factor N^-1) of [batch][N]; natural (or,
// with bitrev, bit-reversed) order in, natural order out.
template <int LOGN>
__global__ void __launch_bounds__(teams_of<LOGN>() * nt_of<LOGN>())
k_ntt_inv(NttArgs A)
{
    constexpr int N = 1 << LOGN, NT = nt_of<LOGN>(), NP = Sched<LOGN>::kPasses;
    extern __shared__ __align__(16) uint32_t smem[];
    const int team = threadIdx.x / NT, tid = threadIdx.x - team * NT;
    const size_t prod = static_cast<size_t>(blockIdx.x) * teams_of<LOGN>() + team;
    const bool valid = prod < A.batch;
    uint32_t *g = A.data + (valid ? prod * N : 0);
    uint32_t *sm = smem + static_cast<size_t>(team) * N;
    for (int k = tid; k < N; k += NT) sm[swz(A.bitrev ? k : brev<LOGN>(k))] = valid ? g[k] : 0u;
    __syncthreads();
    inv_passes<LOGN, NT, NP - 1, 0>(sm, tid, A.tw, A.p);
    if (valid)
        for (int k = tid; k < N; k += NT) g[k] = mont_mul(sm[swz(k)], A.ninv_mont, A.p, A.pp);
}

// Dynamic shared memory above 48 KB must be opted into per kernel and device.
template <typename K>
int ensure_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return MONT_OK;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes)) ==
                   cudaSuccess
               ? MONT_OK
               : MONT_ECUDA;
}

template <int LOGN>
int launch_polymul_smem(const PolyArgs &A, cudaStream_t s)
{
    constexpr int T = teams_of<LOGN>(), NT = nt_of<LOGN>();
    const size_t smem = static_cast<size_t>(T) * 2 * (size_t{1} << LOGN) * sizeof(uint32_t);
    if (ensure_smem(k_polymul<LOGN>, smem) != MONT_OK) return MONT_ECUDA;
    const size_t grid = (A.count + T - 1) / T;
    if (grid > 0x7FFFFFFFu) return MONT_ERANGE;
    k_polymul<LOGN><<<static_cast<unsigned>(grid), T * NT, smem, s>>>(A);
    return launch_status();
}

template <int LOGN>
int launch_ntt_smem(const NttArgs &A, bool inverse, cudaStream_t s)
{
    constexpr int T = teams_of<LOGN>(), NT = nt_of<LOGN>();
    const size_t smem = static_cast<size_t>(T) * (size_t{1} << LOGN) * sizeof(uint32_t);
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

int dispatch_polymul_smem(int log2n, const PolyArgs &A, cudaStream_t s)
{
    switch (log2n) {
#define X(L) \
    case L: return launch_polymul_smem<L>(A, s);
        MONT_LOGN_CASES(X)
#undef X
    default: return MONT_EUNSUPPORTED;
    }
}

int dispatch_ntt_smem(int log2n, const NttArgs &A, bool inverse, cudaStream_t s)
{
    switch (log2n) {
#define X(L) \
    case L: return launch_ntt_smem<L>(A, inverse, s);
        MONT_LOGN_CASES(X)
#undef X
    default: return MONT_EUNSUPPORTED;
    }
}

int ceil_log2(size_t n)
{
    int k = 0;
    while ((size_t{1} << k) < n) k++;
    return k;
}

int ntt_common(const ntt_plan *plan, uint32_t *data, size_t batch, int flags, bool inverse, cudaStream_t s)
{
    if (!plan || (flags & ~NTT_BITREV)) return MONT_EINVAL;
    if (batch == 0) return MONT_OK;
    if (!data) return MONT_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return MONT_ECUDA;
    if (dev != plan->device) return MONT_EINVAL;
    if (plan->log2n > kMaxSmemLog2N) return MONT_EUNSUPPORTED;
    NttArgs A;
    A.data = data;
    A.batch = batch;
    A.tw = inverse ? plan->table->inv : plan->table->fwd;
    A.p = plan->p;
    A.pp = plan->p_prime;
    A.ninv_mont = plan->ninv_mont;
    A.bitrev = (flags & NTT_BITREV) ? 1 : 0;
    return dispatch_ntt_smem(plan->log2n, A, inverse, s);
}

}  // namespace
}  // namespace mont

extern "C" int ntt_fwd(const ntt_plan *plan, uint32_t *data, size_t batch, int flags, cudaStream_t stream)
{
    return mont::ntt_common(plan, data, batch, flags, false, stream);
}

extern "C" int ntt_inv(const ntt_plan *plan, uint32_t *data, size_t batch, int flags, cudaStream_t stream)
{
    return mont::ntt_common(plan, data, batch, flags, true, stream);
}

extern "C" int polymul_many(uint32_t p, const uint32_t *a, size_t la, const uint32_t *b, size_t lb, uint32_t *c,
                            size_t count, cudaStream_t stream)
{
    if (count == 0) return MONT_OK;
    if (!a || !b || !c || la == 0 || lb == 0) return MONT_EINVAL;
    if (la > (size_t{1} << 30) || lb > (size_t{1} << 30)) return MONT_ERANGE;
    const size_t lc = la + lb - 1;
    if (count > SIZE_MAX / 4 / (lc + la + lb)) return MONT_ERANGE;
    const size_t wa = count * la * 4, wb = count * lb * 4, wc = count * lc * 4;
    if (mont::any_overlap(c, wc, a, wa) || mont::any_overlap(c, wc, b, wb)) return MONT_EINVAL;
    const int log2n = mont::ceil_log2(lc);
    if (log2n > mont::kMaxSmemLog2N) return MONT_EUNSUPPORTED;
    ntt_plan plan;
    int rc = mont::make_plan(p, log2n, &plan);
    if (rc != MONT_OK) return rc;
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

extern "C" int polymul(uint32_t p, const uint32_t *a, size_t la, const uint32_t *b, size_t lb, uint32_t *c,
                       cudaStream_t stream)
{
    return polymul_many(p, a, la, b, lb, c, 1, stream);
}
