// ntt_kernels.cuh -- device building blocks and launch helpers shared by the
// single-CTA (ntt.cu), large-N (ntt_large.cu) and batched (polymul_batch.cu)
// polynomial-multiplication kernels.
#pragma once
#include <cstdint>

#include "ntt_core.cuh"
#include "ntt_internal.cuh"

namespace mont {

// Threads per transform of 2^LOGN elements: 16 elements per thread per
// array, except 2^13 on 256 threads and 2^14 on 512 (32 per thread, a
// radix-32 first pass): 2^13 then fits three CTAs and 24 warps per SM where
// 512 threads fit one, and 2^14 (one CTA per SM by its 132 KB of shared
// memory either way) gets up to 128 registers per thread.
template <int LOGN>
constexpr int nt_of()
{
    return LOGN <= 4 ? 1 : (LOGN == 13 ? 256 : (LOGN == 14 ? 512 : (1 << (LOGN - 4))));
}

// Transforms per CTA for the single-CTA kernels (256-thread CTAs below 2^12).
template <int LOGN>
constexpr int teams_of()
{
    return nt_of<LOGN>() >= 256 ? 1 : 256 / nt_of<LOGN>();
}

// CTAs per SM the register budget is sized for: four 256-thread CTAs
// (64 registers per thread, no spills) for the fused products up to 2^12,
// three for 2^13 (their 66 KB of shared memory fits three); one CTA for the
// 512-thread 2^14 transforms.
template <int LOGN>
constexpr int min_ctas_of()
{
    return teams_of<LOGN>() * nt_of<LOGN>() <= 256 ? (LOGN >= 13 ? 3 : 4) : 1;
}

// Shared-memory words one team needs for a product of 2^LOGN (both operands,
// padded layout).
template <int LOGN>
constexpr int team_smem_words()
{
    return 2 * PadLayout::words(1 << LOGN);
}

// 4-byte asynchronous copy global -> shared (cp.async, no register
// staging): a thread can have all of its tile's loads in flight at once.
// src_bytes = 0 writes zero and reads nothing (src must still be a valid
// address).  Completion: cp_async_wait_all, then a barrier for other threads.
__device__ __forceinline__ void cp_async4(uint32_t *dst_smem, const uint32_t *src, uint32_t src_bytes)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst_smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

struct PolyArgs {
    const uint32_t *a, *b;
    uint32_t *c;
    size_t la, lb, lc, count;
    const uint32_t *tw, *itw;
    uint32_t p, pp, k_scale;
};

// Dynamic shared memory above 48 KB must be opted into per kernel.
template <typename K>
int ensure_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return MONT_OK;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes)) ==
                   cudaSuccess
               ? MONT_OK
               : MONT_ECUDA;
}

// Operand loads of a product: the read-only path for a product's own inputs,
// a coherent load for rows of scratch written earlier in the same kernel.
template <bool READ_ONLY>
__device__ __forceinline__ uint32_t load_operand(const uint32_t *p)
{
    if constexpr (READ_ONLY) return __ldg(p);
    else return *p;
}

// Copies the N words of g into a shared-memory layout, word k to position
// at(k), k = tid + i NT.  Every load of the thread is issued before its first
// store, so each thread has N / NT loads in flight (a loop that stores each
// word as it arrives waits out one memory latency per word).  Zeros when
// !valid.
template <int N, int NT, class L, class AT>
__device__ __forceinline__ void stage_in(const L &lay, const uint32_t *g, int tid, bool valid, AT at)
{
    static_assert(N % NT == 0, "the thread count divides the transform");
    constexpr int PER = N / NT;
    uint32_t v[PER];
#pragma unroll
    for (int i = 0; i < PER; i++) v[i] = valid ? g[tid + i * NT] : 0u;
#pragma unroll
    for (int i = 0; i < PER; i++) lay[at(tid + i * NT)] = v[i];
}

// Operand source of a product: element j (< 2^LOGN) of operand 0 (a) or 1
// (b), zero at and beyond the operand's length, b multiplied by k_scale
// through the reduction (b N^-1 R^2 R^-1 = b N^-1 R).
template <bool READ_ONLY, bool SCALE_B, class RED>
struct PlainLoad {
    const uint32_t *a, *b;
    int la, lb;
    uint32_t k_scale;
    Mod m;
    __device__ __forceinline__ uint32_t operator()(int arr, int j) const
    {
        const uint32_t *g = arr ? b : a;
        if (j >= (arr ? lb : la)) return 0u;   // zero padding: no load, no scaling
        const uint32_t v = load_operand<READ_ONLY>(g + j);
        return (SCALE_B && arr) ? RED::mul(v, k_scale, m) : v;
    }
};

// One product (or one row block of a product) by one team of NT threads
// (nt_of<LOGN>() by default, fewer when each thread takes several groups per
// pass) with team_smem_words<LOGN>() words of shared memory at sm:
// c[0 .. lc) = inverse( forward(A) * forward(B) ), A and B element j being
// ld(0, j) and ld(1, j), where the sub-transform is block b_idx of the
// levels s_base .. s_base + LOGN - 1 of the whole transform (s_base = 0,
// b_idx = 0 for a complete product; BASE0 then also means ld returns reduced
// values, otherwise values below 2P are allowed).  All operand reads happen
// before the first barrier, so gc may alias the operands (in-place row
// passes).  Every thread of the CTA must call it (it contains
// __syncthreads).  lc <= 2^LOGN.
template <int LOGN, bool BASE0, int NT, class RED, class LD>
__device__ __forceinline__ void polymul_team_ld(uint32_t *sm, int tid, const LD &ld, uint32_t *gc, size_t lc,
                                                const uint32_t *__restrict__ tw, const uint32_t *__restrict__ itw,
                                                int s_base, int b_idx, Mod md)
{
    constexpr int N = 1 << LOGN, NP = SchedFor<LOGN, NT>::kPasses;
    const uint32_t p = md.p;
    if constexpr (LOGN == 0) {
        if (lc > 0) gc[0] = RED::mul(ld(0, 0), ld(1, 0), md);
    } else {
        const PadLayout lay[2] = {{sm}, {sm + PadLayout::words(N)}};
        using P0 = PassGeom<LOGN, NT, 0>;
        const int lc32 = static_cast<int>(lc);
        if constexpr (NP == 1) {
#pragma unroll
            for (int r = 0; r < P0::GPT; r++) {
                const int base = P0::base(tid, r);
                uint32_t x[2][P0::G];
#pragma unroll
                for (int t = 0; t < P0::G; t++) {
                    const int j = base + t * P0::HMIN;
                    x[0][t] = ld(0, j);
                    x[1][t] = ld(1, j);
                }
                ct_group<P0::E, 2, BASE0, RED>(x, tw, s_base, b_idx, md);
                uint32_t y[1][P0::G];
#pragma unroll
                for (int t = 0; t < P0::G; t++) y[0][t] = RED::mul(csub(x[0][t], p), x[1][t], md);
                gs_group<P0::E, 1, BASE0, RED>(y, itw, s_base, b_idx, md);
#pragma unroll
                for (int t = 0; t < P0::G; t++) {
                    const int j = base + t * P0::HMIN;
                    if (j < lc32) gc[j] = y[0][t];
                }
            }
        } else {
#pragma unroll
            for (int a = 0; a < 2; a++) {
#pragma unroll
                for (int r = 0; r < P0::GPT; r++) {
                    const int base = P0::base(tid, r);
                    uint32_t x[1][P0::G];
#pragma unroll
                    for (int t = 0; t < P0::G; t++) x[0][t] = ld(a, base + t * P0::HMIN);
                    ct_group<P0::E, 1, BASE0, RED>(x, tw, s_base, b_idx, md);
#pragma unroll
                    for (int t = 0; t < P0::G; t++) elem(lay[a], base, t * P0::HMIN) = x[0][t];
                }
            }
        }
        if constexpr (NP > 1) {
            __syncthreads();
            fwd_passes<LOGN, NT, 2, BASE0, 1, NP - 2, RED>(lay, tid, tw, s_base, b_idx, md);
            fused_middle_pass<LOGN, NT, BASE0, RED>(lay, tid, tw, itw, s_base, b_idx, md);
            __syncthreads();
            inv_passes<LOGN, NT, BASE0, NP - 2, 1, RED>(lay[0], tid, itw, s_base, b_idx, md);
#pragma unroll
            for (int r = 0; r < P0::GPT; r++) {
                const int base = P0::base(tid, r);
                uint32_t y[1][P0::G];
#pragma unroll
                for (int t = 0; t < P0::G; t++) y[0][t] = elem(lay[0], base, t * P0::HMIN);
                gs_group<P0::E, 1, BASE0, RED>(y, itw, s_base, b_idx, md);
#pragma unroll
                for (int t = 0; t < P0::G; t++) {
                    const int j = base + t * P0::HMIN;
                    if (j < lc32) gc[j] = y[0][t];
                }
            }
        }
    }
}

// polymul_team_ld on operand arrays a (length la) and b (length lb): the
// product's own inputs (read-only path) when BASE0, scratch rows (coherent
// loads) otherwise; b multiplied by k_scale on load when SCALE_B.
template <int LOGN, bool BASE0, bool SCALE_B, int NT = nt_of<LOGN>(), class RED = RedAlg2>
__device__ __forceinline__ void polymul_team(uint32_t *sm, int tid, const uint32_t *ga, size_t la,
                                             const uint32_t *gb, size_t lb, uint32_t *gc, size_t lc,
                                             const uint32_t *__restrict__ tw, const uint32_t *__restrict__ itw, int s_base,
                                             int b_idx, uint32_t p, uint32_t pp, uint32_t k_scale)
{
    const Mod md{p, pp};
    const PlainLoad<BASE0, SCALE_B, RED> ld{ga, gb, static_cast<int>(la), static_cast<int>(lb), k_scale, md};
    polymul_team_ld<LOGN, BASE0, NT, RED>(sm, tid, ld, gc, lc, tw, itw, s_base, b_idx, md);
}

namespace {

// Fused products of N = 2^LOGN <= 2^14: teams_of<LOGN>() products per CTA,
// one per team, A.count products of [la] x [lb] -> [lc] laid out row-major.
template <int LOGN, class RED>
__global__ void __launch_bounds__(teams_of<LOGN>() * nt_of<LOGN>(), min_ctas_of<LOGN>())
k_polymul(PolyArgs A)
{
    constexpr int NT = nt_of<LOGN>();
    extern __shared__ __align__(16) uint32_t smem[];
    const int team = threadIdx.x / NT, tid = threadIdx.x - team * NT;
    const size_t prod = static_cast<size_t>(blockIdx.x) * teams_of<LOGN>() + team;
    const bool valid = prod < A.count;
    const uint32_t *ga = A.a + (valid ? prod * A.la : 0);
    const uint32_t *gb = A.b + (valid ? prod * A.lb : 0);
    uint32_t *gc = A.c + (valid ? prod * A.lc : 0);
    uint32_t *sm = smem + static_cast<size_t>(team) * team_smem_words<LOGN>();
    polymul_team<LOGN, true, true, NT, RED>(sm, tid, ga, valid ? A.la : 0, gb, valid ? A.lb : 0, gc,
                                            valid ? A.lc : 0, A.tw, A.itw, 0, 0, A.p, A.pp, A.k_scale);
}

template <int LOGN, class RED>
int launch_polymul_smem(const PolyArgs &A, cudaStream_t s)
{
    constexpr int T = teams_of<LOGN>(), NT = nt_of<LOGN>();
    const size_t smem = static_cast<size_t>(T) * team_smem_words<LOGN>() * sizeof(uint32_t);
    if (ensure_smem(k_polymul<LOGN, RED>, smem) != MONT_OK) return MONT_ECUDA;
    const size_t grid = (A.count + T - 1) / T;
    if (grid > 0x7FFFFFFFu) return MONT_ERANGE;
    k_polymul<LOGN, RED><<<static_cast<unsigned>(grid), T * NT, smem, s>>>(A);
    return launch_status();
}

}  // namespace

int ceil_log2(size_t n);
int dispatch_polymul_smem(int log2n, const PolyArgs &A, cudaStream_t s);
int polymul_prepare(uint32_t p, const uint32_t *a, size_t la, const uint32_t *b, size_t lb, const uint32_t *c,
                    size_t count, ntt_plan *plan, int *log2n);
// N > 2^14: column / row / column kernels through ws (2N words per product).
int polymul_large(const ntt_plan &plan, const uint32_t *a, size_t la, const uint32_t *b, size_t lb, uint32_t *c,
                  size_t count, uint32_t *ws, cudaStream_t s);
// Standalone transforms for N > 2^14, in place.
int ntt_large(const ntt_plan *plan, uint32_t *data, size_t batch, int flags, bool inverse, cudaStream_t s);
// Library-owned scratch for (current device, stream), grown on demand.
int stream_workspace(cudaStream_t s, size_t bytes, void **out);

}  // namespace mont
