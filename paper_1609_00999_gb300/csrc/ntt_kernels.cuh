// ntt_kernels.cuh -- device building blocks and launch helpers shared by the
// single-CTA (ntt.cu), large-N (ntt_large.cu) and batched (polymul_batch.cu)
// polynomial-multiplication kernels.
#pragma once
#include <cstdint>

#include "ntt_core.cuh"
#include "ntt_internal.cuh"

namespace mont {

// Threads per transform of 2^LOGN elements (16 elements per thread per array).
template <int LOGN>
constexpr int nt_of()
{
    return LOGN <= 4 ? 1 : (1 << (LOGN - 4));
}

// Transforms per CTA for the single-CTA kernels (256-thread CTAs below 2^12).
template <int LOGN>
constexpr int teams_of()
{
    return nt_of<LOGN>() >= 256 ? 1 : 256 / nt_of<LOGN>();
}

struct PolyArgs {
    const uint32_t *a, *b;
    uint32_t *c;
    size_t la, lb, lc, count;
    const uint2 *tw, *itw;
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

// One product (or one row block of a product) by one team of nt_of<LOGN>()
// threads with 2 * 2^LOGN words of shared memory at sm:
// c[0 .. lc) = inverse( forward(a) * forward(b * scale) ), where the
// sub-transform is block b_idx of the levels s_base .. s_base + LOGN - 1 of
// the whole transform (s_base = 0, b_idx = 0 for a complete product).
// Reads of a and b (lengths la, lb, zero beyond) all happen before the first
// barrier, so gc may alias ga (in-place row passes).  Every thread of the CTA
// must call it (it contains __syncthreads).
template <int LOGN, bool BASE0, bool SCALE_B>
__device__ __forceinline__ void polymul_team(uint32_t *sm, int tid, const uint32_t *ga, size_t la,
                                             const uint32_t *gb, size_t lb, uint32_t *gc, size_t lc,
                                             const uint2 *__restrict__ tw, const uint2 *__restrict__ itw, int s_base,
                                             int b_idx, uint32_t p, uint32_t pp, uint32_t k_scale)
{
    constexpr int N = 1 << LOGN, NT = nt_of<LOGN>(), NP = Sched<LOGN>::kPasses;
    if constexpr (LOGN == 0) {
        if (lc > 0) {
            const uint32_t bb = SCALE_B ? mont_mul(gb[0], k_scale, p, pp) : gb[0];
            gc[0] = mont_mul(ga[0], bb, p, pp);
        }
    } else {
        const SwzLayout lay[2] = {{sm}, {sm + N}};
        using P0 = PassGeom<LOGN, NT, 0>;
#pragma unroll
        for (int r = 0; r < P0::GPT; r++) {
            const int base = P0::base(tid, r);
            uint32_t x[2][P0::G];
#pragma unroll
            for (int t = 0; t < P0::G; t++) {
                const size_t j = static_cast<size_t>(base + t * P0::HMIN);
                x[0][t] = j < la ? __ldg(ga + j) : 0u;
                const uint32_t bj = j < lb ? __ldg(gb + j) : 0u;
                x[1][t] = SCALE_B ? mont_mul(bj, k_scale, p, pp) : bj;
            }
            ct_group<P0::E, 2, BASE0>(x, tw, s_base, b_idx, p);
            if constexpr (NP == 1) {
                uint32_t y[1][P0::G];
#pragma unroll
                for (int t = 0; t < P0::G; t++) y[0][t] = mont_mul(x[0][t], x[1][t], p, pp);
                gs_group<P0::E, 1, BASE0>(y, itw, s_base, b_idx, p);
#pragma unroll
                for (int t = 0; t < P0::G; t++) {
                    const size_t j = static_cast<size_t>(base + t * P0::HMIN);
                    if (j < lc) gc[j] = y[0][t];
                }
            } else {
#pragma unroll
                for (int t = 0; t < P0::G; t++) {
                    lay[0][base + t * P0::HMIN] = x[0][t];
                    lay[1][base + t * P0::HMIN] = x[1][t];
                }
            }
        }
        if constexpr (NP > 1) {
            __syncthreads();
            fwd_passes<LOGN, NT, 2, BASE0, 1, NP - 2>(lay, tid, tw, s_base, b_idx, p);
            fused_middle_pass<LOGN, NT, BASE0>(lay, tid, tw, itw, s_base, b_idx, p, pp);
            __syncthreads();
            inv_passes<LOGN, NT, BASE0, NP - 2, 1>(lay[0], tid, itw, s_base, b_idx, p);
#pragma unroll
            for (int r = 0; r < P0::GPT; r++) {
                const int base = P0::base(tid, r);
                uint32_t y[1][P0::G];
#pragma unroll
                for (int t = 0; t < P0::G; t++) y[0][t] = lay[0][base + t * P0::HMIN];
                gs_group<P0::E, 1, BASE0>(y, itw, s_base, b_idx, p);
#pragma unroll
                for (int t = 0; t < P0::G; t++) {
                    const size_t j = static_cast<size_t>(base + t * P0::HMIN);
                    if (j < lc) gc[j] = y[0][t];
                }
            }
        }
    }
}

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
