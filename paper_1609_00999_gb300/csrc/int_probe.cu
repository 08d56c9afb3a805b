// int_probe.cu -- throughput probes of the integer pipes: the measured
// ceiling for the arithmetic of the transforms.
//
// Every probe thread keeps kChains independent register chains and applies
// one operation to each of them kUnroll x `iterations` times, with no memory
// traffic: a single instruction form (32-bit multiply-add, high-word
// multiply-add, 32x32->64 multiply-add, three-input add), a full REDC
// (Alg. 2, the library's mont_mul), or one of the NTT butterflies exactly as
// the transform kernels inline them (ntt_core.cuh).  Chains that would fold
// under algebraic simplification (repeated adds, repeated butterflies with
// twiddle 1 on unreduced values) take an operand from the neighbouring
// chain, and the level-0 butterfly (adds only) passes its results through an
// empty asm, so each step stays one operation.
//
// The benchmark times each probe with CUDA events; operations per second
// over the whole GPU are the ceiling the roofline of the transform and
// product kernels divides by, weighted by how many of each operation a
// product performs.
#include <algorithm>

#include "common.cuh"
#include "ntt_core.cuh"

namespace mont {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

struct ProbeArgs {
    uint32_t p, pp, d;
    uint32_t iters;
    uint32_t *sink;
};

template <int KIND>
__device__ __forceinline__ void probe_step(uint32_t (&x)[kChains], uint32_t (&y)[kChains],
                                           const uint32_t (&w)[kChains], const ProbeArgs &A)
{
    const Mod m{A.p, A.pp};
#pragma unroll
    for (int i = 0; i < kChains; i++) {
        const int j = (i + 1) % kChains;
        if constexpr (KIND == MONT_PROBE_IMAD) {
            asm("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[i]) : "r"(x[j]), "r"(A.d));
        } else if constexpr (KIND == MONT_PROBE_IMAD_HI) {
            asm("mad.hi.u32 %0, %0, %1, %2;" : "+r"(x[i]) : "r"(x[j]), "r"(A.d));
        } else if constexpr (KIND == MONT_PROBE_IMAD_WIDE) {
            // (y, x) <- x * w + (y, x) as one 64-bit multiply-add
            asm("{\n\t.reg .u64 t;\n\tmov.b64 t, {%0, %1};\n\tmad.wide.u32 t, %0, %2, t;\n\tmov.b64 {%0, %1}, t;\n\t}"
                : "+r"(x[i]), "+r"(y[i])
                : "r"(w[i]));
        } else if constexpr (KIND == MONT_PROBE_IADD3) {
            asm("add.u32 %0, %0, %1;\n\tadd.u32 %0, %0, %2;" : "+r"(x[i]) : "r"(x[j]), "r"(A.d));
        } else if constexpr (KIND == MONT_PROBE_REDC) {
            x[i] = mont_mul(x[i], w[i], m.p, m.pp);
        } else if constexpr (KIND == MONT_PROBE_CT) {
            bfly_ct<RedAlg2>(x[i], y[i], w[i], m);
        } else if constexpr (KIND == MONT_PROBE_CT_ONE) {
            bfly_ct_one(x[i], y[j], m);
        } else if constexpr (KIND == MONT_PROBE_CT_FIRST) {
            // Two adds with no reduction: repeated steps are linear in the
            // starting values, so an empty asm hides each result from the
            // compiler's algebra (no instruction is emitted for it).
            bfly_ct_first(x[i], y[j], m);
            asm("" : "+r"(x[i]), "+r"(y[j]));
        } else if constexpr (KIND == MONT_PROBE_GS) {
            bfly_gs<RedAlg2>(x[i], y[i], w[i], m);
        } else if constexpr (KIND == MONT_PROBE_GS_ONE) {
            bfly_gs_one(x[i], y[j], m);
        }
    }
}

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_int_probe(ProbeArgs A)
{
    // Starting values below 2^28 < P for every supported prime, so the
    // butterflies and REDC see operands in their valid ranges.
    const uint32_t t = blockIdx.x * kProbeThreads + threadIdx.x;
    uint32_t x[kChains], y[kChains], w[kChains];
#pragma unroll
    for (int i = 0; i < kChains; i++) {
        x[i] = (t * 2654435761u + 97u * i) & 0x0FFFFFFFu;
        y[i] = (t * 40503u + 131u * i + 7u) & 0x0FFFFFFFu;
        w[i] = (A.d * (i + 3u)) & 0x0FFFFFFFu;
    }
#pragma unroll 1
    for (uint32_t it = 0; it < A.iters; it++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) probe_step<KIND>(x, y, w, A);
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < kChains; i++) acc ^= x[i] ^ y[i];
    // Data-dependent store, so the chains are live; almost never taken.
    if (acc == A.p) A.sink[0] = acc;
}

template <int KIND>
int launch_probe(const ProbeArgs &A, unsigned ctas_per_sm, unsigned *grid, cudaStream_t s)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_int_probe<KIND>, kProbeThreads, 0) != cudaSuccess ||
        occ <= 0) {
        cudaGetLastError();
        return MONT_ECUDA;
    }
    const unsigned per = ctas_per_sm == 0 ? static_cast<unsigned>(occ)
                                          : std::min(ctas_per_sm, static_cast<unsigned>(occ));
    const int sms = device_sm_count();
    if (sms <= 0) return MONT_ECUDA;
    *grid = per * static_cast<unsigned>(sms);
    k_int_probe<KIND><<<*grid, kProbeThreads, 0, s>>>(A);
    return launch_status();
}

}  // namespace
}  // namespace mont

extern "C" int mont_int_probe(int kind, uint32_t p, uint32_t iterations, uint32_t ctas_per_sm, uint32_t *sink,
                              uint64_t *ops_per_launch, cudaStream_t stream)
{
    using namespace mont;
    if (!sink || iterations == 0 || p < 3u || !(p & 1u) || p >= 0x80000000u) return MONT_EINVAL;
    ProbeArgs A;
    A.p = p;
    A.pp = host_neg_inv32(p);
    A.d = 0x9E3779B9u % p;
    A.iters = iterations;
    A.sink = sink;
    unsigned grid = 0;
    int rc;
    switch (kind) {
    case MONT_PROBE_IMAD: rc = launch_probe<MONT_PROBE_IMAD>(A, ctas_per_sm, &grid, stream); break;
    case MONT_PROBE_IMAD_HI: rc = launch_probe<MONT_PROBE_IMAD_HI>(A, ctas_per_sm, &grid, stream); break;
    case MONT_PROBE_IMAD_WIDE: rc = launch_probe<MONT_PROBE_IMAD_WIDE>(A, ctas_per_sm, &grid, stream); break;
    case MONT_PROBE_IADD3: rc = launch_probe<MONT_PROBE_IADD3>(A, ctas_per_sm, &grid, stream); break;
    case MONT_PROBE_REDC: rc = launch_probe<MONT_PROBE_REDC>(A, ctas_per_sm, &grid, stream); break;
    case MONT_PROBE_CT: rc = launch_probe<MONT_PROBE_CT>(A, ctas_per_sm, &grid, stream); break;
    case MONT_PROBE_CT_ONE: rc = launch_probe<MONT_PROBE_CT_ONE>(A, ctas_per_sm, &grid, stream); break;
    case MONT_PROBE_CT_FIRST: rc = launch_probe<MONT_PROBE_CT_FIRST>(A, ctas_per_sm, &grid, stream); break;
    case MONT_PROBE_GS: rc = launch_probe<MONT_PROBE_GS>(A, ctas_per_sm, &grid, stream); break;
    case MONT_PROBE_GS_ONE: rc = launch_probe<MONT_PROBE_GS_ONE>(A, ctas_per_sm, &grid, stream); break;
    default: return MONT_EINVAL;
    }
    if (rc == MONT_OK && ops_per_launch)
        *ops_per_launch = static_cast<uint64_t>(grid) * kProbeThreads * iterations * kUnroll * kChains;
    return rc;
}
