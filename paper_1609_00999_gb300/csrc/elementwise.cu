// elementwise.cu -- to_mont / from_mont / mont_mul / mont_fma over vectors, and
// the two other reductions of Sec. 3.1 (Barrett, Alg. 1; Montgomery over
// Fourier primes, Alg. 3) as elementwise kernels.
//
// The data-parallel REDC of Sec. 3.2 on sm_103a: each thread is a lane, each
// thread moves 128-bit (uint4) vectors with coalesced loads, and a grid-stride
// loop over a grid sized to fill every SM covers the vector.  The work is
// HBM-bound (12 B per mont_mul element, 16 B per mont_fma element), so the
// kernel's job is to keep enough loads in flight: each thread issues ILP
// independent uint4 loads per operand before using any of them.
#include "common.cuh"
#include "mont_arith.cuh"

namespace mont {
namespace {

enum Op { OP_SCALE = 0, OP_MUL = 1, OP_FMA = 2, OP_BARRETT = 3, OP_FOURIER = 4 };

// Per-launch constants: the modulus, P', and for OP_SCALE the multiplier k;
// for OP_BARRETT k = ceil(log2 P) and aux = floor(2^(2k) / P); for OP_FOURIER
// aux = c 2^n = P - 1.
struct EwParams {
    uint32_t p, pp, k, aux;
};

// Alg. 1 (Barrett): m = floor(ab / 2^k), q = floor(m P' / 2^k), t = ab - qP,
// then subtract P while t >= P (at most three times, t < 4P).  64-bit
// intermediates: ab < 2^62, m P' < 2^63, t < 4P < 2^33.
__device__ __forceinline__ uint32_t barrett(uint32_t a, uint32_t b, uint32_t p, uint32_t k, uint32_t pb)
{
    const uint64_t T = static_cast<uint64_t>(a) * b;
    const uint64_t m = T >> k;
    const uint64_t q = (m * pb) >> k;
    uint64_t t = T - q * p;
#pragma unroll
    for (int i = 0; i < 3; i++) t = t >= p ? t - p : t;
    return static_cast<uint32_t>(t);
}

constexpr int kThreads = 256;
constexpr int kIlp = 2;

template <int OP>
__device__ __forceinline__ uint32_t apply(uint32_t a, uint32_t b, uint32_t c, const EwParams &q)
{
    // OP_SCALE: b is the launch-wide constant k (R^2 mod P for to_mont, 1 for from_mont).
    if constexpr (OP == OP_BARRETT) return barrett(a, b, q.p, q.k, q.aux);
    if constexpr (OP == OP_FOURIER) return fourier_redc(a, b, q.p, q.aux);
    const uint32_t t = mont_mul(a, b, q.p, q.pp);
    if constexpr (OP == OP_FMA) return add_mod(t, c, q.p);
    return t;
}

template <int OP>
__device__ __forceinline__ uint4 apply4(uint4 a, uint4 b, uint4 c, const EwParams &q)
{
    uint4 r;
    r.x = apply<OP>(a.x, b.x, c.x, q);
    r.y = apply<OP>(a.y, b.y, c.y, q);
    r.z = apply<OP>(a.z, b.z, c.z, q);
    r.w = apply<OP>(a.w, b.w, c.w, q);
    return r;
}

// Vector body over n4 uint4 chunks plus a scalar tail of `tail` elements
// starting at element 4 * n4.  For OP_SCALE, b is unused and k is the multiplier.
// out may equal a, b or c (in place), so no pointer is __restrict__: each
// element is read by the thread that writes it, before it writes it.
template <int OP>
__global__ void __launch_bounds__(kThreads)
k_elementwise(const uint32_t *a, const uint32_t *b, const uint32_t *c, uint32_t *out, size_t n4, uint32_t tail,
              EwParams q)
{
    const uint4 *a4 = reinterpret_cast<const uint4 *>(a);
    const uint4 *b4 = reinterpret_cast<const uint4 *>(b);
    const uint4 *c4 = reinterpret_cast<const uint4 *>(c);
    uint4 *o4 = reinterpret_cast<uint4 *>(out);
    const uint32_t k = q.k;
    const uint4 kk = make_uint4(k, k, k, k);
    const uint4 zero = make_uint4(0, 0, 0, 0);
    const size_t stride = static_cast<size_t>(gridDim.x) * kThreads;
    size_t i = static_cast<size_t>(blockIdx.x) * kThreads + threadIdx.x;

    for (; i + (kIlp - 1) * stride < n4; i += kIlp * stride) {
        uint4 va[kIlp], vb[kIlp], vc[kIlp];
#pragma unroll
        for (int u = 0; u < kIlp; u++) {
            va[u] = __ldcs(a4 + i + u * stride);
            vb[u] = OP == OP_SCALE ? kk : __ldcs(b4 + i + u * stride);
            vc[u] = OP == OP_FMA ? __ldcs(c4 + i + u * stride) : zero;
        }
#pragma unroll
        for (int u = 0; u < kIlp; u++) __stcs(o4 + i + u * stride, apply4<OP>(va[u], vb[u], vc[u], q));
    }
    for (; i < n4; i += stride) {
        const uint4 va = __ldcs(a4 + i);
        const uint4 vb = OP == OP_SCALE ? kk : __ldcs(b4 + i);
        const uint4 vc = OP == OP_FMA ? __ldcs(c4 + i) : zero;
        __stcs(o4 + i, apply4<OP>(va, vb, vc, q));
    }
    if (blockIdx.x == 0 && threadIdx.x < tail) {
        const size_t j = 4 * n4 + threadIdx.x;
        const uint32_t vb = OP == OP_SCALE ? k : b[j];
        const uint32_t vc = OP == OP_FMA ? c[j] : 0u;
        out[j] = apply<OP>(a[j], vb, vc, q);
    }
}

// Scalar grid-stride variant for operands that are not all 16-byte aligned.
template <int OP>
__global__ void __launch_bounds__(kThreads)
k_elementwise_scalar(const uint32_t *a, const uint32_t *b, const uint32_t *c, uint32_t *out, size_t n, EwParams q)
{
    const size_t stride = static_cast<size_t>(gridDim.x) * kThreads;
    for (size_t i = static_cast<size_t>(blockIdx.x) * kThreads + threadIdx.x; i < n; i += stride) {
        const uint32_t vb = OP == OP_SCALE ? q.k : b[i];
        const uint32_t vc = OP == OP_FMA ? c[i] : 0u;
        out[i] = apply<OP>(a[i], vb, vc, q);
    }
}

inline bool aligned16(const void *q)
{
    return (reinterpret_cast<uintptr_t>(q) & 15u) == 0;
}

template <int OP>
int launch(const EwParams &q, const uint32_t *a, const uint32_t *b, const uint32_t *c, uint32_t *out, size_t n,
           cudaStream_t stream)
{
    if (n == 0) return MONT_OK;
    if (!a || !out || (OP != OP_SCALE && !b) || (OP == OP_FMA && !c)) return MONT_EINVAL;
    if (n > (SIZE_MAX >> 3)) return MONT_ERANGE;
    const size_t bytes = n * sizeof(uint32_t);
    if (partial_overlap(a, bytes, out, bytes)) return MONT_EINVAL;
    if (OP != OP_SCALE && partial_overlap(b, bytes, out, bytes)) return MONT_EINVAL;
    if (OP == OP_FMA && partial_overlap(c, bytes, out, bytes)) return MONT_EINVAL;

    const int sms = device_sm_count();
    if (sms <= 0) return MONT_ECUDA;
    const size_t max_blocks = static_cast<size_t>(sms) * (2048 / kThreads);
    const bool vec = aligned16(a) && aligned16(out) && (OP == OP_SCALE || aligned16(b)) &&
                     (OP != OP_FMA || aligned16(c));
    if (vec) {
        const size_t n4 = n / 4;
        const size_t want = (n4 + kThreads - 1) / kThreads;
        const unsigned grid = static_cast<unsigned>(want < 1 ? 1 : (want < max_blocks ? want : max_blocks));
        k_elementwise<OP><<<grid, kThreads, 0, stream>>>(a, b, c, out, n4, static_cast<uint32_t>(n & 3), q);
    } else {
        const size_t want = (n + kThreads - 1) / kThreads;
        const unsigned grid = static_cast<unsigned>(want < max_blocks ? want : max_blocks);
        k_elementwise_scalar<OP><<<grid, kThreads, 0, stream>>>(a, b, c, out, n, q);
    }
    return launch_status();
}

template <int OP>
int launch_ctx(const mont_ctx *ctx, const uint32_t *a, const uint32_t *b, const uint32_t *c, uint32_t *out,
               size_t n, uint32_t k, cudaStream_t stream)
{
    const int rc = check_ctx(ctx);
    if (rc != MONT_OK) return rc;
    return launch<OP>(EwParams{ctx->p, ctx->p_prime, k, 0u}, a, b, c, out, n, stream);
}

}  // namespace
}  // namespace mont

extern "C" int to_mont(const mont_ctx *ctx, const uint32_t *in, uint32_t *out, size_t n, cudaStream_t stream)
{
    if (!ctx) return MONT_EINVAL;
    return mont::launch_ctx<mont::OP_SCALE>(ctx, in, nullptr, nullptr, out, n, ctx->r2_mod_p, stream);
}

extern "C" int from_mont(const mont_ctx *ctx, const uint32_t *in, uint32_t *out, size_t n,
                         cudaStream_t stream)
{
    return mont::launch_ctx<mont::OP_SCALE>(ctx, in, nullptr, nullptr, out, n, 1u, stream);
}

extern "C" int mont_mul(const mont_ctx *ctx, const uint32_t *a, const uint32_t *b, uint32_t *out, size_t n,
                        cudaStream_t stream)
{
    return mont::launch_ctx<mont::OP_MUL>(ctx, a, b, nullptr, out, n, 0u, stream);
}

extern "C" int mont_fma(const mont_ctx *ctx, const uint32_t *a, const uint32_t *b, const uint32_t *c,
                        uint32_t *out, size_t n, cudaStream_t stream)
{
    return mont::launch_ctx<mont::OP_FMA>(ctx, a, b, c, out, n, 0u, stream);
}

extern "C" int barrett_mulmod(uint32_t p, const uint32_t *a, const uint32_t *b, uint32_t *out, size_t n,
                              cudaStream_t stream)
{
    if (p < 3 || !(p & 1u) || p >= 0x80000000u) return MONT_EINVAL;
    uint32_t k = 0;
    while ((uint64_t{1} << k) < p) k++;                                // k = ceil(log2 P)
    const uint64_t pb = (uint64_t{1} << (2 * k)) / p;                   // P' = floor(2^(2k) / P) < 2^32
    return mont::launch<mont::OP_BARRETT>(mont::EwParams{p, 0u, k, static_cast<uint32_t>(pb)}, a, b, nullptr, out,
                                          n, stream);
}

extern "C" int fourier_redc_mul(const mont_ctx *ctx, const uint32_t *a, const uint32_t *b, uint32_t *out, size_t n,
                                cudaStream_t stream)
{
    const int rc = mont::check_ctx(ctx);
    if (rc != MONT_OK) return rc;
    const uint32_t w = ctx->p - 1;                                     // c 2^n
    uint32_t n2 = 0;
    while (!((w >> n2) & 1u)) n2++;
    if (2 * n2 < 32 || ctx->p >= (1u << 30)) return MONT_ERANGE;      // Fourier prime with 2n >= 32, P < 2^30
    return mont::launch<mont::OP_FOURIER>(mont::EwParams{ctx->p, ctx->p_prime, 0u, w}, a, b, nullptr, out, n,
                                          stream);
}
