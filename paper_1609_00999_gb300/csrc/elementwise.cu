// elementwise.cu -- to_mont / from_mont / mont_mul / mont_fma over vectors.
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

enum Op { OP_SCALE = 0, OP_MUL = 1, OP_FMA = 2 };

constexpr int kThreads = 256;
constexpr int kIlp = 2;

template <int OP>
__device__ __forceinline__ uint32_t apply(uint32_t a, uint32_t b, uint32_t c, uint32_t p, uint32_t pp)
{
    // OP_SCALE: b is the launch-wide constant k (R^2 mod P for to_mont, 1 for from_mont).
    const uint32_t t = mont_mul(a, b, p, pp);
    if constexpr (OP == OP_FMA) return add_mod(t, c, p);
    return t;
}

template <int OP>
__device__ __forceinline__ uint4 apply4(uint4 a, uint4 b, uint4 c, uint32_t p, uint32_t pp)
{
    uint4 r;
    r.x = apply<OP>(a.x, b.x, c.x, p, pp);
    r.y = apply<OP>(a.y, b.y, c.y, p, pp);
    r.z = apply<OP>(a.z, b.z, c.z, p, pp);
    r.w = apply<OP>(a.w, b.w, c.w, p, pp);
    return r;
}

// Vector body over n4 uint4 chunks plus a scalar tail of `tail` elements
// starting at element 4 * n4.  For OP_SCALE, b is unused and k is the multiplier.
template <int OP>
__global__ void __launch_bounds__(kThreads)
k_elementwise(const uint32_t *__restrict__ a, const uint32_t *__restrict__ b,
              const uint32_t *__restrict__ c, uint32_t *__restrict__ out, size_t n4, uint32_t tail,
              uint32_t p, uint32_t pp, uint32_t k)
{
    const uint4 *a4 = reinterpret_cast<const uint4 *>(a);
    const uint4 *b4 = reinterpret_cast<const uint4 *>(b);
    const uint4 *c4 = reinterpret_cast<const uint4 *>(c);
    uint4 *o4 = reinterpret_cast<uint4 *>(out);
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
        for (int u = 0; u < kIlp; u++) __stcs(o4 + i + u * stride, apply4<OP>(va[u], vb[u], vc[u], p, pp));
    }
    for (; i < n4; i += stride) {
        const uint4 va = __ldcs(a4 + i);
        const uint4 vb = OP == OP_SCALE ? kk : __ldcs(b4 + i);
        const uint4 vc = OP == OP_FMA ? __ldcs(c4 + i) : zero;
        __stcs(o4 + i, apply4<OP>(va, vb, vc, p, pp));
    }
    if (blockIdx.x == 0 && threadIdx.x < tail) {
        const size_t j = 4 * n4 + threadIdx.x;
        const uint32_t vb = OP == OP_SCALE ? k : b[j];
        const uint32_t vc = OP == OP_FMA ? c[j] : 0u;
        out[j] = apply<OP>(a[j], vb, vc, p, pp);
    }
}

// Scalar grid-stride variant for operands that are not all 16-byte aligned.
template <int OP>
__global__ void __launch_bounds__(kThreads)
k_elementwise_scalar(const uint32_t *__restrict__ a, const uint32_t *__restrict__ b,
                     const uint32_t *__restrict__ c, uint32_t *__restrict__ out, size_t n, uint32_t p,
                     uint32_t pp, uint32_t k)
{
    const size_t stride = static_cast<size_t>(gridDim.x) * kThreads;
    for (size_t i = static_cast<size_t>(blockIdx.x) * kThreads + threadIdx.x; i < n; i += stride) {
        const uint32_t vb = OP == OP_SCALE ? k : b[i];
        const uint32_t vc = OP == OP_FMA ? c[i] : 0u;
        out[i] = apply<OP>(a[i], vb, vc, p, pp);
    }
}

inline bool aligned16(const void *q)
{
    return (reinterpret_cast<uintptr_t>(q) & 15u) == 0;
}

template <int OP>
int launch(const mont_ctx *ctx, const uint32_t *a, const uint32_t *b, const uint32_t *c, uint32_t *out,
           size_t n, uint32_t k, cudaStream_t stream)
{
    int rc = check_ctx(ctx);
    if (rc != MONT_OK) return rc;
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
        k_elementwise<OP><<<grid, kThreads, 0, stream>>>(a, b, c, out, n4, static_cast<uint32_t>(n & 3),
                                                         ctx->p, ctx->p_prime, k);
    } else {
        const size_t want = (n + kThreads - 1) / kThreads;
        const unsigned grid = static_cast<unsigned>(want < max_blocks ? want : max_blocks);
        k_elementwise_scalar<OP><<<grid, kThreads, 0, stream>>>(a, b, c, out, n, ctx->p, ctx->p_prime, k);
    }
    return launch_status();
}

}  // namespace
}  // namespace mont

extern "C" int to_mont(const mont_ctx *ctx, const uint32_t *in, uint32_t *out, size_t n, cudaStream_t stream)
{
    if (!ctx) return MONT_EINVAL;
    return mont::launch<mont::OP_SCALE>(ctx, in, nullptr, nullptr, out, n, ctx->r2_mod_p, stream);
}

extern "C" int from_mont(const mont_ctx *ctx, const uint32_t *in, uint32_t *out, size_t n,
                         cudaStream_t stream)
{
    return mont::launch<mont::OP_SCALE>(ctx, in, nullptr, nullptr, out, n, 1u, stream);
}

extern "C" int mont_mul(const mont_ctx *ctx, const uint32_t *a, const uint32_t *b, uint32_t *out, size_t n,
                        cudaStream_t stream)
{
    return mont::launch<mont::OP_MUL>(ctx, a, b, nullptr, out, n, 0u, stream);
}

extern "C" int mont_fma(const mont_ctx *ctx, const uint32_t *a, const uint32_t *b, const uint32_t *c,
                        uint32_t *out, size_t n, cudaStream_t stream)
{
    return mont::launch<mont::OP_FMA>(ctx, a, b, c, out, n, 0u, stream);
}
