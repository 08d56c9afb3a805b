// setup.cu -- host-side Montgomery set-up (Sec. 3.1), error strings, device info.
#include <atomic>
#include <cstdio>

#include "common.cuh"

namespace mont {

// -p^-1 mod 2^32 by Newton (Hensel) lifting: for odd p, x = p is an inverse
// mod 2^3 (p^2 == 1 mod 8); each step x <- x (2 - p x) doubles the correct
// low bits (3 -> 6 -> 12 -> 24 -> 48).
uint32_t host_neg_inv32(uint32_t p)
{
    uint32_t x = p;
    for (int i = 0; i < 4; i++) x *= 2u - p * x;
    return 0u - x;
}

uint32_t host_mulmod(uint32_t a, uint32_t b, uint32_t p)
{
    return static_cast<uint32_t>(static_cast<uint64_t>(a) * b % p);
}

uint32_t host_powmod(uint32_t a, uint64_t e, uint32_t p)
{
    uint32_t r = 1u % p, base = a % p;
    for (; e; e >>= 1) {
        if (e & 1) r = host_mulmod(r, base, p);
        base = host_mulmod(base, base, p);
    }
    return r;
}

uint32_t host_to_mont(uint32_t a, uint32_t p)
{
    return static_cast<uint32_t>((static_cast<uint64_t>(a) << 32) % p);
}

static bool modulus_ok(uint32_t p)
{
    return p >= 3u && (p & 1u) && p < 0x80000000u;
}

int check_ctx(const mont_ctx *ctx)
{
    if (!ctx || !modulus_ok(ctx->p)) return MONT_EINVAL;
    if (ctx->p * ctx->p_prime != 0xFFFFFFFFu) return MONT_EINVAL;   // P P' == -1 mod R
    const uint32_t r = static_cast<uint32_t>((uint64_t{1} << 32) % ctx->p);
    if (ctx->r_mod_p != r || ctx->r2_mod_p != host_mulmod(r, r, ctx->p)) return MONT_EINVAL;
    return MONT_OK;
}

// Calls may come from several host threads at once (the server's launcher
// threads, callers on different streams): the cache entries are atomics,
// and a race only makes two threads store the same count.
int device_sm_count()
{
    static std::atomic<int> cache[128];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return 0;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

}  // namespace mont

extern "C" int mont_setup(uint32_t p, mont_ctx *out)
{
    if (!out || !mont::modulus_ok(p)) return MONT_EINVAL;
    const uint32_t r = static_cast<uint32_t>((uint64_t{1} << 32) % p);
    out->p = p;
    out->p_prime = mont::host_neg_inv32(p);
    out->r_mod_p = r;
    out->r2_mod_p = mont::host_mulmod(r, r, p);
    return MONT_OK;
}

extern "C" const char *mont_strerror(int code)
{
    switch (code) {
    case MONT_OK: return "success";
    case MONT_EINVAL: return "invalid argument";
    case MONT_ENOMEM: return "out of memory";
    case MONT_ERANGE: return "value or size out of range for this modulus or plan";
    case MONT_ETIMEOUT: return "bounded device wait timed out";
    case MONT_ECUDA: return "CUDA runtime error";
    case MONT_EUNSUPPORTED: return "unsupported request";
    default: return "unknown error code";
    }
}
