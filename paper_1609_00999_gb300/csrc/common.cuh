// common.cuh -- host-side helpers shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "mont.h"

namespace mont {

// Streaming multiprocessor count of the current device (cached per device).
int device_sm_count();

// Returns MONT_OK if ctx holds a self-consistent Montgomery context.
int check_ctx(const mont_ctx *ctx);

// True if [a, a+na) and [b, b+nb) (bytes) overlap without being identical.
inline bool partial_overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    if (x == y && na == nb) return false;
    return x < y + nb && y < x + na;
}

// True if the ranges overlap at all.
inline bool any_overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return na && nb && x < y + nb && y < x + na;
}

inline int launch_status()
{
    return cudaGetLastError() == cudaSuccess ? MONT_OK : MONT_ECUDA;
}

// Host-side Montgomery constants (R = 2^32), shared by the host code of the
// CUDA library only.
uint32_t host_neg_inv32(uint32_t p);                    // -p^-1 mod 2^32
uint32_t host_mulmod(uint32_t a, uint32_t b, uint32_t p);
uint32_t host_powmod(uint32_t a, uint64_t e, uint32_t p);
uint32_t host_to_mont(uint32_t a, uint32_t p);          // a R mod P

}  // namespace mont
