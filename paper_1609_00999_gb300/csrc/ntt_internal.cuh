// ntt_internal.cuh -- host-side structures shared by the NTT translation units.
#pragma once
#include <cstdint>

#include "common.cuh"

namespace mont {

constexpr int kMaxLog2N = 24;       // largest transform the library plans
constexpr int kMaxSmemLog2N = 14;   // largest transform done by one CTA

struct TwTable {
    int device = 0;
    uint32_t p = 0, p_prime = 0, g = 0;
    int log2max = 0;
    uint32_t *fwd = nullptr;   // device, 2^log2max forward twiddles (Montgomery form)
    uint32_t *inv = nullptr;   // device, inverse twiddles
};

uint32_t host_primitive_root(uint32_t p);
int two_adicity(uint32_t p);
// Resident twiddle table for (current device, p) covering 2^log2n.
int get_table(uint32_t p, int log2n, const TwTable **out);

}  // namespace mont

struct ntt_plan {
    const mont::TwTable *table;
    uint32_t p, p_prime;
    int log2n;
    int device;
    uint32_t ninv_mont;   // N^-1 R mod P   (REDC(x * it) = x N^-1)
    uint32_t k_scale;     // N^-1 R^2 mod P (REDC(x * it) = x N^-1 R)
};

namespace mont {
int make_plan(uint32_t p, int log2n, ntt_plan *plan);
}
