// twiddles.cu -- resident per-(device, prime) twiddle tables and NTT plans.
//
// Table layout (see ntt_core.cuh): entry 2^s + i, s = 0 .. K-1, i < 2^s,
// holds r = w_(2^(s+1))^bitrev_s(i) (forward) or its inverse, with
// w_(2^(s+1)) = g^((P-1)/2^(s+1)) and g the smallest primitive root of P.
// Each entry is rR mod P (Montgomery form).  The table does
// not depend on the transform size, so one table of 2^K entries serves every
// N <= 2^K; a larger request builds a larger table (older ones stay valid
// for plans that hold them until the library is unloaded).
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "ntt_internal.cuh"

namespace mont {

static bool is_prime32(uint32_t p)
{
    if (p < 2) return false;
    for (uint32_t q = 2; static_cast<uint64_t>(q) * q <= p; q++)
        if (p % q == 0) return false;
    return true;
}

uint32_t host_primitive_root(uint32_t p)
{
    uint32_t f[32];
    int nf = 0;
    uint32_t m = p - 1;
    for (uint32_t q = 2; static_cast<uint64_t>(q) * q <= m; q++) {
        if (m % q) continue;
        f[nf++] = q;
        while (m % q == 0) m /= q;
    }
    if (m > 1) f[nf++] = m;
    for (uint32_t g = 2; g < p; g++) {
        bool ok = true;
        for (int i = 0; i < nf && ok; i++) ok = host_powmod(g, (p - 1) / f[i], p) != 1;
        if (ok) return g;
    }
    return 0;
}

int two_adicity(uint32_t p)
{
    int k = 0;
    for (uint32_t m = p - 1; m && !(m & 1); m >>= 1) k++;
    return k;
}

namespace {

std::mutex g_mu;
std::vector<TwTable *> g_tables;   // never freed before unload; plans point into them

uint32_t bitrev(uint32_t i, int bits)
{
    uint32_t r = 0;
    for (int b = 0; b < bits; b++) r |= ((i >> b) & 1u) << (bits - 1 - b);
    return r;
}

void fill_table(std::vector<uint32_t> &t, uint32_t p, uint32_t g, int log2max, bool inverse)
{
    t.assign(size_t{1} << log2max, 0u);
    std::vector<uint32_t> pw;
    for (int s = 0; s < log2max; s++) {
        const uint32_t m = 1u << s;
        uint32_t w = host_powmod(g, (p - 1) >> (s + 1), p);      // primitive 2^(s+1)-th root
        if (inverse) w = host_powmod(w, p - 2, p);               // p prime: w^-1 = w^(p-2)
        pw.resize(m);
        pw[0] = 1;
        for (uint32_t e = 1; e < m; e++) pw[e] = host_mulmod(pw[e - 1], w, p);
        for (uint32_t i = 0; i < m; i++) {
            t[m + i] = host_to_mont(pw[bitrev(i, s)], p);
        }
    }
}

}  // namespace

int get_table(uint32_t p, int log2n, const TwTable **out)
{
    if (p >= 0x80000000u || p < 3 || !(p & 1u)) return MONT_EINVAL;
    if (log2n < 0 || log2n > kMaxLog2N) return MONT_ERANGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MONT_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    // Existing tables first: the primality test below (trial division, tens
    // of microseconds) runs only when a new table is built.
    for (TwTable *t : g_tables)
        if (t->device == dev && t->p == p && t->log2max >= log2n) {
            *out = t;
            return MONT_OK;
        }
    if (!is_prime32(p)) return MONT_EINVAL;
    if (log2n > two_adicity(p)) return MONT_ERANGE;
    // Build at least 2^12 entries so small sizes share one table.
    int lg = log2n < 12 ? 12 : log2n;
    if (lg > two_adicity(p)) lg = two_adicity(p);
    if (lg > kMaxLog2N) lg = kMaxLog2N;
    TwTable *t = new (std::nothrow) TwTable();
    if (!t) return MONT_ENOMEM;
    t->device = dev;
    t->p = p;
    t->p_prime = host_neg_inv32(p);
    t->log2max = lg;
    t->g = host_primitive_root(p);
    std::vector<uint32_t> h;
    const size_t bytes = (size_t{1} << lg) * sizeof(uint32_t);
    if (cudaMalloc(&t->fwd, bytes) != cudaSuccess || cudaMalloc(&t->inv, bytes) != cudaSuccess) {
        cudaFree(t->fwd);
        delete t;
        cudaGetLastError();
        return MONT_ENOMEM;
    }
    fill_table(h, p, t->g, lg, false);
    cudaError_t e1 = cudaMemcpy(t->fwd, h.data(), bytes, cudaMemcpyHostToDevice);
    fill_table(h, p, t->g, lg, true);
    cudaError_t e2 = cudaMemcpy(t->inv, h.data(), bytes, cudaMemcpyHostToDevice);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        cudaFree(t->fwd);
        cudaFree(t->inv);
        delete t;
        return MONT_ECUDA;
    }
    g_tables.push_back(t);
    *out = t;
    return MONT_OK;
}

int make_plan(uint32_t p, int log2n, ntt_plan *plan)
{
    const TwTable *t = nullptr;
    int rc = get_table(p, log2n, &t);
    if (rc != MONT_OK) return rc;
    plan->table = t;
    plan->p = p;
    plan->p_prime = t->p_prime;
    plan->log2n = log2n;
    plan->device = t->device;
    const uint32_t n_mod = static_cast<uint32_t>((uint64_t{1} << log2n) % p);
    const uint32_t ninv = host_powmod(n_mod, p - 2, p);
    plan->ninv_mont = host_to_mont(ninv, p);                    // N^-1 R mod P
    plan->k_scale = host_to_mont(plan->ninv_mont, p);           // N^-1 R^2 mod P
    return MONT_OK;
}

}  // namespace mont

extern "C" int ntt_plan_create(uint32_t p, uint32_t log2n, ntt_plan **out)
{
    if (!out) return MONT_EINVAL;
    *out = nullptr;
    ntt_plan *plan = new (std::nothrow) ntt_plan();
    if (!plan) return MONT_ENOMEM;
    int rc = mont::make_plan(p, static_cast<int>(log2n), plan);
    if (rc != MONT_OK) {
        delete plan;
        return rc;
    }
    *out = plan;
    return MONT_OK;
}

extern "C" void ntt_plan_destroy(ntt_plan *plan)
{
    delete plan;
}
