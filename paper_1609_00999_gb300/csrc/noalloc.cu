// noalloc.cu -- polymul_noalloc: a polynomial product that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that records work into a CUDA
// graph (stream capture rejects allocation calls), code running inside a
// framework whose own allocator has reserved the device memory, and
// latency-critical paths that cannot afford cudaMalloc's implicit device
// synchronisation.  This entry point runs the same kernels as polymul, but
// products with N > 2^14 take their scratch from a fixed array in the
// library's own device memory instead of a cudaMalloc'ed buffer.
//
// The array lives for as long as the library is loaded, on every device
// that loads it.  Every call shares it and it keeps the previous call's
// contents; nothing needs clearing, because each call writes every scratch
// word before reading it.  Calls whose kernels overlap on the GPU (e.g. on
// two streams at once) race on the array.
#include <mutex>

#include "ntt_kernels.cuh"

namespace mont {
namespace {

// Largest product this entry point accepts: la + lb - 1 <= 2^18, hence
// N <= 2^18 and 2N words of scratch (2 MiB).
constexpr int kNoAllocMaxLog2N = 18;
constexpr size_t kNoAllocWords = size_t{2} << kNoAllocMaxLog2N;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

// Host code cannot use the array's name as a device address; the address is
// looked up once per device (first call with that device current).
std::mutex g_addr_mu;
uint32_t *g_addr[128];

int scratch_address(uint32_t **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return MONT_ECUDA;
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return MONT_ECUDA;
        }
        g_addr[dev] = static_cast<uint32_t *>(ptr);
    }
    *out = g_addr[dev];
    return MONT_OK;
}

}  // namespace
}  // namespace mont

extern "C" int polymul_noalloc(const ntt_plan *plan, const uint32_t *a, size_t la, const uint32_t *b, size_t lb,
                               uint32_t *c, cudaStream_t stream)
{
    if (!plan || !plan->table || !a || !b || !c || la == 0 || lb == 0) return MONT_EINVAL;
    if (la > (size_t{1} << 30) || lb > (size_t{1} << 30)) return MONT_ERANGE;
    const size_t lc = la + lb - 1;
    const int log2n = mont::ceil_log2(lc);
    if (log2n > mont::kNoAllocMaxLog2N) return MONT_ERANGE;
    if (log2n > plan->log2n || log2n > plan->table->log2max) return MONT_ERANGE;   // plan too small
    if (mont::any_overlap(c, lc * 4, a, la * 4) || mont::any_overlap(c, lc * 4, b, lb * 4)) return MONT_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return MONT_ECUDA;
    if (dev != plan->device) return MONT_EINVAL;

    // Plan for this N from the caller's tables: host arithmetic only.
    ntt_plan pl = *plan;
    const uint32_t p = pl.p;
    pl.log2n = log2n;
    const uint32_t n_mod = static_cast<uint32_t>((uint64_t{1} << log2n) % p);
    pl.ninv_mont = mont::host_to_mont(mont::host_powmod(n_mod, p - 2, p), p);
    pl.k_scale = mont::host_to_mont(pl.ninv_mont, p);

    if (log2n <= mont::kMaxSmemLog2N) {
        mont::PolyArgs A;
        A.a = a;
        A.b = b;
        A.c = c;
        A.la = la;
        A.lb = lb;
        A.lc = lc;
        A.count = 1;
        A.tw = pl.table->fwd;
        A.itw = pl.table->inv;
        A.p = p;
        A.pp = pl.p_prime;
        A.k_scale = pl.k_scale;
        return mont::dispatch_polymul_smem(log2n, A, stream);
    }
    uint32_t *ws = nullptr;
    int rc = mont::scratch_address(&ws);
    if (rc != MONT_OK) return rc;
    return mont::polymul_large(pl, a, la, b, lb, c, 1, ws, stream);
}
