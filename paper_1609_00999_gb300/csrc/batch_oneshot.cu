// batch_oneshot.cu -- polymul_batch: one uneven batch without a plan, every
// device-side table of the batch in the caller's workspace.
//
// The same kernels as a batch plan (polymul_batch.cu) in the form the tuner
// picks for uneven batches and the request server runs: the phased form, one
// kernel per job kind, here all in order on the caller's stream, with
// truncated transforms.  Each call builds the job lists on the host and
// queues copies of them and of the product table into the workspace; a plan
// does that once, and can also be tuned and replayed as a CUDA graph.
#include <algorithm>
#include <vector>

#include "batch_internal.cuh"
#include "ntt_internal.cuh"

namespace mont {
namespace {

constexpr size_t kPart = 256;          // every part of the workspace starts 256-byte aligned

size_t round_up(size_t x)
{
    return (x + kPart - 1) / kPart * kPart;
}

// Byte offsets of the workspace parts: the counters (2 + 2 count words), the
// product table, the phased form's job lists, then the split products'
// scratch.
struct Layout {
    size_t sync, prods, jobs, scratch, total;
};

Layout layout_of(const BatchHost &h, const PhasedHost &ph, size_t count)
{
    Layout L;
    L.sync = 0;
    L.prods = round_up((2 + 2 * count) * sizeof(uint32_t));
    L.jobs = L.prods + round_up(count * sizeof(Prod));
    L.scratch = L.jobs + round_up(ph.jobs.size() * sizeof(Job));
    L.total = L.scratch + h.ws_words * sizeof(uint32_t);
    return L;
}

int build(const polymul_desc *descs, size_t count, BatchHost &h, std::vector<uint32_t> &primes,
          std::vector<int> &logs)
{
    if (!descs) return MONT_EINVAL;
    if (count > (size_t{1} << 31)) return MONT_ERANGE;
    return batch_build(descs, count, h, primes, logs, false, true);
}

}  // namespace
}  // namespace mont

extern "C" size_t polymul_batch_workspace_bytes(const polymul_desc *descs, size_t count)
{
    using namespace mont;
    if (count == 0) return 0;
    BatchHost h;
    PhasedHost ph;
    std::vector<uint32_t> primes;
    std::vector<int> logs;
    if (build(descs, count, h, primes, logs) != MONT_OK) return 0;
    phased_build(h, ph);
    return layout_of(h, ph, count).total;
}

extern "C" int polymul_batch(const polymul_desc *descs, size_t count, void *workspace, size_t ws_bytes,
                             cudaStream_t stream)
{
    using namespace mont;
    if (count == 0) return MONT_OK;
    BatchHost h;
    PhasedHost ph;
    std::vector<uint32_t> primes;
    std::vector<int> logs;
    int rc = build(descs, count, h, primes, logs);
    if (rc != MONT_OK) return rc;
    phased_build(h, ph);
    const Layout L = layout_of(h, ph, count);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kPart) != 0 || ws_bytes < L.total)
        return MONT_EINVAL;

    BatchArgs A{};
    for (size_t i = 0; i < primes.size(); i++) {
        const TwTable *t = nullptr;
        rc = get_table(primes[i], std::max(logs[i], kRowLog), &t);
        if (rc != MONT_OK) return rc;
        A.primes[i] = PrimeInfo{t->p, t->p_prime, t->fwd, t->inv};
    }
    uint8_t *base = static_cast<uint8_t *>(workspace);
    batch_rebase(h, reinterpret_cast<uint32_t *>(base + L.scratch));
    Prod *d_prods = reinterpret_cast<Prod *>(base + L.prods);
    Job *d_jobs = reinterpret_cast<Job *>(base + L.jobs);
    const std::vector<Job> &jobs = ph.jobs;
    // Copies from pageable memory return once the data is staged, so the
    // host tables may go out of scope before the copies reach the device.
    if (cudaMemcpyAsync(d_prods, h.prods.data(), count * sizeof(Prod), cudaMemcpyHostToDevice, stream) !=
            cudaSuccess ||
        (!jobs.empty() && cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(Job), cudaMemcpyHostToDevice,
                                          stream) != cudaSuccess)) {
        cudaGetLastError();
        return MONT_ECUDA;
    }
    A.prods = d_prods;
    A.sync = reinterpret_cast<uint32_t *>(base + L.sync);
    A.wait_iters = 1u << 22;
    A.wait_ns = 2000000000ull;   // 2 s per wait
    return batch_launch_phased(A, ph, d_jobs, 2 + 2 * count, stream, nullptr, nullptr, nullptr);
}

// Synchronous: waits for `stream`, then reads the error word (word 1 of the
// workspace) that an expired bounded wait sets.
extern "C" int polymul_batch_check(const void *workspace, cudaStream_t stream)
{
    if (!workspace) return MONT_EINVAL;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return MONT_ECUDA;
    uint32_t err = 0;
    if (cudaMemcpy(&err, static_cast<const uint32_t *>(workspace) + 1, sizeof(err), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return MONT_ECUDA;
    return err ? MONT_ETIMEOUT : MONT_OK;
}
