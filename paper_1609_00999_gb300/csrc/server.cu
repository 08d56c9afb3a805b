// server.cu -- continuous-batching polymul request server on one GPU.
//
// Requests (c = a * b mod p, operands and result in host or device memory)
// are submitted at any time and move through three stages:
//   queued    : waiting for device memory (FIFO);
//   admitted  : a region of the device-memory budget holds the operands, the
//               result and the product's scratch; waiting for a launch slot;
//   in flight : part of a batch running on one of `slots` streams.
// mont_server_progress (non-blocking) retires finished batches (frees their
// memory, reports completions), admits queued requests while the budget
// allows, and, for every idle slot, launches the admitted requests (up to a
// coefficient cap) as one batch: copies of the operands into the budget
// region, the batch's kernels (the phased form of polymul_batch.cu: one
// kernel per job kind, the small products on a side stream of the slot;
// truncated transforms where they save rows), and copies of the results
// back.  Requests that arrive while batches run are admitted as
// memory frees up and launched on the next idle slot, so their work overlaps
// with the batches already on the device.  Each slot has a launcher thread
// that builds its batch and queues the copies and kernels, so the host work of
// several batches proceeds in parallel.  Twiddle tables for the server's
// primes are built once and stay resident; the device job and product tables
// of each slot are reused across batches.  Small requests' copies are one
// copy-kernel launch per direction and batch; large ones use the copy
// engines.
#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "batch_internal.cuh"

namespace mont {
namespace {

constexpr size_t kAlign = 256;
constexpr int kServeOrder = 0;   // job order: column tiles, whole and small products, rows, output tiles
// Batch form: the phased form (one kernel per job kind, small products on a
// side stream of the slot) or the persistent kernel.
constexpr bool kServePhased = true;

// First-fit allocator over one device region, offsets in bytes.
class Arena {
public:
    void init(size_t bytes) { free_[0] = bytes; total_ = bytes; }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = (bytes + kAlign - 1) / kAlign * kAlign;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, start = it->first + bytes;
            free_.erase(it);
            if (rest) free_[start] = rest;
            used_ += bytes;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = (bytes + kAlign - 1) / kAlign * kAlign;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t total() const { return total_; }

private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0, total_ = 0;
};

// One contiguous copy of n words (either side host or device memory: the
// copy kernel reads and writes through unified addresses).
struct CopyDesc {
    const uint32_t *src;
    uint32_t *dst;
    uint64_t n;
};

// Requests with at most this many input coefficients have their operands
// and results moved by the copy kernel (one launch per direction and batch);
// larger ones use the copy engines (one cudaMemcpyAsync per buffer).  Most
// requests are small but most bytes are in the large ones, so this removes
// most per-copy host calls while the bulk still streams on the copy engines.
constexpr uint64_t kKernelCopyMax = uint64_t{1} << 16;

// Many small copies in one launch: CTA i takes descriptors i, i + grid, ...
__global__ void __launch_bounds__(256) k_copy_many(const CopyDesc *__restrict__ d, uint32_t count)
{
    for (uint32_t i = blockIdx.x; i < count; i += gridDim.x) {
        const CopyDesc c = d[i];
        uint64_t j = threadIdx.x;
        for (; j + 3 * 256 < c.n; j += 4 * 256) {
            const uint32_t v0 = c.src[j], v1 = c.src[j + 256], v2 = c.src[j + 512], v3 = c.src[j + 768];
            c.dst[j] = v0;
            c.dst[j + 256] = v1;
            c.dst[j + 512] = v2;
            c.dst[j + 768] = v3;
        }
        for (; j < c.n; j += 256) c.dst[j] = c.src[j];
    }
}

struct Req {
    mont_request r;
    size_t off = 0, bytes = 0;   // arena region: a | b | c | scratch
    uint32_t *da = nullptr, *db = nullptr, *dc = nullptr, *dws = nullptr;
};

// A slot's batch moves IDLE -> PENDING (requests handed to the slot's
// launcher thread) -> LAUNCHED (copies and kernels queued on its stream, or
// launch_rc set) -> IDLE (retired by progress once its event completes).
enum SlotState : int { SLOT_IDLE = 0, SLOT_PENDING = 1, SLOT_LAUNCHED = 2 };

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    std::atomic<int> state{SLOT_IDLE};
    int launch_rc = MONT_OK;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    std::vector<Req> reqs;
    Job *d_jobs = nullptr;
    Prod *d_prods = nullptr;
    uint32_t *d_sync = nullptr;
    size_t cap_jobs = 0, cap_prods = 0;
    Job *h_jobs = nullptr;     // pinned staging
    Prod *h_prods = nullptr;
    uint32_t *h_err = nullptr;
    CopyDesc *d_copy = nullptr, *h_copy = nullptr;
    size_t cap_copy = 0;
    std::vector<CopyDesc> copies;
    BatchHost host;
    PhasedHost phased;
    cudaStream_t aux = nullptr;                 // the phased form's side stream
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

size_t words_bytes(size_t w)
{
    return (w * sizeof(uint32_t) + kAlign - 1) / kAlign * kAlign;
}

}  // namespace
}  // namespace mont

struct mont_server {
    int device = 0;
    std::vector<uint32_t> primes;
    std::vector<int> prime_log2;
    mont::BatchArgs args{};
    int occupancy = 1, sms = 1;
    uint8_t *arena_base = nullptr;
    mont::Arena arena;
    size_t max_batch_coeffs = 0;
    std::vector<std::unique_ptr<mont::Slot>> slots;
    std::deque<mont::Req> queued, admitted;
    std::deque<mont_completion> completed;
    mont_server_stats stats{};
};

namespace mont {
namespace {

int grow_copies(Slot &s, size_t n)
{
    if (n <= s.cap_copy) return MONT_OK;
    const size_t cap = std::max(n, 2 * s.cap_copy);
    cudaFree(s.d_copy);
    cudaFreeHost(s.h_copy);
    s.d_copy = nullptr;
    s.h_copy = nullptr;
    s.cap_copy = 0;
    if (cudaMalloc(&s.d_copy, cap * sizeof(CopyDesc)) != cudaSuccess ||
        cudaMallocHost(&s.h_copy, cap * sizeof(CopyDesc)) != cudaSuccess)
        return MONT_ENOMEM;
    s.cap_copy = cap;
    return MONT_OK;
}

int grow_slot(Slot &s, size_t njobs, size_t nprods)
{
    if (njobs > s.cap_jobs) {
        const size_t cap = std::max(njobs, 2 * s.cap_jobs);
        cudaFree(s.d_jobs);
        cudaFreeHost(s.h_jobs);
        s.d_jobs = nullptr;
        s.h_jobs = nullptr;
        s.cap_jobs = 0;
        if (cudaMalloc(&s.d_jobs, cap * sizeof(Job)) != cudaSuccess ||
            cudaMallocHost(&s.h_jobs, cap * sizeof(Job)) != cudaSuccess)
            return MONT_ENOMEM;
        s.cap_jobs = cap;
    }
    if (nprods > s.cap_prods) {
        const size_t cap = std::max(nprods, 2 * s.cap_prods);
        cudaFree(s.d_prods);
        cudaFreeHost(s.h_prods);
        cudaFree(s.d_sync);
        s.d_prods = nullptr;
        s.h_prods = nullptr;
        s.d_sync = nullptr;
        s.cap_prods = 0;
        if (cudaMalloc(&s.d_prods, cap * sizeof(Prod)) != cudaSuccess ||
            cudaMallocHost(&s.h_prods, cap * sizeof(Prod)) != cudaSuccess ||
            cudaMalloc(&s.d_sync, (2 + 2 * cap) * sizeof(uint32_t)) != cudaSuccess)
            return MONT_ENOMEM;
        s.cap_prods = cap;
    }
    return MONT_OK;
}

size_t request_bytes(const mont_request &r)
{
    const size_t lc = static_cast<size_t>(r.la) + r.lb - 1;
    return words_bytes(r.la) + words_bytes(r.lb) + words_bytes(lc) + words_bytes(batch_ws_words(lc));
}

// Finished batches: report completions and free their memory.
void retire(mont_server *sv)
{
    for (auto &sp : sv->slots) {
        Slot &s = *sp;
        if (s.state.load(std::memory_order_acquire) != SLOT_LAUNCHED) continue;
        int status = s.launch_rc;
        if (status == MONT_OK) {
            const cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaErrorNotReady) continue;
            status = q != cudaSuccess ? MONT_ECUDA : (*s.h_err ? MONT_ETIMEOUT : MONT_OK);
        }
        for (const Req &r : s.reqs) {
            sv->arena.release(r.off, r.bytes);
            sv->completed.push_back(mont_completion{r.r.id, status, 0});
            sv->stats.completed++;
        }
        s.reqs.clear();
        s.state.store(SLOT_IDLE, std::memory_order_release);
    }
}

void admit(mont_server *sv)
{
    while (!sv->queued.empty()) {
        Req &q = sv->queued.front();
        size_t off = 0;
        if (!sv->arena.alloc(q.bytes, &off)) break;
        q.off = off;
        uint8_t *base = sv->arena_base + off;
        const size_t lc = static_cast<size_t>(q.r.la) + q.r.lb - 1;
        q.da = reinterpret_cast<uint32_t *>(base);
        q.db = reinterpret_cast<uint32_t *>(base + words_bytes(q.r.la));
        q.dc = reinterpret_cast<uint32_t *>(base + words_bytes(q.r.la) + words_bytes(q.r.lb));
        q.dws = batch_ws_words(lc) ? reinterpret_cast<uint32_t *>(base + words_bytes(q.r.la) + words_bytes(q.r.lb) +
                                                                words_bytes(lc))
                                   : nullptr;
        sv->admitted.push_back(q);
        sv->queued.pop_front();
        sv->stats.admitted++;
        sv->stats.bytes_in_use = sv->arena.used();
        sv->stats.peak_bytes = std::max<uint64_t>(sv->stats.peak_bytes, sv->arena.used());
    }
}

// Main thread: move admitted requests (arrival order, up to the coefficient
// cap) into an idle slot and hand them to its launcher thread.
void take_batch(mont_server *sv, Slot &s)
{
    size_t coeffs = 0;
    while (!sv->admitted.empty()) {
        const Req &q = sv->admitted.front();
        const size_t c = static_cast<size_t>(q.r.la) + q.r.lb;
        if (!s.reqs.empty() && coeffs + c > sv->max_batch_coeffs) break;
        coeffs += c;
        s.reqs.push_back(q);
        sv->admitted.pop_front();
    }
    if (s.reqs.empty()) return;
    sv->stats.batches++;
    sv->stats.launched += s.reqs.size();
    {
        std::lock_guard<std::mutex> lock(s.mu);
        s.state.store(SLOT_PENDING, std::memory_order_release);
    }
    s.cv.notify_one();
}

// Launcher thread: build the batch and queue copies, kernels and the
// completion event on the slot's stream.
int issue_batch(mont_server *sv, Slot &s)
{
    std::vector<polymul_desc> descs(s.reqs.size());
    for (size_t i = 0; i < s.reqs.size(); i++) {
        const Req &q = s.reqs[i];
        descs[i] = polymul_desc{q.da, q.db, q.dc, q.r.la, q.r.lb, q.r.p, 0};
    }
    int rc = batch_build(descs.data(), descs.size(), s.host, sv->primes, sv->prime_log2, true, true);
    if (rc == MONT_OK) {
        // Each split product uses the scratch of its own request region.
        std::map<const uint32_t *, uint32_t *> ws_of;
        for (const Req &q : s.reqs) ws_of[q.dc] = q.dws;
        for (Prod &P : s.host.prods)
            if (P.k > static_cast<uint32_t>(kSmallLog)) P.ws = ws_of[P.c];
        if (kServePhased) phased_build(s.host, s.phased);
        rc = grow_slot(s, kServePhased ? s.phased.jobs.size() : s.host.jobs[kServeOrder].size(), s.host.prods.size());
    }
    // Small requests' copies as descriptor lists for the copy kernel: operands
    // first [0, ngather), results after.
    size_t ngather = 0;
    if (rc == MONT_OK) {
        s.copies.clear();
        for (const Req &q : s.reqs)
            if (uint64_t{q.r.la} + q.r.lb <= kKernelCopyMax) {
                s.copies.push_back(CopyDesc{q.r.a, q.da, q.r.la});
                s.copies.push_back(CopyDesc{q.r.b, q.db, q.r.lb});
            }
        ngather = s.copies.size();
        for (const Req &q : s.reqs)
            if (uint64_t{q.r.la} + q.r.lb <= kKernelCopyMax)
                s.copies.push_back(CopyDesc{q.dc, q.r.c, static_cast<uint64_t>(q.r.la) + q.r.lb - 1});
        rc = grow_copies(s, s.copies.size());
    }
    if (rc == MONT_OK) {
        for (const Req &q : s.reqs) {
            if (uint64_t{q.r.la} + q.r.lb <= kKernelCopyMax) continue;
            if (cudaMemcpyAsync(q.da, q.r.a, size_t{q.r.la} * 4, cudaMemcpyDefault, s.stream) != cudaSuccess ||
                cudaMemcpyAsync(q.db, q.r.b, size_t{q.r.lb} * 4, cudaMemcpyDefault, s.stream) != cudaSuccess)
                rc = MONT_ECUDA;
        }
        std::copy(s.copies.begin(), s.copies.end(), s.h_copy);
        const std::vector<Job> &jobs = kServePhased ? s.phased.jobs : s.host.jobs[kServeOrder];
        std::copy(jobs.begin(), jobs.end(), s.h_jobs);
        std::copy(s.host.prods.begin(), s.host.prods.end(), s.h_prods);
        if (rc == MONT_OK &&
            ((!s.copies.empty() && cudaMemcpyAsync(s.d_copy, s.h_copy, s.copies.size() * sizeof(CopyDesc),
                                                   cudaMemcpyHostToDevice, s.stream) != cudaSuccess) ||
             (!jobs.empty() && cudaMemcpyAsync(s.d_jobs, s.h_jobs, jobs.size() * sizeof(Job), cudaMemcpyHostToDevice,
                                               s.stream) != cudaSuccess) ||
             cudaMemcpyAsync(s.d_prods, s.h_prods, s.host.prods.size() * sizeof(Prod), cudaMemcpyHostToDevice,
                             s.stream) != cudaSuccess))
            rc = MONT_ECUDA;
    }
    const size_t copy_grid = static_cast<size_t>(sv->sms) * 4;
    if (rc == MONT_OK && ngather) {
        k_copy_many<<<static_cast<unsigned>(std::min(copy_grid, ngather)), 256, 0, s.stream>>>(
            s.d_copy, static_cast<uint32_t>(ngather));
        rc = launch_status();
    }
    if (rc == MONT_OK) {
        BatchArgs A = sv->args;
        A.prods = s.d_prods;
        A.sync = s.d_sync;
        if (kServePhased)
            rc = batch_launch_phased(A, s.phased, s.d_jobs, 2 + 2 * s.host.prods.size(), s.stream, s.aux, s.ev_fork,
                                     s.ev_join);
        else
            rc = batch_launch(A, s.d_jobs, static_cast<uint32_t>(s.host.jobs[kServeOrder].size()),
                              2 + 2 * s.host.prods.size(), sv->sms * sv->occupancy, 1, s.stream);
    }
    if (rc == MONT_OK) {
        const size_t nscatter = s.copies.size() - ngather;
        if (nscatter) {
            k_copy_many<<<static_cast<unsigned>(std::min(copy_grid, nscatter)), 256, 0, s.stream>>>(
                s.d_copy + ngather, static_cast<uint32_t>(nscatter));
            rc = launch_status();
        }
        for (const Req &q : s.reqs) {
            if (uint64_t{q.r.la} + q.r.lb <= kKernelCopyMax) continue;
            const size_t lc = static_cast<size_t>(q.r.la) + q.r.lb - 1;
            if (cudaMemcpyAsync(q.r.c, q.dc, lc * 4, cudaMemcpyDefault, s.stream) != cudaSuccess) rc = MONT_ECUDA;
        }
        if (cudaMemcpyAsync(s.h_err, s.d_sync + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s.stream) != cudaSuccess ||
            cudaEventRecord(s.done, s.stream) != cudaSuccess)
            rc = MONT_ECUDA;
    }
    if (rc != MONT_OK) {
        cudaStreamSynchronize(s.stream);
        cudaGetLastError();
    }
    return rc;
}

void worker_loop(mont_server *sv, Slot *s)
{
    cudaSetDevice(sv->device);
    for (;;) {
        std::unique_lock<std::mutex> lock(s->mu);
        s->cv.wait(lock, [&] { return s->stop || s->state.load(std::memory_order_acquire) == SLOT_PENDING; });
        if (s->stop) return;
        lock.unlock();
        s->launch_rc = issue_batch(sv, *s);
        s->state.store(SLOT_LAUNCHED, std::memory_order_release);
    }
}

void destroy_server(mont_server *sv)
{
    for (auto &sp : sv->slots) {
        if (!sp || !sp->worker.joinable()) continue;
        {
            std::lock_guard<std::mutex> lock(sp->mu);
            sp->stop = true;
        }
        sp->cv.notify_one();
        sp->worker.join();
    }
    for (auto &sp : sv->slots) {
        if (!sp) continue;
        Slot &s = *sp;
        if (s.stream) cudaStreamSynchronize(s.stream);
        cudaFree(s.d_jobs);
        cudaFree(s.d_prods);
        cudaFree(s.d_sync);
        cudaFreeHost(s.h_jobs);
        cudaFreeHost(s.h_prods);
        cudaFreeHost(s.h_err);
        cudaFree(s.d_copy);
        cudaFreeHost(s.h_copy);
        if (s.done) cudaEventDestroy(s.done);
        if (s.ev_fork) cudaEventDestroy(s.ev_fork);
        if (s.ev_join) cudaEventDestroy(s.ev_join);
        if (s.aux) cudaStreamDestroy(s.aux);
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    cudaFree(sv->arena_base);
}

}  // namespace
}  // namespace mont

extern "C" int mont_server_create(const uint32_t *primes, int nprimes, uint32_t max_log2n, size_t budget_bytes,
                                  int slots, size_t max_batch_coeffs, mont_server **out)
{
    using namespace mont;
    if (!out || !primes || nprimes <= 0 || nprimes > kMaxPrimes || slots <= 0 || slots > 64 ||
        budget_bytes < kAlign || max_batch_coeffs == 0)
        return MONT_EINVAL;
    if (max_log2n > static_cast<uint32_t>(kRowLog + kMaxColLog)) return MONT_ERANGE;
    *out = nullptr;
    mont_server *sv = new (std::nothrow) mont_server();
    if (!sv) return MONT_ENOMEM;
    int rc = cudaGetDevice(&sv->device) == cudaSuccess ? MONT_OK : MONT_ECUDA;
    for (int i = 0; i < nprimes && rc == MONT_OK; i++) {
        const TwTable *t = nullptr;
        rc = get_table(primes[i], std::max<int>(static_cast<int>(max_log2n), kRowLog), &t);
        if (rc == MONT_OK) {
            sv->primes.push_back(primes[i]);
            sv->prime_log2.push_back(static_cast<int>(max_log2n));
            sv->args.primes[i] = PrimeInfo{t->p, t->p_prime, t->fwd, t->inv};
        }
    }
    if (rc == MONT_OK) rc = batch_occupancy(1, &sv->occupancy);   // 3-CTA/SM variant: fastest on mixed sizes
    sv->sms = device_sm_count();
    if (rc == MONT_OK && sv->sms <= 0) rc = MONT_ECUDA;
    if (rc == MONT_OK && cudaMalloc(&sv->arena_base, budget_bytes) != cudaSuccess) rc = MONT_ENOMEM;
    for (int i = 0; i < slots; i++) sv->slots.push_back(std::make_unique<Slot>());
    for (int i = 0; i < slots && rc == MONT_OK; i++) {
        Slot &s = *sv->slots[i];
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&s.aux, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.ev_join, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&s.h_err, sizeof(uint32_t)) != cudaSuccess)
            rc = MONT_ECUDA;
        else
            rc = grow_slot(s, 4096, 1024);
    }
    if (rc != MONT_OK) {
        cudaGetLastError();
        destroy_server(sv);
        delete sv;
        return rc;
    }
    sv->arena.init(budget_bytes);
    sv->max_batch_coeffs = max_batch_coeffs;
    sv->args.wait_iters = 1u << 22;
    sv->args.wait_ns = 2000000000ull;
    sv->stats.budget_bytes = budget_bytes;
    for (auto &sp : sv->slots) sp->worker = std::thread(worker_loop, sv, sp.get());
    *out = sv;
    return MONT_OK;
}

extern "C" void mont_server_destroy(mont_server *sv)
{
    if (!sv) return;
    mont::destroy_server(sv);
    delete sv;
}

extern "C" int mont_server_submit(mont_server *sv, const mont_request *reqs, size_t n)
{
    using namespace mont;
    if (!sv || (n && !reqs)) return MONT_EINVAL;
    // Validate everything first so a bad request rejects the call as a whole.
    for (size_t i = 0; i < n; i++) {
        const mont_request &r = reqs[i];
        if (!r.a || !r.b || !r.c || r.la == 0 || r.lb == 0 || r.reserved != 0) return MONT_EINVAL;
        size_t pi = 0;
        while (pi < sv->primes.size() && sv->primes[pi] != r.p) pi++;
        if (pi == sv->primes.size()) return MONT_EINVAL;
        const size_t lc = static_cast<size_t>(r.la) + r.lb - 1;
        if (ceil_log2(lc) > sv->prime_log2[pi]) return MONT_ERANGE;
        if (request_bytes(r) > sv->arena.total()) return MONT_ERANGE;   // could never be admitted
    }
    for (size_t i = 0; i < n; i++) {
        Req q;
        q.r = reqs[i];
        q.bytes = request_bytes(reqs[i]);
        sv->queued.push_back(q);
        sv->stats.submitted++;
    }
    return MONT_OK;
}

extern "C" int mont_server_progress(mont_server *sv, mont_completion *done, size_t cap, size_t *ndone)
{
    using namespace mont;
    if (!sv || !ndone || (cap && !done)) return MONT_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != sv->device) return MONT_EINVAL;
    retire(sv);
    admit(sv);
    int rc = MONT_OK;
    for (auto &sp : sv->slots) {
        if (sv->admitted.empty()) break;
        if (sp->state.load(std::memory_order_acquire) == SLOT_IDLE) take_batch(sv, *sp);
    }
    sv->stats.bytes_in_use = sv->arena.used();
    size_t k = 0;
    while (k < cap && !sv->completed.empty()) {
        done[k++] = sv->completed.front();
        sv->completed.pop_front();
    }
    *ndone = k;
    return rc;
}

extern "C" int mont_server_get_stats(const mont_server *sv, mont_server_stats *out)
{
    if (!sv || !out) return MONT_EINVAL;
    *out = sv->stats;
    out->queued = sv->queued.size();
    out->admitted_waiting = sv->admitted.size();
    size_t inflight = 0;
    for (const auto &sp : sv->slots) inflight += sp->reqs.size();
    out->in_flight = inflight;
    return MONT_OK;
}
