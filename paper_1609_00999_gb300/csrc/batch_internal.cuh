// batch_internal.cuh -- job-list batches shared by the batch plans
// (polymul_batch.cu) and the request server (server.cu).
#pragma once
#include <cstdint>
#include <vector>

#include "ntt_kernels.cuh"

namespace mont {

constexpr int kThreads = 256;         // threads per CTA of the persistent kernel
constexpr int kSmallLog = 13;      // N <= 2^13: whole product in one CTA
constexpr int kRowLog = 13;        // row size 2^13 for split products (N > 2^13)
constexpr int kMaxColLog = 8;      // K1 <= 8: N <= 2^21 in a batch
constexpr int kMaxRegColLog = 4;   // K1 <= 4: column levels in registers
constexpr int kWholeMaxLog = 15;   // split products up to 2^15: one CTA runs all their jobs
constexpr int kMaxPrimes = 8;
constexpr int kMinTftColLog = 2;   // row-granular TFT for 2 <= K1 <= 4 (register column passes)

enum : uint32_t { JOB_SMALL = 0, JOB_COLF = 1, JOB_ROW = 2, JOB_COLI = 3, JOB_WHOLE = 4 };

struct Job {
    uint32_t type, k, prod, idx;   // idx: tile / row index, or the number of products of a SMALL job
};

// A split product (N > 2^13) is 2^K1 rows of 2^13 (K1 = log2 N - 13).  With
// tft set it runs as a truncated transform at row granularity: only the
// first nrows = ceil(lc / 2^13) < 2^K1 rows (the first nrows x 2^13 outputs
// of the forward transforms in bit-reversed order) are computed, and the
// inverse column pass is an inverse TFT of nrows known outputs per column;
// k_scale is then (2^13)^-1 R^2 (the column pass scales exactly) instead of
// N^-1 R^2.
struct Prod {
    const uint32_t *a, *b;
    uint32_t *c;
    uint32_t *ws;         // 2N words, large products only
    uint32_t la, lb, lc, k;
    uint16_t prime, tft;
    uint32_t k_scale;
    uint32_t ntiles, nrows;
};
static_assert(sizeof(Prod) == 64, "product table entry");

struct PrimeInfo {
    uint32_t p, pp;
    const uint32_t *tw, *itw;
};

struct BatchArgs {
    const Job *jobs;
    const Prod *prods;
    uint32_t *sync;    // [0] job counter, [1] error word, then per product: COLF done, ROW done
    uint32_t njobs;
    uint32_t wait_iters;
    unsigned long long wait_ns;
    PrimeInfo primes[kMaxPrimes];
};

// Job orders: 0 = split products' column tiles, then whole small products,
// then rows, then output tiles; 1 = small products first; 2 and 3 =
// software-pipelined: rows of product i follow the column tiles of product
// i + D and the output tiles of product i - D, with the small products spread
// evenly in between (D = 32 and 64), so memory-heavy tile jobs and
// compute-heavy row jobs run at the same time.
constexpr int kJobOrders = 4;

// Host-side form of a batch: the product table (scratch pointers hold word
// offsets from the batch's scratch base until rebased) and the job list for
// every job order.
struct BatchHost {
    std::vector<Prod> prods;
    std::vector<Job> jobs[kJobOrders];
    size_t ws_words = 0;
};

// Validates the descriptors and builds the batch.  Products are stored small
// (N <= 2^13, sorted by size) first, then split ones.  Primes are looked up
// in prime_list (extended, and prime_log2 raised, unless fixed_primes).
// With tft, split products with 2 <= K1 <= 4 whose output leaves rows
// unused run as row-granular truncated transforms.
int batch_build(const polymul_desc *descs, size_t count, BatchHost &out, std::vector<uint32_t> &prime_list,
                std::vector<int> &prime_log2, bool fixed_primes, bool tft);
// Replaces scratch offsets by pointers into ws.
void batch_rebase(BatchHost &b, uint32_t *ws);
// Opts kernel variant (0: 2 CTAs/SM register budget, 1: 3 CTAs/SM) into its
// shared memory and returns its CTAs per SM.
int batch_occupancy(int variant, int *per_sm);
// Resets the counters (sync_words words) and launches `grid` CTAs on jobs.
int batch_launch(BatchArgs A, const Job *jobs, uint32_t njobs, size_t sync_words, int grid, int variant,
                 cudaStream_t s);
// The phased form: the batch's jobs split by kind, each kind its own kernel
// (one CTA per job), ordered by stream dependencies: the small products on a
// side stream forked from s and joined back (aux null or s: all on s, fork
// and join unused), every larger product's forward columns, rows and output
// tiles on s.
enum PhaseList { PH_COLF_REG = 0, PH_COLF_TILE, PH_ROW, PH_COLI_REG, PH_COLI_TILE, PH_LISTS };

struct PhasedHost {
    std::vector<Job> jobs;            // the lists back to back
    uint32_t off[PH_LISTS] = {}, cnt[PH_LISTS] = {};
    std::vector<uint32_t> small;      // (log2 N, first product, count) per size present
};

// Splits a built batch's products into the phased form's lists.
void phased_build(const BatchHost &b, PhasedHost &out);
int batch_launch_phased(BatchArgs A, const PhasedHost &ph, const Job *d_jobs, size_t sync_words, cudaStream_t s,
                        cudaStream_t aux, cudaEvent_t fork, cudaEvent_t join);
// Scratch words for one product of this output length (0 when N <= 2^13).
size_t batch_ws_words(size_t lc);

}  // namespace mont
