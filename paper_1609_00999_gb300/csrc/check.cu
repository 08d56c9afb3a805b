// check.cu -- mont_check_residues: the device-side check of the input
// precondition (every word a residue of Z_P, Sec. 3.1) that the other entry
// points state but do not test on their hot path.
#include "common.cuh"

namespace mont {
namespace {

constexpr int kCheckThreads = 256;

// Sets *bad to 1 if some word of x[0, n) is >= p.  With VEC, x is 16-byte
// aligned: n / 4 uint4 chunks grid-stride plus the n & 3 tail words in
// block 0; otherwise a scalar grid-stride loop.  Every thread reaches the
// block-wide vote.
template <bool VEC>
__global__ void __launch_bounds__(kCheckThreads)
k_check_residues(const uint32_t *__restrict__ x, size_t n, uint32_t p, uint32_t *bad)
{
    const size_t stride = static_cast<size_t>(gridDim.x) * kCheckThreads;
    const size_t i0 = static_cast<size_t>(blockIdx.x) * kCheckThreads + threadIdx.x;
    bool found = false;
    if constexpr (VEC) {
        const uint4 *x4 = reinterpret_cast<const uint4 *>(x);
        const size_t n4 = n / 4;
        for (size_t i = i0; i < n4; i += stride) {
            const uint4 v = __ldcs(x4 + i);
            found |= v.x >= p || v.y >= p || v.z >= p || v.w >= p;
        }
        if (blockIdx.x == 0 && threadIdx.x < (n & 3)) found |= x[4 * n4 + threadIdx.x] >= p;
    } else {
        for (size_t i = i0; i < n; i += stride) found |= x[i] >= p;
    }
    if (__syncthreads_or(found) && threadIdx.x == 0) *bad = 1u;
}

}  // namespace
}  // namespace mont

extern "C" int mont_check_residues(uint32_t p, const uint32_t *x, size_t n, cudaStream_t stream)
{
    using mont::kCheckThreads;
    if (p < 3 || !(p & 1u) || p >= 0x80000000u) return MONT_EINVAL;
    if (n == 0) return MONT_OK;
    if (!x || n > (SIZE_MAX >> 3)) return MONT_EINVAL;
    const int sms = mont::device_sm_count();
    if (sms <= 0) return MONT_ECUDA;
    const bool vec = (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
    const size_t units = vec ? n / 4 : n;
    const size_t max_blocks = static_cast<size_t>(sms) * (2048 / kCheckThreads);
    const size_t want = (units + kCheckThreads - 1) / kCheckThreads;
    const unsigned grid = static_cast<unsigned>(want < 1 ? 1 : (want < max_blocks ? want : max_blocks));

    uint32_t *bad = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void **>(&bad), sizeof(uint32_t), stream) != cudaSuccess) {
        cudaGetLastError();
        return MONT_ENOMEM;
    }
    uint32_t flagged = 0;
    int rc = cudaMemsetAsync(bad, 0, sizeof(uint32_t), stream) == cudaSuccess ? MONT_OK : MONT_ECUDA;
    if (rc == MONT_OK) {
        if (vec) mont::k_check_residues<true><<<grid, kCheckThreads, 0, stream>>>(x, n, p, bad);
        else mont::k_check_residues<false><<<grid, kCheckThreads, 0, stream>>>(x, n, p, bad);
        rc = mont::launch_status();
    }
    if (rc == MONT_OK &&
        cudaMemcpyAsync(&flagged, bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        rc = MONT_ECUDA;
    if (cudaFreeAsync(bad, stream) != cudaSuccess) rc = MONT_ECUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) rc = MONT_ECUDA;
    if (rc != MONT_OK) return rc;
    return flagged ? MONT_ERANGE : MONT_OK;
}
