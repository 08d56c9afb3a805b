// workspace.cu -- library-owned device scratch, one buffer per (device, stream).
//
// Calls queued on one stream run in order, so they can share that stream's
// buffer.  Growing a buffer frees the old one with cudaFree, which waits for
// all work on the device, so no queued kernel can still be using it.
#include <mutex>
#include <vector>

#include "ntt_kernels.cuh"

namespace mont {
namespace {

struct Entry {
    int device;
    cudaStream_t stream;
    void *ptr;
    size_t bytes;
};

std::mutex g_ws_mu;
std::vector<Entry> g_ws;

}  // namespace

int stream_workspace(cudaStream_t s, size_t bytes, void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MONT_ECUDA;
    std::lock_guard<std::mutex> lock(g_ws_mu);
    for (Entry &e : g_ws) {
        if (e.device != dev || e.stream != s) continue;
        if (e.bytes >= bytes) {
            *out = e.ptr;
            return MONT_OK;
        }
        cudaFree(e.ptr);
        e.ptr = nullptr;
        e.bytes = 0;
        if (cudaMalloc(&e.ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            e.ptr = nullptr;
            return MONT_ENOMEM;
        }
        e.bytes = bytes;
        *out = e.ptr;
        return MONT_OK;
    }
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return MONT_ENOMEM;
    }
    g_ws.push_back(Entry{dev, s, p, bytes});
    *out = p;
    return MONT_OK;
}

}  // namespace mont

// Frees every library-owned scratch buffer (not the twiddle tables).
extern "C" int mont_release_workspaces(void)
{
    std::lock_guard<std::mutex> lock(mont::g_ws_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (mont::Entry &e : mont::g_ws) {
        cudaSetDevice(e.device);
        cudaFree(e.ptr);
    }
    mont::g_ws.clear();
    cudaSetDevice(cur);
    return MONT_OK;
}
