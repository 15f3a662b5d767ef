// Allocation-free (key, value) sort: the least-significant-digit radix sort of K4,
// with all of its scratch in one file-scope device array instead of context memory.
//
// For callers that may not call cudaMalloc: code whose device memory is owned by another
// allocator (a framework's caching pool, or a fixed arena reserved when the process starts),
// where a direct cudaMalloc can fail or fragment that reservation, and latency-critical loops in
// which a cudaMalloc / cudaFree would synchronise the device.  The paper has no counterpart.
#include <mutex>

#include "pgs_internal.cuh"

namespace pgs {
namespace {

constexpr int64_t kStaticMaxPairs = int64_t(1) << 18;  // 262,144 pairs
constexpr int64_t kStaticSortBlocks = kStaticMaxPairs / kSortTile;
constexpr int kMaxDevices = 64;

// scratch layout (bytes): other ping-pong keys, other ping-pong values, the sort's look-back
// words (8 passes of 64-bit keys), digit totals of every pass, pair count, sort CTA count, status word
constexpr size_t kOffKeys = 0;
constexpr size_t kOffVals = kOffKeys + sizeof(unsigned long long) * kStaticMaxPairs;
constexpr size_t kOffHist = kOffVals + sizeof(uint32_t) * kStaticMaxPairs;
constexpr size_t kOffTotals = kOffHist + sizeof(uint32_t) * lookback_words(kMaxPasses, kStaticSortBlocks);
constexpr size_t kOffCount = kOffTotals + sizeof(uint32_t) * kTotalWords;
constexpr size_t kOffBlocks = kOffCount + sizeof(unsigned long long);
constexpr size_t kOffStatus = kOffBlocks + sizeof(uint32_t);
constexpr size_t kScratchBytes = (kOffStatus + sizeof(int32_t) + 255) & ~size_t(255);

// Held by every GPU that loads the library until the process exits (3.8 MB).
static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

// Per-call set-up on the device: pair count, active sort CTAs, cleared totals.  The status word
// is not cleared here: a failed check stays recorded until pgs_sort_pairs_static_status reads it
// (the array starts zeroed).
__global__ void k_static_sort_init(unsigned char* base, int64_t count) {
    uint32_t* totals = reinterpret_cast<uint32_t*>(base + kOffTotals);
    for (int k = threadIdx.x; k < kTotalWords; k += blockDim.x) totals[k] = 0;
    if (threadIdx.x == 0) {
        *reinterpret_cast<unsigned long long*>(base + kOffCount) = (unsigned long long)count;
        *reinterpret_cast<uint32_t*>(base + kOffBlocks) = (uint32_t)((count + kSortTile - 1) / kSortTile);
    }
}

std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
int scratch_address(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PGS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return PGS_ERR_CUDA;
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_ptr[dev];
    return PGS_OK;
}

}  // namespace
}  // namespace pgs

using namespace pgs;

extern "C" int pgs_sort_pairs_static(const uint64_t* keys_in, const uint32_t* vals_in,
                                     uint64_t* keys_out, uint32_t* vals_out, int64_t count,
                                     int32_t key_bits, void* cuda_stream) {
    if (count < 0 || key_bits < 1 || key_bits > 64) return PGS_ERR_INVALID_ARG;
    if (count > kStaticMaxPairs) return PGS_ERR_TOO_LARGE;
    if (count == 0) return PGS_OK;
    if (!keys_in || !vals_in || !keys_out || !vals_out) return PGS_ERR_INVALID_ARG;
    unsigned char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != PGS_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    Scratch sc;
    sc.keys[0] = reinterpret_cast<unsigned long long*>(keys_out);
    sc.vals[0] = vals_out;
    sc.keys[1] = reinterpret_cast<unsigned long long*>(base + kOffKeys);
    sc.vals[1] = reinterpret_cast<uint32_t*>(base + kOffVals);
    sc.sort_hist = reinterpret_cast<uint32_t*>(base + kOffHist);
    sc.digit_totals = reinterpret_cast<uint32_t*>(base + kOffTotals);
    sc.pair_count = reinterpret_cast<unsigned long long*>(base + kOffCount);
    sc.sort_blocks = reinterpret_cast<uint32_t*>(base + kOffBlocks);
    sc.status = reinterpret_cast<int32_t*>(base + kOffStatus);
    // the output buffers are the first ping-pong buffer: copy the input there
    cudaError_t e = cudaMemcpyAsync(keys_out, keys_in, sizeof(uint64_t) * (size_t)count,
                                    cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(vals_out, vals_in, sizeof(uint32_t) * (size_t)count,
                            cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return PGS_ERR_CUDA;
    k_static_sort_init<<<1, 256, 0, s>>>(base, count);
    int buf = 0;
    launch_radix_sort_only(kStaticMaxPairs, key_bits, sc, s, &buf);
    if (buf == 1) {  // odd number of passes: the result is in the scratch copy
        e = cudaMemcpyAsync(keys_out, sc.keys[1], sizeof(uint64_t) * (size_t)count,
                            cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(vals_out, sc.vals[1], sizeof(uint32_t) * (size_t)count,
                                cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return PGS_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? PGS_OK : PGS_ERR_CUDA;
}

extern "C" int pgs_sort_pairs_static_status(void* cuda_stream) {
    unsigned char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != PGS_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int32_t st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, base + kOffStatus, sizeof(st), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffStatus, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return PGS_ERR_CUDA;
    return (st & kStatusInternal) ? PGS_ERR_INTERNAL : PGS_OK;
}
