// Internal helpers shared by the libdpp translation units: error handling,
// device buffers, launch geometry and warp/block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/dpp.h"

namespace dpp {

// Exceptions are the internal error path; every extern "C" entry point catches
// them and turns them into a dpp_status plus a thread-local message.
struct Error : std::runtime_error {
    dpp_status status;
    Error(dpp_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define DPP_CK(call)                                                                    \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            throw ::dpp::Error(e_ == cudaErrorMemoryAllocation ? DPP_ERR_OUT_OF_MEMORY  \
                                                               : DPP_ERR_CUDA,          \
                               std::string(#call) + ": " + cudaGetErrorString(e_));     \
        }                                                                               \
    } while (0)

// Checks the launch just issued and counts it (see dpp_launch_count).
#define DPP_LAUNCH_CK()                       \
    do {                                      \
        DPP_CK(cudaGetLastError());           \
        ::dpp::count_launch();                \
    } while (0)

inline void fail(dpp_status s, const std::string& m) { throw Error(s, m); }

// Launch accounting and optional per-family CUDA-event timing (abi.cu).
void count_launch();
bool profiling_enabled();
bool profiling_selected(const char* family);  // enabled and in the dpp_profile_select list
void profile_record(const char* family, cudaEvent_t start, cudaEvent_t stop, double alg_bytes);
// A timing event from a per-device pool that dpp_profile_enable recycles
// (nullptr on failure); creating events in the timed path would cost more
// host time than the launches being timed.
cudaEvent_t profile_event();

// Times everything issued on `s` inside its scope when profiling is enabled.
struct ProfScope {
    const char* fam = nullptr;
    cudaStream_t s = nullptr;
    double bytes = 0;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(const char* family, cudaStream_t st, double alg_bytes) {
        if (!profiling_enabled() || !profiling_selected(family)) return;
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
            return;  // no event records inside a graph capture
        fam = family;
        s = st;
        bytes = alg_bytes;
        a = profile_event();
        b = profile_event();
        if (!a || !b) { fam = nullptr; return; }
        cudaEventRecord(a, s);
    }
    ~ProfScope() { stop(); }
    // End the timed range now; the record is made by stop(), so the algorithmic
    // bytes may still be set in between (for outputs whose size is known later).
    void end_range() {
        if (!fam || ended) return;
        cudaEventRecord(b, s);
        ended = true;
    }
    void stop() {  // end the timed range early (idempotent)
        if (!fam) return;
        end_range();
        profile_record(fam, a, b, bytes);
        fam = nullptr;
    }
    bool ended = false;
};

// Device memory comes from a library-owned, stream-ordered CUDA memory pool
// (one per device, created on first use, which keeps freed memory for reuse):
// an allocation or a free is an operation on the stream of the API call in
// progress (stream_scope below), with no device-wide synchronisation. Outside
// any API call the legacy default stream is used. Allocating on a stream that
// is being captured into a CUDA graph is an error: graph captures must find
// their buffers already allocated.
void* pool_alloc(size_t bytes);
void pool_free(void* p);
cudaStream_t& current_stream();  // thread-local

// Makes `s` the stream of pool allocations and frees for the scope's lifetime.
struct StreamScope {
    cudaStream_t prev;
    explicit StreamScope(cudaStream_t s) : prev(current_stream()) { current_stream() = s; }
    ~StreamScope() { current_stream() = prev; }
    StreamScope(const StreamScope&) = delete;
    StreamScope& operator=(const StreamScope&) = delete;
};

// Owning device buffer, allocated from and returned to the pool in stream
// order (see pool_alloc).
template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    DBuf() = default;
    explicit DBuf(size_t count) { alloc(count); }
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(size_t count) {
        release();
        n = count;
        if (count) p = static_cast<T*>(pool_alloc(count * sizeof(T)));
    }
    void release() {
        if (p) pool_free(p);
        p = nullptr;
        n = 0;
    }
    T* get() const { return p; }
    size_t bytes() const { return n * sizeof(T); }
};

// Pinned host scratch for small device->host reads.
struct HostScratch {
    void* p = nullptr;
    size_t cap = 0;
    void* get(size_t bytes) {
        if (bytes > cap) {
            if (p) cudaFreeHost(p);
            DPP_CK(cudaMallocHost(&p, bytes));
            cap = bytes;
        }
        return p;
    }
    ~HostScratch() { if (p) cudaFreeHost(p); }
};

constexpr int kSMs = 152;        // GB300: 2 dies x 76 SMs
constexpr int kSell = 32;        // SELL slice height = one warp

inline int grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > (1LL << 30)) g = (1LL << 30);
    return (int)g;
}

// Device status word codes (OR-ed by validation kernels).
enum : int {
    kDevOk = 0,
    kDevBadIndex = 1,
    kDevNonFinite = 2,
    kDevDegenerate = 4,
    kDevOverflow = 8,     // a per-node list exceeded its compile-time bound
    kDevNoOwner = 16,     // a boundary facet is not a face of any cell
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum, result valid in thread 0. `sh` needs blockDim/32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0) v = warp_sum(v);
    __syncthreads();
    return v;
}

// ------------------------------------------------------------------ host helpers

// Exclusive prefix sum of n ints (in may alias out); returns the total.
int64_t exclusive_scan(const int* in, int* out, int64_t n, cudaStream_t s, HostScratch& hs);
// Read one device value.
template <class T>
T read_scalar(const T* d, cudaStream_t s, HostScratch& hs) {
    T* h = (T*)hs.get(sizeof(T));
    DPP_CK(cudaMemcpyAsync(h, d, sizeof(T), cudaMemcpyDeviceToHost, s));
    DPP_CK(cudaStreamSynchronize(s));
    return *h;
}

}  // namespace dpp
