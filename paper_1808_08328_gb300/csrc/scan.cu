// Device-wide exclusive prefix sum over int32 counts (setup kernels only).
// Three phases: per-block scan with block totals, a recursive scan of the
// totals, then a uniform add. Deterministic.
#include "common.cuh"

namespace dpp {

namespace {
constexpr int kScanBlock = 512;
constexpr int kScanItems = 4;  // items per thread
constexpr int kScanTile = kScanBlock * kScanItems;

__global__ void k_scan_tiles(const int* __restrict__ in, int* __restrict__ out, int64_t n,
                             int* __restrict__ tile_sums) {
    __shared__ int sh[kScanBlock];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int tsum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t k = base + i;
        v[i] = (k < n) ? in[k] : 0;
        tsum += v[i];
    }
    sh[threadIdx.x] = tsum;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {  // Hillis-Steele inclusive scan
        int t = (threadIdx.x >= off) ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    int run = sh[threadIdx.x] - tsum;  // exclusive prefix of this thread
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t k = base + i;
        if (k < n) out[k] = run;
        run += v[i];
    }
    if (threadIdx.x == kScanBlock - 1) tile_sums[blockIdx.x] = sh[threadIdx.x];
}

__global__ void k_add_tile_offsets(int* __restrict__ out, int64_t n, const int* __restrict__ offs) {
    int64_t k = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
    int add = offs[blockIdx.x];
    for (int i = 0; i < kScanItems; ++i, k += kScanBlock)
        if (k < n && k < (int64_t)(blockIdx.x + 1) * kScanTile) out[k] += add;
}

void scan_rec(const int* in, int* out, int64_t n, cudaStream_t s) {
    int64_t tiles = (n + kScanTile - 1) / kScanTile;
    DBuf<int> sums(tiles + 1);
    k_scan_tiles<<<(unsigned)tiles, kScanBlock, 0, s>>>(in, out, n, sums.get());
    DPP_LAUNCH_CK();
    if (tiles > 1) {
        DBuf<int> offs(tiles + 1);
        scan_rec(sums.get(), offs.get(), tiles, s);
        k_add_tile_offsets<<<(unsigned)tiles, kScanBlock, 0, s>>>(out, n, offs.get());
        DPP_LAUNCH_CK();
        DPP_CK(cudaStreamSynchronize(s));  // keep the temporaries alive until done
    } else {
        DPP_CK(cudaStreamSynchronize(s));
    }
}

// Sum of the (non-negative) counts in 64 bits, so that a total the int32
// prefix sums cannot hold is detected instead of wrapping.
__global__ void k_sum64(const int* __restrict__ in, int64_t n, unsigned long long* total) {
    unsigned long long acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        acc += (unsigned long long)(unsigned)in[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(total, acc);
}
}  // namespace

int64_t exclusive_scan(const int* in, int* out, int64_t n, cudaStream_t s, HostScratch& hs) {
    if (n <= 0) return 0;
    // The total is taken before a possibly aliasing scan overwrites the input.
    DBuf<unsigned long long> total(1);
    DPP_CK(cudaMemsetAsync(total.get(), 0, sizeof(unsigned long long), s));
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4 * kSMs);
    k_sum64<<<(unsigned)blocks, 256, 0, s>>>(in, n, total.get());
    DPP_LAUNCH_CK();
    scan_rec(in, out, n, s);
    const unsigned long long t = read_scalar(total.get(), s, hs);
    if (t > (unsigned long long)INT32_MAX)
        fail(DPP_ERR_INVALID_ARGUMENT, "a matrix has 2^31 or more nonzeros (int32 row pointers)");
    return (int64_t)t;
}

}  // namespace dpp
