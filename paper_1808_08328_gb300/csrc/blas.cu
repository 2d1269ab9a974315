// Vector kernels for the Krylov solver: dot products, the multi-dot and
// multi-update of classical Gram-Schmidt (run twice, CGS2), and simple
// updates. Reductions are deterministic: each of kRedBlocks blocks writes one
// partial in a fixed order, and the last block to finish (found with a
// device-scope counter) sums the partials in index order. No floating-point
// atomics are used.
#include "kernels.cuh"

namespace dpp {

void Reducer::ensure(int rows, cudaStream_t s) {
    if ((int64_t)partial.n < (int64_t)rows * kRedBlocks) partial.alloc((size_t)rows * kRedBlocks);
    if (!counter.get()) {
        counter.alloc(64);
        // reset on s, the stream that uses it (the legacy stream would not
        // wait for work on a non-blocking one)
        DPP_CK(cudaMemsetAsync(counter.get(), 0, 64 * sizeof(unsigned), s));
    }
}

namespace {

constexpr int kRedThreads = 256;

// Blocks reduce a grid-stride range; the last block to finish sums the partials.
__global__ void __launch_bounds__(kRedThreads) k_dot(const double* __restrict__ x,
                                                     const double* __restrict__ y, int64_t n,
                                                     double* __restrict__ partial,
                                                     unsigned* counter, double* out) {
    __shared__ double sh[kRedThreads / 32];
    __shared__ bool last;
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // two independent accumulators for memory-level parallelism
    double acc2 = 0.0;
    for (; i + stride < n; i += 2 * stride) {
        acc += x[i] * y[i];
        acc2 += x[i + stride] * y[i + stride];
    }
    if (i < n) acc += x[i] * y[i];
    acc += acc2;
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = acc;
        __threadfence();
        unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (int k = threadIdx.x; k < gridDim.x; k += blockDim.x) v += ((volatile double*)partial)[k];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) {
        *out = v;
        *counter = 0u;
    }
}

// grid (kRedBlocks, k): partial[j][blk]
__global__ void __launch_bounds__(kRedThreads) k_multidot(const double* __restrict__ V, int64_t ld,
                                                          const double* __restrict__ w, int64_t n,
                                                          double* __restrict__ partial) {
    __shared__ double sh[kRedThreads / 32];
    const int j = blockIdx.y;
    const double* v = V + (int64_t)j * ld;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double acc = 0.0, acc2 = 0.0;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + stride < n; i += 2 * stride) {
        acc += v[i] * w[i];
        acc2 += v[i + stride] * w[i + stride];
    }
    if (i < n) acc += v[i] * w[i];
    acc = block_sum(acc + acc2, sh);
    if (threadIdx.x == 0) partial[(int64_t)j * gridDim.x + blockIdx.x] = acc;
}

__global__ void k_finish_rows(const double* __restrict__ partial, int nblk, double* __restrict__ out) {
    __shared__ double sh[kRedThreads / 32];
    const int j = blockIdx.x;
    double v = 0.0;
    for (int k = threadIdx.x; k < nblk; k += blockDim.x) v += partial[(int64_t)j * nblk + k];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) out[j] = v;
}

__global__ void k_multi_axpy(const double* __restrict__ V, int64_t ld, int k,
                             const double* __restrict__ h, double* __restrict__ w, int64_t n,
                             double sign) {
    __shared__ double hs[64];
    if (threadIdx.x < k) hs[threadIdx.x] = h[threadIdx.x];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double acc = 0.0;
        for (int j = 0; j < k; ++j) acc += hs[j] * V[(int64_t)j * ld + i];
        w[i] += sign * acc;
    }
}

__global__ void k_multi_axpy_f32(const float* __restrict__ Z, int64_t ld, int k,
                                 const double* __restrict__ h, double* __restrict__ x, int64_t n) {
    __shared__ double hs[64];
    if (threadIdx.x < k) hs[threadIdx.x] = h[threadIdx.x];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double acc = 0.0;
        for (int j = 0; j < k; ++j) acc += hs[j] * (double)Z[(int64_t)j * ld + i];
        x[i] += acc;
    }
}

__global__ void k_scale_copy(const double* __restrict__ x, double* __restrict__ y, int64_t n,
                             const double* __restrict__ num, const double* __restrict__ den) {
    const double a = den ? (*num / *den) : *num;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        y[i] = a * x[i];
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y,
                        int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        y[i] = (b == 0.0) ? a * x[i] : a * x[i] + b * y[i];  // b = 0: y is not read (may be unset)
}

__global__ void k_fill(double* __restrict__ x, double v, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) x[i] = v;
}

__global__ void k_to_float_v(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = (float)in[i];
}

inline int stream_grid(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (int)std::min<int64_t>(std::max<int64_t>(g, 1), 8 * kSMs);
}

}  // namespace

void dot(Reducer& R, const double* x, const double* y, int64_t n, double* out, cudaStream_t s) {
    R.ensure(1, s);
    k_dot<<<kRedBlocks, kRedThreads, 0, s>>>(x, y, n, R.partial.get(), R.counter.get(), out);
    DPP_LAUNCH_CK();
}

void multidot(Reducer& R, const double* V, int64_t ld, int k, const double* w, int64_t n,
              double* out, cudaStream_t s) {
    if (k <= 0) return;
    R.ensure(k, s);
    dim3 grid(kRedBlocks, k);
    k_multidot<<<grid, kRedThreads, 0, s>>>(V, ld, w, n, R.partial.get());
    DPP_LAUNCH_CK();
    k_finish_rows<<<k, kRedThreads, 0, s>>>(R.partial.get(), kRedBlocks, out);
    DPP_LAUNCH_CK();
}

void multi_axpy_sub(const double* V, int64_t ld, int k, const double* h, double* w, int64_t n,
                    cudaStream_t s) {
    if (k <= 0) return;
    if (k > 64) fail(DPP_ERR_INVALID_ARGUMENT, "multi_axpy: k > 64");
    k_multi_axpy<<<stream_grid(n), 256, 0, s>>>(V, ld, k, h, w, n, -1.0);
    DPP_LAUNCH_CK();
}

void multi_axpy_add(const double* Z, int64_t ld, int k, const double* y, double* x, int64_t n,
                    cudaStream_t s) {
    if (k <= 0) return;
    if (k > 64) fail(DPP_ERR_INVALID_ARGUMENT, "multi_axpy: k > 64");
    k_multi_axpy<<<stream_grid(n), 256, 0, s>>>(Z, ld, k, y, x, n, 1.0);
    DPP_LAUNCH_CK();
}

void multi_axpy_add_f32(const float* Z, int64_t ld, int k, const double* y, double* x, int64_t n,
                        cudaStream_t s) {
    if (k <= 0) return;
    if (k > 64) fail(DPP_ERR_INVALID_ARGUMENT, "multi_axpy: k > 64");
    k_multi_axpy_f32<<<stream_grid(n), 256, 0, s>>>(Z, ld, k, y, x, n);
    DPP_LAUNCH_CK();
}

void scale_copy(const double* x, double* y, int64_t n, const double* num, const double* den,
                cudaStream_t s) {
    k_scale_copy<<<stream_grid(n), 256, 0, s>>>(x, y, n, num, den);
    DPP_LAUNCH_CK();
}

void axpby(double a, const double* x, double b, double* y, int64_t n, cudaStream_t s) {
    k_axpby<<<stream_grid(n), 256, 0, s>>>(a, x, b, y, n);
    DPP_LAUNCH_CK();
}

void fill(double* x, double v, int64_t n, cudaStream_t s) {
    k_fill<<<stream_grid(n), 256, 0, s>>>(x, v, n);
    DPP_LAUNCH_CK();
}

void to_float(const double* in, float* out, int64_t n, cudaStream_t s) {
    k_to_float_v<<<stream_grid(n), 256, 0, s>>>(in, out, n);
    DPP_LAUNCH_CK();
}

}  // namespace dpp
