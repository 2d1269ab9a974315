// CSR SpMV of the AMG hierarchy's smaller levels and transfer operators: L
// lanes per row, the same output modes as the SELL-32 kernel (level_spmv.cuh,
// included first). Included by amg.cu only.
#pragma once

#include "level_spmv.cuh"

namespace dpp {
namespace {

// MODE 0: y = A x; 1: y = b - A x; 2: y = y + A x; 3: Chebyshev step (above).
// T: values, vectors and arithmetic.
// L lanes share a row; each lane walks its entries U at a time (4 in FP64, 8
// in FP32), so that several gathers are in flight; FP32 keeps U partial sums,
// FP64 one accumulator (the FP64 pipe is a limit, and partial sums cost adds).
template <int L, int MODE, class T>
__global__ void __launch_bounds__(256) k_csr_spmv(int64_t n_rows, const int* __restrict__ rp,
                                                  const int* __restrict__ col,
                                                  const T* __restrict__ val,
                                                  const T* __restrict__ x,
                                                  const T* __restrict__ b, T* __restrict__ y,
                                                  ChebOut<T> ch) {
    constexpr int U = sizeof(T) == 4 ? 8 : 4;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = t / L;
    const int lane = (int)(t % L);
    const bool active = row < n_rows;  // inactive lanes still join the shuffles
    T a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) a[u] = T(0);
    if (active) {
        int p = rp[row] + lane;
        const int e = rp[row + 1];
        for (; p + (U - 1) * L < e; p += U * L) {
            int c[U];
            T v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                c[u] = col[p + u * L];
                v[u] = val[p + u * L];
            }
            T xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) xv[u] = __ldg(x + c[u]);
            if constexpr (sizeof(T) == 8) {  // FP64: one accumulator (no partial sums to add)
#pragma unroll
                for (int u = 0; u < U; ++u) a[0] = fma(v[u], xv[u], a[0]);
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) a[u] += v[u] * xv[u];
            }
        }
        for (; p < e; p += L) a[0] += val[p] * __ldg(x + col[p]);
    }
    if constexpr (sizeof(T) != 8) {
#pragma unroll
        for (int w = U / 2; w > 0; w >>= 1)
#pragma unroll
            for (int u = 0; u < w; ++u) a[u] += a[u + w];
    }
    T acc = a[0];
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, L);
    if (active && lane == 0) spmv_out<MODE, T>(row, acc, x, b, y, ch);
}

}  // namespace
}  // namespace dpp
