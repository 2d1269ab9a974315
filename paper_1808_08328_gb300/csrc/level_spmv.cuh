// Level SpMV kernels of the AMG hierarchy: CSR with L lanes per row and
// SELL-32 (one thread per row, one or two warps per slice), each with the
// Chebyshev step of the smoother fused into its residual (MODE 3). Included
// by amg.cu only.
#pragma once

#include <cstdint>

namespace dpp {
namespace {

// ------------------------------------------------------------------ CSR SpMV
// Chebyshev step fused into the residual SpMV (MODE 3): with r = b - A x,
// d = c1 d + c2 Dinv r and xo = x + d, written to xo (not x, which other rows
// still read). c1 = 0 does not read d.
template <class T>
struct ChebOut {
    const T* dinv = nullptr;
    T* d = nullptr;
    T* xo = nullptr;
    T c1 = T(0), c2 = T(0);
};

template <int MODE, class T>
__device__ __forceinline__ void spmv_out(int64_t row, T acc, const T* __restrict__ x, const T* __restrict__ b,
                                         T* __restrict__ y, const ChebOut<T>& ch) {
    if (MODE == 0) y[row] = acc;
    else if (MODE == 1) y[row] = b[row] - acc;
    else if (MODE == 2) y[row] += acc;
    else {
        const T r = b[row] - acc;
        const T dn = (ch.c1 != T(0) ? ch.c1 * ch.d[row] : T(0)) + ch.c2 * ch.dinv[row] * r;
        ch.d[row] = dn;
        ch.xo[row] = x[row] + dn;
    }
}

// MODE 0: y = A x; 1: y = b - A x; 2: y = y + A x; 3: Chebyshev step (above).
// T: values, vectors and arithmetic.
// L lanes share a row; each lane walks its entries four at a time with four
// independent partial sums, so that several gathers are in flight.
template <int L, int MODE, class T>
__global__ void __launch_bounds__(256) k_csr_spmv(int64_t n_rows, const int* __restrict__ rp,
                                                  const int* __restrict__ col,
                                                  const T* __restrict__ val,
                                                  const T* __restrict__ x,
                                                  const T* __restrict__ b, T* __restrict__ y,
                                                  ChebOut<T> ch) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = t / L;
    const int lane = (int)(t % L);
    const bool active = row < n_rows;  // inactive lanes still join the shuffles
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    if (active) {
        int p = rp[row] + lane;
        const int e = rp[row + 1];
        for (; p + 3 * L < e; p += 4 * L) {
            const int c0 = col[p], c1 = col[p + L], c2 = col[p + 2 * L], c3 = col[p + 3 * L];
            const T v0 = val[p], v1 = val[p + L], v2 = val[p + 2 * L], v3 = val[p + 3 * L];
            a0 += v0 * __ldg(x + c0);
            a1 += v1 * __ldg(x + c1);
            a2 += v2 * __ldg(x + c2);
            a3 += v3 * __ldg(x + c3);
        }
        for (; p < e; p += L) a0 += val[p] * __ldg(x + col[p]);
    }
    T acc = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, L);
    if (active && lane == 0) spmv_out<MODE, T>(row, acc, x, b, y, ch);
}

// ------------------------------------------------------------------ SELL-32 SpMV
// One thread per row; a warp owns a slice, so every column and value load of
// the warp is one contiguous 128 B (int, float) or 256 B (double) transaction.
// U partial sums keep U gathers in flight: 4 in FP64 (the FP64 pipe is the
// other limit there), 8 in FP32. Same MODEs as k_csr_spmv.
//
// H warps may share a slice (H = 2 in FP32): warp h takes the slots
// h, h + H, ... of every row, and the partial sums meet in shared memory.
//
// C16: the column of a slot is base[slice] + col16[slot] (16-bit offsets from
// the slice's smallest column), 2 bytes per nonzero instead of 4.
template <int MODE, class T, int H, bool C16 = false>
__global__ void __launch_bounds__(256) k_sell_spmv(int64_t n_rows, const int* __restrict__ off,
                                                   const int* __restrict__ col,
                                                   const T* __restrict__ val,
                                                   const T* __restrict__ x,
                                                   const T* __restrict__ b, T* __restrict__ y,
                                                   ChebOut<T> ch,
                                                   const int* __restrict__ base = nullptr,
                                                   const uint16_t* __restrict__ col16 = nullptr) {
    constexpr int U = sizeof(T) == 4 ? 8 : 4;
    constexpr int SPB = 8 / H;  // slices per 256-thread block
    static_assert(H == 1 || H == 2, "one or two warps per slice");
    __shared__ T part[H > 1 ? SPB : 1][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, h = warp % H;
    const int64_t sl = (int64_t)blockIdx.x * SPB + warp / H;
    const int64_t row = sl * 32 + lane;
    const bool live = row < n_rows;
    T a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) a[u] = T(0);
    if (live) {
        const int e = off[sl + 1];
        int p = off[sl] + 32 * h + lane;
        constexpr int S = 32 * H;  // stride between this warp's slots
        const int c0 = C16 ? base[sl] : 0;
        auto column = [&](int q) -> int { return C16 ? c0 + (int)col16[q] : col[q]; };
        for (; p + S * (U - 1) < e; p += S * U) {
            int c[U];
            T v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                c[u] = column(p + S * u);
                v[u] = val[p + S * u];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) a[u] += v[u] * __ldg(x + c[u]);
        }
        for (; p < e; p += S) a[0] += val[p] * __ldg(x + column(p));
    }
#pragma unroll
    for (int w = U / 2; w > 0; w >>= 1)
#pragma unroll
        for (int u = 0; u < w; ++u) a[u] += a[u + w];
    T acc = a[0];
    if (H > 1) {
        if (h == 1) part[warp / H][lane] = acc;
        __syncthreads();
        if (h == 1) return;
        acc += part[warp / H][lane];
    }
    if (!live) return;
    spmv_out<MODE, T>(row, acc, x, b, y, ch);
}

}  // namespace
}  // namespace dpp
