// SELL-32 SpMV of the AMG hierarchy's large levels (one thread per row, one or
// two warps per slice), with the Chebyshev step of the smoother fused into its
// residual (MODE 3), and the output modes it shares with the CSR kernel
// (csr_spmv.cuh). Included by amg.cu only.
#pragma once

#include <cstdint>

namespace dpp {
namespace {

// ------------------------------------------------------------------ output modes
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

// RES: for MODE 1 and 3, acc already holds the residual b - A x (the FP64 SELL
// kernel starts its accumulator at b and subtracts the products).
template <int MODE, class T, bool RES = false>
__device__ __forceinline__ void spmv_out(int64_t row, T acc, const T* __restrict__ x, const T* __restrict__ b,
                                         T* __restrict__ y, const ChebOut<T>& ch) {
    if (MODE == 0) y[row] = acc;
    else if (MODE == 1) y[row] = RES ? acc : b[row] - acc;
    else if (MODE == 2) y[row] += acc;
    else {
        const T r = RES ? acc : b[row] - acc;
        const T dn = (ch.c1 != T(0) ? ch.c1 * ch.d[row] : T(0)) + ch.c2 * ch.dinv[row] * r;
        ch.d[row] = dn;
        ch.xo[row] = x[row] + dn;
    }
}

// ------------------------------------------------------------------ SELL-32 SpMV
// One thread per row; a warp owns a slice, so every column and value load of
// the warp is one contiguous 128 B (int, float) or 256 B (double) transaction.
// U gathers are kept in flight: 4 in FP64 (the FP64 pipe is the other limit
// there), 8 in FP32 with U partial sums; FP64 sums into one accumulator,
// which saves the adds of the partial sums. Same MODEs as k_csr_spmv.
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
    // FP64 residual modes: the first warp of the slice starts at b, and the
    // products are subtracted (one multiply-add each, no separate b - A x: the
    // FP64 pipe is a limit here; in FP32 the early load of b measured slower)
    constexpr bool RES = sizeof(T) == 8 && (MODE == 1 || MODE == 3);
    constexpr T sgn = RES ? T(-1) : T(1);
    T a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) a[u] = T(0);
    if (RES && live && h == 0) a[0] = b[row];
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
            T xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) xv[u] = __ldg(x + c[u]);
            if constexpr (sizeof(T) == 8) {
                // FP64: one accumulator, so no partial sums to add up per row (the
                // FP64 pipe is a limit here); the U gathers are still in flight together
#pragma unroll
                for (int u = 0; u < U; ++u) a[0] = fma(sgn * v[u], xv[u], a[0]);
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) a[u] = fma(sgn * v[u], xv[u], a[u]);
            }
        }
        for (; p < e; p += S) a[0] = fma(sgn * val[p], __ldg(x + column(p)), a[0]);
    }
    if constexpr (sizeof(T) != 8) {
#pragma unroll
        for (int w = U / 2; w > 0; w >>= 1)
#pragma unroll
            for (int u = 0; u < w; ++u) a[u] += a[u + w];
    }
    T acc = a[0];
    if (H > 1) {
        if (h == 1) part[warp / H][lane] = acc;
        __syncthreads();
        if (h == 1) return;
        acc += part[warp / H][lane];
    }
    if (!live) return;
    spmv_out<MODE, T, RES>(row, acc, x, b, y, ch);
}

}  // namespace
}  // namespace dpp
