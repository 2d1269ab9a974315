// Node-pair operators on the SELL-32 storage (the hot SpMV of the solve).
//
// K (Eq. "S4_cg_stiffness_matrix") couples node a to node b through one
// (2d+2) x (2d+2) block built from the pair values m1, m2, Kup[d], Kpu[d],
// d1, d2, e:
//   rows u1_i: m1 x_u1_i + Kup_i x_p1      rows u2_i: m2 x_u2_i + Kup_i x_p2
//   row  p1  : Kpu . x_u1 + d1 x_p1 + e x_p2
//   row  p2  : Kpu . x_u2 + d2 x_p2 + e x_p1
// K^T is the same operator with Kup and Kpu negated. The reasons: K_pu =
// -K_up^T, and the mass, K_pp and coupling blocks are symmetric.
//
// Layout: one thread per node row. A warp covers the 32 rows of one SELL
// slice, so every value and column load is one coalesced 128-256 B
// transaction. x is gathered per column node as (2d+2) contiguous values.
//
// Precision: the FP64 path keeps values, vectors and arithmetic in FP64. The
// mixed path (FP32 values, FP32 preconditioner vectors) does its arithmetic in
// FP32. On GB300 the FP64 pipe, not HBM, bounds the FP64 kernels; the FP32
// kernels are HBM-bound.
#include <type_traits>

#include "kernels.cuh"

namespace dpp {

namespace {

// (2d+2)-value node loads and stores with the widest aligned vector type.
template <int NS>
__device__ __forceinline__ void load_node(const double* __restrict__ x, int64_t b, double (&v)[NS]) {
    const double2* p = reinterpret_cast<const double2*>(x + b * NS);
#pragma unroll
    for (int k = 0; k < NS / 2; ++k) {
        double2 t = __ldg(p + k);
        v[2 * k] = t.x;
        v[2 * k + 1] = t.y;
    }
}
template <int NS>
__device__ __forceinline__ void load_node(const float* __restrict__ x, int64_t b, float (&v)[NS]) {
    if constexpr (NS % 4 == 0) {
        const float4* p = reinterpret_cast<const float4*>(x + b * NS);
#pragma unroll
        for (int k = 0; k < NS / 4; ++k) {
            float4 t = __ldg(p + k);
            v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
        }
    } else {
        const float2* p = reinterpret_cast<const float2*>(x + b * NS);
#pragma unroll
        for (int k = 0; k < NS / 2; ++k) {
            float2 t = __ldg(p + k);
            v[2 * k] = t.x; v[2 * k + 1] = t.y;
        }
    }
}
template <int NS, class T>
__device__ __forceinline__ void load_node_as(const T* __restrict__ x, int64_t b, float (&v)[NS]) {
    if constexpr (std::is_same<T, float>::value) {
        load_node<NS>(x, b, v);
    } else {
        double t[NS];
        load_node<NS>(x, b, t);
#pragma unroll
        for (int k = 0; k < NS; ++k) v[k] = (float)t[k];
    }
}
template <int NS, class T>
__device__ __forceinline__ void load_node_as(const T* __restrict__ x, int64_t b, double (&v)[NS]) {
    if constexpr (std::is_same<T, double>::value) {
        load_node<NS>(x, b, v);
    } else {
        float t[NS];
        load_node<NS>(x, b, t);
#pragma unroll
        for (int k = 0; k < NS; ++k) v[k] = (double)t[k];
    }
}

template <int NS, class AT>
__device__ __forceinline__ void store_node(double* __restrict__ y, int64_t a, const AT (&v)[NS]) {
    double2* p = reinterpret_cast<double2*>(y + a * NS);
#pragma unroll
    for (int k = 0; k < NS / 2; ++k) p[k] = make_double2((double)v[2 * k], (double)v[2 * k + 1]);
}
template <int NS, class AT>
__device__ __forceinline__ void store_node(float* __restrict__ y, int64_t a, const AT (&v)[NS]) {
    if constexpr (NS % 4 == 0) {
        float4* p = reinterpret_cast<float4*>(y + a * NS);
#pragma unroll
        for (int k = 0; k < NS / 4; ++k)
            p[k] = make_float4((float)v[4 * k], (float)v[4 * k + 1], (float)v[4 * k + 2],
                               (float)v[4 * k + 3]);
    } else {
        float2* p = reinterpret_cast<float2*>(y + a * NS);
#pragma unroll
        for (int k = 0; k < NS / 2; ++k) p[k] = make_float2((float)v[2 * k], (float)v[2 * k + 1]);
    }
}

// y = K x (or b - K x). Arithmetic in FP32 when both values and x are FP32.
// H warps share a slice (H = 1 or 2): warp h takes the column groups
// g0 + h, g0 + h + H, ..., and warp 1's partial sums are added to warp 0's
// through shared memory (fixed order). H = 2 doubles the loads in flight when
// one thread per node row leaves most of the GPU idle.
template <int DIM, class VT, class XT, class YT, bool TRANS, bool RESID, int H>
__global__ void __launch_bounds__(128) k_apply_K(int64_t n_rows, int64_t n_slices,
                                                 const int* __restrict__ slice_ptr,
                                                 const int* __restrict__ sell_col,
                                                 const VT* __restrict__ val,
                                                 const XT* __restrict__ x,
                                                 const YT* __restrict__ b, YT* __restrict__ y) {
    using AT = typename std::conditional<std::is_same<VT, float>::value &&
                                             std::is_same<XT, float>::value,
                                         float, double>::type;
    constexpr int NS = 2 * DIM + 2;
    constexpr int NV = pair_values(DIM);
    constexpr int SPB = 4 / H;  // slices per 128-thread block
    static_assert(H == 1 || H == 2, "one or two warps per slice");
    __shared__ AT part[H > 1 ? SPB : 1][NS][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, h = warp % H;
    const int64_t s = (int64_t)blockIdx.x * SPB + warp / H;
    const bool live = s < n_slices;
    const int64_t a = s * 32 + lane;
    AT acc[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) acc[k] = AT(0);
    const int g0 = live ? slice_ptr[s] + h : 0, g1 = live ? slice_ptr[s + 1] : 0;
    for (int g = g0; g < g1; g += H) {
        const int cb = sell_col[(int64_t)g * kSell + lane];
        if (cb < 0) continue;
        const VT* v = val + (int64_t)g * NV * kSell + lane;
        const AT m1 = (AT)v[0], m2 = (AT)v[kSell];
        AT bu[DIM], cu[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            bu[k] = (AT)v[(2 + k) * kSell];
            cu[k] = (AT)v[(2 + DIM + k) * kSell];
            if (TRANS) { bu[k] = -bu[k]; cu[k] = -cu[k]; }
        }
        const AT d1 = (AT)v[(2 + 2 * DIM) * kSell];
        const AT d2 = (AT)v[(3 + 2 * DIM) * kSell];
        const AT e = (AT)v[(4 + 2 * DIM) * kSell];
        AT xb[NS];
        load_node_as<NS, XT>(x, cb, xb);
        const AT p1 = xb[DIM], p2 = xb[2 * DIM + 1];
        // every term is a multiply-add straight into its accumulator (22 per pair
        // in 3D): in FP64 the pipe, not memory, bounds this kernel
        acc[DIM] = fma(d1, p1, acc[DIM]);
        acc[DIM] = fma(e, p2, acc[DIM]);
        acc[2 * DIM + 1] = fma(d2, p2, acc[2 * DIM + 1]);
        acc[2 * DIM + 1] = fma(e, p1, acc[2 * DIM + 1]);
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            acc[k] = fma(m1, xb[k], acc[k]);
            acc[k] = fma(bu[k], p1, acc[k]);
            acc[DIM + 1 + k] = fma(m2, xb[DIM + 1 + k], acc[DIM + 1 + k]);
            acc[DIM + 1 + k] = fma(bu[k], p2, acc[DIM + 1 + k]);
            acc[DIM] = fma(cu[k], xb[k], acc[DIM]);
            acc[2 * DIM + 1] = fma(cu[k], xb[DIM + 1 + k], acc[2 * DIM + 1]);
        }
    }
    if (H > 1) {
        if (h == 1)
#pragma unroll
            for (int k = 0; k < NS; ++k) part[warp / H][k][lane] = acc[k];
        __syncthreads();
        if (h == 1) return;
#pragma unroll
        for (int k = 0; k < NS; ++k) acc[k] += part[warp / H][k][lane];
    }
    if (!live || a >= n_rows) return;
    if (RESID) {
        double out[NS], bb[NS];
        load_node_as<NS, YT>(b, a, bb);
#pragma unroll
        for (int k = 0; k < NS; ++k) out[k] = bb[k] - (double)acc[k];
        store_node<NS>(y, a, out);
    } else {
        store_node<NS>(y, a, acc);
    }
}

// Chebyshev step on A = blockdiag(K1_uu, K2_uu); each velocity component of
// network i sees the same scalar matrix with entries m_i. T: vector and
// arithmetic type; the values have the same type.
template <int DIM, class T, int H>
__global__ void __launch_bounds__(128) k_mass_cheb(int64_t n_rows, int64_t n_slices,
                                                   const int* __restrict__ slice_ptr,
                                                   const int* __restrict__ sell_col,
                                                   const T* __restrict__ val,
                                                   const T* __restrict__ mdiag,
                                                   const T* __restrict__ r,
                                                   const T* __restrict__ xin,
                                                   T* __restrict__ xout, T* __restrict__ d,
                                                   T c1, T c2, int first) {
    constexpr int NS = 2 * DIM + 2;
    constexpr int NV = pair_values(DIM);
    constexpr int SPB = 4 / H;  // slices per 128-thread block (H warps per slice, as in k_apply_K)
    static_assert(H == 1 || H == 2, "one or two warps per slice");
    __shared__ T part[H > 1 ? SPB : 1][NS][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, h = warp % H;
    const int64_t s = (int64_t)blockIdx.x * SPB + warp / H;
    const bool live = s < n_slices;
    const int64_t a = s * 32 + lane;
    // acc starts at the row's right-hand side (warp 0 of the slice) and the
    // products are subtracted, so that acc ends as the residual r - A x with
    // one multiply-add per product and no separate subtraction
    T acc[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) acc[k] = T(0);
    if (!first && live && h == 0 && a < n_rows) load_node<NS>(r, a, acc);
    if (!first && live) {
        const int g0 = slice_ptr[s] + h, g1 = slice_ptr[s + 1];
        for (int g = g0; g < g1; g += H) {
            const int cb = sell_col[(int64_t)g * kSell + lane];
            if (cb < 0) continue;
            const T* v = val + (int64_t)g * NV * kSell + lane;
            const T m1 = v[0], m2 = v[kSell];
            T xb[NS];
            load_node<NS>(xin, cb, xb);
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                acc[k] = fma(-m1, xb[k], acc[k]);
                acc[DIM + 1 + k] = fma(-m2, xb[DIM + 1 + k], acc[DIM + 1 + k]);
            }
        }
    }
    if (H > 1) {
        if (h == 1)
#pragma unroll
            for (int k = 0; k < NS; ++k) part[warp / H][k][lane] = acc[k];
        __syncthreads();
        if (h == 1) return;
#pragma unroll
        for (int k = 0; k < NS; ++k) acc[k] += part[warp / H][k][lane];
    }
    if (!live || a >= n_rows) return;
    T rr[NS], dd[NS], xx[NS];
    load_node<NS>(r, a, rr);
    const T i1 = mdiag[2 * a], i2 = mdiag[2 * a + 1];
    if (first) {
#pragma unroll
        for (int k = 0; k < NS; ++k) dd[k] = T(0);
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            dd[k] = c2 * i1 * rr[k];
            dd[DIM + 1 + k] = c2 * i2 * rr[DIM + 1 + k];
        }
        store_node<NS>(d, a, dd);
        store_node<NS>(xout, a, dd);
        return;
    }
    load_node<NS>(d, a, dd);
    load_node<NS>(xin, a, xx);
    const T s1 = c2 * i1, s2 = c2 * i2;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {  // acc = r - A x (see above)
        dd[k] = fma(s1, acc[k], c1 * dd[k]);
        dd[DIM + 1 + k] = fma(s2, acc[DIM + 1 + k], c1 * dd[DIM + 1 + k]);
        xx[k] += dd[k];
        xx[DIM + 1 + k] += dd[DIM + 1 + k];
    }
    store_node<NS>(d, a, dd);
    store_node<NS>(xout, a, xx);
}

template <int DIM, class T, bool TRANS>
__global__ void __launch_bounds__(128) k_C_resid(int64_t n_rows, int64_t n_slices,
                                                 const int* __restrict__ slice_ptr,
                                                 const int* __restrict__ sell_col,
                                                 const T* __restrict__ val,
                                                 const T* __restrict__ r,
                                                 const T* __restrict__ yu, T* __restrict__ tp) {
    constexpr int NS = 2 * DIM + 2;
    constexpr int NV = pair_values(DIM);
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s = a >> 5;
    if (s >= n_slices) return;
    const int lane = (int)(a & 31);
    const int g0 = slice_ptr[s], g1 = slice_ptr[s + 1];
    T c1 = 0, c2 = 0;
    for (int g = g0; g < g1; ++g) {
        const int cb = sell_col[(int64_t)g * kSell + lane];
        if (cb < 0) continue;
        const T* v = val + (int64_t)g * NV * kSell + lane;
        T xb[NS];
        load_node<NS>(yu, cb, xb);
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const T cu = v[(2 + DIM + k) * kSell];
            c1 += cu * xb[k];
            c2 += cu * xb[DIM + 1 + k];
        }
    }
    if (a >= n_rows) return;
    if (TRANS) { c1 = -c1; c2 = -c2; }
    tp[a] = r[a * NS + DIM] - c1;
    tp[n_rows + a] = r[a * NS + 2 * DIM + 1] - c2;
}

template <int DIM, class T, bool TRANS>
__global__ void __launch_bounds__(128) k_B_resid(int64_t n_rows, int64_t n_slices,
                                                 const int* __restrict__ slice_ptr,
                                                 const int* __restrict__ sell_col,
                                                 const T* __restrict__ val,
                                                 const T* __restrict__ r,
                                                 const T* __restrict__ yp, T* __restrict__ su) {
    constexpr int NS = 2 * DIM + 2;
    constexpr int NV = pair_values(DIM);
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s = a >> 5;
    if (s >= n_slices) return;
    const int lane = (int)(a & 31);
    const int g0 = slice_ptr[s], g1 = slice_ptr[s + 1];
    T acc1[DIM], acc2[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) acc1[k] = acc2[k] = T(0);
    for (int g = g0; g < g1; ++g) {
        const int cb = sell_col[(int64_t)g * kSell + lane];
        if (cb < 0) continue;
        const T* v = val + (int64_t)g * NV * kSell + lane;
        const T p1 = yp[cb], p2 = yp[n_rows + cb];
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const T bu = v[(2 + k) * kSell];
            acc1[k] += bu * p1;
            acc2[k] += bu * p2;
        }
    }
    if (a >= n_rows) return;
    const T sg = TRANS ? T(-1) : T(1);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        su[a * NS + k] = r[a * NS + k] - sg * acc1[k];
        su[a * NS + DIM + 1 + k] = r[a * NS + DIM + 1 + k] - sg * acc2[k];
    }
}

template <int DIM>
__global__ void k_mass_diag(int64_t n_rows, const int* __restrict__ row_ptr,
                            const int* __restrict__ col, const int* __restrict__ slice_ptr,
                            const double* __restrict__ val, double* __restrict__ mdiag,
                            int lumped) {
    constexpr int NV = pair_values(DIM);
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_rows) return;
    double s1 = 0, s2 = 0;
    for (int p = row_ptr[a]; p < row_ptr[a + 1]; ++p) {
        if (!lumped && col[p] != a) continue;
        int64_t grp = (int64_t)slice_ptr[a >> 5] + (p - row_ptr[a]);
        const double* v = val + grp * NV * kSell + (a & 31);
        s1 += v[0];
        s2 += v[kSell];
    }
    mdiag[2 * a] = 1.0 / s1;
    mdiag[2 * a + 1] = 1.0 / s2;
}

template <int DIM, class T>
__global__ void k_scatter_p(int64_t n_rows, const T* __restrict__ yp, T* __restrict__ z) {
    constexpr int NS = 2 * DIM + 2;
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_rows) return;
    z[a * NS + DIM] = yp[a];
    z[a * NS + 2 * DIM + 1] = yp[n_rows + a];
}

template <class VT> const VT* vals_of(const ProblemImpl& P);
template <> const double* vals_of<double>(const ProblemImpl& P) { return P.sell_val.get(); }
template <> const float* vals_of<float>(const ProblemImpl& P) { return P.sell_val32.get(); }

template <int DIM, class VT, class XT, class YT>
void apply_K_dim(const ProblemImpl& P, const XT* x, YT* y, const YT* b, bool tr, cudaStream_t s) {
    // algorithmic bytes: every pair's values and column once, x and y once (b once if given)
    const double vecn = (double)P.n_nodes * P.ns;
    const double alg = (double)P.n_pairs * (P.nv * (double)sizeof(VT) + 4.0) +
                       vecn * (double)(sizeof(XT) + sizeof(YT) + (b ? sizeof(YT) : 0));
    ProfScope prof(sizeof(VT) == 8 ? "apply_K" : "apply_K_fp32", s, alg);
    const int B = 128;
    // two warps per slice in FP32 (HBM-bound, latency-limited at one thread per
    // row); one in FP64, where the FP64 pipe is the limit
    constexpr int H = (sizeof(VT) == 4) ? 2 : 1;
    const int grid = grid_for(P.n_slices, 4 / H);
    const VT* val = vals_of<VT>(P);
#define DPP_LAUNCH_APPLY(TR, RS)                                                          \
    k_apply_K<DIM, VT, XT, YT, TR, RS, H><<<grid, B, 0, s>>>(P.n_nodes, P.n_slices,       \
                                                             P.slice_ptr.get(),           \
                                                             P.sell_col.get(), val, x, b, y)
    if (tr) {
        if (b) DPP_LAUNCH_APPLY(true, true);
        else DPP_LAUNCH_APPLY(true, false);
    } else {
        if (b) DPP_LAUNCH_APPLY(false, true);
        else DPP_LAUNCH_APPLY(false, false);
    }
#undef DPP_LAUNCH_APPLY
    DPP_LAUNCH_CK();
}

template <int DIM>
struct DimTag { static constexpr int value = DIM; };

}  // namespace

void apply_K(const ProblemImpl& P, const double* x, double* y, const double* b, bool tr, bool use32,
             cudaStream_t s) {
    if (use32 && !P.sell_val32.get()) fail(DPP_ERR_BAD_STATE, "FP32 values were not assembled");
    if (P.dim == 2) {
        if (use32) apply_K_dim<2, float, double, double>(P, x, y, b, tr, s);
        else apply_K_dim<2, double, double, double>(P, x, y, b, tr, s);
    } else {
        if (use32) apply_K_dim<3, float, double, double>(P, x, y, b, tr, s);
        else apply_K_dim<3, double, double, double>(P, x, y, b, tr, s);
    }
}

void apply_K32(const ProblemImpl& P, const float* x, double* y, bool tr, cudaStream_t s) {
    if (!P.sell_val32.get()) fail(DPP_ERR_BAD_STATE, "FP32 values were not assembled");
    if (P.dim == 2) apply_K_dim<2, float, float, double>(P, x, y, nullptr, tr, s);
    else apply_K_dim<3, float, float, double>(P, x, y, nullptr, tr, s);
}

template <class T>
void mass_cheb_step(const ProblemImpl& P, const T* mdiag, const T* r, const T* xin, T* xout, T* d,
                    double c1, double c2, bool first, cudaStream_t s) {
    const double vecb = (double)P.n_nodes * P.ns * sizeof(T);
    const double alg = first ? 3 * vecb : (double)P.n_pairs * (2.0 * sizeof(T) + 4.0) + 5 * vecb;
    ProfScope prof(sizeof(T) == 8 ? "mass_cheb" : "mass_cheb_fp32", s, alg);
    const int B = 128;
    // one warp per slice: in FP32 the per-row epilogue outweighs the short pair
    // loop, and in FP64 the FP64 pipe bounds the kernel, so the adds that join
    // two warps' partial sums cost more than the extra loads in flight gain
    // (3.56 against 3.65 ms per step at 64^3)
    constexpr int H = 1;
    const int grid = grid_for(P.n_slices, 4 / H);
    const T* val = vals_of<T>(P);
    if (P.dim == 2)
        k_mass_cheb<2, T, H><<<grid, B, 0, s>>>(P.n_nodes, P.n_slices, P.slice_ptr.get(),
                                                P.sell_col.get(), val, mdiag, r, xin, xout, d, (T)c1,
                                                (T)c2, first ? 1 : 0);
    else
        k_mass_cheb<3, T, H><<<grid, B, 0, s>>>(P.n_nodes, P.n_slices, P.slice_ptr.get(),
                                                P.sell_col.get(), val, mdiag, r, xin, xout, d, (T)c1,
                                                (T)c2, first ? 1 : 0);
    DPP_LAUNCH_CK();
}

template <class T>
void apply_C_resid(const ProblemImpl& P, const T* r, const T* yu, T* tp, bool tr, cudaStream_t s) {
    const int B = 128;
    const int grid = grid_for(P.n_slices * kSell, B);
    const T* val = vals_of<T>(P);
    auto go = [&](auto tag) {
        constexpr int DIM = decltype(tag)::value;
        if (tr)
            k_C_resid<DIM, T, true><<<grid, B, 0, s>>>(P.n_nodes, P.n_slices, P.slice_ptr.get(),
                                                       P.sell_col.get(), val, r, yu, tp);
        else
            k_C_resid<DIM, T, false><<<grid, B, 0, s>>>(P.n_nodes, P.n_slices, P.slice_ptr.get(),
                                                        P.sell_col.get(), val, r, yu, tp);
    };
    if (P.dim == 2) go(DimTag<2>());
    else go(DimTag<3>());
    DPP_LAUNCH_CK();
}

template <class T>
void apply_B_resid(const ProblemImpl& P, const T* r, const T* yp, T* su, bool tr, cudaStream_t s) {
    const int B = 128;
    const int grid = grid_for(P.n_slices * kSell, B);
    const T* val = vals_of<T>(P);
    auto go = [&](auto tag) {
        constexpr int DIM = decltype(tag)::value;
        if (tr)
            k_B_resid<DIM, T, true><<<grid, B, 0, s>>>(P.n_nodes, P.n_slices, P.slice_ptr.get(),
                                                       P.sell_col.get(), val, r, yp, su);
        else
            k_B_resid<DIM, T, false><<<grid, B, 0, s>>>(P.n_nodes, P.n_slices, P.slice_ptr.get(),
                                                        P.sell_col.get(), val, r, yp, su);
    };
    if (P.dim == 2) go(DimTag<2>());
    else go(DimTag<3>());
    DPP_LAUNCH_CK();
}

void mass_diag_inv(const ProblemImpl& P, double* mdiag, bool lumped, cudaStream_t s) {
    const int B = 256;
    if (P.dim == 2)
        k_mass_diag<2><<<grid_for(P.n_nodes, B), B, 0, s>>>(P.n_nodes, P.row_ptr.get(), P.col.get(),
                                                            P.slice_ptr.get(), P.sell_val.get(),
                                                            mdiag, lumped ? 1 : 0);
    else
        k_mass_diag<3><<<grid_for(P.n_nodes, B), B, 0, s>>>(P.n_nodes, P.row_ptr.get(), P.col.get(),
                                                            P.slice_ptr.get(), P.sell_val.get(),
                                                            mdiag, lumped ? 1 : 0);
    DPP_LAUNCH_CK();
}

template <class T>
void scatter_p(const ProblemImpl& P, const T* yp, T* z, cudaStream_t s) {
    const int B = 256;
    if (P.dim == 2) k_scatter_p<2, T><<<grid_for(P.n_nodes, B), B, 0, s>>>(P.n_nodes, yp, z);
    else k_scatter_p<3, T><<<grid_for(P.n_nodes, B), B, 0, s>>>(P.n_nodes, yp, z);
    DPP_LAUNCH_CK();
}

#define DPP_INSTANTIATE(T)                                                                       \
    template void mass_cheb_step<T>(const ProblemImpl&, const T*, const T*, const T*, T*, T*,    \
                                    double, double, bool, cudaStream_t);                         \
    template void apply_C_resid<T>(const ProblemImpl&, const T*, const T*, T*, bool,             \
                                   cudaStream_t);                                                \
    template void apply_B_resid<T>(const ProblemImpl&, const T*, const T*, T*, bool,             \
                                   cudaStream_t);                                                \
    template void scatter_p<T>(const ProblemImpl&, const T*, T*, cudaStream_t);
DPP_INSTANTIATE(double)
DPP_INSTANTIATE(float)
#undef DPP_INSTANTIATE

}  // namespace dpp
