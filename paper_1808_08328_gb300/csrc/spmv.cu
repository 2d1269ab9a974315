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
// transaction. x is gathered per column node as (2d+2) contiguous doubles.
#include "kernels.cuh"

namespace dpp {

namespace {

template <int NS>
__device__ __forceinline__ void load_node(const double* __restrict__ x, int b, double (&v)[NS]) {
    const double2* p = reinterpret_cast<const double2*>(x + (int64_t)b * NS);
#pragma unroll
    for (int k = 0; k < NS / 2; ++k) {
        double2 t = __ldg(p + k);
        v[2 * k] = t.x;
        v[2 * k + 1] = t.y;
    }
}

template <int NS>
__device__ __forceinline__ void store_node(double* __restrict__ y, int64_t a, const double (&v)[NS]) {
    double2* p = reinterpret_cast<double2*>(y + a * NS);
#pragma unroll
    for (int k = 0; k < NS / 2; ++k) p[k] = make_double2(v[2 * k], v[2 * k + 1]);
}

template <int DIM, class VT, bool TRANS, bool RESID>
__global__ void __launch_bounds__(128) k_apply_K(int64_t n_rows, int64_t n_slices,
                                                 const int* __restrict__ slice_ptr,
                                                 const int* __restrict__ sell_col,
                                                 const VT* __restrict__ val,
                                                 const double* __restrict__ x,
                                                 const double* __restrict__ b,
                                                 double* __restrict__ y) {
    constexpr int NS = 2 * DIM + 2;
    constexpr int NV = pair_values(DIM);
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s = a >> 5;
    if (s >= n_slices) return;
    const int lane = (int)(a & 31);
    const int g0 = slice_ptr[s], g1 = slice_ptr[s + 1];
    double acc[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) acc[k] = 0.0;
    for (int g = g0; g < g1; ++g) {
        const int cb = sell_col[(int64_t)g * kSell + lane];
        if (cb < 0) continue;
        const VT* v = val + (int64_t)g * NV * kSell + lane;
        const double m1 = (double)v[0], m2 = (double)v[kSell];
        double bu[DIM], cu[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            bu[k] = (double)v[(2 + k) * kSell];
            cu[k] = (double)v[(2 + DIM + k) * kSell];
            if (TRANS) { bu[k] = -bu[k]; cu[k] = -cu[k]; }
        }
        const double d1 = (double)v[(2 + 2 * DIM) * kSell];
        const double d2 = (double)v[(3 + 2 * DIM) * kSell];
        const double e = (double)v[(4 + 2 * DIM) * kSell];
        double xb[NS];
        load_node<NS>(x, cb, xb);
        const double p1 = xb[DIM], p2 = xb[2 * DIM + 1];
        double cp1 = d1 * p1 + e * p2, cp2 = d2 * p2 + e * p1;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            acc[k] += m1 * xb[k] + bu[k] * p1;
            acc[DIM + 1 + k] += m2 * xb[DIM + 1 + k] + bu[k] * p2;
            cp1 += cu[k] * xb[k];
            cp2 += cu[k] * xb[DIM + 1 + k];
        }
        acc[DIM] += cp1;
        acc[2 * DIM + 1] += cp2;
    }
    if (a >= n_rows) return;
    if (RESID) {
        double bb[NS];
        load_node<NS>(b, (int)a, bb);
#pragma unroll
        for (int k = 0; k < NS; ++k) acc[k] = bb[k] - acc[k];
    }
    store_node<NS>(y, a, acc);
}

// Chebyshev step on A = blockdiag(K1_uu, K2_uu); each velocity component of
// network i sees the same scalar matrix with entries m_i.
template <int DIM, class VT>
__global__ void __launch_bounds__(128) k_mass_cheb(int64_t n_rows, int64_t n_slices,
                                                   const int* __restrict__ slice_ptr,
                                                   const int* __restrict__ sell_col,
                                                   const VT* __restrict__ val,
                                                   const double* __restrict__ mdiag,
                                                   const double* __restrict__ r,
                                                   const double* __restrict__ xin,
                                                   double* __restrict__ xout,
                                                   double* __restrict__ d, double c1, double c2,
                                                   int first) {
    constexpr int NS = 2 * DIM + 2;
    constexpr int NV = pair_values(DIM);
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s = a >> 5;
    if (s >= n_slices) return;
    const int lane = (int)(a & 31);
    double acc[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) acc[k] = 0.0;
    if (!first) {
        const int g0 = slice_ptr[s], g1 = slice_ptr[s + 1];
        for (int g = g0; g < g1; ++g) {
            const int cb = sell_col[(int64_t)g * kSell + lane];
            if (cb < 0) continue;
            const VT* v = val + (int64_t)g * NV * kSell + lane;
            const double m1 = (double)v[0], m2 = (double)v[kSell];
            double xb[NS];
            load_node<NS>(xin, cb, xb);
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                acc[k] += m1 * xb[k];
                acc[DIM + 1 + k] += m2 * xb[DIM + 1 + k];
            }
        }
    }
    if (a >= n_rows) return;
    double rr[NS], dd[NS], xx[NS];
    load_node<NS>(r, (int)a, rr);
    const double i1 = mdiag[2 * a], i2 = mdiag[2 * a + 1];
    if (first) {
#pragma unroll
        for (int k = 0; k < NS; ++k) dd[k] = 0.0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            dd[k] = c2 * i1 * rr[k];
            dd[DIM + 1 + k] = c2 * i2 * rr[DIM + 1 + k];
        }
        store_node<NS>(d, a, dd);
        store_node<NS>(xout, a, dd);
        return;
    }
    load_node<NS>(d, (int)a, dd);
    load_node<NS>(xin, (int)a, xx);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        dd[k] = c1 * dd[k] + c2 * i1 * (rr[k] - acc[k]);
        dd[DIM + 1 + k] = c1 * dd[DIM + 1 + k] + c2 * i2 * (rr[DIM + 1 + k] - acc[DIM + 1 + k]);
        xx[k] += dd[k];
        xx[DIM + 1 + k] += dd[DIM + 1 + k];
    }
    store_node<NS>(d, a, dd);
    store_node<NS>(xout, a, xx);
}

template <int DIM, class VT, bool TRANS>
__global__ void __launch_bounds__(128) k_C_resid(int64_t n_rows, int64_t n_slices,
                                                 const int* __restrict__ slice_ptr,
                                                 const int* __restrict__ sell_col,
                                                 const VT* __restrict__ val,
                                                 const double* __restrict__ r,
                                                 const double* __restrict__ yu,
                                                 double* __restrict__ tp) {
    constexpr int NS = 2 * DIM + 2;
    constexpr int NV = pair_values(DIM);
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s = a >> 5;
    if (s >= n_slices) return;
    const int lane = (int)(a & 31);
    const int g0 = slice_ptr[s], g1 = slice_ptr[s + 1];
    double c1 = 0, c2 = 0;
    for (int g = g0; g < g1; ++g) {
        const int cb = sell_col[(int64_t)g * kSell + lane];
        if (cb < 0) continue;
        const VT* v = val + (int64_t)g * NV * kSell + lane;
        double xb[NS];
        load_node<NS>(yu, cb, xb);
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const double cu = (double)v[(2 + DIM + k) * kSell];
            c1 += cu * xb[k];
            c2 += cu * xb[DIM + 1 + k];
        }
    }
    if (a >= n_rows) return;
    if (TRANS) { c1 = -c1; c2 = -c2; }
    tp[a] = r[a * NS + DIM] - c1;
    tp[n_rows + a] = r[a * NS + 2 * DIM + 1] - c2;
}

template <int DIM, class VT, bool TRANS>
__global__ void __launch_bounds__(128) k_B_resid(int64_t n_rows, int64_t n_slices,
                                                 const int* __restrict__ slice_ptr,
                                                 const int* __restrict__ sell_col,
                                                 const VT* __restrict__ val,
                                                 const double* __restrict__ r,
                                                 const double* __restrict__ yp,
                                                 double* __restrict__ su) {
    constexpr int NS = 2 * DIM + 2;
    constexpr int NV = pair_values(DIM);
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s = a >> 5;
    if (s >= n_slices) return;
    const int lane = (int)(a & 31);
    const int g0 = slice_ptr[s], g1 = slice_ptr[s + 1];
    double acc1[DIM], acc2[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) acc1[k] = acc2[k] = 0.0;
    for (int g = g0; g < g1; ++g) {
        const int cb = sell_col[(int64_t)g * kSell + lane];
        if (cb < 0) continue;
        const VT* v = val + (int64_t)g * NV * kSell + lane;
        const double p1 = yp[cb], p2 = yp[n_rows + cb];
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const double bu = (double)v[(2 + k) * kSell];
            acc1[k] += bu * p1;
            acc2[k] += bu * p2;
        }
    }
    if (a >= n_rows) return;
    const double sg = TRANS ? -1.0 : 1.0;
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

template <int DIM>
__global__ void k_scatter_p(int64_t n_rows, const double* __restrict__ yp, double* __restrict__ z) {
    constexpr int NS = 2 * DIM + 2;
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_rows) return;
    z[a * NS + DIM] = yp[a];
    z[a * NS + 2 * DIM + 1] = yp[n_rows + a];
}

template <int DIM, class VT>
void apply_K_t(const ProblemImpl& P, const VT* val, const double* x, double* y, const double* b,
               bool tr, cudaStream_t s) {
    // algorithmic bytes: every pair's values and column once, x and y once (b once if given)
    const double vecb = (double)P.n_nodes * P.ns * 8.0;
    const double alg = (double)P.n_pairs * (P.nv * (double)sizeof(VT) + 4.0) + vecb * (b ? 3 : 2);
    ProfScope prof(sizeof(VT) == 8 ? "apply_K" : "apply_K_fp32", s, alg);
    const int B = 128;
    const int grid = grid_for(P.n_slices * kSell, B);
    if (tr) {
        if (b) k_apply_K<DIM, VT, true, true><<<grid, B, 0, s>>>(P.n_nodes, P.n_slices, P.slice_ptr.get(), P.sell_col.get(), val, x, b, y);
        else k_apply_K<DIM, VT, true, false><<<grid, B, 0, s>>>(P.n_nodes, P.n_slices, P.slice_ptr.get(), P.sell_col.get(), val, x, b, y);
    } else {
        if (b) k_apply_K<DIM, VT, false, true><<<grid, B, 0, s>>>(P.n_nodes, P.n_slices, P.slice_ptr.get(), P.sell_col.get(), val, x, b, y);
        else k_apply_K<DIM, VT, false, false><<<grid, B, 0, s>>>(P.n_nodes, P.n_slices, P.slice_ptr.get(), P.sell_col.get(), val, x, b, y);
    }
    DPP_LAUNCH_CK();
}

}  // namespace

void apply_K(const ProblemImpl& P, const double* x, double* y, const double* b, bool tr, bool use32,
             cudaStream_t s) {
    if (use32 && !P.sell_val32.get()) fail(DPP_ERR_BAD_STATE, "FP32 values were not assembled");
    if (P.dim == 2) {
        if (use32) apply_K_t<2, float>(P, P.sell_val32.get(), x, y, b, tr, s);
        else apply_K_t<2, double>(P, P.sell_val.get(), x, y, b, tr, s);
    } else {
        if (use32) apply_K_t<3, float>(P, P.sell_val32.get(), x, y, b, tr, s);
        else apply_K_t<3, double>(P, P.sell_val.get(), x, y, b, tr, s);
    }
}

#define DPP_DISPATCH_DV(DIMV, USE32, CALL)                     \
    do {                                                        \
        if ((DIMV) == 2) {                                      \
            constexpr int DIM = 2;                              \
            if (USE32) { using VT = float; CALL; }              \
            else { using VT = double; CALL; }                   \
        } else {                                                \
            constexpr int DIM = 3;                              \
            if (USE32) { using VT = float; CALL; }              \
            else { using VT = double; CALL; }                   \
        }                                                       \
    } while (0)

template <class VT> static const VT* vals_of(const ProblemImpl& P);
template <> const double* vals_of<double>(const ProblemImpl& P) { return P.sell_val.get(); }
template <> const float* vals_of<float>(const ProblemImpl& P) { return P.sell_val32.get(); }

void mass_cheb_step(const ProblemImpl& P, const double* mdiag, const double* r, const double* xin,
                    double* xout, double* d, double c1, double c2, bool first, bool use32,
                    cudaStream_t s) {
    const double vecb = (double)P.n_nodes * P.ns * 8.0;
    const double alg = first ? 3 * vecb
                             : (double)P.n_pairs * (2.0 * (use32 ? 4 : 8) + 4.0) + 5 * vecb;
    ProfScope prof("mass_cheb", s, alg);
    const int B = 128;
    const int grid = grid_for(P.n_slices * kSell, B);
    DPP_DISPATCH_DV(P.dim, use32,
                    (k_mass_cheb<DIM, VT><<<grid, B, 0, s>>>(P.n_nodes, P.n_slices,
                                                             P.slice_ptr.get(), P.sell_col.get(),
                                                             vals_of<VT>(P), mdiag, r, xin, xout,
                                                             d, c1, c2, first ? 1 : 0)));
    DPP_LAUNCH_CK();
}

void apply_C_resid(const ProblemImpl& P, const double* r, const double* yu, double* tp, bool tr,
                   bool use32, cudaStream_t s) {
    const int B = 128;
    const int grid = grid_for(P.n_slices * kSell, B);
    if (tr)
        DPP_DISPATCH_DV(P.dim, use32,
                        (k_C_resid<DIM, VT, true><<<grid, B, 0, s>>>(
                            P.n_nodes, P.n_slices, P.slice_ptr.get(), P.sell_col.get(),
                            vals_of<VT>(P), r, yu, tp)));
    else
        DPP_DISPATCH_DV(P.dim, use32,
                        (k_C_resid<DIM, VT, false><<<grid, B, 0, s>>>(
                            P.n_nodes, P.n_slices, P.slice_ptr.get(), P.sell_col.get(),
                            vals_of<VT>(P), r, yu, tp)));
    DPP_LAUNCH_CK();
}

void apply_B_resid(const ProblemImpl& P, const double* r, const double* yp, double* su, bool tr,
                   bool use32, cudaStream_t s) {
    const int B = 128;
    const int grid = grid_for(P.n_slices * kSell, B);
    if (tr)
        DPP_DISPATCH_DV(P.dim, use32,
                        (k_B_resid<DIM, VT, true><<<grid, B, 0, s>>>(
                            P.n_nodes, P.n_slices, P.slice_ptr.get(), P.sell_col.get(),
                            vals_of<VT>(P), r, yp, su)));
    else
        DPP_DISPATCH_DV(P.dim, use32,
                        (k_B_resid<DIM, VT, false><<<grid, B, 0, s>>>(
                            P.n_nodes, P.n_slices, P.slice_ptr.get(), P.sell_col.get(),
                            vals_of<VT>(P), r, yp, su)));
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

void scatter_p(const ProblemImpl& P, const double* yp, double* z, cudaStream_t s) {
    const int B = 256;
    if (P.dim == 2) k_scatter_p<2><<<grid_for(P.n_nodes, B), B, 0, s>>>(P.n_nodes, yp, z);
    else k_scatter_p<3><<<grid_for(P.n_nodes, B), B, 0, s>>>(P.n_nodes, yp, z);
    DPP_LAUNCH_CK();
}

}  // namespace dpp
