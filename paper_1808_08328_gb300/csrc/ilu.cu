// ILU(0) of the velocity mass blocks: the paper's inner solver for A
// (Section 4.2, "inverting the entire A block using ILU(0)"; Section 4.1 and
// the listings: block Jacobi with its default ILU(0) sub-solver). It is
// selected with dpp_pc_opts::mass_solver = 1; the default is Chebyshev-Jacobi.
//
// A = blockdiag(K1_uu, K2_uu). Every velocity component of network i carries
// the same weighted mass matrix M_i (the m_i pair values), so one ILU(0) per
// network serves its d components. The factorisation keeps A's node-pair
// pattern (zero fill) and the natural row order, as a sequential ILU(0)
// would. Row i of the IKJ algorithm needs the finished rows k < i of its
// lower part, so the rows are grouped into dependency levels (level(i) = 1 +
// the largest level among those k), computed once from the pattern on the
// host. One launch per level then factors, or solves, all rows of that level,
// for both networks and all components at once. The backward solve uses the
// levels of the upper part. On a lexicographic 3D N^3 grid there are about 3N
// levels of each kind. The result is the sequential ILU(0) exactly: within a
// level the rows are independent, and every row's own sums run in its column
// order.
#include "kernels.cuh"

#include <algorithm>

namespace dpp {

namespace {

// m1, m2 of every pair, in CSR order: lu[2 p + net]
template <int DIM>
__global__ void k_gather_mass(int64_t n_rows, const int* __restrict__ row_ptr,
                              const int* __restrict__ slice_ptr, const double* __restrict__ val,
                              double* __restrict__ lu, int* __restrict__ dpos,
                              const int* __restrict__ col) {
    constexpr int NV = pair_values(DIM);
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_rows) return;
    for (int p = row_ptr[a]; p < row_ptr[a + 1]; ++p) {
        const int64_t grp = (int64_t)slice_ptr[a >> 5] + (p - row_ptr[a]);
        const double* v = val + grp * NV * kSell + (a & 31);
        lu[2 * (int64_t)p] = v[0];
        lu[2 * (int64_t)p + 1] = v[kSell];
        if (col[p] == a) dpos[a] = p;
    }
}

// IKJ ILU(0) of the rows of one level (both networks).
__global__ void k_ilu_factor_level(int n_level, const int* __restrict__ rows,
                                   const int* __restrict__ row_ptr, const int* __restrict__ col,
                                   const int* __restrict__ dpos, double* __restrict__ lu) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_level) return;
    const int i = rows[t];
    const int p0 = row_ptr[i], p1 = row_ptr[i + 1];
    for (int p = p0; p < p1; ++p) {
        const int k = col[p];
        if (k >= i) break;
        const int dk = dpos[k];
        const double l1 = lu[2 * (int64_t)p] / lu[2 * (int64_t)dk];
        const double l2 = lu[2 * (int64_t)p + 1] / lu[2 * (int64_t)dk + 1];
        lu[2 * (int64_t)p] = l1;
        lu[2 * (int64_t)p + 1] = l2;
        // a_ij -= l_ik u_kj for j > k present in both rows (both sorted: merge)
        int t2 = p + 1;
        for (int q = dk + 1; q < row_ptr[k + 1] && t2 < p1; ++q) {
            const int j = col[q];
            while (t2 < p1 && col[t2] < j) ++t2;
            if (t2 < p1 && col[t2] == j) {
                lu[2 * (int64_t)t2] -= l1 * lu[2 * (int64_t)q];
                lu[2 * (int64_t)t2 + 1] -= l2 * lu[2 * (int64_t)q + 1];
            }
        }
    }
}

__global__ void k_d2f_ilu(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

// Forward solve, one level: y_i = r_i - sum_{k < i} l_ik y_k on the velocity
// slots of both networks (d components each). y may not alias r.
template <int DIM, class T>
__global__ void k_ilu_lower(int n_level, const int* __restrict__ rows,
                            const int* __restrict__ row_ptr, const int* __restrict__ col,
                            const T* __restrict__ lu, const T* __restrict__ r, T* __restrict__ y) {
    constexpr int NS = 2 * DIM + 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_level) return;
    const int i = rows[t];
    T a1[DIM], a2[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        a1[c] = r[(int64_t)i * NS + c];
        a2[c] = r[(int64_t)i * NS + DIM + 1 + c];
    }
    for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
        const int k = col[p];
        if (k >= i) break;
        const T l1 = lu[2 * (int64_t)p], l2 = lu[2 * (int64_t)p + 1];
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            a1[c] -= l1 * y[(int64_t)k * NS + c];
            a2[c] -= l2 * y[(int64_t)k * NS + DIM + 1 + c];
        }
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        y[(int64_t)i * NS + c] = a1[c];
        y[(int64_t)i * NS + DIM + 1 + c] = a2[c];
    }
}

// Backward solve, one level, in place: z_i = (y_i - sum_{j > i} u_ij z_j) / u_ii.
template <int DIM, class T>
__global__ void k_ilu_upper(int n_level, const int* __restrict__ rows,
                            const int* __restrict__ row_ptr, const int* __restrict__ col,
                            const int* __restrict__ dpos, const T* __restrict__ lu,
                            T* __restrict__ z) {
    constexpr int NS = 2 * DIM + 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_level) return;
    const int i = rows[t];
    const int d = dpos[i];
    T a1[DIM], a2[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        a1[c] = z[(int64_t)i * NS + c];
        a2[c] = z[(int64_t)i * NS + DIM + 1 + c];
    }
    for (int p = d + 1; p < row_ptr[i + 1]; ++p) {
        const int j = col[p];
        const T u1 = lu[2 * (int64_t)p], u2 = lu[2 * (int64_t)p + 1];
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            a1[c] -= u1 * z[(int64_t)j * NS + c];
            a2[c] -= u2 * z[(int64_t)j * NS + DIM + 1 + c];
        }
    }
    const T i1 = T(1) / lu[2 * (int64_t)d], i2 = T(1) / lu[2 * (int64_t)d + 1];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        z[(int64_t)i * NS + c] = a1[c] * i1;
        z[(int64_t)i * NS + DIM + 1 + c] = a2[c] * i2;
    }
}

// Rows grouped by dependency level. lower: level(i) = 1 + max level(k), k < i
// in row i; upper: level(i) = 1 + max level(j), j > i in row i.
void make_levels(const std::vector<int>& rp, const std::vector<int>& col, bool lower,
                 std::vector<int>& lev_ptr, std::vector<int>& rows) {
    const int n = (int)rp.size() - 1;
    std::vector<int> lev(n, 0);
    int nlev = 0;
    if (lower) {
        for (int i = 0; i < n; ++i) {
            int l = 0;
            for (int p = rp[i]; p < rp[i + 1] && col[p] < i; ++p) l = std::max(l, lev[col[p]] + 1);
            lev[i] = l;
            nlev = std::max(nlev, l + 1);
        }
    } else {
        for (int i = n - 1; i >= 0; --i) {
            int l = 0;
            for (int p = rp[i + 1] - 1; p >= rp[i] && col[p] > i; --p) l = std::max(l, lev[col[p]] + 1);
            lev[i] = l;
            nlev = std::max(nlev, l + 1);
        }
    }
    lev_ptr.assign(nlev + 1, 0);
    for (int i = 0; i < n; ++i) ++lev_ptr[lev[i] + 1];
    for (int l = 0; l < nlev; ++l) lev_ptr[l + 1] += lev_ptr[l];
    rows.assign(n, 0);
    std::vector<int> cur(lev_ptr.begin(), lev_ptr.end() - 1);
    for (int i = 0; i < n; ++i) rows[cur[lev[i]]++] = i;  // increasing row id within a level
}

}  // namespace

void mass_ilu_setup(const ProblemImpl& P, PcImpl& pc, cudaStream_t s) {
    ProfScope pr("setup_mass_ilu", s, 0);
    const int64_t n = P.n_nodes;
    MassIlu& M = pc.ilu;
    std::vector<int> rp(n + 1), col(P.n_pairs);
    DPP_CK(cudaMemcpyAsync(rp.data(), P.row_ptr.get(), (n + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    DPP_CK(cudaMemcpyAsync(col.data(), P.col.get(), P.n_pairs * sizeof(int), cudaMemcpyDeviceToHost, s));
    DPP_CK(cudaStreamSynchronize(s));
    std::vector<int> lp, lr, up, ur;
    make_levels(rp, col, true, lp, lr);
    make_levels(rp, col, false, up, ur);
    M.lower_ptr = lp;
    M.upper_ptr = up;
    M.lower_rows.alloc(n);
    M.upper_rows.alloc(n);
    DPP_CK(cudaMemcpyAsync(M.lower_rows.get(), lr.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
    DPP_CK(cudaMemcpyAsync(M.upper_rows.get(), ur.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
    M.lu.alloc(2 * P.n_pairs);
    M.dpos.alloc(n);
    const int B = 128;
    if (P.dim == 2)
        k_gather_mass<2><<<grid_for(n, B), B, 0, s>>>(n, P.row_ptr.get(), P.slice_ptr.get(),
                                                      P.sell_val.get(), M.lu.get(), M.dpos.get(),
                                                      P.col.get());
    else
        k_gather_mass<3><<<grid_for(n, B), B, 0, s>>>(n, P.row_ptr.get(), P.slice_ptr.get(),
                                                      P.sell_val.get(), M.lu.get(), M.dpos.get(),
                                                      P.col.get());
    DPP_LAUNCH_CK();
    for (size_t l = 0; l + 1 < lp.size(); ++l) {
        const int cnt = lp[l + 1] - lp[l];
        k_ilu_factor_level<<<grid_for(cnt, B), B, 0, s>>>(cnt, M.lower_rows.get() + lp[l],
                                                          P.row_ptr.get(), P.col.get(),
                                                          M.dpos.get(), M.lu.get());
        DPP_LAUNCH_CK();
    }
    if (pc.precision == DPP_MIXED_FP32_FP64) {
        M.lu32.alloc(2 * P.n_pairs);
        k_d2f_ilu<<<grid_for(2 * P.n_pairs, 256), 256, 0, s>>>(2 * P.n_pairs, M.lu.get(),
                                                               M.lu32.get());
        DPP_LAUNCH_CK();
    }
    DPP_CK(cudaStreamSynchronize(s));  // the host level tables go out of scope
}

template <class T>
void mass_ilu_apply(const ProblemImpl& P, const PcImpl& pc, const T* r, T* target,
                    cudaStream_t s) {
    const MassIlu& M = pc.ilu;
    const T* lu;
    if constexpr (sizeof(T) == 8) lu = M.lu.get();
    else lu = M.lu32.get();
    const double vec = (double)P.n_nodes * 2 * P.dim * sizeof(T);
    const double alg = 2.0 * (double)P.n_pairs * (2 * sizeof(T) + 4.0) + 4.0 * vec;
    ProfScope prof(sizeof(T) == 8 ? "mass_ilu" : "mass_ilu_fp32", s, alg);
    const int B = 128;
    for (size_t l = 0; l + 1 < M.lower_ptr.size(); ++l) {
        const int cnt = M.lower_ptr[l + 1] - M.lower_ptr[l];
        if (P.dim == 2)
            k_ilu_lower<2, T><<<grid_for(cnt, B), B, 0, s>>>(cnt, M.lower_rows.get() + M.lower_ptr[l],
                                                             P.row_ptr.get(), P.col.get(), lu, r,
                                                             target);
        else
            k_ilu_lower<3, T><<<grid_for(cnt, B), B, 0, s>>>(cnt, M.lower_rows.get() + M.lower_ptr[l],
                                                             P.row_ptr.get(), P.col.get(), lu, r,
                                                             target);
        DPP_LAUNCH_CK();
    }
    for (size_t l = 0; l + 1 < M.upper_ptr.size(); ++l) {
        const int cnt = M.upper_ptr[l + 1] - M.upper_ptr[l];
        if (P.dim == 2)
            k_ilu_upper<2, T><<<grid_for(cnt, B), B, 0, s>>>(cnt, M.upper_rows.get() + M.upper_ptr[l],
                                                             P.row_ptr.get(), P.col.get(),
                                                             M.dpos.get(), lu, target);
        else
            k_ilu_upper<3, T><<<grid_for(cnt, B), B, 0, s>>>(cnt, M.upper_rows.get() + M.upper_ptr[l],
                                                             P.row_ptr.get(), P.col.get(),
                                                             M.dpos.get(), lu, target);
        DPP_LAUNCH_CK();
    }
}

template void mass_ilu_apply<double>(const ProblemImpl&, const PcImpl&, const double*, double*,
                                     cudaStream_t);
template void mass_ilu_apply<float>(const ProblemImpl&, const PcImpl&, const float*, float*,
                                    cudaStream_t);

}  // namespace dpp
