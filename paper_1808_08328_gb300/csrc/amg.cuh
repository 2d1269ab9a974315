// Preconditioner-setup and AMG interfaces shared between translation units.
#pragma once

#include "kernels.cuh"

namespace dpp {

// Non-owning view of a CSR matrix.
struct CsrView {
    int64_t n_rows = 0, n_cols = 0, nnz = 0;
    const int* rp = nullptr;
    const int* col = nullptr;
    const double* val = nullptr;
};
inline CsrView view(const Csr& A) {
    CsrView v;
    v.n_rows = A.n_rows;
    v.n_cols = A.n_cols;
    v.nnz = A.nnz;
    v.rp = A.row_ptr.get();
    v.col = A.col.get();
    v.val = A.val.get();
    return v;
}

// C = A B (sorted columns in every row of B are required and produced in C).
// upper_only: only the entries C[i][j] with j >= i (the upper triangle of a
// product known to be symmetric; see symmetrize_upper).
void spgemm(const CsrView& A, const CsrView& B, Csr& C, bool values, cudaStream_t s,
            HostScratch& hs, bool upper_only = false);
// C = U + strict_upper(U)^T for an upper-triangular U (the full symmetric matrix).
void symmetrize_upper(const Csr& U, Csr& C, cudaStream_t s, HostScratch& hs);
// True when A is square and, in every stride-th row, each entry has its mirror
// with |a_ij - a_ji| <= tol (|a_ij| + |a_ji|).
bool is_symmetric(const Csr& A, double tol, int stride, cudaStream_t s, HostScratch& hs);
void transpose(const Csr& A, Csr& T, cudaStream_t s, HostScratch& hs);
// blockdiag(S_p1, S_p2) from the pair values and mdiag = 1/diag(K_uu) per network.
void build_selfp(const ProblemImpl& P, const double* mdiag, Csr& S, cudaStream_t s,
                 HostScratch& hs);

// Build one hierarchy on A0 (SPD) with the options' coarsening parameters.
void amg_setup(Amg& h, const dpp_pc_opts& o, Csr&& A0, cudaStream_t s, HostScratch& hs);
// FP32 copies of every level (values, 1/diag, work vectors) for the mixed mode.
void amg_make_fp32(Amg& h, cudaStream_t s);
// Autotune the SpMV format / CSR lanes of every level for `precision`.
void amg_tune(Amg& h, const dpp_pc_opts& o, int precision, cudaStream_t s);
// x = (one V-cycle) b on level 0; b is not modified. T = double uses the FP64
// hierarchy; T = float the FP32 copies (the coarsest solve stays FP64).
template <class T>
void amg_vcycle(Amg& h, const dpp_pc_opts& o, const T* b, T* x, cudaStream_t s);

}  // namespace dpp
