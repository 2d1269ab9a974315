// Preconditioner-setup and AMG interfaces shared between translation units.
#pragma once

#include "kernels.cuh"

namespace dpp {

// Non-owning view of a CSR matrix. A matrix of the FP32 hierarchy (mixed
// precision) has FP32 values only (val32), one of the FP64 hierarchy FP64
// values (val), and FP32 copies too once amg_make_fp32 has run.
struct CsrView {
    int64_t n_rows = 0, n_cols = 0, nnz = 0;
    const int* rp = nullptr;
    const int* col = nullptr;
    const double* val = nullptr;
    const float* val32 = nullptr;
};
inline CsrView view(const Csr& A) {
    CsrView v;
    v.n_rows = A.n_rows;
    v.n_cols = A.n_cols;
    v.nnz = A.nnz;
    v.rp = A.row_ptr.get();
    v.col = A.col.get();
    v.val = A.val.get();
    v.val32 = A.val32.get();
    return v;
}

// The values of type V of a matrix or view (FP64: val, FP32: val32).
template <class V> inline const V* vals_of(const CsrView& v);
template <> inline const double* vals_of<double>(const CsrView& v) { return v.val; }
template <> inline const float* vals_of<float>(const CsrView& v) { return v.val32; }
template <class V> inline DBuf<V>& vbuf(Csr& A);
template <> inline DBuf<double>& vbuf<double>(Csr& A) { return A.val; }
template <> inline DBuf<float>& vbuf<float>(Csr& A) { return A.val32; }
template <class V> inline const DBuf<V>& vbuf(const Csr& A) { return vbuf<V>(const_cast<Csr&>(A)); }
template <class V> inline DBuf<V>& sell_vbuf(Csr& A);
template <> inline DBuf<double>& sell_vbuf<double>(Csr& A) { return A.sell_val; }
template <> inline DBuf<float>& sell_vbuf<float>(Csr& A) { return A.sell_val32; }
// True when the matrix holds FP32 values only (a matrix of the FP32 hierarchy).
inline bool fp32_only(const Csr& A) { return !A.val.get() && A.val32.get(); }

// C = A B (sorted columns in every row of B are required and produced in C).
// upper_only: only the entries C[i][j] with j >= i (the upper triangle of a
// product known to be symmetric; see symmetrize_upper). The product takes the
// FP64 values when A has them (into C.val), else the FP32 ones (into C.val32).
void spgemm(const CsrView& A, const CsrView& B, Csr& C, bool values, cudaStream_t s,
            HostScratch& hs, bool upper_only = false);
// C = U + strict_upper(U)^T for an upper-triangular U (the full symmetric matrix).
void symmetrize_upper(const Csr& U, Csr& C, cudaStream_t s, HostScratch& hs);
// True when A is square and, in every stride-th row, each entry has its mirror
// with |a_ij - a_ji| <= tol (|a_ij| + |a_ji|).
bool is_symmetric(const Csr& A, double tol, int stride, cudaStream_t s, HostScratch& hs);
void transpose(const Csr& A, Csr& T, cudaStream_t s, HostScratch& hs);
// blockdiag(S_p1, S_p2) from the pair values and mdiag = 1/diag(K_uu) per network:
// in FP64 from the FP64 pair values (S.val), or in FP32 from the FP32 ones (S.val32).
void build_selfp(const ProblemImpl& P, const double* mdiag, Csr& S, cudaStream_t s,
                 HostScratch& hs);
void build_selfp(const ProblemImpl& P, const float* mdiag, Csr& S, cudaStream_t s,
                 HostScratch& hs);

// Build one hierarchy on A0 (SPD) with the options' coarsening parameters.
void amg_setup(Amg& h, const dpp_pc_opts& o, Csr&& A0, cudaStream_t s, HostScratch& hs);
// FP32 copies of every level (values, 1/diag, work vectors) for the mixed mode;
// a hierarchy built in FP32 gets its FP32 work vectors only.
void amg_make_fp32(Amg& h, cudaStream_t s);
// Autotune the SpMV format / CSR lanes of every level for `precision`.
void amg_tune(Amg& h, const dpp_pc_opts& o, int precision, cudaStream_t s);
// x = (one V-cycle) b on level 0; b is not modified. T = double uses the FP64
// hierarchy; T = float the FP32 copies (the coarsest solve stays FP64).
template <class T>
void amg_vcycle(Amg& h, const dpp_pc_opts& o, const T* b, T* x, cudaStream_t s);

}  // namespace dpp
