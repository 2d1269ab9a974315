// Launch wrappers shared between translation units.
#pragma once

#include "impl.cuh"

namespace dpp {

void assemble_problem(ProblemImpl& P, const dpp_problem_desc& d, cudaStream_t s);
void assemble_uploaded(ProblemImpl& P, cudaStream_t s);

// ---- node-pair (SELL-32) operators on node-interleaved vectors ----
// y = K x (transpose: K^T x). If b != nullptr: y = b - K x. use32: FP32 values
// (arithmetic stays FP64 because x is FP64).
void apply_K(const ProblemImpl& P, const double* x, double* y, const double* b, bool transpose,
             bool use32, cudaStream_t s);
// y = K32 x with FP32 values, FP32 x and FP32 arithmetic, FP64 output.
void apply_K32(const ProblemImpl& P, const float* x, double* y, bool transpose, cudaStream_t s);
// One Chebyshev step on the velocity block A = blockdiag(K1_uu, K2_uu), in type T
// (values of the same type). first: x_out = c2 * Dinv r, d = x_out. else:
// res = r - A x_in; d = c1 d + c2 Dinv res; x_out = x_in + d. Only u slots change.
template <class T>
void mass_cheb_step(const ProblemImpl& P, const T* mdiag, const T* r, const T* xin, T* xout, T* d,
                    double c1, double c2, bool first, cudaStream_t s);
// tp[net][a] = r_p(net)[a] - (C y_u)(net)[a]   (sign of C flipped if transpose)
template <class T>
void apply_C_resid(const ProblemImpl& P, const T* r, const T* yu, T* tp, bool transpose,
                   cudaStream_t s);
// su_u = r_u - B yp   (yp split [2][n]; sign of B flipped if transpose); p slots of su untouched
template <class T>
void apply_B_resid(const ProblemImpl& P, const T* r, const T* yp, T* su, bool transpose,
                   cudaStream_t s);
// mdiag[a][net] = 1 / m_net(a, a) (or the row sum when lumped)
void mass_diag_inv(const ProblemImpl& P, double* mdiag, bool lumped, cudaStream_t s);
// z_p(net)[a] = yp[net][a] (copy split pressures into interleaved p slots)
template <class T>
void scatter_p(const ProblemImpl& P, const T* yp, T* z, cudaStream_t s);

// ---- vector kernels (n doubles) ----
struct Reducer {
    DBuf<double> partial;   // [rows][kRedBlocks]
    DBuf<unsigned> counter;
    void ensure(int rows, cudaStream_t s);  // allocation and counter reset ordered on s
};
constexpr int kRedBlocks = 2 * kSMs;
// out[0] = x . y (deterministic two-level reduction)
void dot(Reducer& R, const double* x, const double* y, int64_t n, double* out, cudaStream_t s);
// out[j] = V_j . w for j < k (V row-major [k][ld])
void multidot(Reducer& R, const double* V, int64_t ld, int k, const double* w, int64_t n,
              double* out, cudaStream_t s);
// w -= sum_j h[j] V_j
void multi_axpy_sub(const double* V, int64_t ld, int k, const double* h, double* w, int64_t n,
                    cudaStream_t s);
// x += sum_j y[j] Z_j
void multi_axpy_add(const double* Z, int64_t ld, int k, const double* y, double* x, int64_t n,
                    cudaStream_t s);
void scale_copy(const double* x, double* y, int64_t n, const double* num, const double* den,
                cudaStream_t s);   // y = x * num / den (device scalars; den may be null)
void axpby(double a, const double* x, double b, double* y, int64_t n, cudaStream_t s);
void fill(double* x, double v, int64_t n, cudaStream_t s);
void to_float(const double* in, float* out, int64_t n, cudaStream_t s);
// x += sum_j y[j] Z_j with FP32 Z (FP64 y and x)
void multi_axpy_add_f32(const float* Z, int64_t ld, int k, const double* y, double* x, int64_t n,
                        cudaStream_t s);

}  // namespace dpp
