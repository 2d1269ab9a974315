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
// Matrix-free y = K x (transpose: K^T x) from the cells' geometry and k, with no
// assembled values (matfree.cu): FP64 throughout, or FP32 geometry, k, x and
// arithmetic with FP64 output (after matrix_free_prepare32).
void apply_K_mf(const ProblemImpl& P, const double* x, double* y, bool transpose, cudaStream_t s);
void apply_K32_mf(const ProblemImpl& P, const float* x, double* y, bool transpose, cudaStream_t s);
void matrix_free_prepare32(ProblemImpl& P, cudaStream_t s);
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
// ILU(0) of the velocity mass blocks (ilu.cu): factor at setup; apply writes
// target's velocity slots = (L U)^-1 r's velocity slots (target != r).
void mass_ilu_setup(const ProblemImpl& P, PcImpl& pc, cudaStream_t s);
template <class T>
void mass_ilu_apply(const ProblemImpl& P, const PcImpl& pc, const T* r, T* target, cudaStream_t s);
// mdiag[a][net] = 1 / m_net(a, a) (or the row sum when lumped)
void mass_diag_inv(const ProblemImpl& P, double* mdiag, bool lumped, cudaStream_t s);
// z_p(net)[a] = yp[net][a] (copy split pressures into interleaved p slots)
template <class T>
void scatter_p(const ProblemImpl& P, const T* yp, T* z, cudaStream_t s);

// ---- adjoint sensitivities of one cell (shared by adjoint.cu and noalloc.cu) ----
// For cell c of the CG-VMS form: g1 = dJ/dlog k1_c and g2 = dJ/dlog k2_c, i.e.
// -lambda^T (dK/dlog k_i x - df/dlog k_i) with the derivative -1/2 mu/k_i M_c on
// the velocity block, +1/2 k_i/mu L_c on the pressure block and
// +1/2 k_i/mu |K| g_a . gamma_b on the load; and the cell's share of dJ/dbeta,
// -(1/mu) (lambda_p1 - lambda_p2)^T M_c (x_p1 - x_p2). M_c = |K| (1 + delta_ab) /
// ((d+1)(d+2)) and L_c = |K| g_a . g_b are exact for P1.
template <int DIM>
__device__ __forceinline__ void cell_sensitivity(int64_t c, const int* __restrict__ cells,
                                                 const double* __restrict__ geo,
                                                 const double* __restrict__ kk,
                                                 const double* __restrict__ x,
                                                 const double* __restrict__ lam, double mu,
                                                 const double (&gbv)[3], double& g1, double& g2,
                                                 double& beta_term) {
    constexpr int S = GeoLayout<DIM>::stride;
    constexpr int NS = 2 * DIM + 2;
    constexpr int NV = DIM + 1;
    int v[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = cells[c * NV + a];
    const double* g = geo + c * S;
    const double vol = g[0];
    const double k1 = kk[2 * c], k2 = kk[2 * c + 1];
    const double cm = vol / ((DIM + 1) * (DIM + 2));
    double mu1 = 0, mu2 = 0, lp1 = 0, lp2 = 0, f1 = 0, f2 = 0, mb = 0;
#pragma unroll
    for (int a = 0; a < NV; ++a) {
        const double* la = lam + (int64_t)v[a] * NS;
        const double* ga = g + 1 + a * DIM;
        double gdot = 0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) gdot += ga[k] * gbv[k];
        f1 += la[DIM] * gdot;
        f2 += la[2 * DIM + 1] * gdot;
#pragma unroll
        for (int b = 0; b < NV; ++b) {
            const double* xb = x + (int64_t)v[b] * NS;
            const double* gbb = g + 1 + b * DIM;
            const double m = cm * (a == b ? 2.0 : 1.0);
            double lg = 0, uu1 = 0, uu2 = 0;
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                lg += ga[k] * gbb[k];
                uu1 += la[k] * xb[k];
                uu2 += la[DIM + 1 + k] * xb[DIM + 1 + k];
            }
            mu1 += m * uu1;
            mu2 += m * uu2;
            lp1 += vol * lg * la[DIM] * xb[DIM];
            lp2 += vol * lg * la[2 * DIM + 1] * xb[2 * DIM + 1];
            mb += m * (la[DIM] - la[2 * DIM + 1]) * (xb[DIM] - xb[2 * DIM + 1]);
        }
    }
    // lambda^T dK x with dK = -1/2 mu/k M (uu) + 1/2 k/mu L (pp); minus lambda^T df
    const double t1 = -0.5 * mu / k1 * mu1 + 0.5 * k1 / mu * lp1 - 0.5 * k1 / mu * vol * f1;
    const double t2 = -0.5 * mu / k2 * mu2 + 0.5 * k2 / mu * lp2 - 0.5 * k2 / mu * vol * f2;
    g1 = -t1;
    g2 = -t2;
    beta_term = -mb / mu;
}

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
