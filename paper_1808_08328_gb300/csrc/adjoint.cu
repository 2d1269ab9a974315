// Assembly sensitivities for the adjoint gradient (dpp_adjoint_solve).
//
// With K(theta) x = f(theta) (Eq. "S4_linear_problem") and K^T lambda = dJ/dx:
//   dJ/dtheta = -lambda^T (dK/dtheta x - df/dtheta).
// On one cell c of the CG-VMS form (Eq. "S4_cg_stiffness_matrix"), log k1_c
// enters only two terms. The velocity mass 1/2 (w1; mu/k1 u1) has
// derivative -1/2 mu/k1 M_c. The pressure stiffness 1/2 (grad q1; k1/mu grad p1)
// has derivative +1/2 k1/mu L_c. The load term 1/2 (grad q1; k1/mu gamma b)
// (Eq. "S4_cg_rhs") has derivative 1/2 k1/mu |K| g_a . gamma_b. The
// cross terms -1/2 (w1; grad p1) and 1/2 (grad q1; u1) do not depend on k1.
// log k2 works the same way. beta enters only (q1 - q2; beta/mu (p1 - p2)),
// so dJ/dbeta = -(1/mu) sum_c (lambda_p1 - lambda_p2)^T M_c (x_p1 - x_p2).
// M_c = |K| (1 + delta_ab) / ((d+1)(d+2)) and L_c = |K| g_a . g_b are exact
// for P1. On Q1 cells the same derivatives use the cell's integral tables
// (q1.cuh). One thread per cell; the beta sum is a deterministic two-level
// reduction of per-cell terms.
#include "q1.cuh"

namespace dpp {

namespace {

template <int DIM>
__global__ void k_cell_sensitivity(int64_t n_cells, const int* __restrict__ cells,
                                   const double* __restrict__ geo, const double* __restrict__ kk,
                                   const double* __restrict__ x, const double* __restrict__ lam,
                                   double mu, double gb0, double gb1, double gb2,
                                   double* __restrict__ g1, double* __restrict__ g2,
                                   double* __restrict__ gbeta_cell) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const double gbv[3] = {gb0, gb1, gb2};
    double t1, t2, tb;
    cell_sensitivity<DIM>(c, cells, geo, kk, x, lam, mu, gbv, t1, t2, tb);
    g1[c] = t1;
    g2[c] = t2;
    gbeta_cell[c] = tb;
}

template <int DIM>
__global__ void k_cell_sensitivity_q1(int64_t n_cells, const int* __restrict__ cells,
                                      const double* __restrict__ tab,
                                      const double* __restrict__ kk, const double* __restrict__ x,
                                      const double* __restrict__ lam, double mu, double gb0,
                                      double gb1, double gb2, double* __restrict__ g1,
                                      double* __restrict__ g2, double* __restrict__ gbeta_cell) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const double gbv[3] = {gb0, gb1, gb2};
    double t1, t2, tb;
    q1::cell_sensitivity<DIM>(c, cells, tab, kk, x, lam, mu, gbv, t1, t2, tb);
    g1[c] = t1;
    g2[c] = t2;
    gbeta_cell[c] = tb;
}

}  // namespace

void adjoint_gradients(const ProblemImpl& P, const double* x, const double* lambda, double* g1,
                       double* g2, double* gbeta, cudaStream_t s) {
    DBuf<double> tmp(P.n_cells), ones(P.n_cells);
    const int B = 256;
    if (P.kind == DPP_CELL_Q1) {
        if (P.dim == 2)
            k_cell_sensitivity_q1<2><<<grid_for(P.n_cells, B), B, 0, s>>>(
                P.n_cells, P.cells.get(), P.q1tab.get(), P.kk.get(), x, lambda, P.mu, P.gb[0],
                P.gb[1], P.gb[2], g1, g2, tmp.get());
        else
            k_cell_sensitivity_q1<3><<<grid_for(P.n_cells, B), B, 0, s>>>(
                P.n_cells, P.cells.get(), P.q1tab.get(), P.kk.get(), x, lambda, P.mu, P.gb[0],
                P.gb[1], P.gb[2], g1, g2, tmp.get());
    } else if (P.dim == 2)
        k_cell_sensitivity<2><<<grid_for(P.n_cells, B), B, 0, s>>>(
            P.n_cells, P.cells.get(), P.geo.get(), P.kk.get(), x, lambda, P.mu, P.gb[0], P.gb[1],
            P.gb[2], g1, g2, tmp.get());
    else
        k_cell_sensitivity<3><<<grid_for(P.n_cells, B), B, 0, s>>>(
            P.n_cells, P.cells.get(), P.geo.get(), P.kk.get(), x, lambda, P.mu, P.gb[0], P.gb[1],
            P.gb[2], g1, g2, tmp.get());
    DPP_LAUNCH_CK();
    fill(ones.get(), 1.0, P.n_cells, s);
    Reducer R;
    dot(R, tmp.get(), ones.get(), P.n_cells, gbeta, s);
    DPP_CK(cudaStreamSynchronize(s));
}

}  // namespace dpp
