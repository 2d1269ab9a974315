// Right-preconditioned flexible GMRES(m) (Saad, SIAM J. Sci. Comput. 14(2),
// 1993) on K x = f or K^T x = g. This is the outer Krylov method of the
// paper's Section 4.2; the paper uses PETSc GMRES, and the flexible variant
// tolerates a preconditioner that changes between iterations (the FP32 inner
// solve of the mixed-precision mode).
//
// Each iteration j:
//   z_j = P^-1 v_j;  w = K z_j;
//   classical Gram-Schmidt, h = V^T w, w -= V h, repeated once (h += V^T w,
//   w -= V h') when the first pass left less than reorth_eta of ||w||;
//   h_{j+1,j} = ||w||;  v_{j+1} = w / h_{j+1,j};
//   then a Givens rotation of column j of the Hessenberg matrix gives the
//   residual estimate |g_{j+1}|.
// The vectors and every O(n) operation stay on the device. Only the
// (m+1) x m Hessenberg matrix lives on the host, together with the j+2
// scalars copied back per iteration. The converged test uses the FP64 true
// residual ||f - K x||_2 / ||f||_2, evaluated when the estimate reaches the
// tolerance and at every restart.
//
// Mixed precision (GMRES-IR in the sense of Carson & Higham, SIAM J. Sci.
// Comput. 40(2), 2018): every restart cycle is one refinement step. The outer
// residual r = f - K x uses FP64 values and arithmetic. Inside the cycle,
// z_j = P^-1 v_j runs in the FP32 preconditioner (FP32 values, vectors and
// arithmetic; FP64 coarsest solve) and is stored in FP32, and w = K z_j uses
// the FP32 values with FP32 arithmetic. The Arnoldi basis V, CGS2, the
// Hessenberg matrix and the Givens rotations stay FP64. A cycle ends when its
// estimate has dropped by inner_rtol relative to the cycle's starting
// residual. Then x += Z y in FP64 and the FP64 residual is recomputed.
#include "amg.cuh"

#include <cmath>

namespace dpp {

void pc_apply(const ProblemImpl& P, PcImpl& pc, const double* r, double* z, bool transpose,
              cudaStream_t s);
void pc_apply32(const ProblemImpl& P, PcImpl& pc, const double* r, float* z, bool transpose,
                cudaStream_t s);

namespace {

struct Workspace {
    int m = 0;
    int64_t n = 0;
    DBuf<double> V, Z, w, r, dscal;  // dscal: [0..m] h, [m+1..2m+1] h', [2m+2] ||w||^2, [2m+3] ||r||^2
    DBuf<float> Z32;                 // preconditioned vectors in the mixed mode
    Reducer R;
    void init(int m_, int64_t n_, bool mixed) {
        m = m_;
        n = n_;
        V.alloc((size_t)(m + 1) * n);
        if (mixed) Z32.alloc((size_t)m * n);
        else Z.alloc((size_t)m * n);
        w.alloc(n);
        r.alloc(n);
        dscal.alloc(2 * m + 8);  // h | h' | ||w||^2 after | ||r||^2 | ||w||^2 before
    }
};

double device_norm(Workspace& W, const double* x, int64_t n, cudaStream_t s, HostScratch& hs) {
    dot(W.R, x, x, n, W.dscal.get() + 2 * W.m + 3, s);
    double v = read_scalar(W.dscal.get() + 2 * W.m + 3, s, hs);
    return std::sqrt(v);
}

}  // namespace

// Returns the dpp_status; fills iterations/restarts/rel_residual in info.
dpp_status fgmres(const ProblemImpl& P, PcImpl& pc, const dpp_solve_opts& o, const double* rhs,
                  double* x, bool transpose, dpp_solve_info& info, cudaStream_t s,
                  HostScratch& hs) {
    const int64_t n = P.n_nodes * P.ns;
    const int m = std::min(std::max(o.restart, 1), 64);
    const bool mixed = pc.precision == DPP_MIXED_FP32_FP64;
    Workspace W;
    W.init(m, n, mixed);
    info.iterations = 0;
    info.restarts = 0;
    const double bnorm = device_norm(W, rhs, n, s, hs);
    if (!std::isfinite(bnorm)) return DPP_ERR_NONFINITE;
    if (o.x0_zero) DPP_CK(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    if (bnorm == 0.0) {
        DPP_CK(cudaMemsetAsync(x, 0, n * sizeof(double), s));
        info.rel_residual = 0.0;
        return DPP_OK;
    }
    apply_K(P, x, W.r.get(), rhs, transpose, false, s);
    double beta = device_norm(W, W.r.get(), n, s, hs);
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    auto h_at = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
    dpp_status st = DPP_ERR_NOT_CONVERGED;
    while (true) {
        if (!std::isfinite(beta)) { st = DPP_ERR_NONFINITE; break; }
        info.rel_residual = beta / bnorm;
        if (info.rel_residual <= o.rtol) { st = DPP_OK; break; }
        if (info.iterations >= o.max_iters) { st = DPP_ERR_NOT_CONVERGED; break; }
        double* V = W.V.get();
        double* Z = W.Z.get();
        float* Z32 = W.Z32.get();
        const double cycle_target = mixed ? std::max(o.inner_rtol * beta, 0.5 * o.rtol * bnorm)
                                          : o.rtol * bnorm;
        axpby(1.0 / beta, W.r.get(), 0.0, V, n, s);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int j = 0, ncol = 0;
        bool breakdown = false, nonfinite = false;
        for (j = 0; j < m; ++j) {
            double* vj = V + (size_t)j * n;
            {
                ProfScope pp("krylov_pc", s, 0);
                if (mixed) {
                    float* zj = Z32 + (size_t)j * n;
                    pc_apply32(P, pc, vj, zj, transpose, s);
                    if (o.matrix_free) apply_K32_mf(P, zj, W.w.get(), transpose, s);
                    else apply_K32(P, zj, W.w.get(), transpose, s);
                } else {
                    double* zj = Z + (size_t)j * n;
                    pc_apply(P, pc, vj, zj, transpose, s);
                    if (o.matrix_free) apply_K_mf(P, zj, W.w.get(), transpose, s);
                    else apply_K(P, zj, W.w.get(), nullptr, transpose, false, s);
                }
            }
            double* hd = W.dscal.get();
            ProfScope po("krylov_orth", s, 0);
            // classical Gram-Schmidt; a second pass only when the first left less
            // than reorth_eta of ||w|| (the test of Daniel, Gragg, Kaufman &
            // Stewart, Math. Comp. 30, 1976, with a threshold chosen by measurement)
            ProfScope pk("krylov_orth_kernels", s, 0);
            dot(W.R, W.w.get(), W.w.get(), n, hd + 2 * m + 4, s);
            multidot(W.R, V, n, j + 1, W.w.get(), n, hd, s);
            multi_axpy_sub(V, n, j + 1, hd, W.w.get(), n, s);
            dot(W.R, W.w.get(), W.w.get(), n, hd + 2 * m + 2, s);
            pk.stop();
            ProfScope pw("krylov_orth_wait", s, 0);
            double* hh = (double*)hs.get((2 * m + 8) * sizeof(double));
            DPP_CK(cudaMemcpyAsync(hh, hd, (2 * m + 5) * sizeof(double), cudaMemcpyDeviceToHost, s));
            DPP_CK(cudaStreamSynchronize(s));
            const double eta = std::min(std::max(o.reorth_eta, 0.0), 1.0);
            const bool reorth = hh[2 * m + 2] < eta * eta * hh[2 * m + 4];
            for (int i = 0; i <= j; ++i) h_at(i, j) = hh[i];
            if (reorth) {
                multidot(W.R, V, n, j + 1, W.w.get(), n, hd + m + 1, s);
                multi_axpy_sub(V, n, j + 1, hd + m + 1, W.w.get(), n, s);
                dot(W.R, W.w.get(), W.w.get(), n, hd + 2 * m + 2, s);
                DPP_CK(cudaMemcpyAsync(hh, hd, (2 * m + 5) * sizeof(double), cudaMemcpyDeviceToHost, s));
                DPP_CK(cudaStreamSynchronize(s));
                for (int i = 0; i <= j; ++i) h_at(i, j) += hh[m + 1 + i];
            }
            pw.stop();
            const double hn = std::sqrt(std::max(hh[2 * m + 2], 0.0));
            h_at(j + 1, j) = hn;
            if (!std::isfinite(hn)) { nonfinite = true; ncol = j; break; }
            // apply previous rotations and form the new one
            for (int i = 0; i < j; ++i) {
                double t = cs[i] * h_at(i, j) + sn[i] * h_at(i + 1, j);
                h_at(i + 1, j) = -sn[i] * h_at(i, j) + cs[i] * h_at(i + 1, j);
                h_at(i, j) = t;
            }
            const double a = h_at(j, j), b = h_at(j + 1, j);
            const double rr = std::hypot(a, b);
            cs[j] = (rr > 0) ? a / rr : 1.0;
            sn[j] = (rr > 0) ? b / rr : 0.0;
            h_at(j, j) = rr;
            h_at(j + 1, j) = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++info.iterations;
            ncol = j + 1;
            const double est = std::fabs(g[j + 1]);
            if (hn <= 1e-300 * std::max(1.0, rr)) { breakdown = true; break; }  // exact subspace
            if (j + 1 < m) axpby(1.0 / hn, W.w.get(), 0.0, V + (size_t)(j + 1) * n, n, s);
            if (est <= cycle_target || info.iterations >= o.max_iters) break;
        }
        if (nonfinite) { st = DPP_ERR_NONFINITE; break; }
        // y = H^-1 g (upper triangular, ncol columns)
        for (int i = ncol - 1; i >= 0; --i) {
            double t = g[i];
            for (int k = i + 1; k < ncol; ++k) t -= h_at(i, k) * y[k];
            y[i] = t / h_at(i, i);
        }
        double* yd = W.dscal.get();
        DPP_CK(cudaMemcpyAsync(yd, y.data(), ncol * sizeof(double), cudaMemcpyHostToDevice, s));
        if (mixed) multi_axpy_add_f32(Z32, n, ncol, yd, x, n, s);
        else multi_axpy_add(Z, n, ncol, yd, x, n, s);
        apply_K(P, x, W.r.get(), rhs, transpose, false, s);
        beta = device_norm(W, W.r.get(), n, s, hs);
        ++info.restarts;
        if (breakdown && !mixed && beta / bnorm > o.rtol) {
            info.rel_residual = beta / bnorm;
            st = DPP_ERR_BREAKDOWN;
            break;
        }
    }
    DPP_CK(cudaStreamSynchronize(s));
    return st;
}

}  // namespace dpp
