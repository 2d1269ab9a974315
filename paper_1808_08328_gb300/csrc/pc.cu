// Field-split Schur preconditioner (Section 4.2, Method 2, "splitting by
// fields"; the appendix CG-VMS options: fieldsplit 0,2 | 1,3, schur, full,
// selfp, additive inner split).
//
// With K = [[A, B], [C, D]] (A the velocities of both networks, D the two
// pressures), the full factorisation gives
//   K^-1 = [[I, -A^-1 B], [0, I]] [[A^-1, 0], [0, S^-1]] [[I, 0], [-C A^-1, I]].
// Applied to r = (r_u, r_p) with approximate inverses:
//   y_u = Ainv r_u;  y_p = Sinv (r_p - C y_u);  z_u = Ainv (r_u - B y_p);  z_p = y_p.
// Ainv: a fixed Chebyshev-Jacobi polynomial on A = blockdiag(K1_uu, K2_uu)
// (default), or the paper's own ILU(0) of A (mass_solver = 1, ilu.cu).
// This replaces the paper's one sweep of ILU(0)/block Jacobi, which it
// chose because A is a mass matrix. The Chebyshev interval is exact: for P1
// simplices and any positive per-cell weights, eig(diag(M)^-1 M) lies in
// [1/2, (d+2)/2] (Wathen, IMA J. Numer. Anal. 7, 1987), i.e. [1/2, 2] on
// triangles and [1/2, 5/2] on tetrahedra.
// Sinv: one V-cycle of smoothed-aggregation AMG on blockdiag(S_p1, S_p2).
// This is the additive split of S_p into its diagonal blocks, with
// S_pi = Ki_pp - Ki_pu diag(Ki_uu)^-1 Ki_up (Eqs. "S4_sp1", "S4_sp2"). The
// coupling K12_pp = K21_pp is dropped in the preconditioner only; the outer
// Krylov method sees the full K.
// For K^T (the adjoint solve) B and C change sign and S_p is unchanged.
//
// Method 1 of Section 4.1 ("splitting by scales", composition = 1) groups
// {u1, p1} | {u2, p2}, drops the K12_pp coupling between the groups (additive
// outer split), and preconditions each network's 2x2 block by its own full
// Schur factorisation with the selfp matrix S^i_p of Eqs. "S4_sp1"/"S4_sp2".
// Written out, each group applies y_u^i = Ainv_i r_u^i, y_p^i = Sinv_i (r_p^i -
// K^i_pu y_u^i), z_u^i = Ainv_i (r_u^i - K^i_up y_p^i). Method 2 as composed
// here (A, B, C block-diagonal by network, additive split of S_p) applies the
// same steps. So both share the fused kernels below, which work on both
// networks in one launch. They differ in the multigrid: Method 1 builds one
// SA-AMG hierarchy per network on S^i_p alone, with its own aggregates,
// smoothing bounds and coarsest solve; Method 2 coarsens blockdiag(S_p1, S_p2)
// as one matrix, and its Chebyshev bounds come from the larger of the two
// spectra. With exact inner solves the two preconditioners would be equal,
// which is why the paper's KSP counts for the two methods agree.
#include "amg.cuh"

#include <cmath>

namespace dpp {

namespace {

template <class T>
void mass_chebyshev_poly(const ProblemImpl& P, const PcImpl& pc, const T* mdiag, const T* r,
                         T* target, T* tmp, T* dvec, cudaStream_t s);

// target_u = Ainv r_u: Chebyshev-Jacobi (default) or ILU(0) (mass_solver = 1).
template <class T>
void mass_chebyshev(const ProblemImpl& P, const PcImpl& pc, const T* mdiag, const T* r, T* target,
                    T* tmp, T* dvec, cudaStream_t s) {
    if (pc.opts.mass_solver == 1) mass_ilu_apply<T>(P, pc, r, target, s);
    else mass_chebyshev_poly<T>(P, pc, mdiag, r, target, tmp, dvec, s);
}

template <class T>
void mass_chebyshev_poly(const ProblemImpl& P, const PcImpl& pc, const T* mdiag, const T* r,
                         T* target, T* tmp, T* dvec, cudaStream_t s) {
    const int deg = std::max(1, pc.opts.cheb_degree_mass);
    const double lo = pc.mass_lmin, hi = pc.mass_lmax;
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
    double rho = 1.0 / sigma;
    const T* xin = nullptr;
    for (int k = 0; k < deg; ++k) {
        T* xout = ((deg - 1 - k) % 2 == 0) ? target : tmp;
        if (k == 0) {
            mass_cheb_step<T>(P, mdiag, r, nullptr, xout, dvec, 0.0, 1.0 / theta, true, s);
        } else {
            const double rho_new = 1.0 / (2.0 * sigma - rho);
            mass_cheb_step<T>(P, mdiag, r, xin, xout, dvec, rho_new * rho, 2.0 * rho_new / delta,
                              false, s);
            rho = rho_new;
        }
        xin = xout;
    }
}

__global__ void k_d2f_pc(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = (float)in[i];
}

void d2f(const double* in, float* out, int64_t n, cudaStream_t s) {
    k_d2f_pc<<<(int)std::min<int64_t>((n + 255) / 256, 8 * kSMs), 256, 0, s>>>(n, in, out);
    DPP_LAUNCH_CK();
}

__global__ void k_f2d_pc(int64_t n, const float* __restrict__ in, double* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = (double)in[i];
}


// Rows r0 .. r0+m-1 of S as an m x m matrix (columns shifted by -r0). Flags an
// entry outside the diagonal block: S must be block-diagonal there.
__global__ void k_block_rows_ptr(int64_t m, const int* __restrict__ rp, int64_t r0,
                                 int* __restrict__ orp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= m) orp[i] = rp[r0 + i] - rp[r0];
}
template <class V>
__global__ void k_block_rows_entries(int64_t nnz, int64_t m, const int* __restrict__ col,
                                     const V* __restrict__ val, int64_t e0, int64_t r0,
                                     int* __restrict__ ocol, V* __restrict__ oval, int* bad) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const int64_t c = (int64_t)col[e0 + e] - r0;
    if (c < 0 || c >= m) { atomicOr(bad, 1); ocol[e] = 0; oval[e] = V(0); return; }
    ocol[e] = (int)c;
    oval[e] = val[e0 + e];
}

void diagonal_block(const Csr& S, int64_t r0, int64_t m, Csr& out, cudaStream_t s,
                    HostScratch& hs) {
    const int64_t e0 = read_scalar(S.row_ptr.get() + r0, s, hs);
    const int64_t e1 = read_scalar(S.row_ptr.get() + r0 + m, s, hs);
    out.n_rows = out.n_cols = m;
    out.nnz = e1 - e0;
    out.row_ptr.alloc(m + 1);
    out.col.alloc(std::max<int64_t>(out.nnz, 1));
    const bool f32 = fp32_only(S);  // S_p of the mixed mode (FP32 values only)
    if (f32) out.val32.alloc(std::max<int64_t>(out.nnz, 1));
    else out.val.alloc(std::max<int64_t>(out.nnz, 1));
    k_block_rows_ptr<<<grid_for(m + 1, 256), 256, 0, s>>>(m, S.row_ptr.get(), r0, out.row_ptr.get());
    DPP_LAUNCH_CK();
    DBuf<int> bad(1);
    DPP_CK(cudaMemsetAsync(bad.get(), 0, sizeof(int), s));
    if (out.nnz) {
        if (f32)
            k_block_rows_entries<float><<<grid_for(out.nnz, 256), 256, 0, s>>>(
                out.nnz, m, S.col.get(), S.val32.get(), e0, r0, out.col.get(), out.val32.get(), bad.get());
        else
            k_block_rows_entries<double><<<grid_for(out.nnz, 256), 256, 0, s>>>(
                out.nnz, m, S.col.get(), S.val.get(), e0, r0, out.col.get(), out.val.get(), bad.get());
        DPP_LAUNCH_CK();
    }
    if (read_scalar(bad.get(), s, hs))
        fail(DPP_ERR_INVALID_ARGUMENT, "scale split: S_p couples the two networks");
}

// y_p = Sinv t_p on the split pressures [p1 | p2]: one V-cycle on
// blockdiag(S_p1, S_p2) (field split), or one per network (scale split).
template <class T>
void schur_vcycle(PcImpl& pc, const T* tp, T* yp, cudaStream_t s) {
    if (pc.n_amg == 1) {
        amg_vcycle<T>(pc.amg[0], pc.opts, tp, yp, s);
        return;
    }
    const int64_t n = pc.n_nodes;
    amg_vcycle<T>(pc.amg[0], pc.opts, tp, yp, s);
    amg_vcycle<T>(pc.amg[1], pc.opts, tp + n, yp + n, s);
}

}  // namespace

// FP32 -> FP64 copy (the widened values and results of the FP32 hierarchy)
void f2d(const float* in, double* out, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_f2d_pc<<<(int)std::min<int64_t>((n + 255) / 256, 8 * kSMs), 256, 0, s>>>(n, in, out);
    DPP_LAUNCH_CK();
}

void pc_setup(PcImpl& pc, const ProblemImpl& P, cudaStream_t s) {
    pc.dim = P.dim;
    pc.n_nodes = P.n_nodes;
    const int64_t n = P.n_nodes;
    const int64_t nn = n * P.ns;
    pc.mdiag.alloc(2 * n);
    mass_diag_inv(P, pc.mdiag.get(), pc.opts.use_lumped_diag != 0, s);
    if (P.kind == DPP_CELL_Q1) {
        // Q1 element mass on a parallelepiped: the d-fold tensor product of the
        // 1D P1 mass, so eig(diag(M_e)^-1 M_e) = products of {1/2, 3/2} and
        // eig(lumped(M_e)^-1 M_e) = products of {1/3, 1}; Wathen's argument
        // carries these element bounds to the assembled matrix
        const double d = P.dim;
        pc.mass_lmin = pc.opts.use_lumped_diag ? std::pow(1.0 / 3.0, d) : std::pow(0.5, d);
        pc.mass_lmax = pc.opts.use_lumped_diag ? 1.0 : std::pow(1.5, d);
    } else if (pc.opts.use_lumped_diag) {
        // eig(lumped(M)^-1 M) lies in [1/(d+2), 1] elementwise
        pc.mass_lmin = 1.0 / (P.dim + 2);
        pc.mass_lmax = 1.0;
    } else {
        pc.mass_lmin = 0.5;
        pc.mass_lmax = 0.5 * (P.dim + 2);
    }
    const bool mixed = pc.precision == DPP_MIXED_FP32_FP64;
    if (mixed) {
        // The mixed mode's hierarchy is built in FP32, from the FP32 pair values
        // (converted here if the problem was assembled in FP64 only) and FP32 M^-1.
        auto& Pm = const_cast<ProblemImpl&>(P);
        if (!Pm.sell_val32.get()) {
            Pm.sell_val32.alloc(P.sell_val.n);
            d2f(P.sell_val.get(), Pm.sell_val32.get(), (int64_t)P.sell_val.n, s);
        }
        pc.mdiag32.alloc(2 * n);
        d2f(pc.mdiag.get(), pc.mdiag32.get(), 2 * n, s);
    }
    Csr S;
    {
        ProfScope pr("setup_selfp", s, 0);
        if (mixed) build_selfp(P, pc.mdiag32.get(), S, s, pc.hs);
        else build_selfp(P, pc.mdiag.get(), S, s, pc.hs);
    }
    if (pc.opts.composition == kScaleSplit) {
        // Method 1: S^1_p and S^2_p, each with its own hierarchy
        Csr S1, S2;
        diagonal_block(S, 0, n, S1, s, pc.hs);
        diagonal_block(S, n, n, S2, s, pc.hs);
        S = Csr();
        pc.n_amg = 2;
        amg_setup(pc.amg[0], pc.opts, std::move(S1), s, pc.hs);
        amg_setup(pc.amg[1], pc.opts, std::move(S2), s, pc.hs);
    } else {
        pc.n_amg = 1;
        amg_setup(pc.amg[0], pc.opts, std::move(S), s, pc.hs);
    }
    if (pc.opts.mass_solver == 1) mass_ilu_setup(P, pc, s);
    pc.yu.alloc(nn);
    pc.su.alloc(nn);
    pc.tmp.alloc(nn);
    pc.dcheb.alloc(nn);
    pc.tp.alloc(2 * n);
    pc.yp.alloc(2 * n);
    DPP_CK(cudaMemsetAsync(pc.su.get(), 0, nn * sizeof(double), s));
    if (mixed) {
        // the FP32 hierarchy's work vectors
        for (int h = 0; h < pc.n_amg; ++h) amg_make_fp32(pc.amg[h], s);
        pc.yu32.alloc(nn);
        pc.su32.alloc(nn);
        pc.tmp32.alloc(nn);
        pc.dcheb32.alloc(nn);
        pc.tp32.alloc(2 * n);
        pc.yp32.alloc(2 * n);
        pc.r32.alloc(nn);
        DPP_CK(cudaMemsetAsync(pc.su32.get(), 0, nn * sizeof(float), s));
    }
    for (int h = 0; h < pc.n_amg; ++h) amg_tune(pc.amg[h], pc.opts, pc.precision, s);
    DPP_CK(cudaStreamSynchronize(s));
}

void pc_apply32(const ProblemImpl& P, PcImpl& pc, const double* r, float* z, bool transpose,
                cudaStream_t s);

// z = P^-1 r in FP64 (values, vectors and arithmetic). A mixed-precision
// preconditioner holds its FP32 hierarchy only: there z is its FP32 result,
// widened.
void pc_apply(const ProblemImpl& P, PcImpl& pc, const double* r, double* z, bool transpose,
              cudaStream_t s) {
    if (pc.precision == DPP_MIXED_FP32_FP64) {
        const int64_t nn = P.n_nodes * P.ns;
        DBuf<float> z32(nn);
        pc_apply32(P, pc, r, z32.get(), transpose, s);
        f2d(z32.get(), z, nn, s);
        return;
    }
    // 1. y_u = Ainv r_u
    mass_chebyshev<double>(P, pc, pc.mdiag.get(), r, pc.yu.get(), pc.tmp.get(), pc.dcheb.get(), s);
    // 2. t_p = r_p - C y_u   (split pressures [p1 | p2])
    apply_C_resid<double>(P, r, pc.yu.get(), pc.tp.get(), transpose, s);
    // 3. y_p = Sinv t_p: V-cycles on S_p1 and S_p2 (one shared hierarchy or one each)
    schur_vcycle<double>(pc, pc.tp.get(), pc.yp.get(), s);
    // 4. s_u = r_u - B y_p ;  z_u = Ainv s_u
    apply_B_resid<double>(P, r, pc.yp.get(), pc.su.get(), transpose, s);
    mass_chebyshev<double>(P, pc, pc.mdiag.get(), pc.su.get(), z, pc.tmp.get(), pc.dcheb.get(), s);
    // 5. z_p = y_p
    scatter_p<double>(P, pc.yp.get(), z, s);
}

// z32 = P^-1 r in FP32 (mixed mode): r is converted once, every preconditioner
// step runs on FP32 values and vectors, and the coarsest solve stays FP64.
void pc_apply32(const ProblemImpl& P, PcImpl& pc, const double* r, float* z, bool transpose,
                cudaStream_t s) {
    if (pc.precision != DPP_MIXED_FP32_FP64) fail(DPP_ERR_BAD_STATE, "pc has no FP32 hierarchy");
    float* r32 = pc.r32.get();
    d2f(r, r32, P.n_nodes * P.ns, s);
    mass_chebyshev<float>(P, pc, pc.mdiag32.get(), r32, pc.yu32.get(), pc.tmp32.get(),
                          pc.dcheb32.get(), s);
    apply_C_resid<float>(P, r32, pc.yu32.get(), pc.tp32.get(), transpose, s);
    schur_vcycle<float>(pc, pc.tp32.get(), pc.yp32.get(), s);
    apply_B_resid<float>(P, r32, pc.yp32.get(), pc.su32.get(), transpose, s);
    mass_chebyshev<float>(P, pc, pc.mdiag32.get(), pc.su32.get(), z, pc.tmp32.get(),
                          pc.dcheb32.get(), s);
    scatter_p<float>(P, pc.yp32.get(), z, s);
}

// z_u = Ainv r_u (the inner solve of the velocity block alone), p slots zero.
void pc_apply_mass(const ProblemImpl& P, PcImpl& pc, const double* r, double* z, cudaStream_t s) {
    DPP_CK(cudaMemsetAsync(z, 0, P.n_nodes * P.ns * sizeof(double), s));
    mass_chebyshev<double>(P, pc, pc.mdiag.get(), r, z, pc.tmp.get(), pc.dcheb.get(), s);
}

}  // namespace dpp
