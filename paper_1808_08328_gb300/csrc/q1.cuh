// CG-VMS on Q1 quadrilaterals and hexahedra: the paper's QUAD and HEX meshes
// with the equal-order [Q1 + Q1]^2 spaces (Table "ELE_level_discretization"),
// the same blocks (Eq. "S4_cg_stiffness_matrix") and load (Eq. "S4_cg_rhs")
// as on simplices, with integrals that are no longer closed-form.
//
// A cell's vertices are in tensor order: vertex v sits at the reference
// corner with coordinate bits (v & 1, (v >> 1) & 1, (v >> 2) & 1) of
// [0,1]^d. The map is isoparametric, x(xi) = sum_v x_v phi_v(xi), with phi_v
// the product of xi_k (bit set) or 1 - xi_k. Integrals use the tensor
// 2-point Gauss rule (2^d points). It is exact on parallelepipeds and the
// standard rule otherwise. Per cell one table holds every integral the
// blocks and the load need:
//   M[a][b] = (phi_a; phi_b),  L[a][b] = (grad phi_a; grad phi_b),
//   G[a][b][k] = (phi_a; d_k phi_b),  IP[a] = (phi_a; 1),  IG[a][k] = (d_k phi_a; 1).
// The node-pair values then follow as on simplices:
//   m_i = 1/2 mu/k_i M,  K_up[k] = -(G[b][a][k] + 1/2 G[a][b][k]),
//   K_pu[k] = G[a][b][k] + 1/2 G[b][a][k],  d_i = 1/2 k_i/mu L + beta/mu M,  e = -beta/mu M,
// each summed over the cells holding both nodes in increasing cell id.
// Boundary facets carry W[a][b][k] = (psi_a psi_b; n_k)_F for the weak
// pressure term -(w.n; p0h)_F.
#pragma once

#include "kernels.cuh"

namespace dpp {
namespace q1 {

template <int DIM> struct Layout {
    static constexpr int NVC = 1 << DIM;          // vertices per cell
    static constexpr int NFV = 1 << (DIM - 1);    // vertices per facet
    static constexpr int M = 0;
    static constexpr int L = NVC * NVC;
    static constexpr int G = 2 * NVC * NVC;
    static constexpr int IP = (2 + DIM) * NVC * NVC;
    static constexpr int IG = IP + NVC;
    static constexpr int stride = IG + NVC * DIM;          // doubles per cell table
    static constexpr int fstride = NFV * NFV * DIM;        // doubles per facet table
};

__device__ __forceinline__ double gauss_point(int bit) {
    // 2-point Gauss-Legendre on [0,1]: 1/2 -+ 1/(2 sqrt 3)
    const double g = 0.28867513459481288225;
    return bit ? 0.5 + g : 0.5 - g;
}

// Value and reference gradient of basis function v at xi (D dimensions).
template <int D>
__device__ __forceinline__ double basis(int v, const double* xi, double* dphi) {
    double f[D], df[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const int bit = (v >> k) & 1;
        f[k] = bit ? xi[k] : 1.0 - xi[k];
        df[k] = bit ? 1.0 : -1.0;
    }
    double val = 1.0;
#pragma unroll
    for (int k = 0; k < D; ++k) val *= f[k];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        double p = df[k];
#pragma unroll
        for (int j = 0; j < D; ++j)
            if (j != k) p *= f[j];
        dphi[k] = p;
    }
    return val;
}

// Row a of the cell tables of cell c; one thread per (cell, vertex).
template <int DIM>
__global__ void k_cell_tables(const double* __restrict__ X, const int* __restrict__ cells,
                              int64_t n_cells, const double* __restrict__ lk1,
                              const double* __restrict__ lk2, double* __restrict__ tab,
                              double* __restrict__ kk, int* status) {
    using Lay = Layout<DIM>;
    constexpr int NVC = Lay::NVC;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_cells * NVC) return;
    const int64_t c = t / NVC;
    const int a = (int)(t % NVC);
    const int* cv = cells + c * NVC;
    double Mr[NVC], Lr[NVC], Gr[NVC][DIM], ip = 0.0, ig[DIM];
#pragma unroll
    for (int b = 0; b < NVC; ++b) {
        Mr[b] = Lr[b] = 0.0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) Gr[b][k] = 0.0;
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) ig[k] = 0.0;
    int neg = 0, pos = 0;
    for (int q = 0; q < NVC; ++q) {
        double xi[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) xi[k] = gauss_point((q >> k) & 1);
        // J[r][k] = dx_r / dxi_k
        double J[DIM][DIM];
#pragma unroll
        for (int r = 0; r < DIM; ++r)
#pragma unroll
            for (int k = 0; k < DIM; ++k) J[r][k] = 0.0;
        for (int v = 0; v < NVC; ++v) {
            double dphi[DIM];
            basis<DIM>(v, xi, dphi);
            const double* xv = X + (int64_t)cv[v] * DIM;
#pragma unroll
            for (int r = 0; r < DIM; ++r)
#pragma unroll
                for (int k = 0; k < DIM; ++k) J[r][k] += xv[r] * dphi[k];
        }
        // Jinv[k][r] = dxi_k / dx_r
        double Jinv[DIM][DIM], det;
        if constexpr (DIM == 2) {
            det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            const double id = 1.0 / det;
            Jinv[0][0] = J[1][1] * id;
            Jinv[0][1] = -J[0][1] * id;
            Jinv[1][0] = -J[1][0] * id;
            Jinv[1][1] = J[0][0] * id;
        } else {
            double C[3][3];
            C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
            C[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
            C[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
            C[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
            C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
            C[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
            C[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
            C[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
            C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            det = J[0][0] * C[0][0] + J[0][1] * C[1][0] + J[0][2] * C[2][0];
            const double id = 1.0 / det;
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int r = 0; r < 3; ++r) Jinv[k][r] = C[k][r] * id;
        }
        if (det > 0.0) ++pos;
        else if (det < 0.0) ++neg;
        const double w = fabs(det) / NVC;
        double dpa[DIM], ga[DIM];
        const double pa = basis<DIM>(a, xi, dpa);
#pragma unroll
        for (int r = 0; r < DIM; ++r) {
            ga[r] = 0.0;
#pragma unroll
            for (int k = 0; k < DIM; ++k) ga[r] += dpa[k] * Jinv[k][r];
        }
        ip += w * pa;
#pragma unroll
        for (int r = 0; r < DIM; ++r) ig[r] += w * ga[r];
        for (int b = 0; b < NVC; ++b) {
            double dpb[DIM], gb[DIM];
            const double pb = basis<DIM>(b, xi, dpb);
            double lg = 0.0;
#pragma unroll
            for (int r = 0; r < DIM; ++r) {
                gb[r] = 0.0;
#pragma unroll
                for (int k = 0; k < DIM; ++k) gb[r] += dpb[k] * Jinv[k][r];
                lg += ga[r] * gb[r];
            }
            Mr[b] += w * pa * pb;
            Lr[b] += w * lg;
#pragma unroll
            for (int r = 0; r < DIM; ++r) Gr[b][r] += w * pa * gb[r];
        }
    }
    if ((pos && neg) || pos + neg < NVC) atomicOr(status, kDevDegenerate);
    double* o = tab + c * Lay::stride;
#pragma unroll
    for (int b = 0; b < NVC; ++b) {
        o[Lay::M + a * NVC + b] = Mr[b];
        o[Lay::L + a * NVC + b] = Lr[b];
#pragma unroll
        for (int r = 0; r < DIM; ++r) o[Lay::G + (a * NVC + b) * DIM + r] = Gr[b][r];
    }
    o[Lay::IP + a] = ip;
#pragma unroll
    for (int r = 0; r < DIM; ++r) o[Lay::IG + a * DIM + r] = ig[r];
    if (a == 0) {
        kk[2 * c] = exp(lk1[c]);
        kk[2 * c + 1] = exp(lk2[c]);
    }
}

// One thread per node pair (self pairs included): the pair values, summed
// over the row node's cells that hold both nodes, in increasing cell id.
template <int DIM>
__global__ void k_assemble_pairs(const int* __restrict__ pair_row, const int* __restrict__ col,
                                 const int* __restrict__ row_ptr, int64_t n_pairs,
                                 const int* __restrict__ nc_ptr, const int* __restrict__ nc_list,
                                 const int* __restrict__ cells, const double* __restrict__ tab,
                                 const double* __restrict__ kk, double mu, double beta,
                                 const double* __restrict__ mub, const int* __restrict__ slice_ptr,
                                 double* __restrict__ sell_val) {
    using Lay = Layout<DIM>;
    constexpr int NVC = Lay::NVC;
    constexpr int NV = pair_values(DIM);
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    const int a = pair_row[p], b = col[p];
    double m1 = 0, m2 = 0, d1 = 0, d2 = 0, bm = 0, bu[DIM], cu[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) bu[k] = cu[k] = 0.0;
    for (int q = nc_ptr[a]; q < nc_ptr[a + 1]; ++q) {
        const int c = nc_list[q];
        int la = -1, lb = -1;
#pragma unroll
        for (int v = 0; v < NVC; ++v) {
            const int n = cells[(int64_t)c * NVC + v];
            if (n == a) la = v;
            if (n == b) lb = v;
        }
        if (lb < 0) continue;
        const double* T = tab + (int64_t)c * Lay::stride;
        const double muc = mub ? mub[2 * c] : mu, bc = mub ? mub[2 * c + 1] : beta;
        const double k1 = kk[2 * c], k2 = kk[2 * c + 1];
        const double Mab = T[Lay::M + la * NVC + lb];
        const double Lab = T[Lay::L + la * NVC + lb];
        m1 += 0.5 * muc / k1 * Mab;
        m2 += 0.5 * muc / k2 * Mab;
        bm += bc / muc * Mab;
        d1 += 0.5 * k1 / muc * Lab;
        d2 += 0.5 * k2 / muc * Lab;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const double gab = T[Lay::G + (la * NVC + lb) * DIM + k];  // (phi_a; d_k phi_b)
            const double gba = T[Lay::G + (lb * NVC + la) * DIM + k];  // (phi_b; d_k phi_a)
            bu[k] -= gba + 0.5 * gab;
            cu[k] += gab + 0.5 * gba;
        }
    }
    const int64_t grp = (int64_t)slice_ptr[a >> 5] + (p - row_ptr[a]);
    double* o = sell_val + grp * NV * kSell + (a & 31);
    o[0 * kSell] = m1;
    o[1 * kSell] = m2;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        o[(2 + k) * kSell] = bu[k];
        o[(2 + DIM + k) * kSell] = cu[k];
    }
    o[(2 + 2 * DIM) * kSell] = d1 + bm;
    o[(3 + 2 * DIM) * kSell] = d2 + bm;
    o[(4 + 2 * DIM) * kSell] = -bm;
}

// W[a][b][k] = (psi_a psi_b; n_k)_F per boundary facet, n pointing away from
// the owning cell (the incident cell of the first vertex that holds every
// vertex of the facet).
template <int DIM>
__global__ void k_facet_tables(const int* __restrict__ bf, int64_t n_bf,
                               const int* __restrict__ nc_ptr, const int* __restrict__ nc_list,
                               const int* __restrict__ cells, const double* __restrict__ X,
                               const double* __restrict__ p01, const double* __restrict__ p02,
                               double* __restrict__ W, int* status) {
    using Lay = Layout<DIM>;
    constexpr int NVC = Lay::NVC, NFV = Lay::NFV;
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_bf) return;
    int fv[NFV];
#pragma unroll
    for (int k = 0; k < NFV; ++k) fv[k] = bf[f * NFV + k];
    int owner = -1;
    for (int q = nc_ptr[fv[0]]; q < nc_ptr[fv[0] + 1] && owner < 0; ++q) {
        const int c = nc_list[q];
        int hits = 0;
        for (int v = 0; v < NVC; ++v) {
            const int n = cells[(int64_t)c * NVC + v];
#pragma unroll
            for (int k = 0; k < NFV; ++k) hits += (n == fv[k]);
        }
        if (hits == NFV) owner = c;
    }
    bool bad = false;
#pragma unroll
    for (int k = 0; k < NFV; ++k) bad |= !isfinite(p01[fv[k]]) || !isfinite(p02[fv[k]]);
    if (bad) atomicOr(status, kDevNonFinite);
    double* o = W + f * Lay::fstride;
    for (int i = 0; i < Lay::fstride; ++i) o[i] = 0.0;
    if (owner < 0) {
        atomicOr(status, kDevNoOwner);
        return;
    }
    double cen[DIM];
#pragma unroll
    for (int r = 0; r < DIM; ++r) cen[r] = 0.0;
    for (int v = 0; v < NVC; ++v)
#pragma unroll
        for (int r = 0; r < DIM; ++r) cen[r] += X[(int64_t)cells[(int64_t)owner * NVC + v] * DIM + r];
#pragma unroll
    for (int r = 0; r < DIM; ++r) cen[r] /= NVC;
    for (int sq = 0; sq < NFV; ++sq) {
        double s[DIM];  // facet coordinates (DIM - 1 used)
#pragma unroll
        for (int k = 0; k < DIM - 1; ++k) s[k] = gauss_point((sq >> k) & 1);
        double psi[NFV], x[DIM], T[DIM][DIM];
#pragma unroll
        for (int r = 0; r < DIM; ++r) {
            x[r] = 0.0;
#pragma unroll
            for (int k = 0; k < DIM; ++k) T[k][r] = 0.0;
        }
#pragma unroll
        for (int v = 0; v < NFV; ++v) {
            double dps[DIM];
            psi[v] = basis<DIM - 1>(v, s, dps);
            const double* xv = X + (int64_t)fv[v] * DIM;
#pragma unroll
            for (int r = 0; r < DIM; ++r) {
                x[r] += psi[v] * xv[r];
#pragma unroll
                for (int k = 0; k < DIM - 1; ++k) T[k][r] += dps[k] * xv[r];
            }
        }
        double n[DIM];
        if constexpr (DIM == 2) {
            n[0] = T[0][1];
            n[1] = -T[0][0];
        } else {
            n[0] = T[0][1] * T[1][2] - T[0][2] * T[1][1];
            n[1] = T[0][2] * T[1][0] - T[0][0] * T[1][2];
            n[2] = T[0][0] * T[1][1] - T[0][1] * T[1][0];
        }
        double dA = 0.0, side = 0.0;
#pragma unroll
        for (int r = 0; r < DIM; ++r) dA += n[r] * n[r];
        dA = sqrt(dA);
#pragma unroll
        for (int r = 0; r < DIM; ++r) side += n[r] * (x[r] - cen[r]);
        const double sg = (side < 0.0) ? -1.0 : 1.0;
        const double w = 1.0 / NFV;  // the rule's weight; dA * n_hat = n
#pragma unroll
        for (int a = 0; a < NFV; ++a)
#pragma unroll
            for (int b = 0; b < NFV; ++b)
#pragma unroll
                for (int k = 0; k < DIM; ++k) o[(a * NFV + b) * DIM + k] += w * sg * n[k] * psi[a] * psi[b];
        (void)dA;
    }
}

// Load vector per node: body terms over incident cells, then -(w.n; p0h)_F
// over incident boundary facets.
template <int DIM>
__global__ void k_rhs(int64_t n_nodes, const int* __restrict__ nc_ptr,
                      const int* __restrict__ nc_list, const int* __restrict__ cells,
                      const double* __restrict__ tab, const double* __restrict__ kk,
                      const int* __restrict__ nf_ptr, const int* __restrict__ nf_list,
                      const int* __restrict__ bf, const double* __restrict__ W,
                      const double* __restrict__ p01, const double* __restrict__ p02, double mu,
                      const double* __restrict__ mub, double gb0, double gb1, double gb2,
                      double* __restrict__ f) {
    using Lay = Layout<DIM>;
    constexpr int NVC = Lay::NVC, NFV = Lay::NFV, NS = 2 * DIM + 2;
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_nodes) return;
    const double gbv[3] = {gb0, gb1, gb2};
    double vsum = 0, fp1 = 0, fp2 = 0;
    for (int q = nc_ptr[a]; q < nc_ptr[a + 1]; ++q) {
        const int c = nc_list[q];
        int la = 0;
        for (int v = 0; v < NVC; ++v)
            if (cells[(int64_t)c * NVC + v] == a) la = v;
        const double* T = tab + (int64_t)c * Lay::stride;
        double gdot = 0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) gdot += T[Lay::IG + la * DIM + k] * gbv[k];
        const double muc = mub ? mub[2 * c] : mu;
        vsum += T[Lay::IP + la];
        fp1 += 0.5 * kk[2 * c] / muc * gdot;
        fp2 += 0.5 * kk[2 * c + 1] / muc * gdot;
    }
    double fu1[DIM], fu2[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) fu1[k] = fu2[k] = 0.5 * gbv[k] * vsum;
    for (int q = nf_ptr[a]; q < nf_ptr[a + 1]; ++q) {
        const int F = nf_list[q];
        int la = 0;
#pragma unroll
        for (int v = 0; v < NFV; ++v)
            if (bf[(int64_t)F * NFV + v] == a) la = v;
        const double* w = W + (int64_t)F * Lay::fstride;
#pragma unroll
        for (int v = 0; v < NFV; ++v) {
            const int b = bf[(int64_t)F * NFV + v];
            const double q1v = p01[b], q2v = p02[b];
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                fu1[k] -= w[(la * NFV + v) * DIM + k] * q1v;
                fu2[k] -= w[(la * NFV + v) * DIM + k] * q2v;
            }
        }
    }
    double* o = f + a * NS;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        o[k] = fu1[k];
        o[DIM + 1 + k] = fu2[k];
    }
    o[DIM] = fp1;
    o[2 * DIM + 1] = fp2;
}

// Adjoint sensitivities of one Q1 cell, as dpp::cell_sensitivity for simplices:
// the derivative of the element is -1/2 mu/k_i M (velocity), +1/2 k_i/mu L
// (pressure) and +1/2 k_i/mu IG . gamma_b (load); beta enters through M.
template <int DIM>
__device__ __forceinline__ void cell_sensitivity(int64_t c, const int* __restrict__ cells,
                                                 const double* __restrict__ tab,
                                                 const double* __restrict__ kk,
                                                 const double* __restrict__ x,
                                                 const double* __restrict__ lam, double mu,
                                                 const double (&gbv)[3], double& g1, double& g2,
                                                 double& beta_term) {
    using Lay = Layout<DIM>;
    constexpr int NVC = Lay::NVC, NS = 2 * DIM + 2;
    const double* T = tab + c * Lay::stride;
    const int* cv = cells + c * NVC;
    const double k1 = kk[2 * c], k2 = kk[2 * c + 1];
    double mu1 = 0, mu2 = 0, lp1 = 0, lp2 = 0, f1 = 0, f2 = 0, mb = 0;
    for (int a = 0; a < NVC; ++a) {
        const double* la = lam + (int64_t)cv[a] * NS;
        double gdot = 0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) gdot += T[Lay::IG + a * DIM + k] * gbv[k];
        f1 += la[DIM] * gdot;
        f2 += la[2 * DIM + 1] * gdot;
        for (int b = 0; b < NVC; ++b) {
            const double* xb = x + (int64_t)cv[b] * NS;
            const double m = T[Lay::M + a * NVC + b], l = T[Lay::L + a * NVC + b];
            double uu1 = 0, uu2 = 0;
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                uu1 += la[k] * xb[k];
                uu2 += la[DIM + 1 + k] * xb[DIM + 1 + k];
            }
            mu1 += m * uu1;
            mu2 += m * uu2;
            lp1 += l * la[DIM] * xb[DIM];
            lp2 += l * la[2 * DIM + 1] * xb[2 * DIM + 1];
            mb += m * (la[DIM] - la[2 * DIM + 1]) * (xb[DIM] - xb[2 * DIM + 1]);
        }
    }
    const double t1 = -0.5 * mu / k1 * mu1 + 0.5 * k1 / mu * lp1 - 0.5 * k1 / mu * f1;
    const double t2 = -0.5 * mu / k2 * mu2 + 0.5 * k2 / mu * lp2 - 0.5 * k2 / mu * f2;
    g1 = -t1;
    g2 = -t2;
    beta_term = -mb / mu;
}

}  // namespace q1
}  // namespace dpp
