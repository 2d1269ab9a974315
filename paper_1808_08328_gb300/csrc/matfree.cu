// Matrix-free, element-by-element application of the CG-VMS operator:
// y = K x (or K^T x) without the assembled pair values (dpp_apply_K_mf,
// dpp_apply_K32_mf, and the inner K z of the solver when
// dpp_solve_opts::matrix_free is set).
//
// Paper: the blocks of Eq. "S4_cg_stiffness_matrix" from the form of Eq.
// "CG_VMS_Weak_form". On a P1 simplex with measure |K|, basis gradients g_b,
// M(a, b) = |K| (1 + delta_ab) / ((d+1)(d+2)) and w = |K| / (d+1), the
// element's action on row a needs only these sums over the cell's vertices,
// per network i:
//   S_u = sum_b u_b,  S_p = sum_b p_b,  G_p = sum_b g_b p_b (grad p_h),
//   div = sum_b g_b . u_b (div u_h).
// Row a then receives
//   u_i:  1/2 mu/k_i cm (u_a + S_u)  -  s w (g_a S_p + 1/2 G_p)
//   p_i:  s w (div + 1/2 g_a . S_u) + 1/2 k_i/mu |K| g_a . G_p
//         + beta/mu cm (p_i,a + S_p,i) - beta/mu cm (p_j,a + S_p,j)    (j the other network)
// with cm = |K| / ((d+1)(d+2)), s = +1 for K and -1 for K^T (K^T is K with the
// K_up and K_pu blocks negated).
//
// Layout and order: G = 2 lanes per node take the node's incident cells in
// increasing cell id, G apart. Each lane recomputes the cell's geometry from
// the vertex coordinates (the inverse of the edge matrix) and gathers the four
// (three) vertex vectors. The lanes then add their partial rows in a fixed
// butterfly order, so the result is bit-reproducible. There are no atomics.
//
// Bytes per apply: the node->cell lists, the cells' vertex ids and k values,
// the coordinates, x and y. Each is read once when L2 holds the window of cells
// that neighbouring nodes share. At 3D 64^3 in FP32 that is about 95 MB (DRAM
// measured 81 MB), against 220 MB for the assembled FP32 pair values. But each
// cell's vertex data is gathered once per vertex node: about 220 B of L1
// traffic per (node, cell), 1.45 GB per apply at 64^3. That, not DRAM, bounds
// the kernel (96 us against 51 us for the assembled FP32 apply). In FP64 the
// FP64 pipe bounds the recomputed geometry and the element action (3.1 ms).
#include "kernels.cuh"

namespace dpp {

namespace {

template <class T> __device__ __forceinline__ T ld(const T* p) { return __ldg(p); }

// The FP32 3D path reads through vector loads: coordinates padded to float4,
// the node's 8 unknowns as two float4, the cell's 4 vertex ids as one int4.
template <int DIM, class T> struct MfVec {
    static constexpr bool on = (DIM == 3) && sizeof(T) == 4;
    static constexpr int xs = on ? 4 : DIM;  // coordinate stride
};

template <int DIM, class T, class YT, bool TRANS, int G>
__global__ void __launch_bounds__(256, (sizeof(T) == 4) ? 4 : 2)
k_apply_K_mf(int64_t n_nodes, const int* __restrict__ nc_ptr, const int* __restrict__ nc_list,
             const int* __restrict__ cells, const T* __restrict__ X, const T* __restrict__ kk,
             const T* __restrict__ mub, T mu, T beta, const T* __restrict__ x,
             YT* __restrict__ y) {
    constexpr int NV = DIM + 1;
    constexpr int NS = 2 * DIM + 2;
    static_assert(G == 1 || G == 2 || G == 4 || G == 8 || G == 16 || G == 32,
                  "group of lanes within a warp");
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t a = t / G;
    const int lane = (int)(t % G);
    // whole groups leave together, so the group shuffles below see full groups
    if (a >= n_nodes) return;
    using V = MfVec<DIM, T>;
    constexpr int XS = V::xs;
    const T sB = TRANS ? T(-1) : T(1);
    T acc[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[s] = T(0);
    const int q1 = nc_ptr[a + 1];
    for (int q = nc_ptr[a] + lane; q < q1; q += G) {
        const int c = nc_list[q];
        int v[NV];
        if constexpr (V::on) {
            const int4 cv = __ldg(reinterpret_cast<const int4*>(cells) + c);
            v[0] = cv.x;
            v[1] = cv.y;
            v[2] = cv.z;
            v[3] = cv.w;
        } else {
#pragma unroll
            for (int k = 0; k < NV; ++k) v[k] = ld(cells + (int64_t)c * NV + k);
        }
        // geometry: J = [x_1 - x_0, ..., x_d - x_0]; g_{k+1} = row k of J^-1
        T xv[NV][DIM], J[DIM][DIM];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            if constexpr (V::on) {
                const float4 q = __ldg(reinterpret_cast<const float4*>(X) + v[k]);
                xv[k][0] = q.x;
                xv[k][1] = q.y;
                xv[k][2] = q.z;
            } else {
#pragma unroll
                for (int r = 0; r < DIM; ++r) xv[k][r] = ld(X + (int64_t)v[k] * XS + r);
            }
        }
#pragma unroll
        for (int q2 = 0; q2 < DIM; ++q2)
#pragma unroll
            for (int r = 0; r < DIM; ++r) J[r][q2] = xv[q2 + 1][r] - xv[0][r];
        T g[NV][DIM], det;
        if constexpr (DIM == 2) {
            det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            const T id = T(1) / det;
            g[1][0] = J[1][1] * id;
            g[1][1] = -J[0][1] * id;
            g[2][0] = -J[1][0] * id;
            g[2][1] = J[0][0] * id;
        } else {
            T inv[3][3];
            inv[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
            inv[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
            inv[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
            det = J[0][0] * inv[0][0] + J[0][1] * inv[1][0] + J[0][2] * inv[2][0];
            inv[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
            inv[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
            inv[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
            inv[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
            inv[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
            inv[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            const T id = T(1) / det;
#pragma unroll
            for (int q2 = 0; q2 < 3; ++q2)
#pragma unroll
                for (int r = 0; r < 3; ++r) g[q2 + 1][r] = inv[q2][r] * id;
        }
#pragma unroll
        for (int r = 0; r < DIM; ++r) {
            T s = T(0);
#pragma unroll
            for (int k = 1; k < NV; ++k) s += g[k][r];
            g[0][r] = -s;
        }
        const T vol = (det < T(0) ? -det : det) / T(DIM == 2 ? 2 : 6);
        // the cell-level sums, and the row node's own values
        T Su1[DIM], Su2[DIM], Gp1[DIM], Gp2[DIM], ua1[DIM], ua2[DIM], ga[DIM];
        T Sp1 = 0, Sp2 = 0, dv1 = 0, dv2 = 0, pa1 = 0, pa2 = 0;
#pragma unroll
        for (int r = 0; r < DIM; ++r) Su1[r] = Su2[r] = Gp1[r] = Gp2[r] = ua1[r] = ua2[r] = ga[r] = T(0);
#pragma unroll
        for (int b = 0; b < NV; ++b) {
            const T* xb = x + (int64_t)v[b] * NS;
            T u1[DIM], u2[DIM], p1, p2;
            if constexpr (V::on) {
                const float4 lo = __ldg(reinterpret_cast<const float4*>(xb));
                const float4 hi = __ldg(reinterpret_cast<const float4*>(xb) + 1);
                u1[0] = lo.x;
                u1[1] = lo.y;
                u1[2] = lo.z;
                p1 = lo.w;
                u2[0] = hi.x;
                u2[1] = hi.y;
                u2[2] = hi.z;
                p2 = hi.w;
            } else {
#pragma unroll
                for (int r = 0; r < DIM; ++r) {
                    u1[r] = ld(xb + r);
                    u2[r] = ld(xb + DIM + 1 + r);
                }
                p1 = ld(xb + DIM);
                p2 = ld(xb + 2 * DIM + 1);
            }
            const bool self = (v[b] == (int)a);
#pragma unroll
            for (int r = 0; r < DIM; ++r) {
                Su1[r] += u1[r];
                Su2[r] += u2[r];
                Gp1[r] += g[b][r] * p1;
                Gp2[r] += g[b][r] * p2;
                dv1 += g[b][r] * u1[r];
                dv2 += g[b][r] * u2[r];
                if (self) {
                    ua1[r] = u1[r];
                    ua2[r] = u2[r];
                    ga[r] = g[b][r];
                }
            }
            Sp1 += p1;
            Sp2 += p2;
            if (self) {
                pa1 = p1;
                pa2 = p2;
            }
        }
        T k1, k2;
        if constexpr (V::on) {
            const float2 kv = __ldg(reinterpret_cast<const float2*>(kk) + c);
            k1 = kv.x;
            k2 = kv.y;
        } else {
            k1 = ld(kk + 2 * (int64_t)c);
            k2 = ld(kk + 2 * (int64_t)c + 1);
        }
        const T muc = mub ? ld(mub + 2 * (int64_t)c) : mu;
        const T bc = mub ? ld(mub + 2 * (int64_t)c + 1) : beta;
        const T cm = vol / T((DIM + 1) * (DIM + 2));
        const T w = vol / T(DIM + 1);
        const T m1 = T(0.5) * muc / k1 * cm, m2 = T(0.5) * muc / k2 * cm;
        const T s1 = T(0.5) * k1 / muc * vol, s2 = T(0.5) * k2 / muc * vol;
        const T tb = bc / muc * cm * ((pa1 + Sp1) - (pa2 + Sp2));
        T gs1 = 0, gs2 = 0, gg1 = 0, gg2 = 0;
#pragma unroll
        for (int r = 0; r < DIM; ++r) {
            acc[r] += m1 * (ua1[r] + Su1[r]) - sB * w * (ga[r] * Sp1 + T(0.5) * Gp1[r]);
            acc[DIM + 1 + r] += m2 * (ua2[r] + Su2[r]) - sB * w * (ga[r] * Sp2 + T(0.5) * Gp2[r]);
            gs1 += ga[r] * Su1[r];
            gs2 += ga[r] * Su2[r];
            gg1 += ga[r] * Gp1[r];
            gg2 += ga[r] * Gp2[r];
        }
        acc[DIM] += sB * w * (dv1 + T(0.5) * gs1) + s1 * gg1 + tb;
        acc[2 * DIM + 1] += sB * w * (dv2 + T(0.5) * gs2) + s2 * gg2 - tb;
    }
    // fixed-order butterfly over the group's lanes (only this group's lanes
    // take part: groups past the last node have left)
    const unsigned gmask =
        (G == 32) ? 0xffffffffu : (((1u << (G & 31)) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
        for (int s = 0; s < NS; ++s) acc[s] += __shfl_xor_sync(gmask, acc[s], off, G);
    YT* ya = y + a * NS;
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if (s % G == lane) ya[s] = (YT)acc[s];
}

__global__ void k_pad_coords(int64_t n, const double* __restrict__ X, float* __restrict__ X4) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    X4[4 * i] = (float)X[3 * i];
    X4[4 * i + 1] = (float)X[3 * i + 1];
    X4[4 * i + 2] = (float)X[3 * i + 2];
    X4[4 * i + 3] = 0.0f;
}

__global__ void k_mf_float_copy(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

template <class T> const T* coords_of(const ProblemImpl& P);
template <> const double* coords_of<double>(const ProblemImpl& P) { return P.coords.get(); }
template <> const float* coords_of<float>(const ProblemImpl& P) { return P.coords32.get(); }
template <class T> const T* kk_of(const ProblemImpl& P);
template <> const double* kk_of<double>(const ProblemImpl& P) { return P.kk.get(); }
template <> const float* kk_of<float>(const ProblemImpl& P) { return P.kk32.get(); }
template <class T> const T* mub_of(const ProblemImpl& P);
template <> const double* mub_of<double>(const ProblemImpl& P) { return P.cell_mu_beta.get(); }
template <> const float* mub_of<float>(const ProblemImpl& P) { return P.cell_mu_beta32.get(); }

template <int DIM, class T, class YT>
void apply_mf_dim(const ProblemImpl& P, const T* x, YT* y, bool tr, cudaStream_t s) {
    // lanes per node, measured at 3D 64^3 in FP32: 1: 136 us, 2: 96 us, 4: 100 us,
    // 8: 126 us, 16: 187 us, 32: 289 us (the group's final reduction and idle
    // lanes cost more than the extra parallelism buys)
    constexpr int G = 2;
    const double n = (double)P.n_nodes, nc = (double)P.n_cells;
    const double alg = (n + 1) * 4.0 + nc * (DIM + 1) * 4.0 * 2.0 +
                       nc * 2.0 * sizeof(T) * (P.cell_mu_beta.get() ? 2.0 : 1.0) +
                       n * MfVec<DIM, T>::xs * sizeof(T) + n * P.ns * (double)(sizeof(T) + sizeof(YT));
    ProfScope prof(sizeof(T) == 8 ? "apply_K_mf" : "apply_K_mf_fp32", s, alg);
    const int B = 256;
    const int grid = grid_for(P.n_nodes * G, B);
    const T* mub = mub_of<T>(P);
    if (tr)
        k_apply_K_mf<DIM, T, YT, true, G><<<grid, B, 0, s>>>(
            P.n_nodes, P.nc_ptr.get(), P.nc_list.get(), P.cells.get(), coords_of<T>(P), kk_of<T>(P),
            mub, (T)P.mu, (T)P.beta, x, y);
    else
        k_apply_K_mf<DIM, T, YT, false, G><<<grid, B, 0, s>>>(
            P.n_nodes, P.nc_ptr.get(), P.nc_list.get(), P.cells.get(), coords_of<T>(P), kk_of<T>(P),
            mub, (T)P.mu, (T)P.beta, x, y);
    DPP_LAUNCH_CK();
}

void to_f32(const DBuf<double>& in, DBuf<float>& out, cudaStream_t s) {
    out.alloc(in.n);
    if (in.n) {
        k_mf_float_copy<<<grid_for((int64_t)in.n, 256), 256, 0, s>>>((int64_t)in.n, in.get(),
                                                                      out.get());
        DPP_LAUNCH_CK();
    }
}

}  // namespace

void matrix_free_prepare32(ProblemImpl& P, cudaStream_t s) {
    if (P.coords32.get()) return;
    if (P.dim == 3) {  // padded to 4 floats per node for one float4 load
        P.coords32.alloc(P.n_nodes * 4);
        k_pad_coords<<<grid_for(P.n_nodes, 256), 256, 0, s>>>(P.n_nodes, P.coords.get(),
                                                               P.coords32.get());
        DPP_LAUNCH_CK();
    } else {
        to_f32(P.coords, P.coords32, s);
    }
    to_f32(P.kk, P.kk32, s);
    if (P.cell_mu_beta.get()) to_f32(P.cell_mu_beta, P.cell_mu_beta32, s);
}

void apply_K_mf(const ProblemImpl& P, const double* x, double* y, bool tr, cudaStream_t s) {
    if (P.dim == 2) apply_mf_dim<2, double, double>(P, x, y, tr, s);
    else apply_mf_dim<3, double, double>(P, x, y, tr, s);
}

void apply_K32_mf(const ProblemImpl& P, const float* x, double* y, bool tr, cudaStream_t s) {
    if (!P.coords32.get()) fail(DPP_ERR_BAD_STATE, "FP32 geometry was not prepared");
    if (P.dim == 2) apply_mf_dim<2, float, double>(P, x, y, tr, s);
    else apply_mf_dim<3, float, double>(P, x, y, tr, s);
}

}  // namespace dpp
