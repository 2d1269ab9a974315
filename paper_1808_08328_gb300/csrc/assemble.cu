// Assembly of the CG-VMS P1 system on the device (dpp_assemble).
//
// Paper: the block entries of Eq. "S4_cg_stiffness_matrix" and the load of
// Eq. "S4_cg_rhs" (Section 4), from the stabilised form of Eq.
// "CG_VMS_Weak_form" (Section 3.3). On a P1 simplex K with measure |K| and
// constant basis gradients g_a, the integrals are closed-form:
//   (phi_a; phi_b)_K = |K| (1 + delta_ab) / ((d+1)(d+2)),
//   (phi_a; 1)_K     = |K| / (d+1),
//   (grad phi_a; grad phi_b)_K = |K| g_a . g_b.
// A node pair (a, b) therefore carries
//   m_i   = 1/2 sum_K mu/k_i (phi_a; phi_b)                (K^i_uu, per component)
//   Kup_c = sum_K -|K|/(d+1) (g_a[c] + 1/2 g_b[c])       (K^i_up, both networks)
//   Kpu_c = sum_K  |K|/(d+1) (g_b[c] + 1/2 g_a[c])       (K^i_pu, both networks)
//   d_i   = sum_K 1/2 k_i/mu |K| g_a.g_b + beta/mu (phi_a; phi_b)   (K^i_pp)
//   e     = -sum_K beta/mu (phi_a; phi_b)                 (K^12_pp = K^21_pp)
// Every sum runs over the cells that contain both a and b, in increasing cell
// id. It is a fixed-order gather (no floating-point atomics), so K is
// bit-reproducible.
#include "q1.cuh"

namespace dpp {

namespace {

constexpr int kMaxRow = 96;  // max node-pair row length (distinct neighbours + self)

template <int NVC>
__global__ void k_validate_cells(const int* __restrict__ cells, int64_t n_cells, int64_t n_nodes,
                                 const double* __restrict__ lk1, const double* __restrict__ lk2,
                                 int* status) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    int bad = 0;
#pragma unroll
    for (int v = 0; v < NVC; ++v) {
        int a = cells[c * NVC + v];
        if (a < 0 || a >= n_nodes) bad |= kDevBadIndex;
    }
    if (!isfinite(lk1[c]) || !isfinite(lk2[c])) bad |= kDevNonFinite;
    if (bad) atomicOr(status, bad);
}

__global__ void k_validate_facets(const int* __restrict__ f, int64_t n, int dim, int64_t n_nodes,
                                  int* status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * dim) return;
    int a = f[i];
    if (a < 0 || a >= n_nodes) atomicOr(status, kDevBadIndex);
}

__global__ void k_validate_coords(const double* __restrict__ x, int64_t n, int* status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !isfinite(x[i])) atomicOr(status, kDevNonFinite);
}

// incidence lists: count, fill (unordered), then sort each list
__global__ void k_count_incidence(const int* __restrict__ ent, int64_t n_ent, int per,
                                  int* __restrict__ count) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_ent * per) atomicAdd(&count[ent[i]], 1);
}

__global__ void k_fill_incidence(const int* __restrict__ ent, int64_t n_ent, int per,
                                 int* __restrict__ cursor, int* __restrict__ list) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_ent * per) {
        int slot = atomicAdd(&cursor[ent[i]], 1);
        list[slot] = (int)(i / per);
    }
}

__global__ void k_sort_segments(const int* __restrict__ ptr, int* __restrict__ list, int64_t n) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    int s = ptr[a], e = ptr[a + 1];
    for (int i = s + 1; i < e; ++i) {  // insertion sort (lists are short)
        int v = list[i], j = i - 1;
        while (j >= s && list[j] > v) { list[j + 1] = list[j]; --j; }
        list[j + 1] = v;
    }
}

// Distinct neighbours (self included) of node a, sorted, in a local array
// (NVC vertices per cell).
template <int NVC>
__device__ int gather_neighbours(int a, const int* __restrict__ nc_ptr,
                                 const int* __restrict__ nc_list, const int* __restrict__ cells,
                                 int* nb, bool* overflow) {
    int len = 0;
    for (int k = nc_ptr[a]; k < nc_ptr[a + 1]; ++k) {
        int c = nc_list[k];
#pragma unroll
        for (int v = 0; v < NVC; ++v) {
            int b = cells[(int64_t)c * NVC + v];
            int pos = 0;
            while (pos < len && nb[pos] < b) ++pos;
            if (pos < len && nb[pos] == b) continue;
            if (len >= kMaxRow) { *overflow = true; continue; }
            for (int q = len; q > pos; --q) nb[q] = nb[q - 1];
            nb[pos] = b;
            ++len;
        }
    }
    return len;
}

template <int NVC>
__global__ void k_pair_count(const int* __restrict__ nc_ptr, const int* __restrict__ nc_list,
                             const int* __restrict__ cells, int64_t n_nodes, int* __restrict__ len,
                             int* status) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_nodes) return;
    int nb[kMaxRow];
    bool of = false;
    len[a] = gather_neighbours<NVC>((int)a, nc_ptr, nc_list, cells, nb, &of);
    if (of) atomicOr(status, kDevOverflow);
}

template <int NVC>
__global__ void k_pair_fill(const int* __restrict__ nc_ptr, const int* __restrict__ nc_list,
                            const int* __restrict__ cells, int64_t n_nodes,
                            const int* __restrict__ row_ptr, int* __restrict__ col,
                            int* __restrict__ pair_row) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_nodes) return;
    int nb[kMaxRow];
    bool of = false;
    int len = gather_neighbours<NVC>((int)a, nc_ptr, nc_list, cells, nb, &of);
    int s = row_ptr[a];
    for (int j = 0; j < len; ++j) {
        col[s + j] = nb[j];
        pair_row[s + j] = (int)a;
    }
}

// SELL slice widths (one warp per slice of 32 rows)
__global__ void k_slice_width(const int* __restrict__ row_ptr, int64_t n_rows, int64_t n_slices,
                              int* __restrict__ width) {
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (w >= n_slices) return;
    int64_t r = w * kSell + lane;
    int len = (r < n_rows) ? row_ptr[r + 1] - row_ptr[r] : 0;
    len = warp_max(len);
    if (lane == 0) width[w] = len;
}

__global__ void k_sell_cols(const int* __restrict__ row_ptr, const int* __restrict__ col,
                            int64_t n_rows, int64_t n_slices, const int* __restrict__ slice_ptr,
                            int* __restrict__ sell_col) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t s = r >> 5;
    if (s >= n_slices) return;
    int lane = (int)(r & 31);
    int g0 = slice_ptr[s], g1 = slice_ptr[s + 1];
    int rs = (r < n_rows) ? row_ptr[r] : 0;
    int len = (r < n_rows) ? row_ptr[r + 1] - rs : 0;
    for (int j = 0; j < g1 - g0; ++j)
        sell_col[(int64_t)(g0 + j) * kSell + lane] = (j < len) ? col[rs + j] : -1;
}

// Per-cell factors of the pair values (index: meaning):
// 0: |K|/(d+1)  1: |K|/((d+1)(d+2))  2: mu/(2 k1)  3: mu/(2 k2)  4: k1 |K|/(2 mu)
// 5: k2 |K|/(2 mu)  6: beta/mu  7: unused
template <int DIM>
__global__ void k_cell_geometry(const double* __restrict__ X, const int* __restrict__ cells,
                                int64_t n_cells, const double* __restrict__ lk1,
                                const double* __restrict__ lk2, double mu, double beta,
                                const double* __restrict__ mub, double* __restrict__ geo,
                                double* __restrict__ kk, double* __restrict__ coef, int* status) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    constexpr int S = GeoLayout<DIM>::stride;
    double x[DIM + 1][DIM];
#pragma unroll
    for (int v = 0; v <= DIM; ++v) {
        int a = cells[c * (DIM + 1) + v];
#pragma unroll
        for (int k = 0; k < DIM; ++k) x[v][k] = X[(int64_t)a * DIM + k];
    }
    double g[DIM + 1][DIM];
    double det;
    if constexpr (DIM == 2) {
        const double j00 = x[1][0] - x[0][0], j01 = x[2][0] - x[0][0];
        const double j10 = x[1][1] - x[0][1], j11 = x[2][1] - x[0][1];
        det = j00 * j11 - j01 * j10;
        const double id = 1.0 / det;
        // rows of J^-1 (J has columns x_1 - x_0, x_2 - x_0) are grad lambda_1, grad lambda_2
        g[1][0] = j11 * id;  g[1][1] = -j01 * id;
        g[2][0] = -j10 * id; g[2][1] = j00 * id;
    } else {
        double J[3][3];
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q) J[r][q] = x[q + 1][r] - x[0][r];  // column q = x_{q+1} - x_0
        // adjugate: inv[q][r] = cofactor(r, q) / det; row q of J^-1 is grad lambda_{q+1}
        double inv[3][3];
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
        const double id = 1.0 / det;
        for (int q = 0; q < 3; ++q)
            for (int r = 0; r < 3; ++r) g[q + 1][r] = inv[q][r] * id;
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        double s = 0;
#pragma unroll
        for (int v = 1; v <= DIM; ++v) s += g[v][k];
        g[0][k] = -s;
    }
    double vol = fabs(det) / (DIM == 2 ? 2.0 : 6.0);
    if (!(vol > 0.0) || !isfinite(vol)) atomicOr(status, kDevDegenerate);
    double* o = geo + c * S;
    o[0] = vol;
#pragma unroll
    for (int v = 0; v <= DIM; ++v)
#pragma unroll
        for (int k = 0; k < DIM; ++k) o[1 + v * DIM + k] = g[v][k];
    const double k1 = exp(lk1[c]), k2 = exp(lk2[c]);
    kk[2 * c] = k1;
    kk[2 * c + 1] = k2;
    const double muc = mub ? mub[2 * c] : mu, bc = mub ? mub[2 * c + 1] : beta;
    // per-cell factors of the pair values, with the P1 mass integral
    // (phi_a; phi_b)_K = vol / ((d+1)(d+2)) (times 2 for a = b, applied per
    // pair) folded in, so the pair loop adds them without multiplying
    double* cf = coef + c * kCellCoef;
    const double mass = vol / ((DIM + 1) * (DIM + 2));
    cf[0] = vol / (DIM + 1);           // (grad phi_a; phi_b)_K = g_a vol / (d+1)
    cf[1] = mass * (0.5 * muc / k1);   // 1/2 mu/k1 (phi_a; phi_b)
    cf[2] = mass * (0.5 * muc / k2);
    cf[3] = mass * (bc / muc);         // beta/mu (phi_a; phi_b)
    cf[4] = 0.5 * k1 / muc * vol;      // 1/2 k1/mu |K|, times g_a.g_b
    cf[5] = 0.5 * k2 / muc * vol;
    cf[6] = 0.0;
    cf[7] = 0.0;
}

// Fixed-order gather over the cells of the row node, one thread per node pair.
// The per-cell factors come precomputed from k_cell_geometry (no division here;
// FP64 division is costly on GB300's FP64 pipe).
//
// The FP64 pipe is the limit, and it is charged per warp instruction however
// few lanes are active. So a thread first marks which of its row node's cells
// contain the pair (integer work), then runs the FP64 terms over the marked
// cells only; the lanes of a warp take their terms side by side. Threads
// [0, n_nodes) do the self pairs, which share all of the node's cells, and
// threads [n_nodes, n_nodes + n_pairs) the other pairs (a self pair there is
// skipped), so no warp waits on a 24-cell self pair beside 4-6-cell edge pairs.
// Each pair still sums its cells in the order of the node's cell list.
template <int DIM>
__global__ void k_assemble_pairs(const int* __restrict__ pair_row, const int* __restrict__ col,
                                 const int* __restrict__ row_ptr, int64_t n_pairs, int64_t n_nodes,
                                 const int* __restrict__ nc_ptr, const int* __restrict__ nc_list,
                                 const int* __restrict__ cells, const double* __restrict__ geo,
                                 const double* __restrict__ coef,
                                 const int* __restrict__ slice_ptr, double* __restrict__ sell_val) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_nodes + n_pairs) return;
    constexpr int S = GeoLayout<DIM>::stride;
    constexpr int NV = pair_values(DIM);
    int a, b;
    int64_t p;
    if (t < n_nodes) {  // self pair of node t: its slot in the sorted row
        a = b = (int)t;
        int lo = row_ptr[a], hi = row_ptr[a + 1];
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (col[mid] < a) lo = mid + 1;
            else hi = mid;
        }
        if (lo >= row_ptr[a + 1] || col[lo] != a) return;  // a node in no cell has no pairs
        p = lo;
    } else {
        p = t - n_nodes;
        a = pair_row[p];
        b = col[p];
        if (a == b) return;
    }
    const int j = (int)(p - row_ptr[a]);
    const double self = (a == b) ? 2.0 : 1.0;
    // sums over the cells of the pair: mass factors, d terms and the
    // gradient moments sa = sum vol/(d+1) g_a, sb = sum vol/(d+1) g_b
    double m1 = 0, m2 = 0, d1 = 0, d2 = 0, bm = 0, sa[DIM], sb[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) sa[k] = sb[k] = 0;
    auto local = [&](int c, int& la, int& lb) {
        la = -1;
        lb = -1;
        if constexpr (DIM == 3) {
            const int4 v = *reinterpret_cast<const int4*>(cells + (int64_t)c * 4);
            la = (v.x == a) ? 0 : (v.y == a) ? 1 : (v.z == a) ? 2 : 3;
            lb = (v.x == b) ? 0 : (v.y == b) ? 1 : (v.z == b) ? 2 : (v.w == b) ? 3 : -1;
        } else {
#pragma unroll
            for (int v = 0; v <= DIM; ++v) {
                const int n = cells[(int64_t)c * (DIM + 1) + v];
                if (n == a) la = v;
                if (n == b) lb = v;
            }
        }
    };
    auto term = [&](int c, int la, int lb) {
        const double* g = geo + (int64_t)c * S;
        const double* ga = g + 1 + la * DIM;
        const double* gb = g + 1 + lb * DIM;
        const double* cf = coef + (int64_t)c * kCellCoef;
        double dot = 0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) dot += ga[k] * gb[k];
        m1 += cf[1];
        m2 += cf[2];
        bm += cf[3];
        d1 += cf[4] * dot;
        d2 += cf[5] * dot;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            sa[k] += cf[0] * ga[k];
            sb[k] += cf[0] * gb[k];
        }
    };
    const int q0 = nc_ptr[a], q1 = nc_ptr[a + 1];
    const int qm = min(q1, q0 + 64);
    unsigned long long mask = 0;
    if (a == b) {  // every cell of the node holds the self pair
        mask = (qm - q0 == 64) ? ~0ull : ((1ull << (qm - q0)) - 1ull);
    } else {
        for (int q = q0; q < qm; ++q) {
            int la, lb;
            local(nc_list[q], la, lb);
            if (lb >= 0) mask |= 1ull << (q - q0);
        }
    }
    while (mask) {
        const int q = q0 + __ffsll((long long)mask) - 1;
        mask &= mask - 1ull;
        const int c = nc_list[q];
        int la, lb;
        local(c, la, lb);
        term(c, la, lb);
    }
    for (int q = qm; q < q1; ++q) {  // nodes in more than 64 cells
        const int c = nc_list[q];
        int la, lb;
        local(c, la, lb);
        if (lb >= 0) term(c, la, lb);
    }
    m1 *= self;
    m2 *= self;
    bm *= self;
    double bu[DIM], cu[DIM];  // B: -(sum vol/(d+1) (g_a + g_b/2)), C: sum vol/(d+1) (g_b + g_a/2)
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        bu[k] = -(sa[k] + 0.5 * sb[k]);
        cu[k] = sb[k] + 0.5 * sa[k];
    }
    const int64_t grp = (int64_t)slice_ptr[a >> 5] + j;
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

// Area-weighted outward normal of each boundary facet; the owning cell is the
// one incident cell of the facet's first vertex that contains all its vertices.
template <int DIM>
__global__ void k_facet_normals(const int* __restrict__ bf, int64_t n_bf,
                                const int* __restrict__ nc_ptr, const int* __restrict__ nc_list,
                                const int* __restrict__ cells, const double* __restrict__ X,
                                const double* __restrict__ p01, const double* __restrict__ p02,
                                double* __restrict__ nA, int* status) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_bf) return;
    int fv[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) fv[k] = bf[f * DIM + k];
    int owner = -1, opp = -1;
    for (int q = nc_ptr[fv[0]]; q < nc_ptr[fv[0] + 1] && owner < 0; ++q) {
        int c = nc_list[q];
        int hits = 0, other = -1;
#pragma unroll
        for (int v = 0; v <= DIM; ++v) {
            int n = cells[(int64_t)c * (DIM + 1) + v];
            bool in = false;
#pragma unroll
            for (int k = 0; k < DIM; ++k) in |= (n == fv[k]);
            if (in) ++hits; else other = n;
        }
        if (hits == DIM) { owner = c; opp = other; }
    }
    bool bad = false;
#pragma unroll
    for (int k = 0; k < DIM; ++k) bad |= !isfinite(p01[fv[k]]) || !isfinite(p02[fv[k]]);
    if (bad) atomicOr(status, kDevNonFinite);
    double n[DIM];
    if (owner < 0) {
        atomicOr(status, kDevNoOwner);
#pragma unroll
        for (int k = 0; k < DIM; ++k) nA[f * DIM + k] = 0.0;
        return;
    }
    const double* x0 = X + (int64_t)fv[0] * DIM;
    const double* x1 = X + (int64_t)fv[1] * DIM;
    if constexpr (DIM == 2) {
        n[0] = x1[1] - x0[1];  // |F| times a unit normal of the edge
        n[1] = -(x1[0] - x0[0]);
    } else {
        const double* x2 = X + (int64_t)fv[2] * DIM;
        double e1[3], e2[3];
        for (int k = 0; k < 3; ++k) { e1[k] = x1[k] - x0[k]; e2[k] = x2[k] - x0[k]; }
        n[0] = 0.5 * (e1[1] * e2[2] - e1[2] * e2[1]);  // half the cross product: |F| n
        n[1] = 0.5 * (e1[2] * e2[0] - e1[0] * e2[2]);
        n[2] = 0.5 * (e1[0] * e2[1] - e1[1] * e2[0]);
    }
    const double* xo = X + (int64_t)opp * DIM;
    double s = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) s += n[k] * (xo[k] - x0[k]);
    double sg = (s > 0) ? -1.0 : 1.0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) nA[f * DIM + k] = sg * n[k];
}

// Load vector per node (Eq. "S4_cg_rhs"): body terms over incident cells, then
// -(w . n; p0h)_F over incident boundary facets with the exact facet mass
// (phi_a; phi_b)_F = |F| (1 + delta_ab) / (d (d+1)).
template <int DIM>
__global__ void k_rhs(int64_t n_nodes, const int* __restrict__ nc_ptr,
                      const int* __restrict__ nc_list, const int* __restrict__ cells,
                      const double* __restrict__ geo, const double* __restrict__ kk,
                      const int* __restrict__ nf_ptr, const int* __restrict__ nf_list,
                      const int* __restrict__ bf, const double* __restrict__ nA,
                      const double* __restrict__ p01, const double* __restrict__ p02, double mu,
                      const double* __restrict__ mub, double gb0, double gb1, double gb2,
                      double* __restrict__ f) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_nodes) return;
    constexpr int S = GeoLayout<DIM>::stride;
    constexpr int NS = 2 * DIM + 2;
    const double gbv[3] = {gb0, gb1, gb2};
    double vsum = 0, fp1 = 0, fp2 = 0;
    for (int q = nc_ptr[a]; q < nc_ptr[a + 1]; ++q) {
        int c = nc_list[q];
        int la = 0;
#pragma unroll
        for (int v = 0; v <= DIM; ++v)
            if (cells[(int64_t)c * (DIM + 1) + v] == a) la = v;
        const double* g = geo + (int64_t)c * S;
        double vol = g[0];
        double gdot = 0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) gdot += g[1 + la * DIM + k] * gbv[k];
        const double muc = mub ? mub[2 * c] : mu;
        vsum += vol / (DIM + 1);
        fp1 += 0.5 * vol * kk[2 * c] / muc * gdot;
        fp2 += 0.5 * vol * kk[2 * c + 1] / muc * gdot;
    }
    double fu1[DIM], fu2[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) fu1[k] = fu2[k] = 0.5 * gbv[k] * vsum;
    const double fm = 1.0 / (DIM * (DIM + 1));
    for (int q = nf_ptr[a]; q < nf_ptr[a + 1]; ++q) {
        int F = nf_list[q];
        double s1 = 0, s2 = 0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            int b = bf[(int64_t)F * DIM + k];
            double w = fm * (b == a ? 2.0 : 1.0);
            s1 += w * p01[b];
            s2 += w * p02[b];
        }
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            double n = nA[(int64_t)F * DIM + k];
            fu1[k] -= n * s1;
            fu2[k] -= n * s2;
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

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

void check_status(ProblemImpl& P, cudaStream_t s, const char* where) {
    int st = read_scalar(P.dstatus.get(), s, P.hs);
    if (st == kDevOk) return;
    std::string m = std::string(where) + ":";
    if (st & kDevBadIndex) m += " node index out of range;";
    if (st & kDevNonFinite) m += " non-finite input value;";
    if (st & kDevDegenerate) m += " zero-volume cell;";
    if (st & kDevOverflow) m += " a node has more than 95 distinct neighbours;";
    if (st & kDevNoOwner) m += " a boundary facet is not a face of any cell;";
    fail((st & kDevNonFinite) && !(st & ~kDevNonFinite) ? DPP_ERR_NONFINITE
                                                        : DPP_ERR_INVALID_ARGUMENT, m);
}

template <class T>
void upload(DBuf<T>& dst, const T* src, size_t n, bool host, cudaStream_t s) {
    dst.alloc(n);
    if (n) DPP_CK(cudaMemcpyAsync(dst.get(), src, n * sizeof(T),
                                  host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
}

void build_incidence(const int* ent, int64_t n_ent, int per, int64_t n_nodes, DBuf<int>& ptr,
                     DBuf<int>& list, cudaStream_t s, HostScratch& hs) {
    ptr.alloc(n_nodes + 1);
    DPP_CK(cudaMemsetAsync(ptr.get(), 0, (n_nodes + 1) * sizeof(int), s));
    const int B = 256;
    if (n_ent) {
        k_count_incidence<<<grid_for(n_ent * per, B), B, 0, s>>>(ent, n_ent, per, ptr.get());
        DPP_LAUNCH_CK();
    }
    int64_t total = exclusive_scan(ptr.get(), ptr.get(), n_nodes + 1, s, hs);
    (void)total;
    list.alloc(std::max<int64_t>(n_ent * per, 1));
    DBuf<int> cursor(n_nodes + 1);
    DPP_CK(cudaMemcpyAsync(cursor.get(), ptr.get(), (n_nodes + 1) * sizeof(int),
                           cudaMemcpyDeviceToDevice, s));
    if (n_ent) {
        k_fill_incidence<<<grid_for(n_ent * per, B), B, 0, s>>>(ent, n_ent, per, cursor.get(),
                                                               list.get());
        DPP_LAUNCH_CK();
    }
    k_sort_segments<<<grid_for(n_nodes, B), B, 0, s>>>(ptr.get(), list.get(), n_nodes);
    DPP_LAUNCH_CK();
    DPP_CK(cudaStreamSynchronize(s));
}

// Steps 5-7 for Q1 cells: the cell tables, the pair values and the load.
template <int DIM>
void assemble_q1_values(ProblemImpl& P, cudaStream_t s) {
    using Lay = q1::Layout<DIM>;
    const int B = 128;
    P.q1tab.alloc(P.n_cells * Lay::stride);
    P.kk.alloc(P.n_cells * 2);
    q1::k_cell_tables<DIM><<<grid_for(P.n_cells * Lay::NVC, B), B, 0, s>>>(
        P.coords.get(), P.cells.get(), P.n_cells, P.logk1.get(), P.logk2.get(), P.q1tab.get(),
        P.kk.get(), P.dstatus.get());
    DPP_LAUNCH_CK();
    check_status(P, s, "dpp_assemble cell geometry");
    P.sell_val.alloc(P.n_groups * P.nv * kSell);
    DPP_CK(cudaMemsetAsync(P.sell_val.get(), 0, P.sell_val.bytes(), s));
    q1::k_assemble_pairs<DIM><<<grid_for(P.n_pairs, B), B, 0, s>>>(
        P.pair_row.get(), P.col.get(), P.row_ptr.get(), P.n_pairs, P.nc_ptr.get(), P.nc_list.get(),
        P.cells.get(), P.q1tab.get(), P.kk.get(), P.mu, P.beta, P.cell_mu_beta.get(),
        P.slice_ptr.get(), P.sell_val.get());
    DPP_LAUNCH_CK();
    if (P.precision == DPP_MIXED_FP32_FP64) {
        P.sell_val32.alloc(P.sell_val.n);
        k_to_float<<<grid_for(P.sell_val.n, 256), 256, 0, s>>>(P.sell_val.get(), P.sell_val32.get(),
                                                              P.sell_val.n);
        DPP_LAUNCH_CK();
    }
    P.facet_tab.alloc(std::max<int64_t>(P.n_bfacets * Lay::fstride, 1));
    if (P.n_bfacets) {
        q1::k_facet_tables<DIM><<<grid_for(P.n_bfacets, B), B, 0, s>>>(
            P.bfacets.get(), P.n_bfacets, P.nc_ptr.get(), P.nc_list.get(), P.cells.get(),
            P.coords.get(), P.p01.get(), P.p02.get(), P.facet_tab.get(), P.dstatus.get());
        DPP_LAUNCH_CK();
    }
    P.f.alloc(P.n_nodes * P.ns);
    q1::k_rhs<DIM><<<grid_for(P.n_nodes, B), B, 0, s>>>(
        P.n_nodes, P.nc_ptr.get(), P.nc_list.get(), P.cells.get(), P.q1tab.get(), P.kk.get(),
        P.nf_ptr.get(), P.nf_list.get(), P.bfacets.get(), P.facet_tab.get(), P.p01.get(),
        P.p02.get(), P.mu, P.cell_mu_beta.get(), P.gb[0], P.gb[1], P.gb[2], P.f.get());
    DPP_LAUNCH_CK();
    check_status(P, s, "dpp_assemble");
}

// NVC: vertices per cell (DIM + 1 for simplices, 2^DIM for Q1 cells).
template <int DIM, int NVC>
void assemble_dim(ProblemImpl& P, cudaStream_t s) {
    constexpr bool kQ1 = NVC != DIM + 1;
    constexpr int NFV = kQ1 ? (1 << (DIM - 1)) : DIM;  // vertices per boundary facet
    const int B = 256;
    auto& hs = P.hs;
    // 1. validation of every index and value before any indexed access
    k_validate_cells<NVC><<<grid_for(P.n_cells, B), B, 0, s>>>(
        P.cells.get(), P.n_cells, P.n_nodes, P.logk1.get(), P.logk2.get(), P.dstatus.get());
    DPP_LAUNCH_CK();
    if (P.n_bfacets) {
        k_validate_facets<<<grid_for(P.n_bfacets * NFV, B), B, 0, s>>>(
            P.bfacets.get(), P.n_bfacets, NFV, P.n_nodes, P.dstatus.get());
        DPP_LAUNCH_CK();
    }
    k_validate_coords<<<grid_for(P.n_nodes * DIM, B), B, 0, s>>>(P.coords.get(), P.n_nodes * DIM,
                                                                 P.dstatus.get());
    DPP_LAUNCH_CK();
    check_status(P, s, "dpp_assemble input check");

    // 2. incidence lists node -> cells and node -> boundary facets
    build_incidence(P.cells.get(), P.n_cells, NVC, P.n_nodes, P.nc_ptr, P.nc_list, s, hs);
    build_incidence(P.bfacets.get(), P.n_bfacets, NFV, P.n_nodes, P.nf_ptr, P.nf_list, s, hs);

    // 3. node-pair graph (CSR with sorted columns)
    P.row_ptr.alloc(P.n_nodes + 1);
    DPP_CK(cudaMemsetAsync(P.row_ptr.get(), 0, (P.n_nodes + 1) * sizeof(int), s));
    k_pair_count<NVC><<<grid_for(P.n_nodes, 128), 128, 0, s>>>(
        P.nc_ptr.get(), P.nc_list.get(), P.cells.get(), P.n_nodes, P.row_ptr.get(), P.dstatus.get());
    DPP_LAUNCH_CK();
    check_status(P, s, "dpp_assemble pair graph");
    P.n_pairs = exclusive_scan(P.row_ptr.get(), P.row_ptr.get(), P.n_nodes + 1, s, hs);
    P.col.alloc(P.n_pairs);
    P.pair_row.alloc(P.n_pairs);
    k_pair_fill<NVC><<<grid_for(P.n_nodes, 128), 128, 0, s>>>(
        P.nc_ptr.get(), P.nc_list.get(), P.cells.get(), P.n_nodes, P.row_ptr.get(), P.col.get(),
        P.pair_row.get());
    DPP_LAUNCH_CK();

    // 4. SELL-32 layout
    P.n_slices = (P.n_nodes + kSell - 1) / kSell;
    P.slice_ptr.alloc(P.n_slices + 1);
    DPP_CK(cudaMemsetAsync(P.slice_ptr.get(), 0, (P.n_slices + 1) * sizeof(int), s));
    k_slice_width<<<grid_for(P.n_slices * 32, B), B, 0, s>>>(P.row_ptr.get(), P.n_nodes,
                                                             P.n_slices, P.slice_ptr.get());
    DPP_LAUNCH_CK();
    P.n_groups = exclusive_scan(P.slice_ptr.get(), P.slice_ptr.get(), P.n_slices + 1, s, hs);
    P.sell_col.alloc(P.n_groups * kSell);
    k_sell_cols<<<grid_for(P.n_slices * 32, B), B, 0, s>>>(P.row_ptr.get(), P.col.get(), P.n_nodes,
                                                           P.n_slices, P.slice_ptr.get(),
                                                           P.sell_col.get());
    DPP_LAUNCH_CK();

    if constexpr (kQ1) {
        assemble_q1_values<DIM>(P, s);
        return;
    }

    // 5. cell geometry and permeabilities
    P.geo.alloc(P.n_cells * GeoLayout<DIM>::stride);
    P.kk.alloc(P.n_cells * 2);
    P.ccoef.alloc(P.n_cells * kCellCoef);
    k_cell_geometry<DIM><<<grid_for(P.n_cells, B), B, 0, s>>>(
        P.coords.get(), P.cells.get(), P.n_cells, P.logk1.get(), P.logk2.get(), P.mu, P.beta,
        P.cell_mu_beta.get(), P.geo.get(), P.kk.get(), P.ccoef.get(), P.dstatus.get());
    DPP_LAUNCH_CK();

    // 6. pair values
    P.sell_val.alloc(P.n_groups * P.nv * kSell);
    DPP_CK(cudaMemsetAsync(P.sell_val.get(), 0, P.sell_val.bytes(), s));
    k_assemble_pairs<DIM><<<grid_for(P.n_pairs + P.n_nodes, B), B, 0, s>>>(
        P.pair_row.get(), P.col.get(), P.row_ptr.get(), P.n_pairs, P.n_nodes, P.nc_ptr.get(),
        P.nc_list.get(), P.cells.get(), P.geo.get(), P.ccoef.get(), P.slice_ptr.get(),
        P.sell_val.get());
    DPP_LAUNCH_CK();
    if (P.precision == DPP_MIXED_FP32_FP64) {
        P.sell_val32.alloc(P.sell_val.n);
        k_to_float<<<grid_for(P.sell_val.n, B), B, 0, s>>>(P.sell_val.get(), P.sell_val32.get(),
                                                          P.sell_val.n);
        DPP_LAUNCH_CK();
    }

    // 7. load vector
    P.facet_nA.alloc(std::max<int64_t>(P.n_bfacets * DIM, 1));
    if (P.n_bfacets) {
        k_facet_normals<DIM><<<grid_for(P.n_bfacets, B), B, 0, s>>>(
            P.bfacets.get(), P.n_bfacets, P.nc_ptr.get(), P.nc_list.get(), P.cells.get(),
            P.coords.get(), P.p01.get(), P.p02.get(), P.facet_nA.get(), P.dstatus.get());
        DPP_LAUNCH_CK();
    }
    P.f.alloc(P.n_nodes * P.ns);
    k_rhs<DIM><<<grid_for(P.n_nodes, B), B, 0, s>>>(
        P.n_nodes, P.nc_ptr.get(), P.nc_list.get(), P.cells.get(), P.geo.get(), P.kk.get(),
        P.nf_ptr.get(), P.nf_list.get(), P.bfacets.get(), P.facet_nA.get(), P.p01.get(),
        P.p02.get(), P.mu, P.cell_mu_beta.get(), P.gb[0], P.gb[1], P.gb[2], P.f.get());
    DPP_LAUNCH_CK();
    check_status(P, s, "dpp_assemble");
}

}  // namespace

void assemble_uploaded(ProblemImpl& P, cudaStream_t s);

void assemble_problem(ProblemImpl& P, const dpp_problem_desc& d, cudaStream_t s) {
    const bool host = d.memory == DPP_MEM_HOST;
    P.dim = d.dim;
    P.n_nodes = d.n_nodes;
    P.n_cells = d.n_cells;
    P.n_bfacets = d.n_bfacets;
    P.mu = d.mu;
    P.beta = d.beta;
    for (int k = 0; k < 3; ++k) P.gb[k] = (k < d.dim) ? d.gamma_b[k] : 0.0;
    upload(P.coords, d.coords, (size_t)d.n_nodes * d.dim, host, s);
    P.kind = d.cell_kind;
    P.nvc = (P.kind == DPP_CELL_Q1) ? (1 << d.dim) : d.dim + 1;
    P.nfv = (P.kind == DPP_CELL_Q1) ? (1 << (d.dim - 1)) : d.dim;
    upload(P.cells, d.cells, (size_t)d.n_cells * P.nvc, host, s);
    upload(P.bfacets, d.bfacets, (size_t)d.n_bfacets * P.nfv, host, s);
    upload(P.logk1, d.log_k1, (size_t)d.n_cells, host, s);
    upload(P.logk2, d.log_k2, (size_t)d.n_cells, host, s);
    upload(P.p01, d.p01, (size_t)d.n_nodes, host, s);
    upload(P.p02, d.p02, (size_t)d.n_nodes, host, s);
    assemble_uploaded(P, s);
}

// Assembly from arrays already in P (coords, cells, bfacets, log k, p0, sizes,
// dim, mu, beta, gamma b, and the optional per-cell mu/beta of batches).
void assemble_uploaded(ProblemImpl& P, cudaStream_t s) {
    P.ns = 2 * P.dim + 2;
    P.nv = pair_values(P.dim);
    P.dstatus.alloc(1);
    DPP_CK(cudaMemsetAsync(P.dstatus.get(), 0, sizeof(int), s));
    if (P.kind == DPP_CELL_Q1) {
        if (P.dim == 2) assemble_dim<2, 4>(P, s);
        else assemble_dim<3, 8>(P, s);
    } else {
        if (P.dim == 2) assemble_dim<2, 3>(P, s);
        else assemble_dim<3, 4>(P, s);
    }
}

}  // namespace dpp

namespace dpp {

namespace {
__global__ void k_export_pairs(int64_t n_pairs, int nv, const int* __restrict__ pair_row,
                               const int* __restrict__ row_ptr, const int* __restrict__ slice_ptr,
                               const double* __restrict__ sell_val, double* __restrict__ out) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    const int a = pair_row[p];
    const int64_t grp = (int64_t)slice_ptr[a >> 5] + (p - row_ptr[a]);
    for (int k = 0; k < nv; ++k) out[p * nv + k] = sell_val[(grp * nv + k) * kSell + (a & 31)];
}
}  // namespace

// CSR-ordered copy of the pair graph and its values (inspection entry point).
void export_pairs(const ProblemImpl& P, int* rp, int* col, double* vals, cudaStream_t s) {
    DPP_CK(cudaMemcpyAsync(rp, P.row_ptr.get(), (P.n_nodes + 1) * sizeof(int),
                           cudaMemcpyDeviceToDevice, s));
    DPP_CK(cudaMemcpyAsync(col, P.col.get(), P.n_pairs * sizeof(int), cudaMemcpyDeviceToDevice, s));
    k_export_pairs<<<grid_for(P.n_pairs, 256), 256, 0, s>>>(P.n_pairs, P.nv, P.pair_row.get(),
                                                           P.row_ptr.get(), P.slice_ptr.get(),
                                                           P.sell_val.get(), vals);
    DPP_LAUNCH_CK();
}

}  // namespace dpp
