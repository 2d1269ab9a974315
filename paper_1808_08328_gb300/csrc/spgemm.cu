// Sparse matrix products for the preconditioner setup:
//   * the selfp Schur matrices S_pi = Ki_pp - Ki_pu diag(Ki_uu)^-1 Ki_up
//     (Eqs. "S4_sp1", "S4_sp2", Section 4.2), formed straight from the node-pair
//     values and stored as the block-diagonal matrix blockdiag(S_p1, S_p2);
//   * the general CSR product C = A B. The AMG setup uses it for A P and for
//     the Galerkin product P^T (A P);
//   * the CSR transpose.
//
// Product scheme (deterministic; no floating-point atomics). One warp owns one
// output row, and its lanes form G groups of 32/G lanes. Group g takes the
// entries p = g, g+G, ... of A's row i; its lanes take the entries of B's row
// acol[p]. The group count follows B's mean row length, so short rows of B
// (aggregation prolongators) still keep every lane busy.
//   1. symbolic: the candidate columns go into an open-addressing hash set in
//      shared memory, and the distinct keys are counted. Tables grow in tiers
//      (256, 2048, 8192 slots); a row that overflows one tier is retried in
//      the next;
//   2. numeric: the warp rebuilds the set, compacts it, and ranks the keys
//      (they are distinct, so a key's rank is the number of smaller keys) to
//      get the row's sorted columns. Each group then scatters a_ip * B_p into
//      its own accumulator, at positions found by binary search in the sorted
//      columns. Within one round the positions of a group are distinct
//      (B's row has distinct columns); between rounds the warp synchronises.
//      At the end the group accumulators are added in group order. The
//      summation order is therefore fixed, and the result is deterministic. Rows
//      wider than the largest shared accumulator (1024 columns) use one
//      warp with the accumulator in C's own storage.
#include <climits>

#include "amg.cuh"

namespace dpp {

namespace {
__device__ __forceinline__ unsigned hash_key(int k) { return (unsigned)k * 2654435761u; }

template <int HT>
__device__ __forceinline__ bool hs_insert(int* keys, int key) {
    unsigned h = hash_key(key) & (HT - 1);
    for (int probe = 0; probe < HT; ++probe) {
        int prev = atomicCAS(&keys[h], -1, key);
        if (prev == -1 || prev == key) return true;
        h = (h + 1) & (HT - 1);
    }
    return false;
}

// Fill the warp's hash set with the candidate columns of row i of A*B.
template <int HT, int G>
__device__ bool warp_collect(int i, const int* __restrict__ arp, const int* __restrict__ acol,
                             const int* __restrict__ brp, const int* __restrict__ bcol, int* keys,
                             int lane) {
    constexpr int GL = 32 / G;
    for (int t = lane; t < HT; t += 32) keys[t] = -1;
    __syncwarp();
    const int g = lane / GL, gl = lane % GL;
    bool ok = true;
    for (int p = arp[i] + g; p < arp[i + 1]; p += G) {
        const int k = acol[p];
        for (int q = brp[k] + gl; q < brp[k + 1]; q += GL) ok &= hs_insert<HT>(keys, bcol[q]);
    }
    __syncwarp();
    return __all_sync(0xffffffffu, ok);
}

// Compact the set into list[0..u) and write the keys in ascending order to out.
template <int HT>
__device__ int warp_sorted_keys(const int* keys, int* list, int lane, int* out) {
    int base = 0;
    for (int t0 = 0; t0 < HT; t0 += 32) {
        int k = keys[t0 + lane];
        unsigned m = __ballot_sync(0xffffffffu, k >= 0);
        if (k >= 0) list[base + __popc(m & ((1u << lane) - 1u))] = k;
        base += __popc(m);
    }
    __syncwarp();
    for (int e = lane; e < base; e += 32) {
        int k = list[e], r = 0;
        for (int f = 0; f < base; ++f) r += (list[f] < k);
        out[r] = k;
    }
    __syncwarp();
    return base;
}

__device__ __forceinline__ int bsearch_row(const int* __restrict__ col, int lo, int hi, int key) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int v = col[mid];
        if (v < key) lo = mid + 1;
        else if (v > key) hi = mid;
        else return mid;
    }
    return -1;
}

// Symbolic pass: count[i] = distinct columns of row i (rows[] lists the rows to
// do, with rows[-1] their number; rows == nullptr means every row). Rows that
// overflow the table are appended to ovf (ovf[0] = count).
template <int HT, int G>
__global__ void k_spgemm_count(int64_t n_rows, const int* __restrict__ arp,
                               const int* __restrict__ acol, const int* __restrict__ brp,
                               const int* __restrict__ bcol, int* __restrict__ count,
                               int* __restrict__ ovf, const int* __restrict__ rows,
                               const int* __restrict__ is_long) {
    extern __shared__ int smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    const int64_t n_work = rows ? rows[-1] : n_rows;
    if (w >= n_work) return;
    const int i = rows ? rows[w] : (int)w;
    if (is_long && is_long[i]) return;  // done by the block-per-row kernels
    int* keys = smem + warp * HT;
    const bool ok = warp_collect<HT, G>(i, arp, acol, brp, bcol, keys, lane);
    int c = 0;
    for (int t = lane; t < HT; t += 32) c += (keys[t] >= 0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) {
        count[i] = ok ? c : 0;
        if (!ok) ovf[atomicAdd(&ovf[0], 1) + 1] = i;
    }
}

// Symbolic fill for pattern-only products: sorted columns of each row.
template <int HT, int G>
__global__ void k_spgemm_pattern(int64_t n_rows, const int* __restrict__ arp,
                                 const int* __restrict__ acol, const int* __restrict__ brp,
                                 const int* __restrict__ bcol, const int* __restrict__ crp,
                                 int* __restrict__ ccol, const int* __restrict__ rows) {
    extern __shared__ int smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    const int64_t n_work = rows ? rows[-1] : n_rows;
    if (w >= n_work) return;
    const int i = rows ? rows[w] : (int)w;
    int* keys = smem + warp * 2 * HT;
    if (!warp_collect<HT, G>(i, arp, acol, brp, bcol, keys, lane)) return;
    warp_sorted_keys<HT>(keys, keys + HT, lane, ccol + crp[i]);
}

// Numeric pass for rows with at most CAP distinct columns (shared accumulators).
template <int HT, int G, int CAP>
__global__ void k_spgemm_scatter(int64_t n_rows, const int* __restrict__ arp,
                                 const int* __restrict__ acol, const double* __restrict__ aval,
                                 const int* __restrict__ brp, const int* __restrict__ bcol,
                                 const double* __restrict__ bval, const int* __restrict__ crp,
                                 int* __restrict__ ccol, double* __restrict__ cval,
                                 int* __restrict__ wide, const int* __restrict__ is_long) {
    extern __shared__ int smem[];
    constexpr int WPB = 4;
    constexpr int GL = 32 / G;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * WPB + warp;
    if (w >= n_rows) return;
    const int i = (int)w;
    if (is_long && is_long[i]) return;  // done by the block-per-row kernels
    const int c0 = crp[i];
    if (crp[i + 1] - c0 > CAP) {  // too wide for the shared accumulators
        if (lane == 0) wide[atomicAdd(&wide[0], 1) + 1] = i;
        return;
    }
    int* keys = smem + warp * 2 * HT;
    int* sorted = keys + HT;  // HT >= 2 CAP slots: the compacted list, then the sorted keys
    double* acc = reinterpret_cast<double*>(smem + WPB * 2 * HT) + (size_t)warp * G * CAP;
    warp_collect<HT, G>(i, arp, acol, brp, bcol, keys, lane);  // cannot overflow (HT >= 2 CAP)
    // compact into sorted[CAP..2CAP), rank-sort into sorted[0..u)
    int* list = sorted + CAP;
    int u = 0;
    for (int t0 = 0; t0 < HT; t0 += 32) {
        int k = keys[t0 + lane];
        unsigned m = __ballot_sync(0xffffffffu, k >= 0);
        if (k >= 0) list[u + __popc(m & ((1u << lane) - 1u))] = k;
        u += __popc(m);
    }
    __syncwarp();
    for (int e = lane; e < u; e += 32) {
        int k = list[e], r = 0;
        for (int f = 0; f < u; ++f) r += (list[f] < k);
        sorted[r] = k;
    }
    for (int e = lane; e < G * CAP; e += 32) acc[e] = 0.0;
    __syncwarp();
    for (int e = lane; e < u; e += 32) ccol[c0 + e] = sorted[e];
    const int g = lane / GL, gl = lane % GL;
    double* my = acc + g * CAP;
    const int a0 = arp[i], a1 = arp[i + 1];
    for (int pb = a0; pb < a1; pb += G) {
        const int p = pb + g;
        if (p < a1) {
            const int k = acol[p];
            const double a = aval[p];
            for (int q = brp[k] + gl; q < brp[k + 1]; q += GL)
                my[bsearch_row(sorted, 0, u, bcol[q])] += a * bval[q];
        }
        __syncwarp();
    }
    for (int e = lane; e < u; e += 32) {
        double v = acc[e];
#pragma unroll
        for (int h = 1; h < G; ++h) v += acc[h * CAP + e];
        cval[c0 + e] = v;
    }
}

// Numeric pass for wide rows: one warp per listed row, accumulating in C.
template <int HT>
__global__ void k_spgemm_wide(const int* __restrict__ arp, const int* __restrict__ acol,
                              const double* __restrict__ aval, const int* __restrict__ brp,
                              const int* __restrict__ bcol, const double* __restrict__ bval,
                              const int* __restrict__ crp, int* __restrict__ ccol,
                              double* __restrict__ cval, const int* __restrict__ rows,
                              int* __restrict__ status) {
    extern __shared__ int smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (w >= rows[-1]) return;
    const int i = rows[w];
    int* keys = smem + warp * 2 * HT;
    if (!warp_collect<HT, 1>(i, arp, acol, brp, bcol, keys, lane)) {
        if (lane == 0) atomicOr(status, 1);
        return;
    }
    const int c0 = crp[i];
    const int u = warp_sorted_keys<HT>(keys, keys + HT, lane, ccol + c0);
    for (int e = lane; e < u; e += 32) cval[c0 + e] = 0.0;
    __syncwarp();
    for (int p = arp[i]; p < arp[i + 1]; ++p) {
        const int k = acol[p];
        const double a = aval[p];
        for (int q = brp[k] + lane; q < brp[k + 1]; q += 32)
            cval[bsearch_row(ccol, c0, c0 + u, bcol[q])] += a * bval[q];
        __syncwarp();
    }
}

// Long rows (many products, typically Galerkin products on coarse levels, where
// rows are few): one block of kLongWarps warps per listed row. Warp w takes the
// entries p = w, w + kLongWarps, ... of A's row, and its lanes take B's row.
// The count pass shares one hash table per block. The numeric pass gives each
// warp its own accumulator and adds them in warp order, so the result stays
// deterministic. Rows wider than kLongCap columns are left to k_spgemm_wide.
constexpr int kLongWarps = 8;
constexpr int kLongHT = 8192;
constexpr int kLongCap = 1024;

__global__ void __launch_bounds__(kLongWarps * 32)
k_long_count(const int* __restrict__ arp, const int* __restrict__ acol,
             const int* __restrict__ brp, const int* __restrict__ bcol, int* __restrict__ count,
             const int* __restrict__ rows, int* __restrict__ status) {
    extern __shared__ int keys[];
    __shared__ int part[kLongWarps];
    const int i = rows[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = threadIdx.x; t < kLongHT; t += blockDim.x) keys[t] = -1;
    __syncthreads();
    bool ok = true;
    for (int p = arp[i] + warp; p < arp[i + 1]; p += kLongWarps) {
        const int k = acol[p];
        for (int q = brp[k] + lane; q < brp[k + 1]; q += 32) ok &= hs_insert<kLongHT>(keys, bcol[q]);
    }
    __syncthreads();
    int c = 0;
    for (int t = threadIdx.x; t < kLongHT; t += blockDim.x) c += (keys[t] >= 0);
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) part[warp] = c;
    if (!ok) atomicOr(status, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kLongWarps; ++w) t += part[w];
        count[i] = t;
    }
}

__global__ void __launch_bounds__(kLongWarps * 32)
k_long_numeric(const int* __restrict__ arp, const int* __restrict__ acol,
               const double* __restrict__ aval, const int* __restrict__ brp,
               const int* __restrict__ bcol, const double* __restrict__ bval,
               const int* __restrict__ crp, int* __restrict__ ccol, double* __restrict__ cval,
               const int* __restrict__ rows, int* __restrict__ wide) {
    extern __shared__ int smem[];
    int* keys = smem;                                  // kLongHT
    int* list = keys + kLongHT;                        // kLongCap
    int* sorted = list + kLongCap;                     // kLongCap
    double* acc = reinterpret_cast<double*>(sorted + kLongCap);  // kLongWarps * kLongCap
    __shared__ int nu;
    const int i = rows[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = crp[i], u = crp[i + 1] - c0;
    if (u > kLongCap) {
        if (threadIdx.x == 0) wide[atomicAdd(&wide[0], 1) + 1] = i;
        return;
    }
    for (int t = threadIdx.x; t < kLongHT; t += blockDim.x) keys[t] = -1;
    for (int t = threadIdx.x; t < kLongWarps * kLongCap; t += blockDim.x) acc[t] = 0.0;
    if (threadIdx.x == 0) nu = 0;
    __syncthreads();
    for (int p = arp[i] + warp; p < arp[i + 1]; p += kLongWarps) {
        const int k = acol[p];
        for (int q = brp[k] + lane; q < brp[k + 1]; q += 32) hs_insert<kLongHT>(keys, bcol[q]);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kLongHT; t += blockDim.x)  // compact (order irrelevant)
        if (keys[t] >= 0) list[atomicAdd(&nu, 1)] = keys[t];
    __syncthreads();
    for (int e = threadIdx.x; e < u; e += blockDim.x) {
        int k = list[e], r = 0;
        for (int f = 0; f < u; ++f) r += (list[f] < k);
        sorted[r] = k;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < u; e += blockDim.x) ccol[c0 + e] = sorted[e];
    double* my = acc + warp * kLongCap;
    for (int p = arp[i] + warp; p < arp[i + 1]; p += kLongWarps) {
        const int k = acol[p];
        const double a = aval[p];
        for (int q = brp[k] + lane; q < brp[k + 1]; q += 32)
            my[bsearch_row(sorted, 0, u, bcol[q])] += a * bval[q];
        __syncwarp();
    }
    __syncthreads();
    for (int e = threadIdx.x; e < u; e += blockDim.x) {
        double v = acc[e];
#pragma unroll
        for (int w = 1; w < kLongWarps; ++w) v += acc[w * kLongCap + e];
        cval[c0 + e] = v;
    }
}

// products per row: sum of B's row lengths over A's row; long rows are listed
__global__ void k_split_long(int64_t n, const int* __restrict__ arp, const int* __restrict__ acol,
                             const int* __restrict__ brp, int threshold, int* __restrict__ is_long,
                             int* __restrict__ long_rows) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    int t = 0;
    for (int p = arp[i] + lane; p < arp[i + 1]; p += 32) t += brp[acol[p] + 1] - brp[acol[p]];
    t = __reduce_add_sync(0xffffffffu, t);
    if (lane == 0) {
        is_long[i] = (t > threshold) ? 1 : 0;
        if (t > threshold) long_rows[atomicAdd(&long_rows[0], 1) + 1] = (int)i;
    }
}

__global__ void k_row_len_max(int64_t n, const int* __restrict__ rp, const int* __restrict__ skip,
                              int* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int v = (i < n && !(skip && skip[i])) ? rp[i + 1] - rp[i] : 0;
    v = warp_max(v);
    if ((threadIdx.x & 31) == 0) atomicMax(out, v);
}

// S_p rows for both networks. The pattern is the pair graph squared; it is
// produced by the product kernels above with A = B = pair graph.
template <int DIM>
__global__ void k_selfp_values(int64_t n_nodes, const int* __restrict__ prp,
                               const int* __restrict__ pcol, const int* __restrict__ slice_ptr,
                               const double* __restrict__ pv, const double* __restrict__ mdiag,
                               const int* __restrict__ srp, const int* __restrict__ scol,
                               double* __restrict__ sval, int64_t nnz_half) {
    constexpr int NV = pair_values(DIM);
    const int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (a >= n_nodes) return;
    auto pval = [&](int row, int p, int k) -> double {
        int64_t grp = (int64_t)slice_ptr[row >> 5] + (p - prp[row]);
        return pv[(grp * NV + k) * kSell + (row & 31)];
    };
    for (int e = srp[a] + lane; e < srp[a + 1]; e += 32) {
        const int c = scol[e];
        double s1 = 0.0, s2 = 0.0;
        const int pac = bsearch_row(pcol, prp[a], prp[a + 1], c);
        if (pac >= 0) {
            s1 = pval((int)a, pac, 2 + 2 * DIM);
            s2 = pval((int)a, pac, 3 + 2 * DIM);
        }
        for (int pab = prp[a]; pab < prp[a + 1]; ++pab) {
            const int b = pcol[pab];
            const int pbc = bsearch_row(pcol, prp[b], prp[b + 1], c);
            if (pbc < 0) continue;
            double dot = 0.0;
#pragma unroll
            for (int k = 0; k < DIM; ++k) dot += pval((int)a, pab, 2 + DIM + k) * pval(b, pbc, 2 + k);
            s1 -= dot * mdiag[2 * b];
            s2 -= dot * mdiag[2 * b + 1];
        }
        sval[e] = s1;
        sval[nnz_half + e] = s2;
    }
}

// block-diagonal duplication of the pattern: rows n..2n-1 get columns + n
__global__ void k_dup_pattern(int64_t n, int64_t nnz, int* __restrict__ rp, int* __restrict__ col) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nnz) col[nnz + i] = col[i] + (int)n;
    if (i <= n) rp[n + i] = rp[i] + (int)nnz;
}

// transpose: count, scatter, per-row sort
__global__ void k_col_count(const int* __restrict__ col, int64_t nnz, int* __restrict__ cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nnz) atomicAdd(&cnt[col[i]], 1);
}

__global__ void k_transpose_scatter(int64_t n_rows, const int* __restrict__ rp,
                                    const int* __restrict__ col, const double* __restrict__ val,
                                    int* __restrict__ cursor, int* __restrict__ tcol,
                                    double* __restrict__ tval) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rows) return;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
        int q = atomicAdd(&cursor[col[p]], 1);
        tcol[q] = (int)i;
        tval[q] = val[p];
    }
}

// warp per row: rank sort of (col, val) by col (distinct cols)
__global__ void k_sort_rows(int64_t n_rows, const int* __restrict__ rp, int* __restrict__ col,
                            double* __restrict__ val, int* __restrict__ tmpc,
                            double* __restrict__ tmpv) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n_rows) return;
    const int s = rp[i], e = rp[i + 1];
    for (int p = s + lane; p < e; p += 32) { tmpc[p] = col[p]; tmpv[p] = val[p]; }
    __syncwarp();
    for (int p = s + lane; p < e; p += 32) {
        int k = tmpc[p], r = 0;
        for (int q = s; q < e; ++q) r += (tmpc[q] < k);
        col[s + r] = k;
        val[s + r] = tmpv[p];
    }
}

constexpr int kWarps = 4;  // warps per block of the tiered kernels

template <class K>
void set_smem(K kernel, size_t smem) {
    if (smem > 48 * 1024)
        DPP_CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
}

int groups_for(double avg_b) {  // lane groups per warp ~ 32 / (mean row length of B)
    if (avg_b <= 1.5) return 32;
    if (avg_b <= 3.0) return 16;
    if (avg_b <= 6.0) return 8;
    if (avg_b <= 12.0) return 4;
    if (avg_b <= 24.0) return 2;
    return 1;
}

template <int HT, int G>
void count_tier(const CsrView& A, const CsrView& B, int* count, int* ovf, const int* rows,
                int64_t n_work, int wpb, const int* is_long, cudaStream_t s) {
    const size_t smem = (size_t)wpb * HT * sizeof(int);
    set_smem(k_spgemm_count<HT, G>, smem);
    k_spgemm_count<HT, G><<<grid_for(n_work, wpb), wpb * 32, smem, s>>>(
        A.n_rows, A.rp, A.col, B.rp, B.col, count, ovf, rows, is_long);
    DPP_LAUNCH_CK();
}

template <int HT>
void count_g(int G, const CsrView& A, const CsrView& B, int* count, int* ovf, const int* rows,
             int64_t n_work, int wpb, const int* is_long, cudaStream_t s) {
    switch (G) {
        case 32: count_tier<HT, 32>(A, B, count, ovf, rows, n_work, wpb, is_long, s); break;
        case 16: count_tier<HT, 16>(A, B, count, ovf, rows, n_work, wpb, is_long, s); break;
        case 8: count_tier<HT, 8>(A, B, count, ovf, rows, n_work, wpb, is_long, s); break;
        case 4: count_tier<HT, 4>(A, B, count, ovf, rows, n_work, wpb, is_long, s); break;
        case 2: count_tier<HT, 2>(A, B, count, ovf, rows, n_work, wpb, is_long, s); break;
        default: count_tier<HT, 1>(A, B, count, ovf, rows, n_work, wpb, is_long, s); break;
    }
}

template <int HT, int G>
void pattern_tier(const CsrView& A, const CsrView& B, Csr& C, const int* rows, int64_t n_work,
                  int wpb, cudaStream_t s) {
    const size_t smem = (size_t)wpb * 2 * HT * sizeof(int);
    set_smem(k_spgemm_pattern<HT, G>, smem);
    k_spgemm_pattern<HT, G><<<grid_for(n_work, wpb), wpb * 32, smem, s>>>(
        A.n_rows, A.rp, A.col, B.rp, B.col, C.row_ptr.get(), C.col.get(), rows);
    DPP_LAUNCH_CK();
}

template <int HT, int G, int CAP>
void scatter_tier(const CsrView& A, const CsrView& B, Csr& C, int* wide, const int* is_long,
                  cudaStream_t s) {
    const size_t smem = (size_t)kWarps * 2 * HT * sizeof(int) + (size_t)kWarps * G * CAP * sizeof(double);
    set_smem(k_spgemm_scatter<HT, G, CAP>, smem);
    k_spgemm_scatter<HT, G, CAP><<<grid_for(A.n_rows, kWarps), kWarps * 32, smem, s>>>(
        A.n_rows, A.rp, A.col, A.val, B.rp, B.col, B.val, C.row_ptr.get(), C.col.get(),
        C.val.get(), wide, is_long);
    DPP_LAUNCH_CK();
}

// G is capped so that the accumulators stay at or below 8 KB per warp.
template <int CAP>
void scatter_g(int G, const CsrView& A, const CsrView& B, Csr& C, int* wide, const int* is_long,
               cudaStream_t s) {
    constexpr int HT = 2 * CAP < 64 ? 64 : 2 * CAP;
    constexpr int GMAX = 1024 / CAP < 1 ? 1 : 1024 / CAP;
    G = std::min(G, GMAX);
    switch (G) {
        case 32: scatter_tier<HT, (GMAX >= 32 ? 32 : 1), CAP>(A, B, C, wide, is_long, s); break;
        case 16: scatter_tier<HT, (GMAX >= 16 ? 16 : 1), CAP>(A, B, C, wide, is_long, s); break;
        case 8: scatter_tier<HT, (GMAX >= 8 ? 8 : 1), CAP>(A, B, C, wide, is_long, s); break;
        case 4: scatter_tier<HT, (GMAX >= 4 ? 4 : 1), CAP>(A, B, C, wide, is_long, s); break;
        case 2: scatter_tier<HT, (GMAX >= 2 ? 2 : 1), CAP>(A, B, C, wide, is_long, s); break;
        default: scatter_tier<HT, 1, CAP>(A, B, C, wide, is_long, s); break;
    }
}

constexpr int kHtTiers[3] = {256, 2048, 8192};

}  // namespace

void spgemm(const CsrView& A, const CsrView& B, Csr& C, bool values, cudaStream_t s,
            HostScratch& hs) {
    ProfScope prof(values ? "spgemm_numeric" : "spgemm_pattern", s, 0);
    if (A.n_cols != B.n_rows) fail(DPP_ERR_INVALID_ARGUMENT, "spgemm: shape mismatch");
    const int64_t n = A.n_rows;
    C.n_rows = n;
    C.n_cols = B.n_cols;
    C.row_ptr.alloc(n + 1);
    DPP_CK(cudaMemsetAsync(C.row_ptr.get(), 0, (n + 1) * sizeof(int), s));
    const int G = groups_for(B.n_rows ? (double)B.nnz / (double)B.n_rows : 1.0);
    // symbolic: tiers of hash tables; rows[t] lists the rows retried in tier t
    DBuf<int> lists(2 * (n + 2));
    int* tier_rows[3] = {nullptr, lists.get() + 1, lists.get() + (n + 2) + 1};
    int64_t tier_n[3] = {n, 0, 0};
    DPP_CK(cudaMemsetAsync(lists.get(), 0, sizeof(int), s));
    DPP_CK(cudaMemsetAsync(lists.get() + (n + 2), 0, sizeof(int), s));
    DBuf<int> last_ovf(2);
    DPP_CK(cudaMemsetAsync(last_ovf.get(), 0, sizeof(int), s));
    // rows with many products go to the block-per-row kernels (numeric products only)
    DBuf<int> is_long(values ? n : 1), long_rows(values ? n + 2 : 1);
    int64_t n_long = 0;
    const int* long_flag = nullptr;
    if (values) {
        DPP_CK(cudaMemsetAsync(long_rows.get(), 0, sizeof(int), s));
        // only when rows are too few to fill the GPU with one warp per row
        const int threshold = (n < 16384) ? 2048 : INT_MAX;
        k_split_long<<<grid_for(n * 32, 256), 256, 0, s>>>(n, A.rp, A.col, B.rp, threshold,
                                                          is_long.get(), long_rows.get());
        DPP_LAUNCH_CK();
        n_long = read_scalar(long_rows.get(), s, hs);
        if (n_long > 0) long_flag = is_long.get();
    }
    {
        ProfScope pc("spgemm_count", s, 0);
        count_g<256>(G, A, B, C.row_ptr.get(), tier_rows[1] - 1, nullptr, n, kWarps, long_flag, s);
        tier_n[1] = read_scalar(tier_rows[1] - 1, s, hs);
        if (tier_n[1] > 0) {
            count_g<2048>(G, A, B, C.row_ptr.get(), tier_rows[2] - 1, tier_rows[1], tier_n[1], kWarps,
                          long_flag, s);
            tier_n[2] = read_scalar(tier_rows[2] - 1, s, hs);
        }
        if (tier_n[2] > 0) {
            count_g<8192>(G, A, B, C.row_ptr.get(), last_ovf.get(), tier_rows[2], tier_n[2], 1,
                          long_flag, s);
            if (read_scalar(last_ovf.get(), s, hs) > 0)
                fail(DPP_ERR_INVALID_ARGUMENT, "spgemm: a product row has more than 8191 distinct columns");
        }
        if (n_long > 0) {
            DBuf<int> st(1);
            DPP_CK(cudaMemsetAsync(st.get(), 0, sizeof(int), s));
            const size_t smem = (size_t)kLongHT * sizeof(int);
            set_smem(k_long_count, smem);
            k_long_count<<<(unsigned)n_long, kLongWarps * 32, smem, s>>>(
                A.rp, A.col, B.rp, B.col, C.row_ptr.get(), long_rows.get() + 1, st.get());
            DPP_LAUNCH_CK();
            if (read_scalar(st.get(), s, hs))
                fail(DPP_ERR_INVALID_ARGUMENT, "spgemm: a product row has more than 8191 distinct columns");
        }
    }
    C.nnz = exclusive_scan(C.row_ptr.get(), C.row_ptr.get(), n + 1, s, hs);
    {
        ProfScope pa("spgemm_alloc", s, 0);
        C.col.alloc(std::max<int64_t>(C.nnz, 1));
        if (values) C.val.alloc(std::max<int64_t>(C.nnz, 1));
    }
    ProfScope pf(values ? "spgemm_fill" : "spgemm_fill_pattern", s, 0);
    if (!values) {
        pattern_tier<256, 1>(A, B, C, nullptr, n, kWarps, s);  // rows that fit the first tier
        if (tier_n[1] > 0) pattern_tier<2048, 1>(A, B, C, tier_rows[1], tier_n[1], kWarps, s);
        if (tier_n[2] > 0) pattern_tier<8192, 1>(A, B, C, tier_rows[2], tier_n[2], 1, s);
        DPP_CK(cudaStreamSynchronize(s));
        return;
    }
    DBuf<int> mx(1);
    DPP_CK(cudaMemsetAsync(mx.get(), 0, sizeof(int), s));
    k_row_len_max<<<grid_for(n, 256), 256, 0, s>>>(n, C.row_ptr.get(), long_flag, mx.get());
    DPP_LAUNCH_CK();
    const int max_u = read_scalar(mx.get(), s, hs);
    DBuf<int> wide(n + 2), st(1);
    DPP_CK(cudaMemsetAsync(wide.get(), 0, sizeof(int), s));
    DPP_CK(cudaMemsetAsync(st.get(), 0, sizeof(int), s));
    if (n_long > 0) {
        const size_t smem = (size_t)(kLongHT + 2 * kLongCap) * sizeof(int) +
                            (size_t)kLongWarps * kLongCap * sizeof(double);
        set_smem(k_long_numeric, smem);
        k_long_numeric<<<(unsigned)n_long, kLongWarps * 32, smem, s>>>(
            A.rp, A.col, A.val, B.rp, B.col, B.val, C.row_ptr.get(), C.col.get(), C.val.get(),
            long_rows.get() + 1, wide.get());
        DPP_LAUNCH_CK();
    }
    if (n_long < n) {
        if (max_u <= 32) scatter_g<32>(G, A, B, C, wide.get(), long_flag, s);
        else if (max_u <= 64) scatter_g<64>(G, A, B, C, wide.get(), long_flag, s);
        else if (max_u <= 128) scatter_g<128>(G, A, B, C, wide.get(), long_flag, s);
        else if (max_u <= 256) scatter_g<256>(G, A, B, C, wide.get(), long_flag, s);
        else if (max_u <= 512) scatter_g<512>(G, A, B, C, wide.get(), long_flag, s);
        else scatter_g<1024>(G, A, B, C, wide.get(), long_flag, s);
    }
    const int n_wide = read_scalar(wide.get(), s, hs);
    if (n_wide > 0) {
        const size_t smem = (size_t)2 * 8192 * sizeof(int);
        set_smem(k_spgemm_wide<8192>, smem);
        k_spgemm_wide<8192><<<n_wide, 32, smem, s>>>(A.rp, A.col, A.val, B.rp, B.col, B.val,
                                                     C.row_ptr.get(), C.col.get(), C.val.get(),
                                                     wide.get() + 1, st.get());
        DPP_LAUNCH_CK();
        if (read_scalar(st.get(), s, hs))
            fail(DPP_ERR_INVALID_ARGUMENT, "spgemm: a product row has more than 8191 distinct columns");
    }
    DPP_CK(cudaStreamSynchronize(s));
}

void transpose(const Csr& A, Csr& T, cudaStream_t s, HostScratch& hs) {
    T.n_rows = A.n_cols;
    T.n_cols = A.n_rows;
    T.nnz = A.nnz;
    T.row_ptr.alloc(T.n_rows + 1);
    DPP_CK(cudaMemsetAsync(T.row_ptr.get(), 0, (T.n_rows + 1) * sizeof(int), s));
    const int B = 256;
    if (A.nnz) {
        k_col_count<<<grid_for(A.nnz, B), B, 0, s>>>(A.col.get(), A.nnz, T.row_ptr.get());
        DPP_LAUNCH_CK();
    }
    exclusive_scan(T.row_ptr.get(), T.row_ptr.get(), T.n_rows + 1, s, hs);
    T.col.alloc(std::max<int64_t>(A.nnz, 1));
    T.val.alloc(std::max<int64_t>(A.nnz, 1));
    DBuf<int> cursor(T.n_rows + 1);
    DPP_CK(cudaMemcpyAsync(cursor.get(), T.row_ptr.get(), (T.n_rows + 1) * sizeof(int),
                           cudaMemcpyDeviceToDevice, s));
    k_transpose_scatter<<<grid_for(A.n_rows, B), B, 0, s>>>(A.n_rows, A.row_ptr.get(), A.col.get(),
                                                            A.val.get(), cursor.get(), T.col.get(),
                                                            T.val.get());
    DPP_LAUNCH_CK();
    DBuf<int> tc(std::max<int64_t>(A.nnz, 1));
    DBuf<double> tv(std::max<int64_t>(A.nnz, 1));
    k_sort_rows<<<grid_for(T.n_rows * 32, B), B, 0, s>>>(T.n_rows, T.row_ptr.get(), T.col.get(),
                                                         T.val.get(), tc.get(), tv.get());
    DPP_LAUNCH_CK();
    DPP_CK(cudaStreamSynchronize(s));
}

void build_selfp(const ProblemImpl& P, const double* mdiag, Csr& S, cudaStream_t s,
                 HostScratch& hs) {
    // pattern of G*G with G the pair graph (self pairs included)
    CsrView G;
    G.n_rows = G.n_cols = P.n_nodes;
    G.nnz = P.n_pairs;
    G.rp = P.row_ptr.get();
    G.col = P.col.get();
    Csr Sh;
    spgemm(G, G, Sh, false, s, hs);
    const int64_t n = P.n_nodes, nnz = Sh.nnz;
    S.n_rows = S.n_cols = 2 * n;
    S.nnz = 2 * nnz;
    S.row_ptr.alloc(2 * n + 1);
    S.col.alloc(2 * nnz);
    S.val.alloc(2 * nnz);
    DPP_CK(cudaMemcpyAsync(S.row_ptr.get(), Sh.row_ptr.get(), (n + 1) * sizeof(int),
                           cudaMemcpyDeviceToDevice, s));
    DPP_CK(cudaMemcpyAsync(S.col.get(), Sh.col.get(), nnz * sizeof(int), cudaMemcpyDeviceToDevice, s));
    const int B = 256;
    k_dup_pattern<<<grid_for(std::max<int64_t>(nnz, n + 1), B), B, 0, s>>>(n, nnz, S.row_ptr.get(),
                                                                           S.col.get());
    DPP_LAUNCH_CK();
    if (P.dim == 2)
        k_selfp_values<2><<<grid_for(n * 32, B), B, 0, s>>>(
            n, P.row_ptr.get(), P.col.get(), P.slice_ptr.get(), P.sell_val.get(), mdiag,
            Sh.row_ptr.get(), Sh.col.get(), S.val.get(), nnz);
    else
        k_selfp_values<3><<<grid_for(n * 32, B), B, 0, s>>>(
            n, P.row_ptr.get(), P.col.get(), P.slice_ptr.get(), P.sell_val.get(), mdiag,
            Sh.row_ptr.get(), Sh.col.get(), S.val.get(), nnz);
    DPP_LAUNCH_CK();
    DPP_CK(cudaStreamSynchronize(s));
}

}  // namespace dpp
