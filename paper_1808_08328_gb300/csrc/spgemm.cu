// Sparse matrix products for the preconditioner setup:
//   * the selfp Schur matrices S_pi = Ki_pp - Ki_pu diag(Ki_uu)^-1 Ki_up
//     (Eqs. "S4_sp1", "S4_sp2", Section 4.2), formed straight from the node-pair
//     values and stored as the block-diagonal matrix blockdiag(S_p1, S_p2);
//   * the general CSR product C = A B. The AMG setup uses it for A P and for
//     the Galerkin product P^T (A P);
//   * the CSR transpose.
//
// Product scheme (deterministic; no floating-point atomics). One warp owns one
// output row:
//   1. symbolic: the warp inserts every candidate column of row i (the
//      columns of B's rows named by A's row i) into an open-addressing hash
//      set in shared memory and counts the distinct keys;
//   2. numeric: the warp rebuilds the set, compacts it, and ranks the keys
//      (the keys are distinct, so a key's rank is the number of smaller keys).
//      It writes the sorted columns. For each output column c it then gathers
//      sum_k A_ik B_kc in the fixed order of A's row, finding B_kc by binary
//      search in B's sorted row k.
// Rows whose distinct-column count exceeds the small table are redone with a
// larger table (one warp per block).
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
// pattern_only: when A has no values (pattern products).
template <int HT>
__device__ bool warp_collect(int i, const int* __restrict__ arp, const int* __restrict__ acol,
                             const int* __restrict__ brp, const int* __restrict__ bcol, int* keys,
                             int lane) {
    for (int t = lane; t < HT; t += 32) keys[t] = -1;
    __syncwarp();
    bool ok = true;
    for (int p = arp[i]; p < arp[i + 1]; ++p) {
        const int k = acol[p];
        for (int q = brp[k] + lane; q < brp[k + 1]; q += 32) ok &= hs_insert<HT>(keys, bcol[q]);
    }
    __syncwarp();
    return __all_sync(0xffffffffu, ok);
}

template <int HT>
__global__ void k_spgemm_count(int64_t n_rows, const int* __restrict__ arp,
                               const int* __restrict__ acol, const int* __restrict__ brp,
                               const int* __restrict__ bcol, int* __restrict__ count,
                               int* __restrict__ overflow, const int* __restrict__ rows) {
    extern __shared__ int smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    int64_t n_work = rows ? rows[-1] : n_rows;  // rows[-1] holds the count of listed rows
    if (w >= n_work) return;
    const int i = rows ? rows[w] : (int)w;
    int* keys = smem + warp * 2 * HT;
    bool ok = warp_collect<HT>(i, arp, acol, brp, bcol, keys, lane);
    int c = 0;
    for (int t = lane; t < HT; t += 32) c += (keys[t] >= 0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) {
        count[i] = ok ? c : 0;
        if (!ok) overflow[atomicAdd(&overflow[0], 1) + 1] = i;
    }
}

// Sorted distinct columns of row i into out (global), returns count.
template <int HT>
__device__ int warp_sorted_keys(int* keys, int* list, int lane, int* out) {
    // compact
    int base = 0;
    for (int t0 = 0; t0 < HT; t0 += 32) {
        int k = keys[t0 + lane];
        unsigned m = __ballot_sync(0xffffffffu, k >= 0);
        if (k >= 0) list[base + __popc(m & ((1u << lane) - 1u))] = k;
        base += __popc(m);
    }
    __syncwarp();
    // rank sort (keys are distinct)
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

template <int HT>
__global__ void k_spgemm_fill(int64_t n_rows, const int* __restrict__ arp,
                              const int* __restrict__ acol, const double* __restrict__ aval,
                              const int* __restrict__ brp, const int* __restrict__ bcol,
                              const double* __restrict__ bval, const int* __restrict__ crp,
                              int* __restrict__ ccol, double* __restrict__ cval,
                              const int* __restrict__ rows) {
    extern __shared__ int smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    int64_t n_work = rows ? rows[-1] : n_rows;
    if (w >= n_work) return;
    const int i = rows ? rows[w] : (int)w;
    int* keys = smem + warp * 2 * HT;
    int* list = keys + HT;
    if (!warp_collect<HT>(i, arp, acol, brp, bcol, keys, lane)) return;  // redone with a larger table
    const int c0 = crp[i];
    const int u = warp_sorted_keys<HT>(keys, list, lane, ccol + c0);
    if (!cval) return;
    for (int e = lane; e < u; e += 32) {
        const int c = ccol[c0 + e];
        double v = 0.0;
        for (int p = arp[i]; p < arp[i + 1]; ++p) {
            const int k = acol[p];
            const int q = bsearch_row(bcol, brp[k], brp[k + 1], c);
            if (q >= 0) v += aval[p] * bval[q];
        }
        cval[c0 + e] = v;
    }
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

constexpr int kHtSmall = 512;   // per-warp table (ints), 4 warps per block
constexpr int kHtLarge = 8192;  // one warp per block (64 KB of keys + list)

template <int HT>
void launch_count(const CsrView& A, const CsrView& B, int* count, int* overflow, const int* rows,
                  int64_t n_work, int wpb, cudaStream_t s) {
    size_t smem = (size_t)wpb * 2 * HT * sizeof(int);
    if (smem > 48 * 1024)
        DPP_CK(cudaFuncSetAttribute(k_spgemm_count<HT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    k_spgemm_count<HT><<<grid_for(n_work, wpb), wpb * 32, smem, s>>>(
        A.n_rows, A.rp, A.col, B.rp, B.col, count, overflow, rows);
    DPP_LAUNCH_CK();
}

template <int HT>
void launch_fill(const CsrView& A, const CsrView& B, Csr& C, const int* rows, int64_t n_work,
                 int wpb, bool values, cudaStream_t s) {
    size_t smem = (size_t)wpb * 2 * HT * sizeof(int);
    if (smem > 48 * 1024)
        DPP_CK(cudaFuncSetAttribute(k_spgemm_fill<HT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    k_spgemm_fill<HT><<<grid_for(n_work, wpb), wpb * 32, smem, s>>>(
        A.n_rows, A.rp, A.col, values ? A.val : nullptr, B.rp, B.col, values ? B.val : nullptr,
        C.row_ptr.get(), C.col.get(), values ? C.val.get() : nullptr, rows);
    DPP_LAUNCH_CK();
}

}  // namespace

void spgemm(const CsrView& A, const CsrView& B, Csr& C, bool values, cudaStream_t s,
            HostScratch& hs) {
    if (A.n_cols != B.n_rows) fail(DPP_ERR_INVALID_ARGUMENT, "spgemm: shape mismatch");
    const int64_t n = A.n_rows;
    C.n_rows = n;
    C.n_cols = B.n_cols;
    C.row_ptr.alloc(n + 1);
    DPP_CK(cudaMemsetAsync(C.row_ptr.get(), 0, (n + 1) * sizeof(int), s));
    DBuf<int> ovf(n + 2);  // ovf[0] = count, ovf[1..] = rows
    DPP_CK(cudaMemsetAsync(ovf.get(), 0, sizeof(int), s));
    launch_count<kHtSmall>(A, B, C.row_ptr.get(), ovf.get(), nullptr, n, 4, s);
    const int n_ovf = read_scalar(ovf.get(), s, hs);
    if (n_ovf > 0) {
        DBuf<int> ovf2(2);
        DPP_CK(cudaMemsetAsync(ovf2.get(), 0, sizeof(int), s));
        launch_count<kHtLarge>(A, B, C.row_ptr.get(), ovf2.get(), ovf.get() + 1, n_ovf, 1, s);
        if (read_scalar(ovf2.get(), s, hs) > 0)
            fail(DPP_ERR_INVALID_ARGUMENT, "spgemm: a product row has more than 8191 distinct columns");
    }
    C.nnz = exclusive_scan(C.row_ptr.get(), C.row_ptr.get(), n + 1, s, hs);
    C.col.alloc(std::max<int64_t>(C.nnz, 1));
    if (values) C.val.alloc(std::max<int64_t>(C.nnz, 1));
    launch_fill<kHtSmall>(A, B, C, nullptr, n, 4, values, s);
    if (n_ovf > 0) launch_fill<kHtLarge>(A, B, C, ovf.get() + 1, n_ovf, 1, values, s);
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
