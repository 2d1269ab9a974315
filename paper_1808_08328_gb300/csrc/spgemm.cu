// Sparse matrix products for the preconditioner setup:
//   * the selfp Schur matrices S_pi = Ki_pp - Ki_pu diag(Ki_uu)^-1 Ki_up
//     (Eqs. "S4_sp1", "S4_sp2", Section 4.2), formed straight from the node-pair
//     values and stored as the block-diagonal matrix blockdiag(S_p1, S_p2);
//   * the general CSR product C = A B. The AMG setup uses it for A P and for
//     the Galerkin product P^T (A P);
//   * the CSR transpose.
//
// Product scheme (deterministic; no floating-point atomics). One warp owns one
// output row i of C = A B. The warp takes A's row in chunks of 32 entries, one
// per lane; a warp prefix sum of the lengths of the B rows they select numbers
// the chunk's products t = 0, 1, ... in (p, q) order, and the warp then takes
// 32 consecutive products per round, one per lane, so every lane has a product
// and its own independent loads whatever the lengths of B's rows. A lane finds
// the A entry that owns its product by a binary search over the chunk's prefix
// sums held in the lanes' registers (shuffles).
//   1. symbolic: the candidate columns go into an open-addressing hash set in
//      shared memory, and the distinct keys are counted. Tables grow in tiers
//      (256, 2048, 8192 slots); a row that overflows one tier is retried in
//      the next;
//   2. numeric: the warp rebuilds the set, compacts it and ranks the keys
//      (they are distinct, so a key's rank is the number of smaller keys):
//      the ranks give the row's sorted columns and, stored beside each key in
//      the table, the accumulator slot of each column. Each round then adds
//      a_ip * b_pq into the slot of column q. Lanes of one round that hit the
//      same slot add one after another in lane order (found with a warp
//      match), and rounds follow each other, so every entry of C is summed in
//      the sequential (p, q) order and the result is deterministic. Rows
//      wider than the largest shared accumulator (1024 columns) use one warp
//      with the accumulator in C's own storage.
// Products with many rows (at least 16384) skip the counting pass: each row of
// at most 128 columns is collected, ranked and accumulated once into a
// fixed-capacity staging row, then a scan and a compaction copy build C; only
// the wider rows are counted, and they take a block-per-row kernel. Products
// with few rows give rows with many products to a block of 8 warps each.
// Symmetric Galerkin products may be formed as their upper triangle and
// mirrored (symmetrize_upper). S_p is built the same one-pass way, with its
// pattern (the pair graph squared) collected by the same product loop.
#include <climits>

#include "amg.cuh"

namespace dpp {

namespace {
constexpr unsigned kFull = 0xffffffffu;

// multiplicative (Fibonacci) hashing: the top log2(HT) bits of k * 2^32/phi
template <int HT>
__device__ __forceinline__ unsigned hash_slot(int k) {
    constexpr int bits = __builtin_ctz(HT);
    return ((unsigned)k * 2654435761u) >> (32 - bits);
}

// Most inserts find their key already present, so a plain read comes first and
// only an empty slot takes the atomic.
template <int HT>
__device__ __forceinline__ bool hs_insert(int* keys, int key) {
    unsigned h = hash_slot<HT>(key);
    for (int probe = 0; probe < HT; ++probe) {
        const int cur = reinterpret_cast<volatile int*>(keys)[h];
        if (cur == key) return true;
        if (cur == -1) {
            const int prev = atomicCAS(&keys[h], -1, key);
            if (prev == -1 || prev == key) return true;
        }
        h = (h + 1) & (HT - 1);
    }
    return false;
}

// table position of a key known to be in the set (-1 if absent)
template <int HT>
__device__ __forceinline__ int hs_find(const int* keys, int key) {
    unsigned h = hash_slot<HT>(key);
    for (int probe = 0; probe < HT; ++probe) {
        const int k = keys[h];
        if (k == key) return (int)h;
        if (k < 0) return -1;
        h = (h + 1) & (HT - 1);
    }
    return -1;
}

// first position in the sorted col[lo, hi) with col >= key
__device__ __forceinline__ int lower_bound_col(const int* __restrict__ col, int lo, int hi, int key) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (col[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Start of the part of B's row k that the product row needs: all of it, or,
// for the upper triangle of a symmetric product (col_lo = the row index), the
// columns >= col_lo (B's rows are sorted).
__device__ __forceinline__ int b_row_start(const int* __restrict__ brp, const int* __restrict__ bcol,
                                           int k, int col_lo) {
    return (col_lo == INT_MIN) ? brp[k] : lower_bound_col(bcol, brp[k], brp[k + 1], col_lo);
}

// Calls f(active, q, a_ip) for every product of row i of A B, 32 per round,
// in (p, q) order; every lane of the warp makes every call (f may use warp
// collectives), inactive lanes with active == false. Only columns >= col_lo
// are produced (INT_MIN: all).
template <bool VALS, class V, class F>
__device__ __forceinline__ void for_each_product(int i, const int* __restrict__ arp,
                                                 const int* __restrict__ acol,
                                                 const V* __restrict__ aval,
                                                 const int* __restrict__ brp,
                                                 const int* __restrict__ bcol, int col_lo, int lane,
                                                 F&& f) {
    const int a0 = arp[i], a1 = arp[i + 1];
    for (int pc = a0; pc < a1; pc += 32) {
        const int p = pc + lane;
        int bs = 0, len = 0;
        V a = V(0);
        if (p < a1) {
            const int k = acol[p];
            bs = b_row_start(brp, bcol, k, col_lo);
            len = brp[k + 1] - bs;
            if (VALS) a = aval[p];
        }
        int inc = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += y;
        }
        const int total = __shfl_sync(kFull, inc, 31);
        const int excl = inc - len;
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + lane;
            int j = 0;  // owner: the last lane whose products start at or before t
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int e = __shfl_sync(kFull, excl, j + step);
                if (e <= t) j += step;
            }
            const int q = __shfl_sync(kFull, bs, j) + (t - __shfl_sync(kFull, excl, j));
            const V aj = VALS ? __shfl_sync(kFull, a, j) : V(0);
            f(t < total, q, aj);
        }
    }
}

// Fill the warp's hash set with the candidate columns of row i of A*B.
template <int HT>
__device__ bool warp_collect(int i, const int* __restrict__ arp, const int* __restrict__ acol,
                             const int* __restrict__ brp, const int* __restrict__ bcol, int* keys,
                             int lane, int col_lo) {
    for (int t = lane; t < HT; t += 32) keys[t] = -1;
    __syncwarp();
    bool ok = true;
    for_each_product<false, double>(i, arp, acol, nullptr, brp, bcol, col_lo, lane, [&](bool act, int q, double) {
        if (act) ok &= hs_insert<HT>(keys, bcol[q]);
    });
    __syncwarp();
    return __all_sync(kFull, ok);
}

// Compact the set into list[0..u) (any order); returns u.
template <int HT>
__device__ int warp_compact(const int* keys, int* list, int lane) {
    int base = 0;
    for (int t0 = 0; t0 < HT; t0 += 32) {
        const int k = keys[t0 + lane];
        const unsigned m = __ballot_sync(kFull, k >= 0);
        if (k >= 0) list[base + __popc(m & ((1u << lane) - 1u))] = k;
        base += __popc(m);
    }
    __syncwarp();
    return base;
}

// Rank the distinct keys list[0..u): out[rank] = key and, if slot != nullptr,
// slot[table position of key] = rank. Each lane holds up to 8 keys in
// registers and reads the list once per batch.
template <int HT>
__device__ void warp_rank(const int* list, int u, int lane, int* __restrict__ out,
                          const int* keys, int* slot) {
    constexpr int KR = 8;
    for (int e0 = 0; e0 < u; e0 += 32 * KR) {
        int k[KR], r[KR];
#pragma unroll
        for (int j = 0; j < KR; ++j) {
            const int e = e0 + j * 32 + lane;
            k[j] = (e < u) ? list[e] : INT_MAX;
            r[j] = 0;
        }
        for (int f = 0; f < u; ++f) {
            const int v = list[f];
#pragma unroll
            for (int j = 0; j < KR; ++j) r[j] += (v < k[j]);
        }
#pragma unroll
        for (int j = 0; j < KR; ++j) {
            if (e0 + j * 32 + lane < u) {
                out[r[j]] = k[j];
                if (slot) slot[hs_find<HT>(keys, k[j])] = r[j];
            }
        }
    }
    __syncwarp();
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
template <int HT>
__global__ void k_spgemm_count(int64_t n_rows, const int* __restrict__ arp,
                               const int* __restrict__ acol, const int* __restrict__ brp,
                               const int* __restrict__ bcol, int* __restrict__ count,
                               int* __restrict__ ovf, const int* __restrict__ rows,
                               const int* __restrict__ is_long, int upper) {
    extern __shared__ int smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    const int64_t n_work = rows ? rows[-1] : n_rows;
    if (w >= n_work) return;
    const int i = rows ? rows[w] : (int)w;
    if (is_long && is_long[i]) return;  // done by the block-per-row kernels
    int* keys = smem + warp * HT;
    const bool ok = warp_collect<HT>(i, arp, acol, brp, bcol, keys, lane, upper ? i : INT_MIN);
    int c = 0;
    for (int t = lane; t < HT; t += 32) c += (keys[t] >= 0);
    c = __reduce_add_sync(kFull, c);
    if (lane == 0) {
        count[i] = ok ? c : 0;
        if (!ok) ovf[atomicAdd(&ovf[0], 1) + 1] = i;
    }
}

// Symbolic fill for pattern-only products: sorted columns of each row.
template <int HT>
__global__ void k_spgemm_pattern(int64_t n_rows, const int* __restrict__ arp,
                                 const int* __restrict__ acol, const int* __restrict__ brp,
                                 const int* __restrict__ bcol, const int* __restrict__ crp,
                                 int* __restrict__ ccol, const int* __restrict__ rows, int upper) {
    extern __shared__ int smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    const int64_t n_work = rows ? rows[-1] : n_rows;
    if (w >= n_work) return;
    const int i = rows ? rows[w] : (int)w;
    int* keys = smem + warp * 2 * HT;
    if (!warp_collect<HT>(i, arp, acol, brp, bcol, keys, lane, upper ? i : INT_MIN)) return;
    int* list = keys + HT;
    const int u = warp_compact<HT>(keys, list, lane);
    warp_rank<HT>(list, u, lane, ccol + crp[i], keys, nullptr);
}

// Numeric pass for rows with at most CAP distinct columns (shared accumulators).
// Shared memory per warp: keys[HT], slot[HT], acc[CAP] (the compacted key list
// lives in acc until the ranks are known).
template <int HT, int CAP, class V>
__global__ void k_spgemm_scatter(int64_t n_rows, const int* __restrict__ arp,
                                 const int* __restrict__ acol, const V* __restrict__ aval,
                                 const int* __restrict__ brp, const int* __restrict__ bcol,
                                 const V* __restrict__ bval, const int* __restrict__ crp,
                                 int* __restrict__ ccol, V* __restrict__ cval,
                                 int* __restrict__ wide, const int* __restrict__ is_long,
                                 int upper) {
    static_assert(HT >= 2 * CAP, "table at most half full");
    extern __shared__ int smem[];
    constexpr int WPB = 4;
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
    int* slot = keys + HT;
    V* acc = reinterpret_cast<V*>(smem + WPB * 2 * HT) + (size_t)warp * CAP;
    const int col_lo = upper ? i : INT_MIN;
    warp_collect<HT>(i, arp, acol, brp, bcol, keys, lane, col_lo);  // cannot overflow (HT >= 2 CAP)
    int* list = reinterpret_cast<int*>(acc);
    const int u = warp_compact<HT>(keys, list, lane);
    warp_rank<HT>(list, u, lane, ccol + c0, keys, slot);
    for (int e = lane; e < u; e += 32) acc[e] = V(0);
    __syncwarp();
    for_each_product<true, V>(i, arp, acol, aval, brp, bcol, col_lo, lane, [&](bool act, int q, V a) {
        int s = -1 - lane;  // distinct for idle lanes
        V bv = V(0);
        if (act) {
            const int key = bcol[q];
            bv = bval[q];
            s = slot[hs_find<HT>(keys, key)];
        }
        const unsigned peers = __match_any_sync(kFull, s);
        const int order = __popc(peers & ((1u << lane) - 1u));
        const int n_sub = (int)__reduce_max_sync(kFull, (unsigned)__popc(peers));
        for (int r = 0; r < n_sub; ++r) {  // one fused multiply-add per product
            if (act && order == r) acc[s] = fma(a, bv, acc[s]);
            __syncwarp();
        }
    });
    for (int e = lane; e < u; e += 32) cval[c0 + e] = acc[e];
}

// One-pass product for rows of at most CAP distinct columns: the warp
// collects, ranks and accumulates its row exactly as k_spgemm_scatter does,
// but writes it to a fixed-capacity staging row (tcol/tval + i * CAP) and
// records its length, so no separate counting pass is needed. Rows that do
// not fit get uone[i] = -1 and are listed in ovf (ovf[0] = count) for the
// counting tiers and k_spgemm_wide.
// Per warp the accumulators take CAP values, and at least HT ints: the
// compacted key list lives there until the ranks are known.
template <int HT, int CAP, class V>
__host__ __device__ constexpr size_t onepass_acc_bytes() {
    return CAP * sizeof(V) > HT * sizeof(int) ? CAP * sizeof(V) : HT * sizeof(int);
}

template <int HT, int CAP, class V>
__global__ void k_spgemm_onepass(int64_t n_rows, const int* __restrict__ arp,
                                 const int* __restrict__ acol, const V* __restrict__ aval,
                                 const int* __restrict__ brp, const int* __restrict__ bcol,
                                 const V* __restrict__ bval, int* __restrict__ count,
                                 int* __restrict__ uone, int* __restrict__ tcol,
                                 V* __restrict__ tval, int* __restrict__ ovf, int upper) {
    static_assert(HT == 2 * CAP, "tables at most half full");
    extern __shared__ int smem[];
    constexpr int WPB = 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * WPB + warp;
    if (w >= n_rows) return;
    const int i = (int)w;
    int* keys = smem + warp * 2 * HT;
    int* slot = keys + HT;
    V* acc = reinterpret_cast<V*>(reinterpret_cast<char*>(smem + WPB * 2 * HT) +
                                  (size_t)warp * onepass_acc_bytes<HT, CAP, V>());
    const int col_lo = upper ? i : INT_MIN;
    const bool ok = warp_collect<HT>(i, arp, acol, brp, bcol, keys, lane, col_lo);
    int* list = reinterpret_cast<int*>(acc);  // HT ints
    const int u = ok ? warp_compact<HT>(keys, list, lane) : HT + 1;
    if (u > CAP) {
        if (lane == 0) {
            count[i] = 0;
            uone[i] = -1;
            ovf[atomicAdd(&ovf[0], 1) + 1] = i;
        }
        return;
    }
    int* orow = tcol + (int64_t)i * CAP;
    warp_rank<HT>(list, u, lane, orow, keys, slot);
    for (int e = lane; e < u; e += 32) acc[e] = V(0);
    __syncwarp();
    for_each_product<true, V>(i, arp, acol, aval, brp, bcol, col_lo, lane, [&](bool act, int q, V a) {
        int sl = -1 - lane;
        V bv = V(0);
        if (act) {
            bv = bval[q];
            sl = slot[hs_find<HT>(keys, bcol[q])];
        }
        const unsigned peers = __match_any_sync(kFull, sl);
        const int order = __popc(peers & ((1u << lane) - 1u));
        const int n_sub = (int)__reduce_max_sync(kFull, (unsigned)__popc(peers));
        for (int r = 0; r < n_sub; ++r) {  // one fused multiply-add per product
            if (act && order == r) acc[sl] = fma(a, bv, acc[sl]);
            __syncwarp();
        }
    });
    V* vrow = tval + (int64_t)i * CAP;
    for (int e = lane; e < u; e += 32) vrow[e] = acc[e];
    if (lane == 0) {
        count[i] = u;
        uone[i] = u;
    }
}

// staged rows into C (one warp per row; rows with uone < 0 are done elsewhere)
template <int CAP, class V>
__global__ void k_onepass_compact(int64_t n_rows, const int* __restrict__ uone,
                                  const int* __restrict__ crp, const int* __restrict__ tcol,
                                  const V* __restrict__ tval, int* __restrict__ ccol,
                                  V* __restrict__ cval) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n_rows) return;
    const int u = uone[i];
    const int c0 = crp[i];
    for (int e = lane; e < u; e += 32) {
        ccol[c0 + e] = tcol[i * CAP + e];
        cval[c0 + e] = tval[i * CAP + e];
    }
}

// Numeric pass for wide rows: one warp per listed row, accumulating in C.
template <int HT, class V>
__global__ void k_spgemm_wide(const int* __restrict__ arp, const int* __restrict__ acol,
                              const V* __restrict__ aval, const int* __restrict__ brp,
                              const int* __restrict__ bcol, const V* __restrict__ bval,
                              const int* __restrict__ crp, int* __restrict__ ccol,
                              V* __restrict__ cval, const int* __restrict__ rows,
                              int* __restrict__ status, int upper) {
    extern __shared__ int smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (w >= rows[-1]) return;
    const int i = rows[w];
    const int col_lo = upper ? i : INT_MIN;
    int* keys = smem + warp * 2 * HT;
    if (!warp_collect<HT>(i, arp, acol, brp, bcol, keys, lane, col_lo)) {
        if (lane == 0) atomicOr(status, 1);
        return;
    }
    const int c0 = crp[i];
    const int u = warp_compact<HT>(keys, keys + HT, lane);
    warp_rank<HT>(keys + HT, u, lane, ccol + c0, keys, nullptr);
    for (int e = lane; e < u; e += 32) cval[c0 + e] = V(0);
    __syncwarp();
    for (int p = arp[i]; p < arp[i + 1]; ++p) {
        const int k = acol[p];
        const V a = aval[p];
        for (int q = b_row_start(brp, bcol, k, col_lo) + lane; q < brp[k + 1]; q += 32) {
            V& cq = cval[bsearch_row(ccol, c0, c0 + u, bcol[q])];
            cq = fma(a, bval[q], cq);
        }
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
             const int* __restrict__ rows, int* __restrict__ status, int upper) {
    extern __shared__ int keys[];
    __shared__ int part[kLongWarps];
    const int i = rows[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = threadIdx.x; t < kLongHT; t += blockDim.x) keys[t] = -1;
    __syncthreads();
    bool ok = true;
    for (int p = arp[i] + warp; p < arp[i + 1]; p += kLongWarps) {
        const int k = acol[p];
        for (int q = b_row_start(brp, bcol, k, upper ? i : INT_MIN) + lane; q < brp[k + 1]; q += 32)
            ok &= hs_insert<kLongHT>(keys, bcol[q]);
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

template <class V>
__global__ void __launch_bounds__(kLongWarps * 32)
k_long_numeric(const int* __restrict__ arp, const int* __restrict__ acol,
               const V* __restrict__ aval, const int* __restrict__ brp,
               const int* __restrict__ bcol, const V* __restrict__ bval,
               const int* __restrict__ crp, int* __restrict__ ccol, V* __restrict__ cval,
               const int* __restrict__ rows, int* __restrict__ wide, int upper) {
    extern __shared__ int smem[];
    int* keys = smem;                                  // kLongHT
    int* list = keys + kLongHT;                        // kLongCap
    int* sorted = list + kLongCap;                     // kLongCap
    V* acc = reinterpret_cast<V*>(sorted + kLongCap);  // kLongWarps * kLongCap
    __shared__ int nu;
    const int i = rows[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = crp[i], u = crp[i + 1] - c0;
    if (u > kLongCap) {
        if (threadIdx.x == 0) wide[atomicAdd(&wide[0], 1) + 1] = i;
        return;
    }
    for (int t = threadIdx.x; t < kLongHT; t += blockDim.x) keys[t] = -1;
    for (int t = threadIdx.x; t < kLongWarps * kLongCap; t += blockDim.x) acc[t] = V(0);
    if (threadIdx.x == 0) nu = 0;
    __syncthreads();
    for (int p = arp[i] + warp; p < arp[i + 1]; p += kLongWarps) {
        const int k = acol[p];
        for (int q = b_row_start(brp, bcol, k, upper ? i : INT_MIN) + lane; q < brp[k + 1]; q += 32)
            hs_insert<kLongHT>(keys, bcol[q]);
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
    V* my = acc + warp * kLongCap;
    for (int p = arp[i] + warp; p < arp[i + 1]; p += kLongWarps) {
        const int k = acol[p];
        const V a = aval[p];
        for (int q = b_row_start(brp, bcol, k, upper ? i : INT_MIN) + lane; q < brp[k + 1]; q += 32)
            my[bsearch_row(sorted, 0, u, bcol[q])] += a * bval[q];
        __syncwarp();
    }
    __syncthreads();
    for (int e = threadIdx.x; e < u; e += blockDim.x) {
        V v = acc[e];
#pragma unroll
        for (int w = 1; w < kLongWarps; ++w) v += acc[w * kLongCap + e];
        cval[c0 + e] = v;
    }
}

// Long rows of a product whose B has at most kLongBitCols columns: the row's
// column set is a bitmap in shared memory. A column's place in the sorted row
// is the number of set bits before it (a prefix sum of the words' popcounts and
// one popcount inside the word), so no hash table, sort or search is needed.
// The values are accumulated as in k_long_numeric (one accumulator per warp,
// entries of A in p order, added in warp order), so both give the same sums.
constexpr int kLongBitCols = 65536;
constexpr int kLongBitWords = kLongBitCols / 32;

// false (and nothing written) for a column outside the bitmap's n_words words
__device__ __forceinline__ bool bm_set(unsigned* bm, int c, int n_words) {
    if ((unsigned)c >= 32u * (unsigned)n_words) return false;
    const unsigned bit = 1u << (c & 31);
    if (!(bm[c >> 5] & bit)) atomicOr(&bm[c >> 5], bit);  // plain read first: most bits repeat
    return true;
}

// pre[w] = set bits in words 0..w-1 (block-wide exclusive scan); bm is final.
__device__ __forceinline__ void bm_prefix(const unsigned* bm, int* pre, int n_words, int* warp_tot) {
    const int per = (n_words + (int)blockDim.x - 1) / (int)blockDim.x;
    const int w0 = min((int)threadIdx.x * per, n_words), w1 = min(w0 + per, n_words);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int mine = 0;
    for (int w = w0; w < w1; ++w) mine += __popc(bm[w]);
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int run = incl - mine;
    for (int w = 0; w < warp; ++w) run += warp_tot[w];
    for (int w = w0; w < w1; ++w) {
        pre[w] = run;
        run += __popc(bm[w]);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kLongWarps * 32)
k_long_count_bm(const int* __restrict__ arp, const int* __restrict__ acol,
                const int* __restrict__ brp, const int* __restrict__ bcol, int n_words,
                int* __restrict__ count, const int* __restrict__ rows, int* __restrict__ status,
                int upper) {
    __shared__ unsigned bm[kLongBitWords];
    __shared__ int part[kLongWarps];
    const int i = rows[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = threadIdx.x; t < n_words; t += blockDim.x) bm[t] = 0u;
    __syncthreads();
    bool ok = true;
    for (int p = arp[i] + warp; p < arp[i + 1]; p += kLongWarps) {
        const int k = acol[p];
        for (int q = b_row_start(brp, bcol, k, upper ? i : INT_MIN) + lane; q < brp[k + 1]; q += 32)
            ok &= bm_set(bm, bcol[q], n_words);
    }
    if (!ok) atomicOr(status, 1);
    __syncthreads();
    int c = 0;
    for (int t = threadIdx.x; t < n_words; t += blockDim.x) c += __popc(bm[t]);
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) part[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kLongWarps; ++w) t += part[w];
        count[i] = t;
    }
}

template <class V>
constexpr size_t long_bm_smem() {
    return (size_t)kLongWarps * kLongCap * sizeof(V) + (size_t)kLongBitWords * (sizeof(unsigned) + sizeof(int)) +
           (size_t)kLongWarps * sizeof(int);
}

template <class V>
__global__ void __launch_bounds__(kLongWarps * 32)
k_long_numeric_bm(const int* __restrict__ arp, const int* __restrict__ acol,
                  const V* __restrict__ aval, const int* __restrict__ brp,
                  const int* __restrict__ bcol, const V* __restrict__ bval, int n_words,
                  const int* __restrict__ crp, int* __restrict__ ccol, V* __restrict__ cval,
                  const int* __restrict__ rows, int* __restrict__ wide, int* __restrict__ status,
                  int upper) {
    extern __shared__ __align__(16) unsigned char long_bm_mem[];
    V* acc = reinterpret_cast<V*>(long_bm_mem);                                // kLongWarps * kLongCap
    unsigned* bm = reinterpret_cast<unsigned*>(acc + kLongWarps * kLongCap);  // kLongBitWords
    int* pre = reinterpret_cast<int*>(bm + kLongBitWords);                     // kLongBitWords
    int* warp_tot = pre + kLongBitWords;                                       // kLongWarps
    // (all of it dynamic: the launch sets the opt-in size whenever it passes 48 KB)
    const int i = rows[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = crp[i], u = crp[i + 1] - c0;
    if (u > kLongCap) {
        if (threadIdx.x == 0) wide[atomicAdd(&wide[0], 1) + 1] = i;
        return;
    }
    V* my = acc + warp * kLongCap;
    for (int e = lane; e < u; e += 32) my[e] = V(0);
    for (int t = threadIdx.x; t < n_words; t += blockDim.x) bm[t] = 0u;
    __syncthreads();
    bool ok = true;
    for (int p = arp[i] + warp; p < arp[i + 1]; p += kLongWarps) {
        const int k = acol[p];
        for (int q = b_row_start(brp, bcol, k, upper ? i : INT_MIN) + lane; q < brp[k + 1]; q += 32)
            ok &= bm_set(bm, bcol[q], n_words);
    }
    if (!ok) atomicOr(status, 1);
    __syncthreads();
    bm_prefix(bm, pre, n_words, warp_tot);
    // the row's column count must be the one counted (it sizes C's row)
    if (threadIdx.x == 0 && (n_words > 0 ? pre[n_words - 1] + __popc(bm[n_words - 1]) : 0) != u)
        atomicOr(status, 1);
    for (int w = threadIdx.x; w < n_words; w += blockDim.x) {
        unsigned m = bm[w];
        int r = pre[w];
        while (m && r < u) {
            ccol[c0 + r++] = w * 32 + (__ffs(m) - 1);
            m &= m - 1u;
        }
    }
    for (int p = arp[i] + warp; p < arp[i + 1]; p += kLongWarps) {
        const int k = acol[p];
        const V a = aval[p];
        for (int q = b_row_start(brp, bcol, k, upper ? i : INT_MIN) + lane; q < brp[k + 1]; q += 32) {
            const int c = bcol[q];
            if ((unsigned)c >= 32u * (unsigned)n_words) continue;  // flagged above
            const int pos = pre[c >> 5] + __popc(bm[c >> 5] & ((1u << (c & 31)) - 1u));
            if (pos < u) my[pos] += a * bval[q];                    // else flagged above
        }
        __syncwarp();
    }
    __syncthreads();
    for (int e = threadIdx.x; e < u; e += blockDim.x) {
        V v = acc[e];
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
// produced by the product kernels above with A = B = pair graph. Row a:
//   S_pi[a][c] = D_i[a][c] - sum_b C[a][b] . B[b][c] / M_i[b]
// (C the pressure-velocity and B the velocity-pressure pair blocks, M_i the
// diagonal velocity mass). One warp per node a: the D terms are written into
// shared accumulators first, then the products (b in N(a), c in N(b)) run
// 32 per round in (b, c) order as in the general product kernels, and lanes of
// one round that hit the same column subtract in lane order. Every entry is
// therefore summed over b in increasing order, as the definition reads. Rows
// with more than CAP columns are listed in `wide` for k_selfp_values.
template <int DIM, int CAP, class V>
__global__ void __launch_bounds__(128, 8)
k_selfp_scatter(int64_t n_nodes, const int* __restrict__ prp, const int* __restrict__ pcol,
                const int* __restrict__ slice_ptr, const V* __restrict__ pv,
                const V* __restrict__ mdiag, const int* __restrict__ srp,
                const int* __restrict__ scol, V* __restrict__ sval, int64_t nnz_half,
                int* __restrict__ wide) {
    constexpr int NV = pair_values(DIM);
    constexpr int HT = 2 * CAP;
    constexpr int WPB = 4;
    __shared__ int sh_keys[WPB][HT];
    __shared__ int sh_slot[WPB][HT];
    __shared__ V sh_acc[WPB][2][CAP];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t a = (int64_t)blockIdx.x * WPB + warp;
    if (a >= n_nodes) return;
    const int e0 = srp[a], u = srp[a + 1] - e0;
    if (u > CAP) {
        if (lane == 0) wide[atomicAdd(&wide[0], 1) + 1] = (int)a;
        return;
    }
    int* keys = sh_keys[warp];
    int* slot = sh_slot[warp];
    V* acc1 = sh_acc[warp][0];
    V* acc2 = sh_acc[warp][1];
    auto pval = [&](int row, int p, int k) -> V {
        const int64_t grp = (int64_t)slice_ptr[row >> 5] + (p - prp[row]);
        return pv[(grp * NV + k) * kSell + (row & 31)];
    };
    for (int t = lane; t < HT; t += 32) keys[t] = -1;
    for (int e = lane; e < CAP; e += 32) acc1[e] = acc2[e] = V(0);
    __syncwarp();
    for (int e = lane; e < u; e += 32) {  // the row's columns are distinct
        const int c = scol[e0 + e];
        hs_insert<HT>(keys, c);
    }
    __syncwarp();
    for (int e = lane; e < u; e += 32) slot[hs_find<HT>(keys, scol[e0 + e])] = e;
    __syncwarp();
    const int pa0 = prp[a], pa1 = prp[a + 1];
    for (int pac = pa0 + lane; pac < pa1; pac += 32) {  // D terms: distinct columns
        const int e = slot[hs_find<HT>(keys, pcol[pac])];
        acc1[e] = pval((int)a, pac, 2 + 2 * DIM);
        acc2[e] = pval((int)a, pac, 3 + 2 * DIM);
    }
    __syncwarp();
    for (int pc0 = pa0; pc0 < pa1; pc0 += 32) {
        const int pab = pc0 + lane;
        int b = 0, bs = 0, len = 0;
        V cab[DIM], m1 = V(0), m2 = V(0);
#pragma unroll
        for (int k = 0; k < DIM; ++k) cab[k] = V(0);
        if (pab < pa1) {
            b = pcol[pab];
            bs = prp[b];
            len = prp[b + 1] - bs;
#pragma unroll
            for (int k = 0; k < DIM; ++k) cab[k] = pval((int)a, pab, 2 + DIM + k);
            m1 = mdiag[2 * b];
            m2 = mdiag[2 * b + 1];
        }
        int inc = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += y;
        }
        const int total = __shfl_sync(kFull, inc, 31);
        const int excl = inc - len;
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + lane;
            int j = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int ex = __shfl_sync(kFull, excl, j + step);
                if (ex <= t) j += step;
            }
            const int bj = __shfl_sync(kFull, b, j);
            const int pbc = __shfl_sync(kFull, bs, j) + (t - __shfl_sync(kFull, excl, j));
            V cj[DIM];
#pragma unroll
            for (int k = 0; k < DIM; ++k) cj[k] = __shfl_sync(kFull, cab[k], j);
            const V mj1 = __shfl_sync(kFull, m1, j), mj2 = __shfl_sync(kFull, m2, j);
            const bool act = t < total;
            int e = -1 - lane;
            V dot = V(0);
            if (act) {
#pragma unroll
                for (int k = 0; k < DIM; ++k) dot += cj[k] * pval(bj, pbc, 2 + k);
                e = slot[hs_find<HT>(keys, pcol[pbc])];
            }
            const unsigned peers = __match_any_sync(kFull, e);
            const int order = __popc(peers & ((1u << lane) - 1u));
            const int n_sub = (int)__reduce_max_sync(kFull, (unsigned)__popc(peers));
            for (int r = 0; r < n_sub; ++r) {
                if (act && order == r) {
                    acc1[e] -= dot * mj1;
                    acc2[e] -= dot * mj2;
                }
                __syncwarp();
            }
        }
    }
    __syncwarp();
    for (int e = lane; e < u; e += 32) {
        sval[e0 + e] = acc1[e];
        sval[nnz_half + e0 + e] = acc2[e];
    }
}

// Entry-per-lane form with a binary search per (a, b, c): used for the rows
// listed in rows[0..rows[-1]) that are too wide for k_selfp_scatter.
template <int DIM, class V>
__global__ void k_selfp_values(const int* __restrict__ rows, const int* __restrict__ prp,
                               const int* __restrict__ pcol, const int* __restrict__ slice_ptr,
                               const V* __restrict__ pv, const V* __restrict__ mdiag,
                               const int* __restrict__ srp, const int* __restrict__ scol,
                               V* __restrict__ sval, int64_t nnz_half) {
    constexpr int NV = pair_values(DIM);
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= rows[-1]) return;
    const int64_t a = rows[w];
    auto pval = [&](int row, int p, int k) -> V {
        int64_t grp = (int64_t)slice_ptr[row >> 5] + (p - prp[row]);
        return pv[(grp * NV + k) * kSell + (row & 31)];
    };
    for (int e = srp[a] + lane; e < srp[a + 1]; e += 32) {
        const int c = scol[e];
        V s1 = V(0), s2 = V(0);
        const int pac = bsearch_row(pcol, prp[a], prp[a + 1], c);
        if (pac >= 0) {
            s1 = pval((int)a, pac, 2 + 2 * DIM);
            s2 = pval((int)a, pac, 3 + 2 * DIM);
        }
        for (int pab = prp[a]; pab < prp[a + 1]; ++pab) {
            const int b = pcol[pab];
            const int pbc = bsearch_row(pcol, prp[b], prp[b + 1], c);
            if (pbc < 0) continue;
            V dot = V(0);
#pragma unroll
            for (int k = 0; k < DIM; ++k) dot += pval((int)a, pab, 2 + DIM + k) * pval(b, pbc, 2 + k);
            s1 -= dot * mdiag[2 * b];
            s2 -= dot * mdiag[2 * b + 1];
        }
        sval[e] = s1;
        sval[nnz_half + e] = s2;
    }
}

// One pass for S_p: the warp of node a collects the columns c of its row
// (c in N(b), b in N(a): the products of G G with G the pair graph), ranks
// them, and accumulates the D and Schur terms into slots exactly as
// k_selfp_scatter does; the sorted columns and both networks' values go to
// fixed-capacity staging rows. A row wider than CAP sets *ovf, and the
// caller then builds S_p the two-pass way.
template <int DIM, int CAP, class V>
__global__ void __launch_bounds__(128, 8)
k_selfp_onepass(int64_t n_nodes, const int* __restrict__ prp, const int* __restrict__ pcol,
                const int* __restrict__ slice_ptr, const V* __restrict__ pv,
                const V* __restrict__ mdiag, int* __restrict__ count, int* __restrict__ tcol,
                V* __restrict__ tv1, V* __restrict__ tv2, int* __restrict__ ovf) {
    constexpr int NV = pair_values(DIM);
    constexpr int HT = 2 * CAP;
    constexpr int WPB = 4;
    __shared__ int sh_keys[WPB][HT];
    __shared__ int sh_slot[WPB][HT];
    __shared__ V sh_acc[WPB][2][CAP];
    static_assert(2 * CAP * sizeof(V) >= HT * sizeof(int), "the key list lives in the accumulators");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t a = (int64_t)blockIdx.x * WPB + warp;
    if (a >= n_nodes) return;
    int* keys = sh_keys[warp];
    int* slot = sh_slot[warp];
    V* acc1 = sh_acc[warp][0];
    V* acc2 = sh_acc[warp][1];
    auto pval = [&](int row, int p, int k) -> V {
        const int64_t grp = (int64_t)slice_ptr[row >> 5] + (p - prp[row]);
        return pv[(grp * NV + k) * kSell + (row & 31)];
    };
    const bool ok = warp_collect<HT>((int)a, prp, pcol, prp, pcol, keys, lane, INT_MIN);
    int* list = reinterpret_cast<int*>(sh_acc[warp]);  // 2 CAP values >= HT ints
    const int u = ok ? warp_compact<HT>(keys, list, lane) : HT + 1;
    if (u > CAP) {
        if (lane == 0) {
            count[a] = 0;
            atomicOr(ovf, 1);
        }
        return;
    }
    warp_rank<HT>(list, u, lane, tcol + a * CAP, keys, slot);
    for (int e = lane; e < CAP; e += 32) acc1[e] = acc2[e] = V(0);
    __syncwarp();
    const int pa0 = prp[a], pa1 = prp[a + 1];
    for (int pac = pa0 + lane; pac < pa1; pac += 32) {  // D terms: distinct columns
        const int e = slot[hs_find<HT>(keys, pcol[pac])];
        acc1[e] = pval((int)a, pac, 2 + 2 * DIM);
        acc2[e] = pval((int)a, pac, 3 + 2 * DIM);
    }
    __syncwarp();
    for (int pc0 = pa0; pc0 < pa1; pc0 += 32) {
        const int pab = pc0 + lane;
        int b = 0, bs = 0, len = 0;
        V cab[DIM], m1 = V(0), m2 = V(0);
#pragma unroll
        for (int k = 0; k < DIM; ++k) cab[k] = V(0);
        if (pab < pa1) {
            b = pcol[pab];
            bs = prp[b];
            len = prp[b + 1] - bs;
#pragma unroll
            for (int k = 0; k < DIM; ++k) cab[k] = pval((int)a, pab, 2 + DIM + k);
            m1 = mdiag[2 * b];
            m2 = mdiag[2 * b + 1];
        }
        int inc = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += y;
        }
        const int total = __shfl_sync(kFull, inc, 31);
        const int excl = inc - len;
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + lane;
            int j = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int ex = __shfl_sync(kFull, excl, j + step);
                if (ex <= t) j += step;
            }
            const int bj = __shfl_sync(kFull, b, j);
            const int pbc = __shfl_sync(kFull, bs, j) + (t - __shfl_sync(kFull, excl, j));
            V cj[DIM];
#pragma unroll
            for (int k = 0; k < DIM; ++k) cj[k] = __shfl_sync(kFull, cab[k], j);
            const V mj1 = __shfl_sync(kFull, m1, j), mj2 = __shfl_sync(kFull, m2, j);
            const bool act = t < total;
            int e = -1 - lane;
            V dot = V(0);
            if (act) {
#pragma unroll
                for (int k = 0; k < DIM; ++k) dot += cj[k] * pval(bj, pbc, 2 + k);
                e = slot[hs_find<HT>(keys, pcol[pbc])];
            }
            const unsigned peers = __match_any_sync(kFull, e);
            const int order = __popc(peers & ((1u << lane) - 1u));
            const int n_sub = (int)__reduce_max_sync(kFull, (unsigned)__popc(peers));
            for (int r = 0; r < n_sub; ++r) {
                if (act && order == r) {
                    acc1[e] -= dot * mj1;
                    acc2[e] -= dot * mj2;
                }
                __syncwarp();
            }
        }
    }
    __syncwarp();
    for (int e = lane; e < u; e += 32) {
        tv1[a * CAP + e] = acc1[e];
        tv2[a * CAP + e] = acc2[e];
    }
    if (lane == 0) count[a] = u;
}

// staging rows into blockdiag(S_p1, S_p2): rows a and n + a (columns + n)
template <int CAP, class V>
__global__ void k_selfp_compact(int64_t n, int64_t nnz_half, const int* __restrict__ rp,
                                const int* __restrict__ tcol, const V* __restrict__ tv1,
                                const V* __restrict__ tv2, int* __restrict__ srp,
                                int* __restrict__ scol, V* __restrict__ sval) {
    const int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (a > n) return;
    if (lane == 0) {
        srp[a] = rp[a];
        srp[n + a] = rp[a] + (int)nnz_half;
    }
    if (a == n) return;
    const int c0 = rp[a], u = rp[a + 1] - c0;
    for (int e = lane; e < u; e += 32) {
        const int c = tcol[a * CAP + e];
        scol[c0 + e] = c;
        scol[nnz_half + c0 + e] = c + (int)n;
        sval[c0 + e] = tv1[a * CAP + e];
        sval[nnz_half + c0 + e] = tv2[a * CAP + e];
    }
}

// block-diagonal duplication of the pattern: rows n..2n-1 get columns + n
__global__ void k_dup_pattern(int64_t n, int64_t nnz, int* __restrict__ rp, int* __restrict__ col) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nnz) col[nnz + i] = col[i] + (int)n;
    if (i <= n) rp[n + i] = rp[i] + (int)nnz;
}

// transpose: count, scatter, per-row sort. The count aggregates the lanes of
// a warp that hit the same column into one atomic (P's neighbouring rows share
// their aggregates, so columns repeat within a warp).
__global__ void k_col_count(const int* __restrict__ col, int64_t nnz, int* __restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = (i < nnz) ? col[i] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    const int lane = threadIdx.x & 31;
    if (c >= 0 && lane == __ffs(peers) - 1) atomicAdd(&cnt[c], __popc(peers));
}

template <class V>
__global__ void k_transpose_scatter(int64_t n_rows, const int* __restrict__ rp,
                                    const int* __restrict__ col, const V* __restrict__ val,
                                    int* __restrict__ cursor, int* __restrict__ tcol,
                                    V* __restrict__ tval) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rows) return;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
        int q = atomicAdd(&cursor[col[p]], 1);
        tcol[q] = (int)i;
        tval[q] = val[p];
    }
}

// warp per row: rank sort of (col, val) by col (distinct cols)
template <class V>
__global__ void k_sort_rows(int64_t n_rows, const int* __restrict__ rp, int* __restrict__ col,
                            V* __restrict__ val, int* __restrict__ tmpc,
                            V* __restrict__ tmpv) {
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

template <int HT>
void count_tier(const CsrView& A, const CsrView& B, int* count, int* ovf, const int* rows,
                int64_t n_work, int wpb, const int* is_long, int upper, cudaStream_t s) {
    const size_t smem = (size_t)wpb * HT * sizeof(int);
    set_smem(k_spgemm_count<HT>, smem);
    k_spgemm_count<HT><<<grid_for(n_work, wpb), wpb * 32, smem, s>>>(
        A.n_rows, A.rp, A.col, B.rp, B.col, count, ovf, rows, is_long, upper);
    DPP_LAUNCH_CK();
}

template <int HT>
void pattern_tier(const CsrView& A, const CsrView& B, Csr& C, const int* rows, int64_t n_work,
                  int wpb, int upper, cudaStream_t s) {
    const size_t smem = (size_t)wpb * 2 * HT * sizeof(int);
    set_smem(k_spgemm_pattern<HT>, smem);
    k_spgemm_pattern<HT><<<grid_for(n_work, wpb), wpb * 32, smem, s>>>(
        A.n_rows, A.rp, A.col, B.rp, B.col, C.row_ptr.get(), C.col.get(), rows, upper);
    DPP_LAUNCH_CK();
}

template <int CAP, class V>
void scatter_tier(const CsrView& A, const CsrView& B, Csr& C, int* wide, const int* is_long,
                  int upper, cudaStream_t s) {
    constexpr int HT = 2 * CAP < 64 ? 64 : 2 * CAP;
    const size_t smem = (size_t)kWarps * 2 * HT * sizeof(int) + (size_t)kWarps * CAP * sizeof(V);
    set_smem(k_spgemm_scatter<HT, CAP, V>, smem);
    k_spgemm_scatter<HT, CAP, V><<<grid_for(A.n_rows, kWarps), kWarps * 32, smem, s>>>(
        A.n_rows, A.rp, A.col, vals_of<V>(A), B.rp, B.col, vals_of<V>(B), C.row_ptr.get(), C.col.get(),
        vbuf<V>(C).get(), wide, is_long, upper);
    DPP_LAUNCH_CK();
}

constexpr int kHtTiers[3] = {256, 2048, 8192};

}  // namespace

namespace {
// Products of C = A B actually formed (B's row from b_row_start on), summed
// exactly in 64-bit integers: the FP64 multiply-adds of the product, for the
// profiling records.
__global__ void k_count_products(int64_t n, const int* __restrict__ arp, const int* __restrict__ acol,
                                 const int* __restrict__ brp, const int* __restrict__ bcol, int upper,
                                 unsigned long long* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c = 0;
    if (i < n)
        for (int p = arp[i]; p < arp[i + 1]; ++p) {
            const int k = acol[p];
            c += (unsigned long long)(brp[k + 1] - b_row_start(brp, bcol, k, upper ? (int)i : INT_MIN));
        }
    c = __reduce_add_sync(0xffffffffu, (unsigned)c) + 0ull;
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// Numeric product in one pass for rows of at most kOneCap columns (see
// k_spgemm_onepass); returns false when the staging rows would not fit the
// memory budget, and the caller takes the counting path.
constexpr int kOneCap = 128;

template <class V>
bool spgemm_onepass(const CsrView& A, const CsrView& B, Csr& C, int up, cudaStream_t s,
                    HostScratch& hs) {
    const int64_t n = A.n_rows;
    const int64_t stage = n * (int64_t)kOneCap;
    if (stage * (int64_t)(sizeof(int) + sizeof(V)) > (int64_t(4) << 30)) return false;
    C.n_rows = n;
    C.n_cols = B.n_cols;
    C.row_ptr.alloc(n + 1);
    DPP_CK(cudaMemsetAsync(C.row_ptr.get(), 0, (n + 1) * sizeof(int), s));
    DBuf<int> tcol(stage), uone(n), ovf(n + 2), ovf2(n + 2), last(2);
    DBuf<V> tval(stage);
    DPP_CK(cudaMemsetAsync(ovf.get(), 0, sizeof(int), s));
    DPP_CK(cudaMemsetAsync(ovf2.get(), 0, sizeof(int), s));
    DPP_CK(cudaMemsetAsync(last.get(), 0, sizeof(int), s));
    // The one-pass product is also timed as a kernel family of its own. Its
    // algorithmic bytes: A and B (values, columns, row pointers) read once, and
    // the rows of C written once (known after the launch).
    ProfScope po(sizeof(V) == 8 ? "spgemm_onepass" : "spgemm_onepass_fp32", s, 0);
    // the same launches with their algorithmic work (2 flops per product)
    ProfScope pw(sizeof(V) == 8 ? "spgemm_onepass_flop" : "spgemm_onepass_flop_fp32", s, 0);
    {
        ProfScope pf("spgemm_fill", s, 0);
        constexpr int HT = 2 * kOneCap;
        const size_t smem = (size_t)kWarps * 2 * HT * sizeof(int) +
                            (size_t)kWarps * onepass_acc_bytes<HT, kOneCap, V>();
        set_smem(k_spgemm_onepass<HT, kOneCap, V>, smem);
        k_spgemm_onepass<HT, kOneCap, V><<<grid_for(n, kWarps), kWarps * 32, smem, s>>>(
            n, A.rp, A.col, vals_of<V>(A), B.rp, B.col, vals_of<V>(B), C.row_ptr.get(), uone.get(),
            tcol.get(), tval.get(), ovf.get(), up);
        DPP_LAUNCH_CK();
    }
    po.end_range();
    pw.end_range();
    if (pw.fam) {  // timed: count the products (setup-time only, under profiling)
        DBuf<unsigned long long> prods(1);
        DPP_CK(cudaMemsetAsync(prods.get(), 0, sizeof(unsigned long long), s));
        k_count_products<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp, A.col, B.rp, B.col, up,
                                                          prods.get());
        DPP_LAUNCH_CK();
        pw.bytes = 2.0 * (double)read_scalar(prods.get(), s, hs);
    }
    pw.stop();
    const int64_t n_ovf = read_scalar(ovf.get(), s, hs);
    if (n_ovf > 0) {  // wider rows: counted in the larger tiers
        ProfScope pc("spgemm_count", s, 0);
        count_tier<2048>(A, B, C.row_ptr.get(), ovf2.get(), ovf.get() + 1, n_ovf, kWarps, nullptr, up, s);
        const int64_t n_ovf2 = read_scalar(ovf2.get(), s, hs);
        if (n_ovf2 > 0) {
            count_tier<8192>(A, B, C.row_ptr.get(), last.get(), ovf2.get() + 1, n_ovf2, 1, nullptr, up, s);
            if (read_scalar(last.get(), s, hs) > 0)
                fail(DPP_ERR_INVALID_ARGUMENT, "spgemm: a product row has more than 8191 distinct columns");
        }
    }
    C.nnz = exclusive_scan(C.row_ptr.get(), C.row_ptr.get(), n + 1, s, hs);
    po.bytes = (4.0 + sizeof(V)) * (double)(A.nnz + B.nnz + C.nnz) + 4.0 * (double)(A.n_rows + B.n_rows + 2) +
               4.0 * (double)n;
    po.stop();
    {
        ProfScope pa("spgemm_alloc", s, 0);
        C.col.alloc(std::max<int64_t>(C.nnz, 1));
        vbuf<V>(C).alloc(std::max<int64_t>(C.nnz, 1));
    }
    ProfScope pf("spgemm_fill", s, 0);
    k_onepass_compact<kOneCap, V><<<grid_for(n * 32, 256), 256, 0, s>>>(
        n, uone.get(), C.row_ptr.get(), tcol.get(), tval.get(), C.col.get(), vbuf<V>(C).get());
    DPP_LAUNCH_CK();
    if (n_ovf > 0) {  // one block per overflow row; rows wider than kLongCap: one warp each
        DBuf<int> wide(n_ovf + 2), st(1);
        DPP_CK(cudaMemsetAsync(wide.get(), 0, sizeof(int), s));
        DPP_CK(cudaMemsetAsync(st.get(), 0, sizeof(int), s));
        if (B.n_cols <= kLongBitCols) {
            const size_t smem_b = long_bm_smem<V>();
            set_smem(k_long_numeric_bm<V>, smem_b);
            k_long_numeric_bm<V><<<(unsigned)n_ovf, kLongWarps * 32, smem_b, s>>>(
                A.rp, A.col, vals_of<V>(A), B.rp, B.col, vals_of<V>(B), (int)((B.n_cols + 31) / 32),
                C.row_ptr.get(), C.col.get(), vbuf<V>(C).get(), ovf.get() + 1, wide.get(), st.get(), up);
        } else {
            const size_t smem_l = (size_t)(kLongHT + 2 * kLongCap) * sizeof(int) +
                                  (size_t)kLongWarps * kLongCap * sizeof(V);
            set_smem(k_long_numeric<V>, smem_l);
            k_long_numeric<V><<<(unsigned)n_ovf, kLongWarps * 32, smem_l, s>>>(
                A.rp, A.col, vals_of<V>(A), B.rp, B.col, vals_of<V>(B), C.row_ptr.get(), C.col.get(),
                vbuf<V>(C).get(), ovf.get() + 1, wide.get(), up);
        }
        DPP_LAUNCH_CK();
        const int n_wide = read_scalar(wide.get(), s, hs);
        if (n_wide > 0) {
            const size_t smem = (size_t)2 * 8192 * sizeof(int);
            set_smem(k_spgemm_wide<8192, V>, smem);
            k_spgemm_wide<8192, V><<<(unsigned)n_wide, 32, smem, s>>>(
                A.rp, A.col, vals_of<V>(A), B.rp, B.col, vals_of<V>(B), C.row_ptr.get(), C.col.get(),
                vbuf<V>(C).get(), wide.get() + 1, st.get(), up);
            DPP_LAUNCH_CK();
        }
        if (read_scalar(st.get(), s, hs))
            fail(DPP_ERR_INVALID_ARGUMENT,
                 "spgemm: a product row has more than 8191 distinct columns, or a column index "
                 "outside the operand's columns");
    }
    DPP_CK(cudaStreamSynchronize(s));
    return true;
}
}  // namespace

namespace {
template <class V>
void spgemm_t(const CsrView& A, const CsrView& B, Csr& C, bool values, cudaStream_t s,
              HostScratch& hs, bool upper_only) {
    const int up = upper_only ? 1 : 0;
    ProfScope prof(values ? "spgemm_numeric" : "spgemm_pattern", s, 0);
    if (A.n_cols != B.n_rows) fail(DPP_ERR_INVALID_ARGUMENT, "spgemm: shape mismatch");
    if (values && (!vals_of<V>(A) || !vals_of<V>(B)))
        fail(DPP_ERR_BAD_STATE, "spgemm: operands without values of the product's type");
    const int64_t n = A.n_rows;
    // many rows: one numeric pass, counting only the rows that overflow it
    if (values && n >= 16384 && spgemm_onepass<V>(A, B, C, up, s, hs)) return;
    C.n_rows = n;
    C.n_cols = B.n_cols;
    C.row_ptr.alloc(n + 1);
    DPP_CK(cudaMemsetAsync(C.row_ptr.get(), 0, (n + 1) * sizeof(int), s));
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
        count_tier<256>(A, B, C.row_ptr.get(), tier_rows[1] - 1, nullptr, n, kWarps, long_flag, up, s);
        tier_n[1] = read_scalar(tier_rows[1] - 1, s, hs);
        if (tier_n[1] > 0) {
            count_tier<2048>(A, B, C.row_ptr.get(), tier_rows[2] - 1, tier_rows[1], tier_n[1], kWarps,
                             long_flag, up, s);
            tier_n[2] = read_scalar(tier_rows[2] - 1, s, hs);
        }
        if (tier_n[2] > 0) {
            count_tier<8192>(A, B, C.row_ptr.get(), last_ovf.get(), tier_rows[2], tier_n[2], 1,
                             long_flag, up, s);
            if (read_scalar(last_ovf.get(), s, hs) > 0)
                fail(DPP_ERR_INVALID_ARGUMENT, "spgemm: a product row has more than 8191 distinct columns");
        }
        if (n_long > 0 && B.n_cols <= kLongBitCols) {
            DBuf<int> st(1);
            DPP_CK(cudaMemsetAsync(st.get(), 0, sizeof(int), s));
            k_long_count_bm<<<(unsigned)n_long, kLongWarps * 32, 0, s>>>(
                A.rp, A.col, B.rp, B.col, (int)((B.n_cols + 31) / 32), C.row_ptr.get(),
                long_rows.get() + 1, st.get(), up);
            DPP_LAUNCH_CK();
            if (read_scalar(st.get(), s, hs))
                fail(DPP_ERR_INVALID_ARGUMENT, "spgemm: a column index outside the operand's columns");
        } else if (n_long > 0) {
            DBuf<int> st(1);
            DPP_CK(cudaMemsetAsync(st.get(), 0, sizeof(int), s));
            const size_t smem = (size_t)kLongHT * sizeof(int);
            set_smem(k_long_count, smem);
            k_long_count<<<(unsigned)n_long, kLongWarps * 32, smem, s>>>(
                A.rp, A.col, B.rp, B.col, C.row_ptr.get(), long_rows.get() + 1, st.get(), up);
            DPP_LAUNCH_CK();
            if (read_scalar(st.get(), s, hs))
                fail(DPP_ERR_INVALID_ARGUMENT, "spgemm: a product row has more than 8191 distinct columns");
        }
    }
    C.nnz = exclusive_scan(C.row_ptr.get(), C.row_ptr.get(), n + 1, s, hs);
    {
        ProfScope pa("spgemm_alloc", s, 0);
        C.col.alloc(std::max<int64_t>(C.nnz, 1));
        if (values) vbuf<V>(C).alloc(std::max<int64_t>(C.nnz, 1));
    }
    ProfScope pf(values ? "spgemm_fill" : "spgemm_fill_pattern", s, 0);
    if (!values) {
        pattern_tier<256>(A, B, C, nullptr, n, kWarps, up, s);  // rows that fit the first tier
        if (tier_n[1] > 0) pattern_tier<2048>(A, B, C, tier_rows[1], tier_n[1], kWarps, up, s);
        if (tier_n[2] > 0) pattern_tier<8192>(A, B, C, tier_rows[2], tier_n[2], 1, up, s);
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
    if (n_long > 0 && B.n_cols <= kLongBitCols) {
        const size_t smem = long_bm_smem<V>();
        set_smem(k_long_numeric_bm<V>, smem);
        k_long_numeric_bm<V><<<(unsigned)n_long, kLongWarps * 32, smem, s>>>(
            A.rp, A.col, vals_of<V>(A), B.rp, B.col, vals_of<V>(B), (int)((B.n_cols + 31) / 32),
            C.row_ptr.get(), C.col.get(), vbuf<V>(C).get(), long_rows.get() + 1, wide.get(), st.get(), up);
        DPP_LAUNCH_CK();
    } else if (n_long > 0) {
        const size_t smem = (size_t)(kLongHT + 2 * kLongCap) * sizeof(int) +
                            (size_t)kLongWarps * kLongCap * sizeof(V);
        set_smem(k_long_numeric<V>, smem);
        k_long_numeric<V><<<(unsigned)n_long, kLongWarps * 32, smem, s>>>(
            A.rp, A.col, vals_of<V>(A), B.rp, B.col, vals_of<V>(B), C.row_ptr.get(), C.col.get(),
            vbuf<V>(C).get(), long_rows.get() + 1, wide.get(), up);
        DPP_LAUNCH_CK();
    }
    if (n_long < n) {
        if (max_u <= 32) scatter_tier<32, V>(A, B, C, wide.get(), long_flag, up, s);
        else if (max_u <= 64) scatter_tier<64, V>(A, B, C, wide.get(), long_flag, up, s);
        else if (max_u <= 128) scatter_tier<128, V>(A, B, C, wide.get(), long_flag, up, s);
        else if (max_u <= 256) scatter_tier<256, V>(A, B, C, wide.get(), long_flag, up, s);
        else if (max_u <= 512) scatter_tier<512, V>(A, B, C, wide.get(), long_flag, up, s);
        else scatter_tier<1024, V>(A, B, C, wide.get(), long_flag, up, s);
    }
    const int n_wide = read_scalar(wide.get(), s, hs);
    if (n_wide > 0) {
        const size_t smem = (size_t)2 * 8192 * sizeof(int);
        set_smem(k_spgemm_wide<8192, V>, smem);
        k_spgemm_wide<8192, V><<<n_wide, 32, smem, s>>>(A.rp, A.col, vals_of<V>(A), B.rp, B.col,
                                                        vals_of<V>(B), C.row_ptr.get(), C.col.get(),
                                                        vbuf<V>(C).get(), wide.get() + 1, st.get(), up);
        DPP_LAUNCH_CK();
    }
    if (n_long > 0 || n_wide > 0) {
        if (read_scalar(st.get(), s, hs))
            fail(DPP_ERR_INVALID_ARGUMENT,
                 "spgemm: a product row has more than 8191 distinct columns, or a column index "
                 "outside the operand's columns");
    }
    DPP_CK(cudaStreamSynchronize(s));
}
}  // namespace

void spgemm(const CsrView& A, const CsrView& B, Csr& C, bool values, cudaStream_t s,
            HostScratch& hs, bool upper_only) {
    if (values && !A.val && A.val32) spgemm_t<float>(A, B, C, values, s, hs, upper_only);
    else spgemm_t<double>(A, B, C, values, s, hs, upper_only);
}

namespace {
template <class V>
void transpose_t(const Csr& A, Csr& T, cudaStream_t s, HostScratch& hs) {
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
    vbuf<V>(T).alloc(std::max<int64_t>(A.nnz, 1));
    DBuf<int> cursor(T.n_rows + 1);
    DPP_CK(cudaMemcpyAsync(cursor.get(), T.row_ptr.get(), (T.n_rows + 1) * sizeof(int),
                           cudaMemcpyDeviceToDevice, s));
    k_transpose_scatter<V><<<grid_for(A.n_rows, B), B, 0, s>>>(A.n_rows, A.row_ptr.get(), A.col.get(),
                                                               vbuf<V>(A).get(), cursor.get(), T.col.get(),
                                                               vbuf<V>(T).get());
    DPP_LAUNCH_CK();
    DBuf<int> tc(std::max<int64_t>(A.nnz, 1));
    DBuf<V> tv(std::max<int64_t>(A.nnz, 1));
    k_sort_rows<V><<<grid_for(T.n_rows * 32, B), B, 0, s>>>(T.n_rows, T.row_ptr.get(), T.col.get(),
                                                            vbuf<V>(T).get(), tc.get(), tv.get());
    DPP_LAUNCH_CK();
    DPP_CK(cudaStreamSynchronize(s));
}
}  // namespace

// The FP64 values are transposed when A has them, else the FP32 ones.
void transpose(const Csr& A, Csr& T, cudaStream_t s, HostScratch& hs) {
    if (fp32_only(A)) transpose_t<float>(A, T, s, hs);
    else transpose_t<double>(A, T, s, hs);
}

namespace {
// rows of C = U + strict_upper(U)^T: T = U^T (sorted rows, column <= row),
// count[i] = |T row i without the diagonal| + |U row i|
__global__ void k_sym_count(int64_t n, const int* __restrict__ urp, const int* __restrict__ trp,
                            const int* __restrict__ tcol, int* __restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lt = trp[i + 1] - trp[i];
    if (lt > 0 && tcol[trp[i + 1] - 1] == (int)i) --lt;  // the diagonal comes from U
    count[i] = lt + (urp[i + 1] - urp[i]);
}

// one warp per row: the strictly lower part from T, then U's row (both sorted)
template <class V>
__global__ void k_sym_fill(int64_t n, const int* __restrict__ urp, const int* __restrict__ ucol,
                           const V* __restrict__ uval, const int* __restrict__ trp,
                           const int* __restrict__ tcol, const V* __restrict__ tval,
                           const int* __restrict__ crp, int* __restrict__ ccol,
                           V* __restrict__ cval) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int c0 = crp[i];
    const int nl = crp[i + 1] - c0 - (urp[i + 1] - urp[i]);
    for (int e = lane; e < nl; e += 32) {
        ccol[c0 + e] = tcol[trp[i] + e];
        cval[c0 + e] = tval[trp[i] + e];
    }
    for (int e = lane; e < urp[i + 1] - urp[i]; e += 32) {
        ccol[c0 + nl + e] = ucol[urp[i] + e];
        cval[c0 + nl + e] = uval[urp[i] + e];
    }
}

// one warp per checked row (every stride-th row): flag entries whose mirror
// is missing or differs
template <class V>
__global__ void k_sym_check(int64_t n, int stride, const int* __restrict__ rp, const int* __restrict__ col,
                            const V* __restrict__ val, double tol, int* __restrict__ bad) {
    const int64_t i = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * stride;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    bool ok = true;
    for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) {
        const int j = col[p];
        const int q = bsearch_row(col, rp[j], rp[j + 1], (int)i);
        if (q < 0) { ok = false; continue; }
        const double a = val[p], b = val[q];
        if (!(fabs(a - b) <= tol * (fabs(a) + fabs(b)))) ok = false;
    }
    if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicOr(bad, 1);
}
}  // namespace

namespace {
template <class V>
void symmetrize_upper_t(const Csr& U, Csr& C, cudaStream_t s, HostScratch& hs) {
    Csr T;
    transpose(U, T, s, hs);
    const int64_t n = U.n_rows;
    C.n_rows = C.n_cols = n;
    C.row_ptr.alloc(n + 1);
    DPP_CK(cudaMemsetAsync(C.row_ptr.get(), 0, (n + 1) * sizeof(int), s));
    k_sym_count<<<grid_for(n, 256), 256, 0, s>>>(n, U.row_ptr.get(), T.row_ptr.get(), T.col.get(),
                                                 C.row_ptr.get());
    DPP_LAUNCH_CK();
    C.nnz = exclusive_scan(C.row_ptr.get(), C.row_ptr.get(), n + 1, s, hs);
    C.col.alloc(std::max<int64_t>(C.nnz, 1));
    vbuf<V>(C).alloc(std::max<int64_t>(C.nnz, 1));
    k_sym_fill<V><<<grid_for(n * 32, 256), 256, 0, s>>>(n, U.row_ptr.get(), U.col.get(), vbuf<V>(U).get(),
                                                        T.row_ptr.get(), T.col.get(), vbuf<V>(T).get(),
                                                        C.row_ptr.get(), C.col.get(), vbuf<V>(C).get());
    DPP_LAUNCH_CK();
    DPP_CK(cudaStreamSynchronize(s));
}
}  // namespace

void symmetrize_upper(const Csr& U, Csr& C, cudaStream_t s, HostScratch& hs) {
    if (fp32_only(U)) symmetrize_upper_t<float>(U, C, s, hs);
    else symmetrize_upper_t<double>(U, C, s, hs);
}

bool is_symmetric(const Csr& A, double tol, int stride, cudaStream_t s, HostScratch& hs) {
    if (A.n_rows != A.n_cols) return false;
    DBuf<int> bad(1);
    DPP_CK(cudaMemsetAsync(bad.get(), 0, sizeof(int), s));
    const int64_t rows = (A.n_rows + stride - 1) / stride;
    const int g = grid_for(rows * 32, 256);
    if (fp32_only(A))
        k_sym_check<float><<<g, 256, 0, s>>>(A.n_rows, stride, A.row_ptr.get(), A.col.get(),
                                             A.val32.get(), tol, bad.get());
    else
        k_sym_check<double><<<g, 256, 0, s>>>(A.n_rows, stride, A.row_ptr.get(), A.col.get(),
                                              A.val.get(), tol, bad.get());
    DPP_LAUNCH_CK();
    return read_scalar(bad.get(), s, hs) == 0;
}

namespace {
// one-pass S_p when every row fits kSelfpOneCap columns; false = not built
template <class V> const V* pair_vals(const ProblemImpl& P);
template <> const double* pair_vals<double>(const ProblemImpl& P) { return P.sell_val.get(); }
template <> const float* pair_vals<float>(const ProblemImpl& P) { return P.sell_val32.get(); }

template <int DIM, int CAP, class V>
bool selfp_onepass(const ProblemImpl& P, const V* mdiag, Csr& S, cudaStream_t s,
                   HostScratch& hs) {
    const int64_t n = P.n_nodes;
    DBuf<int> cnt(n + 1), tcol(n * CAP), ovf(1);
    DBuf<V> tv1(n * CAP), tv2(n * CAP);
    DPP_CK(cudaMemsetAsync(cnt.get(), 0, (n + 1) * sizeof(int), s));
    DPP_CK(cudaMemsetAsync(ovf.get(), 0, sizeof(int), s));
    k_selfp_onepass<DIM, CAP, V><<<grid_for(n, 4), 128, 0, s>>>(
        n, P.row_ptr.get(), P.col.get(), P.slice_ptr.get(), pair_vals<V>(P), mdiag, cnt.get(),
        tcol.get(), tv1.get(), tv2.get(), ovf.get());
    DPP_LAUNCH_CK();
    if (read_scalar(ovf.get(), s, hs)) return false;
    const int64_t nnz = exclusive_scan(cnt.get(), cnt.get(), n + 1, s, hs);
    S.n_rows = S.n_cols = 2 * n;
    S.nnz = 2 * nnz;
    S.row_ptr.alloc(2 * n + 1);
    S.col.alloc(std::max<int64_t>(2 * nnz, 1));
    vbuf<V>(S).alloc(std::max<int64_t>(2 * nnz, 1));
    k_selfp_compact<CAP, V><<<grid_for((n + 1) * 32, 256), 256, 0, s>>>(
        n, nnz, cnt.get(), tcol.get(), tv1.get(), tv2.get(), S.row_ptr.get(), S.col.get(),
        vbuf<V>(S).get());
    DPP_LAUNCH_CK();
    DPP_CK(cudaStreamSynchronize(s));
    return true;
}
template <class V>
void build_selfp_t(const ProblemImpl& P, const V* mdiag, Csr& S, cudaStream_t s, HostScratch& hs) {
    if (!pair_vals<V>(P)) fail(DPP_ERR_BAD_STATE, "selfp: pair values of this precision were not assembled");
    if (P.dim == 3 ? selfp_onepass<3, 128, V>(P, mdiag, S, s, hs) : selfp_onepass<2, 64, V>(P, mdiag, S, s, hs))
        return;
    // two passes: pattern of G*G with G the pair graph (self pairs included), then values
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
    vbuf<V>(S).alloc(2 * nnz);
    DPP_CK(cudaMemcpyAsync(S.row_ptr.get(), Sh.row_ptr.get(), (n + 1) * sizeof(int),
                           cudaMemcpyDeviceToDevice, s));
    DPP_CK(cudaMemcpyAsync(S.col.get(), Sh.col.get(), nnz * sizeof(int), cudaMemcpyDeviceToDevice, s));
    const int B = 256;
    k_dup_pattern<<<grid_for(std::max<int64_t>(nnz, n + 1), B), B, 0, s>>>(n, nnz, S.row_ptr.get(),
                                                                           S.col.get());
    DPP_LAUNCH_CK();
    constexpr int kSelfpCap = 128;
    DBuf<int> wide(n + 1);
    DPP_CK(cudaMemsetAsync(wide.get(), 0, sizeof(int), s));
    if (P.dim == 2)
        k_selfp_scatter<2, kSelfpCap, V><<<grid_for(n, 4), 128, 0, s>>>(
            n, P.row_ptr.get(), P.col.get(), P.slice_ptr.get(), pair_vals<V>(P), mdiag,
            Sh.row_ptr.get(), Sh.col.get(), vbuf<V>(S).get(), nnz, wide.get());
    else
        k_selfp_scatter<3, kSelfpCap, V><<<grid_for(n, 4), 128, 0, s>>>(
            n, P.row_ptr.get(), P.col.get(), P.slice_ptr.get(), pair_vals<V>(P), mdiag,
            Sh.row_ptr.get(), Sh.col.get(), vbuf<V>(S).get(), nnz, wide.get());
    DPP_LAUNCH_CK();
    const int n_wide = read_scalar(wide.get(), s, hs);
    if (n_wide > 0) {
        if (P.dim == 2)
            k_selfp_values<2, V><<<grid_for((int64_t)n_wide * 32, B), B, 0, s>>>(
                wide.get() + 1, P.row_ptr.get(), P.col.get(), P.slice_ptr.get(), pair_vals<V>(P),
                mdiag, Sh.row_ptr.get(), Sh.col.get(), vbuf<V>(S).get(), nnz);
        else
            k_selfp_values<3, V><<<grid_for((int64_t)n_wide * 32, B), B, 0, s>>>(
                wide.get() + 1, P.row_ptr.get(), P.col.get(), P.slice_ptr.get(), pair_vals<V>(P),
                mdiag, Sh.row_ptr.get(), Sh.col.get(), vbuf<V>(S).get(), nnz);
        DPP_LAUNCH_CK();
    }
    DPP_CK(cudaStreamSynchronize(s));
}
}  // namespace

void build_selfp(const ProblemImpl& P, const double* mdiag, Csr& S, cudaStream_t s,
                 HostScratch& hs) {
    build_selfp_t<double>(P, mdiag, S, s, hs);
}

void build_selfp(const ProblemImpl& P, const float* mdiag, Csr& S, cudaStream_t s,
                 HostScratch& hs) {
    build_selfp_t<float>(P, mdiag, S, s, hs);
}

}  // namespace dpp
