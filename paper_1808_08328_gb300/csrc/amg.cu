// Smoothed-aggregation AMG on blockdiag(S_p1, S_p2) with Chebyshev-Jacobi
// smoothing. It plays the role the paper gives to one BoomerAMG V-cycle per
// Schur block (Section 4.2, Method 2, "fieldsplit_1" of its appendix
// options).
//
// Setup per level (Vanek, Mandel & Brezina, Computing 56, 1996, for the
// aggregation and prolongator smoothing; Bell, Dalton & Olson, SIAM J. Sci.
// Comput. 34(4), 2012, for the parallel distance-2 independent-set
// aggregation):
//   1. symmetric strength: j is a strong neighbour of i if
//      |a_ij| >= theta sqrt(|a_ii a_jj|);
//   2. a distance-2 maximal independent set of the strength graph. Ties are
//      broken by a fixed integer hash of the row id, so the result is
//      deterministic. Each root plus its strong neighbours forms an
//      aggregate; the remaining rows join the aggregate of a strong
//      neighbour;
//   3. tentative prolongator P0 = aggregate indicator; smoothed prolongator
//      P = (I - omega D^-1 A) P0 with omega = 4 / (3 lambda_max(D^-1 A));
//   4. Galerkin coarse matrix A_c = P^T (A P).
// lambda_max comes from 12 power iterations on D^-1 A. Coarsening stops at
// coarse_max_rows rows, or earlier when a level consists of small diagonal
// blocks only (a batched union of instances). The coarsest matrix is inverted
// block by block (its contiguous diagonal blocks, Gauss-Jordan without
// pivoting, valid for SPD) and applied as block matrix-vector products.
//
// Smoother: Chebyshev polynomial in D^-1 A on [lambda_max / ratio,
// 1.1 lambda_max] (Adams, Brezina, Hu & Tuminaro, J. Comput. Phys. 188,
// 2003).
#include "amg.cuh"
#include "level_spmv.cuh"
#include "csr_spmv.cuh"

#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

namespace dpp {

namespace {

// smallest column of each slice (base[s]) and a flag if any slice's columns
// span 65536 or more; one warp per slice. A lane reads only its own row's
// slots (k * 32 + lane): the slots of rows past n_rows in the last slice are
// never written.
__global__ void k_sell_span(int64_t n_rows, int64_t n_sl, const int* __restrict__ off,
                            const int* __restrict__ scol, int* __restrict__ base, int* __restrict__ wide) {
    const int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (sl >= n_sl) return;
    int lo = INT_MAX, hi = INT_MIN;
    if (sl * 32 + lane < n_rows)
        for (int q = off[sl] + lane; q < off[sl + 1]; q += 32) {
            lo = min(lo, scol[q]);
            hi = max(hi, scol[q]);
        }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) {
        base[sl] = (lo == INT_MAX) ? 0 : lo;
        if (lo != INT_MAX && (int64_t)hi - (int64_t)lo > 65535) atomicOr(wide, 1);
    }
}

// 16-bit columns relative to the slice base; the never-read slots of rows
// past n_rows are set to 0
__global__ void k_sell_col16(int64_t n_rows, int64_t n_sl, const int* __restrict__ off,
                             const int* __restrict__ scol, const int* __restrict__ base,
                             uint16_t* __restrict__ c16) {
    const int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (sl >= n_sl) return;
    const bool live = sl * 32 + lane < n_rows;
    const int b = base[sl];
    for (int q = off[sl] + lane; q < off[sl + 1]; q += 32) c16[q] = live ? (uint16_t)(scol[q] - b) : 0;
}

// slice widths: w[s] = 32 * (longest row of slice s); one warp per slice
__global__ void k_sell_width(int64_t n_rows, const int* __restrict__ rp, int* __restrict__ w) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t sl = t >> 5;
    const int64_t row = t;
    const int64_t n_sl = (n_rows + 31) / 32;
    int len = (row < n_rows) ? rp[row + 1] - rp[row] : 0;
    len = __reduce_max_sync(0xffffffffu, len);
    if ((t & 31) == 0 && sl < n_sl) w[sl] = 32 * len;
    if (t == 0) w[n_sl] = 0;
}

template <class T>
__global__ void k_sell_fill(int64_t n_rows, const int* __restrict__ rp, const int* __restrict__ col,
                            const T* __restrict__ val, const int* __restrict__ off,
                            int* __restrict__ scol, T* __restrict__ sval) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n_rows) return;
    const int64_t sl = row >> 5;
    const int lane = (int)(row & 31);
    const int r0 = rp[row], len = rp[row + 1] - r0;
    const int width = (off[sl + 1] - off[sl]) / 32;
    // padding: (the row's last column, 0.0), a valid column also for a
    // rectangular matrix (P), already loaded for this row
    const int pad = (len > 0) ? col[r0 + len - 1] : 0;
    for (int k = 0; k < width; ++k) {
        const int64_t q = (int64_t)off[sl] + (int64_t)k * 32 + lane;
        scol[q] = (k < len) ? col[r0 + k] : pad;
        sval[q] = (k < len) ? val[r0 + k] : T(0);
    }
}

template <class T> const T* vals(const Csr& A);
template <> const double* vals<double>(const Csr& A) { return A.val.get(); }
template <> const float* vals<float>(const Csr& A) { return A.val32.get(); }

template <int MODE, class T>
void spmv_lanes(int lanes, const Csr& A, const T* x, const T* b, T* y, cudaStream_t s,
                const char* family = nullptr, ChebOut<T> ch = ChebOut<T>()) {
    const bool sell = lanes == 0 && A.has_sell() &&
                      (sizeof(T) == 8 ? A.sell_val.get() != nullptr : A.sell_val32.get() != nullptr);
    // algorithmic bytes: values and column indices of the nonzeros, the row
    // pointers (CSR only), x once, y (and b) once; SELL padding is not counted
    // (MODE 3 moves b, Dinv, d, and writes d and the new x: 5 values per row)
    const bool c16 = sell && sizeof(T) == 4 && A.sell_col16.get();
    const double alg = (double)A.nnz * (sizeof(T) + (c16 ? 2.0 : 4.0)) +
                       (sell ? (c16 ? (double)((A.n_rows + 31) / 32) * 4.0 : 0.0) : (double)(A.n_rows + 1) * 4.0) +
                       (double)A.n_cols * sizeof(T) +
                       (double)A.n_rows * sizeof(T) * (MODE == 0 ? 1 : MODE == 3 ? 5 : 2);
    ProfScope prof(family ? family : (sizeof(T) == 8 ? "amg_spmv_setup" : "amg_spmv_setup_fp32"), s, alg);
    const int B = 256;
    if (sell) {
        const T* sv = (sizeof(T) == 8) ? reinterpret_cast<const T*>(A.sell_val.get())
                                       : reinterpret_cast<const T*>(A.sell_val32.get());
        // two warps per slice in FP32 (latency-limited at one thread per row),
        // one in FP64 (the FP64 pipe is the limit there)
        constexpr int H = sizeof(T) == 4 ? 2 : 1;
        const int64_t n_sl = (A.n_rows + 31) / 32;
        bool done = false;
        if constexpr (sizeof(T) == 4) {
            if (A.sell_col16.get()) {
                k_sell_spmv<MODE, T, H, true><<<grid_for(n_sl, 8 / H), B, 0, s>>>(
                    A.n_rows, A.sell_off.get(), nullptr, sv, x, b, y, ch, A.sell_base.get(), A.sell_col16.get());
                done = true;
            }
        }
        if (!done)
            k_sell_spmv<MODE, T, H><<<grid_for(n_sl, 8 / H), B, 0, s>>>(A.n_rows, A.sell_off.get(),
                                                                       A.sell_col.get(), sv, x, b, y, ch);
        DPP_LAUNCH_CK();
        return;
    }
    if (lanes < 1) lanes = 2;  // SELL requested but not built
    const int64_t thr = A.n_rows * lanes;
    const int g = grid_for(thr, B);
    const int* rp = A.row_ptr.get();
    const int* cl = A.col.get();
    const T* v = vals<T>(A);
    switch (lanes) {
        case 1: k_csr_spmv<1, MODE, T><<<g, B, 0, s>>>(A.n_rows, rp, cl, v, x, b, y, ch); break;
        case 2: k_csr_spmv<2, MODE, T><<<g, B, 0, s>>>(A.n_rows, rp, cl, v, x, b, y, ch); break;
        case 4: k_csr_spmv<4, MODE, T><<<g, B, 0, s>>>(A.n_rows, rp, cl, v, x, b, y, ch); break;
        case 8: k_csr_spmv<8, MODE, T><<<g, B, 0, s>>>(A.n_rows, rp, cl, v, x, b, y, ch); break;
        case 16: k_csr_spmv<16, MODE, T><<<g, B, 0, s>>>(A.n_rows, rp, cl, v, x, b, y, ch); break;
        default: k_csr_spmv<32, MODE, T><<<g, B, 0, s>>>(A.n_rows, rp, cl, v, x, b, y, ch); break;
    }
    DPP_LAUNCH_CK();
}

// Lanes per row from the mean row length and the row count: enough entries per
// lane to keep loads in flight, and enough rows x lanes to fill the GPU.
int pick_lanes(const Csr& A) {
    const double avg = A.n_rows ? (double)A.nnz / (double)A.n_rows : 1.0;
    const double want = std::max(avg / 16.0, 150000.0 / std::max<double>((double)A.n_rows, 1.0));
    int l = 2;
    while (l < 32 && l < want) l <<= 1;
    return l;
}

// SELL-32 copy of a level matrix (the matrix's own values: FP64, to which
// amg_make_fp32 adds FP32 ones, or FP32 for a matrix of the FP32 hierarchy),
// built for matrices with at least opts.sell_min_rows rows (default 65536)
// unless opts.spmv_format asks for CSR only; offsets must fit int32.
int64_t sell_min_rows(const dpp_pc_opts& o) { return o.sell_min_rows > 0 ? o.sell_min_rows : 65536; }

void build_sell(Csr& A, cudaStream_t s, HostScratch& hs) {
    const int64_t n = A.n_rows, n_sl = (n + 31) / 32;
    DBuf<int> off(n_sl + 1);
    k_sell_width<<<grid_for(n_sl * 32, 256), 256, 0, s>>>(n, A.row_ptr.get(), off.get());
    DPP_LAUNCH_CK();
    const int64_t tot = exclusive_scan(off.get(), off.get(), n_sl + 1, s, hs);
    if (tot <= 0 || tot >= INT32_MAX) return;  // keep CSR only
    A.sell_col.alloc(tot);
    if (fp32_only(A)) {  // a matrix of the FP32 hierarchy: FP32 values, 16-bit columns if they fit
        A.sell_val32.alloc(tot);
        k_sell_fill<float><<<grid_for(n, 256), 256, 0, s>>>(n, A.row_ptr.get(), A.col.get(), A.val32.get(),
                                                           off.get(), A.sell_col.get(), A.sell_val32.get());
        DPP_LAUNCH_CK();
        DBuf<int> base(n_sl), wide(1);
        DPP_CK(cudaMemsetAsync(wide.get(), 0, sizeof(int), s));
        k_sell_span<<<grid_for(n_sl * 32, 256), 256, 0, s>>>(n, n_sl, off.get(), A.sell_col.get(), base.get(),
                                                            wide.get());
        DPP_LAUNCH_CK();
        if (read_scalar(wide.get(), s, hs) == 0) {
            A.sell_col16.alloc(tot);
            k_sell_col16<<<grid_for(n_sl * 32, 256), 256, 0, s>>>(n, n_sl, off.get(), A.sell_col.get(),
                                                                 base.get(), A.sell_col16.get());
            DPP_LAUNCH_CK();
            A.sell_base = std::move(base);
        }
    } else {
        A.sell_val.alloc(tot);
        k_sell_fill<double><<<grid_for(n, 256), 256, 0, s>>>(n, A.row_ptr.get(), A.col.get(), A.val.get(),
                                                            off.get(), A.sell_col.get(), A.sell_val.get());
    }
    DPP_LAUNCH_CK();
    A.sell_off = std::move(off);
}

// ------------------------------------------------------------------ vectors
template <class V>
__global__ void k_diag_inv(int64_t n, const int* __restrict__ rp, const int* __restrict__ col,
                           const V* __restrict__ val, V* __restrict__ dinv,
                           V* __restrict__ dabs, int* status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    V d = V(0);
    for (int p = rp[i]; p < rp[i + 1]; ++p)
        if (col[p] == i) d = val[p];
    if (!(d > V(0)) || !isfinite(d)) atomicOr(status, kDevDegenerate);
    dinv[i] = V(1) / d;
    if (dabs) dabs[i] = fabs(d);
}

// First Chebyshev step from a zero start: d = c2 Dinv b, x = d (the later steps
// are fused into the residual SpMV, MODE 3)
template <class T>
__global__ void k_cheb_start(int64_t n, const T* __restrict__ dinv, const T* __restrict__ b,
                             T* __restrict__ d, T* __restrict__ x, T c2) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const T v = c2 * dinv[i] * b[i];
        d[i] = v;
        x[i] = v;
    }
}

__global__ void k_d2f(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = (float)in[i];
}

__global__ void k_fill_int(int64_t n, int v, int* __restrict__ x) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

// y = x / sqrt(*nrm2)
template <class V>
__global__ void k_scale_rsqrt(int64_t n, const V* __restrict__ x, V* __restrict__ y,
                              const double* __restrict__ nrm2) {
    const V a = (V)(1.0 / sqrt(*nrm2));
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        y[i] = a * x[i];
}

__global__ void k_f2d(int64_t n, const float* __restrict__ in, double* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = (double)in[i];
}

template <class V>
__global__ void k_dinv_scale(int64_t n, const V* __restrict__ dinv, V* __restrict__ v) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        v[i] *= dinv[i];
}

__device__ __forceinline__ uint32_t mix32(uint32_t x) {  // murmur3 finaliser
    x ^= x >> 16;
    x *= 0x85ebca6bu;
    x ^= x >> 13;
    x *= 0xc2b2ae35u;
    x ^= x >> 16;
    return x;
}

template <class V>
__global__ void k_hash_vector(int64_t n, V* __restrict__ v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (V)(0.5 + (double)(mix32((uint32_t)i * 2654435761u + 12345u) >> 8) / 16777216.0);
}

// ------------------------------------------------------------------ aggregation
// Strength of connection, one warp per row: j != i is a strong neighbour of i
// when |a_ij| >= theta sqrt(|a_ii| |a_jj|), tested as a_ij^2 >= theta^2 |a_ii| |a_jj|
// (no FP64 square root, which is slow on this GPU's FP64 pipe). Ballots keep
// the row's column order.
template <class V>
__device__ __forceinline__ bool is_strong(int64_t i, int j, V aij, V di, const V* __restrict__ dabs,
                                          V theta2) {
    return j != i && aij * aij >= theta2 * (di * dabs[j]);
}

// One pass: the strong columns of row i go to tmp[rp[i] ...] (the row's own
// range in A) and their number to cnt[i]; k_strength_compact then packs them.
template <class V>
__global__ void k_strength_stage(int64_t n, const int* __restrict__ rp, const int* __restrict__ col,
                                 const V* __restrict__ val, const V* __restrict__ dabs,
                                 V theta2, int* __restrict__ cnt, int* __restrict__ tmp) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const V di = dabs[i];
    const int p1 = rp[i + 1];
    int q = rp[i];
    for (int p0 = rp[i]; p0 < p1; p0 += 32) {
        const int p = p0 + lane;
        const int j = p < p1 ? col[p] : -1;
        const bool st = p < p1 && is_strong(i, j, val[p], di, dabs, theta2);
        const unsigned m = __ballot_sync(0xffffffffu, st);
        if (st) tmp[q + __popc(m & ((1u << lane) - 1u))] = j;
        q += __popc(m);
    }
    if (lane == 0) cnt[i] = q - rp[i];
}

__global__ void k_strength_compact(int64_t n, const int* __restrict__ rp, const int* __restrict__ tmp,
                                   const int* __restrict__ srp, int* __restrict__ scol) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int c = srp[i + 1] - srp[i];
    for (int e = lane; e < c; e += 32) scol[srp[i] + e] = tmp[rp[i] + e];
}


enum : int { kOut = 0, kUnd = 1, kIn = 2 };

__device__ __forceinline__ uint64_t mis_key(int state, int64_t i) {
    return ((uint64_t)state << 62) | ((uint64_t)mix32((uint32_t)i) << 30) | (uint64_t)(i & 0x3fffffff);
}

__global__ void k_mis_t0(int64_t n, const int* __restrict__ state, uint64_t* __restrict__ t0) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) t0[i] = mis_key(state[i], i);
}

// tout[i] = max of tin over i and its strong neighbours; kMisLanes lanes per row
constexpr int kMisLanes = 8;
__global__ void k_mis_max(int64_t n, const int* __restrict__ srp, const int* __restrict__ scol,
                          const uint64_t* __restrict__ tin, uint64_t* __restrict__ tout) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = t / kMisLanes;
    const int sub = (int)(t % kMisLanes);
    const bool valid = i < n;  // every lane stays for the shuffles below
    uint64_t m = 0;
    if (valid) {
        if (sub == 0) m = tin[i];
        for (int p = srp[i] + sub; p < srp[i + 1]; p += kMisLanes) m = max(m, tin[scol[p]]);
    }
#pragma unroll
    for (int o = kMisLanes / 2; o > 0; o >>= 1) {
        const uint64_t y = __shfl_xor_sync(0xffffffffu, m, o, kMisLanes);
        m = max(m, y);
    }
    if (valid && sub == 0) tout[i] = m;
}

// decide the undecided rows, and write the next round's keys (t0_next) for all
__global__ void k_mis_update(int64_t n, int* __restrict__ state, const uint64_t* __restrict__ t0,
                             const uint64_t* __restrict__ t2, uint64_t* __restrict__ t0_next,
                             int* __restrict__ undecided) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int st = state[i];
    if (st == kUnd) {
        if (t2[i] == t0[i]) st = kIn;
        else if ((int)(t2[i] >> 62) == kIn) st = kOut;
        else atomicAdd(undecided, 1);
        state[i] = st;
    }
    t0_next[i] = mis_key(st, i);
}

// flag[0..n) = root indicator, flag[n] = 0 (the scan below runs over n + 1 entries)
__global__ void k_root_flags(int64_t n, const int* __restrict__ state, int* __restrict__ flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (state[i] == kIn) ? 1 : 0;
    if (i == n) flag[n] = 0;
}

__global__ void k_agg_pass1(int64_t n, const int* __restrict__ srp, const int* __restrict__ scol,
                            const int* __restrict__ state, const int* __restrict__ root_id,
                            int* __restrict__ agg) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (state[i] == kIn) { agg[i] = root_id[i]; return; }
    uint64_t best = 0;
    int a = -1;
    for (int p = srp[i]; p < srp[i + 1]; ++p) {
        int j = scol[p];
        if (state[j] != kIn) continue;
        uint64_t k = mis_key(kIn, j);
        if (a < 0 || k > best) { best = k; a = root_id[j]; }
    }
    agg[i] = a;
}

__global__ void k_agg_pass2(int64_t n, const int* __restrict__ srp, const int* __restrict__ scol,
                            const int* __restrict__ agg1, int* __restrict__ agg2, int* status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (agg1[i] >= 0) { agg2[i] = agg1[i]; return; }
    uint64_t best = 0;
    int a = -1;
    for (int p = srp[i]; p < srp[i + 1]; ++p) {
        int j = scol[p];
        if (agg1[j] < 0) continue;
        uint64_t k = mis_key(kUnd, j);
        if (a < 0 || k > best) { best = k; a = agg1[j]; }
    }
    agg2[i] = a;
    if (a < 0) atomicOr(status, kDevOverflow);
}

// Filtered matrix A^F of the prolongator smoother (Vanek, Mandel & Brezina,
// Computing 56, 1996): row i keeps its diagonal and its strong entries (the
// same test as the strength graph), and the weak off-diagonal entries are
// added into the diagonal, a^F_ii = a_ii - sum_weak a_ij (kept as a_ii if that
// is not positive). frp[i] = strong entries before row i + i (one diagonal per
// row). One warp per row; entries keep A's column order, and the weak sum is
// a fixed shuffle tree, so A^F is deterministic.
template <class V>
__global__ void k_filter_rows(int64_t n, const int* __restrict__ rp, const int* __restrict__ col,
                              const V* __restrict__ val, const V* __restrict__ dabs, V theta2,
                              const int* __restrict__ frp, int* __restrict__ fcol, V* __restrict__ fval) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const V di = dabs[i];
    const int p1 = rp[i + 1];
    int q = frp[i];
    int dpos = -1;
    V weak = V(0), aii = V(0);
    for (int p0 = rp[i]; p0 < p1; p0 += 32) {
        const int p = p0 + lane;
        const int j = p < p1 ? col[p] : -1;
        const V v = p < p1 ? val[p] : V(0);
        const bool diag = p < p1 && j == i;
        const bool st = p < p1 && is_strong(i, j, v, di, dabs, theta2);
        const bool keep = diag || st;
        if (p < p1 && !keep) weak += v;
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        const int at = q + __popc(m & ((1u << lane) - 1u));
        if (keep) {
            fcol[at] = j;
            fval[at] = v;
        }
        if (diag) {
            dpos = at;
            aii = v;
        }
        q += __popc(m);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) weak += __shfl_xor_sync(0xffffffffu, weak, o);
    if (dpos >= 0) {
        const V lumped = aii - weak;
        fval[dpos] = lumped > V(0) ? lumped : aii;
    }
}

__global__ void k_filter_ptr(int64_t n, const int* __restrict__ srp, int* __restrict__ frp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) frp[i] = srp[i] + (int)i;
}

template <class V>
__global__ void k_p0(int64_t n, const int* __restrict__ agg, int* __restrict__ rp,
                     int* __restrict__ col, V* __restrict__ val) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        rp[i] = (int)i;
        col[i] = agg[i];
        val[i] = V(1);
    }
    if (i == n) rp[n] = (int)n;
}

// P = P0 - omega D^-1 (A P0), in place on the values of A P0.
template <class V>
__global__ void k_smooth_p(int64_t n, const int* __restrict__ rp, const int* __restrict__ col,
                           V* __restrict__ val, const int* __restrict__ agg,
                           const V* __restrict__ dinv, V omega) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const V w = omega * dinv[i];
    for (int p = rp[i]; p < rp[i + 1]; ++p) val[p] = (col[p] == agg[i] ? V(1) : V(0)) - w * val[p];
}

// ------------------------------------------------------------------ coarse block inverse
// The coarsest matrix is inverted block by block: its contiguous diagonal
// blocks (one per instance and network in a batched union, the two S_p blocks
// of a single problem) are stored compactly, row-major, block c at coff[c].
// blk[3c .. 3c+2] = first row, size, offset of block c; rowblk[i] = block of row i.

// row extents: lo[i] / hi[i] = smallest / largest column of row i (and i itself)
__global__ void k_row_extents(int64_t n, const int* __restrict__ rp, const int* __restrict__ col,
                              int* __restrict__ lo, int* __restrict__ hi) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int a = (int)i, b = (int)i;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
        a = min(a, col[p]);
        b = max(b, col[p]);
    }
    lo[i] = a;
    hi[i] = b;
}

template <class V>
__global__ void k_csr_to_blocks(int64_t n, const int* __restrict__ rp, const int* __restrict__ col,
                                const V* __restrict__ val, const int* __restrict__ blk,
                                const int* __restrict__ rowblk, double* __restrict__ inv) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = rowblk[i];
    const int b0 = blk[3 * c], nb = blk[3 * c + 1], off = blk[3 * c + 2];
    for (int p = rp[i]; p < rp[i + 1]; ++p)
        inv[(int64_t)off + (int64_t)(i - b0) * nb + (col[p] - b0)] = (double)val[p];
}

// Gauss-Jordan of many small blocks at once: one CTA per listed block (list
// entries are block ids), the block held in shared memory.
constexpr int kGjSmall = 96;
constexpr size_t kGjSmem = (size_t)(kGjSmall * kGjSmall + kGjSmall) * sizeof(double);  // dynamic
__global__ void __launch_bounds__(256) k_gj_blocks(const int* __restrict__ list, const int* __restrict__ blk,
                                                   double* __restrict__ inv) {
    extern __shared__ double gj_smem[];
    double* a = gj_smem;                    // [nb][nb]
    double* f = gj_smem + kGjSmall * kGjSmall;
    const int c = list[blockIdx.x];
    const int nb = blk[3 * c + 1];
    double* M = inv + blk[3 * c + 2];
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) a[t] = M[t];
    __syncthreads();
    for (int k = 0; k < nb; ++k) {
        const double piv = a[k * nb + k];
        for (int i = threadIdx.x; i < nb; i += blockDim.x) f[i] = (i == k) ? 0.0 : a[i * nb + k];
        __syncthreads();
        for (int j = threadIdx.x; j < nb; j += blockDim.x) a[k * nb + j] = ((j == k) ? 1.0 : a[k * nb + j]) / piv;
        __syncthreads();
        for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
            const int i = t / nb, j = t % nb;
            if (i == k) continue;
            a[t] = ((j == k) ? 0.0 : a[t]) - f[i] * a[k * nb + j];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) M[t] = a[t];
}

// Gauss-Jordan of the blocks above kGjSmall rows, all in one cooperative
// launch (every CTA resident, which cudaLaunchCooperativeKernel checks). The
// blocks stay in global memory (L2); each warp takes one block row at a time
// and its lanes the row's columns. Pivot k of a block is one phase: with its column k (colb)
// and row k (rowb) as they stood after pivot k - 1,
//   M[k][j] = rowb[j] / rowb[k]               (rowb[k] is the pivot; M[k][k] = 1 / pivot)
//   M[i][j] = M[i][j] - colb[i] M[k][j]       (i != k; column k starts from 0)
// with one reciprocal of the pivot per row and pivot (the FP64 divide is
// many instructions on this part).
// and every thread that writes an element of row or column k + 1 also copies
// it to the other half of rowb / colb, so that one grid barrier per pivot
// separates the phases. Blocks with fewer than k + 1 rows have finished.
// The barrier is a generation counter with a bounded wait: a wait that runs
// out sets err[0] and every CTA returns.
struct GjBarrier {
    unsigned* count;
    unsigned* gen;
    int* err;
};

__device__ __forceinline__ bool gj_grid_barrier(const GjBarrier& b, unsigned nblocks) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* genv = b.gen;
        volatile int* errv = b.err;
        const unsigned g = *genv;
        __threadfence();
        if (atomicAdd(b.count, 1u) + 1u == nblocks) {
            *b.count = 0u;
            __threadfence();
            atomicAdd(b.gen, 1u);
        } else {
            long spins = 0;
            while (*genv == g) {
                if (*errv) { ok = 0; break; }
                if (++spins > (1L << 24)) {  // far beyond any pivot phase (about a second)
                    atomicExch(b.err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_sh = ok && !*errv;
    }
    __syncthreads();
    return ok_sh != 0;
}

__global__ void __launch_bounds__(256) k_gj_coop(int n_large, const int* __restrict__ list,
                                                 const int* __restrict__ blk, double* __restrict__ inv,
                                                 double* __restrict__ colb, double* __restrict__ rowb,
                                                 const int* __restrict__ voff, int max_nb, GjBarrier bar) {
    // one warp per block row at a time; rows are numbered across the blocks
    // (voff is the prefix sum of the block sizes, searched by bisection)
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    const int n_rows = voff[n_large];
    auto locate = [&](int r, int& q, int& i) {
        int lo = 0, hi = n_large - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (voff[mid] <= r) lo = mid;
            else hi = mid - 1;
        }
        q = lo;
        i = r - voff[lo];
    };
    // column 0 and row 0 of every block, before the first pivot
    for (int r = warp; r < n_rows; r += n_warps) {
        int q, i;
        locate(r, q, i);
        const int nb = blk[3 * list[q] + 1];
        const double* M = inv + blk[3 * list[q] + 2] + (int64_t)i * nb;
        if (lane == 0) colb[2 * voff[q] + i] = M[0];
        if (i == 0)
            for (int j = lane; j < nb; j += 32) rowb[2 * voff[q] + j] = M[j];
    }
    if (!gj_grid_barrier(bar, gridDim.x)) return;
    for (int k = 0; k < max_nb; ++k) {
        const int h = k & 1, hn = h ^ 1;
        for (int r = warp; r < n_rows; r += n_warps) {
            int q, i;
            locate(r, q, i);
            const int nb = blk[3 * list[q] + 1];
            if (k >= nb) continue;
            double* M = inv + blk[3 * list[q] + 2] + (int64_t)i * nb;
            const double* rb = rowb + 2 * voff[q] + (int64_t)h * nb;
            double* col_next = colb + 2 * voff[q] + (int64_t)hn * nb;
            double* row_next = rowb + 2 * voff[q] + (int64_t)hn * nb;
            const double rpiv = 1.0 / rb[k];
            const double ci = (i == k) ? 0.0 : colb[2 * voff[q] + (int64_t)h * nb + i];
            for (int j = lane; j < nb; j += 32) {
                const double rkj = (j == k) ? rpiv : rb[j] * rpiv;
                const double mij = (i == k || j == k) ? 0.0 : M[j];
                const double v = (i == k) ? rkj : fma(-ci, rkj, mij);
                M[j] = v;
                if (j == k + 1) col_next[i] = v;
                if (i == k + 1) row_next[j] = v;
            }
        }
        if (!gj_grid_barrier(bar, gridDim.x)) return;
    }
}

// x = Minv b for the block-diagonal inverse: one warp per row; the inverse and
// the accumulation stay FP64 in both modes
template <class T>
__global__ void k_block_mv(int64_t n, const double* __restrict__ inv, const int* __restrict__ blk,
                           const int* __restrict__ rowblk, const T* __restrict__ b, T* __restrict__ x) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const int c = rowblk[row];
    const int b0 = blk[3 * c], nb = blk[3 * c + 1];
    const double* M = inv + blk[3 * c + 2] + (int64_t)(row - b0) * nb;
    double acc = 0.0;
    for (int j = lane; j < nb; j += 32) acc += M[j] * (double)b[b0 + j];
    acc = warp_sum(acc);
    if (lane == 0) x[row] = (T)acc;
}

inline int sgrid(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 8 * kSMs); }

void check_dev(DBuf<int>& st, cudaStream_t s, HostScratch& hs, const char* what) {
    int v = read_scalar(st.get(), s, hs);
    if (v) fail(DPP_ERR_INVALID_ARGUMENT, std::string("AMG setup: ") + what);
}

// ||x||^2 into out[0], summed in FP64 (an FP32 x is widened first into wide)
void sq_norm(Reducer& R, const double* x, int64_t n, double* out, DBuf<double>&, cudaStream_t s) {
    dot(R, x, x, n, out, s);
}
void sq_norm(Reducer& R, const float* x, int64_t n, double* out, DBuf<double>& wide, cudaStream_t s) {
    k_f2d<<<sgrid(n), 256, 0, s>>>(n, x, wide.get());
    DPP_LAUNCH_CK();
    dot(R, wide.get(), wide.get(), n, out, s);
}

// lambda_max(D^-1 A) by 12 power steps in the hierarchy's precision V; the
// vector is renormalised on the device (no host round trip per step) and the
// estimate read once at the end.
template <class V>
double power_lmax(const Csr& A, const V* dinv, int lanes, cudaStream_t s, HostScratch& hs) {
    const int64_t n = A.n_rows;
    DBuf<V> v(n), w(n);
    DBuf<double> nrm(1), wide(sizeof(V) == 4 ? n : 0);
    const int B = 256;
    k_hash_vector<V><<<grid_for(n, B), B, 0, s>>>(n, v.get());
    DPP_LAUNCH_CK();
    Reducer R;
    sq_norm(R, v.get(), n, nrm.get(), wide, s);
    k_scale_rsqrt<V><<<sgrid(n), 256, 0, s>>>(n, v.get(), v.get(), nrm.get());
    DPP_LAUNCH_CK();
    for (int it = 0; it < 12; ++it) {
        spmv_lanes<0, V>(lanes, A, v.get(), nullptr, w.get(), s);
        k_dinv_scale<V><<<sgrid(n), 256, 0, s>>>(n, dinv, w.get());
        DPP_LAUNCH_CK();
        sq_norm(R, w.get(), n, nrm.get(), wide, s);   // ||D^-1 A v||^2 with ||v|| = 1
        k_scale_rsqrt<V><<<sgrid(n), 256, 0, s>>>(n, w.get(), v.get(), nrm.get());
        DPP_LAUNCH_CK();
    }
    const double l2 = read_scalar(nrm.get(), s, hs);
    if (!(l2 > 0.0) || !std::isfinite(l2)) fail(DPP_ERR_NONFINITE, "AMG setup: power iteration");
    return std::sqrt(l2);
}

// Contiguous diagonal blocks of A from its row extents: a boundary falls after
// row i when no row up to i reaches beyond i and no row after i reaches back
// to i or before. Returns (first row, size) pairs.
std::vector<std::pair<int, int>> diag_blocks(const Csr& A, cudaStream_t s) {
    const int64_t n = A.n_rows;
    DBuf<int> d_lo(n), d_hi(n);
    k_row_extents<<<grid_for(n, 256), 256, 0, s>>>(n, A.row_ptr.get(), A.col.get(), d_lo.get(), d_hi.get());
    DPP_LAUNCH_CK();
    std::vector<int> lo(n), hi(n);
    DPP_CK(cudaMemcpyAsync(lo.data(), d_lo.get(), n * sizeof(int), cudaMemcpyDeviceToHost, s));
    DPP_CK(cudaMemcpyAsync(hi.data(), d_hi.get(), n * sizeof(int), cudaMemcpyDeviceToHost, s));
    DPP_CK(cudaStreamSynchronize(s));
    std::vector<int> suffix_lo(n + 1, INT32_MAX);
    for (int64_t i = n - 1; i >= 0; --i) suffix_lo[i] = std::min(suffix_lo[i + 1], lo[i]);
    std::vector<std::pair<int, int>> blocks;
    int start = 0, reach = -1;
    for (int64_t i = 0; i < n; ++i) {
        reach = std::max(reach, hi[i]);
        if (reach <= i && suffix_lo[i + 1] > i) {
            blocks.emplace_back(start, (int)i + 1 - start);
            start = (int)i + 1;
        }
    }
    return blocks;
}

// Inverse of the coarsest matrix (SPD: Gauss-Jordan without pivoting), block
// by block in compact storage. Blocks of at most kGjSmall rows are inverted
// one CTA each in shared memory, in one launch; the larger ones together in
// one cooperative launch, one grid barrier per pivot.
void block_inverse(Amg& pc, const Csr& A, cudaStream_t s) {
    const int64_t n = A.n_rows;
    const auto blocks = diag_blocks(A, s);
    std::vector<int> blk(3 * blocks.size()), rowblk(n), small;
    int64_t off = 0;
    for (size_t c = 0; c < blocks.size(); ++c) {
        const int b0 = blocks[c].first, nb = blocks[c].second;
        if (nb > 4096) fail(DPP_ERR_INVALID_ARGUMENT, "AMG setup: a coarsest diagonal block has more than "
                                                      "4096 rows; raise max_levels or lower strength_theta");
        blk[3 * c] = b0;
        blk[3 * c + 1] = nb;
        blk[3 * c + 2] = (int)off;
        for (int r = 0; r < nb; ++r) rowblk[b0 + r] = (int)c;
        if (nb <= kGjSmall) small.push_back((int)c);
        off += (int64_t)nb * nb;
        if (off >= INT32_MAX) fail(DPP_ERR_INVALID_ARGUMENT, "AMG setup: coarsest blocks too large");
    }
    pc.coarse_blk.alloc(blk.size());
    pc.coarse_rowblk.alloc(n);
    pc.coarse_inv.alloc(std::max<int64_t>(off, 1));
    DPP_CK(cudaMemcpyAsync(pc.coarse_blk.get(), blk.data(), blk.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    DPP_CK(cudaMemcpyAsync(pc.coarse_rowblk.get(), rowblk.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
    DPP_CK(cudaMemsetAsync(pc.coarse_inv.get(), 0, off * sizeof(double), s));
    if (fp32_only(A))  // the FP32 hierarchy: the coarsest matrix is widened, its inverse is FP64
        k_csr_to_blocks<float><<<grid_for(n, 128), 128, 0, s>>>(n, A.row_ptr.get(), A.col.get(), A.val32.get(),
                                                                pc.coarse_blk.get(), pc.coarse_rowblk.get(),
                                                                pc.coarse_inv.get());
    else
        k_csr_to_blocks<double><<<grid_for(n, 128), 128, 0, s>>>(n, A.row_ptr.get(), A.col.get(), A.val.get(),
                                                                 pc.coarse_blk.get(), pc.coarse_rowblk.get(),
                                                                 pc.coarse_inv.get());
    DPP_LAUNCH_CK();
    if (!small.empty()) {
        DBuf<int> d_small(small.size());
        DPP_CK(cudaMemcpyAsync(d_small.get(), small.data(), small.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        DPP_CK(cudaFuncSetAttribute(k_gj_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGjSmem));
        k_gj_blocks<<<(unsigned)small.size(), 256, kGjSmem, s>>>(d_small.get(), pc.coarse_blk.get(),
                                                                 pc.coarse_inv.get());
        DPP_LAUNCH_CK();
    }
    // the larger blocks: one cooperative launch for all of them
    std::vector<int> large, voff(1, 0);
    int max_nb = 0;
    for (size_t c = 0; c < blocks.size(); ++c) {
        const int nb = blocks[c].second;
        if (nb <= kGjSmall) continue;
        large.push_back((int)c);
        voff.push_back(voff.back() + nb);
        max_nb = std::max(max_nb, nb);
    }
    if (!large.empty()) {
        const int nl = (int)large.size();
        DBuf<int> d_large(nl), d_voff(nl + 1), ctl(3);  // ctl: count, generation, error
        DBuf<double> colb(2 * (size_t)voff.back()), rowb(2 * (size_t)voff.back());
        DPP_CK(cudaMemcpyAsync(d_large.get(), large.data(), nl * sizeof(int), cudaMemcpyHostToDevice, s));
        DPP_CK(cudaMemcpyAsync(d_voff.get(), voff.data(), (nl + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
        DPP_CK(cudaMemsetAsync(ctl.get(), 0, 3 * sizeof(int), s));
        const int grid = std::min(kSMs, std::max(1, (voff.back() + 7) / 8));
        int n_large = nl, mx = max_nb;
        const int* a_list = d_large.get();
        const int* a_blk = pc.coarse_blk.get();
        double* a_inv = pc.coarse_inv.get();
        double* a_col = colb.get();
        double* a_row = rowb.get();
        const int* a_voff = d_voff.get();
        GjBarrier bar{reinterpret_cast<unsigned*>(ctl.get()), reinterpret_cast<unsigned*>(ctl.get() + 1),
                      ctl.get() + 2};
        void* args[] = {&n_large, &a_list, &a_blk, &a_inv, &a_col, &a_row, &a_voff, &mx, &bar};
        DPP_CK(cudaLaunchCooperativeKernel((const void*)k_gj_coop, dim3(grid), dim3(256), args, 0, s));
        DPP_LAUNCH_CK();
        int err = 0;
        DPP_CK(cudaMemcpyAsync(&err, ctl.get() + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
        DPP_CK(cudaStreamSynchronize(s));
        if (err) fail(DPP_ERR_TIMEOUT, "AMG setup: the coarse Gauss-Jordan barrier timed out");
    }
    DPP_CK(cudaStreamSynchronize(s));  // host tables go out of scope
}

}  // namespace

namespace {
template <class V> DBuf<V>& dinv_of(Level& L);
template <> DBuf<double>& dinv_of<double>(Level& L) { return L.dinv; }
template <> DBuf<float>& dinv_of<float>(Level& L) { return L.dinv32; }

// The setup in the precision V of A0's values: FP64 (the FP64 hierarchy, of
// which amg_make_fp32 may add FP32 copies), or FP32 (the hierarchy of the
// mixed mode, built in FP32 from the FP32 S_p; only its coarsest inverse is
// FP64).
template <class V>
void amg_setup_t(Amg& pc, const dpp_pc_opts& o, Csr&& A0, cudaStream_t s, HostScratch& hs) {
    ProfScope prof_all("setup_amg", s, 0);
    pc.levels.clear();
    pc.levels.emplace_back();
    pc.levels[0].A = std::move(A0);
    DBuf<int> st(1);
    const int B = 256;
    // Galerkin products of a symmetric A (S_p is, up to rounding in its
    // assembly) may be computed as an upper triangle and mirrored
    constexpr int64_t kMirrorMinRows = 16384;
    constexpr int64_t kBlockCoarseRows = 65536;
    // S_p is symmetric by construction (D symmetric, C = -B^T in exact
    // arithmetic), so a sample of every 16th row only guards against a
    // structural surprise
    const bool symmetric = is_symmetric(pc.levels[0].A, sizeof(V) == 8 ? 1e-10 : 1e-5, 16, s, hs);
    pc.symmetric = symmetric;
    for (int l = 0;; ++l) {
        Level& L = pc.levels[l];
        const int64_t n = L.A.n_rows;
        L.lanes = pick_lanes(L.A);
        if (o.spmv_format != 1 && n >= sell_min_rows(o)) {
            build_sell(L.A, s, hs);
            if (L.A.has_sell()) L.lanes = 0;  // SELL-32 (the autotuner may still pick CSR)
        }
        DBuf<V>& dinv = dinv_of<V>(L);
        dinv.alloc(n);
        DBuf<V> dabs(n);
        DPP_CK(cudaMemsetAsync(st.get(), 0, sizeof(int), s));
        k_diag_inv<V><<<grid_for(n, B), B, 0, s>>>(n, L.A.row_ptr.get(), L.A.col.get(),
                                                   vbuf<V>(L.A).get(), dinv.get(), dabs.get(), st.get());
        DPP_LAUNCH_CK();
        check_dev(st, s, hs, "a level matrix has a non-positive diagonal entry");
        if (sizeof(V) == 8) {  // FP64 work vectors (amg_make_fp32 adds the FP32 ones)
            L.x.alloc(n);
            L.xt.alloc(n);
            L.b.alloc(n);
            L.r.alloc(n);
            L.d.alloc(n);
        }
        bool last = (n <= o.coarse_max_rows) || (l + 1 >= o.max_levels);
        if (!last && n <= kBlockCoarseRows) {
            // a level made of small diagonal blocks only (a batched union that
            // has coarsened to a few rows per instance) is solved directly
            int max_block = 0;
            for (const auto& bl : diag_blocks(L.A, s)) max_block = std::max(max_block, bl.second);
            last = max_block <= kGjSmall;
        }
        if (last) break;  // the coarsest level is solved directly: no smoother, no lambda_max
        {
            ProfScope pr("setup_power", s, 0);
            L.lmax = power_lmax<V>(L.A, dinv.get(), L.lanes, s, hs);
        }

        // strength graph
        ProfScope pr_agg("setup_aggregate", s, 0);
        ProfScope pr_str("setup_strength", s, 0);
        const double theta2 = o.strength_theta * o.strength_theta;
        Csr S;
        S.n_rows = S.n_cols = n;
        S.row_ptr.alloc(n + 1);
        DPP_CK(cudaMemsetAsync(S.row_ptr.get(), 0, (n + 1) * sizeof(int), s));
        DBuf<int> stage(std::max<int64_t>(L.A.nnz, 1));
        k_strength_stage<V><<<grid_for(n * 32, B), B, 0, s>>>(n, L.A.row_ptr.get(), L.A.col.get(),
                                                         vbuf<V>(L.A).get(), dabs.get(), (V)theta2,
                                                         S.row_ptr.get(), stage.get());
        DPP_LAUNCH_CK();
        S.nnz = exclusive_scan(S.row_ptr.get(), S.row_ptr.get(), n + 1, s, hs);
        S.col.alloc(std::max<int64_t>(S.nnz, 1));
        k_strength_compact<<<grid_for(n * 32, B), B, 0, s>>>(n, L.A.row_ptr.get(), stage.get(),
                                                        S.row_ptr.get(), S.col.get());
        DPP_LAUNCH_CK();

        pr_str.stop();
        // distance-2 maximal independent set
        ProfScope pr_mis("setup_mis", s, 0);
        DBuf<int> state(n), undecided(1);
        DBuf<uint64_t> t0a(n), t0b(n), t1(n), t2(n);
        k_fill_int<<<grid_for(n, B), B, 0, s>>>(n, kUnd, state.get());
        DPP_LAUNCH_CK();
        k_mis_t0<<<grid_for(n, B), B, 0, s>>>(n, state.get(), t0a.get());
        DPP_LAUNCH_CK();
        uint64_t* t0 = t0a.get();
        uint64_t* t0n = t0b.get();
        for (int round = 0; round < 64; ++round) {
            DPP_CK(cudaMemsetAsync(undecided.get(), 0, sizeof(int), s));
            k_mis_max<<<grid_for(n * kMisLanes, B), B, 0, s>>>(n, S.row_ptr.get(), S.col.get(), t0, t1.get());
            DPP_LAUNCH_CK();
            k_mis_max<<<grid_for(n * kMisLanes, B), B, 0, s>>>(n, S.row_ptr.get(), S.col.get(), t1.get(), t2.get());
            DPP_LAUNCH_CK();
            k_mis_update<<<grid_for(n, B), B, 0, s>>>(n, state.get(), t0, t2.get(), t0n, undecided.get());
            DPP_LAUNCH_CK();
            std::swap(t0, t0n);
            // the count is read every other round (a round after the last
            // decision changes nothing), which halves the host round trips
            if ((round & 1) && read_scalar(undecided.get(), s, hs) == 0) break;
            if (round == 63) fail(DPP_ERR_INVALID_ARGUMENT, "AMG setup: MIS-2 did not finish");
        }
        pr_mis.stop();
        DBuf<int> root_id(n + 1), agg1(n), agg(n);
        k_root_flags<<<grid_for(n + 1, B), B, 0, s>>>(n, state.get(), root_id.get());
        DPP_LAUNCH_CK();
        const int64_t n_agg = exclusive_scan(root_id.get(), root_id.get(), n + 1, s, hs);
        k_agg_pass1<<<grid_for(n, B), B, 0, s>>>(n, S.row_ptr.get(), S.col.get(), state.get(),
                                                 root_id.get(), agg1.get());
        DPP_LAUNCH_CK();
        DPP_CK(cudaMemsetAsync(st.get(), 0, sizeof(int), s));
        k_agg_pass2<<<grid_for(n, B), B, 0, s>>>(n, S.row_ptr.get(), S.col.get(), agg1.get(),
                                                 agg.get(), st.get());
        DPP_LAUNCH_CK();
        check_dev(st, s, hs, "a row was left without an aggregate");
        if (n_agg <= 0 || n_agg >= n) break;  // no coarsening possible: this level is the last

        // prolongator
        ProfScope pr_rap("setup_prolong_rap", s, 0);
        Csr P0;
        P0.n_rows = n;
        P0.n_cols = n_agg;
        P0.nnz = n;
        P0.row_ptr.alloc(n + 1);
        P0.col.alloc(n);
        vbuf<V>(P0).alloc(n);
        k_p0<V><<<grid_for(n + 1, B), B, 0, s>>>(n, agg.get(), P0.row_ptr.get(), P0.col.get(),
                                                 vbuf<V>(P0).get());
        DPP_LAUNCH_CK();
        Csr Pm;
        if (o.smooth_filter) {
            // P = (I - omega D_F^-1 A^F) P0 with the filtered A^F, omega = 4 / (3 lambda_max(D_F^-1 A^F))
            Csr AF;
            AF.n_rows = AF.n_cols = n;
            AF.nnz = S.nnz + n;
            AF.row_ptr.alloc(n + 1);
            AF.col.alloc(std::max<int64_t>(AF.nnz, 1));
            vbuf<V>(AF).alloc(std::max<int64_t>(AF.nnz, 1));
            k_filter_ptr<<<grid_for(n + 1, B), B, 0, s>>>(n, S.row_ptr.get(), AF.row_ptr.get());
            DPP_LAUNCH_CK();
            k_filter_rows<V><<<grid_for(n * 32, B), B, 0, s>>>(n, L.A.row_ptr.get(), L.A.col.get(),
                                                              vbuf<V>(L.A).get(), dabs.get(), (V)theta2,
                                                              AF.row_ptr.get(), AF.col.get(), vbuf<V>(AF).get());
            DPP_LAUNCH_CK();
            DBuf<V> dinv_f(n);
            DPP_CK(cudaMemsetAsync(st.get(), 0, sizeof(int), s));
            k_diag_inv<V><<<grid_for(n, B), B, 0, s>>>(n, AF.row_ptr.get(), AF.col.get(), vbuf<V>(AF).get(),
                                                       dinv_f.get(), nullptr, st.get());
            DPP_LAUNCH_CK();
            check_dev(st, s, hs, "a filtered level matrix has a non-positive diagonal entry");
            double lmax_f;
            {
                ProfScope pr("setup_power", s, 0);
                lmax_f = power_lmax<V>(AF, dinv_f.get(), pick_lanes(AF), s, hs);
            }
            {
                ProfScope q(l == 0 ? "spgemm_AP0_L0" : "spgemm_AP0_Lc", s, 0);
                spgemm(view(AF), view(P0), Pm, true, s, hs);
            }
            k_smooth_p<V><<<grid_for(n, B), B, 0, s>>>(n, Pm.row_ptr.get(), Pm.col.get(), vbuf<V>(Pm).get(),
                                                       agg.get(), dinv_f.get(), (V)(4.0 / (3.0 * lmax_f)));
            DPP_LAUNCH_CK();
        } else {
            {
                ProfScope q(l == 0 ? "spgemm_AP0_L0" : "spgemm_AP0_Lc", s, 0);
                spgemm(view(L.A), view(P0), Pm, true, s, hs);
            }
            const double omega = 4.0 / (3.0 * L.lmax);
            k_smooth_p<V><<<grid_for(n, B), B, 0, s>>>(n, Pm.row_ptr.get(), Pm.col.get(), vbuf<V>(Pm).get(),
                                                       agg.get(), dinv.get(), (V)omega);
            DPP_LAUNCH_CK();
        }
        L.P = std::move(Pm);
        if (o.spmv_format != 1 && n >= sell_min_rows(o)) build_sell(L.P, s, hs);  // autotuner may pick it
        transpose(L.P, L.R, s, hs);
        Csr AP;
        {
            ProfScope q(l == 0 ? "spgemm_AP_L0" : "spgemm_AP_Lc", s, 0);
            spgemm(view(L.A), view(L.P), AP, true, s, hs);
        }
        Csr Ac;
        {
            ProfScope q(l == 0 ? "spgemm_RAP_L0" : "spgemm_RAP_Lc", s, 0);
            // P^T A P is symmetric too: its upper triangle, mirrored, where the
            // product is large enough (many coarse rows) to repay the mirroring
            if (symmetric && L.R.n_rows >= kMirrorMinRows) {
                Csr U;
                spgemm(view(L.R), view(AP), U, true, s, hs, /*upper_only=*/true);
                symmetrize_upper(U, Ac, s, hs);
            } else {
                spgemm(view(L.R), view(AP), Ac, true, s, hs);
            }
        }
        pc.levels.emplace_back();
        pc.levels.back().A = std::move(Ac);
    }
    // coarse solve
    Level& C = pc.levels.back();
    pc.coarse_n = C.A.n_rows;
    ProfScope pr("setup_coarse_inverse", s, 0);
    block_inverse(pc, C.A, s);
}
}  // namespace

void amg_setup(Amg& pc, const dpp_pc_opts& o, Csr&& A0, cudaStream_t s, HostScratch& hs) {
    if (fp32_only(A0)) amg_setup_t<float>(pc, o, std::move(A0), s, hs);
    else amg_setup_t<double>(pc, o, std::move(A0), s, hs);
}

namespace {

template <class T> T* lv(DBuf<double>& d, DBuf<float>& f);
template <> double* lv<double>(DBuf<double>& d, DBuf<float>&) { return d.get(); }
template <> float* lv<float>(DBuf<double>&, DBuf<float>& f) { return f.get(); }

// Chebyshev degree of level l: cheb_degree_amg, or on the coarser levels
// cheb_degree_coarse when that is set
inline int cheb_degree(const dpp_pc_opts& o, size_t l) {
    return std::max(1, (l > 0 && o.cheb_degree_coarse > 0) ? o.cheb_degree_coarse : o.cheb_degree_amg);
}

template <class T>
void cheb_smooth(const dpp_pc_opts& o, size_t l, Level& L, const T* b, T* x, bool zero_init, cudaStream_t s,
                 const char* fam = nullptr) {
    const int deg = cheb_degree(o, l);
    const double hi = 1.1 * L.lmax, lo = L.lmax / o.cheb_ratio;
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
    const int64_t n = L.A.n_rows;
    T* tmp = lv<T>(L.xt, L.xt32);
    T* d = lv<T>(L.d, L.d32);
    const T* dinv = lv<T>(L.dinv, L.dinv32);
    double rho = 1.0 / sigma;
    // Every step after a zero start is one fused SpMV + update (MODE 3) that
    // writes the new iterate to the other of x and tmp; the start buffer is
    // chosen so that the last step lands in x.
    const int fused = zero_init ? deg - 1 : deg;
    T* cur = x;
    int k = 0;
    if (zero_init) {
        cur = (fused % 2 == 0) ? x : tmp;
        k_cheb_start<T><<<sgrid(n), 256, 0, s>>>(n, dinv, b, d, cur, T(1.0 / theta));
        DPP_LAUNCH_CK();
        k = 1;
    }
    for (; k < deg; ++k) {
        double c1 = 0.0, c2 = 1.0 / theta;
        if (k > 0) {
            const double rho_new = 1.0 / (2.0 * sigma - rho);
            c1 = rho_new * rho;
            c2 = 2.0 * rho_new / delta;
            rho = rho_new;
        }
        ChebOut<T> ch;
        ch.dinv = dinv;
        ch.d = d;
        ch.xo = (cur == x) ? tmp : x;
        ch.c1 = T(c1);
        ch.c2 = T(c2);
        spmv_lanes<3, T>(L.lanes, L.A, cur, b, nullptr, s, fam, ch);
        cur = ch.xo;
    }
    if (cur != x) DPP_CK(cudaMemcpyAsync(x, cur, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
}

template <class T>
void vcycle_level(Amg& pc, const dpp_pc_opts& o, size_t l, const T* b, T* x, cudaStream_t s) {
    Level& L = pc.levels[l];
    if (l + 1 == pc.levels.size()) {
        const int64_t n = pc.coarse_n;
        k_block_mv<T><<<grid_for(n * 32, 256), 256, 0, s>>>(n, pc.coarse_inv.get(), pc.coarse_blk.get(),
                                                            pc.coarse_rowblk.get(), b, x);
        DPP_LAUNCH_CK();
        return;
    }
    Level& C = pc.levels[l + 1];
    T* r = lv<T>(L.r, L.r32);
    T* cb = lv<T>(C.b, C.b32);
    T* cx = lv<T>(C.x, C.x32);
    // timing families: level-0 A, coarser A, and the transfers P and R
    const bool f64 = sizeof(T) == 8;
    const char* fam = (l == 0) ? (f64 ? "amg_spmv_L0" : "amg_spmv_L0_fp32")
                               : (f64 ? "amg_spmv_Lc" : "amg_spmv_Lc_fp32");
    const char* fam_pr = f64 ? "amg_spmv_PR" : "amg_spmv_PR_fp32";
    cheb_smooth<T>(o, l, L, b, x, true, s, fam);
    spmv_lanes<1, T>(L.lanes, L.A, x, b, r, s, fam);
    spmv_lanes<0, T>(L.lanes_R, L.R, r, nullptr, cb, s, fam_pr);
    vcycle_level<T>(pc, o, l + 1, cb, cx, s);
    spmv_lanes<2, T>(L.lanes_P, L.P, cx, nullptr, x, s, fam_pr);
    cheb_smooth<T>(o, l, L, b, x, false, s, fam);
}

void to_f32(const DBuf<double>& in, DBuf<float>& out, cudaStream_t s) {
    out.alloc(in.n);
    if (in.n) {
        k_d2f<<<sgrid((int64_t)in.n), 256, 0, s>>>((int64_t)in.n, in.get(), out.get());
        DPP_LAUNCH_CK();
    }
}

// ------------------------------------------------------------------ autotuner
// Lanes per row of the CSR SpMV, chosen per matrix by timing every candidate
// on the device. Choices are cached for the process per size class (precision,
// operator kind, log2 rows, mean row length). If the environment variable
// DPP_TUNE_CACHE names a file, the cache is read from it and new choices are
// appended to it as JSON lines.
struct TuneKey {
    int fp32, kind, log2_rows, avg_nnz, sell;
    bool operator<(const TuneKey& o) const {
        return std::tie(fp32, kind, log2_rows, avg_nnz, sell) <
               std::tie(o.fp32, o.kind, o.log2_rows, o.avg_nnz, o.sell);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;
bool g_tune_loaded = false;

void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = std::getenv("DPP_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char line[256];
    while (std::fgets(line, sizeof line, f)) {
        TuneKey k;
        int lanes = 0;
        if (std::sscanf(line,
                        "{\"fp32\": %d, \"kind\": %d, \"log2_rows\": %d, \"avg_nnz\": %d, "
                        "\"sell\": %d, \"lanes\": %d}",
                        &k.fp32, &k.kind, &k.log2_rows, &k.avg_nnz, &k.sell, &lanes) == 6 &&
            ((lanes == 0 && k.sell == 1) || lanes == 2 || lanes == 4 || lanes == 8 || lanes == 16 ||
             lanes == 32))
            g_tune[k] = lanes;
    }
    std::fclose(f);
}

void tune_store_locked(const TuneKey& k, int lanes) {
    g_tune[k] = lanes;
    const char* path = std::getenv("DPP_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"fp32\": %d, \"kind\": %d, \"log2_rows\": %d, \"avg_nnz\": %d, \"sell\": %d, "
                 "\"lanes\": %d}\n",
                 k.fp32, k.kind, k.log2_rows, k.avg_nnz, k.sell, lanes);
    std::fclose(f);
}

template <int MODE, class T>
int tune_lanes(const Csr& A, const T* x, const T* b, T* y, int kind, cudaStream_t s) {
    TuneKey key;
    key.fp32 = sizeof(T) == 4;
    key.kind = kind;
    key.log2_rows = 0;
    for (int64_t r = A.n_rows; r > 1; r >>= 1) ++key.log2_rows;
    key.avg_nnz = (int)std::lround(A.n_rows ? (double)A.nnz / (double)A.n_rows : 0.0);
    key.sell = A.has_sell() ? 1 : 0;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load_locked();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) return it->second;
    }
    // candidates: SELL-32 when built (first, so that it wins ties), then the
    // heuristic CSR choice and its neighbours
    const int h = pick_lanes(A);
    std::vector<int> cands;
    if (A.has_sell()) cands.push_back(0);
    for (int c : {std::max(2, h / 2), h, std::min(32, h * 2)}) cands.push_back(c);
    cudaEvent_t e0, e1;
    DPP_CK(cudaEventCreate(&e0));
    DPP_CK(cudaEventCreate(&e1));
    int best = cands[0];
    float best_ms = 1e30f;
    for (int c : cands) {
        spmv_lanes<MODE, T>(c, A, x, b, y, s);  // warm
        for (int trial = 0; trial < 2; ++trial) {
            DPP_CK(cudaEventRecord(e0, s));
            for (int rep = 0; rep < 10; ++rep) spmv_lanes<MODE, T>(c, A, x, b, y, s);
            DPP_CK(cudaEventRecord(e1, s));
            DPP_CK(cudaEventSynchronize(e1));
            float ms = 0;
            DPP_CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_ms * 0.97f) { best_ms = ms; best = c; }  // ties keep the earlier (fewer lanes)
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_store_locked(key, best);
    return best;
}

template <class T>
void tune_levels(Amg& pc, const dpp_pc_opts& o, cudaStream_t s) {
    for (size_t l = 0; l < pc.levels.size(); ++l) {
        Level& L = pc.levels[l];
        T* x = lv<T>(L.x, L.x32);
        T* b = lv<T>(L.b, L.b32);
        T* r = lv<T>(L.r, L.r32);
        DPP_CK(cudaMemsetAsync(x, 0, L.A.n_rows * sizeof(T), s));
        DPP_CK(cudaMemsetAsync(b, 0, L.A.n_rows * sizeof(T), s));
        if (o.spmv_format == 2 && L.A.has_sell()) L.lanes = 0;  // SELL-32 as asked
        else L.lanes = tune_lanes<1, T>(L.A, x, b, r, 0, s);
        if (l + 1 < pc.levels.size()) {
            Level& C = pc.levels[l + 1];
            T* cx = lv<T>(C.x, C.x32);
            T* cb = lv<T>(C.b, C.b32);
            DPP_CK(cudaMemsetAsync(cx, 0, C.A.n_rows * sizeof(T), s));
            L.lanes_R = tune_lanes<0, T>(L.R, r, nullptr, cb, 1, s);
            if (o.spmv_format == 2 && L.P.has_sell()) L.lanes_P = 0;
            else L.lanes_P = tune_lanes<2, T>(L.P, cx, nullptr, x, 2, s);
        }
    }
    DPP_CK(cudaStreamSynchronize(s));
}

}  // namespace

void amg_tune(Amg& pc, const dpp_pc_opts& o, int precision, cudaStream_t s) {
    ProfScope pr("setup_tune", s, 0);
    if (precision == DPP_MIXED_FP32_FP64) tune_levels<float>(pc, o, s);
    else tune_levels<double>(pc, o, s);
}

void amg_make_fp32(Amg& pc, cudaStream_t s) {
    for (size_t l = 0; l < pc.levels.size(); ++l) {
        Level& L = pc.levels[l];
        if (!fp32_only(L.A)) {  // an FP64 hierarchy: FP32 copies of its values
            to_f32(L.A.val, L.A.val32, s);
            if (L.A.has_sell()) to_f32(L.A.sell_val, L.A.sell_val32, s);
            if (L.dinv.get()) to_f32(L.dinv, L.dinv32, s);
            if (l + 1 < pc.levels.size()) {
                to_f32(L.P.val, L.P.val32, s);
                if (L.P.has_sell()) to_f32(L.P.sell_val, L.P.sell_val32, s);
                to_f32(L.R.val, L.R.val32, s);
            }
        }
        const int64_t n = L.A.n_rows;
        L.x32.alloc(n);
        L.xt32.alloc(n);
        L.b32.alloc(n);
        L.r32.alloc(n);
        L.d32.alloc(n);
    }
    DPP_CK(cudaStreamSynchronize(s));
}

template <class T>
void amg_vcycle(Amg& h, const dpp_pc_opts& o, const T* b, T* x, cudaStream_t s) {
    vcycle_level<T>(h, o, 0, b, x, s);
}
template void amg_vcycle<double>(Amg&, const dpp_pc_opts&, const double*, double*, cudaStream_t);
template void amg_vcycle<float>(Amg&, const dpp_pc_opts&, const float*, float*, cudaStream_t);

}  // namespace dpp
