// Batched solves: many independent DPP systems (permeability realisations,
// meshes of uneven size) in one union problem and one lock-step FGMRES.
//
// Union: instance b's nodes and cells are shifted by the totals of the
// instances before it, so the union K is block-diagonal. Assembly, the selfp
// Schur blocks (Eqs. "S4_sp1", "S4_sp2") and the smoothed-aggregation hierarchy
// run unchanged on the union. No strength edge joins two instances, so no
// aggregate spans two instances and every level stays block-diagonal. mu and
// beta may differ between instances; they travel as per-cell values.
//
// Krylov: every instance runs its own right-preconditioned FGMRES(m): its
// own inner products, Hessenberg matrix, Givens rotations, least-squares
// solve and convergence test. All instances share every kernel launch.
// Reductions are segmented by a chunk table whose chunks never straddle two
// instances: each block reduces one chunk, then one pass adds an instance's
// chunk partials in chunk order. The result is deterministic. The small
// per-instance algebra runs as one device thread per instance, including the
// test for a second Gram-Schmidt pass, which then runs only over that
// instance's chunks. The whole solve is one CUDA graph, launched once: a
// conditional WHILE node over restart cycles, whose body is a WHILE node over
// the Arnoldi steps (the step index lives on the device) followed by the end
// of the cycle (least squares, x += Z y, the FP64 true residual and the
// convergence flags). Device kernels end each loop when no instance is still
// iterating (steps) or active (cycles); the restart length and the cycle cap
// derived from max_iters bound them. An instance stops contributing once its
// residual estimate meets its target; its later basis vectors are zero.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "amg.cuh"

namespace dpp {

void pc_setup(PcImpl& pc, const ProblemImpl& P, cudaStream_t s);
void pc_apply(const ProblemImpl& P, PcImpl& pc, const double* r, double* z, bool transpose,
              cudaStream_t s);
void pc_apply32(const ProblemImpl& P, PcImpl& pc, const double* r, float* z, bool transpose,
                cudaStream_t s);
void set_last_error_message(const char* m);

namespace {

constexpr int kChunk = 4096;   // vector entries per reduction chunk
constexpr int kSegThreads = 256;

// ------------------------------------------------------------------ union construction
// Cell checks per instance: vertex ids in range, finite log k, and (ids in
// range) a simplex of nonzero measure. Ids are still the instance's own, so
// its vertices are read at the instance's node offset in the union.
__global__ void k_check_instance_cells(const int* __restrict__ cells, int64_t n_cells, int nv,
                                       const int* __restrict__ cell_inst,
                                       const int64_t* __restrict__ inst_nodes,
                                       const int64_t* __restrict__ inst_noff,
                                       const double* __restrict__ X, int dim,
                                       const double* __restrict__ lk1,
                                       const double* __restrict__ lk2, int* __restrict__ flag) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const int b = cell_inst[c];
    int bad = 0;
    for (int v = 0; v < nv; ++v) {
        int a = cells[c * nv + v];
        if (a < 0 || a >= inst_nodes[b]) bad |= kDevBadIndex;
    }
    if (!isfinite(lk1[c]) || !isfinite(lk2[c])) bad |= kDevNonFinite;
    if (!(bad & kDevBadIndex)) {  // det of the edge vectors from vertex 0
        double e[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        const double* x0 = X + (inst_noff[b] + cells[c * nv]) * dim;
        for (int v = 1; v < nv && v <= 3; ++v) {
            const double* xv = X + (inst_noff[b] + cells[c * nv + v]) * dim;
            for (int k = 0; k < dim; ++k) e[v - 1][k] = xv[k] - x0[k];
        }
        const double det = (dim == 2) ? e[0][0] * e[1][1] - e[0][1] * e[1][0]
                                      : e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                                            e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                                            e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
        if (isfinite(det) && !(fabs(det) > 0.0)) bad |= kDevDegenerate;  // NaN: the node check
    }
    if (bad) atomicOr(&flag[b], bad);
}

__global__ void k_check_instance_nodes(const double* __restrict__ X, int64_t n, int dim,
                                       const int* __restrict__ node_inst,
                                       const double* __restrict__ p01,
                                       const double* __restrict__ p02, int* __restrict__ flag) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    bool bad = !isfinite(p01[a]) || !isfinite(p02[a]);
    for (int k = 0; k < dim; ++k) bad |= !isfinite(X[a * dim + k]);
    if (bad) atomicOr(&flag[node_inst[a]], kDevNonFinite);
}

__global__ void k_check_instance_facets(const int* __restrict__ f, int64_t n, int dim,
                                        const int* __restrict__ facet_inst,
                                        const int64_t* __restrict__ inst_nodes,
                                        int* __restrict__ flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = facet_inst[i];
    for (int k = 0; k < dim; ++k) {
        int a = f[i * dim + k];
        if (a < 0 || a >= inst_nodes[b]) atomicOr(&flag[b], kDevBadIndex);
    }
}

__global__ void k_offset_ids(int* __restrict__ ids, int64_t n, int per,
                             const int* __restrict__ owner, const int64_t* __restrict__ off) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n * per) ids[i] += (int)off[owner[i / per]];
}

// instance owning union element e: the last i with off[i] <= e (off[0] = 0)
__device__ __forceinline__ int owner_of(const int64_t* __restrict__ off, int nl, int64_t e) {
    int lo = 0, hi = nl - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Union gather of one input array: element e (comp values each) comes from
// instance i = owner_of(e) at src[i][(e - off[i]) * comp ...]. Instances with
// src[i] == nullptr were copied from host memory by the caller. owner[e] = i
// when owner != nullptr.
template <class T>
__global__ void k_union_gather(int nl, const int64_t* __restrict__ off, int comp,
                               const T* const* __restrict__ src, T* __restrict__ dst,
                               int* __restrict__ owner) {
    const int64_t total = off[nl];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int i = owner_of(off, nl, e);
        if (owner) owner[e] = i;
        const T* sp = src[i];
        if (!sp) continue;
        const int64_t k = e - off[i];
        for (int c = 0; c < comp; ++c) dst[e * comp + c] = sp[k * comp + c];
    }
}

__global__ void k_fill_mub(int64_t n_cells, const int* __restrict__ cell_inst,
                           const double* __restrict__ mu, const double* __restrict__ beta,
                           double* __restrict__ mub) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n_cells) {
        mub[2 * c] = mu[cell_inst[c]];
        mub[2 * c + 1] = beta[cell_inst[c]];
    }
}

// ------------------------------------------------------------------ segmented Krylov kernels
// partial[chunk][j] = sum over the chunk of V_j * w (j < nvec), V row-major [nvec][ld]
// (nvec_dev != nullptr: nvec = *nvec_dev + 1, the Arnoldi step index kept on the device)
template <class VT>
__global__ void __launch_bounds__(kSegThreads)
k_seg_dots(const int64_t* __restrict__ beg, const int64_t* __restrict__ end, const VT* __restrict__ V,
           int64_t ld, int nvec, const double* __restrict__ w, double* __restrict__ partial,
           int pld, const int* __restrict__ inst, const int* __restrict__ run,
           const int* __restrict__ nvec_dev) {
    __shared__ double sh[kSegThreads / 32];
    if (nvec_dev) nvec = *nvec_dev + 1;
    const int c = blockIdx.x;
    if (run && !run[inst[c]]) return;  // this instance skips the pass (its partials are unused)
    const int64_t b0 = beg[c], b1 = end[c];
    for (int j = 0; j < nvec; ++j) {
        const VT* v = V + (int64_t)j * ld;
        double acc = 0.0;
        for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) acc += (double)v[i] * w[i];
        acc = block_sum(acc, sh);
        if (threadIdx.x == 0) partial[(int64_t)c * pld + j] = acc;
    }
}

// out[b][j] = sum over b's chunks (in order) of partial[chunk][j]
__global__ void k_seg_finish(int nb, const int* __restrict__ inst_ch, const double* __restrict__ partial,
                             int pld, int nvec, double* __restrict__ out, int old,
                             const int* __restrict__ run, const int* __restrict__ nvec_dev) {
    if (nvec_dev) nvec = *nvec_dev + 1;
    const int b = blockIdx.x;
    if (b >= nb) return;
    if (run && !run[b]) return;  // out keeps what k_batch_reorth_flags wrote
    for (int j = threadIdx.x; j < nvec; j += blockDim.x) {
        double s = 0.0;
        for (int c = inst_ch[b]; c < inst_ch[b + 1]; ++c) s += partial[(int64_t)c * pld + j];
        out[(int64_t)b * old + j] = s;
    }
}

// w += sign * sum_j coef[b][j] V_j over each chunk (b = the chunk's instance)
template <class VT>
__global__ void __launch_bounds__(kSegThreads)
k_seg_axpy(const int* __restrict__ inst, const int64_t* __restrict__ beg,
           const int64_t* __restrict__ end, const VT* __restrict__ V, int64_t ld, int nvec,
           const double* __restrict__ coef, int cld, double sign, double* __restrict__ w,
           const int* __restrict__ run, const int* __restrict__ nvec_dev = nullptr) {
    __shared__ double cs[64];
    if (nvec_dev) nvec = *nvec_dev + 1;
    const int c = blockIdx.x;
    const int b = inst[c];
    if (run && !run[b]) return;
    if (threadIdx.x < nvec) cs[threadIdx.x] = sign * coef[(int64_t)b * cld + threadIdx.x];
    __syncthreads();
    for (int64_t i = beg[c] + threadIdx.x; i < end[c]; i += blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < nvec; ++j) acc += cs[j] * (double)V[(int64_t)j * ld + i];
        w[i] += acc;
    }
}

// y = x / div[b] (0 where div[b] == 0: the instance is frozen or done)
__global__ void __launch_bounds__(kSegThreads)
k_seg_scale(const int* __restrict__ inst, const int64_t* __restrict__ beg,
            const int64_t* __restrict__ end, const double* __restrict__ x,
            const double* __restrict__ div, double* __restrict__ y) {
    const int c = blockIdx.x;
    const double d = div[inst[c]];
    const double a = (d != 0.0) ? 1.0 / d : 0.0;
    for (int64_t i = beg[c] + threadIdx.x; i < end[c]; i += blockDim.x) y[i] = a * x[i];
}

// V[j + 1] = x / div[b] with j = *jdev (nothing when j + 1 == m)
__global__ void __launch_bounds__(kSegThreads)
k_seg_scale_next(const int* __restrict__ inst, const int64_t* __restrict__ beg,
                 const int64_t* __restrict__ end, const double* __restrict__ x,
                 const double* __restrict__ div, double* __restrict__ V, int64_t ld,
                 const int* __restrict__ jdev, int m) {
    const int j = *jdev;
    if (j + 1 >= m) return;
    const int c = blockIdx.x;
    const double d = div[inst[c]];
    const double a = (d != 0.0) ? 1.0 / d : 0.0;
    double* y = V + (int64_t)(j + 1) * ld;
    for (int64_t i = beg[c] + threadIdx.x; i < end[c]; i += blockDim.x) y[i] = a * x[i];
}

// out = column *jdev of V (V row-major [.][ld]), or column *jdev of Z = in
template <class T>
__global__ void k_take_col(int64_t n, const T* __restrict__ V, int64_t ld, const int* __restrict__ jdev,
                           T* __restrict__ out) {
    const T* v = V + (int64_t)(*jdev) * ld;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = v[i];
}
template <class T>
__global__ void k_put_col(int64_t n, const T* __restrict__ in, T* __restrict__ Z, int64_t ld,
                          const int* __restrict__ jdev) {
    T* z = Z + (int64_t)(*jdev) * ld;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) z[i] = in[i];
}

struct BatchDev {
    double *H, *cs, *sn, *g, *y, *hcol, *hcol2, *nrm2, *hn, *beta, *bnorm, *target, *relres;
    int *ncol, *active, *status, *iters, *n_active;
    double* nrm0;  // ||w||^2 before the first Gram-Schmidt pass
    int* reo;      // per instance: 1 = run the second Gram-Schmidt pass in this iteration
    int* n_iter;   // instances still iterating after the last column (reset every iteration)
};

// Column j of every instance's Hessenberg matrix: rotations, residual estimate,
// freeze test. One thread per instance.
__global__ void k_batch_givens(int nb, int j, int m, BatchDev d, const int* __restrict__ jdev) {
    if (jdev) j = *jdev;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    if (!d.active[b] || d.ncol[b] <= j) {  // done, or frozen earlier in this cycle
        d.hn[b] = 0.0;
        return;
    }
    double* H = d.H + (int64_t)b * (m + 1) * m;
    double* cs = d.cs + (int64_t)b * m;
    double* sn = d.sn + (int64_t)b * m;
    double* g = d.g + (int64_t)b * (m + 1);
    auto h = [&](int i) -> double& { return H[(int64_t)i * m + j]; };
    for (int i = 0; i <= j; ++i) h(i) = d.hcol[(int64_t)b * (m + 2) + i] + d.hcol2[(int64_t)b * (m + 2) + i];
    const double hn = sqrt(fmax(d.nrm2[b], 0.0));
    h(j + 1) = hn;
    for (int i = 0; i < j; ++i) {
        double t = cs[i] * h(i) + sn[i] * h(i + 1);
        h(i + 1) = -sn[i] * h(i) + cs[i] * h(i + 1);
        h(i) = t;
    }
    const double a = h(j), c = h(j + 1);
    const double rr = hypot(a, c);
    cs[j] = (rr > 0) ? a / rr : 1.0;
    sn[j] = (rr > 0) ? c / rr : 0.0;
    h(j) = rr;
    h(j + 1) = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    d.iters[b] += 1;
    const double est = fabs(g[j + 1]);
    if (!isfinite(est) || !isfinite(hn)) {
        d.status[b] = DPP_ERR_NONFINITE;
        d.active[b] = 0;
        d.ncol[b] = j;
        d.hn[b] = 0.0;
        return;
    }
    if (est <= d.target[b] || hn <= 1e-300 * fmax(1.0, rr) || j + 1 == m) {
        d.ncol[b] = j + 1;
        d.hn[b] = 0.0;  // later basis vectors of this instance are zero
    } else {
        d.hn[b] = hn;
        atomicAdd(d.n_iter, 1);
    }
}

// Second Gram-Schmidt pass needed? (DGKS test per instance, against the norm
// before the first pass). hcol2 is zeroed for the instances that skip it.
__global__ void k_batch_reorth_flags(int nb, int j, int pld, double eta2, BatchDev d,
                                     const int* __restrict__ jdev) {
    if (jdev) j = *jdev;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const bool live = d.active[b] && d.ncol[b] > j;
    const int r = (live && d.nrm2[b] < eta2 * d.nrm0[b]) ? 1 : 0;
    d.reo[b] = r;
    if (!r)
        for (int i = 0; i <= j; ++i) d.hcol2[(int64_t)b * pld + i] = 0.0;
}

// y = H^-1 g over the instance's ncol columns (zero for instances that are done)
__global__ void k_batch_lsq(int nb, int m, BatchDev d) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    double* y = d.y + (int64_t)b * m;
    for (int i = 0; i < m; ++i) y[i] = 0.0;
    if (!d.active[b]) return;
    const double* H = d.H + (int64_t)b * (m + 1) * m;
    const double* g = d.g + (int64_t)b * (m + 1);
    const int n = d.ncol[b];
    for (int i = n - 1; i >= 0; --i) {
        double t = g[i];
        for (int k = i + 1; k < n; ++k) t -= H[(int64_t)i * m + k] * y[k];
        y[i] = t / H[(int64_t)i * m + i];
    }
}

// After the true residual: convergence test, next cycle's start values, and
// the count of instances still active.
__global__ void k_batch_check(int nb, int m, double rtol, double inner_rtol, int mixed,
                              int max_iters, BatchDev d) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const double nrm = sqrt(fmax(d.nrm2[b], 0.0));
    const double rel = (d.bnorm[b] > 0) ? nrm / d.bnorm[b] : 0.0;
    d.ncol[b] = m;
    double* g = d.g + (int64_t)b * (m + 1);
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    if (!d.active[b]) {
        d.beta[b] = 0.0;
        return;
    }
    d.relres[b] = rel;
    if (!isfinite(nrm)) {
        d.status[b] = DPP_ERR_NONFINITE;
        d.active[b] = 0;
        d.beta[b] = 0.0;
        return;
    }
    if (rel <= rtol) {
        d.status[b] = DPP_OK;
        d.active[b] = 0;
        d.beta[b] = 0.0;
        return;
    }
    if (d.iters[b] >= max_iters) {
        d.status[b] = DPP_ERR_NOT_CONVERGED;
        d.active[b] = 0;
        d.beta[b] = 0.0;
        return;
    }
    d.beta[b] = nrm;
    g[0] = nrm;
    d.target[b] = mixed ? fmax(inner_rtol * nrm, 0.5 * rtol * d.bnorm[b]) : rtol * d.bnorm[b];
    atomicAdd(d.n_active, 1);
}

// Loop control of the persistent solve graph (one thread). End of an Arnoldi
// step: advance j; repeat while some instance still iterates and j < m.
__global__ void k_iter_advance(int* __restrict__ jdev, const int* __restrict__ n_iter, int m,
                               int* __restrict__ n_steps, cudaGraphConditionalHandle h_iter) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int j = *jdev + 1;
    *jdev = j;
    *n_steps += 1;
    cudaGraphSetConditional(h_iter, (*n_iter > 0 && j < m) ? 1u : 0u);
}
// End of a restart cycle: another cycle while some instance is active and the
// cycle cap (from max_iters) is not reached; the next cycle starts at j = 0.
__global__ void k_cycle_advance(int* __restrict__ jdev, const int* __restrict__ n_active,
                                int* __restrict__ n_cycles, int max_cycles,
                                cudaGraphConditionalHandle h_cycle,
                                cudaGraphConditionalHandle h_iter) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int c = *n_cycles + 1;
    *n_cycles = c;
    *jdev = 0;
    const bool more = *n_active > 0 && c < max_cycles;
    cudaGraphSetConditional(h_cycle, more ? 1u : 0u);
    cudaGraphSetConditional(h_iter, more ? 1u : 0u);
}

__global__ void k_sqrt_copy(int nb, const double* __restrict__ a, double* __restrict__ out) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) out[b] = sqrt(fmax(a[b], 0.0));
}

__global__ void k_batch_init(int nb, BatchDev d) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    d.active[b] = 1;
    d.status[b] = DPP_ERR_NOT_CONVERGED;
    d.iters[b] = 0;
    d.relres[b] = 1.0;
}

inline int g1(int n) { return (n + 127) / 128; }

template <class T>
void upload_at(T* dst, const T* src, size_t n, bool host, cudaStream_t s) {
    if (n) DPP_CK(cudaMemcpyAsync(dst, src, n * sizeof(T),
                                  host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
}

}  // namespace

// Build the union problem from the valid instances. Returns per-instance
// validation codes (0 = ok) in `codes` (host, size n).
void assemble_union(ProblemImpl& P, int n, const dpp_problem_desc* descs, std::vector<int>& codes,
                    cudaStream_t s) {
    codes.assign(n, 0);
    const int dim = descs[0].dim;
    for (int b = 0; b < n; ++b) {
        const dpp_problem_desc& d = descs[b];
        bool ok = d.dim == dim && (d.dim == 2 || d.dim == 3) &&
                  (d.memory == DPP_MEM_DEVICE || d.memory == DPP_MEM_HOST) && d.n_nodes > 0 &&
                  d.n_cells > 0 && d.n_bfacets >= 0 && d.coords && d.cells && d.log_k1 &&
                  d.log_k2 && d.p01 && d.p02 && (d.n_bfacets == 0 || d.bfacets) && d.mu > 0 &&
                  std::isfinite(d.mu) && d.beta >= 0 && std::isfinite(d.beta) &&
                  d.cell_kind == DPP_CELL_SIMPLEX;  // the batched union takes simplices
        for (int k = 0; k < dim && ok; ++k) ok = d.gamma_b[k] == descs[0].gamma_b[k];
        if (!ok) codes[b] = DPP_ERR_INVALID_ARGUMENT;
    }
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<int> live;
        for (int b = 0; b < n; ++b)
            if (!codes[b]) live.push_back(b);
        if (live.empty()) fail(DPP_ERR_INVALID_ARGUMENT, "dpp_solve_batched: no valid instance");
        const int nl = (int)live.size();
        std::vector<int64_t> noff(nl + 1, 0), coff(nl + 1, 0), foff(nl + 1, 0), nnodes(nl);
        for (int i = 0; i < nl; ++i) {
            const auto& d = descs[live[i]];
            noff[i + 1] = noff[i] + d.n_nodes;
            coff[i + 1] = coff[i] + d.n_cells;
            foff[i + 1] = foff[i] + d.n_bfacets;
            nnodes[i] = d.n_nodes;
        }
        if (noff[nl] >= (1LL << 30) || coff[nl] >= (1LL << 30))
            fail(DPP_ERR_INVALID_ARGUMENT, "dpp_solve_batched: union mesh too large for int32 ids");
        P.dim = dim;
        P.n_nodes = noff[nl];
        P.n_cells = coff[nl];
        P.n_bfacets = foff[nl];
        P.mu = 1.0;
        P.beta = 0.0;
        for (int k = 0; k < 3; ++k) P.gb[k] = (k < dim) ? descs[live[0]].gamma_b[k] : 0.0;
        const int nv = dim + 1;
        P.coords.alloc(P.n_nodes * dim);
        P.cells.alloc(P.n_cells * nv);
        P.bfacets.alloc(std::max<int64_t>(P.n_bfacets * dim, 1));
        P.logk1.alloc(P.n_cells);
        P.logk2.alloc(P.n_cells);
        P.p01.alloc(P.n_nodes);
        P.p02.alloc(P.n_nodes);
        P.cell_mu_beta.alloc(2 * P.n_cells);
        DBuf<int> cell_inst(P.n_cells), node_inst(P.n_nodes), facet_inst(std::max<int64_t>(P.n_bfacets, 1));
        DBuf<int64_t> d_nnodes(nl), d_noff(nl);
        DPP_CK(cudaMemcpyAsync(d_nnodes.get(), nnodes.data(), nl * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        DPP_CK(cudaMemcpyAsync(d_noff.get(), noff.data(), nl * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        // Host-memory instances are copied one by one; device-memory instances
        // are gathered by one kernel per array through a table of their
        // pointers, which also writes the owner of every node, cell and facet.
        std::vector<const void*> tab(7 * (size_t)nl, nullptr);  // [array][instance]
        std::vector<double> mu_b(2 * (size_t)nl);
        for (int i = 0; i < nl; ++i) {
            const auto& d = descs[live[i]];
            mu_b[i] = d.mu;
            mu_b[nl + i] = d.beta;
            if (d.memory == DPP_MEM_HOST) {
                upload_at(P.coords.get() + noff[i] * dim, d.coords, (size_t)d.n_nodes * dim, true, s);
                upload_at(P.cells.get() + coff[i] * nv, d.cells, (size_t)d.n_cells * nv, true, s);
                upload_at(P.bfacets.get() + foff[i] * dim, d.bfacets, (size_t)d.n_bfacets * dim, true, s);
                upload_at(P.logk1.get() + coff[i], d.log_k1, (size_t)d.n_cells, true, s);
                upload_at(P.logk2.get() + coff[i], d.log_k2, (size_t)d.n_cells, true, s);
                upload_at(P.p01.get() + noff[i], d.p01, (size_t)d.n_nodes, true, s);
                upload_at(P.p02.get() + noff[i], d.p02, (size_t)d.n_nodes, true, s);
            } else {
                const void* ptrs[7] = {d.coords, d.cells, d.n_bfacets ? d.bfacets : nullptr, d.log_k1,
                                       d.log_k2, d.p01, d.p02};
                for (int a = 0; a < 7; ++a) tab[(size_t)a * nl + i] = ptrs[a];
            }
        }
        DBuf<int64_t> d_off(3 * ((size_t)nl + 1));  // node, cell, facet offsets
        DBuf<const void*> d_tab(tab.size());
        DBuf<double> d_mub(mu_b.size());
        DPP_CK(cudaMemcpyAsync(d_off.get(), noff.data(), (nl + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        DPP_CK(cudaMemcpyAsync(d_off.get() + (nl + 1), coff.data(), (nl + 1) * sizeof(int64_t),
                               cudaMemcpyHostToDevice, s));
        DPP_CK(cudaMemcpyAsync(d_off.get() + 2 * (nl + 1), foff.data(), (nl + 1) * sizeof(int64_t),
                               cudaMemcpyHostToDevice, s));
        DPP_CK(cudaMemcpyAsync(d_tab.get(), tab.data(), tab.size() * sizeof(void*), cudaMemcpyHostToDevice, s));
        DPP_CK(cudaMemcpyAsync(d_mub.get(), mu_b.data(), mu_b.size() * sizeof(double),
                               cudaMemcpyHostToDevice, s));
        const int64_t* o_node = d_off.get();
        const int64_t* o_cell = d_off.get() + (nl + 1);
        const int64_t* o_facet = d_off.get() + 2 * (nl + 1);
        auto dtab = [&](int a) { return reinterpret_cast<const double* const*>(d_tab.get() + (size_t)a * nl); };
        auto itab = [&](int a) { return reinterpret_cast<const int* const*>(d_tab.get() + (size_t)a * nl); };
        const int gb = 8 * kSMs;
        k_union_gather<double><<<gb, 256, 0, s>>>(nl, o_node, dim, dtab(0), P.coords.get(), node_inst.get());
        DPP_LAUNCH_CK();
        k_union_gather<int><<<gb, 256, 0, s>>>(nl, o_cell, nv, itab(1), P.cells.get(), cell_inst.get());
        DPP_LAUNCH_CK();
        if (P.n_bfacets) {
            k_union_gather<int><<<gb, 256, 0, s>>>(nl, o_facet, dim, itab(2), P.bfacets.get(), facet_inst.get());
            DPP_LAUNCH_CK();
        }
        k_union_gather<double><<<gb, 256, 0, s>>>(nl, o_cell, 1, dtab(3), P.logk1.get(), nullptr);
        DPP_LAUNCH_CK();
        k_union_gather<double><<<gb, 256, 0, s>>>(nl, o_cell, 1, dtab(4), P.logk2.get(), nullptr);
        DPP_LAUNCH_CK();
        k_union_gather<double><<<gb, 256, 0, s>>>(nl, o_node, 1, dtab(5), P.p01.get(), nullptr);
        DPP_LAUNCH_CK();
        k_union_gather<double><<<gb, 256, 0, s>>>(nl, o_node, 1, dtab(6), P.p02.get(), nullptr);
        DPP_LAUNCH_CK();
        k_fill_mub<<<grid_for(P.n_cells, 256), 256, 0, s>>>(P.n_cells, cell_inst.get(), d_mub.get(),
                                                            d_mub.get() + nl, P.cell_mu_beta.get());
        DPP_LAUNCH_CK();
        // per-instance validation before the ids are shifted
        DBuf<int> flags(nl);
        DPP_CK(cudaMemsetAsync(flags.get(), 0, nl * sizeof(int), s));
        k_check_instance_cells<<<grid_for(P.n_cells, 256), 256, 0, s>>>(
            P.cells.get(), P.n_cells, nv, cell_inst.get(), d_nnodes.get(), d_noff.get(), P.coords.get(), dim,
            P.logk1.get(), P.logk2.get(), flags.get());
        DPP_LAUNCH_CK();
        k_check_instance_nodes<<<grid_for(P.n_nodes, 256), 256, 0, s>>>(
            P.coords.get(), P.n_nodes, dim, node_inst.get(), P.p01.get(), P.p02.get(), flags.get());
        DPP_LAUNCH_CK();
        if (P.n_bfacets) {
            k_check_instance_facets<<<grid_for(P.n_bfacets, 256), 256, 0, s>>>(
                P.bfacets.get(), P.n_bfacets, dim, facet_inst.get(), d_nnodes.get(), flags.get());
            DPP_LAUNCH_CK();
        }
        std::vector<int> hf(nl);
        DPP_CK(cudaMemcpyAsync(hf.data(), flags.get(), nl * sizeof(int), cudaMemcpyDeviceToHost, s));
        DPP_CK(cudaStreamSynchronize(s));
        bool any_bad = false;
        for (int i = 0; i < nl; ++i)
            if (hf[i]) {
                codes[live[i]] = (hf[i] & (kDevBadIndex | kDevDegenerate)) ? DPP_ERR_INVALID_ARGUMENT
                                                                           : DPP_ERR_NONFINITE;
                any_bad = true;
            }
        if (any_bad) {
            if (pass == 1) fail(DPP_ERR_INVALID_ARGUMENT, "dpp_solve_batched: validation did not settle");
            continue;  // rebuild without the rejected instances
        }
        k_offset_ids<<<grid_for(P.n_cells * nv, 256), 256, 0, s>>>(P.cells.get(), P.n_cells, nv,
                                                                   cell_inst.get(), d_noff.get());
        DPP_LAUNCH_CK();
        if (P.n_bfacets) {
            k_offset_ids<<<grid_for(P.n_bfacets * dim, 256), 256, 0, s>>>(
                P.bfacets.get(), P.n_bfacets, dim, facet_inst.get(), d_noff.get());
            DPP_LAUNCH_CK();
        }
        P.n_inst = nl;
        P.inst_node_off = noff;
        P.inst_cell_off = coff;
        P.inst_mu.resize(nl);
        P.inst_beta.resize(nl);
        for (int i = 0; i < nl; ++i) {
            P.inst_mu[i] = descs[live[i]].mu;
            P.inst_beta[i] = descs[live[i]].beta;
        }
        assemble_uploaded(P, s);
        return;
    }
}

// Lock-step FGMRES over the instances of a union problem. Per-instance results
// go to status/iters/relres (host vectors, size n_inst).
void fgmres_batched(const ProblemImpl& P, PcImpl& pc, const dpp_solve_opts& o, double* x,
                    std::vector<int>& status, std::vector<int>& iters,
                    std::vector<double>& relres, int64_t& graph_launches, cudaStream_t s,
                    HostScratch& hs) {
    const int nb = P.n_inst;
    const int64_t n = P.n_nodes * P.ns;
    const int m = std::min(std::max(o.restart, 1), 62);
    const bool mixed = pc.precision == DPP_MIXED_FP32_FP64;
    // chunk table over vector entries
    std::vector<int64_t> cb, ce;
    std::vector<int> ci, ich(nb + 1, 0);
    for (int b = 0; b < nb; ++b) {
        const int64_t e0 = P.inst_node_off[b] * P.ns, e1 = P.inst_node_off[b + 1] * P.ns;
        ich[b] = (int)cb.size();
        for (int64_t e = e0; e < e1; e += kChunk) {
            cb.push_back(e);
            ce.push_back(std::min<int64_t>(e + kChunk, e1));
            ci.push_back(b);
        }
    }
    ich[nb] = (int)cb.size();
    const int nch = (int)cb.size();
    DBuf<int64_t> d_cb(nch), d_ce(nch);
    DBuf<int> d_ci(nch), d_ich(nb + 1);
    DPP_CK(cudaMemcpyAsync(d_cb.get(), cb.data(), nch * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    DPP_CK(cudaMemcpyAsync(d_ce.get(), ce.data(), nch * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    DPP_CK(cudaMemcpyAsync(d_ci.get(), ci.data(), nch * sizeof(int), cudaMemcpyHostToDevice, s));
    DPP_CK(cudaMemcpyAsync(d_ich.get(), ich.data(), (nb + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
    const int pld = m + 2;
    DBuf<double> V((size_t)(m + 1) * n), Z(mixed ? 1 : (size_t)m * n), w(n), r(n), partial((size_t)nch * pld);
    DBuf<float> Z32(mixed ? (size_t)m * n : 1);
    // A cycle that ends early leaves later columns of Z from an earlier cycle
    // (zero coefficients in x += Z y); they start at zero so that they are finite.
    if (mixed) DPP_CK(cudaMemsetAsync(Z32.get(), 0, Z32.bytes(), s));
    else DPP_CK(cudaMemsetAsync(Z.get(), 0, Z.bytes(), s));
    DBuf<double> H((size_t)nb * (m + 1) * m), cs((size_t)nb * m), sn((size_t)nb * m), g((size_t)nb * (m + 1)),
        y((size_t)nb * m), hcol((size_t)nb * pld), hcol2((size_t)nb * pld), nrm2(nb), hn(nb), beta(nb),
        bnorm(nb), target(nb), rel(nb);
    DBuf<int> ncol(nb), active(nb), st(nb), it(nb), n_active(1), reo(nb), n_iter(1);
    DBuf<double> nrm0(nb);
    BatchDev d{H.get(), cs.get(), sn.get(), g.get(), y.get(), hcol.get(), hcol2.get(), nrm2.get(),
               hn.get(), beta.get(), bnorm.get(), target.get(), rel.get(), ncol.get(), active.get(),
               st.get(), it.get(), n_active.get(), nrm0.get(), reo.get(), n_iter.get()};
    const double* f = P.f.get();
    auto seg_dot = [&](const double* Vv, int64_t ld, int nvec, const double* wv, double* out, int old,
                       const int* run, const int* nvec_dev = nullptr) {
        k_seg_dots<double><<<nch, kSegThreads, 0, s>>>(d_cb.get(), d_ce.get(), Vv, ld, nvec, wv,
                                                       partial.get(), pld, d_ci.get(), run, nvec_dev);
        DPP_LAUNCH_CK();
        k_seg_finish<<<nb, 64, 0, s>>>(nb, d_ich.get(), partial.get(), pld, nvec, out, old, run,
                                       nvec_dev);
        DPP_LAUNCH_CK();
    };
    // ||f_b||, initial x, residual and flags
    seg_dot(f, 0, 1, f, nrm2.get(), 1, nullptr);
    k_sqrt_copy<<<g1(nb), 128, 0, s>>>(nb, nrm2.get(), bnorm.get());
    DPP_LAUNCH_CK();
    if (o.x0_zero) DPP_CK(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    k_batch_init<<<g1(nb), 128, 0, s>>>(nb, d);
    DPP_LAUNCH_CK();
    auto tail = [&]() {  // true residual, convergence test, v_0 of the next cycle
        apply_K(P, x, r.get(), f, false, false, s);
        seg_dot(r.get(), 0, 1, r.get(), nrm2.get(), 1, nullptr);
        DPP_CK(cudaMemsetAsync(n_active.get(), 0, sizeof(int), s));
        k_batch_check<<<g1(nb), 128, 0, s>>>(nb, m, o.rtol, o.inner_rtol, mixed ? 1 : 0, o.max_iters, d);
        DPP_LAUNCH_CK();
        k_seg_scale<<<nch, kSegThreads, 0, s>>>(d_ci.get(), d_cb.get(), d_ce.get(), r.get(), beta.get(), V.get());
        DPP_LAUNCH_CK();
    };
    tail();
    const double eta = std::min(std::max(o.reorth_eta, 0.0), 1.0);
    // Loop state on the device: the Arnoldi step j of the current cycle, and
    // counters of the steps and cycles run (for the launch accounting).
    DBuf<int> loop(3);  // [0] j, [1] steps run, [2] cycles run
    int* jdev = loop.get();
    DPP_CK(cudaMemsetAsync(loop.get(), 0, 3 * sizeof(int), s));
    // The preconditioner and K read and write fixed vectors; column j of V is
    // copied in and the preconditioned vector copied out to column j of Z.
    DBuf<double> vcur(n), zcur(mixed ? 1 : n);
    DBuf<float> zcur32(mixed ? n : 1);
    const int cgrid = (int)std::min<int64_t>((n + 255) / 256, 8 * kSMs);
    // Arnoldi step j = *jdev for every instance: classical Gram-Schmidt, and a
    // second pass for the instances whose first pass left less than eta of ||w||
    auto iteration = [&](cudaGraphConditionalHandle h_iter) {
        k_take_col<double><<<cgrid, 256, 0, s>>>(n, V.get(), n, jdev, vcur.get());
        DPP_LAUNCH_CK();
        if (mixed) {
            pc_apply32(P, pc, vcur.get(), zcur32.get(), false, s);
            k_put_col<float><<<cgrid, 256, 0, s>>>(n, zcur32.get(), Z32.get(), n, jdev);
            DPP_LAUNCH_CK();
            apply_K32(P, zcur32.get(), w.get(), false, s);
        } else {
            pc_apply(P, pc, vcur.get(), zcur.get(), false, s);
            k_put_col<double><<<cgrid, 256, 0, s>>>(n, zcur.get(), Z.get(), n, jdev);
            DPP_LAUNCH_CK();
            apply_K(P, zcur.get(), w.get(), nullptr, false, false, s);
        }
        seg_dot(w.get(), 0, 1, w.get(), nrm0.get(), 1, nullptr);
        seg_dot(V.get(), n, 1, w.get(), hcol.get(), pld, nullptr, jdev);
        k_seg_axpy<double><<<nch, kSegThreads, 0, s>>>(d_ci.get(), d_cb.get(), d_ce.get(), V.get(), n, 1,
                                                       hcol.get(), pld, -1.0, w.get(), nullptr, jdev);
        DPP_LAUNCH_CK();
        seg_dot(w.get(), 0, 1, w.get(), nrm2.get(), 1, nullptr);
        k_batch_reorth_flags<<<g1(nb), 128, 0, s>>>(nb, 0, pld, eta * eta, d, jdev);
        DPP_LAUNCH_CK();
        seg_dot(V.get(), n, 1, w.get(), hcol2.get(), pld, reo.get(), jdev);
        k_seg_axpy<double><<<nch, kSegThreads, 0, s>>>(d_ci.get(), d_cb.get(), d_ce.get(), V.get(), n, 1,
                                                       hcol2.get(), pld, -1.0, w.get(), reo.get(), jdev);
        DPP_LAUNCH_CK();
        seg_dot(w.get(), 0, 1, w.get(), nrm2.get(), 1, reo.get());
        DPP_CK(cudaMemsetAsync(n_iter.get(), 0, sizeof(int), s));
        k_batch_givens<<<g1(nb), 128, 0, s>>>(nb, 0, m, d, jdev);
        DPP_LAUNCH_CK();
        k_seg_scale_next<<<nch, kSegThreads, 0, s>>>(d_ci.get(), d_cb.get(), d_ce.get(), w.get(), hn.get(),
                                                     V.get(), n, jdev, m);
        DPP_LAUNCH_CK();
        k_iter_advance<<<1, 32, 0, s>>>(jdev, n_iter.get(), m, loop.get() + 1, h_iter);
        DPP_LAUNCH_CK();
    };
    const int max_cycles = (o.max_iters + m - 1) / m + 1;
    auto finish = [&](cudaGraphConditionalHandle h_cycle, cudaGraphConditionalHandle h_iter) {
        k_batch_lsq<<<g1(nb), 128, 0, s>>>(nb, m, d);  // least squares, x += Z y, true residual, test
        DPP_LAUNCH_CK();
        if (mixed)
            k_seg_axpy<float><<<nch, kSegThreads, 0, s>>>(d_ci.get(), d_cb.get(), d_ce.get(), Z32.get(), n, m,
                                                          y.get(), m, 1.0, x, nullptr);
        else
            k_seg_axpy<double><<<nch, kSegThreads, 0, s>>>(d_ci.get(), d_cb.get(), d_ce.get(), Z.get(), n, m,
                                                           y.get(), m, 1.0, x, nullptr);
        DPP_LAUNCH_CK();
        tail();
        k_cycle_advance<<<1, 32, 0, s>>>(jdev, n_active.get(), loop.get() + 2, max_cycles, h_cycle,
                                         h_iter);
        DPP_LAUNCH_CK();
    };
    // The whole solve is one CUDA graph: a WHILE node over restart cycles whose
    // body is a WHILE node over Arnoldi steps followed by the end of the
    // cycle. The device ends each loop (cudaGraphSetConditional) when no
    // instance is still iterating or active; the iteration and cycle caps
    // bound both. The host launches the graph once and waits once.
    struct GraphGuard {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t e = nullptr;
        ~GraphGuard() {
            if (e) cudaGraphExecDestroy(e);
            if (g) cudaGraphDestroy(g);
        }
    } G;
    auto capture_into = [&](cudaGraph_t target, const cudaGraphNode_t* deps, size_t ndeps,
                            auto&& body) {
        DPP_CK(cudaStreamBeginCaptureToGraph(s, target, deps, nullptr, ndeps,
                                             cudaStreamCaptureModeThreadLocal));
        try {
            body();
        } catch (...) {
            cudaGraph_t tmp = nullptr;
            cudaStreamEndCapture(s, &tmp);
            throw;
        }
        cudaGraph_t out = nullptr;
        DPP_CK(cudaStreamEndCapture(s, &out));
    };
    auto while_node = [&](cudaGraph_t parent, cudaGraphConditionalHandle h, cudaGraphNode_t* node,
                          cudaGraph_t* body) {
        cudaGraphNodeParams prm{};
        prm.type = cudaGraphNodeTypeConditional;
        prm.conditional.handle = h;
        prm.conditional.type = cudaGraphCondTypeWhile;
        prm.conditional.size = 1;
        DPP_CK(cudaGraphAddNode(node, parent, nullptr, nullptr, 0, &prm));
        *body = prm.conditional.phGraph_out[0];
    };
    int active_now = read_scalar(n_active.get(), s, hs);
    if (active_now > 0) {
        // host time of building the graph (the device is idle meanwhile)
        ProfScope pg("batched_graph_build", s, 0);
        DPP_CK(cudaGraphCreate(&G.g, 0));
        cudaGraphConditionalHandle h_cycle, h_iter;
        DPP_CK(cudaGraphConditionalHandleCreate(&h_cycle, G.g, 1, cudaGraphCondAssignDefault));
        cudaGraphNode_t w_cycle, w_iter;
        cudaGraph_t body_cycle, body_iter;
        while_node(G.g, h_cycle, &w_cycle, &body_cycle);
        DPP_CK(cudaGraphConditionalHandleCreate(&h_iter, body_cycle, 1, cudaGraphCondAssignDefault));
        while_node(body_cycle, h_iter, &w_iter, &body_iter);
        capture_into(body_iter, nullptr, 0, [&]() { iteration(h_iter); });
        capture_into(body_cycle, &w_iter, 1, [&]() { finish(h_cycle, h_iter); });
        DPP_CK(cudaGraphInstantiate(&G.e, G.g, 0));
        pg.stop();
        DPP_CK(cudaGraphLaunch(G.e, s));
        size_t n_iter_nodes = 0, n_cycle_nodes = 0;
        DPP_CK(cudaGraphGetNodes(body_iter, nullptr, &n_iter_nodes));
        DPP_CK(cudaGraphGetNodes(body_cycle, nullptr, &n_cycle_nodes));
        int counts[3];
        DPP_CK(cudaMemcpyAsync(counts, loop.get(), 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
        DPP_CK(cudaStreamSynchronize(s));
        graph_launches += (int64_t)counts[1] * (int64_t)n_iter_nodes +
                          (int64_t)counts[2] * (int64_t)(n_cycle_nodes - 1);
    }
    status.resize(nb);
    iters.resize(nb);
    relres.resize(nb);
    DPP_CK(cudaMemcpyAsync(status.data(), st.get(), nb * sizeof(int), cudaMemcpyDeviceToHost, s));
    DPP_CK(cudaMemcpyAsync(iters.data(), it.get(), nb * sizeof(int), cudaMemcpyDeviceToHost, s));
    DPP_CK(cudaMemcpyAsync(relres.data(), rel.get(), nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    DPP_CK(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------------ schedule autotuner
// The preconditioner schedule of the batched solve: the AMG Chebyshev degree
// (finest level, then the coarser levels), the AMG Chebyshev interval ratio
// and the mass Chebyshev degree. None of them changes the setup (aggregates,
// Galerkin products, lambda_max), so the candidates are timed as full batched
// solves on the one hierarchy already built, by a coordinate search from the
// given schedule: the AMG degree in {1, 2, 3}, the coarse-level degree in
// {1, 2, 3}, the ratio in {10, 20, 30}, then the mass degree in {1, 2, 3}. A candidate that leaves an instance unconverged is dropped. The
// choice is cached for the process per size class (dimension, precision,
// log2 of the union's nodes, log2 of the mean nodes per instance); if
// DPP_TUNE_CACHE names a file, choices are read from it and new ones appended.
namespace {
struct SchedKey {
    int dim, fp32, log2_nodes, log2_mean;
    bool operator<(const SchedKey& o) const {
        return std::tie(dim, fp32, log2_nodes, log2_mean) <
               std::tie(o.dim, o.fp32, o.log2_nodes, o.log2_mean);
    }
};
struct Sched {
    int amg, mass;
    double ratio;
    int coarse;  // 0: the AMG degree on every level
};
std::mutex g_sched_mu;
std::map<SchedKey, Sched> g_sched;
bool g_sched_loaded = false;

int ilog2(int64_t v) {
    int r = 0;
    while (v > 1) { v >>= 1; ++r; }
    return r;
}

void sched_load_locked() {
    if (g_sched_loaded) return;
    g_sched_loaded = true;
    const char* path = std::getenv("DPP_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char line[256];
    while (std::fgets(line, sizeof line, f)) {
        SchedKey k;
        Sched v;
        if (std::sscanf(line,
                        "{\"schedule\": 2, \"dim\": %d, \"fp32\": %d, \"log2_nodes\": %d, "
                        "\"log2_mean\": %d, \"amg\": %d, \"coarse\": %d, \"mass\": %d, \"ratio\": %lf}",
                        &k.dim, &k.fp32, &k.log2_nodes, &k.log2_mean, &v.amg, &v.coarse, &v.mass,
                        &v.ratio) == 8 &&
            v.amg >= 1 && v.amg <= 16 && v.coarse >= 0 && v.coarse <= 16 && v.mass >= 1 &&
            v.mass <= 16 && v.ratio > 1)
            g_sched[k] = v;
    }
    std::fclose(f);
}

void sched_store_locked(const SchedKey& k, const Sched& v) {
    g_sched[k] = v;
    const char* path = std::getenv("DPP_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"schedule\": 2, \"dim\": %d, \"fp32\": %d, \"log2_nodes\": %d, "
                 "\"log2_mean\": %d, \"amg\": %d, \"coarse\": %d, \"mass\": %d, \"ratio\": %g}\n",
                 k.dim, k.fp32, k.log2_nodes, k.log2_mean, v.amg, v.coarse, v.mass, v.ratio);
    std::fclose(f);
}
}  // namespace

void tune_batched_schedule(const ProblemImpl& P, PcImpl& pc, const dpp_solve_opts& o,
                           cudaStream_t s, HostScratch& hs) {
    ProfScope pr("setup_schedule_tune", s, 0);
    SchedKey key{P.dim, pc.precision == DPP_MIXED_FP32_FP64 ? 1 : 0, ilog2(P.n_nodes),
                 ilog2(P.n_nodes / std::max(P.n_inst, 1))};
    {
        std::lock_guard<std::mutex> lk(g_sched_mu);
        sched_load_locked();
        auto it = g_sched.find(key);
        if (it != g_sched.end()) {
            pc.opts.cheb_degree_amg = it->second.amg;
            pc.opts.cheb_degree_coarse = it->second.coarse;
            pc.opts.cheb_degree_mass = it->second.mass;
            pc.opts.cheb_ratio = it->second.ratio;
            return;
        }
    }
    dpp_solve_opts t = o;
    t.x0_zero = 1;
    DBuf<double> xt(P.n_nodes * P.ns);
    cudaEvent_t e0, e1;
    DPP_CK(cudaEventCreate(&e0));
    DPP_CK(cudaEventCreate(&e1));
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } eg{e0, e1};
    std::map<std::tuple<int, int, int, double>, float> seen;
    auto trial = [&](const Sched& c) -> float {
        auto k = std::make_tuple(c.amg, c.coarse ? c.coarse : c.amg, c.mass, c.ratio);
        auto f = seen.find(k);
        if (f != seen.end()) return f->second;
        pc.opts.cheb_degree_amg = c.amg;
        pc.opts.cheb_degree_coarse = c.coarse;
        pc.opts.cheb_degree_mass = c.mass;
        pc.opts.cheb_ratio = c.ratio;
        std::vector<int> st, it;
        std::vector<double> rr;
        int64_t launches = 0;
        DPP_CK(cudaEventRecord(e0, s));
        fgmres_batched(P, pc, t, xt.get(), st, it, rr, launches, s, hs);
        DPP_CK(cudaEventRecord(e1, s));
        DPP_CK(cudaEventSynchronize(e1));
        for (int64_t q = 0; q < launches; ++q) count_launch();
        float ms = 0;
        DPP_CK(cudaEventElapsedTime(&ms, e0, e1));
        for (int v : st)
            if (v != DPP_OK) ms = 1e30f;  // a candidate must converge every instance
        seen[k] = ms;
        return ms;
    };
    Sched best{pc.opts.cheb_degree_amg, pc.opts.cheb_degree_mass, pc.opts.cheb_ratio,
               pc.opts.cheb_degree_coarse};
    float best_ms = trial(best);
    for (int a : {1, 2, 3}) {
        Sched c = best;
        c.amg = a;
        const float ms = trial(c);
        if (ms < best_ms) { best_ms = ms; best = c; }
    }
    for (int a : {1, 2, 3}) {
        Sched c = best;
        c.coarse = a;
        const float ms = trial(c);
        if (ms < best_ms) { best_ms = ms; best = c; }
    }
    for (double r : {10.0, 20.0, 30.0}) {
        Sched c = best;
        c.ratio = r;
        const float ms = trial(c);
        if (ms < best_ms) { best_ms = ms; best = c; }
    }
    for (int m : {1, 2, 3}) {
        Sched c = best;
        c.mass = m;
        const float ms = trial(c);
        if (ms < best_ms) { best_ms = ms; best = c; }
    }
    pc.opts.cheb_degree_amg = best.amg;
    pc.opts.cheb_degree_coarse = best.coarse;
    pc.opts.cheb_degree_mass = best.mass;
    pc.opts.cheb_ratio = best.ratio;
    std::lock_guard<std::mutex> lk(g_sched_mu);
    sched_store_locked(key, best);
}

}  // namespace dpp
