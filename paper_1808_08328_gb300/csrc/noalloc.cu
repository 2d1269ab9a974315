// dpp_adjoint_gradients_noalloc: the per-cell adjoint sensitivities with no
// device allocation.
//
// Who needs this: callers that run the gradient step inside device memory
// that another framework owns. Examples are a custom call inside an
// XLA/JAX or TensorFlow graph, or an optimisation loop that a serving process
// replays under a fixed memory budget. In those settings cudaMalloc and
// cudaFree are off limits. They synchronise the whole device, they bypass the
// host framework's pool and its accounting, and they can fail or stall once
// that pool has reserved the memory. dpp_adjoint_solve allocates its scratch
// (a per-cell buffer for the beta term and the reduction partials) for every
// call. This variant computes the same three outputs with scratch that lives
// in one fixed array of this file, loaded with the library.
//
// Scratch: g_noalloc_partials, kNoAllocMaxBlocks doubles (128 KiB) per GPU
// that loads the library, held until the process exits. Pass 1 writes one
// partial sum of the beta term per block of kNoAllocThreads cells. Pass 2
// (one block) adds the partials in block order. Every call writes all the
// partials it reads before reading them, so nothing has to start at zero.
// Calls that overlap on the GPU (on different streams, or from different
// threads without ordering) share the array and race. Order them on one
// stream.
//
// Limit: n_cells <= kNoAllocMaxBlocks * kNoAllocThreads = 4,194,304 cells.
// Larger problems are rejected with DPP_ERR_INVALID_ARGUMENT.
#include <mutex>

#include "kernels.cuh"

namespace dpp {
void set_last_error_message(const char* m);
}

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocMaxBlocks = 16384;
constexpr int64_t kNoAllocMaxCells = (int64_t)kNoAllocMaxBlocks * kNoAllocThreads;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks];

// Same cell formula as the allocating path: with the CG-VMS form,
//   dJ/dlog k_i,c = -lambda^T (dK/dlog k_i,c x - df/dlog k_i,c), where the derivative is
//   -1/2 mu/k_i M_c (velocity block), +1/2 k_i/mu L_c (pressure block) and
//   +1/2 k_i/mu |K| g_a.gamma_b (load);
//   dJ/dbeta = -(1/mu) sum_c (lambda_p1 - lambda_p2)^T M_c (x_p1 - x_p2).
template <int DIM>
__global__ void __launch_bounds__(kNoAllocThreads)
k_cell_sensitivity_partials(int64_t n_cells, const int* __restrict__ cells,
                            const double* __restrict__ geo, const double* __restrict__ kk,
                            const double* __restrict__ x, const double* __restrict__ lam, double mu,
                            double gb0, double gb1, double gb2, double* __restrict__ g1,
                            double* __restrict__ g2, double* __restrict__ partials) {
    constexpr int S = dpp::GeoLayout<DIM>::stride;
    constexpr int NS = 2 * DIM + 2;
    constexpr int NV = DIM + 1;
    __shared__ double sh[kNoAllocThreads / 32];
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double beta_term = 0.0;
    if (c < n_cells) {
        const double gbv[3] = {gb0, gb1, gb2};
        int v[NV];
#pragma unroll
        for (int a = 0; a < NV; ++a) v[a] = cells[c * NV + a];
        const double* g = geo + c * S;
        const double vol = g[0];
        const double k1 = kk[2 * c], k2 = kk[2 * c + 1];
        const double cm = vol / ((DIM + 1) * (DIM + 2));
        double mu1 = 0, mu2 = 0, lp1 = 0, lp2 = 0, f1 = 0, f2 = 0, mb = 0;
#pragma unroll
        for (int a = 0; a < NV; ++a) {
            const double* la = lam + (int64_t)v[a] * NS;
            const double* ga = g + 1 + a * DIM;
            double gdot = 0;
#pragma unroll
            for (int k = 0; k < DIM; ++k) gdot += ga[k] * gbv[k];
            f1 += la[DIM] * gdot;
            f2 += la[2 * DIM + 1] * gdot;
#pragma unroll
            for (int b = 0; b < NV; ++b) {
                const double* xb = x + (int64_t)v[b] * NS;
                const double* gbb = g + 1 + b * DIM;
                const double m = cm * (a == b ? 2.0 : 1.0);
                double lg = 0, uu1 = 0, uu2 = 0;
#pragma unroll
                for (int k = 0; k < DIM; ++k) {
                    lg += ga[k] * gbb[k];
                    uu1 += la[k] * xb[k];
                    uu2 += la[DIM + 1 + k] * xb[DIM + 1 + k];
                }
                mu1 += m * uu1;
                mu2 += m * uu2;
                lp1 += vol * lg * la[DIM] * xb[DIM];
                lp2 += vol * lg * la[2 * DIM + 1] * xb[2 * DIM + 1];
                mb += m * (la[DIM] - la[2 * DIM + 1]) * (xb[DIM] - xb[2 * DIM + 1]);
            }
        }
        const double t1 = -0.5 * mu / k1 * mu1 + 0.5 * k1 / mu * lp1 - 0.5 * k1 / mu * vol * f1;
        const double t2 = -0.5 * mu / k2 * mu2 + 0.5 * k2 / mu * lp2 - 0.5 * k2 / mu * vol * f2;
        g1[c] = -t1;
        g2[c] = -t2;
        beta_term = -mb / mu;
    }
    const double s = dpp::block_sum(beta_term, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kNoAllocThreads)
k_sum_partials(const double* __restrict__ partials, int n, double* __restrict__ out) {
    __shared__ double sh[kNoAllocThreads / 32];
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) v += partials[k];
    v = dpp::block_sum(v, sh);
    if (threadIdx.x == 0) *out = v;
}

// Device address of g_noalloc_partials, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
double* g_addr[kMaxDevices] = {};

cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

dpp_status report(dpp_status s, const char* m) {
    dpp::set_last_error_message(m);
    return s;
}

}  // namespace

extern "C" dpp_status dpp_adjoint_gradients_noalloc(dpp_problem prob, const double* x,
                                                   const double* lambda, double* dJ_dlogk1,
                                                   double* dJ_dlogk2, double* dJ_dbeta,
                                                   dpp_stream_t stream) {
    if (!prob || !x || !lambda || !dJ_dlogk1 || !dJ_dlogk2 || !dJ_dbeta)
        return report(DPP_ERR_INVALID_ARGUMENT, "dpp_adjoint_gradients_noalloc: null argument");
    const dpp::ProblemImpl& P = prob->impl;
    if (P.n_cells > kNoAllocMaxCells)
        return report(DPP_ERR_INVALID_ARGUMENT,
                      "dpp_adjoint_gradients_noalloc: n_cells exceeds the fixed scratch limit of "
                      "4194304 cells (use dpp_adjoint_solve for larger meshes)");
    double* partials = nullptr;
    cudaError_t e = scratch_address(&partials);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return report(DPP_ERR_CUDA, "dpp_adjoint_gradients_noalloc: cudaGetSymbolAddress failed");
    }
    const int nblk = (int)((P.n_cells + kNoAllocThreads - 1) / kNoAllocThreads);
    cudaStream_t s = (cudaStream_t)stream;
    if (P.dim == 2)
        k_cell_sensitivity_partials<2><<<nblk, kNoAllocThreads, 0, s>>>(
            P.n_cells, P.cells.get(), P.geo.get(), P.kk.get(), x, lambda, P.mu, P.gb[0], P.gb[1],
            P.gb[2], dJ_dlogk1, dJ_dlogk2, partials);
    else
        k_cell_sensitivity_partials<3><<<nblk, kNoAllocThreads, 0, s>>>(
            P.n_cells, P.cells.get(), P.geo.get(), P.kk.get(), x, lambda, P.mu, P.gb[0], P.gb[1],
            P.gb[2], dJ_dlogk1, dJ_dlogk2, partials);
    e = cudaGetLastError();
    if (e != cudaSuccess) return report(DPP_ERR_CUDA, "dpp_adjoint_gradients_noalloc: launch failed");
    dpp::count_launch();
    k_sum_partials<<<1, kNoAllocThreads, 0, s>>>(partials, nblk, dJ_dbeta);
    e = cudaGetLastError();
    if (e != cudaSuccess) return report(DPP_ERR_CUDA, "dpp_adjoint_gradients_noalloc: launch failed");
    dpp::count_launch();
    return DPP_OK;
}
