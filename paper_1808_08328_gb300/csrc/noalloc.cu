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

// The per-cell formula is dpp::cell_sensitivity, the one the allocating path
// uses; only the reduction of the beta term differs (block partials here).
template <int DIM>
__global__ void __launch_bounds__(kNoAllocThreads)
k_cell_sensitivity_partials(int64_t n_cells, const int* __restrict__ cells,
                            const double* __restrict__ geo, const double* __restrict__ kk,
                            const double* __restrict__ x, const double* __restrict__ lam, double mu,
                            double gb0, double gb1, double gb2, double* __restrict__ g1,
                            double* __restrict__ g2, double* __restrict__ partials) {
    __shared__ double sh[kNoAllocThreads / 32];
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double beta_term = 0.0;
    if (c < n_cells) {
        const double gbv[3] = {gb0, gb1, gb2};
        double t1, t2;
        dpp::cell_sensitivity<DIM>(c, cells, geo, kk, x, lam, mu, gbv, t1, t2, beta_term);
        g1[c] = t1;
        g2[c] = t2;
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
    // Like every other entry point: the thread-local message is cleared on
    // entry, and no exception leaves the library.
    dpp::set_last_error_message("");
    try {
        if (!prob || !x || !lambda || !dJ_dlogk1 || !dJ_dlogk2 || !dJ_dbeta)
            return report(DPP_ERR_INVALID_ARGUMENT, "dpp_adjoint_gradients_noalloc: null argument");
        const dpp::ProblemImpl& P = prob->impl;
        if (P.kind != DPP_CELL_SIMPLEX)
            return report(DPP_ERR_BAD_STATE,
                          "dpp_adjoint_gradients_noalloc: simplicial meshes only (use "
                          "dpp_adjoint_solve for Q1 cells)");
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
    } catch (const dpp::Error& e) {
        return report(e.status, e.what());
    } catch (...) {
        return report(DPP_ERR_CUDA, "dpp_adjoint_gradients_noalloc: unexpected failure");
    }
}
