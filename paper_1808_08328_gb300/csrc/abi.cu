// extern "C" entry points of libdpp (declared in include/dpp.h). Every call
// validates its arguments on the host, runs its work on the caller's stream,
// and converts internal exceptions into a dpp_status plus a thread-local
// message. Nothing here aborts, exits or traps.
#include <atomic>
#include <cstring>
#include <map>
#include <cstdlib>
#include <mutex>
#include <new>
#include <set>

#include "amg.cuh"

namespace dpp {
void pc_setup(PcImpl& pc, const ProblemImpl& P, cudaStream_t s);
void f2d(const float* in, double* out, int64_t n, cudaStream_t s);
void pc_apply(const ProblemImpl& P, PcImpl& pc, const double* r, double* z, bool transpose,
              cudaStream_t s);
void pc_apply_mass(const ProblemImpl& P, PcImpl& pc, const double* r, double* z, cudaStream_t s);
dpp_status fgmres(const ProblemImpl& P, PcImpl& pc, const dpp_solve_opts& o, const double* rhs,
                  double* x, bool transpose, dpp_solve_info& info, cudaStream_t s,
                  HostScratch& hs);
void adjoint_gradients(const ProblemImpl& P, const double* x, const double* lambda, double* g1,
                       double* g2, double* gbeta, cudaStream_t s);
void assemble_union(ProblemImpl& P, int n, const dpp_problem_desc* descs, std::vector<int>& codes,
                    cudaStream_t s);
void fgmres_batched(const ProblemImpl& P, PcImpl& pc, const dpp_solve_opts& o, double* x,
                    std::vector<int>& status, std::vector<int>& iters,
                    std::vector<double>& relres, int64_t& graph_launches, cudaStream_t s,
                    HostScratch& hs);
void tune_batched_schedule(const ProblemImpl& P, PcImpl& pc, const dpp_solve_opts& o,
                           cudaStream_t s, HostScratch& hs);
}  // namespace dpp

namespace dpp {

namespace {
std::atomic<int64_t> g_launches{0};
std::atomic<bool> g_profiling{false};
struct Family {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
    double bytes = 0;
};
std::mutex g_prof_mu;
std::map<std::string, Family> g_prof;
std::map<int, std::vector<cudaEvent_t>> g_event_pool;  // per device
std::map<int, size_t> g_event_next;
std::atomic<bool> g_prof_all{true};
std::set<std::string> g_prof_select;  // timed families when !g_prof_all
}  // namespace

bool profiling_selected(const char* family) {
    if (g_prof_all.load(std::memory_order_relaxed)) return true;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    return g_prof_select.count(family) != 0;
}

cudaEvent_t profile_event() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    auto& pool = g_event_pool[dev];
    size_t& next = g_event_next[dev];
    if (next == pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        pool.push_back(e);
    }
    return pool[next++];
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
namespace {
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};

cudaMemPool_t device_pool(int dev) {
    if (dev < 0 || dev >= kMaxDevices) fail(DPP_ERR_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        DPP_CK(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = UINT64_MAX;  // keep freed memory for reuse until dpp_release_cached_memory
        DPP_CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        g_pools[dev] = pool;
    }
    return g_pools[dev];
}
}  // namespace

cudaStream_t& current_stream() {
    thread_local cudaStream_t s = nullptr;
    return s;
}

void* pool_alloc(size_t bytes) {
    cudaStream_t s = current_stream();
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    DPP_CK(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone)
        fail(DPP_ERR_CUDA, "internal: device allocation while the stream is being captured");
    int dev = 0;
    DPP_CK(cudaGetDevice(&dev));
    void* p = nullptr;
    DPP_CK(cudaMallocFromPoolAsync(&p, bytes, device_pool(dev), s));
    // DPP_POISON_ALLOC=1 fills every new buffer with 0xFF bytes (NaN for
    // floating point, -1 for integers), so that a read of memory the library
    // never wrote shows up in its results.
    static const bool poison = [] {
        const char* e = std::getenv("DPP_POISON_ALLOC");
        return e && e[0] == '1';
    }();
    if (poison) DPP_CK(cudaMemsetAsync(p, 0xFF, bytes, s));
    return p;
}

void pool_free(void* p) { cudaFreeAsync(p, current_stream()); }

void set_last_error_message(const char* m);
bool profiling_enabled() { return g_profiling.load(std::memory_order_relaxed); }
void profile_record(const char* family, cudaEvent_t a, cudaEvent_t b, double bytes) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    auto& f = g_prof[family];
    f.events.emplace_back(a, b);
    f.bytes += bytes;
}

}  // namespace dpp

using namespace dpp;

namespace {

thread_local std::string g_last_error;

dpp_status set_error(dpp_status s, const std::string& m) {
    g_last_error = m;
    return s;
}

template <class F>
dpp_status guarded(const char* name, F&& f) {
    try {
        g_last_error.clear();
        return f();
    } catch (const Error& e) {
        return set_error(e.status, std::string(name) + ": " + e.what());
    } catch (const std::bad_alloc&) {
        return set_error(DPP_ERR_OUT_OF_MEMORY, std::string(name) + ": host allocation failed");
    } catch (const std::exception& e) {
        return set_error(DPP_ERR_CUDA, std::string(name) + ": " + e.what());
    } catch (...) {
        return set_error(DPP_ERR_CUDA, std::string(name) + ": unknown failure");
    }
}

void require(bool ok, const std::string& what) {
    if (!ok) fail(DPP_ERR_INVALID_ARGUMENT, what);
}

void require_aligned(const void* p, const char* what) {
    require(((uintptr_t)p & 15u) == 0, std::string(what) + " must be 16-byte aligned");
}

void ensure_device() {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        fail(DPP_ERR_CUDA, "no CUDA device is available (libdpp has no CPU fallback)");
    }
}

struct EventTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s;
    explicit EventTimer(cudaStream_t st) : s(st) {
        DPP_CK(cudaEventCreate(&a));
        DPP_CK(cudaEventCreate(&b));
        DPP_CK(cudaEventRecord(a, s));
    }
    double stop() {
        DPP_CK(cudaEventRecord(b, s));
        DPP_CK(cudaEventSynchronize(b));
        float ms = 0;
        DPP_CK(cudaEventElapsedTime(&ms, a, b));
        return ms;
    }
    ~EventTimer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

}  // namespace

namespace dpp {
void set_last_error_message(const char* m) { g_last_error = m ? m : ""; }
}  // namespace dpp

extern "C" {

void dpp_pc_opts_default(dpp_pc_opts* o) {
    if (!o) return;
    o->cheb_degree_mass = 2;
    o->cheb_degree_amg = 2;
    o->coarse_max_rows = 384;
    o->max_levels = 12;
    o->strength_theta = 0.02;
    o->cheb_ratio = 10.0;
    o->use_lumped_diag = 0;
    o->precision = DPP_FP64;
    o->sell_min_rows = 0;
    o->spmv_format = 0;
    o->composition = 0;
    o->mass_solver = 0;
    o->schedule_tuning = 0;
    o->smooth_filter = 0;
    o->cheb_degree_coarse = 0;
}

void dpp_solve_opts_default(dpp_solve_opts* o) {
    if (!o) return;
    o->rtol = 1e-10;
    o->restart = 30;
    o->max_iters = 1000;
    o->x0_zero = 1;
    o->x_memory = DPP_MEM_DEVICE;
    o->check_every = 1;
    o->inner_rtol = 1e-4;
    o->wait_budget_cycles = 0;
    o->reorth_eta = 0.1;
    o->matrix_free = 0;
}

const char* dpp_status_string(int32_t s) {
    switch (s) {
        case DPP_OK: return "DPP_OK";
        case DPP_ERR_INVALID_ARGUMENT: return "DPP_ERR_INVALID_ARGUMENT";
        case DPP_ERR_OUT_OF_MEMORY: return "DPP_ERR_OUT_OF_MEMORY";
        case DPP_ERR_CUDA: return "DPP_ERR_CUDA";
        case DPP_ERR_NOT_CONVERGED: return "DPP_ERR_NOT_CONVERGED";
        case DPP_ERR_BREAKDOWN: return "DPP_ERR_BREAKDOWN";
        case DPP_ERR_NONFINITE: return "DPP_ERR_NONFINITE";
        case DPP_ERR_TIMEOUT: return "DPP_ERR_TIMEOUT";
        case DPP_ERR_BAD_STATE: return "DPP_ERR_BAD_STATE";
        default: return "DPP_ERR_UNKNOWN";
    }
}

const char* dpp_last_error(void) { return g_last_error.c_str(); }

dpp_status dpp_assemble(const dpp_problem_desc* d, int32_t precision, dpp_stream_t stream,
                        dpp_problem* out) {
    return guarded("dpp_assemble", [&]() -> dpp_status {
        StreamScope scope_((cudaStream_t)stream);
        require(d != nullptr && out != nullptr, "null descriptor or output handle");
        *out = nullptr;
        require(d->dim == 2 || d->dim == 3, "dim must be 2 or 3");
        require(d->cell_kind == DPP_CELL_SIMPLEX || d->cell_kind == DPP_CELL_Q1,
                "cell_kind must be DPP_CELL_SIMPLEX or DPP_CELL_Q1");
        require(d->memory == DPP_MEM_DEVICE || d->memory == DPP_MEM_HOST, "bad memory kind");
        require(precision == DPP_FP64 || precision == DPP_MIXED_FP32_FP64, "bad precision");
        require(d->n_nodes > 0 && d->n_cells > 0 && d->n_bfacets >= 0, "sizes must be positive");
        require(d->n_nodes < (1LL << 30) && d->n_cells < (1LL << 30), "mesh too large for int32 ids");
        require(d->coords && d->cells && d->log_k1 && d->log_k2 && d->p01 && d->p02,
                "null input array");
        require(d->n_bfacets == 0 || d->bfacets, "null bfacets with n_bfacets > 0");
        require(d->mu > 0 && std::isfinite(d->mu), "mu must be positive and finite");
        require(d->beta >= 0 && std::isfinite(d->beta), "beta must be >= 0 and finite");
        for (int k = 0; k < d->dim; ++k) require(std::isfinite(d->gamma_b[k]), "gamma_b not finite");
        ensure_device();
        cudaStream_t s = (cudaStream_t)stream;
        auto* h = new dpp_problem_s();
        try {
            EventTimer t(s);
            ProfScope pr("assemble", s, 0);
            h->impl.precision = precision;
            assemble_problem(h->impl, *d, s);
            h->impl.ms_assemble = t.stop();
        } catch (...) {
            delete h;
            throw;
        }
        *out = h;
        return DPP_OK;
    });
}

dpp_status dpp_setup_pc(dpp_problem prob, const dpp_pc_opts* opts, dpp_stream_t stream,
                        dpp_pc* out) {
    return guarded("dpp_setup_pc", [&]() -> dpp_status {
        StreamScope scope_((cudaStream_t)stream);
        require(prob != nullptr && out != nullptr, "null problem or output handle");
        *out = nullptr;
        dpp_pc_opts o;
        dpp_pc_opts_default(&o);
        if (opts) o = *opts;
        require(o.cheb_degree_mass >= 1 && o.cheb_degree_mass <= 16, "cheb_degree_mass in [1,16]");
        require(o.cheb_degree_amg >= 1 && o.cheb_degree_amg <= 16, "cheb_degree_amg in [1,16]");
        require(o.coarse_max_rows >= 1 && o.coarse_max_rows <= 4096, "coarse_max_rows in [1,4096]");
        require(o.max_levels >= 1 && o.max_levels <= 32, "max_levels in [1,32]");
        require(o.strength_theta >= 0 && o.strength_theta < 1, "strength_theta in [0,1)");
        require(o.cheb_ratio > 1, "cheb_ratio > 1");
        require(o.precision == DPP_FP64 || o.precision == DPP_MIXED_FP32_FP64, "bad precision");
        require(o.sell_min_rows >= 0, "sell_min_rows >= 0");
        require(o.spmv_format >= 0 && o.spmv_format <= 2, "spmv_format in {0,1,2}");
        require(o.composition == kFieldSplit || o.composition == kScaleSplit,
                "composition in {0 (field split), 1 (scale split)}");
        require(o.mass_solver == 0 || o.mass_solver == 1,
                "mass_solver in {0 (Chebyshev-Jacobi), 1 (ILU(0))}");
        require(o.smooth_filter == 0 || o.smooth_filter == 1, "smooth_filter in {0,1}");
        require(o.cheb_degree_coarse >= 0 && o.cheb_degree_coarse <= 16, "cheb_degree_coarse in [0,16]");
        require(o.schedule_tuning == 0 || o.schedule_tuning == 1, "schedule_tuning in {0,1}");
        cudaStream_t s = (cudaStream_t)stream;
        auto* h = new dpp_pc_s();
        try {
            EventTimer t(s);
            h->impl.opts = o;
            h->impl.precision = o.precision;
            h->owner = prob;
            pc_setup(h->impl, prob->impl, s);
            h->impl.ms_setup = t.stop();
        } catch (...) {
            delete h;
            throw;
        }
        *out = h;
        return DPP_OK;
    });
}

static dpp_status solve_common(const char* name, dpp_problem prob, dpp_pc pc,
                               const dpp_solve_opts* opts, const double* rhs_dev, double* x,
                               bool transpose, dpp_solve_info* info, dpp_stream_t stream) {
    dpp_solve_info local{};
    dpp_solve_info& inf = info ? *info : local;
    std::memset(&inf, 0, sizeof(inf));
    dpp_status st = guarded(name, [&]() -> dpp_status {
        StreamScope scope_((cudaStream_t)stream);
        require(prob && pc && x, "null problem, pc or x");
        require(pc->owner == prob, "pc was built for a different problem");
        dpp_solve_opts o;
        dpp_solve_opts_default(&o);
        if (opts) o = *opts;
        require(o.rtol > 0 && o.rtol < 1, "rtol in (0,1)");
        require(o.restart >= 1 && o.restart <= 64, "restart in [1,64]");
        require(o.max_iters >= 1, "max_iters >= 1");
        require(o.x_memory == DPP_MEM_DEVICE || o.x_memory == DPP_MEM_HOST, "bad x_memory");
        require(o.matrix_free == 0 || o.matrix_free == 1, "matrix_free in {0,1}");
        require(!o.matrix_free || prob->impl.kind == DPP_CELL_SIMPLEX,
                "matrix_free supports simplices only");
        if (o.matrix_free && pc->impl.precision == DPP_MIXED_FP32_FP64)
            matrix_free_prepare32(prob->impl, (cudaStream_t)stream);
        const ProblemImpl& P = prob->impl;
        cudaStream_t s = (cudaStream_t)stream;
        const int64_t n = P.n_nodes * P.ns;
        inf.levels = (int)pc->impl.amg[0].levels.size();
        inf.ms_assemble = P.ms_assemble;
        inf.ms_setup = pc->impl.ms_setup;
        EventTimer t(s);
        DBuf<double> xd;
        double* xw = x;
        if (o.x_memory == DPP_MEM_HOST) {
            xd.alloc(n);
            xw = xd.get();
            if (!o.x0_zero)
                DPP_CK(cudaMemcpyAsync(xw, x, n * sizeof(double), cudaMemcpyHostToDevice, s));
        } else {
            require_aligned(x, "x");
        }
        dpp_status r = fgmres(P, pc->impl, o, rhs_dev ? rhs_dev : P.f.get(), xw, transpose, inf, s,
                              const_cast<HostScratch&>(P.hs));
        if (o.x_memory == DPP_MEM_HOST)
            DPP_CK(cudaMemcpyAsync(x, xw, n * sizeof(double), cudaMemcpyDeviceToHost, s));
        inf.ms_solve = t.stop();
        if (r != DPP_OK) {
            char buf[160];
            snprintf(buf, sizeof buf, "%s after %d iterations, relative residual %.3e",
                     dpp_status_string(r), inf.iterations, inf.rel_residual);
            g_last_error = std::string(name) + ": " + buf;
        }
        return r;
    });
    inf.status = st;
    return st;
}

dpp_status dpp_solve(dpp_problem prob, dpp_pc pc, const dpp_solve_opts* opts, double* x,
                     dpp_solve_info* info, dpp_stream_t stream) {
    return solve_common("dpp_solve", prob, pc, opts, nullptr, x, false, info, stream);
}

dpp_status dpp_solve_rhs(dpp_problem prob, dpp_pc pc, const dpp_solve_opts* opts, const double* b,
                         double* x, dpp_solve_info* info, dpp_stream_t stream) {
    if (!b || ((uintptr_t)b & 15u)) {
        g_last_error = "dpp_solve_rhs: b must be a non-null, 16-byte aligned device pointer";
        if (info) { std::memset(info, 0, sizeof(*info)); info->status = DPP_ERR_INVALID_ARGUMENT; }
        return DPP_ERR_INVALID_ARGUMENT;
    }
    return solve_common("dpp_solve_rhs", prob, pc, opts, b, x, false, info, stream);
}

dpp_status dpp_adjoint_solve(dpp_problem prob, dpp_pc pc, const dpp_solve_opts* opts,
                             const double* x, const double* dJdx, double* lambda,
                             double* dJ_dlogk1, double* dJ_dlogk2, double* dJ_dbeta,
                             dpp_solve_info* info, dpp_stream_t stream) {
    dpp_status st;
    {
        dpp_status pre = guarded("dpp_adjoint_solve", [&]() -> dpp_status {
            StreamScope scope_((cudaStream_t)stream);
            require(prob && x && dJdx && lambda && dJ_dlogk1 && dJ_dlogk2 && dJ_dbeta,
                    "null argument");
            if (opts) require(opts->x_memory == DPP_MEM_DEVICE, "adjoint arrays must be device memory");
            require_aligned(x, "x");
            require_aligned(dJdx, "dJdx");
            return DPP_OK;
        });
        if (pre != DPP_OK) {
            if (info) { std::memset(info, 0, sizeof(*info)); info->status = pre; }
            return pre;
        }
    }
    dpp_solve_opts o;
    dpp_solve_opts_default(&o);
    if (opts) o = *opts;
    st = solve_common("dpp_adjoint_solve", prob, pc, &o, dJdx, lambda, true, info, stream);
    if (st != DPP_OK) return st;
    return guarded("dpp_adjoint_solve", [&]() -> dpp_status {
        StreamScope scope_((cudaStream_t)stream);
        cudaStream_t s = (cudaStream_t)stream;
        adjoint_gradients(prob->impl, x, lambda, dJ_dlogk1, dJ_dlogk2, dJ_dbeta, s);
        DPP_CK(cudaStreamSynchronize(s));
        return DPP_OK;
    });
}

dpp_status dpp_solve_batched(int32_t n_inst, const dpp_problem_desc* descs,
                             const dpp_pc_opts* pc_opts, const dpp_solve_opts* opts,
                             double* const* xs, dpp_solve_info* infos, dpp_stream_t stream) {
    std::vector<int> codes;
    dpp_status st = guarded("dpp_solve_batched", [&]() -> dpp_status {
        StreamScope scope_((cudaStream_t)stream);
        require(n_inst >= 1 && descs && xs && infos, "null argument or n_inst < 1");
        for (int i = 0; i < n_inst; ++i) std::memset(&infos[i], 0, sizeof(dpp_solve_info));
        dpp_pc_opts po;
        dpp_pc_opts_default(&po);
        if (pc_opts) po = *pc_opts;
        dpp_solve_opts o;
        dpp_solve_opts_default(&o);
        if (opts) o = *opts;
        require(o.rtol > 0 && o.rtol < 1 && o.restart >= 1 && o.restart <= 62 && o.max_iters >= 1,
                "bad solve options (rtol in (0,1), restart in [1,62], max_iters >= 1)");
        require(o.x_memory == DPP_MEM_DEVICE || o.x_memory == DPP_MEM_HOST, "bad x_memory");
        require(po.precision == DPP_FP64 || po.precision == DPP_MIXED_FP32_FP64, "bad precision");
        ensure_device();
        cudaStream_t user = (cudaStream_t)stream;
        // graph capture needs a stream other than the legacy default stream
        cudaStream_t s = nullptr;
        DPP_CK(cudaStreamSynchronize(user));
        DPP_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        struct StreamGuard {
            cudaStream_t s;
            ~StreamGuard() { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
        } guard{s};
        StreamScope on_private(s);  // declared after guard: restored before s is destroyed
        dpp_problem_s prob;
        dpp_pc_s pc;
        EventTimer ta(s);
        prob.impl.precision = po.precision;
        try {
            assemble_union(prob.impl, n_inst, descs, codes, s);
        } catch (const Error& e) {  // e.g. no valid instance: every info says why
            for (int i = 0; i < n_inst; ++i)
                infos[i].status = (i < (int)codes.size() && codes[i]) ? codes[i] : e.status;
            throw;
        }
        const double ms_asm = ta.stop();
        EventTimer tb(s);
        pc.impl.opts = po;
        pc.impl.precision = po.precision;
        pc.owner = &prob;
        require(po.schedule_tuning == 0 || po.schedule_tuning == 1, "schedule_tuning in {0,1}");
        require(po.smooth_filter == 0 || po.smooth_filter == 1, "smooth_filter in {0,1}");
        require(po.cheb_degree_coarse >= 0 && po.cheb_degree_coarse <= 16, "cheb_degree_coarse in [0,16]");
        pc_setup(pc.impl, prob.impl, s);
        if (po.schedule_tuning) tune_batched_schedule(prob.impl, pc.impl, o, s, prob.impl.hs);
        const double ms_setup = tb.stop();
        const ProblemImpl& P = prob.impl;
        const int64_t n = P.n_nodes * P.ns;
        DBuf<double> x(n);
        // initial guesses (live instances in order)
        std::vector<int> live;
        for (int i = 0; i < n_inst; ++i)
            if (!codes[i]) live.push_back(i);
        if (!o.x0_zero)
            for (size_t k = 0; k < live.size(); ++k) {
                const int64_t cnt = (P.inst_node_off[k + 1] - P.inst_node_off[k]) * P.ns;
                DPP_CK(cudaMemcpyAsync(x.get() + P.inst_node_off[k] * P.ns, xs[live[k]],
                                       cnt * sizeof(double),
                                       o.x_memory == DPP_MEM_HOST ? cudaMemcpyHostToDevice
                                                                  : cudaMemcpyDeviceToDevice, s));
            }
        EventTimer tc(s);
        std::vector<int> status, iters;
        std::vector<double> relres;
        int64_t graph_launches = 0;
        fgmres_batched(P, pc.impl, o, x.get(), status, iters, relres, graph_launches, s,
                       prob.impl.hs);
        for (int64_t k = 0; k < graph_launches; ++k) count_launch();
        for (size_t k = 0; k < live.size(); ++k) {
            const int64_t cnt = (P.inst_node_off[k + 1] - P.inst_node_off[k]) * P.ns;
            DPP_CK(cudaMemcpyAsync(xs[live[k]], x.get() + P.inst_node_off[k] * P.ns,
                                   cnt * sizeof(double),
                                   o.x_memory == DPP_MEM_HOST ? cudaMemcpyDeviceToHost
                                                              : cudaMemcpyDeviceToDevice, s));
        }
        const double ms_solve = tc.stop();
        dpp_status worst = DPP_OK;
        for (int i = 0; i < n_inst; ++i) {
            dpp_solve_info& inf = infos[i];
            inf.ms_assemble = ms_asm;
            inf.ms_setup = ms_setup;
            inf.ms_solve = ms_solve;
            inf.levels = (int)pc.impl.amg[0].levels.size();
            if (codes[i]) {
                inf.status = codes[i];
                worst = (dpp_status)codes[i];
            }
        }
        for (size_t k = 0; k < live.size(); ++k) {
            dpp_solve_info& inf = infos[live[k]];
            inf.status = status[k];
            inf.iterations = iters[k];
            inf.rel_residual = relres[k];
            inf.restarts = (iters[k] + o.restart - 1) / o.restart;
            if (status[k] != DPP_OK && worst == DPP_OK) worst = (dpp_status)status[k];
        }
        DPP_CK(cudaStreamSynchronize(s));
        if (worst != DPP_OK) g_last_error = "dpp_solve_batched: at least one instance failed (see infos)";
        return worst;
    });
    return st;
}

// The library's buffers go back to its stream-ordered pool, so first wait for
// every stream that may still use them.
void dpp_destroy_problem(dpp_problem p) {
    if (!p) return;
    cudaDeviceSynchronize();
    delete p;
}
void dpp_destroy_pc(dpp_pc p) {
    if (!p) return;
    cudaDeviceSynchronize();
    delete p;
}

dpp_status dpp_release_cached_memory(void) {
    return guarded("dpp_release_cached_memory", [&]() -> dpp_status {
        int dev = 0;
        DPP_CK(cudaGetDevice(&dev));
        DPP_CK(cudaDeviceSynchronize());
        DPP_CK(cudaMemPoolTrimTo(device_pool(dev), 0));
        return DPP_OK;
    });
}

dpp_status dpp_problem_sizes(dpp_problem prob, int64_t out[6]) {
    return guarded("dpp_problem_sizes", [&]() -> dpp_status {
        require(prob && out, "null argument");
        const ProblemImpl& P = prob->impl;
        out[0] = P.n_nodes;
        out[1] = P.n_cells;
        out[2] = P.n_pairs;
        out[3] = P.nv;
        out[4] = P.dim;
        out[5] = P.n_groups;
        return DPP_OK;
    });
}

dpp_status dpp_apply_K(dpp_problem prob, int32_t transpose, const double* x, double* y,
                       dpp_stream_t stream) {
    return guarded("dpp_apply_K", [&]() -> dpp_status {
        StreamScope scope_((cudaStream_t)stream);
        require(prob && x && y && x != y, "null or aliased argument");
        require_aligned(x, "x");
        require_aligned(y, "y");
        apply_K(prob->impl, x, y, nullptr, transpose != 0, false, (cudaStream_t)stream);
        return DPP_OK;
    });
}

dpp_status dpp_apply_K32(dpp_problem prob, int32_t transpose, const float* x, double* y,
                         dpp_stream_t stream) {
    return guarded("dpp_apply_K32", [&]() -> dpp_status {
        StreamScope scope_((cudaStream_t)stream);
        require(prob && x && y, "null argument");
        require_aligned(x, "x");
        require_aligned(y, "y");
        apply_K32(prob->impl, x, y, transpose != 0, (cudaStream_t)stream);
        return DPP_OK;
    });
}

dpp_status dpp_apply_K_mf(dpp_problem prob, int32_t transpose, const double* x, double* y,
                          dpp_stream_t stream) {
    return guarded("dpp_apply_K_mf", [&]() -> dpp_status {
        StreamScope scope_((cudaStream_t)stream);
        require(prob && x && y && x != y, "null or aliased argument");
        if (prob->impl.kind != DPP_CELL_SIMPLEX)
            fail(DPP_ERR_BAD_STATE, "the matrix-free apply supports simplices only");
        apply_K_mf(prob->impl, x, y, transpose != 0, (cudaStream_t)stream);
        return DPP_OK;
    });
}

dpp_status dpp_apply_K32_mf(dpp_problem prob, int32_t transpose, const float* x, double* y,
                            dpp_stream_t stream) {
    return guarded("dpp_apply_K32_mf", [&]() -> dpp_status {
        StreamScope scope_((cudaStream_t)stream);
        require(prob && x && y, "null argument");
        require_aligned(x, "x");
        if (prob->impl.kind != DPP_CELL_SIMPLEX)
            fail(DPP_ERR_BAD_STATE, "the matrix-free apply supports simplices only");
        matrix_free_prepare32(prob->impl, (cudaStream_t)stream);
        apply_K32_mf(prob->impl, x, y, transpose != 0, (cudaStream_t)stream);
        return DPP_OK;
    });
}

dpp_status dpp_get_rhs(dpp_problem prob, double* f, dpp_stream_t stream) {
    return guarded("dpp_get_rhs", [&]() -> dpp_status {
        StreamScope scope_((cudaStream_t)stream);
        require(prob && f, "null argument");
        const ProblemImpl& P = prob->impl;
        DPP_CK(cudaMemcpyAsync(f, P.f.get(), P.n_nodes * P.ns * sizeof(double),
                               cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
        return DPP_OK;
    });
}

}  // extern "C"

namespace dpp {
void export_pairs(const ProblemImpl& P, int* rp, int* col, double* vals, cudaStream_t s);
}

extern "C" {

dpp_status dpp_export_pairs(dpp_problem prob, int32_t* row_ptr, int32_t* col, double* vals,
                            dpp_stream_t stream) {
    return guarded("dpp_export_pairs", [&]() -> dpp_status {
        StreamScope scope_((cudaStream_t)stream);
        require(prob && row_ptr && col && vals, "null argument");
        export_pairs(prob->impl, row_ptr, col, vals, (cudaStream_t)stream);
        return DPP_OK;
    });
}

dpp_status dpp_pc_apply(dpp_problem prob, dpp_pc pc, int32_t transpose, const double* r, double* z,
                        dpp_stream_t stream) {
    return guarded("dpp_pc_apply", [&]() -> dpp_status {
        StreamScope scope_((cudaStream_t)stream);
        require(prob && pc && r && z && r != z, "null or aliased argument");
        require(pc->owner == prob, "pc was built for a different problem");
        require_aligned(r, "r");
        require_aligned(z, "z");
        pc_apply(prob->impl, pc->impl, r, z, transpose != 0, (cudaStream_t)stream);
        return DPP_OK;
    });
}

dpp_status dpp_pc_apply_mass(dpp_problem prob, dpp_pc pc, const double* r, double* z,
                             dpp_stream_t stream) {
    return guarded("dpp_pc_apply_mass", [&]() -> dpp_status {
        StreamScope scope_((cudaStream_t)stream);
        require(prob && pc && r && z && r != z, "null or aliased argument");
        require(pc->owner == prob, "pc was built for a different problem");
        pc_apply_mass(prob->impl, pc->impl, r, z, (cudaStream_t)stream);
        return DPP_OK;
    });
}

dpp_status dpp_pc_hierarchies(dpp_pc pc, int32_t* n) {
    return guarded("dpp_pc_hierarchies", [&]() -> dpp_status {
        require(pc && n, "null argument");
        *n = pc->impl.n_amg;
        return DPP_OK;
    });
}

dpp_status dpp_pc_hierarchy_level_sizes(dpp_pc pc, int32_t hierarchy, int32_t level,
                                        int64_t out[5]) {
    return guarded("dpp_pc_level_sizes", [&]() -> dpp_status {
        require(pc && out, "null argument");
        require(hierarchy >= 0 && hierarchy < pc->impl.n_amg, "hierarchy out of range");
        const auto& L = pc->impl.amg[hierarchy].levels;
        require(level >= 0 && level < (int)L.size(), "level out of range");
        out[0] = L[level].A.n_rows;
        out[1] = L[level].A.nnz;
        out[2] = (int64_t)L.size();
        out[3] = (level + 1 < (int)L.size()) ? L[level].P.n_cols : 0;
        out[4] = (level + 1 < (int)L.size()) ? L[level].P.nnz : 0;
        return DPP_OK;
    });
}

dpp_status dpp_pc_level_sizes(dpp_pc pc, int32_t level, int64_t out[5]) {
    return dpp_pc_hierarchy_level_sizes(pc, 0, level, out);
}

dpp_status dpp_pc_hierarchy_export_level(dpp_pc pc, int32_t hierarchy, int32_t level,
                                         int32_t* row_ptr, int32_t* col, double* val,
                                         int32_t* p_row_ptr, int32_t* p_col, double* p_val,
                                         dpp_stream_t stream) {
    return guarded("dpp_pc_export_level", [&]() -> dpp_status {
        StreamScope scope_((cudaStream_t)stream);
        require(pc && row_ptr && col && val, "null argument");
        require(hierarchy >= 0 && hierarchy < pc->impl.n_amg, "hierarchy out of range");
        const auto& L = pc->impl.amg[hierarchy].levels;
        require(level >= 0 && level < (int)L.size(), "level out of range");
        cudaStream_t s = (cudaStream_t)stream;
        const Csr& A = L[level].A;
        DPP_CK(cudaMemcpyAsync(row_ptr, A.row_ptr.get(), (A.n_rows + 1) * sizeof(int),
                               cudaMemcpyDeviceToDevice, s));
        DPP_CK(cudaMemcpyAsync(col, A.col.get(), A.nnz * sizeof(int), cudaMemcpyDeviceToDevice, s));
        // the FP32 hierarchy of a mixed-precision preconditioner: values widened
        auto values = [&](const Csr& M, double* out) {
            if (fp32_only(M)) f2d(M.val32.get(), out, M.nnz, s);
            else DPP_CK(cudaMemcpyAsync(out, M.val.get(), M.nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
        };
        values(A, val);
        if (p_row_ptr && p_col && p_val && level + 1 < (int)L.size()) {
            const Csr& P = L[level].P;
            DPP_CK(cudaMemcpyAsync(p_row_ptr, P.row_ptr.get(), (P.n_rows + 1) * sizeof(int),
                                   cudaMemcpyDeviceToDevice, s));
            DPP_CK(cudaMemcpyAsync(p_col, P.col.get(), P.nnz * sizeof(int), cudaMemcpyDeviceToDevice, s));
            values(P, p_val);
        }
        DPP_CK(cudaStreamSynchronize(s));
        return DPP_OK;
    });
}

dpp_status dpp_pc_export_level(dpp_pc pc, int32_t level, int32_t* row_ptr, int32_t* col,
                               double* val, int32_t* p_row_ptr, int32_t* p_col, double* p_val,
                               dpp_stream_t stream) {
    return dpp_pc_hierarchy_export_level(pc, 0, level, row_ptr, col, val, p_row_ptr, p_col, p_val,
                                         stream);
}

}  // extern "C"

extern "C" {

int64_t dpp_launch_count(void) { return g_launches.load(); }

dpp_status dpp_profile_enable(int32_t on) {
    return guarded("dpp_profile_enable", [&]() -> dpp_status {
        DPP_CK(cudaDeviceSynchronize());  // recorded events are reused from here on
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof.clear();
        for (auto& kv : g_event_next) kv.second = 0;
        g_profiling.store(on != 0);
        return DPP_OK;
    });
}

dpp_status dpp_profile_select(const char* families) {
    return guarded("dpp_profile_select", [&]() -> dpp_status {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof_select.clear();
        const std::string all = families ? families : "";
        size_t b = 0;
        while (b <= all.size()) {
            size_t e = all.find(',', b);
            if (e == std::string::npos) e = all.size();
            if (e > b) g_prof_select.insert(all.substr(b, e - b));
            b = e + 1;
        }
        g_prof_all.store(g_prof_select.empty());
        return DPP_OK;
    });
}

dpp_status dpp_profile_read(const char* family, int64_t* launches, double* total_ms,
                            double* alg_bytes) {
    return guarded("dpp_profile_read", [&]() -> dpp_status {
        require(family && launches && total_ms && alg_bytes, "null argument");
        std::lock_guard<std::mutex> lk(g_prof_mu);
        *launches = 0;
        *total_ms = 0;
        *alg_bytes = 0;
        auto it = g_prof.find(family);
        if (it == g_prof.end()) return DPP_OK;
        double ms = 0;
        for (auto& e : it->second.events) {
            DPP_CK(cudaEventSynchronize(e.second));
            float t = 0;
            DPP_CK(cudaEventElapsedTime(&t, e.first, e.second));
            ms += t;
        }
        *launches = (int64_t)it->second.events.size();
        *total_ms = ms;
        *alg_bytes = it->second.bytes;
        return DPP_OK;
    });
}

}  // extern "C"
