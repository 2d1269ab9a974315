/*
 * dpp.h -- C ABI of the GB300 solver for the four-field double
 * porosity/permeability (DPP) model.
 *
 * Model and method: Joshaghani, Chang, Nakshatrala & Knepley, "Composable
 * block solvers for the four-field double porosity/permeability model"
 * (2018).
 *   - Governing equations: Eqs. "DG_GE_Darcy_BLM" (Darcy in each network plus
 *     mass balance) and "Composable_mass_transfer" (chi = -beta/mu (p1 - p2)),
 *     Section 2.
 *   - Pressure boundary data p0i on Gamma^p: Eq. "DG_GE_Darcy_pBC". It is
 *     imposed weakly through -(w.n; p0i) in the linear functional (Section 3,
 *     L_Gal; appendix CG-VMS listing, which uses no strong BCs).
 *   - Discretisation: the CG-VMS stabilised mixed form (Eq.
 *     "CG_VMS_Weak_form", Section 3.3), P1 on triangles and tetrahedra.
 *     Blocks: Eq. "S4_cg_stiffness_matrix"; load: Eq. "S4_cg_rhs"; system
 *     K u = f: Eq. "S4_linear_problem" (Section 4).
 *   - Solver: Method 2 of Section 4.2 ("splitting by fields", the default).
 *     A full Schur factorisation of [[A, B], [C, D]] with A =
 *     blockdiag(K1_uu, K2_uu); the selfp Schur matrix S_p = D - C diag(A)^-1
 *     B, additively split into its two diagonal blocks (Eqs. "S4_sp1",
 *     "S4_sp2"); one multigrid V-cycle per block; single-sweep inner solves
 *     inside an outer Krylov method. Method 1 of Section 4.1 ("splitting by
 *     scales") is the other composition (dpp_pc_opts::composition).
 *
 * Conventions for every entry point:
 *   - Device pointers are CUDA global-memory addresses on the current device.
 *     The caller owns them and keeps them valid until the call's stream work
 *     has completed. The library owns its handles and frees them only in
 *     dpp_destroy_*.
 *   - Work is ordered on `stream` (NULL = the legacy default stream). Calls that
 *     must report a host-visible result (dpp_solve*, dpp_setup_pc and
 *     dpp_assemble's size discovery) synchronise that stream before they return.
 *   - The library's own device memory (handles, work vectors, setup
 *     temporaries) comes from a library-owned, stream-ordered CUDA memory
 *     pool per device: allocations and frees are ordered on the call's stream
 *     and never synchronise the device, and freed memory stays cached for
 *     reuse until dpp_release_cached_memory. A handle must not be used from
 *     two streams at once; dpp_destroy_* first waits for the whole device.
 *   - No call aborts, exits or traps. Errors come back as dpp_status, and
 *     dpp_last_error() gives a thread-local message. Input arrays are checked
 *     on the device for index range and finiteness before any kernel uses
 *     them as an index.
 *   - Unknown layout: node-interleaved. Node a holds 2d+2 doubles
 *     [u1_0 .. u1_{d-1}, p1, u2_0 .. u2_{d-1}, p2] at offset a*(2d+2).
 *   - There is no CPU fallback. Without a CUDA device every call that needs
 *     one returns DPP_ERR_CUDA.
 */
#ifndef DPP_H
#define DPP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t, declared here so callers need no CUDA headers. */
typedef struct CUstream_st* dpp_stream_t;

typedef enum {
    DPP_OK = 0,
    DPP_ERR_INVALID_ARGUMENT = 1, /* bad size, null pointer, index out of range, degenerate cell */
    DPP_ERR_OUT_OF_MEMORY = 2,
    DPP_ERR_CUDA = 3,             /* a CUDA runtime error (including "no device") */
    DPP_ERR_NOT_CONVERGED = 4,    /* max_iters reached; x holds the last iterate */
    DPP_ERR_BREAKDOWN = 5,        /* Krylov breakdown before convergence */
    DPP_ERR_NONFINITE = 6,        /* NaN or Inf in an input or in the iteration */
    DPP_ERR_TIMEOUT = 7,          /* a bounded device wait ran out */
    DPP_ERR_BAD_STATE = 8         /* handle mismatch or misuse */
} dpp_status;

typedef enum { DPP_FP64 = 0, DPP_MIXED_FP32_FP64 = 1 } dpp_precision;
typedef enum { DPP_MEM_DEVICE = 0, DPP_MEM_HOST = 1 } dpp_memory;
/* Cell types (Table "ELE_level_discretization"): P1 on triangles/tetrahedra, or
 * Q1 on quadrilaterals/hexahedra with vertices in tensor order (vertex v at
 * the reference corner with coordinate bits (v & 1, (v >> 1) & 1, (v >> 2) & 1)). */
typedef enum { DPP_CELL_SIMPLEX = 0, DPP_CELL_Q1 = 1 } dpp_cell_kind;

typedef struct dpp_problem_s* dpp_problem; /* opaque: graph, K pair values, f */
typedef struct dpp_pc_s* dpp_pc;           /* opaque: S_p blocks and AMG hierarchy */

/*
 * Problem description (Section 2 and the CG-VMS forms of Section 3.3).
 * `memory` says where every array below lives. For DPP_MEM_HOST the library
 * copies the arrays to the device inside dpp_assemble.
 */
typedef struct {
    int32_t dim;              /* 2 (triangles, quadrilaterals) or 3 (tetrahedra, hexahedra) */
    int32_t memory;           /* dpp_memory of the arrays below */
    int64_t n_nodes, n_cells, n_bfacets;
    const double* coords;     /* [n_nodes][dim] */
    const int32_t* cells;     /* [n_cells][dim+1] node ids (simplices; either orientation) */
    const int32_t* bfacets;   /* [n_bfacets][dim] boundary facets on Gamma^p (pressure data) */
    const double* log_k1;     /* [n_cells] natural-log macro permeability k1 */
    const double* log_k2;     /* [n_cells] natural-log micro permeability k2 */
    double mu;                /* viscosity, > 0 */
    double beta;              /* mass-transfer coefficient, >= 0 (Eq. "Composable_mass_transfer") */
    double gamma_b[3];        /* constant gamma*b body force (first dim entries used) */
    const double* p01;        /* [n_nodes] macro pressure data, read at bfacet nodes */
    const double* p02;        /* [n_nodes] micro pressure data, read at bfacet nodes */
    int32_t cell_kind;        /* dpp_cell_kind. For DPP_CELL_Q1, cells are [n_cells][2^dim] and
                                 bfacets [n_bfacets][2^(dim-1)], both in tensor vertex order */
} dpp_problem_desc;

/* Preconditioner options (Section 4; defaults from dpp_pc_opts_default). */
typedef struct {
    int32_t cheb_degree_mass;  /* Chebyshev-Jacobi degree for A^-1 (default 2) */
    int32_t cheb_degree_amg;   /* Chebyshev-Jacobi pre/post smoothing degree (default 2) */
    int32_t coarse_max_rows;   /* stop coarsening at or below this many rows (default 384) */
    int32_t max_levels;        /* hierarchy depth cap (default 12) */
    double strength_theta;     /* SA symmetric strength threshold (default 0.02) */
    double cheb_ratio;         /* AMG smoothing interval [lmax/ratio, 1.1 lmax] (default 10) */
    int32_t use_lumped_diag;   /* 0: diag(K_uu) as written (default); 1: row-sum lumping */
    int32_t precision;         /* dpp_precision of the hierarchy values */
    int32_t sell_min_rows;     /* level matrices with at least this many rows also get a SELL-32
                                  copy (0 = library default, 65536) */
    int32_t spmv_format;       /* AMG SpMV format: 0 = autotuned among SELL-32 (where built) and
                                  CSR (default), 1 = CSR only, 2 = SELL-32 wherever built.
                                  The autotuned choices are cached for the process per size
                                  class; if the environment variable DPP_TUNE_CACHE names a
                                  file, they are read from it and new ones are appended to it
                                  (one JSON object per line). */
    int32_t composition;       /* 0: Method 2 of Section 4.2, splitting by fields (default): one
                                  Schur factorisation over {u1, u2} | {p1, p2} and one SA-AMG
                                  hierarchy on blockdiag(S_p1, S_p2).
                                  1: Method 1 of Section 4.1, splitting by scales: an additive
                                  split {u1, p1} | {u2, p2} (K12_pp dropped), each network with
                                  its own Schur factorisation, selfp matrix S^i_p (Eqs.
                                  "S4_sp1", "S4_sp2") and SA-AMG hierarchy. */
    int32_t mass_solver;       /* inner solve of the velocity block A = blockdiag(K1_uu, K2_uu):
                                  0: Chebyshev-Jacobi of degree cheb_degree_mass on the exact
                                  Wathen interval (default);
                                  1: ILU(0) of each network's mass matrix in natural row order,
                                  the paper's block Jacobi / ILU(0) sub-solver (Sections 4.1,
                                  4.2); level-scheduled, one launch per dependency level. */
    int32_t schedule_tuning;   /* dpp_solve_batched only. 1: the preconditioner schedule (AMG
                                  Chebyshev degrees, cheb_ratio, mass Chebyshev degree) is chosen
                                  by timing candidate batched solves on the hierarchy already
                                  built (coordinate search: AMG degree {1,2,3}, coarse-level
                                  degree {1,2,3}, ratio {10,20,30}, mass degree {1,2,3}),
                                  once per size class (dimension, precision, log2 of the union's
                                  nodes and of the mean instance's); the choice is cached for
                                  the process and in the DPP_TUNE_CACHE file if one is named.
                                  0: the schedule given (default). */
    int32_t smooth_filter;     /* prolongator smoothing: 0 = P = (I - w D^-1 A) P0 with the level
                                  matrix A; 1 = with the filtered matrix A^F of Vanek, Mandel and
                                  Brezina (strong entries of A by strength_theta, the weak ones
                                  added into the diagonal), w = 4 / (3 lambda_max(D_F^-1 A^F)):
                                  sparser P and Galerkin products. */
    int32_t cheb_degree_coarse; /* Chebyshev degree of the AMG smoother on the levels below the
                                  finest; 0 (default) = cheb_degree_amg on every level */
} dpp_pc_opts;

/* Krylov options. */
typedef struct {
    double rtol;               /* stop at FP64 ||f - K x||_2 / ||f||_2 <= rtol (default 1e-10) */
    int32_t restart;           /* FGMRES restart length m (default 30, at most 64) */
    int32_t max_iters;         /* total inner iterations cap (default 1000) */
    int32_t x0_zero;           /* 1: ignore x on entry and start from 0 (default 1) */
    int32_t x_memory;          /* dpp_memory of x / lambda arrays passed to dpp_solve* (default device) */
    int32_t check_every;       /* reserved, ignored: the residual estimate is checked at every
                                  iteration, when the Hessenberg column reaches the host anyway */
    double inner_rtol;         /* mixed precision: inner cycle reduction target (default 1e-4) */
    int64_t wait_budget_cycles;/* reserved, ignored: no kernel of the library spins on a flag */
    double reorth_eta;         /* second Gram-Schmidt pass when ||w|| drops below reorth_eta
                                  times its value before the first pass (DGKS test; 0 = never,
                                  1 = always; default 0.1) */
    int32_t matrix_free;       /* 1: the Krylov step's K z is applied element by element from the
                                  cells' geometry and k (dpp_apply_K_mf; FP32 in the mixed mode,
                                  dpp_apply_K32_mf) instead of from the assembled pair values.
                                  Residuals keep the assembled FP64 K. Default 0. */
} dpp_solve_opts;

typedef struct {
    int32_t status;            /* dpp_status of the call */
    int32_t iterations;        /* inner Krylov iterations */
    int32_t restarts;          /* restarts / refinement steps */
    int32_t levels;            /* AMG levels (from the pc) */
    double rel_residual;       /* FP64 true ||f - K x|| / ||f|| at exit */
    double ms_assemble, ms_setup, ms_solve;
} dpp_solve_info;

void dpp_pc_opts_default(dpp_pc_opts* o);
void dpp_solve_opts_default(dpp_solve_opts* o);

/*
 * Assemble K and f of Eq. "S4_linear_problem" for the CG-VMS P1 form.
 * Per node pair (a, b) the library keeps the distinct block values of
 * Eq. "S4_cg_stiffness_matrix": the two weighted masses 1/2 (w; mu/ki u),
 * the d entries of K_up, the d entries of K_pu, the two K_pp diagonals and
 * the coupling K12_pp = K21_pp. precision = DPP_MIXED_FP32_FP64 also keeps
 * an FP32 copy of the values. On success *out is a new handle.
 * Errors: INVALID_ARGUMENT (null pointers, dim not 2 or 3, an index out of
 * range, a zero-volume cell, mu <= 0 or beta < 0, a bfacet that is not a
 * cell face, a node with more than 95 distinct neighbours), NONFINITE (NaN
 * or Inf in coords, log k or p0), OUT_OF_MEMORY, CUDA. A node may lie in any
 * number of cells.
 */
dpp_status dpp_assemble(const dpp_problem_desc* desc, int32_t precision, dpp_stream_t stream,
                        dpp_problem* out);

/*
 * Build the block preconditioner of Section 4: Method 2 (splitting by fields,
 * the default) or Method 1 (splitting by scales), as opts->composition says.
 * It forms S_pi = Ki_pp - Ki_pu diag(Ki_uu)^-1 Ki_up (Eqs. "S4_sp1",
 * "S4_sp2") on the device, then smoothed-aggregation AMG: one hierarchy on
 * blockdiag(S_p1, S_p2) (Method 2) or one per S_pi (Method 1). With
 * opts->precision = DPP_MIXED_FP32_FP64 the S_pi and the whole hierarchy are
 * built in FP32 from the FP32 pair values (only the coarsest inverse is FP64).
 * Synchronises `stream`. Errors: INVALID_ARGUMENT, OUT_OF_MEMORY, CUDA.
 * Size limit: row pointers are int32, so the nonzeros of blockdiag(S_p1,
 * S_p2), of every level matrix and of every prolongator must each stay below
 * 2^31. blockdiag(S_p1, S_p2) has up to 2 x 65 entries per node on 3D Kuhn
 * meshes, which reaches the limit near 16 M nodes (about 130 M DoF). A larger
 * matrix is detected when its row pointers are formed and fails with
 * INVALID_ARGUMENT (dpp_assemble does the same for the node pairs).
 */
dpp_status dpp_setup_pc(dpp_problem prob, const dpp_pc_opts* opts, dpp_stream_t stream,
                        dpp_pc* out);

/*
 * Solve K x = f with right-preconditioned FGMRES(m), the preconditioner of
 * dpp_setup_pc, in FP64 (or FP64-outer / FP32-inner refinement if the problem
 * and pc were built with DPP_MIXED_FP32_FP64). x: [n_nodes][2d+2], where
 * opts->x_memory says; on entry the initial guess unless opts->x0_zero,
 * on exit the solution. info may be NULL. Returns NOT_CONVERGED (x = last
 * iterate), BREAKDOWN, NONFINITE, INVALID_ARGUMENT or CUDA on failure.
 */
dpp_status dpp_solve(dpp_problem prob, dpp_pc pc, const dpp_solve_opts* opts, double* x,
                     dpp_solve_info* info, dpp_stream_t stream);

/*
 * As dpp_solve, but for K x = b with a caller-supplied right-hand side b
 * (device, [n_nodes][2d+2], 16-byte aligned) instead of the assembled f.
 * It reuses the assembled operator and preconditioner for further
 * right-hand sides, for example corrections K d = f - K x0. opts->rtol is
 * relative to ||b||_2. x follows opts->x_memory like dpp_solve's x.
 */
dpp_status dpp_solve_rhs(dpp_problem prob, dpp_pc pc, const dpp_solve_opts* opts, const double* b,
                         double* x, dpp_solve_info* info, dpp_stream_t stream);

/*
 * Adjoint of the solve for J(x) with a given gradient dJdx (device,
 * [n_nodes][2d+2]). It solves K^T lambda = dJdx with the same preconditioner
 * (S_p is unchanged when B and C change sign). It then forms, for every cell
 * c, dJ/dlog k1_c = -lambda^T (dK/dlog k1_c x - df/dlog k1_c), the same for
 * log k2, and dJ/dbeta = -lambda^T (dK/dbeta) x. Outputs (device): lambda
 * [n_nodes][2d+2], dJ_dlogk1 [n_cells], dJ_dlogk2 [n_cells], dJ_dbeta [1].
 * x must be the forward solution of the same problem.
 */
dpp_status dpp_adjoint_solve(dpp_problem prob, dpp_pc pc, const dpp_solve_opts* opts,
                             const double* x, const double* dJdx, double* lambda,
                             double* dJ_dlogk1, double* dJ_dlogk2, double* dJ_dbeta,
                             dpp_solve_info* info, dpp_stream_t stream);

/*
 * Solve n_inst independent systems (for example permeability realisations on
 * meshes of different sizes) in one batched pass. descs[i] describes instance i
 * exactly as for dpp_assemble (simplicial cells only); dim and gamma_b must
 * agree across instances, and mu and beta may differ. The instances are assembled as one block-diagonal
 * union. One preconditioner (pc_opts, including its precision) is built on the
 * union; because no strength edge joins two instances, each instance keeps its
 * own aggregates. Every instance then runs its own FGMRES, with its own inner
 * products, Givens rotations, least-squares solves and convergence test on
 * ||f_i - K_i x_i|| / ||f_i|| <= rtol, in lock step with the others. The
 * whole solve is one CUDA graph, launched once: a conditional WHILE node over
 * restart cycles around a WHILE node over Arnoldi steps, which the device ends
 * when no instance is still iterating (restart and max_iters bound both
 * loops). xs[i]: [n_nodes_i][2d+2]
 * (device or host per opts->x_memory; the initial guess unless opts->x0_zero).
 * infos[i] receives that instance's status, iterations and residual. An
 * instance with invalid input gets INVALID_ARGUMENT or NONFINITE and is left
 * out; the others are still solved. Returns DPP_OK when every instance
 * converged, else the first failing status. restart is limited to 62.
 * Synchronises `stream`.
 */
dpp_status dpp_solve_batched(int32_t n_inst, const dpp_problem_desc* descs,
                             const dpp_pc_opts* pc_opts, const dpp_solve_opts* opts,
                             double* const* xs, dpp_solve_info* infos, dpp_stream_t stream);

void dpp_destroy_problem(dpp_problem prob);
void dpp_destroy_pc(dpp_pc pc);
const char* dpp_status_string(int32_t status);
const char* dpp_last_error(void); /* thread-local detail of the last failing call */

/* ---------------- inspection entry points (used by the parity tests) ---------------- */

/* Sizes: out[0] = n_nodes, out[1] = n_cells, out[2] = n_pairs (CSR entries
 * of the node-pair graph, self pairs included), out[3] = values per pair,
 * out[4] = dim, out[5] = SELL slot groups. */
dpp_status dpp_problem_sizes(dpp_problem prob, int64_t out[6]);

/* y = K x, or y = K^T x if transpose != 0. x, y: device [n_nodes][2d+2], FP64. */
dpp_status dpp_apply_K(dpp_problem prob, int32_t transpose, const double* x, double* y,
                       dpp_stream_t stream);

/* y = K32 x with the FP32 copy of the pair values, FP32 x and FP32 arithmetic,
 * FP64 y: the operator of the mixed-precision inner iteration. Requires a
 * problem assembled with DPP_MIXED_FP32_FP64 (else DPP_ERR_BAD_STATE).
 * x: device float [n_nodes][2d+2], 16-byte aligned; y: device double. */
dpp_status dpp_apply_K32(dpp_problem prob, int32_t transpose, const float* x, double* y,
                         dpp_stream_t stream);

/*
 * Matrix-free y = K x (transpose != 0: K^T x), element by element (an
 * alternative evaluation of Eq. "S4_cg_stiffness_matrix"). No pair values are
 * read: each node gathers, over its incident cells in increasing cell id, the
 * element's action from the cell's vertex coordinates, k1, k2, mu and beta.
 * The cell-level sums it needs are sum u, sum p, grad p_h and div u_h per
 * network. The gather is deterministic (no atomics). x, y: device
 * [n_nodes][2d+2] FP64. Agrees with dpp_apply_K up to rounding.
 */
dpp_status dpp_apply_K_mf(dpp_problem prob, int32_t transpose, const double* x, double* y,
                          dpp_stream_t stream);

/* As dpp_apply_K_mf with FP32 geometry, k, x and arithmetic, and FP64 output:
 * the matrix-free counterpart of dpp_apply_K32. The first call makes FP32
 * copies of the coordinates and k (kept with the problem). x: device float
 * [n_nodes][2d+2], 16-byte aligned; y: device double. */
dpp_status dpp_apply_K32_mf(dpp_problem prob, int32_t transpose, const float* x, double* y,
                            dpp_stream_t stream);

/* Copy f (device, [n_nodes][2d+2]) into `f`. */
dpp_status dpp_get_rhs(dpp_problem prob, double* f, dpp_stream_t stream);

/* Export the node-pair graph and values in CSR order: row_ptr [n_nodes+1],
 * col [n_pairs], vals [n_pairs][values per pair] (all device). Value order
 * per pair (a, b): m1, m2, Kup[0..d-1], Kpu[0..d-1], d1, d2, e where
 * (u1_i, u1_i) = m1, (u1_i, p1) = Kup[i], (p1, u1_i) = Kpu[i], (p1, p1) = d1,
 * (p2, p2) = d2, (p1, p2) = (p2, p1) = e, with the same pattern for network 2. */
dpp_status dpp_export_pairs(dpp_problem prob, int32_t* row_ptr, int32_t* col, double* vals,
                            dpp_stream_t stream);

/* z = P^-1 r for the preconditioner (device [n_nodes][2d+2]); transpose != 0
 * applies the preconditioner of K^T. A DPP_MIXED_FP32_FP64 preconditioner holds
 * its FP32 hierarchy only: z is then its FP32 result, widened to FP64. */
dpp_status dpp_pc_apply(dpp_problem prob, dpp_pc pc, int32_t transpose, const double* r,
                        double* z, dpp_stream_t stream);

/* z = Ainv r on the velocity slots (the preconditioner's inner solve of A =
 * blockdiag(K1_uu, K2_uu) alone: Chebyshev-Jacobi or ILU(0) per
 * mass_solver); the pressure slots of z are zero. r, z: device
 * [n_nodes][2d+2], distinct. */
dpp_status dpp_pc_apply_mass(dpp_problem prob, dpp_pc pc, const double* r, double* z,
                             dpp_stream_t stream);

/* Number of AMG hierarchies: 1 for the field split (on blockdiag(S_p1, S_p2)),
 * 2 for the scale split (hierarchy 0 on S_p1, hierarchy 1 on S_p2). */
dpp_status dpp_pc_hierarchies(dpp_pc pc, int32_t* n);

/* Sizes of level `level` of AMG hierarchy `hierarchy`: out[0] = rows, out[1] =
 * nnz, out[2] = levels, out[3] = columns of the prolongator P (0 on the
 * coarsest level), out[4] = nnz(P). dpp_pc_level_sizes is hierarchy 0. */
dpp_status dpp_pc_hierarchy_level_sizes(dpp_pc pc, int32_t hierarchy, int32_t level,
                                        int64_t out[5]);
dpp_status dpp_pc_level_sizes(dpp_pc pc, int32_t level, int64_t out[5]);

/* Export the CSR matrix of AMG level `level` of hierarchy `hierarchy` (level 0
 * = blockdiag(S_p1, S_p2) for the field split; S_p1 or S_p2 for the scale
 * split) and, for level < levels-1, its prolongator P (device arrays sized
 * from the level sizes). Null P pointers skip P. dpp_pc_export_level is
 * hierarchy 0. The hierarchy of a DPP_MIXED_FP32_FP64 preconditioner is built
 * in FP32; its values are exported widened to FP64. */
dpp_status dpp_pc_hierarchy_export_level(dpp_pc pc, int32_t hierarchy, int32_t level,
                                         int32_t* row_ptr, int32_t* col, double* val,
                                         int32_t* p_row_ptr, int32_t* p_col, double* p_val,
                                         dpp_stream_t stream);
dpp_status dpp_pc_export_level(dpp_pc pc, int32_t level, int32_t* row_ptr, int32_t* col,
                               double* val, int32_t* p_row_ptr, int32_t* p_col, double* p_val,
                               dpp_stream_t stream);

/*
 * Allocation-free variant of the adjoint's sensitivity step. The paper has no
 * counterpart; this is an interface for callers that cannot allocate device
 * memory. Examples: a custom call inside an XLA/JAX or TensorFlow graph, or a
 * process whose device memory another framework's pool has already reserved.
 * For them cudaMalloc/cudaFree would synchronise the device, bypass the owning
 * pool, or fail.
 * Given the forward solution x and the adjoint lambda (device, [n_nodes][2d+2])
 * of an assembled problem, it writes the same dJ_dlogk1 [n_cells], dJ_dlogk2
 * [n_cells] and dJ_dbeta [1] (all device) as dpp_adjoint_solve does after its
 * transpose solve. It allocates nothing. Its scratch is one fixed array in the
 * library (16384 doubles, 128 KiB on each GPU that loads the library, kept
 * until the process exits), so n_cells must be at most 4,194,304. Larger
 * meshes return DPP_ERR_INVALID_ARGUMENT. The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current, so make that first call before any stream capture. Every call
 * overwrites the part of the array it uses before reading it, so no state
 * carries over. Calls that overlap on the GPU share the array and race: order
 * them on one stream. The work is queued on `stream`, and the call returns
 * without waiting for it.
 */
dpp_status dpp_adjoint_gradients_noalloc(dpp_problem prob, const double* x, const double* lambda,
                                         double* dJ_dlogk1, double* dJ_dlogk2, double* dJ_dbeta,
                                         dpp_stream_t stream);

/* ---------------- instrumentation (no counterpart in the paper) ---------------- */

/* Wait for the current device, then return the memory cached in the
 * library's pool for that device (see the conventions above) to the driver.
 * Live handles keep their memory. Errors: CUDA. */
dpp_status dpp_release_cached_memory(void);

/* Number of kernels this library has launched since it was loaded (every
 * launch site is counted once). */
int64_t dpp_launch_count(void);

/* Enable (on != 0) or disable per-family CUDA-event timing and reset the
 * records (waits for the device first: the timing events are reused). When
 * enabled, the library records a start and a stop event on the launching
 * stream around every launch of the kernel families "apply_K",
 * "apply_K_fp32", "mass_cheb", "mass_cheb_fp32", the V-cycle SpMVs
 * "amg_spmv_L0" (level-0 matrix), "amg_spmv_Lc" (coarser matrices) and
 * "amg_spmv_PR" (prolongation and restriction), each also with an "_fp32"
 * twin, "amg_spmv_setup" and "amg_spmv_setup_fp32" (SpMVs of the setup: power
 * iterations and the autotuner), and around the phases
 * "assemble", "setup_*", "spgemm_*" and "krylov_*" (preconditioner and
 * K applications, orthogonalisation, its kernels and its host wait). For the
 * kernel families it also accumulates the algorithmic bytes: every matrix
 * value, index and vector entry, counted once. Timing adds about a
 * microsecond of host work per timed range; ranges inside a CUDA graph
 * capture are not timed. */
dpp_status dpp_profile_enable(int32_t on);

/* Restrict timing to the comma-separated families in `families` (NULL or ""
 * = every family, the default), so that a long timed run pays for the events
 * of the families it reads only. Takes effect for ranges opened afterwards. */
dpp_status dpp_profile_select(const char* families);

/* Totals for one family since the last dpp_profile_enable: launches, device
 * milliseconds (summed event intervals, synchronising on them), algorithmic
 * bytes. An unknown family gives zeros. */
dpp_status dpp_profile_read(const char* family, int64_t* launches, double* total_ms,
                            double* alg_bytes);

#ifdef __cplusplus
}
#endif

#endif /* DPP_H */
