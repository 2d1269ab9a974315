// Library-internal data structures behind the opaque dpp_problem / dpp_pc handles.
#pragma once

#include "common.cuh"

namespace dpp {

// Per-cell geometry record: |K| then the d+1 constant gradients of the P1
// barycentric basis, padded to a power of two.
template <int DIM> struct GeoLayout;
template <> struct GeoLayout<2> { static constexpr int stride = 8; };
template <> struct GeoLayout<3> { static constexpr int stride = 16; };

// Per-cell factors of the pair values, written by the geometry kernel.
constexpr int kCellCoef = 8;

// Values stored per node pair (a, b): m1, m2, Kup[d], Kpu[d], d1, d2, e.
__host__ __device__ constexpr int pair_values(int dim) { return 2 + 2 * dim + 3; }

// Scalar CSR matrix (AMG levels, S_p, P, R).
struct Csr {
    int64_t n_rows = 0, n_cols = 0, nnz = 0;
    DBuf<int> row_ptr, col;
    DBuf<double> val;
    DBuf<float> val32;
    // Optional SELL-32 copy (slices of 32 rows, column-major within a slice,
    // each slice as wide as its longest row; padding = (the row's last column,
    // 0.0)). Built for level matrices and prolongators with many rows, where
    // one thread per row fills the GPU.
    DBuf<int> sell_off;      // [n_slices + 1] entry offsets
    DBuf<int> sell_col;
    DBuf<double> sell_val;
    DBuf<float> sell_val32;
    // Optional 16-bit columns of the SELL-32 copy (FP32 hierarchy): column =
    // sell_base[slice] + sell_col16[slot], built when every slice's columns
    // span less than 65536.
    DBuf<int> sell_base;
    DBuf<uint16_t> sell_col16;
    bool has_sell() const { return sell_off.get() != nullptr; }
};

struct ProblemImpl {
    int dim = 0, ns = 0, nv = 0;  // dimension, DoF per node (2d+2), values per pair
    int kind = DPP_CELL_SIMPLEX;  // dpp_cell_kind
    int nvc = 0, nfv = 0;         // vertices per cell and per boundary facet
    int64_t n_nodes = 0, n_cells = 0, n_bfacets = 0, n_pairs = 0;
    double mu = 1, beta = 0, gb[3] = {0, 0, 0};
    int precision = DPP_FP64;

    DBuf<double> coords, logk1, logk2, p01, p02;
    DBuf<int> cells, bfacets;
    DBuf<int> nc_ptr, nc_list;   // node -> incident cells (sorted)
    DBuf<int> nf_ptr, nf_list;   // node -> incident boundary facets (sorted)
    DBuf<double> facet_nA;       // [n_bfacets][dim]: |F| times the outward unit normal
    DBuf<int> row_ptr, col, pair_row;  // node-pair CSR (self pairs included, columns sorted)

    // SELL-32 storage of the pair values: slice s holds rows 32s..32s+31,
    // groups slice_ptr[s]..slice_ptr[s+1]-1, one group per column slot.
    int64_t n_slices = 0, n_groups = 0;
    DBuf<int> slice_ptr;    // [n_slices+1]
    DBuf<int> sell_col;     // [n_groups][32], -1 = padding
    DBuf<double> sell_val;  // [n_groups][nv][32]
    DBuf<float> sell_val32; // FP32 copy (mixed precision)

    DBuf<double> cell_mu_beta;  // [n_cells][2]: per-cell mu, beta (batched problems only)
    // batched problems: instance b owns nodes inst_node_off[b] .. inst_node_off[b+1]-1
    int n_inst = 1;
    std::vector<int64_t> inst_node_off, inst_cell_off;
    std::vector<double> inst_mu, inst_beta;
    // FP32 copies for the matrix-free FP32 operator (made on first use)
    DBuf<float> coords32, kk32, cell_mu_beta32;
    DBuf<double> geo;       // [n_cells][GeoLayout<dim>::stride]
    DBuf<double> q1tab;     // Q1 cells: [n_cells][q1::Layout<dim>::stride] element integrals
    DBuf<double> facet_tab; // Q1 cells: [n_bfacets][q1::Layout<dim>::fstride] facet integrals
    DBuf<double> kk;        // [n_cells][2]: k1, k2
    DBuf<double> ccoef;     // [n_cells][kCellCoef]: factors of the pair values
    DBuf<double> f;         // [n_nodes][ns]
    DBuf<int> dstatus;      // device status word
    HostScratch hs;
    double ms_assemble = 0;
};

// One level of the AMG hierarchy on blockdiag(S_p1, S_p2).
struct Level {
    Csr A;            // level matrix
    Csr P, R;         // prolongator to this level from the next coarser, and R = P^T
    DBuf<double> dinv;        // 1 / diag(A)
    DBuf<float> dinv32;
    double lmax = 0;          // estimate of the largest eigenvalue of D^-1 A
    int lanes = 4;            // CSR SpMV lanes per row of A (autotuned)
    int lanes_P = 4, lanes_R = 4;  // lanes per row of P and R (autotuned)
    // V-cycle work vectors (length n_rows); xt: the smoother's second iterate buffer
    DBuf<double> x, xt, b, r, d;
    DBuf<float> x32, xt32, b32, r32, d32;
};

// One smoothed-aggregation hierarchy: its level matrices, transfers, work
// vectors and the inverse of its coarsest matrix.
struct Amg {
    std::vector<Level> levels;
    DBuf<double> coarse_inv;  // inverse of the coarsest matrix: its diagonal blocks, row-major
    DBuf<int> coarse_blk;     // per block: first row, size, offset into coarse_inv
    DBuf<int> coarse_rowblk;  // block of each coarsest row
    int64_t coarse_n = 0;
    bool symmetric = false;   // level-0 matrix found symmetric: Galerkin products mirrored
};

// ILU(0) of the two velocity mass blocks on the node-pair pattern (ilu.cu).
struct MassIlu {
    DBuf<double> lu;          // [n_pairs][2]: packed L (unit lower) and U factors, per network
    DBuf<float> lu32;         // FP32 copy (mixed precision)
    DBuf<int> dpos;           // position of the diagonal in each row
    std::vector<int> lower_ptr, upper_ptr;  // level boundaries (host)
    DBuf<int> lower_rows, upper_rows;       // rows ordered by level
};

// Preconditioner compositions of Section 4 (values of dpp_pc_opts::composition).
enum : int { kFieldSplit = 0, kScaleSplit = 1 };

struct PcImpl {
    int dim = 0;
    int64_t n_nodes = 0;
    int precision = DPP_FP64;
    dpp_pc_opts opts{};
    double mass_lmin = 0.5, mass_lmax = 2.0;  // Wathen bounds of D^-1 M (TRI: [1/2, 2], TET: [1/2, 5/2])
    // Method 2 (field split): one hierarchy on blockdiag(S_p1, S_p2) (n_amg = 1).
    // Method 1 (scale split): amg[i] on S^(i+1)_p alone, one per network (n_amg = 2).
    Amg amg[2];
    int n_amg = 1;
    MassIlu ilu;              // mass_solver = 1 only
    // preconditioner work vectors (node-interleaved, n_nodes * ns)
    DBuf<double> yu, su, tmp, dcheb;
    DBuf<double> tp, yp;      // split pressures [2][n_nodes]
    DBuf<double> mdiag;       // [n_nodes][2]: 1/m1_aa, 1/m2_aa (mass Jacobi)
    // FP32 copies for the mixed-precision preconditioner
    DBuf<float> yu32, su32, tmp32, dcheb32, tp32, yp32, mdiag32, r32;
    HostScratch hs;
    double ms_setup = 0;
};

}  // namespace dpp

struct dpp_problem_s { dpp::ProblemImpl impl; };
struct dpp_pc_s { dpp::PcImpl impl; const dpp_problem_s* owner = nullptr; };
