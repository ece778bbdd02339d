// Internal structures shared by the host analysis and the CUDA numeric phase.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "ndsi.h"

namespace ndsi {

// Operand access modes of the batched complex GEMM, all column-major:
//   OP_N: X(r,c) = X[r + c*ld];  OP_T: X(r,c) = X[c + r*ld];
//   OP_S: symmetric matrix stored in its lower triangle, X(r,c) = X[max + min*ld].
enum OpMode : int32_t { OP_N = 0, OP_T = 1, OP_S = 2 };
// Device buffers addressed by the schedule.  Each holds one slab per pole.
enum BufId : int32_t { BUF_FRONT = 0, BUF_SCR = 1 };

// One sub-matrix product C = alpha*op(A)op(B) + beta*C of a schedule step.  Offsets are in
// complex elements inside the pole's slab of the named buffer.
struct GemmItem {
    int64_t a_off, b_off, c_off;
    int32_t lda, ldb, ldc;
    int32_t M, N, K;
    int32_t pad;
};

// One output tile of a GEMM step: the item and the tile's first row/column.
struct GemmTile {
    int32_t item, m0, n0, pad;
};

// Dense copy dst = scale*src of a rows x cols block between buffers (SCR -> FRONT).
struct CopyItem {
    int64_t src_off, dst_off;
    int32_t lds, ldd, rows, cols;
};

// A diagonal pivot block: nb x nb, lower-valid, at `off` with leading dimension `ld`.
struct DiagItem {
    int64_t off;
    int32_t ld, nb;
};

// Square tile of a node's front (assembly) or of its struct x struct block (gather).
struct NodeTile {
    int32_t node, i0, j0, pad;
};

// Per-node data read by the assembly and gather kernels.
struct NodeDev {
    int64_t front_off;  // complex elements within a pole slab
    int64_t inv_off[2]; // offsets into inv_map for each child (length f of this node), -1 if none
    int64_t rel_off;    // offset into rel_map (length r): struct(J) -> parent's front index
    int32_t f, s, r;
    int32_t nchild;
    int32_t child[2];
    int32_t parent;
    int32_t level;
};

enum LaunchKind : int32_t {
    L_ASSEMBLE = 0,  // pull children's Schur updates into the fronts of a level (and zero)
    L_SCATTER = 1,   // add z*S - H entries of the level's nodes
    L_DIAGINV = 2,   // FP64 inverse of diagonal pivot blocks
    L_GEMM = 3,      // batched complex GEMM step
    L_COPY = 4,      // SCR -> FRONT block copies (scaled by +1 or -1)
    L_GATHER = 5,    // selected-inverse gather of G_RR from the parent front
};

struct Launch {
    int32_t kind;
    int32_t level;
    int32_t opA, opB, bufA, bufB, bufC, lower;
    double alpha, beta;
    int64_t first, count;    // range in the item array of this kind
    int64_t tfirst, tcount;  // GEMM tiles range
    int32_t tile;            // FP64 GEMM output tile edge (16 or 32); pivot-sweep width of a diag launch
    int32_t exact;           // 1: FP64 CUDA-core GEMM in every precision mode (diagonal blocks)
    int32_t phase;           // 0 factor, 1 selinv
    int32_t tag;             // which formula the step implements (for profiling names)
    double flops;            // algorithmic real flops per pole of this launch
    double bytes;            // algorithmic global-memory bytes per pole of this launch
};

// Tags of the schedule steps.
enum StepTag : int32_t {
    T_ASSEMBLE = 0, T_SCATTER, T_DINV, T_PANEL, T_UPDATE, T_PCOPY, T_AINV_T, T_AINV_D,
    T_AINV_COPY, T_LRJ, T_SCHUR, T_LCOPY, T_GATHER, T_SEL_T, T_SEL_D, T_SEL_COPY,
    T_OPANEL, T_OUPDATE, T_OPCOPY, T_OAINV_T, T_OAINV_D, T_OAINV_COPY
};

// GEMM launches that split mode runs on the tensor cores.
inline bool split_eligible(const Launch& l) { return l.kind == L_GEMM && !l.exact; }

struct Plan {
    // input structure
    int64_t n = 0, nnz = 0;
    int32_t n_atoms = 0;
    std::vector<int64_t> rowptr;
    std::vector<int32_t> col;
    ndsi_options opt{};
    // dissection
    std::vector<int32_t> perm_atoms;   // structured position -> atom
    std::vector<int32_t> perm_basis;   // structured position -> basis
    std::vector<int32_t> ipos_basis;   // basis -> structured position
    std::vector<int32_t> node_atom_first;  // [n_nodes+1] atom positions
    std::vector<int32_t> node_first;       // [n_nodes+1] basis positions
    std::vector<int32_t> parent, level, nchild;
    std::vector<int32_t> child0, child1;
    std::vector<int64_t> struct_ptr;       // [n_nodes+1] into struct_atoms
    std::vector<int32_t> struct_atoms;     // atom ids
    std::vector<int64_t> sstruct_ptr;      // [n_nodes+1] into struct_basis
    std::vector<int32_t> struct_basis;     // structured basis positions
    int32_t n_nodes = 0, n_levels = 0;
    std::vector<std::vector<int32_t>> level_nodes;
    // fronts
    std::vector<int32_t> f, s, r;
    std::vector<int64_t> front_off;
    int64_t front_total = 0;               // complex elements per pole
    std::vector<int64_t> scr_off;          // per node, within its level
    int64_t scr_total = 0;                 // complex elements per pole
    int32_t max_front = 0;
    // index tables
    std::vector<int64_t> asm_map;          // [nnz] front offset or -1
    std::vector<int64_t> out_map;          // [nnz] front offset of G_ij (lower storage)
    std::vector<int32_t> inv_map;          // concatenated per child
    std::vector<int32_t> rel_map;          // concatenated per node (length r)
    std::vector<NodeDev> nodes;
    // schedule
    std::vector<int64_t> scatter_idx;      // CSR entries grouped by level
    std::vector<GemmItem> gemm_items;
    std::vector<GemmTile> gemm_tiles;
    std::vector<CopyItem> copy_items;
    std::vector<DiagItem> diag_items;
    std::vector<NodeTile> node_tiles;      // assembly and gather tiles
    std::vector<Launch> launches;
    double flops_per_pole = 0, bytes_per_pole = 0;
    int32_t block = 16;
    int32_t outer = 128;   // diagonal-block size of the two-level factorisation of A_J
    std::vector<std::vector<int64_t>> level_entries;  // CSR entries scattered per level
    // systems of a batched plan (one for a plain plan)
    int32_t n_systems = 1;
    std::vector<int64_t> sys_nnz_first;   // [n_systems+1] pattern-entry offsets
    std::vector<int64_t> sys_n_first;     // [n_systems+1] basis offsets
    std::vector<int32_t> entry_sys;       // [nnz] system of each pattern entry
    // device-side state (owned by the numeric phase)
    void* dev = nullptr;
};

// Host analysis entry (analyze.cpp).  Returns NDSI_OK or an error code, with `err` set.
int analyze(const ndsi_pattern* pat, int32_t n_atoms, const double* centers,
            const int32_t* atom_of_basis, const ndsi_options& opt, Plan& plan, std::string& err);

// Schedule and scratch layout from the node structure; merging of per-system plans.
void compute_scratch(Plan& P);
void build_schedule(Plan& P);
int merge_plans(std::vector<Plan>& parts, Plan& merged, std::string& err);

// Bounds and write-overlap check of every schedule table (plan_check.cpp).
int check_plan(const Plan& P, std::string& err);

// Chemical-potential search over caller-supplied evaluations (mu_search.cpp).
int mu_search(ndsi_mu_eval_fn eval, ndsi_mu_dos_fn dos, void* ctx, double elo, double ehi, double kT,
              double n_electrons, int32_t n_grid, double mu_lo, double mu_hi, double tol, int32_t max_iter,
              double* mu_out, double* dn_out, int32_t* evals_out, std::string& err);

// The same search for several systems in lockstep, one batched callback per round.
int mu_search_batched(int32_t ns, ndsi_mu_eval_batch_fn eval, ndsi_mu_dos_batch_fn dos, void* ctx,
                      const double* elo, const double* ehi, const double* kT, const double* n_electrons,
                      int32_t n_grid, const double* mu_lo, const double* mu_hi, double tol, int32_t max_iter,
                      double* mu_out, double* dn_out, int32_t* evals_out, int32_t* rounds_out, std::string& err);

// Continued-fraction poles (analyze.cpp).
int cf_poles(int32_t M, double* z, double* R, std::string& err);

// Tile sizes shared by the schedule and the kernels.
constexpr int kGemmTile = 32;     // largest FP64 GEMM output tile (rows and columns)
constexpr int kGemmTileSmall = 16;  // output tile for launches whose items are small
constexpr int kNodeTile = 32;     // assembly / gather tile

void set_last_error(const std::string& msg);

}  // namespace ndsi
