/*
 * ndsi.h - nested-dissection selected inversion for contour-integrated density matrices.
 *
 * C ABI of the GB300 (sm_103a) library libndsi.so.  Problem statement (Sec. II.A-II.B of
 * Ozaki, "Numerically exact O(N^{7/3}) method for large-scale electronic structure
 * calculations"): given real symmetric H and S on one sparse pattern (Eq. 2 and the remark
 * that both share the same sparse structure), a chemical potential mu and temperature kT,
 * return the density matrix rho on that pattern (Eq. 8) and the electron count Tr(rho S)
 * (Eq. 40), through the Green function G(Z) = (Z S - H)^{-1} (Eq. 6) evaluated at the poles
 * alpha_p = mu + i z_p / beta of the continued fraction of the Fermi function (Eq. 7).
 *
 * Conventions
 *  - Every function returns an int status (NDSI_OK = 0); the message of the last failure on
 *    the calling thread is available from ndsi_last_error().  No C++ exception crosses the ABI.
 *  - Complex numbers are passed as interleaved (re, im) pairs of double.
 *  - Arrays "on the pattern" are indexed like the CSR arrays of ndsi_pattern (original basis
 *    order, row-major CSR order).
 *  - Pointers documented as "device or host" are classified with cudaPointerGetAttributes:
 *    host memory is staged through the library's device buffers on the given stream.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls are
 *    stream-ordered; results written to device memory are valid after the stream reaches them.
 *  - The caller owns every input and output buffer.  The library owns plan and factor
 *    handles (and the device workspace behind them) and frees them in *_destroy.
 *  - All work runs on the current CUDA device.  A plan may be used by one stream at a time.
 */
#ifndef NDSI_H
#define NDSI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define NDSI_OK               0
#define NDSI_ERR_INVALID      1   /* bad pattern, sizes, options or pointer */
#define NDSI_ERR_SINGULAR     2   /* a diagonal pivot block was singular or non-finite */
#define NDSI_ERR_OOM          3   /* device or host allocation failed, or over the workspace cap */
#define NDSI_ERR_CUDA         4   /* a CUDA runtime call failed */
#define NDSI_ERR_TIMEOUT      5   /* a bounded device wait gave up */
#define NDSI_ERR_UNSUPPORTED  6   /* feature not available on this device or build */

/* Arithmetic of the dense contractions (separator Schur updates and selected-inverse
 * products).  Diagonal pivot blocks, their inverses and the residue sum are FP64 in both. */
#define NDSI_PREC_FP64   0   /* FP64 operands and accumulation on the CUDA cores */
#define NDSI_PREC_SPLIT  1   /* FP64 emulated by BF16 slices on the tcgen05 tensor cores */

typedef struct ndsi_plan ndsi_plan;
typedef struct ndsi_factors ndsi_factors;

/* Symmetric sparsity pattern of H and S (CSR, original basis order).  Every row must hold its
 * diagonal, column indices must be strictly increasing within a row, and (i,j) present implies
 * (j,i) present.  Host pointers; read only during ndsi_analyze. */
typedef struct {
    int64_t n;              /* number of basis functions */
    const int64_t* rowptr;  /* [n+1], rowptr[0] = 0, rowptr[n] = nnz */
    const int32_t* col;     /* [nnz] */
} ndsi_pattern;

typedef struct {
    int32_t leaf_atoms;          /* innermost-domain threshold of the dissection (default 20) */
    int32_t precision;           /* NDSI_PREC_FP64 or NDSI_PREC_SPLIT (default FP64) */
    int32_t split_slices;        /* BF16 slices per operand in split mode, 4..7; 0 (default) = 6 */
    int32_t block;               /* FP64 pivot block size, 16/32/64 (0 = default 16) */
    double m0_radius;            /* R of the zeroth-moment point Z = iR (default 1e7) */
    int64_t max_workspace_bytes; /* device workspace cap; poles are chunked to fit (0 = auto) */
    int32_t outer_block;         /* diagonal-block size of the two-level factorisation of A_J: the
                                    block's own LDL^T and inverse run in FP64 pivot blocks, the
                                    panel, trailing update and inverse assembly outside it are the
                                    GEMMs that split mode moves to the tensor cores; a multiple of
                                    `block` (0 = default 128) */
    int32_t split_bands;         /* TMEM accumulators of the split GEMM: 0 (default) = one per
                                    slice-product scale t+u (every scale exact; 40 complex columns
                                    per tile, 32 with seven slices); 4 (t+u = 2, 3, 4 exact, the
                                    rest in one tail accumulator whose low bits the tensor core
                                    drops; 64 columns) or 5 (t+u = 2..5 exact; 48 columns) */
    double cell[3];              /* periodic cell lengths along x, y, z in the units of `centers`;
                                    0 (default) = open along that axis.  On a periodic axis the
                                    dissection orders atoms by their coordinate wrapped into
                                    [0, L) and sees each neighbour at its image nearest the atom
                                    (Sec. II.C.1 step (i): ordering numbers l*N_d + q in the
                                    periodic cells), so a separator can wrap around the cell */
    int32_t screen_degree;       /* long-tail screening (Sec. II.C.1 step (ii)): atoms adjacent to
                                    more than this many atoms join the root separator before the
                                    dissection; 0 (default) = off */
    double split_far_ratio;      /* split mode, density sweeps only: poles with z_p >= ratio * z_1
                                    (farther from the real axis, Eq. 8) run with split_slices - 1
                                    slices.  The error a GEMM leaves in G(alpha_p) grows with the
                                    condition of alpha_p S - H (~ spectral width / Im alpha_p), and
                                    the pole's weight in rho is ~ 1 / Im alpha_p of its G, so one
                                    digit fewer (2^8 larger product error) at Im alpha_p >= 32 Im
                                    alpha_1 leaves each far pole's contribution below the nearest
                                    pole's.  M0, the moment points of the energy density and every
                                    pole of ndsi_factor_poles / ndsi_dos keep split_slices.
                                    0 (default) = 32; negative = off (every point split_slices) */
} ndsi_options;

/* Summary of a plan, filled by ndsi_plan_info. */
typedef struct {
    int64_t n;                 /* basis functions */
    int64_t nnz;               /* pattern entries */
    int32_t n_atoms;
    int32_t n_nodes;           /* supernodes of the dissection tree (innermost domains + separators) */
    int32_t n_levels;          /* tree levels (0 = innermost domains) */
    int32_t max_front;         /* largest dense front |J| + |struct(J)| */
    int64_t front_elems;       /* sum of front sizes squared (complex elements per pole) */
    double flops_per_pole;     /* algorithmic real FP64 flops of factor + selected inversion */
    double bytes_per_pole;     /* algorithmic front bytes written + read per pole */
    int32_t n_launches;        /* schedule launches per pole batch (factor + selected inversion) */
    int32_t n_systems;         /* systems in the plan (1 unless built by ndsi_analyze_batched) */
    int32_t split_slices;      /* slices per operand of a split plan (0 for an FP64 plan) */
    int32_t split_bands;       /* accumulators of a split plan (the slice count when there is one
                                  per scale; 0 for an FP64 plan) */
} ndsi_plan_summary;

/* Items for ndsi_plan_export. */
#define NDSI_EXPORT_PERM_ATOMS   1  /* int32[n_atoms]: structured position -> atom id */
#define NDSI_EXPORT_PERM_BASIS   2  /* int32[n]: structured position -> basis index */
#define NDSI_EXPORT_NODE_ATOMS   3  /* int32[n_nodes+1]: first structured atom position per node */
#define NDSI_EXPORT_PARENT       4  /* int32[n_nodes]: parent node (-1 = root), nodes in postorder */
#define NDSI_EXPORT_STRUCT_PTR   5  /* int64[n_nodes+1]: offsets into NDSI_EXPORT_STRUCT_ATOMS */
#define NDSI_EXPORT_STRUCT_ATOMS 6  /* int32[...]: struct(J) as atom ids, by structured position */
#define NDSI_EXPORT_LEVEL        7  /* int32[n_nodes]: tree level of each node */
#define NDSI_EXPORT_SCHEDULE     8  /* int32[4*n_launches]: (kind, level, step tag, items) per launch
                                       of one pole batch, in issue order; n_launches from
                                       ndsi_plan_info.n_launches */
#define NDSI_EXPORT_TILE_SHAPES  9  /* int32[n_launches]: per launch of the schedule, -1 (not a GEMM),
                                       0 (a GEMM on the FP64 CUDA cores) or the complex columns per
                                       128-row tile of its tensor-core kernel (40 one accumulator per
                                       slice scale, 48 five bands, 64 four bands, 32 seven slices),
                                       as the split options and ndsi_autotune left them */

/* Fill *opt with the defaults listed above. */
void ndsi_default_options(ndsi_options* opt);

/* Poles z_p (ascending, z_1 ~ pi) and residues R_p (< 0) of the Fermi continued fraction of
 * Eq. 7 truncated after the denominator 4M-1, so that
 *   1/(1+e^x) ~= 1/2 + sum_{p=1..M} R_p/(x - i z_p) + R_p/(x + i z_p).
 * Host arrays z_out[M], R_out[M].  Pure host computation (symmetric tridiagonal eigenproblem
 * of order 2M).  Errors: NDSI_ERR_INVALID if M < 1 or a pointer is NULL. */
int ndsi_poles(int32_t M, double* z_out, double* R_out);

/* Structure analysis (Sec. II.C.1, once per geometry): geometric nested dissection of the
 * atoms along the three axes (steps i-v), the binary separator tree, the supernodal
 * structure struct(J) of every node, and every index table the numeric phase needs
 * (the "table function" of Sec. II.C.2).  Integer only; runs on the host.
 *   pat            - pattern of H and S (host).
 *   n_atoms        - number of atoms.
 *   centers        - host double[n_atoms*3], Cartesian centre of each atom.
 *   atom_of_basis  - host int32[n], atom owning each basis function.
 *   opt            - options (NULL = defaults).
 *   plan_out       - receives the plan; free with ndsi_plan_destroy.
 * Errors: NDSI_ERR_INVALID for a malformed pattern, NDSI_ERR_OOM. */
int ndsi_analyze(const ndsi_pattern* pat, int32_t n_atoms, const double* centers,
                 const int32_t* atom_of_basis, const ndsi_options* opt, ndsi_plan** plan_out);

/* Batched analysis: n_systems independent systems of uneven size in one plan.  Each system is
 * dissected on its own (as by ndsi_analyze); the supernodes of all systems are then merged level by
 * level (level = height above the innermost domains), so every launch of the factor and of the
 * selected inversion processes one tree level of every system and every pole at once.  Pattern
 * arrays of the batch are the systems' arrays concatenated in order.
 *   pats[i], n_atoms[i], centers[i], atom_of_basis[i] - as for ndsi_analyze, per system.
 * ndsi_density_batched, ndsi_find_mu_batched, ndsi_factor_poles and ndsi_selinv accept the plan;
 * ndsi_density, ndsi_density_energy, ndsi_dos, ndsi_find_mu, ndsi_mu_features,
 * ndsi_factors_solve and ndsi_eigenstates need a single-system plan (NDSI_ERR_INVALID
 * otherwise).  The options (including `cell`) apply to every system. */
int ndsi_analyze_batched(int32_t n_systems, const ndsi_pattern* pats, const int32_t* n_atoms,
                         const double* const* centers, const int32_t* const* atom_of_basis,
                         const ndsi_options* opt, ndsi_plan** plan_out);

/* Density matrices of every system of a batched plan, each at its own mu[i] and kT[i] (host
 * arrays of n_systems), with the same pole count: as ndsi_density, with H, S and rho_out the
 * systems' pattern arrays concatenated (device or host) and n_elec_out[i] = Tr(rho_i S_i)
 * (device or host array of n_systems, may be NULL).  Synchronises `stream`. */
int ndsi_density_batched(ndsi_plan* plan, const double* H, const double* S, const double* mu,
                         const double* kT, int32_t n_poles, double* rho_out, double* n_elec_out,
                         void* stream);

/* One rank's share of ndsi_density_batched when the poles are divided among processes (the
 * (pole, system) pairs of the batch, split by pole): for every system of the plan, M0 if with_m0
 * plus the poles pole_begin <= p < pole_end of an n_poles expansion, and each system's
 * Tr(rho_part S) in n_elec_out[i].  Summed over ranks whose ranges partition [0, n_poles) with one
 * with_m0, the shares give ndsi_density_batched's results (ndsi_pole_shard picks the ranges).
 * Arguments, outputs and errors as ndsi_density_batched, plus NDSI_ERR_INVALID for a bad range. */
int ndsi_density_batched_poles(ndsi_plan* plan, const double* H, const double* S, const double* mu,
                               const double* kT, int32_t n_poles, int32_t pole_begin, int32_t pole_end,
                               int32_t with_m0, double* rho_out, double* n_elec_out, void* stream);

/* Sizes and cost figures of a plan (ndsi_plan_summary above) into the caller's *out.
 * Errors: NDSI_ERR_INVALID for NULL arguments. */
int ndsi_plan_info(const ndsi_plan* plan, ndsi_plan_summary* out);

/* Host-only check of a plan's schedule (no GPU work): every index the kernels follow (GEMM items
 * and tiles, copies, pivot blocks, assembly/gather tiles, scatter entries, index maps) stays in
 * its buffer and front, and no two work items of one launch write overlapping memory or read
 * what another item of the launch writes.  NDSI_OK, or NDSI_ERR_INVALID with the first violation
 * in ndsi_last_error. */
int ndsi_plan_check(const ndsi_plan* plan);

/* Copy one structure table of the plan (see NDSI_EXPORT_*) into host memory `out`, which must
 * hold the documented number of elements.  Errors: NDSI_ERR_INVALID for an unknown item. */
int ndsi_plan_export(const ndsi_plan* plan, int32_t what, void* out);

/* Factor X_p = z_p S - H for every p in nested-dissection order as a supernodal block LDL^T
 * (Eqs. 18-21 applied recursively; the Schur complements of Eq. 32 and the recurrence of
 * Eqs. 28-31 appear as dense front updates), no pivoting across supernodes.
 *   H, S     - values on the pattern, double[nnz], device or host.
 *   z        - n_poles complex points, interleaved double[2*n_poles], host.
 *   n_poles  - >= 1.  Im z_p != 0 keeps every leading block nonsingular for S SPD.
 *   f_out    - receives the factors (device fronts of all poles); free with ndsi_factors_destroy.
 * The factors hold all poles at once; NDSI_ERR_OOM if they do not fit.  Singular pivot blocks
 * are reported by ndsi_selinv (the check needs a stream synchronisation). */
int ndsi_factor_poles(ndsi_plan* plan, const double* H, const double* S, const double* z,
                      int32_t n_poles, ndsi_factors** f_out, void* stream);

/* Selected inversion (Eqs. 38-39, Takahashi/Erisman-Tinney form) of factors from
 * ndsi_factor_poles: G_ij(z_p) for every (i,j) of the pattern.
 *   G_out - device or host, interleaved complex double[2 * n_poles * nnz], pole-major
 *           (G_out[2*(p*nnz + k)] is Re G(z_p) at pattern entry k); NULL skips the gather.
 * Synchronises `stream`.  Errors: NDSI_ERR_SINGULAR (pivot check), NDSI_ERR_CUDA. */
int ndsi_selinv(ndsi_factors* f, double* G_out, void* stream);

/* Solve (z_p S - H) X = Y with the factors of pole p (App. B, Eqs. B8-B15, in supernodal form:
 * forward elimination leaves first, y_R(J) -= L_RJ y_J; the diagonal step w_J = A_J^{-1} y_J;
 * back substitution root first, x_J = w_J - L_RJ^T x_R(J)).  Valid until ndsi_selinv runs on the
 * same factors (it overwrites them with G).
 *   pole   - 0 <= pole < n_poles of ndsi_factor_poles.
 *   Y      - k complex right-hand sides, interleaved double[2 * n * k], row-major by basis
 *            index (Y[2*(i*k + c)] is Re of row i of right-hand side c), original basis order;
 *            device or host; not modified.
 *   X_out  - the solutions in the same layout, device or host.
 * Synchronises the stream.  Errors: NDSI_ERR_INVALID (null pointers, k < 1, pole out of range,
 * factors already inverted, a batched plan), NDSI_ERR_OOM, NDSI_ERR_CUDA. */
int ndsi_factors_solve(ndsi_factors* f, int32_t pole, const double* Y, int32_t k, double* X_out,
                       void* stream);

/* Density matrix by the contour sum of Eq. 8 with M = n_poles pole pairs:
 *   rho = M0 + sum_p w_p Re G(alpha_p),  alpha_p = mu + i z_p/beta,  w_p = -4 R_p/beta,
 * with M0 = Re(iR G(iR)) (the zeroth moment, R = opt.m0_radius), and
 *   n_elec = Tr(rho S) = sum_k rho_k S_k.
 *   H, S       - values on the pattern, double[nnz], device or host.
 *   rho_out    - double[nnz], device or host.
 *   n_elec_out - one double, device or host (may be NULL).
 * Runs factor, selected inversion and the residue sum for all poles (chunked to the
 * workspace cap) and synchronises `stream`.  Errors: NDSI_ERR_INVALID (kT <= 0, n_poles < 1),
 * NDSI_ERR_SINGULAR, NDSI_ERR_OOM, NDSI_ERR_CUDA. */
int ndsi_density(ndsi_plan* plan, const double* H, const double* S, double mu, double kT,
                 int32_t n_poles, double* rho_out, double* n_elec_out, void* stream);

/* One rank's share of the contour sum of Eq. 8 when the poles are divided among processes
 * (Sec. III.D: the poles are independent, and the only exchange is the sum of the results):
 *   rho_part   = [M0 if with_m0] + sum_{pole_begin <= p < pole_end} w_p Re G(alpha_p),
 *   n_elec_part = Tr(rho_part S) = sum_k rho_part_k S_k,
 * with the poles, weights and M0 of ndsi_density for the same n_poles, mu and kT.  When the
 * ranges of all ranks partition [0, n_poles) and exactly one rank sets with_m0, the sums over
 * ranks of rho_part and n_elec_part are ndsi_density's rho and Tr(rho S) (equal up to the order
 * of the floating-point additions).  An empty share (pole_begin == pole_end, with_m0 = 0) writes
 * zeros.  Arguments, outputs and synchronisation as ndsi_density; single-system plans only
 * (ndsi_density_batched_poles is the batched form).
 * Errors: NDSI_ERR_INVALID (0 <= pole_begin <= pole_end <= n_poles violated, a batched plan, or
 * as ndsi_density), otherwise as ndsi_density. */
int ndsi_density_poles(ndsi_plan* plan, const double* H, const double* S, double mu, double kT,
                       int32_t n_poles, int32_t pole_begin, int32_t pole_end, int32_t with_m0,
                       double* rho_out, double* n_elec_out, void* stream);

/* The pole range of `rank` among `world` processes for ndsi_density_poles: contiguous ranges
 * [floor(r M / W), floor((r + 1) M / W)), whose sizes differ by at most one, and with_m0 set on
 * the first rank holding the smallest number of poles (rank 0 when all are equal), so that every
 * rank sums about the same number of points.  Host only.  Errors: NDSI_ERR_INVALID (M < 1,
 * world < 1, rank outside [0, world), NULL outputs). */
int ndsi_pole_shard(int32_t n_poles, int32_t rank, int32_t world, int32_t* pole_begin,
                    int32_t* pole_end, int32_t* with_m0);

/* Per-kernel timing.  While enabled, every launch made for this plan by ndsi_factor_poles,
 * ndsi_selinv and ndsi_density is bracketed by CUDA events on its stream; durations, launch
 * counts and the algorithmic flops and bytes of the launches accumulate per kernel family.
 * ndsi_profile_enable(plan, 1) also clears the counters; 2 does the same and splits the GEMM and
 * slicing families by tree level (":L<level>" appended to the name); 0 stops recording. */
typedef struct {
    char name[32];        /* kernel family and schedule step: "gemm_f64:<step>", "slice:<step>",
                             "gemm_split:<step>", diaginv, assemble, scatter, copy, gather,
                             accumulate, reduce */
    int64_t launches;     /* launches recorded */
    double ms;            /* summed event-timed durations of those launches */
    double flops;         /* summed algorithmic real flops (complex MAC = 8 flops) */
    double bytes;         /* summed algorithmic global-memory bytes (reads + writes) */
    double tensor_flops;  /* summed tensor-core flops issued (split GEMM only) */
} ndsi_profile_entry;

/* Start (enable = 1 or 2, counters cleared) or stop (0) the per-kernel timing of the plan.
 * While it is on, density sweeps launch their kernels directly (no graph replay) so that each
 * launch can be bracketed by events.  Errors: NDSI_ERR_INVALID for a NULL plan. */
int ndsi_profile_enable(ndsi_plan* plan, int32_t enable);

/* Autotuner for split-precision plans: times every GEMM step of one density sweep at (mu, kT,
 * n_poles) on H, S (device or host) both on the tensor cores (slicing + emulated-FP64 GEMM) and
 * on the FP64 CUDA cores, with CUDA events per launch after an untimed warm-up of each, and keeps
 * the faster path per step for all later calls on the plan.  Both paths meet the split-mode
 * tolerance, so only speed changes.  Small steps (few tiles, short inner dimension) usually go
 * to the CUDA cores, separator-sized ones to the tensor cores.  A step whose tensor-core time is
 * below the least time the FP64 cores could need for it (its issued FP64 flops at the DFMA rate
 * measured on the device, as ndsi_fp64_peak) is decided without an FP64 run, so on large systems
 * the FP64 sweeps time only the small steps.  A plan with the default accumulators (one per
 * slice scale) then times every tensor-core step once more with five accumulator bands (48
 * complex columns per tile instead of 40, within the same tolerance) and keeps the faster tile per
 * step (NDSI_EXPORT_TILE_SHAPES lists the result); factors made before the call can no longer be
 * inverted by ndsi_selinv.  Counts of the steps left on each path in
 * *n_split_out / *n_fp64_out (either may be NULL).  Runs four to six sweeps; the profiler counters are
 * unchanged and any captured graph is dropped.  FP64 plans: no-op (all steps
 * counted as FP64).  Errors: NDSI_ERR_INVALID for bad arguments or a batched plan; as
 * ndsi_density otherwise. */
int ndsi_autotune(ndsi_plan* plan, const double* H, const double* S, double mu, double kT, int32_t n_poles,
                  int32_t* n_split_out, int32_t* n_fp64_out, void* stream);

/* Density matrix and energy density matrix (Eq. 10) on the pattern in one sweep:
 *   e = M1 + kappa M0 - (4/beta) sum_p R_p Re(alpha_p G(alpha_p)),  kappa = (4/beta) sum_p R_p,
 * with M0 = S^{-1} and M1 = S^{-1} H S^{-1} the zeroth and first moments of G.  The poles and the
 * M0 point are those of ndsi_density (their factors are shared); M1 comes from three more points
 * z = Re, -Re, i Re as (Re^2/4) [G(Re) + G(-Re) - 2 Re G(i Re)]: with the fourth point -i Re (the
 * conjugate of i Re) these are the four roots Re i^k, which cancel every moment but M1, M5, ...,
 * so the truncation is (spectral radius / Re)^4 relative.  Re = 1000 x the Gershgorin bound of
 * the pencil's spectrum (max_i sum_j |H_ij| over min_i (S_ii - sum_{j!=i} |S_ij|)), computed on
 * the device; this replaces the two-point moment formula the paper prints (whose truncation is
 * O(|M2|/R)).  rho_out, e_out: nnz doubles each (device or host); n_elec_out: Tr(rho S) (may be
 * NULL).  Single-system plans only.  Errors as ndsi_density. */
int ndsi_density_energy(ndsi_plan* plan, const double* H, const double* S, double mu, double kT,
                        int32_t n_poles, double* rho_out, double* e_out, double* n_elec_out, void* stream);

/* CUDA graphs.  While enabled (the default) and profiling is off, ndsi_density,
 * ndsi_density_batched and ndsi_find_mu run each density sweep (all chunks of points: assembly,
 * factorisation, selected inversion, residue sum and electron counts) as one CUDA graph,
 * captured on a private stream at the first call and replayed by later calls on the caller's
 * stream.  A graph is recaptured when a buffer it names changes (H, S or output pointers, the
 * workspace, the number of points); the chemical potential and temperature are read from device
 * memory at run time and need no recapture.  ndsi_graph_enable(plan, 0) launches every kernel
 * directly instead and frees the graph.  Errors: NDSI_ERR_INVALID for a NULL plan. */
int ndsi_graph_enable(ndsi_plan* plan, int32_t enable);

/* Kernel nodes of the plan's current captured sweep in *nodes_out (0 when none is held). */
int ndsi_graph_info(const ndsi_plan* plan, int64_t* nodes_out);

/* Copy up to max_entries families into `out` (host) and their number into *n_out.
 * Errors: NDSI_ERR_INVALID for NULL arguments. */
int ndsi_profile_read(const ndsi_plan* plan, ndsi_profile_entry* out, int32_t max_entries,
                      int32_t* n_out);

/* FP64 throughput of the current GPU in TFLOP/s (host *tflops_out): every SM runs 2048 threads
 * of eight independent fused multiply-add chains (2 flops each), timed with CUDA events on
 * `stream`, best of five launches after a warm-up (about 0.1 s in all).  This is the measured
 * ceiling of the FP64 path's kernels (the paper's arithmetic is FP64 throughout, Sec. II; GB300
 * runs FP64 on the CUDA cores only), against which their roofline fractions are quoted.
 * Synchronises `stream`.  Errors: NDSI_ERR_INVALID (NULL output), NDSI_ERR_CUDA. */
int ndsi_fp64_peak(double* tflops_out, void* stream);

/* Residue sum and electron count from caller-held G, allocating no device memory.
 * The paper has no counterpart: this is a library convenience for callers that cannot call
 * cudaMalloc (a host framework that owns the whole device-memory budget, or a latency-critical
 * path where cudaMalloc/cudaFree, which can synchronise the device, are not allowed).  It runs the
 * residue-sum kernel of ndsi_density with its partial traces kept in a fixed 256 KiB
 * file-scope __device__ array instead of an allocated buffer:
 *   rho_out[k]  = sum_q Re(c_q * G[q][k])         (the residue-weighted sum of G),
 *   *n_elec_out = sum_k rho_out[k] * S[k]          (the trace of rho S).
 *   G          - device, interleaved complex double[2 * n_points * nnz], point-major (the layout
 *                ndsi_selinv writes), 16-byte aligned.
 *   c          - device, interleaved complex double[2 * n_points], 16-byte aligned: w_p = -4 R_p kT
 *                for the poles alpha_p, and iR for the zeroth-moment point iR.
 *   S          - device double[nnz]; rho_out device double[nnz]; n_elec_out device double or NULL.
 * Every array must be device memory of the current device (or managed memory).
 * Limit: nnz <= 8,388,608 (32768 blocks of 256 entries); larger nnz -> NDSI_ERR_INVALID.
 * Host pointers, another device's memory, or a misaligned G or c -> NDSI_ERR_INVALID, with no
 * launch.  Stream-ordered, no synchronisation.  The first call on a device resolves the array's
 * device address (cudaGetSymbolAddress) with that device current, so make that first call before
 * any stream capture; the address is kept for the life of the process, so a cudaDeviceReset (or
 * any other teardown of the device's primary context) invalidates this entry point on that
 * device.  Every call on a device shares the one array: calls whose kernels overlap on the GPU
 * (other streams or threads) race on it. */
int ndsi_residue_sum_static(const double* G, const double* c, int32_t n_points, const double* S,
                            int64_t nnz, double* rho_out, double* n_elec_out, void* stream);

/* Selected eigenstates near an energy xi (App. B): the n_states pairs of H c = eps S c with the
 * smallest |eps - xi|, by the block shift-invert iteration (B2)-(B3).  The pencil is factored once
 * at z = xi + i eta (eta > 0 keeps every pivot block nonsingular without pivoting; the paper's
 * real shift is the limit eta -> 0); each step forms b = (z S - H)^{-1} S c for the `block`
 * vectors c with that factorisation (ndsi_factors_solve's three steps), solves (B3) in the real
 * span of Re b and Im b (2 x block vectors; S-Gram directions below 1e-12 of the largest are
 * dropped) and keeps the `block` Ritz pairs nearest xi.  The loop stops when the n_states nearest
 * have |H c - eps S c|_2 < tol (c S-normalised).  In split precision each solve takes one step
 * of FP64 iterative refinement (residual y - (zS - H) b with the exact H and S, solved again with
 * the same factors), so the iteration converges to the pencil's own eigenpairs.
 *   H, S       - values on the pattern, device or host.
 *   xi, eta    - the shift; eta > 0 (about the wanted level spacing or smaller).
 *   n_states   - >= 1;  block - n_states..32, and <= n.
 *   max_iter   - >= 1;  tol > 0;  seed - of the starting block (counter-based uniform [-1, 1)).
 *   eps_out    - host double[n_states], ascending.
 *   C_out      - device or host double[n_states * n]: state j at C_out[j*n + i], original basis
 *                order, S-orthonormal, largest-magnitude component positive.
 *   resid_out  - host double[n_states] or NULL;  iters_out - host or NULL.
 * Synchronises the stream.  Errors: NDSI_ERR_INVALID (arguments, a batched plan),
 * NDSI_ERR_TIMEOUT (not converged in max_iter; the current pairs are still written),
 * NDSI_ERR_SINGULAR (pivot check, non-finite projections or a collapsed search space),
 * NDSI_ERR_OOM, NDSI_ERR_CUDA. */
int ndsi_eigenstates(ndsi_plan* plan, const double* H, const double* S, double xi, double eta,
                     int32_t n_states, int32_t block, int32_t max_iter, double tol, uint64_t seed,
                     double* eps_out, double* C_out, double* resid_out, int32_t* iters_out,
                     void* stream);

/* Density of states from the retarded Green function (Eq. 41):
 *   D(E_k) = -(2/pi) Im Tr(G(E_k + i eta) S),  G(z) = (z S - H)^{-1},
 * the spin-summed density of states broadened by a Lorentzian of half-width eta (for each
 * generalised eigenvalue eps_nu it contributes (2/pi) eta / ((E - eps_nu)^2 + eta^2)).  One
 * sweep of factorisation and selected inversion over the n_energies points (chunked to the
 * workspace), then Tr(G S) = sum over the pattern of G_ij S_ij.  Single-system plans only.
 *   H, S        - values on the pattern, device or host.
 *   energies    - host double[n_energies], the real parts E_k.
 *   eta         - > 0, the imaginary part shared by every point.
 *   dos_out     - host double[n_energies], D(E_k).
 * Synchronises the stream before returning.
 * Errors: NDSI_ERR_INVALID (null or device energies/dos_out, n_energies < 1, eta <= 0, a
 * non-finite energy, a batched plan), NDSI_ERR_OOM, NDSI_ERR_CUDA, and the pivot errors of
 * ndsi_factor_poles (an energy on the real axis exactly at a singular point cannot occur for
 * eta > 0). */
int ndsi_dos(ndsi_plan* plan, const double* H, const double* S, const double* energies,
             int32_t n_energies, double eta, double* dos_out, void* stream);

/* Callbacks of ndsi_mu_search: DeltaN(mu) = Tr(rho(mu) S) - n_electrons into *dn, and the
 * density of states D(E_k) = -(2/pi) Im Tr(G(E_k + i eta) S) for n energies into D.  Return 0 on
 * success; any other value stops the search, which returns it. */
typedef int (*ndsi_mu_eval_fn)(void* ctx, double mu, double* dn);
typedef int (*ndsi_mu_dos_fn)(void* ctx, const double* E, int32_t n, double eta, double* D);

/* The search of ndsi_find_mu over caller-supplied evaluations (host only, no GPU work): solves
 * DeltaN(mu) = 0 (Eq. 40) for an increasing DeltaN inside the spectral bounds [elo, ehi].
 *   With mu_lo < mu_hi the bracket is evaluated first; otherwise, when `dos` is given, one call
 *   of it on n_grid energies evenly spanning [elo, ehi] (eta two grid spacings) builds the
 *   density-of-states model of procedure (2) (Eqs. 41-43) and the search starts where the
 *   model holds n_electrons; without `dos`, at the middle of the bounds.
 *   While all evaluations have one sign it steps by the model anchored at the best point
 *   (DeltaN_i + integral D [f((E - mu)/kT) - f((E - mu_i)/kT)] dE = 0), or by doubling steps
 *   when that stalls.  With both signs it takes the Muller step (procedure (4), Eqs. 45-46) on the
 *   three points of smallest |DeltaN| with both signs, else the linear step (procedure (3),
 *   Eq. 44 with the denominator read as DeltaN_i - DeltaN_j), else the anchored model step, any
 *   of them only strictly inside the bracket, and bisects after a step that does not halve the
 *   smallest |DeltaN|.
 *   mu_out, dn_out, evals_out - host; the best mu, its DeltaN, and the evaluations used (the
 *   density-of-states call counts as one).  They are written on every return.
 * Errors: NDSI_ERR_INVALID (elo >= ehi, kT <= 0, tol <= 0, max_iter < 1, no sign change within
 * the bounds), NDSI_ERR_TIMEOUT (not converged in max_iter), NDSI_ERR_SINGULAR (non-finite
 * DeltaN), or a callback's own non-zero return. */
int ndsi_mu_search(ndsi_mu_eval_fn eval, ndsi_mu_dos_fn dos, void* ctx, double elo, double ehi,
                   double kT, double n_electrons, int32_t n_grid, double mu_lo, double mu_hi,
                   double tol_electrons, int32_t max_iter, double* mu_out, double* dn_out,
                   int32_t* evals_out);

/* Callbacks of ndsi_mu_search_batched, each answering one round for all systems at once:
 * DeltaN_s(mu_s) for every system s into dn[s], and D_s(E_s,k) for the n energies of every system
 * (E and D row-major n_systems x n, eta[s] per system).  active[s] = 1 marks the systems whose
 * search asked for the round; the others' values are ignored.  Return 0 on success. */
typedef int (*ndsi_mu_eval_batch_fn)(void* ctx, int32_t n_systems, const int32_t* active, const double* mu,
                                     double* dn);
typedef int (*ndsi_mu_dos_batch_fn)(void* ctx, int32_t n_systems, const int32_t* active, const double* E,
                                    int32_t n, const double* eta, double* D);

/* ndsi_mu_search for n_systems systems in lockstep (host only): every system runs its own search
 * (per-system elo, ehi, kT, n_electrons and optional brackets mu_lo/mu_hi, NULL for none), and
 * each round answers all pending requests of one kind with one batched callback, so a batched
 * plan needs one sweep per round instead of one per system and step.
 *   mu_out, dn_out, evals_out - host arrays [n_systems] (dn_out, evals_out may be NULL);
 *   rounds_out                - host, the batched callbacks made.
 * The search of each system runs on a worker thread; the callbacks run on the calling thread.
 * Errors: as ndsi_mu_search, for the first failing system (its index in ndsi_last_error). */
int ndsi_mu_search_batched(int32_t n_systems, ndsi_mu_eval_batch_fn eval, ndsi_mu_dos_batch_fn dos,
                           void* ctx, const double* elo, const double* ehi, const double* kT,
                           const double* n_electrons, int32_t n_grid, const double* mu_lo,
                           const double* mu_hi, double tol_electrons, int32_t max_iter, double* mu_out,
                           double* dn_out, int32_t* evals_out, int32_t* rounds_out);

/* Chemical-potential search (Sec. II.C.3): find mu with
 *   DeltaN(mu) = Tr(rho(mu) S) - n_electrons = 0      (Eq. 40)
 * to |DeltaN| < tol_electrons.  Every trial mu is one full contour evaluation (ndsi_density).
 * The bracket [mu_lo, mu_hi] (e.g. from a learned seed) is checked first and, if it does not
 * enclose the root, widened step by step towards the Gershgorin bounds of the pencil (H, S).
 * With mu_lo >= mu_hi the search starts from the density of states of the retarded Green
 * function instead (procedure (2), Eqs. 41-43: ndsi_dos on n_poles + 1 energies spanning the
 * bounds, one sweep of factorisation and selected inversion, counted as one evaluation).  The
 * steps are those of ndsi_mu_search, each trial mu one contour evaluation.
 *   H, S            - values on the pattern, device or host.
 *   rho_out         - rho at the returned mu, device or host (double[nnz]).
 *   mu_out, n_elec_out, iters_out - host scalars (iters = contour sweeps used).
 * Errors: NDSI_ERR_INVALID (kT <= 0, n_poles < 1, tol <= 0, no sign change within the bounds),
 * NDSI_ERR_TIMEOUT if max_iter evaluations do not converge (the best mu is still returned),
 * and every error of ndsi_density. */
int ndsi_find_mu(ndsi_plan* plan, const double* H, const double* S, double kT, int32_t n_poles,
                 double n_electrons, double mu_lo, double mu_hi, double tol_electrons,
                 int32_t max_iter, double* rho_out, double* mu_out, double* n_elec_out,
                 int32_t* iters_out, void* stream);

/* ndsi_find_mu for every system of a batched plan at once: the searches run in lockstep
 * (ndsi_mu_search_batched), each round one batched contour sweep (ndsi_density_batched) or one
 * batched retarded-Green-function sweep with a grid per system, so the cost is that of the
 * slowest system's search, not the sum.
 *   kT, n_electrons       - host double[n_systems];
 *   mu_lo, mu_hi          - host double[n_systems] brackets, or NULL (procedure (2) start);
 *   rho_out               - device or host double[nnz of the batched plan], rho at mu_out;
 *   mu_out, n_elec_out    - host double[n_systems] (n_elec_out may be NULL);
 *   rounds_out            - host, the batched sweeps used (the density-of-states sweep counts).
 * Errors: those of ndsi_find_mu (for the first failing system) and NDSI_ERR_INVALID for a
 * non-positive kT or a non-finite electron count. */
int ndsi_find_mu_batched(ndsi_plan* plan, const double* H, const double* S, const double* kT,
                         int32_t n_poles, const double* n_electrons, const double* mu_lo,
                         const double* mu_hi, double tol_electrons, int32_t max_iter, double* rho_out,
                         double* mu_out, double* n_elec_out, int32_t* rounds_out, void* stream);

/* ---- Learned seed for the chemical-potential search (not in the paper; it only proposes the
 * starting bracket of ndsi_find_mu, whose exact evaluations still decide the result). ----
 * Network: 32 inputs -> 64 tanh -> 64 tanh -> 1 output, FP32, parameters packed as
 * [W1 (64x32 row-major), b1 (64), W2 (64x64), b2 (64), W3 (64), b3 (1)]. */
#define NDSI_MLP_INPUTS 32
#define NDSI_MLP_HIDDEN 64
#define NDSI_MLP_PARAMS 6337

/* Input features of a system (device or host float[32]):
 *   [0..23]  Chebyshev moments (1/N) Tr T_k(H/4), k = 1..24 (fixed window [-4, 4] Ha),
 *   [24..29] Chebyshev moments (1/N) Tr T_k((S - I)/0.75), k = 1..6,
 *   [30] filling n_electrons/(2N), [31] 10*kT (Ha),
 * traces estimated with n_vectors Rademacher vectors from a counter-based generator (seed).
 * Errors: NDSI_ERR_INVALID, NDSI_ERR_OOM, NDSI_ERR_CUDA. */
int ndsi_mu_features(ndsi_plan* plan, const double* H, const double* S, double n_electrons,
                     double kT, int32_t n_vectors, uint64_t seed, float* feat_out, void* stream);

/* params (device float[NDSI_MLP_PARAMS]) <- Glorot-uniform weights, zero biases. */
int ndsi_mlp_init(float* params, uint64_t seed, void* stream);
/* Y[s] = network(X[s, :]) for s < n; X device float[n*32], Y device float[n]. */
int ndsi_mlp_forward(const float* params, const float* X, int32_t n, float* Y, void* stream);
/* grad (device float[NDSI_MLP_PARAMS]) and loss (device float, may be NULL) of the mean squared
 * error (1/n) sum_s (network(X_s) - T_s)^2.  Synchronises the stream. */
int ndsi_mlp_grad(const float* params, const float* X, const float* T, int32_t n, float* grad,
                  float* loss, void* stream);
/* `steps` full-batch Adam steps (beta1 0.9, beta2 0.999) on the mean squared error; final loss
 * to *loss_out (host, may be NULL).  Synchronises the stream. */
int ndsi_mlp_train(float* params, const float* X, const float* T, int32_t n, int32_t steps,
                   float lr, float* loss_out, void* stream);

/* Free a plan (its device tables, workspaces, staging, captured graph) or a factors handle (its
 * fronts of every pole).  NULL is ignored.  Destroy every factors handle of a plan before the
 * plan; no call of the handle may be in flight on any stream. */
void ndsi_plan_destroy(ndsi_plan* plan);
void ndsi_factors_destroy(ndsi_factors* f);

/* Message of the last failing call on this thread ("" if none).  Valid until the next call. */
const char* ndsi_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NDSI_H */
