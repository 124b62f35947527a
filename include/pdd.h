/*
 * pdd.h -- C ABI of the GB300 (sm_103a) library for the explicit interfacial
 * system of "An explicit substructuring method for overlapping domain
 * decomposition based on stochastic calculus" (Moron-Vidal, Bernal, Suzuki).
 *
 * The library assembles the sparse, nonsymmetric system C u = r of Eq. 28-30
 * over a cover of overlapping circles (Sec. 2.1), solves it in FP64 and
 * differentiates a misfit of u.  Every step runs in CUDA kernels on the
 * current device; there is no CPU fallback.
 *
 * Conventions shared by every entry point:
 *   - Handles (pdd_cover, pdd_system) own their device memory and are freed
 *     by the matching destroy call.  Structs passed in are read during the
 *     call only (host pointers inside them are copied).
 *   - "dev" pointers are device pointers owned by the caller; "host"
 *     pointers are host memory.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     queued on it; calls that return counts or statuses synchronise it.
 *   - Every call returns a pdd_status; PDD_OK is 0.  pdd_last_error()
 *     returns a thread-local message for the last failure.
 *   - Sizes are counts of elements unless stated.
 */
#ifndef PDD_H
#define PDD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PDD_OK = 0,
    PDD_EINVAL = 1,            /* bad argument or degenerate discretisation        */
    PDD_ECOVER_GAP = 2,        /* Eq. 5 violated: a point of Omega is uncovered     */
    PDD_ECIRCLE_OUTSIDE = 3,   /* Eq. 5 violated: an explicit circle misses Omega   */
    PDD_EKNOT_UNCOVERED = 4,   /* Sec. 2.1: a knot lies inside no other subdomain  */
    PDD_ENOCONV = 5,           /* iterative refinement or GMRES did not converge   */
    PDD_EPATH_CAP = 6,         /* a Monte Carlo path reached its step cap          */
    PDD_ENOMEM = 7,            /* device allocation failed                          */
    PDD_ECUDA = 8,             /* CUDA runtime error                                */
    PDD_EDUPLICATE_KNOT = 9    /* two knots closer than 1e-12                       */
} pdd_status;

/* ---------------------------------------------------------------------------
 * Problem statement, Eq. 1-3:  L u + c u + f = 0 in Omega, u = g on dOmega,
 * with L = (1/2) Laplacian + b . grad  (sigma = I in Eq. 3).
 * ------------------------------------------------------------------------- */

enum { PDD_DOMAIN_SQUARE = 0,   /* p = {x0, y0, x1, y1}: (x0,x1) x (y0,y1)        */
       PDD_DOMAIN_DISK = 1 };   /* p = {cx, cy, R, unused}                         */

typedef struct {
    int kind;
    double p[4];
} pdd_domain;

enum { PDD_B_ZERO = 0, PDD_B_SINX_COSY = 1 };                 /* b = (sin x, cos y)  */
enum { PDD_C_ZERO = 0, PDD_C_QUADRATIC = 1,                    /* c = -(1+x^2+y^2)    */
       PDD_C_RBF = 2 };              /* c = min(0, sum_p w_p exp(-|x-x_p|^2/(2 s^2))) */
enum { PDD_F_ZERO = 0, PDD_F_ONE = 1,
       PDD_F_MANUFACTURED = 2,       /* f = -(L u* + c u*), u* = sin(pi x) cos(pi y)  */
       PDD_F_EQ46 = 3,               /* f = -(L u46 + c u46), u46 = exact solution of
                                        the Poisson test, Eq. 46:
                                        3 + sin(sqrt(1+x^2/100+y^2/50))/3
                                          + tanh(sin(3x/25+y/20) + sin(x/20-3y/25))/3 */
       PDD_F_RBF = 4 };              /* f = sum_q v_q exp(-|x-x_q|^2/(2 s_f^2))       */
enum { PDD_G_EXP_SIN = 0,            /* g = e^x sin y                                 */
       PDD_G_SIN_COS = 1,            /* g = sin(pi x) cos(pi y)                       */
       PDD_G_BOUNDARY_FOURIER = 2,   /* g(s) = sum_k a_k cos(2 pi k s/P) + b_k sin(.)  */
       PDD_G_ONE = 3, PDD_G_ZERO = 4,
       PDD_G_EQ46 = 5 };             /* g = u46 (Eq. 46)                              */

typedef struct {
    int b_kind, c_kind, f_kind, g_kind;
    int n_rbf;                        /* PDD_C_RBF: number of Gaussians            */
    const double *rbf_x, *rbf_y;      /* host, n_rbf centres                        */
    const double *rbf_w;              /* host, n_rbf weights                        */
    double rbf_sigma;                 /* Gaussian width                             */
    int n_gcoef;                      /* PDD_G_BOUNDARY_FOURIER: K_c + K_s          */
    const double *g_coef;             /* host: a_0..a_{Kc-1}, b_1..b_{Ks}; Kc = ceil(n/2),
                                         s = arclength counter-clockwise from (x0,y0),
                                         P = perimeter of the square               */
    int n_frbf;                       /* PDD_F_RBF: number of Gaussians of f        */
    const double *frbf_x, *frbf_y;    /* host, n_frbf centres                       */
    const double *frbf_w;             /* host, n_frbf weights v_q                   */
    double frbf_sigma;                /* Gaussian width s_f                         */
} pdd_operator;

/* ---------------------------------------------------------------------------
 * Cover (Eq. 4-7) and its discretisation (Eq. 8-12).
 * ------------------------------------------------------------------------- */

enum { PDD_COVER_SQUARE_LATTICE = 0,  /* centres (x_o + i s, y_o + j s)             */
       PDD_COVER_HEX_LATTICE = 1,     /* rows y_o + k s sqrt(3)/2, x_o + i s (+ s/2 on odd k) */
       PDD_COVER_EXPLICIT = 2 };      /* centres, radii and grids given per circle  */

typedef struct {
    int kind;
    int nx, ny;                       /* lattice index box, i < nx, j (or k) < ny   */
    double x_origin, y_origin, spacing, radius;
    int n_knots, n_r, n_theta;        /* uniform discretisation (lattices)          */
    int n_explicit;                   /* PDD_COVER_EXPLICIT: number of circles       */
    const double *cx, *cy, *r;        /* host, n_explicit                           */
    const int *n_knots_per, *n_r_per, *n_theta_per;   /* host, n_explicit           */
    int row_mode;                     /* PDD_ROWS_FARTHEST or PDD_ROWS_AVERAGED     */
} pdd_cover_spec;

/* Which subdomains a knot's row integrates in (Sec. 3.2):
 *   FARTHEST: the one whose interface is farthest from the knot (Eq. 29-30);
 *   AVERAGED: every subdomain whose open disk holds the knot, summed (Eq. 38-39):
 *             C_ii = #Pi_i, C_ij = the subdomains' entries of their stencils,
 *             r_i = the sum of their r's.  The k-th subdomain of a row draws its
 *             paths with Philox counter word 3 = k.  RAS and the adjoint
 *             gradient take FARTHEST covers only (PDD_EINVAL otherwise). */
enum { PDD_ROWS_FARTHEST = 0, PDD_ROWS_AVERAGED = 1 };

typedef struct pdd_cover pdd_cover;
typedef struct pdd_system pdd_system;

/*
 * pdd_build_cover -- Eq. 4-12 and Sec. 3.2 on the device.
 *   Lattice circles that miss Omega are dropped (Eq. 5, right); explicit
 *   circles that miss Omega give PDD_ECIRCLE_OUTSIDE.  Circles are floating
 *   when the closed disk lies in open Omega (Eq. 7).  Knots: theta_j = 2 pi j/n
 *   on full circles; on arcs the same candidates strictly inside Omega and
 *   at least 0.25 * 2 pi/n from every junction, plus one knot per junction
 *   (Dirichlet rows).  Knots are numbered circle by circle, each circle's
 *   knots by local angle from the midpoint of its largest outside arc.
 *   Each interior knot's row goes to the circle maximising r_m - |x_i - c_m|
 *   (Sec. 3.2, footnote 3), ties within 1e-12 r to the lowest index; with
 *   row_mode PDD_ROWS_AVERAGED it goes to every circle m != owner with
 *   r_m - |x_i - c_m| > 1e-12 r_owner (Eq. 38-39).
 *   Requires n_knots and n_theta even, n_r >= 1.  Checks Eq. 5 on a sample
 *   grid of pitch min(r)/4 (PDD_ECOVER_GAP).  Synchronises `stream`.
 */
pdd_status pdd_build_cover(const pdd_domain *domain, const pdd_cover_spec *spec,
                           pdd_cover **out, void *stream);

/* Counts: circles M, floating circles, knots N, nonzeros of C. */
pdd_status pdd_cover_info(const pdd_cover *cov, int *M, int *M_floating, int *N, int64_t *nnz);

/*
 * pdd_cover_arrays -- device pointers (owned by the cover, valid until
 * pdd_destroy_cover) to the cover and its discretisation:
 *   cx, cy, r [M] (double); floating [M] (uint8); knot_ptr [M+1] (int32, the
 *   stencil Xi_m is the knot range [knot_ptr[m], knot_ptr[m+1]));
 *   kx, ky, ku [N] (double; ku = local unwrapped angle); kowner [N] (int32);
 *   kdir [N] (uint8, 1 = knot on dOmega); row_sub [N] (int32, subdomain of
 *   each row, -1 for Dirichlet rows); rowptr [N+1], col [nnz] (int32 CSR
 *   pattern of Eq. 29, columns sorted).  Any output pointer may be NULL.
 */
pdd_status pdd_cover_arrays(const pdd_cover *cov, const double **cx, const double **cy,
                            const double **r, const uint8_t **floating, const int **knot_ptr,
                            const double **kx, const double **ky, const double **ku,
                            const int **kowner, const uint8_t **kdir, const int **row_sub,
                            const int **rowptr, const int **col);

void pdd_destroy_cover(pdd_cover *cov);

/* ---------------------------------------------------------------------------
 * Assembly of C and r (Eq. 28-35, 40-41).
 * ------------------------------------------------------------------------- */

enum { PDD_PREC_FP64 = 0,       /* disk LU, solves and paths all in FP64             */
       PDD_PREC_MIXED = 1 };    /* FP32 disk LU + FP64 refinement; FP32 path
                                   positions, FP64 weights and score sums           */

enum { PDD_FACTOR_RECURSIVE_TC = 0,      /* recursive LU without row interchanges, every step
                                             but the 64 x 64 diagonal blocks on tcgen05 (the
                                             row-equilibrated collocation matrices keep growth
                                             factor 1); a wave with a pivot below 1e-5, or
                                             whose refinement does not converge, is redone
                                             with PDD_FACTOR_PIVOTED_TC.  With lu_leaf_width > 0:
                                             PDD_FACTOR_PIVOTED_TC with that leaf width     */
       PDD_FACTOR_BLOCKED = 1,            /* one CTA per disk, right-looking, partial pivoting,
                                             CUDA cores                                      */
       PDD_FACTOR_PIVOTED_TC = 2 };       /* recursive LU with partial pivoting, Schur updates
                                             on tcgen05; with lu_leaf_width = 0 the library
                                             times the candidate leaf widths and tensor-core
                                             thresholds on the first wave of each grid size
                                             and keeps the fastest                           */          /* one CTA per disk, right-looking, CUDA cores      */

enum { PDD_FLOATING_PSEUDOSPECTRAL = 0,   /* Sec. 3.3 (default)                      */
       PDD_FLOATING_MONTE_CARLO = 1 };    /* integrate floating rows by paths too     */

/* Per-stage overrides of `precision`: the floating disks (a6-a9) and the Monte
 * Carlo paths (a11) may take different forms, e.g. mixed disks with FP64 paths
 * on the oracle's Philox streams. */
enum { PDD_STAGE_DEFAULT = 0,   /* as `precision`                                    */
       PDD_STAGE_FP64 = 1,
       PDD_STAGE_MIXED = 2 };

/* Summation of the IMQ basis moments M_l (a12).  C = -K^-T M amplifies their
 * rounding by up to kappa(K).  AUTO chooses by kappa_1(K) for mixed-form paths and
 * takes FP64 for FP64 paths; a forced choice applies to either path form. */
enum { PDD_SUMS_AUTO = 0,          /* by kappa_1(K): FP32 up to 1e5, double-float up to
                                      1e10, FP64 beyond                              */
       PDD_SUMS_FP32 = 1,          /* FP32 values of phi, FP32 sums of 16 paths       */
       PDD_SUMS_DOUBLE_FLOAT = 2,  /* double-float phi and sums (~1e-13 relative)     */
       PDD_SUMS_FP64 = 3 };

typedef struct {
    int precision;            /* PDD_PREC_*                                          */
    int floating_method;      /* PDD_FLOATING_*                                      */
    int paths;                /* Monte Carlo paths per knot (> 0)                    */
    double h;                 /* Euler-Maruyama time step (> 0)                      */
    uint64_t seed;            /* Philox key word 0 (low 32 bits used)                */
    double imq_c2;            /* IMQ shape c^2 of Eq. 19, the knots' local angle in
                                 radians (1.5 in the paper, Sec. 4)                  */
    int max_refine;           /* refinement sweeps cap (mixed form), e.g. 12         */
    double refine_tol;        /* stop once the correction just applied, or the next
                                 one predicted from the last two, is <= tol |x|_inf
                                 per disk (0 = 1e-12: the refined entries then agree
                                 with FP64 to ~1e-12, against a 1e-10 requirement)  */
    int factor;               /* mixed form's LU: PDD_FACTOR_*                        */
    int lu_leaf_width;        /* recursive LU leaf panel width 8/16/32; 0 = autotune */
    int lu_tensor_min;        /* smallest GEMM side sent to tcgen05; 0 = autotune    */
    int paths_max;            /* > paths: adaptive path counts (pilot = paths)       */
    double se_target;         /* rows whose largest standard error (C entries and r)
                                 exceeds it rerun with paths (se/se_target)^2 paths,
                                 capped at paths_max (rounded up to 32); path ids
                                 continue the pilot's Philox streams                 */
    int boundary_shift;       /* 1: Gobet-Menozzi stopped Euler scheme (Sec. 4: the
                                 paper's perimeter subdomains): exit tests against
                                 the disk and the domain shrunk by c0 sqrt(h),
                                 c0 = -zeta(1/2)/sqrt(2 pi) = 0.5826 (sigma = I), and
                                 the path scored at the projection of its first
                                 point outside onto that piece of the true boundary;
                                 0: plain exit at the first crossing of the segment */
    int max_steps;            /* Euler-Maruyama steps allowed per path; 0 = 50 r^2/h
                                 (about 100 mean exit times).  A path that reaches
                                 the cap is not scored: the call returns
                                 PDD_EPATH_CAP (the system is still created only
                                 when no path was capped)                            */
    int disk_precision;       /* PDD_STAGE_*: form of the floating disks (a6-a9)     */
    int path_precision;       /* PDD_STAGE_*: form of the Monte Carlo paths (a11)    */
    int moment_sums;          /* PDD_SUMS_*: basis sums of the IMQ moments (a12)     */
    int cv_degree;            /* pathwise variance reduction (Sec. 4: the paper's
                                 perimeter rows use one): 0 = off; D = 1..4: the
                                 regression control variate of Milstein and Tretyakov
                                 with the D (D + 3) / 2 martingales
                                 sum_k Y_k sqrt(h) grad psi(X_k) . xi_k of the monomials
                                 psi = ((x - c_x)/r)^a ((y - c_y)/r)^b, 1 <= a + b <= D
                                 (mean zero for any psi); every payoff of a row (basis
                                 moments, r) is regressed on them over the row's paths
                                 and corrected.  pdd_grad takes cv_degree = 0 only     */
} pdd_assembly_opts;

typedef struct {
    int floating_disks;       /* disks solved                                        */
    int floating_rows;        /* rows assembled by the pseudospectral path           */
    int mc_rows;              /* rows assembled by Monte Carlo                       */
    int64_t path_steps;       /* Euler-Maruyama steps taken                          */
    int64_t capped_paths;     /* paths that hit the step cap                          */
    int64_t paths_total;      /* paths run (pilot + adaptive extension)               */
    int extended_rows;        /* rows that ran more than the pilot count              */
    int max_refine_sweeps;    /* most refinement sweeps any disk needed              */
    int unconverged_disks;    /* disks whose refinement missed refine_tol            */
    double ms_cover_rows;     /* device time per stage (CUDA events), milliseconds   */
    double ms_disks;          /*   all floating-disk work (a6-a9)                    */
    double ms_paths;          /*   Euler-Maruyama path kernel (a11)                  */
    double ms_finalize;       /*   Monte Carlo finalize (a12)                         */
    double ms_operator;       /*   collocation operator build (a6)                   */
    double ms_factor;         /*   batched LU (a7)                                    */
    double ms_refine;         /*   solves and refinement residuals (a8)              */
    double ms_eval;           /*   evaluation at the knots (a9)                       */
    int lu_blocked;           /* mixed-form LU used: 1 blocked, 0 recursive with      */
    int lu_leaf_width;        /*   this leaf width (64: the pivot-free LU's diagonal   */
                              /*   blocks) and                                         */
    int lu_tensor_min;        /*   this tensor-core threshold (autotuned or forced)   */
    double ms_trisolve;       /* mixed form: device time of the triangular-solve     */
                              /*   launches alone (CUDA events around each, a8)      */
    double ms_tc_gemm;        /* mixed form: device time of the tensor-core Schur    */
                              /*   update launches alone (a7)                        */
    int64_t disk_solves;      /* (disk, sweep) triangular solves run (a8)            */
    double tc_gemm_flop;      /* useful flops (2MNK per matrix) of those launches    */
    int lu_pivoted_fallback;  /* 1: a wave of the pivot-free LU was redone with partial
                                 pivoting (a tiny pivot or a refinement that missed its
                                 tolerance)                                           */
    double ms_gemm_fused;     /* the part of ms_tc_gemm spent in the kernel that splits
                                 its operands as it stages them (the K = 64 updates) */
    double gemm_fused_flop;   /* their useful flops                                   */
    double gemm_fused_bytes;  /* their algorithmic bytes: A and B read once, C written
                                 (read and written when subtracting)                 */
    int64_t gemm_pipe_launches; /* launches of the kernel that streams pre-split tiles */
} pdd_assembly_stats;

/*
 * pdd_assemble_G -- C (CSR, pattern of the cover) and r on the device.
 *   Dirichlet rows: C_ii = 1, r_i = g(x_i).  Floating rows (Eq. 33, 35): per
 *   disk one Chebyshev(r) x Fourier(theta) collocation matrix, factored once
 *   (partial-pivoting LU), solved for 1 + #Xi right-hand sides and
 *   evaluated at the disk's knots.  Perimeter rows (Eq. 29-30): Euler-Maruyama
 *   paths of dX = b dt + dW, dY = c Y dt, dZ = f Y dt from the knot, stopped
 *   at the exit from the disk n Omega; IMQ cardinals (Eq. 22) on the arc.
 *   Philox4x32-10 normals: key (seed, knot), counter (step, path, 0, 0).
 *   Synchronises `stream`.  PDD_EPATH_CAP when a path exceeds 50 r^2/h steps.
 */
pdd_status pdd_assemble_G(const pdd_cover *cov, const pdd_operator *op,
                          const pdd_assembly_opts *opts, pdd_system **out, void *stream);

/*
 * pdd_system_csr -- device pointers owned by the system: val [nnz] (C in the
 * cover's CSR pattern), b [N] (r), se [nnz] (standard error of Monte Carlo
 * entries, 0 elsewhere), se_b [N].  Any output pointer may be NULL.
 */
pdd_status pdd_system_csr(const pdd_system *sys, const double **val, const double **b,
                          const double **se, const double **se_b);

/*
 * pdd_cover_rows -- the subdomains each row integrates in (device, owned by
 * the cover): Pi_i = pi_sub[pi_ptr[i] .. pi_ptr[i+1]) (int32, ascending); one
 * entry per interior row for PDD_ROWS_FARTHEST, every circle holding the knot
 * for PDD_ROWS_AVERAGED, none for Dirichlet rows.  n_pairs = pi_ptr[N].
 */
pdd_status pdd_cover_rows(const pdd_cover *cov, int *n_pairs, const int **pi_ptr, const int **pi_sub);

/*
 * pdd_system_mc_subs -- the subdomain (device int32, owned by the system) of
 * each Monte Carlo slot of pdd_system_mc: slot k integrates knot rows[k] in
 * circle subs[k].  With averaged rows a knot has one slot per subdomain.
 */
pdd_status pdd_system_mc_subs(const pdd_system *sys, const int **subs);

/*
 * pdd_system_mc -- the raw Monte Carlo estimates (device, owned by the
 * system): for the k-th Monte Carlo slot (row id rows[k], subdomain
 * pdd_system_mc_subs), moments
 * [mom_ptr[k], mom_ptr[k+1]) hold E[1_Gamma Y_tau phi_l(u_tau)] (IMQ basis) or
 * E[1_Gamma Y_tau H_j] (Fourier cardinals), and bmean[k] = E[1_dOmega g Y + Z].
 */
pdd_status pdd_system_mc(const pdd_system *sys, int *n_rows, const int **rows,
                         const int **mom_ptr, const double **moments, const double **bmean);

pdd_status pdd_system_stats(const pdd_system *sys, pdd_assembly_stats *stats);

void pdd_destroy_system(pdd_system *sys);

/* ---------------------------------------------------------------------------
 * Global solve (a13): restarted GMRES(m) in FP64 (Sec. 4) on a CSR sparse
 * matrix-vector product, optionally right-preconditioned (Eq. 45) by the
 * one-level restricted additive Schwarz operator of Eq. 42-44.
 * ------------------------------------------------------------------------- */

enum {
    PDD_PRECOND_NONE = 0,
    /* M^-1 = sum_p R_p^T D_p C_p^-1 R_p (Eq. 44) over subsets w_p = the rows
     * assigned to subdomain p (Sec. 3.2) plus their neighbours in the graph of
     * C, the knots of circle p; D_p the partition of unity of Eq. 43.  The C_p
     * (at most 128 x 128) are inverted once per solve in FP32; the iteration
     * and its stopping test stay FP64.  pdd_solve only (it needs the cover). */
    PDD_PRECOND_RAS = 1
};

typedef struct {
    int restart;              /* Krylov subspace size m (1..256)                    */
    int max_iters;            /* total inner iterations cap                          */
    double rtol;              /* stop at |r - C u|_2 <= rtol |r|_2                   */
    int transpose;            /* 1: solve C^T u = r instead                          */
    int precond;              /* PDD_PRECOND_*; pdd_solve_csr and the allocation-    */
                              /*   free entry point take PDD_PRECOND_NONE only       */
} pdd_solve_opts;

typedef struct {
    int iters;
    double rel_residual;      /* true residual after the last restart              */
    int converged;
} pdd_solve_info;

/* Solve the system's C u = r; u_dev [N] caller-owned device memory. */
pdd_status pdd_solve(const pdd_system *sys, const pdd_solve_opts *opts, double *u_dev,
                     pdd_solve_info *info, void *stream);

/*
 * pdd_ras_apply -- y = M_RAS^-1 v (Eq. 44) for the system's C and cover, the
 * operator pdd_solve applies with PDD_PRECOND_RAS; v_dev, y_dev [N] double
 * in device memory.  Builds the operator for the call (same subsets, same
 * FP32 inverses).  PDD_EINVAL for subsets over 128 knots, PDD_ENOCONV for a
 * singular C_p.
 */
pdd_status pdd_ras_apply(const pdd_system *sys, const double *v_dev, double *y_dev, void *stream);

/*
 * Failure injection (tests): with PDD_INJECT_BARRIER_TIMEOUT=1 in the environment, every grid
 * barrier of the solver's fused Arnoldi kernel waits for one block more than the grid holds,
 * with a short poll limit; the blocks give up, record the error and return, and the solve
 * returns PDD_ECUDA ("grid barrier timed out").  The device context stays usable.
 */

/*
 * pdd_solve_csr -- the same solver on any square CSR matrix in device memory
 * (rowptr [n+1], col [nnz] int32 sorted per row; val [nnz], b [n], u [n]
 * double).  u is overwritten (the initial guess is 0).  Workspace is
 * allocated for the call and freed before return.
 */
pdd_status pdd_solve_csr(int n, const int *rowptr_dev, const int *col_dev, const double *val_dev,
                         const double *b_dev, double *u_dev, const pdd_solve_opts *opts,
                         pdd_solve_info *info, void *stream);

/*
 * pdd_solve_csr_noalloc -- pdd_solve_csr without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory while they run -- a process whose device
 * heap belongs to another allocator (a caching allocator that must not be
 * bypassed or fragmented), a latency-critical loop that cannot absorb the
 * device-wide synchronisation of cudaFree, or a service that must not fail
 * with out-of-memory in the middle of a request.
 *   Workspace: a fixed 64 MiB array in device memory, reserved by every GPU
 *   that loads the library and held until the process exits.  The Krylov
 *   basis, partial sums and Hessenberg state of one solve must fit in it:
 *   about (restart + 2) * n * 8 bytes; larger requests return PDD_EINVAL with
 *   the sizes in pdd_last_error() and touch nothing.
 *   The first call on a device looks up the array's device address once
 *   (with that device current); make that first call before any stream
 *   capture on the device.  The address is kept for the process: do not
 *   reset the device (cudaDeviceReset) between calls.
 *   Every call uses the same array, which keeps the previous call's contents
 *   (the solver clears what must start at zero).  Calls that overlap on the
 *   GPU -- on different streams, or from different host threads, on the same
 *   device -- race on the array and give wrong results: serialise them.
 *   opts->transpose must be 0.  Arguments and results are as pdd_solve_csr.
 */
pdd_status pdd_solve_csr_noalloc(int n, const int *rowptr_dev, const int *col_dev,
                                 const double *val_dev, const double *b_dev, double *u_dev,
                                 const pdd_solve_opts *opts, pdd_solve_info *info, void *stream);

/* y = C x (or C^T x when transpose != 0) for a CSR matrix in device memory. */
pdd_status pdd_spmv_csr(int n, const int *rowptr_dev, const int *col_dev, const double *val_dev,
                        const double *x_dev, double *y_dev, int transpose, void *stream);

/*
 * pdd_batched_gemm_sub_tf32x3 -- C_b -= A_b B_b for b < batch (row-major FP32
 * device matrices: A_b M x K with leading dimension lda at A + b*sA, B_b K x N
 * (ldb), C_b M x N (ldc)).  Runs on the tcgen05 tensor cores with split-TF32
 * products (A_hi B_hi + A_hi B_lo + A_lo B_hi, FP32 accumulation): relative
 * error ~1e-6 of sum |A||B|.  It is the Schur-complement update of the
 * recursive disk LU (a7, Eq. 41 solved by LU) and is exposed for reuse and
 * testing.  Synchronises `stream`.
 */
pdd_status pdd_batched_gemm_sub_tf32x3(int batch, int M, int N, int K, const float *A_dev,
                                       long long sA, int lda, const float *B_dev, long long sB,
                                       int ldb, float *C_dev, long long sC, int ldc, void *stream);

/*
 * pdd_batched_gemm_tf32x3 -- C_b -= A_b B_b (subtract != 0) or C_b = A_b B_b, same operands,
 * layouts and split-TF32 accuracy as pdd_batched_gemm_sub_tf32x3, through the pipelined
 * kernel of the pivot-free disk LU (a7): both operands are first split once into hi/lo TF32
 * tiles (128 rows x 32 K, in device memory allocated for the call), then a persistent
 * warp-specialised tcgen05 kernel streams them with bulk copies.  C may alias A or B only in
 * the C = A B form (the operands are read before C is written).  Synchronises `stream`.
 */
pdd_status pdd_batched_gemm_tf32x3(int batch, int M, int N, int K, const float *A_dev, long long sA, int lda,
                                   const float *B_dev, long long sB, int ldb, float *C_dev, long long sC, int ldc,
                                   int subtract, void *stream);

/* ---------------------------------------------------------------------------
 * Adjoint gradient (a14; not in the paper).
 * ------------------------------------------------------------------------- */

/*
 * pdd_grad -- dJ/dw (RBF weights of c, n_rbf values), dJ/dv (RBF weights of
 * f, n_frbf values) and dJ/da (boundary Fourier coefficients of g, n_gcoef
 * values) of a misfit J(u), given u and dJ/du.  lambda solves
 * C^T lambda = dJ/du; floating disks contribute -z^T diag(psi_q 1{c<0}) V to
 * dJ/dw and -z^T psi^f_q to dJ/dv, with A^T z = sum_i lambda_i E_i (transposed
 * disk solves, factors recomputed per disk) and V the disk solution for the
 * interface data of u; perimeter rows replay their Philox paths (common
 * random numbers) and accumulate the pathwise derivatives of Y_tau and Z_tau
 * (Z_tau = sum_k f(X_k) Y_k h, so dZ/dv_q = sum_k psi^f_q(X_k) Y_k h).
 * The operator and options must be those the system was assembled with.
 * grad_dev [n_rbf + n_frbf + n_gcoef] caller-owned device memory, in that
 * order (a family the operator does not use has no entries).
 * lambda_dev [N] may be NULL.  Synchronises `stream`.
 */
pdd_status pdd_grad(const pdd_cover *cov, const pdd_operator *op, const pdd_assembly_opts *opts,
                    const pdd_system *sys, const double *u_dev, const double *dJdu_dev,
                    double *grad_dev, double *lambda_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Diagnostics.
 * ------------------------------------------------------------------------- */

/*
 * pdd_split_df -- the double-float split that the double-float moment sums (a12,
 * PDD_SUMS_DOUBLE_FLOAT) apply to each path record's weight and exit angle, built
 * from the FP64 bit fields by integer operations: hi = v truncated to 24
 * significant bits, lo = the remaining bits rounded to FP32, so |hi + lo - v| <=
 * 2^-47 |v| for 2^-74 <= |v| < 2^128; 2^-126 <= |v| < 2^-74 gives lo = 0 (error
 * below 2^-23 |v|) and |v| < 2^-126 gives hi = lo = 0 with v's sign.
 * v_dev [n] FP64 in, hilo_dev [n][2] FP32 out (hi, lo), both caller-owned device
 * memory, hilo_dev 8-byte aligned.  Synchronises `stream`.
 */
pdd_status pdd_split_df(const double *v_dev, float *hilo_dev, long long n, void *stream);

const char *pdd_last_error(void);

/* Number of kernels this process has launched through the library. */
int64_t pdd_launch_count(void);

/* Library version string. */
const char *pdd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PDD_H */
