// Handle layouts (opaque behind include/pdd.h) and the stage drivers the
// C ABI calls.  Device arrays are structure-of-arrays in HBM.
#pragma once

#include <vector>

#include "common.cuh"

struct pdd_cover {
    pdd_domain domain;
    int M = 0, M_floating = 0, N = 0;
    int64_t nnz = 0;
    int max_nk = 0, max_stencil = 0;
    double max_r = 0.0, min_r = 0.0;
    // circles
    pdd::DevBuf<double> cx, cy, r, theta_s;
    pdd::DevBuf<uint8_t> floating;
    pdd::DevBuf<int> nk, nr, nt;
    pdd::DevBuf<int> knot_ptr;             // [M+1]
    // knots
    pdd::DevBuf<double> kx, ky, ku;
    pdd::DevBuf<int> kowner, row_sub;
    pdd::DevBuf<uint8_t> kdir;
    // Pi_i, the subdomains row i integrates in (ascending): pi_sub[pi_ptr[i] .. pi_ptr[i+1]);
    // one per interior row, or all that hold the knot for averaged rows (Eq. 38-39)
    int averaged = 0, npairs = 0;
    pdd::DevBuf<int> pi_ptr, pi_sub;
    // rows grouped by subdomain: rows of circle m are sub_rows[sub_ptr[m] .. sub_ptr[m+1]); per
    // entry p: its subdomain sub_m, the position sub_k of that subdomain in Pi_i, the offset
    // sub_off of Xi_m's first column in the CSR row; pair_spos[pi_ptr[i] + k] = p
    pdd::DevBuf<int> sub_ptr, sub_rows, sub_m, sub_k, sub_off, pair_spos;
    // CSR pattern
    pdd::DevBuf<int> rowptr, col;
    // spatial hash of circles (uniform grid of pitch max_r)
    int gx = 0, gy = 0;
    double gx0 = 0, gy0 = 0, gh = 1;
    pdd::DevBuf<int> cell_ptr, cell_items;
    // host copies of small per-circle data
    std::vector<int> h_knot_ptr, h_sub_ptr, h_nk, h_nr, h_nt;
    std::vector<uint8_t> h_floating;
};

struct pdd_system {
    int N = 0;
    int64_t nnz = 0;
    const pdd_cover *cov = nullptr;
    pdd::DevBuf<double> val, b, se, se_b;
    pdd::DevBuf<double> bs, se_bs;         // r and its SE per (row, subdomain) entry of sub_rows
    // Monte Carlo raw estimates
    int n_mc = 0;
    // per Monte Carlo slot: row, subdomain, entry of sub_rows, position of the subdomain in Pi_i
    pdd::DevBuf<int> mc_rows, mc_subs, mc_spos, mc_kword, mom_ptr;
    pdd::DevBuf<double> moments, bmean;
    pdd::DevBuf<int> mc_np;                // paths run for each Monte Carlo row
    pdd_assembly_stats stats{};
    int precision = 0;
};

namespace pdd {

// the form each stage runs in: `precision`, unless the stage's own override is set
inline bool disk_mixed(const pdd_assembly_opts &o) {
    return o.disk_precision != PDD_STAGE_DEFAULT ? o.disk_precision == PDD_STAGE_MIXED : o.precision == PDD_PREC_MIXED;
}
inline bool path_mixed(const pdd_assembly_opts &o) {
    return o.path_precision != PDD_STAGE_DEFAULT ? o.path_precision == PDD_STAGE_MIXED : o.precision == PDD_PREC_MIXED;
}

// device problem description (uploads the operator's host arrays)
struct ProblemHolder {
    Problem P{};
    DevBuf<double> rbf_x, rbf_y, rbf_w, g_coef, frbf_x, frbf_y, frbf_w;
    DevBuf<float> rbf32, frbf32;
    void set(const pdd_domain &dom, const pdd_operator &op, cudaStream_t st);
};

// stage drivers (each file implements its own)
void build_cover_impl(const pdd_domain &dom, const pdd_cover_spec &spec, pdd_cover &cov,
                      cudaStream_t st);
void assemble_dirichlet(const pdd_cover &cov, const Problem &P, pdd_system &sys, cudaStream_t st);

struct DiskStats {
    int disks = 0, rows = 0, max_sweeps = 0, unconverged = 0;
    float ms_operator = 0, ms_factor = 0, ms_refine = 0, ms_eval = 0;
    int lu_blocked = 0, lu_leaf = 0, lu_tmin = 0;          // factorisation used (mixed form)
    int lu_fallback = 0;                                   // a pivot-free wave was redone pivoted
    float ms_trisolve = 0, ms_tc_gemm = 0;                 // kernel-only device times (mixed form)
    int64_t disk_solves = 0;                               // (disk, sweep) triangular solves
    double tc_gemm_flop = 0;                               // useful flops of the tensor-core launches
    float ms_gemm_fused = 0;                               // the fused-split part of ms_tc_gemm
    double gemm_fused_flop = 0, gemm_fused_bytes = 0;      // its flops and algorithmic bytes
    int64_t gemm_pipe_launches = 0;                        // launches of the pre-split (pipelined) kernel
};

// CUDA events bracketing consecutive stages on one stream
struct StageTimer {
    cudaEvent_t ev[8];
    int n = 0;
    cudaStream_t st;
    explicit StageTimer(cudaStream_t s, int count) : n(count), st(s) {
        for (int k = 0; k < n; ++k) PDD_CUDA(cudaEventCreate(&ev[k]));
    }
    void mark(int k) { PDD_CUDA(cudaEventRecord(ev[k], st)); }
    float ms(int a, int b) {
        float t = 0;
        cudaEventElapsedTime(&t, ev[a], ev[b]);
        return t;
    }
    ~StageTimer() {
        for (int k = 0; k < n; ++k) cudaEventDestroy(ev[k]);
    }
};
DiskStats assemble_disks(const pdd_cover &cov, const Problem &P, const pdd_assembly_opts &o,
                         pdd_system &sys, cudaStream_t st);

struct McStats {
    int rows = 0, extended_rows = 0;
    int64_t steps = 0, capped = 0, paths_total = 0;
    float ms_paths = 0, ms_finalize = 0;
};
McStats assemble_mc(const pdd_cover &cov, const Problem &P, const pdd_assembly_opts &o,
                    pdd_system &sys, cudaStream_t st);

struct SolveResult {
    int iters = 0;
    double rel = 0;
    int converged = 0;
};
// one-level RAS preconditioner of Eq. 42-44 (ras.cu)
struct RasPrecond {
    int P = 0, N = 0, NP = 0;                  // subsets, rows, padded subset size
    DevBuf<int> wptr, widx, p1, l1, p2, l2;
    DevBuf<float> cinvT, z;
    void build(const pdd_cover &cov, const int *rowptr, const int *col, const double *val, cudaStream_t st);
    void apply(const double *v, double *y, cudaStream_t st) const;
};

SolveResult gmres_csr(int n, const int *rowptr, const int *col, const double *val, const double *b,
                      double *u, const pdd_solve_opts &o, cudaStream_t st, const RasPrecond *M = nullptr);
void spmv_csr(int n, const int *rowptr, const int *col, const double *val, const double *x,
              double *y, cudaStream_t st);
// explicit transpose of a CSR pattern + values (rows of the result sorted)
void csr_transpose(int n, int64_t nnz, const int *rowptr, const int *col, const double *val,
                   DevBuf<int> &rowptr_t, DevBuf<int> &col_t, DevBuf<double> &val_t,
                   cudaStream_t st);

// adjoint pieces: per-disk (floating rows) and per-row (Monte Carlo) partial
// gradients, summed in a fixed order by grad_impl
void grad_disks(const pdd_cover &cov, const Problem &P, const double *u, const double *lambda,
                DevBuf<double> &partial, int &n_part, cudaStream_t st);
void grad_mc(const pdd_cover &cov, const Problem &P, const pdd_assembly_opts &o, const pdd_system &sys,
             const double *u, const double *lambda, DevBuf<double> &partial, int &n_part,
             cudaStream_t st);
// K^-1 of every perimeter stencil (offsets per circle, -1 when none)
void build_imq_inverses(const pdd_cover &cov, double c2, DevBuf<double> &kinv, DevBuf<long> &koff_m,
                        DevBuf<double> &kcond, cudaStream_t st);

void grad_impl(const pdd_cover &cov, const Problem &P, const pdd_assembly_opts &o,
               const pdd_system &sys, const double *u, const double *dJdu, double *grad,
               double *lambda, cudaStream_t st);

// recursive LU of a batch of FP32 matrices on the tensor cores (lu_rec.cu)
// W = leaf panel width (8, 16, 32); GEMMs with M, N, K >= tensor_min go to the tensor cores
void lu_recursive_f32(float *A, int n, long strideA, int *perm, int *info, int nd, cudaStream_t st, int W,
                      int tensor_min, float *ms_gemm = nullptr, double *gemm_flop = nullptr);

// batched split-TF32 tensor-core GEMM C_b (-)= A_b B_b (tc_gemm.cu); `alias` states how C meets
// the operands, scratch holds pre-split tiles for the cases the fused kernel does not take
enum { TC_ALIAS_NONE = 0, TC_ALIAS_A = 1, TC_ALIAS_B = 2, TC_ALIAS_UNKNOWN = 3 };
// CUDA event pairs around the GEMM kernels (not the operand splits), by kernel form, with the useful
// flops (2MNK per matrix) and, for the fused form, the algorithmic bytes (A and B read once, C
// written, or read and written when subtracting)
struct TcTiming {
    std::vector<cudaEvent_t> pipe, fused;
    double flop_pipe = 0, flop_fused = 0, bytes_fused = 0;
};
void tc_gemm(int batch, int M, int N, int K, const float *A, long sA, int lda, bool transA, const float *B, long sB,
             int ldb, bool transB, float *C, long sC, int ldc, bool sub, int alias, float *scratch,
             size_t scratch_floats, int *err, cudaStream_t st, TcTiming *tt);
bool tc_gemm_fused_ok(int batch, int M, int N, int K, const float *A, long sA, int lda, bool transA, const float *B,
                      long sB, int ldb, bool transB, const float *C, long sC, int ldc, int alias);
size_t tc_tile_floats(int rows, int K);

// device-wide exclusive scan of int32 counts by warp scans (out[n] = the total): the _async form
// queues the work on st and returns at once (the total optionally to *total_dev); exclusive_scan
// also returns the total to the host (one synchronisation)
void exclusive_scan_async(const int *in, int *out, int n, cudaStream_t st, long long *total_dev);
int64_t exclusive_scan(const int *in, int *out, int n, cudaStream_t st);

}  // namespace pdd
