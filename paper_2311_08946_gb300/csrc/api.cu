// C ABI entry points (include/pdd.h): argument checks, handles, stage
// drivers and status plumbing.  Every compute step runs in the kernels of
// cover.cu, disk.cu, mc.cu, krylov.cu and adjoint.cu.
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>

#include <vector>

#include "handles.cuh"

namespace pdd {

static thread_local std::string g_err;
static std::atomic<long long> g_launches{0};

void set_error(const std::string &msg) { g_err = msg; }

std::string cuda_msg(cudaError_t e, const char *what) {
    return std::string("CUDA error ") + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ") in " + what;
}

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void ProblemHolder::set(const pdd_domain &dom, const pdd_operator &op, cudaStream_t st) {
    P = Problem{};
    P.dom_kind = dom.kind;
    for (int k = 0; k < 4; ++k) P.dom[k] = dom.p[k];
    P.b_kind = op.b_kind;
    P.c_kind = op.c_kind;
    P.f_kind = op.f_kind;
    P.g_kind = op.g_kind;
    if (op.c_kind == PDD_C_RBF) {
        if (op.n_rbf <= 0 || !op.rbf_x || !op.rbf_y || !op.rbf_w || !(op.rbf_sigma > 0))
            fail(PDD_EINVAL, "c = RBF needs n_rbf > 0, centres, weights and sigma > 0");
        rbf_x.alloc(op.n_rbf);
        rbf_y.alloc(op.n_rbf);
        rbf_w.alloc(op.n_rbf);
        PDD_CUDA(cudaMemcpyAsync(rbf_x.p, op.rbf_x, op.n_rbf * 8, cudaMemcpyHostToDevice, st));
        PDD_CUDA(cudaMemcpyAsync(rbf_y.p, op.rbf_y, op.n_rbf * 8, cudaMemcpyHostToDevice, st));
        PDD_CUDA(cudaMemcpyAsync(rbf_w.p, op.rbf_w, op.n_rbf * 8, cudaMemcpyHostToDevice, st));
        P.n_rbf = op.n_rbf;
        P.rbf_x = rbf_x.p;
        P.rbf_y = rbf_y.p;
        P.rbf_w = rbf_w.p;
        P.rbf_sigma = op.rbf_sigma;
        std::vector<float> f32(3 * (size_t)op.n_rbf);
        for (int q = 0; q < op.n_rbf; ++q) {
            f32[q] = (float)op.rbf_x[q];
            f32[op.n_rbf + q] = (float)op.rbf_y[q];
            f32[2 * op.n_rbf + q] = (float)op.rbf_w[q];
        }
        rbf32.alloc(f32.size());
        PDD_CUDA(cudaMemcpyAsync(rbf32.p, f32.data(), f32.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        PDD_CUDA(cudaStreamSynchronize(st));
        P.rbf32 = rbf32.p;
        P.rbf_inv2s2 = (float)(1.0 / (2.0 * op.rbf_sigma * op.rbf_sigma));
    }
    if (op.f_kind == PDD_F_RBF) {
        if (op.n_frbf <= 0 || op.n_frbf > 256 || !op.frbf_x || !op.frbf_y || !op.frbf_w || !(op.frbf_sigma > 0))
            fail(PDD_EINVAL, "f = RBF needs 1..256 Gaussians, centres, weights and sigma > 0");
        const int nq = op.n_frbf;
        frbf_x.alloc(nq);
        frbf_y.alloc(nq);
        frbf_w.alloc(nq);
        PDD_CUDA(cudaMemcpyAsync(frbf_x.p, op.frbf_x, nq * 8, cudaMemcpyHostToDevice, st));
        PDD_CUDA(cudaMemcpyAsync(frbf_y.p, op.frbf_y, nq * 8, cudaMemcpyHostToDevice, st));
        PDD_CUDA(cudaMemcpyAsync(frbf_w.p, op.frbf_w, nq * 8, cudaMemcpyHostToDevice, st));
        std::vector<float> f32(3 * (size_t)nq);
        for (int q = 0; q < nq; ++q) {
            f32[q] = (float)op.frbf_x[q];
            f32[nq + q] = (float)op.frbf_y[q];
            f32[2 * nq + q] = (float)op.frbf_w[q];
        }
        frbf32.alloc(f32.size());
        PDD_CUDA(cudaMemcpyAsync(frbf32.p, f32.data(), f32.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        PDD_CUDA(cudaStreamSynchronize(st));
        P.n_frbf = nq;
        P.frbf_x = frbf_x.p;
        P.frbf_y = frbf_y.p;
        P.frbf_w = frbf_w.p;
        P.frbf_sigma = op.frbf_sigma;
        P.frbf32 = frbf32.p;
        P.frbf_inv2s2 = (float)(1.0 / (2.0 * op.frbf_sigma * op.frbf_sigma));
    }
    if (op.g_kind == PDD_G_BOUNDARY_FOURIER) {
        if (op.n_gcoef <= 0 || !op.g_coef) fail(PDD_EINVAL, "g = boundary Fourier needs coefficients");
        g_coef.alloc(op.n_gcoef);
        PDD_CUDA(cudaMemcpyAsync(g_coef.p, op.g_coef, op.n_gcoef * 8, cudaMemcpyHostToDevice, st));
        P.n_gcoef = op.n_gcoef;
        P.g_coef = g_coef.p;
    }
    P.perimeter = (dom.kind == PDD_DOMAIN_SQUARE) ? 2.0 * ((dom.p[2] - dom.p[0]) + (dom.p[3] - dom.p[1]))
                                                  : 2.0 * PDD_PI * dom.p[2];
}

// the diagonal, C_ii = #Pi_i (1 for one subdomain, Eq. 29; Eq. 38 for averaged rows), and
// Dirichlet rows C_ii = 1, r_i = g(x_i); the diagonal sits after the stencils below i
__global__ void k_diag_dirichlet(Problem P, int N, const int *pi_ptr, const int *pi_sub, const int *knot_ptr,
                                 const int *rowptr, const double *kx, const double *ky, double *val, double *b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int e0 = pi_ptr[i], e1 = pi_ptr[i + 1];
    int pos = rowptr[i];
    for (int e = e0; e < e1; ++e) {
        const int m = pi_sub[e];
        if (knot_ptr[m] < i) pos += knot_ptr[m + 1] - knot_ptr[m];
    }
    val[pos] = e1 > e0 ? (double)(e1 - e0) : 1.0;
    if (e1 == e0) {
        const double x = kx[i], y = ky[i];
        double s = 0.0;
        if (P.g_kind == PDD_G_BOUNDARY_FOURIER) s = boundary_s(P, x, y, nearest_edge(P, x, y));
        b[i] = gdata(P, x, y, s);
    }
}

void assemble_dirichlet(const pdd_cover &cov, const Problem &P, pdd_system &sys, cudaStream_t st) {
    PDD_LAUNCH(k_diag_dirichlet, cdiv(cov.N, 256), 256, 0, st, P, cov.N, cov.pi_ptr.p, cov.pi_sub.p,
               cov.knot_ptr.p, cov.rowptr.p, cov.kx.p, cov.ky.p, sys.val.p, sys.b.p);
}

// r_i = the sum of its subdomains' r's in the order of Pi_i (Eq. 30; Eq. 39), and the root sum
// of squares of their standard errors (independent paths)
__global__ void k_gather_rows(int N, const int *pi_ptr, const int *pair_spos, const double *bs,
                              const double *se_bs, double *b, double *se_b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int e0 = pi_ptr[i], e1 = pi_ptr[i + 1];
    if (e1 == e0) return;                          // Dirichlet row
    double s = 0.0, v = 0.0;
    for (int e = e0; e < e1; ++e) {
        const int p = pair_spos[e];
        s += bs[p];
        v += se_bs[p] * se_bs[p];
    }
    b[i] = s;
    se_b[i] = sqrt(v);
}

static void check_domain(const pdd_domain *d) {
    if (!d) fail(PDD_EINVAL, "null domain");
    if (d->kind == PDD_DOMAIN_SQUARE) {
        if (!(d->p[2] > d->p[0]) || !(d->p[3] > d->p[1])) fail(PDD_EINVAL, "empty square domain");
    } else if (d->kind == PDD_DOMAIN_DISK) {
        if (!(d->p[2] > 0)) fail(PDD_EINVAL, "disk domain needs R > 0");
    } else {
        fail(PDD_EINVAL, "unknown domain kind");
    }
    for (int k = 0; k < 4; ++k)
        if (!std::isfinite(d->p[k])) fail(PDD_EINVAL, "non-finite domain parameter");
}

static void check_spec(const pdd_cover_spec *s) {
    if (!s) fail(PDD_EINVAL, "null cover spec");
    if (s->kind == PDD_COVER_SQUARE_LATTICE || s->kind == PDD_COVER_HEX_LATTICE) {
        if (s->nx <= 0 || s->ny <= 0 || (long)s->nx * s->ny > 50000000L) fail(PDD_EINVAL, "lattice size out of range");
        if (!(s->spacing > 0) || !(s->radius > 0)) fail(PDD_EINVAL, "lattice spacing and radius must be > 0");
        if (s->n_knots < 2 || s->n_knots > 248 || (s->n_knots & 1)) fail(PDD_EINVAL, "n_knots must be even in [2, 248]");
        if (s->n_theta < 2 || s->n_theta > 128 || (s->n_theta & 1)) fail(PDD_EINVAL, "n_theta must be even in [2, 128]");
        if (s->n_r < 1 || s->n_r > 64) fail(PDD_EINVAL, "n_r must be in [1, 64]");
    } else if (s->kind == PDD_COVER_EXPLICIT) {
        if (s->n_explicit <= 0 || !s->cx || !s->cy || !s->r || !s->n_knots_per || !s->n_r_per || !s->n_theta_per)
            fail(PDD_EINVAL, "explicit cover needs n_explicit > 0 and every per-circle array");
        for (int m = 0; m < s->n_explicit; ++m) {
            if (s->n_knots_per[m] < 2 || s->n_knots_per[m] > 248 || (s->n_knots_per[m] & 1) ||
                s->n_theta_per[m] < 2 || s->n_theta_per[m] > 128 || (s->n_theta_per[m] & 1) ||
                s->n_r_per[m] < 1 || s->n_r_per[m] > 64 || !(s->r[m] > 0))
                fail(PDD_EINVAL, "explicit circle " + std::to_string(m) + " has an invalid discretisation");
        }
    } else {
        fail(PDD_EINVAL, "unknown cover kind");
    }
    if (s->row_mode != PDD_ROWS_FARTHEST && s->row_mode != PDD_ROWS_AVERAGED) fail(PDD_EINVAL, "unknown row mode");
}

static void check_op(const pdd_operator *op) {
    if (!op) fail(PDD_EINVAL, "null operator");
    if (op->b_kind < 0 || op->b_kind > 1 || op->c_kind < 0 || op->c_kind > 2 || op->f_kind < 0 || op->f_kind > 4 ||
        op->g_kind < 0 || op->g_kind > 5)
        fail(PDD_EINVAL, "unknown coefficient family");
}

static void check_opts(const pdd_assembly_opts *o) {
    if (!o) fail(PDD_EINVAL, "null assembly options");
    if (o->precision != PDD_PREC_FP64 && o->precision != PDD_PREC_MIXED) fail(PDD_EINVAL, "unknown precision");
    if (o->floating_method != 0 && o->floating_method != 1) fail(PDD_EINVAL, "unknown floating method");
    if (o->factor != PDD_FACTOR_RECURSIVE_TC && o->factor != PDD_FACTOR_BLOCKED && o->factor != PDD_FACTOR_PIVOTED_TC)
        fail(PDD_EINVAL, "unknown factorisation");
    if (o->lu_leaf_width != 0 && o->lu_leaf_width != 8 && o->lu_leaf_width != 16 && o->lu_leaf_width != 32)
        fail(PDD_EINVAL, "lu_leaf_width must be 0, 8, 16 or 32");
    if (o->lu_tensor_min < 0) fail(PDD_EINVAL, "lu_tensor_min must be >= 0");
    if (o->paths_max > 0 && o->paths_max > (1 << 28)) fail(PDD_EINVAL, "paths_max too large");
    if (o->paths <= 1 || !(o->h > 0) || !(o->imq_c2 > 0)) fail(PDD_EINVAL, "paths > 1, h > 0 and c^2 > 0 required");
    if (o->max_steps < 0) fail(PDD_EINVAL, "max_steps must be >= 0 (0: 50 r^2/h)");
    if (o->disk_precision < PDD_STAGE_DEFAULT || o->disk_precision > PDD_STAGE_MIXED ||
        o->path_precision < PDD_STAGE_DEFAULT || o->path_precision > PDD_STAGE_MIXED)
        fail(PDD_EINVAL, "unknown stage precision");
    if (o->moment_sums < PDD_SUMS_AUTO || o->moment_sums > PDD_SUMS_FP64) fail(PDD_EINVAL, "unknown moment summation");
    if (o->cv_degree < 0 || o->cv_degree > 4) fail(PDD_EINVAL, "cv_degree must be in [0, 4]");
}

}  // namespace pdd

using namespace pdd;

#define API_BEGIN try {
#define API_END                                                        \
    }                                                                  \
    catch (const Fail &f) {                                            \
        return f.st;                                                   \
    }                                                                  \
    catch (const std::exception &e) {                                  \
        set_error(std::string("internal error: ") + e.what());         \
        return PDD_EINVAL;                                             \
    }                                                                  \
    return PDD_OK;

extern "C" {

const char *pdd_last_error(void) { return g_err.c_str(); }

int64_t pdd_launch_count(void) { return (int64_t)g_launches.load(); }

const char *pdd_version(void) { return "pdd-gb300 1.0 (sm_103a)"; }

pdd_status pdd_build_cover(const pdd_domain *domain, const pdd_cover_spec *spec, pdd_cover **out, void *stream) {
    API_BEGIN
    if (!out) fail(PDD_EINVAL, "null output handle");
    *out = nullptr;
    check_domain(domain);
    check_spec(spec);
    cudaStream_t st = (cudaStream_t)stream;
    pdd_cover *c = new pdd_cover();
    try {
        build_cover_impl(*domain, *spec, *c, st);
    } catch (...) {
        delete c;
        throw;
    }
    *out = c;
    API_END
}

pdd_status pdd_cover_info(const pdd_cover *cov, int *M, int *M_floating, int *N, int64_t *nnz) {
    API_BEGIN
    if (!cov) fail(PDD_EINVAL, "null cover");
    if (M) *M = cov->M;
    if (M_floating) *M_floating = cov->M_floating;
    if (N) *N = cov->N;
    if (nnz) *nnz = cov->nnz;
    API_END
}

pdd_status pdd_cover_arrays(const pdd_cover *cov, const double **cx, const double **cy, const double **r,
                            const uint8_t **floating, const int **knot_ptr, const double **kx, const double **ky,
                            const double **ku, const int **kowner, const uint8_t **kdir, const int **row_sub,
                            const int **rowptr, const int **col) {
    API_BEGIN
    if (!cov) fail(PDD_EINVAL, "null cover");
    if (cx) *cx = cov->cx.p;
    if (cy) *cy = cov->cy.p;
    if (r) *r = cov->r.p;
    if (floating) *floating = cov->floating.p;
    if (knot_ptr) *knot_ptr = cov->knot_ptr.p;
    if (kx) *kx = cov->kx.p;
    if (ky) *ky = cov->ky.p;
    if (ku) *ku = cov->ku.p;
    if (kowner) *kowner = cov->kowner.p;
    if (kdir) *kdir = cov->kdir.p;
    if (row_sub) *row_sub = cov->row_sub.p;
    if (rowptr) *rowptr = cov->rowptr.p;
    if (col) *col = cov->col.p;
    API_END
}

void pdd_destroy_cover(pdd_cover *cov) { delete cov; }

pdd_status pdd_assemble_G(const pdd_cover *cov, const pdd_operator *op, const pdd_assembly_opts *opts,
                          pdd_system **out, void *stream) {
    API_BEGIN
    if (!out) fail(PDD_EINVAL, "null output handle");
    *out = nullptr;
    if (!cov) fail(PDD_EINVAL, "null cover");
    check_op(op);
    check_opts(opts);
    cudaStream_t st = (cudaStream_t)stream;
    pdd_system *s = new pdd_system();
    try {
        s->N = cov->N;
        s->nnz = cov->nnz;
        s->cov = cov;
        s->precision = disk_mixed(*opts) || path_mixed(*opts) ? PDD_PREC_MIXED : PDD_PREC_FP64;
        s->val.alloc(cov->nnz);
        s->b.alloc(cov->N);
        const int nsub = std::max(cov->h_sub_ptr.empty() ? 0 : cov->h_sub_ptr.back(), 1);
        s->bs.alloc(nsub);
        s->se_bs.alloc(nsub);
        PDD_CUDA(cudaMemsetAsync(s->bs.p, 0, sizeof(double) * nsub, st));
        PDD_CUDA(cudaMemsetAsync(s->se_bs.p, 0, sizeof(double) * nsub, st));
        s->se.alloc(cov->nnz);
        s->se_b.alloc(cov->N);
        PDD_CUDA(cudaMemsetAsync(s->val.p, 0, sizeof(double) * cov->nnz, st));
        PDD_CUDA(cudaMemsetAsync(s->b.p, 0, sizeof(double) * cov->N, st));
        PDD_CUDA(cudaMemsetAsync(s->se.p, 0, sizeof(double) * cov->nnz, st));
        PDD_CUDA(cudaMemsetAsync(s->se_b.p, 0, sizeof(double) * cov->N, st));
        ProblemHolder ph;
        ph.set(cov->domain, *op, st);
        cudaEvent_t e0, e1, e2;
        PDD_CUDA(cudaEventCreate(&e0));
        PDD_CUDA(cudaEventCreate(&e1));
        PDD_CUDA(cudaEventCreate(&e2));
        PDD_CUDA(cudaEventRecord(e0, st));
        assemble_dirichlet(*cov, ph.P, *s, st);
        PDD_CUDA(cudaEventRecord(e1, st));
        DiskStats ds;
        if (opts->floating_method == PDD_FLOATING_PSEUDOSPECTRAL) ds = assemble_disks(*cov, ph.P, *opts, *s, st);
        PDD_CUDA(cudaEventRecord(e2, st));
        PDD_CUDA(cudaEventSynchronize(e2));
        float t01 = 0, t12 = 0;
        cudaEventElapsedTime(&t01, e0, e1);
        cudaEventElapsedTime(&t12, e1, e2);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaEventDestroy(e2);
        McStats ms = assemble_mc(*cov, ph.P, *opts, *s, st);
        PDD_LAUNCH(k_gather_rows, cdiv(cov->N, 256), 256, 0, st, cov->N, cov->pi_ptr.p, cov->pair_spos.p, s->bs.p,
                   s->se_bs.p, s->b.p, s->se_b.p);
        PDD_CUDA(cudaStreamSynchronize(st));
        pdd_assembly_stats &S = s->stats;
        S.floating_disks = ds.disks;
        S.floating_rows = ds.rows;
        S.mc_rows = ms.rows;
        S.path_steps = ms.steps;
        S.capped_paths = ms.capped;
        S.paths_total = ms.paths_total;
        S.extended_rows = ms.extended_rows;
        S.max_refine_sweeps = ds.max_sweeps;
        S.unconverged_disks = ds.unconverged;
        S.ms_cover_rows = t01;
        S.ms_disks = t12;
        S.ms_paths = ms.ms_paths;
        S.ms_finalize = ms.ms_finalize;
        S.ms_operator = ds.ms_operator;
        S.ms_factor = ds.ms_factor;
        S.ms_refine = ds.ms_refine;
        S.ms_eval = ds.ms_eval;
        S.lu_blocked = ds.lu_blocked;
        S.lu_leaf_width = ds.lu_leaf;
        S.lu_tensor_min = ds.lu_tmin;
        S.ms_trisolve = ds.ms_trisolve;
        S.ms_tc_gemm = ds.ms_tc_gemm;
        S.disk_solves = ds.disk_solves;
        S.tc_gemm_flop = ds.tc_gemm_flop;
        S.lu_pivoted_fallback = ds.lu_fallback;
        S.ms_gemm_fused = ds.ms_gemm_fused;
        S.gemm_fused_flop = ds.gemm_fused_flop;
        S.gemm_fused_bytes = ds.gemm_fused_bytes;
        S.gemm_pipe_launches = ds.gemm_pipe_launches;
        if (ms.capped) fail(PDD_EPATH_CAP, std::to_string(ms.capped) + " paths reached the step cap");
        if (ds.unconverged)
            fail(PDD_ENOCONV, std::to_string(ds.unconverged) + " disks missed the refinement tolerance");
    } catch (...) {
        delete s;
        throw;
    }
    *out = s;
    API_END
}

pdd_status pdd_system_csr(const pdd_system *sys, const double **val, const double **b, const double **se,
                          const double **se_b) {
    API_BEGIN
    if (!sys) fail(PDD_EINVAL, "null system");
    if (val) *val = sys->val.p;
    if (b) *b = sys->b.p;
    if (se) *se = sys->se.p;
    if (se_b) *se_b = sys->se_b.p;
    API_END
}

pdd_status pdd_system_mc(const pdd_system *sys, int *n_rows, const int **rows, const int **mom_ptr,
                         const double **moments, const double **bmean) {
    API_BEGIN
    if (!sys) fail(PDD_EINVAL, "null system");
    if (n_rows) *n_rows = sys->n_mc;
    if (rows) *rows = sys->mc_rows.p;
    if (mom_ptr) *mom_ptr = sys->mom_ptr.p;
    if (moments) *moments = sys->moments.p;
    if (bmean) *bmean = sys->bmean.p;
    API_END
}

pdd_status pdd_cover_rows(const pdd_cover *cov, int *n_pairs, const int **pi_ptr, const int **pi_sub) {
    API_BEGIN
    if (!cov) fail(PDD_EINVAL, "null cover");
    if (n_pairs) *n_pairs = cov->npairs;
    if (pi_ptr) *pi_ptr = cov->pi_ptr.p;
    if (pi_sub) *pi_sub = cov->pi_sub.p;
    API_END
}

pdd_status pdd_system_mc_subs(const pdd_system *sys, const int **subs) {
    API_BEGIN
    if (!sys) fail(PDD_EINVAL, "null system");
    if (subs) *subs = sys->mc_subs.p;
    API_END
}

pdd_status pdd_system_stats(const pdd_system *sys, pdd_assembly_stats *stats) {
    API_BEGIN
    if (!sys || !stats) fail(PDD_EINVAL, "null argument");
    *stats = sys->stats;
    API_END
}

void pdd_destroy_system(pdd_system *sys) { delete sys; }

static void check_solve_opts(const pdd_solve_opts *o) {
    if (!o) fail(PDD_EINVAL, "null solve options");
    if (o->restart < 1 || o->restart > 256 || o->max_iters < 1 || !(o->rtol > 0))
        fail(PDD_EINVAL, "restart in [1, 256], max_iters >= 1 and rtol > 0 required");
    if (o->precond != PDD_PRECOND_NONE && o->precond != PDD_PRECOND_RAS) fail(PDD_EINVAL, "unknown preconditioner");
}

pdd_status pdd_solve_csr(int n, const int *rowptr, const int *col, const double *val, const double *b, double *u,
                         const pdd_solve_opts *opts, pdd_solve_info *info, void *stream) {
    API_BEGIN
    check_solve_opts(opts);
    if (opts->precond != PDD_PRECOND_NONE) fail(PDD_EINVAL, "the RAS preconditioner needs the cover: use pdd_solve");
    if (n <= 0 || !rowptr || !col || !val || !b || !u) fail(PDD_EINVAL, "null array or n <= 0");
    cudaStream_t st = (cudaStream_t)stream;
    SolveResult r;
    if (opts->transpose) {
        int64_t nnz = 0;
        int hn = 0;
        PDD_CUDA(cudaMemcpyAsync(&hn, rowptr + n, sizeof(int), cudaMemcpyDeviceToHost, st));
        PDD_CUDA(cudaStreamSynchronize(st));
        nnz = hn;
        DevBuf<int> rt, ct;
        DevBuf<double> vt;
        csr_transpose(n, nnz, rowptr, col, val, rt, ct, vt, st);
        r = gmres_csr(n, rt.p, ct.p, vt.p, b, u, *opts, st);
    } else {
        r = gmres_csr(n, rowptr, col, val, b, u, *opts, st);
    }
    if (info) {
        info->iters = r.iters;
        info->rel_residual = r.rel;
        info->converged = r.converged;
    }
    if (!r.converged) fail(PDD_ENOCONV, "GMRES stopped at relative residual " + std::to_string(r.rel));
    API_END
}

pdd_status pdd_solve(const pdd_system *sys, const pdd_solve_opts *opts, double *u, pdd_solve_info *info,
                     void *stream) {
    if (!sys) {
        set_error("null system");
        return PDD_EINVAL;
    }
    if (!opts || opts->precond == PDD_PRECOND_NONE)
        return pdd_solve_csr(sys->N, sys->cov->rowptr.p, sys->cov->col.p, sys->val.p, sys->b.p, u, opts, info, stream);
    API_BEGIN
    check_solve_opts(opts);
    if (opts->transpose) fail(PDD_EINVAL, "the preconditioned solve takes C itself (transpose = 0)");
    if (!u) fail(PDD_EINVAL, "null u");
    if (sys->cov->averaged) fail(PDD_EINVAL, "the RAS subsets need one subdomain per row (a farthest-interface cover)");
    cudaStream_t st = (cudaStream_t)stream;
    RasPrecond M;
    M.build(*sys->cov, sys->cov->rowptr.p, sys->cov->col.p, sys->val.p, st);
    const SolveResult r = gmres_csr(sys->N, sys->cov->rowptr.p, sys->cov->col.p, sys->val.p, sys->b.p, u, *opts, st, &M);
    if (info) {
        info->iters = r.iters;
        info->rel_residual = r.rel;
        info->converged = r.converged;
    }
    if (!r.converged) fail(PDD_ENOCONV, "GMRES stopped at relative residual " + std::to_string(r.rel));
    API_END
}

pdd_status pdd_ras_apply(const pdd_system *sys, const double *v, double *y, void *stream) {
    API_BEGIN
    if (!sys || !v || !y) fail(PDD_EINVAL, "null argument");
    if (sys->cov->averaged) fail(PDD_EINVAL, "the RAS subsets need one subdomain per row (a farthest-interface cover)");
    cudaStream_t st = (cudaStream_t)stream;
    RasPrecond M;
    M.build(*sys->cov, sys->cov->rowptr.p, sys->cov->col.p, sys->val.p, st);
    M.apply(v, y, st);
    PDD_CUDA(cudaStreamSynchronize(st));
    API_END
}

pdd_status pdd_spmv_csr(int n, const int *rowptr, const int *col, const double *val, const double *x, double *y,
                        int transpose, void *stream) {
    API_BEGIN
    if (n <= 0 || !rowptr || !col || !val || !x || !y) fail(PDD_EINVAL, "null array or n <= 0");
    cudaStream_t st = (cudaStream_t)stream;
    if (transpose) {
        int hn = 0;
        PDD_CUDA(cudaMemcpyAsync(&hn, rowptr + n, sizeof(int), cudaMemcpyDeviceToHost, st));
        PDD_CUDA(cudaStreamSynchronize(st));
        DevBuf<int> rt, ct;
        DevBuf<double> vt;
        csr_transpose(n, hn, rowptr, col, val, rt, ct, vt, st);
        spmv_csr(n, rt.p, ct.p, vt.p, x, y, st);
        PDD_CUDA(cudaStreamSynchronize(st));
    } else {
        spmv_csr(n, rowptr, col, val, x, y, st);
    }
    API_END
}

pdd_status pdd_grad(const pdd_cover *cov, const pdd_operator *op, const pdd_assembly_opts *opts,
                    const pdd_system *sys, const double *u, const double *dJdu, double *grad, double *lambda,
                    void *stream) {
    API_BEGIN
    if (!cov || !sys || !u || !dJdu || !grad) fail(PDD_EINVAL, "null argument");
    if (sys->cov != cov) fail(PDD_EINVAL, "system was not assembled on this cover");
    if (cov->averaged) fail(PDD_EINVAL, "the adjoint gradient needs one subdomain per row (a farthest-interface cover)");
    check_op(op);
    check_opts(opts);
    if (opts->cv_degree) fail(PDD_EINVAL, "the adjoint gradient differentiates the plain estimator (cv_degree = 0)");
    cudaStream_t st = (cudaStream_t)stream;
    ProblemHolder ph;
    ph.set(cov->domain, *op, st);
    grad_impl(*cov, ph.P, *opts, *sys, u, dJdu, grad, lambda, st);
    PDD_CUDA(cudaStreamSynchronize(st));
    API_END
}

}  // extern "C"
