// a14: adjoint gradient of a misfit J(u) (not part of the paper).
//   dJ/dtheta = lambda^T (dr/dtheta - (dC/dtheta) u),   C^T lambda = dJ/du.
// lambda comes from GMRES on the explicit transpose of C; the Dirichlet
// rows, the floating disks (disk.cu: transposed disk solves) and the Monte
// Carlo rows (mc.cu: path replay under common random numbers) each give
// partial gradients that k_sum_partials adds in a fixed order.
#include <vector>

#include "handles.cuh"

namespace pdd {

// Dirichlet rows: r_i = g(x_i), so dJ/da_k += lambda_i psi^g_k(s(x_i)); one CTA per coefficient
__global__ void __launch_bounds__(256) k_grad_dirichlet(Problem P, int N, const int *row_sub, const double *kx,
                                                        const double *ky, const double *lambda, double *out) {
    __shared__ double red[8];
    const int kk = blockIdx.x, kc = (P.n_gcoef + 1) / 2;
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += 256) {
        if (row_sub[i] >= 0) continue;
        const double sv = boundary_s(P, kx[i], ky[i], nearest_edge(P, kx[i], ky[i]));
        const double w = PDD_TWO_PI * sv / P.perimeter;
        const double basis = (kk < kc) ? cos(kk * w) : sin((kk - kc + 1) * w);
        s += lambda[i] * basis;
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        out[kk] = t;
    }
}

// grad[q] = sum_d partial_disk[d][q] (q < nw + nf) + sum_s partial_mc[s][q] + dirichlet[q - nw - nf]
// (q >= nw + nf), in the layout [c weights][f weights][g coefficients], each sum in a fixed order
__global__ void k_sum_partials(int nw, int nf, int ng, const double *pd, int nd, const double *pm, int nm,
                               const double *pg, double *grad) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int np = nw + nf + ng;
    if (q >= np) return;
    double s = 0.0;
    if (q < nw + nf)
        for (int d = 0; d < nd; ++d) s += pd[(long)d * (nw + nf) + q];
    for (int r = 0; r < nm; ++r) s += pm[(long)r * np + q];
    if (q >= nw + nf && pg) s += pg[q - nw - nf];
    grad[q] = s;
}

void grad_impl(const pdd_cover &cov, const Problem &P, const pdd_assembly_opts &o, const pdd_system &sys,
               const double *u, const double *dJdu, double *grad, double *lambda_out, cudaStream_t st) {
    const int N = cov.N;
    const int nw = (P.c_kind == PDD_C_RBF) ? P.n_rbf : 0;
    const int nf = (P.f_kind == PDD_F_RBF) ? P.n_frbf : 0;
    const int ng = (P.g_kind == PDD_G_BOUNDARY_FOURIER) ? P.n_gcoef : 0;
    DevBuf<double> lam_own;
    double *lambda = lambda_out;
    if (!lambda) {
        lam_own.alloc(N);
        lambda = lam_own.p;
    }
    // C^T lambda = dJ/du
    {
        DevBuf<int> rt, ct;
        DevBuf<double> vt;
        csr_transpose(N, cov.nnz, cov.rowptr.p, cov.col.p, sys.val.p, rt, ct, vt, st);
        pdd_solve_opts so{64, 20000, 1e-14, 0};
        SolveResult r = gmres_csr(N, rt.p, ct.p, vt.p, dJdu, lambda, so, st);
        if (!r.converged) fail(PDD_ENOCONV, "adjoint GMRES did not converge");
    }
    const int n_all = nw + nf + ng;
    if (n_all == 0) return;
    PDD_CUDA(cudaMemsetAsync(grad, 0, sizeof(double) * n_all, st));
    DevBuf<double> pg;
    if (ng) {
        pg.alloc(ng);
        PDD_LAUNCH(k_grad_dirichlet, ng, 256, 0, st, P, N, cov.row_sub.p, cov.kx.p, cov.ky.p, lambda, pg.p);
    }
    DevBuf<double> pd, pm;
    int nd = 0, nm = 0;
    if ((nw || nf) && o.floating_method == PDD_FLOATING_PSEUDOSPECTRAL) grad_disks(cov, P, u, lambda, pd, nd, st);
    grad_mc(cov, P, o, sys, u, lambda, pm, nm, st);
    // layout of grad: [c weights][f weights][g coefficients] (families the operator does not use
    // have no entries)
    PDD_LAUNCH(k_sum_partials, cdiv(n_all, 128), 128, 0, st, nw, nf, ng, pd.p, nd, pm.p, nm, ng ? pg.p : nullptr,
               grad);
    PDD_CUDA(cudaStreamSynchronize(st));
}

}  // namespace pdd
