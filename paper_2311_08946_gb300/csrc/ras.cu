// a13 (right preconditioner): the one-level restricted additive Schwarz
// operator of Sec. 4, Eq. 42-44,
//     M^-1 = sum_p R_p^T D_p C_p^-1 R_p,   C_p = R_p C R_p^T,
//     (D_p)_ii = 1 / #{q : x_i in w_q}.
// Subsets: the nonoverlapping part of w_p is the set of rows the row
// assignment (Sec. 3.2) gives to subdomain p, and its neighbours in the graph
// of C are the columns of those rows: the knots of circle p (Eq. 29).  So w_p
// lists p's owned rows, then p's knots, and every row lies in at most two
// subsets (its own circle's, and its owner's unless it is a Dirichlet row):
// the sum over subsets becomes a two-term gather in a fixed order.
//
// The C_p (at most 128 x 128, padded with the identity) are assembled from the
// CSR system and inverted once per solve by Gauss-Jordan elimination with
// partial pivoting in shared memory, one CTA per subset, in FP32: the
// preconditioner only has to be close to C^-1; GMRES keeps the FP64 true
// residual, so the solution does not depend on its precision.  Applying M^-1
// is one small dense product per subset (k_ras_local) and the gather
// (k_ras_gather); the fused Arnoldi kernel runs the same two steps inline.
#include <algorithm>
#include <vector>

#include "handles.cuh"

namespace pdd {

static constexpr int kRasThreads = 128;

// w_p: p's owned rows, then p's knots
__global__ void k_ras_index(int P, const int *sub_ptr, const int *sub_rows, const int *knot_ptr, const int *wptr,
                            int *widx) {
    const int p = blockIdx.x;
    if (p >= P) return;
    const int a0 = sub_ptr[p], na = sub_ptr[p + 1] - a0;
    const int k0 = knot_ptr[p], nk = knot_ptr[p + 1] - k0;
    int *w = widx + wptr[p];
    for (int e = threadIdx.x; e < na + nk; e += blockDim.x) w[e] = e < na ? sub_rows[a0 + e] : k0 + (e - na);
}

// where row i sits: (p1, l1) in its own circle's subset, (p2, l2) in its owner's (p2 = -1 for a
// Dirichlet row)
__global__ void k_ras_locate_knots(int N, const int *kowner, const int *sub_ptr, const int *knot_ptr,
                                   const int *row_sub, int *p1, int *l1, int *p2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int p = kowner[i];
    p1[i] = p;
    l1[i] = (sub_ptr[p + 1] - sub_ptr[p]) + (i - knot_ptr[p]);
    p2[i] = row_sub[i];
}

__global__ void k_ras_locate_rows(int nrows, const int *sub_rows, const int *sub_ptr, const int *row_sub, int *l2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nrows) return;
    const int i = sub_rows[e];
    l2[i] = e - sub_ptr[row_sub[i]];
}

// C_p from the CSR system, inverted by Gauss-Jordan with partial pivoting; cinvT[p][b][a] =
// (C_p^-1)[a][b] (column-major, so that the apply reads consecutive addresses across outputs)
__global__ void __launch_bounds__(kRasThreads) k_ras_invert(int P, int NP, const int *wptr, const int *widx,
                                                            const int *rowptr, const int *col, const double *val,
                                                            const int *kowner, const int *row_sub, const int *l1,
                                                            const int *l2, float *cinvT, int *singular) {
    extern __shared__ float gj[];                   // NP x (2 NP + 1): [C_p | I]
    __shared__ float fcol[128];
    __shared__ int piv_s;
    const int p = blockIdx.x, tid = threadIdx.x, LD = 2 * NP + 1;
    const int base = wptr[p], np = wptr[p + 1] - base;
    for (int e = tid; e < NP * LD; e += kRasThreads) {
        const int a = e / LD, c = e - a * LD;
        gj[e] = (c == NP + a || (a >= np && c == a)) ? 1.f : 0.f;
    }
    __syncthreads();
    for (int a = tid; a < np; a += kRasThreads) {
        const int i = widx[base + a];
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const int j = col[k];
            int bcol = -1;
            if (kowner[j] == p) bcol = l1[j];
            else if (row_sub[j] == p) bcol = l2[j];
            if (bcol >= 0) gj[a * LD + bcol] = (float)val[k];
        }
    }
    __syncthreads();
    for (int k = 0; k < NP; ++k) {
        if (tid < 32) {                             // pivot: largest |C[r][k]|, r >= k, lowest r on ties
            float best = -1.f;
            int bi = k;
            for (int r = k + tid; r < NP; r += 32) {
                const float v = fabsf(gj[r * LD + k]);
                if (v > best) {
                    best = v;
                    bi = r;
                }
            }
            for (int o = 16; o; o >>= 1) {
                const float ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) {
                    best = ov;
                    bi = oi;
                }
            }
            if (tid == 0) piv_s = bi;
        }
        __syncthreads();
        const int pr = piv_s;
        if (pr != k)
            for (int c = tid; c < 2 * NP; c += kRasThreads) {
                const float t = gj[k * LD + c];
                gj[k * LD + c] = gj[pr * LD + c];
                gj[pr * LD + c] = t;
            }
        __syncthreads();
        const float d = gj[k * LD + k];
        if (d == 0.f) {
            if (tid == 0) atomicAdd(singular, 1);
            return;                                  // the whole block leaves: d is the same for all
        }
        const float inv = 1.f / d;
        for (int c = tid; c < 2 * NP; c += kRasThreads) gj[k * LD + c] *= inv;
        for (int r = tid; r < NP; r += kRasThreads) fcol[r] = gj[r * LD + k];
        __syncthreads();
        for (int e = tid; e < NP * 2 * NP; e += kRasThreads) {
            const int r = e / (2 * NP), c = e - r * 2 * NP;
            if (r != k) gj[r * LD + c] -= fcol[r] * gj[k * LD + c];
        }
        __syncthreads();
    }
    float *out = cinvT + (long)p * NP * NP;
    for (int e = tid; e < NP * NP; e += kRasThreads) {
        const int b = e / NP, a = e - b * NP;       // out[b][a] = inv[a][b]
        out[e] = gj[a * LD + NP + b];
    }
}

// z_p = C_p^-1 (R_p v), one CTA per subset
__global__ void __launch_bounds__(kRasThreads) k_ras_local(int P, int NP, const int *wptr, const int *widx,
                                                           const float *cinvT, const double *v, float *z) {
    __shared__ float vs[128];
    const int p = blockIdx.x, tid = threadIdx.x;
    const int base = wptr[p], np = wptr[p + 1] - base;
    for (int b = tid; b < NP; b += kRasThreads) vs[b] = b < np ? (float)v[widx[base + b]] : 0.f;
    __syncthreads();
    const float *ci = cinvT + (long)p * NP * NP;
    for (int a = tid; a < NP; a += kRasThreads) {
        float s = 0.f;
        for (int b = 0; b < np; ++b) s = fmaf(ci[(long)b * NP + a], vs[b], s);
        z[(long)p * NP + a] = s;
    }
}

// y_i = sum over the (one or two) subsets holding i of D_ii (z_p)_i
__global__ void k_ras_gather(int N, int NP, const int *p1, const int *l1, const int *p2, const int *l2,
                             const float *z, double *y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int q = p2[i];
    const double a = (double)z[(long)p1[i] * NP + l1[i]];
    y[i] = q >= 0 ? 0.5 * (a + (double)z[(long)q * NP + l2[i]]) : a;
}

void RasPrecond::build(const pdd_cover &cov, const int *rowptr, const int *col, const double *val,
                       cudaStream_t st) {
    P = cov.M;
    N = cov.N;
    std::vector<int> wp(P + 1, 0);
    int mx = 0;
    for (int p = 0; p < P; ++p) {
        const int n_p = (cov.h_sub_ptr[p + 1] - cov.h_sub_ptr[p]) + (cov.h_knot_ptr[p + 1] - cov.h_knot_ptr[p]);
        wp[p + 1] = wp[p] + n_p;
        mx = std::max(mx, n_p);
    }
    NP = std::max(4, (mx + 3) / 4 * 4);
    if (NP > 128) fail(PDD_EINVAL, "RAS subsets larger than 128 knots");
    wptr.alloc(P + 1);
    widx.alloc(std::max(1, wp[P]));
    p1.alloc(N);
    l1.alloc(N);
    p2.alloc(N);
    l2.alloc(N);
    cinvT.alloc((size_t)P * NP * NP);
    z.alloc((size_t)P * NP);
    DevBuf<int> sing;
    sing.alloc(1);
    PDD_CUDA(cudaMemsetAsync(sing.p, 0, sizeof(int), st));
    PDD_CUDA(cudaMemcpyAsync(wptr.p, wp.data(), (P + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    PDD_LAUNCH(k_ras_index, P, 128, 0, st, P, cov.sub_ptr.p, cov.sub_rows.p, cov.knot_ptr.p, wptr.p, widx.p);
    PDD_LAUNCH(k_ras_locate_knots, cdiv(N, 256), 256, 0, st, N, cov.kowner.p, cov.sub_ptr.p, cov.knot_ptr.p,
               cov.row_sub.p, p1.p, l1.p, p2.p);
    const int nrows = cov.h_sub_ptr[P];
    if (nrows > 0)
        PDD_LAUNCH(k_ras_locate_rows, cdiv(nrows, 256), 256, 0, st, nrows, cov.sub_rows.p, cov.sub_ptr.p,
                   cov.row_sub.p, l2.p);
    const size_t sm = (size_t)NP * (2 * NP + 1) * sizeof(float);
    PDD_CUDA(cudaFuncSetAttribute(k_ras_invert, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    PDD_LAUNCH(k_ras_invert, P, kRasThreads, sm, st, P, NP, wptr.p, widx.p, rowptr, col, val, cov.kowner.p,
               cov.row_sub.p, l1.p, l2.p, cinvT.p, sing.p);
    int hs = 0;
    PDD_CUDA(cudaMemcpyAsync(&hs, sing.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    PDD_CUDA(cudaStreamSynchronize(st));
    if (hs) fail(PDD_ENOCONV, "a RAS subset matrix C_p is singular");
}

void RasPrecond::apply(const double *v, double *y, cudaStream_t st) const {
    PDD_LAUNCH(k_ras_local, P, kRasThreads, 0, st, P, NP, wptr.p, widx.p, cinvT.p, v, z.p);
    PDD_LAUNCH(k_ras_gather, cdiv(N, 256), 256, 0, st, N, NP, p1.p, l1.p, p2.p, l2.p, z.p, y);
}

}  // namespace pdd
