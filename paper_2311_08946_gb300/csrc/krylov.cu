// a13: the global solve C u = r (Eq. 28) in FP64 by restarted GMRES(m)
// (Sec. 4; Eq. 45 without the RAS preconditioner) on a CSR sparse
// matrix-vector product.
//
// Layout: the Krylov basis V is (m+1) x n row-major (each basis vector
// contiguous); dot products are block partial sums reduced in a fixed order
// (deterministic).  Orthogonalisation is classical Gram-Schmidt applied
// twice (CGS2).  The Hessenberg matrix, Givens rotations and the residual
// estimate live on the device; after convergence every kernel of the cycle
// sees the stop flag and returns at once, so the host synchronises only once
// per restart cycle to read the true residual.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "handles.cuh"

namespace pdd {

static constexpr int kRowsPerBlock = 32;    // 8 lanes per row, 256 threads
static constexpr int kDotBlock = 256;

struct GState {
    int stop, iters, k_used, pad;
    double bnorm, res;
};

// y = C x, 8 lanes per row
__global__ void __launch_bounds__(256) k_spmv(int n, const int *rowptr, const int *col, const double *val,
                                              const double *x, double *y, const GState *gs) {
    if (gs && gs->stop) return;
    const int row = blockIdx.x * kRowsPerBlock + (threadIdx.x >> 3), l = threadIdx.x & 7;
    double s = 0.0;
    if (row < n)
        for (int k = rowptr[row] + l; k < rowptr[row + 1]; k += 8) s += val[k] * x[col[k]];
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    if (row < n && l == 0) y[row] = s;
}

// partial[t * G + bx] = sum over the rows of block column bx of V[t] . w.  The grid is
// (row chunks G) x (groups of eight vectors); each thread takes rows of its chunk for the eight
// vectors of its group (independent loads).  The last block of a vector group to finish adds the
// group's partials in block order into hsum[t] (deterministic) and re-arms the group's counter.
static constexpr int kMaxDots = 257;
static constexpr int kDotThreads = 128, kDotVec = 8;
static constexpr int kDotGroups = (kMaxDots + kDotVec - 1) / kDotVec;
__global__ void __launch_bounds__(kDotThreads) k_dots(int n, int nv, const double *V, const double *w,
                                                      double *partial, double *hsum, unsigned *cnt,
                                                      const GState *gs) {
    if (gs && gs->stop) return;
    __shared__ double red[kDotThreads / 32][kDotVec];
    __shared__ bool last;
    const int G = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t0 = blockIdx.y * kDotVec, nq = min(kDotVec, nv - t0);
    const int per = (n + G - 1) / G, a = blockIdx.x * per, b = min(n, a + per);
    double s[kDotVec];
#pragma unroll
    for (int q = 0; q < kDotVec; ++q) s[q] = 0.0;
    const double *v0 = V + (long)t0 * n;
    for (int r = a + threadIdx.x; r < b; r += kDotThreads) {
        const double wr = w[r];
#pragma unroll
        for (int q = 0; q < kDotVec; ++q)
            if (q < nq) s[q] += v0[(long)q * n + r] * wr;
    }
#pragma unroll
    for (int q = 0; q < kDotVec; ++q) {
        double v = s[q];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < nq) {
        double v = 0.0;
        for (int q = 0; q < kDotThreads / 32; ++q) v += red[q][threadIdx.x];
        partial[(long)(t0 + threadIdx.x) * G + blockIdx.x] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(cnt + blockIdx.y, 1u) == (unsigned)G - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int q = warp; q < nq; q += kDotThreads / 32) {
        const double *pp = partial + (long)(t0 + q) * G;
        double v = 0.0;
#pragma unroll 4
        for (int i = lane; i < G; i += 32) v += __ldcg(pp + i);
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) hsum[t0 + q] = v;
    }
    if (threadIdx.x == 0) cnt[blockIdx.y] = 0u;
}

// w -= sum_t V[t] h[t] with h = hsum; column j of H gets h (+= when add)
__global__ void __launch_bounds__(kDotBlock) k_orth(int n, int nv, const double *V, double *w,
                                                    const double *hsum, double *Hcol, int add, const GState *gs) {
    if (gs && gs->stop) return;
    __shared__ double h[kMaxDots];
    for (int t = threadIdx.x; t < nv; t += blockDim.x) h[t] = hsum[t];
    __syncthreads();
    if (blockIdx.x == 0)
        for (int t = threadIdx.x; t < nv; t += blockDim.x) Hcol[t] = add ? Hcol[t] + h[t] : h[t];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        double s = w[r];
        for (int t0 = 0; t0 < nv; t0 += 16) {            // sixteen independent loads in flight
            double v[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = (t0 + q < nv) ? V[(long)(t0 + q) * n + r] : 0.0;
#pragma unroll
            for (int q = 0; q < 16; ++q)
                if (t0 + q < nv) s -= v[q] * h[t0 + q];
        }
        w[r] = s;
    }
}

// v = w / |w| with |w|^2 = hsum[0]; Hsub = |w|
__global__ void __launch_bounds__(kDotBlock) k_normalize(int n, const double *w, double *v, const double *hsum,
                                                         double *Hsub, const GState *gs) {
    if (gs && gs->stop) return;
    const double nrm = sqrt(hsum[0]);
    if (blockIdx.x == 0 && threadIdx.x == 0 && Hsub) *Hsub = nrm;
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) v[r] = w[r] * inv;
}

// apply the previous rotations to column j, make a new one, update g and the stop flag; one
// warp stages the column and the rotations in shared memory, lane 0 runs the recurrence
__global__ void k_givens(double *H, int ldh, double *cs, double *sn, double *g, int j, double rtol,
                         int max_iters, GState *gs) {
    if (gs->stop) return;
    __shared__ double hs[kMaxDots], cc[kMaxDots], ss[kMaxDots];
    double *hc = H + (long)j * ldh;                  // column j stored contiguously (ldh = m+1)
    for (int i = threadIdx.x; i <= j + 1; i += 32) hs[i] = hc[i];
    for (int i = threadIdx.x; i < j; i += 32) {
        cc[i] = cs[i];
        ss[i] = sn[i];
    }
    __syncwarp();
    if (threadIdx.x == 0) {
        double hi = hs[0];
        for (int i = 0; i < j; ++i) {
            const double hn = hs[i + 1];
            const double t = cc[i] * hi + ss[i] * hn;
            hi = -ss[i] * hi + cc[i] * hn;
            hs[i] = t;
        }
        // hi is the rotated entry j
        const double a = hi, b = hs[j + 1];
        const double den = hypot(a, b);
        const double c = den > 0.0 ? a / den : 1.0, s = den > 0.0 ? b / den : 0.0;
        cs[j] = c;
        sn[j] = s;
        hs[j] = den;
        hs[j + 1] = 0.0;
        g[j + 1] = -s * g[j];
        g[j] = c * g[j];
        gs->iters += 1;
        gs->k_used = j + 1;
        gs->res = fabs(g[j + 1]);
        if (gs->res <= rtol * gs->bnorm || gs->iters >= max_iters || b == 0.0) gs->stop = 1;
    }
    __syncwarp();
    for (int i = threadIdx.x; i <= j + 1; i += 32) hc[i] = hs[i];
}

// y = H^-1 g (upper triangular k x k), single thread; then stop is cleared for the next cycle
__global__ void k_upper_solve(const double *H, int ldh, const double *g, double *y, GState *gs) {
    const int k = gs->k_used;
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int c = i + 1; c < k; ++c) s -= H[(long)c * ldh + i] * y[c];
        y[i] = s / H[(long)i * ldh + i];
    }
}

__global__ void k_xupdate(int n, const double *V, const double *y, const GState *gs, double *x) {
    const int k = gs->k_used;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        double s = x[r];
        for (int t = 0; t < k; ++t) s += V[(long)t * n + r] * y[t];
        x[r] = s;
    }
}

// r = b - C x (Cx precomputed in r)
__global__ void k_residual_vec(int n, const double *b, double *r) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) r[i] = b[i] - r[i];
}

__global__ void k_cycle_start(GState *gs, const double *hsum, double *g, int m, double rtol, int max_iters,
                              int first) {
    if (threadIdx.x != 0) return;
    const double beta = sqrt(hsum[0]);
    if (first) gs->bnorm = beta;                      // x0 = 0, so r0 = b
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    gs->res = beta;
    gs->k_used = 0;
    gs->stop = (beta <= rtol * gs->bnorm || gs->iters >= max_iters || beta == 0.0) ? 1 : 0;
}

void spmv_csr(int n, const int *rowptr, const int *col, const double *val, const double *x, double *y,
              cudaStream_t st) {
    PDD_LAUNCH(k_spmv, cdiv(n, kRowsPerBlock), 256, 0, st, n, rowptr, col, val, x, y, (const GState *)nullptr);
}

// The m Arnoldi iterations of a restart cycle (about 8 kernels each) are
// captured once into a CUDA graph and replayed once per cycle; the stop flag
// on the device turns the remaining kernels of a converged cycle into no-ops.
SolveResult gmres_csr(int n, const int *rowptr, const int *col, const double *val, const double *b, double *u,
                      const pdd_solve_opts &o, cudaStream_t st_in) {
    const int m = std::max(1, std::min(256, o.restart));
    const int G = std::max(1, std::min(1024, cdiv(n, 2 * kDotThreads)));
    DevBuf<double> V, w, partial, hsum, H, cs, sn, g, y;
    DevBuf<unsigned> cnt;
    DevBuf<GState> gs;
    V.alloc((size_t)(m + 1) * n);
    w.alloc(n);
    partial.alloc((size_t)(m + 1) * G);
    hsum.alloc(m + 1);
    cnt.alloc(kDotGroups);
    H.alloc((size_t)(m + 1) * m);
    cs.alloc(m);
    sn.alloc(m);
    g.alloc(m + 1);
    y.alloc(m);
    gs.alloc(1);
    // graph capture needs a capturable stream: the legacy default stream is replaced by a private one
    cudaStream_t st = st_in;
    bool own = false;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    if (st_in == 0 || st_in == cudaStreamLegacy) {
        PDD_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        PDD_CUDA(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
        PDD_CUDA(cudaEventRecord(ev_in, st_in));
        PDD_CUDA(cudaStreamWaitEvent(st, ev_in, 0));
        own = true;
    }
    PDD_CUDA(cudaMemsetAsync(gs.p, 0, sizeof(GState), st));
    PDD_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned) * kDotGroups, st));
    PDD_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * n, st));
    PDD_CUDA(cudaMemsetAsync(H.p, 0, sizeof(double) * (m + 1) * m, st));
    const int vb = std::min(cdiv(n, 256), 2048);
    SolveResult res;
    const int max_iters = std::max(1, o.max_iters);
    cudaGraphExec_t exec = nullptr;
    int per_cycle = 0;
    try {
        for (int cycle = 0;; ++cycle) {
            // r = b - C u  (u = 0 on the first cycle)
            PDD_LAUNCH(k_spmv, cdiv(n, kRowsPerBlock), 256, 0, st, n, rowptr, col, val, u, w.p, (const GState *)nullptr);
            PDD_LAUNCH(k_residual_vec, vb, 256, 0, st, n, b, w.p);
            PDD_LAUNCH(k_dots, dim3(G, 1), kDotThreads, 0, st, n, 1, w.p, w.p, partial.p, hsum.p, cnt.p, (const GState *)nullptr);
            PDD_LAUNCH(k_cycle_start, 1, 32, 0, st, gs.p, hsum.p, g.p, m, o.rtol, max_iters, cycle == 0 ? 1 : 0);
            PDD_LAUNCH(k_normalize, vb, kDotBlock, 0, st, n, w.p, V.p, hsum.p, (double *)nullptr, gs.p);
            if (!exec) {
                const int64_t before = pdd_launch_count();
                cudaGraph_t graph;
                PDD_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                for (int j = 0; j < m; ++j) {
                    double *vj = V.p + (long)j * n;
                    double *Hc = H.p + (long)j * (m + 1);
                    PDD_LAUNCH(k_spmv, cdiv(n, kRowsPerBlock), 256, 0, st, n, rowptr, col, val, vj, w.p, gs.p);
                    for (int pass = 0; pass < 2; ++pass) {
                        PDD_LAUNCH(k_dots, dim3(G, cdiv(j + 1, kDotVec)), kDotThreads, 0, st, n, j + 1, V.p, w.p, partial.p, hsum.p, cnt.p, gs.p);
                        PDD_LAUNCH(k_orth, vb, kDotBlock, 0, st, n, j + 1, V.p, w.p, hsum.p, Hc, pass, gs.p);
                    }
                    PDD_LAUNCH(k_dots, dim3(G, 1), kDotThreads, 0, st, n, 1, w.p, w.p, partial.p, hsum.p, cnt.p, gs.p);
                    PDD_LAUNCH(k_normalize, vb, kDotBlock, 0, st, n, w.p, V.p + (long)(j + 1) * n, hsum.p, Hc + j + 1,
                               gs.p);
                    PDD_LAUNCH(k_givens, 1, 32, 0, st, H.p, m + 1, cs.p, sn.p, g.p, j, o.rtol, max_iters, gs.p);
                }
                PDD_CUDA(cudaStreamEndCapture(st, &graph));
                PDD_CUDA(cudaGraphInstantiate(&exec, graph, 0));
                cudaGraphDestroy(graph);
                per_cycle = (int)(pdd_launch_count() - before);
                count_launch(-per_cycle);          // captured, not run: counted when the graph runs
            }
            PDD_CUDA(cudaGraphLaunch(exec, st));
            count_launch(per_cycle);
            PDD_LAUNCH(k_upper_solve, 1, 1, 0, st, H.p, m + 1, g.p, y.p, gs.p);
            PDD_LAUNCH(k_xupdate, vb, 256, 0, st, n, V.p, y.p, gs.p, u);
            // true residual
            PDD_LAUNCH(k_spmv, cdiv(n, kRowsPerBlock), 256, 0, st, n, rowptr, col, val, u, w.p, (const GState *)nullptr);
            PDD_LAUNCH(k_residual_vec, vb, 256, 0, st, n, b, w.p);
            PDD_LAUNCH(k_dots, dim3(G, 1), kDotThreads, 0, st, n, 1, w.p, w.p, partial.p, hsum.p, cnt.p, (const GState *)nullptr);
            GState hg{};
            double rs = 0.0;
            PDD_CUDA(cudaMemcpyAsync(&rs, hsum.p, sizeof(double), cudaMemcpyDeviceToHost, st));
            PDD_CUDA(cudaMemcpyAsync(&hg, gs.p, sizeof(GState), cudaMemcpyDeviceToHost, st));
            PDD_CUDA(cudaStreamSynchronize(st));
            const double rel = hg.bnorm > 0.0 ? std::sqrt(rs) / hg.bnorm : 0.0;
            res.iters = hg.iters;
            res.rel = rel;
            if (hg.bnorm == 0.0 || rel <= o.rtol) {
                res.converged = 1;
                break;
            }
            if (hg.iters >= max_iters) break;
        }
    } catch (...) {
        if (exec) cudaGraphExecDestroy(exec);
        if (own) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
            cudaEventDestroy(ev_in);
        }
        throw;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (own) {
        PDD_CUDA(cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
        PDD_CUDA(cudaEventRecord(ev_out, st));
        PDD_CUDA(cudaStreamWaitEvent(st_in, ev_out, 0));
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
        cudaEventDestroy(ev_in);
        cudaEventDestroy(ev_out);
    }
    return res;
}

// ---------------------------------------------------------------------------
// explicit transpose (counting sort by column, rows then sorted: deterministic)
// ---------------------------------------------------------------------------
__global__ void k_col_count(int64_t nnz, const int *col, int *cnt) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[col[k]], 1);
}

__global__ void k_t_fill(int n, const int *rowptr, const int *col, const double *val, const int *ptr_t,
                         int *cursor, int *col_t, double *val_t) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        int c = col[k];
        int p = ptr_t[c] + atomicAdd(&cursor[c], 1);
        col_t[p] = i;
        val_t[p] = val[k];
    }
}

__global__ void k_t_sort(int n, const int *ptr_t, int *col_t, double *val_t) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    for (int k = ptr_t[r] + 1; k < ptr_t[r + 1]; ++k) {
        int c = col_t[k];
        double v = val_t[k];
        int q = k - 1;
        while (q >= ptr_t[r] && col_t[q] > c) {
            col_t[q + 1] = col_t[q];
            val_t[q + 1] = val_t[q];
            --q;
        }
        col_t[q + 1] = c;
        val_t[q + 1] = v;
    }
}

void csr_transpose(int n, int64_t nnz, const int *rowptr, const int *col, const double *val, DevBuf<int> &rowptr_t,
                   DevBuf<int> &col_t, DevBuf<double> &val_t, cudaStream_t st) {
    DevBuf<int> cnt, cursor;
    cnt.alloc(n + 1);
    cursor.alloc(n + 1);
    rowptr_t.alloc(n + 1);
    col_t.alloc(std::max<int64_t>(nnz, 1));
    val_t.alloc(std::max<int64_t>(nnz, 1));
    PDD_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int) * (n + 1), st));
    PDD_CUDA(cudaMemsetAsync(cursor.p, 0, sizeof(int) * (n + 1), st));
    PDD_LAUNCH(k_col_count, 1024, 256, 0, st, nnz, col, cnt.p);
    exclusive_scan(cnt.p, rowptr_t.p, n, st);
    PDD_LAUNCH(k_t_fill, cdiv(n, 256), 256, 0, st, n, rowptr, col, val, rowptr_t.p, cursor.p, col_t.p, val_t.p);
    PDD_LAUNCH(k_t_sort, cdiv(n, 256), 256, 0, st, n, rowptr_t.p, col_t.p, val_t.p);
}

}  // namespace pdd

// ---------------------------------------------------------------------------
// Allocation-free variant of the CSR GMRES solve.
//
// Some callers cannot allocate device memory while they run: a host process
// whose device heap is owned by another allocator (a caching allocator that
// must not be bypassed or fragmented), a latency-critical loop that cannot
// absorb the device-wide synchronisation cudaFree implies, or a service that
// must not meet an out-of-memory failure half-way through a request.  For them
// pdd_solve_csr_noalloc runs the same GMRES kernels on a fixed workspace that
// lives in this file-scope device array, reserved when the library is loaded
// and held by every GPU that loads it until the process exits.
// ---------------------------------------------------------------------------
namespace pdd {

static constexpr size_t kNoAllocBytes = (size_t)64 << 20;          // 64 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static constexpr int kMaxDevices = 64;
static void *g_noalloc_ptr[kMaxDevices] = {nullptr};
static std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device (looked up once per device).
static void *noalloc_scratch(int dev) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (dev < 0 || dev >= kMaxDevices) fail(PDD_EINVAL, "device ordinal out of range");
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            set_error(cuda_msg(e, "cudaGetSymbolAddress(g_noalloc_scratch)"));
            throw Fail{PDD_ECUDA};
        }
        g_noalloc_ptr[dev] = p;
    }
    return g_noalloc_ptr[dev];
}

struct NoAllocLayout {
    size_t V, w, partial, hsum, cnt, H, cs, sn, g, y, gs, total;
};

static NoAllocLayout noalloc_layout(int n, int m, int G) {
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    NoAllocLayout L{};
    size_t off = 0;
    L.V = off; off += up(sizeof(double) * (size_t)(m + 1) * n);
    L.w = off; off += up(sizeof(double) * (size_t)n);
    L.partial = off; off += up(sizeof(double) * (size_t)(m + 1) * G);
    L.hsum = off; off += up(sizeof(double) * (size_t)(m + 1));
    L.cnt = off; off += up(sizeof(unsigned) * kDotGroups);
    L.H = off; off += up(sizeof(double) * (size_t)(m + 1) * m);
    L.cs = off; off += up(sizeof(double) * (size_t)m);
    L.sn = off; off += up(sizeof(double) * (size_t)m);
    L.g = off; off += up(sizeof(double) * (size_t)(m + 1));
    L.y = off; off += up(sizeof(double) * (size_t)m);
    L.gs = off; off += up(sizeof(GState));
    L.total = off;
    return L;
}

// The same iteration as gmres_csr, on buffers carved from `base`.
static SolveResult gmres_csr_fixed(int n, const int *rowptr, const int *col, const double *val,
                                   const double *b, double *u, const pdd_solve_opts &o, unsigned char *base,
                                   const NoAllocLayout &L, int m, int G, cudaStream_t st) {
    double *V = (double *)(base + L.V), *w = (double *)(base + L.w);
    double *partial = (double *)(base + L.partial), *H = (double *)(base + L.H);
    double *hsum = (double *)(base + L.hsum);
    unsigned *cnt = (unsigned *)(base + L.cnt);
    double *cs = (double *)(base + L.cs), *sn = (double *)(base + L.sn);
    double *g = (double *)(base + L.g), *y = (double *)(base + L.y);
    GState *gs = (GState *)(base + L.gs);
    // the array keeps the previous call's contents: clear what must start at zero
    PDD_CUDA(cudaMemsetAsync(gs, 0, sizeof(GState), st));
    PDD_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned) * kDotGroups, st));
    PDD_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * n, st));
    PDD_CUDA(cudaMemsetAsync(H, 0, sizeof(double) * (m + 1) * m, st));
    const int vb = std::min(cdiv(n, 256), 2048);
    const int max_iters = std::max(1, o.max_iters);
    SolveResult res;
    for (int cycle = 0;; ++cycle) {
        PDD_LAUNCH(k_spmv, cdiv(n, kRowsPerBlock), 256, 0, st, n, rowptr, col, val, u, w, (const GState *)nullptr);
        PDD_LAUNCH(k_residual_vec, vb, 256, 0, st, n, b, w);
        PDD_LAUNCH(k_dots, dim3(G, 1), kDotThreads, 0, st, n, 1, w, w, partial, hsum, cnt, (const GState *)nullptr);
        PDD_LAUNCH(k_cycle_start, 1, 32, 0, st, gs, hsum, g, m, o.rtol, max_iters, cycle == 0 ? 1 : 0);
        PDD_LAUNCH(k_normalize, vb, kDotBlock, 0, st, n, w, V, hsum, (double *)nullptr, gs);
        for (int j = 0; j < m; ++j) {
            double *vj = V + (long)j * n;
            double *Hc = H + (long)j * (m + 1);
            PDD_LAUNCH(k_spmv, cdiv(n, kRowsPerBlock), 256, 0, st, n, rowptr, col, val, vj, w, gs);
            for (int pass = 0; pass < 2; ++pass) {
                PDD_LAUNCH(k_dots, dim3(G, cdiv(j + 1, kDotVec)), kDotThreads, 0, st, n, j + 1, V, w, partial, hsum, cnt, gs);
                PDD_LAUNCH(k_orth, vb, kDotBlock, 0, st, n, j + 1, V, w, hsum, Hc, pass, gs);
            }
            PDD_LAUNCH(k_dots, dim3(G, 1), kDotThreads, 0, st, n, 1, w, w, partial, hsum, cnt, gs);
            PDD_LAUNCH(k_normalize, vb, kDotBlock, 0, st, n, w, V + (long)(j + 1) * n, hsum, Hc + j + 1, gs);
            PDD_LAUNCH(k_givens, 1, 32, 0, st, H, m + 1, cs, sn, g, j, o.rtol, max_iters, gs);
        }
        PDD_LAUNCH(k_upper_solve, 1, 1, 0, st, H, m + 1, g, y, gs);
        PDD_LAUNCH(k_xupdate, vb, 256, 0, st, n, V, y, gs, u);
        PDD_LAUNCH(k_spmv, cdiv(n, kRowsPerBlock), 256, 0, st, n, rowptr, col, val, u, w, (const GState *)nullptr);
        PDD_LAUNCH(k_residual_vec, vb, 256, 0, st, n, b, w);
        PDD_LAUNCH(k_dots, dim3(G, 1), kDotThreads, 0, st, n, 1, w, w, partial, hsum, cnt, (const GState *)nullptr);
        GState hg{};
        double rs = 0.0;
        PDD_CUDA(cudaMemcpyAsync(&rs, hsum, sizeof(double), cudaMemcpyDeviceToHost, st));
        PDD_CUDA(cudaMemcpyAsync(&hg, gs, sizeof(GState), cudaMemcpyDeviceToHost, st));
        PDD_CUDA(cudaStreamSynchronize(st));
        const double rel = hg.bnorm > 0.0 ? std::sqrt(rs) / hg.bnorm : 0.0;
        res.iters = hg.iters;
        res.rel = rel;
        if (hg.bnorm == 0.0 || rel <= o.rtol) {
            res.converged = 1;
            break;
        }
        if (hg.iters >= max_iters) break;
    }
    return res;
}

}  // namespace pdd

extern "C" pdd_status pdd_solve_csr_noalloc(int n, const int *rowptr, const int *col, const double *val,
                                            const double *b, double *u, const pdd_solve_opts *opts,
                                            pdd_solve_info *info, void *stream) {
    using namespace pdd;
    try {
        if (!opts) fail(PDD_EINVAL, "null solve options");
        if (opts->restart < 1 || opts->restart > 256 || opts->max_iters < 1 || !(opts->rtol > 0))
            fail(PDD_EINVAL, "restart in [1, 256], max_iters >= 1 and rtol > 0 required");
        if (opts->transpose) fail(PDD_EINVAL, "the allocation-free solve takes C itself (transpose = 0)");
        if (n <= 0 || !rowptr || !col || !val || !b || !u) fail(PDD_EINVAL, "null array or n <= 0");
        const int m = opts->restart;
        const int G = std::max(1, std::min(1024, cdiv(n, 2 * kDotThreads)));
        const NoAllocLayout L = noalloc_layout(n, m, G);
        if (L.total > kNoAllocBytes)
            fail(PDD_EINVAL, "workspace of " + std::to_string(L.total) + " bytes exceeds the fixed " +
                                 std::to_string(kNoAllocBytes) + "-byte array: (restart + 2) * n * 8 bytes "
                                 "must stay below about 64 MiB");
        int dev = 0;
        PDD_CUDA(cudaGetDevice(&dev));
        unsigned char *base = (unsigned char *)noalloc_scratch(dev);
        SolveResult r = gmres_csr_fixed(n, rowptr, col, val, b, u, *opts, base, L, m, G, (cudaStream_t)stream);
        if (info) {
            info->iters = r.iters;
            info->rel_residual = r.rel;
            info->converged = r.converged;
        }
        if (!r.converged) fail(PDD_ENOCONV, "GMRES stopped at relative residual " + std::to_string(r.rel));
    } catch (const Fail &f) {
        return f.st;
    }
    return PDD_OK;
}
