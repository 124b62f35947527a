// a13: the global solve C u = r (Eq. 28) in FP64 by restarted GMRES(m)
// (Sec. 4) on a CSR sparse matrix-vector product, plain or right-
// preconditioned (Eq. 45) by the RAS operator of ras.cu.
//
// Layout: the Krylov basis V is (m+1) x n row-major (each basis vector
// contiguous); dot products are block partial sums reduced in a fixed order
// (deterministic).  Orthogonalisation is classical Gram-Schmidt applied
// twice (CGS2).  The m Arnoldi iterations of a restart cycle run in one
// cooperative kernel (k_arnoldi_fused); the Hessenberg matrix, Givens
// rotations and the residual estimate live on the device, and the host
// synchronises once per restart cycle to read the true residual.
#include <cstdlib>
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

// v = w / |w| with |w|^2 = hsum[0]; Hsub = |w|
__global__ void __launch_bounds__(kDotBlock) k_normalize(int n, const double *w, double *v, const double *hsum,
                                                         double *Hsub, const GState *gs) {
    if (gs && gs->stop) return;
    const double nrm = sqrt(hsum[0]);
    if (blockIdx.x == 0 && threadIdx.x == 0 && Hsub) *Hsub = nrm;
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) v[r] = w[r] * inv;
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

// ---------------------------------------------------------------------------
// One restart cycle's Arnoldi iterations in a single cooperative launch.
// Block b owns rows [b per, (b+1) per): it computes w = C v_j on them, their
// partial dot products with the basis, their part of the CGS2 updates and of
// |w|; partial sums meet in global memory and are added in block order after
// a grid barrier (deterministic).  Block 0 keeps the Hessenberg column, the
// Givens rotations and g in shared memory and writes the stop flag that every
// block reads after the iteration's last barrier.  Four grid barriers per
// iteration; each is a bounded spin that records an error and returns.
// ---------------------------------------------------------------------------
static constexpr int kFusedThreads = 512;
static constexpr long long kBarrierLimit = 1LL << 22;   // polls (an L2 read each, ~0.2 us) before giving up

struct FusedArnoldi {
    int n, m;
    const int *rowptr, *col;
    const double *val;
    double *V, *w, *part;        // part: 3 x kMaxDots x gridDim.x partial sums
    double *H, *cs, *sn, *g;     // H column-major (ldh = m + 1)
    GState *gs;
    unsigned *bar;               // [0] arrivals, [1] generation
    int *err;
    double rtol;
    int max_iters;
    unsigned bar_extra;          // arrivals a barrier waits for beyond the grid (0; 1 = never completes)
    long long bar_limit;         // polls before a barrier wait gives up
    // right preconditioner (Eq. 44-45); ras_P = 0: none
    int ras_P, ras_NP;
    const int *ras_wptr, *ras_widx, *ras_p1, *ras_l1, *ras_p2, *ras_l2;
    const float *ras_cinvT;
    float *ras_z;
    double *ras_Z;               // z_j = M^-1 v_j of the cycle, m x n (flexible GMRES)
};

// The block's writes are ordered before thread 0's device-scope fence by the block barrier
// (the same pattern as a cooperative-groups grid sync), so only thread 0 fences; the waiters
// poll the generation word without sleeping.
__device__ __forceinline__ bool grid_barrier(const FusedArnoldi &F) {
    __shared__ int s_bad;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = F.bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        if (atomicAdd(F.bar, 1u) == gridDim.x - 1 + F.bar_extra) {
            atomicExch(F.bar, 0u);
            __threadfence();
            atomicAdd(F.bar + 1, 1u);
        } else {
            long long it = 0;
            while (*gen == g0) {
                if (++it > F.bar_limit) {
                    atomicExch(F.err, 1);
                    break;
                }
            }
        }
        __threadfence();
        s_bad = *(volatile int *)F.err;
    }
    __syncthreads();
    return s_bad == 0;
}

__device__ __forceinline__ double warp_sum(double s) {
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

__global__ void __launch_bounds__(kFusedThreads) k_arnoldi_fused(FusedArnoldi F) {
    constexpr int NW = kFusedThreads / 32;
    __shared__ double h[kMaxDots], hcol[kMaxDots + 1], cs[kMaxDots], sn[kMaxDots], gv[kMaxDots + 1];
    __shared__ double red[NW];
    __shared__ float vs[4 * 128];
    __shared__ int s_stop;
    const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = F.n, m = F.m, ldh = m + 1;
    const int per = (n + G - 1) / G, r0 = min(n, b * per), r1 = min(n, r0 + per);
    if (b == 0)
        for (int i = tid; i <= m; i += kFusedThreads) gv[i] = F.g[i];
    for (int j = 0; j < m; ++j) {
        if (tid == 0) s_stop = __ldcg(&F.gs->stop);
        __syncthreads();
        if (s_stop) break;
        // w = C v_j on this block's rows, 8 lanes per row; v_j was written by every block
        const double *vj = F.V + (long)j * n;
        if (F.ras_P) {
            // z_j = M^-1 v_j (Eq. 44): this block's subsets z_p = C_p^-1 (R_p v_j), then the gather of
            // its own rows; w = C z_j below (right preconditioning, Eq. 45).  z_j is kept: the cycle
            // ends with u += Z y (the flexible form, exact for the products actually taken, which the
            // FP32 local solves make only nearly linear in v)
            const int NP = F.ras_NP;
            // four groups of 128 threads take four subsets at a time: group g of block b the subsets
            // b + G (4 k + g); eight loads of C_p^-1 in flight per thread
            const int grp = tid >> 7, gt = tid & 127;
            for (int k0 = 0; b + G * k0 < F.ras_P; k0 += 4) {
                const int p = b + G * (k0 + grp);
                const bool has = p < F.ras_P;
                const int wb = has ? F.ras_wptr[p] : 0, np_ = has ? F.ras_wptr[p + 1] - wb : 0;
                if (gt < NP) vs[grp * 128 + gt] = gt < np_ ? (float)__ldcg(vj + F.ras_widx[wb + gt]) : 0.f;
                __syncthreads();
                if (has && gt < NP) {
                    const float *ci = F.ras_cinvT + (long)p * NP * NP + gt;
                    const float *vv = vs + grp * 128;
                    float s = 0.f;
                    for (int q0 = 0; q0 < np_; q0 += 8) {
                        float c[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) c[u] = q0 + u < np_ ? ci[(long)(q0 + u) * NP] : 0.f;
#pragma unroll
                        for (int u = 0; u < 8; ++u) s = fmaf(c[u], vv[q0 + u < 128 ? q0 + u : 0], s);
                    }
                    F.ras_z[(long)p * NP + gt] = s;
                }
                __syncthreads();
            }
            if (!grid_barrier(F)) return;
            double *zj = F.ras_Z + (long)j * n;
            for (int r = r0 + tid; r < r1; r += kFusedThreads) {
                const int q2 = F.ras_p2[r];
                const double a = (double)__ldcg(F.ras_z + (long)F.ras_p1[r] * NP + F.ras_l1[r]);
                zj[r] = q2 >= 0 ? 0.5 * (a + (double)__ldcg(F.ras_z + (long)q2 * NP + F.ras_l2[r])) : a;
            }
            if (!grid_barrier(F)) return;
            vj = zj;
        }
        // (every lane of a warp runs the same number of slots: the shuffles below use the full mask);
        // the row's column indices and values are loaded before the gathers
        for (int base = r0; base < r1; base += kFusedThreads / 8) {
            const int row = base + (tid >> 3), l = tid & 7;
            double s = 0.0;
            if (row < r1) {
                const int ka = F.rowptr[row], kb = F.rowptr[row + 1];
                for (int k0 = ka + l; k0 < kb; k0 += 32) {
                    int c[4];
                    double a[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int k = k0 + 8 * q;
                        c[q] = k < kb ? F.col[k] : 0;
                        a[q] = k < kb ? F.val[k] : 0.0;
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) s += a[q] * __ldcg(vj + c[q]);
                }
            }
            s += __shfl_xor_sync(0xffffffffu, s, 4);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            if (row < r1 && l == 0) F.w[row] = s;
        }
        __syncthreads();
        // two passes of classical Gram-Schmidt against v_0 .. v_j; eight loads in flight per lane
        for (int pass = 0; pass < 2; ++pass) {
            double *pp = F.part + (long)pass * kMaxDots * G;
            for (int t = warp; t <= j; t += NW) {
                const double *vt = F.V + (long)t * n;
                double s = 0.0;
                for (int rb = r0 + lane; rb < r1; rb += 256) {
                    double v[8], x[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int r = rb + 32 * q;
                        v[q] = r < r1 ? vt[r] : 0.0;
                        x[q] = r < r1 ? F.w[r] : 0.0;
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q) s += v[q] * x[q];
                }
                s = warp_sum(s);
                if (lane == 0) pp[(long)t * G + b] = s;
            }
            if (!grid_barrier(F)) return;
            for (int t = warp; t <= j; t += NW) {
                double s = 0.0;
                for (int qb = lane; qb < G; qb += 256) {
                    double v[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[q] = qb + 32 * q < G ? __ldcg(pp + (long)t * G + qb + 32 * q) : 0.0;
#pragma unroll
                    for (int q = 0; q < 8; ++q) s += v[q];
                }
                s = warp_sum(s);
                if (lane == 0) h[t] = s;
            }
            __syncthreads();
            if (b == 0)
                for (int t = tid; t <= j; t += kFusedThreads) hcol[t] = pass ? hcol[t] + h[t] : h[t];
            for (int r = r0 + tid; r < r1; r += kFusedThreads) {
                double s = F.w[r];
                for (int t0 = 0; t0 <= j; t0 += 8) {
                    double v[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[q] = t0 + q <= j ? F.V[(long)(t0 + q) * n + r] : 0.0;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (t0 + q <= j) s -= v[q] * h[t0 + q];
                }
                F.w[r] = s;
            }
            __syncthreads();
        }
        // |w|
        {
            double s = 0.0;
            for (int r = r0 + tid; r < r1; r += kFusedThreads) s += F.w[r] * F.w[r];
            s = warp_sum(s);
            if (lane == 0) red[warp] = s;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int q = 0; q < NW; ++q) t += red[q];
                F.part[2L * kMaxDots * G + b] = t;
            }
        }
        if (!grid_barrier(F)) return;
        if (warp == 0) {
            const double s = warp_sum([&] {
                double a = 0.0;
                for (int q = lane; q < G; q += 32) a += __ldcg(F.part + 2L * kMaxDots * G + q);
                return a;
            }());
            if (lane == 0) red[0] = s;
        }
        __syncthreads();
        const double nrm = sqrt(red[0]);
        const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
        double *vn = F.V + (long)(j + 1) * n;
        for (int r = r0 + tid; r < r1; r += kFusedThreads) vn[r] = F.w[r] * inv;
        if (b == 0 && tid == 0) {
            // Givens: the previous rotations on column j, a new one, g and the stop flag
            hcol[j + 1] = nrm;
            double hi = hcol[0];
            for (int i = 0; i < j; ++i) {
                const double hn = hcol[i + 1];
                const double t = cs[i] * hi + sn[i] * hn;
                hi = -sn[i] * hi + cs[i] * hn;
                hcol[i] = t;
            }
            const double a = hi, bb = hcol[j + 1];
            const double den = hypot(a, bb);
            const double c = den > 0.0 ? a / den : 1.0, sv = den > 0.0 ? bb / den : 0.0;
            cs[j] = c;
            sn[j] = sv;
            hcol[j] = den;
            hcol[j + 1] = 0.0;
            gv[j + 1] = -sv * gv[j];
            gv[j] = c * gv[j];
            GState *gs = F.gs;
            gs->iters += 1;
            gs->k_used = j + 1;
            gs->res = fabs(gv[j + 1]);
            if (gs->res <= F.rtol * gs->bnorm || gs->iters >= F.max_iters || bb == 0.0) gs->stop = 1;
        }
        if (b == 0) {
            __syncthreads();
            double *Hc = F.H + (long)j * ldh;
            for (int i = tid; i <= j + 1; i += kFusedThreads) Hc[i] = hcol[i];
            for (int i = tid; i <= j + 1; i += kFusedThreads) F.g[i] = gv[i];
        }
        if (!grid_barrier(F)) return;
    }
}

// buffers of one GMRES(m) solve; gmres_csr allocates them, the allocation-free entry point carves
// them from its fixed array
struct GmresBufs {
    double *V, *w, *partial, *hsum, *H, *cs, *sn, *g, *y, *fpart;
    unsigned *cnt, *bar;
    GState *gs;
    int *err;
};

// SM count of the current device (the occupancy check once per device: devices may differ)
static int fused_grid(int n) {
    static constexpr int kDevs = 64;
    static int sms_of[kDevs] = {0};
    static std::mutex mu;
    int dev = 0;
    PDD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kDevs) fail(PDD_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(mu);
    if (!sms_of[dev]) {
        int sms = 0, per_sm = 0;
        PDD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        PDD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_arnoldi_fused, kFusedThreads, 0));
        if (per_sm < 1) fail(PDD_ECUDA, "the fused Arnoldi kernel does not fit on an SM");
        sms_of[dev] = sms;
    }
    return std::max(1, std::min(sms_of[dev], cdiv(n, 64)));     // one block per SM: co-resident, cheap barriers
}

// Failure injection on the host (tests): PDD_INJECT_BARRIER_TIMEOUT=1 makes every grid barrier
// of the fused Arnoldi kernel wait for one arrival more than the grid has, with a short poll
// limit; each block gives up after that limit, records the error and returns, and the solve
// reports PDD_ECUDA.  The device context stays usable.
static bool inject_barrier_timeout() {
    const char *v = std::getenv("PDD_INJECT_BARRIER_TIMEOUT");
    return v && v[0] == '1';
}

static SolveResult gmres_run(int n, const int *rowptr, const int *col, const double *val, const double *b, double *u,
                             const pdd_solve_opts &o, const GmresBufs &B, int m, int G, cudaStream_t st,
                             const RasPrecond *Mr = nullptr, double *Z = nullptr) {
    PDD_CUDA(cudaMemsetAsync(B.gs, 0, sizeof(GState), st));
    PDD_CUDA(cudaMemsetAsync(B.cnt, 0, sizeof(unsigned) * kDotGroups, st));
    PDD_CUDA(cudaMemsetAsync(B.bar, 0, sizeof(unsigned) * 2, st));
    PDD_CUDA(cudaMemsetAsync(B.err, 0, sizeof(int), st));
    PDD_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * n, st));
    PDD_CUDA(cudaMemsetAsync(B.H, 0, sizeof(double) * (m + 1) * m, st));
    const int vb = std::min(cdiv(n, 256), 2048);
    const int max_iters = std::max(1, o.max_iters);
    const int Gf = fused_grid(n);
    const bool inject = inject_barrier_timeout();
    FusedArnoldi F{n, m, rowptr, col, val, B.V, B.w, B.fpart, B.H, B.cs, B.sn, B.g, B.gs, B.bar, B.err, o.rtol,
                   max_iters, inject ? 1u : 0u, inject ? (1LL << 14) : kBarrierLimit, 0, 0, nullptr, nullptr, nullptr,
                   nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (Mr) {
        F.ras_P = Mr->P;
        F.ras_NP = Mr->NP;
        F.ras_wptr = Mr->wptr.p;
        F.ras_widx = Mr->widx.p;
        F.ras_p1 = Mr->p1.p;
        F.ras_l1 = Mr->l1.p;
        F.ras_p2 = Mr->p2.p;
        F.ras_l2 = Mr->l2.p;
        F.ras_cinvT = Mr->cinvT.p;
        F.ras_z = Mr->z.p;
        F.ras_Z = Z;
    }
    SolveResult res;
    for (int cycle = 0;; ++cycle) {
        // r = b - C u  (u = 0 on the first cycle)
        PDD_LAUNCH(k_spmv, cdiv(n, kRowsPerBlock), 256, 0, st, n, rowptr, col, val, u, B.w, (const GState *)nullptr);
        PDD_LAUNCH(k_residual_vec, vb, 256, 0, st, n, b, B.w);
        PDD_LAUNCH(k_dots, dim3(G, 1), kDotThreads, 0, st, n, 1, B.w, B.w, B.partial, B.hsum, B.cnt,
                   (const GState *)nullptr);
        PDD_LAUNCH(k_cycle_start, 1, 32, 0, st, B.gs, B.hsum, B.g, m, o.rtol, max_iters, cycle == 0 ? 1 : 0);
        PDD_LAUNCH(k_normalize, vb, kDotBlock, 0, st, n, B.w, B.V, B.hsum, (double *)nullptr, B.gs);
        void *args[] = {&F};
        PDD_CUDA(cudaLaunchCooperativeKernel((const void *)k_arnoldi_fused, dim3(Gf), dim3(kFusedThreads), args, 0,
                                             st));
        count_launch();
        PDD_LAUNCH(k_upper_solve, 1, 1, 0, st, B.H, m + 1, B.g, B.y, B.gs);
        // u += Z y (preconditioned: the z_j = M^-1 v_j of the cycle) or V y
        PDD_LAUNCH(k_xupdate, vb, 256, 0, st, n, Mr ? Z : B.V, B.y, B.gs, u);
        // true residual
        PDD_LAUNCH(k_spmv, cdiv(n, kRowsPerBlock), 256, 0, st, n, rowptr, col, val, u, B.w, (const GState *)nullptr);
        PDD_LAUNCH(k_residual_vec, vb, 256, 0, st, n, b, B.w);
        PDD_LAUNCH(k_dots, dim3(G, 1), kDotThreads, 0, st, n, 1, B.w, B.w, B.partial, B.hsum, B.cnt,
                   (const GState *)nullptr);
        GState hg{};
        double rs = 0.0;
        int herr = 0;
        PDD_CUDA(cudaMemcpyAsync(&rs, B.hsum, sizeof(double), cudaMemcpyDeviceToHost, st));
        PDD_CUDA(cudaMemcpyAsync(&hg, B.gs, sizeof(GState), cudaMemcpyDeviceToHost, st));
        PDD_CUDA(cudaMemcpyAsync(&herr, B.err, sizeof(int), cudaMemcpyDeviceToHost, st));
        PDD_CUDA(cudaStreamSynchronize(st));
        if (herr) fail(PDD_ECUDA, "GMRES grid barrier timed out");
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

SolveResult gmres_csr(int n, const int *rowptr, const int *col, const double *val, const double *b, double *u,
                      const pdd_solve_opts &o, cudaStream_t st, const RasPrecond *Mr) {
    const int m = std::max(1, std::min(256, o.restart));
    const int G = std::max(1, std::min(1024, cdiv(n, 2 * kDotThreads)));
    const int Gf = fused_grid(n);
    DevBuf<double> V, w, partial, hsum, H, cs, sn, g, y, fpart;
    DevBuf<unsigned> cnt, bar;
    DevBuf<GState> gs;
    DevBuf<int> err;
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
    fpart.alloc((size_t)3 * kMaxDots * Gf);
    bar.alloc(2);
    err.alloc(1);
    const GmresBufs B{V.p, w.p, partial.p, hsum.p, H.p, cs.p, sn.p, g.p, y.p, fpart.p, cnt.p, bar.p, gs.p, err.p};
    DevBuf<double> Z;
    if (Mr) Z.alloc((size_t)m * n);
    return gmres_run(n, rowptr, col, val, b, u, o, B, m, G, st, Mr, Z.p);
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
    exclusive_scan_async(cnt.p, rowptr_t.p, n, st, nullptr);
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
    size_t V, w, partial, hsum, cnt, H, cs, sn, g, y, gs, fpart, bar, err, total;
};

static NoAllocLayout noalloc_layout(int n, int m, int G, int Gf) {
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
    L.fpart = off; off += up(sizeof(double) * (size_t)3 * kMaxDots * Gf);
    L.bar = off; off += up(sizeof(unsigned) * 2);
    L.err = off; off += up(sizeof(int));
    L.total = off;
    return L;
}

// The same iteration as gmres_csr, on buffers carved from `base`.
static SolveResult gmres_csr_fixed(int n, const int *rowptr, const int *col, const double *val,
                                   const double *b, double *u, const pdd_solve_opts &o, unsigned char *base,
                                   const NoAllocLayout &L, int m, int G, cudaStream_t st) {
    const GmresBufs B{(double *)(base + L.V), (double *)(base + L.w), (double *)(base + L.partial),
                      (double *)(base + L.hsum), (double *)(base + L.H), (double *)(base + L.cs),
                      (double *)(base + L.sn), (double *)(base + L.g), (double *)(base + L.y),
                      (double *)(base + L.fpart), (unsigned *)(base + L.cnt), (unsigned *)(base + L.bar),
                      (GState *)(base + L.gs), (int *)(base + L.err)};
    return gmres_run(n, rowptr, col, val, b, u, o, B, m, G, st);
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
        if (opts->precond != PDD_PRECOND_NONE) fail(PDD_EINVAL, "the allocation-free solve takes no preconditioner");
        if (n <= 0 || !rowptr || !col || !val || !b || !u) fail(PDD_EINVAL, "null array or n <= 0");
        const int m = opts->restart;
        const int G = std::max(1, std::min(1024, cdiv(n, 2 * kDotThreads)));
        const NoAllocLayout L = noalloc_layout(n, m, G, fused_grid(n));
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
