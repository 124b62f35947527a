// a7 (mixed form): recursive partial-pivoting LU of a batch of n x n FP32
// matrices (row-major, in place), all disks of a wave at once.
//
//   lu(k0, w):   w <= W: k_panel_leaf (one CTA per disk, panel in shared
//                memory, row interchanges applied to whole rows);
//                else    lu(k0, w1); trsm(k0, w1 | cols k0+w1..k0+w);
//                        A22 -= L21 U12 (batched GEMM, K = w1); lu(k0+w1, w-w1)
//   trsm(r0, w): w <= W: k_trsm_leaf (unit lower, one thread per column);
//                else    trsm(r0, w1); B2 -= L21 X1 (batched GEMM); trsm(r0+w1, w-w1)
//
// Most of the 2/3 n^3 flops land in GEMMs with K = n/2, n/4, ..., which
// run on the tcgen05 tensor cores with split-TF32 products
// (gemm_sub_tf32x3); thin updates use a CUDA-core FP32 GEMM.  The result
// is the same factorisation P A = L U as the one-CTA right-looking kernel,
// to FP32 rounding; FP64 iterative refinement (a8) follows.
#include <algorithm>
#include <vector>

#include "handles.cuh"

namespace pdd {

void gemm_sub_tf32x3(int batch, int M, int N, int K, const float *A, long sA, int lda, const float *B, long sB,
                     int ldb, float *C, long sC, int ldc, int *err, cudaStream_t st);

__device__ __forceinline__ void apply_panel_swaps(float *A, int n, int k0, int w, const int *piv, int tid, int nt);

// factor columns [k0, k0+w) of rows [k0, n); perm tracks P A = L U
template <int W>
__global__ void __launch_bounds__(256) k_panel_leaf(float *Aall, int n, long strideA, int k0, int w, int *permAll,
                                                    int *infoAll) {
    extern __shared__ __align__(16) float pn[];          // (n - k0) x (W + 1): padded rows, no bank conflicts
    constexpr int LD = W + 1;
    __shared__ int piv[W];
    __shared__ float rv[8];
    __shared__ int ri[8];
    const int disk = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *A = Aall + disk * strideA;
    int *perm = permAll + (long)disk * n;
    const int rows = n - k0;
    int *ps = reinterpret_cast<int *>(pn + (size_t)rows * LD);   // perm[k0 ..], stored at the end
    for (int idx = tid; idx < rows * w; idx += 256) {
        const int r = idx / w, c = idx - r * w;
        pn[r * LD + c] = A[(long)(k0 + r) * n + k0 + c];
    }
    for (int r = tid; r < rows; r += 256) ps[r] = perm[k0 + r];
    __syncthreads();
    int info = 0;
    for (int c = 0; c < w; ++c) {
        float best = -1.f;
        int bi = c;
        for (int r = c + tid; r < rows; r += 256) {
            const float v = fabsf(pn[r * LD + c]);
            if (v > best) { best = v; bi = r; }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { rv[warp] = best; ri[warp] = bi; }
        __syncthreads();
        if (tid == 0) {
            float b = rv[0];
            int i0 = ri[0];
            for (int q = 1; q < 8; ++q)
                if (rv[q] > b || (rv[q] == b && ri[q] < i0)) { b = rv[q]; i0 = ri[q]; }
            piv[c] = i0;
            if (i0 != c) {
                const int t = ps[c];
                ps[c] = ps[i0];
                ps[i0] = t;
            }
        }
        __syncthreads();
        const int p = piv[c];
        if (p != c && tid < w) {
            const float t = pn[c * LD + tid];
            pn[c * LD + tid] = pn[p * LD + tid];
            pn[p * LD + tid] = t;
        }
        __syncthreads();
        const float d = pn[c * LD + c];
        if (d == 0.f && info == 0) info = k0 + c + 1;
        for (int r = c + 1 + tid; r < rows; r += 256) {
            const float l = (d != 0.f) ? pn[r * LD + c] / d : 0.f;
            pn[r * LD + c] = l;
            for (int cc = c + 1; cc < w; ++cc) pn[r * LD + cc] -= l * pn[c * LD + cc];
        }
        __syncthreads();
    }
    for (int idx = tid; idx < rows * w; idx += 256) {
        const int r = idx / w, c = idx - r * w;
        A[(long)(k0 + r) * n + k0 + c] = pn[r * LD + c];
    }
    for (int r = tid; r < rows; r += 256) perm[k0 + r] = ps[r];
    __syncthreads();
    apply_panel_swaps(A, n, k0, w, piv, tid, 256);
    if (tid == 0 && info && infoAll[disk] == 0) infoAll[disk] = info;
}

// the w pivots of a factored panel, applied to every column outside it
__device__ __forceinline__ void apply_panel_swaps(float *A, int n, int k0, int w, const int *piv, int tid, int nt) {
    for (int c = 0; c < w; ++c) {
        const int p = piv[c];
        if (p != c) {
            float *ra = A + (long)(k0 + c) * n, *rb = A + (long)(k0 + p) * n;
            for (int j = tid; j < n - w; j += nt) {
                const int col = j < k0 ? j : j + w;
                const float t = ra[col];
                ra[col] = rb[col];
                rb[col] = t;
            }
        }
        __syncthreads();
    }
}

// The same panel factorisation with the panel in registers: thread t owns panel rows t and
// t + 512 (panels of at most 1024 rows), all W columns.  Per column: block argmax (lowest row
// index among equal magnitudes), the two rows exchanged through shared memory, and the rank-1
// update of the owned rows from the pivot row (register FMAs).
static constexpr int kPanelThreads = 512, kPanelRows = 2;

template <int W>
__global__ void __launch_bounds__(kPanelThreads, 1) k_panel_reg(float *Aall, int n, long strideA, int k0, int w,
                                                                int *permAll, int *infoAll) {
    constexpr int NT = kPanelThreads, R = kPanelRows, NW = NT / 32;
    __shared__ float xch[2][W];
    __shared__ float rv[NW];
    __shared__ int ri[NW];
    __shared__ int piv[W];
    __shared__ int ps[NT * R];                            // perm[k0 ..], swapped here, stored at the end
    const int disk = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *A = Aall + disk * strideA;
    int *perm = permAll + (long)disk * n;
    const int rows = n - k0;
    for (int r = tid; r < rows; r += NT) ps[r] = perm[k0 + r];
    float a[R][W];
    const bool vec = (n & 3) == 0 && (k0 & 3) == 0 && w == W;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int r = tid + i * NT;
        const float *src = A + (long)(k0 + r) * n + k0;
        if (vec) {
#pragma unroll
            for (int c = 0; c < W; c += 4) {
                const float4 v = r < rows ? *reinterpret_cast<const float4 *>(src + c) : make_float4(0.f, 0.f, 0.f, 0.f);
                a[i][c] = v.x;
                a[i][c + 1] = v.y;
                a[i][c + 2] = v.z;
                a[i][c + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int c = 0; c < W; ++c) a[i][c] = (r < rows && c < w) ? src[c] : 0.f;
        }
    }
    int info = 0;
#pragma unroll
    for (int c = 0; c < W; ++c) {
        if (c >= w) break;
        float best = -1.f;
        int bi = 0x7fffffff;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = tid + i * NT;
            if (r >= c && r < rows) {
                const float v = fabsf(a[i][c]);
                if (v > best || (v == best && r < bi)) {
                    best = v;
                    bi = r;
                }
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            rv[warp] = best;
            ri[warp] = bi;
        }
        __syncthreads();
        if (warp == 0) {
            best = lane < NW ? rv[lane] : -1.f;
            bi = lane < NW ? ri[lane] : 0x7fffffff;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const float ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) {
                    best = ov;
                    bi = oi;
                }
            }
            if (lane == 0) {
                piv[c] = bi;
                if (bi != c) {
                    const int t = ps[c];
                    ps[c] = ps[bi];
                    ps[bi] = t;
                }
            }
        }
        __syncthreads();
        const int p = piv[c];
        // rows c and p through shared memory: xch[0] = row c, xch[1] = row p (the new row c); row c
        // (c < W <= NT) is thread c's first row, row p is row p / NT of thread p % NT
        const int po = p % NT;
        if (tid == c) {
#pragma unroll
            for (int cc = 0; cc < W; ++cc) xch[0][cc] = a[0][cc];
        }
        if (tid == po) {
            if (p < NT) {
#pragma unroll
                for (int cc = 0; cc < W; ++cc) xch[1][cc] = a[0][cc];
            } else {
#pragma unroll
                for (int cc = 0; cc < W; ++cc) xch[1][cc] = a[R - 1][cc];
            }
        }
        __syncthreads();
        if (p != c) {
            if (tid == c) {
#pragma unroll
                for (int cc = 0; cc < W; ++cc) a[0][cc] = xch[1][cc];
            }
            if (tid == po) {
                if (p < NT) {
#pragma unroll
                    for (int cc = 0; cc < W; ++cc) a[0][cc] = xch[0][cc];
                } else {
#pragma unroll
                    for (int cc = 0; cc < W; ++cc) a[R - 1][cc] = xch[0][cc];
                }
            }
        }
        const float d = xch[1][c];
        if (d == 0.f && info == 0) info = k0 + c + 1;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = tid + i * NT;
            if (r > c && r < rows) {
                const float l = (d != 0.f) ? a[i][c] / d : 0.f;
                a[i][c] = l;
#pragma unroll
                for (int cc = c + 1; cc < W; ++cc) a[i][cc] -= l * xch[1][cc];
            }
        }
        __syncthreads();                                  // xch is rewritten by the next column
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int r = tid + i * NT;
        if (r < rows) {
            float *dst = A + (long)(k0 + r) * n + k0;
            if (vec) {
#pragma unroll
                for (int c = 0; c < W; c += 4)
                    *reinterpret_cast<float4 *>(dst + c) = make_float4(a[i][c], a[i][c + 1], a[i][c + 2], a[i][c + 3]);
            } else {
#pragma unroll
                for (int c = 0; c < W; ++c)
                    if (c < w) dst[c] = a[i][c];
            }
        }
    }
    for (int r = tid; r < rows; r += NT) perm[k0 + r] = ps[r];
    __syncthreads();
    apply_panel_swaps(A, n, k0, w, piv, tid, NT);
    if (tid == 0 && info && infoAll[disk] == 0) infoAll[disk] = info;
}

// X = L^-1 X for the unit lower w x w block at (r0, r0), X = A[r0:r0+w, c0:c0+nc]
template <int W>
__global__ void __launch_bounds__(256) k_trsm_leaf(float *Aall, int n, long strideA, int r0, int w, int c0, int nc) {
    __shared__ float L[W * W];
    const int disk = blockIdx.y, tid = threadIdx.x;
    float *A = Aall + disk * strideA;
    for (int idx = tid; idx < w * w; idx += 256) {
        const int i = idx / w, j = idx - i * w;
        L[i * W + j] = A[(long)(r0 + i) * n + r0 + j];
    }
    __syncthreads();
    const int col = blockIdx.x * 256 + tid;
    if (col >= nc) return;
    float x[W];
#pragma unroll
    for (int i = 0; i < W; ++i) {
        if (i < w) {
            float v = A[(long)(r0 + i) * n + c0 + col];
            for (int t = 0; t < i; ++t) v -= L[i * W + t] * x[t];
            x[i] = v;
            A[(long)(r0 + i) * n + c0 + col] = v;
        }
    }
}

// C -= A B on CUDA cores (FP32): 64 x 64 tiles, 4 x 4 per thread, K in chunks of 16
__global__ void __launch_bounds__(256) k_gemm_sub_simt(int M, int N, int K, const float *Aall, int lda,
                                                       const float *Ball, int ldb, float *Call, int ldc,
                                                       long stride) {
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int disk = blockIdx.z, tid = threadIdx.x;
    const float *A = Aall + disk * stride;
    const float *B = Ball + disk * stride;
    float *C = Call + disk * stride;
    const int tm = blockIdx.y * 64, tn = blockIdx.x * 64;
    const int ty = tid >> 4, tx = tid & 15;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = tid; e < 16 * 64; e += 256) {
            const int kk = e & 15, r = e >> 4;
            const int gr = tm + r, gk = k0 + kk;
            As[kk][r] = (gr < M && gk < K) ? A[(long)gr * lda + gk] : 0.f;
            const int kb = e >> 6, j = e & 63;
            const int gk2 = k0 + kb, gj = tn + j;
            Bs[kb][j] = (gk2 < K && gj < N) ? B[(long)gk2 * ldb + gj] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][ty * 4 + q];
                b[q] = Bs[kk][tx * 4 + q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * b[q];
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int r = tm + ty * 4 + p;
        if (r >= M) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = tn + tx * 4 + q;
            if (c < N) C[(long)r * ldc + c] -= acc[p][q];
        }
    }
}

struct RecLU {
    float *A;
    int n;
    long sA;
    int *perm, *info, *err;
    int nd, W;
    cudaStream_t st;
    int tensor_min;     // smallest M, N and K sent to the tensor cores
    std::vector<cudaEvent_t> *gev;   // event pairs around the tensor-core launches, or null
    double flop;                     // useful flops sent to the tensor cores

    float *at(int r, int c) const { return A + (long)r * n + c; }

    void gemm(int r, int c, int M, int N, int K, int ar, int ac, int br, int bc) {
        if (M <= 0 || N <= 0 || K <= 0) return;
        if (M >= tensor_min && N >= tensor_min && K >= tensor_min) {
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (gev) {
                PDD_CUDA(cudaEventCreate(&e0));
                PDD_CUDA(cudaEventCreate(&e1));
                gev->push_back(e0);
                gev->push_back(e1);
                PDD_CUDA(cudaEventRecord(e0, st));
            }
            gemm_sub_tf32x3(nd, M, N, K, at(ar, ac), sA, n, at(br, bc), sA, n, at(r, c), sA, n, err, st);
            if (gev) PDD_CUDA(cudaEventRecord(e1, st));
            flop += 2.0 * M * N * K * nd;
        } else {
            dim3 g(cdiv(N, 64), cdiv(M, 64), nd);
            PDD_LAUNCH(k_gemm_sub_simt, g, 256, 0, st, M, N, K, at(ar, ac), n, at(br, bc), n, at(r, c), n, sA);
        }
    }

    void leaf(int k0, int w) {
        if (n - k0 <= kPanelThreads * kPanelRows) {
            switch (W) {
                case 32: PDD_LAUNCH(k_panel_reg<32>, nd, kPanelThreads, 0, st, A, n, sA, k0, w, perm, info); return;
                case 16: PDD_LAUNCH(k_panel_reg<16>, nd, kPanelThreads, 0, st, A, n, sA, k0, w, perm, info); return;
                default: PDD_LAUNCH(k_panel_reg<8>, nd, kPanelThreads, 0, st, A, n, sA, k0, w, perm, info); return;
            }
        }
        const size_t smem = (size_t)(n - k0) * ((W + 1) * sizeof(float) + sizeof(int));
        switch (W) {
#define PDD_LEAF(WV)                                                                                      \
    case WV:                                                                                              \
        PDD_CUDA(cudaFuncSetAttribute(k_panel_leaf<WV>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                      (int)std::max<size_t>(smem, 1)));                                   \
        PDD_LAUNCH(k_panel_leaf<WV>, nd, 256, smem, st, A, n, sA, k0, w, perm, info);                     \
        break;
            PDD_LEAF(32)
            PDD_LEAF(16)
            PDD_LEAF(8)
#undef PDD_LEAF
            default: fail(PDD_EINVAL, "bad panel width");
        }
    }

    void trsm_leaf(int r0, int w, int c0, int nc) {
        dim3 g(cdiv(nc, 256), nd);
        switch (W) {
            case 32: PDD_LAUNCH(k_trsm_leaf<32>, g, 256, 0, st, A, n, sA, r0, w, c0, nc); break;
            case 16: PDD_LAUNCH(k_trsm_leaf<16>, g, 256, 0, st, A, n, sA, r0, w, c0, nc); break;
            default: PDD_LAUNCH(k_trsm_leaf<8>, g, 256, 0, st, A, n, sA, r0, w, c0, nc); break;
        }
    }

    int split(int w) const { return std::max(W, ((w / 2) / W) * W); }

    void trsm(int r0, int w, int c0, int nc) {
        if (w <= W) {
            trsm_leaf(r0, w, c0, nc);
            return;
        }
        const int w1 = split(w);
        trsm(r0, w1, c0, nc);
        gemm(r0 + w1, c0, w - w1, nc, w1, r0 + w1, r0, r0, c0);
        trsm(r0 + w1, w - w1, c0, nc);
    }

    void lu(int k0, int w) {
        if (w <= W) {
            leaf(k0, w);
            return;
        }
        const int w1 = split(w);
        lu(k0, w1);
        trsm(k0, w1, k0 + w1, w - w1);
        gemm(k0 + w1, k0 + w1, n - (k0 + w1), w - w1, w1, k0 + w1, k0, k0, k0 + w1);
        lu(k0 + w1, w - w1);
    }
};

__global__ void k_iota_perm(int n, int nd, int *perm, int *info) {
    const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx < (long)n * nd) perm[idx] = (int)(idx % n);
    if (idx < nd) info[idx] = 0;
}

void lu_recursive_f32(float *A, int n, long strideA, int *perm, int *info, int nd, cudaStream_t st, int W,
                      int tensor_min, float *ms_gemm, double *gemm_flop) {
    DevBuf<int> err;
    err.alloc(1);
    PDD_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    PDD_LAUNCH(k_iota_perm, cdiv((long)n * nd, 256), 256, 0, st, n, nd, perm, info);
    if (W != 8 && W != 16 && W != 32) fail(PDD_EINVAL, "panel width must be 8, 16 or 32");
    if ((size_t)n * ((W + 1) * sizeof(float) + sizeof(int)) > 200 * 1024)
        fail(PDD_EINVAL, "disk grid too large for the panel width");
    std::vector<cudaEvent_t> gev;
    RecLU r{A, n, strideA, perm, info, err.p, nd, W, st, tensor_min, ms_gemm ? &gev : nullptr, 0.0};
    try {
        r.lu(0, n);
    } catch (...) {
        for (cudaEvent_t e : gev) cudaEventDestroy(e);
        throw;
    }
    int h = 0;
    PDD_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    PDD_CUDA(cudaStreamSynchronize(st));
    if (ms_gemm) {
        float tot = 0.f;
        for (size_t k = 0; k + 1 < gev.size(); k += 2) {
            float t = 0.f;
            cudaEventElapsedTime(&t, gev[k], gev[k + 1]);
            tot += t;
        }
        *ms_gemm += tot;
    }
    if (gemm_flop) *gemm_flop += r.flop;
    for (cudaEvent_t e : gev) cudaEventDestroy(e);
    if (h) fail(PDD_ECUDA, "tensor-core GEMM timed out waiting for its MMAs");
}

}  // namespace pdd
