// a7 (mixed form): recursive LU WITHOUT row interchanges of a batch of n x n
// FP32 matrices (row-major, in place), all disks of a wave at once, with every
// step except the 64 x 64 diagonal blocks on the tcgen05 tensor cores.
//
// The row-equilibrated collocation matrices of Sec. 3.3 (every row scaled to
// max |a_ij| = 1) keep their diagonal as the row maximum, and elimination
// without interchanges shows growth factor 1 on the 16x16, 32x32, 22x44 and
// 48x64 grids (measured in FP32 on the oracle's matrices; partial pivoting
// gives the same growth).  Any pivot below kTinyPivot is recorded per disk,
// and the caller then refactors that wave with partial pivoting; the FP64
// refinement of a8 recovers the accuracy either way.
//
//   lu(k0, w):   w <= 64: factor the diagonal block D (one CTA per disk, the
//                block in registers) and store L_D^-1 and U_D^-1; L21 = A21 U_D^-1 (GEMM);
//                else lu(k0, w1); U12 = L11^-1 A12 (trsm); A22 -= L21 U12
//                (GEMM, K = w1); lu(k0 + w1, w - w1)
//   trsm(r0, w): w <= 64: X = L_D^-1 X (GEMM); else trsm(r0, w1);
//                X2 -= L21 X1 (GEMM); trsm(r0 + w1, w - w1)
// The GEMMs are tc_gemm (tc_gemm.cu), split-TF32 on tcgen05 with FP32
// accumulation in tensor memory: the K = 64 updates through the kernel that
// splits its FP32 operands as it stages them, the longer ones through operands
// split once into tiles and streamed by bulk copies.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "handles.cuh"

namespace pdd {

static constexpr int kLeafW = 64;
static constexpr float kTinyPivot = 1e-5f;       // rows are equilibrated to max |a_ij| = 1

// Factor the w x w diagonal block at (k0, k0) without interchanges (in place) and store the
// inverses of its unit-lower and upper factors: inv[disk][k0 / 64][0] = L_D^-1,
// inv[disk][k0 / 64][1] = U_D^-1 (64 x 64 row-major, zero outside the w x w block).
//
// One sweep over the pivots k with one barrier per step; thread (ty, tx) keeps the 16
// elements (ty + 8a, tx + 32c) in registers for the whole sweep.  An element (i, j) holds its
// Schur-complement value until step min(i, j), then the accumulator of L^-1 (i > j: the
// elimination applied to the identity) or of U^-1 (i < j: X U = I column by column, unscaled
// by 1 / u_jj until the end).  Step k applies one rank-1 form  acc_ij -= m_i r_j  to
//   rows > k (Schur complement for columns > k, L^-1 for columns <= k) and
//   rows <= k, columns > k (U^-1),
// with m_i = (column k of row i) / u_kk (1 / u_kk on row k) and r_j = row k (1 at column k).
// Column k reaches the warp's rows by shuffles from the lane that holds it; row k + 1 is
// published to a double-buffered shared row after step k.  The final factor entries go to a
// shared tile as they become final (row k+1 of U after step k, multipliers of column k in
// step k) and are written out with the inverses at the end.
__global__ void __launch_bounds__(256) k_leaf_diag(float *Aall, int n, long sA, int k0, int w, float *invAll,
                                                   long sInv, int *info) {
    __shared__ float Dout[kLeafW][kLeafW + 1];
    __shared__ float R[2][kLeafW];
    __shared__ float RD[kLeafW];
    const int disk = blockIdx.x, tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    float *A = Aall + disk * sA;
    float acc[8][2];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int i = ty + 8 * a, j = tx + 32 * c;
            acc[a][c] = (i < w && j < w) ? A[(long)(k0 + i) * n + k0 + j] : (i == j ? 1.f : 0.f);
        }
    if (ty == 0) {
        R[0][tx] = Dout[0][tx] = acc[0][0];
        R[0][tx + 32] = Dout[0][tx + 32] = acc[0][1];
    }
    __syncthreads();
    // step k; HI = (k >= 32) names the register that holds column k at compile time
    auto step = [&](int k, auto hi_c) {
        constexpr int HI = decltype(hi_c)::value;
        const int b = k & 1, src = k & 31;
        const float d = R[b][k];
        const float rd = (d != 0.f) ? 1.f / d : 0.f;
        if (tid == 0) {
            RD[k] = rd;
            if (!(fabsf(d) >= kTinyPivot)) atomicCAS(info + disk, 0, k0 + k + 1);
        }
        const float r0 = (tx == k) ? 1.f : R[b][tx];
        const float r1 = (tx + 32 == k) ? 1.f : R[b][tx + 32];
        const bool up0 = tx > k, up1 = tx + 32 > k;
        float m[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) m[a] = __shfl_sync(0xffffffffu, acc[a][HI], src) * rd;
        if (tx == src) {     // column k: multipliers out, then L^-1's column k restarts (1 on the diagonal)
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const int i = ty + 8 * a;
                if (i > k) Dout[i][k] = m[a];
                if (i >= k) acc[a][HI] = (i == k) ? 1.f : 0.f;
            }
        }
        if (ty == (k & 7)) { // row k: U^-1's row k starts from 0 with multiplier 1 / u_kk
            const int ak = k >> 3;
#pragma unroll
            for (int a = 0; a < 8; ++a)
                if (a == ak) {
                    m[a] = rd;
                    if (up0) acc[a][0] = 0.f;
                    if (up1) acc[a][1] = 0.f;
                }
        }
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const bool below = ty + 8 * a > k;
            if (below || up0) acc[a][0] = fmaf(-m[a], r0, acc[a][0]);
            if (below || up1) acc[a][1] = fmaf(-m[a], r1, acc[a][1]);
        }
        if (k + 1 < w && ty == ((k + 1) & 7)) {
            const int ap = (k + 1) >> 3;
#pragma unroll
            for (int a = 0; a < 8; ++a)
                if (a == ap) {
                    R[b ^ 1][tx] = acc[a][0];
                    R[b ^ 1][tx + 32] = acc[a][1];
                    if (up0) Dout[k + 1][tx] = acc[a][0];
                    if (up1) Dout[k + 1][tx + 32] = acc[a][1];
                }
        }
        __syncthreads();
    };
    const int kh = w < 32 ? w : 32;
    for (int k = 0; k < kh; ++k) step(k, std::integral_constant<int, 0>());
    for (int k = 32; k < w; ++k) step(k, std::integral_constant<int, 1>());
    float *inv = invAll + disk * sInv + (long)(k0 / kLeafW) * 2 * kLeafW * kLeafW;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int i = ty + 8 * a, j = tx + 32 * c;
            const bool in = i < w && j < w;
            if (in) A[(long)(k0 + i) * n + k0 + j] = Dout[i][j];
            inv[i * kLeafW + j] = in ? (i > j ? acc[a][c] : (i == j ? 1.f : 0.f)) : 0.f;
            inv[kLeafW * kLeafW + i * kLeafW + j] = (in && i <= j) ? acc[a][c] * RD[j] : 0.f;
        }
}

struct NpLU {
    float *A;
    int n;
    long sA;
    int nd;
    float *inv;
    long sInv;
    int *info, *err;
    float *scratch;
    size_t scratch_floats;
    cudaStream_t st;
    TcTiming *tt;                    // event pairs around the tensor-core GEMM kernels, or null

    float *at(int r, int c) const { return A + (long)r * n + c; }
    const float *invL(int k0) const { return inv + (long)(k0 / kLeafW) * 2 * kLeafW * kLeafW; }
    const float *invU(int k0) const { return invL(k0) + kLeafW * kLeafW; }

    void gemm(int M, int N, int K, const float *a, long sa, int lda, const float *b, long sb, int ldb, float *c,
              bool sub, int alias) {
        if (M <= 0 || N <= 0 || K <= 0) return;
        tc_gemm(nd, M, N, K, a, sa, lda, false, b, sb, ldb, false, c, sA, n, sub, alias, scratch, scratch_floats,
                err, st, tt);
    }

    int split(int w) const { return std::max(kLeafW, ((w / 2) / kLeafW) * kLeafW); }

    // X = L[r0:r0+w, r0:r0+w]^-1 X with X = A[r0:r0+w, c0:c0+nc] (unit lower L)
    void trsm(int r0, int w, int c0, int nc) {
        if (w <= kLeafW) {
            gemm(w, nc, w, invL(r0), sInv, kLeafW, at(r0, c0), sA, n, at(r0, c0), false, TC_ALIAS_B);
            return;
        }
        const int w1 = split(w);
        trsm(r0, w1, c0, nc);
        gemm(w - w1, nc, w1, at(r0 + w1, r0), sA, n, at(r0, c0), sA, n, at(r0 + w1, c0), true, TC_ALIAS_NONE);
        trsm(r0 + w1, w - w1, c0, nc);
    }

    void lu(int k0, int w) {
        if (w <= kLeafW) {
            PDD_LAUNCH(k_leaf_diag, nd, 256, 0, st, A, n, sA, k0, w, inv, sInv, info);
            const int below = n - k0 - w;
            if (below > 0)
                gemm(below, w, w, at(k0 + w, k0), sA, n, invU(k0), sInv, kLeafW, at(k0 + w, k0), false, TC_ALIAS_A);
            return;
        }
        const int w1 = split(w);
        lu(k0, w1);
        trsm(k0, w1, k0 + w1, w - w1);
        gemm(n - (k0 + w1), w - w1, w1, at(k0 + w1, k0), sA, n, at(k0, k0 + w1), sA, n, at(k0 + w1, k0 + w1), true,
             TC_ALIAS_NONE);
        lu(k0 + w1, w - w1);
    }
};

// floats of inverse storage per disk and of GEMM tile scratch per disk (the largest GEMM)
long lu_np_inv_floats(int n) { return (long)cdiv(n, kLeafW) * 2 * kLeafW * kLeafW; }

size_t lu_np_scratch_floats_per_disk(int n) {
    if (n <= kLeafW) return 0;
    const int w1 = std::max(kLeafW, ((n / 2) / kLeafW) * kLeafW);
    // the GEMMs with K > 64 go through pre-split tiles; the top-level Schur update (M = n - w1,
    // N = n - w1, K = w1) bounds them all (the K = 64 updates take the fused kernel)
    return tc_tile_floats(n - w1, w1) * 2;
}

__global__ void k_iota_perm_np(int n, int nd, int *perm) {
    const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx < (long)n * nd) perm[idx] = (int)(idx % n);
}

// info[d] = 1-based index of the first pivot below kTinyPivot of disk d, 0 when none
void lu_nopivot_f32(float *A, int n, long strideA, int *perm, int *info, int nd, float *inv, long sInv,
                    float *scratch, size_t scratch_floats, cudaStream_t st, DiskStats *ds) {
    DevBuf<int> err;
    err.alloc(1);
    PDD_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    PDD_CUDA(cudaMemsetAsync(info, 0, sizeof(int) * nd, st));
    PDD_LAUNCH(k_iota_perm_np, cdiv((long)n * nd, 256), 256, 0, st, n, nd, perm);
    TcTiming tt;
    auto destroy = [&tt]() {
        for (cudaEvent_t e : tt.pipe) cudaEventDestroy(e);
        for (cudaEvent_t e : tt.fused) cudaEventDestroy(e);
    };
    NpLU r{A, n, strideA, nd, inv, sInv, info, err.p, scratch, scratch_floats, st, ds ? &tt : nullptr};
    try {
        r.lu(0, n);
    } catch (...) {
        destroy();
        throw;
    }
    int h = 0;
    PDD_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    PDD_CUDA(cudaStreamSynchronize(st));
    if (ds) {
        auto sum = [](const std::vector<cudaEvent_t> &ev) {
            float tot = 0.f;
            for (size_t k = 0; k + 1 < ev.size(); k += 2) {
                float t = 0.f;
                cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
                tot += t;
            }
            return tot;
        };
        const float mf = sum(tt.fused);
        ds->ms_tc_gemm += sum(tt.pipe) + mf;
        ds->ms_gemm_fused += mf;
        ds->tc_gemm_flop += tt.flop_pipe + tt.flop_fused;
        ds->gemm_fused_flop += tt.flop_fused;
        ds->gemm_fused_bytes += tt.bytes_fused;
        ds->gemm_pipe_launches += (int64_t)(tt.pipe.size() / 2);
    }
    destroy();
    if (h) fail(PDD_ECUDA, "tensor-core GEMM timed out waiting for its pipeline");
}

}  // namespace pdd
