// Batched C -= A * B on the 5th-generation tensor cores (tcgen05), FP32 in and
// out with split-TF32 products: each operand is split into hi = tf32(x) and
// lo = tf32(x - hi); A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped
// lo*lo term is ~2^-22 relative), accumulated in FP32 in tensor memory.
// This is the Schur-complement update of the recursive disk LU (a7) and of
// its triangular solves; it keeps the factors accurate to about FP32, which
// the FP64 refinement of a8 needs (one TF32 product would leave
// kappa(A) u_tf32 > 1 on the 32x32 and 48x64 disk grids).
//
// One CTA (256 threads) computes a 128 x 128 tile of C for one matrix of the
// batch:
//   * the K loop runs in chunks of 16; each chunk is loaded with 16-byte
//     loads into registers two chunks ahead of the tensor cores,
//     split, and stored into shared memory in the canonical no-swizzle
//     K-major layout (8-row x 16-byte core matrices; LBO = K-direction core
//     stride, SBO = 8-row-group stride), hi and lo copies, double-buffered;
//   * one thread issues 4 k-steps x 3 tcgen05.mma.kind::tf32 (M = 128,
//     N = 128, K = 8) into a TMEM accumulator and commits them to the
//     buffer's mbarrier;
//   * the epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM
//     lanes 32(w mod 4).. = rows, and one half of the columns) and subtracts
//     it from C.
//   * 64 KB of shared memory and 128 TMEM columns per CTA: two CTAs share an
//     SM, so one's prologue and epilogue overlap the other's MMAs.
// Every mbarrier wait is bounded: on timeout the kernel records an error,
// waits once more (bounded) for its own MMAs, frees its TMEM and returns.
#include <algorithm>
#include <vector>

#include "handles.cuh"
#include "mbarrier.cuh"

namespace pdd {

static constexpr int kTM = 128, kTN = 128, kTK = 16;
static constexpr int kOpBytes = kTM * kTK * 4;          // one operand copy: 8 KB
static constexpr int kStageBytes = 4 * kOpBytes;        // A_hi, A_lo, B_hi, B_lo
static constexpr int kTcSmem = 2 * kStageBytes;        // two stages (64 KB: two CTAs per SM)
static constexpr int kTmemCols = 128;                   // one 128 x 128 FP32 accumulator

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// shared-memory matrix descriptor, no swizzle, K-major
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;                    // descriptor version for tcgen05
    return d;                                  // base offset 0, LBO mode 0, no swizzle
}

// instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4)                   // D format F32
           | (2u << 7)                 // A format TF32
           | (2u << 10)                // B format TF32
           | ((uint32_t)(N >> 3) << 17)
           | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// element (r, k) of a rows x 32 operand tile in the canonical layout
__device__ __forceinline__ int canon_off(int r, int k, int rows) {
    return (k >> 2) * (rows * 16) + (r >> 3) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

static constexpr int kTcThreads = 256;

// One K chunk (16) of the two operands in registers (vector path): thread (warp w, lane l) holds
//   A: 2 float4 = rows 8 (8 i + w) + (l & 7), k = 4 (l >> 3) .. + 3
//   B: 2 float4 = row k = (l >> 3) + 4 (w >> 1), columns 4 ((l & 7) + 8 (2 (w & 1) + i)) .. + 3
// so that a warp's global loads cover whole 32-byte sectors and its shared-memory stores
// into the canonical layout hit 32 different banks.
struct Chunk {
    float4 a[2], b[2];
};

__device__ __forceinline__ int chunk_a_row(int i, int w, int l) { return 8 * (8 * i + w) + (l & 7); }
__device__ __forceinline__ int chunk_a_k(int l) { return 4 * (l >> 3); }
__device__ __forceinline__ int chunk_b_k(int w, int l) { return (l >> 3) + 4 * (w >> 1); }
__device__ __forceinline__ int chunk_b_j(int i, int w, int l) { return 4 * ((l & 7) + 8 * (2 * (w & 1) + i)); }

__device__ __forceinline__ void load_chunk_vec(Chunk &c, const float *A, int lda, const float *B, int ldb, int M,
                                               int N, int K, int tm, int tn, int k0, int w, int l) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int gr = tm + chunk_a_row(i, w, l), gk = k0 + chunk_a_k(l);
        c.a[i] = (gr < M && gk < K) ? __ldg(reinterpret_cast<const float4 *>(A + (long)gr * lda + gk))
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int gk = k0 + chunk_b_k(w, l), gj = tn + chunk_b_j(i, w, l);
        c.b[i] = (gk < K && gj < N) ? __ldg(reinterpret_cast<const float4 *>(B + (long)gk * ldb + gj))
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__device__ __forceinline__ float4 split_hi(float4 v) {
    return make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
}

__device__ __forceinline__ float4 split_lo(float4 v, float4 h) {
    return make_float4(tf32_round(v.x - h.x), tf32_round(v.y - h.y), tf32_round(v.z - h.z), tf32_round(v.w - h.w));
}

__device__ __forceinline__ float pick4(float4 v, int e) {
    return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

__device__ __forceinline__ void store_chunk_vec(const Chunk &c, float *Ahi, float *Alo, float *Bhi, float *Blo, int w,
                                                int l) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int off = canon_off(chunk_a_row(i, w, l), chunk_a_k(l), kTM) >> 2;
        const float4 h = split_hi(c.a[i]);
        *reinterpret_cast<float4 *>(Ahi + off) = h;
        *reinterpret_cast<float4 *>(Alo + off) = split_lo(c.a[i], h);
    }
    const int rot = (l >> 1) & 3;            // element order rotated per lane: conflict-free stores
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int k = chunk_b_k(w, l), j0 = chunk_b_j(i, w, l);
        const float4 h = split_hi(c.b[i]);
        const float4 lo = split_lo(c.b[i], h);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int ee = (e + rot) & 3;
            const int off = canon_off(j0 + ee, k, kTN) >> 2;
            Bhi[off] = pick4(h, ee);
            Blo[off] = pick4(lo, ee);
        }
    }
}

// scalar staging for shapes or addresses that are not 16-byte aligned
__device__ __forceinline__ void stage_scalar(const float *A, int lda, const float *B, int ldb, int M, int N, int K,
                                             int tm, int tn, int k0, float *Ahi, float *Alo, float *Bhi, float *Blo,
                                             int tid) {
    for (int e = tid; e < kTM * kTK; e += kTcThreads) {
        const int r = e / kTK, k = e % kTK;
        const int gr = tm + r, gk = k0 + k;
        const float v = (gr < M && gk < K) ? A[(long)gr * lda + gk] : 0.f;
        const float hi = tf32_round(v);
        const int off = canon_off(r, k, kTM) >> 2;
        Ahi[off] = hi;
        Alo[off] = tf32_round(v - hi);
    }
    for (int e = tid; e < kTK * kTN; e += kTcThreads) {
        const int k = e >> 7, j = e & 127;
        const int gk = k0 + k, gj = tn + j;
        const float v = (gk < K && gj < N) ? B[(long)gk * ldb + gj] : 0.f;
        const float hi = tf32_round(v);
        const int off = canon_off(j, k, kTN) >> 2;
        Bhi[off] = hi;
        Blo[off] = tf32_round(v - hi);
    }
}

// C (tile rows tm.., columns tn..) -= the TMEM accumulator; warp w reads TMEM lanes 32 (w & 3) ..
// (rows) and the column half (w >> 2)
template <bool VEC>
__device__ __forceinline__ void epilogue(uint32_t tmem, float *C, int ldc, int M, int N, int tm, int tn, int w,
                                         int l) {
    const int row = tm + (w & 3) * 32 + l;
#pragma unroll 1
    for (int c0 = (w >> 2) * 64; c0 < (w >> 2) * 64 + 64; c0 += 32) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)((w & 3) * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
              "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
              "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
              "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < M) {
            float *crow = C + (long)row * ldc + tn + c0;
            if (VEC && tn + c0 + 32 <= N) {
#pragma unroll
                for (int q = 0; q < 32; q += 4) {
                    float4 cv = *reinterpret_cast<float4 *>(crow + q);
                    cv.x -= __uint_as_float(v[q]);
                    cv.y -= __uint_as_float(v[q + 1]);
                    cv.z -= __uint_as_float(v[q + 2]);
                    cv.w -= __uint_as_float(v[q + 3]);
                    *reinterpret_cast<float4 *>(crow + q) = cv;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 32; ++q)
                    if (tn + c0 + q < N) crow[q] -= __uint_as_float(v[q]);
            }
        }
    }
}

template <bool VEC>
__global__ void __launch_bounds__(kTcThreads, 2) k_gemm_sub_tf32x3(int M, int N, int K, const float *A, long sA,
                                                                   int lda, const float *B, long sB, int ldb,
                                                                   float *C, long sC, int ldc, int *err) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int bz = blockIdx.z;
    const int tm = blockIdx.y * kTM, tn = blockIdx.x * kTN;
    A += bz * sA;
    B += bz * sB;
    C += bz * sC;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        failed = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const int nch = (K + kTK - 1) / kTK;
    const uint32_t idesc = idesc_tf32(kTM, kTN);
    const uint32_t lbo = kTM * 16;             // K-direction core-matrix stride (rows = 128)
    const uint32_t sbo = 128;                  // 8-row-group stride
    int issued = -1;                           // last chunk whose MMAs were committed (uniform)
    Chunk cur, nxt;                            // chunks kc and kc + 1 in flight
    if (VEC && nch > 0) load_chunk_vec(cur, A, lda, B, ldb, M, N, K, tm, tn, 0, warp, lane);
    if (VEC && nch > 1) load_chunk_vec(nxt, A, lda, B, ldb, M, N, K, tm, tn, kTK, warp, lane);
    for (int kc = 0; kc < nch; ++kc) {
        const int buf = kc & 1;
        unsigned char *st = tsm + buf * kStageBytes;
        if (kc >= 2 && tid == 0) {
            if (!mbar_wait(smem_u32(&mbar[buf]), ((kc - 2) >> 1) & 1)) failed = 1;
        }
        __syncthreads();
        if (failed) break;
        float *Ahi = (float *)st, *Alo = (float *)(st + kOpBytes);
        float *Bhi = (float *)(st + 2 * kOpBytes), *Blo = (float *)(st + 3 * kOpBytes);
        if (VEC) store_chunk_vec(cur, Ahi, Alo, Bhi, Blo, warp, lane);
        else stage_scalar(A, lda, B, ldb, M, N, K, tm, tn, kc * kTK, Ahi, Alo, Bhi, Blo, tid);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_hi = smem_u32(Ahi), a_lo = smem_u32(Alo);
            const uint32_t b_hi = smem_u32(Bhi), b_lo = smem_u32(Blo);
#pragma unroll
            for (int s = 0; s < kTK / 8; ++s) {
                const uint32_t ko = s * 2 * lbo;               // 8 tf32 = two 16-byte core columns
                const int first = (kc == 0 && s == 0) ? 0 : 1;
                mma_tf32(tmem, smem_desc(a_hi + ko, lbo, sbo), smem_desc(b_hi + ko, lbo, sbo), idesc, first);
                mma_tf32(tmem, smem_desc(a_hi + ko, lbo, sbo), smem_desc(b_lo + ko, lbo, sbo), idesc, 1);
                mma_tf32(tmem, smem_desc(a_lo + ko, lbo, sbo), smem_desc(b_hi + ko, lbo, sbo), idesc, 1);
            }
            mma_commit(smem_u32(&mbar[buf]));
        }
        issued = kc;
        // two chunks' loads are in flight while the tensor cores work on this one
        if (VEC) {
            cur = nxt;
            if (kc + 2 < nch) load_chunk_vec(nxt, A, lda, B, ldb, M, N, K, tm, tn, (kc + 2) * kTK, warp, lane);
        }
    }
    // all MMAs of this tile are complete once the last commit has landed
    if (issued >= 0 && tid == 0) {
        const int last = issued & 1;
        const uint32_t par = (issued >> 1) & 1;
        bool ok = mbar_wait(smem_u32(&mbar[last]), par);
        if (!ok) {
            failed = 1;
            mbar_wait(smem_u32(&mbar[last]), par);          // bounded second wait for in-flight MMAs
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!failed && issued == nch - 1 && nch > 0) epilogue<VEC>(tmem, C, ldc, M, N, tm, tn, warp, lane);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    if (tid == 0 && failed) atomicAdd(err, 1);
}

// ---------------------------------------------------------------------------
// Pipelined form for large batches of Schur updates (the pivot-free recursive
// LU of the disks).  Each operand is split into hi/lo TF32 ONCE, into tiles of
// 128 rows x 32 K that are stored in the exact shared-memory layout the MMAs
// read (the canonical no-swizzle K-major layout above: two 16 KB blocks, hi
// then lo, contiguous).  The GEMM kernel is persistent (one CTA per SM) and
// warp-specialised:
//   warp 0    one lane streams each K chunk's A and B tile pairs (2 x 32 KB)
//             into a 3-stage ring with cp.async.bulk, completion counted by
//             the stage's mbarrier (expect_tx);
//   warp 1    allocates 256 TMEM columns (two 128 x 128 FP32 accumulators) and
//             one lane issues 4 k-steps x 3 tcgen05.mma.kind::tf32 per chunk,
//             releasing the stage with tcgen05.commit and, after a tile's last
//             chunk, handing the accumulator to the epilogue;
//   warps 2-5 read the accumulator with tcgen05.ld (warp w owns TMEM lanes
//             32 (w mod 4) ..) and write C -= acc (or C = acc), then free it, so
//             one tile's epilogue overlaps the next tile's MMAs.
// Every mbarrier wait is bounded; a timeout records an error, the roles stop
// issuing, the MMA lane waits (bounded) for its own MMAs, and TMEM is freed.
// ---------------------------------------------------------------------------
static constexpr int kPipeRows = 128, kPipeK = 32;
static constexpr int kBlkFloats = kPipeRows * kPipeK;         // one hi or lo block: 16 KB
static constexpr int kPairFloats = 2 * kBlkFloats;             // hi + lo: 32 KB
static constexpr int kPipeStages = 3;
static constexpr int kPipeStageBytes = 2 * kPairFloats * 4;    // A pair + B pair: 64 KB
static constexpr int kPipeSmem = kPipeStages * kPipeStageBytes;
static constexpr int kPipeSmemAll = kPipeSmem + kPipeRows * 68 * 4;      // + the epilogue's staging block
static constexpr int kPipeThreads = 192;
static constexpr int kPipeTmemCols = 256;

// X (R x K, row stride ld; TRANS: X is K x R) -> tiles [b][rt][kc][hi, lo][128 x 32 canonical].
// Bandwidth-bound: every thread issues its four 16-byte loads before any shared-memory store
// (scalar loads, with bounds, for a misaligned source or a ragged edge).
template <bool TRANS>
__global__ void __launch_bounds__(256) k_split_tiles(const float *X, long sX, int ld, int R, int K, int rtiles,
                                                     int nkc, float *out, long sOut) {
    __shared__ float t[kPipeRows][kPipeK + 1];
    const int kc = blockIdx.x, rt = blockIdx.y, b = blockIdx.z, tid = threadIdx.x;
    const float *src = X + b * sX;
    const int r0 = rt * kPipeRows, k0 = kc * kPipeK;
    const bool al = ((uintptr_t)src & 15) == 0 && (ld & 3) == 0;
    float4 v[4];
    // float4 group q = tid + 256 i: non-TRANS row r = q >> 3, k = 4 (q & 7); TRANS k = q >> 5, r = 4 (q & 31)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int q = tid + 256 * i;
        int r, k;
        if (TRANS) {
            k = q >> 5;
            r = 4 * (q & 31);
        } else {
            r = q >> 3;
            k = 4 * (q & 7);
        }
        const int gr = r0 + r, gk = k0 + k;
        if (TRANS) {
            const float *p = src + (long)gk * ld + gr;
            if (al && gk < K && gr + 3 < R) {
                v[i] = __ldg(reinterpret_cast<const float4 *>(p));
            } else {
                v[i].x = (gk < K && gr < R) ? p[0] : 0.f;
                v[i].y = (gk < K && gr + 1 < R) ? p[1] : 0.f;
                v[i].z = (gk < K && gr + 2 < R) ? p[2] : 0.f;
                v[i].w = (gk < K && gr + 3 < R) ? p[3] : 0.f;
            }
        } else {
            const float *p = src + (long)gr * ld + gk;
            if (al && gr < R && gk + 3 < K) {
                v[i] = __ldg(reinterpret_cast<const float4 *>(p));
            } else {
                v[i].x = (gr < R && gk < K) ? p[0] : 0.f;
                v[i].y = (gr < R && gk + 1 < K) ? p[1] : 0.f;
                v[i].z = (gr < R && gk + 2 < K) ? p[2] : 0.f;
                v[i].w = (gr < R && gk + 3 < K) ? p[3] : 0.f;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int q = tid + 256 * i;
        if (TRANS) {
            const int k = q >> 5, r = 4 * (q & 31);
            t[r][k] = v[i].x;
            t[r + 1][k] = v[i].y;
            t[r + 2][k] = v[i].z;
            t[r + 3][k] = v[i].w;
        } else {
            const int r = q >> 3, k = 4 * (q & 7);
            t[r][k] = v[i].x;
            t[r][k + 1] = v[i].y;
            t[r][k + 2] = v[i].z;
            t[r][k + 3] = v[i].w;
        }
    }
    __syncthreads();
    float *hi = out + b * sOut + ((long)rt * nkc + kc) * kPairFloats;
    float *lo = hi + kBlkFloats;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int e = tid + 256 * i;
        const int k4 = e >> 7, r = e & 127;            // a warp writes 32 rows of one core column: 512 B
        float4 w = make_float4(t[r][4 * k4], t[r][4 * k4 + 1], t[r][4 * k4 + 2], t[r][4 * k4 + 3]);
        const float4 h = split_hi(w);
        const int off = k4 * (kPipeRows * 4) + (r >> 3) * 32 + (r & 7) * 4;
        *reinterpret_cast<float4 *>(hi + off) = h;
        *reinterpret_cast<float4 *>(lo + off) = split_lo(w, h);
    }
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// epilogue staging row stride of both GEMM forms (64 columns + 4: consecutive rows shift banks)
static constexpr int kStgLd = 68;

struct TcPipeArgs {
    int M, N, mtiles, ntiles, nkc, batch;
    const float *Ap;
    long sAp;                 // floats per matrix of A's tiles
    const float *Bp;
    long sBp;
    float *C;
    long sC;
    int ldc;
    int *err;
};

__device__ __forceinline__ void pipe_tile(long t, const TcPipeArgs &g, int &b, int &mt, int &nt) {
    const long per = (long)g.mtiles * g.ntiles;
    b = (int)(t / per);
    const int rem = (int)(t - (long)b * per);
    mt = rem / g.ntiles;
    nt = rem - mt * g.ntiles;
}

template <bool SUB>
__global__ void __launch_bounds__(kPipeThreads, 1) k_tc_gemm_pipe(TcPipeArgs g) {
    extern __shared__ __align__(1024) unsigned char psm[];
    __shared__ __align__(8) uint64_t full[kPipeStages], empty[kPipeStages], accf[2], acce[2], fin;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int failed;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long total = (long)g.batch * g.mtiles * g.ntiles;
    if (threadIdx.x == 0) {
        failed = 0;
        for (int s = 0; s < kPipeStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&accf[a]), 1);
            mbar_init(smem_u32(&acce[a]), 4);         // one arrival per epilogue warp
        }
        mbar_init(smem_u32(&fin), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kPipeTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t base = smem_u32(psm);
    if (warp == 0) {
        if (lane == 0) {                                   // producer
            long it = 0;
            for (long t = blockIdx.x; t < total && !failed; t += gridDim.x) {
                int b, mt, nt;
                pipe_tile(t, g, b, mt, nt);
                const float *a = g.Ap + b * g.sAp + (long)mt * g.nkc * kPairFloats;
                const float *bb = g.Bp + b * g.sBp + (long)nt * g.nkc * kPairFloats;
                for (int kc = 0; kc < g.nkc; ++kc, ++it) {
                    const int s = (int)(it % kPipeStages);
                    const long r = it / kPipeStages;
                    if (r > 0 && !mbar_wait_sleep(smem_u32(&empty[s]), (uint32_t)((r - 1) & 1))) {
                        failed = 1;
                        break;
                    }
                    if (failed) break;
                    const uint32_t st = base + s * kPipeStageBytes;
                    mbar_expect_tx(smem_u32(&full[s]), kPipeStageBytes);
                    bulk_g2s(st, a + (long)kc * kPairFloats, kPairFloats * 4, smem_u32(&full[s]));
                    bulk_g2s(st + kPairFloats * 4, bb + (long)kc * kPairFloats, kPairFloats * 4, smem_u32(&full[s]));
                }
            }
            // copies still in flight land before the CTA exits: wait (bounded) for the last phase of
            // each stage that was filled
            const long n_it = it;
            for (long q = n_it - kPipeStages < 0 ? 0 : n_it - kPipeStages; q < n_it; ++q)
                mbar_wait_sleep(smem_u32(&full[q % kPipeStages]), (uint32_t)((q / kPipeStages) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {                                   // MMA issuer
            const uint32_t idesc = idesc_tf32(kPipeRows, kPipeRows);
            const uint32_t lbo = kPipeRows * 16, sbo = 128;
            long it = 0;
            int tc = 0;
            bool issued = false;
            for (long t = blockIdx.x; t < total && !failed; t += gridDim.x, ++tc) {
                const int acc = tc & 1, use = tc >> 1;
                if (use > 0 && !mbar_wait_sleep(smem_u32(&acce[acc]), (uint32_t)((use - 1) & 1))) {
                    failed = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(acc * kPipeRows);
                bool ok = true;
                for (int kc = 0; kc < g.nkc; ++kc, ++it) {
                    const int s = (int)(it % kPipeStages);
                    if (!mbar_wait_sleep(smem_u32(&full[s]), (uint32_t)((it / kPipeStages) & 1))) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a_hi = base + s * kPipeStageBytes, a_lo = a_hi + kBlkFloats * 4;
                    const uint32_t b_hi = a_hi + kPairFloats * 4, b_lo = b_hi + kBlkFloats * 4;
#pragma unroll
                    for (int k8 = 0; k8 < kPipeK / 8; ++k8) {
                        const uint32_t ko = k8 * 2 * lbo;
                        mma_tf32(d, smem_desc(a_hi + ko, lbo, sbo), smem_desc(b_hi + ko, lbo, sbo), idesc,
                                 (kc | k8) ? 1 : 0);
                        mma_tf32(d, smem_desc(a_hi + ko, lbo, sbo), smem_desc(b_lo + ko, lbo, sbo), idesc, 1);
                        mma_tf32(d, smem_desc(a_lo + ko, lbo, sbo), smem_desc(b_hi + ko, lbo, sbo), idesc, 1);
                    }
                    issued = true;
                    mma_commit(smem_u32(&empty[s]));
                }
                if (!ok) {
                    failed = 1;
                    break;
                }
                mma_commit(smem_u32(&accf[acc]));
            }
            // every MMA this lane issued is complete before TMEM is freed
            if (issued) {
                mma_commit(smem_u32(&fin));
                if (!mbar_wait_sleep(smem_u32(&fin), 0)) failed = 1;
            }
        }
    } else {                                               // epilogue: warps 2..5
        // warp q owns TMEM lanes 32 q .. = tile rows 32 q ..; C moves through a shared staging block
        // of those 32 rows x 64 columns as whole-row coalesced accesses, a slab's C loads in flight
        // together (the first slab's before the accumulator is ready), as in the fused form
        const int q = warp & 3;
        float *stg = reinterpret_cast<float *>(psm + kPipeSmem) + (size_t)(q * 32) * kStgLd;
        int tc = 0;
        const bool vec = ((uintptr_t)g.C & 15) == 0 && (g.ldc & 3) == 0 && (g.sC & 3) == 0;
        const int hr = lane >> 4, hc = 4 * (lane & 15);
        float4 cl[16];
        for (long t = blockIdx.x; t < total; t += gridDim.x, ++tc) {
            const int acc = tc & 1, use = tc >> 1;
            int b, mt, nt;
            pipe_tile(t, g, b, mt, nt);
            const int rbase = mt * kPipeRows + q * 32;
            float *cbase = g.C + b * g.sC;
            auto cload = [&](int colg) {
                const int ncol = g.N - colg;
#pragma unroll
                for (int it = 0; it < 16; ++it) {
                    const int grow = rbase + 2 * it + hr;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (grow < g.M && hc < ncol) {
                        const float *cp = cbase + (long)grow * g.ldc + colg + hc;
                        if (vec && hc + 4 <= ncol) {
                            v = *reinterpret_cast<const float4 *>(cp);
                        } else {
                            v.x = cp[0];
                            if (hc + 1 < ncol) v.y = cp[1];
                            if (hc + 2 < ncol) v.z = cp[2];
                            if (hc + 3 < ncol) v.w = cp[3];
                        }
                    }
                    cl[it] = v;
                }
            };
            if (SUB) cload(nt * kPipeRows);
            // lane 0 waits for the accumulator; the warp goes on (or leaves) together
            int ok = 1;
            if (lane == 0) ok = mbar_wait_sleep(smem_u32(&accf[acc]), (uint32_t)(use & 1)) ? 1 : 0;
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                failed = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
            for (int sl = 0; sl < kPipeRows / 64; ++sl) {
                const int colg = nt * kPipeRows + sl * 64, ncol = g.N - colg;
                if (SUB) {
#pragma unroll
                    for (int it = 0; it < 16; ++it)
                        *reinterpret_cast<float4 *>(stg + (2 * it + hr) * kStgLd + hc) = cl[it];
                    __syncwarp();
                    if (sl + 1 < kPipeRows / 64) cload(colg + 64);
                }
                uint32_t v0[32], v1[32];
                const uint32_t taddr = tmem + (uint32_t)(acc * kPipeRows + sl * 64) + ((uint32_t)(q * 32) << 16);
                tmem_ld32(taddr, v0);
                tmem_ld32(taddr + 32, v1);
                float *sr = stg + lane * kStgLd;
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const uint32_t *vv = e < 8 ? v0 : v1;
                    const int k = 4 * (e & 7);
                    float4 o = make_float4(__uint_as_float(vv[k]), __uint_as_float(vv[k + 1]),
                                           __uint_as_float(vv[k + 2]), __uint_as_float(vv[k + 3]));
                    if (SUB) {
                        const float4 c = *reinterpret_cast<const float4 *>(sr + 4 * e);
                        o = make_float4(c.x - o.x, c.y - o.y, c.z - o.z, c.w - o.w);
                    }
                    *reinterpret_cast<float4 *>(sr + 4 * e) = o;
                }
                __syncwarp();
#pragma unroll 4
                for (int it = 0; it < 16; ++it) {
                    const int rr = 2 * it + hr, grow = rbase + rr;
                    if (grow < g.M && hc < ncol) {
                        const float4 v = *reinterpret_cast<const float4 *>(stg + rr * kStgLd + hc);
                        float *cp = cbase + (long)grow * g.ldc + colg + hc;
                        if (vec && hc + 4 <= ncol) {
                            *reinterpret_cast<float4 *>(cp) = v;
                        } else {
                            cp[0] = v.x;
                            if (hc + 1 < ncol) cp[1] = v.y;
                            if (hc + 2 < ncol) cp[2] = v.z;
                            if (hc + 3 < ncol) cp[3] = v.w;
                        }
                    }
                }
                __syncwarp();
            }
            // the warp's TMEM reads are done: one arrival per warp (128 single-thread arrivals on one
            // mbarrier serialise, and the MMA lane waits on this before reusing the accumulator)
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acce[acc]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kPipeTmemCols)
                     : "memory");
    if (threadIdx.x == 0 && failed) atomicAdd(g.err, 1);
}

// ---------------------------------------------------------------------------
// Fused form (the recursive disk LU's GEMMs): the operands are read as FP32
// from their matrices and split into hi/lo TF32 inside the GEMM kernel, so no
// split copy of either operand passes through device memory.  Persistent
// (one CTA per SM), warp-specialised, tiles of 128 rows x TN columns
// (TN = 64, 128 or 256 by N), K in chunks of 16 through a 4-stage ring:
//   warps 0-7   converters: each K chunk of the A tile (128 x 16, row-major
//               source: 16-byte loads of 4 k) and of the B tile (16 x TN,
//               row-major source: each thread loads a 4 k x TN/64 block, one
//               float per row of 32 consecutive columns, and writes it
//               transposed as 16-byte rows) is loaded a few chunks ahead
//               into registers, split, and stored in the canonical no-swizzle
//               K-major layout (LBO = rows x 16 B, SBO = 128 B; the 16-byte
//               unit of operand row r is r, so both stores are free of bank
//               conflicts); each warp makes its stores visible to the tensor
//               cores (fence.proxy.async) and arrives on the stage's mbarrier;
//               warp 0 also allocates 2 TN TMEM columns (two accumulators),
//               and its lane 0, once all converters have stored a chunk,
//               issues 2 k-steps x 3 tcgen05.mma.kind::tf32 (M = 128, N = TN)
//               for it and releases the stage with tcgen05.commit (12 warps:
//               three per scheduler, so up to 168 registers per thread);
//   warps 8-11  epilogue: C -= acc (or C = acc) from TMEM (warp w reads lanes
//               32 (w mod 4) ..), each 32-column group of C loaded one group
//               ahead (the first before the accumulator is ready), overlapping
//               the next tile's MMAs.
// C may be one of the operands only when every tile that reads the aliased part
// also writes it: A with N <= TN, or B with M <= 128.
// Every mbarrier wait is bounded, as in the pipelined form.
// ---------------------------------------------------------------------------
static constexpr int kFzK = 16;
static constexpr int kFzStgLd = kStgLd;
static constexpr int kFzConvWarps = 8;
static constexpr int kFzThreads = (kFzConvWarps + 4) * 32;

// ring stages (4; 3 at TN = 256 so that the epilogue's staging fits beside them; 2 at TN = 64,
// where two CTAs share an SM) and shared bytes
__host__ __device__ constexpr int fz_stages(int TN) { return TN >= 256 ? 3 : 2; }
// CTAs per SM: the 64- and 128-wide tiles are bound by the converters' issue, so two CTAs (24 warps,
// at most 85 registers each; TMEM 2 x 2 TN columns) hide each other's stalls
__host__ __device__ constexpr int fz_ctas(int TN) { return TN >= 256 ? 1 : 2; }
__host__ __device__ constexpr int fz_smem(int TN) {
    return fz_stages(TN) * 2 * (128 + TN) * kFzK * 4 + 128 * kFzStgLd * 4;
}
// chunks in flight ahead of the one being stored (the register ring holds FZ_DEPTH + 1 chunks)
__host__ __device__ constexpr int fz_depth(int TN) { return TN >= 256 ? 2 : (TN >= 128 ? 2 : 3); }

struct FzArgs {
    int M, N, K, mtiles, ntiles, nkc, batch;
    const float *A;
    long sA;
    int lda;
    const float *B;
    long sB;
    int ldb;
    float *C;
    long sC;
    int ldc;
    int *err;
};

// where the converters' loads are: tile t (b, mt, nt) and chunk kc
struct FzCursor {
    long t;
    int kc;
    const float *a, *b;   // this tile's A rows (row mt 128) and B columns (column nt TN)
    int rows, cols;       // valid rows of the A tile, valid columns of the B tile
};

template <int TN>
__device__ __forceinline__ void fz_seek(FzCursor &c, const FzArgs &g) {
    const long per = (long)g.mtiles * g.ntiles;
    const int b = (int)(c.t / per);
    const int rem = (int)(c.t - (long)b * per);
    const int mt = rem / g.ntiles, nt = rem - mt * g.ntiles;
    c.a = g.A + b * g.sA + (long)mt * 128 * g.lda;
    c.b = g.B + b * g.sB + (long)nt * TN;
    c.rows = g.M - mt * 128;
    c.cols = g.N - nt * TN;
}

template <int TN>
__device__ __forceinline__ void fz_advance(FzCursor &c, const FzArgs &g) {
    if (++c.kc == g.nkc) {
        c.kc = 0;
        c.t += gridDim.x;
        if (c.t < (long)g.batch * g.mtiles * g.ntiles) fz_seek<TN>(c, g);
    }
}

// one K chunk: A 2 x float4 (rows 8 (8 i + w) + (l & 7), k = 4 (l >> 3) ..), B V x 4 floats
// (k = 4 (w >> 1) + kk, column l + 32 ((w & 1) + 2 e))
template <int TN, bool VEC>
__device__ __forceinline__ void fz_load(float4 (&a)[2], float (&bv)[TN / 64][4], const FzCursor &c,
                                        const FzArgs &g, int w, int l) {
    constexpr int V = TN / 64;
    const int k0 = c.kc * kFzK;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int row = 8 * (8 * i + w) + (l & 7), k = k0 + 4 * (l >> 3);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < c.rows) {
            const float *p = c.a + (long)row * g.lda + k;
            if (VEC && k + 3 < g.K) {
                v = *reinterpret_cast<const float4 *>(p);
            } else {
                if (k < g.K) v.x = p[0];
                if (k + 1 < g.K) v.y = p[1];
                if (k + 2 < g.K) v.z = p[2];
                if (k + 3 < g.K) v.w = p[3];
            }
        }
        a[i] = v;
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const int k = k0 + 4 * (w >> 1) + kk;
        const float *p = c.b + (long)k * g.ldb;
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const int col = l + 32 * ((w & 1) + 2 * e);
            bv[e][kk] = (k < g.K && col < c.cols) ? p[col] : 0.f;
        }
    }
}

template <int TN>
__device__ __forceinline__ void fz_store(const float4 (&a)[2], const float (&bv)[TN / 64][4], float *st, int w,
                                         int l) {
    constexpr int V = TN / 64, AF = 128 * kFzK, BF = TN * kFzK;
    float *ahi = st, *alo = st + AF, *bhi = st + 2 * AF, *blo = st + 2 * AF + BF;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int row = 8 * (8 * i + w) + (l & 7);
        const int off = (l >> 3) * (128 * 4) + row * 4;
        const float4 h = split_hi(a[i]);
        *reinterpret_cast<float4 *>(ahi + off) = h;
        *reinterpret_cast<float4 *>(alo + off) = split_lo(a[i], h);
    }
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const int col = l + 32 * ((w & 1) + 2 * e);
        const int off = (w >> 1) * (TN * 4) + col * 4;
        const float4 v = make_float4(bv[e][0], bv[e][1], bv[e][2], bv[e][3]);
        const float4 h = split_hi(v);
        *reinterpret_cast<float4 *>(bhi + off) = h;
        *reinterpret_cast<float4 *>(blo + off) = split_lo(v, h);
    }
}


template <bool SUB, int TN, bool VEC>
__global__ void __launch_bounds__(kFzThreads, fz_ctas(TN)) k_tc_gemm_fused(FzArgs g) {
    constexpr int V = TN / 64, D = fz_depth(TN), R = D + 1, NS = fz_stages(TN);
    constexpr int AF = 128 * kFzK, BF = TN * kFzK, SF = 2 * (AF + BF);
    extern __shared__ __align__(1024) unsigned char zsm[];
    __shared__ __align__(8) uint64_t full[NS], empty[NS], accf[2], acce[2], fin;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int failed;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long total = (long)g.batch * g.mtiles * g.ntiles;
    if (threadIdx.x == 0) {
        failed = 0;
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&full[s]), kFzConvWarps);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&accf[a]), 1);
            mbar_init(smem_u32(&acce[a]), 4);         // one arrival per epilogue warp
        }
        mbar_init(smem_u32(&fin), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(2 * TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    float *ring = reinterpret_cast<float *>(zsm);
    const uint32_t base = smem_u32(zsm);
    if (warp < kFzConvWarps) {                             // converters (+ the MMA lane)
        const bool mma_lane = warp == 0 && lane == 0;
        const uint32_t idesc = idesc_tf32(128, TN);
        const uint32_t lbo_a = 128 * 16, lbo_b = TN * 16, sbo = 128;
        int m_kc = 0, m_tc = 0;                            // the MMA lane's chunk and tile count
        bool issued = false;
        const long mine = total > blockIdx.x ? (total - 1 - blockIdx.x) / gridDim.x + 1 : 0;
        const long n_items = mine * g.nkc;
        FzCursor cur{(long)blockIdx.x, 0, nullptr, nullptr, 0, 0};
        if (n_items > 0) fz_seek<TN>(cur, g);
        float4 ra[R][2];
        float rb[R][V][4];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            if (j < n_items) {
                fz_load<TN, VEC>(ra[j], rb[j], cur, g, warp, lane);
                fz_advance<TN>(cur, g);
            }
        }
        bool stop = false;
        for (long it0 = 0; it0 < n_items && !stop; it0 += R) {
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const long it = it0 + j;
                if (it >= n_items) break;
                if (it + D < n_items) {
                    fz_load<TN, VEC>(ra[(j + D) % R], rb[(j + D) % R], cur, g, warp, lane);
                    fz_advance<TN>(cur, g);
                }
                const int s = (int)(it % NS);
                const long r = it / NS;
                // lane 0 waits for the stage to be free; the warp leaves together on a failure
                int go = 1;
                if (lane == 0) {
                    if (failed) go = 0;
                    else if (r > 0 && !mbar_wait_sleep(smem_u32(&empty[s]), (uint32_t)((r - 1) & 1))) {
                        failed = 1;
                        go = 0;
                    }
                }
                if (!__shfl_sync(0xffffffffu, go, 0)) {
                    stop = true;
                    break;
                }
                fz_store<TN>(ra[j], rb[j], ring + (size_t)s * SF, warp, lane);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&full[s]));
                if (mma_lane) {
                    // chunk m_kc of this CTA's tile m_tc, once every converter has stored it
                    const int acc = m_tc & 1, use = m_tc >> 1;
                    bool ok = true;
                    if (m_kc == 0 && use > 0) ok = mbar_wait_sleep(smem_u32(&acce[acc]), (uint32_t)((use - 1) & 1));
                    if (ok) ok = mbar_wait_sleep(smem_u32(&full[s]), (uint32_t)(r & 1));
                    if (!ok) {
                        failed = 1;
                    } else {
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t d = tmem + (uint32_t)(acc * TN);
                        const uint32_t a_hi = base + (uint32_t)(s * SF * 4), a_lo = a_hi + AF * 4;
                        const uint32_t b_hi = a_hi + 2 * AF * 4, b_lo = b_hi + BF * 4;
#pragma unroll
                        for (int k8 = 0; k8 < kFzK / 8; ++k8) {
                            const uint32_t koa = k8 * 2 * lbo_a, kob = k8 * 2 * lbo_b;
                            mma_tf32(d, smem_desc(a_hi + koa, lbo_a, sbo), smem_desc(b_hi + kob, lbo_b, sbo), idesc,
                                     (m_kc | k8) ? 1 : 0);
                            mma_tf32(d, smem_desc(a_hi + koa, lbo_a, sbo), smem_desc(b_lo + kob, lbo_b, sbo), idesc,
                                     1);
                            mma_tf32(d, smem_desc(a_lo + koa, lbo_a, sbo), smem_desc(b_hi + kob, lbo_b, sbo), idesc,
                                     1);
                        }
                        issued = true;
                        mma_commit(smem_u32(&empty[s]));
                        if (++m_kc == g.nkc) {
                            mma_commit(smem_u32(&accf[acc]));
                            m_kc = 0;
                            ++m_tc;
                        }
                    }
                }
            }
        }
        // every MMA this lane issued is complete before TMEM is freed
        if (mma_lane && issued) {
            mma_commit(smem_u32(&fin));
            if (!mbar_wait_sleep(smem_u32(&fin), 0)) failed = 1;
        }
    } else {                                               // epilogue: warps 8..11
        // warp q owns TMEM lanes 32 q .. = tile rows 32 q ..; C moves through a shared staging block
        // of those 32 rows x 64 columns as whole-row coalesced accesses (a thread-per-row access of C
        // would touch 32 rows, 32 cache lines, per instruction).  When subtracting, a slab's 16 loads
        // per thread are in flight together: the first slab's before the accumulator is ready, the
        // next slab's while this one is combined and stored.
        const int q = warp & 3;
        float *stg = ring + (size_t)NS * SF + (size_t)(q * 32) * kFzStgLd;
        int tc = 0;
        const bool vec = ((uintptr_t)g.C & 15) == 0 && (g.ldc & 3) == 0 && (g.sC & 3) == 0;
        const int hr = lane >> 4, hc = 4 * (lane & 15);      // coalesced form: 2 rows x 16 float4 per pass
        float4 cl[16];
        for (long t = blockIdx.x; t < total; t += gridDim.x, ++tc) {
            const int acc = tc & 1, use = tc >> 1;
            const long per = (long)g.mtiles * g.ntiles;
            const int b = (int)(t / per);
            const int rem = (int)(t - (long)b * per);
            const int mt = rem / g.ntiles, nt = rem - mt * g.ntiles;
            const int rbase = mt * 128 + q * 32;
            float *cbase = g.C + b * g.sC;
            // the warp's 32 rows x 64 columns of C from column colg, two rows per pass
            auto cload = [&](int colg) {
                const int ncol = g.N - colg;
#pragma unroll
                for (int it = 0; it < 16; ++it) {
                    const int grow = rbase + 2 * it + hr;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (grow < g.M && hc < ncol) {
                        const float *cp = cbase + (long)grow * g.ldc + colg + hc;
                        if (vec && hc + 4 <= ncol) {
                            v = *reinterpret_cast<const float4 *>(cp);
                        } else {
                            v.x = cp[0];
                            if (hc + 1 < ncol) v.y = cp[1];
                            if (hc + 2 < ncol) v.z = cp[2];
                            if (hc + 3 < ncol) v.w = cp[3];
                        }
                    }
                    cl[it] = v;
                }
            };
            // C's slab at column colg straight into the staging rows by asynchronous 16-byte copies (no
            // registers held; partial edges filled directly), for the tiles that run two CTAs per SM
            auto cload_async = [&](int colg) {
                const int ncol = g.N - colg;
#pragma unroll
                for (int it = 0; it < 16; ++it) {
                    const int rr = 2 * it + hr, grow = rbase + rr;
                    float *dst = stg + rr * kFzStgLd + hc;
                    const float *cp = cbase + (long)grow * g.ldc + colg + hc;
                    if (grow < g.M && vec && hc + 4 <= ncol) {
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(cp)
                                     : "memory");
                    } else {
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (grow < g.M && hc < ncol) {
                            v.x = cp[0];
                            if (hc + 1 < ncol) v.y = cp[1];
                            if (hc + 2 < ncol) v.z = cp[2];
                            if (hc + 3 < ncol) v.w = cp[3];
                        }
                        *reinterpret_cast<float4 *>(dst) = v;
                    }
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
            };
            constexpr bool kAsyncC = TN <= 128;
            if (SUB) {
                if constexpr (kAsyncC) cload_async(nt * TN);
                else cload(nt * TN);
            }
            // lane 0 waits for the accumulator; the warp goes on (or leaves) together
            int ok = 1;
            if (lane == 0) ok = (!failed && mbar_wait_sleep(smem_u32(&accf[acc]), (uint32_t)(use & 1))) ? 1 : 0;
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                failed = 1;
                if (SUB && kAsyncC) asm volatile("cp.async.wait_group 0;" ::: "memory");
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
            for (int sl = 0; sl < TN / 64; ++sl) {
                const int colg = nt * TN + sl * 64;          // first column of this slab in C
                const int ncol = g.N - colg;                 // valid columns from colg (may exceed 64)
                if (SUB) {                                   // C's slab into the staging rows
                    if constexpr (kAsyncC) {
                        if (sl > 0) cload_async(colg);       // the staging rows are free again
                        asm volatile("cp.async.wait_group 0;" ::: "memory");
                    } else {
#pragma unroll
                        for (int it = 0; it < 16; ++it)
                            *reinterpret_cast<float4 *>(stg + (2 * it + hr) * kFzStgLd + hc) = cl[it];
                    }
                    __syncwarp();
                    if (!kAsyncC && sl + 1 < TN / 64) cload(colg + 64);
                }
                // this thread's row: the accumulator's 64 columns into the staging row, 16 at a time
                const uint32_t taddr = tmem + (uint32_t)(acc * TN + sl * 64) + ((uint32_t)(q * 32) << 16);
                float *sr = stg + lane * kFzStgLd;
#pragma unroll
                for (int p4 = 0; p4 < 4; ++p4) {
                    uint32_t v[16];
                    tmem_ld16(taddr + 16 * p4, v);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        float4 o = make_float4(__uint_as_float(v[4 * e]), __uint_as_float(v[4 * e + 1]),
                                               __uint_as_float(v[4 * e + 2]), __uint_as_float(v[4 * e + 3]));
                        float *d = sr + 16 * p4 + 4 * e;
                        if (SUB) {
                            const float4 c = *reinterpret_cast<const float4 *>(d);
                            o = make_float4(c.x - o.x, c.y - o.y, c.z - o.z, c.w - o.w);
                        }
                        *reinterpret_cast<float4 *>(d) = o;
                    }
                }
                __syncwarp();
                // the staging rows back to C, coalesced
#pragma unroll 4
                for (int it = 0; it < 16; ++it) {
                    const int rr = 2 * it + hr, grow = rbase + rr;
                    if (grow < g.M && hc < ncol) {
                        const float4 v = *reinterpret_cast<const float4 *>(stg + rr * kFzStgLd + hc);
                        float *cp = cbase + (long)grow * g.ldc + colg + hc;
                        if (vec && hc + 4 <= ncol) {
                            *reinterpret_cast<float4 *>(cp) = v;
                        } else {
                            cp[0] = v.x;
                            if (hc + 1 < ncol) cp[1] = v.y;
                            if (hc + 2 < ncol) cp[2] = v.z;
                            if (hc + 3 < ncol) cp[3] = v.w;
                        }
                    }
                }
                __syncwarp();
            }
            // the warp's TMEM reads are done: one arrival per warp (128 single-thread arrivals on one
            // mbarrier serialise, and the MMA lane waits on this before reusing the accumulator)
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acce[acc]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TN) : "memory");
    if (threadIdx.x == 0 && failed) atomicAdd(g.err, 1);
}

static int g_sms[64] = {0};

static int sm_count() {
    int dev = 0;
    PDD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(PDD_EINVAL, "device ordinal out of range");
    if (!g_sms[dev]) PDD_CUDA(cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev));
    return g_sms[dev];
}

size_t tc_tile_floats(int rows, int K) { return (size_t)cdiv(rows, kPipeRows) * cdiv(K, kPipeK) * kPairFloats; }

static int cur_device() {
    int dev = 0;
    PDD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(PDD_EINVAL, "device ordinal out of range");
    return dev;
}

// C_b (-)= A_b B_b through pre-split tiles (any transposition, any aliasing of C in the C = A B
// form).  scratch: at least chunk * (tc_tile_floats(M, K) + tc_tile_floats(N, K)) floats; the
// batch is processed in chunks that fit.
static void tc_gemm_presplit(int batch, int M, int N, int K, const float *A, long sA, int lda, bool transA,
                             const float *B, long sB, int ldb, bool transB, float *C, long sC, int ldc, bool sub,
                             float *scratch, size_t scratch_floats, int *err, cudaStream_t st,
                             std::vector<cudaEvent_t> *kev) {       // event pairs around the GEMM kernels
    static bool attr[64] = {false};
    const int dev = cur_device();
    if (!attr[dev]) {
        PDD_CUDA(cudaFuncSetAttribute(k_tc_gemm_pipe<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPipeSmemAll));
        PDD_CUDA(cudaFuncSetAttribute(k_tc_gemm_pipe<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPipeSmemAll));
        attr[dev] = true;
    }
    const int mt = cdiv(M, kPipeRows), ntl = cdiv(N, kPipeRows), nkc = cdiv(K, kPipeK);
    const size_t fa = tc_tile_floats(M, K), fb = tc_tile_floats(N, K);
    const int chunk = (int)std::min<size_t>((size_t)batch, scratch_floats / (fa + fb));
    if (chunk < 1) fail(PDD_EINVAL, "tensor-core GEMM scratch smaller than one matrix's tiles");
    if (mt > 65535 || ntl > 65535 || chunk > 65535) fail(PDD_EINVAL, "GEMM too large for the split grid");
    const int sms = sm_count();
    for (int b0 = 0; b0 < batch; b0 += chunk) {
        const int nb = std::min(chunk, batch - b0);
        float *Ap = scratch, *Bp = scratch + (size_t)nb * fa;
        // A tiles: rows of C (M) x K; B tiles: columns of C (N) x K
        if (transA)
            PDD_LAUNCH(k_split_tiles<true>, dim3(nkc, mt, nb), 256, 0, st, A + b0 * sA, sA, lda, M, K, mt, nkc, Ap, (long)fa);
        else
            PDD_LAUNCH(k_split_tiles<false>, dim3(nkc, mt, nb), 256, 0, st, A + b0 * sA, sA, lda, M, K, mt, nkc, Ap, (long)fa);
        if (transB)
            PDD_LAUNCH(k_split_tiles<false>, dim3(nkc, ntl, nb), 256, 0, st, B + b0 * sB, sB, ldb, N, K, ntl, nkc, Bp, (long)fb);
        else
            PDD_LAUNCH(k_split_tiles<true>, dim3(nkc, ntl, nb), 256, 0, st, B + b0 * sB, sB, ldb, N, K, ntl, nkc, Bp, (long)fb);
        const TcPipeArgs g{M, N, mt, ntl, nkc, nb, Ap, (long)fa, Bp, (long)fb, C + b0 * sC, sC, ldc, err};
        const long tiles = (long)nb * mt * ntl;
        const int grid = (int)std::min<long>(tiles, sms);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (kev) {                       // device time of the GEMM kernels alone (not the splits)
            PDD_CUDA(cudaEventCreate(&e0));
            PDD_CUDA(cudaEventCreate(&e1));
            kev->push_back(e0);
            kev->push_back(e1);
            PDD_CUDA(cudaEventRecord(e0, st));
        }
        if (sub) PDD_LAUNCH(k_tc_gemm_pipe<true>, grid, kPipeThreads, kPipeSmemAll, st, g);
        else PDD_LAUNCH(k_tc_gemm_pipe<false>, grid, kPipeThreads, kPipeSmemAll, st, g);
        if (kev) PDD_CUDA(cudaEventRecord(e1, st));
    }
}

// [lo, hi) float addresses touched by a batch of row-major matrices
static void span(const float *p, long s, int batch, int rows, int ld, int cols, uintptr_t &lo, uintptr_t &hi) {
    lo = (uintptr_t)p;
    hi = (uintptr_t)(p + (long)(batch - 1) * s + (long)(rows - 1) * ld + cols);
}

static bool spans_disjoint(const float *a, long sa, int rowsa, int lda, int colsa, const float *c, long sc,
                           int rowsc, int ldc, int colsc, int batch) {
    uintptr_t a0, a1, c0, c1;
    span(a, sa, batch, rowsa, lda, colsa, a0, a1);
    span(c, sc, batch, rowsc, ldc, colsc, c0, c1);
    return a1 <= c0 || c1 <= a0;
}

static int fused_tile_n(int N) { return N > 128 ? 256 : (N > 64 ? 128 : 64); }

// Longest K sent to the fused kernel.  Its converters hold the next chunks in registers, which
// covers the load latency of short updates (K = 64: the leaf panels, the leaf triangular solves
// and the thinnest Schur and TRSM updates, where it beats splitting first: 0.84-0.93x the time
// of split + pipelined GEMM on the 16-disk n = 3072 case) but not the operand rate of long ones
// (K >= 192: 1.2-2x), which the pipelined kernel streams from pre-split tiles with bulk copies.
static constexpr int kFusedMaxK = 64;

// whether tc_gemm takes the fused kernel (needs no scratch) for these operands
bool tc_gemm_fused_ok(int batch, int M, int N, int K, const float *A, long sA, int lda, bool transA, const float *B,
                      long sB, int ldb, bool transB, const float *C, long sC, int ldc, int alias) {
    if (K > kFusedMaxK) return false;
    const int mt = cdiv(M, 128), ntl = cdiv(N, fused_tile_n(N));
    const bool same_a = C == A && sC == sA && ldc == lda;
    const bool same_b = C == B && sC == sB && ldc == ldb;
    if (transA || transB) return false;
    if (alias == TC_ALIAS_A) return same_a && ntl == 1;
    if (alias == TC_ALIAS_B) return same_b && mt == 1;
    if (alias == TC_ALIAS_UNKNOWN)
        return (spans_disjoint(A, sA, M, lda, K, C, sC, M, ldc, N, batch) || (same_a && ntl == 1)) &&
               (spans_disjoint(B, sB, K, ldb, N, C, sC, M, ldc, N, batch) || (same_b && mt == 1));
    return true;
}

template <bool SUB, int TN, bool VEC>
static void launch_fused_t(int grid, cudaStream_t st, const FzArgs &g) {
    static bool attr[64] = {false};
    const int dev = cur_device();
    if (!attr[dev]) {
        PDD_CUDA(cudaFuncSetAttribute(k_tc_gemm_fused<SUB, TN, VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      fz_smem(TN)));
        attr[dev] = true;
    }
    auto kern = k_tc_gemm_fused<SUB, TN, VEC>;
    PDD_LAUNCH(kern, grid, kFzThreads, fz_smem(TN), st, g);
}

// code bits: 1 subtract, 2 16-byte A loads, 4 TN = 128, 8 TN = 256 (neither: TN = 64)
static void launch_fused(int code, int grid, cudaStream_t st, const FzArgs &g) {
    switch (code) {
        case 0: launch_fused_t<false, 64, false>(grid, st, g); break;
        case 1: launch_fused_t<true, 64, false>(grid, st, g); break;
        case 2: launch_fused_t<false, 64, true>(grid, st, g); break;
        case 3: launch_fused_t<true, 64, true>(grid, st, g); break;
        case 4: launch_fused_t<false, 128, false>(grid, st, g); break;
        case 5: launch_fused_t<true, 128, false>(grid, st, g); break;
        case 6: launch_fused_t<false, 128, true>(grid, st, g); break;
        case 7: launch_fused_t<true, 128, true>(grid, st, g); break;
        case 8: launch_fused_t<false, 256, false>(grid, st, g); break;
        case 9: launch_fused_t<true, 256, false>(grid, st, g); break;
        case 10: launch_fused_t<false, 256, true>(grid, st, g); break;
        default: launch_fused_t<true, 256, true>(grid, st, g); break;
    }
}

// C_b (-)= A_b B_b for b < batch.  A: M x K (row stride lda), or with transA its transpose stored
// K x M; B: K x N (ldb), or with transB its transpose stored N x K.  `alias` states how C meets
// the operands: TC_ALIAS_NONE (disjoint: the caller knows, e.g. separate blocks of one matrix),
// TC_ALIAS_A / TC_ALIAS_B (C is that operand, same pointer, stride and row stride), or
// TC_ALIAS_UNKNOWN (checked here by address ranges).  Untransposed operands with K <= 64 go
// through the fused kernel (no scratch) when every aliased part is read and written by the same
// tile (C = A with N <= TN, C = B with M <= 128); the rest through pre-split tiles in `scratch`.
void tc_gemm(int batch, int M, int N, int K, const float *A, long sA, int lda, bool transA, const float *B, long sB,
             int ldb, bool transB, float *C, long sC, int ldc, bool sub, int alias, float *scratch,
             size_t scratch_floats, int *err, cudaStream_t st, TcTiming *tt) {
    if (batch <= 0 || M <= 0 || N <= 0 || K <= 0) return;
    const int TN = fused_tile_n(N);
    const int mt = cdiv(M, 128), ntl = cdiv(N, TN);
    if (!tc_gemm_fused_ok(batch, M, N, K, A, sA, lda, transA, B, sB, ldb, transB, C, sC, ldc, alias)) {
        tc_gemm_presplit(batch, M, N, K, A, sA, lda, transA, B, sB, ldb, transB, C, sC, ldc, sub, scratch,
                         scratch_floats, err, st, tt ? &tt->pipe : nullptr);
        if (tt) tt->flop_pipe += 2.0 * M * N * K * batch;
        return;
    }
    // 16-byte loads of A: its matrices and rows start on 4-float boundaries
    const bool vec = ((uintptr_t)A & 15) == 0 && lda % 4 == 0 && sA % 4 == 0;
    const FzArgs g{M, N, K, mt, ntl, cdiv(K, kFzK), batch, A, sA, lda, B, sB, ldb, C, sC, ldc, err};
    const long tiles = (long)batch * mt * ntl;
    const int grid = (int)std::min<long>(tiles, (long)fz_ctas(TN) * sm_count());
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (tt) {
        PDD_CUDA(cudaEventCreate(&e0));
        PDD_CUDA(cudaEventCreate(&e1));
        tt->fused.push_back(e0);
        tt->fused.push_back(e1);
        PDD_CUDA(cudaEventRecord(e0, st));
        tt->flop_fused += 2.0 * M * N * K * batch;
        tt->bytes_fused += 4.0 * batch * ((double)M * K + (double)K * N + (sub ? 2.0 : 1.0) * M * N);
    }
    const int code = (sub ? 1 : 0) | (vec ? 2 : 0) | (TN == 256 ? 8 : (TN == 128 ? 4 : 0));
    launch_fused(code, grid, st, g);
    if (tt) PDD_CUDA(cudaEventRecord(e1, st));
}

void gemm_sub_tf32x3(int batch, int M, int N, int K, const float *A, long sA, int lda, const float *B, long sB,
                     int ldb, float *C, long sC, int ldc, int *err, cudaStream_t st) {
    if (batch <= 0 || M <= 0 || N <= 0 || K <= 0) return;
    static bool attr = false;
    if (!attr) {
        PDD_CUDA(cudaFuncSetAttribute(k_gemm_sub_tf32x3<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
        PDD_CUDA(cudaFuncSetAttribute(k_gemm_sub_tf32x3<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
        attr = true;
    }
    dim3 grid(cdiv(N, kTN), cdiv(M, kTM), batch);
    if (grid.y > 65535 || grid.z > 65535) fail(PDD_EINVAL, "GEMM batch too large");
    // 16-byte vector path: every row start and the K and N extents on 4-float boundaries
    auto al16 = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    const bool vec = al16(A) && al16(B) && al16(C) && lda % 4 == 0 && ldb % 4 == 0 && ldc % 4 == 0 && sA % 4 == 0 &&
                     sB % 4 == 0 && sC % 4 == 0 && K % 4 == 0 && N % 4 == 0;
    if (vec)
        PDD_LAUNCH(k_gemm_sub_tf32x3<true>, grid, kTcThreads, kTcSmem, st, M, N, K, A, sA, lda, B, sB, ldb, C, sC,
                   ldc, err);
    else
        PDD_LAUNCH(k_gemm_sub_tf32x3<false>, grid, kTcThreads, kTcSmem, st, M, N, K, A, sA, lda, B, sB, ldb, C, sC,
                   ldc, err);
}

}  // namespace pdd

// C ABI: the Schur-update primitive (see include/pdd.h)
extern "C" pdd_status pdd_batched_gemm_sub_tf32x3(int batch, int M, int N, int K, const float *A, long long sA,
                                                  int lda, const float *B, long long sB, int ldb, float *C,
                                                  long long sC, int ldc, void *stream) {
    using namespace pdd;
    try {
        if (batch < 0 || M < 0 || N < 0 || K < 0 || (batch && M && N && K && (!A || !B || !C)))
            fail(PDD_EINVAL, "negative size or null operand");
        if (lda < K || ldb < N || ldc < N) fail(PDD_EINVAL, "leading dimension smaller than the row length");
        cudaStream_t st = (cudaStream_t)stream;
        DevBuf<int> err;
        err.alloc(1);
        PDD_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
        gemm_sub_tf32x3(batch, M, N, K, A, (long)sA, lda, B, (long)sB, ldb, C, (long)sC, ldc, err.p, st);
        int h = 0;
        PDD_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        PDD_CUDA(cudaStreamSynchronize(st));
        if (h) fail(PDD_ECUDA, "tensor-core GEMM timed out waiting for its MMAs");
    } catch (const Fail &f) {
        return f.st;
    }
    return PDD_OK;
}

// C ABI: the pipelined form (see include/pdd.h)
extern "C" pdd_status pdd_batched_gemm_tf32x3(int batch, int M, int N, int K, const float *A, long long sA, int lda,
                                              const float *B, long long sB, int ldb, float *C, long long sC,
                                              int ldc, int subtract, void *stream) {
    using namespace pdd;
    try {
        if (batch < 0 || M < 0 || N < 0 || K < 0 || (batch && M && N && K && (!A || !B || !C)))
            fail(PDD_EINVAL, "negative size or null operand");
        if (lda < K || ldb < N || ldc < N) fail(PDD_EINVAL, "leading dimension smaller than the row length");
        if (batch == 0 || M == 0 || N == 0 || K == 0) return PDD_OK;
        cudaStream_t st = (cudaStream_t)stream;
        DevBuf<int> err;
        err.alloc(1);
        PDD_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
        const size_t per = tc_tile_floats(M, K) + tc_tile_floats(N, K);
        int chunk = 0;
        DevBuf<float> scr;
        if (!tc_gemm_fused_ok(batch, M, N, K, A, (long)sA, lda, false, B, (long)sB, ldb, false, C, (long)sC, ldc,
                              TC_ALIAS_UNKNOWN)) {
            chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)batch, ((size_t)1 << 28) / per));
            scr.alloc(per * chunk);
        }
        tc_gemm(batch, M, N, K, A, (long)sA, lda, false, B, (long)sB, ldb, false, C, (long)sC, ldc, subtract != 0,
                TC_ALIAS_UNKNOWN,
                scr.p, per * chunk, err.p, st, nullptr);
        int h = 0;
        PDD_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        PDD_CUDA(cudaStreamSynchronize(st));
        if (h) fail(PDD_ECUDA, "tensor-core GEMM timed out waiting for its pipeline");
    } catch (const Fail &f) {
        return f.st;
    }
    return PDD_OK;
}
