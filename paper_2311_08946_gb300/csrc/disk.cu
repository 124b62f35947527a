// a6-a9: floating rows by Chebyshev(r) x Fourier(theta) collocation on each
// disk (Sec. 3.3, Eq. 31-35, 40-41), batched over disks.
//
//   a6  k_node_coef + k_fill_operator: per-node FP64 coefficients and row
//       scales (one thread per node), the right-hand sides [A_IB H, -f], then
//       the rows of the row-equilibrated collocation matrix of L + c.
//   a7  FP64 form: k_lu, right-looking blocked LU with partial pivoting, one
//       CTA per disk, panel in shared memory.  Mixed form: the recursive FP32
//       LU of lu_rec.cu (tensor-core Schur updates) or the blocked one, chosen
//       by tune_lu.  The paper factors by QR (Eq. 41); LU solves the same
//       systems.
//   a8  FP64 form: k_lu_solve.  Mixed form: k_lu_solve_rl on the transposed
//       FP32 factors, refined in FP64 (first residual k_residual in FP64,
//       later ones k_residual_df in double-float delta form) until the
//       predicted next correction is below the tolerance.
//   a9  k_disk_eval / k_disk_eval_df: tensor interpolation (barycentric
//       Chebyshev in r over all 2 n_r + 2 points, the Fourier cardinal in
//       theta) at the knots of every row the disk contributes to, written into
//       the CSR values of C and the row's part of r.
//
// Grid: N_c = 2 n_r + 1 Chebyshev points x_k = cos(k pi / N_c); unknowns at
// radius x_k (k = 1..n_r) and angle t_j = 2 pi j / n_theta, index
// p = (k-1) n_theta + j; a point at x_{N_c - k} < 0 is radius x_k at angle
// t_j + pi.  With sigma = I the operator in polar coordinates is
// (1/2)(u_rr + u_r/r + u_tt/r^2) + b_x(cos t u_r - sin t u_t/r)
//   + b_y(sin t u_r + cos t u_t/r) + c u, and d/dr carries 1/R.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <vector>

#include "handles.cuh"

namespace pdd {

struct Shape {
    int nr, nt, nk, nc, n, nrhs;
    double *x, *D, *D2, *F1, *F2, *Hg;   // device tables
    float2 *Dhl, *D2hl, *F1hl, *F2hl;    // the same tables as FP32 (hi, lo) pairs
    float2 *Hghl;
};

struct DiskDesc {
    double cx, cy, R;
    int m, knot_base, row_begin, row_end;
};

// ---------------------------------------------------------------------------
// shape tables: Chebyshev points and differentiation matrix (closed form),
// Fourier differentiation vectors (closed forms), boundary data of each knot
// ---------------------------------------------------------------------------
__device__ double fourier_cardinal_cf(double x, int n) {
    // H(x) = sin(n x / 2) cot(x / 2) / n  (Eq. 18 summed), x reduced to (-pi, pi]
    x = remainder(x, PDD_TWO_PI);
    if (x == 0.0) return 1.0;
    double s = sin(0.5 * n * x), c = cos(0.5 * x), d = sin(0.5 * x);
    return s * c / (d * n);
}

__global__ void k_shape_tables(int nr, int nt, int nk, double *x, double *D, double *F1, double *F2,
                               double *Hg) {
    const int nc = 2 * nr + 1, np = nc + 1;
    for (int k = threadIdx.x; k < np; k += blockDim.x) x[k] = sin(PDD_PI * (nc - 2.0 * k) / (2.0 * nc));
    __syncthreads();
    for (int idx = threadIdx.x; idx < np * np; idx += blockDim.x) {
        int i = idx / np, j = idx % np;
        if (i == j) continue;
        double ci = (i == 0 || i == nc) ? 2.0 : 1.0, cj = (j == 0 || j == nc) ? 2.0 : 1.0;
        double sg = ((i + j) & 1) ? -1.0 : 1.0;
        D[idx] = ci / cj * sg / (x[i] - x[j]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < np; i += blockDim.x) {   // negative-sum diagonal
        double s = 0.0;
        for (int j = 0; j < np; ++j)
            if (j != i) s += D[i * np + j];
        D[i * np + i] = -s;
    }
    const double h = PDD_TWO_PI / nt;
    for (int d = threadIdx.x; d < nt; d += blockDim.x) {
        if (d == 0) {
            F1[0] = 0.0;
            F2[0] = -PDD_PI * PDD_PI / (3.0 * h * h) - 1.0 / 6.0;
        } else {
            double sg = (d & 1) ? -1.0 : 1.0;
            double s = sin(0.5 * d * h), c = cos(0.5 * d * h);
            F1[d] = 0.5 * sg * c / s;
            F2[d] = -0.5 * sg / (s * s);
        }
    }
    for (int idx = threadIdx.x; idx < nt * nk; idx += blockDim.x) {
        int j = idx / nk, col = idx % nk;
        double t = PDD_TWO_PI * j / nt, tk = PDD_TWO_PI * col / nk;
        Hg[idx] = fourier_cardinal_cf(t - tk, nk);
    }
}

__global__ void k_matmul_sq(const double *A, double *C, int np) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= np * np) return;
    int i = idx / np, j = idx % np;
    double s = 0.0;
    for (int k = 0; k < np; ++k) s += A[i * np + k] * A[k * np + j];
    C[idx] = s;
}

// ---------------------------------------------------------------------------
// a6: operator rows
// ---------------------------------------------------------------------------
struct NodeCoef {
    double alpha, beta, gamma, delta, c, s;
};

// per node: coefficients of the polar operator, the row scale 1/max|A_pq| (the
// nonzeros of a row are the radial line through the node, its mirror through
// the centre, the node's ring and the diagonal) and the right-hand sides
__global__ void __launch_bounds__(256) k_node_coef(Problem P, Shape S, const DiskDesc *disks, int nd,
                                                   double *RHS, long strideR, NodeCoef *coef, long strideC) {
    const long gid = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (gid >= (long)nd * S.n) return;
    const int disk = (int)(gid / S.n), p = (int)(gid - (long)disk * S.n);
    const DiskDesc dd = disks[disk];
    const int k = p / S.nt + 1, j = p % S.nt, np = S.nc + 1, half = S.nt >> 1;
    const double rho = S.x[k];
    double st, ct;
    sincos(PDD_TWO_PI * j / S.nt, &st, &ct);
    const double X = dd.cx + dd.R * rho * ct, Y = dd.cy + dd.R * rho * st;
    double bx, by;
    drift(P, X, Y, bx, by);
    const double cv = killing(P, X, Y);
    const double fv = source(P, X, Y);
    const double R2 = dd.R * dd.R;
    const double al = 0.5 / R2;
    const double be = 0.5 / (R2 * rho) + (bx * ct + by * st) / dd.R;
    const double ga = 0.5 / (R2 * rho * rho);
    const double de = (-bx * st + by * ct) / (dd.R * rho);
    // the row scale only equilibrates (any nearby value serves), so the candidates are evaluated
    // on the FP32 pipes (FP64 runs at a small fraction of their rate here): same terms, same order
    const float alf = (float)al, bef = (float)be, gaf = (float)ga, def = (float)de, cvf = (float)cv;
    const float2 *Dk = S.Dhl + k * np, *D2k = S.D2hl + k * np;
    float amax = 0.f;
    for (int l = 1; l <= S.nr; ++l) {
        float v = alf * D2k[l].x + bef * Dk[l].x;
        float vm = alf * D2k[S.nc - l].x + bef * Dk[S.nc - l].x;
        if (l == k) {                              // the node's own ring crosses both lines
            v += gaf * S.F2hl[0].x + def * S.F1hl[0].x + cvf;
            vm += gaf * S.F2hl[half].x + def * S.F1hl[half].x;
        }
        amax = fmaxf(amax, fabsf(v));
        amax = fmaxf(amax, fabsf(vm));
    }
    const int jm = j + half < S.nt ? j + half : j + half - S.nt;
    for (int jp = 0; jp < S.nt; ++jp) {
        if (jp == j || jp == jm) continue;                          // counted with the radial line
        const int d = jp <= j ? j - jp : j - jp + S.nt;
        amax = fmaxf(amax, fabsf(gaf * S.F2hl[d].x + def * S.F1hl[d].x));
    }
    const double sc = amax > 0.f ? 1.0 / (double)amax : 1.0;
    coef[disk * strideC + p] = NodeCoef{al, be, ga, de, cv, sc};
    const double w0 = al * S.D2[k * np + 0] + be * S.D[k * np + 0];
    const double wN = al * S.D2[k * np + S.nc] + be * S.D[k * np + S.nc];
    double *Rrow = RHS + disk * strideR + (long)p * S.nrhs;
    for (int col = 0; col < S.nk; ++col)
        Rrow[col] = sc * (w0 * S.Hg[j * S.nk + col] + wN * S.Hg[jm * S.nk + col]);
    Rrow[S.nk] = -sc * fv;
}

// rows of the equilibrated collocation matrix, one warp per row: the row is
// zeroed in shared memory, its nonzeros (the node's radial line, the mirrored
// line and the node's ring: 2 nr + nt candidates, the crossings computed twice
// with the same value) are evaluated in the matrix's precision (the FP32 rows
// of the mixed form feed only the LU that preconditions the refinement, whose
// residuals use the FP64 coefficients), and the row is stored with 16-byte
// writes
template <typename T>
__global__ void __launch_bounds__(256) k_fill_operator(Shape S, T *A, long strideA, const NodeCoef *coef,
                                                       long strideC, int rows_per_block) {
    extern __shared__ __align__(16) unsigned char fsm_raw[];
    const int disk = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= rows_per_block) return;
    const int p = blockIdx.x * rows_per_block + warp;
    if (p >= S.n) return;
    T *row = reinterpret_cast<T *>(fsm_raw) + (size_t)warp * S.n;
    if ((S.n * sizeof(T)) % 16 == 0) {
        float4 *r4 = reinterpret_cast<float4 *>(row);
        for (int q = lane; q < (int)(S.n * sizeof(T) / 16); q += 32) r4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        for (int q = lane; q < S.n; q += 32) row[q] = (T)0;
    }
    __syncwarp();
    const NodeCoef cf = coef[disk * strideC + p];
    const int k = p / S.nt + 1, j = p % S.nt, half = S.nt >> 1, jm = (j + half) % S.nt, np = S.nc + 1;
    const int ncand = 2 * S.nr + S.nt;
    // the candidates are the radial line through node p, its mirror through the centre and the ring
    // of p; each entry sums the operator's terms that reach it (radial, mirror, ring, diagonal, in
    // that order), the candidate's line and angle known without index division
    if constexpr (std::is_same<T, float>::value) {
        const float al = (float)cf.alpha, be = (float)cf.beta, ga = (float)cf.gamma, de = (float)cf.delta;
        const float cv = (float)cf.c, sc = (float)cf.s;
        const float2 *Dk = S.Dhl + k * np, *D2k = S.D2hl + k * np;
        for (int c = lane; c < ncand; c += 32) {
            int q;
            float v = 0.f;
            if (c < S.nr) {
                const int l = c + 1;
                q = c * S.nt + j;
                v += al * D2k[l].x + be * Dk[l].x;
                if (l == k) {
                    v += ga * S.F2hl[0].x + de * S.F1hl[0].x;
                    v += cv;
                }
            } else if (c < 2 * S.nr) {
                const int l = c - S.nr + 1;
                q = (l - 1) * S.nt + jm;
                v += al * D2k[S.nc - l].x + be * Dk[S.nc - l].x;
                if (l == k) v += ga * S.F2hl[half].x + de * S.F1hl[half].x;
            } else {
                const int jp = c - 2 * S.nr;
                q = (k - 1) * S.nt + jp;
                if (jp == j) v += al * D2k[k].x + be * Dk[k].x;
                if (jp == jm) v += al * D2k[S.nc - k].x + be * Dk[S.nc - k].x;
                int d = j - jp;
                d += d < 0 ? S.nt : 0;
                v += ga * S.F2hl[d].x + de * S.F1hl[d].x;
                if (jp == j) v += cv;
            }
            row[q] = sc * v;
        }
    } else {
        for (int c = lane; c < ncand; c += 32) {
            int q;
            double v = 0.0;
            if (c < S.nr) {                                      // radial line: l = c + 1, angle j
                const int l = c + 1;
                q = c * S.nt + j;
                v += cf.alpha * S.D2[k * np + l] + cf.beta * S.D[k * np + l];
                if (l == k) {
                    v += cf.gamma * S.F2[0] + cf.delta * S.F1[0];
                    v += cf.c;                                   // q == p
                }
            } else if (c < 2 * S.nr) {                           // mirror line: angle jm
                const int l = c - S.nr + 1;
                q = (l - 1) * S.nt + jm;
                v += cf.alpha * S.D2[k * np + S.nc - l] + cf.beta * S.D[k * np + S.nc - l];
                if (l == k) v += cf.gamma * S.F2[half] + cf.delta * S.F1[half];
            } else {                                             // ring of p: l = k, angle jp
                const int jp = c - 2 * S.nr;
                q = (k - 1) * S.nt + jp;
                if (jp == j) v += cf.alpha * S.D2[k * np + k] + cf.beta * S.D[k * np + k];
                if (jp == jm) v += cf.alpha * S.D2[k * np + S.nc - k] + cf.beta * S.D[k * np + S.nc - k];
                int d = j - jp;
                d += d < 0 ? S.nt : 0;
                v += cf.gamma * S.F2[d] + cf.delta * S.F1[d];
                if (jp == j) v += cf.c;                          // q == p
            }
            row[q] = (T)(cf.s * v);
        }
    }
    __syncwarp();
    T *Arow = A + disk * strideA + (long)p * S.n;
    constexpr int V = 16 / sizeof(T);
    if (S.n % V == 0) {
        const int nv = S.n / V;
        const float4 *src = reinterpret_cast<const float4 *>(row);
        float4 *dst = reinterpret_cast<float4 *>(Arow);
        for (int q = lane; q < nv; q += 32) dst[q] = src[q];
    } else {
        for (int q = lane; q < S.n; q += 32) Arow[q] = row[q];
    }
}

// the collocation system of every disk of the wave: node coefficients, then the matrix rows
template <typename T>
static void build_operator(const Problem &P, const Shape &S, const DiskDesc *dd, int nd, T *A, long sA, double *RHS,
                           long sR, NodeCoef *coef, long sC, cudaStream_t st) {
    PDD_LAUNCH(k_node_coef, cdiv((long)nd * S.n, 256), 256, 0, st, P, S, dd, nd, RHS, sR, coef, sC);
    const size_t row_bytes = (size_t)S.n * sizeof(T);
    const int rpb = (int)std::max<size_t>(1, std::min<size_t>(8, (size_t)(96 * 1024) / row_bytes));
    if (row_bytes > (size_t)200 * 1024) fail(PDD_EINVAL, "disk grid too large for the operator kernel");
    const size_t sm = rpb * row_bytes;
    PDD_CUDA(cudaFuncSetAttribute(k_fill_operator<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 g(cdiv(S.n, rpb), nd);
    PDD_LAUNCH(k_fill_operator<T>, g, 32 * rpb, sm, st, S, A, sA, coef, sC, rpb);
}

// ---------------------------------------------------------------------------
// a7: batched LU with partial pivoting (row-major, in place), one CTA per disk
// ---------------------------------------------------------------------------
template <typename T, int NB>
__global__ void __launch_bounds__(256) k_lu(T *Aall, int n, long strideA, int *permAll, int *infoAll) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int LD = NB + 1;                             // padded panel rows: no bank conflicts
    T *Pn = reinterpret_cast<T *>(smem_raw);               // panel rows x LD
    T *Ut = Pn + (size_t)n * LD;                           // NB x 64 tile of U12
    __shared__ int piv[NB];
    __shared__ double rv[8];
    __shared__ int ri[8];
    const int disk = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    T *A = Aall + disk * strideA;
    int *perm = permAll + (long)disk * n;
    for (int i = tid; i < n; i += 256) perm[i] = i;
    int info = 0;
    __syncthreads();
    for (int k0 = 0; k0 < n; k0 += NB) {
        const int kb = min(NB, n - k0), rows = n - k0;
        for (int idx = tid; idx < rows * kb; idx += 256) {
            int r = idx / kb, c = idx - r * kb;
            Pn[r * LD + c] = A[(long)(k0 + r) * n + k0 + c];
        }
        __syncthreads();
        for (int c = 0; c < kb; ++c) {
            double best = -1.0;
            int bi = c;
            for (int r = c + tid; r < rows; r += 256) {
                double v = fabs((double)Pn[r * LD + c]);
                if (v > best) { best = v; bi = r; }
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                double ov = __shfl_xor_sync(0xffffffffu, best, o);
                int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (lane == 0) { rv[warp] = best; ri[warp] = bi; }
            __syncthreads();
            if (tid == 0) {
                double b = rv[0];
                int i0 = ri[0];
                for (int w = 1; w < 8; ++w)
                    if (rv[w] > b || (rv[w] == b && ri[w] < i0)) { b = rv[w]; i0 = ri[w]; }
                piv[c] = i0;
                if (i0 != c) {
                    int t = perm[k0 + c];
                    perm[k0 + c] = perm[k0 + i0];
                    perm[k0 + i0] = t;
                }
            }
            __syncthreads();
            const int p = piv[c];
            if (p != c)
                for (int cc = tid; cc < kb; cc += 256) {
                    T t = Pn[c * LD + cc];
                    Pn[c * LD + cc] = Pn[p * LD + cc];
                    Pn[p * LD + cc] = t;
                }
            __syncthreads();
            const T d = Pn[c * LD + c];
            if (d == (T)0 && info == 0) info = k0 + c + 1;
            for (int r = c + 1 + tid; r < rows; r += 256) {
                T l = (d != (T)0) ? Pn[r * LD + c] / d : (T)0;
                Pn[r * LD + c] = l;
                for (int cc = c + 1; cc < kb; ++cc) Pn[r * LD + cc] -= l * Pn[c * LD + cc];
            }
            __syncthreads();
        }
        // write the panel back
        for (int idx = tid; idx < rows * kb; idx += 256) {
            int r = idx / kb, c = idx - r * kb;
            A[(long)(k0 + r) * n + k0 + c] = Pn[r * LD + c];
        }
        // the panel's row interchanges, applied to the columns outside it
        for (int c = 0; c < kb; ++c) {
            const int p = piv[c];
            if (p != c) {
                T *ra = A + (long)(k0 + c) * n, *rb = A + (long)(k0 + p) * n;
                for (int j = tid; j < n - kb; j += 256) {
                    int col = j < k0 ? j : j + kb;
                    T t = ra[col];
                    ra[col] = rb[col];
                    rb[col] = t;
                }
            }
            __syncthreads();
        }
        const int c0 = k0 + kb, nrem = n - c0;
        if (nrem <= 0) break;
        // U12 = L11^-1 A12 (unit lower triangular solve, one column per thread)
        for (int j = c0 + tid; j < n; j += 256) {
            T u[NB];
#pragma unroll
            for (int rr = 0; rr < NB; ++rr) {
                if (rr < kb) {
                    T v = A[(long)(k0 + rr) * n + j];
                    for (int t = 0; t < rr; ++t) v -= Pn[rr * LD + t] * u[t];
                    u[rr] = v;
                    A[(long)(k0 + rr) * n + j] = v;
                }
            }
        }
        __syncthreads();
        // A22 -= L21 U12 in 64 x 64 tiles, 4 x 4 per thread
        const int tiles = (nrem + 63) / 64;
        const int ty = tid >> 4, tx = tid & 15;
        for (int tj = 0; tj < tiles; ++tj) {
            const int cbase = c0 + tj * 64;
            for (int idx = tid; idx < kb * 64; idx += 256) {
                int t = idx >> 6, jj = idx & 63;
                int col = cbase + jj;
                Ut[t * 64 + jj] = col < n ? A[(long)(k0 + t) * n + col] : (T)0;
            }
            __syncthreads();
            for (int ti = 0; ti < tiles; ++ti) {
                const int rbase = ti * 64;          // index into the panel rows beyond kb
                T acc[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
                for (int t = 0; t < kb; ++t) {
                    T lv[4], uv[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        int pr = kb + rbase + ty * 4 + a;
                        lv[a] = pr < rows ? Pn[pr * LD + t] : (T)0;
                    }
#pragma unroll
                    for (int b = 0; b < 4; ++b) uv[b] = Ut[t * 64 + tx * 4 + b];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] += lv[a] * uv[b];
                }
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    int row = c0 + rbase + ty * 4 + a;
                    if (row >= n) continue;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        int col = cbase + tx * 4 + b;
                        if (col < n) A[(long)row * n + col] -= acc[a][b];
                    }
                }
            }
            __syncthreads();
        }
    }
    if (tid == 0) infoAll[disk] = info;
}

// ---------------------------------------------------------------------------
// a8: multi-RHS solve with the LU factors: W = U^-1 L^-1 P R, then X = W
// (plain form) or X += W with a per-disk convergence test (refinement).
// Row blocks of TB: the off-diagonal part of each block is a small GEMM
// staged through shared memory (QB-wide tiles of the factor and of the
// solved rows), the TB x TB diagonal block is solved column by column.
// ---------------------------------------------------------------------------
static constexpr int kSolveTB = 32, kSolveQB = 64, kSolveMaxOut = 12;   // nrhs <= 96

template <typename T>
__global__ void __launch_bounds__(256) k_lu_solve(const T *LUall, int n, long strideA, const int *permAll,
                                                  const double *Rall, int nrhs, long strideR,
                                                  T *Wall, double *Xall, int accumulate, int *conv,
                                                  int *sweeps, double tol) {
    extern __shared__ __align__(16) unsigned char ssm[];
    T *Ls = reinterpret_cast<T *>(ssm);                     // kSolveTB x kSolveQB (factor tile)
    T *Ys = Ls + kSolveTB * kSolveQB;                       // kSolveQB x nrhs (solved rows)
    T *Dg = Ys + kSolveQB * nrhs;                           // kSolveTB x kSolveTB diagonal block
    T *Xs = Dg + kSolveTB * kSolveTB;                       // kSolveTB x nrhs rows being solved
    const int disk = blockIdx.x, tid = threadIdx.x;
    if (conv && conv[disk]) return;
    const T *LU = LUall + disk * strideA;
    const int *perm = permAll + (long)disk * n;
    const double *R = Rall + disk * strideR;
    T *W = Wall + disk * strideR;
    double *X = Xall + disk * strideR;
    constexpr int TB = kSolveTB, QB = kSolveQB;
    for (int pass = 0; pass < 2; ++pass) {                  // 0: L (unit lower), 1: U (upper)
        const int nblk = (n + TB - 1) / TB;
        for (int bi = 0; bi < nblk; ++bi) {
            const int blk = pass == 0 ? bi : nblk - 1 - bi;
            const int i0 = blk * TB, tb = min(TB, n - i0);
            const int qa = pass == 0 ? 0 : i0 + tb, qb = pass == 0 ? i0 : n;   // already solved rows
            T acc[kSolveMaxOut];
#pragma unroll
            for (int o = 0; o < kSolveMaxOut; ++o) acc[o] = (T)0;
            for (int q0 = qa; q0 < qb; q0 += QB) {
                const int qn = min(QB, qb - q0);
                for (int e = tid; e < TB * QB; e += 256) {
                    const int r = e / QB, q = e - r * QB;
                    Ls[e] = (r < tb && q < qn) ? LU[(long)(i0 + r) * n + q0 + q] : (T)0;
                }
                for (int e = tid; e < QB * nrhs; e += 256) {
                    const int q = e / nrhs, c = e - q * nrhs;
                    Ys[e] = (q < qn) ? W[(long)(q0 + q) * nrhs + c] : (T)0;
                }
                __syncthreads();
#pragma unroll
                for (int o = 0; o < kSolveMaxOut; ++o) {
                    const int e = tid + o * 256;
                    if (e < tb * nrhs) {
                        const int r = e / nrhs, c = e - r * nrhs;
                        T a = acc[o];
                        const T *lr = Ls + r * QB;
                        for (int q = 0; q < qn; ++q) a += lr[q] * Ys[q * nrhs + c];
                        acc[o] = a;
                    }
                }
                __syncthreads();
            }
            for (int e = tid; e < tb * tb; e += 256) {
                const int r = e / tb, c = e - r * tb;
                Dg[r * TB + c] = LU[(long)(i0 + r) * n + i0 + c];
            }
#pragma unroll
            for (int o = 0; o < kSolveMaxOut; ++o) {
                const int e = tid + o * 256;
                if (e < tb * nrhs) {
                    const int r = e / nrhs, c = e - r * nrhs;
                    const T rhs = pass == 0 ? (T)R[(long)perm[i0 + r] * nrhs + c] : W[(long)(i0 + r) * nrhs + c];
                    Xs[r * nrhs + c] = rhs - acc[o];
                }
            }
            __syncthreads();
            // the diagonal block, in shared memory
            for (int c = tid; c < nrhs; c += 256) {
                if (pass == 0) {
                    for (int ii = 1; ii < tb; ++ii) {
                        T v = Xs[ii * nrhs + c];
                        for (int t = 0; t < ii; ++t) v -= Dg[ii * TB + t] * Xs[t * nrhs + c];
                        Xs[ii * nrhs + c] = v;
                    }
                } else {
                    for (int ii = tb - 1; ii >= 0; --ii) {
                        T v = Xs[ii * nrhs + c];
                        for (int t = ii + 1; t < tb; ++t) v -= Dg[ii * TB + t] * Xs[t * nrhs + c];
                        Xs[ii * nrhs + c] = v / Dg[ii * TB + ii];
                    }
                }
            }
            __syncthreads();
            for (int e = tid; e < tb * nrhs; e += 256) W[(long)i0 * nrhs + e] = Xs[e];
            __syncthreads();
        }
    }
    // X = W or X += W; refinement test max|W| <= tol max|X|
    double dmax = 0.0, xmax = 0.0;
    for (long o = tid; o < (long)n * nrhs; o += 256) {
        const double w = (double)W[o];
        const double xv = accumulate ? X[o] + w : w;
        X[o] = xv;
        dmax = fmax(dmax, fabs(w));
        xmax = fmax(xmax, fabs(xv));
    }
    if (!conv) return;
    __shared__ double sd[8], sx[8];
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
    }
    if ((tid & 31) == 0) { sd[tid >> 5] = dmax; sx[tid >> 5] = xmax; }
    __syncthreads();
    if (tid == 0) {
        double d = 0.0, x = 0.0;
        for (int w = 0; w < 8; ++w) { d = fmax(d, sd[w]); x = fmax(x, sx[w]); }
        sweeps[disk] += 1;
        if (d <= tol * x) conv[disk] = 1;
    }
}

template <typename T>
static size_t solve_smem(int nrhs) {
    return sizeof(T) * ((size_t)kSolveTB * kSolveQB + (size_t)kSolveQB * nrhs + (size_t)kSolveTB * kSolveTB +
                        (size_t)kSolveTB * nrhs);
}

template <typename T>
static void launch_solve(const T *LU, int n, long sA, const int *perm, const double *R, int nrhs, long sR, T *W,
                         double *X, int accumulate, int *conv, int *sweeps, double tol, int nd, cudaStream_t st) {
    if (nrhs > 96) fail(PDD_EINVAL, "more than 95 knots per circle");
    const size_t sm = solve_smem<T>(nrhs);
    PDD_CUDA(cudaFuncSetAttribute(k_lu_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    PDD_LAUNCH(k_lu_solve<T>, nd, 256, sm, st, LU, n, sA, perm, R, nrhs, sR, W, X, accumulate, conv, sweeps, tol);
}

// ---------------------------------------------------------------------------
// a8, mixed form: right-looking blocked triangular solves.  One CTA holds a
// group of right-hand-side columns for all n rows in shared memory; for each
// 32-row panel it applies the inverse of the panel's diagonal block (computed
// once after the factorisation) and then subtracts the panel's contribution
// from every row not yet solved.  Each factor entry is read from HBM once per
// solve, and the row updates are independent FP32 FMA chains (broadcast
// shared-memory reads of the solved panel rows).
// ---------------------------------------------------------------------------
static constexpr int kRlTB = 32, kRlThreads = 512;
static constexpr size_t kRlSmemMax = 225 * 1024;        // 227 KB per CTA, less the static arrays

// inverses of the unit-lower and upper 32x32 diagonal blocks of each LU:
// Dinv[disk][blk][0] = inv(L_bb), Dinv[disk][blk][1] = inv(U_bb), zero-padded
__global__ void __launch_bounds__(128) k_diag_inv(const float *LUall, int n, long strideA, int nd, float *Dinv) {
    __shared__ float Ts[4][kRlTB][kRlTB + 1], Xs[4][kRlTB][kRlTB + 1];
    const int w = threadIdx.x >> 5, j = threadIdx.x & 31;
    const int nblk = (n + kRlTB - 1) / kRlTB;
    const long item = (long)blockIdx.x * 4 + w;
    if (item >= (long)nd * nblk * 2) return;
    const int tri = (int)(item & 1);
    const long db = item >> 1;
    const int blk = (int)(db % nblk), disk = (int)(db / nblk);
    const int i0 = blk * kRlTB, tb = min(kRlTB, n - i0);
    const float *LU = LUall + disk * strideA;
    for (int r = 0; r < kRlTB; ++r) Ts[w][r][j] = (r < tb && j < tb) ? LU[(long)(i0 + r) * n + i0 + j] : 0.f;
    __syncwarp();
    // lane j forms column j of the inverse
    if (tri == 0) {
        for (int i = 0; i < kRlTB; ++i) {
            float v = (i == j) ? 1.f : 0.f;
            if (i > j && i < tb)
                for (int k = j; k < i; ++k) v -= Ts[w][i][k] * Xs[w][k][j];
            Xs[w][i][j] = (i < tb && j < tb) ? v : 0.f;
        }
    } else {
        for (int i = kRlTB - 1; i >= 0; --i) {
            float v = 0.f;
            if (i < tb && j < tb && i <= j) {
                v = (i == j) ? 1.f : 0.f;
                for (int k = i + 1; k <= j; ++k) v -= Ts[w][i][k] * Xs[w][k][j];
                v /= Ts[w][i][i];
            }
            Xs[w][i][j] = v;
        }
    }
    __syncwarp();
    float *out = Dinv + (((long)disk * nblk + blk) * 2 + tri) * (kRlTB * kRlTB);
    for (int r = 0; r < kRlTB; ++r) out[r * kRlTB + j] = Xs[w][r][j];
}

// packed FP32 pairs: fma.rn.f32x2 is two correctly rounded FMAs (the same results as fmaf)
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(unsigned long long r, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// shared-memory floats of the right-looking solve: the panel's solved rows padded to 4-float
// rows, the diagonal-block inverse, the n x CG right-hand sides
__host__ __device__ constexpr int rl_cgp(int CG) { return (CG + 3) & ~3; }
static size_t rl_smem_bytes(int n, int CG) {
    return ((size_t)kRlTB * rl_cgp(CG) + (size_t)kRlTB * (kRlTB + 1) + (size_t)n * CG) * sizeof(float);
}

// X += inv(LU) P R for the columns [blockIdx.y CG, ...) of every disk not yet
// converged; the largest |correction| and |X| of each disk go to dmaxb/xmaxb
// (bit patterns of non-negative doubles, ordered like the values)
template <int CG>
__global__ void __launch_bounds__(kRlThreads, 1) k_lu_solve_rl(const float *LUTall, int n, long strideA,
                                                               const int *permAll, const float *DinvAll,
                                                               const double *Rall, int nrhs, long strideR,
                                                               double *Xall, const int *conv,
                                                               unsigned long long *dmaxb, unsigned long long *xmaxb,
                                                               float2 *Dall, int dmode) {
    constexpr int NT = kRlThreads, TB = kRlTB;
    constexpr bool VEC = (CG % 4) == 0;                // 16-byte shared-memory access to the columns
    constexpr int PD = (CG <= 20) ? 32 : (CG <= 36 ? 8 : 2);   // factor entries per row in flight
    constexpr int CGP = rl_cgp(CG);
    constexpr int NP = CG / 2;                         // column pairs (a last odd column is scalar)
    extern __shared__ __align__(16) float rsm[];
    float *Xp = rsm;                                   // TB x CGP: the panel's solved rows, 16-byte rows
    float *Ds = Xp + TB * CGP;                         // TB x (TB + 1) diagonal-block inverse (padded rows)
    float *Bs = Ds + TB * (TB + 1);                    // n x CG: right-hand sides, then solutions
    const int disk = blockIdx.x, tid = threadIdx.x;
    if (conv[disk]) return;
    const int c0 = blockIdx.y * CG, cg = min(CG, nrhs - c0);
    const float *LUT = LUTall + disk * strideA;      // the factors transposed
    const int *perm = permAll + (long)disk * n;
    const double *R = Rall + disk * strideR;
    double *X = Xall + disk * strideR;
    const int nblk = (n + TB - 1) / TB;
    const float *Dv = DinvAll + (long)disk * nblk * 2 * (TB * TB);
    for (int e = tid; e < n * CG; e += NT) {
        const int p = e / CG, c = e - p * CG;
        Bs[e] = (c < cg) ? (float)R[(long)perm[p] * nrhs + c0 + c] : 0.f;
    }
    for (int e = tid; e < TB * CGP; e += NT) Xp[e] = 0.f;
    // each panel's diagonal-block inverse is loaded into registers one panel ahead (NT >= TB TB / 2)
    static_assert(2 * NT >= TB * TB, "two inverse entries per thread");
    float dnext[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int e = tid + h * NT;
        dnext[h] = e < TB * TB ? Dv[e] : 0.f;                       // pass 0, block 0
    }
    for (int pass = 0; pass < 2; ++pass) {             // 0: L (unit lower), 1: U (upper)
        for (int bi = 0; bi < nblk; ++bi) {
            const int blk = pass == 0 ? bi : nblk - 1 - bi;
            const int i0 = blk * TB, tb = min(TB, n - i0);
            const int ra = pass == 0 ? i0 + tb : 0, rb = pass == 0 ? n : i0;
            const bool full = tb == TB;
            // the panel's rows X_b = inv(T_bb) B_b: warp q takes columns 4q .. 4q+3 (one column when CG
            // is not a multiple of 4), lane i the panel row i; the row of the inverse comes from shared
            // memory and the panel's right-hand sides are read as broadcasts
            const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int e = tid + h * NT;
                if (e < TB * TB) Ds[(e >> 5) * (TB + 1) + (e & 31)] = dnext[h];
            }
            {   // the next panel's inverse (L pass in block order, then U pass in reverse)
                const bool last_l = pass == 0 && bi == nblk - 1;
                const int npass = last_l ? 1 : pass;
                const int nblk_i = last_l ? nblk - 1 : (pass == 0 ? blk + 1 : blk - 1);
                if (npass == 1 && nblk_i < 0) {
                    dnext[0] = dnext[1] = 0.f;
                } else {
                    const float *Dn = Dv + ((long)nblk_i * 2 + npass) * (TB * TB);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int e = tid + h * NT;
                        if (e < TB * TB) dnext[h] = Dn[e];
                    }
                }
            }
            __syncthreads();
            constexpr int NQ = VEC ? CG / 4 : CG, NW = NT / 32, QP = (NQ + NW - 1) / NW;
            float4 xo[QP];
#pragma unroll
            for (int qp = 0; qp < QP; ++qp) {
                const int q = warp + qp * NW;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (q < NQ && lane < tb) {
                    const float *dr = Ds + lane * (TB + 1);
                    if constexpr (VEC) {
                        const float *bc = Bs + (size_t)i0 * CG + 4 * q;
                        for (int k = 0; k < tb; ++k) {
                            const float d = dr[k];
                            const float4 b = *reinterpret_cast<const float4 *>(bc + (size_t)k * CG);
                            v.x = fmaf(d, b.x, v.x);
                            v.y = fmaf(d, b.y, v.y);
                            v.z = fmaf(d, b.z, v.z);
                            v.w = fmaf(d, b.w, v.w);
                        }
                    } else {
                        const float *bc = Bs + (size_t)i0 * CG + q;
                        for (int k = 0; k < tb; ++k) v.x = fmaf(dr[k], bc[(size_t)k * CG], v.x);
                    }
                }
                xo[qp] = v;
            }
            __syncthreads();
#pragma unroll
            for (int qp = 0; qp < QP; ++qp) {
                const int q = warp + qp * NW;
                if (q < NQ && lane < tb) {
                    if constexpr (VEC) {
                        *reinterpret_cast<float4 *>(Bs + (size_t)(i0 + lane) * CG + 4 * q) = xo[qp];
                        *reinterpret_cast<float4 *>(Xp + lane * CGP + 4 * q) = xo[qp];
                    } else {
                        Bs[(size_t)(i0 + lane) * CG + q] = xo[qp].x;
                        Xp[lane * CGP + q] = xo[qp].x;
                    }
                }
            }
            __syncthreads();
            // rows still to solve: B_r -= T_rb X_b, two rows per thread so that each broadcast read of
            // a solved row feeds both
            for (int base = ra; base < rb; base += 2 * NT) {
                // the rows of this pass paired as (t, t + half): no thread carries an empty second row
                const int m = min(2 * NT, rb - base), half = (m + 1) >> 1;
                if (tid >= half) continue;
                const int r = base + tid, r2 = r + half;
                const bool two = r2 < base + m;
                float *b0 = Bs + (size_t)r * CG, *b1 = Bs + (size_t)(two ? r2 : r) * CG;
                // factor entries T[r][i0 + k] = LUT[(i0 + k) n + r]: consecutive rows, consecutive addresses
                const float *l0 = LUT + (long)i0 * n + r, *l1 = LUT + (long)i0 * n + (two ? r2 : r);
                if (full) {
                    // the rows as packed column pairs; the panel's solved rows as 16-byte loads, each
                    // feeding both rows; PD factor entries per row in flight before their FMAs
                    unsigned long long p0[NP > 0 ? NP : 1], p1[NP > 0 ? NP : 1];
                    float s0 = 0.f, s1 = 0.f;
#pragma unroll
                    for (int c = 0; c < NP; ++c) {
                        p0[c] = pk2(b0[2 * c], b0[2 * c + 1]);
                        p1[c] = pk2(b1[2 * c], b1[2 * c + 1]);
                    }
                    if (CG & 1) {
                        s0 = b0[CG - 1];
                        s1 = b1[CG - 1];
                    }
#pragma unroll 1
                    for (int k0 = 0; k0 < TB; k0 += PD) {
                        float m0[PD], m1[PD];
#pragma unroll
                        for (int kk = 0; kk < PD; ++kk) {
                            m0[kk] = __ldg(l0 + (long)(k0 + kk) * n);
                            m1[kk] = __ldg(l1 + (long)(k0 + kk) * n);
                        }
#pragma unroll
                        for (int kk = 0; kk < PD; ++kk) {
                            const float4 *xr = reinterpret_cast<const float4 *>(Xp + (k0 + kk) * CGP);
                            const unsigned long long n0 = pk2(-m0[kk], -m0[kk]), n1 = pk2(-m1[kk], -m1[kk]);
#pragma unroll
                            for (int c4 = 0; c4 < CGP / 4; ++c4) {
                                const float4 x = xr[c4];
                                if (2 * c4 < NP) {
                                    const unsigned long long xa = pk2(x.x, x.y);
                                    p0[2 * c4] = fma2(n0, xa, p0[2 * c4]);
                                    p1[2 * c4] = fma2(n1, xa, p1[2 * c4]);
                                } else if ((CG & 1) && 4 * c4 == CG - 1) {
                                    s0 = fmaf(-m0[kk], x.x, s0);
                                    s1 = fmaf(-m1[kk], x.x, s1);
                                }
                                if (2 * c4 + 1 < NP) {
                                    const unsigned long long xb = pk2(x.z, x.w);
                                    p0[2 * c4 + 1] = fma2(n0, xb, p0[2 * c4 + 1]);
                                    p1[2 * c4 + 1] = fma2(n1, xb, p1[2 * c4 + 1]);
                                } else if ((CG & 1) && 4 * c4 + 2 == CG - 1) {
                                    s0 = fmaf(-m0[kk], x.z, s0);
                                    s1 = fmaf(-m1[kk], x.z, s1);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int c = 0; c < NP; ++c) upk2(p0[c], b0[2 * c], b0[2 * c + 1]);
                    if (CG & 1) b0[CG - 1] = s0;
                    if (two) {
#pragma unroll
                        for (int c = 0; c < NP; ++c) upk2(p1[c], b1[2 * c], b1[2 * c + 1]);
                        if (CG & 1) b1[CG - 1] = s1;
                    }
                } else {
                    float acc0[CG], acc1[CG];
#pragma unroll
                    for (int c = 0; c < CG; ++c) {
                        acc0[c] = b0[c];
                        acc1[c] = b1[c];
                    }
                    for (int k = 0; k < tb; ++k) {
                        const float m0 = __ldg(l0 + (long)k * n), m1 = __ldg(l1 + (long)k * n);
                        const float *xr = Xp + k * CGP;
#pragma unroll
                        for (int c = 0; c < CG; ++c) {
                            const float x = xr[c];
                            acc0[c] = fmaf(-m0, x, acc0[c]);
                            acc1[c] = fmaf(-m1, x, acc1[c]);
                        }
                    }
#pragma unroll
                    for (int c = 0; c < CG; ++c) b0[c] = acc0[c];
                    if (two) {
#pragma unroll
                        for (int c = 0; c < CG; ++c) b1[c] = acc1[c];
                    }
                }
            }
            __syncthreads();
        }
    }
    // X += W (and D = W or D += W, in double-float, for the later residuals); the refinement test
    // takes max|W| and max|X| over the disk's columns
    double dmax = 0.0, xmax = 0.0;
    float2 *Dd = dmode ? Dall + disk * strideR : nullptr;
    for (int e = tid; e < n * cg; e += NT) {
        const int p = e / cg, c = e - p * cg;
        const float w32 = Bs[(size_t)p * CG + c];
        const double w = (double)w32;
        const long o = (long)p * nrhs + c0 + c;
        const double xv = X[o] + w;
        X[o] = xv;
        if (dmode == 1) Dd[o] = make_float2(w32, 0.f);
        else if (dmode == 2) Dd[o] = df_add(Dd[o], make_float2(w32, 0.f));
        dmax = fmax(dmax, fabs(w));
        xmax = fmax(xmax, fabs(xv));
    }
    __shared__ double sd[NT / 32], sx[NT / 32];
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
    }
    if ((tid & 31) == 0) {
        sd[tid >> 5] = dmax;
        sx[tid >> 5] = xmax;
    }
    __syncthreads();
    if (tid == 0) {
        double d = 0.0, x = 0.0;
        for (int w = 0; w < NT / 32; ++w) {
            d = fmax(d, sd[w]);
            x = fmax(x, sx[w]);
        }
        atomicMax(dmaxb + disk, (unsigned long long)__double_as_longlong(d));
        atomicMax(xmaxb + disk, (unsigned long long)__double_as_longlong(x));
    }
}

// per disk: count the sweep and stop refining once max|W| <= tol max|X|
// AT = A^T for every disk (32 x 32 tiles through shared memory): the solve then reads the factor
// entries of consecutive rows from consecutive addresses
__global__ void __launch_bounds__(256) k_transpose_f32(const float *Aall, float *ATall, int n, long strideA) {
    __shared__ float t[32][33];
    const int disk = blockIdx.z, bx = blockIdx.x * 32, by = blockIdx.y * 32;
    const float *A = Aall + disk * strideA;
    float *AT = ATall + disk * strideA;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
        const int gr = by + r, gc = bx + tx;
        t[r][tx] = (gr < n && gc < n) ? A[(long)gr * n + gc] : 0.f;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int gr = bx + r, gc = by + tx;
        if (gr < n && gc < n) AT[(long)gr * n + gc] = t[tx][r];
    }
}

// the same transpose in 64 x 64 tiles with 16-byte loads and stores (n a multiple of 4): each
// thread has four loads in flight, and the disk's tiles are a quarter as many blocks
__global__ void __launch_bounds__(256) k_transpose_f32_v4(const float *Aall, float *ATall, int n, long strideA) {
    __shared__ float t[64][65];
    const int disk = blockIdx.z, bx = blockIdx.x * 64, by = blockIdx.y * 64;   // rows by.., columns bx..
    const float *A = Aall + disk * strideA;
    float *AT = ATall + disk * strideA;
    const int c4 = threadIdx.x & 15, rr = threadIdx.x >> 4;                    // 16 float4 per tile row
    float4 v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int gr = by + rr + 16 * k, gc = bx + 4 * c4;
        v[k] = (gr < n && gc < n) ? *reinterpret_cast<const float4 *>(A + (long)gr * n + gc)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float *row = &t[rr + 16 * k][4 * c4];
        row[0] = v[k].x;
        row[1] = v[k].y;
        row[2] = v[k].z;
        row[3] = v[k].w;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int o = rr + 16 * k;                       // row bx + o of AT = column bx + o of A
        const int gr = bx + o, gc = by + 4 * c4;
        if (gr < n && gc < n)
            *reinterpret_cast<float4 *>(AT + (long)gr * n + gc) =
                make_float4(t[4 * c4][o], t[4 * c4 + 1][o], t[4 * c4 + 2][o], t[4 * c4 + 3][o]);
    }
}

// per disk: count the sweep and stop refining once the correction just applied, or the next one
// predicted from the contraction of the last two (|W_s|^2 / |W_{s-1}|, when they contract), is at
// most tol max|X|
__global__ void k_refine_conv(int nd, int *conv, int *sweeps, unsigned long long *dmaxb,
                              unsigned long long *xmaxb, double *dprev, double tol) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= nd) return;
    if (!conv[d]) {
        sweeps[d] += 1;
        const double w = __longlong_as_double((long long)dmaxb[d]);
        const double x = __longlong_as_double((long long)xmaxb[d]);
        const double wp = sweeps[d] > 1 ? dprev[d] : 0.0;
        const bool predicted = wp > 0.0 && w < wp && w * (w / wp) <= tol * x;
        if (w <= tol * x || predicted) conv[d] = 1;
        dprev[d] = w;
    }
    dmaxb[d] = 0ull;
    xmaxb[d] = 0ull;
}

// column-group width of the right-looking solve for n rows and nrhs columns
// (0: the shared-memory block does not fit; the tiled solve is used)
static int rl_width(int n, int nrhs, int &groups) {
    static const int widths[] = {8, 12, 17, 20, 36, 52};     // 17: all 17 columns of 16-knot disks at n = 3072
    for (int g = 1; g <= nrhs; ++g) {
        const int cg = (nrhs + g - 1) / g;
        int W = 0;
        for (int w : widths)
            if (w >= cg) {
                W = w;
                break;
            }
        if (!W) continue;
        const size_t sm = rl_smem_bytes(n, W);
        if (sm <= kRlSmemMax) {
            groups = (nrhs + W - 1) / W;
            return W;
        }
        if (W == 8) break;
    }
    groups = 0;
    return 0;
}

struct RlArgs {
    const float *LU;
    int n;
    long sA;
    const int *perm;
    const float *Dinv;
    const double *R;
    int nrhs;
    long sR;
    double *X;
    const int *conv;
    unsigned long long *dmb, *xmb;
    float2 *D;
    int dmode, nd, groups;
};

template <int CG>
static void launch_rl_cg(const RlArgs &a, cudaStream_t st) {
    const size_t sm = rl_smem_bytes(a.n, CG);
    PDD_CUDA(cudaFuncSetAttribute(k_lu_solve_rl<CG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    PDD_LAUNCH(k_lu_solve_rl<CG>, dim3(a.nd, a.groups), kRlThreads, sm, st, a.LU, a.n, a.sA, a.perm, a.Dinv, a.R,
               a.nrhs, a.sR, a.X, a.conv, a.dmb, a.xmb, a.D, a.dmode);
}

static void launch_rl(int W, const RlArgs &a, cudaStream_t st) {
    switch (W) {
        case 8: launch_rl_cg<8>(a, st); break;
        case 12: launch_rl_cg<12>(a, st); break;
        case 17: launch_rl_cg<17>(a, st); break;
        case 20: launch_rl_cg<20>(a, st); break;
        case 36: launch_rl_cg<36>(a, st); break;
        default: launch_rl_cg<52>(a, st); break;
    }
}

__global__ void k_split_df(const double *v, float2 *out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = df_split(v[i]);
}

// R = RHS - A X in FP64 without forming A (equilibrated rows).  A block takes
// kResNP nodes; their combined radial and angular weights go to shared memory
// and the (node, column) outputs are spread over all threads of the block.
// With R1 non-null the residual is also stored as (hi, lo) FP32 pairs.  Both forms take 32 nodes
// per block (41 KB of weights for the double-float one, five blocks per SM): their FP64 and
// double-float sums are long dependent chains, so more resident warps hide their latency.
static constexpr int kResNP = 32;
static constexpr int kResNPdf = 32;

__global__ void __launch_bounds__(256) k_residual(Shape S, const NodeCoef *coefAll, long strideC,
                                                  const double *RHSall, const double *Xall,
                                                  double *Rall, long strideR, const int *conv, float2 *R1all) {
    const int disk = blockIdx.y;
    if (conv[disk]) return;
    extern __shared__ double wsm[];                 // per node: nc-1 radial + nt angular weights
    const int nw = (S.nc - 1) + S.nt, np = S.nc + 1, half = S.nt >> 1;
    const int p0 = blockIdx.x * kResNP, npb = min(kResNP, S.n - p0);
    for (int e = threadIdx.x; e < npb * nw; e += blockDim.x) {
        const int pl = e / nw, l = e - pl * nw;
        const NodeCoef cf = coefAll[disk * strideC + p0 + pl];
        const int k = (p0 + pl) / S.nt + 1;
        double v;
        if (l < S.nc - 1) {
            v = cf.alpha * S.D2[k * np + l + 1] + cf.beta * S.D[k * np + l + 1];
        } else {
            const int d = l - (S.nc - 1);
            v = cf.gamma * S.F2[d] + cf.delta * S.F1[d];
        }
        wsm[e] = v;
    }
    __syncthreads();
    const double *X = Xall + disk * strideR;
    for (int e = threadIdx.x; e < npb * S.nrhs; e += blockDim.x) {
        const int pl = e / S.nrhs, col = e - pl * S.nrhs, p = p0 + pl;
        const double *w = wsm + pl * nw;
        const NodeCoef cf = coefAll[disk * strideC + p];
        const int k = p / S.nt + 1, j = p % S.nt;
        const int jm = (j + half) % S.nt;
        double acc = cf.c * X[(long)p * S.nrhs + col];
        // the radial line and its mirror, then the ring; eight loads in flight, summed in order
        const long ls = (long)S.nt * S.nrhs;
        const double *xj = X + (long)j * S.nrhs + col, *xjm = X + (long)jm * S.nrhs + col;
        for (int l0 = 1; l0 <= S.nr; l0 += 4) {
            double a[4], bm[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = l0 + u <= S.nr;
                a[u] = ok ? xj[(l0 + u - 1) * ls] : 0.0;
                bm[u] = ok ? xjm[(l0 + u - 1) * ls] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int l = l0 + u;
                if (l <= S.nr) {
                    acc += w[l - 1] * a[u];
                    acc += w[S.nc - l - 1] * bm[u];
                }
            }
        }
        const double *wa = w + S.nc - 1;
        const double *xr = X + (long)(k - 1) * S.nt * S.nrhs + col;
        for (int jp0 = 0; jp0 < S.nt; jp0 += 8) {
            double xv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) xv[u] = jp0 + u < S.nt ? xr[(long)(jp0 + u) * S.nrhs] : 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int jp = jp0 + u;
                if (jp < S.nt) {
                    int d = j - jp;
                    d += (d < 0) ? S.nt : 0;
                    acc += wa[d] * xv[u];
                }
            }
        }
        const long o = disk * strideR + (long)p * S.nrhs + col;
        const double r = RHSall[o] - cf.s * acc;
        Rall[o] = r;
        if (R1all) R1all[o] = df_split(r);
    }
}

// Later refinement sweeps: with X = X1 + D (X1 the first solve's FP32 result,
// D the sum of the later FP32 corrections), R = R1 - A D where R1 = RHS - A X1
// came from k_residual.  |D| is about the first solve's error, so A D needs
// far fewer digits than the first residual; it is formed in double-float
// arithmetic on the FP32 pipes (FP64 runs at a small fraction of the FP32
// rate on this part).  The result is rounded to FP32, the precision in which
// the triangular solves read it.
__global__ void __launch_bounds__(256) k_residual_df(Shape S, const NodeCoef *coefAll, long strideC,
                                                     const float2 *R1all, const float2 *Dall, double *Rall,
                                                     long strideR, const int *conv) {
    const int disk = blockIdx.y;
    if (conv[disk]) return;
    extern __shared__ float2 wdf[];                 // per node: weights, then (c, s)
    const int nw = (S.nc - 1) + S.nt, np = S.nc + 1, half = S.nt >> 1;
    const int p0 = blockIdx.x * kResNPdf, npb = min(kResNPdf, S.n - p0);
    float2 *cab = wdf + (size_t)kResNPdf * nw;      // per node: alpha, beta, gamma, delta, c, s
    for (int pl = threadIdx.x; pl < npb; pl += blockDim.x) {
        const NodeCoef cf = coefAll[disk * strideC + p0 + pl];
        cab[6 * pl + 0] = df_split(cf.alpha);
        cab[6 * pl + 1] = df_split(cf.beta);
        cab[6 * pl + 2] = df_split(cf.gamma);
        cab[6 * pl + 3] = df_split(cf.delta);
        cab[6 * pl + 4] = df_split(cf.c);
        cab[6 * pl + 5] = df_split(cf.s);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < npb * nw; e += blockDim.x) {
        const int pl = e / nw, l = e - pl * nw;
        const int k = (p0 + pl) / S.nt + 1;
        const float2 *cf = cab + 6 * pl;
        float2 v;
        if (l < S.nc - 1) {
            v = df_add(df_mul(cf[0], S.D2hl[k * np + l + 1]), df_mul(cf[1], S.Dhl[k * np + l + 1]));
        } else {
            const int d = l - (S.nc - 1);
            v = df_add(df_mul(cf[2], S.F2hl[d]), df_mul(cf[3], S.F1hl[d]));
        }
        wdf[e] = v;
    }
    __syncthreads();
    const float2 *D = Dall + disk * strideR;
    for (int e = threadIdx.x; e < npb * S.nrhs; e += blockDim.x) {
        const int pl = e / S.nrhs, col = e - pl * S.nrhs, p = p0 + pl;
        const float2 *w = wdf + pl * nw;
        const int k = p / S.nt + 1, j = p % S.nt;
        const int jm = (j + half) % S.nt;
        const float2 x0 = D[(long)p * S.nrhs + col];
        const float2 c0 = df_mul(cab[6 * pl + 4], x0);
        float sh = c0.x, sl = c0.y;
        // the radial line and its mirror, then the ring; eight loads in flight, summed in order
        const long ls = (long)S.nt * S.nrhs;
        const float2 *dj = D + (long)j * S.nrhs + col, *djm = D + (long)jm * S.nrhs + col;
        for (int l0 = 1; l0 <= S.nr; l0 += 4) {
            float2 a[4], bm[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = l0 + u <= S.nr;
                a[u] = ok ? dj[(l0 + u - 1) * ls] : make_float2(0.f, 0.f);
                bm[u] = ok ? djm[(l0 + u - 1) * ls] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int l = l0 + u;
                if (l <= S.nr) {
                    df_acc(sh, sl, w[l - 1], a[u]);
                    df_acc(sh, sl, w[S.nc - l - 1], bm[u]);
                }
            }
        }
        const float2 *wa = w + S.nc - 1;
        const float2 *dr = D + (long)(k - 1) * S.nt * S.nrhs + col;
        for (int jp0 = 0; jp0 < S.nt; jp0 += 8) {
            float2 xv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                xv[u] = jp0 + u < S.nt ? dr[(long)(jp0 + u) * S.nrhs] : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int jp = jp0 + u;
                if (jp < S.nt) {
                    int d = j - jp;
                    d += (d < 0) ? S.nt : 0;
                    df_acc(sh, sl, wa[d], xv[u]);
                }
            }
        }
        const float h = sh + sl;
        const float2 ad = df_mul(cab[6 * pl + 5], make_float2(h, sl - (h - sh)));
        const long o = disk * strideR + (long)p * S.nrhs + col;
        const float2 r = df_add(R1all[o], make_float2(-ad.x, -ad.y));
        Rall[o] = (double)r.x;
    }
}

// ---------------------------------------------------------------------------
// a9: evaluate at the disk's knots and scatter into C and r
// ---------------------------------------------------------------------------
// Entry p of sub_rows (row i, this disk) writes Xi_m's block of row i at rowptr[i] + sub_off[p] and
// its part of r_i to bs[p] (rows that average several subdomains sum the parts afterwards).
__global__ void __launch_bounds__(256) k_disk_eval(Shape S, const DiskDesc *disks, const int *sub_rows,
                                                   const int *sub_off, const double *kx, const double *ky,
                                                   const int *rowptr, const double *Xall,
                                                   long strideR, int group, int per, double *val,
                                                   double *bs) {
    extern __shared__ double esm[];                 // per rows x (n + nt) evaluation weights
    __shared__ double lr[8][130];                   // radial barycentric weights, l = 0..nc
    __shared__ double sa[8][130];                   // angular cardinals at the grid angles
    const int disk = blockIdx.x, tid = threadIdx.x;
    const DiskDesc dd = disks[disk];
    const double *X = Xall + disk * strideR;
    const int nE = S.n + S.nt, half = S.nt >> 1;
    const int gid = tid / group, gl = tid % group;
    const bool in_group = gid < per;
    for (int r0 = dd.row_begin; r0 < dd.row_end; r0 += per) {
        const int row = r0 + gid;
        const bool active = in_group && row < dd.row_end;
        double *E = esm + gid * nE;
        double rho = 0.0;
        if (active) {
            const int i = sub_rows[row];
            const double dx = kx[i] - dd.cx, dy = ky[i] - dd.cy;
            rho = sqrt(dx * dx + dy * dy) / dd.R;
            const double phi = atan2(dy, dx);
            for (int l = gl; l <= S.nc; l += group) {
                const double wl = ((l & 1) ? -1.0 : 1.0) * ((l == 0 || l == S.nc) ? 0.5 : 1.0);
                const double d = rho - S.x[l];
                lr[gid][l] = (d == 0.0) ? 0.0 : wl / d;
            }
            for (int a = gl; a < S.nt; a += group)
                sa[gid][a] = fourier_cardinal_cf(phi - PDD_TWO_PI * a / S.nt, S.nt);
        }
        __syncthreads();
        if (active && gl == 0) {                    // normalise (barycentric formula, 2nd kind)
            int hit = -1;
            double den = 0.0;
            for (int l = 0; l <= S.nc; ++l) {
                if (rho == S.x[l]) hit = l;
                den += lr[gid][l];
            }
            for (int l = 0; l <= S.nc; ++l)
                lr[gid][l] = (hit >= 0) ? (l == hit ? 1.0 : 0.0) : lr[gid][l] / den;
        }
        __syncthreads();
        if (active) {
            // E[k][a] = l_{k+1} S_a + l_{nc-1-k} S_{a+half};  E_B[a] = l_0 S_a + l_nc S_{a+half}
            for (int q = gl; q < nE; q += group) {
                if (q < S.n) {
                    const int kk = q / S.nt, a = q - kk * S.nt;
                    E[q] = lr[gid][kk + 1] * sa[gid][a] + lr[gid][S.nc - 1 - kk] * sa[gid][(a + half) % S.nt];
                } else {
                    const int a = q - S.n;
                    E[q] = lr[gid][0] * sa[gid][a] + lr[gid][S.nc] * sa[gid][(a + half) % S.nt];
                }
            }
        }
        __syncthreads();
        if (active) {
            const int i = sub_rows[row];
            for (int col = gl; col < S.nrhs; col += group) {
                double acc = 0.0;
                for (int q = 0; q < S.n; ++q) acc += E[q] * X[(long)q * S.nrhs + col];
                if (col < S.nk) {
                    // boundary ring: G_j = -H_j on the circle
                    for (int a = 0; a < S.nt; ++a) acc -= E[S.n + a] * S.Hg[a * S.nk + col];
                    val[rowptr[i] + sub_off[row] + col] = acc;
                } else {
                    bs[row] = acc;
                }
            }
        }
        __syncthreads();
    }
}

// mixed form: the same evaluation with the 1024-term sums in double-float
// arithmetic (the weights are built in FP64 and split; X comes split by
// k_split_x).  A block takes one disk, its knots eight at a time; the
// (knot, column) outputs are spread over all threads.
static constexpr int kEvalKnots = 8;

__global__ void k_split_x(long count, const double *X, float2 *Xhl) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < count; e += (long)gridDim.x * blockDim.x)
        Xhl[e] = df_split(X[e]);
}

__global__ void __launch_bounds__(256) k_disk_eval_df(Shape S, const DiskDesc *disks, const int *sub_rows,
                                                      const int *sub_off, const double *kx, const double *ky,
                                                      const int *rowptr, const float2 *Xhl, long strideR, int kper,
                                                      double *val, double *bs) {
    extern __shared__ float2 edf[];                 // kper (<= kEvalKnots) x (n + nt) weights
    __shared__ double lr[kEvalKnots][130];          // radial barycentric weights, l = 0..nc
    __shared__ double sa[kEvalKnots][130];          // angular cardinals at the grid angles
    __shared__ double rho_s[kEvalKnots];
    const int disk = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const DiskDesc dd = disks[disk];
    const float2 *X = Xhl + disk * strideR;
    const int nE = S.n + S.nt, half = S.nt >> 1;
    for (int r0 = dd.row_begin; r0 < dd.row_end; r0 += kper) {
        const int nkn = min(kper, dd.row_end - r0);
        // radial and angular weights of each knot: warp g takes knot g
        if (warp < nkn) {
            const int i = sub_rows[r0 + warp];
            const double dx = kx[i] - dd.cx, dy = ky[i] - dd.cy;
            const double rho = sqrt(dx * dx + dy * dy) / dd.R;
            const double phi = atan2(dy, dx);
            for (int l = lane; l <= S.nc; l += 32) {
                const double wl = ((l & 1) ? -1.0 : 1.0) * ((l == 0 || l == S.nc) ? 0.5 : 1.0);
                const double d = rho - S.x[l];
                lr[warp][l] = (d == 0.0) ? 0.0 : wl / d;
            }
            for (int a = lane; a < S.nt; a += 32) sa[warp][a] = fourier_cardinal_cf(phi - PDD_TWO_PI * a / S.nt, S.nt);
            if (lane == 0) rho_s[warp] = rho;
        }
        __syncthreads();
        if (warp < nkn && lane == 0) {             // normalise (barycentric formula, 2nd kind)
            const double rho = rho_s[warp];
            int hit = -1;
            double den = 0.0;
            for (int l = 0; l <= S.nc; ++l) {
                if (rho == S.x[l]) hit = l;
                den += lr[warp][l];
            }
            for (int l = 0; l <= S.nc; ++l)
                lr[warp][l] = (hit >= 0) ? (l == hit ? 1.0 : 0.0) : lr[warp][l] / den;
        }
        __syncthreads();
        // E[k][a] = l_{k+1} S_a + l_{nc-1-k} S_{a+half};  E_B[a] = l_0 S_a + l_nc S_{a+half}
        for (int e = tid; e < nkn * nE; e += blockDim.x) {
            const int g = e / nE, q = e - g * nE;
            double v;
            if (q < S.n) {
                const int kk = q / S.nt, a = q - kk * S.nt;
                v = lr[g][kk + 1] * sa[g][a] + lr[g][S.nc - 1 - kk] * sa[g][(a + half) % S.nt];
            } else {
                const int a = q - S.n;
                v = lr[g][0] * sa[g][a] + lr[g][S.nc] * sa[g][(a + half) % S.nt];
            }
            edf[e] = df_split(v);
        }
        __syncthreads();
        for (int o = tid; o < nkn * S.nrhs; o += blockDim.x) {
            const int g = o / S.nrhs, col = o - g * S.nrhs;
            const float2 *E = edf + g * nE;
            float sh = 0.f, sl = 0.f;
            const float2 *xc = X + col;
            for (int q0 = 0; q0 < S.n; q0 += 8) {             // eight loads in flight
                float2 xv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    xv[u] = q0 + u < S.n ? xc[(long)(q0 + u) * S.nrhs] : make_float2(0.f, 0.f);
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (q0 + u < S.n) df_acc(sh, sl, E[q0 + u], xv[u]);
            }
            const int i = sub_rows[r0 + g];
            if (col < S.nk) {
                // boundary ring: G_j = -H_j on the circle
                for (int a = 0; a < S.nt; ++a) {
                    const float2 hg = S.Hghl[a * S.nk + col];
                    df_acc(sh, sl, E[S.n + a], make_float2(-hg.x, -hg.y));
                }
                val[rowptr[i] + sub_off[r0 + g] + col] = (double)sh + (double)sl;
            } else {
                bs[r0 + g] = (double)sh + (double)sl;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
struct ShapeTables {
    DevBuf<double> x, D, D2, F1, F2, Hg;
    DevBuf<float2> Dhl, D2hl, F1hl, F2hl, Hghl;
    Shape S{};
    void build(int nr, int nt, int nk, cudaStream_t st) {
        const int nc = 2 * nr + 1, np = nc + 1;
        x.alloc(np);
        D.alloc((size_t)np * np);
        D2.alloc((size_t)np * np);
        F1.alloc(nt);
        F2.alloc(nt);
        Hg.alloc((size_t)nt * nk);
        PDD_CUDA(cudaMemsetAsync(D.p, 0, sizeof(double) * np * np, st));
        PDD_LAUNCH(k_shape_tables, 1, 256, 0, st, nr, nt, nk, x.p, D.p, F1.p, F2.p, Hg.p);
        PDD_LAUNCH(k_matmul_sq, cdiv((long)np * np, 256), 256, 0, st, D.p, D2.p, np);
        Dhl.alloc((size_t)np * np);
        D2hl.alloc((size_t)np * np);
        F1hl.alloc(nt);
        F2hl.alloc(nt);
        PDD_LAUNCH(k_split_df, cdiv((long)np * np, 256), 256, 0, st, D.p, Dhl.p, np * np);
        PDD_LAUNCH(k_split_df, cdiv((long)np * np, 256), 256, 0, st, D2.p, D2hl.p, np * np);
        PDD_LAUNCH(k_split_df, cdiv(nt, 256), 256, 0, st, F1.p, F1hl.p, nt);
        PDD_LAUNCH(k_split_df, cdiv(nt, 256), 256, 0, st, F2.p, F2hl.p, nt);
        Hghl.alloc((size_t)nt * nk);
        PDD_LAUNCH(k_split_df, cdiv(nt * nk, 256), 256, 0, st, Hg.p, Hghl.p, nt * nk);
        S = Shape{nr, nt, nk, nc, nr * nt, nk + 1, x.p, D.p, D2.p, F1.p, F2.p, Hg.p,
                  Dhl.p, D2hl.p, F1hl.p, F2hl.p, Hghl.p};
    }
};

static int lu_nb(int n, size_t elem) {
    // panel n x (NB + 1) plus an NB x 64 tile must fit in ~200 KB of shared memory
    int nb = 32;
    while (nb > 4 && ((size_t)n * (nb + 1) + (size_t)nb * 64) * elem > 200 * 1024) nb >>= 1;
    return nb;
}

template <typename T>
static void launch_lu(T *A, int n, long strideA, int *perm, int *info, int nd, cudaStream_t st) {
    const int nb = lu_nb(n, sizeof(T));
    const size_t smem = ((size_t)n * (nb + 1) + (size_t)nb * 64) * sizeof(T);
    switch (nb) {
#define PDD_LU_CASE(NBV)                                                                      \
    case NBV:                                                                                  \
        PDD_CUDA(cudaFuncSetAttribute(k_lu<T, NBV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                      (int)smem));                                            \
        PDD_LAUNCH((k_lu<T, NBV>), nd, 256, smem, st, A, n, strideA, perm, info);              \
        break;
        PDD_LU_CASE(32)
        PDD_LU_CASE(16)
        PDD_LU_CASE(8)
        PDD_LU_CASE(4)
#undef PDD_LU_CASE
        default: fail(PDD_EINVAL, "disk grid too large for the panel kernel");
    }
}

// ---------------------------------------------------------------------------
// Autotuner of the mixed-form LU: on the first wave of each grid size n, the
// candidates (one-CTA blocked LU; recursive LU with leaf width 32/16/8 and a
// tensor-core threshold of 64 or 128) are timed with CUDA events on a copy
// of up to 64 of the wave's matrices; the fastest is kept for the process.
// ---------------------------------------------------------------------------
void lu_nopivot_f32(float *A, int n, long strideA, int *perm, int *info, int nd, float *inv, long sInv,
                    float *scratch, size_t scratch_floats, cudaStream_t st, DiskStats *ds);
long lu_np_inv_floats(int n);
size_t lu_np_scratch_floats_per_disk(int n);

struct LuChoice {
    int blocked, W, tmin;
    float ms;
};
static std::map<int, LuChoice> g_lu_choice;
static std::mutex g_lu_mu;

static void run_lu_choice(const LuChoice &c, float *A, int n, long sA, int *perm, int *info, int nd, cudaStream_t st,
                          float *ms_gemm = nullptr, double *gemm_flop = nullptr) {
    if (c.blocked) launch_lu<float>(A, n, sA, perm, info, nd, st);
    else lu_recursive_f32(A, n, sA, perm, info, nd, st, c.W, c.tmin, ms_gemm, gemm_flop);
}

static LuChoice tune_lu(float *A, int n, long sA, int nd, cudaStream_t st) {
    {
        std::lock_guard<std::mutex> lk(g_lu_mu);
        auto it = g_lu_choice.find(n);
        if (it != g_lu_choice.end()) return it->second;
    }
    std::vector<LuChoice> cand{{1, 0, 0, 0.f}};
    for (int W : {32, 16, 8})
        if ((size_t)n * ((W + 1) * sizeof(float) + sizeof(int)) <= 200 * 1024)
            for (int tmin : {32, 64, 128}) cand.push_back({0, W, tmin, 0.f});
    const int nt = std::min(nd, 304);           // two disks per SM: the occupancy of a full wave
    DevBuf<float> pristine, work;
    DevBuf<int> perm, info;
    pristine.alloc((size_t)nt * sA);
    work.alloc((size_t)nt * sA);
    perm.alloc((size_t)nt * n);
    info.alloc(nt);
    PDD_CUDA(cudaMemcpyAsync(pristine.p, A, sizeof(float) * nt * sA, cudaMemcpyDeviceToDevice, st));
    StageTimer tm(st, 2);
    LuChoice best{1, 0, 0, 1e30f};
    for (auto &c : cand) {
        float t = 0.f;
        for (int rep = 0; rep < 2; ++rep) {           // the first run warms the code paths
            PDD_CUDA(cudaMemcpyAsync(work.p, pristine.p, sizeof(float) * nt * sA, cudaMemcpyDeviceToDevice, st));
            tm.mark(0);
            run_lu_choice(c, work.p, n, sA, perm.p, info.p, nt, st);
            tm.mark(1);
            PDD_CUDA(cudaStreamSynchronize(st));
            t = tm.ms(0, 1);
        }
        c.ms = t;
        if (t < best.ms) best = c;
    }
    std::lock_guard<std::mutex> lk(g_lu_mu);
    g_lu_choice[n] = best;
    return best;
}

template <typename T>
static DiskStats run_group(const pdd_cover &cov, const Problem &P, const pdd_assembly_opts &o,
                           pdd_system &sys, const ShapeTables &tab, const std::vector<DiskDesc> &disks,
                           cudaStream_t st) {
    const Shape S = tab.S;
    const bool mixed = sizeof(T) == 4;
    const size_t perA = (size_t)S.n * S.n * sizeof(T);
    const size_t perR = (size_t)S.n * S.nrhs * sizeof(double);
    int rl_groups = 0;
    const int rlW = mixed ? rl_width(S.n, S.nrhs, rl_groups) : 0;
    const int nblk = (S.n + kRlTB - 1) / kRlTB;
    const size_t perDinv = rlW ? (size_t)nblk * 2 * kRlTB * kRlTB * sizeof(float) + 2 * perR + perA : 0;
    const bool use_np = mixed && o.factor == PDD_FACTOR_RECURSIVE_TC && o.lu_leaf_width == 0 && S.n > 64;
    const size_t perNp = use_np ? (size_t)lu_np_inv_floats(S.n) * sizeof(float) : 0;
    const size_t perDisk = perA + perR * (mixed ? 3 : 1) + (size_t)S.n * S.nrhs * sizeof(T) +
                           (size_t)S.n * sizeof(NodeCoef) + (size_t)S.n * sizeof(int) + perDinv + perNp + 64;
    size_t freeb = 0, totb = 0;
    PDD_CUDA(cudaMemGetInfo(&freeb, &totb));
    size_t budget = std::min<size_t>((size_t)(0.6 * freeb), (size_t)64 << 30);
    if (use_np) {           // the GEMM tile scratch comes out of the same budget
        const size_t scr = lu_np_scratch_floats_per_disk(S.n) * sizeof(float) *
                           std::min<size_t>(disks.size(), 256);
        budget = budget > 2 * scr ? budget - scr : budget / 2;
    }
    int wave = (int)std::max<size_t>(1, budget / perDisk);
    wave = std::min<int>(wave, (int)disks.size());
    if ((size_t)wave * perDisk > freeb) fail(PDD_ENOMEM, "not enough device memory for one disk");
    {
        // equal waves, as many as fill the SMs in the fewest rounds: the kernels that take one CTA
        // per disk (the triangular solves, one per SM; the leaf blocks, four) otherwise leave the
        // last round of every wave part empty.  From the fewest waves memory allows to two more.
        int dev = 0, sms = 0;
        PDD_CUDA(cudaGetDevice(&dev));
        PDD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const long total = (long)disks.size(), nw0 = (total + wave - 1) / wave;
        long best = wave, best_rounds = -1;
        for (long nw = nw0; nw <= std::min(nw0 + 2, total); ++nw) {
            const long w = (total + nw - 1) / nw, rounds = nw * ((w + sms - 1) / sms);
            if (best_rounds < 0 || rounds < best_rounds) {
                best_rounds = rounds;
                best = w;
            }
        }
        wave = (int)best;
    }
    DevBuf<T> A, W;
    DevBuf<double> RHS, X, Rr;
    DevBuf<NodeCoef> coef;
    DevBuf<int> perm, info, conv, sweeps;
    DevBuf<DiskDesc> dd;
    DevBuf<float> dinv, AT;
    DevBuf<unsigned long long> dmaxb, xmaxb;
    DevBuf<double> dprev;
    DevBuf<float2> R1hl, Dhl;
    if (rlW) {
        dinv.alloc((size_t)wave * nblk * 2 * kRlTB * kRlTB);
        AT.alloc((size_t)wave * S.n * S.n);
        dmaxb.alloc(wave);
        xmaxb.alloc(wave);
        dprev.alloc(wave);
        R1hl.alloc((size_t)wave * S.n * S.nrhs);
        Dhl.alloc((size_t)wave * S.n * S.nrhs);
    }
    A.alloc((size_t)wave * S.n * S.n);
    W.alloc((size_t)wave * S.n * S.nrhs);
    RHS.alloc((size_t)wave * S.n * S.nrhs);
    X.alloc((size_t)wave * S.n * S.nrhs);
    if (mixed) Rr.alloc((size_t)wave * S.n * S.nrhs);
    coef.alloc((size_t)wave * S.n);
    perm.alloc((size_t)wave * S.n);
    info.alloc(wave);
    conv.alloc(wave);
    sweeps.alloc(wave);
    dd.alloc(wave);
    // pivot-free LU: inverses of the 64 x 64 diagonal blocks and the GEMMs' hi/lo tile scratch
    // (enough for min(wave, 256) disks of the largest update; larger waves run in chunks)
    DevBuf<float> npinv, npscr;
    const long np_inv_per = use_np ? lu_np_inv_floats(S.n) : 0;
    size_t np_scr_floats = 0;
    if (use_np) {
        npinv.alloc((size_t)wave * np_inv_per);
        np_scr_floats = lu_np_scratch_floats_per_disk(S.n) * (size_t)std::min(wave, 256);
        npscr.alloc(std::max<size_t>(np_scr_floats, 1));
    }
    const long sA = (long)S.n * S.n, sR = (long)S.n * S.nrhs, sC = S.n;
    DiskStats ds;
    for (size_t w0 = 0; w0 < disks.size(); w0 += wave) {
        const int nd = (int)std::min<size_t>(wave, disks.size() - w0);
        for (int attempt = 0; attempt < 2; ++attempt) {
        DiskStats wv;                                   // this wave's statistics (kept on success)
        PDD_CUDA(cudaMemcpyAsync(dd.p, disks.data() + w0, nd * sizeof(DiskDesc), cudaMemcpyHostToDevice, st));
        StageTimer tm(st, 5);
        tm.mark(0);
        build_operator<T>(P, S, dd.p, nd, A.p, sA, RHS.p, sR, coef.p, sC, st);
        tm.mark(1);
        bool np_used = false;
        if constexpr (sizeof(T) == 4) {
            if (use_np && attempt == 0) {
                // pivot-free tensor-core LU; a pivot below the threshold sends the wave to the
                // pivoted factorisation (the operator is rebuilt: the factor overwrote it)
                lu_nopivot_f32(A.p, S.n, sA, perm.p, info.p, nd, npinv.p, np_inv_per, npscr.p, np_scr_floats, st,
                               &wv);
                std::vector<int> hi(nd);
                PDD_CUDA(cudaMemcpyAsync(hi.data(), info.p, nd * sizeof(int), cudaMemcpyDeviceToHost, st));
                PDD_CUDA(cudaStreamSynchronize(st));
                np_used = std::all_of(hi.begin(), hi.end(), [](int v) { return v == 0; });
                if (!np_used) {
                    wv.ms_tc_gemm = 0.f;
                    wv.tc_gemm_flop = 0.0;
                    wv.ms_gemm_fused = 0.f;
                    wv.gemm_fused_flop = wv.gemm_fused_bytes = 0.0;
                    wv.gemm_pipe_launches = 0;
                    build_operator<T>(P, S, dd.p, nd, A.p, sA, RHS.p, sR, coef.p, sC, st);
                }
            }
            if (np_used) {
                wv.lu_blocked = 0;
                wv.lu_leaf = 64;
                wv.lu_tmin = 0;
            } else if (o.factor == PDD_FACTOR_BLOCKED) {
                launch_lu<T>(A.p, S.n, sA, perm.p, info.p, nd, st);
                wv.lu_blocked = 1;
            } else if (o.lu_leaf_width > 0) {
                const LuChoice c{0, o.lu_leaf_width, o.lu_tensor_min > 0 ? o.lu_tensor_min : 128, 0.f};
                run_lu_choice(c, A.p, S.n, sA, perm.p, info.p, nd, st, &wv.ms_tc_gemm, &wv.tc_gemm_flop);
                wv.lu_blocked = 0;
                wv.lu_leaf = c.W;
                wv.lu_tmin = c.tmin;
            } else {
                const LuChoice c = tune_lu(A.p, S.n, sA, nd, st);       // cached after the first wave
                if (!use_np) tm.mark(1);                               // factor time excludes tuning
                run_lu_choice(c, A.p, S.n, sA, perm.p, info.p, nd, st, &wv.ms_tc_gemm, &wv.tc_gemm_flop);
                wv.lu_blocked = c.blocked;
                wv.lu_leaf = c.W;
                wv.lu_tmin = c.tmin;
            }
            if (use_np && !np_used) wv.lu_fallback = 1;
        } else {
            launch_lu<T>(A.p, S.n, sA, perm.p, info.p, nd, st);
        }
        if (rlW) {
            const long items = (long)nd * nblk * 2;
            PDD_LAUNCH(k_diag_inv, (int)((items + 3) / 4), 128, 0, st, reinterpret_cast<const float *>(A.p), S.n, sA,
                       nd, dinv.p);
            if ((S.n & 3) == 0)       // rows and disks start on 16-byte boundaries (cudaMalloc'd buffers)
                PDD_LAUNCH(k_transpose_f32_v4, dim3(cdiv(S.n, 64), cdiv(S.n, 64), nd), 256, 0, st,
                           reinterpret_cast<const float *>(A.p), AT.p, S.n, sA);
            else
                PDD_LAUNCH(k_transpose_f32, dim3(cdiv(S.n, 32), cdiv(S.n, 32), nd), 256, 0, st,
                           reinterpret_cast<const float *>(A.p), AT.p, S.n, sA);
        }
        tm.mark(2);
        if (!mixed) {
            launch_solve<T>(A.p, S.n, sA, perm.p, RHS.p, S.nrhs, sR, W.p, X.p, 0, nullptr, nullptr, 0.0, nd, st);
        } else {
            PDD_CUDA(cudaMemsetAsync(conv.p, 0, nd * sizeof(int), st));
            PDD_CUDA(cudaMemsetAsync(sweeps.p, 0, nd * sizeof(int), st));
            PDD_CUDA(cudaMemsetAsync(X.p, 0, (size_t)nd * sR * sizeof(double), st));
            const int maxs = std::max(1, o.max_refine);
            const double tol = o.refine_tol > 0 ? o.refine_tol : 1e-12;
            const int nw = (S.nc - 1) + S.nt;
            const size_t rsm = (size_t)kResNP * nw * sizeof(double);
            const size_t rsm_df = ((size_t)kResNPdf * nw + 6 * kResNPdf) * sizeof(float2);
            PDD_CUDA(cudaFuncSetAttribute(k_residual, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
            PDD_CUDA(cudaFuncSetAttribute(k_residual_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm_df));
            dim3 g_res(cdiv(S.n, kResNP), nd), g_res_df(cdiv(S.n, kResNPdf), nd);
            std::vector<cudaEvent_t> sev(rlW ? 2 * maxs : 0);
            for (cudaEvent_t &e : sev) PDD_CUDA(cudaEventCreate(&e));
            struct EvFree {
                std::vector<cudaEvent_t> &v;
                ~EvFree() {
                    for (cudaEvent_t e : v) cudaEventDestroy(e);
                }
            } ev_free{sev};
            if (rlW) {
                PDD_CUDA(cudaMemsetAsync(dmaxb.p, 0, nd * sizeof(unsigned long long), st));
                PDD_CUDA(cudaMemsetAsync(xmaxb.p, 0, nd * sizeof(unsigned long long), st));
            }
            for (int s = 0; s < maxs; ++s) {
                const double *rhs_now = (s == 0) ? RHS.p : Rr.p;
                if (rlW) {
                    const RlArgs ra{AT.p, S.n, sA, perm.p, dinv.p, rhs_now, S.nrhs, sR,
                                    X.p, conv.p, dmaxb.p, xmaxb.p, Dhl.p, s == 0 ? 0 : (s == 1 ? 1 : 2), nd,
                                    rl_groups};
                    PDD_CUDA(cudaEventRecord(sev[2 * s], st));
                    launch_rl(rlW, ra, st);
                    PDD_CUDA(cudaEventRecord(sev[2 * s + 1], st));
                    PDD_LAUNCH(k_refine_conv, cdiv(nd, 256), 256, 0, st, nd, conv.p, sweeps.p, dmaxb.p, xmaxb.p, dprev.p,
                               tol);
                    if (s + 1 < maxs) {
                        if (s == 0)
                            PDD_LAUNCH(k_residual, g_res, 256, rsm, st, S, coef.p, sC, RHS.p, X.p, Rr.p, sR, conv.p,
                                       R1hl.p);
                        else
                            PDD_LAUNCH(k_residual_df, g_res_df, 256, rsm_df, st, S, coef.p, sC, R1hl.p, Dhl.p, Rr.p, sR,
                                       conv.p);
                    }
                } else {
                    launch_solve<T>(A.p, S.n, sA, perm.p, rhs_now, S.nrhs, sR, W.p, X.p, 1, conv.p, sweeps.p, tol,
                                    nd, st);
                    if (s + 1 < maxs)
                        PDD_LAUNCH(k_residual, g_res, 256, rsm, st, S, coef.p, sC, RHS.p, X.p, Rr.p, sR, conv.p,
                                   (float2 *)nullptr);
                }
            }
            tm.mark(3);
            std::vector<int> hc(nd), hs(nd);
            PDD_CUDA(cudaMemcpyAsync(hc.data(), conv.p, nd * sizeof(int), cudaMemcpyDeviceToHost, st));
            PDD_CUDA(cudaMemcpyAsync(hs.data(), sweeps.p, nd * sizeof(int), cudaMemcpyDeviceToHost, st));
            PDD_CUDA(cudaStreamSynchronize(st));
            for (int d = 0; d < nd; ++d) {
                wv.max_sweeps = std::max(wv.max_sweeps, hs[d]);
                wv.unconverged += hc[d] ? 0 : 1;
                wv.disk_solves += hs[d];
            }
            if (rlW)
                for (int s = 0; s < maxs; ++s) {
                    float t = 0.f;
                    cudaEventElapsedTime(&t, sev[2 * s], sev[2 * s + 1]);
                    wv.ms_trisolve += t;
                }
        }
        if (!mixed) tm.mark(3);
        if (S.nc + 1 > 130 || S.nt > 130) fail(PDD_EINVAL, "disk grid too large for the evaluation kernel");
        if (rlW) {
            // mixed form: double-float sums on X split into FP32 pairs (the correction buffer is free now)
            const long cnt = (long)nd * sR;
            PDD_LAUNCH(k_split_x, (int)std::min<long>(cdiv(cnt, 256), 4096), 256, 0, st, cnt, X.p, Dhl.p);
            const size_t rowdf = (size_t)(S.n + S.nt) * sizeof(float2);
            // knots per pass: all (knot, column) outputs of a pass in one sweep of the 256 threads
            const int kper = (int)std::min<size_t>(std::max(1, std::min(kEvalKnots, 256 / S.nrhs)), (200 * 1024) / rowdf);
            if (kper < 1) fail(PDD_EINVAL, "disk grid too large for the evaluation kernel");
            const size_t esm = kper * rowdf;
            PDD_CUDA(cudaFuncSetAttribute(k_disk_eval_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)esm));
            PDD_LAUNCH(k_disk_eval_df, nd, 256, esm, st, S, dd.p, cov.sub_rows.p, cov.sub_off.p, cov.kx.p, cov.ky.p,
                       cov.rowptr.p, Dhl.p, sR, kper, sys.val.p, sys.bs.p);
        } else {
            const int group = (S.nrhs <= 32) ? 32 : ((S.nrhs <= 64) ? 64 : 128);
            const size_t rowb = (size_t)(S.n + S.nt) * sizeof(double);
            const int per = (int)std::min<size_t>(256 / group, (180 * 1024) / rowb);
            if (per < 1) fail(PDD_EINVAL, "disk grid too large for the evaluation kernel");
            const size_t esm = per * rowb;
            PDD_CUDA(cudaFuncSetAttribute(k_disk_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)esm));
            PDD_LAUNCH(k_disk_eval, nd, 256, esm, st, S, dd.p, cov.sub_rows.p, cov.sub_off.p, cov.kx.p, cov.ky.p,
                       cov.rowptr.p, X.p, sR, group, per, sys.val.p, sys.bs.p);
        }
        tm.mark(4);
        std::vector<int> hinfo(nd);
        PDD_CUDA(cudaMemcpyAsync(hinfo.data(), info.p, nd * sizeof(int), cudaMemcpyDeviceToHost, st));
        PDD_CUDA(cudaStreamSynchronize(st));
        // a pivot-free factorisation whose refinement missed the tolerance: redo the wave pivoted
        if (np_used && wv.unconverged > 0) {
            ds.lu_fallback = 1;
            continue;
        }
        ds.ms_operator += tm.ms(0, 1);
        ds.ms_factor += tm.ms(1, 2);
        ds.ms_refine += tm.ms(2, 3);
        ds.ms_eval += tm.ms(3, 4);
        ds.ms_tc_gemm += wv.ms_tc_gemm;
        ds.tc_gemm_flop += wv.tc_gemm_flop;
        ds.ms_gemm_fused += wv.ms_gemm_fused;
        ds.gemm_fused_flop += wv.gemm_fused_flop;
        ds.gemm_fused_bytes += wv.gemm_fused_bytes;
        ds.gemm_pipe_launches += wv.gemm_pipe_launches;
        ds.ms_trisolve += wv.ms_trisolve;
        ds.max_sweeps = std::max(ds.max_sweeps, wv.max_sweeps);
        ds.unconverged += wv.unconverged;
        ds.disk_solves += wv.disk_solves;
        ds.lu_blocked = wv.lu_blocked;
        ds.lu_leaf = wv.lu_leaf;
        ds.lu_tmin = wv.lu_tmin;
        ds.lu_fallback |= wv.lu_fallback;
        for (int d = 0; d < nd; ++d)
            if (hinfo[d] && !np_used) fail(PDD_ENOCONV, "singular collocation matrix");
        ds.disks += nd;
        for (int d = 0; d < nd; ++d) ds.rows += disks[w0 + d].row_end - disks[w0 + d].row_begin;
        break;
        }
    }
    return ds;
}

DiskStats assemble_disks(const pdd_cover &cov, const Problem &P, const pdd_assembly_opts &o,
                         pdd_system &sys, cudaStream_t st) {
    std::map<std::tuple<int, int, int>, std::vector<DiskDesc>> groups;
    std::vector<double> hcx(cov.M), hcy(cov.M), hr(cov.M);
    PDD_CUDA(cudaMemcpyAsync(hcx.data(), cov.cx.p, cov.M * 8, cudaMemcpyDeviceToHost, st));
    PDD_CUDA(cudaMemcpyAsync(hcy.data(), cov.cy.p, cov.M * 8, cudaMemcpyDeviceToHost, st));
    PDD_CUDA(cudaMemcpyAsync(hr.data(), cov.r.p, cov.M * 8, cudaMemcpyDeviceToHost, st));
    PDD_CUDA(cudaStreamSynchronize(st));
    for (int m = 0; m < cov.M; ++m) {
        if (!cov.h_floating[m]) continue;
        int a = cov.h_sub_ptr[m], b = cov.h_sub_ptr[m + 1];
        if (b <= a) continue;
        if (cov.h_knot_ptr[m + 1] - cov.h_knot_ptr[m] != cov.h_nk[m]) fail(PDD_EINVAL, "floating circle lost knots");
        groups[{cov.h_nr[m], cov.h_nt[m], cov.h_nk[m]}].push_back(
            DiskDesc{hcx[m], hcy[m], hr[m], m, cov.h_knot_ptr[m], a, b});
    }
    DiskStats all;
    for (auto &kv : groups) {
        ShapeTables tab;
        tab.build(std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first), st);
        DiskStats d = disk_mixed(o)
                          ? run_group<float>(cov, P, o, sys, tab, kv.second, st)
                          : run_group<double>(cov, P, o, sys, tab, kv.second, st);
        all.disks += d.disks;
        all.rows += d.rows;
        all.max_sweeps = std::max(all.max_sweeps, d.max_sweeps);
        all.unconverged += d.unconverged;
        all.ms_operator += d.ms_operator;
        all.ms_factor += d.ms_factor;
        all.ms_refine += d.ms_refine;
        all.ms_eval += d.ms_eval;
        all.ms_trisolve += d.ms_trisolve;
        all.ms_tc_gemm += d.ms_tc_gemm;
        all.ms_gemm_fused += d.ms_gemm_fused;
        all.gemm_fused_flop += d.gemm_fused_flop;
        all.gemm_fused_bytes += d.gemm_fused_bytes;
        all.gemm_pipe_launches += d.gemm_pipe_launches;
        all.disk_solves += d.disk_solves;
        all.tc_gemm_flop += d.tc_gemm_flop;
        if (d.lu_leaf || d.lu_blocked) {
            all.lu_blocked = d.lu_blocked;
            all.lu_leaf = d.lu_leaf;
            all.lu_tmin = d.lu_tmin;
        }
        all.lu_fallback |= d.lu_fallback;
    }
    return all;
}

}  // namespace pdd

// ---------------------------------------------------------------------------
// a14 (floating rows): with V the disk solution for the interface data of u
// (V = B - sum_j u_j G_j) and A^T z = sum_i lambda_i E_i, the weights of c
// get -sum_p z_p V_p 1{c<0} psi_q(x_p).  FP64 throughout; factors recomputed.
// ---------------------------------------------------------------------------
namespace pdd {

__global__ void __launch_bounds__(256) k_adjoint_vecs(Shape S, const DiskDesc *disks, const int *sub_rows,
                                                      const double *kx, const double *ky, const double *Xall,
                                                      long strideR, const double *u, const double *lambda,
                                                      double *Vall, double *Eall) {
    __shared__ double lr[130], sa[130];
    const int disk = blockIdx.x, tid = threadIdx.x;
    const DiskDesc dd = disks[disk];
    const double *X = Xall + disk * strideR;
    double *V = Vall + (long)disk * S.n, *E = Eall + (long)disk * S.n;
    const int half = S.nt >> 1;
    for (int p = tid; p < S.n; p += 256) {
        double v = X[(long)p * S.nrhs + S.nk];
        for (int c = 0; c < S.nk; ++c) v -= u[dd.knot_base + c] * X[(long)p * S.nrhs + c];
        V[p] = v;
        E[p] = 0.0;
    }
    for (int row = dd.row_begin; row < dd.row_end; ++row) {
        const int i = sub_rows[row];
        const double dx = kx[i] - dd.cx, dy = ky[i] - dd.cy;
        const double rho = sqrt(dx * dx + dy * dy) / dd.R, phi = atan2(dy, dx);
        __syncthreads();
        for (int l = tid; l <= S.nc; l += 256) {
            const double wl = ((l & 1) ? -1.0 : 1.0) * ((l == 0 || l == S.nc) ? 0.5 : 1.0);
            const double d = rho - S.x[l];
            lr[l] = (d == 0.0) ? 0.0 : wl / d;
        }
        for (int a = tid; a < S.nt; a += 256) sa[a] = fourier_cardinal_cf(phi - PDD_TWO_PI * a / S.nt, S.nt);
        __syncthreads();
        if (tid == 0) {
            int hit = -1;
            double den = 0.0;
            for (int l = 0; l <= S.nc; ++l) {
                if (rho == S.x[l]) hit = l;
                den += lr[l];
            }
            for (int l = 0; l <= S.nc; ++l) lr[l] = (hit >= 0) ? (l == hit ? 1.0 : 0.0) : lr[l] / den;
        }
        __syncthreads();
        const double li = lambda[i];
        for (int q = tid; q < S.n; q += 256) {
            const int kk = q / S.nt, a = q - kk * S.nt;
            E[q] += li * (lr[kk + 1] * sa[a] + lr[S.nc - 1 - kk] * sa[(a + half) % S.nt]);
        }
    }
}

// z = S A_s^-T e with P A_s = L U (A_s the equilibrated matrix, S its row scales)
__global__ void __launch_bounds__(256) k_lu_solve_T(const double *LUall, int n, long strideA, const int *permAll,
                                                    const NodeCoef *coefAll, long strideC, const double *Eall,
                                                    double *Wall, double *Zall) {
    __shared__ double red[8];
    const int disk = blockIdx.x, tid = threadIdx.x;
    const double *LU = LUall + disk * strideA;
    const int *perm = permAll + (long)disk * n;
    const double *e = Eall + (long)disk * n;
    double *w = Wall + (long)disk * n, *z = Zall + (long)disk * n;
    // U^T y = e (lower, non-unit): y_i = (e_i - sum_{k<i} U_ki y_k) / U_ii
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int k = tid; k < i; k += 256) s += LU[(long)k * n + i] * w[k];
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((tid & 31) == 0) red[tid >> 5] = s;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < 8; ++q) t += red[q];
            w[i] = (e[i] - t) / LU[(long)i * n + i];
        }
        __syncthreads();
    }
    // L^T v = y (upper, unit): v_i = y_i - sum_{k>i} L_ki v_k
    for (int i = n - 1; i >= 0; --i) {
        double s = 0.0;
        for (int k = i + 1 + tid; k < n; k += 256) s += LU[(long)k * n + i] * w[k];
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((tid & 31) == 0) red[tid >> 5] = s;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < 8; ++q) t += red[q];
            w[i] -= t;
        }
        __syncthreads();
    }
    // P z' = v  ->  z'[perm[i]] = v[i];  z = S z'
    for (int i = tid; i < n; i += 256) {
        const int r = perm[i];
        z[r] = coefAll[disk * strideC + r].s * w[i];
    }
}

// per disk: the c-weight partials -sum_p z_p V_p 1{c<0} psi_q(x_p) and the f-weight partials
// -sum_p z_p psi^f_q(x_p), in the layout [disk][c weights, f weights]
__global__ void __launch_bounds__(256) k_adjoint_contract(Problem P, Shape S, const DiskDesc *disks,
                                                          const double *Vall, const double *Zall,
                                                          double *partial) {
    extern __shared__ double csm[];             // per node: x, y, z V 1{c<0}, z
    const int disk = blockIdx.x, tid = threadIdx.x;
    const DiskDesc dd = disks[disk];
    const int nw = (P.c_kind == PDD_C_RBF) ? P.n_rbf : 0;
    const int nf = (P.f_kind == PDD_F_RBF) ? P.n_frbf : 0;
    double *nx = csm, *ny = csm + S.n, *tv = csm + 2 * S.n, *zz = csm + 3 * S.n;
    for (int p = tid; p < S.n; p += 256) {
        const int k = p / S.nt + 1, j = p % S.nt;
        double st, ct;
        sincos(PDD_TWO_PI * j / S.nt, &st, &ct);
        const double X = dd.cx + dd.R * S.x[k] * ct, Y = dd.cy + dd.R * S.x[k] * st;
        nx[p] = X;
        ny[p] = Y;
        const double act = (P.c_kind == PDD_C_RBF && rbf_sum(P, X, Y) < 0.0) ? 1.0 : 0.0;
        tv[p] = Zall[(long)disk * S.n + p] * Vall[(long)disk * S.n + p] * act;
        zz[p] = Zall[(long)disk * S.n + p];
    }
    __syncthreads();
    const double inv = nw ? 1.0 / (2.0 * P.rbf_sigma * P.rbf_sigma) : 0.0;
    const double invf = nf ? 1.0 / (2.0 * P.frbf_sigma * P.frbf_sigma) : 0.0;
    for (int q = tid; q < nw + nf; q += 256) {
        double s = 0.0;
        if (q < nw) {
            for (int p = 0; p < S.n; ++p) {
                const double dx = nx[p] - P.rbf_x[q], dy = ny[p] - P.rbf_y[q];
                s += tv[p] * exp(-(dx * dx + dy * dy) * inv);
            }
        } else {
            const int qf = q - nw;
            for (int p = 0; p < S.n; ++p) {
                const double dx = nx[p] - P.frbf_x[qf], dy = ny[p] - P.frbf_y[qf];
                s += zz[p] * exp(-(dx * dx + dy * dy) * invf);
            }
        }
        partial[(long)disk * (nw + nf) + q] = -s;
    }
}

void grad_disks(const pdd_cover &cov, const Problem &P, const double *u, const double *lambda,
                DevBuf<double> &partial, int &n_part, cudaStream_t st) {
    n_part = 0;
    const int nw = (P.c_kind == PDD_C_RBF) ? P.n_rbf : 0;
    const int nf = (P.f_kind == PDD_F_RBF) ? P.n_frbf : 0;
    if (nw + nf == 0) return;
    std::map<std::tuple<int, int, int>, std::vector<DiskDesc>> groups;
    std::vector<double> hcx(cov.M), hcy(cov.M), hr(cov.M);
    PDD_CUDA(cudaMemcpyAsync(hcx.data(), cov.cx.p, cov.M * 8, cudaMemcpyDeviceToHost, st));
    PDD_CUDA(cudaMemcpyAsync(hcy.data(), cov.cy.p, cov.M * 8, cudaMemcpyDeviceToHost, st));
    PDD_CUDA(cudaMemcpyAsync(hr.data(), cov.r.p, cov.M * 8, cudaMemcpyDeviceToHost, st));
    PDD_CUDA(cudaStreamSynchronize(st));
    int total = 0;
    for (int m = 0; m < cov.M; ++m) {
        if (!cov.h_floating[m]) continue;
        int a = cov.h_sub_ptr[m], b = cov.h_sub_ptr[m + 1];
        if (b <= a) continue;
        groups[{cov.h_nr[m], cov.h_nt[m], cov.h_nk[m]}].push_back(
            DiskDesc{hcx[m], hcy[m], hr[m], m, cov.h_knot_ptr[m], a, b});
        ++total;
    }
    if (!total) return;
    partial.alloc((size_t)total * (nw + nf));
    int done = 0;
    for (auto &kv : groups) {
        ShapeTables tab;
        tab.build(std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first), st);
        const Shape S = tab.S;
        const auto &disks = kv.second;
        const size_t perDisk = (size_t)S.n * S.n * 8 + (size_t)S.n * S.nrhs * 8 * 3 + (size_t)S.n * 8 * 4 +
                               (size_t)S.n * sizeof(NodeCoef) + (size_t)S.n * 4 + 64;
        size_t freeb = 0, totb = 0;
        PDD_CUDA(cudaMemGetInfo(&freeb, &totb));
        int wave = (int)std::max<size_t>(1, std::min<size_t>((size_t)(0.5 * freeb), (size_t)32 << 30) / perDisk);
        wave = std::min<int>(wave, (int)disks.size());
        DevBuf<double> A, W, RHS, X, Vb, Eb, Zb, Wt;
        DevBuf<NodeCoef> coef;
        DevBuf<int> perm, info;
        DevBuf<DiskDesc> dd;
        A.alloc((size_t)wave * S.n * S.n);
        W.alloc((size_t)wave * S.n * S.nrhs);
        RHS.alloc((size_t)wave * S.n * S.nrhs);
        X.alloc((size_t)wave * S.n * S.nrhs);
        Vb.alloc((size_t)wave * S.n);
        Eb.alloc((size_t)wave * S.n);
        Zb.alloc((size_t)wave * S.n);
        Wt.alloc((size_t)wave * S.n);
        coef.alloc((size_t)wave * S.n);
        perm.alloc((size_t)wave * S.n);
        info.alloc(wave);
        dd.alloc(wave);
        const long sA = (long)S.n * S.n, sR = (long)S.n * S.nrhs, sC = S.n;
        for (size_t w0 = 0; w0 < disks.size(); w0 += wave) {
            const int nd = (int)std::min<size_t>(wave, disks.size() - w0);
            PDD_CUDA(cudaMemcpyAsync(dd.p, disks.data() + w0, nd * sizeof(DiskDesc), cudaMemcpyHostToDevice, st));
            build_operator<double>(P, S, dd.p, nd, A.p, sA, RHS.p, sR, coef.p, sC, st);
            launch_lu<double>(A.p, S.n, sA, perm.p, info.p, nd, st);
            launch_solve<double>(A.p, S.n, sA, perm.p, RHS.p, S.nrhs, sR, W.p, X.p, 0, nullptr, nullptr, 0.0, nd,
                                 st);
            PDD_LAUNCH(k_adjoint_vecs, nd, 256, 0, st, S, dd.p, cov.sub_rows.p, cov.kx.p, cov.ky.p, X.p, sR, u,
                       lambda, Vb.p, Eb.p);
            PDD_LAUNCH(k_lu_solve_T, nd, 256, 0, st, A.p, S.n, sA, perm.p, coef.p, sC, Eb.p, Wt.p, Zb.p);
            const size_t csm = (size_t)4 * S.n * sizeof(double);
            PDD_CUDA(cudaFuncSetAttribute(k_adjoint_contract, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
            PDD_LAUNCH(k_adjoint_contract, nd, 256, csm, st, P, S, dd.p, Vb.p, Zb.p,
                       partial.p + (size_t)(done + w0) * (nw + nf));
        }
        PDD_CUDA(cudaStreamSynchronize(st));
        done += (int)disks.size();
    }
    n_part = total;
}

}  // namespace pdd
