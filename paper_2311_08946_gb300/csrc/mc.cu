// a10-a12: Monte Carlo rows (Eq. 25-30 with the representation of Eq. 53,
// 56 and sigma = I), IMQ cardinals on perimeter arcs (Eq. 19-22).
//
//   a10 k_imq_inverse: K_lk = ((u_l - u_k)^2 + c^2)^-1/2 per perimeter stencil
//       (u the knots' local angles in radians), Cholesky factor and K^-1 in FP64
//       (one CTA per circle), and kappa_1(K).
//   a11 k_paths: Euler-Maruyama paths of dX = b dt + dW, dY = c Y dt,
//       dZ = f Y dt from the knot, stopped at the first step whose end point
//       leaves the open disk or the open domain (optionally both shrunk by the
//       Gobet-Menozzi shift).  One CTA per (row, subdomain) slot; a lane takes
//       the row's next path id as soon as its path exits.  Exit point: the
//       first crossing of the segment with the circle or dOmega (ties to
//       dOmega).  Normals: Philox4x32-10, key (seed, knot), counter (step,
//       path, 0, k) with k the subdomain's position in the row's list.  FP64
//       form: every quantity in FP64.  Mixed form: position, drift and normals
//       in FP32, weights Y, Z and all scores in FP64.  Per-path exit records
//       (side, angle or arclength, Y, Z) go to a device scratch buffer.
//   a12 k_mc_finalize: one CTA of 16 warps per slot; warp w owns batches w and
//       w + 16 (paths p = b mod 32) and its lanes own basis functions.  The
//       moments M_l = E[1_Gamma Y phi_l(u)], C_ij = -sum_l (K^-1)_lj M_l (IMQ)
//       or -M_j (Fourier cardinals), the slot's part of r_i = E[1_dOmega g Y +
//       Z]; standard errors by batch means over the 32 batches.
#include <algorithm>
#include <vector>

#include "handles.cuh"

namespace pdd {

static constexpr int kBatches = 32;
static constexpr int kMaxStencil = 96;
static constexpr double kFastKappa = 1e5;      // largest kappa_1(K) summed in FP32 (mixed form)
static constexpr double kDfKappa = 1e10;       // largest kappa_1(K) summed in double-float (mixed form)

// ---------------------------------------------------------------------------
// a10
// ---------------------------------------------------------------------------
// largest column sum of |A| (n x n in shared memory), by the block
__device__ double norm1_block(const double *A, int n, double *red) {
    double mx = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double s = 0.0;
        for (int l = 0; l < n; ++l) s += fabs(A[l * n + c]);
        mx = fmax(mx, s);
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int t = 0; t < blockDim.x; ++t) v = fmax(v, red[t]);
        red[0] = v;
    }
    __syncthreads();
    const double v = red[0];
    __syncthreads();
    return v;
}

__global__ void __launch_bounds__(128) k_imq_inverse(const int *circles, const int *knot_ptr,
                                                     const double *ku, const long *kinv_off,
                                                     double c2, double *kinv, double *kcond, int *bad) {
    extern __shared__ double sm[];                    // K (n x n), then L in place
    __shared__ double red[128];
    const int m = circles[blockIdx.x];
    const int a = knot_ptr[m], n = knot_ptr[m + 1] - a;
    double *K = sm;
    double *Z = sm + n * n;                           // n x n work for the inverse
    const int tid = threadIdx.x;
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        int l = idx / n, k = idx % n;
        double d = ku[a + l] - ku[a + k];
        K[idx] = 1.0 / sqrt(d * d + c2);
    }
    __syncthreads();
    const double nK = norm1_block(K, n, red);
    // right-looking Cholesky, lower triangle
    for (int j = 0; j < n; ++j) {
        if (tid == 0) {
            double v = K[j * n + j];
            if (!(v > 0.0)) atomicAdd(bad, 1);
            K[j * n + j] = sqrt(fmax(v, 1e-300));
        }
        __syncthreads();
        const double d = K[j * n + j];
        for (int i = j + 1 + tid; i < n; i += blockDim.x) K[i * n + j] /= d;
        __syncthreads();
        for (int idx = tid; idx < (n - j - 1) * (n - j - 1); idx += blockDim.x) {
            int i = j + 1 + idx / (n - j - 1), k = j + 1 + idx % (n - j - 1);
            if (k <= i) K[i * n + k] -= K[i * n + j] * K[k * n + j];
        }
        __syncthreads();
    }
    // K^-1 = L^-T L^-1: column c of the identity per thread
    for (int c = tid; c < n; c += blockDim.x) {
        for (int i = 0; i < n; ++i) {                 // L y = e_c
            double v = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) v -= K[i * n + k] * Z[k * n + c];
            Z[i * n + c] = v / K[i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {            // L^T x = y
            double v = Z[i * n + c];
            for (int k = i + 1; k < n; ++k) v -= K[k * n + i] * Z[k * n + c];
            Z[i * n + c] = v / K[i * n + i];
        }
    }
    __syncthreads();
    const double nZ = norm1_block(Z, n, red);
    if (tid == 0) kcond[m] = nK * nZ;                 // kappa_1(K)
    double *out = kinv + kinv_off[blockIdx.x];
    for (int idx = tid; idx < n * n; idx += blockDim.x) out[idx] = Z[idx];
}

// ---------------------------------------------------------------------------
// a11
// ---------------------------------------------------------------------------
struct PathArgs {
    // per slot: the row (knot) i; per global slot gs: its subdomain and the position of that
    // subdomain in Pi_i (Philox counter word 3; null: 0)
    const int *rows, *subs, *kword;
    const double *kx, *ky, *ccx, *ccy, *cr, *theta_s;
    int paths;                       // paths per row when npaths is null
    double h;
    uint64_t seed;
    int8_t *side;
    double *su, *Y, *Z;
    unsigned long long *steps;
    int *capped;
    const int *npaths;               // per-row path counts (adaptive), or null
    const long *rec_off;             // per-row record offsets, or null (slot * paths)
    float2 *ez;                      // mixed form: the unfolded FP32 increments (e, z) of each record
    double shift;                    // Gobet-Menozzi boundary shift c0 sqrt(h), or 0 (plain exit)
    const int *gslot;                // global slot of each launched slot, or null (slot)
    int max_steps;                   // step cap per path (0: 50 r^2 / h)
    int cvd, ncv;                    // control-variate monomial degree (0: none) and feature count
    double *cvq;                     // per-path features [rec][ncv]
};

// c0 = -zeta(1/2) / sqrt(2 pi): the Gobet-Menozzi shift in units of |sigma^T n| sqrt(h) (sigma = I)
static constexpr double kGmC0 = 0.5825971579390108;

__device__ __forceinline__ double circle_exit_t(double px, double py, double dx, double dy, double ox,
                                                double oy, double rad) {
    const double qx = px - ox, qy = py - oy;
    const double a = dx * dx + dy * dy;
    const double b = qx * dx + qy * dy;
    const double c = qx * qx + qy * qy - rad * rad;
    double disc = b * b - a * c;
    if (disc < 0.0) disc = 0.0;
    const double sq = sqrt(disc);
    return (b >= 0.0) ? -c / (b + sq) : (sq - b) / a;
}

// first crossing of the segment P -> P + D with the circle |z - o| = rad (P inside), in R
template <typename R>
__device__ __forceinline__ R circle_exit_tr(R px, R py, R dx, R dy, R ox, R oy, R rad) {
    const R qx = px - ox, qy = py - oy;
    const R a = dx * dx + dy * dy;
    const R b = qx * dx + qy * dy;
    const R c = qx * qx + qy * qy - rad * rad;
    R disc = b * b - a * c;
    if (disc < (R)0) disc = (R)0;
    const R sq = sqrt(disc);
    return (b >= (R)0) ? -c / (b + sq) : (sq - b) / a;
}

template <typename R>
struct Num;
template <>
struct Num<double> {
    __device__ static void normals(uint64_t s, uint32_t k, uint32_t q, uint32_t st, uint32_t p, double &a, double &b) {
        normals64(s, k, q, st, p, a, b);
    }
    __device__ static void drift(const Problem &P, double x, double y, double &bx, double &by) {
        pdd::drift(P, x, y, bx, by);
    }
    __device__ static double sq(double v) { return sqrt(v); }
};
template <>
struct Num<float> {
    __device__ static void normals(uint64_t s, uint32_t k, uint32_t q, uint32_t st, uint32_t p, float &a, float &b) {
        normals32(s, k, q, st, p, a, b);
    }
    __device__ static void drift(const Problem &P, float x, float y, float &bx, float &by) {
        if (P.b_kind == PDD_B_SINX_COSY) {
            bx = __sinf(reduce_2pi(x));
            by = __cosf(reduce_2pi(y));
        } else {
            bx = 0.f;
            by = 0.f;
        }
    }
    __device__ static float sq(float v) { return sqrtf(v); }
};

__device__ __forceinline__ float killing32(const Problem &P, float x, float y) {
    if (P.c_kind == PDD_C_QUADRATIC) return -(1.0f + x * x + y * y);
    if (P.c_kind == PDD_C_RBF) {
        float s = 0.f;
        const int nr = P.n_rbf;
        const float *cx = P.rbf32, *cy = P.rbf32 + nr, *cw = P.rbf32 + 2 * nr;
        for (int q = 0; q < nr; ++q) {
            const float dx = x - cx[q], dy = y - cy[q];
            s += cw[q] * __expf(-(dx * dx + dy * dy) * P.rbf_inv2s2);
        }
        return s < 0.f ? s : 0.f;
    }
    return 0.f;
}

// f of the manufactured solution from already evaluated b and c (FP32)
__device__ __forceinline__ float source32_given(const Problem &P, float x, float y, float bx, float by, float cv) {
    if (P.f_kind == PDD_F_RBF) {
        const int nq = P.n_frbf;
        const float *fx = P.frbf32, *fy = P.frbf32 + nq, *fw = P.frbf32 + 2 * nq;
        float s = 0.f;
        for (int q = 0; q < nq; ++q) {
            const float dx = x - fx[q], dy = y - fy[q];
            s += fw[q] * __expf(-(dx * dx + dy * dy) * P.frbf_inv2s2);
        }
        return s;
    }
    if (P.f_kind == PDD_F_ONE) return 1.0f;
    if (P.f_kind == PDD_F_MANUFACTURED) {
        float spx, cpx, spy, cpy;
        fast_sincospi(x, spx, cpx);
        fast_sincospi(y, spy, cpy);
        const float pi = 3.14159265358979f;
        const float u = spx * cpy, ux = pi * cpx * cpy, uy = -pi * spx * spy;
        return -(-pi * pi * u + bx * ux + by * uy + cv * u);
    }
    if (P.f_kind == PDD_F_EQ46) {
        float u, ux, uy, lap;
        u46_derivs(x, y, u, ux, uy, lap);
        return -(0.5f * lap + bx * ux + by * uy + cv * u);
    }
    return 0.f;
}

__device__ __forceinline__ float source32(const Problem &P, float x, float y) {
    float bx, by;
    Num<float>::drift(P, x, y, bx, by);
    return source32_given(P, x, y, bx, by, killing32(P, x, y));
}

// Control-variate features (CV): for the monomials psi = xr^a yr^b (1 <= a + b <= D <= 4) of
// xr = (x - cx) / r, yr = (y - cy) / r, the sums Q = sum_k Y_k sqrt(h) grad psi(X_k) . xi_k, which have
// mean zero whatever psi (xi_k is independent of X_k and Y_k): the regression control variate of
// Milstein and Tretyakov (features in the order d = a + b = 1..D, a = d..0).
static constexpr int kMaxCv = 14;

template <typename R>
__device__ __forceinline__ void cv_accumulate(R (&cq)[kMaxCv], int D, R xr, R yr, R s, R xi0, R xi1) {
    R px[5], py[5];
    px[0] = (R)1;
    py[0] = (R)1;
#pragma unroll
    for (int e = 1; e <= 4; ++e) {
        px[e] = px[e - 1] * xr;
        py[e] = py[e - 1] * yr;
    }
    int q = 0;
#pragma unroll
    for (int d = 1; d <= 4; ++d) {
        if (d > D) break;
#pragma unroll
        for (int a = d; a >= 0; --a) {
            const int b = d - a;
            R g = (R)0;
            if (a > 0) g += (R)a * px[a - 1] * py[b] * xi0;
            if (b > 0) g += (R)b * px[a] * py[b - 1] * xi1;
            cq[q] += s * g;
            ++q;
        }
    }
}

template <typename R, bool KILL, bool SRC, bool CV>
__global__ void __launch_bounds__(256) k_paths(Problem P, PathArgs A) {
    __shared__ int next_path;
    const int slot = blockIdx.x;
    const int gsl = A.gslot ? A.gslot[slot] : slot;
    const int i = A.rows[slot], m = A.subs[gsl];
    const uint32_t kw = A.kword ? (uint32_t)A.kword[gsl] : 0u;
    const double rad = A.cr[m], ts = A.theta_s[m];
    // exit tests against the disk and the domain shrunk by the boundary shift (0: the true ones), in
    // the position type; computed once into shared memory so that the loop reads them instead of
    // recomputing FP64 expressions: circle centre, r^2, r, the square's (x0, y0, x1, y1) or the
    // disk domain's (cx, cy, R) and R^2, the starting point and the step constants
    __shared__ R kc[14];
    if (threadIdx.x == 0) {
        const double rs = rad - A.shift, sft = A.shift;
        const bool sqd = P.dom_kind == 0;
        kc[0] = (R)A.ccx[m];
        kc[1] = (R)A.ccy[m];
        kc[2] = (R)(rs * rs);
        kc[3] = (R)rs;
        kc[4] = (R)(sqd ? P.dom[0] + sft : P.dom[0]);
        kc[5] = (R)(sqd ? P.dom[1] + sft : P.dom[1]);
        kc[6] = (R)(P.dom[2] - sft);
        kc[7] = (R)(P.dom[3] - sft);
        kc[8] = (R)((P.dom[2] - sft) * (P.dom[2] - sft));
        kc[9] = (R)A.kx[i];
        kc[10] = (R)A.ky[i];
        kc[11] = (R)A.h;
        kc[12] = Num<R>::sq((R)A.h);
        kc[13] = (R)ts;
    }
    __syncthreads();
    const R rcx = kc[0], rcy = kc[1], r2 = kc[2];
    const int max_steps = A.max_steps > 0 ? A.max_steps : (int)fmin(2147483647.0, ceil(50.0 * rad * rad / A.h));
    const R h = kc[11], sh = kc[12];
    const float hf = (float)kc[11];
    const bool sq_dom = P.dom_kind == 0;
    const R d0 = kc[4], d1 = kc[5], d2 = kc[6], d3 = kc[7];
    const R dr2 = kc[8];
    const R x_start = kc[9], y_start = kc[10];
    const int npath = A.npaths ? A.npaths[slot] : A.paths;
    const long rbase = A.rec_off ? A.rec_off[slot] : (long)slot * A.paths;
    unsigned long long my_steps = 0;
    int my_capped = 0;
    if (threadIdx.x == 0) next_path = blockDim.x;
    __syncthreads();
    // One loop iteration is one Euler-Maruyama step of this lane's current path; a lane whose
    // path exits writes its record and starts its next path (the row's next free path id) in
    // the same iteration, so the lanes of a warp stay converged whatever the path lengths.
    int p = threadIdx.x;
    R x = x_start, y = y_start;
    R cq[kMaxCv];
#pragma unroll
    for (int q = 0; q < kMaxCv; ++q) cq[q] = (R)0;
    const R crad = (R)rad;
    double Yv = 1.0, Zv = 0.0;
    float e = 0.f, z = 0.f;    // mixed form: Y = Yv (1 + e), Z = Zv + Yv z (FP32 block increments)
    int k = 0;
    unsigned it = 0;           // loop iterations, equal in all active lanes
    while (p < npath) {
        const long rec = rbase + p;
        bool done = false;
        if (k >= max_steps) {
            A.side[rec] = 2;
            A.su[rec] = 0.0;
            A.Y[rec] = 0.0;
            A.Z[rec] = 0.0;
            if constexpr (sizeof(R) == 4) A.ez[rec] = make_float2(0.f, 0.f);
            if constexpr (CV)
                for (int q = 0; q < A.ncv; ++q) A.cvq[rec * A.ncv + q] = 0.0;
            ++my_capped;
            done = true;
        } else {
            R xi0, xi1;
            Num<R>::normals(A.seed, (uint32_t)i, kw, (uint32_t)k, (uint32_t)p, xi0, xi1);
            if constexpr (CV) {
                // Y_k sqrt(h) grad psi(X_k) . xi_k / r, with Y_k the weight before this step
                const R yk = sizeof(R) == 8 ? (R)Yv : (R)((float)Yv * (1.0f + e));
                cv_accumulate<R>(cq, A.cvd, (x - rcx) / crad, (y - rcy) / crad, yk * sh / crad, xi0, xi1);
            }
            R bx, by;
            Num<R>::drift(P, x, y, bx, by);
            double Yn = Yv, Zn = Zv;
            float en = e, zn = z;
            if constexpr (sizeof(R) == 8) {
                // FP64 form: the same expressions as the definition (identical streams)
                if (KILL) Yn = Yv * (1.0 + killing(P, (double)x, (double)y) * A.h);
                if (SRC) Zn = Zv + source(P, (double)x, (double)y) * Yv * A.h;
            } else {
                const float cv = KILL ? killing32(P, (float)x, (float)y) : 0.f;
                // Z_{k+1} = Z_k + f_k h Y_k and Y_{k+1} = Y_k (1 + c_k h), with Y_k = Yv (1 + e)
                if (SRC) zn = fmaf(source32_given(P, (float)x, (float)y, (float)bx, (float)by, cv) * hf, 1.0f + e, z);
                if (KILL) en = fmaf(cv * hf, 1.0f + e, e);
            }
            const R nx = x + bx * h + sh * xi0;
            const R ny = y + by * h + sh * xi1;
            ++k;
            const R ddx = nx - rcx, ddy = ny - rcy;
            const bool out_c = !(ddx * ddx + ddy * ddy < r2);
            bool in_d;
            if (P.dom_kind == 0) {
                in_d = nx > d0 && nx < d2 && ny > d1 && ny < d3;
            } else {
                const R ex0 = nx - d0, ey0 = ny - d1;
                in_d = ex0 * ex0 + ey0 * ey0 < dr2;
            }
            const bool out_d = !in_d;
            if constexpr (sizeof(R) == 4) {
                // fold the FP32 increments into the FP64 weights every 8 iterations of the loop (the
                // same iterations in every lane of the warp, so the FP64 work is not divergent); the
                // increments left at the exit go to the record and the finalize folds them
                if ((++it & 7) == 0) {
                    Zn = fma(Yv, (double)zn, Zv);
                    Yn = fma(Yv, (double)en, Yv);
                    en = 0.f;
                    zn = 0.f;
                }
            }
            if (!out_c && !out_d) {
                x = nx;
                y = ny;
                Yv = Yn;
                Zv = Zn;
                e = en;
                z = zn;
            } else {
                // exit point on the segment, in the position type (FP64 form: FP64; mixed: FP32); with
                // the boundary shift the piece crossed first (on the shrunk boundaries) is scored at the
                // projection of the first point outside onto the true boundary
                const R dx = nx - x, dy = ny - y;
                R tc = (R)2, td = (R)2;
                int ed = -1;
                if (out_c) tc = circle_exit_tr<R>(x, y, dx, dy, rcx, rcy, kc[3]);
                if (out_d) {
                    if (sq_dom) {
                        R t;
                        if (nx <= d0) { t = (d0 - x) / dx; if (t < td) { td = t; ed = 3; } }
                        if (nx >= d2) { t = (d2 - x) / dx; if (t < td) { td = t; ed = 1; } }
                        if (ny <= d1) { t = (d1 - y) / dy; if (t < td) { td = t; ed = 0; } }
                        if (ny >= d3) { t = (d3 - y) / dy; if (t < td) { td = t; ed = 2; } }
                    } else {
                        td = circle_exit_tr<R>(x, y, dx, dy, d0, d1, d2);
                        ed = 0;
                    }
                }
                const bool proj = A.shift > 0.0;
                if (td <= tc) {
                    R ex = x + td * dx, ey = y + td * dy;
                    if (proj) {
                        ex = nx;
                        ey = ny;
                        if (sq_dom) {
                            const R x0 = (R)P.dom[0], y0 = (R)P.dom[1], x1 = (R)P.dom[2], y1 = (R)P.dom[3];
                            ex = ex < x0 ? x0 : (ex > x1 ? x1 : ex);
                            ey = ey < y0 ? y0 : (ey > y1 ? y1 : ey);
                            if (ed == 0) ey = y0;
                            else if (ed == 1) ex = x1;
                            else if (ed == 2) ey = y1;
                            else ex = x0;
                        }                                  // disk domain: the arclength is the angle's
                    }
                    A.side[rec] = 1;
                    A.su[rec] = boundary_s(P, (double)ex, (double)ey, ed);
                } else {
                    const R ex = proj ? nx : x + tc * dx, ey = proj ? ny : y + tc * dy;
                    R th = atan2(ey - rcy, ex - rcx);
                    const R two_pi = (R)PDD_TWO_PI;
                    if (th < (R)0) th += two_pi;
                    R u = th - kc[13];
                    if (u < (R)0) u += two_pi;
                    if (u >= two_pi) u -= two_pi;
                    A.side[rec] = 0;
                    A.su[rec] = (double)u;
                }
                A.Y[rec] = Yn;
                A.Z[rec] = Zn;
                if constexpr (sizeof(R) == 4) A.ez[rec] = make_float2(en, zn);
                if constexpr (CV) {
#pragma unroll
                    for (int q = 0; q < kMaxCv; ++q)
                        if (q < A.ncv) A.cvq[rec * A.ncv + q] = (double)cq[q];
                }
                done = true;
            }
        }
        if (done) {
            my_steps += (unsigned long long)k;
            p = atomicAdd(&next_path, 1);
            x = x_start;
            y = y_start;
            Yv = 1.0;
            Zv = 0.0;
            e = 0.f;
            z = 0.f;
            k = 0;
            if constexpr (CV) {
#pragma unroll
                for (int q = 0; q < kMaxCv; ++q) cq[q] = (R)0;
            }
        }
    }
    // block totals
    __shared__ unsigned long long ss[8];
    __shared__ int sc[8];
    for (int o = 16; o; o >>= 1) {
        my_steps += __shfl_xor_sync(0xffffffffu, my_steps, o);
        my_capped += __shfl_xor_sync(0xffffffffu, my_capped, o);
    }
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = my_steps;
        sc[threadIdx.x >> 5] = my_capped;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        int c = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t += ss[w];
            c += sc[w];
        }
        atomicAdd(A.steps, t);
        if (c) atomicAdd(A.capped, c);
    }
}

// ---------------------------------------------------------------------------
// a12
// ---------------------------------------------------------------------------
// Dirichlet data in FP32 (mixed form's boundary scores)
__device__ __forceinline__ float gdata32(const Problem &P, float x, float y, float s) {
    switch (P.g_kind) {
        case PDD_G_EXP_SIN: return expf(x) * sinf(y);
        case PDD_G_SIN_COS: return sinpif(x) * cospif(y);
        case PDD_G_BOUNDARY_FOURIER: {
            const int kc = (P.n_gcoef + 1) / 2, ks = P.n_gcoef - kc;
            const float w = s * (float)(2.0 / P.perimeter);
            float acc = 0.f;
            for (int k = 0; k < kc; ++k) acc += (float)P.g_coef[k] * cospif(k * w);
            for (int k = 1; k <= ks; ++k) acc += (float)P.g_coef[kc + k - 1] * sinpif(k * w);
            return acc;
        }
        case PDD_G_ONE: return 1.f;
        case PDD_G_EQ46: {
            float u, ux, uy, lap;
            u46_derivs(x, y, u, ux, uy, lap);
            return u;
        }
        default: return 0.f;
    }
}

// Fourier cardinal of a knot (Eq. 18) at angular distance t, closed form; out of line (Monte Carlo
// rows of floating circles only) for the same reason as boundary_score
__device__ __noinline__ double fourier_cardinal_at(double t, int n) {
    const double x = remainder(t, PDD_TWO_PI);
    return (x == 0.0) ? 1.0 : sin(0.5 * n * x) * cos(0.5 * x) / (sin(0.5 * x) * n);
}

// g at the boundary point of arclength s (FP32 data in the mixed form); kept out of line so that
// the data families do not add to the register pressure of the finalize loop (taken only for
// paths that exit through dOmega)
__device__ __noinline__ double boundary_score(const Problem &P, double s, int mixed) {
    double ex, ey;
    boundary_point(P, s, ex, ey);
    return mixed ? (double)gdata32(P, (float)ex, (float)ey, (float)s) : gdata(P, ex, ey, s);
}

struct FinalArgs {
    // per slot: the row i; per global slot gs: its subdomain and its entry p of sub_rows, whose
    // stencil block starts at rowptr[i] + sub_off[p] and whose part of r_i goes to bs[p]
    const int *rows, *subs, *spos, *sub_off, *knot_ptr, *rowptr;
    const uint8_t *floating;
    const double *ku;
    const long *kinv_off;     // per circle (-1 when not IMQ)
    const double *kinv;
    const double *kcond;      // per circle: kappa_1(K) (0 when not IMQ)
    double c2;
    int paths, mc_floating, mixed;
    const int *npaths;               // per-row path counts, or null (paths)
    const long *rec_off;             // per-row record offsets, or null (slot * paths)
    const int *gslot;                // index of the row in the system's Monte Carlo arrays, or null (slot)
    const int8_t *side;
    const double *su, *Y, *Z;
    const float2 *ez;                // mixed form: unfolded increments, Y (1 + e) and Z + Y z
    const int *mom_ptr;
    double *moments, *bmean, *val, *se, *bs, *se_bs;
    int sums;                        // PDD_SUMS_* of the mixed form (AUTO: by kappa_1(K))
    // regression control variate (null: none): per launched slot, beta [ns_max + 1][ncv] (the basis
    // moments' rows, then r's) and the per-batch feature sums [32][ncv]
    const double *cv_beta, *cv_sq;
    int ncv, cv_stride;              // features, beta rows per slot (the launch's largest stencil + 1)
};

// v = hi + lo with hi = v truncated to 24 significant bits and lo the rest rounded to FP32, built
// from the bit fields by integer operations (the FP64 pipe of this part is 1/64 of the FP32 rate).
// |v| < 2^-126 gives (0, 0) and |v| < 2^-74 drops lo (relative error up to 2^-23 there); above
// that the split is within 2^-47 relative (an emulation over 2e4 values per decade); the Monte Carlo
// weights and exit angles are far from either.
__device__ __forceinline__ float2 split_df_bits(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FF);
    const int eh = e - 896;                                 // FP32 biased exponent of hi
    if (eh >= 255) return make_float2((float)v, 0.f);       // beyond FP32 range (not reached)
    if (eh <= 0) return make_float2(__uint_as_float(sign), 0.f);
    const float hi = __uint_as_float(sign | ((unsigned)eh << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
    const int el = e - 948;                                 // FP32 biased exponent of 2^(e - 1075)
    float lo = 0.f;
    if (el > 0) lo = __fmul_rn(__uint2float_rn((unsigned)(b & 0x1FFFFFFFull)), __uint_as_float((unsigned)el << 23));
    return make_float2(hi, __uint_as_float(__float_as_uint(lo) | sign));
}

// 1 / sqrt(q) for q = qh + ql in double-float: one Newton step from rsqrtf, whose residual
// t = 1 - q r0^2 is formed without rounding error in its leading part (r0^2 and q r0^2 by FMA
// splits; 1 - h is exact because h is within 2^-22 of 1); relative error below 1e-13
__device__ __forceinline__ float2 df_rsqrt(float qh, float ql) {
    const float r0 = rsqrtf(qh);
    const float a = __fmul_rn(r0, r0);
    const float ae = fmaf(r0, r0, -a);
    const float h = __fmul_rn(qh, a);
    float he = fmaf(qh, a, -h);
    he = fmaf(qh, ae, he);
    he = fmaf(ql, a, he);
    const float t = __fsub_rn(__fsub_rn(1.0f, h), he);
    return make_float2(r0, __fmul_rn(__fmul_rn(0.5f, r0), t));
}

// Per-row finalize.  NQ = register slices of 32 stencil knots (the launch's largest stencil).
// Basis sums of the mixed form (sum mode, per stencil):
//   0: FP32 phi and FP32 sums of 16 paths (kappa_1(K) <= kFastKappa);
//   1: double-float phi and sums (kappa_1(K) <= kDfKappa);
//   2: FP64 (the FP64 form, Fourier cardinals, and larger kappa).
// C = -K^-T M amplifies the rounding of the moments by up to kappa(K): FP32 sums of FP32 phi
// were measured off by ~5e-11 kappa in C (0.03 at kappa 5.6e8); double-float phi is within
// 1e-13 relative (an emulation over 2e4 random angles), FP64 within 2^-52.
template <int NQ>
__global__ void __launch_bounds__(512) k_mc_finalize(Problem P, FinalArgs F) {
    extern __shared__ double fsm[];                   // [32 batches][ns] moments, then per-batch C
    __shared__ double bsum[kBatches];
    __shared__ int bcnt[kBatches];
    const int slot = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gs = F.gslot ? F.gslot[slot] : slot;
    const int i = F.rows[slot], m = F.subs[gs], pe = F.spos[gs];
    const int a = F.knot_ptr[m], ns = F.knot_ptr[m + 1] - a;
    const bool imq = !F.floating[m];
    double *Mb = fsm;                                 // kBatches x ns
    double *Cb = fsm + kBatches * ns;                 // kBatches x ns
    const int npath = F.npaths ? F.npaths[slot] : F.paths;
    const long base = F.rec_off ? F.rec_off[slot] : (long)slot * F.paths;
    // this lane's stencil angles (IMQ) or knot angles (Fourier cardinals), also as hi + lo FP32
    double uk[NQ];
    float ukf[NQ], ukl[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int l = lane + 32 * q;
        uk[q] = (l < ns) ? (imq ? F.ku[a + l] : PDD_TWO_PI * l / ns) : 0.0;
        ukf[q] = (float)uk[q];
        ukl[q] = (float)(uk[q] - (double)ukf[q]);
    }
    const float c2f = (float)F.c2, c2l = (float)(F.c2 - (double)c2f);
    // a forced mode applies to either path form (FP64 records carry no FP32 increments); the
    // automatic choice keeps FP64 sums for FP64 paths
    int mode = 2;
    if (imq) {
        if (F.sums != PDD_SUMS_AUTO) mode = F.sums - 1;
        else if (F.mixed) mode = F.kcond[m] <= kFastKappa ? 0 : (F.kcond[m] <= kDfKappa ? 1 : 2);
    }
    const int nq = (ns + 31) >> 5;                     // slices holding stencil knots (block-uniform)
    for (int bt = warp; bt < kBatches; bt += 16) {         // 16 warps, two batches each (p mod 32)
        double acc[NQ];
        float accf[NQ], accl[NQ];                          // FP32 or double-float sums of 16 paths
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            acc[q] = 0.0;
            accf[q] = 0.f;
            accl[q] = 0.f;
        }
        int pend = 0;                                      // mode 0: paths in the FP32 sums since the last fold
        double bs = 0.0;
        int cnt = 0;
        // chunks of 32 paths of this batch: lane l loads path bt + 32 (t0 + l)
        for (int t0 = 0; bt + kBatches * t0 < npath; t0 += 32) {
            const int pl = bt + kBatches * (t0 + lane);
            int sd = 2;
            double yv = 0.0, zv = 0.0, su = 0.0;
            double yraw = 0.0;
            float ey = 0.f;                                // mixed form: the unfolded increment of Y
            if (pl < npath) {
                sd = F.side[base + pl];
                yraw = F.Y[base + pl];
                zv = F.Z[base + pl];
                su = F.su[base + pl];
                if (F.mixed) {
                    const float2 q = F.ez[base + pl];
                    zv = fma(yraw, (double)q.y, zv);
                    ey = q.x;
                }
            }
            // Y (1 + e) in FP64 where it is used in FP64: always, except for the double-float basis
            // sums, which need it only for a boundary score
            yv = yraw;
            if (F.mixed && ey != 0.f && (mode != 1 || sd == 1)) yv = fma(yraw, (double)ey, yraw);
            if (sd != 2) {                                 // this lane's own contribution to r_i
                ++cnt;
                if (sd == 1) {
                    bs += boundary_score(P, su, F.mixed) * yv + zv;
                } else {
                    bs += zv;
                }
            }
            // the chunk's interface exits, in path order, into every lane's basis sums
            if (mode == 0) {
                // each lane converts its own record once; FP32 values are shuffled
                const float yf = (float)yv, suf = (float)su;
                for (int src = 0; src < 32; ++src) {
                    const int s_sd = __shfl_sync(0xffffffffu, sd, src);
                    const float s_yf = __shfl_sync(0xffffffffu, yf, src);
                    const float s_suf = __shfl_sync(0xffffffffu, suf, src);
                    if (s_sd != 0) continue;
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        if (q >= nq) break;                // slices past the stencil hold no knot
                        const float df = s_suf - ukf[q];
                        accf[q] = fmaf(s_yf, rsqrtf(df * df + c2f), accf[q]);
                    }
                    if (++pend == 16) {
#pragma unroll
                        for (int q = 0; q < NQ; ++q) {
                            acc[q] += (double)accf[q];
                            accf[q] = 0.f;
                        }
                        pend = 0;
                    }
                }
            } else if (mode == 1) {
                // double-float: the record's Y and angle split once per lane by integer operations
                // (no FP64 instruction), Y (1 + e) formed in double-float, then shuffled
                float2 y2 = split_df_bits(yraw);
                if (ey != 0.f) {
                    const float p = __fmul_rn(y2.x, ey);
                    float pe = fmaf(y2.x, ey, -p);
                    pe = fmaf(y2.y, ey, pe);
                    y2 = df_add(y2, make_float2(p, pe));
                }
                const float2 s2 = split_df_bits(su);
                const float yh = y2.x, yl = y2.y, sh = s2.x, sl = s2.y;
                for (int src = 0; src < 32; ++src) {
                    const int s_sd = __shfl_sync(0xffffffffu, sd, src);
                    const float s_yh = __shfl_sync(0xffffffffu, yh, src);
                    const float s_yl = __shfl_sync(0xffffffffu, yl, src);
                    const float s_sh = __shfl_sync(0xffffffffu, sh, src);
                    const float s_sl = __shfl_sync(0xffffffffu, sl, src);
                    if (s_sd != 0) continue;
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        if (q >= nq) break;
                        // d = u - u_l, then q = d^2 + c^2, both in double-float
                        float dh, dl;
                        two_sum(s_sh, -ukf[q], dh, dl);
                        dl = __fadd_rn(dl, __fsub_rn(s_sl, ukl[q]));
                        const float p = __fmul_rn(dh, dh);
                        float pe2 = fmaf(dh, dh, -p);
                        pe2 = fmaf(__fmul_rn(2.0f, dh), dl, pe2);
                        float qh, ql;
                        two_sum(p, c2f, qh, ql);
                        ql = __fadd_rn(ql, __fadd_rn(pe2, c2l));
                        const float2 phi = df_rsqrt(qh, ql);
                        // (accf, accl) += Y phi
                        const float mh = __fmul_rn(s_yh, phi.x);
                        float me = fmaf(s_yh, phi.x, -mh);
                        me = fmaf(s_yh, phi.y, me);
                        me = fmaf(s_yl, phi.x, me);
                        float sh2, se2;
                        two_sum(accf[q], mh, sh2, se2);
                        accf[q] = sh2;
                        accl[q] = __fadd_rn(accl[q], __fadd_rn(se2, me));
                    }
                    // (no periodic fold: a double-float sum of a batch's paths stays within ~1e-13)
                }
            } else {
                for (int src = 0; src < 32; ++src) {
                    const int s_sd = __shfl_sync(0xffffffffu, sd, src);
                    const double s_y = __shfl_sync(0xffffffffu, yv, src);
                    const double s_su = __shfl_sync(0xffffffffu, su, src);
                    if (s_sd != 0) continue;
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        const int l = lane + 32 * q;
                        if (l >= ns) continue;
                        double phi;
                        if (imq) {
                            const double d = s_su - uk[q];
                            phi = F.mixed ? rsqrt(d * d + F.c2) : 1.0 / sqrt(d * d + F.c2);
                        } else {
                            phi = fourier_cardinal_at(s_su - uk[q], ns);
                        }
                        acc[q] += s_y * phi;
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int l = lane + 32 * q;
            if (l < ns) Mb[bt * ns + l] = acc[q] + (double)accf[q] + (double)accl[q];
        }
        for (int o = 16; o; o >>= 1) {
            bs += __shfl_xor_sync(0xffffffffu, bs, o);
            cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        }
        if (lane == 0) {
            bsum[bt] = bs;
            bcnt[bt] = cnt;
        }
    }
    __syncthreads();
    // regression control variate: every batch sum of a payoff loses beta^T (the batch's feature sums)
    if (F.cv_beta) {
        const double *beta = F.cv_beta + (long)slot * F.cv_stride * F.ncv;
        const double *sq = F.cv_sq + (long)slot * kBatches * F.ncv;
        for (int e = threadIdx.x; e < kBatches * (ns + 1); e += blockDim.x) {
            const int bt = e / (ns + 1), l = e - bt * (ns + 1);
            const double *bl = beta + (long)(l < ns ? l : F.cv_stride - 1) * F.ncv;
            double c = 0.0;
            for (int q = 0; q < F.ncv; ++q) c += bl[q] * sq[bt * F.ncv + q];
            if (l < ns) Mb[bt * ns + l] -= c;
            else bsum[bt] -= c;
        }
        __syncthreads();
    }
    // per-batch C estimates (batch means)
    const double *Ki = imq ? F.kinv + F.kinv_off[m] : nullptr;
    for (int bt = warp; bt < kBatches; bt += 16)
        for (int j = lane; j < ns; j += 32) {
            double v = 0.0;
            const int nb = bcnt[bt];
            if (imq) {
                for (int l = 0; l < ns; ++l) v -= Ki[l * ns + j] * Mb[bt * ns + l];
            } else {
                v = -Mb[bt * ns + j];
            }
            Cb[bt * ns + j] = nb ? v / nb : 0.0;
        }
    __syncthreads();
    // (the batch loops below stay partly rolled: fully unrolled they spilled)
    if (warp == 0) {
        int ntot = 0;
#pragma unroll 4
        for (int w = 0; w < kBatches; ++w) ntot += bcnt[w];
        const double inv = ntot ? 1.0 / ntot : 0.0;
        const int off = F.sub_off[pe];
        const long rp = F.rowptr[i];
        for (int j = lane; j < ns; j += 32) {
            double mean = 0.0, msum = 0.0;
#pragma unroll 4
            for (int w = 0; w < kBatches; ++w) {
                mean += bcnt[w] * Cb[w * ns + j];
                msum += Mb[w * ns + j];
            }
            mean *= inv;
            double var = 0.0;
#pragma unroll 4
            for (int w = 0; w < kBatches; ++w) {
                double f = bcnt[w] * inv, d = Cb[w * ns + j] - mean;
                var += f * f * d * d;
            }
            var *= (double)kBatches / (kBatches - 1);
            F.val[rp + off + j] = mean;
            F.se[rp + off + j] = sqrt(var);
            F.moments[F.mom_ptr[gs] + j] = msum * inv;
        }
        if (lane == 0) {
            double tot = 0.0;
            for (int w = 0; w < kBatches; ++w) tot += bsum[w];
            const double bm = tot * inv;
            double var = 0.0;
            for (int w = 0; w < kBatches; ++w) {
                if (!bcnt[w]) continue;
                double f = bcnt[w] * inv, d = bsum[w] / bcnt[w] - bm;
                var += f * f * d * d;
            }
            var *= (double)kBatches / (kBatches - 1);
            F.bs[pe] = bm;
            F.bmean[gs] = bm;
            F.se_bs[pe] = sqrt(var);
        }
    }
}

// (row, subdomain) entries integrated by Monte Carlo: flag + compaction over sub_rows
__global__ void k_mc_flag(int nsub, const int *sub_m, const uint8_t *floating, int mc_floating, int *flag) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nsub) return;
    flag[p] = (!floating[sub_m[p]] || mc_floating) ? 1 : 0;
}

__global__ void k_mc_compact(int nsub, const int *flag, const int *pos, const int *sub_rows, const int *sub_m,
                             const int *sub_k, const int *knot_ptr, int *rows, int *subs, int *spos, int *kword,
                             int *ns) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nsub || !flag[p]) return;
    int s = pos[p], m = sub_m[p];
    rows[s] = sub_rows[p];
    subs[s] = m;
    spos[s] = p;
    kword[s] = sub_k[p];
    ns[s] = knot_ptr[m + 1] - knot_ptr[m];
}

void build_imq_inverses(const pdd_cover &cov, double c2, DevBuf<double> &kinv, DevBuf<long> &koff_m,
                        DevBuf<double> &kcond, cudaStream_t st) {
    if (cov.max_stencil > kMaxStencil) fail(PDD_EINVAL, "stencil larger than the Monte Carlo kernels support");
    std::vector<int> per;
    std::vector<long> off(cov.M, -1);
    long tot = 0;
    for (int m = 0; m < cov.M; ++m) {
        int n = cov.h_knot_ptr[m + 1] - cov.h_knot_ptr[m];
        if (!cov.h_floating[m] && n > 0) {
            per.push_back(m);
            off[m] = tot;
            tot += (long)n * n;
        }
    }
    DevBuf<long> koff_c;
    DevBuf<int> circ, bad;
    kinv.alloc(std::max<long>(tot, 1));
    koff_m.alloc(cov.M);
    kcond.alloc(std::max(cov.M, 1));
    PDD_CUDA(cudaMemsetAsync(kcond.p, 0, sizeof(double) * std::max(cov.M, 1), st));
    bad.alloc(1);
    PDD_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    PDD_CUDA(cudaMemcpyAsync(koff_m.p, off.data(), cov.M * sizeof(long), cudaMemcpyHostToDevice, st));
    if (!per.empty()) {
        std::vector<long> offc(per.size());
        for (size_t q = 0; q < per.size(); ++q) offc[q] = off[per[q]];
        circ.alloc(per.size());
        koff_c.alloc(per.size());
        PDD_CUDA(cudaMemcpyAsync(circ.p, per.data(), per.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        PDD_CUDA(cudaMemcpyAsync(koff_c.p, offc.data(), per.size() * sizeof(long), cudaMemcpyHostToDevice, st));
        const size_t smem = (size_t)2 * cov.max_stencil * cov.max_stencil * sizeof(double);
        PDD_CUDA(cudaFuncSetAttribute(k_imq_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        PDD_LAUNCH(k_imq_inverse, (int)per.size(), 128, smem, st, circ.p, cov.knot_ptr.p, cov.ku.p, koff_c.p, c2,
                   kinv.p, kcond.p, bad.p);
    }
    int hb = 0;
    PDD_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    PDD_CUDA(cudaStreamSynchronize(st));
    if (hb) fail(PDD_EINVAL, "IMQ matrix not positive definite (coincident stencil angles)");
}

// ---------------------------------------------------------------------------
// Regression control variate (Milstein and Tretyakov): per slot, beta = Cov(Q)^-1 Cov(Q, P) for the
// payoffs P = (1_Gamma Y phi_l(u), l < ns; the boundary payoff of r), covariances normalised by the
// path count, and the per-batch sums of the features Q.  Any beta leaves the estimators unbiased
// (E[Q] = 0); this one is the sample's least-squares choice.  FP64 throughout (the basis values
// too, in both forms: beta only needs to be near the optimum).  One CTA per slot; paths go
// through shared memory 256 at a time.
// ---------------------------------------------------------------------------
static constexpr int kCvThreads = 256;

__global__ void __launch_bounds__(kCvThreads) k_cv_regress(Problem P, FinalArgs F, const double *cvq,
                                                           double *beta_out, double *sq_out) {
    const int M = F.ncv;
    extern __shared__ double cvs[];
    double *Qs = cvs;                                 // [256][M] this chunk's features
    double *Ys = Qs + kCvThreads * M;                 // [256] Y at the exit (0: not an interface exit)
    double *Us = Ys + kCvThreads;                     // [256] exit angle
    double *QQ = Us + kCvThreads;                     // [M][M]
    double *QP = QQ + M * M;                          // [ns + 1][M]
    double *Pm = QP + (F.cv_stride) * M;              // [ns + 1] payoff sums
    double *Qm = Pm + F.cv_stride;                    // [M] feature sums
    double *SQ = Qm + M;                              // [32][M] per-batch feature sums
    double *L = SQ + kBatches * M;                    // [M][M] Cholesky factor
    __shared__ int s_cnt;
    const int slot = blockIdx.x, tid = threadIdx.x;
    const int gs = F.gslot ? F.gslot[slot] : slot;
    const int m = F.subs[gs];
    const int a = F.knot_ptr[m], ns = F.knot_ptr[m + 1] - a;
    const bool imq = !F.floating[m];
    const int npath = F.npaths ? F.npaths[slot] : F.paths;
    const long base = F.rec_off ? F.rec_off[slot] : (long)slot * F.paths;
    for (int e = tid; e < M * M + F.cv_stride * M + F.cv_stride + M + kBatches * M; e += kCvThreads) QQ[e] = 0.0;
    __syncthreads();
    // per-thread sums: the thread's paths are p = tid (mod 256), all in batch tid mod 32
    double my_sq[kMaxCv], my_bq[kMaxCv], my_b = 0.0;
#pragma unroll
    for (int q = 0; q < kMaxCv; ++q) {
        my_sq[q] = 0.0;
        my_bq[q] = 0.0;
    }
    int my_cnt = 0;
    // QQ entry (i, j) per thread (M (M + 1) / 2 <= 105 < 256); QP rows per thread l = tid (mod ns + 1)
    int qi = -1, qj = -1;
    {
        int e = tid;
        for (int i = 0; i < M && qi < 0; ++i) {
            if (e < M - i) {
                qi = i;
                qj = i + e;
            } else {
                e -= M - i;
            }
        }
    }
    double acc_qq = 0.0;
    for (int c0 = 0; c0 < npath; c0 += kCvThreads) {
        const int p = c0 + tid;
        double yv = 0.0, ut = 0.0;
        if (p < npath) {
            const long rec = base + p;
            const int sd = F.side[rec];
            double y = F.Y[rec], z = F.Z[rec];
            if (F.mixed) {
                const float2 q = F.ez[rec];
                z = fma(y, (double)q.y, z);
                y = fma(y, (double)q.x, y);
            }
            for (int q = 0; q < M; ++q) Qs[tid * M + q] = (sd != 2) ? cvq[rec * M + q] : 0.0;
            if (sd != 2) {
                ++my_cnt;
                const double bp = (sd == 1) ? boundary_score(P, F.su[rec], F.mixed) * y + z : z;
                my_b += bp;
                for (int q = 0; q < M; ++q) {
                    const double qv = cvq[rec * M + q];
                    my_sq[q] += qv;
                    my_bq[q] += bp * qv;
                }
                if (sd == 0) {
                    yv = y;
                    ut = F.su[rec];
                }
            }
        } else {
            for (int q = 0; q < M; ++q) Qs[tid * M + q] = 0.0;
        }
        Ys[tid] = yv;
        Us[tid] = ut;
        __syncthreads();
        if (qi >= 0)
            for (int t = 0; t < kCvThreads; ++t) acc_qq += Qs[t * M + qi] * Qs[t * M + qj];
        // basis payoffs: thread l < ns accumulates sum_p Y phi_l(u_p) Q_p and sum_p Y phi_l(u_p)
        for (int l = tid; l < ns; l += kCvThreads) {
            const double ul = imq ? F.ku[a + l] : PDD_TWO_PI * l / ns;
            double acc[kMaxCv], ps = 0.0;
#pragma unroll
            for (int q = 0; q < kMaxCv; ++q) acc[q] = 0.0;
            for (int t = 0; t < kCvThreads; ++t) {
                if (Ys[t] == 0.0) continue;
                const double d = Us[t] - ul;
                const double phi = imq ? 1.0 / sqrt(d * d + F.c2) : fourier_cardinal_at(d, ns);
                const double w = Ys[t] * phi;
                ps += w;
#pragma unroll
                for (int q = 0; q < kMaxCv; ++q)
                    if (q < M) acc[q] += w * Qs[t * M + q];
            }
            Pm[l] += ps;
            for (int q = 0; q < M; ++q) QP[l * M + q] += acc[q];
        }
        __syncthreads();
    }
    if (qi >= 0) {
        QQ[qi * M + qj] = acc_qq;
        QQ[qj * M + qi] = acc_qq;
    }
    // the features' sums per batch (lane = batch; the 8 warps added in order), then over batches;
    // the boundary payoff's sums by warp shuffles and the 8 warps in order (deterministic)
    __shared__ double wb[8][kMaxCv + 1];
    __shared__ int wc[8];
    for (int q = 0; q < M; ++q) Qs[tid * M + q] = my_sq[q];
#pragma unroll
    for (int q = 0; q <= kMaxCv; ++q) {
        double v = q < kMaxCv ? my_bq[q] : my_b;
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) wb[tid >> 5][q] = v;
    }
    for (int o = 16; o; o >>= 1) my_cnt += __shfl_xor_sync(0xffffffffu, my_cnt, o);
    if ((tid & 31) == 0) wc[tid >> 5] = my_cnt;
    __syncthreads();
    for (int e = tid; e < kBatches * M; e += kCvThreads) {
        const int bt = e / M, q = e - bt * M;
        double v = 0.0;
        for (int w = 0; w < kCvThreads / 32; ++w) v += Qs[(w * 32 + bt) * M + q];
        SQ[e] = v;
    }
    if (tid <= M) {
        double v = 0.0;
        for (int w = 0; w < kCvThreads / 32; ++w) v += wb[w][tid < M ? tid : kMaxCv];
        if (tid < M) QP[(F.cv_stride - 1) * M + tid] = v;
        else Pm[F.cv_stride - 1] = v;
    }
    if (tid == 0) {
        int c = 0;
        for (int w = 0; w < kCvThreads / 32; ++w) c += wc[w];
        s_cnt = c;
    }
    __syncthreads();
    if (tid < M) {
        double v = 0.0;
        for (int bt = 0; bt < kBatches; ++bt) v += SQ[bt * M + tid];
        Qm[tid] = v;
    }
    __syncthreads();
    // Cov(Q) = QQ / n - qm qm^T, Cholesky in place (thread 0; M <= 14)
    const double inv_n = s_cnt ? 1.0 / s_cnt : 0.0;
    if (tid == 0) {
        for (int i = 0; i < M; ++i)
            for (int j = 0; j < M; ++j) L[i * M + j] = QQ[i * M + j] * inv_n - Qm[i] * inv_n * Qm[j] * inv_n;
        for (int j = 0; j < M; ++j) {
            double dg = L[j * M + j];
            for (int k = 0; k < j; ++k) dg -= L[j * M + k] * L[j * M + k];
            dg = dg > 0.0 ? sqrt(dg) : 0.0;
            L[j * M + j] = dg;
            for (int i = j + 1; i < M; ++i) {
                double v = L[i * M + j];
                for (int k = 0; k < j; ++k) v -= L[i * M + k] * L[j * M + k];
                L[i * M + j] = dg > 0.0 ? v / dg : 0.0;
            }
        }
    }
    __syncthreads();
    // beta for each payoff row: rows l < ns (basis moments) and row cv_stride - 1 (r); zero when the
    // covariance is singular (no paths, or a feature that never moved)
    double *bo = beta_out + (long)slot * F.cv_stride * M;
    for (int l = tid; l < F.cv_stride; l += kCvThreads) {
        if (l >= ns && l != F.cv_stride - 1) {
            for (int q = 0; q < M; ++q) bo[l * M + q] = 0.0;
            continue;
        }
        double y[kMaxCv];
        bool ok = s_cnt > 1;
        for (int i = 0; i < M; ++i) {
            double v = QP[l * M + i] * inv_n - Qm[i] * inv_n * Pm[l] * inv_n;
            for (int k = 0; k < i; ++k) v -= L[i * M + k] * y[k];
            ok = ok && L[i * M + i] > 0.0;
            y[i] = ok ? v / L[i * M + i] : 0.0;
        }
        for (int i = M - 1; i >= 0; --i) {
            double v = y[i];
            for (int k = i + 1; k < M; ++k) v -= L[k * M + i] * y[k];
            y[i] = ok ? v / L[i * M + i] : 0.0;
        }
        for (int q = 0; q < M; ++q) bo[l * M + q] = y[q];
    }
    for (int e = tid; e < kBatches * M; e += kCvThreads) sq_out[(long)slot * kBatches * M + e] = SQ[e];
}

// adaptive path count of each row from its pilot standard errors
__global__ void k_need(int nmc, const int *rows, const int *subs, const int *spos, const int *sub_off,
                       const int *knot_ptr, const int *rowptr, const double *se, const double *se_bs, int P0,
                       int Pmax, double target, int *need) {
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= nmc) return;
    const int i = rows[slot], m = subs[slot], pe = spos[slot];
    const int a = knot_ptr[m], ns = knot_ptr[m + 1] - a, off = sub_off[pe];
    double mx = se_bs[pe];
    for (int j = 0; j < ns; ++j) mx = fmax(mx, se[rowptr[i] + off + j]);
    // rows at or below the target keep the pilot; the others rerun with ceil(P0 (se/target)^2)
    // paths rounded up to a multiple of 32, capped at Pmax
    if (!(mx > target)) {
        need[slot] = P0;
        return;
    }
    const double r = mx / target;
    const double want = fmin(ceil(P0 * r * r), (double)Pmax);
    int w = (int)want;
    w = ((w + 31) / 32) * 32;
    need[slot] = w > Pmax ? Pmax : w;
}

template <typename R, bool CV>
static void launch_paths_cv(const Problem &P, const PathArgs &A, int nrows, cudaStream_t st) {
    const bool kill = P.c_kind != PDD_C_ZERO, src = P.f_kind != PDD_F_ZERO;
    if (kill && src) PDD_LAUNCH((k_paths<R, true, true, CV>), nrows, 256, 0, st, P, A);
    else if (kill) PDD_LAUNCH((k_paths<R, true, false, CV>), nrows, 256, 0, st, P, A);
    else if (src) PDD_LAUNCH((k_paths<R, false, true, CV>), nrows, 256, 0, st, P, A);
    else PDD_LAUNCH((k_paths<R, false, false, CV>), nrows, 256, 0, st, P, A);
}

template <typename R>
static void launch_paths(const Problem &P, const PathArgs &A, int nrows, cudaStream_t st) {
    if (A.cvd > 0) launch_paths_cv<R, true>(P, A, nrows, st);
    else launch_paths_cv<R, false>(P, A, nrows, st);
}

McStats assemble_mc(const pdd_cover &cov, const Problem &P, const pdd_assembly_opts &o, pdd_system &sys,
                    cudaStream_t st) {
    McStats ms;
    const int mcf = o.floating_method == PDD_FLOATING_MONTE_CARLO ? 1 : 0;
    const int nsub = cov.h_sub_ptr.empty() ? 0 : cov.h_sub_ptr.back();
    DevBuf<int> flag, pos;
    flag.alloc(nsub + 1);
    pos.alloc(nsub + 1);
    if (nsub > 0) PDD_LAUNCH(k_mc_flag, cdiv(nsub, 256), 256, 0, st, nsub, cov.sub_m.p, cov.floating.p, mcf, flag.p);
    const int nmc = nsub > 0 ? (int)exclusive_scan(flag.p, pos.p, nsub, st) : 0;
    sys.n_mc = nmc;
    ms.rows = nmc;
    if (nmc == 0) return ms;
    sys.mc_rows.alloc(nmc);
    sys.mc_subs.alloc(nmc);
    sys.mc_spos.alloc(nmc);
    sys.mc_kword.alloc(nmc);
    DevBuf<int> ns;
    ns.alloc(nmc + 1);
    sys.mom_ptr.alloc(nmc + 1);
    PDD_LAUNCH(k_mc_compact, cdiv(nsub, 256), 256, 0, st, nsub, flag.p, pos.p, cov.sub_rows.p, cov.sub_m.p,
               cov.sub_k.p, cov.knot_ptr.p, sys.mc_rows.p, sys.mc_subs.p, sys.mc_spos.p, sys.mc_kword.p, ns.p);
    const int nmom = (int)exclusive_scan(ns.p, sys.mom_ptr.p, nmc, st);
    sys.moments.alloc(std::max(nmom, 1));
    sys.bmean.alloc(nmc);

    // a10: IMQ inverses for every perimeter circle with a stencil
    DevBuf<double> kinv, kcond;
    DevBuf<long> koff_m;
    build_imq_inverses(cov, o.imq_c2, kinv, koff_m, kcond, st);

    // a11: paths into the record scratch, in waves that bound the scratch size
    const long P_ = o.paths;
    const int mixed = path_mixed(o) ? 1 : 0;
    const int cvd = o.cv_degree, ncv = cvd * (cvd + 3) / 2;          // control-variate features per path
    const int cv_stride = cov.max_stencil + 1;
    const size_t rec_bytes = 1 + 3 * sizeof(double) + (mixed ? sizeof(float2) : 0) + (size_t)ncv * sizeof(double);
    const size_t per_row = (size_t)P_ * rec_bytes;
    const int wave = (int)std::max<size_t>(1, std::min<size_t>(nmc, ((size_t)8 << 30) / per_row));
    DevBuf<int8_t> side;
    DevBuf<double> su, Y, Z;
    side.alloc((size_t)wave * P_);
    su.alloc((size_t)wave * P_);
    Y.alloc((size_t)wave * P_);
    Z.alloc((size_t)wave * P_);
    DevBuf<float2> ez;
    if (mixed) ez.alloc((size_t)wave * P_);
    DevBuf<double> cvq, cvbeta, cvsq;
    if (ncv) cvq.alloc((size_t)wave * P_ * ncv);
    const size_t cv_smem = ((size_t)kCvThreads * ncv + 2 * kCvThreads + 2 * ncv * ncv + (size_t)cv_stride * ncv +
                            cv_stride + ncv + (size_t)kBatches * ncv) * sizeof(double);
    if (ncv) PDD_CUDA(cudaFuncSetAttribute(k_cv_regress, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cv_smem));
    DevBuf<unsigned long long> steps;
    DevBuf<int> capped;
    steps.alloc(1);
    capped.alloc(1);
    PDD_CUDA(cudaMemsetAsync(steps.p, 0, sizeof(unsigned long long), st));
    PDD_CUDA(cudaMemsetAsync(capped.p, 0, sizeof(int), st));
    cudaEvent_t e0, e1, e2;
    PDD_CUDA(cudaEventCreate(&e0));
    PDD_CUDA(cudaEventCreate(&e1));
    PDD_CUDA(cudaEventCreate(&e2));
    float tp = 0, tf = 0;
    const size_t fsm = (size_t)2 * kBatches * cov.max_stencil * sizeof(double);
    const int nq_launch = std::max(1, (cov.max_stencil + 31) / 32);
    PDD_CUDA(cudaFuncSetAttribute(k_mc_finalize<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm));
    PDD_CUDA(cudaFuncSetAttribute(k_mc_finalize<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm));
    PDD_CUDA(cudaFuncSetAttribute(k_mc_finalize<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm));
    // per-slot arrays (subs, spos, kword, momp, bmean) are indexed like the global slot gs: offset to
    // the wave's first slot when gsl is null, or the whole arrays with gsl
    auto run_wave = [&](const int *rows, int nr, const int *np, const long *roff, const int *gsl, const int *momp,
                        double *bmean, size_t w0) {
        const int *subs = sys.mc_subs.p + w0, *spos = sys.mc_spos.p + w0, *kword = sys.mc_kword.p + w0;
        PathArgs A{rows, subs, kword, cov.kx.p, cov.ky.p, cov.cx.p, cov.cy.p, cov.r.p,
                   cov.theta_s.p, o.paths, o.h, o.seed, side.p, su.p, Y.p, Z.p, steps.p, capped.p, np, roff, ez.p,
                   o.boundary_shift ? kGmC0 * sqrt(o.h) : 0.0, gsl, o.max_steps, cvd, ncv, cvq.p};
        PDD_CUDA(cudaEventRecord(e0, st));
        if (mixed) launch_paths<float>(P, A, nr, st);
        else launch_paths<double>(P, A, nr, st);
        PDD_CUDA(cudaEventRecord(e1, st));
        FinalArgs F{rows, subs, spos, cov.sub_off.p, cov.knot_ptr.p, cov.rowptr.p, cov.floating.p,
                    cov.ku.p, koff_m.p, kinv.p, kcond.p, o.imq_c2, o.paths, mcf, mixed, np, roff, gsl, side.p, su.p,
                    Y.p, Z.p,
                    ez.p, momp, sys.moments.p, bmean, sys.val.p, sys.se.p, sys.bs.p, sys.se_bs.p, o.moment_sums,
                    nullptr, nullptr, ncv, cv_stride};
        if (ncv) {
            if (cvbeta.n < (size_t)nr * cv_stride * ncv) cvbeta.alloc((size_t)nr * cv_stride * ncv);
            if (cvsq.n < (size_t)nr * kBatches * ncv) cvsq.alloc((size_t)nr * kBatches * ncv);
            PDD_LAUNCH(k_cv_regress, nr, kCvThreads, cv_smem, st, P, F, cvq.p, cvbeta.p, cvsq.p);
            F.cv_beta = cvbeta.p;
            F.cv_sq = cvsq.p;
        }
        if (nq_launch == 1) PDD_LAUNCH(k_mc_finalize<1>, nr, 512, fsm, st, P, F);
        else if (nq_launch == 2) PDD_LAUNCH(k_mc_finalize<2>, nr, 512, fsm, st, P, F);
        else PDD_LAUNCH(k_mc_finalize<3>, nr, 512, fsm, st, P, F);
        PDD_CUDA(cudaEventRecord(e2, st));
        PDD_CUDA(cudaEventSynchronize(e2));
        float ta = 0, tb = 0;
        cudaEventElapsedTime(&ta, e0, e1);
        cudaEventElapsedTime(&tb, e1, e2);
        tp += ta;
        tf += tb;
    };
    for (int w0 = 0; w0 < nmc; w0 += wave) {
        const int nr = std::min(wave, nmc - w0);
        run_wave(sys.mc_rows.p + w0, nr, nullptr, nullptr, nullptr, sys.mom_ptr.p + w0, sys.bmean.p + w0, w0);
    }
    ms.paths_total = (int64_t)nmc * P_;
    sys.mc_np.alloc(nmc);
    std::vector<int> need(nmc, (int)P_);
    // adaptive path counts: rows whose largest standard error exceeds the target rerun with
    // P0 (se/target)^2 paths (capped at paths_max); path ids continue the pilot's streams
    if (o.paths_max > o.paths && o.se_target > 0.0) {
        DevBuf<int> dneed;
        dneed.alloc(nmc);
        PDD_LAUNCH(k_need, cdiv(nmc, 256), 256, 0, st, nmc, sys.mc_rows.p, sys.mc_subs.p, sys.mc_spos.p,
                   cov.sub_off.p, cov.knot_ptr.p, cov.rowptr.p, sys.se.p, sys.se_bs.p, o.paths, o.paths_max,
                   o.se_target, dneed.p);
        PDD_CUDA(cudaMemcpyAsync(need.data(), dneed.p, nmc * sizeof(int), cudaMemcpyDeviceToHost, st));
        PDD_CUDA(cudaStreamSynchronize(st));
        std::vector<int> ext_slot, ext_row_host;
        std::vector<int> hrows(nmc);
        PDD_CUDA(cudaMemcpyAsync(hrows.data(), sys.mc_rows.p, nmc * sizeof(int), cudaMemcpyDeviceToHost, st));
        PDD_CUDA(cudaStreamSynchronize(st));
        for (int k = 0; k < nmc; ++k)
            if (need[k] > P_) ext_slot.push_back(k);
        size_t q = 0;
        const size_t budget = (size_t)8 << 30;
        while (q < ext_slot.size()) {
            std::vector<int> rows, np, gsl;
            std::vector<long> roff;
            size_t used = 0;
            long off = 0;
            while (q < ext_slot.size() && (rows.empty() || used + (size_t)need[ext_slot[q]] * rec_bytes <= budget)) {
                const int k = ext_slot[q++];
                rows.push_back(hrows[k]);
                np.push_back(need[k]);
                gsl.push_back(k);
                roff.push_back(off);
                off += need[k];
                used += (size_t)need[k] * rec_bytes;
                ms.paths_total += need[k];
                ++ms.extended_rows;
            }
            DevBuf<int> drows, dnp, dgsl;
            DevBuf<long> droff;
            drows.alloc(rows.size());
            dnp.alloc(rows.size());
            dgsl.alloc(rows.size());
            droff.alloc(rows.size());
            PDD_CUDA(cudaMemcpyAsync(drows.p, rows.data(), rows.size() * sizeof(int), cudaMemcpyHostToDevice, st));
            PDD_CUDA(cudaMemcpyAsync(dnp.p, np.data(), np.size() * sizeof(int), cudaMemcpyHostToDevice, st));
            PDD_CUDA(cudaMemcpyAsync(dgsl.p, gsl.data(), gsl.size() * sizeof(int), cudaMemcpyHostToDevice, st));
            PDD_CUDA(cudaMemcpyAsync(droff.p, roff.data(), roff.size() * sizeof(long), cudaMemcpyHostToDevice, st));
            if ((size_t)off > side.n) {
                side.alloc(off);
                su.alloc(off);
                Y.alloc(off);
                Z.alloc(off);
                if (mixed) ez.alloc(off);
                if (ncv) cvq.alloc((size_t)off * ncv);
            }
            run_wave(drows.p, (int)rows.size(), dnp.p, droff.p, dgsl.p, sys.mom_ptr.p, sys.bmean.p, 0);
        }
    }
    PDD_CUDA(cudaMemcpyAsync(sys.mc_np.p, need.data(), nmc * sizeof(int), cudaMemcpyHostToDevice, st));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    unsigned long long hs = 0;
    int hc = 0;
    PDD_CUDA(cudaMemcpyAsync(&hs, steps.p, sizeof(hs), cudaMemcpyDeviceToHost, st));
    PDD_CUDA(cudaMemcpyAsync(&hc, capped.p, sizeof(hc), cudaMemcpyDeviceToHost, st));
    PDD_CUDA(cudaStreamSynchronize(st));
    ms.steps = (int64_t)hs;
    ms.capped = hc;
    ms.ms_paths = tp;
    ms.ms_finalize = tf;
    return ms;
}

}  // namespace pdd

// ---------------------------------------------------------------------------
// a14 (perimeter rows): replay each row's paths with the same Philox streams
// (common random numbers).  The paths X do not depend on c, f or g; only the
// weights do.  With S_q = sum_k 1{c<0} psi_q(X_k) h / (1 + c(X_k) h),
// dY_tau/dw_q = Y_tau S_q and dZ/dw_q = sum_k f(X_k) h Y_k S_q(k).  The row adds
// lambda_i E[(1_dOmega g + 1_Gamma u_hat) dY_q + dZ_q] to dJ/dw_q and
// lambda_i E[1_dOmega psi^g_k(s) Y_tau] to dJ/da_k.
// ---------------------------------------------------------------------------
namespace pdd {

struct GradArgs {
    const double *u, *lambda;
    const int *knot_ptr;
    const uint8_t *floating;
    const double *ku;
    const long *kinv_off;
    const double *kinv;
    double c2;
    int n_par;
    double *partial;          // [slot][n_rbf + n_gcoef]
};

template <typename R, bool SRC>
__global__ void __launch_bounds__(64) k_paths_grad(Problem P, PathArgs A, GradArgs G) {
    extern __shared__ double gsm[];
    const int T = blockDim.x, tid = threadIdx.x;
    const int nw = P.n_rbf, ng = (P.g_kind == PDD_G_BOUNDARY_FOURIER) ? P.n_gcoef : 0;
    const int nf = (P.f_kind == PDD_F_RBF) ? P.n_frbf : 0;
    double *alpha = gsm;                         // kMaxStencil
    double *S = alpha + kMaxStencil;             // [nw][T]
    double *dZ = S + (size_t)nw * T;             // [nw][T]
    double *Gw = dZ + (size_t)nw * T;            // [nw][T]
    double *Gg = Gw + (size_t)nw * T;            // [ng][T]
    double *Gf = Gg + (size_t)ng * T;            // [nf][T]: sum over paths of dZ_tau / dv_q
    const int slot = blockIdx.x;
    const int gsl = A.gslot ? A.gslot[slot] : slot;
    const int i = A.rows[slot], m = A.subs[gsl];
    const uint32_t kw = A.kword ? (uint32_t)A.kword[gsl] : 0u;
    const int a = G.knot_ptr[m], ns = G.knot_ptr[m + 1] - a;
    const bool imq = !G.floating[m];
    // u_hat(u) = sum_l alpha_l phi_l(u) (IMQ) or sum_j u_j H_j(theta) (Fourier cardinals)
    for (int l = tid; l < ns; l += T) {
        double v = 0.0;
        if (imq) {
            const double *Ki = G.kinv + G.kinv_off[m];
            for (int j = 0; j < ns; ++j) v += Ki[l * ns + j] * G.u[a + j];
        } else {
            v = G.u[a + l];
        }
        alpha[l] = v;
    }
    for (int q = 0; q < nw; ++q) Gw[q * T + tid] = 0.0;
    for (int k = 0; k < ng; ++k) Gg[k * T + tid] = 0.0;
    for (int q = 0; q < nf; ++q) Gf[q * T + tid] = 0.0;
    __syncthreads();
    const double inv2f = nf ? 1.0 / (2.0 * P.frbf_sigma * P.frbf_sigma) : 0.0;
    const double cx = A.ccx[m], cy = A.ccy[m], rad = A.cr[m];
    // the same exit rule as k_paths: disk and domain shrunk by the boundary shift (0: plain)
    const double rs = rad - A.shift;
    const R rcx = (R)cx, rcy = (R)cy, r2 = (R)(rs * rs);
    Problem Ps = P;
    if (P.dom_kind == 0) {
        Ps.dom[0] += A.shift;
        Ps.dom[1] += A.shift;
        Ps.dom[2] -= A.shift;
        Ps.dom[3] -= A.shift;
    } else {
        Ps.dom[2] -= A.shift;
    }
    const int max_steps = A.max_steps > 0 ? A.max_steps : (int)fmin(2147483647.0, ceil(50.0 * rad * rad / A.h));
    const R h = (R)A.h, sh = Num<R>::sq((R)A.h);
    const double inv2s = nw ? 1.0 / (2.0 * P.rbf_sigma * P.rbf_sigma) : 0.0;
    const int npath = A.npaths ? A.npaths[slot] : A.paths;
    for (int p = tid; p < npath; p += T) {
        R x = (R)A.kx[i], y = (R)A.ky[i];
        double Yv = 1.0, Zv = 0.0;
        for (int q = 0; q < nw; ++q) {
            S[q * T + tid] = 0.0;
            dZ[q * T + tid] = 0.0;
        }
        int k = 0;
        int side = 2;
        double su = 0.0;
        for (;;) {
            if (k >= max_steps) break;
            R xi0, xi1;
            Num<R>::normals(A.seed, (uint32_t)i, kw, (uint32_t)k, (uint32_t)p, xi0, xi1);
            R bx, by;
            Num<R>::drift(P, x, y, bx, by);
            const double xd = (double)x, yd = (double)y;
            double cv = 0.0;
            if (P.c_kind == PDD_C_RBF) {
                double s = 0.0;
                for (int q = 0; q < nw; ++q) {
                    const double ddx = xd - P.rbf_x[q], ddy = yd - P.rbf_y[q];
                    s += P.rbf_w[q] * exp(-(ddx * ddx + ddy * ddy) * inv2s);
                }
                cv = s < 0.0 ? s : 0.0;
            } else {
                cv = (sizeof(R) == 8) ? killing(P, xd, yd) : (double)killing32(P, (float)x, (float)y);
            }
            const double fv = SRC ? ((sizeof(R) == 8) ? source(P, xd, yd) : (double)source32(P, (float)x, (float)y)) : 0.0;
            if (nw && cv < 0.0) {
                const double fac = A.h / (1.0 + cv * A.h);
                for (int q = 0; q < nw; ++q) {
                    const double ddx = xd - P.rbf_x[q], ddy = yd - P.rbf_y[q];
                    const double psi = exp(-(ddx * ddx + ddy * ddy) * inv2s);
                    if (SRC) dZ[q * T + tid] += fv * A.h * Yv * S[q * T + tid];
                    S[q * T + tid] += psi * fac;
                }
            } else if (SRC && nw) {
                for (int q = 0; q < nw; ++q) dZ[q * T + tid] += fv * A.h * Yv * S[q * T + tid];
            }
            const double Yn = Yv * (1.0 + cv * A.h);
            const double Zn = Zv + fv * Yv * A.h;
            // f's weights: dZ_{k+1} / dv_q = dZ_k / dv_q + psi^f_q(X_k) Y_k h (kept for the paths that exit)
            for (int q = 0; q < nf; ++q) {
                const double ddx = xd - P.frbf_x[q], ddy = yd - P.frbf_y[q];
                Gf[q * T + tid] += exp(-(ddx * ddx + ddy * ddy) * inv2f) * Yv * A.h;
            }
            const R nx = x + bx * h + sh * xi0;
            const R ny = y + by * h + sh * xi1;
            ++k;
            const R ddx = nx - rcx, ddy = ny - rcy;
            const bool out_c = !(ddx * ddx + ddy * ddy < r2);
            const bool out_d = !inside_domain(Ps, (double)nx, (double)ny);
            if (!out_c && !out_d) {
                x = nx;
                y = ny;
                Yv = Yn;
                Zv = Zn;
                continue;
            }
            const double dx = (double)nx - xd, dy = (double)ny - yd;
            double tc = 2.0, td = 2.0;
            int ed = -1;
            if (out_c) tc = circle_exit_t(xd, yd, dx, dy, cx, cy, rs);
            if (out_d) {
                if (Ps.dom_kind == 0) {
                    double t;
                    if ((double)nx <= Ps.dom[0]) { t = (Ps.dom[0] - xd) / dx; if (t < td) { td = t; ed = 3; } }
                    if ((double)nx >= Ps.dom[2]) { t = (Ps.dom[2] - xd) / dx; if (t < td) { td = t; ed = 1; } }
                    if ((double)ny <= Ps.dom[1]) { t = (Ps.dom[1] - yd) / dy; if (t < td) { td = t; ed = 0; } }
                    if ((double)ny >= Ps.dom[3]) { t = (Ps.dom[3] - yd) / dy; if (t < td) { td = t; ed = 2; } }
                } else {
                    td = circle_exit_t(xd, yd, dx, dy, Ps.dom[0], Ps.dom[1], Ps.dom[2]);
                    ed = 0;
                }
            }
            const bool proj = A.shift > 0.0;
            if (td <= tc) {
                side = 1;
                double ex = xd + td * dx, ey = yd + td * dy;
                if (proj) {                          // projection onto the true boundary
                    ex = (double)nx;
                    ey = (double)ny;
                    if (P.dom_kind == 0) {
                        ex = ex < P.dom[0] ? P.dom[0] : (ex > P.dom[2] ? P.dom[2] : ex);
                        ey = ey < P.dom[1] ? P.dom[1] : (ey > P.dom[3] ? P.dom[3] : ey);
                        if (ed == 0) ey = P.dom[1];
                        else if (ed == 1) ex = P.dom[2];
                        else if (ed == 2) ey = P.dom[3];
                        else ex = P.dom[0];
                    }
                }
                su = boundary_s(P, ex, ey, ed);
            } else {
                const double ex = proj ? (double)nx : xd + tc * dx, ey = proj ? (double)ny : yd + tc * dy;
                double th = atan2(ey - cy, ex - cx);
                if (th < 0.0) th += PDD_TWO_PI;
                double uu = th - A.theta_s[m];
                if (uu < 0.0) uu += PDD_TWO_PI;
                if (uu >= PDD_TWO_PI) uu -= PDD_TWO_PI;
                side = 0;
                su = uu;
            }
            Yv = Yn;
            Zv = Zn;
            break;
        }
        if (side == 2) continue;
        double payoff;
        if (side == 1) {
            double ex, ey;
            boundary_point(P, su, ex, ey);
            payoff = gdata(P, ex, ey, su);
            if (ng) {
                const int kc = (P.n_gcoef + 1) / 2;
                const double wv = PDD_TWO_PI * su / P.perimeter;
                for (int kk = 0; kk < ng; ++kk) {
                    const double basis = (kk < kc) ? cos(kk * wv) : sin((kk - kc + 1) * wv);
                    Gg[kk * T + tid] += Yv * basis;
                }
            }
        } else {
            payoff = 0.0;
            for (int l = 0; l < ns; ++l) {
                double ph;
                if (imq) {
                    const double d = su - G.ku[a + l];
                    ph = 1.0 / sqrt(d * d + G.c2);
                } else {
                    double xx = remainder(su - PDD_TWO_PI * l / ns, PDD_TWO_PI);
                    ph = (xx == 0.0) ? 1.0 : sin(0.5 * ns * xx) * cos(0.5 * xx) / (sin(0.5 * xx) * ns);
                }
                payoff += alpha[l] * ph;
            }
        }
        for (int q = 0; q < nw; ++q) Gw[q * T + tid] += payoff * Yv * S[q * T + tid] + dZ[q * T + tid];
    }
    __syncthreads();
    // partial layout [c weights][f weights][g coefficients]
    const double scale = G.lambda[i] / npath;
    for (int q = tid; q < nw + nf + ng; q += T) {
        const double *src = (q < nw) ? Gw + (size_t)q * T
                                     : (q < nw + nf ? Gf + (size_t)(q - nw) * T : Gg + (size_t)(q - nw - nf) * T);
        double s = 0.0;
        for (int t = 0; t < T; ++t) s += src[t];
        G.partial[(long)slot * G.n_par + q] = scale * s;
    }
}

void grad_mc(const pdd_cover &cov, const Problem &P, const pdd_assembly_opts &o, const pdd_system &sys,
             const double *u, const double *lambda, DevBuf<double> &partial, int &n_part, cudaStream_t st) {
    n_part = 0;
    const int nmc = sys.n_mc;
    const int nw = (P.c_kind == PDD_C_RBF) ? P.n_rbf : 0;
    const int ng = (P.g_kind == PDD_G_BOUNDARY_FOURIER) ? P.n_gcoef : 0;
    const int nf = (P.f_kind == PDD_F_RBF) ? P.n_frbf : 0;
    if (nmc == 0 || nw + nf + ng == 0) return;
    DevBuf<double> kinv, kcond;
    DevBuf<long> koff_m;
    build_imq_inverses(cov, o.imq_c2, kinv, koff_m, kcond, st);
    const int n_par = nw + nf + ng;
    partial.alloc((size_t)nmc * n_par);
    PDD_CUDA(cudaMemsetAsync(partial.p, 0, sizeof(double) * nmc * n_par, st));
    DevBuf<unsigned long long> steps;
    DevBuf<int> capped;
    steps.alloc(1);
    capped.alloc(1);
    PathArgs A{sys.mc_rows.p, sys.mc_subs.p, sys.mc_kword.p, cov.kx.p, cov.ky.p, cov.cx.p, cov.cy.p, cov.r.p,
               cov.theta_s.p, o.paths, o.h, o.seed, nullptr, nullptr, nullptr, nullptr, steps.p, capped.p,
               sys.mc_np.p, nullptr, nullptr, o.boundary_shift ? kGmC0 * sqrt(o.h) : 0.0, nullptr, o.max_steps, 0, 0,
               nullptr};
    GradArgs G{u, lambda, cov.knot_ptr.p, cov.floating.p, cov.ku.p, koff_m.p, kinv.p, o.imq_c2, n_par, partial.p};
    const int T = 64;
    const size_t smem = (size_t)(kMaxStencil + (3 * nw + ng + nf) * T) * sizeof(double);
    if (smem > 220 * 1024) fail(PDD_EINVAL, "too many gradient parameters for the replay kernel");
    const bool src = P.f_kind != PDD_F_ZERO;
#define PDD_GRAD_LAUNCH(R, SRCV)                                                                          \
    do {                                                                                                  \
        PDD_CUDA(cudaFuncSetAttribute(k_paths_grad<R, SRCV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                      (int)smem));                                                       \
        PDD_LAUNCH((k_paths_grad<R, SRCV>), nmc, T, smem, st, P, A, G);                                   \
    } while (0)
    if (path_mixed(o)) {
        if (src) PDD_GRAD_LAUNCH(float, true); else PDD_GRAD_LAUNCH(float, false);
    } else {
        if (src) PDD_GRAD_LAUNCH(double, true); else PDD_GRAD_LAUNCH(double, false);
    }
#undef PDD_GRAD_LAUNCH
    n_part = nmc;
}

}  // namespace pdd

namespace pdd {
__global__ void k_split_df(const double *v, float2 *out, long n) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t < n) out[t] = split_df_bits(v[t]);
}
}  // namespace pdd

// C ABI: the double-float split of the finalize's sum mode 1 (see include/pdd.h)
extern "C" pdd_status pdd_split_df(const double *v_dev, float *hilo_dev, long long n, void *stream) {
    using namespace pdd;
    try {
        if (n < 0 || (n > 0 && (!v_dev || !hilo_dev))) fail(PDD_EINVAL, "negative count or null buffer");
        if (((uintptr_t)hilo_dev & 7) != 0) fail(PDD_EINVAL, "output not 8-byte aligned");
        if (n == 0) return PDD_OK;
        cudaStream_t st = (cudaStream_t)stream;
        PDD_LAUNCH(k_split_df, (unsigned)cdiv((long)n, 256), 256, 0, st, v_dev, reinterpret_cast<float2 *>(hilo_dev),
                   (long)n);
        PDD_CUDA(cudaStreamSynchronize(st));
    } catch (const Fail &f) {
        return f.st;
    }
    return PDD_OK;
}
