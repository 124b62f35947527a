// Internal header of the GB300 library: status plumbing, launch accounting,
// the device-side problem description (Eq. 1-3) and the Philox4x32-10
// generator.  Nothing here is part of the C ABI (include/pdd.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "../../include/pdd.h"

namespace pdd {

// ---------------------------------------------------------------------------
// status plumbing
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
std::string cuda_msg(cudaError_t e, const char *what);
void count_launch(int n = 1);

struct Fail {
    pdd_status st;
};

#define PDD_CUDA(call)                                                          \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) {                                                \
            ::pdd::set_error(::pdd::cuda_msg(e_, #call));                       \
            throw ::pdd::Fail{e_ == cudaErrorMemoryAllocation ? PDD_ENOMEM     \
                                                               : PDD_ECUDA};   \
        }                                                                       \
    } while (0)

// launch accounting: every kernel launch goes through this macro
#define PDD_LAUNCH(kernel, grid, block, smem, stream, ...)                      \
    do {                                                                        \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);             \
        ::pdd::count_launch();                                                  \
        PDD_CUDA(cudaGetLastError());                                           \
    } while (0)

inline void fail(pdd_status st, const std::string &msg) {
    set_error(msg);
    throw Fail{st};
}

// device buffer owned by a handle
template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    void alloc(size_t count) {
        release();
        if (count == 0) return;
        PDD_CUDA(cudaMalloc((void **)&p, count * sizeof(T)));
        n = count;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    ~DevBuf() { release(); }
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
};

inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// problem description passed by value to kernels (Eq. 1-3 with sigma = I)
// ---------------------------------------------------------------------------
struct Problem {
    int dom_kind;          // 0 square (x0,y0,x1,y1), 1 disk (cx,cy,R)
    double dom[4];
    int b_kind, c_kind, f_kind, g_kind;
    int n_rbf;
    const double *rbf_x, *rbf_y, *rbf_w;   // device
    double rbf_sigma;
    int n_gcoef;
    const double *g_coef;                  // device
    double perimeter;
    const float *rbf32;                    // device: the RBF centres and weights as FP32, x[n] y[n] w[n]
    float rbf_inv2s2;                      // 1 / (2 sigma^2) in FP32
    int n_frbf;                            // f = sum_q v_q exp(-|x - x_q|^2 / (2 s_f^2)) (PDD_F_RBF)
    const double *frbf_x, *frbf_y, *frbf_w;   // device
    double frbf_sigma;
    const float *frbf32;                   // device: FP32 x[n] y[n] v[n]
    float frbf_inv2s2;
};

#define PDD_PI 3.141592653589793
#define PDD_TWO_PI 6.283185307179586

__device__ __forceinline__ bool inside_domain(const Problem &P, double x, double y) {
    if (P.dom_kind == 0) return x > P.dom[0] && x < P.dom[2] && y > P.dom[1] && y < P.dom[3];
    double dx = x - P.dom[0], dy = y - P.dom[1];
    return dx * dx + dy * dy < P.dom[2] * P.dom[2];
}

__device__ __forceinline__ void drift(const Problem &P, double x, double y, double &bx, double &by) {
    if (P.b_kind == PDD_B_SINX_COSY) {
        bx = sin(x);
        by = cos(y);
    } else {
        bx = 0.0;
        by = 0.0;
    }
}

__device__ __forceinline__ double rbf_sum(const Problem &P, double x, double y) {
    double s = 0.0;
    const double inv = 1.0 / (2.0 * P.rbf_sigma * P.rbf_sigma);
    for (int q = 0; q < P.n_rbf; ++q) {
        double dx = x - P.rbf_x[q], dy = y - P.rbf_y[q];
        s += P.rbf_w[q] * exp(-(dx * dx + dy * dy) * inv);
    }
    return s;
}

__device__ __forceinline__ double killing(const Problem &P, double x, double y) {
    if (P.c_kind == PDD_C_QUADRATIC) return -(1.0 + x * x + y * y);
    if (P.c_kind == PDD_C_RBF) {
        double s = rbf_sum(P, x, y);
        return s < 0.0 ? s : 0.0;
    }
    return 0.0;
}

// exact solution of the Poisson test (Eq. 46) with its gradient and Laplacian:
// u = 3 + sin(s)/3 + tanh(w)/3, s = sqrt(1 + x^2/100 + y^2/50), w = sin(a) + sin(b),
// a = 3x/25 + y/20, b = x/20 - 3y/25.  Lap s = (1/100 + 1/50 - |grad s|^2)/s and
// Lap w = -((3/25)^2 + (1/20)^2) w; tanh'' = -2 tanh sech^2.
__device__ __forceinline__ void sincos_t(double v, double *s, double *c) { sincos(v, s, c); }
__device__ __forceinline__ void sincos_t(float v, float *s, float *c) { sincosf(v, s, c); }
__device__ __forceinline__ double sqrt_t(double v) { return sqrt(v); }
__device__ __forceinline__ float sqrt_t(float v) { return sqrtf(v); }
__device__ __forceinline__ double tanh_t(double v) { return tanh(v); }
__device__ __forceinline__ float tanh_t(float v) { return tanhf(v); }

template <typename T>
__device__ __forceinline__ void u46_derivs(T x, T y, T &u, T &ux, T &uy, T &lap) {
    const T s = sqrt_t(T(1) + x * x * T(0.01) + y * y * T(0.02));
    const T rs = T(1) / s;
    const T sx = x * T(0.01) * rs, sy = y * T(0.02) * rs;
    const T g2s = sx * sx + sy * sy;
    const T lap_s = (T(0.03) - g2s) * rs;
    const T a = x * T(0.12) + y * T(0.05), b = x * T(0.05) - y * T(0.12);
    T sa, ca, sb, cb, ss, cs;
    sincos_t(a, &sa, &ca);
    sincos_t(b, &sb, &cb);
    sincos_t(s, &ss, &cs);
    const T w = sa + sb;
    const T wx = T(0.12) * ca + T(0.05) * cb, wy = T(0.05) * ca - T(0.12) * cb;
    const T lap_w = T(-0.0169) * w;
    const T t = tanh_t(w), sech2 = T(1) - t * t;
    const T third = T(1) / T(3);
    u = T(3) + (ss + t) * third;
    ux = (cs * sx + sech2 * wx) * third;
    uy = (cs * sy + sech2 * wy) * third;
    lap = (cs * lap_s - ss * g2s + sech2 * (lap_w - T(2) * t * (wx * wx + wy * wy))) * third;
}

__device__ __forceinline__ double source(const Problem &P, double x, double y) {
    if (P.f_kind == PDD_F_RBF) {
        const double inv = 1.0 / (2.0 * P.frbf_sigma * P.frbf_sigma);
        double s = 0.0;
        for (int q = 0; q < P.n_frbf; ++q) {
            const double dx = x - P.frbf_x[q], dy = y - P.frbf_y[q];
            s += P.frbf_w[q] * exp(-(dx * dx + dy * dy) * inv);
        }
        return s;
    }
    if (P.f_kind == PDD_F_ONE) return 1.0;
    if (P.f_kind == PDD_F_MANUFACTURED) {
        double spx, cpx, spy, cpy;
        sincospi(x, &spx, &cpx);
        sincospi(y, &spy, &cpy);
        double u = spx * cpy;
        double ux = PDD_PI * cpx * cpy;
        double uy = -PDD_PI * spx * spy;
        double bx, by;
        drift(P, x, y, bx, by);
        return -(-PDD_PI * PDD_PI * u + bx * ux + by * uy + killing(P, x, y) * u);
    }
    if (P.f_kind == PDD_F_EQ46) {
        double u, ux, uy, lap, bx, by;
        u46_derivs(x, y, u, ux, uy, lap);
        drift(P, x, y, bx, by);
        return -(0.5 * lap + bx * ux + by * uy + killing(P, x, y) * u);
    }
    return 0.0;
}

// boundary Fourier series at arclength s (a_0..a_{Kc-1} cos, b_1..b_Ks sin)
__device__ __forceinline__ double g_fourier(const Problem &P, double s) {
    int kc = (P.n_gcoef + 1) / 2, ks = P.n_gcoef - kc;
    double w = PDD_TWO_PI * s / P.perimeter;
    double acc = 0.0;
    for (int k = 0; k < kc; ++k) acc += P.g_coef[k] * cos(k * w);
    for (int k = 1; k <= ks; ++k) acc += P.g_coef[kc + k - 1] * sin(k * w);
    return acc;
}

// boundary point of arclength s (square: counter-clockwise from (x0, y0))
__device__ __forceinline__ void boundary_point(const Problem &P, double s, double &x, double &y) {
    if (P.dom_kind == 0) {
        double x0 = P.dom[0], y0 = P.dom[1], x1 = P.dom[2], y1 = P.dom[3];
        double w = x1 - x0, h = y1 - y0;
        if (s < w) { x = x0 + s; y = y0; }
        else if (s < w + h) { x = x1; y = y0 + (s - w); }
        else if (s < 2.0 * w + h) { x = x1 - (s - w - h); y = y1; }
        else { x = x0; y = y1 - (s - 2.0 * w - h); }
    } else {
        double t = s / P.dom[2];
        double st, ct;
        sincos(t, &st, &ct);
        x = P.dom[0] + P.dom[2] * ct;
        y = P.dom[1] + P.dom[2] * st;
    }
}

// arclength of a boundary point on edge e (square) or the disk
__device__ __forceinline__ double boundary_s(const Problem &P, double x, double y, int e) {
    if (P.dom_kind == 0) {
        double x0 = P.dom[0], y0 = P.dom[1], x1 = P.dom[2], y1 = P.dom[3];
        double w = x1 - x0, h = y1 - y0;
        if (e == 0) return x - x0;
        if (e == 1) return w + (y - y0);
        if (e == 2) return w + h + (x1 - x);
        return 2.0 * w + h + (y1 - y);
    }
    double t = atan2(y - P.dom[1], x - P.dom[0]);
    if (t < 0.0) t += PDD_TWO_PI;
    return P.dom[2] * t;
}

__device__ __forceinline__ double gdata(const Problem &P, double x, double y, double s) {
    switch (P.g_kind) {
        case PDD_G_EXP_SIN: return exp(x) * sin(y);
        case PDD_G_SIN_COS: {
            double a, b;
            a = sinpi(x);
            b = cospi(y);
            return a * b;
        }
        case PDD_G_BOUNDARY_FOURIER: return g_fourier(P, s);
        case PDD_G_ONE: return 1.0;
        case PDD_G_EQ46: {
            double u, ux, uy, lap;
            u46_derivs(x, y, u, ux, uy, lap);
            return u;
        }
        default: return 0.0;
    }
}

// nearest edge of the square (for Dirichlet knots of the Fourier data)
__device__ __forceinline__ int nearest_edge(const Problem &P, double x, double y) {
    if (P.dom_kind != 0) return 0;
    double d[4] = {fabs(y - P.dom[1]), fabs(x - P.dom[2]), fabs(y - P.dom[3]), fabs(x - P.dom[0])};
    int e = 0;
    for (int k = 1; k < 4; ++k)
        if (d[k] < d[e]) e = k;
    return e;
}

// ---------------------------------------------------------------------------
// double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32
// numbers (Dekker 1971; Knuth's two-sum).  Products use __fmul_rn so that the
// compiler cannot contract them into the following addition.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 df_split(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
    const float h = p + e;
    return make_float2(h, e - (h - p));
}

__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    e += a.y + b.y;
    const float h = s + e;
    return make_float2(h, e - (h - s));
}

// (sh, sl) += w x, the accumulator left unnormalised
__device__ __forceinline__ void df_acc(float &sh, float &sl, float2 w, float2 x) {
    const float p = __fmul_rn(w.x, x.x);
    float e = fmaf(w.x, x.x, -p);
    e = fmaf(w.x, x.y, fmaf(w.y, x.x, e));
    float s, t;
    two_sum(sh, p, s, t);
    sh = s;
    sl += t + e;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // each 32 x 32 -> 64-bit product as one wide multiply (both halves from one instruction)
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

// two 53-bit uniforms in (0, 1] from the four words
__device__ __forceinline__ double uniform53(uint32_t a, uint32_t b) {
    uint64_t m = ((uint64_t)a << 21) ^ (uint64_t)(b >> 11);
    return ((double)m + 0.5) * 1.1102230246251565e-16;
}

// key (seed_lo32, knot), counter (step, path, 0, sub): sub is the position of the subdomain in the
// row's list Pi_i (0 unless the row averages several subdomains)
__device__ __forceinline__ void normals64(uint64_t seed, uint32_t knot, uint32_t sub, uint32_t step, uint32_t path,
                                          double &xi0, double &xi1) {
    U4 w = philox10(step, path, 0u, sub, (uint32_t)(seed & 0xffffffffu), knot);
    double u1 = uniform53(w.x, w.y);
    double u2 = uniform53(w.z, w.w);
    double rr = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    xi0 = rr * c;
    xi1 = rr * s;
}

// round to the nearest integer with FP32 additions (exact for |x| < 2^22):
// adding and subtracting 1.5 2^23 leaves x rounded to an integer, on the FMA
// pipe instead of a round instruction
__device__ __forceinline__ float round_fma(float x) {
    const float big = 12582912.0f;
    return __fsub_rn(__fadd_rn(x, big), big);
}

// FP32 sine and cosine for the mixed form: the argument is reduced to [-pi, pi]
// (where the hardware approximations __sinf/__cosf/__sincosf keep an absolute
// error near 2^-21) and the approximation is taken there
__device__ __forceinline__ float reduce_2pi(float x) {
    return x - 6.28318530717958647692f * round_fma(x * 0.159154943091895335769f);
}

// sin(pi x) and cos(pi x): x - 2 round(x / 2) is exact, then as above
__device__ __forceinline__ void fast_sincospi(float x, float &s, float &c) {
    const float t = x - 2.0f * round_fma(0.5f * x);
    __sincosf(3.14159265358979323846f * t, &s, &c);
}

// 23-bit uniforms in (0, 1) for the mixed-precision form, built from the
// mantissa bits (no conversion instruction): [1.m] - 1 = m 2^-23 with
// m = w >> 9 (exact), plus half a step; u follows the leading bits of w like
// the 53-bit form does
__device__ __forceinline__ float uniform23(uint32_t w) {
    return (__uint_as_float(0x3f800000u | (w >> 9)) - 1.0f) + 0x1p-24f;
}

__device__ __forceinline__ void normals32(uint64_t seed, uint32_t knot, uint32_t sub, uint32_t step, uint32_t path,
                                          float &xi0, float &xi1) {
    U4 w = philox10(step, path, 0u, sub, (uint32_t)(seed & 0xffffffffu), knot);
    const float u1 = uniform23(w.x);
    const float u2 = uniform23(w.z);
    const float rr = sqrtf(-2.0f * __logf(u1));
    float s, c;
    fast_sincospi(2.0f * u2, s, c);
    xi0 = rr * c;
    xi1 = rr * s;
}

}  // namespace pdd
