/*
 * Plain FP64 Euler-Maruyama Feynman-Kac paths for one knot (a11).
 * TEST INFRASTRUCTURE ONLY: part of the oracle; never linked into the library.
 *
 * The elliptic Feynman-Kac representation (Appendix, Eq. 53 and 56, and
 * Eq. 25-30 of the paper) with sigma = I:
 *     dX = b(X) dt + dW,   dY = c(X) Y dt,   dZ = f(X) Y dt,
 *     X_0 = x_i, Y_0 = 1, Z_0 = 0,
 * stopped at the first exit tau from the subdomain O_m n Omega (Eq. 26).
 *
 * Discretisation (plain Euler-Maruyama, step h, left-point weights):
 *     X_{k+1} = X_k + b(X_k) h + sqrt(h) xi_k
 *     Y_{k+1} = Y_k (1 + c(X_k) h)
 *     Z_{k+1} = Z_k + f(X_k) Y_k h
 * The path exits at the first step whose end point is outside the open disk
 * or outside the open domain.  The exit point is where the segment
 * X_k -> X_{k+1} first meets the circle or dOmega (smaller segment parameter;
 * a tie goes to dOmega).  The weights are the ones after the exit step.
 *
 * Boundary shift (the Gobet-Menozzi stopped-diffusion correction, Stoch.
 * Proc. Appl. 120 (2010); the paper's perimeter subdomains use it, Sec. 4):
 * with shift = c0 |sigma^T n| sqrt(h) > 0 (sigma = I; c0 = -zeta(1/2)/sqrt(2 pi)
 * = 0.5826) the exit test uses the disk and the domain shrunk by `shift`, the
 * piece left first is chosen as above on the shrunk boundaries, and the path
 * is scored at the projection of its first point outside onto that piece of
 * the true boundary (radial for circles, onto the edge for the square).
 *
 * Normals: Philox4x32-10 (Salmon et al., SC'11) with key (seed_lo32, knot) and
 * counter (step, path, 0, k), k = the position of the subdomain in the row's
 * list Pi_i (0 unless the row averages several subdomains, Eq. 38-39).  The four 32-bit words (a, b, c, d) give two
 * 53-bit uniforms u1 = ((a << 21) ^ (b >> 11) + 0.5) 2^-53 and likewise u2
 * from (c, d); Box-Muller gives xi = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).
 *
 * Control-variate features (optional, cv_degree = D > 0): for the monomials
 * psi = xr^a yr^b (1 <= a + b <= D) of xr = (x - cx) / r, yr = (y - cy) / r, the
 * discrete martingales Q = sum_k Y_k grad psi(X_k) . sqrt(h) xi_k (sigma = I),
 * which have mean zero for any psi because xi_k is independent of X_k and Y_k
 * (Newton 1994; Milstein and Tretyakov, SIAM J. Numer. Anal. 47 (2009)):
 *   grad psi . xi = (a xr^(a-1) yr^b xi_x + b xr^a yr^(b-1) xi_y) / r.
 * Stored per path in the order d = a + b = 1..D, a = d..0: D (D + 3) / 2
 * features (at most 14, D <= 4).
 *
 * Output per path: side (0 interface, 1 domain boundary, 2 step cap),
 * boundary edge, exit point, exit angle about the centre, Y_tau, Z_tau,
 * number of steps, the control-variate features, and optionally the pathwise
 * derivatives of Y_tau and Z_tau with respect to the RBF weights of c (for the
 * adjoint check).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef struct {
    int dom_kind;            /* 0 square (x0,y0,x1,y1), 1 disk (cx,cy,R) */
    double dom[4];
    int b_kind;              /* 0 zero, 1 (sin x, cos y) */
    int c_kind;              /* 0 zero, 1 -(1+x^2+y^2), 2 rbf */
    int f_kind;              /* 0 zero, 1 one, 2 manufactured sin(pi x)cos(pi y), 3 Eq. 46, 4 rbf */
    int n_rbf;
    const double *rbf_x, *rbf_y, *rbf_w;
    double rbf_sigma;
    int n_frbf;              /* f = sum_q v_q exp(-|x - x_q|^2 / (2 s_f^2)) (f_kind 4) */
    const double *frbf_x, *frbf_y, *frbf_w;
    double frbf_sigma;
} oracle_problem;

typedef struct {
    double cx, cy, r;        /* the subdomain's circle */
    double x0, y0;           /* the knot */
    uint32_t knot;
    uint32_t sub;            /* position of the subdomain in Pi_i (Philox counter word 3) */
    uint64_t seed;
    double h;
    int n_paths;
    int max_steps;
    double shift;            /* 0: plain exit; > 0: shrunk boundaries, projected exit point */
    int cv_degree;           /* 0: no control-variate features; D: 2 D features per path */
} oracle_walk;

static void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        if (round < 9) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* exported for the generator tests */
void oracle_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    philox4x32_10(ctr, key, out);
}

static double uniform53(uint32_t a, uint32_t b)
{
    uint64_t m = ((uint64_t)a << 21) ^ (uint64_t)(b >> 11);
    return ((double)m + 0.5) * 1.1102230246251565e-16;   /* 2^-53 */
}

void oracle_normals(uint64_t seed, uint32_t knot, uint32_t sub, uint32_t step, uint32_t path, double *xi)
{
    uint32_t ctr[4] = {step, path, 0u, sub};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), knot};
    uint32_t w[4];
    philox4x32_10(ctr, key, w);
    double u1 = uniform53(w[0], w[1]);
    double u2 = uniform53(w[2], w[3]);
    double rr = sqrt(-2.0 * log(u1));
    double ang = 2.0 * M_PI * u2;
    xi[0] = rr * cos(ang);
    xi[1] = rr * sin(ang);
}

static void drift(const oracle_problem *p, double x, double y, double *bx, double *by)
{
    if (p->b_kind == 1) { *bx = sin(x); *by = cos(y); }
    else { *bx = 0.0; *by = 0.0; }
}

static double rbf_sum(const oracle_problem *p, double x, double y)
{
    double s = 0.0;
    double two_s2 = 2.0 * p->rbf_sigma * p->rbf_sigma;
    for (int q = 0; q < p->n_rbf; ++q) {
        double dx = x - p->rbf_x[q], dy = y - p->rbf_y[q];
        s += p->rbf_w[q] * exp(-(dx * dx + dy * dy) / two_s2);
    }
    return s;
}

static double killing(const oracle_problem *p, double x, double y)
{
    if (p->c_kind == 1) return -(1.0 + x * x + y * y);
    if (p->c_kind == 2) { double s = rbf_sum(p, x, y); return s < 0.0 ? s : 0.0; }
    return 0.0;
}

/* Exact solution of the Poisson test (Eq. 46) with its gradient and Laplacian:
 * u = 3 + sin(s)/3 + tanh(w)/3, s = sqrt(1 + x^2/100 + y^2/50),
 * w = sin(3x/25 + y/20) + sin(x/20 - 3y/25) (chain rule as in problem.py). */
static void u46(double x, double y, double *u, double *ux, double *uy, double *lap)
{
    double s = sqrt(1.0 + x * x / 100.0 + y * y / 50.0);
    double sx = x / (100.0 * s), sy = y / (50.0 * s);
    double g2s = sx * sx + sy * sy;
    double lap_s = (1.0 / 100.0 + 1.0 / 50.0 - g2s) / s;
    double a = 3.0 * x / 25.0 + y / 20.0, b = x / 20.0 - 3.0 * y / 25.0;
    double w = sin(a) + sin(b);
    double wx = 3.0 / 25.0 * cos(a) + cos(b) / 20.0;
    double wy = cos(a) / 20.0 - 3.0 / 25.0 * cos(b);
    double lap_w = -((3.0 / 25.0) * (3.0 / 25.0) + (1.0 / 20.0) * (1.0 / 20.0)) * w;
    double t = tanh(w), sech2 = 1.0 - t * t;
    *u = 3.0 + sin(s) / 3.0 + t / 3.0;
    *ux = (cos(s) * sx + sech2 * wx) / 3.0;
    *uy = (cos(s) * sy + sech2 * wy) / 3.0;
    *lap = (cos(s) * lap_s - sin(s) * g2s + sech2 * (lap_w - 2.0 * t * (wx * wx + wy * wy))) / 3.0;
}

static double frbf_psi(const oracle_problem *p, int q, double x, double y)
{
    double dx = x - p->frbf_x[q], dy = y - p->frbf_y[q];
    return exp(-(dx * dx + dy * dy) / (2.0 * p->frbf_sigma * p->frbf_sigma));
}

static double source(const oracle_problem *p, double x, double y)
{
    if (p->f_kind == 4) {
        double s = 0.0;
        for (int q = 0; q < p->n_frbf; ++q) s += p->frbf_w[q] * frbf_psi(p, q, x, y);
        return s;
    }
    if (p->f_kind == 1) return 1.0;
    if (p->f_kind == 2) {
        double pi = M_PI;
        double u = sin(pi * x) * cos(pi * y);
        double ux = pi * cos(pi * x) * cos(pi * y);
        double uy = -pi * sin(pi * x) * sin(pi * y);
        double bx, by;
        drift(p, x, y, &bx, &by);
        return -(-pi * pi * u + bx * ux + by * uy + killing(p, x, y) * u);
    }
    if (p->f_kind == 3) {
        double u, ux, uy, lap, bx, by;
        u46(x, y, &u, &ux, &uy, &lap);
        drift(p, x, y, &bx, &by);
        return -(0.5 * lap + bx * ux + by * uy + killing(p, x, y) * u);
    }
    return 0.0;
}

static int inside_domain(const oracle_problem *p, double x, double y)
{
    if (p->dom_kind == 0)
        return x > p->dom[0] && x < p->dom[2] && y > p->dom[1] && y < p->dom[3];
    double dx = x - p->dom[0], dy = y - p->dom[1];
    return dx * dx + dy * dy < p->dom[2] * p->dom[2];
}

/* Smallest t in (0, 1] where P + t D leaves the disk |z - o| < rad, P inside. */
static double circle_exit_t(double px, double py, double dx, double dy,
                            double ox, double oy, double rad)
{
    double qx = px - ox, qy = py - oy;
    double a = dx * dx + dy * dy;
    double b = qx * dx + qy * dy;
    double c = qx * qx + qy * qy - rad * rad;      /* < 0 inside */
    double disc = b * b - a * c;
    if (disc < 0.0) disc = 0.0;
    double sq = sqrt(disc);
    if (b >= 0.0) return -c / (b + sq);
    return (sq - b) / a;
}

int oracle_walk_knot(const oracle_problem *p, const oracle_walk *w,
                     int8_t *side, int8_t *edge, double *ex, double *ey, double *etheta,
                     double *Ytau, double *Ztau, int32_t *steps,
                     double *dY, double *dZ, double *Q, double *dZf)
{
    /* dZf (optional, n_paths x n_frbf): d Z_tau / d v_q = sum_k psi^f_q(X_k) Y_k h */
    const int nf = (dZf != NULL && p->f_kind == 4) ? p->n_frbf : 0;
    if (nf > 256) return -1;
    double Sf[256];
    const int ncv = (Q != NULL && w->cv_degree > 0) ? w->cv_degree * (w->cv_degree + 3) / 2 : 0;
    if (w->cv_degree > 4) return -2;
    const double sh = sqrt(w->h);
    const double dl = w->shift > 0.0 ? w->shift : 0.0;
    const double rs = w->r - dl;                         /* shrunk circle and domain */
    const double r2 = rs * rs;
    oracle_problem ps = *p;
    if (p->dom_kind == 0) {
        ps.dom[0] += dl; ps.dom[1] += dl; ps.dom[2] -= dl; ps.dom[3] -= dl;
    } else {
        ps.dom[2] -= dl;
    }
    int capped = 0;
    double S[256], dZacc[256];      /* running sums for the RBF-weight derivatives */
    int nr = (dY != NULL) ? p->n_rbf : 0;
    if (nr > 256) return -1;
    for (int path = 0; path < w->n_paths; ++path) {
        double x = w->x0, y = w->y0, Y = 1.0, Z = 0.0;
        double cvq[16];
        for (int q = 0; q < ncv; ++q) cvq[q] = 0.0;
        for (int q = 0; q < nf; ++q) Sf[q] = 0.0;
        for (int q = 0; q < nr; ++q) { S[q] = 0.0; dZacc[q] = 0.0; }
        int k = 0;
        int done = 0;
        while (!done) {
            if (k >= w->max_steps) {
                side[path] = 2; edge[path] = -1; ex[path] = x; ey[path] = y;
                etheta[path] = 0.0; Ytau[path] = Y; Ztau[path] = Z; steps[path] = k;
                for (int q = 0; q < ncv; ++q) Q[(size_t)path * ncv + q] = 0.0;
                for (int q = 0; q < nf; ++q) dZf[(size_t)path * nf + q] = 0.0;
                ++capped;
                break;
            }
            double xi[2];
            oracle_normals(w->seed, w->knot, w->sub, (uint32_t)k, (uint32_t)path, xi);
            double bx, by;
            drift(p, x, y, &bx, &by);
            double cv = killing(p, x, y);
            double fv = source(p, x, y);
            double nx = x + bx * w->h + sh * xi[0];
            double ny = y + by * w->h + sh * xi[1];
            double Yn = Y * (1.0 + cv * w->h);
            double Zn = Z + fv * Y * w->h;
            for (int q = 0; q < nf; ++q) Sf[q] += frbf_psi(p, q, x, y) * Y * w->h;
            if (ncv) {
                /* Y_k sqrt(h) grad psi(X_k) . xi_k for psi = xr^a yr^b */
                double xr = (x - w->cx) / w->r, yr = (y - w->cy) / w->r;
                double s = Y * sh / w->r;
                double px[5], py[5];
                px[0] = 1.0; py[0] = 1.0;
                for (int e = 1; e <= w->cv_degree; ++e) { px[e] = px[e - 1] * xr; py[e] = py[e - 1] * yr; }
                int q = 0;
                for (int d = 1; d <= w->cv_degree; ++d)
                    for (int a = d; a >= 0; --a) {
                        int b = d - a;
                        double g = 0.0;
                        if (a > 0) g += a * px[a - 1] * py[b] * xi[0];
                        if (b > 0) g += b * px[a] * py[b - 1] * xi[1];
                        cvq[q++] += s * g;
                    }
            }
            if (nr) {
                /* d/dw_q of Y_{k+1} = Y_k (1 + c_k h):  S_q accumulates psi_q h / (1 + c_k h),
                 * and dZ_{k+1} = dZ_k + f_k h dY_k with dY_k = Y_k S_q (before the update). */
                double two_s2 = 2.0 * p->rbf_sigma * p->rbf_sigma;
                double sum = rbf_sum(p, x, y);
                double active = (p->c_kind == 2 && sum < 0.0) ? 1.0 : 0.0;
                for (int q = 0; q < nr; ++q) {
                    double ddx = x - p->rbf_x[q], ddy = y - p->rbf_y[q];
                    double psi = exp(-(ddx * ddx + ddy * ddy) / two_s2);
                    dZacc[q] += fv * w->h * Y * S[q];
                    S[q] += active * psi * w->h / (1.0 + cv * w->h);
                }
            }
            ++k;
            double ddx = nx - w->cx, ddy = ny - w->cy;
            int out_c = !(ddx * ddx + ddy * ddy < r2);
            int out_d = !inside_domain(&ps, nx, ny);
            if (!out_c && !out_d) { x = nx; y = ny; Y = Yn; Z = Zn; continue; }
            double dx = nx - x, dy = ny - y;
            double tc = 2.0, td = 2.0;
            int ed = -1;
            if (out_c) tc = circle_exit_t(x, y, dx, dy, w->cx, w->cy, rs);
            if (out_d) {
                if (ps.dom_kind == 0) {
                    double t;
                    if (nx <= ps.dom[0]) { t = (ps.dom[0] - x) / dx; if (t < td) { td = t; ed = 3; } }
                    if (nx >= ps.dom[2]) { t = (ps.dom[2] - x) / dx; if (t < td) { td = t; ed = 1; } }
                    if (ny <= ps.dom[1]) { t = (ps.dom[1] - y) / dy; if (t < td) { td = t; ed = 0; } }
                    if (ny >= ps.dom[3]) { t = (ps.dom[3] - y) / dy; if (t < td) { td = t; ed = 2; } }
                } else {
                    td = circle_exit_t(x, y, dx, dy, ps.dom[0], ps.dom[1], ps.dom[2]);
                    ed = 0;
                }
            }
            if (td <= tc) {
                side[path] = 1; edge[path] = (int8_t)ed;
                if (dl > 0.0) {
                    /* projection of the first point outside onto the true boundary piece */
                    if (p->dom_kind == 0) {
                        double qx = nx < p->dom[0] ? p->dom[0] : (nx > p->dom[2] ? p->dom[2] : nx);
                        double qy = ny < p->dom[1] ? p->dom[1] : (ny > p->dom[3] ? p->dom[3] : ny);
                        if (ed == 0) qy = p->dom[1];
                        else if (ed == 1) qx = p->dom[2];
                        else if (ed == 2) qy = p->dom[3];
                        else qx = p->dom[0];
                        ex[path] = qx; ey[path] = qy;
                    } else {
                        double th = atan2(ny - p->dom[1], nx - p->dom[0]);
                        ex[path] = p->dom[0] + p->dom[2] * cos(th);
                        ey[path] = p->dom[1] + p->dom[2] * sin(th);
                    }
                } else {
                    ex[path] = x + td * dx; ey[path] = y + td * dy;
                }
                etheta[path] = 0.0;
            } else {
                side[path] = 0; edge[path] = -1;
                double qx = x + tc * dx, qy = y + tc * dy;
                if (dl > 0.0) { qx = nx; qy = ny; }          /* radial projection below */
                double th = atan2(qy - w->cy, qx - w->cx);
                if (th < 0.0) th += 2.0 * M_PI;
                etheta[path] = th;
                if (dl > 0.0) {
                    ex[path] = w->cx + w->r * cos(th); ey[path] = w->cy + w->r * sin(th);
                } else {
                    ex[path] = qx; ey[path] = qy;
                }
            }
            Ytau[path] = Yn; Ztau[path] = Zn; steps[path] = k;
            for (int q = 0; q < ncv; ++q) Q[(size_t)path * ncv + q] = cvq[q];
            for (int q = 0; q < nf; ++q) dZf[(size_t)path * nf + q] = Sf[q];
            for (int q = 0; q < nr; ++q) {
                dY[(size_t)path * nr + q] = Yn * S[q];
                dZ[(size_t)path * nr + q] = dZacc[q];
            }
            done = 1;
        }
        if (nr && side[path] == 2) {
            for (int q = 0; q < nr; ++q) {
                dY[(size_t)path * nr + q] = 0.0;
                dZ[(size_t)path * nr + q] = 0.0;
            }
        }
    }
    return capped;
}
