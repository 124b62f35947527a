// a1-a5 on the device: cover (Eq. 4-7), interfaces and junctions (Eq. 8, 11),
// knots and stencils (Eq. 9, 12), row assignment (Sec. 3.2 and footnote 3)
// and the CSR pattern of Eq. 29.
//
// This file is compiled with -fmad=false: its FP64 geometry (lattice
// positions, junction points, distances, scores) must round exactly like
// the plain IEEE expressions that define it, so that every integer output
// (which circles are kept or floating, knot counts and order, row owners,
// CSR columns) is reproducible.
//
// Rules where the paper is silent:
//   * knots on a full circle at theta_j = 2 pi j / n;
//   * on an arc: the same candidates strictly inside Omega and at least
//     0.25 * 2 pi / n from every junction, plus one knot per junction;
//   * local order by angle measured from the midpoint of the largest arc
//     outside Omega (first such arc in angle order when lengths agree to 1e-9);
//   * row i goes to the circle with the largest r_m - |x_i - c_m| among those
//     (other than its owner) whose score exceeds 1e-12 r_owner; scores within
//     1e-12 r_owner of the best tie to the lowest circle index;
//   * averaged rows (Eq. 38-39): row i goes to every such circle, ascending.
#include <algorithm>

#include "handles.cuh"

namespace pdd {

static constexpr int kMaxJ = 8;          // junctions per circle (4 square edges x 2)
static constexpr int kMaxKnots = 256;    // knots per circle
static constexpr double kJunctionGap = 0.25;
static constexpr double kScoreEps = 1e-12;

// ---------------------------------------------------------------------------
// Device-wide exclusive scan of int32 counts by warp scans (reduce, scan of the
// tile sums, scan within the tiles): a tile is 1024 threads x 4 counts; a warp
// scans its threads' sums with shuffles, the block its 32 warp sums the same
// way.  out[n] = the total.  64-bit partial sums; no host synchronisation
// unless the caller needs the total (exclusive_scan).
// ---------------------------------------------------------------------------
static constexpr int kScanThreads = 1024, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ long long warp_incl_scan(long long v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive prefix of v over the block (and the block total)
__device__ __forceinline__ long long block_excl_scan(long long v, long long *total) {
    __shared__ long long ws[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long inc = warp_incl_scan(v);
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const long long w = (lane < (int)(blockDim.x >> 5)) ? ws[lane] : 0;
        ws[lane] = warp_incl_scan(w);
    }
    __syncthreads();
    const long long before = (warp > 0 ? ws[warp - 1] : 0) + inc - v;
    if (total) *total = ws[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int *in, int n, long long *tile_sum) {
    const long base = (long)blockIdx.x * kScanTile + (long)threadIdx.x * kScanItems;
    long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += in[base + k];
    long long tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// one block: exclusive offsets of the tile sums (in place), chunk by chunk
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(long long *tile_sum, int ntiles, int *out_last,
                                                            long long *total) {
    long long carry = 0;
    for (int c0 = 0; c0 < ntiles; c0 += kScanThreads) {
        const int i = c0 + threadIdx.x;
        const long long v = i < ntiles ? tile_sum[i] : 0;
        long long tot;
        const long long ex = block_excl_scan(v, &tot);
        if (i < ntiles) tile_sum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        *out_last = (int)carry;
        if (total) *total = carry;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int *in, int *out, int n,
                                                            const long long *tile_off) {
    const long base = (long)blockIdx.x * kScanTile + (long)threadIdx.x * kScanItems;
    int v[kScanItems];
    long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    long long run = tile_off[blockIdx.x] + block_excl_scan(s, nullptr);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) {
            out[base + k] = (int)run;
            run += v[k];
        }
}

// out[0..n] = exclusive prefix sums of in[0..n), out[n] = total; queued on st (no synchronisation);
// the total also goes to *total_dev when given
void exclusive_scan_async(const int *in, int *out, int n, cudaStream_t st, long long *total_dev) {
    const int ntiles = std::max(1, cdiv(n, kScanTile));
    long long *ts = nullptr;                     // stream-ordered: freed after the launches that read it
    PDD_CUDA(cudaMallocAsync((void **)&ts, sizeof(long long) * ntiles, st));
    if (n > 0) PDD_LAUNCH(k_scan_reduce, ntiles, kScanThreads, 0, st, in, n, ts);
    else PDD_CUDA(cudaMemsetAsync(ts, 0, sizeof(long long), st));
    PDD_LAUNCH(k_scan_tiles, 1, kScanThreads, 0, st, ts, ntiles, out + n, total_dev);
    if (n > 0) PDD_LAUNCH(k_scan_apply, ntiles, kScanThreads, 0, st, in, out, n, ts);
    PDD_CUDA(cudaFreeAsync(ts, st));
}

int64_t exclusive_scan(const int *in, int *out, int n, cudaStream_t st) {
    DevBuf<long long> tot;
    tot.alloc(1);
    exclusive_scan_async(in, out, n, st, tot.p);
    long long h = 0;
    PDD_CUDA(cudaMemcpyAsync(&h, tot.p, sizeof(long long), cudaMemcpyDeviceToHost, st));
    PDD_CUDA(cudaStreamSynchronize(st));
    if (h > 0x7fffffffLL) fail(PDD_EINVAL, "count exceeds the int32 index range");
    return h;
}

// ---------------------------------------------------------------------------
// a1: lattice -> keep circles meeting Omega -> classify
// ---------------------------------------------------------------------------
__device__ double dist_closed(const Problem &P, double x, double y) {
    if (P.dom_kind == 0) {
        double dx = fmax(fmax(P.dom[0] - x, 0.0), x - P.dom[2]);
        double dy = fmax(fmax(P.dom[1] - y, 0.0), y - P.dom[3]);
        return sqrt(dx * dx + dy * dy);
    }
    double dx = x - P.dom[0], dy = y - P.dom[1];
    return fmax(sqrt(dx * dx + dy * dy) - P.dom[2], 0.0);
}

__device__ bool contains_closed_disk(const Problem &P, double cx, double cy, double r) {
    if (P.dom_kind == 0)
        return (cx - r > P.dom[0]) && (cx + r < P.dom[2]) && (cy - r > P.dom[1]) && (cy + r < P.dom[3]);
    double dx = cx - P.dom[0], dy = cy - P.dom[1];
    return sqrt(dx * dx + dy * dy) + r < P.dom[2];
}

struct LatticeArgs {
    int kind, nx, ny, n_lat;
    double xo, yo, s, rad;
    const double *ecx, *ecy, *er;
    const int *enk, *enr, *ent;
    int unk, unr, unt;
};

__global__ void k_lattice(Problem P, LatticeArgs L, double *cx, double *cy, double *r, int *nk, int *nr,
                          int *nt, int *keep) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= L.n_lat) return;
    double x, y, rr;
    int a = L.unk, b = L.unr, c = L.unt;
    if (L.kind == PDD_COVER_SQUARE_LATTICE) {
        int j = idx / L.nx, i = idx % L.nx;
        x = L.xo + (double)i * L.s;
        y = L.yo + (double)j * L.s;
        rr = L.rad;
    } else if (L.kind == PDD_COVER_HEX_LATTICE) {
        int k = idx / L.nx, i = idx % L.nx;
        double dy = L.s * sqrt(3.0) * 0.5;
        x = L.xo + (double)i * L.s;
        if (k & 1) x = x + 0.5 * L.s;
        y = L.yo + (double)k * dy;
        rr = L.rad;
    } else {
        x = L.ecx[idx];
        y = L.ecy[idx];
        rr = L.er[idx];
        a = L.enk[idx];
        b = L.enr[idx];
        c = L.ent[idx];
    }
    cx[idx] = x;
    cy[idx] = y;
    r[idx] = rr;
    nk[idx] = a;
    nr[idx] = b;
    nt[idx] = c;
    keep[idx] = dist_closed(P, x, y) < rr ? 1 : 0;
}

__global__ void k_compact_circles(int n_lat, const int *keep, const int *pos, const double *cx,
                                  const double *cy, const double *r, const int *nk, const int *nr,
                                  const int *nt, Problem P, double *ocx, double *ocy, double *orr,
                                  int *onk, int *onr, int *ont, uint8_t *ofl) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_lat || !keep[idx]) return;
    int m = pos[idx];
    ocx[m] = cx[idx];
    ocy[m] = cy[idx];
    orr[m] = r[idx];
    onk[m] = nk[idx];
    onr[m] = nr[idx];
    ont[m] = nt[idx];
    ofl[m] = contains_closed_disk(P, cx[idx], cy[idx], r[idx]) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// a2-a3: junctions, unwrap origin, knots of one circle
// ---------------------------------------------------------------------------
struct Junction {
    double ang, x, y;
};

__device__ double norm_angle(double t) { return t < 0.0 ? t + PDD_TWO_PI : t; }

__device__ int circle_junctions(const Problem &P, double cx, double cy, double r, Junction *J,
                                int *degenerate) {
    int nj = 0;
    if (P.dom_kind == 0) {
        const double x0 = P.dom[0], y0 = P.dom[1], x1 = P.dom[2], y1 = P.dom[3];
        const double vx[2] = {x0, x1};
        for (int e = 0; e < 2; ++e) {            // vertical edges x = X
            double d = vx[e] - cx;
            if (fabs(d) < r) {
                double h = sqrt(r * r - d * d);
                double ys[2] = {cy + h, cy - h};
                for (int q = 0; q < 2; ++q)
                    if (ys[q] >= y0 && ys[q] <= y1) J[nj++] = Junction{0.0, vx[e], ys[q]};
            }
        }
        const double hy[2] = {y0, y1};
        for (int e = 0; e < 2; ++e) {            // horizontal edges y = Y
            double d = hy[e] - cy;
            if (fabs(d) < r) {
                double h = sqrt(r * r - d * d);
                double xs[2] = {cx + h, cx - h};
                for (int q = 0; q < 2; ++q)
                    if (xs[q] >= x0 && xs[q] <= x1) J[nj++] = Junction{0.0, xs[q], hy[e]};
            }
        }
    } else {
        const double ox = P.dom[0], oy = P.dom[1], R = P.dom[2];
        double dx = ox - cx, dy = oy - cy;
        double d = sqrt(dx * dx + dy * dy);
        if (fabs(r - R) < d && d < r + R) {
            double a = (d * d + r * r - R * R) / (2.0 * d);
            double hh = sqrt(r * r - a * a);
            double bx = cx + a * dx / d, by = cy + a * dy / d;
            J[nj++] = Junction{0.0, bx - hh * dy / d, by + hh * dx / d};
            J[nj++] = Junction{0.0, bx + hh * dy / d, by - hh * dx / d};
        }
    }
    for (int k = 0; k < nj; ++k) J[k].ang = norm_angle(atan2(J[k].y - cy, J[k].x - cx));
    for (int k = 1; k < nj; ++k) {               // insertion sort by angle
        Junction v = J[k];
        int q = k - 1;
        while (q >= 0 && J[q].ang > v.ang) {
            J[q + 1] = J[q];
            --q;
        }
        J[q + 1] = v;
    }
    for (int k = 1; k < nj; ++k)
        if (J[k].ang - J[k - 1].ang < 1e-12) *degenerate = 1;
    return nj;
}

__device__ double unwrap_origin(const Problem &P, double cx, double cy, double r, const Junction *J,
                                int nj) {
    double best = -1.0, ts = 0.0;
    for (int k = 0; k < nj; ++k) {
        double a0 = J[k].ang;
        double a1 = (k + 1 < nj) ? J[k + 1].ang : J[0].ang + PDD_TWO_PI;
        double mid = 0.5 * (a0 + a1);
        double s, c;
        sincos(mid, &s, &c);
        bool outside = !inside_domain(P, cx + r * c, cy + r * s);
        if (outside && (a1 - a0) > best + 1e-9) {
            best = a1 - a0;
            ts = mid < PDD_TWO_PI ? mid : mid - PDD_TWO_PI;
        }
    }
    return ts;
}

__device__ double unwrap(double t, double ts) {
    double u = t - ts;
    if (u < 0.0) u += PDD_TWO_PI;
    if (u >= PDD_TWO_PI) u -= PDD_TWO_PI;
    return u;
}

struct KnotRec {
    double x, y, u;
    int dir;
};

// count (out == nullptr) or emit the knots of circle m in local order
__device__ int circle_knots(const Problem &P, double cx, double cy, double r, int n, KnotRec *out,
                            double *theta_s, int *degenerate) {
    Junction J[kMaxJ];
    int nj = circle_junctions(P, cx, cy, r, J, degenerate);
    double ts = unwrap_origin(P, cx, cy, r, J, nj);
    if (theta_s) *theta_s = ts;
    const double gap = kJunctionGap * PDD_TWO_PI / n;
    int cnt = 0;
    for (int j = 0; j < n; ++j) {
        double t = PDD_TWO_PI * j / n;
        double s, c;
        sincos(t, &s, &c);
        double x = cx + r * c, y = cy + r * s;
        if (!inside_domain(P, x, y)) continue;
        bool near = false;
        for (int k = 0; k < nj; ++k) {
            double d = fabs(t - J[k].ang);
            d = fmin(d, PDD_TWO_PI - d);
            if (d < gap) near = true;
        }
        if (near) continue;
        if (out) out[cnt] = KnotRec{x, y, unwrap(t, ts), 0};
        ++cnt;
    }
    for (int k = 0; k < nj; ++k) {
        if (out) out[cnt] = KnotRec{J[k].x, J[k].y, unwrap(J[k].ang, ts), 1};
        ++cnt;
    }
    if (out) {
        for (int k = 1; k < cnt; ++k) {          // insertion sort by local angle
            KnotRec v = out[k];
            int q = k - 1;
            while (q >= 0 && out[q].u > v.u) {
                out[q + 1] = out[q];
                --q;
            }
            out[q + 1] = v;
        }
    }
    return cnt;
}

__global__ void k_count_knots(Problem P, int M, const double *cx, const double *cy, const double *r,
                              const int *nk, int *cnt, int *err) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    int deg = 0;
    if (nk[m] + kMaxJ > kMaxKnots) {
        atomicAdd(&err[0], 1);
        cnt[m] = 0;
        return;
    }
    cnt[m] = circle_knots(P, cx[m], cy[m], r[m], nk[m], nullptr, nullptr, &deg);
    if (deg) atomicAdd(&err[0], 1);
}

__global__ void k_emit_knots(Problem P, int M, const double *cx, const double *cy, const double *r,
                             const int *nk, const int *knot_ptr, double *theta_s, double *kx,
                             double *ky, double *ku, int *kowner, uint8_t *kdir) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    if (nk[m] + kMaxJ > kMaxKnots) return;        // flagged by k_count_knots
    KnotRec buf[kMaxKnots];
    int deg = 0;
    double ts = 0.0;
    int cnt = circle_knots(P, cx[m], cy[m], r[m], nk[m], buf, &ts, &deg);
    theta_s[m] = ts;
    int base = knot_ptr[m];
    for (int k = 0; k < cnt; ++k) {
        kx[base + k] = buf[k].x;
        ky[base + k] = buf[k].y;
        ku[base + k] = buf[k].u;
        kowner[base + k] = m;
        kdir[base + k] = (uint8_t)buf[k].dir;
    }
}

// ---------------------------------------------------------------------------
// spatial hash of circles (or knots) on a uniform grid of pitch h
// ---------------------------------------------------------------------------
struct Grid {
    int gx, gy;
    double x0, y0, h;
    __device__ int cell_of(double x, double y) const {
        int ix = (int)floor((x - x0) / h), iy = (int)floor((y - y0) / h);
        ix = max(0, min(gx - 1, ix));
        iy = max(0, min(gy - 1, iy));
        return iy * gx + ix;
    }
};

__global__ void k_cell_count(Grid G, int n, const double *x, const double *y, int *cnt, int *cell) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = G.cell_of(x[i], y[i]);
    cell[i] = c;
    atomicAdd(&cnt[c], 1);
}

__global__ void k_cell_fill(int n, const int *cell, const int *ptr, int *cursor, int *items) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = cell[i];
    int p = atomicAdd(&cursor[c], 1);
    items[ptr[c] + p] = i;
}

static void build_grid(Grid G, int n, const double *x, const double *y, DevBuf<int> &ptr,
                       DevBuf<int> &items, cudaStream_t st) {
    int ncell = G.gx * G.gy;
    DevBuf<int> cnt, cell, cursor;
    cnt.alloc(ncell + 1);
    cell.alloc(std::max(n, 1));
    cursor.alloc(ncell + 1);
    ptr.alloc(ncell + 1);
    items.alloc(std::max(n, 1));
    PDD_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int) * (ncell + 1), st));
    PDD_CUDA(cudaMemsetAsync(cursor.p, 0, sizeof(int) * (ncell + 1), st));
    if (n) PDD_LAUNCH(k_cell_count, cdiv(n, 256), 256, 0, st, G, n, x, y, cnt.p, cell.p);
    exclusive_scan_async(cnt.p, ptr.p, ncell, st, nullptr);
    if (n) PDD_LAUNCH(k_cell_fill, cdiv(n, 256), 256, 0, st, n, cell.p, ptr.p, cursor.p, items.p);
}

// ---------------------------------------------------------------------------
// Eq. 5 (left) on a sample grid of pitch min(r)/4
// ---------------------------------------------------------------------------
__global__ void k_coverage(Problem P, Grid G, int sx, int sy, double bx0, double by0, double bx1,
                           double by1, const int *cptr, const int *citems, const double *cx,
                           const double *cy, const double *r, int *uncovered) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= sx * sy) return;
    int i = idx % sx, j = idx / sx;
    double x = bx0 + (i + 0.5) * (bx1 - bx0) / sx;
    double y = by0 + (j + 0.5) * (by1 - by0) / sy;
    if (!inside_domain(P, x, y)) return;
    int c = G.cell_of(x, y), ix = c % G.gx, iy = c / G.gx;
    for (int b = max(0, iy - 1); b <= min(G.gy - 1, iy + 1); ++b)
        for (int a = max(0, ix - 1); a <= min(G.gx - 1, ix + 1); ++a) {
            int cc = b * G.gx + a;
            for (int q = cptr[cc]; q < cptr[cc + 1]; ++q) {
                int m = citems[q];
                double dx = x - cx[m], dy = y - cy[m];
                if (dx * dx + dy * dy < r[m] * r[m]) return;
            }
        }
    atomicAdd(uncovered, 1);
}

// ---------------------------------------------------------------------------
// a4: row assignment
// ---------------------------------------------------------------------------
__global__ void k_assign_rows(Grid G, int N, const double *kx, const double *ky, const int *kowner,
                              const uint8_t *kdir, const int *cptr, const int *citems,
                              const double *cx, const double *cy, const double *r, int *row_sub,
                              int *uncovered) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (kdir[i]) {
        row_sub[i] = -1;
        return;
    }
    const double x = kx[i], y = ky[i];
    const int own = kowner[i];
    const double eps = kScoreEps * r[own];
    int c = G.cell_of(x, y), ix = c % G.gx, iy = c / G.gx;
    double best = -1.0;
    bool any = false;
    for (int pass = 0; pass < 2; ++pass) {
        int pick = 0x7fffffff;
        for (int b = max(0, iy - 1); b <= min(G.gy - 1, iy + 1); ++b)
            for (int a = max(0, ix - 1); a <= min(G.gx - 1, ix + 1); ++a) {
                int cc = b * G.gx + a;
                for (int q = cptr[cc]; q < cptr[cc + 1]; ++q) {
                    int m = citems[q];
                    if (m == own) continue;
                    double dx = x - cx[m], dy = y - cy[m];
                    double s = r[m] - sqrt(dx * dx + dy * dy);
                    if (!(s > eps)) continue;
                    if (pass == 0) {
                        if (!any || s > best) best = s;
                        any = true;
                    } else if (s >= best - eps && m < pick) {
                        pick = m;
                    }
                }
            }
        if (pass == 0 && !any) {
            row_sub[i] = -2;
            atomicAdd(uncovered, 1);
            return;
        }
        if (pass == 1) row_sub[i] = pick;
    }
}

// ---------------------------------------------------------------------------
// duplicate knots (closer than 1e-12)
// ---------------------------------------------------------------------------
__global__ void k_dup_knots(Grid G, int N, const double *kx, const double *ky, const int *kptr,
                            const int *kitems, int *dups) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double x = kx[i], y = ky[i];
    int c = G.cell_of(x, y), ix = c % G.gx, iy = c / G.gx;
    for (int b = max(0, iy - 1); b <= min(G.gy - 1, iy + 1); ++b)
        for (int a = max(0, ix - 1); a <= min(G.gx - 1, ix + 1); ++a) {
            int cc = b * G.gx + a;
            for (int q = kptr[cc]; q < kptr[cc + 1]; ++q) {
                int j = kitems[q];
                if (j <= i) continue;
                if (fabs(kx[j] - x) < 1e-12 && fabs(ky[j] - y) < 1e-12) atomicAdd(dups, 1);
            }
        }
}

// ---------------------------------------------------------------------------
// Pi_i: the subdomains a row integrates in.  One (the farthest interface, Sec.
// 3.2) or, for averaged rows (Eq. 38-39), every subdomain whose open disk holds
// the knot -- the same "inside" test as the candidates of k_assign_rows --
// listed in ascending order.
// ---------------------------------------------------------------------------
__global__ void k_pi_count(Grid G, int N, int averaged, const double *kx, const double *ky, const int *kowner,
                           const int *row_sub, const int *cptr, const int *citems, const double *cx,
                           const double *cy, const double *r, int *cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (row_sub[i] < 0) {
        cnt[i] = 0;
        return;
    }
    if (!averaged) {
        cnt[i] = 1;
        return;
    }
    const double x = kx[i], y = ky[i];
    const int own = kowner[i];
    const double eps = kScoreEps * r[own];
    int c = G.cell_of(x, y), ix = c % G.gx, iy = c / G.gx, n = 0;
    for (int b = max(0, iy - 1); b <= min(G.gy - 1, iy + 1); ++b)
        for (int a = max(0, ix - 1); a <= min(G.gx - 1, ix + 1); ++a) {
            int cc = b * G.gx + a;
            for (int q = cptr[cc]; q < cptr[cc + 1]; ++q) {
                int m = citems[q];
                if (m == own) continue;
                double dx = x - cx[m], dy = y - cy[m];
                if (r[m] - sqrt(dx * dx + dy * dy) > eps) ++n;
            }
        }
    cnt[i] = n;
}

__global__ void k_pi_fill(Grid G, int N, int averaged, const double *kx, const double *ky, const int *kowner,
                          const int *row_sub, const int *cptr, const int *citems, const double *cx,
                          const double *cy, const double *r, const int *pi_ptr, int *pi_sub) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || row_sub[i] < 0) return;
    int *out = pi_sub + pi_ptr[i];
    if (!averaged) {
        out[0] = row_sub[i];
        return;
    }
    const double x = kx[i], y = ky[i];
    const int own = kowner[i];
    const double eps = kScoreEps * r[own];
    int c = G.cell_of(x, y), ix = c % G.gx, iy = c / G.gx, n = 0;
    for (int b = max(0, iy - 1); b <= min(G.gy - 1, iy + 1); ++b)
        for (int a = max(0, ix - 1); a <= min(G.gx - 1, ix + 1); ++a) {
            int cc = b * G.gx + a;
            for (int q = cptr[cc]; q < cptr[cc + 1]; ++q) {
                int m = citems[q];
                if (m == own) continue;
                double dx = x - cx[m], dy = y - cy[m];
                if (!(r[m] - sqrt(dx * dx + dy * dy) > eps)) continue;
                int k = n++;                               // insertion into the ascending list
                while (k > 0 && out[k - 1] > m) {
                    out[k] = out[k - 1];
                    --k;
                }
                out[k] = m;
            }
        }
}

// ---------------------------------------------------------------------------
// a5: CSR pattern (Eq. 29; Eq. 38 for averaged rows) and rows grouped by
// subdomain.  Row i holds the diagonal and the stencils Xi_m of every m in
// Pi_i; the stencils are disjoint knot ranges in the order of m, and i lies in
// none of them (a knot is on its own circle, not inside it).
// ---------------------------------------------------------------------------
__global__ void k_row_len(int N, const int *pi_ptr, const int *pi_sub, const int *knot_ptr, int *len,
                          int *sub_cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int n = 1;
    for (int e = pi_ptr[i]; e < pi_ptr[i + 1]; ++e) {
        const int m = pi_sub[e];
        n += knot_ptr[m + 1] - knot_ptr[m];
        atomicAdd(&sub_cnt[m], 1);
    }
    len[i] = n;
}

__global__ void k_csr_cols(int N, const int *pi_ptr, const int *pi_sub, const int *knot_ptr, const int *rowptr,
                           int *col) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int p = rowptr[i];
    bool diag = false;
    for (int e = pi_ptr[i]; e < pi_ptr[i + 1]; ++e) {
        const int m = pi_sub[e], a = knot_ptr[m], b = knot_ptr[m + 1];
        if (!diag && i < a) {
            col[p++] = i;
            diag = true;
        }
        for (int j = a; j < b; ++j) col[p++] = j;
    }
    if (!diag) col[p] = i;
}

__global__ void k_sub_fill(int N, const int *pi_ptr, const int *pi_sub, const int *sub_ptr, int *cursor,
                           int *sub_rows) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int e = pi_ptr[i]; e < pi_ptr[i + 1]; ++e) {
        const int m = pi_sub[e];
        int p = atomicAdd(&cursor[m], 1);
        sub_rows[sub_ptr[m] + p] = i;
    }
}

// per entry p of sub_rows (subdomain m, row i): the position k of m in Pi_i, the offset of
// Xi_m's first column in row i, and the inverse map pair_spos[pi_ptr[i] + k] = p
__global__ void k_sub_meta(int M, const int *sub_ptr, const int *sub_rows, const int *pi_ptr, const int *pi_sub,
                           const int *knot_ptr, int *sub_m, int *sub_k, int *sub_off, int *pair_spos) {
    const int m = blockIdx.x;
    if (m >= M) return;
    const int a = knot_ptr[m];
    for (int p = sub_ptr[m] + threadIdx.x; p < sub_ptr[m + 1]; p += blockDim.x) {
        const int i = sub_rows[p];
        int off = (i < a) ? 1 : 0, k = 0;
        for (int e = pi_ptr[i]; e < pi_ptr[i + 1]; ++e) {
            const int q = pi_sub[e];
            if (q == m) {
                k = e - pi_ptr[i];
                break;
            }
            off += knot_ptr[q + 1] - knot_ptr[q];
        }
        sub_m[p] = m;
        sub_k[p] = k;
        sub_off[p] = off;
        pair_spos[pi_ptr[i] + k] = p;
    }
}

__global__ void k_sub_sort(int M, const int *sub_ptr, int *sub_rows) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    int a = sub_ptr[m], b = sub_ptr[m + 1];
    for (int k = a + 1; k < b; ++k) {
        int v = sub_rows[k], q = k - 1;
        while (q >= a && sub_rows[q] > v) {
            sub_rows[q + 1] = sub_rows[q];
            --q;
        }
        sub_rows[q + 1] = v;
    }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
template <typename T>
static std::vector<T> to_host(const DevBuf<T> &d, size_t n, cudaStream_t st) {
    std::vector<T> h(n);
    if (n) PDD_CUDA(cudaMemcpyAsync(h.data(), d.p, n * sizeof(T), cudaMemcpyDeviceToHost, st));
    PDD_CUDA(cudaStreamSynchronize(st));
    return h;
}

void build_cover_impl(const pdd_domain &dom, const pdd_cover_spec &spec, pdd_cover &cov,
                      cudaStream_t st) {
    Problem P{};
    P.dom_kind = dom.kind;
    for (int k = 0; k < 4; ++k) P.dom[k] = dom.p[k];
    cov.domain = dom;
    cov.averaged = spec.row_mode == PDD_ROWS_AVERAGED ? 1 : 0;

    LatticeArgs L{};
    L.kind = spec.kind;
    L.nx = spec.nx;
    L.ny = spec.ny;
    L.xo = spec.x_origin;
    L.yo = spec.y_origin;
    L.s = spec.spacing;
    L.rad = spec.radius;
    L.unk = spec.n_knots;
    L.unr = spec.n_r;
    L.unt = spec.n_theta;
    DevBuf<double> ecx, ecy, er;
    DevBuf<int> enk, enr, ent;
    if (spec.kind == PDD_COVER_EXPLICIT) {
        int n = spec.n_explicit;
        L.n_lat = n;
        ecx.alloc(n);
        ecy.alloc(n);
        er.alloc(n);
        enk.alloc(n);
        enr.alloc(n);
        ent.alloc(n);
        PDD_CUDA(cudaMemcpyAsync(ecx.p, spec.cx, n * 8, cudaMemcpyHostToDevice, st));
        PDD_CUDA(cudaMemcpyAsync(ecy.p, spec.cy, n * 8, cudaMemcpyHostToDevice, st));
        PDD_CUDA(cudaMemcpyAsync(er.p, spec.r, n * 8, cudaMemcpyHostToDevice, st));
        PDD_CUDA(cudaMemcpyAsync(enk.p, spec.n_knots_per, n * 4, cudaMemcpyHostToDevice, st));
        PDD_CUDA(cudaMemcpyAsync(enr.p, spec.n_r_per, n * 4, cudaMemcpyHostToDevice, st));
        PDD_CUDA(cudaMemcpyAsync(ent.p, spec.n_theta_per, n * 4, cudaMemcpyHostToDevice, st));
        L.ecx = ecx.p;
        L.ecy = ecy.p;
        L.er = er.p;
        L.enk = enk.p;
        L.enr = enr.p;
        L.ent = ent.p;
    } else {
        L.n_lat = spec.nx * spec.ny;
    }
    const int nl = L.n_lat;
    DevBuf<double> lcx, lcy, lr;
    DevBuf<int> lnk, lnr, lnt, keep, pos;
    lcx.alloc(nl);
    lcy.alloc(nl);
    lr.alloc(nl);
    lnk.alloc(nl);
    lnr.alloc(nl);
    lnt.alloc(nl);
    keep.alloc(nl + 1);
    pos.alloc(nl + 1);
    PDD_LAUNCH(k_lattice, cdiv(nl, 256), 256, 0, st, P, L, lcx.p, lcy.p, lr.p, lnk.p, lnr.p, lnt.p,
               keep.p);
    const int M = (int)exclusive_scan(keep.p, pos.p, nl, st);
    if (M == 0) fail(PDD_EINVAL, "no circle meets the domain");
    cov.M = M;
    cov.cx.alloc(M);
    cov.cy.alloc(M);
    cov.r.alloc(M);
    cov.nk.alloc(M);
    cov.nr.alloc(M);
    cov.nt.alloc(M);
    cov.floating.alloc(M);
    cov.theta_s.alloc(M);
    PDD_LAUNCH(k_compact_circles, cdiv(nl, 256), 256, 0, st, nl, keep.p, pos.p, lcx.p, lcy.p, lr.p,
               lnk.p, lnr.p, lnt.p, P, cov.cx.p, cov.cy.p, cov.r.p, cov.nk.p, cov.nr.p, cov.nt.p,
               cov.floating.p);
    cov.h_nk = to_host(cov.nk, M, st);
    cov.h_nr = to_host(cov.nr, M, st);
    cov.h_nt = to_host(cov.nt, M, st);
    cov.h_floating = to_host(cov.floating, M, st);
    std::vector<double> hr = to_host(cov.r, M, st);
    std::vector<double> hcx = to_host(cov.cx, M, st), hcy = to_host(cov.cy, M, st);
    cov.max_nk = 0;
    cov.M_floating = 0;
    for (int m = 0; m < M; ++m) {
        if (cov.h_nk[m] < 2 || (cov.h_nk[m] & 1) || (cov.h_nt[m] & 1) || cov.h_nt[m] < 2 ||
            cov.h_nr[m] < 1)
            fail(PDD_EINVAL, "n_knots and n_theta must be even and >= 2, n_r >= 1");
        if (!(hr[m] > 0.0)) fail(PDD_EINVAL, "non-positive radius");
        cov.max_nk = std::max(cov.max_nk, cov.h_nk[m]);
        cov.M_floating += cov.h_floating[m];
    }
    cov.max_r = *std::max_element(hr.begin(), hr.end());
    cov.min_r = *std::min_element(hr.begin(), hr.end());

    // spatial hash of circle centres, pitch max_r
    double bx0 = hcx[0], bx1 = hcx[0], by0 = hcy[0], by1 = hcy[0];
    for (int m = 0; m < M; ++m) {
        bx0 = std::min(bx0, hcx[m]);
        bx1 = std::max(bx1, hcx[m]);
        by0 = std::min(by0, hcy[m]);
        by1 = std::max(by1, hcy[m]);
    }
    Grid G;
    G.h = cov.max_r;
    G.x0 = bx0 - cov.max_r;
    G.y0 = by0 - cov.max_r;
    G.gx = (int)std::ceil((bx1 - bx0 + 2 * cov.max_r) / G.h) + 1;
    G.gy = (int)std::ceil((by1 - by0 + 2 * cov.max_r) / G.h) + 1;
    if ((double)G.gx * G.gy > 5e7) fail(PDD_EINVAL, "circle radii too disparate for the spatial hash");
    cov.gx = G.gx;
    cov.gy = G.gy;
    cov.gx0 = G.x0;
    cov.gy0 = G.y0;
    cov.gh = G.h;
    build_grid(G, M, cov.cx.p, cov.cy.p, cov.cell_ptr, cov.cell_items, st);

    DevBuf<int> err;
    err.alloc(8);
    PDD_CUDA(cudaMemsetAsync(err.p, 0, 8 * sizeof(int), st));

    // Eq. 5 (left): sampled coverage
    {
        double x0, y0, x1, y1;
        if (dom.kind == 0) {
            x0 = dom.p[0]; y0 = dom.p[1]; x1 = dom.p[2]; y1 = dom.p[3];
        } else {
            x0 = dom.p[0] - dom.p[2]; y0 = dom.p[1] - dom.p[2];
            x1 = dom.p[0] + dom.p[2]; y1 = dom.p[1] + dom.p[2];
        }
        double h = 0.25 * cov.min_r;
        int sx = (int)std::ceil((x1 - x0) / h), sy = (int)std::ceil((y1 - y0) / h);
        if ((double)sx * sy > 4e8) fail(PDD_EINVAL, "coverage sample grid too large");
        PDD_LAUNCH(k_coverage, cdiv((long)sx * sy, 256), 256, 0, st, P, G, sx, sy, x0, y0, x1, y1,
                   cov.cell_ptr.p, cov.cell_items.p, cov.cx.p, cov.cy.p, cov.r.p, err.p + 3);
    }

    // a2-a3: knots
    DevBuf<int> cnt;
    cnt.alloc(M + 1);
    cov.knot_ptr.alloc(M + 1);
    PDD_LAUNCH(k_count_knots, cdiv(M, 128), 128, 0, st, P, M, cov.cx.p, cov.cy.p, cov.r.p, cov.nk.p,
               cnt.p, err.p);
    const int N = (int)exclusive_scan(cnt.p, cov.knot_ptr.p, M, st);
    cov.N = N;
    cov.kx.alloc(N);
    cov.ky.alloc(N);
    cov.ku.alloc(N);
    cov.kowner.alloc(N);
    cov.kdir.alloc(N);
    cov.row_sub.alloc(N);
    PDD_LAUNCH(k_emit_knots, cdiv(M, 64), 64, 0, st, P, M, cov.cx.p, cov.cy.p, cov.r.p, cov.nk.p,
               cov.knot_ptr.p, cov.theta_s.p, cov.kx.p, cov.ky.p, cov.ku.p, cov.kowner.p, cov.kdir.p);

    // duplicate knots
    {
        DevBuf<int> kptr, kitems;
        build_grid(G, N, cov.kx.p, cov.ky.p, kptr, kitems, st);
        PDD_LAUNCH(k_dup_knots, cdiv(N, 256), 256, 0, st, G, N, cov.kx.p, cov.ky.p, kptr.p, kitems.p,
                   err.p + 2);
    }
    // a4: rows
    PDD_LAUNCH(k_assign_rows, cdiv(N, 256), 256, 0, st, G, N, cov.kx.p, cov.ky.p, cov.kowner.p,
               cov.kdir.p, cov.cell_ptr.p, cov.cell_items.p, cov.cx.p, cov.cy.p, cov.r.p,
               cov.row_sub.p, err.p + 1);
    std::vector<int> herr = to_host(err, 8, st);
    if (herr[0]) fail(PDD_EINVAL, "degenerate junction (a circle through a corner) or too many knots");
    if (herr[3]) fail(PDD_ECOVER_GAP, std::to_string(herr[3]) + " sample points of the domain are uncovered");
    if (herr[2]) fail(PDD_EDUPLICATE_KNOT, "two knots coincide");
    if (herr[1]) fail(PDD_EKNOT_UNCOVERED, std::to_string(herr[1]) + " knots lie inside no other circle");

    // Pi_i (one subdomain, or all that hold the knot for averaged rows)
    DevBuf<int> picnt;
    picnt.alloc(N + 1);
    PDD_LAUNCH(k_pi_count, cdiv(N, 256), 256, 0, st, G, N, cov.averaged, cov.kx.p, cov.ky.p, cov.kowner.p,
               cov.row_sub.p, cov.cell_ptr.p, cov.cell_items.p, cov.cx.p, cov.cy.p, cov.r.p, picnt.p);
    cov.pi_ptr.alloc(N + 1);
    cov.npairs = (int)exclusive_scan(picnt.p, cov.pi_ptr.p, N, st);
    cov.pi_sub.alloc(std::max(cov.npairs, 1));
    PDD_LAUNCH(k_pi_fill, cdiv(N, 256), 256, 0, st, G, N, cov.averaged, cov.kx.p, cov.ky.p, cov.kowner.p,
               cov.row_sub.p, cov.cell_ptr.p, cov.cell_items.p, cov.cx.p, cov.cy.p, cov.r.p, cov.pi_ptr.p,
               cov.pi_sub.p);

    // a5: CSR pattern + rows by subdomain
    DevBuf<int> len, sub_cnt, cursor;
    len.alloc(N + 1);
    sub_cnt.alloc(M + 1);
    cursor.alloc(M + 1);
    PDD_CUDA(cudaMemsetAsync(sub_cnt.p, 0, sizeof(int) * (M + 1), st));
    PDD_CUDA(cudaMemsetAsync(cursor.p, 0, sizeof(int) * (M + 1), st));
    PDD_LAUNCH(k_row_len, cdiv(N, 256), 256, 0, st, N, cov.pi_ptr.p, cov.pi_sub.p, cov.knot_ptr.p, len.p,
               sub_cnt.p);
    cov.rowptr.alloc(N + 1);
    cov.nnz = exclusive_scan(len.p, cov.rowptr.p, N, st);
    cov.col.alloc(cov.nnz);
    PDD_LAUNCH(k_csr_cols, cdiv(N, 256), 256, 0, st, N, cov.pi_ptr.p, cov.pi_sub.p, cov.knot_ptr.p,
               cov.rowptr.p, cov.col.p);
    cov.sub_ptr.alloc(M + 1);
    int nsub = (int)exclusive_scan(sub_cnt.p, cov.sub_ptr.p, M, st);
    cov.sub_rows.alloc(std::max(nsub, 1));
    PDD_LAUNCH(k_sub_fill, cdiv(N, 256), 256, 0, st, N, cov.pi_ptr.p, cov.pi_sub.p, cov.sub_ptr.p, cursor.p,
               cov.sub_rows.p);
    PDD_LAUNCH(k_sub_sort, cdiv(M, 128), 128, 0, st, M, cov.sub_ptr.p, cov.sub_rows.p);
    const int np1 = std::max(nsub, 1);
    cov.sub_m.alloc(np1);
    cov.sub_k.alloc(np1);
    cov.sub_off.alloc(np1);
    cov.pair_spos.alloc(np1);
    if (M > 0)
        PDD_LAUNCH(k_sub_meta, M, 128, 0, st, M, cov.sub_ptr.p, cov.sub_rows.p, cov.pi_ptr.p, cov.pi_sub.p,
                   cov.knot_ptr.p, cov.sub_m.p, cov.sub_k.p, cov.sub_off.p, cov.pair_spos.p);
    cov.h_knot_ptr = to_host(cov.knot_ptr, M + 1, st);
    cov.h_sub_ptr = to_host(cov.sub_ptr, M + 1, st);
    cov.max_stencil = 0;
    for (int m = 0; m < M; ++m)
        cov.max_stencil = std::max(cov.max_stencil, cov.h_knot_ptr[m + 1] - cov.h_knot_ptr[m]);
}

}  // namespace pdd
