// Setup kernels: staircase classification, IBM-point lists, weights (delta,
// lambda, wall source), per-stage implicit coefficients and Poisson pivots.
//
// This translation unit is compiled with -fmad=false and writes its level-set
// arithmetic with explicitly rounded operations, so the sign of phi at every
// grid point is the same as an FP64 evaluation of the same formula in the
// same order on any IEEE machine (classification is bit-exact).
#include "common.cuh"

#include <cmath>
#include <vector>

namespace {

constexpr double TWO_PI = 6.283185307179586;

// ---------------------------------------------------------------------------
// Level set: phi < 0 fluid, phi >= 0 solid (Sec. 3.3, "true boundary")
// ---------------------------------------------------------------------------
__device__ double phi_at(const GeomP& g, double x, double y, double z) {
    const double* p = g.p;
    switch (g.kind) {
        case IBM_GEOM_PLANES:
            return fmax(__dsub_rn(p[0], y), __dsub_rn(y, p[1]));
        case IBM_GEOM_CYLINDER: {
            double dx = __dsub_rn(x, p[0]);
            double dy = __dsub_rn(y, p[1]);
            double q = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
            return __dmul_rn(p[3], __dsub_rn(q, __dmul_rn(p[2], p[2])));
        }
        case IBM_GEOM_SPHERE: {
            double dx = __dsub_rn(x, p[0]);
            double dy = __dsub_rn(y, p[1]);
            double dz = __dsub_rn(z, p[2]);
            double q = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            return __dmul_rn(p[4], __dsub_rn(q, __dmul_rn(p[3], p[3])));
        }
        case IBM_GEOM_SINE_WALL: {
            double yw = __dadd_rn(p[0], __dmul_rn(p[1], sin(__dmul_rn(TWO_PI, __ddiv_rn(x, p[2])))));
            return fmax(__dsub_rn(yw, y), __dsub_rn(y, p[3]));
        }
        case IBM_GEOM_TUBES: {
            // min over tubes and segments of |X - C| - r(t): C the projection of X on the
            // segment [A, B], t in [0,1] its position, r linear between the end radii
            double best = 1e300;
            for (int tb = 0; tb < g.ntubes; ++tb) {
                const double* q = g.tube + tb * g.npts * 4;
                for (int sgi = 0; sgi + 1 < g.npts; ++sgi) {
                    const double* a = q + 4 * sgi;
                    const double* b = a + 4;
                    const double ex = __dsub_rn(b[0], a[0]), ey = __dsub_rn(b[1], a[1]), ez = __dsub_rn(b[2], a[2]);
                    const double ee = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
                    const double wx = __dsub_rn(x, a[0]), wy = __dsub_rn(y, a[1]), wz = __dsub_rn(z, a[2]);
                    const double we = __dadd_rn(__dadd_rn(__dmul_rn(wx, ex), __dmul_rn(wy, ey)), __dmul_rn(wz, ez));
                    const double t = fmin(fmax(__ddiv_rn(we, ee), 0.0), 1.0);
                    const double dx = __dsub_rn(x, __dadd_rn(a[0], __dmul_rn(t, ex)));
                    const double dy = __dsub_rn(y, __dadd_rn(a[1], __dmul_rn(t, ey)));
                    const double dz = __dsub_rn(z, __dadd_rn(a[2], __dmul_rn(t, ez)));
                    const double dist = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                                             __dmul_rn(dz, dz)));
                    const double r = __dadd_rn(a[3], __dmul_rn(t, __dsub_rn(b[3], a[3])));
                    best = fmin(best, __dsub_rn(dist, r));
                }
            }
            return best;
        }
        default:
            return -1.0;
    }
}

// coordinate of component c (0..2; 3 = cell centre) of index idx along direction d; on a
// stretched y the tabulated centre or face height
__device__ __forceinline__ double coord(const GridP& g, int d, int idx, int c) {
    if (d == 1 && g.ystr) return ytab(g, c == 1 ? YT_YF : YT_YC, idx);
    double off = (d == c) ? 1.0 : 0.5;
    double o = d == 0 ? g.ox : (d == 1 ? g.oy : g.oz);
    double D = d == 0 ? g.dx : (d == 1 ? g.dy : g.dz);
    return __dadd_rn(o, __dmul_rn(__dadd_rn((double)idx, off), D));
}

// Is (i,j,k) of component c a prescribed box-face point: v on the +y wall, or u
// on the outflow face of an inflow/outflow x?  Such points are never solved.
__device__ __forceinline__ bool bface(const GridP& g, int c, int i, int j) {
    return (c == 1 && j == g.ny - 1) || (c == 0 && !g.xper && i == g.nx - 1);
}

// ---------------------------------------------------------------------------
// Classification
// ---------------------------------------------------------------------------
__global__ void k_classify_vel(GridP g, GeomP geo, uint8_t* __restrict__ velbits) {
    long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    int i = (int)(id % g.nx);
    int j = (int)((id / g.nx) % g.ny);
    int k = (int)(id / ((long long)g.nx * g.ny));
    uint8_t b = 0;
    for (int c = 0; c < g.ncomp; ++c) {
        if (bface(g, c, i, j)) continue;
        double phi;
        if (geo.kind == IBM_GEOM_SAMPLED) {
            phi = geo.sdf[c][id];
        } else {
            double x = coord(g, 0, i, c), y = coord(g, 1, j, c), z = coord(g, 2, k, c);
            phi = phi_at(geo, x, y, z);
        }
        if (phi < 0.0) b |= (uint8_t)(1u << c);
    }
    if (!g.xper) {
        // bit 7: the inflow face (u at i = -1, i.e. x = origin) of row (j, k) is fluid at i = 0,
        // the outflow face (u at i = nx-1) is fluid at i = nx-1
        double yy = coord(g, 1, j, 0), zz = coord(g, 2, k, 0);
        if (i == 0 && phi_at(geo, coord(g, 0, -1, 0), yy, zz) < 0.0) b |= IBM_MASK_FACE;
        if (i == g.nx - 1 && phi_at(geo, coord(g, 0, i, 0), yy, zz) < 0.0) b |= IBM_MASK_FACE;
    }
    velbits[id] = b;
}

// A translating body at the start of a step: velocity points that turn fluid (internal in the new
// classification vb, not in the previous mask) take the body velocity.
template <typename T>
__global__ void k_fresh_fill(GridP g, const uint8_t* __restrict__ vb, const uint8_t* __restrict__ mask, BodyP body,
                             T* __restrict__ u0, T* __restrict__ u1, T* __restrict__ u2) {
    long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    const uint8_t fresh = vb[id] & (uint8_t)~mask[id] & 7u;
    if (!fresh) return;
    T* u[3] = {u0, u1, u2};
    for (int c = 0; c < g.ncomp; ++c)
        if ((fresh >> c) & 1u) u[c][id] = (T)body.ub[c];
}

__device__ __forceinline__ bool vel_internal(const GridP& g, const uint8_t* vb, int c, int i, int j, int k) {
    return (vb[i + (long long)g.nx * (j + (long long)g.ny * k)] >> c) & 1u;
}

// external = a stored point, not on a box face, that is not internal
__device__ __forceinline__ bool vel_external(const GridP& g, const uint8_t* vb, int c, int i, int j, int k) {
    if (bface(g, c, i, j)) return false;
    return !vel_internal(g, vb, c, i, j, k);
}

// Neighbour of (i,j,k) along d by s on component c's grid; false if beyond a box face.
__device__ __forceinline__ bool neighbour(const GridP& g, int d, int s, int& i, int& j, int& k) {
    if (d == 0) {
        if (g.xper) { i = wrapi(i + s, g.nx); return true; }
        i += s;
        return i >= 0 && i < g.nx;
    }
    if (d == 2) { k = wrapi(k + s, g.nz); return true; }
    j += s;
    return j >= 0 && j < g.ny;
}

__global__ void k_classify_final(GridP g, const uint8_t* __restrict__ vb, uint8_t* __restrict__ mask) {
    long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    int i = (int)(id % g.nx);
    int j = (int)((id / g.nx) % g.ny);
    int k = (int)(id / ((long long)g.nx * g.ny));
    uint8_t own = vb[id];
    uint8_t m = own;
    // internal pressure: any of the cell's face velocities internal (the inflow face is not one)
    bool pint = (own & 7u) != 0;
    for (int c = 0; c < g.ncomp && !pint; ++c) {
        int ii = i, jj = j, kk = k;
        if (c == 0) {
            ii = g.xper ? wrapi(i - 1, g.nx) : i - 1;
            if (ii < 0) continue;
        }
        else if (c == 2) kk = wrapi(k - 1, g.nz);
        else { jj = j - 1; if (jj < 0) continue; }
        if (vel_internal(g, vb, c, ii, jj, kk)) pint = true;
    }
    if (pint) m |= IBM_MASK_P;
    // IBM point: internal with an external same-component neighbour along an arm
    for (int c = 0; c < g.ncomp; ++c) {
        if (!((own >> c) & 1u)) continue;
        bool ext = false;
        for (int d = 0; d < g.ndim && !ext; ++d)
            for (int s = 1; s >= -1 && !ext; s -= 2) {
                int ii = i, jj = j, kk = k;
                if (!neighbour(g, d, s, ii, jj, kk)) continue;
                if (vel_external(g, vb, c, ii, jj, kk)) ext = true;
            }
        if (ext) m |= (uint8_t)(IBM_MASK_IBM_U << c);
    }
    mask[id] = m;
}

// One warp per 32-point x segment: IBM points per component
__global__ void k_segcount(GridP g, long long nseg, const uint8_t* __restrict__ mask, int* cnt0, int* cnt1, int* cnt2) {
    long long seg = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / IBM_WARP;
    int lane = threadIdx.x & 31;
    if (seg >= nseg) return;
    int sx = (int)(seg % g.nsegx);
    long long row = seg / g.nsegx;
    int i = sx * IBM_WARP + lane;
    uint8_t m = i < g.nx ? mask[row * g.nx + i] : 0;
    int* cnt[3] = {cnt0, cnt1, cnt2};
    for (int c = 0; c < 3; ++c) {
        unsigned b = __ballot_sync(0xffffffffu, (m >> (4 + c)) & 1u);
        if (lane == 0) cnt[c][seg] = __popc(b);
    }
}

__global__ void k_compact(GridP g, long long nseg, const uint8_t* __restrict__ mask, const int* off0,
                          const int* off1, const int* off2, int* idx0, int* idx1, int* idx2) {
    long long seg = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / IBM_WARP;
    int lane = threadIdx.x & 31;
    if (seg >= nseg) return;
    int sx = (int)(seg % g.nsegx);
    long long row = seg / g.nsegx;
    int i = sx * IBM_WARP + lane;
    long long lin = row * g.nx + i;
    uint8_t m = i < g.nx ? mask[lin] : 0;
    const int* off[3] = {off0, off1, off2};
    int* idx[3] = {idx0, idx1, idx2};
    for (int c = 0; c < 3; ++c) {
        bool bit = (m >> (4 + c)) & 1u;
        unsigned b = __ballot_sync(0xffffffffu, bit);
        if (bit) idx[c][off[c][seg] + __popc(b & lanemask_lt())] = (int)lin;
    }
}

// ---------------------------------------------------------------------------
// Exclusive scan of int counts (three arrays, blockIdx.y = component)
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 512;      // threads per block
constexpr int SCAN_E = 8;        // elements per thread
constexpr int SCAN_CH = SCAN_T * SCAN_E;

__device__ int block_exclusive_scan(int v, int* sh, int& total) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        int y = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += t;
        }
        if (lane < nw) sh[lane] = y;
    }
    __syncthreads();
    int warp_off = wid > 0 ? sh[wid - 1] : 0;
    total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_off + x - v;
}

struct ScanArgs {
    const int* in[3];
    int* out[3];
};

__global__ void k_scan_partials(ScanArgs a, long long n, int* bsum, int nblocks) {
    __shared__ int sh[32];
    int c = blockIdx.y;
    long long base = (long long)blockIdx.x * SCAN_CH + (long long)threadIdx.x * SCAN_E;
    int s = 0;
    for (int e = 0; e < SCAN_E; ++e)
        if (base + e < n) s += a.in[c][base + e];
    int total;
    block_exclusive_scan(s, sh, total);
    if (threadIdx.x == 0) bsum[c * nblocks + blockIdx.x] = total;
}

__global__ void k_scan_top(int* bsum, int nblocks, int* totals) {
    __shared__ int sh[32];
    int c = blockIdx.x;
    int run = 0;
    for (int base = 0; base < nblocks; base += blockDim.x) {
        int t = base + threadIdx.x;
        int v = t < nblocks ? bsum[c * nblocks + t] : 0;
        int total;
        int ex = block_exclusive_scan(v, sh, total);
        if (t < nblocks) bsum[c * nblocks + t] = run + ex;
        run += total;
    }
    if (threadIdx.x == 0) totals[c] = run;
}

__global__ void k_scan_apply(ScanArgs a, long long n, const int* boff, int nblocks) {
    __shared__ int sh[32];
    int c = blockIdx.y;
    long long base = (long long)blockIdx.x * SCAN_CH + (long long)threadIdx.x * SCAN_E;
    int v[SCAN_E];
    int s = 0;
    for (int e = 0; e < SCAN_E; ++e) {
        v[e] = (base + e < n) ? a.in[c][base + e] : 0;
        s += v[e];
    }
    int total;
    int ex = block_exclusive_scan(s, sh, total) + boff[c * nblocks + blockIdx.x];
    for (int e = 0; e < SCAN_E; ++e) {
        if (base + e < n) a.out[c][base + e] = ex;
        ex += v[e];
    }
}

// ---------------------------------------------------------------------------
// Weights: delta per crossed arm, lambda and the wall source (Sec. 2.2)
// ---------------------------------------------------------------------------
__device__ double delta_bisect(const GeomP& geo, const double P[3], int d, int s, double D) {
    double lo = 0.0, hi = D;
    for (int it = 0; it < 200; ++it) {
        double mid = __dmul_rn(0.5, __dadd_rn(lo, hi));
        if (mid <= lo || mid >= hi) break;
        double Q[3] = {P[0], P[1], P[2]};
        Q[d] = __dadd_rn(P[d], __dmul_rn((double)s, mid));
        if (phi_at(geo, Q[0], Q[1], Q[2]) < 0.0) lo = mid;
        else hi = mid;
    }
    return hi;
}

// closed-form distance, or a negative value when none applies
__device__ double delta_closed(const GeomP& geo, const double P[3], int d, int s, double D) {
    const double* p = geo.p;
    if (geo.kind == IBM_GEOM_PLANES && d == 1) return s < 0 ? __dsub_rn(P[1], p[0]) : __dsub_rn(p[1], P[1]);
    if (geo.kind == IBM_GEOM_SINE_WALL && d == 1) {
        if (s < 0) {
            double yw = __dadd_rn(p[0], __dmul_rn(p[1], sin(__dmul_rn(TWO_PI, __ddiv_rn(P[0], p[2])))));
            return __dsub_rn(P[1], yw);
        }
        return __dsub_rn(p[3], P[1]);
    }
    if (geo.kind == IBM_GEOM_CYLINDER || geo.kind == IBM_GEOM_SPHERE) {
        bool sph = geo.kind == IBM_GEOM_SPHERE;
        double ctr[3] = {p[0], p[1], sph ? p[2] : 0.0};
        double R = sph ? p[3] : p[2];
        int nd = sph ? 3 : 2;
        if (d >= nd) return -1.0;
        double rho2 = 0.0;
        for (int e = 0; e < nd; ++e) {
            if (e == d) continue;
            double t = __dsub_rn(P[e], ctr[e]);
            rho2 = __dadd_rn(rho2, __dmul_rn(t, t));
        }
        double h2 = __dsub_rn(__dmul_rn(R, R), rho2);
        if (h2 < 0.0) return -1.0;
        double hh = __dsqrt_rn(h2);
        double xp = P[d];
        double xq = __dadd_rn(xp, __dmul_rn((double)s, D));
        double lo = fmin(xp, xq), hi = fmax(xp, xq);
        double r1 = __dsub_rn(ctr[d], hh), r2 = __dadd_rn(ctr[d], hh);
        bool in1 = lo <= r1 && r1 <= hi, in2 = lo <= r2 && r2 <= hi;
        if (in1 == in2) return -1.0;
        return fabs(__dsub_rn(in1 ? r1 : r2, xp));
    }
    return -1.0;
}

__device__ double wall_factor(int kind, int d, int s) {
    if (kind == IBM_GEOM_PLANES) return (d == 1 && s > 0) ? 1.0 : 0.0;
    if (kind == IBM_GEOM_SINE_WALL) return (d == 1 && s > 0) ? 0.0 : 1.0;
    return 1.0;
}

struct WeightArgs {
    const int* idx[3];
    double* lam[3];
    double* src[3];
    int count[3];
    double nu;
    double wall_u[3];
    int no_ibm;
    BodyP body;      // a moving body: the body-frame source (below)
};

__global__ void k_weights(GridP g, GeomP geo, WeightArgs a, const uint8_t* __restrict__ mask) {
    int c = blockIdx.y;
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncomp || m >= a.count[c]) return;
    int lin = a.idx[c][m];
    int i = lin % g.nx;
    int j = (lin / g.nx) % g.ny;
    int k = lin / (g.nx * g.ny);
    double lam = 0.0, src = 0.0;
    if (!a.no_ibm) {
        const bool sampled = geo.kind == IBM_GEOM_SAMPLED;
        double P[3] = {coord(g, 0, i, c), coord(g, 1, j, c), coord(g, 2, k, c)};
        double phiP = sampled ? geo.sdf[c][lin] : phi_at(geo, P[0], P[1], P[2]);
        for (int d = 0; d < g.ndim; ++d) {
            for (int s = 1; s >= -1; s -= 2) {
                double D = d == 0 ? g.dx : (d == 1 ? g.dy : g.dz);
                // a stretched y arm (reading R23): the distance to this neighbour on the
                // component's own grid, and d(s) = 2 / (D (D_- + D_+)) in place of 1 / D^2
                double Dsum = 2.0 * D;
                if (d == 1 && g.ystr) {
                    const double hm = ytab(g, c == 1 ? YT_DYC : YT_HC, j);
                    const double hp = c == 1 ? (j + 1 < g.ny ? ytab(g, YT_DYC, j + 1) : ytab(g, YT_DYC, g.ny - 1))
                                             : ytab(g, YT_HC, j + 1);
                    D = s > 0 ? hp : hm;
                    Dsum = hm + hp;
                }
                int ii = i, jj = j, kk = k;
                if (!neighbour(g, d, s, ii, jj, kk)) continue;
                if (bface(g, c, ii, jj)) continue;
                long long q = ii + (long long)g.nx * (jj + (long long)g.ny * kk);
                if ((mask[q] >> c) & 1u) continue;       // internal neighbour
                double phiQ = sampled ? geo.sdf[c][q]
                                      : phi_at(geo, coord(g, 0, ii, c), coord(g, 1, jj, c), coord(g, 2, kk, c));
                double dl;
                if (phiQ == 0.0) {
                    dl = D;
                } else if (sampled) {
                    // the root of the straight line through the two samples
                    dl = __dmul_rn(D, __ddiv_rn(phiP, __dsub_rn(phiP, phiQ)));
                } else {
                    dl = delta_closed(geo, P, d, s, D);
                    if (dl < 0.0) dl = delta_bisect(geo, P, d, s, D);
                }
                dl = fmin(fmax(dl, 1e-12 * D), D);
                if (d == 1 && g.ystr) {
                    lam = lam + a.nu * 2.0 * (D - dl) / (dl * D * Dsum);
                    src = src + a.nu * (a.wall_u[c] * wall_factor(geo.kind, d, s)) * 2.0 / (dl * Dsum);
                } else if (a.body.kind != 0) {
                    // a moving body: the wall velocity at the crossing X = P + s delta e_d, in the
                    // body-frame form that pairs with the operator reading the body's point Q as
                    // its own velocity: nu (U(X) / (delta D) - U(Q) / D^2) per crossed arm (for a
                    // translating body lambda_arm U_b, so the wall term is -lambda (w - U_b))
                    double X[3] = {P[0], P[1], P[2]};
                    X[d] = X[d] + s * dl;
                    const double uw = bodyvel(a.body, c, X[0], X[1]);
                    const double uq = bodyvel(a.body, c, coord(g, 0, ii, c), coord(g, 1, jj, c));
                    lam = lam + a.nu * (D - dl) / (dl * D * D);
                    src = src + a.nu * (uw / (dl * D) - uq / (D * D));
                } else {
                    lam = lam + a.nu * (D - dl) / (dl * D * D);
                    src = src + a.nu * (a.wall_u[c] * wall_factor(geo.kind, d, s)) / (dl * D);
                }
            }
        }
    }
    a.lam[c][m] = lam;
    a.src[c][m] = src;
}

// ---------------------------------------------------------------------------
// Per-stage implicit coefficients (Eq. Bexpr / expint / rk3-rai)
// ---------------------------------------------------------------------------
__device__ double B_of_x(double x, int mode) { return ibm_B_of_x(x, mode); }

template <typename T>
struct CoefArgs {
    const double* lam[3];
    const double* src[3];
    Coef4<T>* coef[3];   // [3 stages][count]
    int count[3];
    double ckdt[3];
    double dta[3];      // dt a_k
    int bmode;
};

template <typename T>
__global__ void k_coefs(CoefArgs<T> a) {
    int c = blockIdx.y;
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= a.count[c]) return;
    double lam = a.lam[c][m];
    double s = a.src[c][m];
    for (int st = 0; st < 3; ++st) {
        Coef4<T> q;
        q.s = (T)s;
        if (a.bmode == IBM_B_EXPLICIT) {
            // -lambda u joins N (through pad) and u* = u + R: alpha = 1 - dt a_k lambda, beta = 1
            q.a = (T)(1.0 - a.dta[st] * lam);
            q.b = (T)1;
            q.pad = (T)lam;
        } else {
            double x = lam * a.ckdt[st];
            double B = B_of_x(x, a.bmode);
            q.a = (T)(B / (B + x));
            q.b = (T)(1.0 / (B + x));
            q.pad = (T)0;
        }
        a.coef[c][(long long)st * a.count[c] + m] = q;
    }
}

// Flux control response: sum over the u IBM points of (1 - beta_k) and the
// number of internal u points (the exact beta of non-IBM points is 1).
__global__ void k_flux_response(GridP g, const uint8_t* __restrict__ mask, const double* __restrict__ lam_u,
                                const int* __restrict__ idx_u, int count_u, double ck0, double ck1, double ck2, int bmode, double* out) {
    __shared__ double sh[4][32];
    double acc[4] = {0, 0, 0, 0};
    long long stride = (long long)gridDim.x * blockDim.x;
    // a stretched y weighs each point by its cell height (the volumes differ by row)
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < g.N; id += stride)
        acc[0] += (mask[id] & IBM_MASK_U) ? (g.ystr ? ytab(g, YT_DYC, (int)((id / g.nx) % g.ny)) : 1.0) : 0.0;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < count_u; m += stride) {
        double l = lam_u[m];
        const double wy = g.ystr ? ytab(g, YT_DYC, (int)((idx_u[m] / g.nx) % g.ny)) : 1.0;
        double ck[3] = {ck0, ck1, ck2};
        for (int st = 0; st < 3; ++st) {
            double x = bmode == IBM_B_EXPLICIT ? 0.0 : l * ck[st];
            double B = B_of_x(x, bmode);
            acc[1 + st] += (1.0 - 1.0 / (B + x)) * wy;
        }
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = 0; q < 4; ++q) {
        double v = warp_sum(acc[q]);
        if (lane == 0) sh[q][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[threadIdx.x][w];
        out[blockIdx.x * 4 + threadIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------
// Fluid inflow and outflow faces of an inflow/outflow x: out[0] += inflow faces,
// out[1] += outflow faces (integer counts, exact)
__global__ void k_face_count(GridP g, const uint8_t* __restrict__ mask, int* __restrict__ out) {
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;   // row (j, k)
    if (r >= (long long)g.ny * g.nz) return;
    const long long base = r * g.nx;
    if (mask[base] & IBM_MASK_FACE) atomicAdd(out, 1);
    if (mask[base + g.nx - 1] & IBM_MASK_FACE) atomicAdd(out + 1, 1);
}

// Stretched y: the summed cell heights of the fluid inflow (out[0]) and outflow (out[1]) faces
__global__ void k_face_area(GridP g, const uint8_t* __restrict__ mask, double* __restrict__ out) {
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;   // row (j, k)
    if (r >= (long long)g.ny * g.nz) return;
    const long long base = r * g.nx;
    const double A = ytab(g, YT_DYC, (int)(r % g.ny));
    if (mask[base] & IBM_MASK_FACE) atomicAdd(out, A);
    if (mask[base + g.nx - 1] & IBM_MASK_FACE) atomicAdd(out + 1, A);
}

// Thomas pivots of the y systems, one thread per (kz, kx)
// ---------------------------------------------------------------------------
__global__ void k_pivots(GridP g, double* __restrict__ piv, float* __restrict__ piv32, uint8_t* __restrict__ use32,
                         double tau) {
    long long sys = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long nsys = (long long)g.nzs * g.nxh;
    if (sys >= nsys) return;
    int kx = (int)(sys % g.nxh);
    int kz = (int)(sys / g.nxh);
    const double PI = 3.141592653589793;
    // periodic x: Fourier modes, 4 sin^2(pi k/n)/dx^2; Neumann x: cosine modes, 4 sin^2(pi k/2n)/dx^2
    double sx = g.xper ? sin(PI * kx / g.nx) : sin(PI * kx / (2.0 * g.nx));
    double K = 4.0 * sx * sx / (g.dx * g.dx);
    if (g.ndim == 3 && g.nz > 1) {
        double sz = sin(PI * kz / g.nz);
        K += 4.0 * sz * sz / (g.dz * g.dz);
    }
    double Kd = K * g.dy * g.dy;
    bool zero = (kx == 0 && kz == 0);
    if (g.ystr) {     // the symmetric unit off-diagonal form: dominant when K s_j^2 dyc_j >= 1 in every row
        double mn = 1e300;
        for (int j = 0; j < g.ny; ++j) mn = fmin(mn, K * ytab(g, YT_PBK, j));
        Kd = mn;
    }
    use32[sys] = (!zero && Kd >= tau) ? 1 : 0;
    double wprev = 0.0;
    for (int j = 0; j < g.ny; ++j) {
        bool end = (j == 0 || j == g.ny - 1);
        double b = g.ystr ? ytab(g, YT_PBE, j) - K * ytab(g, YT_PBK, j) : (end ? -1.0 : -2.0) - Kd;
        double w;
        if (j == 0) w = zero ? 0.0 : 1.0 / b;
        else w = 1.0 / (b - wprev);
        piv[((long long)kz * g.ny + j) * g.nxh + kx] = w;
        piv32[((long long)kz * g.ny + j) * g.nxh + kx] = (float)w;
        wprev = w;
    }
}

// Wall-shear stress along a lower wall: per u IBM point whose -y arm crosses the wall,
// nu times the slope at the wall of the quadratic through 0 (wall), u_P (delta) and u_Q
// (delta + dy, the point above; u_P / delta when Q is not internal), summed per x column
// with a count, into acc[0..nx) and acc[nx..2nx).
template <typename T>
__global__ void k_wall_shear(GridP g, GeomP geo, const int* __restrict__ idx, int count,
                             const uint8_t* __restrict__ mask, const T* __restrict__ u, double nu,
                             double* __restrict__ acc) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= count) return;
    const int lin = idx[m];
    const int i = lin % g.nx;
    const int j = (lin / g.nx) % g.ny;
    const int k = lin / (g.nx * g.ny);
    if (j == 0) return;
    const int below = lin - g.nx;
    if (mask[below] & IBM_MASK_U) return;             // no wall below this point
    // a stretched y: the arm below P and the step up to Q are the row's own centre distances
    const double D = g.ystr ? ytab(g, YT_HC, j) : g.dy;
    const double Dp = g.ystr ? ytab(g, YT_HC, j + 1) : g.dy;
    const double P[3] = {coord(g, 0, i, 0), coord(g, 1, j, 0), coord(g, 2, k, 0)};
    const bool sampled = geo.kind == IBM_GEOM_SAMPLED;
    const double phiP = sampled ? geo.sdf[0][lin] : phi_at(geo, P[0], P[1], P[2]);
    const double phiQ = sampled ? geo.sdf[0][below] : phi_at(geo, P[0], coord(g, 1, j - 1, 0), P[2]);
    double dl;
    if (phiQ == 0.0) {
        dl = D;
    } else if (sampled) {
        dl = __dmul_rn(D, __ddiv_rn(phiP, __dsub_rn(phiP, phiQ)));
    } else {
        dl = delta_closed(geo, P, 1, -1, D);
        if (dl < 0.0) dl = delta_bisect(geo, P, 1, -1, D);
    }
    dl = fmin(fmax(dl, 1e-12 * D), D);
    const double uP = (double)u[lin];
    double slope;
    if (j + 1 < g.ny && (mask[lin + g.nx] & IBM_MASK_U)) {
        const double uQ = (double)u[lin + g.nx];
        const double a = dl + Dp;
        slope = (uP * (a * a) - uQ * (dl * dl)) / (dl * Dp * a);
    } else {
        slope = uP / dl;
    }
    atomicAdd(acc + i, nu * slope);
    atomicAdd(acc + g.nx + i, 1.0);
}

}  // namespace

ibm_status geom_wall_shear(ibm_solver* h, double wavelength, double* tau_x, double* tau1) {
    const GridP& g = h->gp;
    double* acc = (double*)h->rhs;                     // scratch between steps
    IBM_CUDA_TRY(cudaMemsetAsync(acc, 0, 2 * (size_t)g.nx * sizeof(double), h->stream));
    const int cnt = h->counts[0];
    if (cnt > 0) {
        const int nb = (cnt + 127) / 128;
        if (h->prec == IBM_FP64)
            k_wall_shear<double><<<nb, 128, 0, h->stream>>>(g, h->geo, h->idx[0], cnt, h->mask,
                                                           (const double*)h->buf.u[0], h->phys.nu, acc);
        else
            k_wall_shear<float><<<nb, 128, 0, h->stream>>>(g, h->geo, h->idx[0], cnt, h->mask,
                                                          (const float*)h->buf.u[0], h->phys.nu, acc);
        IBM_LAUNCH_CHECK();
    }
    std::vector<double> v(2 * (size_t)g.nx);
    IBM_CUDA_TRY(cudaMemcpyAsync(v.data(), acc, v.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    IBM_CUDA_TRY(cudaStreamSynchronize(h->stream));
    double c1 = 0.0, s1 = 0.0;
    const double two_pi = 6.283185307179586;
    for (int i = 0; i < g.nx; ++i) {
        const double t = v[g.nx + i] > 0.0 ? v[i] / v[g.nx + i] : std::nan("");
        if (tau_x) tau_x[i] = t;
        if (v[g.nx + i] > 0.0) {
            const double xi = g.ox + (i + 1.0) * g.dx;
            c1 += t * std::cos(two_pi * xi / wavelength);
            s1 += t * std::sin(two_pi * xi / wavelength);
        }
    }
    if (tau1) {
        tau1[0] = 2.0 / g.nx * c1;
        tau1[1] = 2.0 / g.nx * s1;
    }
    return IBM_OK;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
ibm_status geom_classify(ibm_solver* h, bool fresh_fill) {
    const GridP& g = h->gp;
    int nb = (int)((g.N + 255) / 256);
    cudaEvent_t t;
    timer_begin(h, "classify", &t);
    k_classify_vel<<<nb, 256, 0, h->stream>>>(g, h->geo, h->velbits);
    IBM_LAUNCH_CHECK();
    if (fresh_fill) {     // before the new mask replaces the previous one
        if (h->prec == IBM_FP64)
            k_fresh_fill<double><<<nb, 256, 0, h->stream>>>(g, h->velbits, h->mask, h->body, (double*)h->buf.u[0],
                                                            (double*)h->buf.u[1],
                                                            (double*)h->buf.u[g.ncomp == 3 ? 2 : 0]);
        else
            k_fresh_fill<float><<<nb, 256, 0, h->stream>>>(g, h->velbits, h->mask, h->body, (float*)h->buf.u[0],
                                                           (float*)h->buf.u[1],
                                                           (float*)h->buf.u[g.ncomp == 3 ? 2 : 0]);
        IBM_LAUNCH_CHECK();
    }
    k_classify_final<<<nb, 256, 0, h->stream>>>(g, h->velbits, h->mask);
    IBM_LAUNCH_CHECK();
    timer_end(h, t, "classify");
    long long nthreads = h->nseg * IBM_WARP;
    int nbs = (int)((nthreads + 255) / 256);
    k_segcount<<<nbs, 256, 0, h->stream>>>(g, h->nseg, h->mask, h->segcnt[0], h->segcnt[1], h->segcnt[2]);
    IBM_LAUNCH_CHECK();
    int nblocks = (int)((h->nseg + SCAN_CH - 1) / SCAN_CH);
    ScanArgs sa;
    for (int c = 0; c < 3; ++c) { sa.in[c] = h->segcnt[c]; sa.out[c] = h->segoff[c]; }
    k_scan_partials<<<dim3(nblocks, 3), SCAN_T, 0, h->stream>>>(sa, h->nseg, h->scan_tmp, nblocks);
    IBM_LAUNCH_CHECK();
    k_scan_top<<<3, 1024, 0, h->stream>>>(h->scan_tmp, nblocks, h->d_counts);
    IBM_LAUNCH_CHECK();
    k_scan_apply<<<dim3(nblocks, 3), SCAN_T, 0, h->stream>>>(sa, h->nseg, h->scan_tmp, nblocks);
    IBM_LAUNCH_CHECK();
    int faces[2] = {0, 0};
    if (!g.xper) {
        IBM_CUDA_TRY(cudaMemsetAsync(h->d_counts + 4, 0, 2 * sizeof(int), h->stream));
        const long long rows = (long long)g.ny * g.nz;
        k_face_count<<<(int)((rows + 255) / 256), 256, 0, h->stream>>>(g, h->mask, h->d_counts + 4);
        IBM_LAUNCH_CHECK();
        IBM_CUDA_TRY(cudaMemcpyAsync(faces, h->d_counts + 4, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    }
    IBM_CUDA_TRY(cudaMemcpyAsync(h->counts, h->d_counts, 3 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    IBM_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->nfaces[0] = faces[0];
    h->nfaces[1] = faces[1];
    h->aface[0] = faces[0];
    h->aface[1] = faces[1];
    if (!g.xper && g.ystr) {           // faces of unequal height: their summed heights
        double a[2] = {0.0, 0.0};
        IBM_CUDA_TRY(cudaMemsetAsync(h->partials, 0, 2 * sizeof(double), h->stream));
        const long long rows = (long long)g.ny * g.nz;
        k_face_area<<<(int)((rows + 255) / 256), 256, 0, h->stream>>>(g, h->mask, h->partials);
        IBM_LAUNCH_CHECK();
        IBM_CUDA_TRY(cudaMemcpyAsync(a, h->partials, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        IBM_CUDA_TRY(cudaStreamSynchronize(h->stream));
        h->aface[0] = a[0];
        h->aface[1] = a[1];
    }
    return IBM_OK;
}

ibm_status geom_build_lists_and_weights(ibm_solver* h) {
    const GridP& g = h->gp;
    long long nthreads = h->nseg * IBM_WARP;
    int nbs = (int)((nthreads + 255) / 256);
    k_compact<<<nbs, 256, 0, h->stream>>>(g, h->nseg, h->mask, h->segoff[0], h->segoff[1], h->segoff[2],
                                          h->idx[0], h->idx[1], h->idx[2]);
    IBM_LAUNCH_CHECK();
    WeightArgs a;
    int maxc = 1;
    for (int c = 0; c < 3; ++c) {
        a.idx[c] = h->idx[c];
        a.lam[c] = h->lam[c];
        a.src[c] = h->src[c];
        a.count[c] = h->counts[c];
        a.wall_u[c] = h->phys.wall_u[c];
        if (h->counts[c] > maxc) maxc = h->counts[c];
    }
    a.nu = h->phys.nu;
    a.no_ibm = h->phys.no_ibm;
    a.body = h->body;
    k_weights<<<dim3((maxc + 127) / 128, 3), 128, 0, h->stream>>>(g, h->geo, a, h->mask);
    IBM_LAUNCH_CHECK();
    return IBM_OK;
}

ibm_status geom_stage_coefficients(ibm_solver* h) {
    const double rkc[3] = {64.0 / 120.0, 16.0 / 120.0, 40.0 / 120.0};
    const double rka[3] = {64.0 / 120.0, 50.0 / 120.0, 90.0 / 120.0};
    int maxc = 1;
    for (int c = 0; c < 3; ++c) maxc = h->counts[c] > maxc ? h->counts[c] : maxc;
    dim3 grid((maxc + 127) / 128, 3);
    if (h->prec == IBM_FP64) {
        CoefArgs<double> a;
        for (int c = 0; c < 3; ++c) {
            a.lam[c] = h->lam[c]; a.src[c] = h->src[c]; a.count[c] = h->counts[c];
            a.coef[c] = (Coef4<double>*)h->coef[c]; a.ckdt[c] = rkc[c] * h->phys.dt;
            a.dta[c] = rka[c] * h->phys.dt;
        }
        a.bmode = h->phys.bmode;
        k_coefs<double><<<grid, 128, 0, h->stream>>>(a);
    } else {
        CoefArgs<float> a;
        for (int c = 0; c < 3; ++c) {
            a.lam[c] = h->lam[c]; a.src[c] = h->src[c]; a.count[c] = h->counts[c];
            a.coef[c] = (Coef4<float>*)h->coef[c]; a.ckdt[c] = rkc[c] * h->phys.dt;
            a.dta[c] = rka[c] * h->phys.dt;
        }
        a.bmode = h->phys.bmode;
        k_coefs<float><<<grid, 128, 0, h->stream>>>(a);
    }
    IBM_LAUNCH_CHECK();
    // flux-control response S_k = c_k dt dV sum_internal beta_k
    const GridP& g = h->gp;
    int nb = 120;
    k_flux_response<<<nb, 256, 0, h->stream>>>(g, h->mask, h->lam[0], h->idx[0], h->counts[0], rkc[0] * h->phys.dt,
                                               rkc[1] * h->phys.dt, rkc[2] * h->phys.dt, h->phys.bmode, h->partials);
    IBM_LAUNCH_CHECK();
    std::vector<double> part(nb * 4);
    IBM_CUDA_TRY(cudaMemcpyAsync(part.data(), h->partials, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                 h->stream));
    IBM_CUDA_TRY(cudaStreamSynchronize(h->stream));
    double acc[4] = {0, 0, 0, 0};
    for (int b = 0; b < nb; ++b)
        for (int q = 0; q < 4; ++q) acc[q] += part[b * 4 + q];
    double dV = g.dx * (g.ystr ? 1.0 : g.dy) * (g.ndim == 3 ? g.dz : 1.0);   // stretched: dy in the sums
    for (int st = 0; st < 3; ++st) h->S[st] = rkc[st] * h->phys.dt * dV * (acc[0] - acc[1 + st]);
    return IBM_OK;
}

ibm_status geom_pivots(ibm_solver* h) {
    long long nsys = (long long)h->gp.nzs * h->gp.nxh;
    // FP32 sweeps only in FP32 mode, for systems with K dy^2 >= 1
    double tau = h->prec == IBM_FP32 ? 1.0 : 1e300;
    k_pivots<<<(int)((nsys + 127) / 128), 128, 0, h->stream>>>(h->gp, h->pivots, h->pivots32, h->use32, tau);
    IBM_LAUNCH_CHECK();
    // system order: FP64 systems first, each group sorted by (kz, kx)
    std::vector<uint8_t> use(nsys);
    IBM_CUDA_TRY(cudaMemcpyAsync(use.data(), h->use32, nsys, cudaMemcpyDeviceToHost, h->stream));
    IBM_CUDA_TRY(cudaStreamSynchronize(h->stream));
    std::vector<int> order;
    order.reserve(nsys);
    for (long long q = 0; q < nsys; ++q)
        if (!use[q]) order.push_back((int)q);
    h->n64 = (int)order.size();
    for (long long q = 0; q < nsys; ++q)
        if (use[q]) order.push_back((int)q);
    IBM_CUDA_TRY(cudaMemcpyAsync(h->sys_order, order.data(), nsys * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    IBM_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return IBM_OK;
}
