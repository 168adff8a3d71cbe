// Hot-path kernels of one RK3 substage:
//   momentum predictor with the fused implicit IBM division   (Sec. 2.4, Eq. rk3-rai)
//   constant-flow-rate forcing                                 (reading: uniform forcing)
//   divergence                                                 (Sec. 2.1 projection)
//   FFT (cuFFT) + batched FP64 tridiagonal Poisson solve + inverse FFT
//   gradient correction and pressure update
// plus the diagnostics reductions.
#include "common.cuh"

#include <cstdio>

namespace {

// ---------------------------------------------------------------------------
// Masked loads with the y-wall rules
// ---------------------------------------------------------------------------
// Value of component c at (i,j,k) as the momentum operator sees it:
//   * x and z wrap (periodic);
//   * beyond a y wall: the wall-normal component reads the wall value (0),
//     a tangential component reads the mirror ghost sig * (adjacent value);
//   * every non-internal point (external or wall face) reads 0, so the ghost
//     term of the IBM vanishes on its own (Sec. 2.4, before Eq. semidisc-mom-comp).
template <typename T>
__device__ __forceinline__ T ld(const GridP& g, const T* __restrict__ f, const uint8_t* __restrict__ mask, int c,
                                int i, int j, int k) {
    i = wrapi(i, g.nx);
    k = wrapi(k, g.nz);
    T s = T(1);
    if (j < 0) {
        if (c == 1) return T(0);
        s = (T)g.sig_lo;
        j = 0;
    } else if (j >= g.ny) {
        if (c == 1) return T(0);
        s = (T)g.sig_hi;
        j = g.ny - 1;
    }
    long long id = i + (long long)g.nx * (j + (long long)g.ny * k);
    return ((__ldg(mask + id) >> c) & 1u) ? s * __ldg(f + id) : T(0);
}

template <typename T> __device__ __forceinline__ T sq(T a) { return a * a; }

template <typename T>
struct MomF {
    const T* u[3];
    const T* p;
    const uint8_t* mask;
    T* us[3];
    T* Nn[3];
};

// N_u = -C_u + nu L u + g_x at an internal u point (Harlow-Welch flux form)
template <typename T, bool THREE>
__device__ __forceinline__ T rhs_u(const GridP& g, const MomF<T>& F, const StageP<T>& sp, T uP, int i, int j, int k) {
    const uint8_t* M = F.mask;
    const T *U = F.u[0], *V = F.u[1], *W = F.u[2];
    T uE = ld(g, U, M, 0, i + 1, j, k), uW = ld(g, U, M, 0, i - 1, j, k);
    T uN = ld(g, U, M, 0, i, j + 1, k), uS = ld(g, U, M, 0, i, j - 1, k);
    T h = T(0.5);
    T cx = (sq(h * (uP + uE)) - sq(h * (uW + uP))) * sp.idx;
    T vN = h * (ld(g, V, M, 1, i, j, k) + ld(g, V, M, 1, i + 1, j, k));
    T vS = h * (ld(g, V, M, 1, i, j - 1, k) + ld(g, V, M, 1, i + 1, j - 1, k));
    T cy = (vN * (h * (uP + uN)) - vS * (h * (uS + uP))) * sp.idy;
    T lap = (uE - T(2) * uP + uW) * sp.idx2 + (uN - T(2) * uP + uS) * sp.idy2;
    T cz = T(0);
    if (THREE) {
        T uT = ld(g, U, M, 0, i, j, k + 1), uB = ld(g, U, M, 0, i, j, k - 1);
        T wT = h * (ld(g, W, M, 2, i, j, k) + ld(g, W, M, 2, i + 1, j, k));
        T wB = h * (ld(g, W, M, 2, i, j, k - 1) + ld(g, W, M, 2, i + 1, j, k - 1));
        cz = (wT * (h * (uP + uT)) - wB * (h * (uB + uP))) * sp.idz;
        lap += (uT - T(2) * uP + uB) * sp.idz2;
    }
    return -(cx + cy + cz) + sp.nu * lap + sp.g[0];
}

template <typename T, bool THREE>
__device__ __forceinline__ T rhs_v(const GridP& g, const MomF<T>& F, const StageP<T>& sp, T vP, int i, int j, int k) {
    const uint8_t* M = F.mask;
    const T *U = F.u[0], *V = F.u[1], *W = F.u[2];
    T vE = ld(g, V, M, 1, i + 1, j, k), vW = ld(g, V, M, 1, i - 1, j, k);
    T vN = ld(g, V, M, 1, i, j + 1, k), vS = ld(g, V, M, 1, i, j - 1, k);
    T h = T(0.5);
    T uE = h * (ld(g, U, M, 0, i, j, k) + ld(g, U, M, 0, i, j + 1, k));
    T uW = h * (ld(g, U, M, 0, i - 1, j, k) + ld(g, U, M, 0, i - 1, j + 1, k));
    T cx = (uE * (h * (vP + vE)) - uW * (h * (vW + vP))) * sp.idx;
    T cy = (sq(h * (vP + vN)) - sq(h * (vS + vP))) * sp.idy;
    T lap = (vE - T(2) * vP + vW) * sp.idx2 + (vN - T(2) * vP + vS) * sp.idy2;
    T cz = T(0);
    if (THREE) {
        T vT = ld(g, V, M, 1, i, j, k + 1), vB = ld(g, V, M, 1, i, j, k - 1);
        T wT = h * (ld(g, W, M, 2, i, j, k) + ld(g, W, M, 2, i, j + 1, k));
        T wB = h * (ld(g, W, M, 2, i, j, k - 1) + ld(g, W, M, 2, i, j + 1, k - 1));
        cz = (wT * (h * (vP + vT)) - wB * (h * (vB + vP))) * sp.idz;
        lap += (vT - T(2) * vP + vB) * sp.idz2;
    }
    return -(cx + cy + cz) + sp.nu * lap + sp.g[1];
}

template <typename T>
__device__ __forceinline__ T rhs_w(const GridP& g, const MomF<T>& F, const StageP<T>& sp, T wP, int i, int j, int k) {
    const uint8_t* M = F.mask;
    const T *U = F.u[0], *V = F.u[1], *W = F.u[2];
    T wE = ld(g, W, M, 2, i + 1, j, k), wW = ld(g, W, M, 2, i - 1, j, k);
    T wN = ld(g, W, M, 2, i, j + 1, k), wS = ld(g, W, M, 2, i, j - 1, k);
    T wT = ld(g, W, M, 2, i, j, k + 1), wB = ld(g, W, M, 2, i, j, k - 1);
    T h = T(0.5);
    T uE = h * (ld(g, U, M, 0, i, j, k) + ld(g, U, M, 0, i, j, k + 1));
    T uW = h * (ld(g, U, M, 0, i - 1, j, k) + ld(g, U, M, 0, i - 1, j, k + 1));
    T cx = (uE * (h * (wP + wE)) - uW * (h * (wW + wP))) * sp.idx;
    T vN = h * (ld(g, V, M, 1, i, j, k) + ld(g, V, M, 1, i, j, k + 1));
    T vS = h * (ld(g, V, M, 1, i, j - 1, k) + ld(g, V, M, 1, i, j - 1, k + 1));
    T cy = (vN * (h * (wP + wN)) - vS * (h * (wS + wP))) * sp.idy;
    T cz = (sq(h * (wP + wT)) - sq(h * (wB + wP))) * sp.idz;
    T lap = (wE - T(2) * wP + wW) * sp.idx2 + (wN - T(2) * wP + wS) * sp.idy2 + (wT - T(2) * wP + wB) * sp.idz2;
    return -(cx + cy + cz) + sp.nu * lap + sp.g[2];
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    int lane = threadIdx.x & 31;
    int nthr = blockDim.x * blockDim.y * blockDim.z;
    int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    int wid = tid >> 5;
    v = warp_sum(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
        for (int w = 0; w < (nthr >> 5); ++w) s += sh[w];
    return s;
}

// ---------------------------------------------------------------------------
// K3: momentum predictor with the implicit IBM diagonal division.
// One thread per cell computes u*, v*, w* of its cell; blockDim.x = 32 so
// that each warp covers one aligned 32-point x segment of a row, which
// gives the list position of an IBM point as segoff + (IBM points of lower
// lanes) with one ballot.
// ---------------------------------------------------------------------------
template <typename T, bool THREE>
__global__ void __launch_bounds__(256) k_momentum(GridP g, MomF<T> F, StageP<T> sp, IbmStage<T> ib,
                                                  double* __restrict__ flux_part) {
    __shared__ double sh[32];
    int i = blockIdx.x * IBM_WARP + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z * blockDim.z + threadIdx.z;
    double fsum = 0.0;
    if (j < g.ny && k < g.nz) {
        long long row = j + (long long)g.ny * k;
        long long id = i + (long long)g.nx * row;
        long long seg = row * g.nsegx + blockIdx.x;
        uint8_t m = i < g.nx ? F.mask[id] : 0;
        int pos[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            unsigned b = __ballot_sync(0xffffffffu, (m >> (4 + c)) & 1u);
            pos[c] = __popc(b & lanemask_lt());
        }
        if (i < g.nx) {
            const int ncomp = THREE ? 3 : 2;
#pragma unroll
            for (int c = 0; c < ncomp; ++c) {
                T out = T(0), Nv = T(0);
                if ((m >> c) & 1u) {
                    T uP = F.u[c][id];
                    T N;
                    T gp;
                    if (c == 0) {
                        N = rhs_u<T, THREE>(g, F, sp, uP, i, j, k);
                        gp = (F.p[(long long)wrapi(i + 1, g.nx) + g.nx * row] - F.p[id]) * sp.idx;
                    } else if (c == 1) {
                        N = rhs_v<T, THREE>(g, F, sp, uP, i, j, k);
                        gp = (F.p[id + g.nx] - F.p[id]) * sp.idy;   // j < ny-1 for internal v
                    } else {
                        N = rhs_w<T>(g, F, sp, uP, i, j, k);
                        long long idT = i + (long long)g.nx * (j + (long long)g.ny * wrapi(k + 1, g.nz));
                        gp = (F.p[idT] - F.p[id]) * sp.idz;
                    }
                    bool isibm = (m >> (4 + c)) & 1u;
                    Coef4<T> q;
                    if (isibm) {
                        q = ib.coef[c][ib.segoff[c][seg] + pos[c]];
                        N += q.s;
                    }
                    T R = sp.dta * N - sp.ckdt * gp;
                    if (sp.read_prev) R += sp.dtb * F.Nn[c][id];
                    out = isibm ? (q.a * uP + q.b * R) : (uP + R);
                    Nv = N;
                    if (c == 0) fsum = (double)out;
                }
                F.us[c][id] = out;
                if (sp.write_n) F.Nn[c][id] = Nv;
            }
        }
    }
    if (sp.flux_sum) {
        double s = block_sum(fsum, sh);
        int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
        if (tid == 0) flux_part[blockIdx.x + gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z)] = s;
    }
}

// Pi = (Q_target - Q(u*)) / S_k  (one block, fixed summation order)
__global__ void k_flux_pi(const double* __restrict__ part, int n, double dV, double target, double S,
                          double* __restrict__ scal) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) s += part[t];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double q = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) q += sh[w];
        scal[0] = (target - q * dV) / S;
    }
}

// u* += Pi c_k dt beta at internal u points (beta = 1, or the stage's IBM beta)
template <typename T>
__global__ void __launch_bounds__(256) k_flux_apply(GridP g, T* __restrict__ us, const uint8_t* __restrict__ mask,
                                                    IbmStage<T> ib, const double* __restrict__ scal, T ckdt) {
    int i = blockIdx.x * IBM_WARP + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (j >= g.ny || k >= g.nz) return;
    long long row = j + (long long)g.ny * k;
    long long id = i + (long long)g.nx * row;
    uint8_t m = i < g.nx ? mask[id] : 0;
    unsigned b = __ballot_sync(0xffffffffu, (m >> 4) & 1u);
    if (i >= g.nx || !(m & IBM_MASK_U)) return;
    T beta = T(1);
    if ((m >> 4) & 1u) beta = ib.coef[0][ib.segoff[0][row * g.nsegx + blockIdx.x] + __popc(b & lanemask_lt())].b;
    us[id] += (T)scal[0] * ckdt * beta;
}

// ---------------------------------------------------------------------------
// K4: divergence of the predictor, D u* (FP64 arithmetic)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_divergence(GridP g, const T* __restrict__ u, const T* __restrict__ v,
                                                    const T* __restrict__ w, T* __restrict__ rhs) {
    long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    int i = (int)(id % g.nx);
    long long row = id / g.nx;
    int j = (int)(row % g.ny);
    int k = (int)(row / g.ny);
    double d = ((double)u[id] - (double)u[row * g.nx + wrapi(i - 1, g.nx)]) / g.dx;
    double vm = j > 0 ? (double)v[id - g.nx] : 0.0;
    d += ((double)v[id] - vm) / g.dy;
    if (g.ndim == 3) {
        long long idB = i + (long long)g.nx * (j + (long long)g.ny * wrapi(k - 1, g.nz));
        d += ((double)w[id] - (double)w[idB]) / g.dz;
    }
    rhs[id] = (T)d;
}

// ---------------------------------------------------------------------------
// K6: batched tridiagonal solve along y for every (kz, kx), FP64 arithmetic.
// Unit off-diagonals after scaling by dy^2; pivots w_j precomputed:
//   forward  d'_j = (d_j - d'_{j-1}) w_j      (w_0 = 0 for the zero mode: phi_0 = 0)
//   backward x_j  = d'_j - w_j x_{j+1}
// The zero mode's solution is shifted to zero mean (box-mean gauge).
// ---------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(128) k_tridiag(GridP g, C* spec, double2* tmp,
                                                 const double* __restrict__ piv, double scale) {
    long long sys = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long nsys = (long long)g.nz * g.nxh;
    if (sys >= nsys) return;
    int kx = (int)(sys % g.nxh);
    int kz = (int)(sys / g.nxh);
    long long base = (long long)kz * g.ny * g.nxh + kx;
    long long st = g.nxh;
    double2 dp = make_double2(0.0, 0.0);
    for (int j = 0; j < g.ny; ++j) {
        long long o = base + j * st;
        C r = spec[o];
        double w = piv[o];
        double dr = (double)r.x * scale, di = (double)r.y * scale;
        if (j == 0) dp = make_double2(dr * w, di * w);
        else dp = make_double2((dr - dp.x) * w, (di - dp.y) * w);
        tmp[o] = dp;
    }
    double2 x = dp;
    double sr = x.x, si = x.y;
    {
        long long o = base + (long long)(g.ny - 1) * st;
        C out;
        out.x = x.x;
        out.y = x.y;
        spec[o] = out;
    }
    for (int j = g.ny - 2; j >= 0; --j) {
        long long o = base + j * st;
        double2 d = tmp[o];
        double w = piv[o];
        x = make_double2(d.x - w * x.x, d.y - w * x.y);
        sr += x.x;
        si += x.y;
        C out;
        out.x = x.x;
        out.y = x.y;
        spec[o] = out;
    }
    if (kx == 0 && kz == 0) {
        double mr = sr / g.ny, mi = si / g.ny;
        for (int j = 0; j < g.ny; ++j) {
            long long o = base + j * st;
            C v = spec[o];
            v.x = (double)v.x - mr;
            v.y = (double)v.y - mi;
            spec[o] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// K7: u = u* - G psi on every non-wall face, p += psi / (c_k dt)
// (psi = c_k dt phi is what the Poisson solve returns for rhs = D u*)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_correct(GridP g, const T* __restrict__ us0, const T* __restrict__ us1,
                                                 const T* __restrict__ us2, const T* __restrict__ psi,
                                                 T* __restrict__ u0, T* __restrict__ u1, T* __restrict__ u2,
                                                 T* __restrict__ p, T inv_ckdt, int update_p) {
    long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    int i = (int)(id % g.nx);
    long long row = id / g.nx;
    int j = (int)(row % g.ny);
    int k = (int)(row / g.ny);
    T ph = psi[id];
    u0[id] = us0[id] - (psi[row * g.nx + wrapi(i + 1, g.nx)] - ph) * (T)(1.0 / g.dx);
    u1[id] = j < g.ny - 1 ? us1[id] - (psi[id + g.nx] - ph) * (T)(1.0 / g.dy) : us1[id];
    if (g.ndim == 3) {
        long long idT = i + (long long)g.nx * (j + (long long)g.ny * wrapi(k + 1, g.nz));
        u2[id] = us2[id] - (psi[idT] - ph) * (T)(1.0 / g.dz);
    }
    if (update_p) p[id] += ph * inv_ckdt;
}

// initial-condition projection: copy the velocity with non-internal points zeroed
template <typename T>
__global__ void k_mask_copy(GridP g, const uint8_t* __restrict__ mask, const T* __restrict__ a0,
                            const T* __restrict__ a1, const T* __restrict__ a2, T* __restrict__ b0,
                            T* __restrict__ b1, T* __restrict__ b2) {
    long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    uint8_t m = mask[id];
    b0[id] = (m & IBM_MASK_U) ? a0[id] : T(0);
    b1[id] = (m & IBM_MASK_V) ? a1[id] : T(0);
    if (g.ndim == 3) b2[id] = (m & IBM_MASK_W) ? a2[id] : T(0);
}

// ---------------------------------------------------------------------------
// K8: diagnostics partials (12 doubles per block), then a fixed-order final sum
//   [0] sum div^2  [1] max |div|  [2..4] max |u_c|  [5..7] sum u_c  [8..10] sum u_c^2  [11] non-finite count
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_diag(GridP g, const T* __restrict__ u, const T* __restrict__ v,
                                              const T* __restrict__ w, const T* __restrict__ p,
                                              const uint8_t* __restrict__ mask, double* __restrict__ part) {
    __shared__ double sh[12][8];
    double a[12];
    for (int q = 0; q < 12; ++q) a[q] = 0.0;
    long long stride = (long long)gridDim.x * blockDim.x;
    const T* f[3] = {u, v, w};
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < g.N; id += stride) {
        int i = (int)(id % g.nx);
        long long row = id / g.nx;
        int j = (int)(row % g.ny);
        int k = (int)(row / g.ny);
        double d = ((double)u[id] - (double)u[row * g.nx + wrapi(i - 1, g.nx)]) / g.dx;
        d += ((double)v[id] - (j > 0 ? (double)v[id - g.nx] : 0.0)) / g.dy;
        if (g.ndim == 3)
            d += ((double)w[id] - (double)w[i + (long long)g.nx * (j + (long long)g.ny * wrapi(k - 1, g.nz))]) / g.dz;
        a[0] += d * d;
        a[1] = fmax(a[1], fabs(d));
        uint8_t m = mask[id];
        for (int c = 0; c < g.ncomp; ++c) {
            double x = (double)f[c][id];
            if (!isfinite(x)) a[11] += 1.0;
            if (!((m >> c) & 1u)) continue;
            a[2 + c] = fmax(a[2 + c], fabs(x));
            a[5 + c] += x;
            a[8 + c] += x * x;
        }
        if (!isfinite((double)p[id])) a[11] += 1.0;
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = 0; q < 12; ++q) {
        double x = a[q];
        if (q == 1 || (q >= 2 && q <= 4)) x = warp_max(x);
        else x = warp_sum(x);
        if (lane == 0) sh[q][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        int q = threadIdx.x;
        double s = 0.0;
        for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww)
            s = (q == 1 || (q >= 2 && q <= 4)) ? fmax(s, sh[q][ww]) : s + sh[q][ww];
        part[blockIdx.x * 12 + q] = s;
    }
}

__global__ void k_diag_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
    int q = threadIdx.x;
    if (q >= 12) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b)
        s = (q == 1 || (q >= 2 && q <= 4)) ? fmax(s, part[b * 12 + q]) : s + part[b * 12 + q];
    out[q] = s;
}

constexpr int DIAG_BLOCKS = 304;
const double RK_A[3] = {64.0 / 120.0, 50.0 / 120.0, 90.0 / 120.0};
const double RK_B[3] = {0.0, -34.0 / 120.0, -50.0 / 120.0};
const double RK_C[3] = {64.0 / 120.0, 16.0 / 120.0, 40.0 / 120.0};

dim3 mom_block(const GridP& g) {
    return g.ndim == 3 ? dim3(32, 4, 2) : dim3(32, 8, 1);
}

template <typename T>
ibm_status poisson_t(ibm_solver* h, void* rhs_inout) {
    const GridP& g = h->gp;
    cudaEvent_t t;
    timer_begin(h, "fft_forward", &t);
    cufftResult r;
    if (h->prec == IBM_FP64) r = cufftExecD2Z(h->plan_f, (cufftDoubleReal*)rhs_inout, (cufftDoubleComplex*)h->spec);
    else r = cufftExecR2C(h->plan_f, (cufftReal*)rhs_inout, (cufftComplex*)h->spec);
    if (r != CUFFT_SUCCESS) { h->failed = true; return ibm_set_error(IBM_E_CUDA, "cufft forward failed"); }
    timer_end(h, t, "fft_forward");
    long long nsys = (long long)g.nz * g.nxh;
    double scale = g.dy * g.dy / ((double)g.nx * (double)g.nz);
    timer_begin(h, "tridiag", &t);
    if (h->prec == IBM_FP64)
        k_tridiag<double2><<<(int)((nsys + 127) / 128), 128, 0, h->stream>>>(g, (double2*)h->spec, (double2*)h->spec,
                                                                            h->pivots, scale);
    else
        k_tridiag<float2><<<(int)((nsys + 127) / 128), 128, 0, h->stream>>>(g, (float2*)h->spec, (double2*)h->dtemp,
                                                                           h->pivots, scale);
    IBM_LAUNCH_CHECK();
    timer_end(h, t, "tridiag");
    timer_begin(h, "fft_inverse", &t);
    if (h->prec == IBM_FP64) r = cufftExecZ2D(h->plan_i, (cufftDoubleComplex*)h->spec, (cufftDoubleReal*)rhs_inout);
    else r = cufftExecC2R(h->plan_i, (cufftComplex*)h->spec, (cufftReal*)rhs_inout);
    if (r != CUFFT_SUCCESS) { h->failed = true; return ibm_set_error(IBM_E_CUDA, "cufft inverse failed"); }
    timer_end(h, t, "fft_inverse");
    return IBM_OK;
}

template <typename T>
ibm_status divergence_and_solve(ibm_solver* h, T* const us[3]) {
    const GridP& g = h->gp;
    int nb = (int)((g.N + 255) / 256);
    cudaEvent_t t;
    timer_begin(h, "divergence", &t);
    k_divergence<T><<<nb, 256, 0, h->stream>>>(g, us[0], us[1], us[2], (T*)h->rhs);
    IBM_LAUNCH_CHECK();
    timer_end(h, t, "divergence");
    return poisson_t<T>(h, h->rhs);
}

template <typename T>
ibm_status substage_t(ibm_solver* h, int k, bool predictor_only) {
    const GridP& g = h->gp;
    MomF<T> F;
    for (int c = 0; c < 3; ++c) {
        F.u[c] = (const T*)h->buf.u[c];
        F.us[c] = (T*)h->ustar[c];
        F.Nn[c] = (T*)h->Nh[c];
    }
    if (g.ndim == 2) { F.u[2] = F.u[0]; F.us[2] = F.us[0]; F.Nn[2] = F.Nn[0]; }
    F.p = (const T*)h->buf.p;
    F.mask = h->mask;
    StageP<T> sp;
    double dt = h->phys.dt;
    sp.dta = (T)(dt * RK_A[k]);
    sp.dtb = (T)(dt * RK_B[k]);
    sp.ckdt = (T)(dt * RK_C[k]);
    sp.nu = (T)h->phys.nu;
    for (int c = 0; c < 3; ++c) sp.g[c] = (T)h->phys.g[c];
    sp.idx = (T)(1.0 / g.dx); sp.idy = (T)(1.0 / g.dy); sp.idz = (T)(1.0 / g.dz);
    sp.idx2 = (T)(1.0 / (g.dx * g.dx)); sp.idy2 = (T)(1.0 / (g.dy * g.dy)); sp.idz2 = (T)(1.0 / (g.dz * g.dz));
    sp.read_prev = k > 0;
    sp.write_n = k < 2;
    bool cflux = h->phys.flow_mode == IBM_FLOW_CONST_FLUX;
    sp.flux_sum = cflux;
    IbmStage<T> ib;
    for (int c = 0; c < 3; ++c) {
        ib.segoff[c] = h->segoff[c];
        ib.coef[c] = (const Coef4<T>*)h->coef[c] + (long long)k * h->counts[c];
    }
    dim3 blk = mom_block(g);
    dim3 grd(g.nsegx, (g.ny + blk.y - 1) / blk.y, (g.nz + blk.z - 1) / blk.z);
    cudaEvent_t t;
    timer_begin(h, "momentum", &t);
    if (g.ndim == 3) k_momentum<T, true><<<grd, blk, 0, h->stream>>>(g, F, sp, ib, h->partials);
    else k_momentum<T, false><<<grd, blk, 0, h->stream>>>(g, F, sp, ib, h->partials);
    IBM_LAUNCH_CHECK();
    timer_end(h, t, "momentum");
    if (cflux) {
        int nparts = grd.x * grd.y * grd.z;
        double dV = g.dx * g.dy * (g.ndim == 3 ? g.dz : 1.0);
        timer_begin(h, "flux_control", &t);
        k_flux_pi<<<1, 1024, 0, h->stream>>>(h->partials, nparts, dV, h->phys.target_flux, h->S[k], h->scal);
        IBM_LAUNCH_CHECK();
        k_flux_apply<T><<<grd, blk, 0, h->stream>>>(g, (T*)h->ustar[0], h->mask, ib, h->scal, sp.ckdt);
        IBM_LAUNCH_CHECK();
        timer_end(h, t, "flux_control");
    }
    T* us[3] = {(T*)h->ustar[0], (T*)h->ustar[1], (T*)h->ustar[2]};
    if (predictor_only) {
        for (int c = 0; c < g.ncomp; ++c)
            IBM_CUDA_TRY(cudaMemcpyAsync(h->buf.u[c], h->ustar[c], g.N * sizeof(T), cudaMemcpyDeviceToDevice, h->stream));
        return IBM_OK;
    }
    ibm_status st = divergence_and_solve<T>(h, us);
    if (st != IBM_OK) return st;
    int nb = (int)((g.N + 255) / 256);
    timer_begin(h, "correct", &t);
    k_correct<T><<<nb, 256, 0, h->stream>>>(g, us[0], us[1], us[2], (const T*)h->rhs, (T*)h->buf.u[0],
                                            (T*)h->buf.u[1], g.ndim == 3 ? (T*)h->buf.u[2] : (T*)h->buf.u[0],
                                            (T*)h->buf.p, (T)(1.0 / (dt * RK_C[k])), 1);
    IBM_LAUNCH_CHECK();
    timer_end(h, t, "correct");
    return IBM_OK;
}

template <typename T>
ibm_status project_t(ibm_solver* h) {
    const GridP& g = h->gp;
    int nb = (int)((g.N + 255) / 256);
    T* us[3] = {(T*)h->ustar[0], (T*)h->ustar[1], g.ndim == 3 ? (T*)h->ustar[2] : (T*)h->ustar[0]};
    const T* u2 = g.ndim == 3 ? (const T*)h->buf.u[2] : (const T*)h->buf.u[0];
    k_mask_copy<T><<<nb, 256, 0, h->stream>>>(g, h->mask, (const T*)h->buf.u[0], (const T*)h->buf.u[1], u2, us[0],
                                              us[1], us[2]);
    IBM_LAUNCH_CHECK();
    ibm_status st = divergence_and_solve<T>(h, us);
    if (st != IBM_OK) return st;
    k_correct<T><<<nb, 256, 0, h->stream>>>(g, us[0], us[1], us[2], (const T*)h->rhs, (T*)h->buf.u[0],
                                            (T*)h->buf.u[1], g.ndim == 3 ? (T*)h->buf.u[2] : (T*)h->buf.u[0],
                                            (T*)h->buf.p, (T)1, 0);
    IBM_LAUNCH_CHECK();
    return IBM_OK;
}

template <typename T>
ibm_status diag_t(ibm_solver* h, double* out) {
    const GridP& g = h->gp;
    const T* w = g.ndim == 3 ? (const T*)h->buf.u[2] : (const T*)h->buf.u[0];
    k_diag<T><<<DIAG_BLOCKS, 256, 0, h->stream>>>(g, (const T*)h->buf.u[0], (const T*)h->buf.u[1], w,
                                                  (const T*)h->buf.p, h->mask, h->partials);
    IBM_LAUNCH_CHECK();
    k_diag_final<<<1, 32, 0, h->stream>>>(h->partials, DIAG_BLOCKS, h->scal + 4);
    IBM_LAUNCH_CHECK();
    IBM_CUDA_TRY(cudaMemcpyAsync(out, h->scal, 16 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    IBM_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return IBM_OK;
}

}  // namespace

int diag_blocks() { return DIAG_BLOCKS; }

ibm_status run_substage(ibm_solver* h, int k, bool predictor_only) {
    return h->prec == IBM_FP64 ? substage_t<double>(h, k, predictor_only) : substage_t<float>(h, k, predictor_only);
}

ibm_status run_project(ibm_solver* h) { return h->prec == IBM_FP64 ? project_t<double>(h) : project_t<float>(h); }

ibm_status run_poisson(ibm_solver* h, void* rhs_inout) {
    return h->prec == IBM_FP64 ? poisson_t<double>(h, rhs_inout) : poisson_t<float>(h, rhs_inout);
}

// out: [0] Pi, [4..15] the 12 diagnostics sums
ibm_status run_diagnostics(ibm_solver* h, double* out16) {
    return h->prec == IBM_FP64 ? diag_t<double>(h, out16) : diag_t<float>(h, out16);
}
