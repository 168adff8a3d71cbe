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
// K3: momentum predictor with the implicit IBM diagonal division.
//
// 2.5D shared-memory tiling: a block owns a 32 x 8 (x, y) column of cells
// and marches KZ planes along z, keeping the planes k-1, k, k+1 of u, v, w
// (with a one-cell halo) in a rolling three-slot buffer.  Each plane is
// loaded once, already in the form the operator reads it:
//   * x and z wrap (periodic);
//   * beyond a y wall the wall-normal component v reads the wall value 0 and
//     the tangential components read the mirror ghost sig * (adjacent value);
//   * every non-internal point (external or wall face) reads 0, so the ghost
//     term of the IBM vanishes by itself (Sec. 2.4, before Eq. semidisc-mom-comp).
// The stencil then reads shared memory with no branches.  Warps cover aligned
// 32-point x segments, so an IBM point's list position is segoff + the
// number of IBM points in the lower lanes (one ballot).
// ---------------------------------------------------------------------------
constexpr int TX = MOM_TX, TY = MOM_TY, KZ = MOM_KZ;
constexpr int HX = TX + 2, HY = TY + 2, HP = HX * HY;

template <typename T>
struct MomF {
    const T* u[3];
    const T* p;
    const uint8_t* mask;
    T* us[3];
    T* Nn[3];
};

// The halo tile of a plane has HP = 34 x 10 cells; each thread owns two of
// them (t = 0, 1).  Their in-plane source offsets, wall flags and ghost
// factors do not change from plane to plane and are computed once.
template <typename T>
struct TileSrc {
    int off[2];        // i + nx * j of the (wrapped / clamped) source point
    bool valid[2];
    bool beyond[2];    // beyond a y wall: ghost rule
    T fac[2];
};

template <typename T, int NC>
struct PlaneRegs {
    T v[2][NC];
    uint8_t m[2];
};

template <typename T>
__device__ __forceinline__ void tile_sources(const GridP& g, TileSrc<T>& S, int i0, int j0, T sig_lo, T sig_hi) {
    const int tid = threadIdx.x + TX * threadIdx.y;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int q = tid + t * TX * TY;
        S.valid[t] = q < HP;
        const int r = q % HX, s = q / HX;
        int i = i0 - 1 + r;
        if (i < 0) i += g.nx;
        while (i >= g.nx) i -= g.nx;
        int j = j0 - 1 + s;
        S.fac[t] = T(1);
        S.beyond[t] = false;
        if (j < 0) { j = 0; S.fac[t] = sig_lo; S.beyond[t] = true; }
        else if (j >= g.ny) { j = g.ny - 1; S.fac[t] = sig_hi; S.beyond[t] = true; }
        S.off[t] = i + g.nx * j;
    }
}

template <typename T, int NC>
__device__ __forceinline__ void fetch_plane(const MomF<T>& F, const TileSrc<T>& S, PlaneRegs<T, NC>& R, int pbase) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        if (S.valid[t]) {
            const int id = pbase + S.off[t];
            R.m[t] = __ldg(F.mask + id);
#pragma unroll
            for (int c = 0; c < NC; ++c) R.v[t][c] = __ldg(F.u[c] + id);
        }
    }
}

template <typename T, int NC>
__device__ __forceinline__ void store_plane(const TileSrc<T>& S, const PlaneRegs<T, NC>& R, T (*tile)[HP]) {
    const int tid = threadIdx.x + TX * threadIdx.y;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        if (S.valid[t]) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                T v = ((R.m[t] >> c) & 1u) ? R.v[t][c] : T(0);
                if (S.beyond[t]) v = (c == 1) ? T(0) : S.fac[t] * v;
                tile[c][tid + t * TX * TY] = v;
            }
        }
    }
}

// K3 kernel.  Four rotating plane slots let one barrier per plane suffice:
// the slot written for plane k+1 last held plane k-3, which no warp still
// computing plane k-1 reads.  Convection uses a^2 - b^2 = (a - b)(a + b) and
// all constant factors are folded into the StageP coefficients.
template <typename T, bool THREE>
__global__ void __launch_bounds__(TX * TY, sizeof(T) == 4 ? 4 : 3)
    k_momentum(GridP g, MomF<T> F, StageP<T> sp, IbmStage<T> ib, double* __restrict__ flux_part) {
    constexpr int NC = THREE ? 3 : 2;
    constexpr int NS = THREE ? 4 : 1;
    __shared__ T tile[NS][NC][HP];
    __shared__ double shd[TY];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int i = i0 + tx, j = j0 + ty;
    const int kbeg = THREE ? blockIdx.z * KZ : 0;
    const int kend = THREE ? min(kbeg + KZ, g.nz) : 1;
    const int c0 = (ty + 1) * HX + (tx + 1);       // own cell in a plane tile
    const int plane = g.nx * g.ny;
    const int rowbase = i + g.nx * j;
    const int dxp = (i + 1 < g.nx) ? 1 : 1 - g.nx;  // offset of the +x neighbour (periodic)
    const bool live_row = j < g.ny;
    const bool live = live_row && i < g.nx;
    T fsum = T(0);

    TileSrc<T> S;
    tile_sources<T>(g, S, i0, j0, sp.sig_lo, sp.sig_hi);
    PlaneRegs<T, NC> R;
    if (THREE) {
        fetch_plane<T, NC>(F, S, R, wrapi(kbeg - 1, g.nz) * plane);
        store_plane<T, NC>(S, R, tile[(kbeg - 1 - kbeg + 4) & 3]);
        fetch_plane<T, NC>(F, S, R, kbeg * plane);
        store_plane<T, NC>(S, R, tile[0]);
        fetch_plane<T, NC>(F, S, R, wrapi(kbeg + 1, g.nz) * plane);
    } else {
        fetch_plane<T, NC>(F, S, R, 0);
        store_plane<T, NC>(S, R, tile[0]);
    }
    for (int k = kbeg; k < kend; ++k) {
        const int rel = k - kbeg;
        const int s0 = THREE ? (rel & 3) : 0, sm = (rel + 3) & 3, spl = (rel + 1) & 3;
        if (THREE) {
            store_plane<T, NC>(S, R, tile[spl]);                                   // plane k+1
            if (k + 1 < kend) fetch_plane<T, NC>(F, S, R, wrapi(k + 2, g.nz) * plane);
        }
        __syncthreads();
        if (live_row) {
            const int id = rowbase + k * plane;
            const int seg = (j + g.ny * k) * g.nsegx + blockIdx.x;
            const uint8_t m = i < g.nx ? F.mask[id] : 0;
            int pos[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                unsigned b = __ballot_sync(0xffffffffu, (m >> (4 + c)) & 1u);
                pos[c] = __popc(b & lanemask_lt());
            }
            if (live) {
                const T* U0 = tile[s0][0];
                const T* V0 = tile[s0][1];
                const T pP = F.p[id];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    T out = T(0), Nv = T(0);
                    if ((m >> c) & 1u) {
                        T N, gp, uP;
                        if (c == 0) {
                            uP = U0[c0];
                            const T uE = U0[c0 + 1], uW = U0[c0 - 1], uN = U0[c0 + HX], uS = U0[c0 - HX];
                            const T sx = uE + uW, sy = uN + uS;
                            T conv = (uE - uW) * (sx + T(2) * uP) * sp.qx;
                            conv += ((V0[c0] + V0[c0 + 1]) * (uP + uN) - (V0[c0 - HX] + V0[c0 - HX + 1]) * (uS + uP)) * sp.qy;
                            T lap = (sx - T(2) * uP) * sp.nx2 + (sy - T(2) * uP) * sp.ny2;
                            if (THREE) {
                                const T* Um = tile[sm][0];
                                const T* Up = tile[spl][0];
                                const T* W0 = tile[s0][NC - 1];
                                const T* Wm = tile[sm][NC - 1];
                                const T uT = Up[c0], uB = Um[c0];
                                conv += ((W0[c0] + W0[c0 + 1]) * (uP + uT) - (Wm[c0] + Wm[c0 + 1]) * (uB + uP)) * sp.qz;
                                lap += (uT + uB - T(2) * uP) * sp.nz2;
                            }
                            N = lap - conv + sp.g[0];
                            gp = (F.p[id + dxp] - pP) * sp.idx;
                        } else if (c == 1) {
                            uP = V0[c0];
                            const T vE = V0[c0 + 1], vW = V0[c0 - 1], vN = V0[c0 + HX], vS = V0[c0 - HX];
                            const T sx = vE + vW, sy = vN + vS;
                            T conv = ((U0[c0] + U0[c0 + HX]) * (uP + vE) - (U0[c0 - 1] + U0[c0 - 1 + HX]) * (vW + uP)) * sp.qx;
                            conv += (vN - vS) * (sy + T(2) * uP) * sp.qy;
                            T lap = (sx - T(2) * uP) * sp.nx2 + (sy - T(2) * uP) * sp.ny2;
                            if (THREE) {
                                const T* Vm = tile[sm][1];
                                const T* Vp = tile[spl][1];
                                const T* W0 = tile[s0][NC - 1];
                                const T* Wm = tile[sm][NC - 1];
                                const T vT = Vp[c0], vB = Vm[c0];
                                conv += ((W0[c0] + W0[c0 + HX]) * (uP + vT) - (Wm[c0] + Wm[c0 + HX]) * (vB + uP)) * sp.qz;
                                lap += (vT + vB - T(2) * uP) * sp.nz2;
                            }
                            N = lap - conv + sp.g[1];
                            gp = (F.p[id + g.nx] - pP) * sp.idy;   // j < ny-1 for internal v
                        } else {
                            const T* W0 = tile[s0][NC - 1];
                            const T* Wm = tile[sm][NC - 1];
                            const T* Wp = tile[spl][NC - 1];
                            const T* Up = tile[spl][0];
                            const T* Vp = tile[spl][1];
                            uP = W0[c0];
                            const T wE = W0[c0 + 1], wW = W0[c0 - 1], wN = W0[c0 + HX], wS = W0[c0 - HX];
                            const T wT = Wp[c0], wB = Wm[c0];
                            const T sz = wT + wB;
                            T conv = ((U0[c0] + Up[c0]) * (uP + wE) - (U0[c0 - 1] + Up[c0 - 1]) * (wW + uP)) * sp.qx;
                            conv += ((V0[c0] + Vp[c0]) * (uP + wN) - (V0[c0 - HX] + Vp[c0 - HX]) * (wS + uP)) * sp.qy;
                            conv += (wT - wB) * (sz + T(2) * uP) * sp.qz;
                            const T lap = (wE + wW - T(2) * uP) * sp.nx2 + (wN + wS - T(2) * uP) * sp.ny2 +
                                          (sz - T(2) * uP) * sp.nz2;
                            N = lap - conv + sp.g[2];
                            const int dzp = (k + 1 < g.nz) ? plane : plane - (int)g.N;
                            gp = (F.p[id + dzp] - pP) * sp.idz;
                        }
                        const bool isibm = (m >> (4 + c)) & 1u;
                        Coef4<T> q;
                        if (isibm) {
                            q = ib.coef[c][ib.segoff[c][seg] + pos[c]];
                            N += q.s;
                        }
                        T R = sp.dta * N - sp.ckdt * gp;
                        if (sp.read_prev) R += sp.dtb * F.Nn[c][id];
                        out = isibm ? (q.a * uP + q.b * R) : (uP + R);
                        Nv = N;
                        if (c == 0) fsum += out;
                    }
                    F.us[c][id] = out;
                    if (sp.write_n) F.Nn[c][id] = Nv;
                }
            }
        }
        if (!THREE) break;
    }
    if (sp.flux_sum) {
        // FP32 sums within a warp, FP64 across warps and blocks
        T ws = warp_sum(fsum);
        if (tx == 0) shd[ty] = (double)ws;
        __syncthreads();
        if (tx == 0 && ty == 0) {
            double s = 0.0;
            for (int w = 0; w < TY; ++w) s += shd[w];
            flux_part[blockIdx.x + gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z)] = s;
        }
    }
}

// Pi = (Q_target - Q(u*)) / S_k  (one block, fixed summation order)
template <typename T>
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
        double pi = (target - q * dV) / S;
        scal[0] = pi;
        *reinterpret_cast<T*>(scal + 2) = (T)pi;   // typed copy read by k_flux_apply
    }
}

// u* += Pi c_k dt beta at internal u points (beta = 1, or the stage's IBM beta)
template <typename T>
__global__ void __launch_bounds__(256) k_flux_apply(GridP g, T* __restrict__ us, const uint8_t* __restrict__ mask,
                                                    IbmStage<T> ib, const double* __restrict__ scal, T ckdt) {
    const int i = blockIdx.x * IBM_WARP + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (j >= g.ny) return;                      // whole warp
    const long long row = j + (long long)g.ny * k;
    const long long id = i + (long long)g.nx * row;
    const uint8_t m = i < g.nx ? mask[id] : 0;
    const unsigned b = __ballot_sync(0xffffffffu, (m >> 4) & 1u);
    if (i >= g.nx || !(m & IBM_MASK_U)) return;
    T beta = T(1);
    if ((m >> 4) & 1u) beta = ib.coef[0][ib.segoff[0][row * g.nsegx + blockIdx.x] + __popc(b & lanemask_lt())].b;
    const T pi = *reinterpret_cast<const T*>(scal + 2);
    us[id] += pi * ckdt * beta;
}

// ---------------------------------------------------------------------------
// K4: divergence of the predictor, D u* (in the field precision)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_divergence(GridP g, const T* __restrict__ u, const T* __restrict__ v,
                                                    const T* __restrict__ w, T* __restrict__ rhs, T idx, T idy,
                                                    T idz) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const long long row = j + (long long)g.ny * k;
    const long long id = i + (long long)g.nx * row;
    T d = (u[id] - u[row * g.nx + wrapi(i - 1, g.nx)]) * idx;
    const T vm = j > 0 ? v[id - g.nx] : T(0);
    d += (v[id] - vm) * idy;
    if (g.ndim == 3) {
        const long long idB = i + (long long)g.nx * (j + (long long)g.ny * wrapi(k - 1, g.nz));
        d += (w[id] - w[idB]) * idz;
    }
    rhs[id] = d;
}

// ---------------------------------------------------------------------------
// K6: batched tridiagonal solve along y for every (kz, kx).
// After scaling by dy^2 the off-diagonals are 1 and the pivots w_j are
// precomputed (FP64):
//   forward  e_j = (d_j - e_{j-1}) w_j      (w_0 = 0 for the zero mode: phi_0 = 0)
//   backward x_j = e_j - w_j x_{j+1}
// and the solution is multiplied by `scale` (dy^2 and the FFT normalisation)
// on the way out.  The zero mode's solution is shifted to zero mean (box-mean
// gauge).  Each system runs in FP64 unless its flag says it is strongly
// diagonally dominant (K dy^2 >= tau, condition number <= 4/tau + 1), in which
// case FP32 arithmetic with FP32 pivots is as accurate as the FP32 transforms
// that feed it; that sweep works in place on the spectrum.
// One warp covers 32 consecutive kx of one kz, so loads coalesce across systems.
// ---------------------------------------------------------------------------
template <typename C>
__device__ __forceinline__ void tridiag_fp64(const GridP& g, C* spec, double2* tmp, const double* __restrict__ piv,
                                             long long base, double scale, bool zero_mode) {
    constexpr bool F32 = sizeof(C) == sizeof(float2);
    constexpr int B = 8;
    const long long st = g.nxh;
    const int ny = g.ny;
    // FP32 storage: the scale is applied to the FP32 input (exact to FP32
    // rounding, like the data); FP64 storage: applied in FP64 on output.
    const float sf = (float)scale;
    const double so = F32 ? 1.0 : scale;
    double2 e = make_double2(0.0, 0.0);
    for (int j0 = 0; j0 < ny; j0 += B) {
        C r[B];
        double w[B];
#pragma unroll
        for (int t = 0; t < B; ++t)
            if (j0 + t < ny) {
                r[t] = spec[base + (j0 + t) * st];
                w[t] = piv[base + (j0 + t) * st];
            }
#pragma unroll
        for (int t = 0; t < B; ++t)
            if (j0 + t < ny) {
                const double rx = F32 ? (double)((float)r[t].x * sf) : (double)r[t].x;
                const double ry = F32 ? (double)((float)r[t].y * sf) : (double)r[t].y;
                e = make_double2((rx - e.x) * w[t], (ry - e.y) * w[t]);    // e_{-1} = 0
                tmp[base + (j0 + t) * st] = e;
            }
    }
    double2 x = e;
    double sr = 0.0, si = 0.0;
    {
        C out;
        out.x = x.x * so;
        out.y = x.y * so;
        spec[base + (long long)(ny - 1) * st] = out;
        if (zero_mode) { sr += x.x; si += x.y; }
    }
    for (int j1 = ny - 2; j1 >= 0; j1 -= B) {
        double2 d[B];
        double w[B];
#pragma unroll
        for (int t = 0; t < B; ++t)
            if (j1 - t >= 0) {
                d[t] = tmp[base + (j1 - t) * st];
                w[t] = piv[base + (j1 - t) * st];
            }
#pragma unroll
        for (int t = 0; t < B; ++t)
            if (j1 - t >= 0) {
                x = make_double2(d[t].x - w[t] * x.x, d[t].y - w[t] * x.y);
                C out;
                out.x = x.x * so;
                out.y = x.y * so;
                spec[base + (j1 - t) * st] = out;
                if (zero_mode) { sr += x.x; si += x.y; }
            }
    }
    if (zero_mode) {
        const double mr = sr / ny * so, mi = si / ny * so;
        for (int j = 0; j < ny; ++j) {
            const long long o = base + j * st;
            C v = spec[o];
            v.x = (double)v.x - mr;
            v.y = (double)v.y - mi;
            spec[o] = v;
        }
    }
}

// FP32 sweep in place; loads are issued 16 rows ahead of the dependent chain
// so that enough bytes are in flight to cover HBM latency.
__device__ __forceinline__ void tridiag_fp32(const GridP& g, float2* spec, const float* __restrict__ piv,
                                             long long base, float scale) {
    constexpr int B = 16;
    const long long st = g.nxh;
    const int ny = g.ny;
    float2 e = make_float2(0.f, 0.f);
    for (int j0 = 0; j0 < ny; j0 += B) {
        float2 r[B];
        float w[B];
#pragma unroll
        for (int t = 0; t < B; ++t) {
            if (j0 + t < ny) {
                r[t] = spec[base + (j0 + t) * st];
                w[t] = piv[base + (j0 + t) * st];
            }
        }
#pragma unroll
        for (int t = 0; t < B; ++t) {
            if (j0 + t < ny) {
                e = make_float2((r[t].x - e.x) * w[t], (r[t].y - e.y) * w[t]);   // e_{-1} = 0
                spec[base + (j0 + t) * st] = e;
            }
        }
    }
    float2 x = e;
    spec[base + (long long)(ny - 1) * st] = make_float2(x.x * scale, x.y * scale);
    for (int j1 = ny - 2; j1 >= 0; j1 -= B) {
        float2 d[B];
        float w[B];
#pragma unroll
        for (int t = 0; t < B; ++t) {
            if (j1 - t >= 0) {
                d[t] = spec[base + (j1 - t) * st];
                w[t] = piv[base + (j1 - t) * st];
            }
        }
#pragma unroll
        for (int t = 0; t < B; ++t) {
            if (j1 - t >= 0) {
                x = make_float2(d[t].x - w[t] * x.x, d[t].y - w[t] * x.y);
                spec[base + (j1 - t) * st] = make_float2(x.x * scale, x.y * scale);
            }
        }
    }
}

// One warp per block; `order` lists the systems (kz * nxh + kx) with every
// FP64 system first, so the scarce FP64 pipes of all SMs share the low modes.
template <typename C>
__global__ void __launch_bounds__(32) k_tridiag(GridP g, C* spec, double2* tmp, const double* __restrict__ piv,
                                                const float* __restrict__ piv32, const int* __restrict__ order,
                                                int n64, int nsys, double scale) {
    const int nb64 = (n64 + 31) / 32;
    int q;
    bool fp64;
    if ((int)blockIdx.x < nb64) {
        q = blockIdx.x * 32 + threadIdx.x;
        if (q >= n64) return;
        fp64 = true;
    } else {
        q = n64 + (blockIdx.x - nb64) * 32 + threadIdx.x;
        if (q >= nsys) return;
        fp64 = false;
    }
    const int sys = order[q];
    const int kx = sys % g.nxh;
    const int kz = sys / g.nxh;
    const long long base = (long long)kz * g.ny * g.nxh + kx;
    if constexpr (sizeof(C) == sizeof(float2)) {
        if (!fp64) {
            tridiag_fp32(g, reinterpret_cast<float2*>(spec), piv32, base, (float)scale);
            return;
        }
    }
    tridiag_fp64<C>(g, spec, tmp, piv, base, scale, kx == 0 && kz == 0);
}

// ---------------------------------------------------------------------------
// K7: u = u* - G psi on every non-wall face, p += psi / (c_k dt)
// (psi = c_k dt phi is what the Poisson solve returns for rhs = D u*)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_correct(GridP g, const T* __restrict__ us0, const T* __restrict__ us1,
                                                 const T* __restrict__ us2, const T* __restrict__ psi,
                                                 T* __restrict__ u0, T* __restrict__ u1, T* __restrict__ u2,
                                                 T* __restrict__ p, T idx, T idy, T idz, T inv_ckdt,
                                                 int update_p) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const long long row = j + (long long)g.ny * k;
    const long long id = i + (long long)g.nx * row;
    T ph = psi[id];
    u0[id] = us0[id] - (psi[row * g.nx + wrapi(i + 1, g.nx)] - ph) * idx;
    u1[id] = j < g.ny - 1 ? us1[id] - (psi[id + g.nx] - ph) * idy : us1[id];
    if (g.ndim == 3) {
        long long idT = i + (long long)g.nx * (j + (long long)g.ny * wrapi(k + 1, g.nz));
        u2[id] = us2[id] - (psi[idT] - ph) * idz;
    }
    if (update_p) p[id] += ph * inv_ckdt;
}

// initial-condition projection: copy the velocity with non-internal points zeroed
template <typename T>
__global__ void k_mask_copy(GridP g, const uint8_t* __restrict__ mask, const T* __restrict__ a0,
                            const T* __restrict__ a1, const T* __restrict__ a2, T* __restrict__ b0,
                            T* __restrict__ b1, T* __restrict__ b2) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const long long id = i + (long long)g.nx * (j + (long long)g.ny * blockIdx.z);
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

// 32 x 8 cells per block, one z plane per blockIdx.z
dim3 cell_grid(const GridP& g) { return dim3(g.nsegx, (g.ny + 7) / 8, g.nz); }
const double RK_A[3] = {64.0 / 120.0, 50.0 / 120.0, 90.0 / 120.0};
const double RK_B[3] = {0.0, -34.0 / 120.0, -50.0 / 120.0};
const double RK_C[3] = {64.0 / 120.0, 16.0 / 120.0, 40.0 / 120.0};


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
    double scale = g.dy * g.dy / ((double)g.nx * (double)g.nz);
    const int nsys = g.nz * g.nxh;
    const int nblk = (h->n64 + 31) / 32 + (nsys - h->n64 + 31) / 32;
    timer_begin(h, "tridiag", &t);
    if (h->prec == IBM_FP64)
        k_tridiag<double2><<<nblk, 32, 0, h->stream>>>(g, (double2*)h->spec, (double2*)h->spec, h->pivots,
                                                       h->pivots32, h->sys_order, h->n64, nsys, scale);
    else
        k_tridiag<float2><<<nblk, 32, 0, h->stream>>>(g, (float2*)h->spec, (double2*)h->dtemp, h->pivots,
                                                      h->pivots32, h->sys_order, h->n64, nsys, scale);
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
    cudaEvent_t t;
    timer_begin(h, "divergence", &t);
    k_divergence<T><<<cell_grid(g), dim3(32, 8), 0, h->stream>>>(g, us[0], us[1], us[2], (T*)h->rhs, (T)(1.0 / g.dx),
                                                (T)(1.0 / g.dy), (T)(1.0 / g.dz));
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
    sp.nx2 = (T)(h->phys.nu / (g.dx * g.dx)); sp.ny2 = (T)(h->phys.nu / (g.dy * g.dy));
    sp.nz2 = (T)(h->phys.nu / (g.dz * g.dz));
    sp.qx = (T)(0.25 / g.dx); sp.qy = (T)(0.25 / g.dy); sp.qz = (T)(0.25 / g.dz);
    sp.sig_lo = (T)g.sig_lo;
    sp.sig_hi = (T)g.sig_hi;
    sp.read_prev = k > 0;
    sp.write_n = k < 2;
    bool cflux = h->phys.flow_mode == IBM_FLOW_CONST_FLUX;
    sp.flux_sum = cflux;
    IbmStage<T> ib;
    for (int c = 0; c < 3; ++c) {
        ib.segoff[c] = h->segoff[c];
        ib.coef[c] = (const Coef4<T>*)h->coef[c] + (long long)k * h->counts[c];
    }
    dim3 blk(TX, TY, 1);
    dim3 grd = momentum_grid(g);
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
        k_flux_pi<T><<<1, 1024, 0, h->stream>>>(h->partials, nparts, dV, h->phys.target_flux, h->S[k], h->scal);
        IBM_LAUNCH_CHECK();
        dim3 fgrd(g.nsegx, (g.ny + 7) / 8, g.nz);
        k_flux_apply<T><<<fgrd, dim3(32, 8, 1), 0, h->stream>>>(g, (T*)h->ustar[0], h->mask, ib, h->scal, sp.ckdt);
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
    timer_begin(h, "correct", &t);
    k_correct<T><<<cell_grid(g), dim3(32, 8), 0, h->stream>>>(g, us[0], us[1], us[2], (const T*)h->rhs, (T*)h->buf.u[0],
                                            (T*)h->buf.u[1], g.ndim == 3 ? (T*)h->buf.u[2] : (T*)h->buf.u[0],
                                            (T*)h->buf.p, (T)(1.0 / g.dx), (T)(1.0 / g.dy), (T)(1.0 / g.dz),
                                            (T)(1.0 / (dt * RK_C[k])), 1);
    IBM_LAUNCH_CHECK();
    timer_end(h, t, "correct");
    return IBM_OK;
}

template <typename T>
ibm_status project_t(ibm_solver* h) {
    const GridP& g = h->gp;
    T* us[3] = {(T*)h->ustar[0], (T*)h->ustar[1], g.ndim == 3 ? (T*)h->ustar[2] : (T*)h->ustar[0]};
    const T* u2 = g.ndim == 3 ? (const T*)h->buf.u[2] : (const T*)h->buf.u[0];
    k_mask_copy<T><<<cell_grid(g), dim3(32, 8), 0, h->stream>>>(g, h->mask, (const T*)h->buf.u[0], (const T*)h->buf.u[1], u2, us[0],
                                              us[1], us[2]);
    IBM_LAUNCH_CHECK();
    ibm_status st = divergence_and_solve<T>(h, us);
    if (st != IBM_OK) return st;
    k_correct<T><<<cell_grid(g), dim3(32, 8), 0, h->stream>>>(g, us[0], us[1], us[2], (const T*)h->rhs,
                                                               (T*)h->buf.u[0], (T*)h->buf.u[1],
                                                               g.ndim == 3 ? (T*)h->buf.u[2] : (T*)h->buf.u[0],
                                                               (T*)h->buf.p, (T)(1.0 / g.dx), (T)(1.0 / g.dy),
                                                               (T)(1.0 / g.dz), (T)1, 0);
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
