// Hot-path kernels of one RK3 substage:
//   momentum predictor with the fused implicit IBM division   (Sec. 2.4, Eq. rk3-rai)
//   constant-flow-rate forcing                                 (reading: uniform forcing)
//   divergence                                                 (Sec. 2.1 projection)
//   FFT (cuFFT) + batched FP64 tridiagonal Poisson solve + inverse FFT
//   gradient correction and pressure update
// plus the diagnostics reductions.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <type_traits>


namespace {

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
        *reinterpret_cast<T*>(scal + 2) = (T)pi;   // typed copy read by the flux corrections
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
// Constant-flow-rate correction Pi c_k dt beta of an internal u point, applied
// on the fly by the divergence and correction kernels (so the corrected u* is
// never written): beta = 1 at a regular internal point, the stage's IBM beta
// at an IBM point, and the point is skipped when not internal.
// ---------------------------------------------------------------------------
template <typename T>
struct FluxCorr {
    const double* scal;    // the typed Pi sits at scal + 2
    T ckdt;
    const int* segoff;     // u component
    const Coef4<T>* coef;  // u component, this stage
};

template <typename T>
__device__ __forceinline__ T flux_increment(const FluxCorr<T>& fc, T pic, uint8_t m, unsigned ibm_ballot, int seg,
                                            int lane) {
    if (!(m & IBM_MASK_U)) return T(0);
    T beta = T(1);
    if (m & IBM_MASK_IBM_U) beta = fc.coef[fc.segoff[seg] + __popc(ibm_ballot & ((1u << lane) - 1u))].b;
    return pic * beta;
}

// ---------------------------------------------------------------------------
// K4: divergence of the predictor, D u*, in the field precision.  Each block
// marches g.kzd planes along z carrying w*(k-1) in a register; u*(i-1) comes
// from the neighbouring lane.  A thread issues the loads of DZ_DIV planes before
// it uses any of them, so several planes' bytes are in flight per warp.
// ---------------------------------------------------------------------------
constexpr int DZ = 4;        // correction: planes whose loads go out together
constexpr int DZ_DIV = 3;    // divergence: measured best of 1-4 (0.110 ms against 0.121 at 4 on 384x256x256)

template <typename T, bool THREE, bool FLUX, bool XF>
__global__ void __launch_bounds__(256) k_divergence(GridP g, const T* __restrict__ u, const T* __restrict__ v,
                                                    const T* __restrict__ w, const uint8_t* __restrict__ mask,
                                                    T* __restrict__ rhs, T idx, T idy, T idz, FluxCorr<T> fc) {
    constexpr int ZB = THREE ? DZ_DIV : 1;
    const int lane = threadIdx.x;
    const int i = blockIdx.x * 32 + lane;
    const int j = blockIdx.y * 8 + threadIdx.y;
    if (j >= g.ny) return;                                   // whole warp
    const int kbeg = THREE ? blockIdx.z * g.kzd : 0;
    const int kend = THREE ? min(kbeg + g.kzd, g.nz) : 1;
    const bool live = i < g.nx;
    const int plane = g.nx * g.ny;
    // left neighbour of lane 0 (periodic in x) and its place in its 32-point segment
    const int il = wrapi((int)blockIdx.x * 32 - 1, g.nx);
    const int segl = il / 32, lanel = il % 32;
    const int il_probe = segl * 32 + lane;                  // the warp reads that segment's mask bits
    const T pic = FLUX ? *reinterpret_cast<const T*>(fc.scal + 2) * fc.ckdt : T(0);
    if (g.ystr) idy = (T)ytab(g, YT_IDYC, j);                // a stretched y: this row's cell height
    // the first segment of an inflow/outflow x: lane 0 (cell 0) reads the inflow face
    const bool inflow_seg = XF && blockIdx.x == 0;
    T wprev = T(0);
    if (THREE && live) wprev = w[i + g.nx * j + plane * wrapi(kbeg - 1, g.nz)];
    for (int k0 = kbeg; k0 < kend; k0 += ZB) {
        T uc[ZB], ul0[ZB], vc[ZB], vm[ZB], wc[ZB];
        uint8_t mc[ZB], ml[ZB];
#pragma unroll
        for (int t = 0; t < ZB; ++t) {
            uc[t] = ul0[t] = vc[t] = vm[t] = wc[t] = T(0);
            mc[t] = ml[t] = 0;
            const int k = k0 + t;
            if (k < kend) {
                const int rowb = g.nx * (j + g.ny * k);
                const int id = rowb + i;
                ul0[t] = u[rowb + il];
                if (live) {
                    uc[t] = u[id];
                    vc[t] = v[id];
                    if (j > 0) vm[t] = v[id - g.nx];
                    if (THREE) wc[t] = w[id];
                    if (FLUX || inflow_seg) mc[t] = mask[id];
                }
                if (FLUX && il_probe < g.nx) ml[t] = mask[rowb + il_probe];
            }
        }
#pragma unroll
        for (int t = 0; t < ZB; ++t) {
            const int k = k0 + t;
            if (k >= kend) break;
            const int rowb = g.nx * (j + g.ny * k);
            T ucc = uc[t], ulane0 = ul0[t];
            if (FLUX) {
                const int rowseg = (j + g.ny * k) * g.nsegx;
                const unsigned b = __ballot_sync(0xffffffffu, (mc[t] & IBM_MASK_IBM_U) != 0);
                if (live) ucc += flux_increment(fc, pic, mc[t], b, rowseg + (int)blockIdx.x, lane);
                const unsigned bl = __ballot_sync(0xffffffffu, (ml[t] & IBM_MASK_IBM_U) != 0);
                const uint8_t mln = __shfl_sync(0xffffffffu, ml[t], lanel);
                ulane0 += flux_increment(fc, pic, mln, bl, rowseg + segl, lanel);
            }
            T ul = __shfl_up_sync(0xffffffffu, ucc, 1);
            if (lane == 0) ul = inflow_seg ? ((mc[t] & IBM_MASK_FACE) ? (T)g.uin : T(0)) : ulane0;   // inflow face
            if (live) {
                T d = (ucc - ul) * idx;
                d += (vc[t] - vm[t]) * idy;
                if (THREE) {
                    d += (wc[t] - wprev) * idz;
                    wprev = wc[t];
                }
                rhs[rowb + i] = d;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// K6: batched tridiagonal solve along y for every (kz, kx).
// After scaling by dy^2 the off-diagonals are 1 and the pivots w_j are
// precomputed (FP64):
//   forward  e_j = (d_j - e_{j-1}) w_j      (w_0 = 0 for the zero mode: phi_0 = 0)
//   backward x_j = e_j - w_j x_{j+1}
// and the solution is multiplied by `scale` (dy^2 and the FFT normalisation)
// on the way out.  The zero mode's solution is shifted to zero mean (box-mean
// gauge).  Each system sweeps in FP64 arithmetic unless its flag says it is
// strongly diagonally dominant (K dy^2 >= tau, condition number <= 4/tau + 1):
// in FP32 mode those sweep in FP32 with FP32 pivots, as accurate as the FP32
// transforms that feed them, in place on the spectrum.
// ---------------------------------------------------------------------------
// FP64 sweep of one complex system by one thread (real and imaginary parts are
// two independent chains).  The forward recurrence runs divide-free on
// f_j = e_j / w_j:  f_j = d_j - w_{j-1} f_{j-1}, one fused multiply-add on the
// dependent chain, and e_j = w_j f_j goes to the FP64 temporary `tmp` (the
// spectrum itself for FP64 storage: row j is read before it is overwritten).
// The backward sweep is one fused multiply-add per row.  This is the least FP64
// work per system (the scarce FP64 pipes bound it when there are many systems);
// the warp form below has the shorter chain for few systems.  Loads run B rows
// ahead of the chain.
template <typename C>
__device__ __forceinline__ void tridiag_thread64(const GridP& g, C* spec, double2* tmp, const double* __restrict__ piv,
                                                 long long base, double scale, bool zero_mode) {
    constexpr bool F32 = sizeof(C) == sizeof(float2);
    using S = typename std::conditional<F32, float, double>::type;   // storage scalar
    constexpr int B = 8;
    const long long st = g.nxh;
    const int ny = g.ny;
    const float sf = (float)scale;
    C r[B], rn[B];
    double w[B], wn[B];
#pragma unroll
    for (int t = 0; t < B; ++t)
        if (t < ny) {
            r[t] = spec[base + t * st];
            w[t] = piv[base + t * st];
        }
    double fr = 0.0, fi = 0.0, wp = 0.0;      // f_{j-1}, w_{j-1}
    for (int j0 = 0; j0 < ny; j0 += B) {
#pragma unroll
        for (int t = 0; t < B; ++t)
            if (j0 + B + t < ny) {
                rn[t] = spec[base + (j0 + B + t) * st];
                wn[t] = piv[base + (j0 + B + t) * st];
            }
#pragma unroll
        for (int t = 0; t < B; ++t)
            if (j0 + t < ny) {
                // FP32 storage: the scale is applied in FP32 on the input (exact to FP32 rounding)
                const double dr = F32 ? (double)((float)r[t].x * sf) : (double)r[t].x;
                const double di = F32 ? (double)((float)r[t].y * sf) : (double)r[t].y;
                fr = fma(-wp, fr, dr);
                fi = fma(-wp, fi, di);
                wp = w[t];
                tmp[base + (j0 + t) * st] = make_double2(wp * fr, wp * fi);
            }
#pragma unroll
        for (int t = 0; t < B; ++t) { r[t] = rn[t]; w[t] = wn[t]; }
    }
    double2 e[B], en[B];
#pragma unroll
    for (int t = 0; t < B; ++t)
        if (ny - 1 - t >= 0) {
            e[t] = tmp[base + (ny - 1 - t) * st];
            w[t] = piv[base + (ny - 1 - t) * st];
        }
    double xr = 0.0, xi = 0.0, sr = 0.0, si = 0.0;    // x_{ny} = 0
    for (int j1 = ny - 1; j1 >= 0; j1 -= B) {
#pragma unroll
        for (int t = 0; t < B; ++t)
            if (j1 - B - t >= 0) {
                en[t] = tmp[base + (j1 - B - t) * st];
                wn[t] = piv[base + (j1 - B - t) * st];
            }
#pragma unroll
        for (int t = 0; t < B; ++t)
            if (j1 - t >= 0) {
                xr = fma(-w[t], xr, e[t].x);
                xi = fma(-w[t], xi, e[t].y);
                C o;
                o.x = (S)(F32 ? xr : xr * scale);
                o.y = (S)(F32 ? xi : xi * scale);
                spec[base + (j1 - t) * st] = o;
                sr += xr;
                si += xi;
            }
#pragma unroll
        for (int t = 0; t < B; ++t) { e[t] = en[t]; w[t] = wn[t]; }
    }
    if (zero_mode) {                                  // box-mean gauge
        const double mr = sr / ny * (F32 ? 1.0 : scale);
        const double mi = si / ny * (F32 ? 1.0 : scale);
        for (int j = 0; j < ny; ++j) {
            const long long o = base + j * st;
            C v = spec[o];
            v.x = (S)((double)v.x - mr);
            v.y = (S)((double)v.y - mi);
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

// Exact FP32 -> FP64 from the IEEE-754 bit layouts, on the integer pipes (the FP64 pipes
// are the scarce resource of the FP64 sweeps): the sign, the exponent rebiased from 127 to
// 1023 and the 23 mantissa bits at the top of the 52-bit field.  Zero keeps its sign;
// subnormal, infinite and NaN inputs take the hardware conversion.
__device__ __forceinline__ double f32_to_f64(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e == 0u && (b & 0x7fffffu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
    if (e == 0u || e == 0xffu) return (double)f;
    const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
}

// FP64 -> FP32 rounded to nearest, ties to even, from the bit layouts on the integer pipes:
// the top 23 mantissa bits are kept and the 29 dropped bits decide the rounding; a carry
// runs into the exponent (and past the largest finite value to infinity, as the rounding
// requires).  Results that would be subnormal or zero, and infinite or NaN inputs, take
// the hardware conversion.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t E = (hi >> 20) & 0x7ffu;
    if (E <= 896u || E >= 1151u) return __double2float_rn(x);
    uint32_t v = ((E - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const uint32_t rem = lo & 0x1fffffffu;
    v += (rem > 0x10000000u || (rem == 0x10000000u && (v & 1u))) ? 1u : 0u;
    return __uint_as_float((hi & 0x80000000u) | v);
}

// FP64 sweep of one system by a whole warp (ny <= 32 * TW_ROWS rows per lane).  The
// forward recurrence runs divide-free on f_j = e_j / w_j:
//   f_j = d_j - w_{j-1} f_{j-1}      (w_{-1} = 0),   e_j = w_j f_j,
// and the backward one is x_j = e_j - w_j x_{j+1} (x_{ny} = 0).  Both are first order and
// affine, so each lane composes the maps of its run of consecutive rows (one fused
// multiply-add per row and part), a five-step shuffle scan composes them across the lanes
// (affine maps compose like the recurrence itself), and each lane replays its rows from the
// value handed in.  The dependent FP64 chain is about 2 (rows per lane + 5) long instead of
// 2 ny.  Real and imaginary parts go through together.  FP32 storage converts on the
// integer pipes (f32_to_f64, f64_to_f32_rn), which leaves the FP64 pipes to the sweeps.
constexpr int TW_ROWS = 32;   // rows per lane at most: the warp path covers ny <= 1024

template <typename C, int TW_ROWS>
__device__ __forceinline__ void tridiag_warp64(const GridP& g, C* spec, const double* __restrict__ piv,
                                               long long base, double scale, bool zero_mode) {
    constexpr bool F32 = sizeof(C) == sizeof(float2);
    using S = typename std::conditional<F32, float, double>::type;
    const int lane = threadIdx.x & 31;
    const int ny = g.ny;
    const int E = (ny + 31) / 32;
    const int j0 = lane * E;
    const long long st = g.nxh;
    const float sf = (float)scale;
    double dr[TW_ROWS], di[TW_ROWS], w[TW_ROWS];
    // w_{j0-1}: the last pivot of the lane below (0 below row 0), read directly (selecting it
    // from the lane below's registers by a run-time row count would force the array into
    // local memory)
    const double wb = (lane > 0 && j0 - 1 < ny) ? piv[base + (long long)(j0 - 1) * st] : 0.0;
#pragma unroll
    for (int t = 0; t < TW_ROWS; ++t) {
        dr[t] = di[t] = w[t] = 0.0;
        if (t < E && j0 + t < ny) {
            const long long o = base + (long long)(j0 + t) * st;
            const C r = spec[o];
            // FP32 storage: the scale is applied in FP32 on the input (exact to FP32 rounding)
            if constexpr (F32) {
                dr[t] = f32_to_f64((float)r.x * sf);
                di[t] = f32_to_f64((float)r.y * sf);
            } else {
                dr[t] = (double)r.x;
                di[t] = (double)r.y;
            }
            w[t] = piv[o];
        }
    }
    // forward: this lane's map f_out = A + B f_in
    double Ar = 0.0, Ai = 0.0, B = 1.0;
    {
        double wp = wb;
#pragma unroll
        for (int t = 0; t < TW_ROWS; ++t)
            if (t < E && j0 + t < ny) {
                Ar = fma(-wp, Ar, dr[t]);
                Ai = fma(-wp, Ai, di[t]);
                B = -wp * B;
                wp = w[t];
            }
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {          // inclusive scan: compose with the lanes below
        const double pr = __shfl_up_sync(0xffffffffu, Ar, off);
        const double pi = __shfl_up_sync(0xffffffffu, Ai, off);
        const double pb = __shfl_up_sync(0xffffffffu, B, off);
        if (lane >= off) {
            Ar = fma(B, pr, Ar);
            Ai = fma(B, pi, Ai);
            B *= pb;
        }
    }
    double fr = __shfl_up_sync(0xffffffffu, Ar, 1), fi = __shfl_up_sync(0xffffffffu, Ai, 1);
    if (lane == 0) fr = fi = 0.0;
    {
        double wp = wb;
#pragma unroll
        for (int t = 0; t < TW_ROWS; ++t)
            if (t < E && j0 + t < ny) {
                fr = fma(-wp, fr, dr[t]);
                fi = fma(-wp, fi, di[t]);
                wp = w[t];
                dr[t] = wp * fr;                       // e_j
                di[t] = wp * fi;
            }
    }
    // backward: this lane's map x_first = Cm + D x_in, x_in the value above the run
    double Cr = 0.0, Ci = 0.0, D = 1.0;
#pragma unroll
    for (int t = TW_ROWS - 1; t >= 0; --t)
        if (t < E && j0 + t < ny) {
            Cr = fma(-w[t], Cr, dr[t]);
            Ci = fma(-w[t], Ci, di[t]);
            D = -w[t] * D;
        }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {          // compose with the lanes above
        const double pr = __shfl_down_sync(0xffffffffu, Cr, off);
        const double pi = __shfl_down_sync(0xffffffffu, Ci, off);
        const double pd = __shfl_down_sync(0xffffffffu, D, off);
        if (lane + off < 32) {
            Cr = fma(D, pr, Cr);
            Ci = fma(D, pi, Ci);
            D *= pd;
        }
    }
    double xr = __shfl_down_sync(0xffffffffu, Cr, 1), xi = __shfl_down_sync(0xffffffffu, Ci, 1);
    if (lane == 31) xr = xi = 0.0;
#pragma unroll
    for (int t = TW_ROWS - 1; t >= 0; --t)
        if (t < E && j0 + t < ny) {
            xr = fma(-w[t], xr, dr[t]);
            xi = fma(-w[t], xi, di[t]);
            dr[t] = xr;
            di[t] = xi;
        }
    if (zero_mode) {                                   // box-mean gauge (one system: the sums run only here)
        double sr = 0.0, si = 0.0;
#pragma unroll
        for (int t = 0; t < TW_ROWS; ++t)
            if (t < E && j0 + t < ny) {
                sr += dr[t];
                si += di[t];
            }
        sr = warp_sum(sr);
        si = warp_sum(si);
        const double mr = __shfl_sync(0xffffffffu, sr, 0) / ny;
        const double mi = __shfl_sync(0xffffffffu, si, 0) / ny;
#pragma unroll
        for (int t = 0; t < TW_ROWS; ++t) {
            dr[t] -= mr;
            di[t] -= mi;
        }
    }
#pragma unroll
    for (int t = 0; t < TW_ROWS; ++t)
        if (t < E && j0 + t < ny) {
            const long long o = base + (long long)(j0 + t) * st;
            C r;
            if constexpr (F32) {
                r.x = f64_to_f32_rn(dr[t]);
                r.y = f64_to_f32_rn(di[t]);
            } else {
                r.x = (S)(dr[t] * scale);
                r.y = (S)(di[t] * scale);
            }
            spec[o] = r;
        }
}

// The warp sweep of one strongly dominant FP32 system in FP32 (FP32 pivots, the
// scale applied on the way out as the thread-per-system sweep does).  Used when
// there are too few systems for one thread each to fill the GPU (the 2D cylinder:
// 1024 such systems of 768 rows, one dependent chain per thread).
template <int TW_ROWS>
__device__ __forceinline__ void tridiag_warp_f32(const GridP& g, float2* spec, const float* __restrict__ piv,
                                                 long long base, float scale) {
    const int lane = threadIdx.x & 31;
    const int ny = g.ny;
    const int E = (ny + 31) / 32;
    const int j0 = lane * E;
    const long long st = g.nxh;
    float dr[TW_ROWS], di[TW_ROWS], w[TW_ROWS];
#pragma unroll
    for (int t = 0; t < TW_ROWS; ++t) {
        dr[t] = di[t] = w[t] = 0.f;
        if (t < E && j0 + t < ny) {
            const long long o = base + (long long)(j0 + t) * st;
            const float2 r = spec[o];
            dr[t] = r.x;
            di[t] = r.y;
            w[t] = piv[o];
        }
    }
    float Ar = 0.f, Ai = 0.f, B = 1.f;
#pragma unroll
    for (int t = 0; t < TW_ROWS; ++t)
        if (t < E && j0 + t < ny) {
            Ar = (dr[t] - Ar) * w[t];
            Ai = (di[t] - Ai) * w[t];
            B = -w[t] * B;
        }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const float pr = __shfl_up_sync(0xffffffffu, Ar, off);
        const float pi = __shfl_up_sync(0xffffffffu, Ai, off);
        const float pb = __shfl_up_sync(0xffffffffu, B, off);
        if (lane >= off) {
            Ar += B * pr;
            Ai += B * pi;
            B *= pb;
        }
    }
    float er = __shfl_up_sync(0xffffffffu, Ar, 1), ei = __shfl_up_sync(0xffffffffu, Ai, 1);
    if (lane == 0) er = ei = 0.f;
#pragma unroll
    for (int t = 0; t < TW_ROWS; ++t)
        if (t < E && j0 + t < ny) {
            er = (dr[t] - er) * w[t];
            ei = (di[t] - ei) * w[t];
            dr[t] = er;
            di[t] = ei;
        }
    float Cr = 0.f, Ci = 0.f, D = 1.f;
#pragma unroll
    for (int t = TW_ROWS - 1; t >= 0; --t)
        if (t < E && j0 + t < ny) {
            Cr = dr[t] - w[t] * Cr;
            Ci = di[t] - w[t] * Ci;
            D = -w[t] * D;
        }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const float pr = __shfl_down_sync(0xffffffffu, Cr, off);
        const float pi = __shfl_down_sync(0xffffffffu, Ci, off);
        const float pd = __shfl_down_sync(0xffffffffu, D, off);
        if (lane + off < 32) {
            Cr += D * pr;
            Ci += D * pi;
            D *= pd;
        }
    }
    float xr = __shfl_down_sync(0xffffffffu, Cr, 1), xi = __shfl_down_sync(0xffffffffu, Ci, 1);
    if (lane == 31) xr = xi = 0.f;
#pragma unroll
    for (int t = TW_ROWS - 1; t >= 0; --t)
        if (t < E && j0 + t < ny) {
            xr = dr[t] - w[t] * xr;
            xi = di[t] - w[t] * xi;
            spec[base + (long long)(j0 + t) * st] = make_float2(xr * scale, xi * scale);
        }
}

// Stretched y: every spectral point of row j times the per-row factor ytab(tab, j)
template <typename C>
__global__ void k_spec_rows(GridP g, C* __restrict__ spec, long long n, int tab) {
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int j = (int)((id / g.nxh) % g.ny);
    using S = decltype(spec[0].x);
    const S f = (S)ytab(g, tab, j);
    C v = spec[id];
    v.x *= f;
    v.y *= f;
    spec[id] = v;
}

// Stretched y: the zero mode (kx = kz = 0) shifted to zero plain mean over the rows (FP64 sums)
template <typename C>
__global__ void k_zero_gauge(GridP g, C* __restrict__ spec) {
    __shared__ double sh[2][8];
    __shared__ double mean[2];
    double sr = 0.0, si = 0.0;
    for (int j = threadIdx.x; j < g.ny; j += blockDim.x) {
        const C v = spec[(long long)j * g.nxh];
        sr += (double)v.x;
        si += (double)v.y;
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = sr; sh[1][threadIdx.x >> 5] = si; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += sh[0][w]; b += sh[1][w]; }
        mean[0] = a / g.ny;
        mean[1] = b / g.ny;
    }
    __syncthreads();
    using S = decltype(spec[0].x);
    for (int j = threadIdx.x; j < g.ny; j += blockDim.x) {
        C v = spec[(long long)j * g.nxh];
        v.x = (S)((double)v.x - mean[0]);
        v.y = (S)((double)v.y - mean[1]);
        spec[(long long)j * g.nxh] = v;
    }
}

// One warp per block; `order` lists the systems (kz * nxh + kx) with every
// FP64 system first, so the scarce FP64 pipes of all SMs share the low modes.
// FP64 systems take one warp each (thr64 = 0; R rows per lane, ny <= 32 R) or one
// thread each (thr64 = 1, or R = 0 when ny > 32 * TW_ROWS); FP32 systems one
// thread each, or one warp each when warp32 is set.
template <typename C, int R>
__global__ void __launch_bounds__(32) k_tridiag(GridP g, C* spec, double2* tmp, const double* __restrict__ piv,
                                                const float* __restrict__ piv32, const int* __restrict__ order,
                                                int n64, int nsys, double scale, int warp32, int thr64, int gauge) {
    const bool warp64 = R > 0 && !thr64;
    const int nb64 = warp64 ? n64 : (n64 + 31) / 32;
    if ((int)blockIdx.x < nb64) {
        if constexpr (R > 0) {
            if (warp64) {                          // one warp (block) per FP64 system
                const int sys = order[blockIdx.x];
                const int kx = sys % g.nxh, kz = sys / g.nxh;
                const long long base = (long long)kz * g.ny * g.nxh + kx;
                tridiag_warp64<C, R>(g, spec, piv, base, scale, gauge && kx == 0 && kz == 0);
                return;
            }
        }
        const int t = blockIdx.x * 32 + threadIdx.x;
        if (t >= n64) return;
        const int sys = order[t];
        const int kx = sys % g.nxh, kz = sys / g.nxh;
        const long long base = (long long)kz * g.ny * g.nxh + kx;
        tridiag_thread64<C>(g, spec, tmp, piv, base, scale, gauge && kx == 0 && kz == 0);
        return;
    }
    if constexpr (sizeof(C) == sizeof(float2)) {
        if constexpr (R > 0) {
            if (warp32) {                          // one warp per FP32 system
                const int sys = order[n64 + (blockIdx.x - nb64)];
                const int kx = sys % g.nxh, kz = sys / g.nxh;
                tridiag_warp_f32<R>(g, reinterpret_cast<float2*>(spec), piv32,
                                    (long long)kz * g.ny * g.nxh + kx, (float)scale);
                return;
            }
        }
        const int q = n64 + (blockIdx.x - nb64) * 32 + threadIdx.x;
        if (q >= nsys) return;
        const int sys = order[q];
        const int kx = sys % g.nxh, kz = sys / g.nxh;
        const long long base = (long long)kz * g.ny * g.nxh + kx;
        tridiag_fp32(g, reinterpret_cast<float2*>(spec), piv32, base, (float)scale);
    }
}

// The FP32 systems of the FP32 mode in a launch of their own (one thread each, blocks of 128,
// held to 80 registers), beside the FP64 systems' launch on a second stream: in one launch they
// ran at the register count of the FP64 warp scans (136 a thread, twelve warps per SM), and the
// FP64 scans, bound by the FP64 pipe, and these sweeps, bound by memory latency, now overlap.
// 0.141 -> 0.113 ms per solve on 384x256x256, 0.308 -> 0.246 ms on 512x384x256 (one after the
// other instead: 0.168-0.191 and 0.289-0.324 ms; 64 registers instead of 80: 0.251 ms).
__global__ void __launch_bounds__(128, 6) k_tridiag32(GridP g, float2* spec, const float* __restrict__ piv32,
                                                   const int* __restrict__ order, int n64, int nsys, double scale) {
    const int q = n64 + blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nsys) return;
    const int sys = order[q];
    const int kx = sys % g.nxh, kz = sys / g.nxh;
    tridiag_fp32(g, spec, piv32, (long long)kz * g.ny * g.nxh + kx, (float)scale);
}

// ---------------------------------------------------------------------------
// K7: u = u* (+ flux correction) - G psi on every non-wall face, p += psi/(c_k dt)
// (psi = c_k dt phi is what the Poisson solve returns for rhs = D u*).  Blocks
// march g.kzd planes carrying psi(k+1) into the next plane; psi(i+1) comes from
// the neighbouring lane.  Loads of DZ planes are issued before any is used.
// ---------------------------------------------------------------------------
template <typename T, bool THREE, bool FLUX, bool XF>
__global__ void __launch_bounds__(256) k_correct(GridP g, const T* __restrict__ us0, const T* __restrict__ us1,
                                                 const T* __restrict__ us2, const T* __restrict__ psi,
                                                 const uint8_t* __restrict__ mask, T* __restrict__ u0,
                                                 T* __restrict__ u1, T* __restrict__ u2, T* __restrict__ p, T idx,
                                                 T idy, T idz, T inv_ckdt, int update_p, FluxCorr<T> fc) {
    constexpr int ZB = THREE ? DZ : 1;
    const int lane = threadIdx.x;
    const int i = blockIdx.x * 32 + lane;
    const int j = blockIdx.y * 8 + threadIdx.y;
    if (j >= g.ny) return;                                   // whole warp
    const int kbeg = THREE ? blockIdx.z * g.kzd : 0;
    const int kend = THREE ? min(kbeg + g.kzd, g.nz) : 1;
    const bool live = i < g.nx;
    const int plane = g.nx * g.ny;
    const int ir = (i + 1 < g.nx) ? i + 1 : 0;              // +x neighbour (periodic)
    const bool from_lane = lane < 31 && i + 1 < g.nx;
    const bool top = j == g.ny - 1;
    const bool outface = XF && i == g.nx - 1;               // the outflow face keeps u*
    const T pic = FLUX ? *reinterpret_cast<const T*>(fc.scal + 2) * fc.ckdt : T(0);
    if (g.ystr) idy = (T)ytab(g, YT_IHV, j);                 // a stretched y: the centre distance across v's face
    T ph = live ? psi[i + g.nx * j + plane * kbeg] : T(0);
    for (int k0 = kbeg; k0 < kend; k0 += ZB) {
        T a0[ZB], a1[ZB], a2[ZB], pT[ZB], pN[ZB], pE[ZB], pp[ZB];
        uint8_t mc[ZB];
#pragma unroll
        for (int t = 0; t < ZB; ++t) {
            a0[t] = a1[t] = a2[t] = pT[t] = pN[t] = pE[t] = pp[t] = T(0);
            mc[t] = 0;
            const int k = k0 + t;
            if (k < kend && live) {
                const int rowb = g.nx * (j + g.ny * k);
                const int id = rowb + i;
                a0[t] = us0[id];
                a1[t] = us1[id];
                if (THREE) {
                    a2[t] = us2[id];
                    pT[t] = psi[id + ((k + 1 < g.nz) ? plane : plane - (int)g.N)];
                }
                if (!top) pN[t] = psi[id + g.nx];
                if (!from_lane) pE[t] = psi[rowb + ir];
                if (FLUX) mc[t] = mask[id];
                if (update_p) pp[t] = p[id];
            }
        }
#pragma unroll
        for (int t = 0; t < ZB; ++t) {
            const int k = k0 + t;
            if (k >= kend) break;
            const int id = g.nx * (j + g.ny * k) + i;
            T e = __shfl_down_sync(0xffffffffu, ph, 1);
            if (!from_lane) e = pE[t];
            T uc = T(0);
            if (FLUX) {
                const unsigned b = __ballot_sync(0xffffffffu, (mc[t] & IBM_MASK_IBM_U) != 0);
                if (live) uc = flux_increment(fc, pic, mc[t], b, (j + g.ny * k) * g.nsegx + (int)blockIdx.x, lane);
            }
            if (live) {
                u0[id] = outface ? a0[t] : a0[t] + uc - (e - ph) * idx;
                u1[id] = top ? a1[t] : a1[t] - (pN[t] - ph) * idy;
                if (THREE) u2[id] = a2[t] - (pT[t] - ph) * idz;
                if (update_p) p[id] = pp[t] + ph * inv_ckdt;
            }
            ph = pT[t];
        }
    }
}

// initial-condition projection: copy the velocity with non-internal points zeroed
template <typename T>
__global__ void k_mask_copy(GridP g, const uint8_t* __restrict__ mask, const T* __restrict__ a0,
                            const T* __restrict__ a1, const T* __restrict__ a2, T* __restrict__ b0,
                            T* __restrict__ b1, T* __restrict__ b2, BodyP body) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const long long id = i + (long long)g.nx * (j + (long long)g.ny * blockIdx.z);
    uint8_t m = mask[id];
    const bool readable_u = (m & IBM_MASK_U) || (!g.xper && i == g.nx - 1 && (m & IBM_MASK_FACE));
    // a moving body's points hold its velocity (periodic x: v on the +y wall is the only box face)
    T r[3] = {T(0), T(0), T(0)};
    if (body.kind != 0)
        for (int c = 0; c < g.ncomp; ++c)
            if (!(c == 1 && j == g.ny - 1))
                r[c] = (T)bodyvel(body, c, g.ox + (i + (c == 0 ? 1.0 : 0.5)) * g.dx,
                                  g.oy + (j + (c == 1 ? 1.0 : 0.5)) * g.dy);
    b0[id] = readable_u ? a0[id] : r[0];
    b1[id] = (m & IBM_MASK_V) ? a1[id] : r[1];
    if (g.ndim == 3) b2[id] = (m & IBM_MASK_W) ? a2[id] : r[2];
}

// ---------------------------------------------------------------------------
// K8: diagnostics partials (12 doubles per block), then a fixed-order final sum
//   [0] sum div^2  [1] max |div|  [2..4] max |u_c|  [5..7] sum u_c  [8..10] sum u_c^2  [11] non-finite count
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_diag(GridP g, const T* __restrict__ u, const T* __restrict__ v,
                                              const T* __restrict__ w, const T* __restrict__ p,
                                              const uint8_t* __restrict__ mask, double* __restrict__ part, double idx,
                                              double idy, double idz) {
    // A block (32 x 8 threads) takes work tiles of 32 x 8 (x, y) points and up to
    // DIAG_Z planes; a thread marches its point's column, carrying w(k-1), and
    // takes u(i-1) from the neighbouring lane.
    constexpr int DIAG_Z = 8;
    __shared__ double sh[12][8];
    DiagAcc<T> acc;
    const DiagInv<T> inv(idx, idy, idz);
    const int lane = threadIdx.x, wy = threadIdx.y;
    const int nty = (g.ny + 7) / 8, nzc = (g.nz + DIAG_Z - 1) / DIAG_Z;
    const long long ntiles = (long long)g.nsegx * nty * nzc;
    const int plane = g.nx * g.ny;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int tx = (int)(t % g.nsegx);
        const long long r = t / g.nsegx;
        const int ty = (int)(r % nty);
        const int kc = (int)(r / nty);
        const int i = tx * 32 + lane, j = ty * 8 + wy;
        if (j >= g.ny) continue;                              // whole warp
        const bool live = i < g.nx;
        const int il = wrapi(tx * 32 - 1, g.nx);              // left neighbour of lane 0
        const int kbeg = kc * DIAG_Z, kend = min(kbeg + DIAG_Z, g.nz);
        T wm = T(0);
        if (g.ndim == 3 && live) wm = w[i + g.nx * j + plane * wrapi(kbeg - 1, g.nz)];
        for (int k0 = kbeg; k0 < kend; k0 += DZ) {
            // the loads of DZ planes go out before any is used
            T uc[DZ], ul0[DZ], vc[DZ], vm[DZ], wc[DZ], pc[DZ];
            uint8_t mc[DZ];
#pragma unroll
            for (int t = 0; t < DZ; ++t) {
                uc[t] = ul0[t] = vc[t] = vm[t] = wc[t] = pc[t] = T(0);
                mc[t] = 0;
                const int k = k0 + t;
                if (k < kend) {
                    const int rowb = g.nx * (j + g.ny * k);
                    const int id = rowb + i;
                    if (lane == 0) {
                        if (g.xper || tx != 0) ul0[t] = u[rowb + il];
                        else ul0[t] = (mask[rowb] & IBM_MASK_FACE) ? (T)g.uin : T(0);   // the inflow face
                    }
                    if (live) {
                        uc[t] = u[id];
                        vc[t] = v[id];
                        if (j > 0) vm[t] = v[id - g.nx];
                        if (g.ndim == 3) wc[t] = w[id];
                        pc[t] = p[id];
                        mc[t] = mask[id];
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < DZ; ++t) {
                if (k0 + t >= kend) break;
                T ul = __shfl_up_sync(0xffffffffu, uc[t], 1);
                if (lane == 0) ul = ul0[t];
                if (live) acc.cell(g.ncomp, inv.v, uc[t], ul, vc[t], vm[t], wc[t], wm, pc[t], mc[t]);
                wm = wc[t];
            }
        }
    }
    double a[12];
    acc.finish(a);
    for (int q = 0; q < 12; ++q) {
        double x = a[q];
        if (q == 1 || (q >= 2 && q <= 4)) x = warp_max(x);
        else x = warp_sum(x);
        if (lane == 0) sh[q][wy] = x;
    }
    __syncthreads();
    const int tid = lane + 32 * wy;
    if (tid < 12) {
        int q = tid;
        double s = 0.0;
        for (int ww = 0; ww < 8; ++ww)
            s = (q == 1 || (q >= 2 && q <= 4)) ? fmax(s, sh[q][ww]) : s + sh[q][ww];
        part[blockIdx.x * 12 + q] = s;
    }
}

// one warp per quantity, fixed order: lane-strided partial sums, then a shuffle tree
// The same partials on a stretched y, in FP64 per cell: the divergence with the row's cell
// height, the sums weighted by it (volumes differ by row), and each velocity maximum already
// divided by its spacing (v: the smaller of the two cells its face joins), as the host expects.
template <typename T>
__global__ void __launch_bounds__(256) k_diag_str(GridP g, const T* __restrict__ u, const T* __restrict__ v,
                                                  const T* __restrict__ w, const T* __restrict__ p,
                                                  const uint8_t* __restrict__ mask, double* __restrict__ part) {
    __shared__ double sh[12][8];
    double a[12];
    for (int q = 0; q < 12; ++q) a[q] = 0.0;
    const double idx = 1.0 / g.dx, idz = 1.0 / g.dz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < g.N; id += stride) {
        const int i = (int)(id % g.nx);
        const long long row = id / g.nx;
        const int j = (int)(row % g.ny);
        const int k = (int)(row / g.ny);
        const uint8_t m = mask[id];
        const double uc = (double)u[id];
        // the -x face of the first cell is the inflow face in an inflow/outflow box
        const double ul = (g.xper || i > 0) ? (double)u[row * g.nx + wrapi(i - 1, g.nx)]
                                            : ((m & IBM_MASK_FACE) ? g.uin : 0.0);
        const double vc = (double)v[id], vm = j > 0 ? (double)v[id - g.nx] : 0.0;
        double d = (uc - ul) * idx + (vc - vm) * ytab(g, YT_IDYC, j);
        double wc = 0.0;
        if (g.ndim == 3) {
            wc = (double)w[id];
            const double wm = (double)w[i + (long long)g.nx * (j + (long long)g.ny * wrapi(k - 1, g.nz))];
            d += (wc - wm) * idz;
        }
        a[0] += d * d;
        a[1] = fmax(a[1], fabs(d));
        const double dyc = ytab(g, YT_DYC, j);
        const double isp[3] = {idx, ytab(g, YT_IVSP, j), idz};
        const double x3[3] = {uc, vc, wc};
        for (int c = 0; c < g.ncomp; ++c) {
            const double x = x3[c];
            if (!isfinite(x)) a[11] += 1.0;
            if (!((m >> c) & 1u)) continue;
            a[2 + c] = fmax(a[2 + c], fabs(x) * isp[c]);
            a[5 + c] += x * dyc;
            a[8 + c] += x * x * dyc;
        }
        if (!isfinite((double)p[id])) a[11] += 1.0;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = 0; q < 12; ++q) {
        const bool mx = q == 1 || (q >= 2 && q <= 4);
        const double x = mx ? warp_max(a[q]) : warp_sum(a[q]);
        if (lane == 0) sh[q][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        const int q = threadIdx.x;
        const bool mx = q == 1 || (q >= 2 && q <= 4);
        double t = 0.0;
        for (int ww = 0; ww < 8; ++ww) t = mx ? fmax(t, sh[q][ww]) : t + sh[q][ww];
        part[blockIdx.x * 12 + q] = t;
    }
}

__global__ void k_diag_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (q >= 12) return;
    const bool mx = q == 1 || (q >= 2 && q <= 4);
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s = mx ? fmax(s, part[b * 12 + q]) : s + part[b * 12 + q];
    s = mx ? warp_max(s) : warp_sum(s);
    if (lane == 0) out[q] = s;
}


// 32 x 8 cells per block, one z plane per blockIdx.z
dim3 cell_grid(const GridP& g) { return dim3(g.nsegx, (g.ny + 7) / 8, g.nz); }


// ---------------------------------------------------------------------------
// Neumann x (inflow/outflow): the type-II DCT of every x row,
//   X[k] = sum_n x[n] cos(pi k (2n+1) / 2nx),
// through one nx-point real FFT (Makhoul's reordering), and its inverse.
//   forward:  v[pos(n)] = x[n], even n ascending and odd n descending;
//             V = FFT(v);  X[k] = Re(e^{-i pi k/2nx} V[k])  (V[k] = conj V[nx-k] past nx/2)
//   inverse:  V[k] = e^{i pi k/2nx} (X[k] - i X[nx-k])  (X[nx] = 0),  v = IFFT(V),  x[n] = v[pos(n)]
// The 1/nx of the inverse sits in the tridiagonal's scale with the 1/nz of z.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int dct_pos(int n, int N) { return (n & 1) ? N - 1 - (n >> 1) : (n >> 1); }

template <typename T>
__global__ void k_dct_reorder(GridP g, const T* __restrict__ in, T* __restrict__ out, int inverse) {
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    const int n = (int)(id % g.nx);
    const long long m = id - n + dct_pos(n, g.nx);
    if (inverse) out[id] = in[m];
    else out[m] = in[id];
}

template <typename T>
__global__ void k_dct_twiddles(int nx, T* __restrict__ tw) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nx) return;
    double sn, cs;
    sincospi((double)k / (2.0 * nx), &sn, &cs);
    tw[2 * k] = (T)cs;
    tw[2 * k + 1] = (T)sn;
}

// ---------------------------------------------------------------------------
// Own real FFT of the x rows (replaces cuFFT's R2C / C2R along x, whose kernel for
// the 384-point rows moved 2 TB/s).  A row of N = 2M reals is M complex values
// z_n = x_2n + i x_2n+1 (the row read as complex pairs); one warp transforms one
// row in shared memory with a self-sorting (Stockham) mixed-radix FFT of length M,
// radices 4, 2, 3, 5, and the split of the two interleaved real transforms gives
// X_k, k = 0..M (Sec. 2.1: the periodic directions are solved "exactly" by
// transforms).  The inverse undoes each step (unnormalised, like cuFFT's C2R).
// Stage s of radix R with Ns the product of the earlier radices: for j < M/R,
// k = j mod Ns, v_q = x[j + q M/R] exp(-+2 pi i q k / (Ns R)), V = DFT_R(v),
// y[(j / Ns) Ns R + k + q Ns] = V_q.
// ---------------------------------------------------------------------------
template <typename C> struct CT;
template <> struct CT<float2> { using T = float; };
template <> struct CT<double2> { using T = double; };
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) { return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
template <typename C> __device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }
// multiply by -i (SIGN = -1) or +i (SIGN = +1)
template <int SIGN, typename C> __device__ __forceinline__ C cmuli(C a) {
    return SIGN < 0 ? C{a.y, -a.x} : C{-a.y, a.x};
}

// in-place DFT of R points with kernel exp(SIGN 2 pi i q p / R)
template <int SIGN, typename C>
__device__ __forceinline__ void dft_small(C* v, int R) {
    using T = typename CT<C>::T;
    if (R == 2) {
        const C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if (R == 4) {
        const C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        const C c = cadd(v[1], v[3]), d = cmuli<SIGN>(csub(v[1], v[3]));
        v[0] = cadd(a, c);
        v[2] = csub(a, c);
        v[1] = cadd(b, d);
        v[3] = csub(b, d);
    } else if (R == 3) {
        const T h = (T)0.5, s3 = (T)(SIGN * 0.86602540378443864676);   // sin(2 pi / 3)
        const C t = cadd(v[1], v[2]);
        const C u = csub(v[1], v[2]);
        const C m = C{v[0].x - h * t.x, v[0].y - h * t.y};
        const C r = C{-s3 * u.y, s3 * u.x};                              // i s3 u
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    } else {   // R == 5
        const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;   // cos(2 pi/5), cos(4 pi/5)
        const T s1 = (T)(SIGN * 0.95105651629515357212), s2 = (T)(SIGN * 0.58778525229247312917);
        const C a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
        const C a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
        const C x0 = v[0];
        const C m1 = C{x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y};
        const C m2 = C{x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y};
        const C n1 = C{-(s1 * b1.y + s2 * b2.y), s1 * b1.x + s2 * b2.x};    // i (s1 b1 + s2 b2)
        const C n2 = C{-(s2 * b1.y - s1 * b2.y), s2 * b1.x - s1 * b2.x};    // i (s2 b1 - s1 b2)
        v[0] = cadd(x0, cadd(a1, a2));
        v[1] = cadd(m1, n1);
        v[4] = csub(m1, n1);
        v[2] = cadd(m2, n2);
        v[3] = csub(m2, n2);
    }
}

// DFT of 8 points: two DFTs of 4 (even and odd points) joined by exp(SIGN 2 pi i p / 8)
template <int SIGN, typename C>
__device__ __forceinline__ void dft8(C* v) {
    using T = typename CT<C>::T;
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    dft_small<SIGN>(e, 4);
    dft_small<SIGN>(o, 4);
    const T r = (T)0.70710678118654752440;
    const C w1 = C{r * (o[1].x - SIGN * o[1].y), r * (o[1].y + SIGN * o[1].x)};     // (1 + SIGN i)/sqrt2 o1
    const C w2 = cmuli<SIGN>(o[2]);                                                   // SIGN i o2
    const C w3 = C{r * (-o[3].x - SIGN * o[3].y), r * (-o[3].y + SIGN * o[3].x)};   // (-1 + SIGN i)/sqrt2 o3
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], w1);
    v[5] = csub(e[1], w1);
    v[2] = cadd(e[2], w2);
    v[6] = csub(e[2], w2);
    v[3] = cadd(e[3], w3);
    v[7] = csub(e[3], w3);
}

struct FftPlan {
    int M, nrad;
    int rad[16];
};

// Shared-memory place of complex value i of a row buffer: one pad slot after every 16,
// so that the stride-R and stride-NS stores of the early stages spread over the banks
// (unpadded, the first radix-8 stage's stores hit the same two banks 16 times).
__device__ __forceinline__ int pz(int i) { return i + (i >> 4); }
// ... and of real value r of a row buffer viewed as reals
__device__ __forceinline__ int pzr(int r) { return 2 * pz(r >> 1) + (r & 1); }
// complex slots of one row buffer (values 0 .. M + 2 with their pads)
__host__ __device__ inline int fft_ps(int M) { return M + (M >> 4) + 4; }

// The warp's FFT of length M from src (shared or global) to a shared buffer; returns the
// buffer holding the result.  tw[t] = exp(-2 pi i t / M).
template <int SIGN, bool GS, typename C>
__device__ __forceinline__ C* warp_fft(const FftPlan& pl, const C* __restrict__ src, C* b0, C* b1,
                                       const C* __restrict__ tw) {
    const int lane = threadIdx.x & 31;
    const int M = pl.M;
    const C* x = src;
    C* y = b0;
    int Ns = 1;
    for (int s = 0; s < pl.nrad; ++s) {
        const int R = pl.rad[s];
        const int MR = M / R;
        const int step = M / (Ns * R);     // twiddle index step: exp(-2 pi i q k / (Ns R)) = tw[q k step]
        for (int j = lane; j < MR; j += 32) {
            const int k = j % Ns;
            C v[5];
#pragma unroll
            for (int q = 0; q < 5; ++q)
                if (q < R) {
                    C a = (GS && s == 0) ? x[j + q * MR] : x[pz(j + q * MR)];
                    if (q > 0 && k > 0) {
                        C w = tw[q * k * step];
                        if (SIGN > 0) w = cconj(w);
                        a = cmul(a, w);
                    }
                    v[q] = a;
                }
            dft_small<SIGN>(v, R);
            const int base = (j / Ns) * Ns * R + k;
#pragma unroll
            for (int q = 0; q < 5; ++q)
                if (q < R) y[pz(base + q * Ns)] = v[q];
        }
        __syncwarp();
        x = y;
        y = (y == b0) ? b1 : b0;
        Ns *= R;
    }
    return const_cast<C*>(x);
}

// The same FFT with the length known at compile time: the stage loop unrolled, the
// index arithmetic by constants, radix 8 where it divides (then 4, 2, 3, 5).
template <int SIGN, int M, int R, int NS, bool GS, typename C>
__device__ __forceinline__ void fft_stage(const C* __restrict__ x, C* __restrict__ y, const C* __restrict__ tw) {
    constexpr int MR = M / R;
    constexpr int STEP = M / (NS * R);
    const int lane = threadIdx.x & 31;
#pragma unroll 2
    for (int j = lane; j < MR; j += 32) {
        const int k = j % NS;
        C v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            C a = GS ? x[j + q * MR] : x[pz(j + q * MR)];
            if (q > 0 && NS > 1) {
                C w = tw[q * k * STEP];
                if (SIGN > 0) w = cconj(w);
                a = cmul(a, w);
            }
            v[q] = a;
        }
        C vv[8];
#pragma unroll
        for (int q = 0; q < R; ++q) vv[q] = v[q];
        if (R == 8) dft8<SIGN>(vv);
        else dft_small<SIGN>(vv, R);
        const int base = (j / NS) * NS * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) y[pz(base + q * NS)] = vv[q];
    }
}

template <int SIGN, int M, int NS, int REM, bool GS>
struct FftRun {
    static constexpr int R = REM % 8 == 0 ? 8 : (REM % 4 == 0 ? 4 : (REM % 2 == 0 ? 2 : (REM % 3 == 0 ? 3 : 5)));
    template <typename C>
    static __device__ __forceinline__ const C* run(const C* x, C* b0, C* b1, const C* tw) {
        fft_stage<SIGN, M, R, NS, GS>(x, b0, tw);
        __syncwarp();
        return FftRun<SIGN, M, NS * R, REM / R, false>::run(b0, b1, b0, tw);
    }
};
template <int SIGN, int M, int NS, bool GS>
struct FftRun<SIGN, M, NS, 1, GS> {
    template <typename C>
    static __device__ __forceinline__ const C* run(const C* x, C*, C*, const C*) { return x; }
};

// lengths with a compiled form (the workloads' rows: 384, 512 and 1536 reals)
// GS: src is the row in global memory (unpadded); else a padded shared row buffer.
template <int SIGN, typename C, bool GS = false>
__device__ __forceinline__ const C* warp_fft_any(const FftPlan& pl, const C* src, C* b0, C* b1, const C* tw) {
    switch (pl.M) {
        case 192: return FftRun<SIGN, 192, 1, 192, GS>::run(src, b0, b1, tw);
        case 256: return FftRun<SIGN, 256, 1, 256, GS>::run(src, b0, b1, tw);
        case 768: return FftRun<SIGN, 768, 1, 768, GS>::run(src, b0, b1, tw);
        default: return warp_fft<SIGN, GS, C>(pl, src, b0, b1, tw);
    }
}

// The split of the two interleaved real transforms: X_k, k = 0..M, from Z = FFT(z).
template <typename C>
__device__ __forceinline__ void rfft_post(int M, const C* Z, C* __restrict__ o, const C* __restrict__ twN) {
    using T = typename CT<C>::T;
    const int lane = threadIdx.x & 31;
    for (int k = lane; k <= M; k += 32) {
        const C zk = Z[pz(k == M ? 0 : k)];
        const C zc = cconj(Z[pz(k == 0 ? 0 : M - k)]);
        const C e = C{(zk.x + zc.x) * (T)0.5, (zk.y + zc.y) * (T)0.5};        // (Z_k + conj Z_{M-k}) / 2
        const C d = C{(zk.x - zc.x) * (T)0.5, (zk.y - zc.y) * (T)0.5};
        const C od = C{d.y, -d.x};                                              // d / i
        o[k] = cadd(e, cmul(twN[k], od));
    }
}

// Forward: rows of N = 2M reals (as M complex pairs) to M + 1 complex values each.
template <typename C>
__global__ void __launch_bounds__(256) k_rfft_rows(FftPlan pl, long long rows, const C* __restrict__ in,
                                                   C* __restrict__ out, const C* __restrict__ tab) {
    extern __shared__ unsigned char fft_smem[];
    using T = typename CT<C>::T;
    const int M = pl.M;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long row = (long long)blockIdx.x * (blockDim.x >> 5) + w;
    C* b0 = reinterpret_cast<C*>(fft_smem) + (size_t)w * 3 * fft_ps(M);
    C* b1 = b0 + fft_ps(M);
    if (row >= rows) return;                              // whole warp
    const C* twM = tab;                                   // exp(-2 pi i t / M)
    const C* twN = tab + M;                               // exp(-2 pi i k / 2M)
    const C* Z = warp_fft_any<-1, C, true>(pl, in + row * M, b0, b1, twM);
    rfft_post<C>(M, Z, out + row * (M + 1), twN);
}

// Inverse: M + 1 complex values per row to N = 2M reals (written as M complex pairs),
// unnormalised.
template <typename C>
__global__ void __launch_bounds__(256) k_irfft_rows(FftPlan pl, long long rows, const C* __restrict__ in,
                                                    C* __restrict__ out, const C* __restrict__ tab) {
    extern __shared__ unsigned char fft_smem[];
    const int M = pl.M;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long row = (long long)blockIdx.x * (blockDim.x >> 5) + w;
    C* b0 = reinterpret_cast<C*>(fft_smem) + (size_t)w * 3 * fft_ps(M);
    C* b1 = b0 + fft_ps(M);
    C* b2 = b1 + fft_ps(M);
    if (row >= rows) return;
    const C* twM = tab;
    const C* twN = tab + M;
    const C* X = in + row * (M + 1);
    for (int k = lane; k < M; k += 32) {
        const C xk = X[k];
        const C xc = cconj(X[M - k]);
        const C e = cadd(xk, xc);
        const C d = cmul(csub(xk, xc), cconj(twN[k]));        // (X_k - conj X_{M-k}) exp(+2 pi i k / 2M)
        b2[pz(k)] = cadd(e, C{-d.y, d.x});                    // e + i d
    }
    __syncwarp();
    const C* z = warp_fft_any<+1, C>(pl, b2, b0, b1, twM);
    C* o = out + row * M;
    for (int n = lane; n < M; n += 32) o[n] = z[pz(n)];
}

// The divergence of u* fused with the forward transform of its x rows (periodic x; XF below):
// one warp computes the divergence of a whole row (32 cells per pass, the constant-flow-rate
// increment of the internal u points as in k_divergence, u*(x-1) from the lane below or
// carried from the previous pass) into shared memory and transforms it there, so the
// divergence never goes through HBM.
// XF: an inflow/outflow x instead: the inflow face value is the left neighbour of x = 0,
// the row goes into the DCT order, and the twiddled DCT coefficients are written over the
// row of xout (as k_dct_rows) instead of a half spectrum.
// The divergence of one x row by one warp for FP32 fields with nx a multiple of 128: each
// lane takes 4 consecutive cells of a 128-cell chunk with 16-byte loads, u*(x-1) of its first
// cell comes from the lane below (or the previous chunk), and the results go to the row
// buffer as pairs (the padded real layout, or the DCT order of an inflow/outflow x).
// The constant-flow-rate increment of an IBM point finds its coefficient from the number of
// IBM points before it in its 32-point segment (a prefix over the segment's 8 lanes).
template <bool THREE, bool FLUX, bool XF>
__device__ __forceinline__ void div_row_vec4(const GridP& g, const float* __restrict__ ur, const float* __restrict__ vr,
                                             const float* __restrict__ vmr, const float* __restrict__ wr,
                                             const float* __restrict__ wmr, const uint8_t* __restrict__ mr,
                                             bool has_below, const FluxCorr<float>& fc, float pic, float idx,
                                             float idy, float idz, int rowseg, float carry, float* __restrict__ d,
                                             int N) {
    const int lane = threadIdx.x & 31;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int c0 = 0; c0 < g.nx; c0 += 128) {
        const int x0 = c0 + 4 * lane;
        const float4 u4 = *reinterpret_cast<const float4*>(ur + x0);
        const float4 v4 = *reinterpret_cast<const float4*>(vr + x0);
        const float4 m4 = has_below ? *reinterpret_cast<const float4*>(vmr + x0) : z4;
        float4 w4 = z4, q4 = z4;
        if (THREE) {
            w4 = *reinterpret_cast<const float4*>(wr + x0);
            q4 = *reinterpret_cast<const float4*>(wmr + x0);
        }
        float uc[4] = {u4.x, u4.y, u4.z, u4.w};
        if (FLUX) {
            const uint32_t mb = *reinterpret_cast<const uint32_t*>(mr + x0);
            uint32_t ibm = 0;                                  // IBM-point bits of the 4 cells
#pragma unroll
            for (int e = 0; e < 4; ++e) ibm |= ((mb >> (8 * e + 4)) & 1u) << e;
            if (__any_sync(0xffffffffu, ibm != 0u)) {
                // IBM points before this lane's first cell within its 32-point segment (8 lanes)
                const int cnt = __popc(ibm);
                int pre = cnt;
#pragma unroll
                for (int o = 1; o < 8; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, pre, o, 8);
                    if ((lane & 7) >= o) pre += t;
                }
                pre -= cnt;
                const int seg = rowseg + (x0 >> 5);
                const int base = fc.segoff[seg] + pre;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const uint32_t me = (mb >> (8 * e)) & 0xffu;
                    if (!(me & IBM_MASK_U)) continue;
                    float beta = 1.f;
                    if (me & IBM_MASK_IBM_U) beta = fc.coef[base + __popc(ibm & ((1u << e) - 1u))].b;
                    uc[e] += pic * beta;
                }
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if ((mb >> (8 * e)) & IBM_MASK_U) uc[e] += pic;
            }
        }
        float ul = __shfl_up_sync(0xffffffffu, uc[3], 1);
        if (lane == 0) ul = carry;
        carry = __shfl_sync(0xffffffffu, uc[3], 31);
        const float vv[4] = {v4.x, v4.y, v4.z, v4.w}, vm[4] = {m4.x, m4.y, m4.z, m4.w};
        const float ww[4] = {w4.x, w4.y, w4.z, w4.w}, wm[4] = {q4.x, q4.y, q4.z, q4.w};
        float dv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float t = (uc[e] - (e == 0 ? ul : uc[e - 1])) * idx;
            t += (vv[e] - vm[e]) * idy;
            if (THREE) t += (ww[e] - wm[e]) * idz;
            dv[e] = t;
        }
        if (XF) {
            // DCT order: even x at x / 2, odd x at N - 1 - (x - 1) / 2 (each pair in one complex slot)
            const int re = x0 >> 1, ro = N - 2 - (x0 >> 1);
            *reinterpret_cast<float2*>(d + pzr(re)) = make_float2(dv[0], dv[2]);
            *reinterpret_cast<float2*>(d + pzr(ro)) = make_float2(dv[3], dv[1]);
        } else {
            *reinterpret_cast<float2*>(d + pzr(x0)) = make_float2(dv[0], dv[1]);
            *reinterpret_cast<float2*>(d + pzr(x0 + 2)) = make_float2(dv[2], dv[3]);
        }
    }
}

template <typename T, typename C, bool THREE, bool FLUX, bool XF>
__device__ __forceinline__ void div_rfft_rows(const GridP& g, const T* __restrict__ u, const T* __restrict__ v,
                                              const T* __restrict__ w, const uint8_t* __restrict__ mask,
                                              const FluxCorr<T>& fc, T idx, T idy, T idz, const FftPlan& pl,
                                              C* __restrict__ out, const C* __restrict__ tab,
                                              T* __restrict__ xout, const T* __restrict__ tw) {
    extern __shared__ unsigned char fft_smem[];
    const int M = pl.M;
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const long long rows = (long long)g.ny * g.nz;
    const long long row = (long long)blockIdx.x * (blockDim.x >> 5) + wq;
    C* b0 = reinterpret_cast<C*>(fft_smem) + (size_t)wq * 3 * fft_ps(M);
    C* b1 = b0 + fft_ps(M);
    C* b2 = b1 + fft_ps(M);
    if (row >= rows) return;                              // whole warp
    const int N = 2 * M;
    const int j = (int)(row % g.ny), k = (int)(row / g.ny);
    const long long rowb = row * g.nx;
    const long long rowm = THREE ? (long long)(k > 0 ? k - 1 : g.nz - 1) * g.ny * g.nx + (long long)j * g.nx : 0;
    T* d = reinterpret_cast<T*>(b2);
    const T pic = FLUX ? *reinterpret_cast<const T*>(fc.scal + 2) * fc.ckdt : T(0);
    const int nseg = g.nsegx;
    const int rowseg = (j + g.ny * k) * nseg;
    // u* at x = nx - 1 (with its increment): the left neighbour of x = 0; the inflow face
    // value for an inflow/outflow x
    T carry;
    if (XF) {
        carry = (mask[rowb] & IBM_MASK_FACE) ? (T)g.uin : T(0);
    } else {
        const int s = nseg - 1;
        const int x = s * 32 + lane;
        const bool live = x < g.nx;
        T uc = live ? u[rowb + x] : T(0);
        if (FLUX) {
            const uint8_t m = live ? mask[rowb + x] : 0;
            const unsigned b = __ballot_sync(0xffffffffu, (m & IBM_MASK_IBM_U) != 0);
            if (live) uc += flux_increment(fc, pic, m, b, rowseg + s, lane);
        }
        carry = __shfl_sync(0xffffffffu, uc, (g.nx - 1) & 31);
    }
    // the row's own pointers: the loads below index them with 32-bit offsets
    const T* __restrict__ ur = u + rowb;
    const T* __restrict__ vr = v + rowb;
    const T* __restrict__ vmr = v + rowb - (j > 0 ? g.nx : 0);
    const T* __restrict__ wr = w + rowb;
    const T* __restrict__ wmr = w + rowm;
    const uint8_t* __restrict__ mr = mask + rowb;
    if constexpr (sizeof(T) == 4) {
        if ((g.nx & 127) == 0) {
            div_row_vec4<THREE, FLUX, XF>(g, ur, vr, vmr, wr, wmr, mr, j > 0, fc, pic, idx, idy, idz, rowseg,
                                               carry, reinterpret_cast<float*>(d), N);
            goto transform;
        }
    }
    {
    constexpr int SB = 6;      // passes whose loads go out together (measured: 3, 4, 6, 12 -> 0.150, 0.146, 0.139, 0.187 ms)
        for (int s0 = 0; s0 < nseg; s0 += SB) {
            T uc[SB], vc[SB], vm[SB], wc[SB], wm[SB];
            uint8_t m[SB];
    #pragma unroll
            for (int t = 0; t < SB; ++t) {
                const int x = (s0 + t) * 32 + lane;
                uc[t] = vc[t] = vm[t] = wc[t] = wm[t] = T(0);
                m[t] = 0;
                if (s0 + t < nseg && x < g.nx) {
                    uc[t] = ur[x];
                    vc[t] = vr[x];
                    if (j > 0) vm[t] = vmr[x];
                    if (THREE) {
                        wc[t] = wr[x];
                        wm[t] = wmr[x];
                    }
                    if (FLUX) m[t] = mr[x];
                }
            }
    #pragma unroll
            for (int t = 0; t < SB; ++t) {
                const int s = s0 + t;
                if (s >= nseg) continue;          // (not break: the loop must unroll, keeping the arrays in registers)
                const int x = s * 32 + lane;
                const bool live = x < g.nx;
                T ucc = uc[t];
                if (FLUX) {
                    const unsigned b = __ballot_sync(0xffffffffu, (m[t] & IBM_MASK_IBM_U) != 0);
                    if (live) ucc += flux_increment(fc, pic, m[t], b, rowseg + s, lane);
                }
                T ul = __shfl_up_sync(0xffffffffu, ucc, 1);
                if (lane == 0) ul = carry;
                carry = __shfl_sync(0xffffffffu, ucc, 31);
                if (live) {
                    T dv = (ucc - ul) * idx;
                    dv += (vc[t] - vm[t]) * idy;
                    if (THREE) dv += (wc[t] - wm[t]) * idz;
                    d[pzr(XF ? ((x & 1) ? N - 1 - (x >> 1) : (x >> 1)) : x)] = dv;
                }
            }
        }
    }
transform:
    __syncwarp();
    const C* Z = warp_fft_any<-1, C, false>(pl, reinterpret_cast<const C*>(d), b0, b1, tab);
    if (!XF) {
        rfft_post<C>(M, Z, out + row * (M + 1), tab + M);
        return;
    }
    // DCT twiddle as in k_dct_rows
    C* V = (Z == b0) ? b1 : b0;
    const C* twN = tab + M;
    for (int kk = lane; kk < M; kk += 32) {
        const C zk = Z[pz(kk)];
        const C zc = cconj(Z[pz(kk == 0 ? 0 : M - kk)]);
        const C e = C{(zk.x + zc.x) * (T)0.5, (zk.y + zc.y) * (T)0.5};
        const C dd = C{(zk.x - zc.x) * (T)0.5, (zk.y - zc.y) * (T)0.5};
        V[pz(kk)] = cadd(e, cmul(twN[kk], C{dd.y, -dd.x}));
    }
    const C z0 = Z[0];
    __syncwarp();
    T* xr = xout + row * N;
    const C* tw2 = reinterpret_cast<const C*>(tw);        // (cos, sin) pairs, one load each
#pragma unroll 4
    for (int kk = lane; kk < N; kk += 32) {
        const C t = tw2[kk];
        C vk;
        if (kk < M) vk = V[pz(kk)];
        else if (kk == M) vk = C{z0.x - z0.y, (T)0};
        else { vk = V[pz(N - kk)]; vk.y = -vk.y; }
        xr[kk] = t.x * vk.x + t.y * vk.y;
    }
}

#define IBM_DIV_RFFT_PARAMS                                                                                      \
    GridP g, const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ w,                          \
        const uint8_t* __restrict__ mask, FluxCorr<T> fc, T idx, T idy, T idz, const __grid_constant__ FftPlan pl, \
        C* __restrict__ out, const C* __restrict__ tab, T* __restrict__ xout, const T* __restrict__ tw
template <typename T, typename C, bool THREE, bool FLUX, bool XF>
__global__ void __launch_bounds__(256) k_div_rfft_rows(IBM_DIV_RFFT_PARAMS) {
    div_rfft_rows<T, C, THREE, FLUX, XF>(g, u, v, w, mask, fc, idx, idy, idz, pl, out, tab, xout, tw);
}
// The FP32 constant-flow-rate instance held to 64 registers, four blocks of eight warps per SM: it is
// latency-bound, and the extra warps outweigh a few spilled bytes (0.126 -> 0.108 ms on 384x256x256).
template <typename T, typename C, bool THREE, bool FLUX, bool XF>
__global__ void __launch_bounds__(256, 4) k_div_rfft_rows_flux(IBM_DIV_RFFT_PARAMS) {
    div_rfft_rows<T, C, THREE, FLUX, XF>(g, u, v, w, mask, fc, idx, idy, idz, pl, out, tab, xout, tw);
}
#undef IBM_DIV_RFFT_PARAMS

template <typename T, typename C, bool THREE, bool FLUX, bool XF, typename... A>
void launch_div_rfft_rows(int nb, int nt, size_t smem, cudaStream_t st, A... a) {
    if constexpr (FLUX && sizeof(T) == 4)
        k_div_rfft_rows_flux<T, C, THREE, FLUX, XF><<<nb, nt, smem, st>>>(a...);
    else
        k_div_rfft_rows<T, C, THREE, FLUX, XF><<<nb, nt, smem, st>>>(a...);
}

// The type-II DCT of whole x rows in one pass (inflow/outflow x): the row is read, placed in
// the Makhoul order v[n/2] = x[n] (n even), v[N-1-(n-1)/2] = x[n] (n odd) in shared memory,
// transformed there as M complex pairs, and X_k = cos(pi k/2N) Re V_k + sin(pi k/2N) Im V_k,
// with V_k = conj V_{N-k} above N/2, is written back over the row.  Replaces the reorder
// pass, cuFFT's R2C and the twiddle pass (three trips through HBM).
template <typename T, typename C>
__global__ void __launch_bounds__(256) k_dct_rows(FftPlan pl, long long rows, T* __restrict__ x,
                                                  const C* __restrict__ tab, const T* __restrict__ tw) {
    extern __shared__ unsigned char fft_smem[];
    const int M = pl.M, N = 2 * pl.M;
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const long long row = (long long)blockIdx.x * (blockDim.x >> 5) + wq;
    C* b0 = reinterpret_cast<C*>(fft_smem) + (size_t)wq * 3 * fft_ps(M);
    C* b1 = b0 + fft_ps(M);
    C* b2 = b1 + fft_ps(M);                               // M + 2 values
    if (row >= rows) return;
    T* xr = x + row * N;
    T* v = reinterpret_cast<T*>(b2);
    for (int n = lane; n < N; n += 32) v[pzr((n & 1) ? N - 1 - (n >> 1) : (n >> 1))] = xr[n];
    __syncwarp();
    const C* Z = warp_fft_any<-1, C>(pl, reinterpret_cast<const C*>(v), b0, b1, tab);
    // V_k, k = 0..M, into the other buffer (the one Z is not in), then the twiddle
    C* V = (Z == b0) ? b1 : b0;
    const C* twN = tab + M;
    for (int k = lane; k < M; k += 32) {
        const C zk = Z[pz(k)];
        const C zc = cconj(Z[pz(k == 0 ? 0 : M - k)]);
        const C e = C{(zk.x + zc.x) * (T)0.5, (zk.y + zc.y) * (T)0.5};
        const C d = C{(zk.x - zc.x) * (T)0.5, (zk.y - zc.y) * (T)0.5};
        V[pz(k)] = cadd(e, cmul(twN[k], C{d.y, -d.x}));
    }
    const C z0 = Z[0];                                    // V_M = Re Z_0 - Im Z_0 (real)
    __syncwarp();
    const C* tw2 = reinterpret_cast<const C*>(tw);        // (cos, sin) pairs, one load each
#pragma unroll 4
    for (int k = lane; k < N; k += 32) {
        const C t = tw2[k];
        C vk;
        if (k < M) vk = V[pz(k)];
        else if (k == M) vk = C{z0.x - z0.y, (T)0};
        else { vk = V[pz(N - k)]; vk.y = -vk.y; }
        xr[k] = t.x * vk.x + t.y * vk.y;
    }
}

// The inverse: V_k = (c a + s b, s a - c b) from a = X_k, b = X_{N-k} (0 at k = 0), the
// unnormalised inverse real transform of V, and x[n] = v[pos(n)] written back over the row.
template <typename T, typename C>
__global__ void __launch_bounds__(256) k_idct_rows(FftPlan pl, long long rows, T* __restrict__ x,
                                                   const C* __restrict__ tab, const T* __restrict__ tw) {
    extern __shared__ unsigned char fft_smem[];
    const int M = pl.M, N = 2 * pl.M;
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const long long row = (long long)blockIdx.x * (blockDim.x >> 5) + wq;
    C* b0 = reinterpret_cast<C*>(fft_smem) + (size_t)wq * 3 * fft_ps(M);
    C* b1 = b0 + fft_ps(M);
    C* b2 = b1 + fft_ps(M);                               // V_0..V_M
    if (row >= rows) return;
    T* xr = x + row * N;
    const C* tw2 = reinterpret_cast<const C*>(tw);        // (cos, sin) pairs, one load each
#pragma unroll 4
    for (int k = lane; k <= M; k += 32) {
        const T a = xr[k];
        const T b = k == 0 ? T(0) : xr[N - k];
        const C t = tw2[k];
        const T c = t.x, sn = t.y;
        b2[pz(k)] = C{c * a + sn * b, sn * a - c * b};
    }
    __syncwarp();
    // the pre-processing of the inverse real transform, into b0
    const C* twN = tab + M;
    for (int k = lane; k < M; k += 32) {
        const C xk = b2[pz(k)];
        const C xc = cconj(b2[pz(M - k)]);
        const C e = cadd(xk, xc);
        const C d = cmul(csub(xk, xc), cconj(twN[k]));
        b0[pz(k)] = cadd(e, C{-d.y, d.x});
    }
    __syncwarp();
    // the transform reads b0 and alternates between b1 and b2 (V is no longer needed)
    const C* z = warp_fft_any<+1, C>(pl, b0, b1, b2, tab);
    const T* v = reinterpret_cast<const T*>(z);
    __syncwarp();
    for (int n = lane; n < N; n += 32) xr[n] = v[pzr((n & 1) ? N - 1 - (n >> 1) : (n >> 1))];
}

template <typename T>
__global__ void k_fft_tables(int M, T* __restrict__ tab) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < M) {
        double sn, cs;
        sincospi(2.0 * t / M, &sn, &cs);
        tab[2 * t] = (T)cs;
        tab[2 * t + 1] = (T)(-sn);
    }
    if (t <= M) {
        double sn, cs;
        sincospi((double)t / M, &sn, &cs);                  // 2 pi t / (2M)
        tab[2 * (M + t)] = (T)cs;
        tab[2 * (M + t) + 1] = (T)(-sn);
    }
}

// Dynamic shared memory of the row kernels: the FP32 inverse rows opt in to 64 KB (512-point rows
// then take eight warps a block, four blocks per SM, where 48 KB held seven: C4 inverse 0.238 ->
// 0.232 ms, the 1536-point rows of C2 0.0195 -> 0.0184); the forward rows keep 48 KB (the fused
// divergence with the DCT rows went 0.231 -> 0.252 ms with 64), and so do FP64 rows, where more rows
// per block would cost blocks per SM at their register count.
inline size_t row_smem_limit(size_t csz, bool inverse) { return csz == 8 && inverse ? 64 * 1024 : 48 * 1024; }

// rows per block of the row kernels (three padded row buffers per warp)
inline int fft_rows_per_block(int M, size_t csz, bool inverse = false) {
    const size_t per = 3 * (size_t)fft_ps(M) * csz;
    int r = (int)(row_smem_limit(csz, inverse) / per);
    return r < 1 ? 1 : (r > 8 ? 8 : r);
}

template <typename T, typename C>
void dct_rows(ibm_solver* h, T* x, bool inverse);

template <typename C>
ibm_status own_rfft(ibm_solver* h, const void* in, void* out, bool inverse) {
    const GridP& g = h->gp;
    FftPlan pl;
    pl.M = g.nx / 2;
    pl.nrad = h->fft_nrad;
    for (int s = 0; s < 16; ++s) pl.rad[s] = h->fft_rad[s];
    const long long rows = (long long)g.ny * g.nz;
    const int rpb = fft_rows_per_block(pl.M, sizeof(C), inverse);
    const size_t smem = 3 * (size_t)fft_ps(pl.M) * sizeof(C) * rpb;
    const int nb = (int)((rows + rpb - 1) / rpb);
    if (inverse)
        k_irfft_rows<C><<<nb, 32 * rpb, smem, h->stream>>>(pl, rows, (const C*)in, (C*)out, (const C*)h->fftab);
    else
        k_rfft_rows<C><<<nb, 32 * rpb, smem, h->stream>>>(pl, rows, (const C*)in, (C*)out, (const C*)h->fftab);
    IBM_LAUNCH_CHECK();
    return IBM_OK;
}

template <typename T, typename C>
void dct_rows(ibm_solver* h, T* x, bool inverse) {
    const GridP& g = h->gp;
    FftPlan pl;
    pl.M = g.nx / 2;
    pl.nrad = h->fft_nrad;
    for (int q = 0; q < 16; ++q) pl.rad[q] = h->fft_rad[q];
    const long long rows = (long long)g.ny * g.nz;
    const int rpb = fft_rows_per_block(pl.M, sizeof(C), inverse);
    const size_t smem = 3 * (size_t)fft_ps(pl.M) * sizeof(C) * rpb;
    const int nb = (int)((rows + rpb - 1) / rpb);
    if (inverse)
        k_idct_rows<T, C><<<nb, 32 * rpb, smem, h->stream>>>(pl, rows, x, (const C*)h->fftab, (const T*)h->twid);
    else
        k_dct_rows<T, C><<<nb, 32 * rpb, smem, h->stream>>>(pl, rows, x, (const C*)h->fftab, (const T*)h->twid);
}


template <typename T, typename C>
__global__ void k_dct_post(GridP g, const C* __restrict__ V, T* __restrict__ X, const T* __restrict__ tw) {
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    const int k = (int)(id % g.nx);
    const long long row = id / g.nx;
    const int nxr = g.nx / 2 + 1;
    C v;
    if (k < nxr) {
        v = V[row * nxr + k];
    } else {
        v = V[row * nxr + g.nx - k];
        v.y = -v.y;
    }
    X[id] = tw[2 * k] * v.x + tw[2 * k + 1] * v.y;
}

template <typename T, typename C>
__global__ void k_idct_pre(GridP g, const T* __restrict__ X, C* __restrict__ V, const T* __restrict__ tw) {
    const int nxr = g.nx / 2 + 1;
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= (long long)g.ny * g.nz * nxr) return;
    const int k = (int)(id % nxr);
    const long long row = id / nxr;
    const T a = X[row * g.nx + k];
    const T b = k == 0 ? T(0) : X[row * g.nx + g.nx - k];
    const T c = tw[2 * k], sn = tw[2 * k + 1];
    C v;
    v.x = c * a + sn * b;
    v.y = sn * a - c * b;
    V[id] = v;
}

template <typename T, typename C>
__global__ void k_pack_real(long long n, const T* __restrict__ x, C* __restrict__ y) {
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= n) return;
    C v;
    v.x = x[id];
    v.y = T(0);
    y[id] = v;
}

template <typename T, typename C>
__global__ void k_unpack_real(long long n, const C* __restrict__ y, T* __restrict__ x) {
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= n) return;
    x[id] = y[id].x;
}

// ---------------------------------------------------------------------------
// Convective outflow (inflow/outflow x), readings as in the header: on every
// fluid outflow face u_b = u(nx-1) the RK3 stage of du/dt = -U_c (u_b - u_{b-1})/dx,
// with the momentum stage's combination (dt a_k N + dt b_k N^{k-2}) and no
// pressure or IBM term; then one constant shift of all fluid outflow faces so
// that the outflow flux equals the inflow flux.  With update = 0 the first
// kernel only sums the present outflow values (initial projection).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_outflow(GridP g, const T* __restrict__ u, const uint8_t* __restrict__ mask,
                                                 T* __restrict__ us, T* __restrict__ Nh, T dta, T dtb, T ucx,
                                                 int read_prev, int write_n, int update, double* __restrict__ part) {
    __shared__ double sh[8];
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;   // row (j, k)
    double s = 0.0;
    if (r < (long long)g.ny * g.nz) {
        const long long ib = r * g.nx + g.nx - 1;
        const bool fluid = mask[ib] & IBM_MASK_FACE;
        if (update) {
            T o = T(0), Nb = T(0);
            if (fluid) {
                const T ub = u[ib];
                const T um = (mask[ib - 1] & IBM_MASK_U) ? u[ib - 1] : T(0);
                Nb = -ucx * (ub - um);
                T R = dta * Nb;
                if (read_prev) R += dtb * Nh[ib];
                o = ub + R;
            }
            us[ib] = o;
            if (write_n) Nh[ib] = Nb;
            s = (double)o;
        } else if (fluid) {
            s = (double)us[ib];
        }
        if (g.ystr) s *= ytab(g, YT_DYC, (int)(r % g.ny));   // the face's height (a flux, not a sum of speeds)
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

// Every block sums the partials itself (the same order in each, so all find the
// same shift) and shifts its own rows: one block looping over every row was
// bound by the latency of its strided accesses (72 us on 384 x 256 rows).
template <typename T>
__global__ void __launch_bounds__(256) k_outflow_fix(GridP g, const uint8_t* __restrict__ mask, T* __restrict__ us,
                                                     const double* __restrict__ part, int nparts, double qin,
                                                     double nout) {
    __shared__ double sh[8];
    __shared__ double shift;
    double s = 0.0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += part[b];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        shift = nout > 0.0 ? (qin - t) / nout : 0.0;
    }
    __syncthreads();
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;   // row (j, k)
    if (r < (long long)g.ny * g.nz) {
        const long long ib = r * g.nx + g.nx - 1;
        if (mask[ib] & IBM_MASK_FACE) us[ib] += (T)shift;
    }
}

template <typename T>
ibm_status poisson_t(ibm_solver* h, void* rhs_inout, bool x_done = false) {
    using C = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
    const GridP& g = h->gp;
    cudaEvent_t t;
    const int nbN = (int)((g.N + 255) / 256);
    auto fwd = [&](cufftHandle p, void* in, void* out) {
        return h->prec == IBM_FP64 ? cufftExecD2Z(p, (cufftDoubleReal*)in, (cufftDoubleComplex*)out)
                                   : cufftExecR2C(p, (cufftReal*)in, (cufftComplex*)out);
    };
    auto inv = [&](cufftHandle p, void* in, void* out) {
        return h->prec == IBM_FP64 ? cufftExecZ2D(p, (cufftDoubleComplex*)in, (cufftDoubleReal*)out)
                                   : cufftExecC2R(p, (cufftComplex*)in, (cufftReal*)out);
    };
    // x rows: the own kernels where the row length allows them, else cuFFT's R2C / C2R
    auto xfwd = [&](void* in, void* out) -> cufftResult {
        if (h->own_fft) return own_rfft<C>(h, in, out, false) == IBM_OK ? CUFFT_SUCCESS : CUFFT_EXEC_FAILED;
        return fwd(h->plan_f, in, out);
    };
    auto xinv = [&](void* in, void* out) -> cufftResult {
        if (h->own_fft) return own_rfft<C>(h, in, out, true) == IBM_OK ? CUFFT_SUCCESS : CUFFT_EXEC_FAILED;
        return inv(h->plan_i, in, out);
    };
    // in-place C2C along z over the half spectrum (periodic x, 3D)
    auto zc2c = [&](int dir) {
        return h->prec == IBM_FP64
                   ? cufftExecZ2Z(h->plan_fz, (cufftDoubleComplex*)h->spec, (cufftDoubleComplex*)h->spec, dir)
                   : cufftExecC2C(h->plan_fz, (cufftComplex*)h->spec, (cufftComplex*)h->spec, dir);
    };
    timer_begin(h, "fft_forward", &t);
    cufftResult r = CUFFT_SUCCESS;
    if (g.xper) {
        if (!x_done) r = xfwd(rhs_inout, h->spec);     // else the divergence kernel did the x rows
        if (r == CUFFT_SUCCESS && g.nz > 1) r = zc2c(CUFFT_FORWARD);
    } else {
        // DCT of the x rows into rhs, then (3D) the real FFT along z into the spectrum
        T* x = (T*)rhs_inout;
        if (x_done) {
            // the divergence kernel wrote the DCT coefficients of the rows
        } else if (h->dct_rows) {
            dct_rows<T, C>(h, x, false);                  // reorder, row FFT and twiddle in one pass
        } else {
            k_dct_reorder<T><<<nbN, 256, 0, h->stream>>>(g, x, (T*)h->rtmp, 0);
            IBM_LAUNCH_CHECK();
            r = xfwd(h->rtmp, h->spec);
            if (r == CUFFT_SUCCESS) {
                k_dct_post<T, C><<<nbN, 256, 0, h->stream>>>(g, (const C*)h->spec, x, (const T*)h->twid);
                IBM_LAUNCH_CHECK();
            }
        }
        if (r == CUFFT_SUCCESS) {
            if (g.nz > 1) {
                r = fwd(h->plan_fz, x, h->spec);
            } else {
                k_pack_real<T, C><<<nbN, 256, 0, h->stream>>>(g.N, x, (C*)h->spec);
                IBM_LAUNCH_CHECK();
            }
        }
    }
    if (r != CUFFT_SUCCESS) { h->failed = true; return ibm_set_error(IBM_E_CUDA, "cufft forward failed"); }
    timer_end(h, t, "fft_forward");
    double scale = g.dy * g.dy / ((double)g.nx * (double)g.nz);
    const int nsys = g.nzs * g.nxh;
    // a stretched y solves the symmetric unit off-diagonal form of its rows: the right-hand side
    // takes the per-row factor s_j dyc_j, the solution s_j, and the zero mode's gauge (the plain
    // mean of phi) is removed after that scaling
    const int gauge = g.ystr ? 0 : 1;
    const int nbs = (int)((h->nspec + 255) / 256);
    if (g.ystr) {
        scale = 1.0 / ((double)g.nx * (double)g.nz);
        k_spec_rows<C><<<nbs, 256, 0, h->stream>>>(g, (C*)h->spec, h->nspec, YT_PIN);
        IBM_LAUNCH_CHECK();
    }
    // FP64 systems: one warp each wherever the warp form covers ny (measured faster: all rows
    // of a system are loaded at once, where one thread per system waits on memory every few
    // rows), one thread each for taller grids or when asked
    const int thr64 = (g.ny > 32 * TW_ROWS || h->tri_form == 2) ? 1 : 0;
    const int nb64 = thr64 ? (h->n64 + 31) / 32 : h->n64;
    // FP32 systems: one warp each when one thread each would leave the GPU nearly idle
    const int warp32 = (h->prec == IBM_FP32 && g.ny <= 32 * TW_ROWS && nsys - h->n64 < 16384) ? 1 : 0;
    // one thread per FP32 system: those go to k_tridiag32 on the solver's stream, and the launch
    // below takes the FP64 ones on the second stream (forked and joined by events, so that a
    // captured step holds both as one fork-join)
    const int n32 = nsys - h->n64;
    const bool split32 = h->prec == IBM_FP32 && !warp32 && n32 > 0 && h->tri_stream;
    const int nblk = split32 ? nb64 : nb64 + (warp32 ? n32 : (n32 + 31) / 32);
    timer_begin(h, "tridiag", &t);
    cudaStream_t s64 = h->stream;
    if (split32 && nb64 > 0) {
        IBM_CUDA_TRY(cudaEventRecord(h->tri_fork, h->stream));
        IBM_CUDA_TRY(cudaStreamWaitEvent(h->tri_stream, h->tri_fork, 0));
        s64 = h->tri_stream;
    }
    if (split32) {
        k_tridiag32<<<(n32 + 127) / 128, 128, 0, h->stream>>>(g, (float2*)h->spec, h->pivots32, h->sys_order,
                                                              h->n64, nsys, scale);
        IBM_LAUNCH_CHECK();
    }
    // rows per lane of the warp path, rounded up to a compiled size
#define IBM_TRIDIAG(RR)                                                                                          \
    do {                                                                                                         \
        if (h->prec == IBM_FP64)                                                                                 \
            k_tridiag<double2, RR><<<nblk, 32, 0, s64>>>(g, (double2*)h->spec, (double2*)h->spec, h->pivots,       \
                                                               h->pivots32, h->sys_order, h->n64, nsys, scale, warp32, thr64, gauge); \
        else                                                                                                     \
            k_tridiag<float2, RR><<<nblk, 32, 0, s64>>>(g, (float2*)h->spec, (double2*)h->dtemp, h->pivots,        \
                                                              h->pivots32, h->sys_order, h->n64, nsys, scale, warp32, thr64, gauge); \
    } while (0)
    if (nblk > 0) {
        if (g.ny <= 32 * 8) IBM_TRIDIAG(8);
        else if (g.ny <= 32 * 16) IBM_TRIDIAG(16);
        else if (g.ny <= 32 * 24) IBM_TRIDIAG(24);
        else if (g.ny <= 32 * 32) IBM_TRIDIAG(32);
        else IBM_TRIDIAG(0);
        IBM_LAUNCH_CHECK();
    }
#undef IBM_TRIDIAG
    if (s64 != h->stream) {
        IBM_CUDA_TRY(cudaEventRecord(h->tri_join, s64));
        IBM_CUDA_TRY(cudaStreamWaitEvent(h->stream, h->tri_join, 0));
    }
    if (g.ystr) {
        k_spec_rows<C><<<nbs, 256, 0, h->stream>>>(g, (C*)h->spec, h->nspec, YT_POUT);
        IBM_LAUNCH_CHECK();
        k_zero_gauge<C><<<1, 256, 0, h->stream>>>(g, (C*)h->spec);
        IBM_LAUNCH_CHECK();
    }
    timer_end(h, t, "tridiag");
    timer_begin(h, "fft_inverse", &t);
    if (g.xper) {
        if (g.nz > 1) r = zc2c(CUFFT_INVERSE);
        if (r == CUFFT_SUCCESS) r = xinv(h->spec, rhs_inout);
    } else {
        T* x = (T*)rhs_inout;
        if (g.nz > 1) {
            r = inv(h->plan_iz, h->spec, x);
        } else {
            k_unpack_real<T, C><<<nbN, 256, 0, h->stream>>>(g.N, (const C*)h->spec, x);
            IBM_LAUNCH_CHECK();
        }
        if (r == CUFFT_SUCCESS && h->dct_rows) {
            dct_rows<T, C>(h, x, true);
        } else if (r == CUFFT_SUCCESS) {
            const long long nh = (long long)g.ny * g.nz * (g.nx / 2 + 1);
            k_idct_pre<T, C><<<(int)((nh + 255) / 256), 256, 0, h->stream>>>(g, x, (C*)h->spec, (const T*)h->twid);
            IBM_LAUNCH_CHECK();
            r = xinv(h->spec, h->rtmp);
            if (r == CUFFT_SUCCESS) {
                k_dct_reorder<T><<<nbN, 256, 0, h->stream>>>(g, (const T*)h->rtmp, x, 1);
                IBM_LAUNCH_CHECK();
            }
        }
    }
    if (r != CUFFT_SUCCESS) { h->failed = true; return ibm_set_error(IBM_E_CUDA, "cufft inverse failed"); }
    timer_end(h, t, "fft_inverse");
    return IBM_OK;
}

dim3 zmarch_grid(const GridP& g) {
    return dim3(g.nsegx, (g.ny + 7) / 8, g.ndim == 3 ? (g.nz + g.kzd - 1) / g.kzd : 1);
}

template <typename T>
FluxCorr<T> flux_corr(ibm_solver* h, int k) {
    FluxCorr<T> fc;
    fc.scal = h->scal;
    fc.ckdt = (T)(h->phys.dt * RK_C[k]);
    fc.segoff = h->segoff[0];
    fc.coef = (const Coef4<T>*)h->coef[0] + (long long)k * h->counts[0];
    return fc;
}

// ---------------------------------------------------------------------------
// Masked projection (IBM_PROJ_MASKED): conjugate gradients on A' = -D M G over the
// internal cells, preconditioned with the full-box solve (z = -(D G)^{-1} r), FP64
// vectors that are zero outside the internal cells.  Block partial sums of the inner
// products go to h->partials; the host adds them in a fixed order.
// ---------------------------------------------------------------------------
constexpr int PCG_BLOCKS = 4 * 152;

__device__ __forceinline__ double block_sum256(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < 8; ++w) t += sh[w];
    return t;
}

// b = -(D u*) on the internal cells; x = 0; r = b; partial sums of r.r
template <typename T>
__global__ void __launch_bounds__(256) k_pcg_init(long long N, const uint8_t* __restrict__ mask,
                                                  const T* __restrict__ rhs, double* __restrict__ x,
                                                  double* __restrict__ r, double* __restrict__ part) {
    __shared__ double sh[8];
    double s = 0.0;
    for (long long id = blockIdx.x * 256LL + threadIdx.x; id < N; id += (long long)gridDim.x * 256) {
        const double b = (mask[id] & IBM_MASK_P) ? -(double)rhs[id] : 0.0;
        x[id] = 0.0;
        r[id] = b;
        s += b * b;
    }
    s = block_sum256(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// y = -(D M G x) on the internal cells (zero elsewhere); partial sums of x.y
__global__ void __launch_bounds__(256) k_pcg_matvec(GridP g, const uint8_t* __restrict__ mask,
                                                    const double* __restrict__ x, double* __restrict__ y,
                                                    double* __restrict__ part) {
    __shared__ double sh[8];
    double s = 0.0;
    const double inv2[3] = {1.0 / (g.dx * g.dx), 1.0 / (g.dy * g.dy), 1.0 / (g.dz * g.dz)};
    for (long long id = blockIdx.x * 256LL + threadIdx.x; id < g.N; id += (long long)gridDim.x * 256) {
        const uint32_t m = mask[id];
        double out = 0.0;
        if (m & IBM_MASK_P) {
            const int i = (int)(id % g.nx);
            const int j = (int)((id / g.nx) % g.ny);
            const int k = (int)(id / ((long long)g.nx * g.ny));
            const double xc = x[id];
            double acc = 0.0;
            for (int d = 0; d < g.ndim; ++d) {
                const int n = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
                const int q = d == 0 ? i : (d == 1 ? j : k);
                const long long st = d == 0 ? 1 : (d == 1 ? (long long)g.nx : (long long)g.nx * g.ny);
                const bool per = d == 2 || (d == 0 && g.xper);
                // +d face: the velocity point of this cell
                if ((m >> d) & 1u) {
                    const long long ip = q + 1 < n ? id + st : id - (long long)(n - 1) * st;
                    acc += (x[ip] - xc) * inv2[d];
                }
                // -d face: the velocity point of the cell below
                if (q > 0 || per) {
                    const long long im = q > 0 ? id - st : id + (long long)(n - 1) * st;
                    if ((mask[im] >> d) & 1u) acc -= (xc - x[im]) * inv2[d];
                }
            }
            out = -acc;
        }
        y[id] = out;
        s += x[id] * out;
    }
    s = block_sum256(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// x += alpha p; r -= alpha Ap; partial sums of r.r
__global__ void __launch_bounds__(256) k_pcg_update(long long N, double alpha, double* __restrict__ x,
                                                    double* __restrict__ r, const double* __restrict__ p,
                                                    const double* __restrict__ Ap, double* __restrict__ part) {
    __shared__ double sh[8];
    double s = 0.0;
    for (long long id = blockIdx.x * 256LL + threadIdx.x; id < N; id += (long long)gridDim.x * 256) {
        x[id] += alpha * p[id];
        const double rn = r[id] - alpha * Ap[id];
        r[id] = rn;
        s += rn * rn;
    }
    s = block_sum256(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// the preconditioner's input: -r in the grid precision
template <typename T>
__global__ void k_pcg_to_field(long long N, const double* __restrict__ r, T* __restrict__ f) {
    for (long long id = blockIdx.x * 256LL + threadIdx.x; id < N; id += (long long)gridDim.x * 256)
        f[id] = (T)(-r[id]);
}

// z = the full-box solution on the internal cells (0 elsewhere); partial sums of z.r and z.Ap
template <typename T>
__global__ void __launch_bounds__(256) k_pcg_from_field(long long N, const uint8_t* __restrict__ mask,
                                                        const T* __restrict__ f, double* __restrict__ z,
                                                        const double* __restrict__ r, const double* __restrict__ Ap,
                                                        double* __restrict__ part, int nb) {
    __shared__ double sh[8];
    double s1 = 0.0, s2 = 0.0;
    for (long long id = blockIdx.x * 256LL + threadIdx.x; id < N; id += (long long)gridDim.x * 256) {
        const double v = (mask[id] & IBM_MASK_P) ? (double)f[id] : 0.0;
        z[id] = v;
        s1 += v * r[id];
        s2 += v * Ap[id];
    }
    s1 = block_sum256(s1, sh);
    __syncthreads();
    s2 = block_sum256(s2, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s1;
        part[nb + blockIdx.x] = s2;
    }
}

__global__ void k_pcg_direction(long long N, double beta, const double* __restrict__ z, double* __restrict__ p) {
    for (long long id = blockIdx.x * 256LL + threadIdx.x; id < N; id += (long long)gridDim.x * 256)
        p[id] = z[id] + beta * p[id];
}

template <typename T>
__global__ void k_pcg_out(long long N, const double* __restrict__ x, T* __restrict__ f) {
    for (long long id = blockIdx.x * 256LL + threadIdx.x; id < N; id += (long long)gridDim.x * 256)
        f[id] = (T)x[id];
}

// reads back nsum groups of nb block partials and adds each group in order
ibm_status pcg_sums(ibm_solver* h, int nb, int nsum, double* out) {
    std::vector<double> buf((size_t)nb * nsum);
    IBM_CUDA_TRY(cudaMemcpyAsync(buf.data(), h->partials, buf.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                 h->stream));
    IBM_CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int q = 0; q < nsum; ++q) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += buf[(size_t)q * nb + b];
        out[q] = s;
    }
    return IBM_OK;
}

// D M G psi = rhs over the internal cells; rhs (the divergence, grid precision) in h->rhs is
// replaced by psi.  Host-driven: one read-back of inner products per iteration.
template <typename T>
ibm_status masked_solve_t(ibm_solver* h) {
    const GridP& g = h->gp;
    const int nb = std::min(PCG_BLOCKS, h->npartials / 2);
    double* x = h->pcg[0];
    double* r = h->pcg[1];
    double* z = h->pcg[2];
    double* p = h->pcg[3];
    double* Ap = h->pcg[4];
    T* f = (T*)h->rhs;
    double sums[2];
    k_pcg_init<T><<<nb, 256, 0, h->stream>>>(g.N, h->mask, f, x, r, h->partials);
    IBM_LAUNCH_CHECK();
    ibm_status st = pcg_sums(h, nb, 1, sums);
    if (st != IBM_OK) return st;
    const double bnorm = std::sqrt(sums[0]);
    int it = 0;
    double rr = sums[0];
    auto precondition = [&](bool with_ap) -> ibm_status {
        k_pcg_to_field<T><<<nb, 256, 0, h->stream>>>(g.N, r, f);
        IBM_LAUNCH_CHECK();
        ibm_status s2 = poisson_t<T>(h, f);
        if (s2 != IBM_OK) return s2;
        k_pcg_from_field<T><<<nb, 256, 0, h->stream>>>(g.N, h->mask, f, z, r, with_ap ? Ap : r, h->partials, nb);
        IBM_LAUNCH_CHECK();
        return pcg_sums(h, nb, 2, sums);
    };
    if (bnorm > 0.0 && std::isfinite(bnorm)) {
        st = precondition(false);
        if (st != IBM_OK) return st;
        double rz = sums[0];
        k_pcg_direction<<<nb, 256, 0, h->stream>>>(g.N, 0.0, z, p);
        IBM_LAUNCH_CHECK();
        double best = rr;
        int best_it = 0;
        for (it = 1; it <= h->proj_maxit; ++it) {
            k_pcg_matvec<<<nb, 256, 0, h->stream>>>(g, h->mask, p, Ap, h->partials);
            IBM_LAUNCH_CHECK();
            if ((st = pcg_sums(h, nb, 1, sums)) != IBM_OK) return st;
            const double pAp = sums[0];
            if (!(pAp > 0.0)) break;                      // the search direction vanished
            const double alpha = rz / pAp;
            k_pcg_update<<<nb, 256, 0, h->stream>>>(g.N, alpha, x, r, p, Ap, h->partials);
            IBM_LAUNCH_CHECK();
            if ((st = pcg_sums(h, nb, 1, sums)) != IBM_OK) return st;
            rr = sums[0];
            if (!std::isfinite(rr) || std::sqrt(rr) <= h->proj_tol * bnorm) break;
            // stagnation at the round-off floor (the right-hand side sums to zero over each
            // group of internal cells only to round-off): stop after 25 iterations without gain
            if (rr < best) {
                best = rr;
                best_it = it;
            } else if (it - best_it > 25) {
                break;
            }
            if ((st = precondition(true)) != IBM_OK) return st;
            // Polak-Ribiere: z_new.(r_new - r_old) / rz_old = -alpha z_new.Ap / rz_old
            const double beta = -alpha * sums[1] / rz;
            rz = sums[0];
            k_pcg_direction<<<nb, 256, 0, h->stream>>>(g.N, beta, z, p);
            IBM_LAUNCH_CHECK();
        }
    } else {
        rr = 0.0;
    }
    h->proj_iters = std::min(it, h->proj_maxit);
    h->proj_resid = bnorm > 0.0 ? std::sqrt(rr) / bnorm : 0.0;
    k_pcg_out<T><<<nb, 256, 0, h->stream>>>(g.N, x, f);
    IBM_LAUNCH_CHECK();
    return IBM_OK;
}

// u = u* - G psi on the internal faces only (+ the constant-flow-rate increment at internal
// u points), u = u* on every other face; p += psi / (c_k dt)
template <typename T, bool FLUX>
__global__ void k_correct_masked(GridP g, const T* __restrict__ us0, const T* __restrict__ us1,
                                 const T* __restrict__ us2, const T* __restrict__ psi, const uint8_t* __restrict__ mask,
                                 T* __restrict__ u0, T* __restrict__ u1, T* __restrict__ u2, T* __restrict__ p, T idx,
                                 T idy, T idz, T inv_ckdt, int update_p, FluxCorr<T> fc) {
    const int lane = threadIdx.x;
    const int i = blockIdx.x * 32 + lane;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    if (j >= g.ny) return;                                   // whole warp
    const bool live = i < g.nx;
    const long long id = live ? i + (long long)g.nx * (j + (long long)g.ny * k) : 0;
    const uint32_t m = live ? mask[id] : 0u;
    T uc = T(0);
    if (FLUX) {
        const T pic = *reinterpret_cast<const T*>(fc.scal + 2) * fc.ckdt;
        const unsigned b = __ballot_sync(0xffffffffu, (m & IBM_MASK_IBM_U) != 0);
        if (live) uc = flux_increment(fc, pic, (uint8_t)m, b, (j + g.ny * k) * g.nsegx + (int)blockIdx.x, lane);
    }
    if (!live) return;
    const T pc = psi[id];
    if (m & IBM_MASK_U) {
        const long long ie = i + 1 < g.nx ? id + 1 : id - (g.nx - 1);
        u0[id] = us0[id] + uc - (psi[ie] - pc) * idx;
    } else {
        u0[id] = us0[id];
    }
    if (m & IBM_MASK_V) u1[id] = us1[id] - (psi[id + g.nx] - pc) * idy;   // internal v: j + 1 < ny
    else u1[id] = us1[id];
    if (g.ndim == 3) {
        const long long plane = (long long)g.nx * g.ny;
        if (m & IBM_MASK_W) {
            const long long it = k + 1 < g.nz ? id + plane : id - (long long)(g.nz - 1) * plane;
            u2[id] = us2[id] - (psi[it] - pc) * idz;
        } else {
            u2[id] = us2[id];
        }
    }
    if (update_p) p[id] = p[id] + pc * inv_ckdt;
}

template <typename T>
ibm_status divergence_and_solve(ibm_solver* h, T* const us[3], bool flux, const FluxCorr<T>& fc) {
    const GridP& g = h->gp;
    cudaEvent_t t;
    // (a stretched y keeps the divergence separate: the fused kernel has no per-row metric)
    const bool fuse_x = (g.xper ? h->own_fft : h->dct_rows) && !g.ystr;
    if (fuse_x && h->proj_mode != IBM_PROJ_MASKED) {
        // the divergence fused with the forward transform of the x rows (own real FFT on a periodic
        // x, own DCT rows on an inflow/outflow x)
        using C = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
        timer_begin(h, "div_fft_x", &t);
        const T ix = (T)(1.0 / g.dx), iy = (T)(1.0 / g.dy), iz = (T)(1.0 / g.dz);
        T* w = g.ndim == 3 ? us[2] : us[0];
        FftPlan pl;
        pl.M = g.nx / 2;
        pl.nrad = h->fft_nrad;
        for (int q = 0; q < 16; ++q) pl.rad[q] = h->fft_rad[q];
        const long long rows = (long long)g.ny * g.nz;
        // the FP32 flow-rate instance in blocks of four rows (eight blocks of four warps per SM):
        // 0.1047 -> 0.1020 ms on 384 x 256 x 256; the DCT instance keeps its seven (4, 5, 6 rows:
        // 0.246, 0.252, 0.252 against 0.229 ms on 512 x 384 x 256)
        const int rpb = (flux && g.xper && sizeof(T) == 4) ? std::min(4, fft_rows_per_block(pl.M, sizeof(C)))
                                                           : fft_rows_per_block(pl.M, sizeof(C));
        const size_t smem = 3 * (size_t)fft_ps(pl.M) * sizeof(C) * rpb;
        const int nb = (int)((rows + rpb - 1) / rpb);
        C* out = (C*)h->spec;
        const C* tab = (const C*)h->fftab;
        T* xo = (T*)h->rhs;
        const T* twd = (const T*)h->twid;
#define IBM_DIVFFT(THREE_, FLUX_, XF_)                                                                          \
    launch_div_rfft_rows<T, C, THREE_, FLUX_, XF_>(nb, 32 * rpb, smem, h->stream, g, us[0], us[1], w, h->mask, fc, \
                                                     ix, iy, iz, pl, out, tab, xo, twd)
        if (!g.xper) {   // inflow/outflow x (no constant flow rate)
            if (g.ndim == 3) IBM_DIVFFT(true, false, true);
            else IBM_DIVFFT(false, false, true);
        } else if (g.ndim == 3) {
            if (flux) IBM_DIVFFT(true, true, false);
            else IBM_DIVFFT(true, false, false);
        } else {
            if (flux) IBM_DIVFFT(false, true, false);
            else IBM_DIVFFT(false, false, false);
        }
#undef IBM_DIVFFT
        IBM_LAUNCH_CHECK();
        timer_end(h, t, "div_fft_x");
        return poisson_t<T>(h, h->rhs, true);
    }
    timer_begin(h, "divergence", &t);
    const T ix = (T)(1.0 / g.dx), iy = (T)(1.0 / g.dy), iz = (T)(1.0 / g.dz);
    const dim3 grd = zmarch_grid(g), blk(32, 8);
    T* rhs = (T*)h->rhs;
    T* w = g.ndim == 3 ? us[2] : us[0];
    if (!g.xper) {   // inflow/outflow x (no constant flow rate)
        if (g.ndim == 3) k_divergence<T, true, false, true><<<grd, blk, 0, h->stream>>>(g, us[0], us[1], w, h->mask, rhs, ix, iy, iz, fc);
        else k_divergence<T, false, false, true><<<grd, blk, 0, h->stream>>>(g, us[0], us[1], w, h->mask, rhs, ix, iy, iz, fc);
    } else if (g.ndim == 3) {
        if (flux) k_divergence<T, true, true, false><<<grd, blk, 0, h->stream>>>(g, us[0], us[1], w, h->mask, rhs, ix, iy, iz, fc);
        else k_divergence<T, true, false, false><<<grd, blk, 0, h->stream>>>(g, us[0], us[1], w, h->mask, rhs, ix, iy, iz, fc);
    } else {
        if (flux) k_divergence<T, false, true, false><<<grd, blk, 0, h->stream>>>(g, us[0], us[1], w, h->mask, rhs, ix, iy, iz, fc);
        else k_divergence<T, false, false, false><<<grd, blk, 0, h->stream>>>(g, us[0], us[1], w, h->mask, rhs, ix, iy, iz, fc);
    }
    IBM_LAUNCH_CHECK();
    timer_end(h, t, "divergence");
    if (h->proj_mode == IBM_PROJ_MASKED) {
        timer_begin(h, "masked_solve", &t);
        ibm_status st = masked_solve_t<T>(h);
        if (st != IBM_OK) return st;
        timer_end(h, t, "masked_solve");
        return IBM_OK;
    }
    return poisson_t<T>(h, h->rhs);
}

template <typename T>
ibm_status launch_correct(ibm_solver* h, T* const us[3], T inv_ckdt, int update_p, bool flux, const FluxCorr<T>& fc) {
    const GridP& g = h->gp;
    const T ix = (T)(1.0 / g.dx), iy = (T)(1.0 / g.dy), iz = (T)(1.0 / g.dz);
    const dim3 grd = zmarch_grid(g), blk(32, 8);
    const T* psi = (const T*)h->rhs;
    T* u0 = (T*)h->buf.u[0];
    T* u1 = (T*)h->buf.u[1];
    T* u2 = g.ndim == 3 ? (T*)h->buf.u[2] : u0;
    T* us2 = g.ndim == 3 ? us[2] : us[0];
    T* p = (T*)h->buf.p;
    if (h->proj_mode == IBM_PROJ_MASKED) {
        const dim3 cg = cell_grid(g);
        if (flux)
            k_correct_masked<T, true><<<cg, blk, 0, h->stream>>>(g, us[0], us[1], us2, psi, h->mask, u0, u1, u2, p, ix, iy,
                                                                 iz, inv_ckdt, update_p, fc);
        else
            k_correct_masked<T, false><<<cg, blk, 0, h->stream>>>(g, us[0], us[1], us2, psi, h->mask, u0, u1, u2, p, ix,
                                                                  iy, iz, inv_ckdt, update_p, fc);
        IBM_LAUNCH_CHECK();
        return IBM_OK;
    }
#define IBM_CORRECT(THREE_, FLUX_, XF_)                                                                        \
    k_correct<T, THREE_, FLUX_, XF_><<<grd, blk, 0, h->stream>>>(g, us[0], us[1], us2, psi, h->mask, u0, u1, u2, p, \
                                                                 ix, iy, iz, inv_ckdt, update_p, fc)
    if (!g.xper) {   // inflow/outflow x (no constant flow rate)
        if (g.ndim == 3) IBM_CORRECT(true, false, true);
        else IBM_CORRECT(false, false, true);
    } else if (g.ndim == 3) {
        if (flux) IBM_CORRECT(true, true, false);
        else IBM_CORRECT(true, false, false);
    } else {
        if (flux) IBM_CORRECT(false, true, false);
        else IBM_CORRECT(false, false, false);
    }
#undef IBM_CORRECT
    IBM_LAUNCH_CHECK();
    return IBM_OK;
}


// ---------------------------------------------------------------------------
// Force of the fluid on the body (diagnostic, per substage): the body's share
// of the discrete momentum budget of the internal points.  Per IBM point P of
// component c:
//   I  = -x u* + (1 - B)(u* - u)   what the implicit division adds to u* - u
//        beyond the explicit R (from (B + x) u* = B u + R)
//   BN = wall source + over the arms toward external points: -s F / D_d
//        + nu (0 - u) / D_d^2, F the face's convective flux as the right-hand
//        side forms it (the external value reads 0)
//   PQ = over the arms along c: +q(cell P + e_c) (s = +1), -q(cell P) (s = -1),
//        q = p + psi / (c_k dt) the new pressure (the solve returns psi = c_k dt phi),
//        the pressure at the end of a run of internal points
// A final single block turns the sums into the stage's impulse
//   dV (sum I - c_k dt PQ / D_c + dt (a_k BN + b_k BN_prev))
// and, after the third stage, adds -impulse / dt to the force sums.
// ---------------------------------------------------------------------------
template <typename T>
struct BodyArgs {
    GridP g;
    const T* u[3];
    const T* us[3];
    const T* p;
    const T* psi;            // c_k dt phi
    const uint8_t* mask;
    const int* idx[3];
    const double* lam[3];
    const double* src[3];
    int cnt[3];
    double ckdt, inv_ckdt, nu;
    int bmode;
    double* part;
};

// value of component d at (i, j, k) as the right-hand side reads it (0 unless
// internal or the fluid outflow face of u); i may be nx or -1 only in a periodic x
template <typename T>
__device__ __forceinline__ double body_rd(const BodyArgs<T>& a, int d, int i, int j, int k) {
    const GridP& g = a.g;
    if (g.xper) i = (i + g.nx) % g.nx;
    if (g.ndim == 3) k = (k + g.nz) % g.nz;
    const long long l = i + (long long)g.nx * (j + (long long)g.ny * k);
    const uint32_t m = a.mask[l];
    bool rd = (m >> d) & 1u;
    if (d == 0 && !g.xper && i == g.nx - 1) rd = (m & IBM_MASK_FACE) != 0;
    return rd ? (double)a.u[d][l] : 0.0;
}

template <typename T>
__global__ void __launch_bounds__(256) k_body_force(BodyArgs<T> a) {
    const GridP& g = a.g;
    const int c = blockIdx.y;
    double sI = 0.0, sBN = 0.0, sPQ = 0.0;
    const int nd = g.ndim;
    const double D[3] = {g.dx, g.dy, g.dz};
    const int n[3] = {g.nx, g.ny, g.nz};
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < a.cnt[c]; m += gridDim.x * blockDim.x) {
        const long long lin = a.idx[c][m];
        const int pi = (int)(lin % g.nx);
        const int pj = (int)((lin / g.nx) % g.ny);
        const int pk = (int)(lin / ((long long)g.nx * g.ny));
        const double u0 = (double)a.u[c][lin];
        const double us = (double)a.us[c][lin];
        if (a.bmode == IBM_B_EXPLICIT) {
            // -lambda u is part of N; the update has no division (I = 0)
            sBN += a.src[c][m] - a.lam[c][m] * u0;
        } else {
            const double x = a.lam[c][m] * a.ckdt;
            const double B = ibm_B_of_x(x, a.bmode);
            sI += -x * us + (1.0 - B) * (us - u0);
            sBN += a.src[c][m];
        }
        const int P[3] = {pi, pj, pk};
        for (int d = 0; d < nd; ++d) {
            const bool per = d == 2 || (d == 0 && g.xper);
            for (int s = 1; s >= -1; s -= 2) {
                int Q[3] = {P[0], P[1], P[2]};
                Q[d] += s;
                if (per) Q[d] = (Q[d] + n[d]) % n[d];
                else if (Q[d] < 0 || Q[d] >= n[d]) continue;
                // box-boundary points (v on the +y wall, u on the outflow face) are not arms
                if ((c == 1 && Q[1] == g.ny - 1) || (c == 0 && !g.xper && Q[0] == g.nx - 1)) continue;
                const long long lq = Q[0] + (long long)g.nx * (Q[1] + (long long)g.ny * Q[2]);
                if ((a.mask[lq] >> c) & 1u) continue;          // internal: its flux cancels
                const double h = (u0 + 0.0) / 2.0;
                double F;
                if (d == c) {
                    F = h * h;
                } else {
                    int e[3] = {0, 0, 0};
                    e[c] = 1;
                    const int o = s > 0 ? 0 : -1;   // the face's advecting points: P (+ e_c), shifted by -e_d for s = -1
                    int A[3] = {P[0], P[1], P[2]};
                    A[d] += o;
                    const double adv = (body_rd(a, d, A[0], A[1], A[2]) +
                                        body_rd(a, d, A[0] + e[0], A[1] + e[1], A[2] + e[2])) / 2.0;
                    F = adv * h;
                }
                sBN += -s * F / D[d] + a.nu * (0.0 - u0) / (D[d] * D[d]);
                if (d == c) {
                    if (s > 0) {
                        const long long lc = Q[0] + (long long)g.nx * (Q[1] + (long long)g.ny * Q[2]);
                        sPQ += (double)a.p[lc] + (double)a.psi[lc] * a.inv_ckdt;
                    } else {
                        sPQ -= (double)a.p[lin] + (double)a.psi[lin] * a.inv_ckdt;
                    }
                }
            }
        }
    }
    __shared__ double sh[3][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double v[3] = {sI, sBN, sPQ};
    for (int q = 0; q < 3; ++q) {
        double t = v[q];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) sh[q][wid] = t;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[threadIdx.x][w];
        a.part[((long long)c * gridDim.x + blockIdx.x) * 3 + threadIdx.x] = t;
    }
}

__global__ void k_body_force_final(const double* __restrict__ part, int nbx, double* __restrict__ scal,
                                   double dV, double dt, double ak, double bk, double ckdt, double dx, double dy,
                                   double dz, int last) {
    // warp c sums component c's block partials in a fixed order
    __shared__ double tot[3][3];
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (c < 3) {
        for (int q = 0; q < 3; ++q) {
            double t = 0.0;
            for (int b = lane; b < nbx; b += 32) t += part[((long long)c * nbx + b) * 3 + q];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) tot[c][q] = t;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double D[3] = {dx, dy, dz};
        for (int q = 0; q < 3; ++q) {
            const double BN = tot[q][1];
            const double imp = dV * (tot[q][0] - ckdt * tot[q][2] / D[q] + dt * (ak * BN + bk * scal[SCAL_BNPREV + q]));
            scal[SCAL_IMP + q] += imp;
            scal[SCAL_BNPREV + q] = BN;
        }
        if (last) {
            for (int q = 0; q < 3; ++q) {
                scal[SCAL_FORCE + q] += -scal[SCAL_IMP + q] / dt;
                scal[SCAL_IMP + q] = 0.0;
            }
            scal[SCAL_FSTEPS] += 1.0;
        }
    }
}

template <typename T>
ibm_status body_force_t(ibm_solver* h, int k) {
    const GridP& g = h->gp;
    BodyArgs<T> a;
    a.g = g;
    int mx = 0;
    for (int c = 0; c < 3; ++c) {
        const bool on = c < g.ncomp;
        a.u[c] = (const T*)h->buf.u[on ? c : 0];
        a.us[c] = (const T*)h->ustar[on ? c : 0];
        a.idx[c] = h->idx[c];
        a.lam[c] = h->lam[c];
        a.src[c] = h->src[c];
        a.cnt[c] = on ? h->counts[c] : 0;
        mx = std::max(mx, a.cnt[c]);
    }
    a.p = (const T*)h->buf.p;
    a.psi = (const T*)h->rhs;
    a.mask = h->mask;
    a.ckdt = h->phys.dt * RK_C[k];
    a.inv_ckdt = 1.0 / a.ckdt;
    a.nu = h->phys.nu;
    a.bmode = h->phys.bmode;
    a.part = h->partials;
    int nbx = std::max(1, std::min((mx + 255) / 256, std::min(256, h->npartials / 9)));
    k_body_force<T><<<dim3(nbx, 3), 256, 0, h->stream>>>(a);
    IBM_LAUNCH_CHECK();
    const double dV = g.dx * g.dy * (g.ndim == 3 ? g.dz : 1.0);
    k_body_force_final<<<1, 96, 0, h->stream>>>(h->partials, nbx, h->scal, dV, h->phys.dt, RK_A[k], RK_B[k],
                                                h->phys.dt * RK_C[k], g.dx, g.dy, g.dz, k == 2 ? 1 : 0);
    IBM_LAUNCH_CHECK();
    return IBM_OK;
}

// Outflow face of stage k (update) or, for the initial projection, only the flux balance.
template <typename T>
ibm_status outflow_t(ibm_solver* h, int k, bool update) {
    const GridP& g = h->gp;
    const long long rows = (long long)g.ny * g.nz;
    const int nb = (int)((rows + 255) / 256);
    if (nb > h->npartials) return ibm_set_error(IBM_E_INVALID, "too many outflow rows for the partials buffer");
    const double dt = h->phys.dt;
    // U_c: the inflow flux over the fluid outflow area (face counts, or summed heights on a stretched y)
    const double ucx = h->aface[1] > 0.0 ? g.uin * h->aface[0] / h->aface[1] / g.dx : 0.0;
    k_outflow<T><<<nb, 256, 0, h->stream>>>(g, (const T*)h->buf.u[0], h->mask, (T*)h->ustar[0], (T*)h->Nh[0],
                                           (T)(dt * RK_A[k]), (T)(dt * RK_B[k]), (T)ucx, k > 0, k < 2, update ? 1 : 0,
                                           h->partials);
    IBM_LAUNCH_CHECK();
    k_outflow_fix<T><<<nb, 256, 0, h->stream>>>(g, h->mask, (T*)h->ustar[0], h->partials, nb,
                                               g.uin * h->aface[0], h->aface[1]);
    IBM_LAUNCH_CHECK();
    return IBM_OK;
}

template <typename T>
ibm_status substage_t(ibm_solver* h, int k, bool predictor_only) {
    const GridP& g = h->gp;
    const double dt = h->phys.dt;
    const bool cflux = h->phys.flow_mode == IBM_FLOW_CONST_FLUX;
    cudaEvent_t t;
    int nparts = 0;
    timer_begin(h, "momentum", &t);
    ibm_status st0 = IBM_OK;
    if (h->mom_external) {       // a batch's persistent job kernel computed u* already
        const dim3 d = momentum_grid(g);
        nparts = (int)(d.x * d.y * d.z);
    } else {
        st0 = momentum_launch(h, k, &nparts);
    }
    if (st0 != IBM_OK) return st0;
    timer_end(h, t, "momentum");
    if (!g.xper) {
        timer_begin(h, "outflow", &t);
        st0 = outflow_t<T>(h, k, true);
        if (st0 != IBM_OK) return st0;
        timer_end(h, t, "outflow");
    }
    if (cflux) {
        double dV = g.dx * (g.ystr ? 1.0 : g.dy) * (g.ndim == 3 ? g.dz : 1.0);   // stretched: dy in the partials
        timer_begin(h, "flux_control", &t);
        k_flux_pi<T><<<1, 1024, 0, h->stream>>>(h->partials, nparts, dV, h->phys.target_flux, h->S[k], h->scal);
        IBM_LAUNCH_CHECK();
        timer_end(h, t, "flux_control");
    }
    T* us[3] = {(T*)h->ustar[0], (T*)h->ustar[1], (T*)h->ustar[2]};
    if (predictor_only) {
        // the caller gets u* itself, so the flux correction is applied explicitly here
        if (cflux) {
            dim3 fgrd(g.nsegx, (g.ny + 7) / 8, g.nz);
            k_flux_apply<T><<<fgrd, dim3(32, 8, 1), 0, h->stream>>>(g, (T*)h->ustar[0], h->mask, stage_coefs<T>(h, k),
                                                                     h->scal, (T)(dt * RK_C[k]));
            IBM_LAUNCH_CHECK();
        }
        for (int c = 0; c < g.ncomp; ++c)
            IBM_CUDA_TRY(cudaMemcpyAsync(h->buf.u[c], h->ustar[c], g.N * sizeof(T), cudaMemcpyDeviceToDevice, h->stream));
        return IBM_OK;
    }
    const FluxCorr<T> fc = flux_corr<T>(h, k);
    ibm_status st = divergence_and_solve<T>(h, us, cflux, fc);
    if (st != IBM_OK) return st;
    if (h->phys.body_force) {
        timer_begin(h, "body_force", &t);
        st = body_force_t<T>(h, k);
        if (st != IBM_OK) return st;
        timer_end(h, t, "body_force");
    }
    timer_begin(h, "correct", &t);
    st = launch_correct<T>(h, us, (T)(1.0 / (dt * RK_C[k])), 1, cflux, fc);
    if (st != IBM_OK) return st;
    timer_end(h, t, "correct");
    return IBM_OK;
}

template <typename T>
ibm_status project_t(ibm_solver* h) {
    const GridP& g = h->gp;
    T* us[3] = {(T*)h->ustar[0], (T*)h->ustar[1], g.ndim == 3 ? (T*)h->ustar[2] : (T*)h->ustar[0]};
    const T* u2 = g.ndim == 3 ? (const T*)h->buf.u[2] : (const T*)h->buf.u[0];
    k_mask_copy<T><<<cell_grid(g), dim3(32, 8), 0, h->stream>>>(g, h->mask, (const T*)h->buf.u[0], (const T*)h->buf.u[1], u2, us[0],
                                              us[1], us[2], h->body);
    IBM_LAUNCH_CHECK();
    if (!g.xper) {
        ibm_status st0 = outflow_t<T>(h, 0, false);
        if (st0 != IBM_OK) return st0;
    }
    const FluxCorr<T> fc = flux_corr<T>(h, 0);
    ibm_status st = divergence_and_solve<T>(h, us, false, fc);
    if (st != IBM_OK) return st;
    return launch_correct<T>(h, us, (T)1, 0, false, fc);
}

template <typename T>
ibm_status diag_t(ibm_solver* h, double* out) {
    const GridP& g = h->gp;
    const T* w = g.ndim == 3 ? (const T*)h->buf.u[2] : (const T*)h->buf.u[0];
    if (g.ystr)
        k_diag_str<T><<<DIAG_BLOCKS, 256, 0, h->stream>>>(g, (const T*)h->buf.u[0], (const T*)h->buf.u[1], w,
                                                          (const T*)h->buf.p, h->mask, h->partials);
    else
        k_diag<T><<<DIAG_BLOCKS, dim3(32, 8), 0, h->stream>>>(g, (const T*)h->buf.u[0], (const T*)h->buf.u[1], w,
                                                              (const T*)h->buf.p, h->mask, h->partials, 1.0 / g.dx,
                                                              1.0 / g.dy, 1.0 / g.dz);
    IBM_LAUNCH_CHECK();
    k_diag_final<<<1, 12 * 32, 0, h->stream>>>(h->partials, DIAG_BLOCKS, h->scal + 4);
    IBM_LAUNCH_CHECK();
    IBM_CUDA_TRY(cudaMemcpyAsync(out, h->scal, SCAL_N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    IBM_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return IBM_OK;
}

// Times the momentum predictor (stage 1, scratch outputs only) for every
// z-chunk choice and the divergence kernel for every march choice, keeping the
// fastest of each.  Overwrites only the predictor and RHS scratch buffers.
template <typename T>
ibm_status autotune_t(ibm_solver* h, int* kzm_out, int* kzd_out) {
    GridP& g = h->gp;
    if (g.ndim != 3) { *kzm_out = g.kzm; *kzd_out = g.kzd; return IBM_OK; }
    cudaEvent_t a, b;
    IBM_CUDA_TRY(cudaEventCreate(&a));
    IBM_CUDA_TRY(cudaEventCreate(&b));
    const bool saved_timing = h->timing;
    h->timing = false;
    auto time_it = [&](auto&& launch) -> float {
        for (int w = 0; w < 2; ++w) launch();
        cudaEventRecord(a, h->stream);
        for (int r = 0; r < 5; ++r) launch();
        cudaEventRecord(b, h->stream);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    };
    float best = 1e30f;
    int best_kzm = g.kzm;
    for (int kz : KZM_CHOICES) {
        if (kz > 2 * g.nz && kz != KZM_CHOICES[0]) continue;
        g.kzm = kz;
        float ms = time_it([&] {
            int np = 0;
            momentum_launch(h, 0, &np);
        });
        if (ms < best) { best = ms; best_kzm = kz; }
    }
    g.kzm = best_kzm;
    best = 1e30f;
    int best_kzd = g.kzd;
    T* us[3] = {(T*)h->ustar[0], (T*)h->ustar[1], (T*)h->ustar[2]};
    const T ix = (T)(1.0 / g.dx), iy = (T)(1.0 / g.dy), iz = (T)(1.0 / g.dz);
    const FluxCorr<T> fc = flux_corr<T>(h, 0);
    for (int kz : KZD_CHOICES) {
        if (kz > 2 * g.nz && kz != KZD_CHOICES[0]) continue;
        g.kzd = kz;
        float ms = time_it([&] {
            k_divergence<T, true, false, false><<<zmarch_grid(g), dim3(32, 8), 0, h->stream>>>(
                g, us[0], us[1], us[2], h->mask, (T*)h->rhs, ix, iy, iz, fc);
        });
        if (ms < best) { best = ms; best_kzd = kz; }
    }
    g.kzd = best_kzd;
    h->timing = saved_timing;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        h->failed = true;
        return ibm_set_error(IBM_E_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
    }
    *kzm_out = g.kzm;
    *kzd_out = g.kzd;
    return IBM_OK;
}

// Self-test of the integer-pipe conversions against the hardware conversions, bit for bit:
// each thread draws a bit pattern from a counter-based hash of its index (splitmix64, a
// published mixer), shaped by i % 4 into a random double, an exact FP32 rounding tie, a
// random float, or a double near the FP32 underflow and overflow thresholds.
__device__ unsigned long long g_selftest_bad;

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

__global__ void k_selftest_conversions(long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t r = splitmix64((uint64_t)i);
    bool bad = false;
    const int kind = (int)(i & 3);
    if (kind == 2) {                                    // float -> double
        const float f = __uint_as_float((uint32_t)r);
        const double a = f32_to_f64(f), b = (double)f;
        bad = __double_as_longlong(a) != __double_as_longlong(b) && !(a != a && b != b);
    } else {
        if (kind == 1) {                               // an exact tie between two floats
            r = (r & ~0x1fffffffull) | 0x10000000ull;
        } else if (kind == 3) {                        // exponents around the FP32 range ends
            const uint64_t E = (r >> 60) & 1 ? 890 + ((r >> 52) & 15) : 1144 + ((r >> 52) & 15);
            r = (r & 0x800fffffffffffffull) | (E << 52);
        }
        const double x = __longlong_as_double((long long)r);
        const float a = f64_to_f32_rn(x), b = __double2float_rn(x);
        bad = __float_as_uint(a) != __float_as_uint(b) && !(a != a && b != b);
    }
    if (bad) atomicAdd(&g_selftest_bad, 1ull);
}

}  // namespace

int diag_blocks() { return DIAG_BLOCKS; }

ibm_status selftest_conversions(long long n, long long* bad) {
    unsigned long long zero = 0, got = 0;
    cudaError_t e = cudaMemcpyToSymbol(g_selftest_bad, &zero, sizeof(zero));
    if (e == cudaSuccess) {
        k_selftest_conversions<<<(unsigned)((n + 255) / 256), 256>>>(n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&got, g_selftest_bad, sizeof(got));
    if (e != cudaSuccess) return ibm_set_error(IBM_E_CUDA, std::string("self-test: ") + cudaGetErrorString(e));
    *bad = (long long)got;
    return IBM_OK;
}

// The inverse row kernels of one precision may take row_smem_limit bytes of dynamic shared memory.
template <typename T, typename C>
void row_kernels_optin() {
    const int b = (int)row_smem_limit(sizeof(C), true);
    cudaFuncSetAttribute(k_irfft_rows<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    cudaFuncSetAttribute(k_idct_rows<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
}

ibm_status poisson_prepare(ibm_solver* h) {
    // the own row FFT: nx = 2M with M a product of 2, 3 and 5, three M-long buffers per warp
    // within 48 KB of shared memory
    {
        const int M = h->gp.nx / 2;
        int m = M, nr = 0;
        int rad[16];
        while (m % 4 == 0 && nr < 16) { rad[nr++] = 4; m /= 4; }
        while (m % 2 == 0 && nr < 16) { rad[nr++] = 2; m /= 2; }
        while (m % 3 == 0 && nr < 16) { rad[nr++] = 3; m /= 3; }
        while (m % 5 == 0 && nr < 16) { rad[nr++] = 5; m /= 5; }
        const size_t csz = 2 * h->esz;
        const bool ok = h->gp.nx % 2 == 0 && M >= 2 && m == 1 && 3 * (size_t)fft_ps(M) * csz <= 48 * 1024;
        // automatic: where the rows have a factor 3 or 5 (384 reals: 0.073 against cuFFT's 0.101 ms
        // per pass on 384 x 256 x 256); cuFFT is faster on power-of-two rows (512: 0.56 against 0.53)
        const bool pow2 = (M & (M - 1)) == 0;
        h->own_fft = ok && (h->own_fft_mode == 1 || (h->own_fft_mode == 2 && !pow2));
        // the DCT rows of an inflow/outflow x: fused whenever the own FFT can run (the fusion saves
        // two passes over the field, which outweighs cuFFT's edge on power-of-two rows)
        h->dct_rows = ok && !h->gp.xper && h->own_fft_mode != 0;
        h->fft_nrad = ok ? nr : 0;
        for (int q = 0; q < 16; ++q) h->fft_rad[q] = (ok && q < nr) ? rad[q] : 0;
        if (ok) {
            if (h->prec == IBM_FP64) row_kernels_optin<double, double2>();
            else row_kernels_optin<float, float2>();
            IBM_CUDA_TRY(cudaGetLastError());
            const int nbt = (M + 1 + 255) / 256;
            if (h->prec == IBM_FP64) k_fft_tables<double><<<nbt, 256, 0, h->stream>>>(M, (double*)h->fftab);
            else k_fft_tables<float><<<nbt, 256, 0, h->stream>>>(M, (float*)h->fftab);
            IBM_LAUNCH_CHECK();
        }
    }
    if (h->gp.xper) return IBM_OK;
    const int nb = (h->gp.nx + 255) / 256;
    if (h->prec == IBM_FP64) k_dct_twiddles<double><<<nb, 256, 0, h->stream>>>(h->gp.nx, (double*)h->twid);
    else k_dct_twiddles<float><<<nb, 256, 0, h->stream>>>(h->gp.nx, (float*)h->twid);
    IBM_LAUNCH_CHECK();
    return IBM_OK;
}


ibm_status run_autotune(ibm_solver* h, int* kzm, int* kzd) {
    return h->prec == IBM_FP64 ? autotune_t<double>(h, kzm, kzd) : autotune_t<float>(h, kzm, kzd);
}

ibm_status run_substage(ibm_solver* h, int k, bool predictor_only) {
    return h->prec == IBM_FP64 ? substage_t<double>(h, k, predictor_only) : substage_t<float>(h, k, predictor_only);
}

ibm_status run_project(ibm_solver* h) { return h->prec == IBM_FP64 ? project_t<double>(h) : project_t<float>(h); }

ibm_status run_poisson(ibm_solver* h, void* rhs_inout) {
    return h->prec == IBM_FP64 ? poisson_t<double>(h, rhs_inout) : poisson_t<float>(h, rhs_inout);
}

// out: [0] Pi, [4..15] the 12 diagnostics sums
ibm_status run_diagnostics(ibm_solver* h, double* out) {
    return h->prec == IBM_FP64 ? diag_t<double>(h, out) : diag_t<float>(h, out);
}
