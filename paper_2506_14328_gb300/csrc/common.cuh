// Shared declarations of libibm: kernel parameter blocks, small device helpers,
// and the host-side solver handle.  Layout conventions are those of include/ibm.h.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/ibm.h"

#define IBM_WARP 32

// ---------------------------------------------------------------------------
// Kernel parameter blocks (passed by value)
// ---------------------------------------------------------------------------
struct GridP {
    int nx, ny, nz;
    int ndim, ncomp;
    int nsegx;              // x segments of 32 points per row
    int nxh;                // spectrum extent in x: nx/2 + 1 (periodic x), nx (Neumann x, DCT modes)
    int nzs;                // spectrum extent in z: nz (periodic x), nz/2 + 1 or 1 (Neumann x)
    int xper;               // 1: x periodic; 0: inflow at -x, convective outflow at +x
    double uin;             // inflow velocity (x inflow/outflow)
    long long N;            // cells
    double dx, dy, dz;
    double ox, oy, oz;
    double sig_lo, sig_hi;  // tangential ghost factor at the y walls (-1 no-slip, +1 free-slip)
    int kzm;                // z planes one momentum block marches (autotuned)
    int kzd;                // z planes one divergence / correction block marches (autotuned)
    int ystr;               // 1: stretched wall-normal grid, per-row tables at yt
    const double* yt;       // device: YT_N tables of ny + 1 doubles (ytab(g, YT_*, j)), or NULL
};

// Per-row tables of a stretched wall-normal grid (reading R23), computed on the host in
// FP64 from the ny + 1 face heights yf and stored one after another, ny + 1 doubles each.
// hc[j] is the distance from centre j-1 to centre j (mirror ghosts of the first and last
// centres past the walls), dyc the cell heights, dyc_up[j] the height of the cell above
// (the last cell's own at the top).
enum {
    YT_YC = 0,     // cell-centre height (u, w, p rows)
    YT_YF,         // v-face height yf[j + 1]
    YT_DYC,        // cell height
    YT_HC,         // hc[j], j = 0..ny
    YT_IDYC,       // 1 / dyc
    YT_IHV,        // 1 / (distance between the centres on either side of v face j; dyc at the top)
    YT_ALO,        // face above row j: weight of row j in the linear interpolation of a
    YT_AHI,        //   cell-centred value (dyc_up / (dyc + dyc_up)), and of row j + 1
    YT_DCM,        // uneven second difference at centre rows: d(-1), d(0), d(+1)
    YT_DC0,
    YT_DCP,
    YT_DVM,        // ... at v rows (face spacing)
    YT_DV0,
    YT_DVP,
    YT_IVSP,       // 1 / min(dyc, dyc_up): v's CFL spacing
    YT_PIN,        // Poisson: input factor s_j dyc_j of the symmetric, unit off-diagonal form
    YT_POUT,       // Poisson: output factor s_j
    YT_PBE,        // Poisson: diagonal -s_j^2 (1/hc_j + 1/hc_{j+1}) (wall ends: one term)
    YT_PBK,        // Poisson: s_j^2 dyc_j, the factor of K on the diagonal
    YT_N
};
__host__ __device__ __forceinline__ double ytab(const GridP& g, int t, int j) { return g.yt[(long long)t * (g.ny + 1) + j]; }

// Union of tubes (IBM_GEOM_TUBES): polylines of (x, y, z, r) points, at most
// TUBE_MAX tubes of TUBE_PTS points; passed by value with the other parameters.
constexpr int TUBE_MAX = 12, TUBE_PTS = 32;

struct GeomP {
    int kind;
    double p[8];
    int ntubes, npts;
    double tube[TUBE_MAX * TUBE_PTS * 4];
    const double* sdf[3];   // IBM_GEOM_SAMPLED: phi of each component at its points (device)
};

// A moving body (reading R24): kind 0 at rest, 1 translating with ub, 2 a cylinder rotating
// about its axis (xc, yc) at the rate om.  Its points hold bodyvel(); the momentum operator
// reads them as that velocity.
struct BodyP {
    int kind;
    double ub[3];
    double om, xc, yc;
};

// velocity of the body at the point of component c with coordinates (x, y)
__host__ __device__ __forceinline__ double bodyvel(const BodyP& b, int c, double x, double y) {
    if (b.kind == 1) return b.ub[c];
    if (b.kind == 2) return c == 0 ? -b.om * (y - b.yc) : (c == 1 ? b.om * (x - b.xc) : 0.0);
    return 0.0;
}

// The IBM coefficients of one stage for one component: indexed by list
// position; segoff gives the list position of the first IBM point of every
// 32-point x segment (lists are sorted by linear index).
// 16-byte aligned: one vector load per coefficient set (the lists start on 256-byte boundaries
// and every entry is 16 or 32 bytes)
template <typename T> struct alignas(16) Coef4 { T a, b, s, pad; };

template <typename T> struct IbmStage {
    const int* segoff[3];
    const Coef4<T>* coef[3];   // already offset to the stage
};

template <typename T> struct StageP {
    T sig_lo, sig_hi;  // tangential ghost factors at the y walls
    T dta, dtb;        // dt a_k, dt b_k
    T ckdt;            // c_k dt
    T nu;
    T g[3];
    T idx, idy, idz;   // 1/dx ...
    T nx2, ny2, nz2;   // nu/dx^2 ...
    T qx, qy, qz;      // 1/(4 dx) ...: the two-point averages' 1/2 squared, over the spacing
    T cgx, cgy, cgz;   // c_k dt / dx ...: pressure-gradient factors
    T lc;              // 2 (nu/dx^2 + nu/dy^2 + nu/dz^2): the Laplacian's centre weight (3D)
    T uin;             // inflow velocity (inflow/outflow x)
    int read_prev;     // stage k > 1: add b_k N^{k-2}
    int write_n;       // stage k < 3: store N^{k-1}
    int flux_sum;      // accumulate the predictor flux (constant flow rate)
};

// Low-storage RK3 coefficients a_k, b_k and c_k = a_k + b_k (Sec. 2.4, Eq. rk3-rai)
inline constexpr double RK_A[3] = {64.0 / 120.0, 50.0 / 120.0, 90.0 / 120.0};
inline constexpr double RK_B[3] = {0.0, -34.0 / 120.0, -50.0 / 120.0};
inline constexpr double RK_C[3] = {64.0 / 120.0, 16.0 / 120.0, 40.0 / 120.0};
// stage times as fractions of the step: the sums of the c of the earlier stages
inline constexpr double RK_T[3] = {0.0, 64.0 / 120.0, 80.0 / 120.0};

// Momentum tiling: blocks of 32 x 8 threads own 32 x 16 cells in (x, y) and
// march g.kzm planes in z.  The autotuner picks kzm from KZM_CHOICES; the flux
// partials are sized for the smallest choice.
constexpr int MOM_TX = 32, MOM_WARPS = 8, MOM_TY = 16, MOM_KZ_MIN = 8;
// blocks (and flux partials) of the IBM division after the TMA predictor, at most (one thread per
// point instead, up to 4096 blocks, measured the same: the kernel is bound by the DRAM sectors of
// its scattered accesses, not by their latency)
constexpr int IBM_DIV_PARTS = 256;
constexpr int KZM_CHOICES[8] = {8, 12, 16, 24, 32, 48, 64, 86};
constexpr int KZD_CHOICES[4] = {4, 8, 16, 32};
inline dim3 momentum_grid(const GridP& g, int kzm) {
    return dim3(g.nsegx, (g.ny + MOM_TY - 1) / MOM_TY, g.ndim == 3 ? (g.nz + kzm - 1) / kzm : 1);
}
inline dim3 momentum_grid(const GridP& g) { return momentum_grid(g, g.kzm); }

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// ---------------------------------------------------------------------------
// Diagnostics accumulated cell by cell, shared by ibm_diagnostics and
// ibm_diagnostics_noalloc so that the two agree cell by cell.  Results (a[12]):
//   [0] sum div^2  [1] max |div|  [2..4] max |u_c|  [5..7] sum u_c  [8..10] sum u_c^2
//   [11] non-finite count;  velocity terms over the internal points of component c.
// FP64 fields: FP64 per cell.  FP32 fields: the same quantities to about 1e-14
// relative with FP32 instructions only (GB300's FP64 rate is 1/64 of FP32):
// differences and products are split exactly into float pairs (two-sum, two-
// product), sums run in pairs and are folded into FP64 every DIAG_FOLD cells.
// ---------------------------------------------------------------------------
constexpr int DIAG_FOLD = 8;
constexpr int DIAG_BLOCKS = 4 * 304;   // blocks of the diagnostics kernel (12 partials each)

// Device scalars (h->scal): [0] Pi of the substage, [2] its typed copy, [3] momentum timeout flag,
// [4..15] diagnostics sums, then the body-force sums.
constexpr int SCAL_N = 32;
constexpr int SCAL_FORCE = 16;    // 3: force on the body summed over the counted steps
constexpr int SCAL_BNPREV = 19;   // 3: the right-hand side's body share of the previous substage
constexpr int SCAL_FSTEPS = 22;   // counted steps
constexpr int SCAL_IMP = 24;      // 3: impulse of the current step so far

// B of the implicit update (Eq. Bexpr and the Taylor options): B = x / (e^x - 1), 1 at x = 0.
__device__ __forceinline__ double ibm_B_of_x(double x, int mode) {
    if (mode == IBM_B_EULER || mode == IBM_B_EXPLICIT) return 1.0;
    if (mode == IBM_B_TAYLOR2) return 1.0 / (1.0 + x / 2.0);
    if (!(x > 0.0)) return 1.0;
    return x / expm1(x);
}

struct FF { float hi, lo; };   // value hi + lo, |lo| <= ulp(hi) / 2

// Each rounding whose error is kept is an explicit _rn operation, so no
// multiply-add contraction can change it.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ FF ff_norm(float s, float e) {   // fast two-sum: |s| >= |e|
    FF r;
    r.hi = __fadd_rn(s, e);
    r.lo = e - (r.hi - s);
    return r;
}

__device__ __forceinline__ FF ff_add(FF a, float bh, float bl) {
    float s, e;
    two_sum(a.hi, bh, s, e);
    return ff_norm(s, e + (a.lo + bl));
}

__device__ __forceinline__ FF ff_mul(FF a, float bh, float bl) {   // (a.hi + a.lo)(bh + bl), to ~2^-46
    const float p = __fmul_rn(a.hi, bh);
    const float pe = fmaf(a.hi, bh, -p) + (a.hi * bl + a.lo * bh);
    return ff_norm(p, pe);
}

template <typename T> struct DiagAcc;

template <> struct DiagAcc<double> {
    double a[12];
    double vmax[3];
    __device__ DiagAcc() {
        for (int q = 0; q < 12; ++q) a[q] = 0.0;
        vmax[0] = vmax[1] = vmax[2] = 0.0;
    }
    __device__ __forceinline__ void cell(int ncomp, const double (&id)[3], double uc, double ul, double vc, double vm,
                                         double wc, double wm, double pc, uint8_t m) {
        double d = (uc - ul) * id[0] + (vc - vm) * id[1];
        if (ncomp == 3) d += (wc - wm) * id[2];
        a[0] += d * d;
        a[1] = fmax(a[1], fabs(d));
        const double x3[3] = {uc, vc, wc};
        for (int c = 0; c < ncomp; ++c) {
            const double x = x3[c];
            if (!isfinite(x)) a[11] += 1.0;
            if (!((m >> c) & 1u)) continue;
            vmax[c] = fmax(vmax[c], fabs(x));
            a[5 + c] += x;
            a[8 + c] += x * x;
        }
        if (!isfinite(pc)) a[11] += 1.0;
    }
    __device__ __forceinline__ void finish(double (&out)[12]) {
        for (int q = 0; q < 12; ++q) out[q] = a[q];
        for (int c = 0; c < 3; ++c) out[2 + c] = vmax[c];
    }
};

template <> struct DiagAcc<float> {
    double a[12];           // folded sums
    FF s[7];                // running pairs: sum u_c (0..2), sum u_c^2 (3..5), sum div^2 (6)
    FF dmax;                // max |div| as a normalised pair (compared exactly)
    float vmax[3];
    int nonfinite, n;
    __device__ DiagAcc() {
        for (int q = 0; q < 12; ++q) a[q] = 0.0;
        for (int q = 0; q < 7; ++q) s[q] = FF{0.f, 0.f};
        dmax = FF{0.f, 0.f};
        vmax[0] = vmax[1] = vmax[2] = 0.f;
        nonfinite = n = 0;
    }
    __device__ __forceinline__ void fold() {
        for (int c = 0; c < 3; ++c) {
            a[5 + c] += (double)s[c].hi + (double)s[c].lo;
            a[8 + c] += (double)s[3 + c].hi + (double)s[3 + c].lo;
        }
        a[0] += (double)s[6].hi + (double)s[6].lo;
        for (int q = 0; q < 7; ++q) s[q] = FF{0.f, 0.f};
        n = 0;
    }
    // id: the inverse spacings split into float pairs (hi, lo) per direction
    __device__ __forceinline__ void cell(int ncomp, const float (&id)[6], float uc, float ul, float vc, float vm,
                                         float wc, float wm, float pc, uint8_t m) {
        FF t, d;
        two_sum(uc, -ul, t.hi, t.lo);                  // exact difference
        d = ff_mul(t, id[0], id[1]);
        two_sum(vc, -vm, t.hi, t.lo);
        t = ff_mul(t, id[2], id[3]);
        d = ff_add(d, t.hi, t.lo);
        if (ncomp == 3) {
            two_sum(wc, -wm, t.hi, t.lo);
            t = ff_mul(t, id[4], id[5]);
            d = ff_add(d, t.hi, t.lo);
        }
        if (!isfinite(d.hi)) d = FF{d.hi, 0.f};
        const FF d2 = ff_mul(d, d.hi, d.lo);
        s[6] = ff_add(s[6], d2.hi, d2.lo);
        const FF ad = d.hi < 0.f ? FF{-d.hi, -d.lo} : d;
        if (ad.hi > dmax.hi || (ad.hi == dmax.hi && ad.lo > dmax.lo)) dmax = ad;
        const float x3[3] = {uc, vc, wc};
        for (int c = 0; c < ncomp; ++c) {
            const float x = x3[c];
            if (!isfinite(x)) ++nonfinite;
            if (!((m >> c) & 1u)) continue;
            vmax[c] = fmaxf(vmax[c], fabsf(x));
            s[c] = ff_add(s[c], x, 0.f);
            const float p = __fmul_rn(x, x);
            s[3 + c] = ff_add(s[3 + c], p, fmaf(x, x, -p));
        }
        if (!isfinite(pc)) ++nonfinite;
        if (++n == DIAG_FOLD) fold();
    }
    __device__ __forceinline__ void finish(double (&out)[12]) {
        fold();
        for (int q = 0; q < 12; ++q) out[q] = a[q];
        out[1] = (double)dmax.hi + (double)dmax.lo;
        for (int c = 0; c < 3; ++c) out[2 + c] = (double)vmax[c];
        out[11] = (double)nonfinite;
    }
};

// The inverse spacings in the form DiagAcc<T>::cell takes them.
template <typename T> struct DiagInv;
template <> struct DiagInv<double> {
    double v[3];
    __host__ __device__ DiagInv(double ix, double iy, double iz) { v[0] = ix; v[1] = iy; v[2] = iz; }
};
template <> struct DiagInv<float> {
    float v[6];
    __host__ __device__ DiagInv(double ix, double iy, double iz) {
        const double x[3] = {ix, iy, iz};
        for (int d = 0; d < 3; ++d) {
            v[2 * d] = (float)x[d];
            v[2 * d + 1] = (float)(x[d] - (double)v[2 * d]);
        }
    }
};

// ---------------------------------------------------------------------------
// Host-side handle
// ---------------------------------------------------------------------------
struct KernelTimer {
    const char* name;   // a string literal
    cudaEvent_t a, b;
};

struct ibm_solver {
    ibm_grid_desc grid;
    ibm_geom_desc geom;
    ibm_buffers buf;
    cudaStream_t stream = nullptr;
    // state import / export: the field copies go out on their own streams (several copy
    // engines), ordered after the solver's stream by an event; created on first use
    cudaStream_t copy_streams[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t tri_stream = nullptr;             // the FP64 tridiagonal systems beside the FP32 ones
    cudaEvent_t tri_fork = nullptr, tri_join = nullptr;
    cudaEvent_t copy_fork = nullptr;
    GridP gp;
    GeomP geo;
    int prec = IBM_FP64;
    size_t esz = 8;            // field element size
    long long N = 0;
    long long nspec = 0;       // nz * ny * nxh
    long long nseg = 0;

    // workspace carve-out
    uint8_t* mask = nullptr;
    uint8_t* velbits = nullptr;
    int* segcnt[3] = {nullptr, nullptr, nullptr};
    int* segoff[3] = {nullptr, nullptr, nullptr};
    int* scan_tmp = nullptr;
    int* d_counts = nullptr;
    void* ustar[3] = {nullptr, nullptr, nullptr};
    void* Nh[3] = {nullptr, nullptr, nullptr};
    void* rhs = nullptr;
    void* spec = nullptr;
    double* pivots = nullptr;
    float* pivots32 = nullptr;     // FP32 copy for the strongly dominant systems
    uint8_t* use32 = nullptr;      // per (kz, kx) system: 1 = FP32 sweep
    int* sys_order = nullptr;      // systems, FP64 ones first
    int n64 = 0;                   // number of FP64 systems
    int tri_form = 0;              // ibm_set_tridiag_form: 0 automatic, 1 warp, 2 thread per FP64 system
    bool mom_external = false;     // a batch launches this solve's momentum predictor (job kernel)
    void* dtemp = nullptr;
    void* fft_work = nullptr;
    double* partials = nullptr;
    double* scal = nullptr;    // device scalars: [0] = Pi of the current substage
    size_t fft_work_bytes = 0;
    int npartials = 0;

    int counts[3] = {0, 0, 0};
    int cap[3] = {0, 0, 0};    // IBM points the weights buffer holds per component (counts, or
                               // 3 counts / 2 + 1024 for a translating body)
    BodyP body = {0, {0.0, 0.0, 0.0}, 0.0, 0.0, 0.0};
    double geo0[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // geometry parameters at t = 0 (a translating body)
    int nfaces[2] = {0, 0};    // inflow/outflow x: fluid inflow and outflow faces
    double aface[2] = {0, 0};  // ... their areas over dx dz: counts, or the summed cell heights (stretched y)
    std::vector<double> ytab_host;   // stretched y: the YT_N per-row tables (also in the workspace)
    double* ytab = nullptr;

    // weights
    bool weights_ready = false;
    ibm_physics phys;
    int* idx[3] = {nullptr, nullptr, nullptr};
    double* lam[3] = {nullptr, nullptr, nullptr};
    double* src[3] = {nullptr, nullptr, nullptr};
    void* coef[3] = {nullptr, nullptr, nullptr};
    double S[3] = {0, 0, 0};   // flux-control response per stage
    double last_pi = 0.0;

    cufftHandle plan_f = 0, plan_i = 0;
    cufftHandle plan_fz = 0, plan_iz = 0;   // Neumann x, 3D: transforms along z
    void* rtmp = nullptr;                    // Neumann x: reordered rows of the DCT (N reals)
    void* twid = nullptr;                    // Neumann x: cos, sin of pi k / 2nx (field precision)
    // own real FFT of the x rows (field precision): radices of nx/2, the table
    // exp(-2 pi i t / (nx/2)), t < nx/2, then exp(-2 pi i k / nx), k <= nx/2
    bool own_fft = false;                    // the rows run the own kernels (nx supported)
    bool dct_rows = false;                   // inflow/outflow x: the DCT rows in one pass each way
    int own_fft_mode = 2;                    // ibm_set_own_fft: 0 never, 1 where supported, 2 automatic
    int fft_nrad = 0;
    int fft_rad[16] = {0};
    void* fftab = nullptr;
    bool plans = false;

    bool failed = false;
    long long steps = 0;
    long long launches = 0;

    bool timing = false;
    std::vector<KernelTimer> timers;

    void* mom_maps = nullptr;  // tensor maps of the TMA momentum kernel (momentum.cu), or NULL
    bool mom_tma = true;       // use the TMA momentum kernel where the grid allows it

    cudaGraphExec_t graph = nullptr;
    bool graph_ready = false;
    long long graph_launches = 0;   // kernels of this library in one captured step

    // masked projection (IBM_PROJ_MASKED): conjugate-gradient vectors x, r, z, p, A p (FP64)
    int proj_mode = IBM_PROJ_FULLBOX;
    double proj_tol = 1e-10;
    int proj_maxit = 500;
    double* pcg[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int proj_iters = 0;
    double proj_resid = 0.0;
};

// The IBM coefficient lists of RK stage k (list position -> {alpha, beta, s}).
template <typename T>
inline IbmStage<T> stage_coefs(const ibm_solver* h, int k) {
    IbmStage<T> ib;
    for (int c = 0; c < 3; ++c) {
        ib.segoff[c] = h->segoff[c];
        ib.coef[c] = (const Coef4<T>*)h->coef[c] + (long long)k * h->counts[c];
    }
    return ib;
}

// ---------------------------------------------------------------------------
// Host entry points between translation units
// ---------------------------------------------------------------------------
ibm_status ibm_set_error(ibm_status st, const std::string& msg);

// geometry.cu
ibm_status geom_classify(ibm_solver* h, bool fresh_fill = false);   // fresh_fill: points that turn fluid take the body velocity
ibm_status geom_build_lists_and_weights(ibm_solver* h);
ibm_status geom_stage_coefficients(ibm_solver* h);
ibm_status geom_pivots(ibm_solver* h);
ibm_status geom_wall_shear(ibm_solver* h, double wavelength, double* tau_x, double* tau1);

// step.cu
ibm_status run_substage(ibm_solver* h, int k, bool predictor_only);
ibm_status run_autotune(ibm_solver* h, int* kzm, int* kzd);

// momentum.cu
// Launches the momentum predictor of RK stage k on the solver's stream;
// *nparts receives the number of flux partials it wrote.
ibm_status momentum_launch(ibm_solver* h, int k, int* nparts);
// stage k's momentum predictors of n solves of one precision in one persistent launch on stream
constexpr int MOM_MAX_JOBS = 40;
ibm_status momentum_jobs_launch(ibm_solver* const* hs, int n, int k, cudaStream_t stream);
int momentum_default_kzm(const GridP& g, int prec, bool tma);
// Builds (or drops) the TMA kernel's tensor maps over the solver's buffers.
void momentum_prepare(ibm_solver* h);
void momentum_release(ibm_solver* h);
bool momentum_uses_tma(const ibm_solver* h);
ibm_status run_project(ibm_solver* h);
ibm_status run_poisson(ibm_solver* h, void* rhs_inout);
ibm_status run_diagnostics(ibm_solver* h, double* out);   // SCAL_N doubles
ibm_status poisson_prepare(ibm_solver* h);
ibm_status selftest_conversions(long long n, long long* bad);   // legacy default stream, blocking   // the own row-FFT plan and tables; Neumann x: the DCT twiddles

// timing hooks used by both
void timer_begin(ibm_solver* h, const char* name, cudaEvent_t* ev);
void timer_end(ibm_solver* h, cudaEvent_t ev_begin, const char* name);

#define IBM_CUDA_TRY(expr)                                                                  \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess) {                                                            \
            h->failed = true;                                                               \
            return ibm_set_error(IBM_E_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
        }                                                                                   \
    } while (0)

#define IBM_LAUNCH_CHECK()                                                                  \
    do {                                                                                    \
        cudaError_t _e = cudaGetLastError();                                                \
        if (_e != cudaSuccess) {                                                            \
            h->failed = true;                                                               \
            return ibm_set_error(IBM_E_CUDA, std::string("kernel launch: ") + cudaGetErrorString(_e)); \
        }                                                                                   \
        h->launches++;                                                                      \
    } while (0)
