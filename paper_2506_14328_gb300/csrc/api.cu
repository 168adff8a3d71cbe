// C ABI of libibm (declared in include/ibm.h): argument checking, workspace
// carve-out, cuFFT plans, stream capture, event timing and state export.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>

namespace {

thread_local std::string g_last_error;

constexpr size_t ALIGN = 256;
constexpr int DIAG_PART = DIAG_BLOCKS * 12;
constexpr int SCAN_CH = 512 * 8;
constexpr uint64_t STATE_MAGIC = 0x31534d4249ull;     // "IBMS1"

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

ibm_status check_grid(const ibm_grid_desc* d) {
    if (!d) return ibm_set_error(IBM_E_INVALID, "grid descriptor is NULL");
    if (d->ndim != 2 && d->ndim != 3) return ibm_set_error(IBM_E_INVALID, "ndim must be 2 or 3");
    for (int i = 0; i < 3; ++i) {
        if (d->n[i] < 1) return ibm_set_error(IBM_E_INVALID, "n[d] must be >= 1");
        if (!(d->L[i] > 0.0) || !std::isfinite(d->L[i])) return ibm_set_error(IBM_E_INVALID, "L[d] must be > 0");
        if (!std::isfinite(d->origin[i])) return ibm_set_error(IBM_E_INVALID, "origin must be finite");
    }
    if (d->ndim == 2 && d->n[2] != 1) return ibm_set_error(IBM_E_INVALID, "2D grids have n[2] == 1");
    if (d->n[1] < 2) return ibm_set_error(IBM_E_INVALID, "ny must be >= 2");
    long long N = (long long)d->n[0] * d->n[1] * d->n[2];
    if (N >= (1ll << 31)) return ibm_set_error(IBM_E_INVALID, "more than 2^31-1 cells");
    if (d->precision != IBM_FP64 && d->precision != IBM_FP32) return ibm_set_error(IBM_E_INVALID, "bad precision");
    if (d->bc_lo[2] != IBM_BC_PERIODIC || d->bc_hi[2] != IBM_BC_PERIODIC)
        return ibm_set_error(IBM_E_UNSUPPORTED, "z must be periodic in this build");
    const bool xper = d->bc_lo[0] == IBM_BC_PERIODIC && d->bc_hi[0] == IBM_BC_PERIODIC;
    const bool xflow = d->bc_lo[0] == IBM_BC_INFLOW && d->bc_hi[0] == IBM_BC_OUTFLOW;
    if (!xper && !xflow)
        return ibm_set_error(IBM_E_UNSUPPORTED, "x must be periodic, or an inflow at -x with an outflow at +x");
    if (xflow && (d->n[0] < 2 || !std::isfinite(d->inflow[0])))
        return ibm_set_error(IBM_E_INVALID, "an inflow/outflow x needs nx >= 2 and a finite inflow velocity");
    for (int b : {d->bc_lo[1], d->bc_hi[1]})
        if (b != IBM_BC_NOSLIP && b != IBM_BC_FREESLIP)
            return ibm_set_error(IBM_E_UNSUPPORTED, "y faces must be no-slip or free-slip walls in this build");
    if (d->y_faces) {
        const double* yf = d->y_faces;
        for (int j = 0; j <= d->n[1]; ++j)
            if (!std::isfinite(yf[j]) || (j > 0 && !(yf[j] > yf[j - 1])))
                return ibm_set_error(IBM_E_INVALID, "y_faces: n[1] + 1 finite, strictly increasing heights");
        const double tol = 1e-12 * d->L[1];
        if (std::fabs(yf[0] - d->origin[1]) > tol || std::fabs(yf[d->n[1]] - d->origin[1] - d->L[1]) > tol)
            return ibm_set_error(IBM_E_INVALID, "y_faces must span the box from origin[1] to origin[1] + L[1]");
    }
    return IBM_OK;
}

// The per-row tables of a stretched wall-normal grid (reading R23; layout YT_* in common.cuh).
std::vector<double> y_tables(const ibm_grid_desc* d) {
    const int ny = d->n[1];
    const int S = ny + 1;
    const double* yf = d->y_faces;
    std::vector<double> t((size_t)YT_N * S, 0.0);
    auto at = [&](int k, int j) -> double& { return t[(size_t)k * S + j]; };
    std::vector<double> yc(ny), dyc(ny), dup(ny), hc(ny + 1);
    for (int j = 0; j < ny; ++j) {
        yc[j] = 0.5 * (yf[j] + yf[j + 1]);
        dyc[j] = yf[j + 1] - yf[j];
    }
    for (int j = 0; j < ny; ++j) dup[j] = j + 1 < ny ? dyc[j + 1] : dyc[ny - 1];
    // centres with the mirror ghosts past the walls
    std::vector<double> ext(ny + 2);
    ext[0] = 2.0 * yf[0] - yc[0];
    for (int j = 0; j < ny; ++j) ext[j + 1] = yc[j];
    ext[ny + 1] = 2.0 * yf[ny] - yc[ny - 1];
    for (int j = 0; j <= ny; ++j) hc[j] = ext[j + 1] - ext[j];
    // the symmetric, unit off-diagonal form of the Poisson rows: s_{j-1} s_j = hc_j
    std::vector<double> sj(ny);
    sj[0] = std::sqrt(hc[1]);
    for (int j = 1; j < ny; ++j) sj[j] = hc[j] / sj[j - 1];
    for (int j = 0; j < ny; ++j) {
        at(YT_YC, j) = yc[j];
        at(YT_YF, j) = yf[j + 1];
        at(YT_DYC, j) = dyc[j];
        at(YT_IDYC, j) = 1.0 / dyc[j];
        at(YT_IHV, j) = 1.0 / (j + 1 < ny ? hc[j + 1] : dyc[ny - 1]);
        at(YT_ALO, j) = dup[j] / (dyc[j] + dup[j]);
        at(YT_AHI, j) = dyc[j] / (dyc[j] + dup[j]);
        const double hm = hc[j], hp = hc[j + 1];
        at(YT_DCM, j) = 2.0 / (hm * (hm + hp));
        at(YT_DC0, j) = -2.0 / (hm * hp);
        at(YT_DCP, j) = 2.0 / (hp * (hm + hp));
        const double vm = dyc[j], vp = dup[j];
        at(YT_DVM, j) = 2.0 / (vm * (vm + vp));
        at(YT_DV0, j) = -2.0 / (vm * vp);
        at(YT_DVP, j) = 2.0 / (vp * (vm + vp));
        at(YT_IVSP, j) = 1.0 / std::min(dyc[j], dup[j]);
        const double e_lo = j > 0 ? 1.0 / hc[j] : 0.0, e_hi = j + 1 < ny ? 1.0 / hc[j + 1] : 0.0;
        at(YT_PIN, j) = sj[j] * dyc[j];
        at(YT_POUT, j) = sj[j];
        at(YT_PBE, j) = -sj[j] * sj[j] * (e_lo + e_hi);
        at(YT_PBK, j) = sj[j] * sj[j] * dyc[j];
    }
    for (int j = 0; j <= ny; ++j) at(YT_HC, j) = hc[j];
    return t;
}

GridP make_gridp(const ibm_grid_desc* d) {
    GridP g;
    g.nx = d->n[0];
    g.ny = d->n[1];
    g.nz = d->n[2];
    g.ndim = d->ndim;
    g.ncomp = d->ndim == 3 ? 3 : 2;
    g.nsegx = (g.nx + IBM_WARP - 1) / IBM_WARP;
    g.xper = d->bc_lo[0] != IBM_BC_INFLOW;
    // spectrum extents: periodic x: half complex in x, full in z; Neumann x: all DCT modes
    // in x, half complex in z (3D)
    g.nxh = g.xper ? g.nx / 2 + 1 : g.nx;
    g.nzs = g.xper ? g.nz : (g.nz > 1 ? g.nz / 2 + 1 : 1);
    g.uin = g.xper ? 0.0 : d->inflow[0];
    g.N = (long long)g.nx * g.ny * g.nz;
    g.dx = d->L[0] / d->n[0];
    g.dy = d->L[1] / d->n[1];
    g.dz = d->L[2] / d->n[2];
    g.ox = d->origin[0];
    g.oy = d->origin[1];
    g.oz = d->origin[2];
    g.sig_lo = d->bc_lo[1] == IBM_BC_NOSLIP ? -1.0 : 1.0;
    g.sig_hi = d->bc_hi[1] == IBM_BC_NOSLIP ? -1.0 : 1.0;
    g.kzm = 32;             // replaced by momentum_default_kzm at setup
    g.kzd = 16;
    g.ystr = d->y_faces != nullptr;
    g.yt = nullptr;         // set once the workspace is carved
    return g;
}

// flux partials: one per momentum block at the smallest z-chunk the autotuner may pick
int momentum_blocks(const GridP& g) {
    dim3 d = momentum_grid(g, MOM_KZ_MIN);
    return (int)(d.x * d.y * d.z);
}

// Creates the transform plans with auto-allocation off; returns the largest work size.
// Periodic x: an R2C / C2R pair along the contiguous x rows and, in 3D, one in-place C2C
// plan along z over the half spectrum (*pfz; *piz = 0); the same passes a 2D (z, x) plan
// makes, with the same spectrum layout.
// Neumann x: an R2C / C2R pair along x (the FFT inside the DCT) and, in 3D, a strided
// R2C / C2R pair along z over the real DCT coefficients.
ibm_status make_plans(const GridP& g, int prec, cufftHandle* pf, cufftHandle* pi, cufftHandle* pfz,
                      cufftHandle* piz, size_t* work) {
    cufftType tf = prec == IBM_FP64 ? CUFFT_D2Z : CUFFT_R2C;
    cufftType ti = prec == IBM_FP64 ? CUFFT_Z2D : CUFFT_C2R;
    long long nx = g.nx, ny = g.ny, nz = g.nz;
    size_t wf = 0, wi = 0, wfz = 0, wiz = 0;
    *pfz = *piz = 0;
    if (cufftCreate(pf) != CUFFT_SUCCESS || cufftCreate(pi) != CUFFT_SUCCESS)
        return ibm_set_error(IBM_E_CUDA, "cufftCreate failed");
    cufftSetAutoAllocation(*pf, 0);
    cufftSetAutoAllocation(*pi, 0);
    cufftResult r1 = CUFFT_SUCCESS, r2 = CUFFT_SUCCESS, r3 = CUFFT_SUCCESS, r4 = CUFFT_SUCCESS;
    {
        long long nxr = nx / 2 + 1;   // half spectrum of a real row
        long long n[1] = {nx};
        long long ie[1] = {nx};
        long long oe[1] = {nxr};
        r1 = cufftMakePlanMany64(*pf, 1, n, ie, 1, nx, oe, 1, nxr, tf, ny * nz, &wf);
        r2 = cufftMakePlanMany64(*pi, 1, n, oe, 1, nxr, ie, 1, nx, ti, ny * nz, &wi);
        if (g.xper && g.nz > 1) {
            if (cufftCreate(pfz) != CUFFT_SUCCESS) return ibm_set_error(IBM_E_CUDA, "cufftCreate failed");
            cufftSetAutoAllocation(*pfz, 0);
            const long long nxh = g.nxh;
            long long nzn[1] = {nz};
            long long ze[1] = {nz};
            r3 = cufftMakePlanMany64(*pfz, 1, nzn, ze, ny * nxh, 1, ze, ny * nxh, 1,
                                     prec == IBM_FP64 ? CUFFT_Z2Z : CUFFT_C2C, ny * nxh, &wfz);
        }
        if (!g.xper && g.nz > 1) {
            if (cufftCreate(pfz) != CUFFT_SUCCESS || cufftCreate(piz) != CUFFT_SUCCESS)
                return ibm_set_error(IBM_E_CUDA, "cufftCreate failed");
            cufftSetAutoAllocation(*pfz, 0);
            cufftSetAutoAllocation(*piz, 0);
            long long nzn[1] = {nz};
            long long ize[1] = {nz};
            long long oze[1] = {nz / 2 + 1};
            r3 = cufftMakePlanMany64(*pfz, 1, nzn, ize, ny * nx, 1, oze, ny * nx, 1, tf, ny * nx, &wfz);
            r4 = cufftMakePlanMany64(*piz, 1, nzn, oze, ny * nx, 1, ize, ny * nx, 1, ti, ny * nx, &wiz);
        }
    }
    if (r1 != CUFFT_SUCCESS || r2 != CUFFT_SUCCESS || r3 != CUFFT_SUCCESS || r4 != CUFFT_SUCCESS) {
        cufftDestroy(*pf);
        cufftDestroy(*pi);
        if (*pfz) cufftDestroy(*pfz);
        if (*piz) cufftDestroy(*piz);
        *pfz = *piz = 0;
        return ibm_set_error(IBM_E_CUDA, "cufftMakePlanMany64 failed (codes " + std::to_string((int)r1) + "/" +
                                             std::to_string((int)r2) + "/" + std::to_string((int)r3) + "/" +
                                             std::to_string((int)r4) + ")");
    }
    size_t w = wf > wi ? wf : wi;
    w = w > wfz ? w : wfz;
    w = w > wiz ? w : wiz;
    *work = w;
    return IBM_OK;
}

// Carve the workspace; with base == nullptr only the size is computed.
size_t carve(ibm_solver* h, const GridP& g, int prec, size_t fft_work, char* base) {
    size_t off = 0;
    size_t esz = prec == IBM_FP64 ? 8 : 4;
    long long nseg = (long long)g.nsegx * g.ny * g.nz;
    long long nspec = (long long)g.nzs * g.ny * g.nxh;
    // the spectrum buffer also holds the half spectra of the x rows inside the DCT (Neumann x)
    long long nspec_buf = g.xper ? nspec : std::max(nspec, (long long)g.nz * g.ny * (g.nx / 2 + 1));
    int nscanb = (int)((nseg + SCAN_CH - 1) / SCAN_CH);
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off += align_up(bytes > 0 ? bytes : 1);
        return p;
    };
    char* mask = take(g.N);
    char* velbits = take(g.N);
    char* segcnt[3];
    char* segoff[3];
    for (int c = 0; c < 3; ++c) segcnt[c] = take(nseg * sizeof(int));
    for (int c = 0; c < 3; ++c) segoff[c] = take(nseg * sizeof(int));
    char* scan_tmp = take(3 * (size_t)nscanb * sizeof(int));
    char* counts = take(8 * sizeof(int));
    char* ustar[3] = {nullptr, nullptr, nullptr};
    char* Nh[3] = {nullptr, nullptr, nullptr};
    for (int c = 0; c < g.ncomp; ++c) ustar[c] = take(g.N * esz);
    for (int c = 0; c < g.ncomp; ++c) Nh[c] = take(g.N * esz);
    char* rhs = take(g.N * esz);
    char* spec = take(nspec_buf * 2 * esz);
    char* piv = take(nspec * sizeof(double));
    char* piv32 = take(nspec * sizeof(float));
    char* use32 = take((size_t)g.nzs * g.nxh);
    char* order = take((size_t)g.nzs * g.nxh * sizeof(int));
    char* rtmp = g.xper ? nullptr : take(g.N * esz);            // reordered rows of the DCT
    char* twid = g.xper ? nullptr : take((size_t)g.nx * 2 * esz);   // cos, sin of pi k / 2nx
    char* fftab = take(((size_t)g.nx + 2) * 2 * esz);                 // own row-FFT twiddles
    char* dtemp = prec == IBM_FP32 ? take(nspec * 2 * sizeof(double)) : nullptr;
    char* fftw = take(fft_work);
    int npart = momentum_blocks(g) + IBM_DIV_PARTS;
    if (npart < DIAG_PART) npart = DIAG_PART;
    if (npart < 120 * 4) npart = 120 * 4;
    char* partials = take((size_t)npart * sizeof(double));
    char* scal = take(SCAL_N * sizeof(double));
    char* ytab = g.ystr ? take((size_t)YT_N * (g.ny + 1) * sizeof(double)) : nullptr;
    if (h && base) {
        h->ytab = (double*)ytab;
        h->mask = (uint8_t*)mask;
        h->velbits = (uint8_t*)velbits;
        for (int c = 0; c < 3; ++c) {
            h->segcnt[c] = (int*)segcnt[c];
            h->segoff[c] = (int*)segoff[c];
            h->ustar[c] = ustar[c];
            h->Nh[c] = Nh[c];
        }
        h->scan_tmp = (int*)scan_tmp;
        h->d_counts = (int*)counts;
        h->rhs = rhs;
        h->spec = spec;
        h->pivots = (double*)piv;
        h->pivots32 = (float*)piv32;
        h->use32 = (uint8_t*)use32;
        h->sys_order = (int*)order;
        h->dtemp = dtemp;
        h->rtmp = rtmp;
        h->twid = twid;
        h->fftab = fftab;
        h->fft_work = fftw;
        h->partials = (double*)partials;
        h->npartials = npart;
        h->scal = (double*)scal;
    }
    return off;
}

// IBM points per component a translating body's weights buffer holds
int moving_capacity(int count) { return count + count / 2 + 1024; }

// cap: IBM points per component to lay out (the counts, or a moving body's capacities)
size_t weights_layout(ibm_solver* h, char* base, const int* cap) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off += align_up(bytes > 0 ? bytes : 1);
        return p;
    };
    for (int c = 0; c < 3; ++c) {
        size_t n = (size_t)cap[c];
        char* idx = take(n * sizeof(int));
        char* lam = take(n * sizeof(double));
        char* src = take(n * sizeof(double));
        char* coef = take(3 * n * 4 * h->esz);
        if (base) {
            h->idx[c] = (int*)idx;
            h->lam[c] = (double*)lam;
            h->src[c] = (double*)src;
            h->coef[c] = coef;
        }
    }
    return off;
}

ibm_status check_handle(const ibm_solver* h) {
    if (!h) return ibm_set_error(IBM_E_INVALID, "handle is NULL");
    if (h->failed) return ibm_set_error(IBM_E_STATE, "handle failed after an earlier CUDA error");
    return IBM_OK;
}

void drop_graph(ibm_solver* h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_ready = false;
}

// A translating body at the start of a full step (reading R24): the level set with the centre at
// its place at t_n, the points classified again (those that turn fluid take the body velocity),
// the IBM lists, weights and stage coefficients rebuilt.  Blocking (reads the new counts back).
ibm_status body_advance(ibm_solver* h) {
    const double t = (double)h->steps * h->phys.dt;
    const int nd = h->geo.kind == IBM_GEOM_CYLINDER ? 2 : 3;
    for (int d = 0; d < nd; ++d) h->geo.p[d] = h->geo0[d] + h->body.ub[d] * t;
    ibm_status st = geom_classify(h, true);
    if (st != IBM_OK) return st;
    for (int c = 0; c < 3; ++c)
        if (h->counts[c] > h->cap[c]) {
            h->failed = true;
            return ibm_set_error(IBM_E_NOMEM, "the moving body's IBM points outgrew the weights buffer (component " +
                                                  std::to_string(c) + ": " + std::to_string(h->counts[c]) + " > " +
                                                  std::to_string(h->cap[c]) + ")");
        }
    st = geom_build_lists_and_weights(h);
    if (st == IBM_OK) st = geom_stage_coefficients(h);
    return st;
}

}  // namespace

ibm_status ibm_set_error(ibm_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

void timer_begin(ibm_solver* h, const char* name, cudaEvent_t* ev) {
    (void)name;
    *ev = nullptr;
    if (!h->timing) return;
    if (cudaEventCreate(ev) != cudaSuccess) { *ev = nullptr; return; }
    cudaEventRecord(*ev, h->stream);
}

void timer_end(ibm_solver* h, cudaEvent_t a, const char* name) {
    if (!h->timing || !a) return;
    cudaEvent_t b;
    if (cudaEventCreate(&b) != cudaSuccess) return;
    cudaEventRecord(b, h->stream);
    h->timers.push_back(KernelTimer{name, a, b});
}

extern "C" {

int ibm_version(void) { return 10000; }

const char* ibm_last_error(void) { return g_last_error.c_str(); }

ibm_status ibm_workspace_bytes(const ibm_grid_desc* grid, size_t* bytes) {
    ibm_status st = check_grid(grid);
    if (st != IBM_OK) return st;
    if (!bytes) return ibm_set_error(IBM_E_INVALID, "bytes is NULL");
    GridP g = make_gridp(grid);
    // cuFFT's work size depends only on the transform shapes (grid, periodic or Neumann x) and
    // the precision; remember it
    // so that repeated queries (a server admitting many solves) build no temporary plans
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, int>, size_t> known;
    const auto key = std::make_tuple(g.nx, g.ny, g.nz, grid->precision, g.xper);
    size_t work = 0;
    bool hit = false;
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = known.find(key);
        if (it != known.end()) { work = it->second; hit = true; }
    }
    if (!hit) {
        cufftHandle pf, pi, pfz, piz;
        st = make_plans(g, grid->precision, &pf, &pi, &pfz, &piz, &work);
        if (st != IBM_OK) return st;
        cufftDestroy(pf);
        cufftDestroy(pi);
        if (pfz) cufftDestroy(pfz);
        if (piz) cufftDestroy(piz);
        std::lock_guard<std::mutex> lock(mu);
        known[key] = work;
    }
    *bytes = carve(nullptr, g, grid->precision, work, nullptr);
    return IBM_OK;
}

ibm_status ibm_setup_geometry(const ibm_grid_desc* grid, const ibm_geom_desc* geom, const ibm_buffers* buffers,
                              void* stream, ibm_solver** out) {
    ibm_status st = check_grid(grid);
    if (st != IBM_OK) return st;
    if (!geom || !buffers || !out) return ibm_set_error(IBM_E_INVALID, "NULL argument");
    *out = nullptr;
    int kind = geom->kind;
    int need = kind == IBM_GEOM_PLANES ? 2 : kind == IBM_GEOM_CYLINDER ? 4 : kind == IBM_GEOM_SPHERE ? 5
             : kind == IBM_GEOM_SINE_WALL ? 4 : 0;
    if (kind == IBM_GEOM_SAMPLED) {
        const int nc = grid->ndim == 3 ? 3 : 2;
        for (int c = 0; c < nc; ++c)
            if (!geom->sdf[c] || ((uintptr_t)geom->sdf[c] & 7u))
                return ibm_set_error(IBM_E_INVALID, "sampled geometry: sdf[c] must be 8-byte aligned device arrays");
        if (grid->bc_lo[0] != IBM_BC_PERIODIC)
            return ibm_set_error(IBM_E_UNSUPPORTED, "sampled geometry needs a periodic x (the inflow face is not sampled)");
    }
    if (kind == IBM_GEOM_TUBES) {
        if (!geom->data || geom->ndata < 2) return ibm_set_error(IBM_E_INVALID, "tubes: data is missing");
        const double nt = geom->data[0], np = geom->data[1];
        if (!(nt >= 1 && nt <= TUBE_MAX && nt == (int)nt) || !(np >= 2 && np <= TUBE_PTS && np == (int)np))
            return ibm_set_error(IBM_E_INVALID, "tubes: need 1..12 tubes of 2..32 points");
        if (geom->ndata != 2 + (int)nt * (int)np * 4) return ibm_set_error(IBM_E_INVALID, "tubes: ndata mismatch");
        for (int q = 2; q < geom->ndata; ++q)
            if (!std::isfinite(geom->data[q])) return ibm_set_error(IBM_E_INVALID, "tubes: non-finite data");
    }
    if (kind < IBM_GEOM_NONE || kind > IBM_GEOM_SAMPLED) return ibm_set_error(IBM_E_INVALID, "bad geometry kind");
    if (geom->nparam < need) return ibm_set_error(IBM_E_INVALID, "too few geometry parameters");
    if (kind == IBM_GEOM_SINE_WALL && !(geom->param[2] != 0.0))
        return ibm_set_error(IBM_E_INVALID, "sine wall wavelength must be nonzero");
    if ((kind == IBM_GEOM_CYLINDER && std::fabs(geom->param[3]) != 1.0) ||
        (kind == IBM_GEOM_SPHERE && std::fabs(geom->param[4]) != 1.0))
        return ibm_set_error(IBM_E_INVALID, "body sign s must be +1 or -1");
    GridP g = make_gridp(grid);
    for (int c = 0; c < g.ncomp; ++c)
        if (!buffers->u[c]) return ibm_set_error(IBM_E_INVALID, "velocity buffer is NULL");
    if (!buffers->p || !buffers->work) return ibm_set_error(IBM_E_INVALID, "pressure or workspace buffer is NULL");
    if ((uintptr_t)buffers->work % ALIGN) return ibm_set_error(IBM_E_INVALID, "workspace must be 256-byte aligned");

    ibm_solver* h = new (std::nothrow) ibm_solver();
    if (!h) return ibm_set_error(IBM_E_INVALID, "host allocation failed");
    h->grid = *grid;
    h->geom = *geom;
    h->buf = *buffers;
    h->stream = (cudaStream_t)stream;
    h->gp = g;
    h->geo.kind = kind;
    for (int q = 0; q < 8; ++q) h->geo.p[q] = q < geom->nparam ? geom->param[q] : 0.0;
    for (int q = 0; q < 8; ++q) h->geo0[q] = h->geo.p[q];
    h->geo.ntubes = h->geo.npts = 0;
    std::memset(h->geo.tube, 0, sizeof(h->geo.tube));
    if (kind == IBM_GEOM_TUBES) {
        h->geo.ntubes = (int)geom->data[0];
        h->geo.npts = (int)geom->data[1];
        std::memcpy(h->geo.tube, geom->data + 2, (size_t)h->geo.ntubes * h->geo.npts * 4 * sizeof(double));
    }
    for (int c = 0; c < 3; ++c)
        h->geo.sdf[c] = (kind == IBM_GEOM_SAMPLED && c < g.ncomp) ? geom->sdf[c] : nullptr;
    h->geom.data = nullptr;   // the caller's array is not kept
    h->geom.ndata = 0;
    h->prec = grid->precision;
    h->esz = grid->precision == IBM_FP64 ? 8 : 4;
    h->N = g.N;
    h->nspec = (long long)g.nzs * g.ny * g.nxh;
    h->nseg = (long long)g.nsegx * g.ny * g.nz;

    size_t work = 0;
    st = make_plans(g, h->prec, &h->plan_f, &h->plan_i, &h->plan_fz, &h->plan_iz, &work);
    if (st != IBM_OK) { delete h; return st; }
    h->plans = true;
    size_t need_bytes = carve(nullptr, g, h->prec, work, nullptr);
    if (buffers->work_bytes < need_bytes) {
        ibm_destroy(h);
        return ibm_set_error(IBM_E_NOMEM, "workspace too small: need " + std::to_string(need_bytes) + " bytes");
    }
    carve(h, g, h->prec, work, (char*)buffers->work);
    h->fft_work_bytes = work;
    h->grid.y_faces = nullptr;   // the caller's array is not kept
    if (g.ystr) {
        h->ytab_host = y_tables(grid);
        cudaError_t e = cudaMemcpyAsync(h->ytab, h->ytab_host.data(), h->ytab_host.size() * sizeof(double),
                                        cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) {
            ibm_destroy(h);
            return ibm_set_error(IBM_E_CUDA, std::string("y tables: ") + cudaGetErrorString(e));
        }
        h->gp.yt = h->ytab;
    }
    if (h->prec == IBM_FP32) {   // the tridiagonal solve's FP64 systems run on a second stream
        cudaError_t e = cudaStreamCreateWithFlags(&h->tri_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->tri_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->tri_join, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            ibm_destroy(h);
            return ibm_set_error(IBM_E_CUDA, std::string("tridiagonal stream: ") + cudaGetErrorString(e));
        }
    }
    momentum_prepare(h);
    h->gp.kzm = momentum_default_kzm(h->gp, h->prec, momentum_uses_tma(h));
    bool plan_ok = true;
    for (cufftHandle p : {h->plan_f, h->plan_i, h->plan_fz, h->plan_iz})
        if (p && (cufftSetWorkArea(p, h->fft_work) != CUFFT_SUCCESS || cufftSetStream(p, h->stream) != CUFFT_SUCCESS))
            plan_ok = false;
    if (!plan_ok) {
        ibm_destroy(h);
        return ibm_set_error(IBM_E_CUDA, "cufft work area / stream setup failed");
    }
    st = geom_classify(h);
    if (st == IBM_OK) st = geom_pivots(h);
    if (st == IBM_OK) st = poisson_prepare(h);
    if (st == IBM_OK) {
        cudaError_t e = cudaMemsetAsync(h->scal, 0, SCAL_N * sizeof(double), h->stream);
        if (e != cudaSuccess) st = ibm_set_error(IBM_E_CUDA, cudaGetErrorString(e));
    }
    if (st != IBM_OK) {
        ibm_destroy(h);
        return st;
    }
    *out = h;
    return IBM_OK;
}

ibm_status ibm_weights_bytes(const ibm_solver* h, size_t* bytes) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    if (!bytes) return ibm_set_error(IBM_E_INVALID, "bytes is NULL");
    *bytes = weights_layout(const_cast<ibm_solver*>(h), nullptr, h->counts);
    return IBM_OK;
}

ibm_status ibm_weights_bytes_moving(const ibm_solver* h, size_t* bytes) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    if (!bytes) return ibm_set_error(IBM_E_INVALID, "bytes is NULL");
    int cap[3];
    for (int c = 0; c < 3; ++c) cap[c] = moving_capacity(h->counts[c]);
    *bytes = weights_layout(const_cast<ibm_solver*>(h), nullptr, cap);
    return IBM_OK;
}

ibm_status ibm_build_weights(ibm_solver* h, const ibm_physics* phys, void* weights, size_t weights_bytes) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    if (!phys || !weights) return ibm_set_error(IBM_E_INVALID, "NULL argument");
    if (!(phys->dt > 0.0) || !(phys->nu >= 0.0) || !std::isfinite(phys->dt) || !std::isfinite(phys->nu))
        return ibm_set_error(IBM_E_INVALID, "need dt > 0 and nu >= 0");
    if (phys->bmode < IBM_B_EXACT || phys->bmode > IBM_B_EXPLICIT) return ibm_set_error(IBM_E_INVALID, "bad bmode");
    if (!std::isfinite(phys->g_freq) || !std::isfinite(phys->g_amp[0]) || !std::isfinite(phys->g_amp[1]) ||
        !std::isfinite(phys->g_amp[2]))
        return ibm_set_error(IBM_E_INVALID, "g_amp and g_freq must be finite");
    if (phys->flow_mode != IBM_FLOW_FORCED && phys->flow_mode != IBM_FLOW_CONST_FLUX)
        return ibm_set_error(IBM_E_INVALID, "bad flow_mode");
    if (phys->flow_mode == IBM_FLOW_CONST_FLUX && !h->gp.xper)
        return ibm_set_error(IBM_E_INVALID, "a constant flow rate needs a periodic x direction");
    if ((uintptr_t)weights % ALIGN) return ibm_set_error(IBM_E_INVALID, "weights must be 256-byte aligned");
    // a moving body (reading R24)
    const bool translating = phys->body_u[0] != 0.0 || phys->body_u[1] != 0.0 || phys->body_u[2] != 0.0;
    const bool rotating = phys->body_omega != 0.0;
    for (double v : {phys->body_u[0], phys->body_u[1], phys->body_u[2], phys->body_omega})
        if (!std::isfinite(v)) return ibm_set_error(IBM_E_INVALID, "body_u and body_omega must be finite");
    if (translating || rotating) {
        const int kind = h->geo.kind;
        if (translating && rotating) return ibm_set_error(IBM_E_UNSUPPORTED, "a body that translates and rotates");
        if (translating && kind != IBM_GEOM_CYLINDER && kind != IBM_GEOM_SPHERE)
            return ibm_set_error(IBM_E_UNSUPPORTED, "a translating body is a cylinder or a sphere");
        if (rotating && kind != IBM_GEOM_CYLINDER)
            return ibm_set_error(IBM_E_UNSUPPORTED, "a rotating body is a cylinder about its own axis");
        if (!h->gp.xper || h->gp.ystr || phys->flow_mode != IBM_FLOW_FORCED || phys->body_force)
            return ibm_set_error(IBM_E_UNSUPPORTED, "a moving body needs a periodic x, a uniform y, the forced flow "
                                                    "and no body-force accounting");
    }
    int cap[3];
    for (int c = 0; c < 3; ++c) cap[c] = translating ? moving_capacity(h->counts[c]) : h->counts[c];
    size_t need = weights_layout(h, nullptr, cap);
    if (weights_bytes < need) return ibm_set_error(IBM_E_NOMEM, "weights buffer too small: need " + std::to_string(need));
    drop_graph(h);
    if (phys->body_force != 0 && phys->body_force != 1) return ibm_set_error(IBM_E_INVALID, "body_force is 0 or 1");
    if (phys->body_force && h->gp.ystr)
        return ibm_set_error(IBM_E_UNSUPPORTED, "the force accounting is written for a uniform y (a stretched "
                                                "second difference does not conserve momentum)");
    h->phys = *phys;
    for (int c = 0; c < 3; ++c) h->cap[c] = cap[c];
    weights_layout(h, (char*)weights, cap);
    h->body.kind = translating ? 1 : (rotating ? 2 : 0);
    for (int c = 0; c < 3; ++c) h->body.ub[c] = phys->body_u[c];
    h->body.om = phys->body_omega;
    h->body.xc = h->geo0[0];
    h->body.yc = h->geo0[1];
    {   // new physics: the force sums start again
        cudaError_t e = cudaMemsetAsync(h->scal + SCAL_FORCE, 0, (SCAL_N - SCAL_FORCE) * sizeof(double), h->stream);
        if (e != cudaSuccess) return ibm_set_error(IBM_E_CUDA, cudaGetErrorString(e));
    }
    st = geom_build_lists_and_weights(h);
    if (st == IBM_OK) st = geom_stage_coefficients(h);
    if (st != IBM_OK) return st;
    if (phys->flow_mode == IBM_FLOW_CONST_FLUX)
        for (int k = 0; k < 3; ++k)
            if (!(h->S[k] > 0.0)) return ibm_set_error(IBM_E_INVALID, "constant flow rate needs internal u points");
    h->weights_ready = true;
    return IBM_OK;
}

ibm_status ibm_step(ibm_solver* h, int nsteps, unsigned flags) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    if (!h->weights_ready) return ibm_set_error(IBM_E_STATE, "ibm_build_weights has not run");
    if (nsteps < 0) return ibm_set_error(IBM_E_INVALID, "nsteps < 0");
    if (flags & IBM_STEP_PREDICTOR_ONLY) {
        drop_graph(h);
        return run_substage(h, 0, true);
    }
    if (flags & IBM_STEP_GRAPH) {
        if (h->timing) return ibm_set_error(IBM_E_STATE, "timing is not available in graph mode");
        if (h->body.kind == 1)
            return ibm_set_error(IBM_E_UNSUPPORTED, "a translating body is classified again every step: no graph mode");
        if (h->proj_mode == IBM_PROJ_MASKED)
            return ibm_set_error(IBM_E_UNSUPPORTED, "the masked projection reads back its inner products: no graph mode");
        if (h->phys.g_amp[0] != 0.0 || h->phys.g_amp[1] != 0.0 || h->phys.g_amp[2] != 0.0)
            return ibm_set_error(IBM_E_UNSUPPORTED, "a time-periodic forcing changes every step: no graph mode");
        if (!h->graph_ready) {
            cudaGraph_t graph;
            IBM_CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
            long long before = h->launches;
            for (int k = 0; k < 3 && st == IBM_OK; ++k) st = run_substage(h, k, false);
            cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
            if (st != IBM_OK) return st;
            if (e != cudaSuccess) { h->failed = true; return ibm_set_error(IBM_E_CUDA, cudaGetErrorString(e)); }
            e = cudaGraphInstantiate(&h->graph, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) { h->failed = true; return ibm_set_error(IBM_E_CUDA, cudaGetErrorString(e)); }
            h->graph_launches = h->launches - before;
            h->launches = before;
            h->graph_ready = true;
        }
        for (int n = 0; n < nsteps; ++n) {
            IBM_CUDA_TRY(cudaGraphLaunch(h->graph, h->stream));
            h->launches += h->graph_launches;
            h->steps++;
        }
        return IBM_OK;
    }
    for (int n = 0; n < nsteps; ++n) {
        if (h->body.kind == 1) {
            st = body_advance(h);
            if (st != IBM_OK) return st;
        }
        for (int k = 0; k < 3; ++k) {
            st = run_substage(h, k, false);
            if (st != IBM_OK) return st;
        }
        h->steps++;
    }
    return IBM_OK;
}

ibm_status ibm_project(ibm_solver* h) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    return run_project(h);
}

ibm_status ibm_poisson(ibm_solver* h, void* rhs_inout) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    if (!rhs_inout) return ibm_set_error(IBM_E_INVALID, "rhs is NULL");
    return run_poisson(h, rhs_inout);
}

ibm_status ibm_diagnostics(ibm_solver* h, ibm_diag* out) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    if (!out) return ibm_set_error(IBM_E_INVALID, "out is NULL");
    double r[SCAL_N];
    st = run_diagnostics(h, r);
    if (st != IBM_OK) return st;
    {   // the force sums restart with the next step
        cudaError_t e = cudaMemsetAsync(h->scal + SCAL_FORCE, 0, 3 * sizeof(double), h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->scal + SCAL_FSTEPS, 0, sizeof(double), h->stream);
        if (e != cudaSuccess) {
            h->failed = true;
            return ibm_set_error(IBM_E_CUDA, cudaGetErrorString(e));
        }
    }
    const GridP& g = h->gp;
    // a stretched y: the sums carry each row's cell height and the velocity maxima are
    // already divided by their spacings (v's per row)
    double dV = g.dx * (g.ystr ? 1.0 : g.dy) * (g.ndim == 3 ? g.dz : 1.0);
    const double* s = r + 4;
    std::memset(out, 0, sizeof(*out));
    out->div_l2 = std::sqrt(s[0] / (double)g.N);
    out->div_linf = s[1];
    double d[3] = {g.dx, g.dy, g.dz};
    double cfl = 0.0;
    for (int c = 0; c < g.ncomp; ++c) {
        cfl += g.ystr ? s[2 + c] : s[2 + c] / d[c];
        out->flux[c] = s[5 + c] * dV;
        out->ke += 0.5 * s[8 + c] * dV;
    }
    out->cfl = cfl * h->phys.dt;
    out->pi = r[0];
    out->step = h->steps;
    out->force_steps = (long long)r[SCAL_FSTEPS];
    out->proj_iters = h->proj_mode == IBM_PROJ_MASKED ? h->proj_iters : 0;
    out->proj_resid = h->proj_mode == IBM_PROJ_MASKED ? h->proj_resid : 0.0;
    for (int c = 0; c < 3; ++c)
        out->force[c] = out->force_steps > 0 ? r[SCAL_FORCE + c] / r[SCAL_FSTEPS] : std::nan("");
    if (r[3] != 0.0) {
        // a TMA momentum block gave up waiting for its plane loads (a bounded wait ran out)
        out->status = IBM_E_TIMEOUT;
        h->failed = true;
        return ibm_set_error(IBM_E_TIMEOUT, "momentum predictor: a plane load did not complete");
    }
    bool finite = s[11] == 0.0 && std::isfinite(out->div_l2) && std::isfinite(out->ke);
    out->status = finite ? IBM_OK : IBM_E_DIVERGED;
    if (!finite) return ibm_set_error(IBM_E_DIVERGED, "non-finite values in the fields");
    return IBM_OK;
}

ibm_status ibm_wall_shear(ibm_solver* h, double wavelength, double* tau_x, double* tau1) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    if (!h->weights_ready) return ibm_set_error(IBM_E_STATE, "ibm_build_weights has not run");
    if (!(wavelength > 0.0) || !std::isfinite(wavelength)) return ibm_set_error(IBM_E_INVALID, "wavelength must be > 0");
    if ((size_t)h->N * h->esz < 2 * (size_t)h->gp.nx * sizeof(double))
        return ibm_set_error(IBM_E_UNSUPPORTED, "grid too small for the wall-shear scratch");
    return geom_wall_shear(h, wavelength, tau_x, tau1);
}

ibm_status ibm_projection_bytes(const ibm_solver* h, size_t* bytes) {
    if (!h) return ibm_set_error(IBM_E_INVALID, "NULL handle");
    if (!bytes) return ibm_set_error(IBM_E_INVALID, "bytes is NULL");
    const size_t one = ((size_t)h->N * sizeof(double) + ALIGN - 1) / ALIGN * ALIGN;
    *bytes = 5 * one;
    return IBM_OK;
}

ibm_status ibm_set_projection(ibm_solver* h, int mode, double tol, int maxit, void* buffer, size_t bytes) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    if (mode != IBM_PROJ_FULLBOX && mode != IBM_PROJ_MASKED) return ibm_set_error(IBM_E_INVALID, "bad projection mode");
    drop_graph(h);
    if (mode == IBM_PROJ_FULLBOX) {
        h->proj_mode = mode;
        for (double*& v : h->pcg) v = nullptr;
        return IBM_OK;
    }
    if (!(tol > 0.0) || !std::isfinite(tol) || maxit < 1) return ibm_set_error(IBM_E_INVALID, "need tol > 0 and maxit >= 1");
    if (h->gp.ystr) return ibm_set_error(IBM_E_UNSUPPORTED, "the masked projection is written for a uniform y");
    size_t need = 0;
    ibm_projection_bytes(h, &need);
    if (!buffer || (uintptr_t)buffer % ALIGN) return ibm_set_error(IBM_E_INVALID, "buffer must be 256-byte aligned");
    if (bytes < need) return ibm_set_error(IBM_E_NOMEM, "projection buffer too small: need " + std::to_string(need));
    const size_t one = need / 5;
    for (int q = 0; q < 5; ++q) h->pcg[q] = (double*)((char*)buffer + q * one);
    h->proj_mode = mode;
    h->proj_tol = tol;
    h->proj_maxit = maxit;
    h->proj_iters = 0;
    h->proj_resid = 0.0;
    return IBM_OK;
}

ibm_status ibm_get_classification(ibm_solver* h, unsigned char* host_mask, int* host_idx[3], int counts[3]) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    if (!counts) return ibm_set_error(IBM_E_INVALID, "counts is NULL");
    for (int c = 0; c < 3; ++c) counts[c] = h->counts[c];
    if (host_mask)
        IBM_CUDA_TRY(cudaMemcpyAsync(host_mask, h->mask, h->N, cudaMemcpyDeviceToHost, h->stream));
    if (host_idx) {
        for (int c = 0; c < 3; ++c) {
            if (!host_idx[c] || h->counts[c] == 0) continue;
            if (!h->weights_ready) return ibm_set_error(IBM_E_STATE, "lists are built by ibm_build_weights");
            IBM_CUDA_TRY(cudaMemcpyAsync(host_idx[c], h->idx[c], h->counts[c] * sizeof(int), cudaMemcpyDeviceToHost,
                                         h->stream));
        }
    }
    IBM_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return IBM_OK;
}

ibm_status ibm_get_weights(ibm_solver* h, double* host_lambda[3], double* host_src[3]) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    if (!h->weights_ready) return ibm_set_error(IBM_E_STATE, "ibm_build_weights has not run");
    for (int c = 0; c < 3; ++c) {
        if (h->counts[c] == 0) continue;
        if (host_lambda && host_lambda[c])
            IBM_CUDA_TRY(cudaMemcpyAsync(host_lambda[c], h->lam[c], h->counts[c] * sizeof(double),
                                         cudaMemcpyDeviceToHost, h->stream));
        if (host_src && host_src[c])
            IBM_CUDA_TRY(cudaMemcpyAsync(host_src[c], h->src[c], h->counts[c] * sizeof(double), cudaMemcpyDeviceToHost,
                                         h->stream));
    }
    IBM_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return IBM_OK;
}

ibm_status ibm_state_bytes(const ibm_solver* h, size_t* bytes) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    if (!bytes) return ibm_set_error(IBM_E_INVALID, "bytes is NULL");
    *bytes = 64 + (size_t)(h->gp.ncomp + 1) * h->N * h->esz;
    return IBM_OK;
}

ibm_status ibm_export_state(ibm_solver* h, void* host, size_t bytes) {
    size_t need = 0;
    ibm_status st = ibm_state_bytes(h, &need);
    if (st != IBM_OK) return st;
    if (!host || bytes < need) return ibm_set_error(IBM_E_INVALID, "host buffer NULL or too small");
    uint64_t hdr[8] = {STATE_MAGIC, (uint64_t)h->prec, (uint64_t)h->N, (uint64_t)h->gp.ncomp, (uint64_t)h->steps, 0, 0, 0};
    std::memcpy(host, hdr, sizeof(hdr));
    char* p = (char*)host + 64;
    size_t fb = h->N * h->esz;
    for (int c = 0; c < h->gp.ncomp; ++c, p += fb)
        IBM_CUDA_TRY(cudaMemcpyAsync(p, h->buf.u[c], fb, cudaMemcpyDeviceToHost, h->stream));
    IBM_CUDA_TRY(cudaMemcpyAsync(p, h->buf.p, fb, cudaMemcpyDeviceToHost, h->stream));
    IBM_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return IBM_OK;
}

ibm_status ibm_import_state(ibm_solver* h, const void* host, size_t bytes) {
    size_t need = 0;
    ibm_status st = ibm_state_bytes(h, &need);
    if (st != IBM_OK) return st;
    if (!host || bytes < need) return ibm_set_error(IBM_E_INVALID, "host buffer NULL or too small");
    uint64_t hdr[8];
    std::memcpy(hdr, host, sizeof(hdr));
    if (hdr[0] != STATE_MAGIC || hdr[1] != (uint64_t)h->prec || hdr[2] != (uint64_t)h->N ||
        hdr[3] != (uint64_t)h->gp.ncomp)
        return ibm_set_error(IBM_E_INVALID, "state snapshot does not match this solver");
    const char* p = (const char*)host + 64;
    size_t fb = h->N * h->esz;
    // one stream per field, after everything already queued on the solver's stream
    if (!h->copy_fork) {
        IBM_CUDA_TRY(cudaEventCreateWithFlags(&h->copy_fork, cudaEventDisableTiming));
        for (cudaStream_t& s : h->copy_streams) IBM_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    }
    IBM_CUDA_TRY(cudaEventRecord(h->copy_fork, h->stream));
    void* dst[4] = {h->buf.u[0], h->buf.u[1], h->gp.ncomp == 3 ? h->buf.u[2] : nullptr, h->buf.p};
    for (int q = 0; q < 4; ++q) {
        if (!dst[q]) continue;
        IBM_CUDA_TRY(cudaStreamWaitEvent(h->copy_streams[q], h->copy_fork, 0));
        IBM_CUDA_TRY(cudaMemcpyAsync(dst[q], p, fb, cudaMemcpyHostToDevice, h->copy_streams[q]));
        p += fb;
    }
    h->steps = (long long)hdr[4];
    for (cudaStream_t s : h->copy_streams) IBM_CUDA_TRY(cudaStreamSynchronize(s));
    return IBM_OK;
}

ibm_status ibm_timing(ibm_solver* h, int enable) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    for (auto& t : h->timers) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    h->timers.clear();
    h->timing = enable != 0;
    return IBM_OK;
}

ibm_status ibm_get_timing(ibm_solver* h, ibm_kernel_time* out, int max, int* count) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    if (!count) return ibm_set_error(IBM_E_INVALID, "count is NULL");
    IBM_CUDA_TRY(cudaStreamSynchronize(h->stream));
    std::vector<ibm_kernel_time> agg;
    for (auto& t : h->timers) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t.a, t.b);
        bool found = false;
        for (auto& a : agg)
            if (std::strcmp(a.name, t.name) == 0) {
                a.launches++;
                a.total_ms += ms;
                found = true;
            }
        if (!found) agg.push_back(ibm_kernel_time{t.name, 1, (double)ms});
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    h->timers.clear();
    *count = (int)agg.size();
    for (int q = 0; q < (int)agg.size() && q < max && out; ++q) out[q] = agg[q];
    return IBM_OK;
}

ibm_status ibm_autotune(ibm_solver* h, int* kz_momentum, int* kz_march) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    if (!h->weights_ready) return ibm_set_error(IBM_E_STATE, "ibm_build_weights has not run");
    int a = 0, b = 0;
    drop_graph(h);
    st = run_autotune(h, &a, &b);
    if (st != IBM_OK) return st;
    if (kz_momentum) *kz_momentum = a;
    if (kz_march) *kz_march = b;
    return IBM_OK;
}

ibm_status ibm_set_tiles(ibm_solver* h, int kz_momentum, int kz_march) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    const bool okm = kz_momentum >= MOM_KZ_MIN && kz_momentum <= KZM_CHOICES[7];
    bool okd = false;
    for (int v : KZD_CHOICES) okd |= v == kz_march;
    if (!okm || !okd) return ibm_set_error(IBM_E_INVALID, "z-chunk not among the supported choices");
    drop_graph(h);
    h->gp.kzm = kz_momentum;
    h->gp.kzd = kz_march;
    return IBM_OK;
}

ibm_status ibm_get_tiles(ibm_solver* h, int* kz_momentum, int* kz_march, int* tma) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    if (kz_momentum) *kz_momentum = h->gp.kzm;
    if (kz_march) *kz_march = h->gp.kzd;
    if (tma) *tma = momentum_uses_tma(h) ? 1 : 0;
    return IBM_OK;
}

ibm_status ibm_set_momentum_tma(ibm_solver* h, int enable) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    drop_graph(h);
    h->mom_tma = enable != 0;
    return IBM_OK;
}

ibm_status ibm_set_own_fft(ibm_solver* h, int mode, int* own) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    if (mode < 0 || mode > 2) return ibm_set_error(IBM_E_INVALID, "mode is 0, 1 or 2");
    drop_graph(h);
    h->own_fft_mode = mode;
    st = poisson_prepare(h);
    if (own) *own = (h->own_fft || h->dct_rows) ? 1 : 0;
    return st;
}

ibm_status ibm_set_tridiag_form(ibm_solver* h, int form) {
    ibm_status st = check_handle(h);
    if (st != IBM_OK) return st;
    if (form < 0 || form > 2) return ibm_set_error(IBM_E_INVALID, "form is 0, 1 or 2");
    drop_graph(h);
    h->tri_form = form;
    return IBM_OK;
}

ibm_status ibm_selftest_conversions(long long n, long long* mismatches) {
    if (n < 0 || !mismatches) return ibm_set_error(IBM_E_INVALID, "n >= 0 and a mismatch counter");
    return selftest_conversions(n, mismatches);
}

ibm_status ibm_launch_count(const ibm_solver* h, long long* count) {
    if (!h || !count) return ibm_set_error(IBM_E_INVALID, "NULL argument");
    *count = h->launches;
    return IBM_OK;
}

struct ibm_batch {
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> joins;
    cudaGraphExec_t exec = nullptr;
    std::vector<ibm_solver*> members;
    std::vector<int> steps;
    std::vector<long long> launches;   // kernels of each member in one replay
    long long job_cells = 0;           // members of at most this many cells: momentum by job kernel
    cudaEvent_t jobev = nullptr;
    bool failed = false;
};

ibm_status ibm_batch_create(void* stream, ibm_batch** out) {
    if (!out) return ibm_set_error(IBM_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!stream) return ibm_set_error(IBM_E_INVALID, "a batch needs a non-default stream (capture is not allowed on the legacy stream)");
    ibm_batch* b = new (std::nothrow) ibm_batch();
    if (!b) return ibm_set_error(IBM_E_INVALID, "host allocation failed");
    b->stream = (cudaStream_t)stream;
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        delete b;
        return ibm_set_error(IBM_E_CUDA, "cudaEventCreate failed");
    }
    *out = b;
    return IBM_OK;
}

ibm_status ibm_batch_set(ibm_batch* b, ibm_solver* const* members, const int* steps, int n) {
    if (!b || (n > 0 && (!members || !steps)) || n < 0) return ibm_set_error(IBM_E_INVALID, "bad batch arguments");
    if (b->failed) return ibm_set_error(IBM_E_STATE, "batch failed earlier");
    for (int q = 0; q < n; ++q) {
        ibm_status st = check_handle(members[q]);
        if (st != IBM_OK) return st;
        if (!members[q]->weights_ready) return ibm_set_error(IBM_E_STATE, "a member has no weights");
        if (members[q]->timing) return ibm_set_error(IBM_E_STATE, "disable member timing before batching");
        if (members[q]->proj_mode == IBM_PROJ_MASKED)
            return ibm_set_error(IBM_E_UNSUPPORTED, "a member uses the masked projection (no graph capture)");
        if (members[q]->phys.g_amp[0] != 0.0 || members[q]->phys.g_amp[1] != 0.0 || members[q]->phys.g_amp[2] != 0.0)
            return ibm_set_error(IBM_E_UNSUPPORTED, "a member has a time-periodic forcing (no graph capture)");
        if (members[q]->body.kind == 1)
            return ibm_set_error(IBM_E_UNSUPPORTED, "a member has a translating body (no graph capture)");
        if (steps[q] < 0) return ibm_set_error(IBM_E_INVALID, "negative step count");
    }
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    b->members.assign(members, members + n);
    b->steps.assign(steps, steps + n);
    while ((int)b->joins.size() < n) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return ibm_set_error(IBM_E_CUDA, "cudaEventCreate failed");
        b->joins.push_back(e);
    }
    if (n == 0) return IBM_OK;
    if (b->job_cells > 0 && !b->jobev) {
        if (cudaEventCreateWithFlags(&b->jobev, cudaEventDisableTiming) != cudaSuccess)
            return ibm_set_error(IBM_E_CUDA, "cudaEventCreate failed");
    }
    // job members (small, uniform y, no moving body): their momentum predictors run in one
    // persistent launch per substage and precision; the rest of each substage on their own streams
    std::vector<int> solo, jobs[2];
    for (int q = 0; q < n; ++q) {
        ibm_solver* h = b->members[q];
        const bool job = b->job_cells > 0 && h->N <= b->job_cells && !h->gp.ystr && h->body.kind == 0;
        if (job) jobs[h->prec == IBM_FP64 ? 1 : 0].push_back(q);
        else solo.push_back(q);
    }
    int maxsteps = 0;
    for (int p = 0; p < 2; ++p) {
        if ((int)jobs[p].size() > MOM_MAX_JOBS) return ibm_set_error(IBM_E_INVALID, "more job members than one launch takes");
        // most steps first, so that the members still stepping are always a prefix
        std::stable_sort(jobs[p].begin(), jobs[p].end(), [&](int a, int c) { return b->steps[a] > b->steps[c]; });
        if (!jobs[p].empty()) maxsteps = std::max(maxsteps, b->steps[jobs[p][0]]);
    }
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return ibm_set_error(IBM_E_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    ibm_status st = IBM_OK;
    b->launches.assign(n, 0);
    std::vector<long long> before(n);
    for (int q = 0; q < n; ++q) before[q] = b->members[q]->launches;
    cudaEventRecord(b->fork, b->stream);
    for (int q : solo) {
        if (st != IBM_OK) break;
        ibm_solver* h = b->members[q];
        cudaStreamWaitEvent(h->stream, b->fork, 0);
        for (int s = 0; s < b->steps[q] && st == IBM_OK; ++s)
            for (int k = 0; k < 3 && st == IBM_OK; ++k) st = run_substage(h, k, false);
        cudaEventRecord(b->joins[q], h->stream);
    }
    for (int s = 0; s < maxsteps && st == IBM_OK; ++s)
        for (int k = 0; k < 3 && st == IBM_OK; ++k) {
            std::vector<ibm_solver*> act[2];
            for (int p = 0; p < 2; ++p)
                for (int q : jobs[p])
                    if (b->steps[q] > s) act[p].push_back(b->members[q]);
            for (int p = 0; p < 2 && st == IBM_OK; ++p)
                st = momentum_jobs_launch(act[p].data(), (int)act[p].size(), k, b->stream);
            cudaEventRecord(b->jobev, b->stream);
            for (int p = 0; p < 2 && st == IBM_OK; ++p)
                for (int q : jobs[p]) {
                    if (b->steps[q] <= s || st != IBM_OK) continue;
                    ibm_solver* h = b->members[q];
                    cudaStreamWaitEvent(h->stream, b->jobev, 0);
                    h->mom_external = true;
                    st = run_substage(h, k, false);
                    h->mom_external = false;
                    cudaEventRecord(b->joins[q], h->stream);
                    cudaStreamWaitEvent(b->stream, b->joins[q], 0);
                }
        }
    for (int q : solo) cudaStreamWaitEvent(b->stream, b->joins[q], 0);
    for (int q = 0; q < n; ++q) {
        b->launches[q] = b->members[q]->launches - before[q];
        b->members[q]->launches = before[q];
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->stream, &graph);
    if (st != IBM_OK) {
        if (graph) cudaGraphDestroy(graph);
        b->failed = true;
        return st;
    }
    if (e != cudaSuccess) { b->failed = true; return ibm_set_error(IBM_E_CUDA, std::string("end capture: ") + cudaGetErrorString(e)); }
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { b->failed = true; return ibm_set_error(IBM_E_CUDA, std::string("instantiate: ") + cudaGetErrorString(e)); }
    return IBM_OK;
}

ibm_status ibm_batch_run(ibm_batch* b) {
    if (!b) return ibm_set_error(IBM_E_INVALID, "batch is NULL");
    if (b->failed) return ibm_set_error(IBM_E_STATE, "batch failed earlier");
    if (b->members.empty()) return IBM_OK;
    if (!b->exec) return ibm_set_error(IBM_E_STATE, "ibm_batch_set has not captured a graph");
    cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) { b->failed = true; return ibm_set_error(IBM_E_CUDA, cudaGetErrorString(e)); }
    for (size_t q = 0; q < b->members.size(); ++q) {
        b->members[q]->steps += b->steps[q];
        b->members[q]->launches += b->launches[q];
    }
    return IBM_OK;
}

ibm_status ibm_batch_jobs(ibm_batch* b, long long max_cells) {
    if (!b || max_cells < 0) return ibm_set_error(IBM_E_INVALID, "bad batch or max_cells < 0");
    b->job_cells = max_cells;
    return IBM_OK;
}

void ibm_batch_destroy(ibm_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->jobev) cudaEventDestroy(b->jobev);
    for (auto e : b->joins) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

void ibm_destroy(ibm_solver* h) {
    if (!h) return;
    for (auto& t : h->timers) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    drop_graph(h);
    for (cudaStream_t s : h->copy_streams)
        if (s) cudaStreamDestroy(s);
    if (h->copy_fork) cudaEventDestroy(h->copy_fork);
    if (h->tri_stream) cudaStreamDestroy(h->tri_stream);
    if (h->tri_fork) cudaEventDestroy(h->tri_fork);
    if (h->tri_join) cudaEventDestroy(h->tri_join);
    if (h->plans) {
        cufftDestroy(h->plan_f);
        cufftDestroy(h->plan_i);
        if (h->plan_fz) cufftDestroy(h->plan_fz);
        if (h->plan_iz) cufftDestroy(h->plan_iz);
    }
    momentum_release(h);
    delete h;
}

}  // extern "C"
