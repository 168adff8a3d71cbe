// Diagnostics for callers that cannot allocate device memory.
//
// ibm_diagnostics needs a solver handle, and a handle needs a caller-allocated
// workspace; its reduction kernel keeps per-block partial sums there.  This
// variant computes the same quantities from field pointers alone and keeps
// its partial sums in a fixed-size array of this library's own device memory
// (g_noalloc_scratch below), so it never calls cudaMalloc, cudaFree or any
// allocating library routine.
//
// Limits and sharing:
//   * at most NA_MAX_BLOCKS blocks of NA_CELLS_PER_BLOCK cells, i.e. grids of
//     up to 134,217,728 cells; larger grids are rejected with IBM_E_INVALID;
//   * the array exists once per GPU that loads the library, for as long as the
//     process lives (2048 * 12 + 16 doubles = 196,736 bytes);
//   * every call shares it and it keeps the last call's contents; each call
//     writes every slot it reads before reading it, so nothing has to start at
//     zero;  calls whose kernels overlap on the GPU (different streams, no
//     ordering between them) race on it and must be serialised by the caller.
#include "common.cuh"

#include <cmath>
#include <cstring>
#include <mutex>

namespace {

constexpr int NA_CELLS_PER_BLOCK = 65536;
constexpr int NA_MAX_BLOCKS = 2048;
constexpr int NA_VALS = 12;
constexpr int NA_THREADS = 256;
constexpr long long NA_MAX_CELLS = (long long)NA_MAX_BLOCKS * NA_CELLS_PER_BLOCK;
constexpr int NA_MAX_DEVICES = 64;

// [0, NA_MAX_BLOCKS * NA_VALS): per-block partials; then 16 slots for the final sums.
static __device__ __align__(256) double g_noalloc_scratch[NA_MAX_BLOCKS * NA_VALS + 16];

// Device address of g_noalloc_scratch per device ordinal (host code may not
// use the symbol itself as a device pointer).
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[NA_MAX_DEVICES] = {};

// Per-block partials of the diagnostics of ibm_diagnostics:
//   [0] sum div^2  [1] max |div|  [2..4] max |u_c|  [5..7] sum u_c  [8..10] sum u_c^2  [11] non-finite count
// with u_c summed over the internal points of component c.
template <typename T>
__global__ void __launch_bounds__(NA_THREADS) k_noalloc_partials(GridP g, const T* __restrict__ u,
                                                                 const T* __restrict__ v, const T* __restrict__ w,
                                                                 const T* __restrict__ p,
                                                                 const uint8_t* __restrict__ mask,
                                                                 double* __restrict__ part) {
    __shared__ double sh[NA_VALS][NA_THREADS / 32];
    DiagAcc<T> acc;
    const DiagInv<T> inv(1.0 / g.dx, 1.0 / g.dy, 1.0 / g.dz);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < g.N; id += stride) {
        const int i = (int)(id % g.nx);
        const long long row = id / g.nx;
        const int j = (int)(row % g.ny);
        const int k = (int)(row / g.ny);
        const T wc = g.ndim == 3 ? w[id] : T(0);
        const T wm = g.ndim == 3 ? w[i + (long long)g.nx * (j + (long long)g.ny * wrapi(k - 1, g.nz))] : T(0);
        // the -x face of the first cell is the inflow face in an inflow/outflow box
        const T uw = (g.xper || i > 0) ? u[row * g.nx + wrapi(i - 1, g.nx)]
                                       : ((mask[id] & IBM_MASK_FACE) ? (T)g.uin : T(0));
        acc.cell(g.ncomp, inv.v, u[id], uw, v[id], j > 0 ? v[id - g.nx] : T(0), wc, wm, p[id], mask[id]);
    }
    double a[NA_VALS];
    acc.finish(a);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = 0; q < NA_VALS; ++q) {
        const bool mx = (q == 1 || (q >= 2 && q <= 4));
        double x = mx ? warp_max(a[q]) : warp_sum(a[q]);
        if (lane == 0) sh[q][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < NA_VALS) {
        const int q = threadIdx.x;
        const bool mx = (q == 1 || (q >= 2 && q <= 4));
        double s = 0.0;
        for (int ww = 0; ww < NA_THREADS / 32; ++ww) s = mx ? fmax(s, sh[q][ww]) : s + sh[q][ww];
        part[blockIdx.x * NA_VALS + q] = s;
    }
}

__global__ void k_noalloc_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
    const int q = threadIdx.x;
    if (q >= NA_VALS) return;
    const bool mx = (q == 1 || (q >= 2 && q <= 4));
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s = mx ? fmax(s, part[b * NA_VALS + q]) : s + part[b * NA_VALS + q];
    out[q] = s;
}

// Once per device, with that device current: the device address of the scratch array.
ibm_status noalloc_scratch(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ibm_set_error(IBM_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return ibm_set_error(IBM_E_UNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        double* ptr = nullptr;
        e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return ibm_set_error(IBM_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
    return IBM_OK;
}

template <typename T>
ibm_status noalloc_run(const GridP& g, const void* u, const void* v, const void* w, const void* p,
                       const unsigned char* mask, cudaStream_t stream, double* scratch, double* host12) {
    const int nb = (int)((g.N + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK);
    const T* wt = g.ndim == 3 ? (const T*)w : (const T*)u;
    k_noalloc_partials<T><<<nb, NA_THREADS, 0, stream>>>(g, (const T*)u, (const T*)v, wt, (const T*)p, mask, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ibm_set_error(IBM_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    double* fin = scratch + (size_t)NA_MAX_BLOCKS * NA_VALS;
    k_noalloc_final<<<1, 32, 0, stream>>>(scratch, nb, fin);
    e = cudaGetLastError();
    if (e != cudaSuccess) return ibm_set_error(IBM_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    e = cudaMemcpyAsync(host12, fin, NA_VALS * sizeof(double), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return ibm_set_error(IBM_E_CUDA, std::string("read-back: ") + cudaGetErrorString(e));
    return IBM_OK;
}

}  // namespace

extern "C" ibm_status ibm_diagnostics_noalloc(const ibm_grid_desc* grid, const void* u, const void* v, const void* w,
                                              const void* p, const unsigned char* mask, double dt, void* stream,
                                              ibm_diag* out) {
    if (!grid || !out) return ibm_set_error(IBM_E_INVALID, "grid or out is NULL");
    if (grid->ndim != 2 && grid->ndim != 3) return ibm_set_error(IBM_E_INVALID, "ndim must be 2 or 3");
    for (int d = 0; d < 3; ++d)
        if (grid->n[d] < 1 || !(grid->L[d] > 0.0)) return ibm_set_error(IBM_E_INVALID, "n[d] >= 1 and L[d] > 0");
    if (grid->n[1] < 2 || (grid->ndim == 2 && grid->n[2] != 1))
        return ibm_set_error(IBM_E_INVALID, "need ny >= 2, and nz == 1 in 2D");
    if (grid->precision != IBM_FP64 && grid->precision != IBM_FP32)
        return ibm_set_error(IBM_E_INVALID, "bad precision");
    if (grid->bc_lo[2] != IBM_BC_PERIODIC || grid->bc_hi[2] != IBM_BC_PERIODIC)
        return ibm_set_error(IBM_E_UNSUPPORTED, "z must be periodic");
    if (grid->y_faces) return ibm_set_error(IBM_E_UNSUPPORTED, "a stretched y needs its per-row tables: use ibm_diagnostics");
    const bool xper = grid->bc_lo[0] == IBM_BC_PERIODIC && grid->bc_hi[0] == IBM_BC_PERIODIC;
    const bool xio = grid->bc_lo[0] == IBM_BC_INFLOW && grid->bc_hi[0] == IBM_BC_OUTFLOW;
    if (!xper && !xio)
        return ibm_set_error(IBM_E_UNSUPPORTED, "x must be periodic, or an inflow at -x with an outflow at +x");
    // the cell count is checked factor by factor, so that the product cannot overflow
    const long long n0 = grid->n[0], n1 = grid->n[1], n2 = grid->n[2];
    if (n0 > NA_MAX_CELLS || n1 > NA_MAX_CELLS / n0 || n2 > NA_MAX_CELLS / (n0 * n1))
        return ibm_set_error(IBM_E_INVALID, "grid of " + std::to_string(n0) + " x " + std::to_string(n1) + " x " +
                                                std::to_string(n2) +
                                                " cells exceeds the 134217728-cell limit of ibm_diagnostics_noalloc");
    const long long N = n0 * n1 * n2;
    if (!u || !v || !p || !mask || (grid->ndim == 3 && !w))
        return ibm_set_error(IBM_E_INVALID, "field or mask pointer is NULL");

    double* scratch = nullptr;
    ibm_status st = noalloc_scratch(&scratch);
    if (st != IBM_OK) return st;

    GridP g;
    std::memset(&g, 0, sizeof(g));
    g.nx = grid->n[0];
    g.ny = grid->n[1];
    g.nz = grid->n[2];
    g.ndim = grid->ndim;
    g.ncomp = grid->ndim == 3 ? 3 : 2;
    g.N = N;
    g.dx = grid->L[0] / grid->n[0];
    g.dy = grid->L[1] / grid->n[1];
    g.dz = grid->L[2] / grid->n[2];
    g.xper = xper;
    g.uin = xper ? 0.0 : grid->inflow[0];
    double s[NA_VALS];
    st = grid->precision == IBM_FP64
             ? noalloc_run<double>(g, u, v, w, p, mask, (cudaStream_t)stream, scratch, s)
             : noalloc_run<float>(g, u, v, w, p, mask, (cudaStream_t)stream, scratch, s);
    if (st != IBM_OK) return st;
    const double dV = g.dx * g.dy * (g.ndim == 3 ? g.dz : 1.0);
    const double dd[3] = {g.dx, g.dy, g.dz};
    std::memset(out, 0, sizeof(*out));
    out->div_l2 = std::sqrt(s[0] / (double)N);
    out->div_linf = s[1];
    double cfl = 0.0;
    for (int c = 0; c < g.ncomp; ++c) {
        cfl += s[2 + c] / dd[c];
        out->flux[c] = s[5 + c] * dV;
        out->ke += 0.5 * s[8 + c] * dV;
    }
    out->cfl = cfl * dt;
    out->step = -1;
    for (int c = 0; c < 3; ++c) out->force[c] = std::nan("");   // needs a solver's IBM points
    out->force_steps = 0;
    const bool finite = s[11] == 0.0 && std::isfinite(out->div_l2) && std::isfinite(out->ke);
    out->status = finite ? IBM_OK : IBM_E_DIVERGED;
    if (!finite) return ibm_set_error(IBM_E_DIVERGED, "non-finite values in the fields");
    return IBM_OK;
}
