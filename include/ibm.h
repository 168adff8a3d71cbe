/*
 * ibm.h -- C ABI of libibm.so: the per-time-step hot path of the implicit,
 * second-order sharp-interface immersed-boundary method of Luchini, Gatti,
 * Chiarini, Gattere, Atzori and Quadrio ("A simple and efficient second-order
 * immersed-boundary method for the incompressible Navier-Stokes equations"),
 * on one GB300 GPU (sm_103a).
 *
 * Problem (paper Sec. 2.1, Eq. ns): du/dt + (u.grad)u - nu lap u + grad p = g,
 * div u = 0, on a staggered Cartesian grid with 3-point central differences.
 * The body enters only as a per-point increase lambda of the Laplacian's
 * centre weight (Sec. 2.2, Eq. disclapl-extr / lambda), applied implicitly
 * (Sec. 2.4, Eq. Bexpr / expint) inside the Rai-Moin RK3 (Eq. rk3-rai); each
 * substage ends with the unmodified pressure projection (Sec. 2.1, Sec. 3.3).
 *
 * Conventions
 *   - Every array is (nz, ny, nx) with x fastest; linear index i + nx*(j + ny*k).
 *     Cell (i,j,k) has its centre at origin + ((i+1/2)dx, (j+1/2)dy, (k+1/2)dz),
 *     dx = L[0]/n[0] etc.; u(i,j,k) sits on the cell's +x face, v on its +y
 *     face, w on its +z face.  In 2D, nz = 1 and w is absent.
 *   - z must be periodic; y is bounded by box walls (no-slip or free-slip),
 *     and v(i, ny-1, k) lies on the +y wall and is held at zero.  x is either
 *     periodic, or has an inflow at -x (bc_lo[0] = IBM_BC_INFLOW, velocity
 *     inflow[0] on the fluid part of the face, zero tangential velocity) and a
 *     convective outflow at +x (bc_hi[0] = IBM_BC_OUTFLOW): u(nx-1, j, k) lies
 *     on the outflow face and follows du/dt + U_c du/dx = 0, U_c the inflow
 *     flux over the fluid outflow area, shifted each substage so that outflow
 *     and inflow fluxes balance; the Poisson problem is then Neumann in x.
 *     Other combinations return IBM_E_UNSUPPORTED.
 *   - Memory: the caller allocates every device buffer (fields, workspace,
 *     weights) and keeps it alive until ibm_destroy.  The library never
 *     allocates or frees device memory except inside cuFFT plans (twiddle
 *     tables); cuFFT's work area comes from the caller's workspace.
 *   - Streams: all device work is enqueued on the stream given at setup.
 *     An IBM_FP32 handle also owns one internal stream (created at setup,
 *     destroyed by ibm_destroy): the tridiagonal solve forks its FP64 systems
 *     onto it and joins back with events recorded on the setup stream, so the
 *     work stays ordered on that stream and a captured step holds both.
 *     Calls are asynchronous except where stated ("blocking").
 *   - Errors: every call returns an ibm_status; nothing throws across the
 *     ABI.  ibm_last_error() gives a thread-local message.  After a CUDA
 *     error the handle is failed and later calls return IBM_E_STATE.
 *   - Precision: IBM_FP64 runs every step in FP64.  IBM_FP32 stores fields in
 *     FP32 and runs the momentum stencil, the IBM division, the per-cell
 *     divergence and the FFTs in FP32.  FP64 arithmetic is kept for the
 *     tridiagonal sweeps of the near-singular spectral systems (K dy^2 < 1,
 *     the low modes), the Thomas pivots of every system, the IBM weights,
 *     and the sums of every reduction (flow rate, outflow balance,
 *     diagnostics); the strongly dominant systems (K dy^2 >= 1, condition
 *     number <= 5) sweep in FP32.
 */
#ifndef IBM_H
#define IBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IBM_OK = 0,
    IBM_E_INVALID = -1,      /* bad argument, size or pointer */
    IBM_E_CUDA = -2,         /* a CUDA or cuFFT call failed */
    IBM_E_NOMEM = -3,        /* a caller buffer is smaller than required */
    IBM_E_UNSUPPORTED = -4,  /* valid request outside what this build implements */
    IBM_E_DIVERGED = -5,     /* non-finite field found by ibm_diagnostics */
    IBM_E_TIMEOUT = -6,      /* a bounded device wait gave up */
    IBM_E_STATE = -7         /* handle failed earlier, or call out of order */
} ibm_status;

/* box boundary condition per face */
enum { IBM_BC_PERIODIC = 0, IBM_BC_NOSLIP = 1, IBM_BC_FREESLIP = 2, IBM_BC_INFLOW = 3, IBM_BC_OUTFLOW = 4 };
/* field precision */
enum { IBM_FP64 = 0, IBM_FP32 = 1 };
/* geometry kinds: level set phi < 0 is fluid, phi >= 0 is solid (Sec. 3.3) */
enum {
    IBM_GEOM_NONE = 0,      /* no body                                                      */
    IBM_GEOM_PLANES = 1,    /* param = {a, b}: fluid for a < y < b; the plane y=b moves       */
    IBM_GEOM_CYLINDER = 2,  /* param = {xc, yc, R, s}: axis along z; s=+1 fluid inside,
                               s=-1 fluid outside; phi = s((x-xc)^2+(y-yc)^2-R^2)            */
    IBM_GEOM_SPHERE = 3,    /* param = {xc, yc, zc, R, s}                                    */
    IBM_GEOM_SINE_WALL = 4, /* param = {y0, A, lam, ytop}: fluid for
                               y0 + A sin(2 pi x/lam) < y < ytop; the wavy wall moves         */
    IBM_GEOM_TUBES = 5,     /* union of tubes: data = {ntubes, npts, then per tube npts points
                             * (x, y, z, r)}, ntubes <= 12, 2 <= npts <= 32; fluid inside.
                             * phi = min over tubes and segments of |X - C| - r(t), with C the
                             * projection of X on the segment, t in [0,1] its position and r
                             * interpolated linearly between the segment's end radii        */
    IBM_GEOM_SAMPLED = 6    /* phi sampled at the velocity points: sdf[c] of ibm_geom_desc.
                             * Fluid where phi < 0; delta = Delta phi_P / (phi_P - phi_Q)
                             * (linear interpolation, Sec. 2.2 leaves the root-finding open).
                             * Needs a periodic x (the inflow face is not a sample point).   */
};
/* B(x) of Eq. (Bexpr), x = lambda c_k dt */
enum { IBM_B_EXACT = 0, IBM_B_EULER = 1, IBM_B_TAYLOR2 = 2,
       IBM_B_EXPLICIT = 3 /* the classic explicit treatment the paper compares against (end of
                           * Sec. 2.5): -lambda w in the explicit right-hand side, no division */ };
/* forcing */
enum { IBM_FLOW_FORCED = 0, IBM_FLOW_CONST_FLUX = 1 };
/* ibm_step flags */
enum {
    IBM_STEP_PREDICTOR_ONLY = 1u, /* run only the stage-1 predictor: fields <- u*, no projection */
    IBM_STEP_GRAPH = 2u           /* replay the step from a CUDA graph captured on first use   */
};
/* packed mask bits returned by ibm_get_classification */
enum { IBM_MASK_U = 1, IBM_MASK_V = 2, IBM_MASK_W = 4, IBM_MASK_P = 8,
       IBM_MASK_IBM_U = 16, IBM_MASK_IBM_V = 32, IBM_MASK_IBM_W = 64,
       /* x inflow/outflow only: at i = 0 the inflow face of the row is fluid, at
        * i = nx-1 the outflow face (u there) is fluid */
       IBM_MASK_FACE = 128 };

typedef struct {
    int ndim;           /* 2 or 3 */
    int n[3];           /* cells nx, ny, nz; nz = 1 when ndim = 2; ny >= 2 */
    double L[3];        /* box lengths */
    double origin[3];   /* box lower corner */
    int bc_lo[3];       /* IBM_BC_* per direction, low face */
    int bc_hi[3];       /* IBM_BC_* per direction, high face */
    int precision;      /* IBM_FP64 or IBM_FP32 */
    double inflow[3];   /* x = IBM_BC_INFLOW / IBM_BC_OUTFLOW: velocity through the inflow face
                         * (inflow[0] used; uniform on the fluid part of the face) */
    const double* y_faces; /* stretched wall-normal grid (Sec. 4.2 and Table wavy-parameters
                         * stretch the wall-normal spacing): host array of the n[1] + 1 face
                         * heights, strictly increasing from origin[1] to origin[1] + L[1]
                         * (within 1e-12 L[1]), read once by ibm_setup_geometry; NULL for a
                         * uniform y.  Cell centres lie midway between faces and v sits on
                         * the faces.  Not with the masked projection, the body force or
                         * ibm_diagnostics_noalloc (IBM_E_UNSUPPORTED). */
} ibm_grid_desc;

typedef struct {
    int kind;           /* IBM_GEOM_* */
    int nparam;         /* number of valid entries in param */
    double param[32];   /* kind-specific parameters (see the enum) */
    const double* data; /* IBM_GEOM_TUBES: host array of ndata doubles (see the enum), read at
                         * setup; NULL for the other kinds */
    int ndata;
    const double* sdf[3]; /* IBM_GEOM_SAMPLED: DEVICE arrays, FP64, layout (nz, ny, nx) x fastest,
                           * phi of component c at its own points (u on +x faces, v on +y, w on +z);
                           * sdf[2] unused in 2D.  Caller-owned: read by ibm_setup_geometry and by
                           * every ibm_build_weights call, so they must stay valid and unchanged
                           * while weights may be rebuilt.  NULL for the other kinds. */
} ibm_geom_desc;

typedef struct {
    void* u[3];         /* device: u, v, w fields, N elements of the grid precision each;
                           u[2] unused in 2D.  Hold the current velocity between calls. */
    void* p;            /* device: pressure, N elements */
    void* work;         /* device workspace, 256-byte aligned, ibm_workspace_bytes() bytes */
    size_t work_bytes;
} ibm_buffers;

typedef struct {
    double nu;          /* kinematic viscosity (1/Re) */
    double dt;          /* time step */
    double g[3];        /* uniform body force */
    int bmode;          /* IBM_B_* */
    int flow_mode;      /* IBM_FLOW_* */
    double target_flux; /* IBM_FLOW_CONST_FLUX: target volume integral of u over internal u points */
    double wall_u[3];   /* velocity of the moving surface (see the geometry kinds) */
    int no_ibm;         /* 1: lambda := 0, no wall source (the staircase baseline) */
    int body_force;     /* 1: every full step adds the force of the fluid on the body to the
                         * sums ibm_diagnostics reports (two small launches per substage over the
                         * IBM points); 0: not computed */
    double g_amp[3];    /* time-periodic forcing (Sec. 2.5): the body force is g + g_amp sin(2 pi
                         * g_freq t), t taken at each RK3 stage's own time (t_n, t_n + 8/15 dt,
                         * t_n + 2/3 dt) with t_n = completed steps * dt.  Nonzero g_amp refuses
                         * IBM_STEP_GRAPH and batches (the stage values change every step). */
    double g_freq;
    double body_u[3];   /* a translating body (Sec. 3.1, end: the IBM applies in the frame in which the
                         * body is at rest; reading R24): a CYLINDER or SPHERE whose centre moves with
                         * this constant velocity.  At the start of every full step the points are
                         * classified again with the centre at its place at t_n = completed steps *
                         * dt, the IBM weights rebuilt with the wall moving at body_u, and points
                         * that became fluid take body_u; the body's own points read and hold
                         * body_u.  Zero: at rest. */
    double body_omega;  /* a CYLINDER rotating about its own axis at this rate (counter-clockwise):
                         * its points hold omega x r and each crossed arm's wall velocity is
                         * omega x r at the crossing.  Not with body_u.  A moving body needs a
                         * periodic x, a uniform y, the forced flow (no constant flow rate) and
                         * body_force = 0; a translating one refuses IBM_STEP_GRAPH and batches
                         * (its weights change every step) and sizes the weights buffer with room
                         * for 1.5 x its first IBM-point counts + 1024 per component
                         * (IBM_E_NOMEM at a step that would exceed it). */
} ibm_physics;

typedef struct {
    double div_l2;      /* sqrt(mean over cells of (D u)^2) */
    double div_linf;    /* max over cells |D u| */
    double cfl;         /* dt * sum_c max_internal |u_c| / d_c */
    double flux[3];     /* sum over internal points of u_c * cell volume */
    double ke;          /* 1/2 sum over internal points of u_c^2 * cell volume */
    double pi;          /* forcing of the last constant-flow-rate substage */
    long long step;     /* completed full steps */
    int status;         /* IBM_OK or IBM_E_DIVERGED */
    double force[3];    /* ibm_physics.body_force = 1: mean over the full steps since the previous
                         * ibm_diagnostics call (or ibm_build_weights) of the force of the fluid on
                         * the body, from the discrete momentum budget: the momentum the IBM
                         * division, the right-hand side's faces toward solid points and the
                         * pressure at the ends of the runs of internal points exchange with the
                         * fluid (the paper reports drag and lift, Sec. 4.1, without a method;
                         * this is the reading taken).  NaN when no step was counted. */
    long long force_steps; /* full steps in that mean; the call resets the sums */
    int proj_iters;     /* IBM_PROJ_MASKED: iterations of the last projection solve (0 otherwise) */
    double proj_resid;  /* its final residual over the right-hand side (2-norms) */
} ibm_diag;

typedef struct {
    const char* name;   /* kernel name */
    int launches;       /* timed launches since the last reset */
    double total_ms;    /* summed CUDA-event duration */
} ibm_kernel_time;

typedef struct ibm_solver ibm_solver;
typedef struct ibm_batch ibm_batch;

/* Library version (major*10000 + minor*100 + patch). */
int ibm_version(void);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char* ibm_last_error(void);

/* Bytes of device workspace a grid needs (mask, RK history, predictor,
 * Poisson spectrum and pivots, cuFFT work area, reduction scratch).
 * Creates and destroys a temporary cuFFT plan to size its work area, so a
 * CUDA device must be present.  Blocking. */
ibm_status ibm_workspace_bytes(const ibm_grid_desc* grid, size_t* bytes);

/* Classify the staggered grids against the geometry (Sec. 3.3) and prepare
 * the Poisson solver.  `stream` is a cudaStream_t (NULL = legacy default).
 * On success *out holds a new handle.  Copies grid and geometry; keeps the
 * buffer pointers.  Blocking: the IBM-point counts are read back. */
ibm_status ibm_setup_geometry(const ibm_grid_desc* grid, const ibm_geom_desc* geom,
                              const ibm_buffers* buffers, void* stream, ibm_solver** out);

/* Device bytes the weights need (IBM-point lists, lambda, wall source and
 * per-stage coefficients), known after ibm_setup_geometry. */
ibm_status ibm_weights_bytes(const ibm_solver* h, size_t* bytes);
/* The weights buffer a translating body needs (ibm_physics.body_u, reading R24 of Sec. 3.1):
 * room for 3/2 of the present IBM-point counts + 1024 per component, since the counts change
 * as the body crosses the grid. */
ibm_status ibm_weights_bytes_moving(const ibm_solver* h, size_t* bytes);

/* Compute delta per crossed stencil arm, lambda (Sec. 2.2, Eq. lambda) and
 * the per-stage implicit coefficients (Eq. Bexpr, rk3-rai) into the caller's
 * device buffer `weights` (256-byte aligned).  May be called again with new
 * physics.  Blocking (reads back the flux-control sums). */
ibm_status ibm_build_weights(ibm_solver* h, const ibm_physics* phys, void* weights,
                             size_t weights_bytes);

/* Advance nsteps full RK3 steps (3 substages, each: predictor with the
 * implicit IBM division, then projection).  Asynchronous on the stream. */
ibm_status ibm_step(ibm_solver* h, int nsteps, unsigned flags);

/* Zero the velocity outside the fluid and project it onto divergence-free
 * fields (initial conditions); the pressure is unchanged.  Asynchronous. */
ibm_status ibm_project(ibm_solver* h);

/* Solve D G phi = rhs on the full box (x, z periodic, homogeneous Neumann in
 * y), zero box mean; `rhs_inout` is a device array of N grid-precision values
 * overwritten by phi.  The rhs must sum to zero.  Asynchronous. */
ibm_status ibm_poisson(ibm_solver* h, void* rhs_inout);

/* Wall-shear stress of the current velocity along a lower wall (Sec. 4.2 reports the Fourier
 * components tau_1c, tau_1s of the time-averaged tau(x) over the wavy wall).  Per column of u
 * points, the lowest internal point P whose -y arm crosses the wall (distance delta, found as for
 * the weights) and the internal point Q above it: tau = nu u'(0) of the quadratic through 0 at the
 * wall, u_P and u_Q (u_P / delta when Q is not internal), averaged over z.  tau_x: host array of nx
 * values (NaN in columns without such a point) or NULL; tau1: host [2] = {tau_1c, tau_1s} =
 * (2/nx) sum_i tau(x_i) {cos, sin}(2 pi x_i / wavelength), x_i the u points' x, or NULL.
 * Uses the divergence scratch (call between steps).  Blocking. */
ibm_status ibm_wall_shear(ibm_solver* h, double wavelength, double* tau_x, double* tau1);

/* Projection operators.  IBM_PROJ_FULLBOX (the default): the unmodified projection, D G of the
 * whole box, every face whose velocity is not prescribed corrected.  IBM_PROJ_MASKED: the
 * literal reading of Sec. 3.3 ("only the internal pressure points are updated"): D M G phi =
 * D u* over the internal cells, M keeping only internal faces, and only internal faces
 * corrected, so external faces keep u* = 0 and every internal cell of the field the operators
 * read is divergence-free.  Solved by conjugate gradients in FP64 preconditioned with the
 * full-box solve; each iteration reads back its inner products (no graph capture). */
enum { IBM_PROJ_FULLBOX = 0, IBM_PROJ_MASKED = 1 };

/* Device bytes IBM_PROJ_MASKED needs: five FP64 fields of N values. */
ibm_status ibm_projection_bytes(const ibm_solver* h, size_t* bytes);

/* Select the projection.  IBM_PROJ_MASKED: `buffer` is a caller-owned device buffer of at
 * least ibm_projection_bytes (256-byte aligned, kept until the mode changes or the solver is
 * destroyed); the iteration stops at a residual of tol times the right-hand side (2-norm) or
 * after maxit iterations (the last count and residual are in ibm_diag).  IBM_PROJ_FULLBOX:
 * buffer, tol and maxit are ignored.  IBM_STEP_GRAPH and batches refuse IBM_PROJ_MASKED
 * (IBM_E_UNSUPPORTED).  Blocking only in that it drops a captured graph. */
ibm_status ibm_set_projection(ibm_solver* h, int mode, double tol, int maxit, void* buffer, size_t bytes);

/* Norms, CFL, flux, kinetic energy of the current fields.  Blocking; returns
 * IBM_E_DIVERGED (and fills out->status) if a field is not finite. */
ibm_status ibm_diagnostics(ibm_solver* h, ibm_diag* out);

/* Blocking copies of the classification: host_mask (N bytes, or NULL), the
 * IBM-point lists (ascending linear index; host_idx[c] may be NULL) and
 * their lengths counts[3] (always written). */
ibm_status ibm_get_classification(ibm_solver* h, unsigned char* host_mask, int* host_idx[3],
                                  int counts[3]);

/* Blocking copies of lambda and the wall source per IBM point, in list order
 * (either array pointer may be NULL).  Needs ibm_build_weights first. */
ibm_status ibm_get_weights(ibm_solver* h, double* host_lambda[3], double* host_src[3]);

/* Bytes of a state snapshot (u, v, w, p, RK history, step counter). */
ibm_status ibm_state_bytes(const ibm_solver* h, size_t* bytes);
/* Blocking copy of the state to / from a host buffer of ibm_state_bytes(). */
ibm_status ibm_export_state(ibm_solver* h, void* host, size_t bytes);
ibm_status ibm_import_state(ibm_solver* h, const void* host, size_t bytes);

/* Kernel timing with CUDA events on the solver's stream: enable (1) or
 * disable (0); enabling resets the counters.  Not available in graph mode. */
ibm_status ibm_timing(ibm_solver* h, int enable);
/* Blocking: per-kernel launches and summed durations since the last reset. */
ibm_status ibm_get_timing(ibm_solver* h, ibm_kernel_time* out, int max, int* count);
/* Tile autotuner (not in the paper: a GB300 tuning aid).  Times the momentum
 * predictor for every z-chunk in {8, 12, 16, 24, 32, 48, 64, 86} and the divergence
 * kernel for every z-chunk in {4, 8, 16, 32} on this solver's own grid and
 * keeps the fastest of each; returns the choices (either pointer may be NULL).
 * Overwrites only scratch (predictor, RHS history, divergence), so call it
 * between full steps, outside stream capture.  Blocking.  2D grids keep the
 * defaults. */
ibm_status ibm_autotune(ibm_solver* h, int* kz_momentum, int* kz_march);
/* Set the z-chunks directly (values from a cached autotune).  kz_momentum:
 * the planes one momentum block marches, 8 to 86 (the last chunk takes the
 * rest); kz_march one of {4, 8, 16, 32}.  IBM_E_INVALID otherwise. */
ibm_status ibm_set_tiles(ibm_solver* h, int kz_momentum, int kz_march);
/* The z-chunks in use, and whether the momentum predictor runs its TMA form
 * (*tma = 1: plane tiles arrive by tensor copies into a shared-memory ring;
 * 0: loads through registers).  Any pointer may be NULL. */
ibm_status ibm_get_tiles(ibm_solver* h, int* kz_momentum, int* kz_march, int* tma);
/* Allow (1, the default) or forbid (0) the TMA form of the momentum
 * predictor.  It is used only on 3D grids with nx a multiple of 16; both forms
 * compute the same update (a tuning and testing aid, not in the paper). */
ibm_status ibm_set_momentum_tma(ibm_solver* h, int enable);
/* The library's own real FFT of the x rows (a warp per row, self-sorting mixed-radix FFT in
 * shared memory) against cuFFT's R2C / C2R.  It can run where nx = 2M with M a product of 2, 3
 * and 5 (M <= 1920 in FP32, 960 in FP64).  mode 0: never; 1: wherever it can; 2 (the default):
 * on a periodic x where M has a factor 3 or 5 (measured faster than cuFFT there, slower on
 * powers of two), on an inflow/outflow x wherever it can (the DCT of a row in one pass).  Where
 * it runs, the divergence is computed inside the forward row transform (except under the masked
 * projection).  *own reports whether it runs on this grid (may be NULL).  Both paths compute
 * the same transform. */
ibm_status ibm_set_own_fft(ibm_solver* h, int mode, int* own);
/* Form of the FP64 tridiagonal sweeps (the near-singular systems K dy^2 < 1 in FP32 mode,
 * every system in FP64 mode).  form 0 (the default) and 1: one warp per system (affine-map
 * scans over the lanes; all rows of a system in flight at once) where ny <= 1024, else one
 * thread per system; 2: one thread per system (the least FP64 work, but a dependent chain
 * of 2 ny steps that waits on memory).  Both compute the same Thomas solve in FP64
 * arithmetic (a tuning and testing aid, not in the paper).  IBM_E_INVALID for other values. */
ibm_status ibm_set_tridiag_form(ibm_solver* h, int form);
/* Self-test (no counterpart in the paper): the FP64 tridiagonal sweeps of FP32 fields
 * convert between FP32 and FP64 with integer instructions (exact widening; narrowing
 * rounded to nearest, ties to even).  This runs n bit patterns (random doubles, exact
 * rounding ties, random floats, doubles near the FP32 range ends) through both those
 * conversions and the hardware's, on the current device's legacy default stream, and
 * returns in *mismatches the count whose results differ in any bit.  Blocking. */
ibm_status ibm_selftest_conversions(long long n, long long* mismatches);

/* Batched stepping of many resident solves (continuous batching for serving
 * many small solves; the paper has no counterpart).  A batch owns a
 * non-default stream.  ibm_batch_set captures ONE CUDA graph that forks onto
 * every member's own stream, runs steps[i] full steps of member i there and
 * joins back, so the members' kernels overlap on the device; call it again
 * whenever the member set or the step counts change.  Members must have
 * weights, timing off, and streams other than the legacy default stream.
 * ibm_batch_run replays the graph once (asynchronous on the batch stream)
 * and advances each member's step counter by steps[i].  Members must not be
 * stepped outside the batch while a replay may be running. */
ibm_status ibm_batch_create(void* stream, ibm_batch** out);
ibm_status ibm_batch_set(ibm_batch* b, ibm_solver* const* members, const int* steps, int n);
ibm_status ibm_batch_run(ibm_batch* b);
/* Members of at most max_cells cells (uniform y, no moving body) advance their momentum
 * predictors -- the fused RHS, RK3 and implicit IBM division of Sec. 2.4 -- in ONE
 * persistent launch per substage and precision: a fixed grid of blocks walks a work list of
 * every such member's (column, z chunk) tiles, each with its own grid, fields, stage constants
 * and coefficients (at most 40 members per precision).  The rest of each member's substage
 * (flow-rate control, projection) stays on its own stream between those launches, so these
 * members step in lockstep, substage by substage.  Their update is the register form of the
 * predictor (compiled into another kernel: FP32 results may differ from the member's own
 * launch in the last bits).  0 (the default) turns
 * this off.  Takes effect at the next ibm_batch_set. */
ibm_status ibm_batch_jobs(ibm_batch* b, long long max_cells);
void ibm_batch_destroy(ibm_batch* b);

/* Kernels this library has launched through this handle (a running count). */
ibm_status ibm_launch_count(const ibm_solver* h, long long* count);

/* Diagnostics without a handle and without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * must not allocate device memory themselves or through this library --
 * for instance code whose device memory is owned entirely by another
 * allocator (a framework's caching pool), or a latency-critical loop that
 * cannot afford cudaMalloc's implicit synchronisation.  It computes what
 * ibm_diagnostics computes (pi = 0, step = -1) from device pointers to the
 * fields u, v, w (w unused in 2D), p and the packed mask of
 * ibm_get_classification (N bytes each in the grid precision, mask 1 byte),
 * on `stream` (a cudaStream_t, NULL = legacy default).  Blocking.
 *   - Scratch: the per-block partial sums live in a fixed array of this
 *     library's own device memory (196,736 bytes, present on every GPU that
 *     loads the library until the process exits); nothing is allocated.
 *   - Grids: the boundary conditions ibm_setup_geometry accepts (x periodic,
 *     or inflow at -x with a convective outflow at +x, whose inflow face
 *     value inflow[0] enters the divergence of the first cells as it does in
 *     ibm_diagnostics; z periodic).
 *   - Limit: grids of at most 134,217,728 cells; larger ones return
 *     IBM_E_INVALID with a message (checked factor by factor, so no size
 *     overflows).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture on the device.
 *   - All calls share the array: calls that overlap on the GPU (unordered
 *     streams) race on it and must be serialised by the caller.
 * Returns IBM_E_DIVERGED (and fills out->status) on non-finite values. */
ibm_status ibm_diagnostics_noalloc(const ibm_grid_desc* grid, const void* u, const void* v, const void* w,
                                   const void* p, const unsigned char* mask, double dt, void* stream,
                                   ibm_diag* out);

/* Release host metadata, events, graphs and cuFFT plans; never frees the
 * caller's device buffers.  Safe on NULL. */
void ibm_destroy(ibm_solver* h);

#ifdef __cplusplus
}
#endif
#endif /* IBM_H */
