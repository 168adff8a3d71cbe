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

// ---------------------------------------------------------------------------
// K3: momentum predictor with the implicit IBM diagonal division.
//
// A block owns a 32 x 16 (x, y) column of cells and marches g.kzm planes
// along z.  Warp w holds the rows j0 + 2w and j0 + 2w + 1 (cells A and B of
// each lane).  Plane tiles of u, v, w with a one-cell halo (34 x 18) sit in a
// ring of three shared-memory slots; each plane is stored once, already in
// the form the operator reads:
//   * x and z wrap (periodic);
//   * beyond a y wall the wall-normal component v reads the wall value 0 and
//     the tangential components read the mirror ghost sig * (adjacent value);
//   * every non-internal point (external or wall face) reads 0, so the ghost
//     term of the IBM vanishes by itself (Sec. 2.4, before Eq. semidisc-mom-comp).
// Global loads of a plane are issued two planes before it is computed (two
// register sets, so the plane loop is unrolled by two); pressure and the
// previous RHS are loaded one plane ahead.  Products shared by neighbouring
// stencils are formed once: a cell's flux through its top z face is carried
// to the next plane as that cell's bottom flux, the u-flux through the face
// between rows A and B serves both, and each corner product serves the two
// components that meet there; each is rounded once, so the flux that
// leaves one cell is bit for bit the flux that enters its neighbour, whatever
// the z-chunking.  The update is branch-free; a warp reads the
// IBM coefficient lists only when one of its points is an IBM point (a vote).
// An IBM point's list position is segoff + the number of IBM points in the
// lower lanes of its 32-point row segment (one ballot).
// ---------------------------------------------------------------------------
constexpr int MX = MOM_TX, MW = MOM_WARPS, MY = MOM_TY;
constexpr int HX = MX + 2, HY = MY + 2, HP = HX * HY;
static_assert(MY == 2 * MW, "two rows per thread");

template <typename T>
struct MomF {
    const T* u[3];
    const T* p;
    const uint8_t* mask;
    T* us[3];
    T* Nn[3];
};

// Where a thread's points come from and where they go in a plane tile; fixed
// over the planes.  Points A and B are the thread's own cells, H a halo point
// (warps 0-3 only).
template <typename T>
struct MomSrc {
    int oa, ob, oh;          // in-plane source offsets (x wrapped, y clamped)
    int ta, tb, th;          // positions in a plane tile
    int oea, oeb, onb;       // pressure: +x neighbour of A and B, +y neighbour of B (clamped)
    bool hh;                 // this thread loads a halo point
    bool ga, gb, gh;         // beyond a y wall: v reads 0, u and w read f * (adjacent)
    T fa, fb, fh;
};

template <typename T, int NC>
struct MomRegs {
    T a[NC], b[NC], h[NC];
    uint32_t m;              // mask bytes: A | B << 8 | H << 16
};

template <typename T>
struct MomPre {              // pressure and previous RHS of one plane
    T eA, eB, nB, tA, tB;
    T qA[3], qB[3];
};

// A product rounded on its own, never fused into a neighbouring add: a flux
// product that two stencils (or two planes) share must have one value.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <typename T>
__device__ __forceinline__ int mom_row(const GridP& g, int j, T sig_lo, T sig_hi, T& f, bool& beyond) {
    f = T(1);
    beyond = false;
    if (j < 0) { f = sig_lo; beyond = true; return 0; }
    if (j >= g.ny) { f = sig_hi; beyond = true; return g.ny - 1; }
    return j;
}

template <typename T>
__device__ __forceinline__ void mom_sources(const GridP& g, MomSrc<T>& S, int i0, int j0, T sig_lo, T sig_hi) {
    const int tx = threadIdx.x, w = threadIdx.y;
    const int ix = (i0 + tx) % g.nx;
    const int ixe = (ix + 1 < g.nx) ? ix + 1 : 0;
    const int ja = mom_row(g, j0 + 2 * w, sig_lo, sig_hi, S.fa, S.ga);
    const int jb = mom_row(g, j0 + 2 * w + 1, sig_lo, sig_hi, S.fb, S.gb);
    const int jn = min(j0 + 2 * w + 2, g.ny - 1);
    S.oa = ix + g.nx * ja;
    S.ob = ix + g.nx * jb;
    S.oea = ixe + g.nx * ja;
    S.oeb = ixe + g.nx * jb;
    S.onb = ix + g.nx * jn;
    S.ta = (2 * w + 1) * HX + tx + 1;
    S.tb = S.ta + HX;
    S.hh = false;
    S.oh = 0;
    S.th = 0;
    S.fh = T(1);
    S.gh = false;
    if (w == 0 || w == 1) {                       // halo rows below and above the tile
        const int jh = mom_row(g, w == 0 ? j0 - 1 : j0 + MY, sig_lo, sig_hi, S.fh, S.gh);
        S.hh = true;
        S.oh = ix + g.nx * jh;
        S.th = (w == 0 ? 0 : (HY - 1) * HX) + tx + 1;
    } else if ((w == 2 || w == 3) && tx < HY) {   // halo columns left and right (with corners)
        const int jh = mom_row(g, j0 - 1 + tx, sig_lo, sig_hi, S.fh, S.gh);
        const int ih = w == 2 ? (i0 - 1 + g.nx) % g.nx : (i0 + MX) % g.nx;
        S.hh = true;
        S.oh = ih + g.nx * jh;
        S.th = tx * HX + (w == 2 ? 0 : HX - 1);
    }
}

template <typename T, int NC>
__device__ __forceinline__ void mom_fetch(const MomF<T>& F, const MomSrc<T>& S, MomRegs<T, NC>& R, int pb) {
    const uint32_t ma = __ldg(F.mask + pb + S.oa);
    const uint32_t mb = __ldg(F.mask + pb + S.ob);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        R.a[c] = __ldg(F.u[c] + pb + S.oa);
        R.b[c] = __ldg(F.u[c] + pb + S.ob);
    }
    uint32_t mh = 0;
    if (S.hh) {
        mh = __ldg(F.mask + pb + S.oh);
#pragma unroll
        for (int c = 0; c < NC; ++c) R.h[c] = __ldg(F.u[c] + pb + S.oh);
    }
    R.m = ma | (mb << 8) | (mh << 16);
}

// value as the operator reads it: 0 unless internal; the ghost rule beyond a wall
template <typename T, bool EDGE>
__device__ __forceinline__ T mom_masked(T x, uint32_t m, int bit, int c, bool beyond, T f) {
    x = ((m >> bit) & 1u) ? x : T(0);
    if (EDGE && beyond) x = (c == 1) ? T(0) : f * x;
    return x;
}

template <typename T, int NC, bool EDGE>
__device__ __forceinline__ void mom_store(T* tile, const MomSrc<T>& S, const MomRegs<T, NC>& R) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        tile[c * HP + S.ta] = mom_masked<T, EDGE>(R.a[c], R.m, c, c, S.ga, S.fa);
        tile[c * HP + S.tb] = mom_masked<T, EDGE>(R.b[c], R.m, 8 + c, c, S.gb, S.fb);
        if (S.hh) tile[c * HP + S.th] = mom_masked<T, EDGE>(R.h[c], R.m, 16 + c, c, S.gh, S.fh);
    }
}

template <typename T, int NC>
__device__ __forceinline__ void mom_store_plane(T* tile, const MomSrc<T>& S, const MomRegs<T, NC>& R, bool yedge) {
    if (yedge) mom_store<T, NC, true>(tile, S, R);
    else mom_store<T, NC, false>(tile, S, R);
}

template <typename T>
__device__ __forceinline__ void mom_pre(const MomF<T>& F, const MomSrc<T>& S, MomPre<T>& P, const GridP& g, int k,
                                        int plane, bool read_prev) {
    const int pb = k * plane;
    const int tb = (k + 1 < g.nz ? k + 1 : 0) * plane;
    P.eA = F.p[pb + S.oea];
    P.eB = F.p[pb + S.oeb];
    P.nB = F.p[pb + S.onb];
    P.tA = F.p[tb + S.oa];
    P.tB = F.p[tb + S.ob];
    if (read_prev) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            P.qA[c] = F.Nn[c][pb + S.oa];
            P.qB[c] = F.Nn[c][pb + S.ob];
        }
    }
}

// carried state of a thread's two cells from one plane to the next
template <typename T>
struct MomCarry {
    T uA, uB, vA, vB, wA, wB;          // own values at plane k
    T uWA, uWB, vSA;                   // u(i-1) of A and B, v(j-1) of A, plane k
    T ubA, ubB, vbA, vbB, wbA, wbB;    // own values at plane k-1
    T fuA, fuB, fvA, fvB;              // bottom z-face fluxes of u and v
    T pA, pB;                          // pressure at plane k
};

// The stage update of one component of one cell before the IBM division:
// out = uP + R with R = dt a_k N - c_k dt gp (+ dt b_k N^{k-2}).
template <typename T>
__device__ __forceinline__ void mom_update(const StageP<T>& sp, T uP, T N, T gp, T Nprev, T& out, T& R) {
    R = sp.dta * N - sp.ckdt * gp;
    if (sp.read_prev) R += sp.dtb * Nprev;
    out = uP + R;
}

// the implicit IBM division of one IBM point (Eq. rk3-rai): the wall source s
// joins N, and u* = alpha u + beta R
template <typename T>
__device__ __forceinline__ void mom_ibm(const StageP<T>& sp, const Coef4<T>& q, T uP, T R, T& out, T& N) {
    N += q.s;
    out = q.a * uP + q.b * (R + sp.dta * q.s);
}

template <typename T, int NC>
__device__ __forceinline__ void mom_ibm_fix(const IbmStage<T>& ib, const StageP<T>& sp, uint32_t mA, uint32_t mB,
                                            int segA, int segB, const T (&uA)[3], const T (&uB)[3], const T (&RA)[3],
                                            const T (&RB)[3], T (&oA)[3], T (&oB)[3], T (&NA)[3], T (&NB)[3]) {
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const bool ia = (mA >> (4 + c)) & 1u, ibb = (mB >> (4 + c)) & 1u;
        const unsigned ba = __ballot_sync(0xffffffffu, ia);
        const unsigned bb = __ballot_sync(0xffffffffu, ibb);
        if (ia) mom_ibm(sp, ib.coef[c][ib.segoff[c][segA] + __popc(ba & lt)], uA[c], RA[c], oA[c], NA[c]);
        if (ibb) mom_ibm(sp, ib.coef[c][ib.segoff[c][segB] + __popc(bb & lt)], uB[c], RB[c], oB[c], NB[c]);
    }
}

template <typename T, int NC>
__device__ __forceinline__ void mom_write(const MomF<T>& F, const StageP<T>& sp, int ida, int idb, bool liveA,
                                          bool liveB, uint32_t mA, uint32_t mB, T (&oA)[3], T (&oB)[3], T (&NA)[3],
                                          T (&NB)[3], T& fsum) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const bool ia = (mA >> c) & 1u, ibb = (mB >> c) & 1u;
        oA[c] = ia ? oA[c] : T(0);
        oB[c] = ibb ? oB[c] : T(0);
        NA[c] = ia ? NA[c] : T(0);
        NB[c] = ibb ? NB[c] : T(0);
        if (liveA) F.us[c][ida] = oA[c];
        if (liveB) F.us[c][idb] = oB[c];
        if (sp.write_n) {
            if (liveA) F.Nn[c][ida] = NA[c];
            if (liveB) F.Nn[c][idb] = NB[c];
        }
    }
    fsum += oA[0] + oB[0];
}

// One plane k of the 3D update.  t0 / t1: the tiles of planes k and k+1.
template <typename T>
__device__ __forceinline__ void mom_plane3(const GridP& g, const MomF<T>& F, const StageP<T>& sp,
                                           const IbmStage<T>& ib, const MomSrc<T>& S, const T* __restrict__ t0,
                                           const T* __restrict__ t1, MomCarry<T>& C, const MomPre<T>& P,
                                           uint32_t m, int k, int ida, int idb, bool liveA, bool liveB, int segA,
                                           T& fsum) {
    const int a = S.ta, b = S.tb;
    const T* U0 = t0;
    const T* V0 = t0 + HP;
    const T* W0 = t0 + 2 * HP;
    const T* U1 = t1;
    const T* V1 = t1 + HP;
    const T* W1 = t1 + 2 * HP;
    const T two = T(2);
    // plane k (the own column and u(i-1), v(j-1) of A are carried)
    const T uEA = U0[a + 1], uEB = U0[b + 1], uSA = U0[a - HX], uNB = U0[b + HX], uNWB = U0[b + HX - 1];
    const T vEA = V0[a + 1], vEB = V0[b + 1], vWA = V0[a - 1], vWB = V0[b - 1], vNB = V0[b + HX];
    const T vSEA = V0[a - HX + 1];
    const T wEA = W0[a + 1], wEB = W0[b + 1], wWA = W0[a - 1], wWB = W0[b - 1], wSA = W0[a - HX];
    const T wNB = W0[b + HX];
    // plane k+1
    const T uTA = U1[a], uTB = U1[b], uTWA = U1[a - 1], uTWB = U1[b - 1];
    const T vTA = V1[a], vTB = V1[b], vTSA = V1[a - HX];
    const T wTA = W1[a], wTB = W1[b];
    const T uA = C.uA, uB = C.uB, vA = C.vA, vB = C.vB, wA = C.wA, wB = C.wB;
    const T uWA = C.uWA, uWB = C.uWB, vSA = C.vSA;

    // corner products, each shared by the two components that meet there
    const T xyA = mul_rn(vA + vEA, uA + uB);          // u: top of A, bottom of B;  v: right of A
    const T xyB = mul_rn(vB + vEB, uB + uNB);         // u: top of B;               v: right of B
    const T xyAs = mul_rn(vSA + vSEA, uSA + uA);      // u: bottom of A
    const T xyAw = mul_rn(uWA + uWB, vWA + vA);       // v: left of A
    const T xyBw = mul_rn(uWB + uNWB, vWB + vB);      // v: left of B
    const T xzA = mul_rn(wA + wEA, uA + uTA);         // u: z-top of A;  w: right of A
    const T xzB = mul_rn(wB + wEB, uB + uTB);
    const T xzAw = mul_rn(uWA + uTWA, wWA + wA);      // w: left of A
    const T xzBw = mul_rn(uWB + uTWB, wWB + wB);
    const T yzA = mul_rn(wA + wB, vA + vTA);          // v: z-top of A;  w: y-top of A, y-bottom of B
    const T yzB = mul_rn(wB + wNB, vB + vTB);         // v: z-top of B;  w: y-top of B
    const T yzAs = mul_rn(vSA + vTSA, wSA + wA);      // w: y-bottom of A

    T NA[3], NB[3], oA[3], oB[3], RA[3], RB[3];
    const T pA = C.pA, pB = C.pB;
    {   // u
        T conv = (uEA - uWA) * (uEA + uWA + two * uA) * sp.qx;
        conv += (xyA - xyAs) * sp.qy;
        conv += (xzA - C.fuA) * sp.qz;
        T lap = (uEA + uWA - two * uA) * sp.nx2 + (uB + uSA - two * uA) * sp.ny2;
        lap += (uTA + C.ubA - two * uA) * sp.nz2;
        NA[0] = lap - conv + sp.g[0];
        mom_update(sp, uA, NA[0], (P.eA - pA) * sp.idx, P.qA[0], oA[0], RA[0]);
        conv = (uEB - uWB) * (uEB + uWB + two * uB) * sp.qx;
        conv += (xyB - xyA) * sp.qy;
        conv += (xzB - C.fuB) * sp.qz;
        lap = (uEB + uWB - two * uB) * sp.nx2 + (uNB + uA - two * uB) * sp.ny2;
        lap += (uTB + C.ubB - two * uB) * sp.nz2;
        NB[0] = lap - conv + sp.g[0];
        mom_update(sp, uB, NB[0], (P.eB - pB) * sp.idx, P.qB[0], oB[0], RB[0]);
    }
    {   // v
        T conv = (xyA - xyAw) * sp.qx;
        conv += (vB - vSA) * (vB + vSA + two * vA) * sp.qy;
        conv += (yzA - C.fvA) * sp.qz;
        T lap = (vEA + vWA - two * vA) * sp.nx2 + (vB + vSA - two * vA) * sp.ny2;
        lap += (vTA + C.vbA - two * vA) * sp.nz2;
        NA[1] = lap - conv + sp.g[1];
        mom_update(sp, vA, NA[1], (pB - pA) * sp.idy, P.qA[1], oA[1], RA[1]);
        conv = (xyB - xyBw) * sp.qx;
        conv += (vNB - vA) * (vNB + vA + two * vB) * sp.qy;
        conv += (yzB - C.fvB) * sp.qz;
        lap = (vEB + vWB - two * vB) * sp.nx2 + (vNB + vA - two * vB) * sp.ny2;
        lap += (vTB + C.vbB - two * vB) * sp.nz2;
        NB[1] = lap - conv + sp.g[1];
        mom_update(sp, vB, NB[1], (P.nB - pB) * sp.idy, P.qB[1], oB[1], RB[1]);
    }
    {   // w
        T conv = (xzA - xzAw) * sp.qx;
        conv += (yzA - yzAs) * sp.qy;
        conv += (wTA - C.wbA) * (wTA + C.wbA + two * wA) * sp.qz;
        T lap = (wEA + wWA - two * wA) * sp.nx2 + (wB + wSA - two * wA) * sp.ny2;
        lap += (wTA + C.wbA - two * wA) * sp.nz2;
        NA[2] = lap - conv + sp.g[2];
        mom_update(sp, wA, NA[2], (P.tA - pA) * sp.idz, P.qA[2], oA[2], RA[2]);
        conv = (xzB - xzBw) * sp.qx;
        conv += (yzB - yzA) * sp.qy;
        conv += (wTB - C.wbB) * (wTB + C.wbB + two * wB) * sp.qz;
        lap = (wEB + wWB - two * wB) * sp.nx2 + (wNB + wA - two * wB) * sp.ny2;
        lap += (wTB + C.wbB - two * wB) * sp.nz2;
        NB[2] = lap - conv + sp.g[2];
        mom_update(sp, wB, NB[2], (P.tB - pB) * sp.idz, P.qB[2], oB[2], RB[2]);
    }
    const uint32_t mA = m & 0xffu, mB = (m >> 8) & 0xffu;
    if (__any_sync(0xffffffffu, (mA | mB) & (IBM_MASK_IBM_U | IBM_MASK_IBM_V | IBM_MASK_IBM_W))) {
        const T ua3[3] = {uA, vA, wA}, ub3[3] = {uB, vB, wB};
        mom_ibm_fix<T, 3>(ib, sp, mA, mB, segA, segA + g.nsegx, ua3, ub3, RA, RB, oA, oB, NA, NB);
    }
    mom_write<T, 3>(F, sp, ida, idb, liveA, liveB, mA, mB, oA, oB, NA, NB, fsum);

    // carry this column into the next plane
    C.ubA = uA; C.ubB = uB; C.vbA = vA; C.vbB = vB; C.wbA = wA; C.wbB = wB;
    C.uA = uTA; C.uB = uTB; C.vA = vTA; C.vB = vTB; C.wA = wTA; C.wB = wTB;
    C.uWA = uTWA; C.uWB = uTWB; C.vSA = vTSA;
    C.fuA = xzA; C.fuB = xzB; C.fvA = yzA; C.fvB = yzB;
    C.pA = P.tA; C.pB = P.tB;
}

// One plane of the 2D update (u, v only).
template <typename T>
__device__ __forceinline__ void mom_plane2(const GridP& g, const MomF<T>& F, const StageP<T>& sp,
                                           const IbmStage<T>& ib, const MomSrc<T>& S, const T* __restrict__ t0,
                                           const MomPre<T>& P, T pA, T pB, uint32_t m, int ida, int idb,
                                           bool liveA, bool liveB, int segA, T& fsum) {
    const int a = S.ta, b = S.tb;
    const T* U0 = t0;
    const T* V0 = t0 + HP;
    const T two = T(2);
    const T uA = U0[a], uB = U0[b], uEA = U0[a + 1], uEB = U0[b + 1], uWA = U0[a - 1], uWB = U0[b - 1];
    const T uSA = U0[a - HX], uNB = U0[b + HX], uNWB = U0[b + HX - 1];
    const T vA = V0[a], vB = V0[b], vEA = V0[a + 1], vEB = V0[b + 1], vWA = V0[a - 1], vWB = V0[b - 1];
    const T vSA = V0[a - HX], vNB = V0[b + HX], vSEA = V0[a - HX + 1];
    const T xyA = mul_rn(vA + vEA, uA + uB);
    const T xyB = mul_rn(vB + vEB, uB + uNB);
    const T xyAs = mul_rn(vSA + vSEA, uSA + uA);
    const T xyAw = mul_rn(uWA + uWB, vWA + vA);
    const T xyBw = mul_rn(uWB + uNWB, vWB + vB);
    T NA[3], NB[3], oA[3], oB[3], RA[3], RB[3];
    {
        T conv = (uEA - uWA) * (uEA + uWA + two * uA) * sp.qx + (xyA - xyAs) * sp.qy;
        T lap = (uEA + uWA - two * uA) * sp.nx2 + (uB + uSA - two * uA) * sp.ny2;
        NA[0] = lap - conv + sp.g[0];
        mom_update(sp, uA, NA[0], (P.eA - pA) * sp.idx, P.qA[0], oA[0], RA[0]);
        conv = (uEB - uWB) * (uEB + uWB + two * uB) * sp.qx + (xyB - xyA) * sp.qy;
        lap = (uEB + uWB - two * uB) * sp.nx2 + (uNB + uA - two * uB) * sp.ny2;
        NB[0] = lap - conv + sp.g[0];
        mom_update(sp, uB, NB[0], (P.eB - pB) * sp.idx, P.qB[0], oB[0], RB[0]);
    }
    {
        T conv = (xyA - xyAw) * sp.qx + (vB - vSA) * (vB + vSA + two * vA) * sp.qy;
        T lap = (vEA + vWA - two * vA) * sp.nx2 + (vB + vSA - two * vA) * sp.ny2;
        NA[1] = lap - conv + sp.g[1];
        mom_update(sp, vA, NA[1], (pB - pA) * sp.idy, P.qA[1], oA[1], RA[1]);
        conv = (xyB - xyBw) * sp.qx + (vNB - vA) * (vNB + vA + two * vB) * sp.qy;
        lap = (vEB + vWB - two * vB) * sp.nx2 + (vNB + vA - two * vB) * sp.ny2;
        NB[1] = lap - conv + sp.g[1];
        mom_update(sp, vB, NB[1], (P.nB - pB) * sp.idy, P.qB[1], oB[1], RB[1]);
    }
    const uint32_t mA = m & 0xffu, mB = (m >> 8) & 0xffu;
    if (__any_sync(0xffffffffu, (mA | mB) & (IBM_MASK_IBM_U | IBM_MASK_IBM_V))) {
        const T ua3[3] = {uA, vA, T(0)}, ub3[3] = {uB, vB, T(0)};
        mom_ibm_fix<T, 2>(ib, sp, mA, mB, segA, segA + g.nsegx, ua3, ub3, RA, RB, oA, oB, NA, NB);
    }
    mom_write<T, 2>(F, sp, ida, idb, liveA, liveB, mA, mB, oA, oB, NA, NB, fsum);
}

// One step of the 3D plane loop: store plane k+1 (register set R) into its
// slot, refill R with plane k+3, load pressure / previous RHS of plane k+1
// into Pn, wait for the block, compute plane k with Pc.
template <typename T>
__device__ __forceinline__ void mom_iter3(const GridP& g, const MomF<T>& F, const StageP<T>& sp,
                                          const IbmStage<T>& ib, const MomSrc<T>& S, T* tiles, int& s0, int& s1,
                                          int& s2, MomRegs<T, 3>& R, MomPre<T>& Pc, MomPre<T>& Pn, uint32_t& mc,
                                          uint32_t& mn, MomCarry<T>& C, int k, int kend, int plane, bool yedge,
                                          int rowA, bool liveA, bool liveB, int segrow, T& fsum) {
    mom_store_plane<T, 3>(tiles + s1, S, R, yedge);               // plane k+1
    mn = R.m & 0xffffu;
    if (k + 3 <= kend) mom_fetch<T, 3>(F, S, R, wrapi(k + 3, g.nz) * plane);
    if (k + 1 < kend) mom_pre(F, S, Pn, g, k + 1, plane, sp.read_prev);
    __syncthreads();
    const int ida = rowA + k * plane;
    mom_plane3<T>(g, F, sp, ib, S, tiles + s0, tiles + s1, C, Pc, mc, k, ida, ida + g.nx, liveA, liveB,
                  segrow + k * g.ny * g.nsegx, fsum);
    const int t = s0;
    s0 = s1;
    s1 = s2;
    s2 = t;
}

template <typename T, bool THREE>
__global__ void __launch_bounds__(MX * MW, sizeof(T) == 4 ? 2 : 1)
    k_momentum(GridP g, MomF<T> F, StageP<T> sp, IbmStage<T> ib, double* __restrict__ flux_part) {
    constexpr int NC = THREE ? 3 : 2;
    constexpr int NS = THREE ? 3 : 1;
    constexpr int SLOT = 3 * HP;                 // one plane tile (u, v, w)
    __shared__ T tiles[NS * SLOT];
    __shared__ double shd[MW];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = blockIdx.x * MX, j0 = blockIdx.y * MY;
    const int i = i0 + tx, jA = j0 + 2 * ty;
    const bool liveA = i < g.nx && jA < g.ny;
    const bool liveB = i < g.nx && jA + 1 < g.ny;
    const bool yedge = j0 == 0 || j0 + MY >= g.ny;
    const int plane = g.nx * g.ny;
    const int rowA = i + g.nx * jA;               // in-plane index of A (B: + nx)
    const int segrow = jA * g.nsegx + blockIdx.x;  // row segment of A at plane 0
    // the point masks of dead cells read 0, so they take part in no ballot
    const uint32_t live_bits = (liveA ? 0xffu : 0u) | (liveB ? 0xff00u : 0u);
    T fsum = T(0);

    MomSrc<T> S;
    mom_sources<T>(g, S, i0, j0, sp.sig_lo, sp.sig_hi);
    MomRegs<T, NC> X, Y;
    MomPre<T> P0, P1;
#pragma unroll
    for (int c = 0; c < 3; ++c) P0.qA[c] = P0.qB[c] = P1.qA[c] = P1.qB[c] = T(0);

    if constexpr (THREE) {
        const int kbeg = blockIdx.z * g.kzm;
        const int kend = min(kbeg + g.kzm, g.nz);
        int s0 = 0, s1 = SLOT, s2 = 2 * SLOT;
        // prologue: planes kbeg-1 (slot 2) and kbeg (slot 0) give the carried state
        mom_fetch<T, 3>(F, S, X, wrapi(kbeg - 1, g.nz) * plane);
        mom_fetch<T, 3>(F, S, Y, kbeg * plane);
        mom_pre(F, S, P0, g, kbeg, plane, sp.read_prev);
        MomCarry<T> C;
        C.pA = F.p[kbeg * plane + S.oa];
        C.pB = F.p[kbeg * plane + S.ob];
        mom_store_plane<T, 3>(tiles + s2, S, X, yedge);
        mom_store_plane<T, 3>(tiles + s0, S, Y, yedge);
        uint32_t m0 = Y.m & live_bits, m1 = 0;
        __syncthreads();
        {
            const int a = S.ta, b = S.tb;
            const T* Ub = tiles + s2;
            const T* Vb = Ub + HP;
            const T* Wb = Ub + 2 * HP;
            const T* U0 = tiles + s0;
            const T* V0 = U0 + HP;
            const T* W0 = U0 + 2 * HP;
            C.ubA = Ub[a]; C.ubB = Ub[b]; C.vbA = Vb[a]; C.vbB = Vb[b]; C.wbA = Wb[a]; C.wbB = Wb[b];
            C.uA = U0[a]; C.uB = U0[b]; C.vA = V0[a]; C.vB = V0[b]; C.wA = W0[a]; C.wB = W0[b];
            C.uWA = U0[a - 1]; C.uWB = U0[b - 1]; C.vSA = V0[a - HX];
            C.fuA = mul_rn(Wb[a] + Wb[a + 1], Ub[a] + U0[a]);
            C.fuB = mul_rn(Wb[b] + Wb[b + 1], Ub[b] + U0[b]);
            C.fvA = mul_rn(Wb[a] + Wb[a + HX], Vb[a] + V0[a]);
            C.fvB = mul_rn(Wb[b] + Wb[b + HX], Vb[b] + V0[b]);
        }
        mom_fetch<T, 3>(F, S, X, wrapi(kbeg + 1, g.nz) * plane);
        if (kbeg + 2 <= kend) mom_fetch<T, 3>(F, S, Y, wrapi(kbeg + 2, g.nz) * plane);
        for (int k = kbeg; k < kend; k += 2) {
            mom_iter3<T>(g, F, sp, ib, S, tiles, s0, s1, s2, X, P0, P1, m0, m1, C, k, kend, plane, yedge, rowA,
                         liveA, liveB, segrow, fsum);
            m1 &= live_bits;
            if (k + 1 >= kend) break;
            mom_iter3<T>(g, F, sp, ib, S, tiles, s0, s1, s2, Y, P1, P0, m1, m0, C, k + 1, kend, plane, yedge, rowA,
                         liveA, liveB, segrow, fsum);
            m0 &= live_bits;
        }
    } else {
        mom_fetch<T, NC>(F, S, X, 0);
        mom_pre(F, S, P0, g, 0, plane, sp.read_prev);
        const T pA = F.p[S.oa], pB = F.p[S.ob];
        mom_store_plane<T, NC>(tiles, S, X, yedge);
        __syncthreads();
        mom_plane2<T>(g, F, sp, ib, S, tiles, P0, pA, pB, X.m & live_bits, rowA, rowA + g.nx, liveA, liveB, segrow,
                      fsum);
    }
    if (sp.flux_sum) {
        // FP32 sums within a warp, FP64 across warps and blocks
        T ws = warp_sum(fsum);
        if (tx == 0) shd[ty] = (double)ws;
        __syncthreads();
        if (tx == 0 && ty == 0) {
            double s = 0.0;
            for (int w = 0; w < MW; ++w) s += shd[w];
            flux_part[blockIdx.x + gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z)] = s;
        }
    }
}

// ---------------------------------------------------------------------------
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
// from the neighbouring lane.
// ---------------------------------------------------------------------------
template <typename T, bool THREE, bool FLUX>
__global__ void __launch_bounds__(256) k_divergence(GridP g, const T* __restrict__ u, const T* __restrict__ v,
                                                    const T* __restrict__ w, const uint8_t* __restrict__ mask,
                                                    T* __restrict__ rhs, T idx, T idy, T idz, FluxCorr<T> fc) {
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
    T wprev = T(0);
    if (THREE && live) wprev = w[i + g.nx * j + plane * wrapi(kbeg - 1, g.nz)];
#pragma unroll 2
    for (int k = kbeg; k < kend; ++k) {
        const int rowb = g.nx * (j + g.ny * k);
        const int id = rowb + i;
        T uc = live ? u[id] : T(0);
        T ulane0 = u[rowb + il];
        if (FLUX) {
            const int rowseg = (j + g.ny * k) * g.nsegx;
            const uint8_t m = live ? mask[id] : 0;
            const unsigned b = __ballot_sync(0xffffffffu, (m & IBM_MASK_IBM_U) != 0);
            if (live) uc += flux_increment(fc, pic, m, b, rowseg + (int)blockIdx.x, lane);
            const uint8_t ml = il_probe < g.nx ? mask[rowb + il_probe] : 0;
            const unsigned bl = __ballot_sync(0xffffffffu, (ml & IBM_MASK_IBM_U) != 0);
            const uint8_t mln = __shfl_sync(0xffffffffu, ml, lanel);
            ulane0 += flux_increment(fc, pic, mln, bl, rowseg + segl, lanel);
        }
        T ul = __shfl_up_sync(0xffffffffu, uc, 1);
        if (lane == 0) ul = ulane0;
        if (live) {
            T d = (uc - ul) * idx;
            const T vm = j > 0 ? v[id - g.nx] : T(0);
            d += (v[id] - vm) * idy;
            if (THREE) {
                const T wc = w[id];
                d += (wc - wprev) * idz;
                wprev = wc;
            }
            rhs[id] = d;
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
// gauge).  Each system runs in FP64 unless its flag says it is strongly
// diagonally dominant (K dy^2 >= tau, condition number <= 4/tau + 1), in which
// case FP32 arithmetic with FP32 pivots is as accurate as the FP32 transforms
// that feed it; that sweep works in place on the spectrum.
// One warp covers 32 consecutive kx of one kz, so loads coalesce across systems.
// ---------------------------------------------------------------------------
// FP64 sweep of one component (real or imaginary part) of one system: the two
// parts are independent recurrences, so two threads share a system and the
// FP64 work is spread over twice as many warps.  The next batch of loads is
// issued before the current batch is consumed.
template <typename C>
__device__ __forceinline__ void tridiag_fp64(const GridP& g, C* spec, double2* tmp, const double* __restrict__ piv,
                                             long long base, int comp, double scale, bool zero_mode) {
    constexpr bool F32 = sizeof(C) == sizeof(float2);
    using S = typename std::conditional<F32, float, double>::type;   // storage scalar
    constexpr int B = 8;
    const long long st = g.nxh;
    const int ny = g.ny;
    S* sp = reinterpret_cast<S*>(spec) + comp;      // component `comp` of spec[o] at sp[2 o]
    double* tp = reinterpret_cast<double*>(tmp) + comp;
    const float sf = (float)scale;
    double e = 0.0;
    S r[B], rn[B];
    double w[B], wn[B];
#pragma unroll
    for (int t = 0; t < B; ++t)
        if (t < ny) {
            r[t] = sp[2 * (base + t * st)];
            w[t] = piv[base + t * st];
        }
    for (int j0 = 0; j0 < ny; j0 += B) {
#pragma unroll
        for (int t = 0; t < B; ++t)
            if (j0 + B + t < ny) {
                rn[t] = sp[2 * (base + (j0 + B + t) * st)];
                wn[t] = piv[base + (j0 + B + t) * st];
            }
#pragma unroll
        for (int t = 0; t < B; ++t)
            if (j0 + t < ny) {
                // FP32 storage: the scale is applied in FP32 on the input (exact to FP32 rounding)
                const double rv = F32 ? (double)((float)r[t] * sf) : (double)r[t];
                e = (rv - e) * w[t];                                          // e_{-1} = 0
                tp[2 * (base + (j0 + t) * st)] = e;
            }
#pragma unroll
        for (int t = 0; t < B; ++t) { r[t] = rn[t]; w[t] = wn[t]; }
    }
    double x = e;
    double sum = 0.0;
    auto put = [&](long long o, double val) {
        if (F32) sp[2 * o] = (S)val;
        else sp[2 * o] = (S)(val * scale);
    };
    put(base + (long long)(ny - 1) * st, x);
    if (zero_mode) sum += x;
    double d[B], dn[B];
#pragma unroll
    for (int t = 0; t < B; ++t)
        if (ny - 2 - t >= 0) {
            d[t] = tp[2 * (base + (ny - 2 - t) * st)];
            w[t] = piv[base + (ny - 2 - t) * st];
        }
    for (int j1 = ny - 2; j1 >= 0; j1 -= B) {
#pragma unroll
        for (int t = 0; t < B; ++t)
            if (j1 - B - t >= 0) {
                dn[t] = tp[2 * (base + (j1 - B - t) * st)];
                wn[t] = piv[base + (j1 - B - t) * st];
            }
#pragma unroll
        for (int t = 0; t < B; ++t)
            if (j1 - t >= 0) {
                x = d[t] - w[t] * x;
                put(base + (j1 - t) * st, x);
                if (zero_mode) sum += x;
            }
#pragma unroll
        for (int t = 0; t < B; ++t) { d[t] = dn[t]; w[t] = wn[t]; }
    }
    if (zero_mode) {
        const double mean = sum / ny * (F32 ? 1.0 : scale);
        for (int j = 0; j < ny; ++j) {
            const long long o = base + j * st;
            sp[2 * o] = (S)((double)sp[2 * o] - mean);
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
// FP64 systems take two threads (real and imaginary part), FP32 systems one.
template <typename C>
__global__ void __launch_bounds__(32) k_tridiag(GridP g, C* spec, double2* tmp, const double* __restrict__ piv,
                                                const float* __restrict__ piv32, const int* __restrict__ order,
                                                int n64, int nsys, double scale) {
    const int nb64 = (2 * n64 + 31) / 32;
    if ((int)blockIdx.x < nb64) {
        const int t = blockIdx.x * 32 + threadIdx.x;
        if (t >= 2 * n64) return;
        const int sys = order[t >> 1];
        const int kx = sys % g.nxh, kz = sys / g.nxh;
        const long long base = (long long)kz * g.ny * g.nxh + kx;
        tridiag_fp64<C>(g, spec, tmp, piv, base, t & 1, scale, kx == 0 && kz == 0);
        return;
    }
    if constexpr (sizeof(C) == sizeof(float2)) {
        const int q = n64 + (blockIdx.x - nb64) * 32 + threadIdx.x;
        if (q >= nsys) return;
        const int sys = order[q];
        const int kx = sys % g.nxh, kz = sys / g.nxh;
        const long long base = (long long)kz * g.ny * g.nxh + kx;
        tridiag_fp32(g, reinterpret_cast<float2*>(spec), piv32, base, (float)scale);
    }
}

// ---------------------------------------------------------------------------
// K7: u = u* (+ flux correction) - G psi on every non-wall face, p += psi/(c_k dt)
// (psi = c_k dt phi is what the Poisson solve returns for rhs = D u*).  Blocks
// march g.kzd planes carrying psi(k+1) into the next plane; psi(i+1) comes from
// the neighbouring lane.
// ---------------------------------------------------------------------------
template <typename T, bool THREE, bool FLUX>
__global__ void __launch_bounds__(256) k_correct(GridP g, const T* __restrict__ us0, const T* __restrict__ us1,
                                                 const T* __restrict__ us2, const T* __restrict__ psi,
                                                 const uint8_t* __restrict__ mask, T* __restrict__ u0,
                                                 T* __restrict__ u1, T* __restrict__ u2, T* __restrict__ p, T idx,
                                                 T idy, T idz, T inv_ckdt, int update_p, FluxCorr<T> fc) {
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
    const T pic = FLUX ? *reinterpret_cast<const T*>(fc.scal + 2) * fc.ckdt : T(0);
    T ph = live ? psi[i + g.nx * j + plane * kbeg] : T(0);
#pragma unroll 2
    for (int k = kbeg; k < kend; ++k) {
        const int rowb = g.nx * (j + g.ny * k);
        const int id = rowb + i;
        T pE = __shfl_down_sync(0xffffffffu, ph, 1);
        T uc = T(0);
        if (FLUX) {
            const uint8_t m = live ? mask[id] : 0;
            const unsigned b = __ballot_sync(0xffffffffu, (m & IBM_MASK_IBM_U) != 0);
            if (live) uc = flux_increment(fc, pic, m, b, (j + g.ny * k) * g.nsegx + (int)blockIdx.x, lane);
        }
        T pT = T(0);
        if (THREE && live) pT = psi[id + ((k + 1 < g.nz) ? plane : plane - (int)g.N)];
        if (live) {
            if (!from_lane) pE = psi[rowb + ir];
            u0[id] = us0[id] + uc - (pE - ph) * idx;
            u1[id] = j < g.ny - 1 ? us1[id] - (psi[id + g.nx] - ph) * idy : us1[id];
            if (THREE) u2[id] = us2[id] - (pT - ph) * idz;
            if (update_p) p[id] += ph * inv_ckdt;
        }
        ph = pT;
    }
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
    const int nblk = (2 * h->n64 + 31) / 32 + (nsys - h->n64 + 31) / 32;
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

template <typename T>
ibm_status divergence_and_solve(ibm_solver* h, T* const us[3], bool flux, const FluxCorr<T>& fc) {
    const GridP& g = h->gp;
    cudaEvent_t t;
    timer_begin(h, "divergence", &t);
    const T ix = (T)(1.0 / g.dx), iy = (T)(1.0 / g.dy), iz = (T)(1.0 / g.dz);
    const dim3 grd = zmarch_grid(g), blk(32, 8);
    T* rhs = (T*)h->rhs;
    if (g.ndim == 3) {
        if (flux) k_divergence<T, true, true><<<grd, blk, 0, h->stream>>>(g, us[0], us[1], us[2], h->mask, rhs, ix, iy, iz, fc);
        else k_divergence<T, true, false><<<grd, blk, 0, h->stream>>>(g, us[0], us[1], us[2], h->mask, rhs, ix, iy, iz, fc);
    } else {
        if (flux) k_divergence<T, false, true><<<grd, blk, 0, h->stream>>>(g, us[0], us[1], us[0], h->mask, rhs, ix, iy, iz, fc);
        else k_divergence<T, false, false><<<grd, blk, 0, h->stream>>>(g, us[0], us[1], us[0], h->mask, rhs, ix, iy, iz, fc);
    }
    IBM_LAUNCH_CHECK();
    timer_end(h, t, "divergence");
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
    if (g.ndim == 3) {
        if (flux) k_correct<T, true, true><<<grd, blk, 0, h->stream>>>(g, us[0], us[1], us2, psi, h->mask, u0, u1, u2, p, ix, iy, iz, inv_ckdt, update_p, fc);
        else k_correct<T, true, false><<<grd, blk, 0, h->stream>>>(g, us[0], us[1], us2, psi, h->mask, u0, u1, u2, p, ix, iy, iz, inv_ckdt, update_p, fc);
    } else {
        if (flux) k_correct<T, false, true><<<grd, blk, 0, h->stream>>>(g, us[0], us[1], us2, psi, h->mask, u0, u1, u2, p, ix, iy, iz, inv_ckdt, update_p, fc);
        else k_correct<T, false, false><<<grd, blk, 0, h->stream>>>(g, us[0], us[1], us2, psi, h->mask, u0, u1, u2, p, ix, iy, iz, inv_ckdt, update_p, fc);
    }
    IBM_LAUNCH_CHECK();
    return IBM_OK;
}

template <typename T>
ibm_status launch_momentum(ibm_solver* h, int k, StageP<T>& sp, IbmStage<T>& ib, dim3& grd) {
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
    sp.flux_sum = h->phys.flow_mode == IBM_FLOW_CONST_FLUX;
    for (int c = 0; c < 3; ++c) {
        ib.segoff[c] = h->segoff[c];
        ib.coef[c] = (const Coef4<T>*)h->coef[c] + (long long)k * h->counts[c];
    }
    dim3 blk(MX, MW, 1);
    grd = momentum_grid(g);
    if (g.ndim == 3) k_momentum<T, true><<<grd, blk, 0, h->stream>>>(g, F, sp, ib, h->partials);
    else k_momentum<T, false><<<grd, blk, 0, h->stream>>>(g, F, sp, ib, h->partials);
    IBM_LAUNCH_CHECK();
    return IBM_OK;
}

template <typename T>
ibm_status substage_t(ibm_solver* h, int k, bool predictor_only) {
    const GridP& g = h->gp;
    StageP<T> sp;
    IbmStage<T> ib;
    dim3 grd;
    const double dt = h->phys.dt;
    const bool cflux = h->phys.flow_mode == IBM_FLOW_CONST_FLUX;
    cudaEvent_t t;
    timer_begin(h, "momentum", &t);
    ibm_status st0 = launch_momentum<T>(h, k, sp, ib, grd);
    if (st0 != IBM_OK) return st0;
    timer_end(h, t, "momentum");
    if (cflux) {
        int nparts = grd.x * grd.y * grd.z;
        double dV = g.dx * g.dy * (g.ndim == 3 ? g.dz : 1.0);
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
            k_flux_apply<T><<<fgrd, dim3(32, 8, 1), 0, h->stream>>>(g, (T*)h->ustar[0], h->mask, ib, h->scal, sp.ckdt);
            IBM_LAUNCH_CHECK();
        }
        for (int c = 0; c < g.ncomp; ++c)
            IBM_CUDA_TRY(cudaMemcpyAsync(h->buf.u[c], h->ustar[c], g.N * sizeof(T), cudaMemcpyDeviceToDevice, h->stream));
        return IBM_OK;
    }
    const FluxCorr<T> fc = flux_corr<T>(h, k);
    ibm_status st = divergence_and_solve<T>(h, us, cflux, fc);
    if (st != IBM_OK) return st;
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
                                              us[1], us[2]);
    IBM_LAUNCH_CHECK();
    const FluxCorr<T> fc = flux_corr<T>(h, 0);
    ibm_status st = divergence_and_solve<T>(h, us, false, fc);
    if (st != IBM_OK) return st;
    return launch_correct<T>(h, us, (T)1, 0, false, fc);
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
            StageP<T> sp;
            IbmStage<T> ib;
            dim3 grd;
            launch_momentum<T>(h, 0, sp, ib, grd);
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
            k_divergence<T, true, false><<<zmarch_grid(g), dim3(32, 8), 0, h->stream>>>(
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

}  // namespace

int diag_blocks() { return DIAG_BLOCKS; }

// Default z-chunk of the momentum predictor.  Per choice: the last wave's
// fill (waves / whole waves) and the share of planes a block loads only for
// its stencil (two per chunk).  Choices with at least four waves are
// preferred: with fewer, one slow SM or a half-empty last wave shows.
int momentum_default_kzm(const GridP& g, int prec) {
    if (g.ndim != 3) return KZM_CHOICES[0];
    int dev = 0, sms = 0, per = 0;
    const int threads = MOM_TX * MOM_WARPS;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 0;
    cudaError_t e = prec == IBM_FP64
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_momentum<double, true>, threads, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_momentum<float, true>, threads, 0);
    if (e != cudaSuccess || sms <= 0 || per <= 0) {
        cudaGetLastError();
        return 24;
    }
    const double slots = (double)sms * per;
    const double cols = (double)g.nsegx * ((g.ny + MOM_TY - 1) / MOM_TY);
    double best = 1e300;
    int pick = KZM_CHOICES[0];
    for (int pass = 0; pass < 2 && best == 1e300; ++pass)
        for (int kz : KZM_CHOICES) {
            const double waves = cols * ((g.nz + kz - 1) / kz) / slots;
            if (pass == 0 && waves < 4.0) continue;
            const double len = std::min(kz, g.nz);
            const double cost = std::ceil(waves) / waves * (len + 2.0) / len;
            if (cost < best) { best = cost; pick = kz; }
        }
    return pick;
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
ibm_status run_diagnostics(ibm_solver* h, double* out16) {
    return h->prec == IBM_FP64 ? diag_t<double>(h, out16) : diag_t<float>(h, out16);
}
