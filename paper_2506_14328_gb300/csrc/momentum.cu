// The momentum predictor (K3): explicit RHS of the RK3 substage fused with the
// implicit IBM diagonal division (Sec. 2.4, Eq. rk3-rai).
//
// Two kernels compute the same update:
//   * k_momentum      - plane loads through registers; any grid, 2D and 3D;
//   * k_momentum_tma  - 3D grids whose x extent is a multiple of 16: plane
//                       tiles arrive by TMA (cp.async.bulk.tensor) into a ring
//                       of shared-memory stages completed on mbarriers, so
//                       loads run several planes ahead without holding
//                       registers.
#include "common.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>

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
    // inflow/outflow x: xa (cells A, B) and xh (halo) are 1 beyond the inflow face, 2 beyond
    // the outflow face, else 0; outa / outh: the point is the outflow face column of u
    int xa, xh;
    bool outa, outh;
};

// Source column of tile column i: wrapped (periodic x), or the adjacent column with
// a ghost kind beyond an inflow (1) or outflow (2) face.
__device__ __forceinline__ int mom_col(const GridP& g, int i, int& xk) {
    xk = 0;
    if (g.xper) return ((i % g.nx) + g.nx) % g.nx;
    if (i < 0) { xk = 1; return 0; }
    if (i >= g.nx) { xk = 2; return g.nx - 1; }
    return i;
}

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
    const int ix = mom_col(g, i0 + tx, S.xa);
    S.outa = !g.xper && S.xa == 0 && ix == g.nx - 1;
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
    S.xh = S.xa;
    S.outh = S.outa;
    if (w == 0 || w == 1) {                       // halo rows below and above the tile
        const int jh = mom_row(g, w == 0 ? j0 - 1 : j0 + MY, sig_lo, sig_hi, S.fh, S.gh);
        S.hh = true;
        S.oh = ix + g.nx * jh;
        S.th = (w == 0 ? 0 : (HY - 1) * HX) + tx + 1;
    } else if ((w == 2 || w == 3) && tx < HY) {   // halo columns left and right (with corners)
        const int jh = mom_row(g, j0 - 1 + tx, sig_lo, sig_hi, S.fh, S.gh);
        const int ih = mom_col(g, w == 2 ? i0 - 1 : i0 + MX, S.xh);
        S.outh = !g.xper && S.xh == 0 && ih == g.nx - 1;
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

// value as the operator reads it: 0 unless internal (or the fluid outflow face
// of u); beyond an inflow face u reads the inflow velocity and v, w the negated
// adjacent value, beyond an outflow face v, w repeat it; then the y-wall rule.
// sh selects the point's mask byte in m.
template <typename T, bool EDGE>
__device__ __forceinline__ T mom_masked(T x, uint32_t m, int sh, int c, bool beyond, T f, int xk, bool outc, T uin) {
    const uint32_t mb = (m >> sh) & 0xffu;
    bool rd = (mb >> c) & 1u;
    if (EDGE && c == 0 && outc) rd = (mb & IBM_MASK_FACE) != 0;
    x = rd ? x : T(0);
    if (EDGE && xk == 1) x = (c == 0) ? ((mb & IBM_MASK_FACE) ? uin : T(0)) : -x;
    else if (EDGE && xk == 2) x = (c == 0) ? T(0) : x;
    if (EDGE && beyond) x = (c == 1) ? T(0) : f * x;
    return x;
}

template <typename T, int NC, bool EDGE>
__device__ __forceinline__ void mom_store(T* tile, const MomSrc<T>& S, const MomRegs<T, NC>& R, T uin) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        tile[c * HP + S.ta] = mom_masked<T, EDGE>(R.a[c], R.m, 0, c, S.ga, S.fa, S.xa, S.outa, uin);
        tile[c * HP + S.tb] = mom_masked<T, EDGE>(R.b[c], R.m, 8, c, S.gb, S.fb, S.xa, S.outa, uin);
        if (S.hh) tile[c * HP + S.th] = mom_masked<T, EDGE>(R.h[c], R.m, 16, c, S.gh, S.fh, S.xh, S.outh, uin);
    }
}

template <typename T, int NC>
__device__ __forceinline__ void mom_store_plane(T* tile, const MomSrc<T>& S, const MomRegs<T, NC>& R, bool edge,
                                                T uin) {
    if (edge) mom_store<T, NC, true>(tile, S, R, uin);
    else mom_store<T, NC, false>(tile, S, R, uin);
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
// out = uP + R with R = dt a_k N - (c_k dt / dx_c) dp (+ dt b_k N^{k-2}), dp the
// pressure difference across the point.
template <typename T>
__device__ __forceinline__ void mom_update(const StageP<T>& sp, T uP, T N, T dp, T cg, T Nprev, T& out, T& R) {
    R = sp.dta * N - cg * dp;
    if (sp.read_prev) R += sp.dtb * Nprev;
    out = uP + R;
}

// the implicit IBM division of one IBM point (Eq. rk3-rai): the wall source s
// joins N, and u* = alpha u + beta R.  The explicit treatment stores lambda in pad
// (0 otherwise), so that -lambda u joins N as well.
template <typename T>
__device__ __forceinline__ void mom_ibm(const StageP<T>& sp, const Coef4<T>& q, T uP, T R, T& out, T& N) {
    N += q.s - q.pad * uP;
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

// DEFER: an IBM point keeps R (its update before the division) in u* and N without the wall
// source; k_ibm_division finishes u* (and, for the explicit IBM, N), and the flow-rate sum
// leaves the point out.
template <typename T, int NC, bool DEFER = false>
__device__ __forceinline__ void mom_write(const MomF<T>& F, const StageP<T>& sp, int ida, int idb, bool liveA,
                                          bool liveB, uint32_t mA, uint32_t mB, T (&oA)[3], T (&oB)[3], T (&NA)[3],
                                          T (&NB)[3], T& fsum, bool outcol, const T (&RA)[3], const T (&RB)[3]) {
    if (DEFER) {
        const T fa = ((mA >> 4) & 1u) ? T(0) : oA[0], fb = ((mB >> 4) & 1u) ? T(0) : oB[0];
        fsum += ((mA & 1u) ? fa : T(0)) + ((mB & 1u) ? fb : T(0));
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        if (c == 0 && outcol) continue;   // u on the outflow face: the outflow update writes it
        const bool ia = (mA >> c) & 1u, ibb = (mB >> c) & 1u;
        if (DEFER) {
            if ((mA >> (4 + c)) & 1u) oA[c] = RA[c];
            if ((mB >> (4 + c)) & 1u) oB[c] = RB[c];
        }
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
    if (!DEFER) fsum += oA[0] + oB[0];
}

// One plane k of the 3D update.  t0 / t1: the tiles of planes k and k+1, with
// rows RS apart and components CS apart; a, b: the tile positions of A and B.
// DEFER: the IBM division is left to k_ibm_division (see mom_write).
template <typename T, int RS, int CS, bool OWN, bool DEFER = false>
__device__ __forceinline__ void mom_plane3(const GridP& g, const MomF<T>& F, const StageP<T>& sp,
                                           const IbmStage<T>& ib, int a, int b, const T* __restrict__ t0,
                                           const T* __restrict__ t1, MomCarry<T>& C, const MomPre<T>& P,
                                           const T (&ownA)[3], const T (&ownB)[3], uint32_t m, int k, int ida,
                                           int idb, bool liveA, bool liveB, int segA, T& fsum, bool outcol) {
    constexpr int HX = RS;
    const T* U0 = t0;
    const T* V0 = t0 + CS;
    const T* W0 = t0 + 2 * CS;
    const T* U1 = t1;
    const T* V1 = t1 + CS;
    const T* W1 = t1 + 2 * CS;
    const T two = T(2);
    // plane k (the own column and u(i-1), v(j-1) of A are carried)
    const T uEA = U0[a + 1], uEB = U0[b + 1], uSA = U0[a - HX], uNB = U0[b + HX], uNWB = U0[b + HX - 1];
    const T vEA = V0[a + 1], vEB = V0[b + 1], vWA = V0[a - 1], vWB = V0[b - 1], vNB = V0[b + HX];
    const T vSEA = V0[a - HX + 1];
    const T wEA = W0[a + 1], wEB = W0[b + 1], wWA = W0[a - 1], wWB = W0[b - 1], wSA = W0[a - HX];
    const T wNB = W0[b + HX];
    // plane k+1
    // plane k+1 at A and B: already in registers when OWN (ownA, ownB = u, v, w)
    const T uTA = OWN ? ownA[0] : U1[a], uTB = OWN ? ownB[0] : U1[b];
    const T vTA = OWN ? ownA[1] : V1[a], vTB = OWN ? ownB[1] : V1[b];
    const T wTA = OWN ? ownA[2] : W1[a], wTB = OWN ? ownB[2] : W1[b];
    const T uTWA = U1[a - 1], uTWB = U1[b - 1], vTSA = V1[a - HX];
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
        T lap = (uEA + uWA) * sp.nx2 + (uB + uSA) * sp.ny2 + (uTA + C.ubA) * sp.nz2 - sp.lc * uA;
        NA[0] = lap - conv + sp.g[0];
        mom_update(sp, uA, NA[0], P.eA - pA, sp.cgx, P.qA[0], oA[0], RA[0]);
        conv = (uEB - uWB) * (uEB + uWB + two * uB) * sp.qx;
        conv += (xyB - xyA) * sp.qy;
        conv += (xzB - C.fuB) * sp.qz;
        lap = (uEB + uWB) * sp.nx2 + (uNB + uA) * sp.ny2 + (uTB + C.ubB) * sp.nz2 - sp.lc * uB;
        NB[0] = lap - conv + sp.g[0];
        mom_update(sp, uB, NB[0], P.eB - pB, sp.cgx, P.qB[0], oB[0], RB[0]);
    }
    {   // v
        T conv = (xyA - xyAw) * sp.qx;
        conv += (vB - vSA) * (vB + vSA + two * vA) * sp.qy;
        conv += (yzA - C.fvA) * sp.qz;
        T lap = (vEA + vWA) * sp.nx2 + (vB + vSA) * sp.ny2 + (vTA + C.vbA) * sp.nz2 - sp.lc * vA;
        NA[1] = lap - conv + sp.g[1];
        mom_update(sp, vA, NA[1], pB - pA, sp.cgy, P.qA[1], oA[1], RA[1]);
        conv = (xyB - xyBw) * sp.qx;
        conv += (vNB - vA) * (vNB + vA + two * vB) * sp.qy;
        conv += (yzB - C.fvB) * sp.qz;
        lap = (vEB + vWB) * sp.nx2 + (vNB + vA) * sp.ny2 + (vTB + C.vbB) * sp.nz2 - sp.lc * vB;
        NB[1] = lap - conv + sp.g[1];
        mom_update(sp, vB, NB[1], P.nB - pB, sp.cgy, P.qB[1], oB[1], RB[1]);
    }
    {   // w
        T conv = (xzA - xzAw) * sp.qx;
        conv += (yzA - yzAs) * sp.qy;
        conv += (wTA - C.wbA) * (wTA + C.wbA + two * wA) * sp.qz;
        T lap = (wEA + wWA) * sp.nx2 + (wB + wSA) * sp.ny2 + (wTA + C.wbA) * sp.nz2 - sp.lc * wA;
        NA[2] = lap - conv + sp.g[2];
        mom_update(sp, wA, NA[2], P.tA - pA, sp.cgz, P.qA[2], oA[2], RA[2]);
        conv = (xzB - xzBw) * sp.qx;
        conv += (yzB - yzA) * sp.qy;
        conv += (wTB - C.wbB) * (wTB + C.wbB + two * wB) * sp.qz;
        lap = (wEB + wWB) * sp.nx2 + (wNB + wA) * sp.ny2 + (wTB + C.wbB) * sp.nz2 - sp.lc * wB;
        NB[2] = lap - conv + sp.g[2];
        mom_update(sp, wB, NB[2], P.tB - pB, sp.cgz, P.qB[2], oB[2], RB[2]);
    }
    const uint32_t mA = m & 0xffu, mB = (m >> 8) & 0xffu;
    if (!DEFER && __any_sync(0xffffffffu, (mA | mB) & (IBM_MASK_IBM_U | IBM_MASK_IBM_V | IBM_MASK_IBM_W))) {
        const T ua3[3] = {uA, vA, wA}, ub3[3] = {uB, vB, wB};
        mom_ibm_fix<T, 3>(ib, sp, mA, mB, segA, segA + g.nsegx, ua3, ub3, RA, RB, oA, oB, NA, NB);
    }
    mom_write<T, 3, DEFER>(F, sp, ida, idb, liveA, liveB, mA, mB, oA, oB, NA, NB, fsum, outcol, RA, RB);

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
                                           bool liveA, bool liveB, int segA, T& fsum, bool outcol) {
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
        mom_update(sp, uA, NA[0], P.eA - pA, sp.cgx, P.qA[0], oA[0], RA[0]);
        conv = (uEB - uWB) * (uEB + uWB + two * uB) * sp.qx + (xyB - xyA) * sp.qy;
        lap = (uEB + uWB - two * uB) * sp.nx2 + (uNB + uA - two * uB) * sp.ny2;
        NB[0] = lap - conv + sp.g[0];
        mom_update(sp, uB, NB[0], P.eB - pB, sp.cgx, P.qB[0], oB[0], RB[0]);
    }
    {
        T conv = (xyA - xyAw) * sp.qx + (vB - vSA) * (vB + vSA + two * vA) * sp.qy;
        T lap = (vEA + vWA - two * vA) * sp.nx2 + (vB + vSA - two * vA) * sp.ny2;
        NA[1] = lap - conv + sp.g[1];
        mom_update(sp, vA, NA[1], pB - pA, sp.cgy, P.qA[1], oA[1], RA[1]);
        conv = (xyB - xyBw) * sp.qx + (vNB - vA) * (vNB + vA + two * vB) * sp.qy;
        lap = (vEB + vWB - two * vB) * sp.nx2 + (vNB + vA - two * vB) * sp.ny2;
        NB[1] = lap - conv + sp.g[1];
        mom_update(sp, vB, NB[1], P.nB - pB, sp.cgy, P.qB[1], oB[1], RB[1]);
    }
    const uint32_t mA = m & 0xffu, mB = (m >> 8) & 0xffu;
    if (__any_sync(0xffffffffu, (mA | mB) & (IBM_MASK_IBM_U | IBM_MASK_IBM_V))) {
        const T ua3[3] = {uA, vA, T(0)}, ub3[3] = {uB, vB, T(0)};
        mom_ibm_fix<T, 2>(ib, sp, mA, mB, segA, segA + g.nsegx, ua3, ub3, RA, RB, oA, oB, NA, NB);
    }
    mom_write<T, 2>(F, sp, ida, idb, liveA, liveB, mA, mB, oA, oB, NA, NB, fsum, outcol, RA, RB);
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
    mom_store_plane<T, 3>(tiles + s1, S, R, yedge, sp.uin);       // plane k+1
    mn = R.m & 0xffffu;
    if (k + 3 <= kend) mom_fetch<T, 3>(F, S, R, wrapi(k + 3, g.nz) * plane);
    if (k + 1 < kend) mom_pre(F, S, Pn, g, k + 1, plane, sp.read_prev);
    __syncthreads();
    const int ida = rowA + k * plane;
    const T none[3] = {T(0), T(0), T(0)};
    mom_plane3<T, HX, HP, false>(g, F, sp, ib, S.ta, S.tb, tiles + s0, tiles + s1, C, Pc, none, none, mc, k, ida,
                                 ida + g.nx, liveA, liveB, segrow + k * g.ny * g.nsegx, fsum, S.outa);
    const int t = s0;
    s0 = s1;
    s1 = s2;
    s2 = t;
}

// One block's work of the register form: the 32 x 16 column (bx, by) over z chunk bz; the
// flux partial goes to flux_part[pidx].  tiles: 3 plane slots (3D) or 1 (2D) of 3 * HP values.
template <typename T, bool THREE>
__device__ __forceinline__ void mom_block(const GridP& g, const MomF<T>& F, const StageP<T>& sp,
                                          const IbmStage<T>& ib, double* __restrict__ flux_part, int bx, int by,
                                          int bz, long long pidx, T* tiles, double* shd) {
    constexpr int NC = THREE ? 3 : 2;
    constexpr int SLOT = 3 * HP;                 // one plane tile (u, v, w)
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = bx * MX, j0 = by * MY;
    const int i = i0 + tx, jA = j0 + 2 * ty;
    const bool liveA = i < g.nx && jA < g.ny;
    const bool liveB = i < g.nx && jA + 1 < g.ny;
    // blocks that touch a y wall, or an x face of an inflow/outflow box, apply the ghost rules
    const bool yedge = j0 == 0 || j0 + MY >= g.ny || (!g.xper && (i0 == 0 || i0 + MX >= g.nx));
    const int plane = g.nx * g.ny;
    const int rowA = i + g.nx * jA;               // in-plane index of A (B: + nx)
    const int segrow = jA * g.nsegx + bx;          // row segment of A at plane 0
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
        const int kbeg = bz * g.kzm;
        const int kend = min(kbeg + g.kzm, g.nz);
        int s0 = 0, s1 = SLOT, s2 = 2 * SLOT;
        // prologue: planes kbeg-1 (slot 2) and kbeg (slot 0) give the carried state
        mom_fetch<T, 3>(F, S, X, wrapi(kbeg - 1, g.nz) * plane);
        mom_fetch<T, 3>(F, S, Y, kbeg * plane);
        mom_pre(F, S, P0, g, kbeg, plane, sp.read_prev);
        MomCarry<T> C;
        C.pA = F.p[kbeg * plane + S.oa];
        C.pB = F.p[kbeg * plane + S.ob];
        mom_store_plane<T, 3>(tiles + s2, S, X, yedge, sp.uin);
        mom_store_plane<T, 3>(tiles + s0, S, Y, yedge, sp.uin);
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
        mom_store_plane<T, NC>(tiles, S, X, yedge, sp.uin);
        __syncthreads();
        mom_plane2<T>(g, F, sp, ib, S, tiles, P0, pA, pB, X.m & live_bits, rowA, rowA + g.nx, liveA, liveB, segrow,
                      fsum, S.outa);
    }
    if (sp.flux_sum) {
        // FP32 sums within a warp, FP64 across warps and blocks
        T ws = warp_sum(fsum);
        if (tx == 0) shd[ty] = (double)ws;
        __syncthreads();
        if (tx == 0 && ty == 0) {
            double s = 0.0;
            for (int w = 0; w < MW; ++w) s += shd[w];
            flux_part[pidx] = s;
        }
    }
}

template <typename T, bool THREE>
__global__ void __launch_bounds__(MX * MW, sizeof(T) == 4 ? 2 : 1)
    k_momentum(GridP g, MomF<T> F, StageP<T> sp, IbmStage<T> ib, double* __restrict__ flux_part) {
    constexpr int NS = THREE ? 3 : 1;
    __shared__ T tiles[NS * 3 * HP];
    __shared__ double shd[MW];
    mom_block<T, THREE>(g, F, sp, ib, flux_part, blockIdx.x, blockIdx.y, blockIdx.z,
                        blockIdx.x + gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z), tiles, shd);
}

// ---------------------------------------------------------------------------
// Many solves' momentum predictors in one persistent launch (serving many small grids):
// one block per SM slot walks a work list of (solve, column, z chunk) tiles of every job,
// each job carrying its own grid, fields, stage constants and IBM coefficients.  The tile
// work is the register form's (mom_block), so each solve's update is bit for bit what its
// own k_momentum launch computes.  tile0[q]: the first tile of job q (prefix sums); the table
// (at most MOM_MAX_JOBS jobs) goes by value with the launch.
// ---------------------------------------------------------------------------
template <typename T>
struct MomJob {
    GridP g;
    MomF<T> F;
    StageP<T> sp;
    IbmStage<T> ib;
    double* part;
    int nbx, nby, nbz;
};

template <typename T>
struct MomJobs {
    int njobs, ntiles;
    int tile0[MOM_MAX_JOBS];
    MomJob<T> job[MOM_MAX_JOBS];
};

template <typename T>
__global__ void __launch_bounds__(MX * MW, sizeof(T) == 4 ? 2 : 1)
    k_momentum_jobs(const __grid_constant__ MomJobs<T> jobs) {
    __shared__ T tiles[3 * 3 * HP];
    __shared__ double shd[MW];
    for (int t = blockIdx.x; t < jobs.ntiles; t += gridDim.x) {
        int lo = 0, hi = jobs.njobs - 1;             // the job whose tile range holds t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs.tile0[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const MomJob<T>& J = jobs.job[lo];
        const int l = t - jobs.tile0[lo];
        const int bx = l % J.nbx, by = (l / J.nbx) % J.nby, bz = l / (J.nbx * J.nby);
        const long long pidx = bx + (long long)J.nbx * (by + (long long)J.nby * bz);
        __syncthreads();                             // the previous tile is done with the shared tiles
        if (J.g.ndim == 3) mom_block<T, true>(J.g, J.F, J.sp, J.ib, J.part, bx, by, bz, pidx, tiles, shd);
        else mom_block<T, false>(J.g, J.F, J.sp, J.ib, J.part, bx, by, bz, pidx, tiles, shd);
    }
}

// ---------------------------------------------------------------------------
// K3 in its general form: the update of k_momentum on a stretched wall-normal grid
// (STR, reading R23) and/or with a moving body (BODY, reading R24).
//   * STR: the y terms on uneven rows, from the per-row tables (ytab): the Laplacian's y
//     part is the uneven three-point second difference of the point's own grid (centre rows
//     for u and w, face rows for v); the convective y fluxes stay in flux form, u and w
//     carried to a v face by linear interpolation between the centres on either side, v to a
//     centre by the plain average, the flux difference divided by the point's own control
//     height (the cell height for u and w, the centre distance across the face for v); v's
//     pressure gradient is divided by the centre distance across its face.
//   * BODY: the body's points (not internal, not a box face) are read as the body's velocity
//     by the convective terms and the Laplacian alike, and hold it in u*; the wall source of
//     the weights is then in its body-frame form (-lambda (w - U_b) for a translating body).
// A 32 x 8 block covers the same 32 x 16 column and z chunk as k_momentum (so the flux
// partials line up); each thread updates its two cells plane by plane, reading every
// neighbour through the operator's rules straight from memory.
// ---------------------------------------------------------------------------
template <typename T, bool BODY>
__device__ __forceinline__ T mom_op(const GridP& g, const T* __restrict__ f, const uint8_t* __restrict__ mask, int c,
                                    int i, int j, int k, const StageP<T>& sp, const BodyP& body) {
    int xk = 0, ii = i;
    if (g.xper) ii = wrapi(i, g.nx);
    else if (i < 0) { xk = 1; ii = 0; }
    else if (i >= g.nx) { xk = 2; ii = g.nx - 1; }
    T fct = T(1);
    bool beyond = false;
    int jj = j;
    if (j < 0) { beyond = true; fct = sp.sig_lo; jj = 0; }
    else if (j >= g.ny) { beyond = true; fct = sp.sig_hi; jj = g.ny - 1; }
    const int kk = g.ndim == 3 ? wrapi(k, g.nz) : 0;
    const long long id = ii + (long long)g.nx * (jj + (long long)g.ny * kk);
    const uint32_t m = (uint32_t)__ldg(mask + id);
    T x = __ldg(f + id);
    if constexpr (BODY) {
        // (a moving body needs a periodic x: the only box-face point is v on the +y wall)
        if (!((m >> c) & 1u) && !(c == 1 && jj == g.ny - 1)) {
            const double xc = g.ox + ((double)ii + (c == 0 ? 1.0 : 0.5)) * g.dx;
            const double yc = g.oy + ((double)jj + (c == 1 ? 1.0 : 0.5)) * g.dy;
            x = (T)bodyvel(body, c, xc, yc);
            return beyond ? ((c == 1) ? T(0) : fct * x) : x;
        }
    }
    const bool outc = !g.xper && xk == 0 && ii == g.nx - 1;
    return mom_masked<T, true>(x, m, 0, c, beyond, fct, xk, outc, sp.uin);
}

template <typename T, bool THREE, bool STR, bool BODY>
__global__ void __launch_bounds__(MX * MW) k_momentum_gen(GridP g, MomF<T> F, StageP<T> sp, IbmStage<T> ib,
                                                          BodyP body, double* __restrict__ flux_part) {
    __shared__ double shd[MW];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.x * MX + tx;
    const bool livex = i < g.nx;
    const int kbeg = THREE ? blockIdx.z * g.kzm : 0;
    const int kend = THREE ? min(kbeg + g.kzm, g.nz) : 1;
    const unsigned lt = lanemask_lt();
    double fsum = 0.0;
    for (int r = 0; r < 2; ++r) {
        const int j = blockIdx.y * MY + 2 * ty + r;
        if (j >= g.ny) break;                                    // whole warp
        // per-row constants: the tables of a stretched y, else the uniform spacing
        const T half = T(0.5);
        const T dyc = STR ? (T)ytab(g, YT_DYC, j) : (T)g.dy;
        const T idyc = STR ? (T)ytab(g, YT_IDYC, j) : sp.idy;
        const T ihv = STR ? (T)ytab(g, YT_IHV, j) : sp.idy;
        const T alo = STR ? (T)ytab(g, YT_ALO, j) : half, ahi = STR ? (T)ytab(g, YT_AHI, j) : half;
        const T blo = (STR && j > 0) ? (T)ytab(g, YT_ALO, j - 1) : half;
        const T bhi = (STR && j > 0) ? (T)ytab(g, YT_AHI, j - 1) : half;
        const T cm = STR ? sp.nu * (T)ytab(g, YT_DCM, j) : sp.ny2;
        const T c0 = STR ? sp.nu * (T)ytab(g, YT_DC0, j) : T(-2) * sp.ny2;
        const T cp = STR ? sp.nu * (T)ytab(g, YT_DCP, j) : sp.ny2;
        const T vm_ = STR ? sp.nu * (T)ytab(g, YT_DVM, j) : sp.ny2;
        const T v0_ = STR ? sp.nu * (T)ytab(g, YT_DV0, j) : T(-2) * sp.ny2;
        const T vp_ = STR ? sp.nu * (T)ytab(g, YT_DVP, j) : sp.ny2;
        const T cgy = STR ? sp.ckdt * ihv : sp.cgy;
        for (int k = kbeg; k < kend; ++k) {
            auto U = [&](int di, int dj, int dk) { return mom_op<T, BODY>(g, F.u[0], F.mask, 0, i + di, j + dj, k + dk, sp, body); };
            auto V = [&](int di, int dj, int dk) { return mom_op<T, BODY>(g, F.u[1], F.mask, 1, i + di, j + dj, k + dk, sp, body); };
            auto W = [&](int di, int dj, int dk) { return mom_op<T, BODY>(g, F.u[2], F.mask, 2, i + di, j + dj, k + dk, sp, body); };
            const long long id = (long long)i + (long long)g.nx * (j + (long long)g.ny * k);
            const int ic = livex ? i : g.nx - 1;
            const long long idc = (long long)ic + (long long)g.nx * (j + (long long)g.ny * k);
            const uint32_t m = livex ? (uint32_t)__ldg(F.mask + idc) : 0u;
            T Nv[3] = {T(0), T(0), T(0)}, Pv[3] = {T(0), T(0), T(0)};
            T own[3] = {T(0), T(0), T(0)};
            if (livex) {
                const T pc = F.p[idc];
                const T pE = F.p[(long long)(g.xper ? wrapi(i + 1, g.nx) : min(i + 1, g.nx - 1)) +
                                 (long long)g.nx * (j + (long long)g.ny * k)];
                const T pN = F.p[idc + (j + 1 < g.ny ? g.nx : 0)];
                const T pT = THREE ? F.p[(long long)i + (long long)g.nx * (j + (long long)g.ny * wrapi(k + 1, g.nz))]
                                   : T(0);
                // ---- u
                const T u0 = U(0, 0, 0), uE = U(1, 0, 0), uW = U(-1, 0, 0), uN = U(0, 1, 0), uS = U(0, -1, 0);
                const T v0 = V(0, 0, 0), vE1 = V(1, 0, 0), vS0 = V(0, -1, 0), vSE = V(1, -1, 0);
                T conv = ((u0 + uE) * (u0 + uE) - (uW + u0) * (uW + u0)) * sp.qx;
                conv += ((v0 + vE1) * (alo * u0 + ahi * uN) - (vS0 + vSE) * (blo * uS + bhi * u0)) * half * idyc;
                T lap = (uE - T(2) * u0 + uW) * sp.nx2 + cm * uS + c0 * u0 + cp * uN;
                T wc = T(0), wT = T(0), wB = T(0), uT = T(0), uB = T(0), wE = T(0), wW = T(0), wN = T(0), wS = T(0);
                if (THREE) {
                    wc = W(0, 0, 0);
                    uT = U(0, 0, 1);
                    uB = U(0, 0, -1);
                    const T wE1 = W(1, 0, 0), wB0 = W(0, 0, -1), wBE = W(1, 0, -1);
                    conv += ((wc + wE1) * (u0 + uT) - (wB0 + wBE) * (uB + u0)) * sp.qz;
                    lap += (uT - T(2) * u0 + uB) * sp.nz2;
                    wE = wE1;
                    wB = wB0;
                }
                Nv[0] = lap - conv + sp.g[0];
                Pv[0] = pE - pc;
                // ---- v
                {
                    const T vW = V(-1, 0, 0), vN = V(0, 1, 0);
                    const T uWN = U(-1, 1, 0);
                    T cv = ((alo * u0 + ahi * uN) * (v0 + vE1) - (alo * uW + ahi * uWN) * (vW + v0)) * half * sp.idx;
                    cv += ((v0 + vN) * (v0 + vN) - (vS0 + v0) * (vS0 + v0)) * T(0.25) * ihv;
                    T lv = (vE1 - T(2) * v0 + vW) * sp.nx2 + vm_ * vS0 + v0_ * v0 + vp_ * vN;
                    if (THREE) {
                        const T vT = V(0, 0, 1), vB = V(0, 0, -1);
                        const T wN1 = W(0, 1, 0), wBN = W(0, 1, -1);
                        cv += ((alo * wc + ahi * wN1) * (v0 + vT) - (alo * wB + ahi * wBN) * (vB + v0)) * half * sp.idz;
                        lv += (vT - T(2) * v0 + vB) * sp.nz2;
                        wN = wN1;
                    }
                    Nv[1] = lv - cv + sp.g[1];
                    Pv[1] = pN - pc;
                }
                // ---- w
                if (THREE) {
                    wW = W(-1, 0, 0);
                    wS = W(0, -1, 0);
                    wT = W(0, 0, 1);
                    const T uWT = U(-1, 0, 1), vT0 = V(0, 0, 1), vST = V(0, -1, 1);
                    T cw = ((u0 + uT) * (wc + wE) - (uW + uWT) * (wW + wc)) * sp.qx;
                    cw += ((v0 + vT0) * (alo * wc + ahi * wN) - (vS0 + vST) * (blo * wS + bhi * wc)) * half * idyc;
                    cw += ((wc + wT) * (wc + wT) - (wB + wc) * (wB + wc)) * sp.qz;
                    T lw = (wE - T(2) * wc + wW) * sp.nx2 + cm * wS + c0 * wc + cp * wN + (wT - T(2) * wc + wB) * sp.nz2;
                    Nv[2] = lw - cw + sp.g[2];
                    Pv[2] = pT - pc;
                }
                own[0] = u0;
                own[1] = v0;
                own[2] = wc;
            }
            // stage combination, the implicit IBM division at IBM points, stores
            const T cg[3] = {sp.cgx, cgy, sp.cgz};
            const int seg = (j + g.ny * k) * g.nsegx + (int)blockIdx.x;
#pragma unroll
            for (int c = 0; c < (THREE ? 3 : 2); ++c) {
                T R = sp.dta * Nv[c] - cg[c] * Pv[c];
                if (sp.read_prev && livex) R += sp.dtb * F.Nn[c][id];
                T out = own[c] + R;
                T Nc = Nv[c];
                const bool ibmp = (m >> (4 + c)) & 1u;
                const unsigned b = __ballot_sync(0xffffffffu, ibmp);
                if (ibmp) mom_ibm(sp, ib.coef[c][ib.segoff[c][seg] + __popc(b & lt)], own[c], R, out, Nc);
                if (!livex) continue;
                if (c == 0 && !g.xper && i == g.nx - 1) continue;   // the outflow face: written by the outflow update
                const bool in = (m >> c) & 1u;
                // a moving body's points hold its velocity (own[c] is what the operator reads there)
                const T rest = (BODY && !(c == 1 && j == g.ny - 1)) ? own[c] : T(0);
                out = in ? out : rest;
                Nc = in ? Nc : T(0);
                F.us[c][id] = out;
                if (sp.write_n) F.Nn[c][id] = Nc;
                if (c == 0) fsum += (double)out * (double)dyc;
            }
        }
    }
    if (sp.flux_sum) {
        const double ws = warp_sum(fsum);
        if (tx == 0) shd[ty] = ws;
        __syncthreads();
        if (tx == 0 && ty == 0) {
            double t = 0.0;
            for (int w = 0; w < MW; ++w) t += shd[w];
            flux_part[blockIdx.x + gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z)] = t;
        }
    }
}

// ---------------------------------------------------------------------------
// K3 with TMA plane loads (3D, nx a multiple of 16).
//
// Each block owns the same 32 x 16 column of cells as k_momentum.  One thread
// issues, per plane, tensor copies of the boxes the stencil needs into one
// stage of a ring of D stages in shared memory, completed on that stage's
// mbarrier:
//   u, v, w  40 x 18 at (i0-4, j0-1)   x start rounded down to 16 bytes
//   mask     64 x 18 at (i0-16, j0-1)  (one byte per cell)
//   p        40 x 17 at (i0, j0)       (+x and +y neighbours; planes kbeg..kend)
//   N^{k-2}  32 x 16 at (i0, j0)       (stages 2 and 3; planes kbeg..kend-1)
// Rows or columns outside the box read 0 (the copy's fill).  Periodic x is
// completed from small wrap boxes (the last 4 / 16 columns for the block at
// x = 0, the first ones for the block that reaches nx); an inflow/outflow x
// takes its ghost columns from the box's own first or last grid column.  Before
// a plane is computed its u, v, w tile is rewritten in place into the form the
// operator reads (non-internal -> 0, ghost rows beyond a y wall, wrapped or
// ghost columns, the outflow face of u), and
// the thread keeps its own two cells' values and masks in registers.  Plane
// k+D-1 is requested while plane k is computed (D = 3 for FP32, 4 for FP64),
// so two or three planes of every block are in flight without register cost.
// ---------------------------------------------------------------------------
template <typename T>
struct TmaLay {
    static constexpr int es = (int)sizeof(T);
    // ring depth in planes: FP32 keeps three blocks of 256 threads per SM
    static constexpr int D = sizeof(T) == 4 ? 3 : 4;
    static constexpr int RX = 40, RY = 18;      // u, v, w box
    static constexpr int MXB = 64;              // mask box width (bytes)
    static constexpr int PX = 40, PY = 17;      // pressure box
    static constexpr int QX = 32, QY = 16;      // previous-RHS box
    static constexpr int WX = 4, WMX = 16;      // wrap boxes (values, mask)
    static constexpr int a128(int b) { return (b + 127) / 128 * 128; }
    static constexpr int CSB = a128(RX * RY * es);       // bytes per component tile
    static constexpr int CS = CSB / es;                   // ... in elements
    static constexpr int oM = 3 * CSB;
    static constexpr int oP = oM + a128(MXB * RY);
    static constexpr int oQ = oP + a128(PX * PY * es);
    static constexpr int QCSB = a128(QX * QY * es);
    static constexpr int oWL = oQ + 3 * QCSB;
    static constexpr int WCSB = a128(WX * RY * es);
    static constexpr int oWR = oWL + 3 * WCSB;
    static constexpr int oWML = oWR + 3 * WCSB;
    static constexpr int oWMR = oWML + a128(WMX * RY);
    static constexpr int oWPR = oWMR + a128(WMX * RY);
    static constexpr int SB = oWPR + a128(WX * PY * es);  // one stage
    static constexpr int SMEM = D * SB + D * 8 + 128;   // + mbarriers + alignment slack
};

struct MomMaps {
    CUtensorMap u[3], uw[3];   // velocity components: main box, wrap box
    CUtensorMap m, mw;         // mask
    CUtensorMap p, pw;         // pressure
    CUtensorMap q[3];          // previous RHS N^{k-2}
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity; gives up after about a second.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* b, unsigned parity) {
    for (int it = 0; it < (1 << 21); ++it)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// Orders this thread's shared-memory writes before later tensor copies into
// the same bytes.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Producer: request plane kk (periodic in z) into stage st, completing on bar.
template <typename T>
__device__ __forceinline__ void tma_issue(const MomMaps& M, unsigned char* st, uint64_t* bar, int kk, const GridP& g,
                                          int i0, int j0, bool withP, bool withQ, bool xl, bool xr) {
    using L = TmaLay<T>;
    constexpr unsigned es = L::es;
    unsigned bytes = 3u * L::RX * L::RY * es + L::MXB * L::RY;
    if (withP) bytes += L::PX * L::PY * es;
    if (withQ) bytes += 3u * L::QX * L::QY * es;
    if (xl) bytes += 3u * L::WX * L::RY * es + L::WMX * L::RY;
    if (xr) bytes += 3u * L::WX * L::RY * es + L::WMX * L::RY + (withP ? L::WX * L::PY * es : 0u);
    mbar_expect_tx(bar, bytes);
    const int z = kk < 0 ? kk + g.nz : (kk >= g.nz ? kk - g.nz : kk);
#pragma unroll
    for (int c = 0; c < 3; ++c) tma_load3(st + c * L::CSB, &M.u[c], i0 - 4, j0 - 1, z, bar);
    tma_load3(st + L::oM, &M.m, i0 - 16, j0 - 1, z, bar);
    if (withP) tma_load3(st + L::oP, &M.p, i0, j0, z, bar);
    if (withQ) {
#pragma unroll
        for (int c = 0; c < 3; ++c) tma_load3(st + L::oQ + c * L::QCSB, &M.q[c], i0, j0, z, bar);
    }
    if (xl) {
#pragma unroll
        for (int c = 0; c < 3; ++c) tma_load3(st + L::oWL + c * L::WCSB, &M.uw[c], g.nx - L::WX, j0 - 1, z, bar);
        tma_load3(st + L::oWML, &M.mw, g.nx - L::WMX, j0 - 1, z, bar);
    }
    if (xr) {
#pragma unroll
        for (int c = 0; c < 3; ++c) tma_load3(st + L::oWR + c * L::WCSB, &M.uw[c], 0, j0 - 1, z, bar);
        tma_load3(st + L::oWMR, &M.mw, 0, j0 - 1, z, bar);
        if (withP) tma_load3(st + L::oWPR, &M.pw, 0, j0, z, bar);
    }
}

// A point of the u, v, w tile that one thread rewrites into operator form:
// destination d (element offset of component 0 in the stage), source so with
// component stride cs (the box itself, or a wrap box), mask byte at mo.
template <typename T>
struct TmaPt {
    int d, so, cs, mo;
    bool ghost;      // beyond a y wall: v reads 0, u and w read f * (adjacent)
    T f;
    int xk;          // inflow/outflow x: 1 beyond the inflow face, 2 beyond the outflow face
    bool outc;       // the u point is the outflow face (readable where the face is fluid)
};

template <typename T, bool XP>
__device__ __forceinline__ TmaPt<T> tma_point(const GridP& g, int i0, int j0, int rx, int ry, T sig_lo, T sig_hi) {
    using L = TmaLay<T>;
    TmaPt<T> q;
    q.d = ry * L::RX + rx;
    const int j = j0 - 1 + ry;
    const int jc = min(max(j, 0), g.ny - 1);
    const int sry = jc - (j0 - 1);
    q.ghost = j != jc;
    q.f = j < 0 ? sig_lo : (j >= g.ny ? sig_hi : T(1));
    const int i = i0 - 4 + rx;
    q.xk = 0;
    q.outc = false;
    if (!XP) {                        // ghost columns repeat the first or last grid column
        const int ic = i < 0 ? 0 : (i >= g.nx ? g.nx - 1 : i);
        q.xk = i < 0 ? 1 : (i >= g.nx ? 2 : 0);
        q.outc = i == g.nx - 1;
        q.so = sry * L::RX + ic - i0 + 4;
        q.cs = L::CS;
        q.mo = L::oM + sry * L::MXB + ic - i0 + 16;
    } else if (i < 0) {               // x = -1: the last column, from the left wrap box
        q.so = L::oWL / L::es + sry * L::WX + L::WX - 1;
        q.cs = L::WCSB / L::es;
        q.mo = L::oWML + sry * L::WMX + L::WMX - 1;
    } else if (i >= g.nx) {           // x = nx (the first column past the grid): column 0
        q.so = L::oWR / L::es + sry * L::WX;
        q.cs = L::WCSB / L::es;
        q.mo = L::oWMR + sry * L::WMX;
    } else {
        q.so = sry * L::RX + rx;
        q.cs = L::CS;
        q.mo = L::oM + sry * L::MXB + rx + 12;
    }
    return q;
}

// Rewrites one point in place; returns its mask byte and its three values.
// A ghost column may read a grid column that its own thread rewrites at the
// same time: the rule below re-applies that column's mask, so the raw and the
// rewritten value give the same result.
template <typename T, bool GEN, bool XP>
__device__ __forceinline__ uint32_t tma_mask_pt(unsigned char* st, const TmaPt<T>& q, T uin, T (&out)[3]) {
    using L = TmaLay<T>;
    T* f = reinterpret_cast<T*>(st);
    const uint32_t m = st[q.mo];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T x = GEN ? f[q.so + c * q.cs] : f[q.d + c * L::CS];
        bool rd = (m >> c) & 1u;
        if (!XP && GEN && c == 0 && q.outc) rd = (m & IBM_MASK_FACE) != 0;
        x = rd ? x : T(0);
        if (!XP && GEN && q.xk == 1) x = (c == 0) ? ((m & IBM_MASK_FACE) ? uin : T(0)) : -x;
        else if (!XP && GEN && q.xk == 2) x = (c == 0) ? T(0) : x;
        if (GEN && q.ghost) x = (c == 1) ? T(0) : q.f * x;
        f[q.d + c * L::CS] = x;
        out[c] = x;
    }
    return m;
}

// The operator-form pass over one stage: this thread's cells A and B (fast
// path unless the block is ragged), its halo point, and the wrapped +x
// pressure column of the block that reaches nx.  Returns A | B << 8.
template <typename T, bool XP>
__device__ __forceinline__ uint32_t tma_pass(unsigned char* st, const TmaPt<T>& qa, const TmaPt<T>& qb,
                                             const TmaPt<T>& qh, bool own_gen, bool has_h, int pfix_row,
                                             int pfix_col, T uin, T (&ua)[3], T (&ub)[3]) {
    using L = TmaLay<T>;
    uint32_t ma, mb;
    if (own_gen) {
        ma = tma_mask_pt<T, true, XP>(st, qa, uin, ua);
        mb = tma_mask_pt<T, true, XP>(st, qb, uin, ub);
    } else {
        ma = tma_mask_pt<T, false, XP>(st, qa, uin, ua);
        mb = tma_mask_pt<T, false, XP>(st, qb, uin, ub);
    }
    if (has_h) {
        T uh[3];
        tma_mask_pt<T, true, XP>(st, qh, uin, uh);
    }
    if (pfix_row >= 0) {
        T* P = reinterpret_cast<T*>(st + L::oP);
        const T* W = reinterpret_cast<const T*>(st + L::oWPR);
        P[pfix_row * L::PX + pfix_col] = W[pfix_row * L::WX];
    }
    return ma | (mb << 8);
}

// XP: periodic x (wrap boxes) or inflow/outflow x (ghost columns from the box)
template <typename T, bool XP>
__global__ void __launch_bounds__(MX * MW, sizeof(T) == 4 ? 3 : 1)
    k_momentum_tma(GridP g, MomF<T> F, StageP<T> sp, IbmStage<T> ib, double* __restrict__ flux_part,
                   double* __restrict__ status, const __grid_constant__ MomMaps maps) {
    using L = TmaLay<T>;
    extern __shared__ unsigned char dyn_smem[];
    __shared__ double shd[MW];
    unsigned char* ring = dyn_smem + ((128u - (smem_addr(dyn_smem) & 127u)) & 127u);
    uint64_t* full = reinterpret_cast<uint64_t*>(ring + L::D * L::SB);
    const int tx = threadIdx.x, w = threadIdx.y, tid = tx + MX * w;
    const int i0 = blockIdx.x * MX, j0 = blockIdx.y * MY;
    const int i = i0 + tx, jA = j0 + 2 * w;
    const bool liveA = i < g.nx && jA < g.ny;
    const bool liveB = i < g.nx && jA + 1 < g.ny;
    const uint32_t live_bits = (liveA ? 0xffu : 0u) | (liveB ? 0xff00u : 0u);
    const int plane = g.nx * g.ny;
    const int rowA = i + g.nx * jA;
    const int segrow = jA * g.nsegx + blockIdx.x;
    // wrap boxes only for a periodic x; an inflow/outflow x rewrites the block holding the
    // outflow column in the general form
    const bool xl = XP && i0 == 0, xr = XP && i0 + MX >= g.nx;
    const bool own_gen = i0 + MX > g.nx || j0 + MY > g.ny || (!XP && i0 + MX >= g.nx);
    const bool outcol = !XP && i == g.nx - 1;
    const int kbeg = blockIdx.z * g.kzm;
    const int kend = min(kbeg + g.kzm, g.nz);
    const int nrel = kend - kbeg + 2;          // planes kbeg-1 .. kend

    // this thread's points in the u, v, w tile (raw x = i - i0 + 4, raw y = j - j0 + 1)
    const TmaPt<T> qa = tma_point<T, XP>(g, i0, j0, tx + 4, 2 * w + 1, sp.sig_lo, sp.sig_hi);
    const TmaPt<T> qb = tma_point<T, XP>(g, i0, j0, tx + 4, 2 * w + 2, sp.sig_lo, sp.sig_hi);
    bool has_h = false;
    TmaPt<T> qh = qa;
    if (w == 0 || w == 1) {
        has_h = true;
        qh = tma_point<T, XP>(g, i0, j0, tx + 4, w == 0 ? 0 : L::RY - 1, sp.sig_lo, sp.sig_hi);
    } else if ((w == 2 || w == 3) && tx < L::RY) {
        has_h = true;
        qh = tma_point<T, XP>(g, i0, j0, w == 2 ? 3 : 4 + MX, tx, sp.sig_lo, sp.sig_hi);
    }
    // the block that reaches nx copies p(x = 0) next to its last column
    const int pfix_row = (xr && w == 4 && tx < L::PY) ? tx : -1;
    const int pfix_col = min(g.nx - i0, L::PX - 1);
    // pressure offsets in the p box; rows past the grid fall back to the cell itself
    const int pa = 2 * w * L::PX + tx;
    const int pb = (jA + 1 < g.ny) ? pa + L::PX : pa;
    const int pnb = (jA + 2 < g.ny) ? pb + L::PX : pb;
    const int qoa = 2 * w * L::QX + tx, qob = qoa + L::QX;
    const int ta = (2 * w + 1) * L::RX + tx + 4, tb = ta + L::RX;

    if (tid == 0) {
        for (int s = 0; s < L::D; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int rel_issued = -1;                       // producer only
    auto issue = [&](int rel) {
        const int kk = kbeg - 1 + rel;
        tma_issue<T>(maps, ring + (rel % L::D) * L::SB, &full[rel % L::D], kk, g, i0, j0, kk >= kbeg,
                     sp.read_prev && kk >= kbeg && kk < kend, xl, xr);
        rel_issued = rel;
    };
    if (tid == 0)
        for (int rel = 0; rel < L::D && rel < nrel; ++rel) issue(rel);
    auto stage = [&](int rel) { return ring + (rel % L::D) * L::SB; };
    auto abort_block = [&](int rel_from) {
        if (tid == 0) {
            status[3] = 1.0;                   // read back by ibm_diagnostics as a timeout
            for (int r = rel_from; r <= rel_issued; ++r) mbar_wait_bounded(&full[r % L::D], (r / L::D) & 1);
        }
    };

    // prologue: planes kbeg-1 (rel 0) and kbeg (rel 1)
    T ua[3], ub[3];
    bool ok = mbar_wait_bounded(&full[0], 0);
    if (ok) tma_pass<T, XP>(stage(0), qa, qb, qh, own_gen, has_h, -1, 0, sp.uin, ua, ub);
    ok = ok && mbar_wait_bounded(&full[1], 0);
    uint32_t mc = 0;
    if (ok) mc = tma_pass<T, XP>(stage(1), qa, qb, qh, own_gen, has_h, pfix_row, pfix_col, sp.uin, ua, ub) & live_bits;
    fence_proxy_async();
    if (__syncthreads_or(!ok)) {
        abort_block(0);
        return;
    }
    MomCarry<T> C;
    {
        const T* Ub = reinterpret_cast<const T*>(stage(0));
        const T* Vb = Ub + L::CS;
        const T* Wb = Ub + 2 * L::CS;
        const T* U0 = reinterpret_cast<const T*>(stage(1));
        const T* V0 = U0 + L::CS;
        const T* W0 = U0 + 2 * L::CS;
        const T* P0 = reinterpret_cast<const T*>(stage(1) + L::oP);
        const int a = ta, b = tb;
        C.ubA = Ub[a]; C.ubB = Ub[b]; C.vbA = Vb[a]; C.vbB = Vb[b]; C.wbA = Wb[a]; C.wbB = Wb[b];
        C.uA = ua[0]; C.uB = ub[0]; C.vA = ua[1]; C.vB = ub[1]; C.wA = ua[2]; C.wB = ub[2];
        C.uWA = U0[a - 1]; C.uWB = U0[b - 1]; C.vSA = V0[a - L::RX];
        C.fuA = mul_rn(Wb[a] + Wb[a + 1], Ub[a] + U0[a]);
        C.fuB = mul_rn(Wb[b] + Wb[b + 1], Ub[b] + U0[b]);
        C.fvA = mul_rn(Wb[a] + Wb[a + L::RX], Vb[a] + V0[a]);
        C.fvB = mul_rn(Wb[b] + Wb[b + L::RX], Vb[b] + V0[b]);
        C.pA = P0[pa];
        C.pB = P0[pb];
    }
    T fsum = T(0);
    MomPre<T> P;
#pragma unroll
    for (int c = 0; c < 3; ++c) P.qA[c] = P.qB[c] = T(0);

    for (int k = kbeg; k < kend; ++k) {
        const int rel = k - kbeg + 1;
        // plane k+1 into operator form
        ok = mbar_wait_bounded(&full[(rel + 1) % L::D], ((rel + 1) / L::D) & 1);
        uint32_t mn = 0;
        if (ok) mn = tma_pass<T, XP>(stage(rel + 1), qa, qb, qh, own_gen, has_h, pfix_row, pfix_col, sp.uin, ua, ub);
        fence_proxy_async();
        if (__syncthreads_or(!ok)) {
            abort_block(rel + 1);
            return;
        }
        // the stage of plane k-1 is free: request plane k+D-1 into it
        if (tid == 0 && rel + L::D - 1 < nrel) issue(rel + L::D - 1);
        const unsigned char* s0 = stage(rel);
        const unsigned char* s1 = stage(rel + 1);
        const T* Pk = reinterpret_cast<const T*>(s0 + L::oP);
        const T* Pk1 = reinterpret_cast<const T*>(s1 + L::oP);
        P.eA = Pk[pa + 1];
        P.eB = Pk[pb + 1];
        P.nB = Pk[pnb];
        P.tA = Pk1[pa];
        P.tB = Pk1[pb];
        if (sp.read_prev) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T* Q = reinterpret_cast<const T*>(s0 + L::oQ + c * L::QCSB);
                P.qA[c] = Q[qoa];
                P.qB[c] = Q[qob];
            }
        }
        const int ida = rowA + k * plane;
        mom_plane3<T, L::RX, L::CS, true, true>(g, F, sp, ib, ta, tb, reinterpret_cast<const T*>(s0),
                                          reinterpret_cast<const T*>(s1), C, P, ua, ub, mc, k, ida, ida + g.nx,
                                          liveA, liveB, segrow + k * g.ny * g.nsegx, fsum, outcol);
        mc = mn & live_bits;
    }
    if (sp.flux_sum) {
        T ws = warp_sum(fsum);
        if (tx == 0) shd[w] = (double)ws;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int q = 0; q < MW; ++q) s += shd[q];
            flux_part[blockIdx.x + gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z)] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// The implicit IBM division (Eq. rk3-rai) of the points that k_momentum_tma
// leaves undivided: one thread per entry of each component's IBM list (block
// row = component), in list order.  u* holds R there and N lacks the wall
// source; mom_ibm finishes u* with the predictor's own division arithmetic.
// The division needs a point's list position, which the predictor could find
// only by two dependent global loads (segment offset, then coefficient) in the
// warps that hold IBM points; the plane barrier then held every warp of the
// block to the slowest.  Here the position is the thread index.  With a
// constant flow rate the blocks of component u add their divided values into
// flux partials after the predictor's own.
// ---------------------------------------------------------------------------
struct IbmDivLists {
    const int* idx[3];
    int count[3];
};

// NUPD: the explicit IBM (pad = lambda) adds s - pad u to N here.  Otherwise N stays without the
// wall source s (the same at every stage), and the next stage, whose R then lacks dt b s, adds it
// back here: the division touches u and u* only (two scattered sectors a point instead of three).
template <typename T, bool NUPD>
__global__ void __launch_bounds__(256) k_ibm_division(GridP g, MomF<T> F, StageP<T> sp, IbmStage<T> ib,
                                                       IbmDivLists d, double* __restrict__ flux_part) {
    __shared__ double shd[8];
    const int c = blockIdx.y;
    // the component's arrays by branches, not by a dynamic index into the parameter arrays
    // (which would copy them to a local frame)
    auto pick = [c](auto a, auto b, auto e) { return c == 0 ? a : (c == 1 ? b : e); };
    const int n = pick(d.count[0], d.count[1], d.count[2]);
    const int* __restrict__ idx = pick(d.idx[0], d.idx[1], d.idx[2]);
    const Coef4<T>* __restrict__ coef = pick(ib.coef[0], ib.coef[1], ib.coef[2]);
    const T* __restrict__ u = pick(F.u[0], F.u[1], F.u[2]);
    T* __restrict__ us = pick(F.us[0], F.us[1], F.us[2]);
    T* __restrict__ Nn = pick(F.Nn[0], F.Nn[1], F.Nn[2]);
    T fs = T(0);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int i = idx[p];
        if (c == 0 && !g.xper && i % g.nx == g.nx - 1) continue;   // the outflow update writes u there
        const T uP = u[i];
        const Coef4<T> q = coef[p];
        T R = us[i];
        if (!NUPD && sp.read_prev) R += sp.dtb * q.s;
        T N = (NUPD && sp.write_n) ? Nn[i] : T(0);
        T out;
        mom_ibm(sp, q, uP, R, out, N);
        us[i] = out;
        if (NUPD && sp.write_n) Nn[i] = N;
        fs += out;
    }
    if (sp.flux_sum && c == 0) {   // the same branch in every thread of the block
        const T ws = warp_sum(fs);
        if ((threadIdx.x & 31) == 0) shd[threadIdx.x >> 5] = (double)ws;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += shd[q];
            flux_part[blockIdx.x] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// Host side of the TMA variant: tensor maps over the solver's own buffers
// (fixed for the handle's life), built once at setup.
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    }
    return fn;
}

// A 3D (x, y, z) map over an nx x ny x nz array of es-byte elements with box bx x by x 1.
bool encode_map(CUtensorMap* m, const void* base, CUtensorMapDataType dt, int es, const GridP& g, int bx, int by) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn || ((uintptr_t)base & 15u)) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nx * es, (cuuint64_t)g.nx * g.ny * es};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return fn(m, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T>
MomMaps* build_maps(const ibm_solver* h) {
    using L = TmaLay<T>;
    const GridP& g = h->gp;
    const CUtensorMapDataType dt = sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    MomMaps* M = new (std::nothrow) MomMaps;
    if (!M) return nullptr;
    bool ok = true;
    for (int c = 0; c < 3; ++c) {
        ok = ok && encode_map(&M->u[c], h->buf.u[c], dt, L::es, g, L::RX, L::RY);
        ok = ok && encode_map(&M->uw[c], h->buf.u[c], dt, L::es, g, L::WX, L::RY);
        ok = ok && encode_map(&M->q[c], h->Nh[c], dt, L::es, g, L::QX, L::QY);
    }
    ok = ok && encode_map(&M->m, h->mask, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, g, L::MXB, L::RY);
    ok = ok && encode_map(&M->mw, h->mask, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, g, L::WMX, L::RY);
    ok = ok && encode_map(&M->p, h->buf.p, dt, L::es, g, L::PX, L::PY);
    ok = ok && encode_map(&M->pw, h->buf.p, dt, L::es, g, L::WX, L::PY);
    if (!ok) {
        delete M;
        return nullptr;
    }
    return M;
}

// Opts the TMA kernel into its shared-memory size, once per device.
template <typename T>
bool tma_smem_ready() {
    static int state[64] = {};   // per device: 0 unknown, 1 ok, -1 refused
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    if (state[dev] == 0) {
        const bool ok = cudaFuncSetAttribute(k_momentum_tma<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             TmaLay<T>::SMEM) == cudaSuccess &&
                        cudaFuncSetAttribute(k_momentum_tma<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             TmaLay<T>::SMEM) == cudaSuccess;
        state[dev] = ok ? 1 : -1;
        cudaGetLastError();
    }
    return state[dev] == 1;
}

// The fields, stage constants and IBM coefficients of stage k of one solve.
template <typename T>
void momentum_params(ibm_solver* h, int k, MomF<T>& F, StageP<T>& sp, IbmStage<T>& ib);
template <typename T>
ibm_status launch_momentum_kernels(ibm_solver* h, const MomF<T>& F, const StageP<T>& sp, const IbmStage<T>& ib,
                                   dim3 grd, dim3 blk, int* nextra = nullptr);

template <typename T>
ibm_status launch_momentum(ibm_solver* h, int k, StageP<T>& sp, IbmStage<T>& ib, dim3& grd, int* nextra) {
    const GridP& g = h->gp;
    MomF<T> F;
    momentum_params<T>(h, k, F, sp, ib);
    dim3 blk(MX, MW, 1);
    grd = momentum_grid(g);
    return launch_momentum_kernels<T>(h, F, sp, ib, grd, blk, nextra);
}

template <typename T>
void momentum_params(ibm_solver* h, int k, MomF<T>& F, StageP<T>& sp, IbmStage<T>& ib) {
    const GridP& g = h->gp;
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
    {   // the body force at the stage's own time (time-periodic forcing, Sec. 2.5)
        const double tk = ((double)h->steps + RK_T[k]) * dt;
        const double sk = h->phys.g_freq != 0.0 ? std::sin(2.0 * M_PI * h->phys.g_freq * tk) : 0.0;
        for (int c = 0; c < 3; ++c) sp.g[c] = (T)(h->phys.g[c] + h->phys.g_amp[c] * sk);
    }
    sp.idx = (T)(1.0 / g.dx); sp.idy = (T)(1.0 / g.dy); sp.idz = (T)(1.0 / g.dz);
    sp.nx2 = (T)(h->phys.nu / (g.dx * g.dx)); sp.ny2 = (T)(h->phys.nu / (g.dy * g.dy));
    sp.nz2 = (T)(h->phys.nu / (g.dz * g.dz));
    sp.qx = (T)(0.25 / g.dx); sp.qy = (T)(0.25 / g.dy); sp.qz = (T)(0.25 / g.dz);
    sp.cgx = (T)(dt * RK_C[k] / g.dx); sp.cgy = (T)(dt * RK_C[k] / g.dy); sp.cgz = (T)(dt * RK_C[k] / g.dz);
    sp.lc = (T)(2.0 * h->phys.nu * (1.0 / (g.dx * g.dx) + 1.0 / (g.dy * g.dy) + 1.0 / (g.dz * g.dz)));
    sp.uin = (T)g.uin;
    sp.sig_lo = (T)g.sig_lo;
    sp.sig_hi = (T)g.sig_hi;
    sp.read_prev = k > 0;
    sp.write_n = k < 2;
    sp.flux_sum = h->phys.flow_mode == IBM_FLOW_CONST_FLUX;
    ib = stage_coefs<T>(h, k);
}

// nextra: flux partials written after the predictor's own (the IBM division's)
template <typename T>
ibm_status launch_momentum_kernels(ibm_solver* h, const MomF<T>& F, const StageP<T>& sp, const IbmStage<T>& ib,
                                   dim3 grd, dim3 blk, int* nextra) {
    if (nextra) *nextra = 0;
    const GridP& g = h->gp;
    if (g.ystr || h->body.kind != 0) {
        const BodyP& bd = h->body;
        if (g.ystr) {   // (a moving body needs a uniform y)
            if (g.ndim == 3) k_momentum_gen<T, true, true, false><<<grd, blk, 0, h->stream>>>(g, F, sp, ib, bd, h->partials);
            else k_momentum_gen<T, false, true, false><<<grd, blk, 0, h->stream>>>(g, F, sp, ib, bd, h->partials);
        } else {
            if (g.ndim == 3) k_momentum_gen<T, true, false, true><<<grd, blk, 0, h->stream>>>(g, F, sp, ib, bd, h->partials);
            else k_momentum_gen<T, false, false, true><<<grd, blk, 0, h->stream>>>(g, F, sp, ib, bd, h->partials);
        }
    }
    else if (g.ndim == 3 && h->mom_maps && h->mom_tma && tma_smem_ready<T>()) {
        const MomMaps& maps = *static_cast<const MomMaps*>(h->mom_maps);
        if (g.xper)
            k_momentum_tma<T, true><<<grd, blk, TmaLay<T>::SMEM, h->stream>>>(g, F, sp, ib, h->partials, h->scal, maps);
        else
            k_momentum_tma<T, false><<<grd, blk, TmaLay<T>::SMEM, h->stream>>>(g, F, sp, ib, h->partials, h->scal,
                                                                               maps);
        IBM_LAUNCH_CHECK();
        IbmDivLists d;
        int most = 0;
        for (int c = 0; c < 3; ++c) {
            d.idx[c] = h->idx[c];
            d.count[c] = c < g.ncomp ? h->counts[c] : 0;
            most = std::max(most, d.count[c]);
        }
        if (most > 0) {
            const int gx = std::min(IBM_DIV_PARTS, (most + 255) / 256);
            if ((long long)grd.x * grd.y * grd.z + gx > h->npartials)
                return ibm_set_error(IBM_E_INVALID, "flux partials buffer too small for the IBM division");
            cudaEvent_t t;
            timer_begin(h, "ibm_division", &t);   // (inside the "momentum" interval)
            if (h->phys.bmode == IBM_B_EXPLICIT)
                k_ibm_division<T, true><<<dim3(gx, g.ncomp), 256, 0, h->stream>>>(
                    g, F, sp, ib, d, h->partials + (size_t)grd.x * grd.y * grd.z);
            else
                k_ibm_division<T, false><<<dim3(gx, g.ncomp), 256, 0, h->stream>>>(
                    g, F, sp, ib, d, h->partials + (size_t)grd.x * grd.y * grd.z);
            IBM_LAUNCH_CHECK();
            timer_end(h, t, "ibm_division");
            if (nextra && sp.flux_sum) *nextra = gx;
        }
        return IBM_OK;
    }
    else if (g.ndim == 3) k_momentum<T, true><<<grd, blk, 0, h->stream>>>(g, F, sp, ib, h->partials);
    else k_momentum<T, false><<<grd, blk, 0, h->stream>>>(g, F, sp, ib, h->partials);
    IBM_LAUNCH_CHECK();
    return IBM_OK;
}

// The momentum predictors of stage k of several solves of one precision in one persistent
// launch (k_momentum_jobs); the job table goes by value with the launch.
template <typename T>
ibm_status launch_momentum_jobs(ibm_solver* const* hs, int n, int k, cudaStream_t stream) {
    MomJobs<T> J;
    J.njobs = n;
    int tiles = 0;
    for (int q = 0; q < n; ++q) {
        ibm_solver* h = hs[q];
        MomJob<T>& j = J.job[q];
        j.g = h->gp;
        IbmStage<T> ib;
        momentum_params<T>(h, k, j.F, j.sp, ib);
        j.ib = ib;
        j.part = h->partials;
        const dim3 d = momentum_grid(h->gp);
        j.nbx = (int)d.x;
        j.nby = (int)d.y;
        j.nbz = (int)d.z;
        J.tile0[q] = tiles;
        tiles += (int)(d.x * d.y * d.z);
    }
    J.ntiles = tiles;
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_momentum_jobs<T>, MX * MW, 0) != cudaSuccess || per < 1)
        return ibm_set_error(IBM_E_CUDA, "momentum jobs: device attributes");
    const int blocks = std::max(1, std::min(tiles, sms * per));
    k_momentum_jobs<T><<<blocks, dim3(MX, MW, 1), 0, stream>>>(J);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ibm_set_error(IBM_E_CUDA, std::string("momentum jobs: ") + cudaGetErrorString(e));
    for (int q = 0; q < n; ++q) hs[q]->launches += 1;
    return IBM_OK;
}

}  // namespace

ibm_status momentum_jobs_launch(ibm_solver* const* hs, int n, int k, cudaStream_t stream) {
    if (n <= 0) return IBM_OK;
    if (n > MOM_MAX_JOBS) return ibm_set_error(IBM_E_INVALID, "too many momentum jobs in one launch");
    return hs[0]->prec == IBM_FP64 ? launch_momentum_jobs<double>(hs, n, k, stream)
                                   : launch_momentum_jobs<float>(hs, n, k, stream);
}

void momentum_release(ibm_solver* h) {
    delete static_cast<MomMaps*>(h->mom_maps);
    h->mom_maps = nullptr;
}

void momentum_prepare(ibm_solver* h) {
    momentum_release(h);
    // the TMA form covers 3D grids whose x extent is a multiple of 16 (a uniform y)
    if (h->gp.ndim != 3 || h->gp.nx % 16 != 0 || h->gp.ystr) return;
    h->mom_maps = h->prec == IBM_FP64 ? static_cast<void*>(build_maps<double>(h))
                                      : static_cast<void*>(build_maps<float>(h));
}

bool momentum_uses_tma(const ibm_solver* h) {
    if (h->gp.ndim != 3 || !h->mom_maps || !h->mom_tma) return false;
    return h->prec == IBM_FP64 ? tma_smem_ready<double>() : tma_smem_ready<float>();
}

ibm_status momentum_launch(ibm_solver* h, int k, int* nparts) {
    StageP<float> spf;
    StageP<double> spd;
    IbmStage<float> ibf;
    IbmStage<double> ibd;
    dim3 grd;
    int nextra = 0;
    ibm_status st = h->prec == IBM_FP64 ? launch_momentum<double>(h, k, spd, ibd, grd, &nextra)
                                        : launch_momentum<float>(h, k, spf, ibf, grd, &nextra);
    if (nparts) *nparts = (int)(grd.x * grd.y * grd.z) + nextra;
    return st;
}

// Default z-chunk of the momentum predictor.  Per choice: the last wave's
// fill (waves / whole waves) and the share of planes a block loads only for
// its stencil (two per chunk).  Choices with at least four waves are
// preferred: with fewer, one slow SM or a half-empty last wave shows.  Chunks
// longer than 16 planes are not taken: the planes the resident blocks stream
// then outgrow L2 and the halo rows and planes come from DRAM a second time
// (measured on 512 x 384 x 256: 0.594 ms per launch at 32 planes, 0.558 at 16;
// 384 x 256 x 256: 0.308 at 32, 0.275 at 16).
int momentum_default_kzm(const GridP& g, int prec, bool tma) {
    if (g.ndim != 3) return KZM_CHOICES[0];
    int dev = 0, sms = 0, per = 0;
    const int threads = MOM_TX * MOM_WARPS;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 0;
    cudaError_t e;
    if (tma)
        e = prec == IBM_FP64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_momentum_tma<double, true>, threads,
                                                                            TmaLay<double>::SMEM)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_momentum_tma<float, true>, threads,
                                                                            TmaLay<float>::SMEM);
    else
        e = prec == IBM_FP64
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
            if (kz > 16) continue;
            const double waves = cols * ((g.nz + kz - 1) / kz) / slots;
            if (pass == 0 && waves < 4.0) continue;
            const double len = std::min(kz, g.nz);
            const double cost = std::ceil(waves) / waves * (len + 2.0) / len;
            if (cost < best) { best = cost; pick = kz; }
        }
    return pick;
}
