"""Projection pieces: divergence, gradient and the pressure-correction Poisson solve.

Paper Sec. 2.1: after the momentum predictor the velocity is projected onto a
solenoidal field; the pressure increment solves a Poisson equation.  Sec. 3.3:
no pressure boundary condition at the body, and the continuity equation is
solved everywhere "as though there was no boundary".  Reading taken (the
"unmodified projection"): the Poisson operator is the plain D G of the full
box, with the box boundary conditions only:
  * periodic directions wrap;
  * wall directions: the wall-normal velocity is prescribed, so G phi is not
    applied on wall faces (homogeneous Neumann for phi);
  * an inflow/outflow x direction likewise: the inflow velocity and the
    (balanced) outflow velocity are prescribed, G phi is not applied on the
    outflow face, and phi is homogeneous Neumann in x.
The correction u = u* - c_k Delta t G phi is applied on every non-wall face
and p += phi in every cell.  The operator is singular (constants); the gauge
is: mean of phi over the box = 0.

Two solvers, which must agree:
  * solve_direct: the definition written out, a sparse LU of D G augmented
    with the zero-mean constraint (small grids, used as a pin);
  * solve_spectral: FFT (numpy, a library primitive) in the periodic
    directions x and z and a Thomas solve along y for every wavenumber pair,
    with the modified wavenumbers 4 sin^2(pi k/n)/Delta^2 of the 3-point
    second difference.  A Neumann x direction takes the type-II discrete
    cosine transform instead (scipy, a library primitive), whose cosines
    cos(pi k (2i+1) / 2n) diagonalise the cell-centred Neumann second
    difference with eigenvalues 4 sin^2(pi k / 2n)/Delta^2.  The (0,0) mode
    fixes phi_0 = 0, solves the rest and then removes the mean over y.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .grid import AX


def divergence(grid, vel, inflow_face=None):
    """(D u) at every cell: sum_d (u_d(idx) - u_d(idx - e_d)) / Delta_d; the -y wall face
    is 0, the -x face of an inflow/outflow box carries inflow_face (nz, ny, 1)."""
    out = np.zeros(grid.shape)
    for d in range(grid.ncomp):
        q = vel[d]
        if grid.periodic(d):
            qm = np.roll(q, 1, axis=AX[d])
        else:
            qm = np.zeros_like(q)
            if d == 0 and inflow_face is not None:
                qm[..., :1] = inflow_face
            n = grid.n[d]
            a = [slice(None)] * 3
            b = [slice(None)] * 3
            a[AX[d]] = slice(1, n)
            b[AX[d]] = slice(0, n - 1)
            qm[tuple(a)] = q[tuple(b)]
        out = out + (q - qm) / (grid.cell_heights() if (d == 1 and grid.stretched) else grid.d[d])
    return out


def gradient(grid, phi):
    """(G phi) on every non-wall face; zero on wall faces."""
    out = []
    for c in range(3):
        if c >= grid.ncomp:
            out.append(np.zeros(grid.shape))
            continue
        if grid.periodic(c):
            out.append((np.roll(phi, -1, axis=AX[c]) - phi) / grid.d[c])
        else:
            g = np.zeros(grid.shape)
            n = grid.n[c]
            a = [slice(None)] * 3
            b = [slice(None)] * 3
            a[AX[c]] = slice(1, n)
            b[AX[c]] = slice(0, n - 1)
            if c == 1 and grid.stretched:     # between the centres on either side of each face
                g[tuple(b)] = (phi[tuple(a)] - phi[tuple(b)]) / grid.face_heights()[:, :-1, :]
            else:
                g[tuple(b)] = (phi[tuple(a)] - phi[tuple(b)]) / grid.d[c]
            out.append(g)
    return out


def thomas(a, b, c, d):
    """Plain Thomas algorithm along axis 0 for many systems at once.

    a: sub-diagonal (a[0] unused), b: diagonal, c: super-diagonal (c[-1] unused),
    d: right-hand sides; a, b, c broadcast against d."""
    n = d.shape[0]
    cp = np.zeros(np.broadcast(b[0], d[0]).shape, dtype=np.float64)
    cps = []
    dps = []
    bet = b[0] * np.ones_like(cp)
    dp = d[0] / bet
    cp = c[0] / bet
    cps.append(cp)
    dps.append(dp)
    for j in range(1, n):
        bet = b[j] - a[j] * cps[-1]
        dp = (d[j] - a[j] * dps[-1]) / bet
        cp = (c[j] / bet) if j < n - 1 else np.zeros_like(bet)
        cps.append(cp)
        dps.append(dp)
    x = [None] * n
    x[n - 1] = dps[n - 1]
    for j in range(n - 2, -1, -1):
        x[j] = dps[j] - cps[j] * x[j + 1]
    return np.stack(x, axis=0)


def modified_wavenumbers(n: int, Delta: float) -> np.ndarray:
    k = np.arange(n)
    return 4.0 * np.sin(np.pi * k / n) ** 2 / Delta ** 2


def neumann_wavenumbers(n: int, Delta: float) -> np.ndarray:
    k = np.arange(n)
    return 4.0 * np.sin(np.pi * k / (2 * n)) ** 2 / Delta ** 2


def solve_spectral(grid, rhs):
    nx, ny, nz = grid.n
    dy = grid.d[1]
    if not grid.periodic(0):
        import scipy.fft as sf
        rh = np.fft.fft(sf.dct(rhs, type=2, axis=2), axis=0)      # (kz, y, kx)
        K = neumann_wavenumbers(nx, grid.d[0])[None, :]
    else:
        rh = np.fft.fft2(rhs, axes=(0, 2))                 # (kz, y, kx)
        K = modified_wavenumbers(nx, grid.d[0])[None, :]
    if grid.ndim == 3:
        K = K + modified_wavenumbers(nz, grid.d[2])[:, None]
    else:
        K = K + np.zeros((nz, 1))
    # y-systems: (phi_{j-1} - 2 phi_j + phi_{j+1})/dy^2 - K phi_j = r_j, Neumann ends
    d = np.moveaxis(rh, 1, 0)                          # (y, kz, kx)
    if grid.stretched:
        # D G along y: (phi_{j+1} - phi_j)/h_{j+1/2} - (phi_j - phi_{j-1})/h_{j-1/2}, over the
        # cell height; h the distance between the centres on either side of a face
        a = 1.0 / (grid.dyc * grid.hc[:-1])
        c = 1.0 / (grid.dyc * grid.hc[1:])
        a[0] = 0.0
        c[-1] = 0.0
        diag = -(a + c)
    else:
        inv = 1.0 / dy ** 2
        a = np.full(ny, inv)
        c = np.full(ny, inv)
        a[0] = 0.0
        c[-1] = 0.0
        diag = np.full(ny, -2.0 * inv)
        diag[0] = -inv
        diag[-1] = -inv
    b = diag[:, None, None] - K[None, :, :]
    zero = (K == 0.0)
    b_safe = np.where(zero[None], -1.0, b)            # placeholder; the zero mode is solved below
    sol = thomas(a[:, None, None], b_safe, c[:, None, None], d)
    # zero mode (kx = kz = 0): phi_0 = 0, rows 1..ny-1, then zero mean along y
    zk = np.argwhere(zero)
    for (kz, kx) in zk:
        dz = d[:, kz, kx]
        a1 = a[1:].copy()
        a1[0] = 0.0
        b1 = diag[1:].copy()
        c1 = c[1:].copy()
        x = np.zeros(ny, dtype=complex)
        x[1:] = thomas(a1, b1, c1, dz[1:])
        x -= x.mean()
        sol[:, kz, kx] = x
    ph = np.moveaxis(sol, 0, 1)
    if not grid.periodic(0):
        import scipy.fft as sf
        return sf.idct(np.real(np.fft.ifft(ph, axis=0)), type=2, axis=2)
    return np.real(np.fft.ifft2(ph, axes=(0, 2)))


def operator_matrix(grid):
    """Sparse D G on the full box (periodic x,z; Neumann y)."""
    nx, ny, nz = grid.n
    N = nx * ny * nz
    idx = np.arange(N).reshape(grid.shape)
    rows, cols, vals = [], [], []
    for d in range(grid.ncomp):
        inv = 1.0 / grid.d[d] ** 2
        ax = AX[d]
        n = grid.n[d]
        for s in (+1, -1):
            if d == 1 and grid.stretched:     # per cell: 1 / (cell height x centre distance)
                h = grid.hc[1:] if s > 0 else grid.hc[:-1]
                inv = np.broadcast_to(grid.ycol(1.0 / (grid.dyc * h)), grid.shape)
            nbr = np.roll(idx, -s, axis=ax)
            valid = np.ones(grid.shape, dtype=bool)
            if not grid.periodic(d):
                pos = np.arange(n)
                shp = [1, 1, 1]
                shp[ax] = n
                pos = pos.reshape(shp)
                valid = np.broadcast_to((pos + s >= 0) & (pos + s <= n - 1), grid.shape)
            if n == 1 and grid.periodic(d):
                continue
            r = idx[valid]
            q = nbr[valid]
            w = inv[valid] if isinstance(inv, np.ndarray) else np.full(r.size, inv)
            rows += [r, r]
            cols += [q, r]
            vals += [w, -w]
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


def solve_direct(grid, rhs):
    A = operator_matrix(grid)
    N = A.shape[0]
    e = np.ones((N, 1))
    M = sp.bmat([[A, sp.csr_matrix(e)], [sp.csr_matrix(e.T), None]], format="csc")
    b = np.concatenate([rhs.ravel(), [0.0]])
    x = spla.spsolve(M, b)
    return x[:N].reshape(grid.shape)


# ---- reading B of the projection: the masked (consistent) operator ---------------------------
#
# Sec. 3.3 says that only the internal pressure points are updated.  Read literally, the
# correction acts only on internal velocity points (the faces between two internal cells)
# and the Poisson operator is D M G, M zeroing G on every other face.  Summed over the
# internal faces f between cells a and b (b = a + e_d):
#     (D M G phi)_a += (phi_b - phi_a) / Delta_d^2,   (D M G phi)_b -= (phi_b - phi_a) / Delta_d^2.
# The unknowns are the internal (pressure) cells; the operator is singular with one constant
# per connected group of them, and the gauge is a zero mean over each group.

def masked_operator_matrix(grid, cls):
    """Sparse D M G over all cells: the 2 x 2 stencil of every internal velocity point."""
    N = grid.shape[0] * grid.shape[1] * grid.shape[2]
    idx = np.arange(N).reshape(grid.shape)
    rows, cols, vals = [], [], []
    for d in range(grid.ncomp):
        inv = 1.0 / grid.d[d] ** 2
        face = cls.internal[d]                     # internal velocity point = face between a and a + e_d
        b_idx = np.roll(idx, -1, axis=AX[d])       # never wraps at an internal face of a wall direction
        a = idx[face]
        b = b_idx[face]
        rows += [a, a, b, b]
        cols += [b, a, a, b]
        vals += [np.full(a.size, inv), np.full(a.size, -inv), np.full(a.size, inv), np.full(a.size, -inv)]
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


def solve_masked(grid, cls, rhs):
    """phi on the internal cells with D M G phi = rhs there (zero mean over each connected
    group of internal cells), zero on every other cell.  The operator is singular with one
    constant per group: phi is fixed to 0 at the first cell of each group, the rest is a
    sparse solve (conjugate gradients of scipy on the symmetric positive definite negative of
    the reduced operator, to a relative residual of 1e-14: a sparse LU fills in too much on
    3D grids), and each group is then shifted to zero mean (the right-hand side sums to zero
    over a group, so the fixed cell's equation holds as well)."""
    from scipy.sparse.csgraph import connected_components
    if grid.stretched:
        raise NotImplementedError("the masked projection on a stretched grid")
    A = masked_operator_matrix(grid, cls)
    inside = np.flatnonzero(cls.p_internal.ravel())
    Ai = A[inside][:, inside].tocsr()
    ngroups, label = connected_components(Ai != 0, directed=False)
    n = inside.size
    first = np.array([np.flatnonzero(label == q)[0] for q in range(ngroups)])
    keep = np.setdiff1d(np.arange(n), first)
    x = np.zeros(n)
    K = -Ai[keep][:, keep].tocsr()
    b = -rhs.ravel()[inside][keep]
    y, info = spla.cg(K, b, rtol=1e-14, atol=0.0, maxiter=50 * keep.size)
    if info != 0 or not np.abs(K @ y - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-300):
        raise RuntimeError("masked Poisson solve did not converge")
    x[keep] = y
    for q in range(ngroups):
        sel = label == q
        x[sel] -= x[sel].mean()
    out = np.zeros(grid.shape[0] * grid.shape[1] * grid.shape[2])
    out[inside] = x
    return out.reshape(grid.shape)
