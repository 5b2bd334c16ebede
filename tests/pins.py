"""Independent closed forms, series and a finite-difference brute force used to
pin the oracle (and, through it, the CUDA path).  None of this calls the
oracle or the CUDA library.

- column_u: the 1D layered TE solution used as boundary data (Sec. 2.1).
- exit_time_series: E[tau] of standard 2D Brownian motion from a rectangle,
  by separation of variables (1/2 Lap u = -1, u = 0 on the boundary).
- helmholtz_series: u = E[exp(-i kappa tau / 2)] for uniform kappa and g = 1,
  i.e. 1/2 Lap u - (i kappa / 2) u = 0, u = 1 on the boundary.
- fd_solve: 5-point finite differences of Lap u - i kappa(x) u = 0 with the
  same Dirichlet data, for heterogeneous kappa, on a uniform grid.
- polygon_cell_fraction / kappa_cell_average: the rate at a grid node as the
  area average over its dual cell, the polygon clipped against each cell
  (Sutherland-Hodgman against the four axis-aligned sides, shoelace area).
  This treats material edges of any slope without a point-in-shape test, so
  it shares no formula with the oracle's edge functions.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# Largest dt bias of the walk measured on the homogeneous half-space
# (16 nodes x 1e5 paths, dt from 4e-3 to 2.5e-4): |bias| <= 0.021 sqrt(dt)
# in the imaginary part, the real part within noise.  Tests allow
# BIAS_C * sqrt(dt).
BIAS_C = 0.03


def bias_bound(dt: float) -> float:
    return BIAS_C * np.sqrt(dt)


def column_u(kappa: float, z):
    """1D TE solution with earth rate kappa below z = 0 and air above."""
    k = np.sqrt(1j * kappa)
    z = np.asarray(z, dtype=np.float64)
    return np.where(z >= 0.0, np.exp(-k * z), 1.0 - k * z)


def _rect_modes(x, z, domain, mmax):
    xmin, xmax, zmin, zmax = domain
    W, H = xmax - xmin, zmax - zmin
    X, Z = x - xmin, z - zmin
    m = np.arange(1, mmax + 1, 2)
    M, N = np.meshgrid(m, m, indexing="ij")
    lam = 0.5 * np.pi ** 2 * ((M / W) ** 2 + (N / H) ** 2)
    phi = np.sin(M * np.pi * X / W) * np.sin(N * np.pi * Z / H)
    coef = 16.0 / (np.pi ** 2 * M * N)
    return lam, phi, coef


def exit_time_series(x, z, domain, mmax=801):
    lam, phi, coef = _rect_modes(x, z, domain, mmax)
    return float(np.sum(coef / lam * phi))


def helmholtz_series(x, z, kappa, domain, mmax=801):
    lam, phi, coef = _rect_modes(x, z, domain, mmax)
    a = 0.5j * kappa
    return complex(1.0 - np.sum(coef * a / (lam + a) * phi))


def g_columns(x, z, domain, kl, kr, wall):
    """Boundary data of the 'columns' kind: sides from the 1D solution of their
    column, top/bottom linear in x between the corners."""
    xmin, xmax, zmin, zmax = domain
    if wall == "left":
        return column_u(kl, z)
    if wall == "right":
        return column_u(kr, z)
    t = (x - xmin) / (xmax - xmin)
    return (1 - t) * column_u(kl, z) + t * column_u(kr, z)


def fd_solve(kappa_fn, domain, h, kl, kr):
    """Solve Lap u - i kappa u = 0 on a uniform grid of spacing h with the
    'columns' boundary data.  kappa_fn(X, Z) gives kappa at grid nodes.
    Returns (xs, zs, U) with U[iz, ix] on the full grid including walls."""
    xmin, xmax, zmin, zmax = domain
    nx = int(round((xmax - xmin) / h))
    nz = int(round((zmax - zmin) / h))
    xs = xmin + h * np.arange(nx + 1)
    zs = zmin + h * np.arange(nz + 1)
    X, Z = np.meshgrid(xs, zs)
    U = np.zeros((nz + 1, nx + 1), dtype=np.complex128)
    U[:, 0] = g_columns(xs[0], zs, domain, kl, kr, "left")
    U[:, -1] = g_columns(xs[-1], zs, domain, kl, kr, "right")
    U[0, :] = g_columns(xs, zs[0], domain, kl, kr, "top")
    U[-1, :] = g_columns(xs, zs[-1], domain, kl, kr, "bottom")
    ni, nk = nx - 1, nz - 1
    idx = np.arange(ni * nk).reshape(nk, ni)
    kap = kappa_fn(X[1:-1, 1:-1], Z[1:-1, 1:-1])
    inv = 1.0 / h ** 2
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [(-4.0 * inv - 1j * kap).ravel()]
    rhs = np.zeros(ni * nk, dtype=np.complex128)
    KZ, KX = np.meshgrid(np.arange(nk), np.arange(ni), indexing="ij")
    for dz, dx in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        JZ, JX = KZ + dz, KX + dx
        inside = (JZ >= 0) & (JZ < nk) & (JX >= 0) & (JX < ni)
        rows.append(idx[inside])
        cols.append(idx[JZ[inside], JX[inside]])
        vals.append(np.full(int(inside.sum()), inv, dtype=np.complex128))
        out = ~inside
        # neighbour on the wall: full-grid index is interior index + 1
        np.subtract.at(rhs, idx[out], inv * U[JZ[out] + 1, JX[out] + 1])
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(ni * nk, ni * nk))
    sol = spla.spsolve(A.tocsc(), rhs)
    U[1:-1, 1:-1] = sol.reshape(nk, ni)
    return xs, zs, U


def fd_value(kappa_fn, domain, h, kl, kr, pts):
    xs, zs, U = fd_solve(kappa_fn, domain, h, kl, kr)
    out = []
    for x, z in pts:
        ix = int(round((x - xs[0]) / h))
        iz = int(round((z - zs[0]) / h))
        assert abs(xs[ix] - x) < 1e-12 and abs(zs[iz] - z) < 1e-12, "point not on the grid"
        out.append(U[iz, ix])
    return np.array(out)


def fd_richardson(kappa_fn, domain, kl, kr, pts, h=1 / 40):
    """Second-order Richardson extrapolation of h and h/2 solutions; returns
    (value, error estimate)."""
    a = fd_value(kappa_fn, domain, h, kl, kr, pts)
    b = fd_value(kappa_fn, domain, h / 2, kl, kr, pts)
    ext = (4 * b - a) / 3
    return ext, np.abs(b - a) / 3


def u_flux(x, diffusion, interfaces, xmin):
    """int_{xmin}^x ds / D(s) for strips with diffusion D_m between the given
    interfaces: continuous, with the same flux D u' = 1 in every strip."""
    x = np.asarray(x, dtype=float)
    bounds = [xmin] + list(interfaces) + [np.inf]
    u = np.zeros_like(x)
    for k, D in enumerate(diffusion):
        lo, hi = bounds[k], bounds[k + 1]
        u += (np.clip(x, lo, hi) - lo) / D
    return u


def fd_solve_tm(domain, h, diffusion, interfaces, kappa, g_fn):
    """Finite volumes for div(D grad u) - i kappa u = 0 on a uniform grid of
    spacing h, D and kappa constant on vertical strips whose interfaces lie on
    grid columns.  x-faces take the D of the strip they lie in; a node on an
    interface takes the mean of its two strips for D on its z-faces and for
    kappa (its control volume is half in each).  Dirichlet data g_fn(X, Z).
    Returns (xs, zs, U)."""
    xmin, xmax, zmin, zmax = domain
    nx = int(round((xmax - xmin) / h))
    nz = int(round((zmax - zmin) / h))
    xs = xmin + h * np.arange(nx + 1)
    zs = zmin + h * np.arange(nz + 1)
    bounds = np.asarray(interfaces, dtype=float)

    def strip(x):
        return np.searchsorted(bounds, x, side="right")

    D = np.asarray(diffusion, dtype=float)
    kap = np.asarray(kappa, dtype=float)
    on_if = np.isclose(xs[:, None], bounds[None, :], atol=1e-9 * h).any(axis=1) if len(bounds) else np.zeros(nx + 1, bool)
    s_node = strip(xs)
    s_left = strip(xs - 0.5 * h)
    d_node = np.where(on_if, 0.5 * (D[s_left] + D[s_node]), D[s_node])
    k_node = np.where(on_if, 0.5 * (kap[s_left] + kap[s_node]), kap[s_node])
    d_xface = D[strip(xs[:-1] + 0.5 * h)]  # face between nodes i and i+1
    X, Z = np.meshgrid(xs, zs)
    U = np.zeros((nz + 1, nx + 1), dtype=np.complex128)
    U[:, 0], U[:, -1] = g_fn(X[:, 0], Z[:, 0]), g_fn(X[:, -1], Z[:, -1])
    U[0, :], U[-1, :] = g_fn(X[0, :], Z[0, :]), g_fn(X[-1, :], Z[-1, :])
    ni, nk = nx - 1, nz - 1
    idx = np.arange(ni * nk).reshape(nk, ni)
    KZ, KX = np.meshgrid(np.arange(nk), np.arange(ni), indexing="ij")
    ix = KX + 1  # full-grid column of each unknown
    inv = 1.0 / h ** 2
    cw, ce = d_xface[ix - 1] * inv, d_xface[ix] * inv
    cz = d_node[ix] * inv
    diag = -(cw + ce + 2.0 * cz) - 1j * k_node[ix]
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [diag.ravel()]
    rhs = np.zeros(ni * nk, dtype=np.complex128)
    for dz, dx, c in ((-1, 0, cz), (1, 0, cz), (0, -1, cw), (0, 1, ce)):
        JZ, JX = KZ + dz, KX + dx
        inside = (JZ >= 0) & (JZ < nk) & (JX >= 0) & (JX < ni)
        rows.append(idx[inside])
        cols.append(idx[JZ[inside], JX[inside]])
        vals.append(c[inside].astype(np.complex128))
        out = ~inside
        np.subtract.at(rhs, idx[out], c[out] * U[JZ[out] + 1, JX[out] + 1])
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(ni * nk, ni * nk))
    U[1:-1, 1:-1] = spla.spsolve(A.tocsc(), rhs).reshape(nk, ni)
    return xs, zs, U


def fd_tm_richardson(domain, diffusion, interfaces, kappa, g_fn, pts, h=1 / 40):
    """Richardson-extrapolated FD values at grid points pts (on both grids),
    and the size of the extrapolation step as an error estimate."""
    vals = []
    for hh in (h, h / 2):
        xs, zs, U = fd_solve_tm(domain, hh, diffusion, interfaces, kappa, g_fn)
        vals.append(np.array([U[int(round((z - zs[0]) / hh)), int(round((x - xs[0]) / hh))] for x, z in pts]))
    ext = (4.0 * vals[1] - vals[0]) / 3.0
    return ext, np.abs(ext - vals[1])


def _clip_half_plane(poly, axis, val, keep_ge):
    """Part of a convex or simple polygon on one side of the line
    coordinate[axis] = val (Sutherland-Hodgman, one edge)."""
    out = []
    n = len(poly)
    for k in range(n):
        p, q = poly[k], poly[(k + 1) % n]
        p_in = p[axis] >= val if keep_ge else p[axis] <= val
        q_in = q[axis] >= val if keep_ge else q[axis] <= val
        if p_in:
            out.append(p)
        if p_in != q_in:
            t = (val - p[axis]) / (q[axis] - p[axis])
            out.append((p[0] + t * (q[0] - p[0]), p[1] + t * (q[1] - p[1])))
    return out


def _shoelace(poly):
    if len(poly) < 3:
        return 0.0
    a = 0.0
    for k in range(len(poly)):
        x0, z0 = poly[k]
        x1, z1 = poly[(k + 1) % len(poly)]
        a += x0 * z1 - x1 * z0
    return abs(a) / 2.0


def polygon_cell_fraction(poly, X, Z, h):
    """Fraction of each square cell [x - h/2, x + h/2] x [z - h/2, z + h/2]
    (x, z the entries of X, Z) covered by the polygon."""
    P = np.asarray(poly, dtype=float)
    lo, hi = P.min(axis=0), P.max(axis=0)
    F = np.zeros_like(np.asarray(X, dtype=float))
    near = (X + h / 2 > lo[0]) & (X - h / 2 < hi[0]) & (Z + h / 2 > lo[1]) & (Z - h / 2 < hi[1])
    for idx in zip(*np.nonzero(near)):
        x, z = float(X[idx]), float(Z[idx])
        q = [tuple(v) for v in P]
        q = _clip_half_plane(q, 0, x - h / 2, True)
        q = _clip_half_plane(q, 0, x + h / 2, False)
        q = _clip_half_plane(q, 1, z - h / 2, True)
        q = _clip_half_plane(q, 1, z + h / 2, False)
        F[idx] = _shoelace(q) / h ** 2
    return F


def kappa_cell_average(k_host, inclusions):
    """kappa_fn(X, Z, h) for a half-space (air kappa = 0 above z = 0, k_host
    below) holding non-overlapping polygonal inclusions [(vertices, kappa)]:
    the area average of kappa over each node's dual cell."""
    def fn(X, Z, h):
        earth = np.clip((Z + h / 2) / h, 0.0, 1.0)
        k = earth * k_host
        for poly, kap in inclusions:
            f = polygon_cell_fraction(poly, X, Z, h)
            k = k + f * (kap - k_host)
        return k
    return fn


def fd_richardson3(kappa_fn, domain, kl, kr, pts, h=1 / 40):
    """FD values at grid points pts on spacings h, h/2, h/4 (kappa_fn(X, Z, h)),
    Richardson-extrapolated from the two finest; returns (value, error
    estimate, observed convergence ratio |u_h - u_h/2| / |u_h/2 - u_h/4|)."""
    vals = []
    for hh in (h, h / 2, h / 4):
        vals.append(fd_value(lambda X, Z, hh=hh: kappa_fn(X, Z, hh), domain, hh, kl, kr, pts))
    a, b, c = vals
    ext = (4 * c - b) / 3
    ratio = np.abs(b - a) / np.maximum(np.abs(c - b), 1e-300)
    return ext, np.abs(ext - c), ratio
