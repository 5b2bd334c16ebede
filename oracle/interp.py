"""Interpolation of interface values along an interface (FP64, numpy).

TEST INFRASTRUCTURE ONLY: the plain reference that the library's
interpolation kernels are checked against.  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this module.  It imports nothing from the CUDA library's package.

Sec. 5 of arXiv:1603.09311 names a way to cut the Monte Carlo work: compute
the stochastic solution at some points along an interface only and
interpolate the remaining interface values.  The paper gives no scheme, so
the reading taken here is:

- the nodes of one interface are an ordered polyline p_0 .. p_{n-1}; the
  interpolation variable is the arc length s_i = sum_{k<i} |p_{k+1} - p_k|;
- the Monte Carlo nodes ("knots") are every stride-th node, 0, stride,
  2 stride, ..., and always the last node;
- each real component of each evaluation is interpolated on its own, either
  piecewise linearly in s or by the natural cubic spline in s (second
  derivative zero at both end knots);
- both interpolants are linear in the knot values, v(s) = sum_j c_j(s) v_j,
  and the knots' estimates are independent, so the standard error of an
  interpolated value is sqrt(sum_j c_j(s)^2 se_j^2).  It is the Monte Carlo
  part of the error only: the interpolation error itself is not in it.

Everything is written from the definitions: the weights c_j(s) are formed
explicitly as a dense matrix (one row per target), the spline's second
derivatives by a dense solve of the natural-spline equations.
"""
from __future__ import annotations

import numpy as np

LINEAR = 0
SPLINE = 1


def arc_length(nodes) -> np.ndarray:
    """Cumulative arc length s_i of the polyline through nodes [n][2]."""
    p = np.asarray(nodes, dtype=np.float64)
    s = np.zeros(len(p))
    for i in range(1, len(p)):
        s[i] = s[i - 1] + np.hypot(p[i, 0] - p[i - 1, 0], p[i, 1] - p[i - 1, 1])
    return s


def knot_indices(n: int, stride: int) -> np.ndarray:
    """Indices of the Monte Carlo nodes: 0, stride, 2 stride, ... and n - 1."""
    idx = list(range(0, n, stride))
    if idx[-1] != n - 1:
        idx.append(n - 1)
    return np.asarray(idx, dtype=np.int64)


def segment(s_knots, t: float) -> int:
    """The segment [s_i, s_{i+1}] holding t: the largest i <= n - 2 with
    s_i <= t (a target on an inner knot belongs to the segment it starts)."""
    i = 0
    while i + 2 < len(s_knots) and s_knots[i + 1] <= t:
        i += 1
    return i


def spline_moments(s_knots) -> np.ndarray:
    """Second derivatives of the natural cubic spline of every unit knot
    vector: column j holds M(e_j), so M(v) = G @ v.

    With h_i = s_{i+1} - s_i, the spline is C2 at the inner knots when
        h_{i-1} M_{i-1} + 2 (h_{i-1} + h_i) M_i + h_i M_{i+1}
            = 6 ((v_{i+1} - v_i) / h_i - (v_i - v_{i-1}) / h_{i-1}),
    i = 1 .. n - 2, and natural when M_0 = M_{n-1} = 0."""
    s = np.asarray(s_knots, dtype=np.float64)
    n = len(s)
    G = np.zeros((n, n))
    if n <= 2:
        return G
    h = np.diff(s)
    m = n - 2
    A = np.zeros((m, m))
    R = np.zeros((m, n))
    for r in range(m):
        i = r + 1
        A[r, r] = 2.0 * (h[i - 1] + h[i])
        if r > 0:
            A[r, r - 1] = h[i - 1]
        if r < m - 1:
            A[r, r + 1] = h[i]
        R[r, i - 1] += 6.0 / h[i - 1]
        R[r, i] -= 6.0 / h[i - 1] + 6.0 / h[i]
        R[r, i + 1] += 6.0 / h[i]
    G[1:n - 1, :] = np.linalg.solve(A, R)
    return G


def weights(s_knots, s_targets, kind: int) -> np.ndarray:
    """Dense weights C [n_targets][n_knots]: v(t) = C @ v_knots."""
    s = np.asarray(s_knots, dtype=np.float64)
    t_all = np.asarray(s_targets, dtype=np.float64)
    n = len(s)
    C = np.zeros((len(t_all), n))
    G = spline_moments(s) if kind == SPLINE else None
    for r, t in enumerate(t_all):
        i = segment(s, t)
        h = s[i + 1] - s[i]
        a = (s[i + 1] - t) / h
        b = (t - s[i]) / h
        C[r, i] += a
        C[r, i + 1] += b
        if kind == SPLINE:
            # S(t) = a v_i + b v_{i+1} + ((a^3 - a) M_i + (b^3 - b) M_{i+1}) h^2 / 6
            C[r, :] += (a ** 3 - a) * h * h / 6.0 * G[i, :] + (b ** 3 - b) * h * h / 6.0 * G[i + 1, :]
    return C


def interpolate(s_knots, values, se, s_targets, kind: int):
    """Interpolated values and standard errors at s_targets.

    values, se: [n_knots][V] real components (e.g. [n_knots][E][2] flattened);
    returns (values [n_targets][V], se [n_targets][V])."""
    C = weights(s_knots, s_targets, kind)
    v = np.asarray(values, dtype=np.float64).reshape(len(s_knots), -1)
    e = np.asarray(se, dtype=np.float64).reshape(len(s_knots), -1)
    return C @ v, np.sqrt((C * C) @ (e * e))


def interface_interp(values_at_knots, se_at_knots, nodes, stride: int, kind: int):
    """Values at every node of the polyline from the Monte Carlo values at
    its knots (knot_indices(n, stride)); knots keep their own estimates.

    values_at_knots, se_at_knots: [n_knots][E][2] real arrays (re, im)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    n = len(nodes)
    k = knot_indices(n, stride)
    s = arc_length(nodes)
    v = np.asarray(values_at_knots, dtype=np.float64)
    e = np.asarray(se_at_knots, dtype=np.float64)
    shape = v.shape[1:]
    vi, ei = interpolate(s[k], v.reshape(len(k), -1), e.reshape(len(k), -1), s, kind)
    vi[k] = v.reshape(len(k), -1)
    ei[k] = e.reshape(len(k), -1)
    return vi.reshape((n,) + shape), ei.reshape((n,) + shape)
