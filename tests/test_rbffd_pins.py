"""Pins of the RBF-FD oracle (Sec. 3.2) against the calculus and the PDE.

- the multiquadric's Laplacian formula against a finite-difference
  Laplacian of the function itself;
- stencils on a grid: the 3 x 3 block in the interior, the nearest nodes at
  a corner; weights symmetric under the grid's reflections;
- the weights' Laplacian of smooth functions converges at second order;
- the sub-domain solution of Lap u = i kappa u converges to exact
  solutions (plane waves exp(a x + b z) with a^2 + b^2 = i kappa, and the
  TE column solution) at second order.
"""
import cmath
import math

import numpy as np
import pytest

from oracle import rbffd as R
from paper_1603_09311_gb300 import inputs as I


@pytest.mark.parametrize("eps", [0.5, 1.0, 20.0])
def test_mq_laplacian_formula(eps):
    x0, z0 = 0.3, -0.2
    h = 1e-4
    for xj, zj in [(0.0, 0.0), (0.5, 0.1), (-1.0, 2.0)]:
        f = lambda x, z: R.mq(math.hypot(x - xj, z - zj), eps)
        lap = (f(x0 + h, z0) + f(x0 - h, z0) + f(x0, z0 + h) + f(x0, z0 - h) - 4 * f(x0, z0)) / h ** 2
        assert R.mq_lap(math.hypot(x0 - xj, z0 - zj), eps) == pytest.approx(lap, rel=1e-5)


def test_stencils_on_a_grid():
    nodes, _ = I.rect_grid(0, 1, 0, 1.25, 5, 5)  # spacing 0.25 x 0.3125
    st = R.stencils(nodes, 9)
    c = 2 * 5 + 2
    block = {r * 5 + q for r in (1, 2, 3) for q in (1, 2, 3)}
    assert st[c, 0] == c and set(st[c]) == block
    # corner (0, 0): itself, (0.25, 0), (0, 0.3125), (0.25, 0.3125), (0.5, 0), (0.5, 0.3125),
    # (0, 0.625), (0.25, 0.625), (0.75, 0)
    assert list(st[0]) == [0, 1, 5, 6, 2, 7, 10, 11, 3]


def test_weights_symmetric_on_a_square_grid():
    nodes, _ = I.rect_grid(0, 1, 0, 1, 7, 7)
    st, w = R.weights(nodes, 9, 1.0)
    i = 3 * 7 + 3
    wmap = dict(zip(st[i], w[i]))
    e = [wmap[i + d] for d in (1, -1, 7, -7)]
    c = [wmap[i + d] for d in (8, -8, 6, -6)]
    assert max(e) - min(e) < 1e-6 * abs(e[0])
    assert max(c) - min(c) < 1e-6 * max(abs(c[0]), 1.0)
    # close to a consistent Laplacian (exactly so only in the flat limit
    # eps h -> 0; here eps h = 1/6): the weights sum to ~0 and the second
    # moment in x is ~2
    h = 1.0 / 6
    assert abs(sum(w[i])) < 1e-3 / h ** 2
    mx = sum(wmap[j] * (nodes[j, 0] - nodes[i, 0]) ** 2 for j in st[i])
    assert mx == pytest.approx(2.0, rel=2e-2)


def test_laplacian_of_smooth_functions_second_order():
    f = lambda x, z: np.sin(1.3 * x) * np.exp(0.7 * z)
    lap = lambda x, z: (0.49 - 1.69) * f(x, z)
    errs = []
    for n in (9, 17, 33):
        nodes, edge = I.rect_grid(0, 1, 0, 1, n, n)
        st, w = R.weights(nodes, 9, 1.0)
        fv = f(nodes[:, 0], nodes[:, 1])
        approx = (w * fv[st]).sum(axis=1)
        inner = edge == 0
        errs.append(np.abs(approx[inner] - lap(nodes[inner, 0], nodes[inner, 1])).max())
    rates = [math.log2(errs[j] / errs[j + 1]) for j in range(2)]
    assert all(r > 1.7 for r in rates), (errs, rates)


def _plane_wave(kappa, theta):
    k = cmath.sqrt(1j * kappa)
    a, b = k * math.cos(theta), k * math.sin(theta)
    return lambda x, z: np.exp(a * x + b * z)


@pytest.mark.parametrize("kappa,theta", [(2.0, 0.3), (20.0, 1.1), (5.0, math.pi / 2)])
def test_subdomain_solution_converges(kappa, theta):
    u_x = _plane_wave(kappa, theta)
    errs = []
    for n in (9, 17, 33):
        nodes, edge = I.rect_grid(0, 1, 0, 1, n, n)
        exact = u_x(nodes[:, 0], nodes[:, 1])
        u = R.solve(nodes, edge, np.where(edge == 1, exact, 0.0), np.full(len(nodes), kappa), 9, 1.0)
        np.testing.assert_array_equal(u[edge == 1], exact[edge == 1])
        errs.append(np.abs(u - exact).max() / np.abs(exact).max())
    rates = [math.log2(errs[j] / errs[j + 1]) for j in range(2)]
    assert errs[-1] < 2e-3 and all(r > 1.7 for r in rates), (errs, rates)


def test_te_column_solution_in_an_earth_block():
    """The right earth block of a half-space, [0, 1] x [0, 1], with the 1D
    column solution e^{-kz} on its edges: the solution is e^{-kz} inside."""
    kappa = 20.0
    k = cmath.sqrt(1j * kappa)
    nodes, edge = I.rect_grid(0, 1, 0, 1, 33, 33)
    exact = np.exp(-k * nodes[:, 1])
    u = R.solve(nodes, edge, np.where(edge == 1, exact, 0.0), np.full(len(nodes), kappa), 9, 1.0)
    assert np.abs(u - exact).max() < 2e-3
