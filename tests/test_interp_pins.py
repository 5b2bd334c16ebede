"""Pins of the interpolation oracle (interface values between Monte Carlo
nodes, Sec. 5) against library routines and the definitions of the two
interpolants.

The spline checks do not go through the oracle's equations: they fit each
segment's cubic from four of its values and test the C2 joins and the
natural end conditions directly, and they compare with scipy's natural
spline.  The standard-error rule is checked by sampling.
"""
import math

import numpy as np
import pytest

from oracle import interp as OI


def _knots(rng, n, uniform=False):
    if uniform:
        return np.linspace(0.0, 1.0, n)
    h = rng.uniform(0.2, 1.8, n - 1)
    return np.concatenate([[0.0], np.cumsum(h)]) / h.sum()


@pytest.mark.parametrize("n", [2, 3, 7, 40])
def test_linear_matches_numpy_interp(n):
    rng = np.random.default_rng(n)
    s = _knots(rng, n)
    v = rng.normal(size=(n, 3))
    t = np.concatenate([s, rng.uniform(0, 1, 50)])
    got, _ = OI.interpolate(s, v, np.ones_like(v), t, OI.LINEAR)
    for c in range(3):
        np.testing.assert_allclose(got[:, c], np.interp(t, s, v[:, c]), rtol=0, atol=1e-14)


@pytest.mark.parametrize("n,uniform", [(3, True), (5, False), (17, True), (64, False)])
def test_spline_matches_scipy_natural(n, uniform):
    interpolate = pytest.importorskip("scipy.interpolate")
    rng = np.random.default_rng(100 + n)
    s = _knots(rng, n, uniform)
    v = rng.normal(size=(n, 2))
    t = np.concatenate([s, rng.uniform(0, 1, 80)])
    got, _ = OI.interpolate(s, v, np.ones_like(v), t, OI.SPLINE)
    for c in range(2):
        ref = interpolate.CubicSpline(s, v[:, c], bc_type="natural")(t)
        np.testing.assert_allclose(got[:, c], ref, rtol=0, atol=1e-12)


def test_spline_joins_and_natural_ends():
    """Each segment is a cubic; first and second derivatives agree at every
    inner knot and the second derivative vanishes at both ends."""
    rng = np.random.default_rng(7)
    n = 9
    s = _knots(rng, n)
    v = rng.normal(size=(n, 1))
    d1 = np.zeros((n - 1, 2))
    d2 = np.zeros((n - 1, 2))
    for i in range(n - 1):
        a, b = s[i], s[i + 1]
        # four points inside the segment define its cubic exactly
        u = a + (b - a) * np.array([0.1, 0.4, 0.6, 0.9])
        y, _ = OI.interpolate(s, v, np.ones_like(v), u, OI.SPLINE)
        p = np.polyfit(u - a, y[:, 0], 3)
        # the cubic through four interior points is the segment's own: its
        # values at the knots are the knot values
        assert np.polyval(p, 0.0) == pytest.approx(v[i, 0], abs=1e-9)
        assert np.polyval(p, b - a) == pytest.approx(v[i + 1, 0], abs=1e-9)
        dp, ddp = np.polyder(p), np.polyder(p, 2)
        d1[i] = np.polyval(dp, 0.0), np.polyval(dp, b - a)
        d2[i] = np.polyval(ddp, 0.0), np.polyval(ddp, b - a)
    np.testing.assert_allclose(d1[1:, 0], d1[:-1, 1], atol=1e-7)
    np.testing.assert_allclose(d2[1:, 0], d2[:-1, 1], atol=1e-6)
    assert abs(d2[0, 0]) < 1e-6 and abs(d2[-1, 1]) < 1e-6


@pytest.mark.parametrize("kind", [OI.LINEAR, OI.SPLINE])
def test_partition_of_unity_and_linear_exactness(kind):
    rng = np.random.default_rng(11)
    s = _knots(rng, 12)
    t = rng.uniform(0, 1, 100)
    C = OI.weights(s, t, kind)
    np.testing.assert_allclose(C.sum(axis=1), 1.0, atol=1e-13)
    f = 3.0 - 2.5 * s
    np.testing.assert_allclose(C @ f, 3.0 - 2.5 * t, atol=1e-13)


@pytest.mark.parametrize("kind", [OI.LINEAR, OI.SPLINE])
def test_knots_are_reproduced(kind):
    rng = np.random.default_rng(12)
    s = _knots(rng, 10)
    C = OI.weights(s, s, kind)
    np.testing.assert_allclose(C, np.eye(10), atol=1e-15)


@pytest.mark.parametrize("kind,order", [(OI.LINEAR, 2), (OI.SPLINE, 4)])
def test_convergence_order(kind, order):
    """sin(pi s) on [0, 1] (zero second derivative at both ends, so the
    natural conditions hold): the maximum error falls as h^2 for the linear
    interpolant and h^4 for the spline."""
    t = np.linspace(0, 1, 2001)
    errs = []
    for n in (9, 17, 33):
        s = np.linspace(0, 1, n)
        y, _ = OI.interpolate(s, np.sin(math.pi * s)[:, None], np.ones((n, 1)), t, kind)
        errs.append(np.abs(y[:, 0] - np.sin(math.pi * t)).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - order) < 0.25 for r in rates), rates


@pytest.mark.parametrize("kind", [OI.LINEAR, OI.SPLINE])
def test_standard_error_by_sampling(kind):
    """Independent noisy knot values with standard errors se_j: the sample
    s.d. of the interpolated value over many draws equals the propagated se."""
    rng = np.random.default_rng(13)
    n = 8
    s = _knots(rng, n)
    se = rng.uniform(0.5, 2.0, (n, 1))
    t = np.array([0.05, 0.31, 0.5, 0.77, 0.99])
    _, want = OI.interpolate(s, np.zeros((n, 1)), se, t, kind)
    draws = 40000
    C = OI.weights(s, t, kind)
    noise = rng.normal(size=(draws, n)) * se[:, 0]
    got = (noise @ C.T).std(axis=0, ddof=1)
    # the sample s.d. of 40000 normal draws is within 4 / sqrt(2 * 40000) relative
    np.testing.assert_allclose(got, want[:, 0], rtol=4 / math.sqrt(2 * draws))


def test_arc_length_closed_forms():
    line = np.stack([np.linspace(0, 3, 7), np.linspace(0, 4, 7)], axis=1)
    np.testing.assert_allclose(OI.arc_length(line), np.linspace(0, 5, 7), atol=1e-15)
    square = np.array([[0, 0], [1, 0], [1, 1], [0, 1], [0, 0]], dtype=float)
    np.testing.assert_allclose(OI.arc_length(square), [0, 1, 2, 3, 4], atol=0)
    # inscribed polygon of a unit circle: perimeter 2 m sin(pi / m) -> 2 pi
    m = 1000
    a = np.linspace(0, 2 * math.pi, m + 1)
    circ = np.stack([np.cos(a), np.sin(a)], axis=1)
    assert OI.arc_length(circ)[-1] == pytest.approx(2 * m * math.sin(math.pi / m), rel=1e-12)


def test_knot_indices():
    assert list(OI.knot_indices(10, 3)) == [0, 3, 6, 9]
    assert list(OI.knot_indices(11, 3)) == [0, 3, 6, 9, 10]
    assert list(OI.knot_indices(2, 5)) == [0, 1]
    assert list(OI.knot_indices(5, 1)) == [0, 1, 2, 3, 4]


@pytest.mark.parametrize("kind", [OI.LINEAR, OI.SPLINE])
def test_interface_interp_keeps_knots_and_reproduces_linear_data(kind):
    """Along a bent polyline, knot values of a linear function of arc length
    give that function at every node; knots keep their own values."""
    rng = np.random.default_rng(14)
    n, stride = 23, 4
    p = np.cumsum(rng.uniform(0.01, 0.05, (n, 2)), axis=0)
    s = OI.arc_length(p)
    k = OI.knot_indices(n, stride)
    f = np.stack([1.0 + 2.0 * s, -0.5 * s], axis=1)[:, None, :]  # [n][E=1][2]
    se = rng.uniform(0.1, 0.2, f.shape)
    v, e = OI.interface_interp(f[k], se[k], p, stride, kind)
    np.testing.assert_allclose(v, f, atol=1e-13)
    np.testing.assert_array_equal(v[k], f[k])
    np.testing.assert_array_equal(e[k], se[k])
