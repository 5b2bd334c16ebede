"""Interpolation between Monte Carlo interface nodes (Sec. 5) on the GPU,
through the C ABI, against the FP64 interpolation oracle.

Both sides compute in FP64 and differ only in rounding order (a Thomas
sweep per spline column on the GPU, a dense solve in the oracle), so values
agree to 1e-12 of the largest knot value and standard errors to 1e-12
relative.  The end-to-end call is checked without handing any GPU result to
the oracle: its knots against sdd_interface_values on the whole polyline
(same node ids), its other nodes against sdd_interpolate of those knots,
and the whole of it against the oracle's own walks and interpolation within
4 combined standard errors + 1e-4.
"""
import numpy as np
import pytest

from oracle import interp as OI
from oracle import oracle as O
from paper_1603_09311_gb300 import build as B
from paper_1603_09311_gb300 import inputs as I
from paper_1603_09311_gb300 import sdd

pytestmark = pytest.mark.gpu

KINDS = [sdd.SDD_INTERP_LINEAR, sdd.SDD_INTERP_SPLINE]


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    sdd.lib()


def _close(got, want, scale):
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * scale)


def _knots(rng, n):
    h = rng.uniform(0.1, 1.9, n - 1)
    return np.concatenate([[0.0], np.cumsum(h)]) * (3.0 / h.sum())


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("nk,V,nt", [(2, 1, 5), (3, 2, 33), (17, 4, 129), (300, 64, 1000),
                                     (1025, 2, 257)])
def test_interpolate_matches_oracle(kind, nk, V, nt):
    rng = np.random.default_rng(1000 * nk + V + kind)
    s = _knots(rng, nk)
    v = rng.normal(size=(nk, V)) * 2.0
    e = rng.uniform(0.01, 0.5, (nk, V))
    # random targets, every knot, both ends and the midpoints
    t = np.concatenate([rng.uniform(s[0], s[-1], nt), s, 0.5 * (s[1:] + s[:-1])])
    gv, ge = sdd.sdd_interpolate(s, v, e, t, kind)
    ov, oe = OI.interpolate(s, v, e, t, kind)
    _close(gv, ov, np.abs(v).max())
    np.testing.assert_allclose(ge, oe, rtol=1e-12, atol=1e-15)
    # a target on a knot gets the knot's value and standard error exactly
    gk, gke = sdd.sdd_interpolate(s, v, e, s, kind)
    np.testing.assert_array_equal(gk, v)
    np.testing.assert_allclose(gke, e, rtol=1e-15, atol=0)


def test_spline_at_the_knot_limit():
    rng = np.random.default_rng(5)
    nk = sdd.SDD_INTERP_MAX_SPLINE_KNOTS
    s = _knots(rng, nk)
    v = rng.normal(size=(nk, 2))
    e = rng.uniform(0.01, 0.5, (nk, 2))
    t = rng.uniform(s[0], s[-1], 300)
    gv, ge = sdd.sdd_interpolate(s, v, e, t, sdd.SDD_INTERP_SPLINE)
    ov, oe = OI.interpolate(s, v, e, t, OI.SPLINE)
    _close(gv, ov, np.abs(v).max())
    np.testing.assert_allclose(ge, oe, rtol=1e-12, atol=1e-15)


def test_interpolate_without_standard_errors():
    rng = np.random.default_rng(6)
    s = _knots(rng, 9)
    v = rng.normal(size=(9, 3))
    t = rng.uniform(s[0], s[-1], 50)
    gv, ge = sdd.sdd_interpolate(s, v, None, t, sdd.SDD_INTERP_SPLINE)
    assert ge is None
    _close(gv, OI.interpolate(s, v, np.zeros_like(v), t, OI.SPLINE)[0], np.abs(v).max())


def _interp_of_knots(nodes, k, m, se, kind):
    """sdd_interpolate of the GPU's knot values at every node (arc lengths of
    the test's polyline)."""
    s = OI.arc_length(nodes)
    E = m.shape[1]
    kv = np.stack([m[k].real, m[k].imag], axis=-1).reshape(len(k), -1)
    gv, ge = sdd.sdd_interpolate(s[k], kv, se[k].reshape(len(k), -1), s, kind)
    gv = gv.reshape(len(nodes), E, 2)
    return gv[..., 0] + 1j * gv[..., 1], ge.reshape(len(nodes), E, 2)


def _line(n):
    # a bent interface polyline inside the quarter-space model: down x = 0,
    # then along a slanted segment
    a = np.stack([np.zeros(n // 2), np.linspace(0.02, 0.6, n // 2)], axis=1)
    b = np.stack([np.linspace(0.02, 0.5, n - n // 2), np.linspace(0.62, 0.85, n - n // 2)], axis=1)
    return np.concatenate([a, b])


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n,stride", [(2, 1), (7, 3), (41, 4), (64, 1), (65, 8)])
def test_interface_interp_end_to_end(kind, n, stride):
    w = I.workload("quarterspace")
    nodes = _line(n)
    ctx = sdd.sdd_create(w["model"])
    try:
        paths, dt, seed = 4000, 1e-3, 21
        m, se, st = sdd.sdd_interface_values_interp(ctx, nodes, stride, paths, kind, dt, seed)
        k = OI.knot_indices(n, stride)
        assert st["walks"] == len(k) * paths
        full, fse, _ = sdd.sdd_interface_values(ctx, nodes, paths, dt, seed,
                                                node_ids=np.arange(n, dtype=np.uint32))
        # knots: the estimates of a call on the whole polyline, up to the FP64
        # summation order of the walks' samples
        np.testing.assert_allclose(m[k], full[k], rtol=0, atol=1e-12)
        np.testing.assert_allclose(se[k], fse[k], rtol=1e-10, atol=1e-15)
        # other nodes: the standalone interpolation of those knot values
        gv, ge = _interp_of_knots(nodes, k, m, se, kind)
        np.testing.assert_allclose(m, gv, rtol=0, atol=1e-12)
        np.testing.assert_allclose(se, ge, rtol=1e-12, atol=1e-15)
    finally:
        ctx.close()


@pytest.mark.parametrize("kind,n,stride", [(sdd.SDD_INTERP_SPLINE, 41, 4), (sdd.SDD_INTERP_LINEAR, 9, 3)])
def test_interface_interp_against_the_oracle_pipeline(kind, n, stride):
    """The oracle's walks at the knots (same streams) and its interpolation,
    against the GPU call, at every node within 4 combined standard errors
    + 1e-4 (the propagated errors of both)."""
    w = I.workload("quarterspace")
    nodes = _line(n)
    paths, dt, seed = 3000, 1e-3, 24
    ctx = sdd.sdd_create(w["model"])
    try:
        m, se, _ = sdd.sdd_interface_values_interp(ctx, nodes, stride, paths, kind, dt, seed)
    finally:
        ctx.close()
    k = OI.knot_indices(n, stride)
    refs = [O.interface_values(w["model"], nodes[j], paths, dt, seed, urule=23, node_id0=int(j)) for j in k]
    kv = np.stack([np.concatenate([r["mean"] for r in refs]).real,
                   np.concatenate([r["mean"] for r in refs]).imag], axis=-1)
    kse = np.concatenate([r["se"] for r in refs])
    ov, oe = OI.interface_interp(kv, kse, nodes, stride, kind)
    tol = 4 * np.sqrt(se ** 2 + oe ** 2) + 1e-4
    assert np.all(np.abs(m.real - ov[..., 0]) <= tol[..., 0])
    assert np.all(np.abs(m.imag - ov[..., 1]) <= tol[..., 1])


def test_interface_interp_knots_against_walk_oracle():
    """The knots' Monte Carlo values agree with the FP64 oracle's walks on the
    single-precision stream within 4 combined standard errors + 1e-4."""
    w = I.workload("quarterspace")
    nodes = _line(9)
    ctx = sdd.sdd_create(w["model"])
    try:
        paths, dt, seed = 3000, 1e-3, 22
        m, se, _ = sdd.sdd_interface_values_interp(ctx, nodes, 4, paths, sdd.SDD_INTERP_SPLINE, dt, seed)
        k = OI.knot_indices(9, 4)
        refs = [O.interface_values(w["model"], nodes[j], paths, dt, seed, urule=23, node_id0=int(j))
                for j in k]
        rm = np.concatenate([r["mean"] for r in refs])
        rse = np.concatenate([r["se"] for r in refs])
        d = m[k] - rm
        tol = 4 * np.sqrt(se[k] ** 2 + rse ** 2) + 1e-4
        assert np.all(np.abs(d.real) <= tol[..., 0]) and np.all(np.abs(d.imag) <= tol[..., 1])
    finally:
        ctx.close()


def test_interface_interp_full_size():
    """The bench's configuration: the quarter-space line of 64 nodes at
    1e5 walks per Monte Carlo node, every 4th node (and the last) walked."""
    w = I.workload("quarterspace")
    nodes = w["nodes"]
    n = len(nodes)
    ctx = sdd.sdd_create(w["model"])
    try:
        k = OI.knot_indices(n, 4)
        for kind in KINDS:
            m, se, st = sdd.sdd_interface_values_interp(ctx, nodes, 4, 100_000, kind, w["dt"], w["seed"])
            assert st["walks"] == len(k) * 100_000
            gv, ge = _interp_of_knots(nodes, k, m, se, kind)
            np.testing.assert_allclose(m, gv, rtol=0, atol=1e-12)
            np.testing.assert_allclose(se, ge, rtol=1e-12, atol=1e-15)
    finally:
        ctx.close()
    # one knot recomputed by the oracle's walks under its node id
    j = int(k[len(k) // 2])
    ref = O.interface_values(w["model"], nodes[j], 100_000, w["dt"], w["seed"], urule=23, node_id0=j)
    d = m[j] - ref["mean"][0]
    tol = 4 * np.sqrt(se[j] ** 2 + ref["se"][0] ** 2) + 1e-4
    assert np.all(np.abs(d.real) <= tol[..., 0]) and np.all(np.abs(d.imag) <= tol[..., 1])


def test_interface_interp_rejects_bad_polylines():
    w = I.workload("quarterspace")
    ctx = sdd.sdd_create(w["model"])
    try:
        nodes = _line(6)
        nodes[3] = nodes[2]
        with pytest.raises(sdd.SddError) as e:
            sdd.sdd_interface_values_interp(ctx, nodes, 2, 10, 0, 1e-3, 0)
        assert e.value.status == sdd.SDD_E_ARG
        with pytest.raises(sdd.SddError) as e:
            sdd.sdd_interface_values_interp(ctx, _line(6), 0, 10, 0, 1e-3, 0)
        assert e.value.status == sdd.SDD_E_ARG
    finally:
        ctx.close()


@pytest.mark.parametrize("kind", KINDS)
def test_interface_interp_with_16_evaluations(kind):
    """The block model's 16 evaluations (32 real components per node) along
    the block's top edge and down its side."""
    w = I.workload("block")
    a = np.stack([np.linspace(-0.3, 0.2, 21), np.full(21, 0.15)], axis=1)
    b = np.stack([np.full(20, 0.25), np.linspace(0.2, 0.6, 20)], axis=1)
    nodes = np.concatenate([a, b])
    n, stride = len(nodes), 5
    ctx = sdd.sdd_create(w["model"])
    try:
        m, se, st = sdd.sdd_interface_values_interp(ctx, nodes, stride, 3000, kind, 1e-3, 23)
        k = OI.knot_indices(n, stride)
        assert m.shape == (n, 16) and st["walks"] == len(k) * 3000
        gv, ge = _interp_of_knots(nodes, k, m, se, kind)
        np.testing.assert_allclose(m, gv, rtol=0, atol=1e-12)
        np.testing.assert_allclose(se, ge, rtol=1e-12, atol=1e-15)
    finally:
        ctx.close()
