"""Apparent resistivity and phase at measurement sites (Sec. 2.1, Sec. 4.2)
on the GPU, through the C ABI.

- The kernel's arithmetic (the standalone entry point) against the oracle
  (`oracle/mt.py`) on the same test-generated three-point values: 1e-12
  relative (both FP64); the site call equals the walks followed by that
  arithmetic.
- The whole path against closed forms: a TE half-space (the column solution
  is the exact field, so the centred difference of e^{-kz} gives rho and
  phi at any h), and the TM analytic test model (u linear in z, so the
  centred difference is exact), within 4 standard errors plus the walks'
  time-step bias carried through the formulas.
"""
import cmath
import math

import numpy as np
import pytest

import pins
from oracle import mt as OM
from oracle import oracle as O
from paper_1603_09311_gb300 import build as B
from paper_1603_09311_gb300 import inputs as I
from paper_1603_09311_gb300 import sdd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    sdd.lib()


def _halfspace3():
    # three evaluations of a half-space (air, earth): earth rates 2, 8, 0.5
    m = I.halfspace(2.0)
    m["kappa"] = np.array([[0.0, 2.0], [0.0, 8.0], [0.0, 0.5]])
    return m, np.array([2.0, 8.0, 0.5])


def _points_values(ctx, sites, h, paths, dt, seed):
    pts = OM.site_points(sites, h)
    m, se, _ = sdd.sdd_interface_values(ctx, pts, paths, dt, seed,
                                        node_ids=np.arange(len(pts), dtype=np.uint32))
    return m.reshape(-1, 3, m.shape[1]), se.reshape(-1, 3, se.shape[1], 2)


@pytest.mark.parametrize("which", ["te", "tm"])
def test_formulas_match_oracle_on_given_values(which):
    """The kernel's arithmetic on test-generated three-point values (the
    standalone entry point) against the oracle's formulas on the same values."""
    rng = np.random.default_rng(40 + (which == "tm"))
    n, E, h = 50, 3, 0.05
    base = rng.normal(size=(n, 1, E)) + 1j * rng.normal(size=(n, 1, E))
    slope = rng.normal(size=(n, 1, E)) + 1j * rng.normal(size=(n, 1, E))
    v = base + slope * h * np.array([-1.0, 0.0, 1.0])[None, :, None] \
        + 0.01 * (rng.normal(size=(n, 3, E)) + 1j * rng.normal(size=(n, 3, E)))
    se = rng.uniform(1e-4, 1e-2, (n, 3, E, 2))
    kr = rng.uniform(0.5, 20.0, E)
    d_site = rng.uniform(0.1, 10.0, n) if which == "tm" else None
    mode = OM.TE if which == "te" else OM.TM
    ds = 1.0 if d_site is None else d_site[:, None]
    r = sdd.sdd_apparent_from_values(v, se, h, kr, d_site)
    rho, phi, uz = OM.apparent(v[:, 0], v[:, 1], v[:, 2], h, kr, mode, d_site=ds)
    rse, pse = OM.apparent_se(v[:, 0], v[:, 1], v[:, 2], se[:, 0], se[:, 1], se[:, 2], h, kr, mode, d_site=ds)
    np.testing.assert_allclose(r["rho"], rho, rtol=1e-12)
    np.testing.assert_allclose(r["phase"], phi, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["rho_se"], rse, rtol=1e-11)
    np.testing.assert_allclose(r["phase_se"], pse, rtol=1e-11)
    np.testing.assert_array_equal(r["u0"], v[:, 1])
    np.testing.assert_allclose(r["uz"], uz, rtol=1e-13)


@pytest.mark.parametrize("which", ["te", "tm"])
def test_sites_equal_the_standalone_arithmetic(which):
    """sdd_apparent_resistivity is the walks at the three points (the values
    sdd_interface_values gives them under the same node ids) followed by the
    standalone arithmetic."""
    if which == "te":
        model, kr = _halfspace3()
        sites = np.array([[-0.5, 0.3], [0.0, 0.02], [0.4, 0.6], [0.9, 0.1]])
        d_site = None
    else:
        model = I.tm_analytic()
        kr = np.array([10.0])
        sites = np.array([[-0.5, 0.2], [0.3, -0.4], [0.6, 0.5], [0.0, 0.1]])
        d_site = np.array([OM.strip_diffusion(model, x) for x in sites[:, 0]])
    ctx = sdd.sdd_create(model)
    try:
        h, paths, dt, seed = 0.05, 3000, 1e-3, 31
        r = sdd.sdd_apparent_resistivity(ctx, sites, h, paths, kr, dt, seed)
        assert r["stats"]["walks"] == 3 * len(sites) * paths
        m, se = _points_values(ctx, sites, h, paths, dt, seed)
    finally:
        ctx.close()
    q = sdd.sdd_apparent_from_values(m, se, h, kr, d_site)
    for k in ("rho", "phase", "rho_se", "phase_se", "u0", "uz"):
        np.testing.assert_allclose(r[k], q[k], rtol=1e-10, atol=1e-12)


def _bias(rho, u, uz, h, dt):
    """The walks' time-step bias (at most pins.bias_bound(dt) per value)
    carried to rho: |d rho| <= 2 rho (b/|u| + b/(h |u_z|))."""
    b = pins.bias_bound(dt)
    return 2 * rho * (b / np.abs(u) + b / (h * np.abs(uz)))


def test_te_halfspace_closed_form():
    model, kap = _halfspace3()
    kr = np.full(3, 2.0)
    sites = np.array([[-0.5, 0.3], [0.0, 0.3], [0.5, 0.3]])
    h, paths, dt, seed = 0.05, 400_000, 1e-4, 32
    ctx = sdd.sdd_create(model)
    try:
        r = sdd.sdd_apparent_resistivity(ctx, sites, h, paths, kr, dt, seed)
    finally:
        ctx.close()
    k = np.sqrt(1j * kap)
    w = -h / np.sinh(k * h)  # u / u_z of e^{-kz} with the centred difference
    rho_x = np.broadcast_to(kr * np.abs(w) ** 2, r["rho"].shape)
    phi_x = np.broadcast_to(np.angle(-1j * w), r["phase"].shape)
    u = np.exp(-k * 0.3)
    tol_r = 4 * r["rho_se"] + _bias(rho_x, u, u / w, h, dt)
    assert np.all(np.abs(r["rho"] - rho_x) <= tol_r), (r["rho"], rho_x, tol_r)
    tol_p = 4 * r["phase_se"] + np.broadcast_to(_bias(1.0, u, u / w, h, dt) / 2, r["phase"].shape)
    assert np.all(np.abs(r["phase"] - phi_x) <= tol_p), (r["phase"], phi_x, tol_p)
    # the half-space's own resistivity and 45 degrees, to the centred difference's O(h^2)
    assert np.all(np.abs(phi_x - math.pi / 4) < 0.03)


def test_tm_analytic_closed_form():
    """u = (z + 1) cosh(a x): rho = D^2 / ((z0 + 1)^2 kappa_ref), phi = 0."""
    model = I.tm_analytic()
    sites = np.array([[-0.5, 0.2], [0.4, 0.0], [0.6, -0.3]])
    h, paths, dt, seed, kr = 0.1, 200_000, 1e-4, 33, 10.0
    ctx = sdd.sdd_create(model)
    try:
        r = sdd.sdd_apparent_resistivity(ctx, sites, h, paths, [kr], dt, seed)
    finally:
        ctx.close()
    D = np.array([OM.strip_diffusion(model, x) for x in sites[:, 0]])
    rho_x = (D ** 2 / ((sites[:, 1] + 1) ** 2 * kr))[:, None]
    a = np.sqrt(-10j / D)
    u = ((sites[:, 1] + 1) * np.cosh(a * sites[:, 0]))[:, None]
    uz = np.cosh(a * sites[:, 0])[:, None]
    # the TM walk's bias is up to 0.3 sqrt(dt) next to an interface
    b = 10 * pins.bias_bound(dt)
    tol_r = 4 * r["rho_se"] + 2 * rho_x * (b / np.abs(u) + b / (h * np.abs(uz)))
    assert np.all(np.abs(r["rho"] - rho_x) <= tol_r), (r["rho"], rho_x, tol_r)
    tol_p = 4 * r["phase_se"] + (b / np.abs(u) + b / (h * np.abs(uz)))
    assert np.all(np.abs(r["phase"]) <= tol_p), (r["phase"], tol_p)


def test_three_points_against_walk_oracle():
    model, kr = _halfspace3()
    sites = np.array([[0.2, 0.1]])
    h, paths, dt, seed = 0.04, 4000, 1e-3, 34
    ctx = sdd.sdd_create(model)
    try:
        r = sdd.sdd_apparent_resistivity(ctx, sites, h, paths, kr, dt, seed)
        m, se = _points_values(ctx, sites, h, paths, dt, seed)
    finally:
        ctx.close()
    ref = O.interface_values(model, OM.site_points(sites, h), paths, dt, seed, urule=23)
    d = m.reshape(3, -1) - ref["mean"]
    tol = 4 * np.sqrt(se.reshape(3, -1, 2) ** 2 + ref["se"] ** 2) + 1e-4
    assert np.all(np.abs(d.real) <= tol[..., 0]) and np.all(np.abs(d.imag) <= tol[..., 1])
    np.testing.assert_allclose(r["u0"][0], m[0, 1], atol=1e-12)
    # the oracle's whole path (its walks, then its formulas) against the
    # GPU's, within 4 combined first-order standard errors
    om, ose = ref["mean"], ref["se"]
    rho_o, phi_o, _ = OM.apparent(om[0], om[1], om[2], h, kr, OM.TE)
    rse_o, pse_o = OM.apparent_se(om[0], om[1], om[2], ose[0], ose[1], ose[2], h, kr, OM.TE)
    assert np.all(np.abs(r["rho"][0] - rho_o) <= 4 * np.hypot(r["rho_se"][0], rse_o) + 1e-6)
    assert np.all(np.abs(r["phase"][0] - phi_o) <= 4 * np.hypot(r["phase_se"][0], pse_o) + 1e-6)


def test_edge_cases():
    model, kr = _halfspace3()
    ctx = sdd.sdd_create(model)
    try:
        r = sdd.sdd_apparent_resistivity(ctx, np.zeros((0, 2)), 0.05, 10, kr, 1e-3, 0)
        assert r["rho"].shape == (0, 3) and r["stats"]["walks"] == 0
        # a point outside the domain (z0 + h beyond the bottom wall)
        with pytest.raises(sdd.SddError) as e:
            sdd.sdd_apparent_resistivity(ctx, [[0.0, 0.95]], 0.1, 10, kr, 1e-3, 0)
        assert e.value.status == sdd.SDD_E_ARG
        with pytest.raises(sdd.SddError) as e:
            sdd.sdd_apparent_resistivity(ctx, [[0.0, 0.3]], 0.0, 10, kr, 1e-3, 0)
        assert e.value.status == sdd.SDD_E_ARG
        with pytest.raises(sdd.SddError) as e:
            sdd.sdd_apparent_resistivity(ctx, [[0.0, 0.3]], 0.05, 10, [1.0, -1.0, 1.0], 1e-3, 0)
        assert e.value.status == sdd.SDD_E_ARG
        # one walk per point: the standard errors are NaN, the values finite
        r = sdd.sdd_apparent_resistivity(ctx, [[0.0, 0.3]], 0.05, 1, kr, 1e-3, 0)
        assert np.all(np.isfinite(r["rho"])) and np.all(np.isnan(r["rho_se"]))
    finally:
        ctx.close()
