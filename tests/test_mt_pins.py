"""Pins of the apparent-resistivity oracle (secondary fields by centred
differences, Sec. 2.1 and Sec. 4.2) against closed forms.

- a uniform half-space: the centred difference of e^{-kz} is -e^{-kz}
  sinh(kh)/h exactly, so rho and phi have closed forms at every h, and tend
  to the half-space's resistivity and 45 degrees (TE), -135 degrees (TM);
- a two-layer earth: the textbook recursion of the 1D response
  c = -u/u_z (tanh form) against the exact layered field;
- the TM analytic test model of Sec. 4.1, u = (z + 1) cosh(a x), for which
  the centred difference is exact;
- the delta-method standard errors against the spread of sampled inputs.
"""
import cmath
import math

import numpy as np
import pytest

from oracle import mt as OM


def _k(kappa, d=1.0):
    k = cmath.sqrt(1j * kappa / d)
    return k if k.real > 0 else -k


@pytest.mark.parametrize("kappa,kref", [(2.0, 2.0), (20.0, 2.0), (0.5, 3.0)])
def test_te_halfspace(kappa, kref):
    k = _k(kappa)
    z0 = 0.3
    errs = []
    for h in (0.04, 0.02, 0.01):
        u = [cmath.exp(-k * (z0 + dz)) for dz in (-h, 0.0, h)]
        rho, phi, uz = OM.apparent(u[0], u[1], u[2], h, kref, OM.TE)
        w = -h / cmath.sinh(k * h)  # u / u_z exactly
        assert rho == pytest.approx(kref * abs(w) ** 2, rel=1e-12)
        assert phi == pytest.approx(cmath.phase(-1j * w), abs=1e-12)
        errs.append((abs(rho - kref / kappa), abs(phi - math.pi / 4)))
    assert rho == pytest.approx(kref / kappa, rel=1e-3)
    assert phi == pytest.approx(math.pi / 4, abs=1e-3)
    # sinh(kh)/(kh) = 1 + (kh)^2/6 + ... with (kh)^2 = i kappa h^2 imaginary:
    # the phase error is second order in h, the modulus error fourth order
    e = np.array(errs)
    assert all(14.0 < e[j, 0] / e[j + 1, 0] < 18.0 for j in range(2))
    assert all(3.6 < e[j, 1] / e[j + 1, 1] < 4.4 for j in range(2))


@pytest.mark.parametrize("kappa,d,kref", [(2.0, 1.0, 2.0), (2.0, 10.0, 2.0), (5.0, 0.25, 1.0)])
def test_tm_halfspace(kappa, d, kref):
    k = _k(kappa, d)
    z0, h = 0.4, 0.005
    u = [cmath.exp(-k * (z0 + dz)) for dz in (-h, 0.0, h)]
    rho, phi, _ = OM.apparent(u[0], u[1], u[2], h, kref, OM.TM, d_site=d)
    wz = -cmath.sinh(k * h) / h  # u_z / u exactly
    assert rho == pytest.approx(d * d * abs(wz) ** 2 / kref, rel=1e-12)
    # -> D kappa / kappa_ref = sigma_ref / sigma, and -135 degrees
    assert rho == pytest.approx(d * kappa / kref, rel=1e-4)
    assert phi == pytest.approx(-3 * math.pi / 4, abs=1e-4)


@pytest.mark.parametrize("k1,k2,thick", [(2.0, 20.0, 0.3), (20.0, 2.0, 0.1), (5.0, 0.5, 0.6)])
def test_te_two_layer_response(k1, k2, thick):
    """Layer of rate kappa1 and thickness d over a half-space of rate kappa2.
    The field in the layer is u = cosh(k1 s) + (k2/k1) sinh(k1 s), s = d - z;
    the recursion of the 1D response gives c(z) = (1/k1) (k1 c2 + tanh(k1 s))
    / (1 + k1 c2 tanh(k1 s)), c2 = 1/k2, and rho = kappa_ref |c|^2,
    phi = arg(i c)."""
    a, b = _k(k1), _k(k2)
    kref = 1.0
    for z0 in (0.02, 0.5 * thick):
        h = 1e-4

        def u(z):
            s = thick - z
            return cmath.cosh(a * s) + (b / a) * cmath.sinh(a * s)

        rho, phi, _ = OM.apparent(u(z0 - h), u(z0), u(z0 + h), h, kref, OM.TE)
        t = cmath.tanh(a * (thick - z0))
        c = (1 / a) * (a / b + t) / (1 + (a / b) * t)
        assert rho == pytest.approx(kref * abs(c) ** 2, rel=1e-6)
        assert phi == pytest.approx(cmath.phase(1j * c), abs=1e-6)


@pytest.mark.parametrize("d", [1.0, 10.0])
def test_tm_analytic_model_is_exact(d):
    """u = (z + 1) cosh(a x), linear in z: the centred difference is exact,
    u_z / u = 1 / (z0 + 1), rho = D^2 / ((z0 + 1)^2 kappa_ref), phi = 0."""
    a = cmath.sqrt(-10j / d)
    x, z0, h, kref = 0.3, 0.25, 0.1, 10.0
    u = [(z0 + dz + 1) * cmath.cosh(a * x) for dz in (-h, 0.0, h)]
    rho, phi, uz = OM.apparent(u[0], u[1], u[2], h, kref, OM.TM, d_site=d)
    assert rho == pytest.approx(d * d / ((z0 + 1) ** 2 * kref), rel=1e-13)
    assert phi == pytest.approx(0.0, abs=1e-13)
    assert uz == pytest.approx(cmath.cosh(a * x), rel=1e-13)


@pytest.mark.parametrize("mode", [OM.TE, OM.TM])
def test_standard_errors_by_sampling(mode):
    rng = np.random.default_rng(30 + mode)
    n = 200_000
    h, kref, d = 0.05, 2.0, 3.0
    k = _k(2.0)
    u = np.array([cmath.exp(-k * (0.3 + dz)) for dz in (-h, 0.0, h)])
    se = np.array([[2e-4, 3e-4], [1e-4, 2.5e-4], [3e-4, 1e-4]])
    noisy = [u[j] + rng.normal(size=n) * se[j, 0] + 1j * rng.normal(size=n) * se[j, 1] for j in range(3)]
    rho, phi, _ = OM.apparent(noisy[0], noisy[1], noisy[2], h, kref, mode, d_site=d)
    sr, sp = OM.apparent_se(u[0], u[1], u[2], se[0], se[1], se[2], h, kref, mode, d_site=d)
    # sample s.d. of 2e5 draws: within 4 / sqrt(2 n) relative, plus second-order terms
    tol = 4 / math.sqrt(2 * n) + 0.01
    assert rho.std(ddof=1) == pytest.approx(float(sr), rel=tol)
    assert phi.std(ddof=1) == pytest.approx(float(sp), rel=tol)


def test_site_points_and_strip_diffusion():
    p = OM.site_points([[0.1, 0.2], [-0.3, 0.5]], 0.05)
    np.testing.assert_allclose(p, [[0.1, 0.15], [0.1, 0.2], [0.1, 0.25],
                                   [-0.3, 0.45], [-0.3, 0.5], [-0.3, 0.55]], atol=1e-15)
    m = {"diffusion": [1.0, 10.0, 3.0], "interfaces": [0.0, 0.5]}
    assert [OM.strip_diffusion(m, x) for x in (-0.2, 0.0, 0.3, 0.5, 0.9)] == [1.0, 10.0, 10.0, 3.0, 3.0]
