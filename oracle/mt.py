"""Secondary fields, apparent resistivities and phases from pointwise
Monte Carlo values (FP64, numpy).

TEST INFRASTRUCTURE ONLY: the plain reference that the library's
apparent-resistivity kernel is checked against.  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this module.  It imports nothing from the CUDA library's package.

Definitions (Sec. 2.1 of arXiv:1603.09311): the secondary field of the TE
mode is H^x = -(1/(i omega mu)) dE^y/dz, that of the TM mode
E^x = (1/sigma) dH^y/dz, and
    rho_TE = |E^y / H^x|^2 / (omega mu),  phi_TE = arg(E^y / H^x),
    rho_TM = |E^x / H^y|^2 / (omega mu),  phi_TM = arg(E^x / H^y).
Sec. 4.2 computes the solution at three points near the surface of each
site and the z-derivative by the centred difference.

In the library's dimensionless form (lengths in units of L, kappa =
omega mu sigma L^2) the primary field u is E^y (TE) or H^y (TM), and with
u_z = (u(z0 + h) - u(z0 - h)) / (2 h) and a reference conductivity
sigma_ref, kappa_ref = omega mu sigma_ref L^2:
    TE  E^y / H^x = -i omega mu L u / u_z
        rho / rho_ref = kappa_ref |u / u_z|^2,   phi = arg(-i u / u_z)
    TM  (D = sigma_ref / sigma at the site, the strip's diffusion)
        E^x / H^y = D u_z / (sigma_ref L u)
        rho / rho_ref = D^2 |u_z / u|^2 / kappa_ref,   phi = arg(u_z / u)
(rho_ref = 1 / sigma_ref; the positive factors omega mu L and
D / (sigma_ref L) leave the phases unchanged).

Standard errors: the three points' estimates are independent, and so are
the real and imaginary parts of each as the library reports them, so the
first-order (delta-method) error is sqrt(sum_k (d f / d x_k)^2 se_k^2) over
the six real inputs x_k.
"""
from __future__ import annotations

import numpy as np

TE = 0
TM = 1


def centred_derivative(u_minus, u_plus, h: float):
    """u_z at the centre from the values at z0 - h and z0 + h."""
    return (np.asarray(u_plus) - np.asarray(u_minus)) / (2.0 * h)


def _w(u0, uz, mode):
    return u0 / uz if mode == TE else uz / u0


def apparent(u_minus, u0, u_plus, h: float, kappa_ref, mode: int, d_site=1.0):
    """(rho / rho_ref, phi, u_z) from the complex values at the three points."""
    u_minus, u0, u_plus = (np.asarray(a, dtype=np.complex128) for a in (u_minus, u0, u_plus))
    uz = centred_derivative(u_minus, u_plus, h)
    w = _w(u0, uz, mode)
    if mode == TE:
        rho = np.asarray(kappa_ref) * np.abs(w) ** 2
        phi = np.angle(-1j * w)
    else:
        rho = np.asarray(d_site) ** 2 * np.abs(w) ** 2 / np.asarray(kappa_ref)
        phi = np.angle(w)
    return rho, phi, uz


def apparent_se(u_minus, u0, u_plus, se_minus, se0, se_plus, h: float, kappa_ref, mode: int,
                d_site=1.0):
    """Delta-method standard errors of (rho / rho_ref, phi).

    se_* are [..., 2] (re, im).  The perturbation of w = u0 / u_z (TE) or
    u_z / u0 (TM) by a change e of one input is
        TE: e / u_z (u0),  -w e' / u_z (u_z)
        TM: -w e / u0 (u0),  e' / u0 (u_z)
    with e' = +-e / (2 h) the change of u_z (+ for u(z0 + h), - for
    u(z0 - h)); then d rho = 2 C Re(conj(w) dw) with C the factor of |w|^2,
    and d phi = Im(dw / w)."""
    u_minus, u0, u_plus = (np.asarray(a, dtype=np.complex128) for a in (u_minus, u0, u_plus))
    uz = centred_derivative(u_minus, u_plus, h)
    w = _w(u0, uz, mode)
    C = np.asarray(kappa_ref) if mode == TE else np.asarray(d_site) ** 2 / np.asarray(kappa_ref)
    var_r = np.zeros(np.shape(w))
    var_p = np.zeros(np.shape(w))
    for which, se in (("minus", se_minus), ("centre", se0), ("plus", se_plus)):
        se = np.asarray(se, dtype=np.float64)
        for comp, e in ((0, 1.0), (1, 1j)):
            if which == "centre":
                dw = e / uz if mode == TE else -w * e / u0
            else:
                de = (e if which == "plus" else -e) / (2.0 * h)
                dw = -w * de / uz if mode == TE else de / u0
            g_r = 2.0 * C * np.real(np.conj(w) * dw)
            g_p = np.imag(dw / w)
            var_r = var_r + (g_r * se[..., comp]) ** 2
            var_p = var_p + (g_p * se[..., comp]) ** 2
    return np.sqrt(var_r), np.sqrt(var_p)


def site_points(sites_xz, h: float) -> np.ndarray:
    """The three points of each site, [3 n][2]: (x, z0 - h), (x, z0), (x, z0 + h);
    site i's points run under node ids 3 i, 3 i + 1, 3 i + 2."""
    s = np.asarray(sites_xz, dtype=np.float64).reshape(-1, 2)
    out = np.repeat(s, 3, axis=0)
    out[0::3, 1] -= h
    out[2::3, 1] += h
    return out


def strip_diffusion(model: dict, x: float) -> float:
    """Diffusion of the strip holding x (TM models): strip m is
    [x_{m-1}, x_m), so x on an interface belongs to the strip on its right."""
    xs = list(model.get("interfaces", []))
    m = 0
    while m < len(xs) and x >= xs[m]:
        m += 1
    return float(model["diffusion"][m])
