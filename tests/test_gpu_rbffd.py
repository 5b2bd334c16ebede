"""RBF-FD sub-domain solve (Sec. 3.2) on the GPU, through the C ABI.

- Stencils: identical to the oracle's (integer work, ties to the lower
  index).
- Weights: both sides solve the same multiquadric systems in FP64 by
  Gaussian elimination with pivoting in different orders, and the systems
  are ill-conditioned near the flat limit (cond up to ~1e10 at eps h 0.03).
  So the GPU's weights must be backward stable (residual within 1e-12 of
  the system's scale) and agree with the oracle's to cond x 1e-14.
- Solution: against the oracle's direct solve on exact boundary data, to
  1e-8 relative (BiCGStab to 1e-12 plus the weights' conditioning); against
  exact solutions to the discretisation error.
- The whole stochastic domain decomposition: walks at the boundary nodes of
  a sub-domain of the quarter-space model, RBF-FD inside, against a
  Richardson-extrapolated finite-difference solution of the whole model.
"""
import cmath
import math

import numpy as np
import pytest

import pins
from oracle import rbffd as R
from paper_1603_09311_gb300 import build as B
from paper_1603_09311_gb300 import inputs as I
from paper_1603_09311_gb300 import sdd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    sdd.lib()


def _scattered(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, (n, 2))


NODESETS = {
    "square": lambda: I.rect_grid(0, 1, 0, 1, 17, 17)[0],
    "uneven_spacing": lambda: I.rect_grid(-1, 1, 0, 1.25, 21, 11)[0],
    "fine": lambda: I.rect_grid(0, 1, 0, 1, 33, 33)[0],
    "scattered": lambda: _scattered(700, 3),
}


@pytest.mark.parametrize("name", list(NODESETS))
@pytest.mark.parametrize("ns,eps", [(9, 1.0), (5, 2.0), (13, 0.5)])
def test_stencils_and_weights_match_oracle(name, ns, eps):
    nodes = NODESETS[name]()
    st_g, w_g = sdd.sdd_rbffd_weights(nodes, ns, eps)
    st_o, w_o = R.weights(nodes, ns, eps)
    np.testing.assert_array_equal(st_g, st_o)
    for i in range(len(nodes)):
        q = nodes[st_o[i]]
        r = np.hypot(q[:, None, 0] - q[None, :, 0], q[:, None, 1] - q[None, :, 1])
        A = R.mq(r, eps)
        b = R.mq_lap(np.hypot(q[:, 0] - nodes[i, 0], q[:, 1] - nodes[i, 1]), eps)
        scale = np.linalg.norm(A, 2) * np.linalg.norm(w_g[i]) + np.linalg.norm(b)
        assert np.linalg.norm(A @ w_g[i] - b) <= 1e-12 * scale
        cond = np.linalg.cond(A)
        assert np.linalg.norm(w_g[i] - w_o[i]) <= 1e-14 * cond * np.linalg.norm(w_o[i]) + 1e-300


def _plane_wave(kappa, theta):
    k = cmath.sqrt(1j * kappa)
    a, b = k * math.cos(theta), k * math.sin(theta)
    return lambda x, z: np.exp(a * x + b * z)


@pytest.mark.parametrize("n,kappa,theta", [(9, 2.0, 0.3), (17, 20.0, 1.1), (33, 5.0, 2.0), (3, 1.0, 0.0)])
def test_solution_matches_oracle_and_exact(n, kappa, theta):
    u_x = _plane_wave(kappa, theta)
    nodes, edge = I.rect_grid(0, 1, 0, 1, n, n)
    exact = u_x(nodes[:, 0], nodes[:, 1])
    vals = np.where(edge == 1, exact, 0.0)
    kap = np.full(len(nodes), kappa)
    ug, st = sdd.sdd_rbffd_solve(nodes, edge, vals, kap, 9, 1.0, tol=1e-12)
    uo = R.solve(nodes, edge, vals, kap, 9, 1.0)
    np.testing.assert_array_equal(ug[edge == 1], exact[edge == 1])
    assert st["unknowns"] == int((edge == 0).sum())
    assert st["rel_residual"] <= 1e-12
    assert np.abs(ug - uo).max() <= 1e-8 * np.abs(uo).max()
    if n >= 17:
        assert np.abs(ug - exact).max() < 1e-2 * np.abs(exact).max()


def _disc_nodes(seed, h=0.06):
    """A jittered grid (+-0.2 h) inside the unit disc, and Dirichlet nodes on
    its circle at spacing h."""
    rng = np.random.default_rng(seed)
    g = np.arange(-1, 1 + 1e-9, h)
    X, Z = np.meshgrid(g, g)
    p = np.stack([X.ravel(), Z.ravel()], axis=1)
    p = p + rng.uniform(-0.2 * h, 0.2 * h, p.shape)
    p = p[np.hypot(p[:, 0], p[:, 1]) < 1 - 0.7 * h]
    m = int(round(2 * math.pi / h))
    a = np.linspace(0, 2 * math.pi, m, endpoint=False)
    nodes = np.concatenate([np.stack([np.cos(a), np.sin(a)], axis=1), p])
    return nodes, np.concatenate([np.ones(m), np.zeros(len(p))]).astype(np.uint8)


def test_scattered_nodes_with_varying_kappa():
    """Jittered nodes in a disc, Dirichlet values on its circle; kappa
    varies per node (the system's diagonal)."""
    nodes, flag = _disc_nodes(9)
    vals = np.where(flag == 1, np.exp(nodes[:, 0] - 0.5j * nodes[:, 1]), 0.0)
    kap = 3.0 + nodes[:, 0]
    ug, st = sdd.sdd_rbffd_solve(nodes, flag, vals, kap, 9, 1.0, tol=1e-12)
    uo = R.solve(nodes, flag, vals, kap, 9, 1.0)
    assert np.abs(ug - uo).max() <= 1e-8 * np.abs(uo).max()


def test_badly_spread_nodes_report_a_breakdown():
    """Uniformly random nodes (some pairs 1e-3 apart) give an RBF-FD matrix
    with eigenvalues of positive real part; BiCGStab breaks down on it and
    the call says so."""
    rng = np.random.default_rng(9)
    m = 120
    a = np.linspace(0, 2 * math.pi, m, endpoint=False)
    r = np.sqrt(rng.uniform(0, 0.85 ** 2, 600))
    t = rng.uniform(0, 2 * math.pi, 600)
    nodes = np.concatenate([np.stack([np.cos(a), np.sin(a)], axis=1),
                            np.stack([r * np.cos(t), r * np.sin(t)], axis=1)])
    flag = np.concatenate([np.ones(m), np.zeros(600)]).astype(np.uint8)
    vals = np.where(flag == 1, np.exp(nodes[:, 0] - 0.5j * nodes[:, 1]), 0.0)
    u, st = sdd.sdd_rbffd_solve(nodes, flag, vals, 3.0 + nodes[:, 0], 9, 1.0, tol=1e-12,
                                allow_unconverged=True)
    assert st["status"] == sdd.SDD_E_TIMEOUT and st["rel_residual"] > 1e-12


def test_unconverged_and_bad_nodes():
    nodes, edge = I.rect_grid(0, 1, 0, 1, 17, 17)
    exact = _plane_wave(2.0, 0.5)(nodes[:, 0], nodes[:, 1])
    vals = np.where(edge == 1, exact, 0.0)
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_rbffd_solve(nodes, edge, vals, 2.0, max_iter=1, tol=1e-14)
    assert e.value.status == sdd.SDD_E_TIMEOUT
    u, st = sdd.sdd_rbffd_solve(nodes, edge, vals, 2.0, max_iter=1, tol=1e-14, allow_unconverged=True)
    assert st["iterations"] == 1 and st["rel_residual"] > 1e-14 and np.all(np.isfinite(u))
    dup = nodes.copy()
    dup[5] = dup[6]
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_rbffd_weights(dup, 9, 1.0)
    assert e.value.status == sdd.SDD_E_ARG
    # a zero right-hand side gives the zero solution without iterating
    u, st = sdd.sdd_rbffd_solve(nodes, edge, np.zeros(len(nodes)), 2.0)
    assert np.all(u == 0) and st["iterations"] == 0


def _kappa_quarter(X, Z):
    k = np.where(X < 0, 2.0, 20.0)
    k = np.where(X == 0, 11.0, k)
    k = np.where(Z < 0, 0.0, k)
    return np.where(Z == 0, k / 2, k)


def test_stochastic_domain_decomposition_of_the_quarter_space():
    """Sub-domain [0, 0.9]^2 of the quarter-space model (rate 20 inside; its
    top edge is the air-earth interface, its left edge the vertical contact):
    walks at its 144 boundary nodes, RBF-FD at the 1225 inner ones.  Against
    the finite-difference solution of the whole model, within 4 boundary
    standard errors + the walks' time-step bias + the RBF-FD discretisation
    error (measured with the reference's own boundary values) + the
    reference's error estimate."""
    w = I.workload("quarterspace")
    nodes, edge = I.rect_grid(0, 0.9, 0, 0.9, 37, 37)
    bnd = np.flatnonzero(edge == 1)
    dt, paths = 1e-4, 100_000
    ctx = sdd.sdd_create(w["model"])
    try:
        m, se, _ = sdd.sdd_interface_values(ctx, nodes[bnd], paths, dt, 51)
    finally:
        ctx.close()
    vals = np.zeros(len(nodes), dtype=complex)
    vals[bnd] = m[:, 0]
    u, st = sdd.sdd_rbffd_solve(nodes, edge, vals, np.full(len(nodes), 20.0), 9, 1.0, tol=1e-12)
    inner = np.flatnonzero(edge == 0)
    pts = [tuple(p) for p in nodes]
    ref, ref_err = pins.fd_richardson(_kappa_quarter, I.DOMAIN, 2.0, 20.0, pts)
    # discretisation error of RBF-FD on this grid, from the reference's boundary values
    u_ref_bnd = R.solve(nodes, edge, np.where(edge == 1, ref, 0.0), np.full(len(nodes), 20.0), 9, 1.0)
    disc = np.abs(u_ref_bnd[inner] - ref[inner]).max()
    se_c = np.sqrt(se[:, 0, 0] ** 2 + se[:, 0, 1] ** 2).max()
    tol = 4 * se_c + 2 * pins.bias_bound(dt) + 2 * disc + ref_err.max()
    assert np.abs(u[inner] - ref[inner]).max() <= tol, (np.abs(u[inner] - ref[inner]).max(), tol)


def test_weights_at_the_node_limit():
    """SDD_RBFFD_MAX_NODES nodes (a jittered 512 x 512 grid): the stencils
    and weights of 64 sampled nodes against the definition evaluated for
    those nodes alone (nearest nodes by a full scan, a dense solve)."""
    n_side = 512
    assert n_side * n_side == sdd.SDD_RBFFD_MAX_NODES
    rng = np.random.default_rng(17)
    nodes, _ = I.rect_grid(0, 1, 0, 1, n_side, n_side)
    h = 1.0 / (n_side - 1)
    nodes = nodes + rng.uniform(-0.2 * h, 0.2 * h, nodes.shape)
    eps = 20.0
    st_g, w_g = sdd.sdd_rbffd_weights(nodes, 9, eps)
    idx = np.arange(len(nodes))
    for i in rng.choice(len(nodes), 64, replace=False):
        dx = nodes[:, 0] - nodes[i, 0]
        dz = nodes[:, 1] - nodes[i, 1]
        want = np.lexsort((idx, dx * dx + dz * dz))[:9]
        np.testing.assert_array_equal(st_g[i], want)
        q = nodes[want]
        r = np.hypot(q[:, None, 0] - q[None, :, 0], q[:, None, 1] - q[None, :, 1])
        A = R.mq(r, eps)
        b = R.mq_lap(np.hypot(q[:, 0] - nodes[i, 0], q[:, 1] - nodes[i, 1]), eps)
        w_o = np.linalg.solve(A, b)
        scale = np.linalg.norm(A, 2) * np.linalg.norm(w_g[i]) + np.linalg.norm(b)
        assert np.linalg.norm(A @ w_g[i] - b) <= 1e-12 * scale
        assert np.linalg.norm(w_g[i] - w_o) <= 1e-14 * np.linalg.cond(A) * np.linalg.norm(w_o)
