"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code: published
known-answer vectors, closed forms, series solutions, a finite-difference
brute force, textbook probabilities and exact special cases.  Tolerances for
Monte Carlo results are 4 standard errors plus the measured time-step bias
(pins.bias_bound) plus, for FD, its Richardson error estimate.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import pins
from oracle import oracle as O
from paper_1603_09311_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
DOM = I.DOMAIN


def _kat():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat())
def test_philox_known_answers(ctr, key, want):
    assert list(O.philox4x32_10(ctr, key)) == want


def test_uniform_rules_open_interval():
    # (w + 1/2) 2^-32 and (w mod 2^23 + 1/2) 2^-23: never 0 or 1
    assert O.uniform(0, 32) == 2.0 ** -33
    assert O.uniform(0xFFFFFFFF, 32) == 1.0 - 2.0 ** -33
    assert O.uniform(0, 23) == 2.0 ** -24
    assert O.uniform(0xFFFFFFFF, 23) == 1.0 - 2.0 ** -24
    assert O.uniform(1, 23) == 3 * 2.0 ** -24 and O.uniform(1 << 23, 23) == 2.0 ** -24


@pytest.mark.parametrize("urule", [32, 23])
def test_box_muller_normals_are_standard(urule):
    # Sec. 3.1 draws W ~ N(0, I2); check the first four moments and a KS test
    vals = np.array([O.normals(7, node, path, n, urule)
                     for node in range(2) for path in range(50) for n in range(200)])
    n = len(vals)
    a, b = vals[:, 0], vals[:, 1]
    for v in (a, b):
        assert abs(v.mean()) < 5 / math.sqrt(n)
        assert abs(v.var() - 1) < 5 * math.sqrt(2 / n)
        assert abs(np.mean(v ** 4) - 3) < 5 * math.sqrt(96 / n)
        assert stats.kstest(v, "norm").pvalue > 1e-4
    assert abs(np.mean(a * b)) < 5 / math.sqrt(n)
    # consecutive steps of one walk use different words of the same Philox call
    w_even = O.normals(1, 0, 0, 0, urule)
    w_odd = O.normals(1, 0, 0, 1, urule)
    assert w_even != w_odd


@pytest.mark.parametrize("urule", [32, 23])
def test_bridge_uniform_stream_is_uniform(urule):
    u = np.array([O.bridge_uniform(3, 0, p, n, urule) for p in range(40) for n in range(250)])
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    assert u.min() > 0 and u.max() < 1
    # independent of the same step's normals (23: disjoint bits of the same words)
    z = np.array([O.normals(3, 0, p, n, urule)[0] for p in range(40) for n in range(250)])
    assert abs(np.corrcoef(u, z)[0, 1]) < 5 / np.sqrt(len(u))


def test_material_rules():
    m = {"domain": DOM, "kappa": [[0, 1, 2, 3]], "bg": (0, 1),
         "shapes": [(0, 2, (-0.2, 0.2, 0.2, 0.5, 0, 0)), (1, 3, (-0.3, 0.6, 0.3, 0.6, 0.0, 0.7))]}
    assert O.material(m, 0.0, -0.1) == 0          # air z < 0
    assert O.material(m, 0.0, 0.0) == 1           # earth z >= 0
    assert O.material(m, -0.2, 0.2) == 2          # rectangle half-open: lower corner in
    assert O.material(m, 0.2, 0.3) == 1           # right edge out
    assert O.material(m, 0.0, 0.5) == 1           # bottom edge out
    assert O.material(m, 0.0, 0.6) == 3           # triangle edge in (closed)
    assert O.material(m, 0.3, 0.6) == 3           # triangle vertex in
    assert O.material(m, 0.0, 0.7) == 3           # apex
    assert O.material(m, 0.0, 0.71) == 1
    # raster: cell index floor((x - xmin) nx / W), clamped
    r = np.arange(12, dtype=np.int8).reshape(3, 4) % 4
    mr = {"domain": (0.0, 4.0, 0.0, 3.0), "kappa": [[0, 1, 2, 3]], "raster": r}
    assert O.material(mr, 0.5, 0.5) == r[0, 0]
    assert O.material(mr, 3.999, 2.999) == r[2, 3]
    assert O.material(mr, 1.0, 2.0) == r[2, 1]
    assert O.material(mr, -5.0, 10.0) == r[2, 0]


def test_g_columns_solves_the_1d_te_equation():
    # u'' = i kappa u for z > 0, u'' = 0 in air, u and u' continuous at 0,
    # u(0) = 1 (the 1D half-space boundary data of Sec. 2.1)
    m = I.quarterspace(2.0, 20.0)
    for wall, kap in ((0, 2.0), (1, 20.0)):
        x = -1.0 if wall == 0 else 1.0
        f = lambda z: O.g_value(m, 0, wall, x, z)
        h = 1e-4
        for z in (0.1, 0.4, 0.9):
            d2 = (f(z + h) - 2 * f(z) + f(z - h)) / h ** 2
            assert abs(d2 - 1j * kap * f(z)) < 1e-4 * max(1.0, abs(kap * f(z)))
        for z in (-0.3, -0.1):
            assert abs((f(z + h) - 2 * f(z) + f(z - h)) / h ** 2) < 1e-3
        assert abs(f(0.0) - 1.0) < 1e-15
        dp = (f(h) - f(0.0)) / h
        dm = (f(0.0) - f(-h)) / h
        assert abs(dp - dm) < 1e-3 * abs(dm)
        assert abs(dm + np.sqrt(1j * kap)) < 1e-12 * abs(dm)
    # half-space kappa = 2: k = 1 + i, top wall z = -0.5 gives 1 + 0.5 k
    hs = I.halfspace(2.0)
    assert abs(O.g_value(hs, 0, 2, 0.3, -0.5) - (1.5 + 0.5j)) < 1e-15
    assert abs(O.g_value(hs, 0, 3, -0.7, 1.0) - np.exp(-(1 + 1j))) < 1e-15
    # top/bottom interpolate linearly between the column corner values
    q = I.quarterspace(2.0, 20.0)
    gl, gr = O.g_value(q, 0, 0, -1.0, 1.0), O.g_value(q, 0, 1, 1.0, 1.0)
    assert abs(O.g_value(q, 0, 3, 0.5, 1.0) - (0.25 * gl + 0.75 * gr)) < 1e-15


def test_exit_rule_overshoot_cases():
    m = I.halfspace(2.0)
    # right wall: d = 0.1, d' = -0.1 -> theta = d / (d + |d'|) = 0.5
    hit, th, w, ex, ez = O.exit_rule(m, 0.9, 0.3, 1.1, 0.5, 1e-3, 0.5)
    assert hit and w == 1 and abs(th - 0.5) < 1e-14 and ex == 1.0 and abs(ez - 0.4) < 1e-14
    # exactly on the wall counts as reached: theta = 1
    hit, th, w, ex, ez = O.exit_rule(m, 0.9, 0.3, 1.0, 0.3, 1e-3, 0.5)
    assert hit and w == 1 and th == 1.0
    # two walls crossed: the smaller theta wins (top wall first here)
    hit, th, w, ex, ez = O.exit_rule(m, -0.95, -0.45, -1.05, -0.65, 1e-3, 0.5)
    assert hit and w == 2 and abs(th - 0.25) < 1e-14 and ez == -0.5
    # a tie goes to the first wall in the order left, right, top, bottom
    hit, th, w, ex, ez = O.exit_rule(m, -0.875, -0.375, -1.125, -0.625, 1e-3, 0.5)
    assert hit and w == 0 and th == 0.5 and ex == -1.0 and ez == -0.5


def test_exit_rule_bridge_matches_brownian_bridge_crossing_probability():
    # P(a Brownian bridge from distance d to d' over time dt touches the wall)
    # = exp(-2 d d' / dt) (textbook reflection principle); the rule draws one
    # uniform U and hits iff 2 d d'/dt <= -log U.
    m = I.halfspace(2.0)
    dt, d, dn = 1e-3, 0.01, 0.02
    p_exact = math.exp(-2 * d * dn / dt)
    M = 20000
    hits = 0
    for k in range(M):
        U = (k + 0.5) / M
        hit, th, w, ex, ez = O.exit_rule(m, 0.3, 1.0 - d, 0.31, 1.0 - dn, dt, U)
        if hit:
            hits += 1
            assert w == 3 and ez == 1.0 and 0 < th <= 1
            assert abs(th - (2 * d * dn / dt) / (-math.log(U))) < 1e-14
    assert abs(hits / M - p_exact) <= 1.0 / M
    # far from every wall the bridge never fires
    assert not O.exit_rule(m, 0.0, 0.3, 0.01, 0.31, dt, 1e-300)[0]


def test_unit_data_without_phase_is_exactly_one():
    # kappa = 0 and g = 1: every sample is exactly 1, the mean is exactly 1
    m = I.uniform_model(0.0, g=("affine", 1.0, 0.0, 0.0))
    nodes = [(0.0, 0.25), (0.9, 0.9), (-0.99, -0.49)]
    r = O.interface_values(m, nodes, 3000, 1e-3, 5)
    assert np.all(r["mean"] == 1.0)
    assert np.all(r["se"] == 0.0)
    assert r["truncated"] == 0 and r["walks"] == 9000


def test_halfspace_matches_closed_form():
    # homogeneous half-space, kappa = 2: u = exp(-(1+i) z) everywhere
    w = I.workload("halfspace")
    r = O.interface_values(w["model"], w["nodes"], w["n_paths"], w["dt"], w["seed"])
    exact = np.exp(-(1 + 1j) * 0.25)
    tol_b = pins.bias_bound(w["dt"])
    dev = r["mean"][:, 0] - exact
    se = r["se"][:, 0, :]
    assert np.all(np.abs(dev.real) <= 4 * se[:, 0] + tol_b)
    assert np.all(np.abs(dev.imag) <= 4 * se[:, 1] + tol_b)
    pooled = dev.mean()
    pse = np.sqrt((se ** 2).sum(0)) / len(dev)
    assert abs(pooled.real) <= 4 * pse[0] + tol_b
    assert abs(pooled.imag) <= 4 * pse[1] + tol_b


@pytest.mark.parametrize("x,z", [(0.0, 0.25), (0.5, 0.25), (0.0, 0.9)])
def test_mean_exit_time_matches_series(x, z):
    dt = 1e-3
    rec = O.walk_records(I.halfspace(2.0), (x, z), 0, 0, 20000, dt, 9)
    tau = ((rec["steps"] - 1) + rec["exit"][:, 2]) * dt
    se = tau.std(ddof=1) / math.sqrt(len(tau))
    assert abs(tau.mean() - pins.exit_time_series(x, z, DOM)) <= 4 * se + 2 * dt


@pytest.mark.parametrize("x,z", [(0.0, 0.25), (0.5, 0.6)])
def test_uniform_kappa_matches_helmholtz_series(x, z):
    kap, dt = 10.0, 1e-3
    r = O.interface_values(I.uniform_model(kap), [(x, z)], 40000, dt, 21)
    exact = pins.helmholtz_series(x, z, kap, DOM)
    dev = r["mean"][0, 0] - exact
    se = r["se"][0, 0]
    assert abs(dev.real) <= 4 * se[0] + pins.bias_bound(dt)
    assert abs(dev.imag) <= 4 * se[1] + pins.bias_bound(dt)


def test_harmonic_affine_data_reproduces_itself():
    # kappa = 0, g harmonic: u = g(x0) (optional stopping of a martingale)
    a, b, c = 0.3 + 0.1j, 1.0 - 0.5j, -0.7 + 0.2j
    m = I.uniform_model(0.0, g=("affine", a, b, c))
    nodes = [(0.0, 0.25), (0.6, 0.7), (-0.8, -0.3)]
    dt = 1e-3
    r = O.interface_values(m, nodes, 40000, dt, 8)
    for (x, z), mu, se in zip(nodes, r["mean"][:, 0], r["se"][:, 0, :]):
        g0 = a + b * x + c * z
        assert abs((mu - g0).real) <= 4 * se[0] + pins.bias_bound(dt)
        assert abs((mu - g0).imag) <= 4 * se[1] + pins.bias_bound(dt)
    m2 = I.uniform_model(0.0, g=("x2mz2",))
    r2 = O.interface_values(m2, nodes, 40000, dt, 8)
    for (x, z), mu, se in zip(nodes, r2["mean"][:, 0], r2["se"][:, 0, :]):
        assert abs(mu.real - (x * x - z * z)) <= 4 * se[0] + pins.bias_bound(dt)
        assert mu.imag == 0.0


def _kappa_quarter(X, Z):
    k = np.where(X < 0, 2.0, 20.0)
    k = np.where(X == 0, 11.0, k)
    k = np.where(Z < 0, 0.0, k)
    return np.where(Z == 0, k / 2, k)


@pytest.mark.slow
def test_quarterspace_matches_finite_differences():
    pts = [(0.0, 0.25), (-0.25, 0.5), (0.25, 0.5)]
    fd, fd_err = pins.fd_richardson(_kappa_quarter, DOM, 2.0, 20.0, pts)
    dt = 1e-3
    r = O.interface_values(I.quarterspace(2.0, 20.0), pts, 100000, dt, 13)
    for mu, se, ref, err in zip(r["mean"][:, 0], r["se"][:, 0, :], fd, fd_err):
        assert abs((mu - ref).real) <= 4 * se[0] + pins.bias_bound(dt) + err
        assert abs((mu - ref).imag) <= 4 * se[1] + pins.bias_bound(dt) + err


# --------------------------------------------------------- occupation rule

@pytest.mark.parametrize("urule", [32, 23])
def test_occupation_counts_the_material_at_the_end_of_each_step(urule):
    # Sec. 3.1 gives a step's dt to the material in which beta^(n+1) lies.
    # With every wall far away (no walk can exit in a few steps) and a
    # material B = {x >= b}, step k is counted in B with probability
    # P(x0 + sqrt(k dt) N >= b) = Phi((x0 - b) / sqrt(k dt)), so the expected
    # count in B after n steps is that sum over k = 1..n.  Counting the left
    # endpoint instead would give 0 (x0 < b) or 1 (x0 >= b) for n = 1.
    dt, b = 1e-2, 0.0
    m = {"domain": (-5.0, 5.0, -5.0, 5.0), "kappa": [[0.0, 0.0]], "bg": (0, 0),
         "shapes": [(0, 1, (b, 10.0, -10.0, 10.0, 0.0, 0.0))], "g": ("affine", 1.0, 0.0, 0.0)}
    N = 40000
    for x0, n_steps in ((b - 0.05, 1), (b + 0.03, 1), (b - 0.1, 4)):
        rec = O.walk_records(m, (x0, 0.3), 0, 0, N, dt, 19, urule=urule, max_steps=n_steps)
        assert np.all(rec["truncated"] == 1) and np.all(rec["steps"] == n_steps)
        assert np.all(rec["counts"].sum(1) == n_steps)
        cnt = rec["counts"][:, 1].astype(float)
        want = sum(stats.norm.cdf((x0 - b) / math.sqrt(k * dt)) for k in range(1, n_steps + 1))
        se = cnt.std(ddof=1) / math.sqrt(N)
        assert abs(cnt.mean() - want) <= 4 * se, (x0, n_steps, cnt.mean(), want, se)


# ------------------------------------------------ finite-difference brute force

@pytest.mark.slow
def test_triangle_matches_finite_differences():
    # The triangle model of the dt sweep (rate 50 inside, host 2) has no
    # closed form.  Finite differences with the rate averaged over each
    # node's dual cell (the triangle clipped against the cell, so the slanted
    # edges need no point-in-triangle test) on h = 1/40, 1/80, 1/160,
    # Richardson-extrapolated from the two finest; nodes on two edges, inside,
    # outside and below.  A triangle of the wrong orientation (empty) or the
    # wrong rate misses by hundreds of standard errors.
    pts = [(0.0, 0.2), (0.0, 0.4), (0.15, 0.4), (0.5, 0.5), (0.0, 0.7)]
    kfn = pins.kappa_cell_average(2.0, [(I.TRIANGLE, 50.0)])
    ref, err, ratio = pins.fd_richardson3(kfn, DOM, 2.0, 2.0, pts)
    assert np.all((ratio > 3.5) & (ratio < 4.5)), ratio  # second order observed
    dt = 1e-3
    r = O.interface_values(I.triangle(), pts, 200000, dt, 13)
    for mu, se, want, e in zip(r["mean"][:, 0], r["se"][:, 0, :], ref, err):
        assert abs((mu - want).real) <= 4 * se[0] + pins.bias_bound(dt) + e
        assert abs((mu - want).imag) <= 4 * se[1] + pins.bias_bound(dt) + e


@pytest.mark.slow
def test_block_matches_finite_differences():
    # The block of the batched workload at frequency scale 1, both block
    # rates (20 and 0.2, host 2) as the two rows of one evaluation table:
    # finite differences as for the triangle, the block clipped against each
    # dual cell; nodes on the block's top and right edges, at its centre,
    # outside and below it.
    pts = [(0.0, 0.2), (0.2, 0.35), (0.0, 0.35), (-0.45, 0.35), (0.0, 0.6)]
    m = I.block_batched(scales=[1.0])
    dt = 1e-3
    r = O.interface_values(m, pts, 150000, dt, 23)
    verts = I.rect_vertices(I.BLOCK)
    for e, kb in enumerate((20.0, 0.2)):
        kfn = pins.kappa_cell_average(2.0, [(verts, kb)])
        ref, err, ratio = pins.fd_richardson3(kfn, DOM, 2.0, 2.0, pts)
        assert np.all((ratio > 3.5) & (ratio < 4.5)), ratio
        for mu, se, want, er in zip(r["mean"][:, e], r["se"][:, e, :], ref, err):
            assert abs((mu - want).real) <= 4 * se[0] + pins.bias_bound(dt) + er, (e, mu, want, se)
            assert abs((mu - want).imag) <= 4 * se[1] + pins.bias_bound(dt) + er, (e, mu, want, se)


def test_block_model_is_symmetric_in_x():
    m = I.block_batched(scales=[1.0, 10.0])
    pts = [(-0.2, 0.35), (0.15, 0.55)]
    mir = [(-x, z) for x, z in pts]
    a = O.interface_values(m, pts, 20000, 1e-3, 1)
    b = O.interface_values(m, mir, 20000, 1e-3, 2)
    d = a["mean"] - b["mean"]
    s = np.sqrt(a["se"] ** 2 + b["se"] ** 2)
    assert np.all(np.abs(d.real) <= 4 * s[..., 0] + 1e-12)
    assert np.all(np.abs(d.imag) <= 4 * s[..., 1] + 1e-12)


def test_raster_model_agrees_with_its_analytic_shapes():
    m = I.triangle()
    mr = dict(m)
    mr["raster"] = I.rasterize(m)
    mr["shapes"] = []
    pts = [(0.0, 0.3), (0.1, 0.62)]
    a = O.interface_values(m, pts, 20000, 1e-3, 4)
    b = O.interface_values(mr, pts, 20000, 1e-3, 4)
    s = np.sqrt(a["se"] ** 2 + b["se"] ** 2)
    d = a["mean"] - b["mean"]
    assert np.all(np.abs(d.real) <= 4 * s[..., 0] + 2e-3)
    assert np.all(np.abs(d.imag) <= 4 * s[..., 1] + 2e-3)


def test_sums_do_not_depend_on_thread_count():
    w = I.scaled(I.workload("quarterspace"), paths_per_node=3000, n_nodes=4, dt=1e-3)
    a = O.interface_values(w["model"], w["nodes"], w["n_paths"], w["dt"], 0, threads=1)
    b = O.interface_values(w["model"], w["nodes"], w["n_paths"], w["dt"], 0, threads=3)
    assert np.array_equal(a["mean"], b["mean"]) and np.array_equal(a["se"], b["se"])


def test_truncated_walks_are_counted_and_excluded():
    m = I.halfspace(2.0)
    r = O.interface_values(m, [(0.0, 0.25)], 2000, 1e-3, 0, max_steps=300)
    rec = O.walk_records(m, (0.0, 0.25), 0, 0, 2000, 1e-3, 0, max_steps=300)
    assert r["truncated"] == int(rec["truncated"].sum()) > 0
    assert np.all(rec["steps"][rec["truncated"] == 1] == 300)
    assert r["walks"] == 2000
    # a walk's occupation counts add up to its non-exiting steps
    ok = rec["truncated"] == 0
    assert np.all(rec["counts"][ok].sum(1) == rec["steps"][ok] - 1)
    assert np.all(rec["counts"][~ok].sum(1) == rec["steps"][~ok])


def test_each_evaluation_row_uses_its_own_rates():
    # three evaluations sharing one walk, each a uniform medium of its own
    # rate (air and earth rates equal): every row must match the Helmholtz
    # series of its own kappa, so a transposed [E][K] table fails
    rows = [[1.0, 1.0], [5.0, 5.0], [20.0, 20.0]]
    m = {"domain": DOM, "kappa": rows, "bg": (0, 1), "shapes": [], "g": ("affine", 1.0, 0.0, 0.0)}
    dt = 1e-3
    x, z = 0.2, 0.4
    r = O.interface_values(m, [(x, z)], 40000, dt, 17)
    for e, (kap, _) in enumerate(rows):
        ref = pins.helmholtz_series(x, z, kap, DOM)
        dev = r["mean"][0, e] - ref
        se = r["se"][0, e]
        assert abs(dev.real) <= 4 * se[0] + pins.bias_bound(dt)
        assert abs(dev.imag) <= 4 * se[1] + pins.bias_bound(dt)


# ------------------------------------------------------------------ TM mode
# Diffusion coefficient that jumps across vertical interfaces (Sec. 2.2 and
# the interface rules of Sec. 3.1).  The interface treatment is first order:
# its bias is O(sqrt(dt)); TM_BIAS_C sqrt(dt) bounds what a dt sweep of these
# pins measured (<= 0.028 sqrt(dt) away from interfaces started on, at
# dt = 1e-4 and 1e-3).
TM_BIAS_C = 0.3
TM_DOM = (-1.0, 1.0, -0.5, 1.0)


def _tm(diffusion, interfaces, kappa, g=("tm_flux",), domain=TM_DOM):
    return {"domain": domain, "kappa": [list(kappa)], "diffusion": list(diffusion),
            "interfaces": list(interfaces), "g": g}


def _tm_close(mean, se, exact, dt):
    tol_re = 4.0 * se[..., 0] + TM_BIAS_C * np.sqrt(dt)
    tol_im = 4.0 * se[..., 1] + TM_BIAS_C * np.sqrt(dt)
    d = mean - exact
    return bool(np.all(np.abs(d.real) <= tol_re) and np.all(np.abs(d.imag) <= tol_im))


def test_tm_uniforms_are_the_words_of_their_own_philox_call():
    for urule in (32, 23):
        U = O.tm_uniforms(77, 3, 11, 5, urule)
        w = O.philox4x32_10([5, 11, 3, 2], [77, 0])
        assert np.array_equal(U, [O.uniform(int(x), urule) for x in w])


@pytest.mark.parametrize("diffusion,interfaces", [((1.0, 10.0), (0.3,)), ((4.0, 0.5, 2.0), (-0.4, 0.2))])
def test_tm_flux_continuous_solution_without_phase(diffusion, interfaces):
    # kappa = 0: u(x) = int dx / D solves div(D grad u) = 0 with the same flux
    # on both sides of every interface; its kink pins the crossing probability
    # D_i / (D_i + D_j) and the side of the resampling disc (a probability of
    # 1/2, or the disc on the wrong side, miss by tens of standard errors)
    dt = 1e-3
    m = _tm(diffusion, interfaces, [0.0] * len(diffusion))
    xs = np.array([-0.8, -0.45, -0.4, 0.0, 0.25, 0.3, 0.6, 0.9])
    nodes = np.stack([xs, np.full_like(xs, 0.25)], axis=1)
    r = O.interface_values(m, nodes, 20000, dt, 11)
    exact = pins.u_flux(xs, diffusion, interfaces, TM_DOM[0])
    assert _tm_close(r["mean"][:, 0], r["se"][:, 0], exact, dt)


def test_tm_analytic_test_model():
    # the analytic test of Sec. 4.1 on [-1,1]^2: D = 1 | 10 across x = 0,
    # lambda = 10i, i.e. D Lap u = i kappa u with kappa = -10; exact solution
    # (z + 1) cosh(a x), D a^2 = i kappa, read with the square root over
    # lambda / kappa_j only (the printed form is garbled)
    dt = 1e-4
    m = _tm((1.0, 10.0), (0.0,), (-10.0, -10.0), g=("tm_cosh",), domain=(-1.0, 1.0, -1.0, 1.0))
    nodes = np.array([[0.6, 0.6], [-0.5, 0.2], [0.0, -0.3]])
    r = O.interface_values(m, nodes, 20000, dt, 7)
    exact = np.array([(z + 1.0) * np.cosh(np.sqrt(1j * -10.0 / (1.0 if x < 0 else 10.0)) * x) for x, z in nodes])
    assert _tm_close(r["mean"][:, 0], r["se"][:, 0], exact, dt)


def test_tm_matches_finite_volumes_with_phase_and_flux():
    # kappa = 2 | 20 and D = 1 | 10 across x = 0 with boundary data int dx / D:
    # no closed form; Richardson-extrapolated finite volumes on h = 1/40, 1/80
    # (flux-conservative faces, the interface on a grid column); one node on
    # the interface itself
    dt = 1e-4
    D, xif, kap = (1.0, 10.0), (0.0,), (2.0, 20.0)
    pts = [(-0.5, 0.25), (-0.1, 0.25), (0.0, 0.5), (0.1, 0.25), (0.5, 0.75)]
    ref, err = pins.fd_tm_richardson(TM_DOM, D, xif, kap,
                                     lambda X, Z: pins.u_flux(X, D, xif, TM_DOM[0]) + 0.0j, pts)
    r = O.interface_values(_tm(D, xif, kap), np.array(pts), 12000, dt, 5)
    assert _tm_close(r["mean"][:, 0], r["se"][:, 0] + err[:, None], ref, dt)


def test_tm_equal_diffusion_is_the_te_walk():
    # D the same in every strip: no interface events, so every walk equals the
    # TE walk through the same material map (strip = material), step by step
    dt = 1e-3
    tm = _tm((1.0, 1.0), (0.3,), (2.0, 20.0), g=("affine", 0.5, 1.0, 0.25))
    te = {"domain": TM_DOM, "kappa": [[2.0, 20.0]], "bg": (0, 0),
          "shapes": [(0, 1, (0.3, 2.0, -1.0, 2.0, 0.0, 0.0))], "g": ("affine", 0.5, 1.0, 0.25)}
    a = O.walk_records(tm, (0.1, 0.2), 4, 0, 500, dt, 3)
    b = O.walk_records(te, (0.1, 0.2), 4, 0, 500, dt, 3)
    for k in ("steps", "counts", "exit", "wall", "m_last"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["occ"], a["counts"]) and a["hits"].sum() == 0
    # a uniform D = 4 is Brownian motion run 4 times faster: mean exit time / 4
    fast = _tm((4.0, 4.0), (0.3,), (0.0, 0.0))
    nodes = np.array([[0.0, 0.25], [0.5, 0.25]])
    rf = O.interface_values(fast, nodes, 20000, dt, 9)
    for (x, z), t in zip(nodes, rf["tau_mean"]):
        assert abs(t - pins.exit_time_series(x, z, TM_DOM) / 4.0) <= 0.02 * pins.exit_time_series(x, z, TM_DOM) / 4.0 + 0.002


def test_tm_walks_hit_interfaces_and_conserve_time():
    dt = 1e-3
    m = _tm((1.0, 10.0), (0.0,), (2.0, 20.0))
    rec = O.walk_records(m, (0.0, 0.25), 0, 0, 2000, dt, 5)
    assert rec["hits"].min() >= 1  # every walk starts on the interface
    ok = rec["truncated"] == 0
    # occupation per walk, in units of dt: every step but the exiting one
    # (which contributes theta through the last material), or every step when
    # the walk ended because a resampled point fell outside the domain
    # (theta = 0; the step's dt was split at the interface)
    disc_exit = rec["exit"][:, 2] == 0.0
    want = rec["steps"] - 1 + disc_exit
    assert np.allclose(rec["occ"][ok].sum(1), want[ok], rtol=0, atol=1e-9)
    assert 0 < disc_exit.sum() < 50


# The TM occupation split (Sec. 3.1, read as: staying on side i gives
# T_i = dt - (1/2)(dt - t_g) p_i, T_j = (1/2)(dt - t_g) p_i; moving to side j
# gives T_i = t_g + (1/2)(dt - t_g) p_j and T_j the rest of dt).  Averaged over
# the side drawn with p_i = D_i/(D_i + D_j), a hit at t_g = th dt leaves
# E[T_i] = (th + (1/2)(1 - th)) dt whatever the diffusions: the time after the
# hit is shared evenly on average.  Swapping p_i and p_j in the split gives
# E[T_i] = (1 - p_j (1 - th)) dt instead.

def _tm_one_step_expectation(c):
    """E[(1 - th) 1{hit}] for one step of standard deviation s from distance
    a = c s to a straight interface (no wall within reach): crossed steps
    (w >= c) have th = c / w; the others hit with probability exp(-g),
    g = 2 c (c - w), at th = g / (g + E), E ~ Exp(1), whose mean of 1 - th is
    1 - g e^g E1(g)."""
    from scipy import integrate, special
    phi = stats.norm.pdf
    crossed, _ = integrate.quad(lambda w: phi(w) * (1.0 - c / w), c, np.inf, epsabs=1e-12)

    def bridge(w):
        g = 2.0 * c * (c - w)
        return phi(w) * (np.exp(-g) - (g * special.exp1(g) if g > 0 else 0.0))
    bridged, _ = integrate.quad(bridge, -np.inf, c, epsabs=1e-12)
    return crossed + bridged


@pytest.mark.parametrize("start", ["left", "right"])
def test_tm_occupation_split_after_one_hit(start):
    # One step from distance a of the interface x = 0 (D = 1 | 10), walls far
    # away.  The hit probability is the reflection principle's 2 Phi(-a/s)
    # (s the step's standard deviation); the occupation of the starting
    # strip has mean 1 - (1/2) E[(1 - th) 1{hit}] (in units of dt).
    dt = 1e-3
    D = (1.0, 10.0)
    m = _tm(D, (0.0,), (0.0, 0.0), domain=(-3.0, 3.0, -3.0, 3.0))
    i = 0 if start == "left" else 1
    s = math.sqrt(D[i] * dt)
    c = 0.6
    x0 = -c * s if start == "left" else c * s
    N = 100000
    rec = O.walk_records(m, (x0, 0.2), 0, 0, N, dt, 29, max_steps=1)
    assert np.all(rec["steps"] == 1) and np.all(rec["truncated"] == 1)
    assert np.allclose(rec["occ"].sum(1), 1.0, rtol=0, atol=1e-12)
    hit = rec["hits"].astype(float)
    p_hit = 2.0 * stats.norm.cdf(-c)
    assert abs(hit.mean() - p_hit) <= 4 * math.sqrt(p_hit * (1 - p_hit) / N)
    Ti = rec["occ"][:, i]
    want = 1.0 - 0.5 * _tm_one_step_expectation(c)
    assert abs(Ti.mean() - want) <= 4 * Ti.std(ddof=1) / math.sqrt(N), (Ti.mean(), want)
    # the swapped split would sit (1/2 - p_j) E[(1 - th) 1{hit}] away
    pj = D[1 - i] / (D[0] + D[1])
    assert abs(0.5 - pj) * _tm_one_step_expectation(c) > 40 * Ti.std(ddof=1) / math.sqrt(N)


def test_tm_occupation_split_of_a_start_on_the_interface():
    # A walk that starts on the interface has hit it at t_g = 0 from the left
    # strip: each strip's mean occupation of the first step is dt/2, and the
    # walk resumes on the right with the crossing probability D_R/(D_L + D_R)
    # (the disc is tangent to the interface on the side drawn).
    dt = 1e-3
    for D in ((1.0, 10.0), (10.0, 1.0), (4.0, 0.5)):
        m = _tm(D, (0.0,), (0.0, 0.0), domain=(-3.0, 3.0, -3.0, 3.0))
        N = 60000
        rec = O.walk_records(m, (0.0, 0.2), 0, 0, N, dt, 31, max_steps=1)
        assert np.all(rec["hits"] == 1)
        occ = rec["occ"]
        assert np.allclose(occ.sum(1), 1.0, rtol=0, atol=1e-12)
        for k in (0, 1):
            assert abs(occ[:, k].mean() - 0.5) <= 4 * occ[:, k].std(ddof=1) / math.sqrt(N)
        right = (rec["m_last"] == 1).astype(float)
        pr = D[1] / (D[0] + D[1])
        assert abs(right.mean() - pr) <= 4 * math.sqrt(pr * (1 - pr) / N)
