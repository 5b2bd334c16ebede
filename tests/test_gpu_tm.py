"""TM mode on the GPU (a diffusion coefficient jumping across vertical
interfaces), through the C ABI, against the FP64 oracle.

FP64 walk: every walk's steps, exit wall, last strip and interface
randomisations equal the oracle's, its occupation times and exit point to
1e-12, node means to 1e-10 relative to the largest |g|.  FP32 walk: node
means within 4 combined standard errors + 1e-4 of the oracle's on the
single-precision stream.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1603_09311_gb300 import build as B
from paper_1603_09311_gb300 import inputs as I
from paper_1603_09311_gb300 import sdd

pytestmark = pytest.mark.gpu

MODELS = {
    "analytic": (I.tm_analytic(), [(0.6, 0.6), (0.0, 0.2), (-0.5, -0.3)]),
    "two_strips": (I.tm_strips((1.0, 10.0), (0.3,), [[2.0, 20.0], [0.5, -3.0]]),
                   [(0.3, 0.25), (-0.2, 0.5), (0.6, 0.1)]),
    "three_strips": (I.tm_strips((4.0, 0.5, 2.0), (-0.4, 0.2), [[0.0, 1.0, 5.0]],
                                 g=("affine", 0.3, 1.0 + 0.5j, -0.2)), [(-0.4, 0.25), (0.0, 0.6), (0.7, 0.3)]),
    "equal_d": (I.tm_strips((2.0, 2.0), (0.1,), [[1.0, 8.0]], g=("x2mz2",)), [(0.1, 0.3), (-0.5, 0.2)]),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    sdd.lib()


def _gmax(name):
    return {"analytic": 2.0 * np.cosh(np.sqrt(10.0)), "two_strips": 2.5, "three_strips": 3.0,
            "equal_d": 1.0}[name]


@pytest.mark.parametrize("name", sorted(MODELS))
def test_tm_fp64_walks_equal_oracle_path_by_path(name):
    model, nodes = MODELS[name]
    ctx = sdd.sdd_create(model)
    for j, (x0, z0) in enumerate(nodes):
        g = sdd.sdd_walk_occupation(ctx, x0, z0, j, 0, 400, 1e-3, 21, precision="fp64")
        o = O.walk_records(model, (x0, z0), j, 0, 400, 1e-3, 21, urule=32)
        for k in ("steps", "wall", "m_last", "hits"):
            assert np.array_equal(g[k], o[k]), (name, j, k)
        assert np.allclose(g["occ"], o["occ"], rtol=0, atol=1e-12), (name, j)
        assert np.allclose(g["exit"], o["exit"], rtol=0, atol=1e-12), (name, j)
        if name != "equal_d":
            assert o["hits"].sum() > 0


@pytest.mark.parametrize("name", sorted(MODELS))
def test_tm_fp64_node_values_match_oracle(name):
    model, nodes = MODELS[name]
    nodes = np.array(nodes)
    n_paths = np.array([1, 33, 2049][: len(nodes)])
    ctx = sdd.sdd_create(model)
    mean, se, st = sdd.sdd_interface_values(ctx, nodes, n_paths, 1e-3, 5, precision="fp64", chunk_paths=64)
    ref = O.interface_values(model, nodes, n_paths, 1e-3, 5, urule=32)
    tol = 1e-10 * _gmax(name)
    assert np.allclose(mean.real, ref["mean"].real, rtol=0, atol=tol)
    assert np.allclose(mean.imag, ref["mean"].imag, rtol=0, atol=tol)
    assert st["steps"] == ref["steps"] and st["walks"] == n_paths.sum()


@pytest.mark.parametrize("name", sorted(MODELS))
def test_tm_fp32_node_values_match_oracle(name):
    model, nodes = MODELS[name]
    nodes = np.array(nodes)
    n_paths = np.full(len(nodes), 6000)
    ctx = sdd.sdd_create(model)
    mean, se, st = sdd.sdd_interface_values(ctx, nodes, n_paths, 1e-3, 8)
    ref = O.interface_values(model, nodes, n_paths, 1e-3, 8, urule=23)
    tol = 4.0 * np.sqrt(se ** 2 + ref["se"] ** 2) + 1e-4
    d = mean - ref["mean"]
    assert np.all(np.abs(d.real) <= tol[..., 0]) and np.all(np.abs(d.imag) <= tol[..., 1])
    assert abs(st["steps"] - ref["steps"]) <= 0.01 * ref["steps"]


def test_tm_fp32_walks_follow_the_oracle_streams():
    model, nodes = MODELS["two_strips"]
    ctx = sdd.sdd_create(model)
    g = sdd.sdd_walk_occupation(ctx, 0.1, 0.3, 2, 0, 3000, 1e-3, 13)
    o = O.walk_records(model, (0.1, 0.3), 2, 0, 3000, 1e-3, 13, urule=23)
    assert np.mean(g["steps"] == o["steps"]) >= 0.8
    ok = g["exit"][:, 2] > 0
    assert np.allclose(g["occ"][ok].sum(1), g["steps"][ok] - 1, rtol=0, atol=1e-3)


def test_tm_truncation_and_records_entry_points():
    model, _ = MODELS["two_strips"]
    ctx = sdd.sdd_create(model)
    for prec in ("fp64", "fp32"):
        g = sdd.sdd_walk_occupation(ctx, -0.2, 0.5, 0, 0, 300, 1e-3, 3, precision=prec, max_steps=16)
        o = O.walk_records(model, (-0.2, 0.5), 0, 0, 300, 1e-3, 3, urule=32 if prec == "fp64" else 23,
                           max_steps=16)
        assert np.array_equal(g["wall"] < 0, o["wall"] < 0) or prec == "fp32"
        assert (g["wall"] < 0).sum() > 100
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_walk_records(ctx, 0.0, 0.5, 0, 0, 10, 1e-3, 1)
    assert e.value.status == sdd.SDD_E_UNSUPPORTED


def test_tm_full_size_sampled_node():
    # the analytic test's 51 x 51 grid with 1e4 walks per node (dt 1e-4); one
    # node recomputed by the oracle under its node id
    w = I.workload("tm_analytic")
    ctx = sdd.sdd_create(w["model"])
    mean, se, st = sdd.sdd_interface_values(ctx, w["nodes"], w["n_paths"], w["dt"], w["seed"])
    assert st["walks"] == len(w["nodes"]) * 10_000 and st["truncated"] == 0
    j = int(np.argmin(np.abs(w["nodes"] - np.array([0.6, 0.6])).sum(1)))
    r = O.interface_values(w["model"], w["nodes"][j:j + 1], w["n_paths"][j:j + 1], w["dt"], w["seed"],
                           urule=23, node_id0=j)
    tol = 4.0 * np.sqrt(se[j] ** 2 + r["se"][0] ** 2) + 1e-4
    d = mean[j] - r["mean"][0]
    assert np.all(np.abs(d.real) <= tol[..., 0]) and np.all(np.abs(d.imag) <= tol[..., 1])
    # and the analytic solution itself, within 4 SE + the interface's O(sqrt(dt)) bias
    x, z = w["nodes"][j]
    exact = (z + 1.0) * np.cosh(np.sqrt(1j * -10.0 / 10.0) * x)
    assert abs(mean[j, 0].real - exact.real) <= 4 * se[j, 0, 0] + 0.3 * np.sqrt(w["dt"])
    assert abs(mean[j, 0].imag - exact.imag) <= 4 * se[j, 0, 1] + 0.3 * np.sqrt(w["dt"])
