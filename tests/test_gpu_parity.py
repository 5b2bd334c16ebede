"""Parity of the CUDA library with the FP64 oracle, through the C ABI.

FP64 mode (same Philox streams, same uniform rule (w + 1/2) 2^-32): every
discrete outcome of every walk -- its number of steps, its per-material step
counts, the wall it leaves by and its last material -- must equal the
oracle's, its exit point and hit fraction to 1e-12, and the node means to
1e-10 relative to the largest |g| (last-ulp differences of log/sin/cos
between the two math libraries are the only source of difference).

FP32 mode (same streams, uniform rule (w mod 2^23 + 1/2) 2^-23, FP32
positions): node means within 4 combined standard errors + 1e-4 of the
oracle's on the same streams.  On the same streams the FP32 walks take the
oracle's decisions (measured: every walk's step count and wall equal at dt
1e-3 and 1e-4), so the actual difference is far below that bound: it is
asserted below FP32_SAME_NSE standard errors.  A few walks (0.1-0.3 %) count
one step in a neighbouring material: a position within FP32 rounding (about
1e-6 after hundreds of steps) of a material edge.  With independent seeds
the two estimates agree within 4 combined standard errors.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1603_09311_gb300 import build as B
from paper_1603_09311_gb300 import inputs as I
from paper_1603_09311_gb300 import sdd

pytestmark = pytest.mark.gpu

FP64_REL = 1e-10        # relative to max |g| on the boundary
FP32_NSE, FP32_ABS = 4.0, 1e-4
# Same streams: the walks agree step for step, so the means differ by the
# rounding of exit points and samples (about 1e-5 of |g|), a small fraction
# of a standard error.
FP32_SAME_NSE = 0.1


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    sdd.lib()


def _triangle_raster():
    m = I.triangle()
    r = dict(m)
    r["raster"] = I.rasterize(m)
    r["shapes"] = []
    return r


def _many_materials():
    # K = 8: air, host and six shapes (rectangles and triangles), overlapping
    shapes = [(0, 2, (-0.8, -0.4, 0.1, 0.4, 0, 0)), (1, 3, (-0.5, 0.2, -0.1, 0.2, -0.3, 0.7)),
              (0, 4, (0.1, 0.5, 0.3, 0.6, 0, 0)), (1, 5, (0.2, 0.0, 0.8, 0.1, 0.6, 0.5)),
              (0, 6, (-0.2, 0.2, 0.6, 0.9, 0, 0)), (1, 7, (0.4, 0.7, 0.9, 0.7, 0.7, 0.95))]
    kap = [[0.0, 2.0, 5.0, 20.0, 0.5, 50.0, 1.0, 10.0]]
    return {"domain": I.DOMAIN, "kappa": kap, "bg": (0, 1), "shapes": shapes, "g": ("columns", 1, 1)}


def _one_rect(rect):
    # one rectangle of material 2 (rate 20) in the layered half-space
    return {"domain": I.DOMAIN, "kappa": [[0.0, 2.0, 20.0]], "bg": (0, 1),
            "shapes": [(0, 2, tuple(rect) + (0.0, 0.0))], "g": ("columns", 1, 1)}


MODELS = {
    "halfspace": (I.halfspace(2.0), (0.3, 0.25)),
    # one rectangle wholly in the air, and one across the surface (the
    # single-rectangle program counts regions only for a shape on one side)
    "rect_air": (_one_rect((-0.3, 0.3, -0.4, -0.1)), (0.0, -0.05)),
    "rect_straddle": (_one_rect((-0.2, 0.3, -0.2, 0.3)), (0.0, 0.1)),
    # one triangle wholly in the air (the single-triangle program's other side)
    "tri_air": ({"domain": I.DOMAIN, "kappa": [[0.0, 2.0, 20.0]], "bg": (0, 1),
                 "shapes": [(1, 2, (-0.4, -0.45, 0.3, -0.35, -0.1, -0.05))], "g": ("columns", 1, 1)},
                (-0.05, -0.2)),
    "quarterspace": (I.quarterspace(2.0, 20.0), (0.0, 0.5)),
    "block16": (I.block_batched(), (0.2, 0.35)),
    "triangle": (I.triangle(), (0.05, 0.4)),
    "triangle_raster": (_triangle_raster(), (0.05, 0.4)),
    "eight_materials": (_many_materials(), (0.0, 0.45)),
    "affine_g": (I.uniform_model(3.0, g=("affine", 0.5 + 0.1j, 1.0 - 0.2j, -0.3 + 0.4j)), (0.4, 0.1)),
    "x2mz2_g": (I.uniform_model(0.0, g=("x2mz2",)), (-0.6, 0.8)),
}


def _gmax(model):
    # a bound on |g| over the boundary (all test models)
    kap = np.asarray(model["kappa"], dtype=float).max()
    return max(2.0, 1.0 + 0.5 * np.sqrt(kap) * 1.5)


@pytest.mark.parametrize("name", sorted(MODELS))
def test_fp64_walks_equal_oracle_path_by_path(name):
    model, (x0, z0) = MODELS[name]
    dt, seed, nid, p0, count = 1e-3, 12345, 7, 101, 3000
    ctx = sdd.sdd_create(model)
    g = sdd.sdd_walk_records(ctx, x0, z0, nid, p0, count, dt, seed, precision="fp64")
    o = O.walk_records(model, (x0, z0), nid, p0, count, dt, seed, urule=32)
    assert np.array_equal(g["steps"], o["steps"])
    assert np.array_equal(g["counts"], o["counts"])
    assert np.array_equal(g["wall"], np.where(o["truncated"] == 1, -1, o["wall"]))
    assert np.array_equal(g["m_last"], o["m_last"])
    assert np.allclose(g["exit"], o["exit"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("name", sorted(MODELS))
def test_fp64_node_values_match_oracle(name):
    model, _ = MODELS[name]
    nodes = np.array([[0.0, 0.25], [-0.55, 0.6], [0.35, -0.2], [0.7, 0.85], [0.05, 0.4]])
    n_paths = np.array([1, 31, 33, 700, 2049])  # ragged: single walk, partial warps, several items
    dt, seed = 1e-3, 99
    ctx = sdd.sdd_create(model)
    mean, se, st = sdd.sdd_interface_values(ctx, nodes, n_paths, dt, seed, precision="fp64",
                                            chunk_paths=64)
    ref = O.interface_values(model, nodes, n_paths, dt, seed, urule=32)
    tol = FP64_REL * _gmax(model)
    assert np.allclose(mean.real, ref["mean"].real, rtol=0, atol=tol)
    assert np.allclose(mean.imag, ref["mean"].imag, rtol=0, atol=tol)
    ok = n_paths > 1
    assert np.allclose(se[ok], ref["se"][ok], rtol=1e-8, atol=1e-12)
    assert np.all(np.isnan(se[~ok]))
    assert st["walks"] == n_paths.sum() and st["steps"] == ref["steps"]


@pytest.mark.parametrize("name", sorted(MODELS))
def test_fp32_node_values_match_oracle(name):
    model, _ = MODELS[name]
    nodes = np.array([[0.0, 0.25], [-0.55, 0.6], [0.35, -0.2], [0.7, 0.85], [0.05, 0.4], [-0.9, 0.05]])
    n_paths = np.array([4096, 3001, 5000, 4096, 2500, 4500])
    dt, seed = 1e-3, 2024
    ctx = sdd.sdd_create(model)
    mean, se, st = sdd.sdd_interface_values(ctx, nodes, n_paths, dt, seed)
    ref = O.interface_values(model, nodes, n_paths, dt, seed, urule=23)
    tol = FP32_NSE * np.sqrt(se ** 2 + ref["se"] ** 2) + FP32_ABS
    d = mean - ref["mean"]
    assert np.all(np.abs(d.real) <= tol[..., 0])
    assert np.all(np.abs(d.imag) <= tol[..., 1])
    # what the same streams actually give: a small fraction of a standard error
    assert np.all(np.abs(d.real) <= FP32_SAME_NSE * ref["se"][..., 0] + 1e-6), np.abs(d.real) / ref["se"][..., 0]
    assert np.all(np.abs(d.imag) <= FP32_SAME_NSE * ref["se"][..., 1] + 1e-6), np.abs(d.imag) / ref["se"][..., 1]
    assert st["walks"] == n_paths.sum() and st["truncated"] == 0
    # same streams: the step totals agree to a small fraction of a percent
    assert abs(st["steps"] - ref["steps"]) <= 1e-3 * ref["steps"]


@pytest.mark.parametrize("name", sorted(MODELS))
def test_fp32_independent_seeds_agree_with_oracle(name):
    # the FP32 walk and the FP64 oracle on unrelated streams (other seed,
    # other uniform rule): both estimate the same expectation, so they agree
    # within 4 combined standard errors
    model, _ = MODELS[name]
    nodes = np.array([[0.0, 0.25], [-0.55, 0.6], [0.35, -0.2]])
    dt = 1e-3
    ctx = sdd.sdd_create(model)
    mean, se, _ = sdd.sdd_interface_values(ctx, nodes, 20000, dt, 5150)
    ref = O.interface_values(model, nodes, 20000, dt, 8088, urule=32)
    assert _fp32_close(mean, se, ref["mean"], ref["se"])


@pytest.mark.parametrize("name,dt", [("quarterspace", 1e-3), ("quarterspace", 1e-4), ("block16", 1e-3),
                                     ("rect_air", 1e-3), ("rect_straddle", 1e-3), ("triangle", 1e-3),
                                     ("tri_air", 1e-3)])
def test_fp32_walks_follow_the_oracle_streams(name, dt):
    # walk by walk: the FP32 walk takes the oracle's steps, wall and
    # per-material counts (the one-shape programs count regions and derive
    # the material counts at the exit)
    model, (x0, z0) = MODELS[name]
    ctx = sdd.sdd_create(model)
    n = 4000 if dt == 1e-3 else 1000
    g = sdd.sdd_walk_records(ctx, x0, z0, 3, 0, n, dt, 77)
    o = O.walk_records(model, (x0, z0), 3, 0, n, dt, 77, urule=23)
    same = g["steps"] == o["steps"]
    assert same.mean() >= 0.99, same.mean()
    assert np.array_equal(g["wall"][same], o["wall"][same])
    assert np.abs(g["exit"][same, :2] - o["exit"][same, :2]).max() <= 1e-3
    assert np.array_equal(g["counts"].sum(1), g["steps"] - 1)
    eq = np.all(g["counts"][same] == o["counts"][same], axis=1)
    assert eq.mean() >= 0.99


@pytest.mark.parametrize("name", ["quarterspace", "triangle_raster", "eight_materials"])
def test_fp32_cooperative_tail_gives_the_same_walks(name):
    # A launch of a few walks runs them in the cooperative tail (the warp's
    # lanes compute the step increments, each walk only moves); the same paths
    # inside one launch of 2048 walks run in full warps for most of their
    # steps.  Every record must be identical, truncation included.
    model, (x0, z0) = MODELS[name]
    ctx = sdd.sdd_create(model)
    full = sdd.sdd_walk_records(ctx, x0, z0, 5, 0, 2048, 1e-3, 91, chunk_paths=2048)
    for p0, cnt in ((0, 1), (7, 3), (100, 8), (2040, 8), (513, 5)):
        part = sdd.sdd_walk_records(ctx, x0, z0, 5, p0, cnt, 1e-3, 91)
        for k in ("steps", "counts", "exit", "wall", "m_last"):
            assert np.array_equal(part[k], full[k][p0:p0 + cnt]), (name, p0, cnt, k)
    full = sdd.sdd_walk_records(ctx, x0, z0, 5, 0, 512, 1e-3, 92, max_steps=40, chunk_paths=512)
    part = sdd.sdd_walk_records(ctx, x0, z0, 5, 200, 3, 1e-3, 92, max_steps=40)
    assert (full["wall"] < 0).sum() > 100 and (full["wall"] >= 0).any()
    for k in ("steps", "counts", "exit", "wall", "m_last"):
        assert np.array_equal(part[k], full[k][200:203]), (name, k)


def test_empty_and_single_inputs():
    ctx = sdd.sdd_create(I.halfspace(2.0))
    mean, se, st = sdd.sdd_interface_values(ctx, np.zeros((0, 2)), np.zeros(0, dtype=np.int64), 1e-3, 0)
    assert mean.shape == (0, 1) and st["walks"] == 0
    mean, se, st = sdd.sdd_interface_values(ctx, [[0.0, 0.25]], [1], 1e-3, 0, precision="fp64")
    ref = O.interface_values(I.halfspace(2.0), [[0.0, 0.25]], [1], 1e-3, 0, urule=32)
    assert abs(mean[0, 0] - ref["mean"][0, 0]) <= 1e-12 and np.all(np.isnan(se))


def test_nodes_next_to_walls_and_node_ids():
    model = I.halfspace(2.0)
    eps = 1e-6
    nodes = np.array([[-1 + eps, 0.3], [1 - eps, 0.3], [0.2, -0.5 + eps], [0.2, 1 - eps],
                      [-1 + eps, -0.5 + eps]])
    ids = np.array([40, 41, 42, 43, 44], dtype=np.uint32)
    ctx = sdd.sdd_create(model)
    mean, se, st = sdd.sdd_interface_values(ctx, nodes, 500, 1e-3, 5, node_ids=ids, precision="fp64")
    ref = O.interface_values(model, nodes, 500, 1e-3, 5, urule=32, node_id0=40)
    assert np.allclose(mean, ref["mean"], rtol=0, atol=1e-10)
    # permuting the nodes together with their ids permutes the results
    perm = np.array([3, 0, 4, 2, 1])
    m2, _, _ = sdd.sdd_interface_values(ctx, nodes[perm], 500, 1e-3, 5, node_ids=ids[perm],
                                        precision="fp64")
    assert np.allclose(m2, mean[perm], rtol=0, atol=1e-12)


def test_truncation_matches_oracle_exactly():
    model = I.quarterspace(2.0, 20.0)
    nodes = np.array([[0.0, 0.4], [0.3, 0.2]])
    ctx = sdd.sdd_create(model)
    mean, se, st = sdd.sdd_interface_values(ctx, nodes, 3000, 1e-3, 8, precision="fp64", max_steps=120)
    ref = O.interface_values(model, nodes, 3000, 1e-3, 8, urule=32, max_steps=120)
    assert st["status"] == sdd.SDD_E_TRUNCATED
    assert st["truncated"] == ref["truncated"] > 0
    assert np.allclose(mean, ref["mean"], rtol=0, atol=1e-10 * 30)


def test_launch_shape_does_not_change_results():
    w = I.scaled(I.workload("block"), n_nodes=12, paths_per_node=3000, dt=1e-3)
    ctx = sdd.sdd_create(w["model"])
    base, _, _ = sdd.sdd_interface_values(ctx, w["nodes"], w["n_paths"], w["dt"], 1)
    scale = np.abs(base).max()
    for cfg in ({"block_threads": 128}, {"chunk_paths": 32}, {"chunk_paths": 2048},
                {"ctas_per_sm": 1, "block_threads": 64}, {"guided_factor": 1}, {"guided_factor": 64}):
        m, _, _ = sdd.sdd_interface_values(ctx, w["nodes"], w["n_paths"], w["dt"], 1, **cfg)
        assert np.allclose(m, base, rtol=0, atol=1e-12 * scale), cfg


def test_device_api_matches_host_api():
    torch = pytest.importorskip("torch")
    w = I.scaled(I.workload("quarterspace"), n_nodes=8, paths_per_node=5000, dt=1e-3)
    ctx = sdd.sdd_create(w["model"])
    hm, hs, _ = sdd.sdd_interface_values(ctx, w["nodes"], w["n_paths"], w["dt"], 4)
    dev = torch.device("cuda:0")
    d_nodes = torch.tensor(w["nodes"], dtype=torch.float64, device=dev)
    d_mean = torch.empty((8, 1, 2), dtype=torch.float64, device=dev)
    d_se = torch.empty((8, 1, 2), dtype=torch.float64, device=dev)
    d_cnt = torch.zeros(3, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    sdd.sdd_interface_values_device(ctx, d_nodes.data_ptr(), 8, w["n_paths"], w["dt"], 4,
                                    d_mean.data_ptr(), d_se.data_ptr(),
                                    d_counters_ptr=d_cnt.data_ptr(), stream=stream.cuda_stream)
    torch.cuda.synchronize()
    dm = d_mean.cpu().numpy()
    assert np.allclose(dm[..., 0] + 1j * dm[..., 1], hm, rtol=0, atol=1e-12)
    assert np.allclose(d_se.cpu().numpy(), hs, rtol=1e-9, atol=0)
    assert int(d_cnt[1]) == 8 * 5000


def _kappa_quarter(X, Z):
    # the quarter-space rates at grid nodes, averaged over a node's dual cell
    # on the contact x = 0 and on the surface z = 0
    k = np.where(X < 0, 2.0, 20.0)
    k = np.where(np.abs(X) < 1e-12, 11.0, k)
    k = np.where(Z < 0, 0.0, k)
    return np.where(np.abs(Z) < 1e-12, k / 2, k)


@pytest.mark.slow
def test_full_size_quarterspace_sampled_nodes():
    # the benchmarked launch: 64 nodes x 1e5 paths, dt = 1e-4, default launch;
    # two nodes recomputed by the oracle in full, and every node against
    # finite differences (h = 1/70 and 1/140 put the nodes z = 0.9 k/63 = k/70
    # on both grids; Richardson-extrapolated)
    import pins
    w = I.workload("quarterspace")
    ctx = sdd.sdd_create(w["model"])
    mean, se, st = sdd.sdd_interface_values(ctx, w["nodes"], w["n_paths"], w["dt"], w["seed"])
    assert st["walks"] == 6_400_000 and st["truncated"] == 0
    a = pins.fd_value(_kappa_quarter, I.DOMAIN, 1 / 70, 2.0, 20.0, w["nodes"])
    b = pins.fd_value(_kappa_quarter, I.DOMAIN, 1 / 140, 2.0, 20.0, w["nodes"])
    fd, fd_err = (4 * b - a) / 3, np.abs(b - a) / 3
    d = mean[:, 0] - fd
    tb = pins.bias_bound(w["dt"])
    assert np.all(np.abs(d.real) <= 4 * se[:, 0, 0] + tb + fd_err), np.abs(d.real) / se[:, 0, 0]
    assert np.all(np.abs(d.imag) <= 4 * se[:, 0, 1] + tb + fd_err), np.abs(d.imag) / se[:, 0, 1]
    # each sampled node keeps its own node id (its index in the full call)
    for j in (9, 50):
        r = O.interface_values(w["model"], w["nodes"][j:j + 1], w["n_paths"][j:j + 1], w["dt"],
                               w["seed"], urule=23, node_id0=j)
        tol = FP32_NSE * np.sqrt(se[j] ** 2 + r["se"][0] ** 2) + FP32_ABS
        d = mean[j] - r["mean"][0]
        assert np.all(np.abs(d.real) <= tol[..., 0]) and np.all(np.abs(d.imag) <= tol[..., 1])
    assert np.all(np.isfinite(mean)) and np.all(se > 0)


def _fp32_close(mean, se, ref_mean, ref_se):
    tol = FP32_NSE * np.sqrt(se ** 2 + ref_se ** 2) + FP32_ABS
    d = mean - ref_mean
    return bool(np.all(np.abs(d.real) <= tol[..., 0]) and np.all(np.abs(d.imag) <= tol[..., 1]))


def test_full_size_halfspace_every_node():
    # the half-space workload in full (16 nodes x 1e4 paths, dt 1e-3), every
    # node recomputed by the oracle, in both precisions
    w = I.workload("halfspace")
    ctx = sdd.sdd_create(w["model"])
    m32, s32, st = sdd.sdd_interface_values(ctx, w["nodes"], w["n_paths"], w["dt"], w["seed"])
    r32 = O.interface_values(w["model"], w["nodes"], w["n_paths"], w["dt"], w["seed"], urule=23)
    assert st["walks"] == 160_000 and _fp32_close(m32, s32, r32["mean"], r32["se"])
    m64, _, _ = sdd.sdd_interface_values(ctx, w["nodes"], w["n_paths"], w["dt"], w["seed"], precision="fp64")
    r64 = O.interface_values(w["model"], w["nodes"], w["n_paths"], w["dt"], w["seed"], urule=32)
    tol = FP64_REL * _gmax(w["model"])
    assert np.allclose(m64.real, r64["mean"].real, rtol=0, atol=tol)
    assert np.allclose(m64.imag, r64["mean"].imag, rtol=0, atol=tol)


def test_full_size_block_sampled_nodes():
    # the batched block workload in full (256 nodes, 1e4..1e6 paths, 16
    # evaluations per walk, dt 1e-4); the three nodes with the fewest paths are
    # recomputed by the oracle under their own node ids
    w = I.workload("block")
    ctx = sdd.sdd_create(w["model"])
    mean, se, st = sdd.sdd_interface_values(ctx, w["nodes"], w["n_paths"], w["dt"], w["seed"])
    assert st["walks"] == w["n_paths"].sum() and st["truncated"] == 0 and mean.shape == (256, 16)
    for j in np.argsort(w["n_paths"])[:3]:
        r = O.interface_values(w["model"], w["nodes"][j:j + 1], w["n_paths"][j:j + 1], w["dt"],
                               w["seed"], urule=23, node_id0=int(j))
        assert _fp32_close(mean[j], se[j], r["mean"][0], r["se"][0]), j
    assert np.all(np.isfinite(mean)) and np.all(se > 0)


@pytest.mark.parametrize("dt", [1e-3, 3e-4, 1e-4, 3e-5])
def test_triangle_dt_sweep_both_precisions(dt):
    # the triangle workload's time-step sweep on four of its nodes: the FP64
    # walk equals the oracle's to 1e-10, the FP32 walk is within 4 combined SE
    w = I.workload("triangle")
    nodes = w["nodes"][[0, 40, 85, 127]]
    n_paths = np.full(4, 3000, dtype=np.int64)
    ctx = sdd.sdd_create(w["model"])
    m64, _, st64 = sdd.sdd_interface_values(ctx, nodes, n_paths, dt, w["seed"], precision="fp64")
    r64 = O.interface_values(w["model"], nodes, n_paths, dt, w["seed"], urule=32)
    tol = FP64_REL * _gmax(w["model"])
    assert np.allclose(m64.real, r64["mean"].real, rtol=0, atol=tol)
    assert np.allclose(m64.imag, r64["mean"].imag, rtol=0, atol=tol)
    assert st64["steps"] == r64["steps"]
    m32, s32, _ = sdd.sdd_interface_values(ctx, nodes, n_paths, dt, w["seed"])
    r32 = O.interface_values(w["model"], nodes, n_paths, dt, w["seed"], urule=23)
    assert _fp32_close(m32, s32, r32["mean"], r32["se"])


def test_full_size_triangle_sampled_node():
    # the triangle workload at its full path count (128 nodes x 1e6 paths) at
    # the sweep's largest step, dt 1e-3; one node recomputed by the oracle
    w = I.workload("triangle")
    dt = 1e-3
    ctx = sdd.sdd_create(w["model"])
    mean, se, st = sdd.sdd_interface_values(ctx, w["nodes"], w["n_paths"], dt, w["seed"])
    assert st["walks"] == 128_000_000 and st["truncated"] == 0
    j = 70
    r = O.interface_values(w["model"], w["nodes"][j:j + 1], w["n_paths"][j:j + 1], dt, w["seed"],
                           urule=23, node_id0=j)
    assert _fp32_close(mean[j], se[j], r["mean"][0], r["se"][0])
    assert np.all(np.isfinite(mean)) and np.all(se > 0)


def test_target_se_equals_fixed_counts_and_meets_target():
    # adaptive path counts: pilot, then top-up to N = var / se^2; the result
    # must be the fixed-count evaluation with n_paths = N (same walks), and
    # each node not capped at n_max must meet the target
    w = I.scaled(I.workload("quarterspace"), n_nodes=8, dt=1e-3)
    ctx = sdd.sdd_create(w["model"])
    target, n_pilot, n_max = 4e-3, 2000, 60000
    mean, se, used, st = sdd.sdd_interface_values_target(ctx, w["nodes"], n_pilot, n_max, target,
                                                         w["dt"], 21)
    assert np.all(used >= n_pilot) and np.all(used <= n_max)
    assert st["walks"] == used.sum()
    se_c = np.sqrt((se ** 2).sum(-1))[:, 0]
    free = used < n_max
    # N comes from the pilot's variance, itself an estimate (relative s.d. about
    # sqrt(2 / n_pilot) times the kurtosis factor, a few percent here): allow 15 %
    assert np.all(se_c[free] <= target * 1.15)
    fixed, fse, fst = sdd.sdd_interface_values(ctx, w["nodes"], used, w["dt"], 21)
    assert np.allclose(mean, fixed, rtol=0, atol=1e-12)
    assert np.allclose(se, fse, rtol=1e-9, atol=0)
    ref = O.interface_values(w["model"], w["nodes"], used, w["dt"], 21, urule=23)
    tol = FP32_NSE * np.sqrt(se ** 2 + ref["se"] ** 2) + FP32_ABS
    d = mean - ref["mean"]
    assert np.all(np.abs(d.real) <= tol[..., 0]) and np.all(np.abs(d.imag) <= tol[..., 1])


def test_batched_models_equal_each_model_alone():
    # several raster models (random serving requests, K up to 6) in one launch:
    # each entry's walks keep their streams, so every entry equals its own
    # evaluation alone up to FP64 summation order; one entry against the oracle
    rng = np.random.default_rng(7)
    entries = []
    for i in range(5):
        r = I.random_request(rng, i)
        nodes = r["nodes"][:: max(1, len(r["nodes"]) // 9)][:9]
        npth = np.array([1, 33, 700, 1500, 2049, 900, 1200, 64, 3000])[: len(nodes)]
        entries.append({"ctx": sdd.sdd_create(r["model"]), "model": r["model"], "nodes": nodes,
                        "n_paths": npth, "node_ids": np.arange(len(nodes)) + 50 * i})
    outs, st = sdd.sdd_batch_values(entries, 1e-3, 77)
    assert st["walks"] == sum(int(e["n_paths"].sum()) for e in entries)
    for e, (m, s_) in zip(entries, outs):
        ma, sa, _ = sdd.sdd_interface_values(e["ctx"], e["nodes"], e["n_paths"], 1e-3, 77,
                                             node_ids=e["node_ids"])
        scale = max(1.0, np.abs(ma[np.isfinite(ma)]).max())
        ok = e["n_paths"] > 1
        assert np.allclose(m[ok], ma[ok], rtol=0, atol=1e-12 * scale)
        assert np.allclose(s_[ok], sa[ok], rtol=1e-9, atol=0)
    e = entries[2]
    ref = O.interface_values(e["model"], e["nodes"], e["n_paths"], 1e-3, 77, urule=23,
                             node_id0=int(e["node_ids"][0]))
    m, s_ = outs[2]
    ok = e["n_paths"] > 1
    tol = FP32_NSE * np.sqrt(s_ ** 2 + ref["se"] ** 2) + FP32_ABS
    d = m - ref["mean"]
    assert np.all(np.abs(d.real)[ok] <= tol[..., 0][ok]) and np.all(np.abs(d.imag)[ok] <= tol[..., 1][ok])


def test_fp32_raster_walks_count_materials_like_the_oracle():
    # the single-precision walk reads rasters through a two-level tile map;
    # on the same streams its per-material step counts must equal the oracle's
    # (which reads the raster cell by cell) for walks whose steps agree
    rng = np.random.default_rng(5)
    r = [I.random_request(rng, i) for i in range(4)][3]  # six materials
    ctx = sdd.sdd_create(r["model"])
    assert ctx.K == 6
    for (x0, z0) in r["nodes"][:: max(1, len(r["nodes"]) // 3)][:3]:
        g = sdd.sdd_walk_records(ctx, x0, z0, 9, 0, 3000, 1e-3, 31)
        o = O.walk_records(r["model"], (x0, z0), 9, 0, 3000, 1e-3, 31, urule=23)
        same = g["steps"] == o["steps"]
        assert same.mean() >= 0.99
        eq = np.all(g["counts"][same] == o["counts"][same], axis=1)
        assert eq.mean() >= 0.99, eq.mean()
        # a differing walk has one step counted in a neighbouring material: a
        # position within FP32 rounding of a cell edge
        moved = np.abs(g["counts"][same][~eq] - o["counts"][same][~eq]).sum(1)
        assert np.all(moved == 2), moved


def test_graph_mode_equals_direct_launches():
    torch = pytest.importorskip("torch")
    w = I.scaled(I.workload("quarterspace"), n_nodes=8, paths_per_node=4000, dt=1e-3)
    ctx = sdd.sdd_create(w["model"])
    dev = torch.device("cuda:0")
    d_nodes = torch.tensor(w["nodes"], dtype=torch.float64, device=dev)
    outs = {}
    for mode, seed in (("direct", 1), ("graph", 1), ("graph", 2), ("direct", 2)):
        m = torch.empty((8, 1, 2), dtype=torch.float64, device=dev)
        s_ = torch.empty((8, 1, 2), dtype=torch.float64, device=dev)
        c = torch.zeros(3, dtype=torch.int64, device=dev)
        sdd.sdd_interface_values_device(ctx, d_nodes.data_ptr(), 8, w["n_paths"], w["dt"], seed,
                                        m.data_ptr(), s_.data_ptr(), d_counters_ptr=c.data_ptr(),
                                        stream=torch.cuda.current_stream().cuda_stream,
                                        use_graph=int(mode == "graph"))
        torch.cuda.synchronize()
        outs[(mode, seed)] = (m.cpu().numpy(), s_.cpu().numpy(), c.cpu().numpy())
    for seed in (1, 2):  # the second graph call updates the first graph in place
        a, b = outs[("direct", seed)], outs[("graph", seed)]
        assert np.allclose(a[0], b[0], rtol=0, atol=1e-12)
        assert np.allclose(a[1], b[1], rtol=1e-9, atol=0)
        assert np.array_equal(a[2], b[2])
    assert not np.allclose(outs[("graph", 1)][0], outs[("graph", 2)][0])


def test_autotune_keeps_results_and_caches_the_shape(tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("SDD_TUNE_CACHE", str(cache))
    w = I.scaled(I.workload("quarterspace"), n_nodes=16, paths_per_node=20000, dt=1e-3)
    ctx = sdd.sdd_create(w["model"])
    cfg, rate = sdd.sdd_autotune(ctx, w["nodes"], w["n_paths"], w["dt"], 3)
    assert cfg["block_threads"] in (128, 192, 256) and cfg["guided_factor"] in (1, 2, 4, 8) and rate > 0
    tuned, _, st = sdd.sdd_interface_values(ctx, w["nodes"], w["n_paths"], w["dt"], 5)
    assert st["block"] == cfg["block_threads"]
    plain = sdd.sdd_create(w["model"])
    monkeypatch.delenv("SDD_TUNE_CACHE")
    ref, _, st0 = sdd.sdd_interface_values(plain, w["nodes"], w["n_paths"], w["dt"], 5, block_threads=256,
                                           chunk_paths=32)
    assert np.allclose(tuned, ref, rtol=0, atol=1e-12)  # the same walks, another launch shape
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and "|" in lines[0]
    monkeypatch.setenv("SDD_TUNE_CACHE", str(cache))
    fresh = sdd.sdd_create(w["model"])  # reads the cached shape
    _, _, st2 = sdd.sdd_interface_values(fresh, w["nodes"], w["n_paths"], w["dt"], 5)
    assert st2["block"] == cfg["block_threads"]


def test_limits_32_evaluations_8_materials_many_nodes():
    # the largest tables (E = 32 evaluations x K = 8 materials; one lane per
    # evaluation in the sample pass) in both precisions, and a plan of 3000
    # nodes with 1..9 walks each (many tiny work items)
    base = _many_materials()
    rng = np.random.default_rng(17)
    kap = np.concatenate([np.array(base["kappa"]) * s for s in np.logspace(-1, 1.5, 32)])
    model = dict(base, kappa=kap)
    nodes = np.array([[0.0, 0.45], [-0.55, 0.6], [0.3, 0.1]])
    n_paths = np.array([700, 33, 2049])
    ctx = sdd.sdd_create(model)
    assert ctx.E == 32 and ctx.K == 8
    m64, _, st = sdd.sdd_interface_values(ctx, nodes, n_paths, 1e-3, 12, precision="fp64")
    r64 = O.interface_values(model, nodes, n_paths, 1e-3, 12, urule=32)
    tol = FP64_REL * _gmax(model)
    assert m64.shape == (3, 32)
    assert np.allclose(m64.real, r64["mean"].real, rtol=0, atol=tol)
    assert np.allclose(m64.imag, r64["mean"].imag, rtol=0, atol=tol)
    m32, s32, _ = sdd.sdd_interface_values(ctx, nodes, n_paths, 1e-3, 12)
    r32 = O.interface_values(model, nodes, n_paths, 1e-3, 12, urule=23)
    t32 = FP32_NSE * np.sqrt(s32 ** 2 + r32["se"] ** 2) + FP32_ABS
    d = m32 - r32["mean"]
    assert np.all(np.abs(d.real) <= t32[..., 0]) and np.all(np.abs(d.imag) <= t32[..., 1])
    many = np.stack([rng.uniform(-0.9, 0.9, 3000), rng.uniform(-0.4, 0.9, 3000)], axis=1)
    small = rng.integers(1, 10, 3000)
    mm, ss, st2 = sdd.sdd_interface_values(ctx, many, small, 1e-3, 13)
    assert st2["walks"] == small.sum() and np.all(np.isfinite(mm))
    # a node computed alone under its node id in the big call equals its value there
    for j in (0, 1234, 2999):
        one, _, _ = sdd.sdd_interface_values(ctx, many[j:j + 1], small[j:j + 1], 1e-3, 13,
                                             node_ids=np.array([j], dtype=np.uint32))
        assert np.allclose(one, mm[j:j + 1], rtol=0, atol=1e-12 * max(1.0, np.abs(mm).max()))
