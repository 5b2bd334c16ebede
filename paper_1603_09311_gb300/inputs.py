"""Seeded synthetic workloads shaped like the experiments of arXiv:1603.09311.

This module only builds inputs: node lists, path counts, material models
(domain, per-material phase rates, shapes or an int8 raster) and request
streams.  It holds none of the method's arithmetic, and both the CUDA library
and the oracle consume what it returns.

All models use the dimensionless TE form Lap u = i kappa(x) u on the domain
[-1, 1] x [-0.5, 1] (z positive down, air z < 0 with kappa = 0, earth z >= 0).
The experiments they stand in for are the quarter-space (Sec. 4.2), the
COMMEMI 2D-1 block in a half-space (Sec. 4.3) and the triangle in a
half-space (Sec. 4.4); the paper's own conductivities, frequencies and
metre-scale geometry are replaced by the dimensionless rates below.

Model dict keys: domain, kappa [E][K], bg (air, earth material), shapes
[(kind, material, v[6])] with kind 0 = rectangle [v0,v1)x[v2,v3) and kind 1 =
closed triangle, raster (optional int8 [nz][nx]), g (("columns", mL, mR) |
("affine", a, b, c) | ("x2mz2",)).
"""
from __future__ import annotations

import math

import numpy as np

DOMAIN = (-1.0, 1.0, -0.5, 1.0)
BIG = 1.0e30


def _model(kappa, shapes=(), g=("columns", 1, 1), bg=(0, 1), raster=None):
    m = {"domain": DOMAIN, "kappa": np.atleast_2d(np.asarray(kappa, dtype=np.float64)),
         "bg": tuple(bg), "shapes": list(shapes), "g": tuple(g)}
    if raster is not None:
        m["raster"] = raster
    return m


def halfspace(kappa_host: float = 2.0):
    """Homogeneous half-space: air (material 0), earth (material 1)."""
    return _model([[0.0, kappa_host]])


def quarterspace(kappa_left: float = 2.0, kappa_right: float = 20.0):
    """Quarter-space: earth split at x = 0 (materials 1 left, 2 right)."""
    return _model([[0.0, kappa_left, kappa_right]],
                  shapes=[(0, 2, (0.0, BIG, 0.0, BIG, 0.0, 0.0))], g=("columns", 1, 2))


BLOCK = (-0.2, 0.2, 0.2, 0.5)
TRIANGLE = ((-0.3, 0.2), (0.3, 0.2), (0.0, 0.6))


def block_batched(kappa_host=2.0, kappa_block=(20.0, 0.2), scales=None):
    """Block in a half-space, one evaluation per (block rate, frequency scale):
    E = len(kappa_block) * len(scales) rows of [air, host, block] rates."""
    if scales is None:
        scales = np.logspace(-1.0, 2.0, 8)
    rows = [[0.0, s * kappa_host, s * kb] for kb in kappa_block for s in scales]
    return _model(rows, shapes=[(0, 2, (BLOCK[0], BLOCK[1], BLOCK[2], BLOCK[3], 0.0, 0.0))])


def triangle(kappa_host=2.0, kappa_tri=50.0):
    (ax, az), (bx, bz), (cx, cz) = TRIANGLE
    return _model([[0.0, kappa_host, kappa_tri]], shapes=[(1, 2, (ax, az, bx, bz, cx, cz))])


def uniform_model(kappa: float, g=("affine", 1.0, 0.0, 0.0)):
    """One material everywhere (bg air = earth = 0) with rate kappa."""
    return _model([[kappa]], g=g, bg=(0, 0))


# ------------------------------------------------------------------ TM models
# Vertical strips with their own diffusion D_m (TM mode): D_m Lap u = i kappa_m u.

def tm_strips(diffusion, interfaces, kappa, g=("tm_flux",), domain=DOMAIN):
    k = np.atleast_2d(np.asarray(kappa, dtype=np.float64))
    return {"domain": domain, "kappa": k.tolist(), "diffusion": [float(d) for d in diffusion],
            "interfaces": [float(x) for x in interfaces], "g": g}


def tm_analytic():
    """The analytic test model of Sec. 4.1: [-1,1]^2, D = 1 | 10 across x = 0,
    lambda = 10i (kappa = -10), boundary data (z + 1) cosh(a x)."""
    return tm_strips((1.0, 10.0), (0.0,), [[-10.0, -10.0]], g=("tm_cosh",), domain=(-1.0, 1.0, -1.0, 1.0))


# ------------------------------------------------------------------ nodes

def rect_grid(x0, x1, z0, z1, nx, nz):
    """Nodes of an nx x nz grid on [x0, x1] x [z0, z1] (row-major in z, then
    x) and a flag per node: 1 on the rectangle's edge, else 0."""
    xs = np.linspace(x0, x1, nx)
    zs = np.linspace(z0, z1, nz)
    X, Z = np.meshgrid(xs, zs)
    nodes = np.stack([X.ravel(), Z.ravel()], axis=1)
    edge = np.zeros((nz, nx), dtype=np.uint8)
    edge[0, :] = edge[-1, :] = 1
    edge[:, 0] = edge[:, -1] = 1
    return np.ascontiguousarray(nodes), edge.ravel()


def nodes_line(p0, p1, n):
    t = np.linspace(0.0, 1.0, n)
    return np.stack([p0[0] + t * (p1[0] - p0[0]), p0[1] + t * (p1[1] - p0[1])], axis=1)


def nodes_on_polygon(verts, n):
    """n points evenly spaced in arc length on a closed polygon, starting at
    its first vertex."""
    v = np.asarray(verts, dtype=np.float64)
    segs = np.roll(v, -1, axis=0) - v
    lens = np.hypot(segs[:, 0], segs[:, 1])
    cum = np.concatenate([[0.0], np.cumsum(lens)])
    s = np.arange(n) * (cum[-1] / n)
    out = np.zeros((n, 2))
    for i, si in enumerate(s):
        k = min(np.searchsorted(cum, si, side="right") - 1, len(lens) - 1)
        t = (si - cum[k]) / lens[k]
        out[i] = v[k] + t * segs[k]
    return out


def rect_vertices(r):
    x0, x1, z0, z1 = r
    return [(x0, z0), (x1, z0), (x1, z1), (x0, z1)]


# --------------------------------------------------------------- workloads

def workload(name: str):
    """The five workload shapes (dimensionless), as dicts with keys
    model, nodes [n][2], n_paths [n], dt, seed, name."""
    if name == "halfspace":
        return {"name": name, "model": halfspace(2.0),
                "nodes": nodes_line((-0.5, 0.25), (0.5, 0.25), 16),
                "n_paths": np.full(16, 10_000, dtype=np.int64), "dt": 1e-3, "seed": 0}
    if name == "quarterspace":
        return {"name": name, "model": quarterspace(2.0, 20.0),
                "nodes": nodes_line((0.0, 0.0), (0.0, 0.9), 64),
                "n_paths": np.full(64, 100_000, dtype=np.int64), "dt": 1e-4, "seed": 0}
    if name == "block":
        rng = np.random.default_rng(3)
        npth = np.exp(rng.uniform(math.log(1e4), math.log(1e6), 256)).astype(np.int64)
        return {"name": name, "model": block_batched(),
                "nodes": nodes_on_polygon(rect_vertices(BLOCK), 256),
                "n_paths": npth, "dt": 1e-4, "seed": 3}
    if name == "triangle":
        return {"name": name, "model": triangle(),
                "nodes": nodes_on_polygon(TRIANGLE, 128),
                "n_paths": np.full(128, 1_000_000, dtype=np.int64), "dt": 1e-4, "seed": 4}
    if name == "tm_analytic":
        # the analytic test's 51 x 51 grid (interior points), 1e4 walks each
        g = np.linspace(-1.0, 1.0, 51)[1:-1]
        X, Z = np.meshgrid(g, g)
        nodes = np.stack([X.ravel(), Z.ravel()], axis=1)
        return {"name": name, "model": tm_analytic(), "nodes": nodes,
                "n_paths": np.full(len(nodes), 10_000, dtype=np.int64), "dt": 1e-4, "seed": 6}
    raise KeyError(name)


def scaled(w: dict, paths_per_node: int | None = None, n_nodes: int | None = None,
           dt: float | None = None):
    """A smaller copy of a workload (fewer paths and/or nodes, other dt)."""
    out = dict(w)
    nodes = w["nodes"]
    npth = w["n_paths"]
    if n_nodes is not None and n_nodes < len(nodes):
        idx = np.linspace(0, len(nodes) - 1, n_nodes).round().astype(int)
        nodes = nodes[idx]
        npth = npth[idx]
    if paths_per_node is not None:
        npth = np.full(len(nodes), paths_per_node, dtype=np.int64)
    out["nodes"] = np.ascontiguousarray(nodes)
    out["n_paths"] = np.ascontiguousarray(npth)
    if dt is not None:
        out["dt"] = dt
    return out


# --------------------------------------------------------- raster models

RASTER_NX, RASTER_NZ = 1024, 768


def rasterize(model: dict, nx: int = RASTER_NX, nz: int = RASTER_NZ) -> np.ndarray:
    """int8 material map of an analytic model, sampled at cell centres."""
    xmin, xmax, zmin, zmax = model["domain"]
    xc = xmin + (np.arange(nx) + 0.5) * ((xmax - xmin) / nx)
    zc = zmin + (np.arange(nz) + 0.5) * ((zmax - zmin) / nz)
    X, Z = np.meshgrid(xc, zc)
    air, earth = model["bg"]
    mat = np.where(Z >= 0.0, earth, air).astype(np.int8)
    for kind, m, v in model["shapes"]:
        if kind == 0:
            inside = (X >= v[0]) & (X < v[1]) & (Z >= v[2]) & (Z < v[3])
        else:
            ax, az, bx, bz, cx, cz = v
            area = (bx - ax) * (cz - az) - (bz - az) * (cx - ax)
            s = 1.0 if area >= 0 else -1.0
            e0 = s * ((bx - ax) * (Z - az) - (bz - az) * (X - ax))
            e1 = s * ((cx - bx) * (Z - bz) - (cz - bz) * (X - bx))
            e2 = s * ((ax - cx) * (Z - cz) - (az - cz) * (X - cx))
            inside = (e0 >= 0) & (e1 >= 0) & (e2 >= 0)
        mat[inside] = m
    return mat


def random_request(rng: np.random.Generator, rid: int):
    """One serving request: a random half-space model with 1-4 rectangles or
    triangles, rasterised to 1024 x 768 int8, nodes on the shape perimeters."""
    k_host = math.exp(rng.uniform(math.log(0.1), math.log(100.0)))
    n_shapes = int(rng.integers(1, 5))
    shapes, kap, polys = [], [0.0, k_host], []
    for s in range(n_shapes):
        cx, cz = rng.uniform(-0.7, 0.7), rng.uniform(0.05, 0.8)
        w, h = rng.uniform(0.05, 0.4), rng.uniform(0.05, 0.4)
        ratio = math.exp(rng.uniform(math.log(0.01), math.log(100.0)))
        kap.append(k_host * ratio)
        mat = 2 + s
        if rng.uniform() < 0.5:
            r = (cx - w / 2, cx + w / 2, max(cz - h / 2, 0.0), cz + h / 2)
            shapes.append((0, mat, (r[0], r[1], r[2], r[3], 0.0, 0.0)))
            polys.append(rect_vertices(r))
        else:
            tri = [(cx - w / 2, cz + h / 2), (cx + w / 2, cz + h / 2), (cx, max(cz - h / 2, 0.0))]
            shapes.append((1, mat, tuple(c for p in tri for c in p)))
            polys.append(tri)
    model = _model([kap], shapes=shapes)
    model["raster"] = rasterize(model)
    model["shapes"] = []
    n_nodes = int(round(math.exp(rng.uniform(math.log(16), math.log(1024)))))
    per = np.diff(np.linspace(0, n_nodes, len(polys) + 1).round().astype(int))
    nodes = np.concatenate([nodes_on_polygon(p, max(int(c), 1)) for p, c in zip(polys, per)])
    xmin, xmax, zmin, zmax = DOMAIN
    nodes[:, 0] = np.clip(nodes[:, 0], xmin + 1e-3, xmax - 1e-3)
    nodes[:, 1] = np.clip(nodes[:, 1], zmin + 1e-3, zmax - 1e-3)
    return {"id": rid, "model": model, "nodes": nodes, "seed": 1000 + rid, "dt": 1e-3,
            "target_se": 1e-3, "n_pilot": 4096, "n_max": 1_000_000}


def request_stream(n: int, rate_per_s: float, seed: int = 5):
    """n requests with Poisson arrival times (seconds from the start)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, n))
    return [dict(random_request(rng, i), arrival=float(t[i])) for i in range(n)]
