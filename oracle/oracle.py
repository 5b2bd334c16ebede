"""ctypes wrapper of the FP64 oracle (``sdd_oracle.c``).

TEST INFRASTRUCTURE ONLY: the plain reference of the TE Feynman-Kac walk of
arXiv:1603.09311 (Sec. 3.1) that the CUDA library is checked against.  Only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It imports nothing from the CUDA
library's package and the library imports nothing from here.

A model is described by a plain dict (see ``sdd_inputs.py``):
    domain   (xmin, xmax, zmin, zmax)
    kappa    [E][K] phase rates per evaluation and material
    bg       (air material, earth material) for the layered background
    shapes   list of (kind, material, v[6]); kind 0 rectangle [v0,v1)x[v2,v3),
             kind 1 closed triangle (v0,v1),(v2,v3),(v4,v5)
    raster   optional int8 [nz][nx] material map (replaces bg and shapes)
    g        ("columns", left_material, right_material) | ("affine", a, b, c)
             | ("x2mz2",) | ("tm_cosh",) | ("tm_flux",)
TM mode (a diffusion coefficient that jumps across vertical interfaces):
    diffusion  [K] diffusion coefficient of strip m (material m)
    interfaces [K-1] increasing strip boundaries x; strip m = [x_{m-1}, x_m)
    (bg, shapes and raster are then unused: the material is the strip)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MAX_K = 8
MAX_E = 32


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (plain gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
           _SRC, "-o", _LIB + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Model(ctypes.Structure):
    _fields_ = [
        ("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
        ("zmin", ctypes.c_double), ("zmax", ctypes.c_double),
        ("K", ctypes.c_int), ("E", ctypes.c_int),
        ("kappa", ctypes.POINTER(ctypes.c_double)),
        ("bg_air", ctypes.c_int), ("bg_earth", ctypes.c_int),
        ("n_shapes", ctypes.c_int),
        ("shape_kind", ctypes.POINTER(ctypes.c_int)),
        ("shape_mat", ctypes.POINTER(ctypes.c_int)),
        ("shape_v", ctypes.POINTER(ctypes.c_double)),
        ("raster", ctypes.POINTER(ctypes.c_int8)),
        ("nx", ctypes.c_int), ("nz", ctypes.c_int),
        ("g_kind", ctypes.c_int),
        ("g_left", ctypes.c_int), ("g_right", ctypes.c_int),
        ("g_coef", ctypes.POINTER(ctypes.c_double)),
        ("urule", ctypes.c_int),
        ("max_steps", ctypes.c_int64),
        ("tm", ctypes.c_int),
        ("diff", ctypes.POINTER(ctypes.c_double)),
        ("xif", ctypes.POINTER(ctypes.c_double)),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        L.orc_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
        L.orc_philox4x32_10.restype = None
        L.orc_uniform.argtypes = [ctypes.c_uint32, ctypes.c_int]
        L.orc_uniform.restype = ctypes.c_double
        L.orc_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64,
                                  ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double)]
        L.orc_normals.restype = None
        L.orc_bridge_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.c_int64, ctypes.c_int]
        L.orc_bridge_uniform.restype = ctypes.c_double
        L.orc_material.argtypes = [P(_Model), ctypes.c_double, ctypes.c_double]
        L.orc_material.restype = ctypes.c_int
        L.orc_g.argtypes = [P(_Model), ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                            P(ctypes.c_double), P(ctypes.c_double)]
        L.orc_g.restype = None
        L.orc_exit_rule.argtypes = [P(_Model)] + [ctypes.c_double] * 6 + [
            P(ctypes.c_double), P(ctypes.c_int), P(ctypes.c_double), P(ctypes.c_double)]
        L.orc_exit_rule.restype = ctypes.c_int
        L.orc_interface_values.argtypes = [
            P(_Model), P(ctypes.c_double), ctypes.c_int, P(ctypes.c_int64), ctypes.c_uint32,
            ctypes.c_double, ctypes.c_uint64, ctypes.c_int, P(ctypes.c_double),
            P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_int64)]
        L.orc_interface_values.restype = ctypes.c_int64
        L.orc_walk_records.argtypes = [
            P(_Model), ctypes.c_double, ctypes.c_double, ctypes.c_uint32, ctypes.c_uint32,
            ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_int, P(ctypes.c_int64),
            P(ctypes.c_int64), P(ctypes.c_double), P(ctypes.c_int), P(ctypes.c_int),
            P(ctypes.c_int), P(ctypes.c_double), P(ctypes.c_int64)]
        L.orc_tm_uniforms.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_int64, ctypes.c_int, P(ctypes.c_double)]
        L.orc_tm_uniforms.restype = None
        L.orc_walk_records.restype = None
        L.orc_range_sums.argtypes = [
            P(_Model), P(ctypes.c_double), P(ctypes.c_uint32), ctypes.c_int, P(ctypes.c_int64),
            P(ctypes.c_int64), ctypes.c_double, ctypes.c_uint64, ctypes.c_int, P(ctypes.c_double),
            P(ctypes.c_int64), P(ctypes.c_int64)]
        L.orc_range_sums.restype = None
        L.orc_max_threads.argtypes = []
        L.orc_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class OracleModel:
    """Holds the ctypes struct and keeps its arrays alive."""

    def __init__(self, model: dict, urule: int = 32, max_steps: int | None = None, dt: float | None = None):
        kappa = np.ascontiguousarray(np.atleast_2d(np.asarray(model["kappa"], dtype=np.float64)))
        E, K = kappa.shape
        if K > MAX_K or E > MAX_E:
            raise ValueError("oracle supports K <= 8 materials and E <= 32 evaluations")
        self.kappa = kappa
        shapes = model.get("shapes", [])
        self.shape_kind = np.array([s[0] for s in shapes] or [0], dtype=np.int32)
        self.shape_mat = np.array([s[1] for s in shapes] or [0], dtype=np.int32)
        v = np.zeros((max(len(shapes), 1), 6), dtype=np.float64)
        for i, s in enumerate(shapes):
            v[i, : len(s[2])] = s[2]
        self.shape_v = v
        raster = model.get("raster")
        self.raster = None if raster is None else np.ascontiguousarray(raster, dtype=np.int8)
        g = model.get("g", ("columns", 1, 1))
        coef = np.zeros(6, dtype=np.float64)
        if g[0] == "columns":
            g_kind, gl, gr = 0, int(g[1]), int(g[2])
        elif g[0] == "affine":
            g_kind, gl, gr = 1, 0, 0
            a, b, c = (complex(t) for t in g[1:4])
            coef[:] = [a.real, a.imag, b.real, b.imag, c.real, c.imag]
        elif g[0] == "x2mz2":
            g_kind, gl, gr = 2, 0, 0
        elif g[0] == "tm_cosh":
            g_kind, gl, gr = 3, 0, 0
        elif g[0] == "tm_flux":
            g_kind, gl, gr = 4, 0, 0
        else:
            raise ValueError(f"unknown g kind {g[0]}")
        self.g_coef = coef
        if max_steps is None:
            if dt is None:
                raise ValueError("give max_steps or dt")
            max_steps = int(np.ceil(20.0 / dt))
        dom = model["domain"]
        bg = model.get("bg", (0, 1))
        self.s = _Model(
            float(dom[0]), float(dom[1]), float(dom[2]), float(dom[3]), K, E,
            _ptr(self.kappa, ctypes.c_double), int(bg[0]), int(bg[1]), len(shapes),
            _ptr(self.shape_kind, ctypes.c_int), _ptr(self.shape_mat, ctypes.c_int),
            _ptr(self.shape_v, ctypes.c_double),
            None if self.raster is None else _ptr(self.raster, ctypes.c_int8),
            0 if self.raster is None else self.raster.shape[1],
            0 if self.raster is None else self.raster.shape[0],
            g_kind, gl, gr, _ptr(self.g_coef, ctypes.c_double), int(urule), int(max_steps))
        self.diff = np.ascontiguousarray(np.asarray(model.get("diffusion", [1.0] * K), dtype=np.float64))
        self.xif = np.ascontiguousarray(np.asarray(list(model.get("interfaces", [])) + [0.0], dtype=np.float64))
        if "diffusion" in model:
            if self.diff.shape != (K,) or len(model.get("interfaces", [])) != K - 1:
                raise ValueError("TM mode needs K diffusion coefficients and K-1 interfaces")
            self.s.tm = 1
        elif g_kind in (3, 4):
            raise ValueError("tm_cosh and tm_flux boundary data need TM mode")
        self.s.diff = _ptr(self.diff, ctypes.c_double)
        self.s.xif = _ptr(self.xif, ctypes.c_double)
        self.E, self.K = E, K


def philox4x32_10(ctr, key):
    L = lib()
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    L.orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def uniform(w: int, urule: int = 32) -> float:
    return lib().orc_uniform(ctypes.c_uint32(w), urule)


def normals(seed: int, node: int, path: int, n: int, urule: int = 32):
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().orc_normals(seed, node, path, n, urule, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def bridge_uniform(seed: int, node: int, path: int, n: int, urule: int = 32) -> float:
    return lib().orc_bridge_uniform(seed, node, path, n, urule)


def tm_uniforms(seed: int, node: int, path: int, n: int, urule: int = 32):
    out = np.zeros(4)
    lib().orc_tm_uniforms(seed, node, path, n, urule, _ptr(out, ctypes.c_double))
    return out


def material(model: dict, x: float, z: float) -> int:
    om = OracleModel(model, max_steps=1)
    return lib().orc_material(ctypes.byref(om.s), x, z)


def g_value(model: dict, e: int, wall: int, x: float, z: float) -> complex:
    om = OracleModel(model, max_steps=1)
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().orc_g(ctypes.byref(om.s), e, wall, x, z, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def exit_rule(model: dict, x, z, xn, zn, dt, U):
    """Returns (exited, theta, wall, ex, ez) of the oracle's exit rule."""
    om = OracleModel(model, max_steps=1)
    th, ex, ez = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    w = ctypes.c_int()
    hit = lib().orc_exit_rule(ctypes.byref(om.s), x, z, xn, zn, dt, U, ctypes.byref(th),
                              ctypes.byref(w), ctypes.byref(ex), ctypes.byref(ez))
    return bool(hit), th.value, w.value, ex.value, ez.value


def interface_values(model: dict, nodes, n_paths, dt: float, seed: int, urule: int = 32,
                     max_steps: int | None = None, node_id0: int = 0, threads: int = 0):
    """Oracle Monte Carlo values.  Returns dict with
    mean complex [n][E], se float [n][E][2] (re, im), tau_mean [n],
    steps, walks, truncated."""
    om = OracleModel(model, urule=urule, max_steps=max_steps, dt=dt)
    nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64).reshape(-1, 2))
    n = nodes.shape[0]
    npth = np.asarray(n_paths, dtype=np.int64)
    if npth.ndim == 0:
        npth = np.full(n, int(npth), dtype=np.int64)
    npth = np.ascontiguousarray(npth)
    mean = np.zeros((n, om.E, 2))
    se = np.zeros((n, om.E, 2))
    tau = np.zeros(n)
    stats = np.zeros(3, dtype=np.int64)
    lib().orc_interface_values(ctypes.byref(om.s), _ptr(nodes, ctypes.c_double), n,
                               _ptr(npth, ctypes.c_int64), node_id0, dt, seed, threads,
                               _ptr(mean, ctypes.c_double), _ptr(se, ctypes.c_double),
                               _ptr(tau, ctypes.c_double), _ptr(stats, ctypes.c_int64))
    return {"mean": mean[..., 0] + 1j * mean[..., 1], "se": se, "tau_mean": tau,
            "steps": int(stats[0]), "walks": int(stats[1]), "truncated": int(stats[2])}


def walk_records(model: dict, node_xz, node_id: int, p0: int, count: int, dt: float, seed: int,
                 urule: int = 32, max_steps: int | None = None, threads: int = 0):
    """Per-path records: steps, counts [count][K], exit (x, z, theta), wall, m_last, truncated,
    occ [count][K] (occupation time per material in units of dt; TE: the counts), hits
    (TM interface randomisations)."""
    om = OracleModel(model, urule=urule, max_steps=max_steps, dt=dt)
    steps = np.zeros(count, dtype=np.int64)
    counts = np.zeros((count, om.K), dtype=np.int64)
    ext = np.zeros((count, 3))
    wall = np.zeros(count, dtype=np.int32)
    mlast = np.zeros(count, dtype=np.int32)
    trunc = np.zeros(count, dtype=np.int32)
    occ = np.zeros((count, om.K))
    hits = np.zeros(count, dtype=np.int64)
    lib().orc_walk_records(ctypes.byref(om.s), float(node_xz[0]), float(node_xz[1]), node_id, p0,
                           count, dt, seed, threads, _ptr(steps, ctypes.c_int64),
                           _ptr(counts, ctypes.c_int64), _ptr(ext, ctypes.c_double),
                           _ptr(wall, ctypes.c_int), _ptr(mlast, ctypes.c_int),
                           _ptr(trunc, ctypes.c_int), _ptr(occ, ctypes.c_double),
                           _ptr(hits, ctypes.c_int64))
    return {"steps": steps, "counts": counts, "exit": ext, "wall": wall, "m_last": mlast,
            "truncated": trunc, "occ": occ, "hits": hits}


def range_sums(model: dict, nodes, node_ids, path_begin, path_count, dt: float, seed: int,
               urule: int = 32, max_steps: int | None = None, threads: int = 0):
    """Raw sums of path ranges (range i: paths [path_begin[i], +path_count[i]) of
    nodes[i] under node id node_ids[i]).  Returns (sums [n][E][4] = sum re, sum im,
    sum re^2, sum im^2; n_valid [n]; total steps)."""
    om = OracleModel(model, urule=urule, max_steps=max_steps, dt=dt)
    nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64).reshape(-1, 2))
    n = nodes.shape[0]
    ids = np.ascontiguousarray(np.asarray(node_ids, dtype=np.uint32))
    b = np.ascontiguousarray(np.asarray(path_begin, dtype=np.int64))
    c = np.ascontiguousarray(np.asarray(path_count, dtype=np.int64))
    sums = np.zeros((n, om.E, 4))
    nv = np.zeros(n, dtype=np.int64)
    st = np.zeros(1, dtype=np.int64)
    lib().orc_range_sums(ctypes.byref(om.s), _ptr(nodes, ctypes.c_double), _ptr(ids, ctypes.c_uint32), n,
                         _ptr(b, ctypes.c_int64), _ptr(c, ctypes.c_int64), dt, seed, threads,
                         _ptr(sums, ctypes.c_double), _ptr(nv, ctypes.c_int64), _ptr(st, ctypes.c_int64))
    return sums, nv, int(st[0])


def max_threads() -> int:
    return lib().orc_max_threads()
