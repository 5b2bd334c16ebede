"""Thin ctypes binding of libsdd (include/sdd.h): argument marshalling only.

Every step of the Monte Carlo evaluation runs in the CUDA library; there is
no CPU fallback.  If libsdd.so is missing or cannot be loaded, ``lib()``
raises and nothing here computes anything.

The functions carry the names of the C entry points:
    sdd_create(model)                           -> Context
    sdd_destroy(ctx)
    sdd_interface_values(ctx, nodes, n_paths, dt, seed, ...)        host arrays
    sdd_interface_values_device(ctx, d_nodes, n_paths, dt, seed, d_mean, d_se, ...)
    sdd_walk_records(ctx, x0, z0, node_id, p0, count, dt, seed, ...)
    sdd_walk_occupation(ctx, x0, z0, node_id, p0, count, dt, seed, ...)   TE and TM
    sdd_interpolate(knots_s, values, se, targets_s, kind)
    sdd_interface_values_interp(ctx, nodes, stride, n_paths, kind, dt, seed, ...)
    sdd_apparent_resistivity(ctx, sites, h, n_paths, kappa_ref, dt, seed, ...)
    sdd_apparent_from_values(values, se, h, kappa_ref, d_site=None)
    sdd_rbffd_weights(nodes, n_stencil, eps), sdd_rbffd_solve(nodes, dirichlet, values, kappa, ...)
    sdd_status_str(status), sdd_last_error()
Models are the plain dicts of ``inputs.py``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsdd.so")

SDD_OK, SDD_E_ARG, SDD_E_OOM, SDD_E_CUDA, SDD_E_TRUNCATED = 0, 1, 2, 3, 4
SDD_E_CANCELLED, SDD_E_TIMEOUT, SDD_E_UNSUPPORTED, SDD_E_BUSY = 5, 6, 7, 8
SDD_FP32, SDD_FP64 = 0, 1
SDD_INTERP_LINEAR, SDD_INTERP_SPLINE = 0, 1
SDD_INTERP_MAX_SPLINE_KNOTS, SDD_INTERP_MAX_NODES = 4096, 1 << 20
SDD_MT_MAX_SITES = 1 << 20
SDD_RBFFD_MAX_NODES, SDD_RBFFD_MAX_STENCIL = 1 << 18, 16
MAX_K, MAX_E, MAX_SHAPES = 8, 32, 16


class SddError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().sdd_last_error().decode()
        super().__init__(f"{where}: {lib().sdd_status_str(status).decode()} ({msg})")


class sdd_domain(ctypes.Structure):
    _fields_ = [("x_min", ctypes.c_double), ("x_max", ctypes.c_double),
                ("z_min", ctypes.c_double), ("z_max", ctypes.c_double)]


class sdd_shape(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("material", ctypes.c_int32), ("v", ctypes.c_double * 6)]


class sdd_model_desc(ctypes.Structure):
    _fields_ = [
        ("domain", sdd_domain),
        ("n_materials", ctypes.c_int32), ("n_eval", ctypes.c_int32),
        ("kappa", ctypes.POINTER(ctypes.c_double)),
        ("bg_air", ctypes.c_int32), ("bg_earth", ctypes.c_int32),
        ("shapes", ctypes.POINTER(sdd_shape)), ("n_shapes", ctypes.c_int32),
        ("raster", ctypes.POINTER(ctypes.c_int8)), ("nx", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("g_kind", ctypes.c_int32), ("g_left", ctypes.c_int32), ("g_right", ctypes.c_int32),
        ("g_coef", ctypes.c_double * 6),
        ("diffusion", ctypes.POINTER(ctypes.c_double)), ("interfaces", ctypes.POINTER(ctypes.c_double)),
    ]


class sdd_config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("max_steps", ctypes.c_int64),
                ("block_threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("chunk_paths", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("guided_factor", ctypes.c_int32)]


class sdd_batch_entry(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("nodes_xz", ctypes.POINTER(ctypes.c_double)),
                ("node_ids", ctypes.POINTER(ctypes.c_uint32)), ("n_nodes", ctypes.c_int32),
                ("n_paths", ctypes.POINTER(ctypes.c_int64)), ("mean", ctypes.POINTER(ctypes.c_double)),
                ("se", ctypes.POINTER(ctypes.c_double))]


class sdd_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint64), ("walks", ctypes.c_uint64),
                ("truncated", ctypes.c_uint64), ("kernel_ms", ctypes.c_double),
                ("launches", ctypes.c_int32), ("items", ctypes.c_int32),
                ("grid", ctypes.c_int32), ("block", ctypes.c_int32),
                ("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64),
                ("post_ms", ctypes.c_double)]


class sdd_rbffd_stats(ctypes.Structure):
    _fields_ = [("unknowns", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("knn_ms", ctypes.c_double),
                ("weights_ms", ctypes.c_double), ("solve_ms", ctypes.c_double)]


class sdd_server_config(ctypes.Structure):
    _fields_ = [("domain", sdd_domain), ("nx", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("n_eval", ctypes.c_int32), ("g_kind", ctypes.c_int32),
                ("max_requests", ctypes.c_int32), ("max_bytes", ctypes.c_int64),
                ("n_streams", ctypes.c_int32), ("max_batch_models", ctypes.c_int32),
                ("max_batch_walks", ctypes.c_int64),
                ("dt", ctypes.c_double), ("seed", ctypes.c_uint64), ("launch", sdd_config)]


class sdd_request_desc(ctypes.Structure):
    _fields_ = [("model", ctypes.POINTER(sdd_model_desc)), ("nodes_xz", ctypes.POINTER(ctypes.c_double)),
                ("node_ids", ctypes.POINTER(ctypes.c_uint32)), ("n_nodes", ctypes.c_int32),
                ("n_paths", ctypes.POINTER(ctypes.c_int64)), ("target_se", ctypes.c_double),
                ("n_pilot", ctypes.c_int64), ("n_max", ctypes.c_int64)]


class sdd_request_stats(ctypes.Structure):
    _fields_ = [("queue_us", ctypes.c_double), ("latency_us", ctypes.c_double),
                ("walks", ctypes.c_uint64), ("truncated", ctypes.c_uint64),
                ("launches", ctypes.c_int32), ("status", ctypes.c_int32)]


class sdd_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("refused", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("cancelled", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("steps", ctypes.c_uint64), ("walks", ctypes.c_uint64),
                ("gpu_busy_ms", ctypes.c_double), ("in_flight", ctypes.c_int32),
                ("bytes_in_use", ctypes.c_int64)]


P = ctypes.POINTER
_lib = None

# (name, restype, argtypes) of every entry point declared in include/sdd.h
SIGNATURES = [
    ("sdd_create", ctypes.c_int, [P(sdd_model_desc), P(ctypes.c_void_p)]),
    ("sdd_destroy", None, [ctypes.c_void_p]),
    ("sdd_interface_values", ctypes.c_int,
     [ctypes.c_void_p, P(ctypes.c_double), P(ctypes.c_uint32), ctypes.c_int32, P(ctypes.c_int64),
      ctypes.c_double, ctypes.c_uint64, P(sdd_config), P(ctypes.c_double), P(ctypes.c_double),
      P(sdd_stats)]),
    ("sdd_interface_values_device", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_int64),
      ctypes.c_double, ctypes.c_uint64, P(sdd_config), ctypes.c_void_p, ctypes.c_void_p,
      ctypes.c_void_p, ctypes.c_void_p]),
    ("sdd_interface_values_target", ctypes.c_int,
     [ctypes.c_void_p, P(ctypes.c_double), P(ctypes.c_uint32), ctypes.c_int32, ctypes.c_int64,
      ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_uint64, P(sdd_config),
      P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_int64), P(sdd_stats)]),
    ("sdd_interface_values_noalloc", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_int64),
      ctypes.c_double, ctypes.c_uint64, P(sdd_config), ctypes.c_void_p, ctypes.c_void_p,
      ctypes.c_void_p, ctypes.c_void_p]),
    ("sdd_range_sums", ctypes.c_int,
     [ctypes.c_void_p, P(ctypes.c_double), P(ctypes.c_uint32), ctypes.c_int32, P(ctypes.c_int64),
      P(ctypes.c_int64), ctypes.c_double, ctypes.c_uint64, P(sdd_config), P(ctypes.c_double),
      P(ctypes.c_int64), P(sdd_stats)]),
    ("sdd_range_sums_device", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_int64),
      P(ctypes.c_int64), ctypes.c_double, ctypes.c_uint64, P(sdd_config), ctypes.c_void_p,
      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("sdd_reduce_sums", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_double),
      P(ctypes.c_int64), P(ctypes.c_double), P(ctypes.c_double)]),
    ("sdd_reduce_sums_device", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int32), ctypes.c_void_p,
      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("sdd_interface_values_async", ctypes.c_int,
     [ctypes.c_void_p, P(ctypes.c_double), P(ctypes.c_uint32), ctypes.c_int32, P(ctypes.c_int64),
      ctypes.c_double, ctypes.c_uint64, P(sdd_config), ctypes.c_void_p, P(ctypes.c_void_p)]),
    ("sdd_poll", ctypes.c_int, [ctypes.c_void_p]),
    ("sdd_wait", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    ("sdd_cancel", ctypes.c_int, [ctypes.c_void_p]),
    ("sdd_request_result", ctypes.c_int, [ctypes.c_void_p, P(ctypes.c_double), P(ctypes.c_double), P(sdd_stats)]),
    ("sdd_request_free", None, [ctypes.c_void_p]),
    ("sdd_batch_values", ctypes.c_int,
     [P(sdd_batch_entry), ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, P(sdd_config),
      P(sdd_stats)]),
    ("sdd_walk_records", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_uint32, ctypes.c_uint32,
      ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, P(sdd_config), P(ctypes.c_int64),
      P(ctypes.c_int64), P(ctypes.c_double), P(ctypes.c_int32), P(ctypes.c_int32)]),
    ("sdd_walk_occupation", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_uint32, ctypes.c_uint32,
      ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, P(sdd_config), P(ctypes.c_int64),
      P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int64)]),
    ("sdd_interpolate", ctypes.c_int,
     [P(ctypes.c_double), ctypes.c_int32, P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int32,
      P(ctypes.c_double), ctypes.c_int32, ctypes.c_int32, P(ctypes.c_double), P(ctypes.c_double)]),
    ("sdd_interface_values_interp", ctypes.c_int,
     [ctypes.c_void_p, P(ctypes.c_double), ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
      ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, P(sdd_config), P(ctypes.c_double),
      P(ctypes.c_double), P(sdd_stats)]),
    ("sdd_apparent_resistivity", ctypes.c_int,
     [ctypes.c_void_p, P(ctypes.c_double), ctypes.c_int32, ctypes.c_double, ctypes.c_int64,
      P(ctypes.c_double), ctypes.c_double, ctypes.c_uint64, P(sdd_config), P(ctypes.c_double),
      P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
      P(ctypes.c_double), P(sdd_stats)]),
    ("sdd_apparent_from_values", ctypes.c_int,
     [P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
      P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
      P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double)]),
    ("sdd_rbffd_weights", ctypes.c_int,
     [P(ctypes.c_double), ctypes.c_int32, ctypes.c_int32, ctypes.c_double, P(ctypes.c_int32),
      P(ctypes.c_double)]),
    ("sdd_rbffd_solve", ctypes.c_int,
     [P(ctypes.c_double), ctypes.c_int32, P(ctypes.c_uint8), P(ctypes.c_double), P(ctypes.c_double),
      ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32, P(ctypes.c_double),
      P(sdd_rbffd_stats)]),
    ("sdd_server_create", ctypes.c_int, [P(sdd_server_config), P(ctypes.c_void_p)]),
    ("sdd_server_destroy", None, [ctypes.c_void_p]),
    ("sdd_server_submit", ctypes.c_int, [ctypes.c_void_p, P(sdd_request_desc), P(ctypes.c_uint64)]),
    ("sdd_server_poll", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, P(ctypes.c_int32)]),
    ("sdd_server_wait", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64]),
    ("sdd_server_result", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_uint64, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_int64),
      P(sdd_request_stats)]),
    ("sdd_server_cancel", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    ("sdd_server_get_stats", ctypes.c_int, [ctypes.c_void_p, P(sdd_server_stats)]),
    ("sdd_autotune", ctypes.c_int,
     [ctypes.c_void_p, P(ctypes.c_double), ctypes.c_int32, P(ctypes.c_int64), ctypes.c_double,
      ctypes.c_uint64, P(sdd_config), P(sdd_config), P(ctypes.c_double)]),
    ("sdd_n_eval", ctypes.c_int32, [ctypes.c_void_p]),
    ("sdd_n_materials", ctypes.c_int32, [ctypes.c_void_p]),
    ("sdd_model_program", ctypes.c_int, [P(sdd_model_desc), P(ctypes.c_int32), P(ctypes.c_int32)]),
    ("sdd_plan_items", ctypes.c_int, [ctypes.c_int32, P(ctypes.c_int64), ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_uint32),
                                      P(ctypes.c_int32), P(ctypes.c_int32)]),
    ("sdd_status_str", ctypes.c_char_p, [ctypes.c_int]),
    ("sdd_last_error", ctypes.c_char_p, []),
]


def lib():
    """Load libsdd.so (built by ``paper_1603_09311_gb300.build``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libsdd.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(P(ctypes.c_double))


def make_desc(model: dict):
    """sdd_model_desc of a model dict, plus the arrays it points into."""
    kappa = np.ascontiguousarray(np.atleast_2d(np.asarray(model["kappa"], dtype=np.float64)))
    E, K = kappa.shape
    keep = [kappa]
    d = sdd_model_desc()
    dom = model["domain"]
    d.domain = sdd_domain(*[float(v) for v in dom])
    d.n_materials, d.n_eval = K, E
    d.kappa = _dp(kappa)
    bg = model.get("bg", (0, 1))
    d.bg_air, d.bg_earth = int(bg[0]), int(bg[1])
    shapes = model.get("shapes", [])
    if shapes:
        arr = (sdd_shape * len(shapes))()
        for i, (kind, mat, v) in enumerate(shapes):
            arr[i].kind, arr[i].material = int(kind), int(mat)
            vv = list(v) + [0.0] * (6 - len(v))
            for j in range(6):
                arr[i].v[j] = float(vv[j])
        keep.append(arr)
        d.shapes = ctypes.cast(arr, P(sdd_shape))
    d.n_shapes = len(shapes)
    raster = model.get("raster")
    if raster is not None:
        r = np.ascontiguousarray(raster, dtype=np.int8)
        keep.append(r)
        d.raster = r.ctypes.data_as(P(ctypes.c_int8))
        d.nz, d.nx = r.shape
    g = model.get("g", ("columns", 1, 1))
    if g[0] == "columns":
        d.g_kind, d.g_left, d.g_right = 0, int(g[1]), int(g[2])
    elif g[0] == "affine":
        d.g_kind = 1
        a, b, c = (complex(t) for t in g[1:4])
        for j, v in enumerate([a.real, a.imag, b.real, b.imag, c.real, c.imag]):
            d.g_coef[j] = v
    elif g[0] == "x2mz2":
        d.g_kind = 2
    elif g[0] == "tm_cosh":
        d.g_kind = 3
    elif g[0] == "tm_flux":
        d.g_kind = 4
    else:
        raise ValueError(f"unknown g kind {g[0]}")
    if "diffusion" in model:
        # TM mode: strips of their own diffusion between vertical interfaces
        dif = np.ascontiguousarray(np.asarray(model["diffusion"], dtype=np.float64))
        xif = np.ascontiguousarray(np.asarray(list(model.get("interfaces", [])) + [0.0], dtype=np.float64))
        keep += [dif, xif]
        d.diffusion = _dp(dif)
        d.interfaces = _dp(xif)
        d.n_shapes = 0
    return d, keep


def make_config(precision="fp32", max_steps=0, block_threads=0, ctas_per_sm=0, chunk_paths=0,
                use_graph=0, guided_factor=0):
    c = sdd_config()
    c.precision = SDD_FP64 if precision in ("fp64", SDD_FP64) else SDD_FP32
    c.max_steps, c.block_threads = int(max_steps), int(block_threads)
    c.ctas_per_sm, c.chunk_paths = int(ctas_per_sm), int(chunk_paths)
    c.use_graph, c.guided_factor = int(use_graph), int(guided_factor)
    return c


class Context:
    """Owns an sdd_ctx; closes it on close() or garbage collection."""

    def __init__(self, handle, E, K):
        self.handle, self.E, self.K = handle, E, K

    def close(self):
        if self.handle:
            lib().sdd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sdd_create(model: dict) -> Context:
    d, _keep = make_desc(model)
    h = ctypes.c_void_p()
    st = lib().sdd_create(ctypes.byref(d), ctypes.byref(h))
    if st != SDD_OK:
        raise SddError(st, "sdd_create")
    return Context(h, d.n_eval, d.n_materials)


# lookup programs of the single-precision walk (SDD_PROGRAM_* in include/sdd.h)
PROGRAMS = {0: "layers", 1: "rect", 2: "triangle", 3: "shapes4", 4: "shapes16", 5: "raster",
            6: "contact", 8: "tm"}


def sdd_model_program(model: dict):
    """The lookup program sdd_create would give the model (host only, no GPU):
    (program name, shape side) with side 0 earth, 1 air, -1 not a one-shape
    program."""
    d, _keep = make_desc(model)
    prog, side = ctypes.c_int32(), ctypes.c_int32()
    st = lib().sdd_model_program(ctypes.byref(d), ctypes.byref(prog), ctypes.byref(side))
    if st != SDD_OK:
        raise SddError(st, "sdd_model_program")
    return PROGRAMS[prog.value], side.value


def sdd_plan_items(n_paths, warps: int, guided_factor: int = 2, chunk_paths: int = 0):
    """The work items of one evaluation in queue order (host only, no GPU):
    arrays node, path0, count."""
    npth = np.ascontiguousarray(np.asarray(n_paths, dtype=np.int64).reshape(-1))
    n = ctypes.c_int32()
    args = (len(npth), npth.ctypes.data_as(P(ctypes.c_int64)), int(warps), int(guided_factor), int(chunk_paths))
    lib().sdd_plan_items(*args, 0, None, None, None, ctypes.byref(n))  # the number of items
    m = max(n.value, 1)
    node = np.zeros(m, dtype=np.int32)
    path0 = np.zeros(m, dtype=np.uint32)
    count = np.zeros(m, dtype=np.int32)
    st = lib().sdd_plan_items(*args, m, node.ctypes.data_as(P(ctypes.c_int32)),
                              path0.ctypes.data_as(P(ctypes.c_uint32)), count.ctypes.data_as(P(ctypes.c_int32)),
                              ctypes.byref(n))
    if st != SDD_OK:
        raise SddError(st, "sdd_plan_items")
    return node[:n.value], path0[:n.value], count[:n.value]


def sdd_destroy(ctx: Context) -> None:
    ctx.close()


def _paths(n_paths, n):
    npth = np.asarray(n_paths, dtype=np.int64)
    if npth.ndim == 0:
        npth = np.full(n, int(npth), dtype=np.int64)
    return np.ascontiguousarray(npth)


def sdd_interface_values(ctx: Context, nodes, n_paths, dt: float, seed: int, node_ids=None,
                         config: sdd_config | None = None, **cfg):
    """Host-buffer call.  Returns (mean complex [n][E], se [n][E][2], stats dict);
    raises SddError unless the status is SDD_OK or SDD_E_TRUNCATED."""
    nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64).reshape(-1, 2))
    n = nodes.shape[0]
    npth = _paths(n_paths, n)
    mean = np.zeros((n, ctx.E, 2))
    se = np.zeros((n, ctx.E, 2))
    st_out = sdd_stats()
    ids = None
    if node_ids is not None:
        ids = np.ascontiguousarray(np.asarray(node_ids, dtype=np.uint32))
    c = config if config is not None else make_config(**cfg)
    st = lib().sdd_interface_values(
        ctx.handle, _dp(nodes), None if ids is None else ids.ctypes.data_as(P(ctypes.c_uint32)),
        n, npth.ctypes.data_as(P(ctypes.c_int64)), float(dt), int(seed) & (2 ** 64 - 1),
        ctypes.byref(c), _dp(mean), _dp(se), ctypes.byref(st_out))
    if st not in (SDD_OK, SDD_E_TRUNCATED):
        raise SddError(st, "sdd_interface_values")
    stats = {f: getattr(st_out, f) for f, _ in sdd_stats._fields_}
    stats["status"] = st
    return mean[..., 0] + 1j * mean[..., 1], se, stats


def sdd_interface_values_target(ctx: Context, nodes, n_pilot: int, n_max: int, target_se: float,
                                dt: float, seed: int, node_ids=None,
                                config: sdd_config | None = None, **cfg):
    """Adaptive path counts: returns (mean complex [n][E], se [n][E][2],
    n_used [n], stats dict)."""
    nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64).reshape(-1, 2))
    n = nodes.shape[0]
    mean = np.zeros((n, ctx.E, 2))
    se = np.zeros((n, ctx.E, 2))
    used = np.zeros(n, dtype=np.int64)
    st_out = sdd_stats()
    ids = None if node_ids is None else np.ascontiguousarray(np.asarray(node_ids, dtype=np.uint32))
    c = config if config is not None else make_config(**cfg)
    st = lib().sdd_interface_values_target(
        ctx.handle, _dp(nodes), None if ids is None else ids.ctypes.data_as(P(ctypes.c_uint32)), n,
        int(n_pilot), int(n_max), float(target_se), float(dt), int(seed) & (2 ** 64 - 1),
        ctypes.byref(c), _dp(mean), _dp(se), used.ctypes.data_as(P(ctypes.c_int64)),
        ctypes.byref(st_out))
    if st not in (SDD_OK, SDD_E_TRUNCATED):
        raise SddError(st, "sdd_interface_values_target")
    stats = {f: getattr(st_out, f) for f, _ in sdd_stats._fields_}
    stats["status"] = st
    return mean[..., 0] + 1j * mean[..., 1], se, used, stats


def sdd_interface_values_device(ctx: Context, d_nodes_ptr: int, n_nodes: int, n_paths, dt: float,
                                seed: int, d_mean_ptr: int, d_se_ptr: int, d_node_ids_ptr: int = 0,
                                d_counters_ptr: int = 0, stream: int = 0,
                                config: sdd_config | None = None, **cfg) -> int:
    """Device-buffer call queued on `stream` (raw pointers, e.g. torch data_ptr())."""
    npth = _paths(n_paths, n_nodes)
    c = config if config is not None else make_config(**cfg)
    st = lib().sdd_interface_values_device(
        ctx.handle, ctypes.c_void_p(d_nodes_ptr), ctypes.c_void_p(d_node_ids_ptr or None), n_nodes,
        npth.ctypes.data_as(P(ctypes.c_int64)), float(dt), int(seed) & (2 ** 64 - 1),
        ctypes.byref(c), ctypes.c_void_p(d_mean_ptr), ctypes.c_void_p(d_se_ptr),
        ctypes.c_void_p(d_counters_ptr or None), ctypes.c_void_p(stream or None))
    if st != SDD_OK:
        raise SddError(st, "sdd_interface_values_device")
    return st


def sdd_interface_values_noalloc(ctx: Context, d_nodes_ptr: int, n_nodes: int, n_paths, dt: float,
                                 seed: int, d_mean_ptr: int, d_se_ptr: int, d_node_ids_ptr: int = 0,
                                 d_counters_ptr: int = 0, stream: int = 0,
                                 config: sdd_config | None = None, **cfg) -> int:
    """Like sdd_interface_values_device, for callers that cannot allocate
    device memory: the library's fixed scratch array replaces its per-call
    allocations (at most SDD_NOALLOC_MAX_NODES nodes per call; calls that
    overlap on the GPU race)."""
    npth = _paths(n_paths, n_nodes)
    c = config if config is not None else make_config(**cfg)
    st = lib().sdd_interface_values_noalloc(
        ctx.handle, ctypes.c_void_p(d_nodes_ptr), ctypes.c_void_p(d_node_ids_ptr or None), n_nodes,
        npth.ctypes.data_as(P(ctypes.c_int64)), float(dt), int(seed) & (2 ** 64 - 1),
        ctypes.byref(c), ctypes.c_void_p(d_mean_ptr), ctypes.c_void_p(d_se_ptr),
        ctypes.c_void_p(d_counters_ptr or None), ctypes.c_void_p(stream or None))
    if st != SDD_OK:
        raise SddError(st, "sdd_interface_values_noalloc")
    return st


class Request:
    """An sdd_request: poll(), wait(timeout_ms), cancel(), result(), free()."""

    def __init__(self, handle, n_nodes, E):
        self.handle, self.n, self.E = handle, n_nodes, E

    def poll(self) -> int:
        return lib().sdd_poll(self.handle)

    def wait(self, timeout_ms: int = -1) -> int:
        return lib().sdd_wait(self.handle, int(timeout_ms))

    def cancel(self) -> int:
        return lib().sdd_cancel(self.handle)

    def result(self):
        """(mean complex [n][E], se [n][E][2], stats dict); raises SddError unless
        the request ended with SDD_OK or SDD_E_TRUNCATED."""
        mean = np.zeros((self.n, self.E, 2))
        se = np.zeros((self.n, self.E, 2))
        st_out = sdd_stats()
        st = lib().sdd_request_result(self.handle, _dp(mean), _dp(se), ctypes.byref(st_out))
        if st not in (SDD_OK, SDD_E_TRUNCATED):
            raise SddError(st, "sdd_request_result")
        stats = {f: getattr(st_out, f) for f, _ in sdd_stats._fields_}
        stats["status"] = st
        return mean[..., 0] + 1j * mean[..., 1], se, stats

    def free(self):
        if self.handle:
            lib().sdd_request_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sdd_interface_values_async(ctx: Context, nodes, n_paths, dt: float, seed: int, node_ids=None, stream: int = 0,
                               config: sdd_config | None = None, **cfg) -> Request:
    """Queue an evaluation (inputs copied at once); returns a Request."""
    nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64).reshape(-1, 2))
    n = nodes.shape[0]
    npth = _paths(n_paths, n)
    ids = None if node_ids is None else np.ascontiguousarray(np.asarray(node_ids, dtype=np.uint32))
    c = config if config is not None else make_config(**cfg)
    h = ctypes.c_void_p()
    st = lib().sdd_interface_values_async(
        ctx.handle, _dp(nodes), None if ids is None else ids.ctypes.data_as(P(ctypes.c_uint32)), n,
        npth.ctypes.data_as(P(ctypes.c_int64)), float(dt), int(seed) & (2 ** 64 - 1), ctypes.byref(c),
        ctypes.c_void_p(stream or None), ctypes.byref(h))
    if st != SDD_OK:
        raise SddError(st, "sdd_interface_values_async")
    return Request(h, n, ctx.E)


def sdd_range_sums(ctx: Context, nodes, path_begin, path_count, dt: float, seed: int, node_ids=None,
                   config: sdd_config | None = None, **cfg):
    """Raw sums of path ranges (range i: paths [path_begin[i], +path_count[i]) of
    nodes[i]).  Returns (sums [n][E][4], n_valid [n], stats dict)."""
    nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64).reshape(-1, 2))
    n = nodes.shape[0]
    b = np.ascontiguousarray(np.asarray(path_begin, dtype=np.int64).reshape(n))
    c = np.ascontiguousarray(np.asarray(path_count, dtype=np.int64).reshape(n))
    ids = None if node_ids is None else np.ascontiguousarray(np.asarray(node_ids, dtype=np.uint32))
    sums = np.zeros((n, ctx.E, 4))
    nv = np.zeros(n, dtype=np.int64)
    st_out = sdd_stats()
    c_ = config if config is not None else make_config(**cfg)
    st = lib().sdd_range_sums(ctx.handle, _dp(nodes), None if ids is None else ids.ctypes.data_as(P(ctypes.c_uint32)),
                              n, b.ctypes.data_as(P(ctypes.c_int64)), c.ctypes.data_as(P(ctypes.c_int64)),
                              float(dt), int(seed) & (2 ** 64 - 1), ctypes.byref(c_), _dp(sums),
                              nv.ctypes.data_as(P(ctypes.c_int64)), ctypes.byref(st_out))
    if st not in (SDD_OK, SDD_E_TRUNCATED):
        raise SddError(st, "sdd_range_sums")
    stats = {f: getattr(st_out, f) for f, _ in sdd_stats._fields_}
    stats["status"] = st
    return sums, nv, stats


def sdd_range_sums_device(ctx: Context, d_nodes_ptr: int, n_ranges: int, path_begin, path_count, dt: float,
                          seed: int, d_sums_ptr: int, d_n_valid_ptr: int, d_node_ids_ptr: int = 0,
                          d_counters_ptr: int = 0, stream: int = 0, config: sdd_config | None = None, **cfg) -> int:
    """Device-buffer range sums queued on `stream` (raw pointers)."""
    b = np.ascontiguousarray(np.asarray(path_begin, dtype=np.int64).reshape(n_ranges))
    c = np.ascontiguousarray(np.asarray(path_count, dtype=np.int64).reshape(n_ranges))
    c_ = config if config is not None else make_config(**cfg)
    st = lib().sdd_range_sums_device(
        ctx.handle, ctypes.c_void_p(d_nodes_ptr), ctypes.c_void_p(d_node_ids_ptr or None), n_ranges,
        b.ctypes.data_as(P(ctypes.c_int64)), c.ctypes.data_as(P(ctypes.c_int64)), float(dt),
        int(seed) & (2 ** 64 - 1), ctypes.byref(c_), ctypes.c_void_p(d_sums_ptr), ctypes.c_void_p(d_n_valid_ptr),
        ctypes.c_void_p(d_counters_ptr or None), ctypes.c_void_p(stream or None))
    if st != SDD_OK:
        raise SddError(st, "sdd_range_sums_device")
    return st


def sdd_reduce_sums(ctx: Context, n_nodes: int, range_node, sums, n_valid):
    """Per-node mean (complex [n_nodes][E]) and se ([n_nodes][E][2]) from range sums,
    a node's ranges added in range order."""
    rn = np.ascontiguousarray(np.asarray(range_node, dtype=np.int32))
    sums = np.ascontiguousarray(np.asarray(sums, dtype=np.float64))
    nv = np.ascontiguousarray(np.asarray(n_valid, dtype=np.int64))
    mean = np.zeros((n_nodes, ctx.E, 2))
    se = np.zeros((n_nodes, ctx.E, 2))
    st = lib().sdd_reduce_sums(ctx.handle, int(n_nodes), len(rn), rn.ctypes.data_as(P(ctypes.c_int32)), _dp(sums),
                               nv.ctypes.data_as(P(ctypes.c_int64)), _dp(mean), _dp(se))
    if st != SDD_OK:
        raise SddError(st, "sdd_reduce_sums")
    return mean[..., 0] + 1j * mean[..., 1], se


def sdd_reduce_sums_device(ctx: Context, n_nodes: int, range_node, d_sums_ptr: int, d_n_valid_ptr: int,
                           d_mean_ptr: int, d_se_ptr: int, stream: int = 0) -> int:
    rn = np.ascontiguousarray(np.asarray(range_node, dtype=np.int32))
    st = lib().sdd_reduce_sums_device(ctx.handle, int(n_nodes), len(rn), rn.ctypes.data_as(P(ctypes.c_int32)),
                                      ctypes.c_void_p(d_sums_ptr), ctypes.c_void_p(d_n_valid_ptr),
                                      ctypes.c_void_p(d_mean_ptr), ctypes.c_void_p(d_se_ptr),
                                      ctypes.c_void_p(stream or None))
    if st != SDD_OK:
        raise SddError(st, "sdd_reduce_sums_device")
    return st


def sdd_batch_values(entries, dt: float, seed: int, config: sdd_config | None = None, **cfg):
    """One launch over several raster models.  entries: list of dicts with
    ctx, nodes, n_paths and optional node_ids.  Returns ([(mean, se)], stats)."""
    arr = (sdd_batch_entry * len(entries))()
    keep, outs = [], []
    for i, e in enumerate(entries):
        nodes = np.ascontiguousarray(np.asarray(e["nodes"], dtype=np.float64).reshape(-1, 2))
        n = nodes.shape[0]
        npth = _paths(e["n_paths"], n)
        mean = np.zeros((n, e["ctx"].E, 2))
        se = np.zeros((n, e["ctx"].E, 2))
        ids = e.get("node_ids")
        if ids is not None:
            ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint32))
        keep += [nodes, npth, ids]
        outs.append((mean, se))
        arr[i].ctx = e["ctx"].handle
        arr[i].nodes_xz = _dp(nodes)
        arr[i].node_ids = None if ids is None else ids.ctypes.data_as(P(ctypes.c_uint32))
        arr[i].n_nodes = n
        arr[i].n_paths = npth.ctypes.data_as(P(ctypes.c_int64))
        arr[i].mean = _dp(mean)
        arr[i].se = _dp(se)
    st_out = sdd_stats()
    c = config if config is not None else make_config(**cfg)
    st = lib().sdd_batch_values(arr, len(entries), float(dt), int(seed) & (2 ** 64 - 1),
                                ctypes.byref(c), ctypes.byref(st_out))
    if st not in (SDD_OK, SDD_E_TRUNCATED):
        raise SddError(st, "sdd_batch_values")
    stats = {f: getattr(st_out, f) for f, _ in sdd_stats._fields_}
    stats["status"] = st
    return [(m[..., 0] + 1j * m[..., 1], s_) for m, s_ in outs], stats


def sdd_walk_records(ctx: Context, x0: float, z0: float, node_id: int, p0: int, count: int,
                     dt: float, seed: int, config: sdd_config | None = None, **cfg):
    """Per-path records (steps, counts [count][K], exit [count][3], wall, m_last)."""
    steps = np.zeros(count, dtype=np.int64)
    counts = np.zeros((count, ctx.K), dtype=np.int64)
    ext = np.zeros((count, 3))
    wall = np.zeros(count, dtype=np.int32)
    mlast = np.zeros(count, dtype=np.int32)
    c = config if config is not None else make_config(**cfg)
    st = lib().sdd_walk_records(ctx.handle, float(x0), float(z0), int(node_id), int(p0), int(count),
                                float(dt), int(seed) & (2 ** 64 - 1), ctypes.byref(c),
                                steps.ctypes.data_as(P(ctypes.c_int64)),
                                counts.ctypes.data_as(P(ctypes.c_int64)), _dp(ext),
                                wall.ctypes.data_as(P(ctypes.c_int32)),
                                mlast.ctypes.data_as(P(ctypes.c_int32)))
    if st != SDD_OK:
        raise SddError(st, "sdd_walk_records")
    return {"steps": steps, "counts": counts, "exit": ext, "wall": wall, "m_last": mlast,
            "truncated": (wall < 0).astype(np.int32)}


def sdd_walk_occupation(ctx: Context, x0: float, z0: float, node_id: int, p0: int, count: int,
                        dt: float, seed: int, config: sdd_config | None = None, **cfg):
    """Per-path records with occupation times (TE and TM models): steps,
    occ [count][K] (units of dt), exit [count][3], wall, m_last, hits."""
    steps = np.zeros(count, dtype=np.int64)
    occ = np.zeros((count, ctx.K))
    ext = np.zeros((count, 3))
    wall = np.zeros(count, dtype=np.int32)
    mlast = np.zeros(count, dtype=np.int32)
    hits = np.zeros(count, dtype=np.int64)
    c = config if config is not None else make_config(**cfg)
    st = lib().sdd_walk_occupation(ctx.handle, float(x0), float(z0), int(node_id), int(p0), int(count),
                                   float(dt), int(seed) & (2 ** 64 - 1), ctypes.byref(c),
                                   steps.ctypes.data_as(P(ctypes.c_int64)), _dp(occ), _dp(ext),
                                   wall.ctypes.data_as(P(ctypes.c_int32)),
                                   mlast.ctypes.data_as(P(ctypes.c_int32)),
                                   hits.ctypes.data_as(P(ctypes.c_int64)))
    if st != SDD_OK:
        raise SddError(st, "sdd_walk_occupation")
    return {"steps": steps, "occ": occ, "exit": ext, "wall": wall, "m_last": mlast, "hits": hits,
            "truncated": (wall < 0).astype(np.int32)}


def sdd_interpolate(knots_s, values, se, targets_s, kind: int):
    """Interpolate knot data [n_knots][V] (and standard errors, or None) to
    targets_s.  Returns (values [n_targets][V], se [n_targets][V] or None)."""
    ks = np.ascontiguousarray(np.asarray(knots_s, dtype=np.float64))
    v = np.ascontiguousarray(np.asarray(values, dtype=np.float64).reshape(len(ks), -1))
    e = None if se is None else np.ascontiguousarray(np.asarray(se, dtype=np.float64).reshape(v.shape))
    t = np.ascontiguousarray(np.asarray(targets_s, dtype=np.float64).reshape(-1))
    ov = np.zeros((len(t), v.shape[1]))
    oe = None if e is None else np.zeros_like(ov)
    st = lib().sdd_interpolate(_dp(ks), len(ks), _dp(v), None if e is None else _dp(e), v.shape[1],
                               _dp(t), len(t), int(kind), _dp(ov), None if oe is None else _dp(oe))
    if st != SDD_OK:
        raise SddError(st, "sdd_interpolate")
    return ov, oe


def sdd_interface_values_interp(ctx: Context, nodes, stride: int, n_paths: int, kind: int, dt: float,
                                seed: int, config: sdd_config | None = None, **cfg):
    """Walks at every stride-th node of an interface polyline (and its last
    node), interpolation in arc length for the others.  Returns (mean complex
    [n][E], se [n][E][2], stats dict of the walks)."""
    nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64).reshape(-1, 2))
    n = nodes.shape[0]
    mean = np.zeros((n, ctx.E, 2))
    se = np.zeros((n, ctx.E, 2))
    st_out = sdd_stats()
    c = config if config is not None else make_config(**cfg)
    st = lib().sdd_interface_values_interp(ctx.handle, _dp(nodes), n, int(stride), int(n_paths), int(kind),
                                           float(dt), int(seed) & (2 ** 64 - 1), ctypes.byref(c),
                                           _dp(mean), _dp(se), ctypes.byref(st_out))
    if st not in (SDD_OK, SDD_E_TRUNCATED):
        raise SddError(st, "sdd_interface_values_interp")
    stats = {f: getattr(st_out, f) for f, _ in sdd_stats._fields_}
    stats["status"] = st
    return mean[..., 0] + 1j * mean[..., 1], se, stats


def sdd_apparent_resistivity(ctx: Context, sites, h: float, n_paths: int, kappa_ref, dt: float, seed: int,
                             config: sdd_config | None = None, **cfg):
    """Apparent resistivity (units of rho_ref) and phase (radians) at sites
    [n][2] from walks at (x, z0 - h), (x, z0), (x, z0 + h).  Returns a dict of
    rho, phase, rho_se, phase_se [n][E], u0, uz (complex [n][E]) and the
    walks' stats."""
    sites = np.ascontiguousarray(np.asarray(sites, dtype=np.float64).reshape(-1, 2))
    n = sites.shape[0]
    kr = np.ascontiguousarray(np.broadcast_to(np.asarray(kappa_ref, dtype=np.float64), (ctx.E,)))
    out = {k: np.zeros((n, ctx.E)) for k in ("rho", "phase", "rho_se", "phase_se")}
    u0 = np.zeros((n, ctx.E, 2))
    uz = np.zeros((n, ctx.E, 2))
    st_out = sdd_stats()
    c = config if config is not None else make_config(**cfg)
    st = lib().sdd_apparent_resistivity(ctx.handle, _dp(sites), n, float(h), int(n_paths), _dp(kr), float(dt),
                                        int(seed) & (2 ** 64 - 1), ctypes.byref(c), _dp(out["rho"]),
                                        _dp(out["phase"]), _dp(out["rho_se"]), _dp(out["phase_se"]), _dp(u0),
                                        _dp(uz), ctypes.byref(st_out))
    if st not in (SDD_OK, SDD_E_TRUNCATED):
        raise SddError(st, "sdd_apparent_resistivity")
    out["u0"] = u0[..., 0] + 1j * u0[..., 1]
    out["uz"] = uz[..., 0] + 1j * uz[..., 1]
    stats = {f: getattr(st_out, f) for f, _ in sdd_stats._fields_}
    stats["status"] = st
    out["stats"] = stats
    return out


def sdd_apparent_from_values(values, se, h: float, kappa_ref, d_site=None):
    """The resistivity arithmetic on given values (complex [n][3][E]) and
    standard errors ([n][3][E][2]); d_site [n] for TM, None for TE.  Returns
    the dict of sdd_apparent_resistivity without stats."""
    v = np.asarray(values, dtype=np.complex128)
    n, _, E = v.shape
    vv = np.ascontiguousarray(np.stack([v.real, v.imag], axis=-1))
    ee = np.ascontiguousarray(np.asarray(se, dtype=np.float64).reshape(n, 3, E, 2))
    kr = np.ascontiguousarray(np.broadcast_to(np.asarray(kappa_ref, dtype=np.float64), (E,)))
    ds = None if d_site is None else np.ascontiguousarray(np.asarray(d_site, dtype=np.float64).reshape(n))
    out = {k: np.zeros((n, E)) for k in ("rho", "phase", "rho_se", "phase_se")}
    u0 = np.zeros((n, E, 2))
    uz = np.zeros((n, E, 2))
    st = lib().sdd_apparent_from_values(_dp(vv), _dp(ee), n, E, float(h), _dp(kr), None if ds is None else _dp(ds),
                                        _dp(out["rho"]), _dp(out["phase"]), _dp(out["rho_se"]),
                                        _dp(out["phase_se"]), _dp(u0), _dp(uz))
    if st != SDD_OK:
        raise SddError(st, "sdd_apparent_from_values")
    out["u0"] = u0[..., 0] + 1j * u0[..., 1]
    out["uz"] = uz[..., 0] + 1j * uz[..., 1]
    return out


def sdd_rbffd_weights(nodes, n_stencil: int = 9, eps: float = 1.0):
    """Stencils [n][n_stencil] (int32) and Laplacian weights [n][n_stencil]."""
    p = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64).reshape(-1, 2))
    n = p.shape[0]
    st = np.zeros((n, n_stencil), dtype=np.int32)
    w = np.zeros((n, n_stencil))
    s = lib().sdd_rbffd_weights(_dp(p), n, int(n_stencil), float(eps), st.ctypes.data_as(P(ctypes.c_int32)),
                                _dp(w))
    if s != SDD_OK:
        raise SddError(s, "sdd_rbffd_weights")
    return st, w


def sdd_rbffd_solve(nodes, dirichlet, values, kappa, n_stencil: int = 9, eps: float = 1.0, tol: float = 1e-12,
                    max_iter: int = 20000, allow_unconverged: bool = False):
    """RBF-FD solution u (complex [n]) of Lap u = i kappa u with the values at
    Dirichlet nodes; returns (u, stats dict).  Raises SddError on
    SDD_E_TIMEOUT unless allow_unconverged."""
    p = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64).reshape(-1, 2))
    n = p.shape[0]
    fl = np.ascontiguousarray(np.asarray(dirichlet, dtype=np.uint8).reshape(n))
    v = np.asarray(values)
    if np.iscomplexobj(v) or v.shape == (n,):
        v = v.astype(np.complex128)
        v = np.stack([v.real, v.imag], axis=-1)
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(n, 2))
    k = np.ascontiguousarray(np.broadcast_to(np.asarray(kappa, dtype=np.float64), (n,)))
    u = np.zeros((n, 2))
    so = sdd_rbffd_stats()
    s = lib().sdd_rbffd_solve(_dp(p), n, fl.ctypes.data_as(P(ctypes.c_uint8)), _dp(v), _dp(k), int(n_stencil),
                              float(eps), float(tol), int(max_iter), _dp(u), ctypes.byref(so))
    stats = {f: getattr(so, f) for f, _ in sdd_rbffd_stats._fields_}
    stats["status"] = s
    if s != SDD_OK and not (allow_unconverged and s == SDD_E_TIMEOUT):
        raise SddError(s, "sdd_rbffd_solve")
    return u[:, 0] + 1j * u[:, 1], stats


def sdd_autotune(ctx: Context, nodes, n_paths, dt: float, seed: int, **base):
    """Time candidate launch shapes on this workload; the context keeps the
    fastest.  Returns ({block_threads, guided_factor}, walk-steps/s)."""
    nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64).reshape(-1, 2))
    npth = _paths(n_paths, nodes.shape[0])
    b = make_config(**base)
    out = sdd_config()
    rate = ctypes.c_double()
    st = lib().sdd_autotune(ctx.handle, _dp(nodes), nodes.shape[0], npth.ctypes.data_as(P(ctypes.c_int64)),
                            float(dt), int(seed) & (2 ** 64 - 1), ctypes.byref(b), ctypes.byref(out),
                            ctypes.byref(rate))
    if st != SDD_OK:
        raise SddError(st, "sdd_autotune")
    return {"block_threads": out.block_threads, "guided_factor": out.guided_factor}, rate.value


def sdd_status_str(status: int) -> str:
    return lib().sdd_status_str(status).decode()


def sdd_last_error() -> str:
    return lib().sdd_last_error().decode()


class Server:
    """A serving loop (sdd_server_*): admission, continuous batching into
    multi-model launches, completion.  Requests are raster models that match
    the server's domain, raster size, n_eval and g_kind."""

    def __init__(self, domain, nx, nz, dt, seed, n_eval=1, g_kind=0, max_requests=64, max_bytes=0,
                 n_streams=4, max_batch_models=64, max_batch_walks=0, **launch):
        c = sdd_server_config()
        c.domain = sdd_domain(*[float(v) for v in domain])
        c.nx, c.nz, c.n_eval, c.g_kind = int(nx), int(nz), int(n_eval), int(g_kind)
        c.max_requests, c.max_bytes = int(max_requests), int(max_bytes)
        c.n_streams, c.max_batch_models = int(n_streams), int(max_batch_models)
        c.max_batch_walks = int(max_batch_walks)
        c.dt, c.seed = float(dt), int(seed) & (2 ** 64 - 1)
        c.launch = make_config(**launch)
        self.n_eval = int(n_eval)
        self.handle = ctypes.c_void_p()
        st = lib().sdd_server_create(ctypes.byref(c), ctypes.byref(self.handle))
        if st != SDD_OK:
            raise SddError(st, "sdd_server_create")
        self.pending = {}

    def submit(self, model: dict, nodes, n_paths=None, target_se=0.0, n_pilot=0, n_max=0, node_ids=None):
        """Returns the request id, or None when the server refused it (SDD_E_BUSY)."""
        d, keep = make_desc(model)
        nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64).reshape(-1, 2))
        r = sdd_request_desc()
        r.model = ctypes.pointer(d)
        r.nodes_xz = _dp(nodes)
        r.n_nodes = nodes.shape[0]
        ids = None
        if node_ids is not None:
            ids = np.ascontiguousarray(np.asarray(node_ids, dtype=np.uint32))
            r.node_ids = ids.ctypes.data_as(P(ctypes.c_uint32))
        npth = None
        if n_paths is not None:
            npth = _paths(n_paths, nodes.shape[0])
            r.n_paths = npth.ctypes.data_as(P(ctypes.c_int64))
        r.target_se, r.n_pilot, r.n_max = float(target_se), int(n_pilot), int(n_max)
        rid = ctypes.c_uint64()
        st = lib().sdd_server_submit(self.handle, ctypes.byref(r), ctypes.byref(rid))
        if st == SDD_E_BUSY:
            return None
        if st != SDD_OK:
            raise SddError(st, "sdd_server_submit")
        self.pending[rid.value] = nodes.shape[0]
        return rid.value

    def poll(self, rid: int) -> bool:
        done = ctypes.c_int32()
        st = lib().sdd_server_poll(self.handle, rid, ctypes.byref(done))
        if st != SDD_OK:
            raise SddError(st, "sdd_server_poll")
        return bool(done.value)

    def wait(self, rid: int, timeout_ms: int = -1) -> bool:
        """True when finished, False on timeout."""
        st = lib().sdd_server_wait(self.handle, rid, int(timeout_ms))
        if st == SDD_E_TIMEOUT:
            return False
        if st != SDD_OK:
            raise SddError(st, "sdd_server_wait")
        return True

    def result(self, rid: int):
        """(status, mean complex [n][E], se [n][E][2], n_used [n], stats dict); frees the slot."""
        n = self.pending[rid]
        mean = np.zeros((n, self.n_eval, 2))
        se = np.zeros((n, self.n_eval, 2))
        used = np.zeros(n, dtype=np.int64)
        rs = sdd_request_stats()
        st = lib().sdd_server_result(self.handle, rid, _dp(mean), _dp(se),
                                     used.ctypes.data_as(P(ctypes.c_int64)), ctypes.byref(rs))
        if st == SDD_E_BUSY:
            raise SddError(st, "sdd_server_result")
        if st == SDD_E_ARG:
            raise SddError(st, "sdd_server_result")
        del self.pending[rid]
        stats = {f: getattr(rs, f) for f, _ in sdd_request_stats._fields_}
        return st, mean[..., 0] + 1j * mean[..., 1], se, used, stats

    def cancel(self, rid: int) -> None:
        st = lib().sdd_server_cancel(self.handle, rid)
        if st != SDD_OK:
            raise SddError(st, "sdd_server_cancel")

    def stats(self) -> dict:
        s = sdd_server_stats()
        st = lib().sdd_server_get_stats(self.handle, ctypes.byref(s))
        if st != SDD_OK:
            raise SddError(st, "sdd_server_get_stats")
        return {f: getattr(s, f) for f, _ in sdd_server_stats._fields_}

    def close(self):
        if self.handle:
            lib().sdd_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
