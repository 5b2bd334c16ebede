"""Host-side checks of the C ABI (no GPU): the library builds and loads,
exports every entry point declared in include/sdd.h, its struct layouts match
the ctypes binding, and argument errors are reported before any CUDA call."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1603_09311_gb300 import build as B
from paper_1603_09311_gb300 import inputs as I
from paper_1603_09311_gb300 import sdd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sdd.h")


@pytest.fixture(scope="module")
def L():
    B.build()
    return sdd.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sdd_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 8
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/sdd.h but not exported"
    bound = {s[0] for s in sdd.SIGNATURES}
    assert set(names) == bound, "binding and header disagree"
    nm = subprocess.run(["nm", "-D", "--defined-only", sdd.LIB_PATH], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}\b", nm), f"{n} is not a C (unmangled) export"


def test_struct_layout_matches_header(tmp_path):
    probe = tmp_path / "probe.c"
    probe.write_text(f'''
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu %zu %zu\\n", sizeof(sdd_model_desc), sizeof(sdd_shape), sizeof(sdd_config),
         sizeof(sdd_stats), sizeof(sdd_domain));
  printf("%zu %zu %zu %zu\\n", offsetof(sdd_model_desc, raster), offsetof(sdd_model_desc, g_coef),
         offsetof(sdd_config, chunk_paths), offsetof(sdd_stats, block));
  printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(sdd_server_config), offsetof(sdd_server_config, launch),
         sizeof(sdd_request_desc), offsetof(sdd_request_desc, n_max), sizeof(sdd_request_stats),
         sizeof(sdd_server_stats), sizeof(sdd_batch_entry));
  printf("%zu %zu %zu\\n", sizeof(sdd_rbffd_stats), offsetof(sdd_rbffd_stats, rel_residual),
         offsetof(sdd_stats, post_ms));
  return 0;
}}''')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", str(probe), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    want = [ctypes.sizeof(sdd.sdd_model_desc), ctypes.sizeof(sdd.sdd_shape),
            ctypes.sizeof(sdd.sdd_config), ctypes.sizeof(sdd.sdd_stats), ctypes.sizeof(sdd.sdd_domain),
            sdd.sdd_model_desc.raster.offset, sdd.sdd_model_desc.g_coef.offset,
            sdd.sdd_config.chunk_paths.offset, sdd.sdd_stats.block.offset,
            ctypes.sizeof(sdd.sdd_server_config), sdd.sdd_server_config.launch.offset,
            ctypes.sizeof(sdd.sdd_request_desc), sdd.sdd_request_desc.n_max.offset,
            ctypes.sizeof(sdd.sdd_request_stats), ctypes.sizeof(sdd.sdd_server_stats),
            ctypes.sizeof(sdd.sdd_batch_entry),
            ctypes.sizeof(sdd.sdd_rbffd_stats), sdd.sdd_rbffd_stats.rel_residual.offset,
            sdd.sdd_stats.post_ms.offset]
    assert [int(v) for v in out] == want


def test_status_strings(L):
    for s in range(9):
        assert sdd.sdd_status_str(s)
    assert "unknown" in sdd.sdd_status_str(99)


@pytest.mark.parametrize("mutate,msg", [
    (lambda m: m.update(kappa=[[0.0, -1.0]]), "kappa"),
    (lambda m: m.update(kappa=[[0.0, float("nan")]]), "kappa"),
    (lambda m: m.update(domain=(1.0, -1.0, 0.0, 1.0)), "domain"),
    (lambda m: m.update(bg=(0, 5)), "background"),
    (lambda m: m.update(shapes=[(0, 7, (0, 1, 0, 1, 0, 0))]), "shape material"),
    (lambda m: m.update(shapes=[(3, 1, (0, 1, 0, 1, 0, 0))]), "shape kind"),
    (lambda m: m.update(g=("columns", 0, 9)), "g_left"),
    (lambda m: m.update(kappa=np.zeros((33, 2))), "n_eval"),
    (lambda m: m.update(kappa=np.zeros((1, 9))), "n_materials"),
    (lambda m: m.update(raster=np.full((4, 4), 3, dtype=np.int8)), "raster"),
    (lambda m: m.update(raster=np.zeros((1, (1 << 20) + 1), dtype=np.int8)), "raster size"),
])
def test_bad_models_are_rejected_before_any_cuda_call(L, mutate, msg):
    m = I.halfspace(2.0)
    mutate(m)
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_create(m)
    assert e.value.status == sdd.SDD_E_ARG
    assert msg in str(e.value)


def test_null_context_is_an_argument_error(L):
    n = np.zeros(2)
    p = np.ones(1, dtype=np.int64)
    st = L.sdd_interface_values(None, n.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, 1,
                                p.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 1e-3, 0, None,
                                None, None, None)
    assert st == sdd.SDD_E_ARG
    L.sdd_destroy(None)  # allowed


@pytest.mark.parametrize("case,msg", [
    ("kind", "kind must be"),
    ("one_knot", "n_knots must be at least 2"),
    ("not_increasing", "strictly increasing"),
    ("nan_knot", "finite"),
    ("target_outside", "targets must lie within"),
    ("spline_too_many", "SDD_INTERP_MAX_SPLINE_KNOTS"),
    ("no_values", "must not be NULL"),
])
def test_interpolate_arguments_rejected_before_any_cuda_call(L, case, msg):
    k = np.array([0.0, 0.5, 1.0])
    kind = sdd.SDD_INTERP_LINEAR
    v = np.zeros((3, 2))
    t = np.array([0.25])
    if case == "kind":
        kind = 7
    elif case == "one_knot":
        k = k[:1]
    elif case == "not_increasing":
        k = np.array([0.0, 0.5, 0.5])
    elif case == "nan_knot":
        k = np.array([0.0, np.nan, 1.0])
    elif case == "target_outside":
        t = np.array([1.5])
    elif case == "spline_too_many":
        kind = sdd.SDD_INTERP_SPLINE
        k = np.linspace(0, 1, sdd.SDD_INTERP_MAX_SPLINE_KNOTS + 1)
        v = np.zeros((len(k), 2))
    if case == "no_values":
        with pytest.raises(sdd.SddError) as e:
            dp = ctypes.POINTER(ctypes.c_double)
            st = L.sdd_interpolate(k.ctypes.data_as(dp), 3, None, None, 2, t.ctypes.data_as(dp), 1, 0,
                                   None, None)
            raise sdd.SddError(st, "sdd_interpolate")
    else:
        with pytest.raises(sdd.SddError) as e:
            sdd.sdd_interpolate(k, v, None, t, kind)
    assert e.value.status == sdd.SDD_E_ARG
    assert msg in sdd.sdd_last_error()


def test_interpolate_without_targets_does_nothing(L):
    v, e = sdd.sdd_interpolate([0.0, 1.0], np.ones((2, 3)), None, np.zeros(0), sdd.SDD_INTERP_SPLINE)
    assert v.shape == (0, 3) and e is None


def test_interface_interp_null_context(L):
    dp = ctypes.POINTER(ctypes.c_double)
    n = np.zeros(4)
    st = L.sdd_interface_values_interp(None, n.ctypes.data_as(dp), 2, 1, 10, 0, 1e-3, 0, None, None,
                                       None, None)
    assert st == sdd.SDD_E_ARG


def test_apparent_resistivity_null_context(L):
    dp = ctypes.POINTER(ctypes.c_double)
    s = np.zeros(2)
    k = np.ones(1)
    st = L.sdd_apparent_resistivity(None, s.ctypes.data_as(dp), 1, 0.05, 10, k.ctypes.data_as(dp), 1e-3, 0,
                                    None, None, None, None, None, None, None, None)
    assert st == sdd.SDD_E_ARG
    assert "ctx" in sdd.sdd_last_error()


@pytest.mark.parametrize("case,msg", [
    ("stencil", "n_stencil"),
    ("few_nodes", "n must be in"),
    ("eps", "eps"),
    ("nan", "finite"),
])
def test_rbffd_weights_arguments_rejected_before_any_cuda_call(L, case, msg):
    nodes, _ = I.rect_grid(0, 1, 0, 1, 4, 4)
    ns, eps = 9, 1.0
    if case == "stencil":
        ns = 17
    elif case == "few_nodes":
        nodes = nodes[:5]
    elif case == "eps":
        eps = 0.0
    elif case == "nan":
        nodes = nodes.copy()
        nodes[3, 0] = np.nan
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_rbffd_weights(nodes, ns, eps)
    assert e.value.status == sdd.SDD_E_ARG
    assert msg in sdd.sdd_last_error()


@pytest.mark.parametrize("case,msg", [
    ("tol", "tol"),
    ("iters", "max_iter"),
    ("flag", "dirichlet flags"),
    ("kappa", "kappa"),
])
def test_rbffd_solve_arguments_rejected_before_any_cuda_call(L, case, msg):
    nodes, edge = I.rect_grid(0, 1, 0, 1, 4, 4)
    vals = np.zeros((16, 2))
    kap = np.ones(16)
    tol, iters = 1e-10, 100
    if case == "tol":
        tol = -1.0
    elif case == "iters":
        iters = 0
    elif case == "flag":
        edge = edge.copy()
        edge[5] = 2
    elif case == "kappa":
        kap[2] = np.inf
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_rbffd_solve(nodes, edge, vals, kap, tol=tol, max_iter=iters)
    assert e.value.status == sdd.SDD_E_ARG
    assert msg in sdd.sdd_last_error()


def test_rbffd_solve_all_dirichlet_needs_no_gpu(L):
    nodes, _ = I.rect_grid(0, 1, 0, 1, 4, 4)
    vals = np.arange(32, dtype=float).reshape(16, 2)
    u, st = sdd.sdd_rbffd_solve(nodes, np.ones(16, dtype=np.uint8), vals, np.ones(16))
    np.testing.assert_array_equal(u, vals[:, 0] + 1j * vals[:, 1])
    assert st["unknowns"] == 0
