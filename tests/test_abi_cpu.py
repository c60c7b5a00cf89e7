"""CPU-side checks of the C ABI: the library loads, exports every function
include/ems.h declares, and rejects invalid inputs in host code (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import ems_synth as es

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2604_10743_gb300 import build as B
    from paper_2604_10743_gb300 import _abi as A
    B.build()
    return A.lib()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(ems_[a-z_0-9]+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(L):
    from paper_2604_10743_gb300 import _abi as A
    decl = _declared()
    assert "ems_stress_advance" in decl and "ems_ttf" in decl
    for name in decl:
        assert hasattr(L, name), name
    assert decl == set(A.EXPORTS)


def _ws(L, g, **kw):
    from paper_2604_10743_gb300 import _abi as A
    prm = A.make_params(es.default_params(), **kw)
    gd = A.GridDesc(g)
    return L.ems_workspace_bytes(ctypes.byref(prm), ctypes.byref(gd.desc))


def test_workspace_sizes(L):
    small = _ws(L, es.tiny_grid())
    assert small > 0
    assert _ws(L, es.mc_grid(n_samples=4)) > small


def test_rejects_cycle(L):
    g = es.stripe_mesh(2, 10e-6)
    g["seg_layer"][:] = 0
    g["pad_node"] = np.array([0], np.int32); g["pad_V"] = np.ones(1)
    assert _ws(L, g) == 0


def test_rejects_nan_current_and_bad_geometry(L):
    g = es.tiny_grid()
    g["sink_I"] = g["sink_I"].copy(); g["sink_I"][3] = np.nan
    assert _ws(L, g) == 0
    g = es.tiny_grid()
    g["seg_L"] = g["seg_L"].copy(); g["seg_L"][0] = -1.0
    assert _ws(L, g) == 0


def test_rejects_island(L):
    g = es.tiny_grid()
    # an extra node linked to nothing
    g["node_x"] = np.append(g["node_x"], 1.0); g["node_y"] = np.append(g["node_y"], 1.0)
    assert _ws(L, g) == 0


def test_rejects_bad_params(L):
    from paper_2604_10743_gb300 import _abi as A
    prm = A.make_params(es.default_params(sigma_crit=-1.0))
    gd = A.GridDesc(es.tiny_grid())
    assert L.ems_workspace_bytes(ctypes.byref(prm), ctypes.byref(gd.desc)) == 0
    prm = A.make_params(es.default_params(), max_voids=0)
    assert L.ems_workspace_bytes(ctypes.byref(prm), ctypes.byref(gd.desc)) == 0


def test_branched_trees_accepted(L):
    for kind in ("T", "comb", "star", "chain"):
        assert _ws(L, es.tree_grid(kind)) > 0


def test_null_context_calls_fail_cleanly(L):
    assert L.ems_ir_solve(None, None, None) == 1       # EMS_E_INVAL
    assert L.ems_destroy(None) == 1


def test_surrogate_calls_reject_bad_arguments_without_a_device(L):
    import ctypes
    h = ctypes.c_void_p()
    assert L.ems_mlp_create(0, 0, None, ctypes.byref(h)) == 1          # n_hidden out of range
    assert L.ems_mlp_create(9, 0, None, ctypes.byref(h)) == 1
    assert L.ems_mlp_create(4, 0, None, None) == 1
    assert L.ems_mlp_param_count(None) == 0
    for M, N, K in ((0, 16, 64), (8, 8, 64), (8, 264, 64), (8, 24, 64), (8, 16, 32), (8, 16, 100)):
        assert L.ems_gemm_bf16(ctypes.c_void_p(256), ctypes.c_void_p(256), M, N, K, None, 0, 1.0,
                               None, None, None) == 1
    assert L.ems_surrogate_features(None, None) == 1
    assert L.ems_surrogate_targets(None, 10.0, 0, None) == 1
    assert L.ems_surrogate_schedule(None, None, 0.1, 16, 0.8, None, None) == 1
    assert L.ems_surrogate_clear(None) == 1
    b = ctypes.c_double()
    cand = (ctypes.c_double * 2)(0.0, 0.5)
    assert L.ems_surrogate_validate(None, 1, None, cand, 2, 16, 0.8, 5e-4, 0.1, ctypes.byref(b), None) == 1
    ctxs = (ctypes.c_void_p * 1)(None)
    assert L.ems_surrogate_validate(ctxs, 1, ctypes.c_void_p(8), cand, 2, 1, 0.8, 5e-4, 0.1,
                                    ctypes.byref(b), None) == 1                    # coarsen < 2
    assert L.ems_surrogate_validate(ctxs, 1, ctypes.c_void_p(8), cand, 2, 16, 1.5, 5e-4, 0.1,
                                    ctypes.byref(b), None) == 1                    # guard > 1
    assert L.ems_surrogate_validate(ctxs, 1, ctypes.c_void_p(8), cand, 2, 16, 0.8, 5e-4, 0.1,
                                    ctypes.byref(b), None) == 1                    # null context


def test_window_layout_sizes(L):
    """Monte Carlo windows: the per-sample part of the workspace shrinks to
    the state (stress, resistances, voltages, factors, voids) and the
    per-node coefficients are held for W samples only; the reduced models
    need the full layout."""
    g = es.mc_grid(n_samples=64)
    full = _ws(L, g)
    w8 = _ws(L, g, window=8)
    w64 = _ws(L, g, window=64)
    assert 0 < w8 < full and w64 == full and _ws(L, g, window=0) == full
    assert _ws(L, g, window=-1) == 0
    from paper_2604_10743_gb300 import _abi as A
    assert _ws(L, g, window=8, method=A.EMS_KRYLOV) == 0
    assert _ws(L, g, window=64, method=A.EMS_KRYLOV) > 0
    # growth per extra sample with windows: state only (well under the
    # full layout's per-sample coefficient arrays)
    g2 = es.mc_grid(n_samples=128)
    per_full = (_ws(L, g2) - full) / 64
    per_win = (_ws(L, g2, window=8) - w8) / 64
    assert per_win < 0.25 * per_full
