"""ctypes binding of the C ABI declared in include/ems.h (argument marshalling only).

Every computation runs in libems.so.  The library must have been built
(__graft_entry__.build() or paper_2604_10743_gb300.build.build()); a missing
library raises instead of falling back to anything else.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libems.so")

EMS_OK, EMS_E_INVAL, EMS_E_STATE, EMS_E_NOMEM, EMS_E_CUDA, EMS_E_NOCONV, EMS_E_TIMEOUT, \
    EMS_E_BREAKDOWN, EMS_E_OVERFLOW = range(9)
STATUS_NAMES = ["EMS_OK", "EMS_E_INVAL", "EMS_E_STATE", "EMS_E_NOMEM", "EMS_E_CUDA", "EMS_E_NOCONV",
                "EMS_E_TIMEOUT", "EMS_E_BREAKDOWN", "EMS_E_OVERFLOW"]
EMS_F64, EMS_F32 = 0, 1
EMS_BE, EMS_KRYLOV, EMS_AUTO = 0, 1, 2
EMS_PC_AUTO, EMS_PC_JACOBI = 0, 1

c_double_p = ctypes.POINTER(ctypes.c_double)
c_int32_p = ctypes.POINTER(ctypes.c_int32)
c_uint8_p = ctypes.POINTER(ctypes.c_uint8)


class EmsParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("e_charge", "k_B", "Omega", "rho_Cu", "B_modulus", "Z_star", "D0", "Ea", "Q_star",
                 "delta", "rho_Ta", "h_Ta", "sigma_T", "sigma_crit", "T0", "horizon")] + [
        ("n_outer", ctypes.c_int), ("n_inner", ctypes.c_int),
        ("ir_fail_frac", ctypes.c_double), ("Vdd", ctypes.c_double),
        ("precision", ctypes.c_int), ("method", ctypes.c_int), ("krylov_q", ctypes.c_int),
        ("krylov_eta", ctypes.c_double), ("ir_rtol", ctypes.c_double), ("ir_max_iter", ctypes.c_int),
        ("max_voids_per_tree", ctypes.c_int), ("ir_precond", ctypes.c_int),
        ("window_samples", ctypes.c_int), ("krylov_eps", ctypes.c_double)]


class EmsGridDesc(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int), ("node_x", c_double_p), ("node_y", c_double_p),
                ("n_seg", ctypes.c_int), ("seg_a", c_int32_p), ("seg_b", c_int32_p),
                ("seg_layer", c_int32_p), ("seg_cells", c_int32_p),
                ("seg_R0", c_double_p), ("seg_W", c_double_p), ("seg_H", c_double_p), ("seg_L", c_double_p),
                ("n_pads", ctypes.c_int), ("pad_node", c_int32_p), ("pad_V", c_double_p),
                ("n_sinks", ctypes.c_int), ("sink_node", c_int32_p), ("sink_I", c_double_p),
                ("n_samples", ctypes.c_int), ("kappa_factor", c_double_p), ("sigc_factor", c_double_p),
                ("seg_via", ctypes.POINTER(ctypes.c_int8))]


class EmsChainRule(ctypes.Structure):
    _fields_ = [("n_lo", ctypes.c_int64), ("n_hi", ctypes.c_int64), ("kind", ctypes.c_int), ("M", ctypes.c_int),
                ("CL", ctypes.c_int), ("T", ctypes.c_int)]


CHAIN_KINDS = {0: "default", 1: "global", 2: "shared", 3: "register", 4: "cluster", 5: "cluster_shared"}


class EmsSpiceOpts(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int), ("W", c_double_p), ("H", c_double_p), ("via_W", ctypes.c_double),
                ("via_H", ctypes.c_double), ("coord_unit", ctypes.c_double), ("dx", ctypes.c_double)]


class EmsTtfOpts(ctypes.Structure):
    _fields_ = [("screen", ctypes.c_int), ("n_outer", ctypes.c_int), ("no_graph", ctypes.c_int)]


class EmsTtfResult(ctypes.Structure):
    _fields_ = [("ttf", c_double_p), ("drop0", c_double_p), ("final_drop", c_double_p),
                ("n_voids", c_int32_p), ("n_mortal", c_int32_p), ("drops", c_double_p),
                ("node_steps", ctypes.c_double), ("stress_ms", ctypes.c_double), ("ir_ms", ctypes.c_double),
                ("ir_iterations", ctypes.c_double), ("ttf_mean", ctypes.c_double), ("ttf_std", ctypes.c_double),
                ("ttf_cov", ctypes.c_double), ("n_censored", ctypes.c_double), ("graph_launch", ctypes.c_double),
                ("node_steps_executed", ctypes.c_double)]


_LIB = None

EXPORTS = ["ems_workspace_bytes", "ems_create", "ems_destroy", "ems_last_error", "ems_load_grid", "ems_dims",
           "ems_set_thermal_map", "ems_ir_solve", "ems_immortality_check", "ems_stress_advance",
           "ems_krylov_reduce", "ems_void_update", "ems_ttf", "ems_get_sigma", "ems_get_currents",
           "ems_get_resistance", "ems_get_voids", "ems_state_export", "ems_state_import",
           "ems_launch_count", "ems_ir_iterations", "ems_ir_pcg_noalloc", "ems_joule_profile", "ems_set_wait_limit",
           "ems_get_node_temperature", "ems_set_thermal_perturbation", "ems_spice_parse", "ems_netlist_desc",
           "ems_netlist_error", "ems_netlist_free", "ems_chain_candidates", "ems_set_chain_rules",
           "ems_workspace_bytes_rules", "ems_autotune", "ems_autotune_log",
           # include/ems_surrogate.h
           "ems_mlp_create", "ems_mlp_destroy", "ems_mlp_last_error", "ems_mlp_param_count",
           "ems_mlp_set_params", "ems_mlp_get_params", "ems_mlp_set_norm", "ems_mlp_fit_norm", "ems_mlp_gradients",
           "ems_mlp_train_step", "ems_mlp_train", "ems_mlp_predict", "ems_gemm_bf16",
           "ems_surrogate_features", "ems_surrogate_targets", "ems_surrogate_schedule", "ems_surrogate_clear",
           "ems_surrogate_validate"]


def lib(path=None):
    """Load libems.so and declare every exported prototype."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libems.so not built (%s): run __graft_entry__.build()" % p)
    L = ctypes.CDLL(p)
    vp = ctypes.c_void_p
    S = ctypes.c_int
    L.ems_workspace_bytes.restype = ctypes.c_size_t
    L.ems_workspace_bytes.argtypes = [ctypes.POINTER(EmsParams), ctypes.POINTER(EmsGridDesc)]
    L.ems_create.restype = S
    L.ems_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(EmsParams), vp, vp, ctypes.c_size_t]
    L.ems_destroy.restype = S; L.ems_destroy.argtypes = [vp]
    L.ems_last_error.restype = ctypes.c_char_p; L.ems_last_error.argtypes = [vp]
    L.ems_load_grid.restype = S; L.ems_load_grid.argtypes = [vp, ctypes.POINTER(EmsGridDesc)]
    L.ems_dims.restype = S
    L.ems_dims.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64),
                           ctypes.POINTER(ctypes.c_int)]
    L.ems_set_thermal_map.restype = S
    L.ems_set_thermal_map.argtypes = [vp, c_double_p, S, S] + [ctypes.c_double] * 4
    L.ems_ir_solve.restype = S; L.ems_ir_solve.argtypes = [vp, c_double_p, c_double_p]
    L.ems_immortality_check.restype = S
    L.ems_immortality_check.argtypes = [vp, c_uint8_p, c_double_p, c_double_p]
    L.ems_stress_advance.restype = S
    L.ems_stress_advance.argtypes = [vp, ctypes.c_double, S, S, ctypes.POINTER(ctypes.c_int)]
    L.ems_krylov_reduce.restype = S
    L.ems_krylov_reduce.argtypes = [vp, S, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int)]
    L.ems_void_update.restype = S; L.ems_void_update.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.ems_ttf.restype = S
    L.ems_ttf.argtypes = [vp, ctypes.POINTER(EmsTtfOpts), ctypes.POINTER(EmsTtfResult)]
    L.ems_get_sigma.restype = S; L.ems_get_sigma.argtypes = [vp, c_double_p]
    L.ems_get_currents.restype = S; L.ems_get_currents.argtypes = [vp, c_double_p]
    L.ems_get_resistance.restype = S; L.ems_get_resistance.argtypes = [vp, c_double_p]
    L.ems_get_voids.restype = S
    L.ems_get_voids.argtypes = [vp, S, c_int32_p, c_int32_p, c_int32_p, c_double_p, c_double_p,
                                ctypes.POINTER(ctypes.c_int)]
    L.ems_state_export.restype = S
    L.ems_state_export.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
    L.ems_ir_iterations.restype = S
    L.ems_ir_iterations.argtypes = [vp, c_int32_p]
    L.ems_launch_count.restype = S
    L.ems_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    L.ems_state_import.restype = S
    L.ems_state_import.argtypes = [vp, vp, ctypes.c_size_t]
    L.ems_spice_parse.restype = S
    L.ems_spice_parse.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(EmsSpiceOpts), ctypes.POINTER(vp)]
    L.ems_netlist_desc.restype = S
    L.ems_netlist_desc.argtypes = [vp, ctypes.POINTER(EmsGridDesc)]
    L.ems_netlist_error.restype = ctypes.c_char_p
    L.ems_netlist_error.argtypes = [vp]
    L.ems_netlist_free.restype = None
    L.ems_netlist_free.argtypes = [vp]
    L.ems_set_thermal_perturbation.restype = S
    L.ems_set_thermal_perturbation.argtypes = [vp, c_double_p, S, S]
    L.ems_set_wait_limit.restype = S
    L.ems_set_wait_limit.argtypes = [vp, ctypes.c_longlong]
    rp = ctypes.POINTER(EmsChainRule)
    L.ems_chain_candidates.restype = S
    L.ems_chain_candidates.argtypes = [ctypes.c_int64, S, rp, S, ctypes.POINTER(ctypes.c_int)]
    L.ems_set_chain_rules.restype = S
    L.ems_set_chain_rules.argtypes = [vp, rp, S]
    L.ems_workspace_bytes_rules.restype = ctypes.c_size_t
    L.ems_workspace_bytes_rules.argtypes = [ctypes.POINTER(EmsParams), ctypes.POINTER(EmsGridDesc), rp, S]
    L.ems_autotune.restype = S
    L.ems_autotune.argtypes = [vp, S, S, rp, c_double_p, c_double_p, S, ctypes.POINTER(ctypes.c_int)]
    L.ems_autotune_log.restype = S
    L.ems_autotune_log.argtypes = [vp, S, rp, c_double_p, c_int32_p, ctypes.POINTER(ctypes.c_int)]
    L.ems_joule_profile.restype = S
    L.ems_joule_profile.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.ems_get_node_temperature.restype = S
    L.ems_get_node_temperature.argtypes = [vp, c_double_p]
    L.ems_ir_pcg_noalloc.restype = S
    L.ems_ir_pcg_noalloc.argtypes = [S, vp, vp, vp, vp, vp, ctypes.c_double, S, ctypes.POINTER(ctypes.c_int), vp]
    fp = ctypes.POINTER(ctypes.c_float)
    i64, u64, f32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_float
    for name, res, args in (
            ("ems_mlp_create", S, [S, u64, vp, ctypes.POINTER(vp)]),
            ("ems_mlp_destroy", None, [vp]),
            ("ems_mlp_last_error", ctypes.c_char_p, [vp]),
            ("ems_mlp_param_count", i64, [vp]),
            ("ems_mlp_set_params", S, [vp, fp]),
            ("ems_mlp_get_params", S, [vp, fp]),
            ("ems_mlp_set_norm", S, [vp, fp, fp, fp, fp]),
            ("ems_mlp_fit_norm", S, [vp, vp, vp, i64, ctypes.POINTER(ctypes.c_double)]),
            ("ems_mlp_gradients", S, [vp, vp, vp, S, fp, fp]),
            ("ems_mlp_train_step", S, [vp, vp, vp, S, f32, fp]),
            ("ems_mlp_train", S, [vp, vp, vp, i64, S, S, f32, u64, fp]),
            ("ems_mlp_predict", S, [vp, vp, i64, vp]),
            ("ems_gemm_bf16", S, [vp, vp, S, S, S, vp, S, f32, vp, vp, vp]),
            ("ems_surrogate_features", S, [vp, vp]),
            ("ems_surrogate_targets", S, [vp, ctypes.c_double, S, vp]),
            ("ems_surrogate_schedule", S, [vp, vp, ctypes.c_double, S, ctypes.c_double, c_int32_p, vp]),
            ("ems_surrogate_clear", S, [vp]),
            ("ems_surrogate_validate", S, [ctypes.POINTER(vp), S, vp, ctypes.POINTER(ctypes.c_double), S, S,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)])):
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _LIB = L
    return L


class EmsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, msg))
        self.status = status


def make_params(p, precision=EMS_F64, method=EMS_BE, ir_rtol=1e-13, ir_max_iter=20000, max_voids=16,
                ir_precond=0, window=0):
    """ems_params from a parameter dict (ems_synth.default_params())."""
    e = EmsParams()
    for name, _ in EmsParams._fields_:
        if name in p:
            setattr(e, name, p[name])
    e.precision = precision
    e.method = method
    e.krylov_q = int(p.get("krylov_q", 10))
    e.krylov_eta = float(p.get("krylov_eta", 1.0))
    e.ir_rtol = ir_rtol
    e.ir_max_iter = ir_max_iter
    e.max_voids_per_tree = max_voids
    e.ir_precond = ir_precond
    e.window_samples = int(window)
    e.krylov_eps = float(p.get("krylov_eps", 0.0))
    return e


def _ptr(a, t):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(t))


class GridDesc:
    """Keeps the contiguous arrays of a grid dict alive behind an EmsGridDesc."""

    def __init__(self, g):
        f64 = lambda k: np.ascontiguousarray(g[k], np.float64)
        i32 = lambda k: np.ascontiguousarray(g[k], np.int32)
        self.keep = {k: f64(k) for k in ("node_x", "node_y", "seg_R0", "seg_W", "seg_H", "seg_L", "pad_V",
                                         "sink_I")}
        self.keep.update({k: i32(k) for k in ("seg_a", "seg_b", "seg_layer", "seg_cells", "pad_node",
                                              "sink_node")})
        kf, sf = g.get("kappa_factor"), g.get("sigc_factor")
        S = 0
        if kf is not None or sf is not None:
            S = (kf if kf is not None else sf).shape[0]
        self.keep["kf"] = None if kf is None else np.ascontiguousarray(kf, np.float64)
        self.keep["sf"] = None if sf is None else np.ascontiguousarray(sf, np.float64)
        k = self.keep
        d = EmsGridDesc()
        d.n_nodes = k["node_x"].size; d.node_x = _ptr(k["node_x"], ctypes.c_double)
        d.node_y = _ptr(k["node_y"], ctypes.c_double)
        d.n_seg = k["seg_a"].size
        for n in ("seg_a", "seg_b", "seg_layer", "seg_cells", "pad_node", "sink_node"):
            setattr(d, n, _ptr(k[n], ctypes.c_int32))
        for n in ("seg_R0", "seg_W", "seg_H", "seg_L", "pad_V", "sink_I"):
            setattr(d, n, _ptr(k[n], ctypes.c_double))
        d.n_pads = k["pad_node"].size; d.n_sinks = k["sink_node"].size
        d.n_samples = S
        d.kappa_factor = _ptr(k["kf"], ctypes.c_double)
        d.sigc_factor = _ptr(k["sf"], ctypes.c_double)
        sv = g.get("seg_via")
        self.keep["via"] = None if sv is None else np.ascontiguousarray(sv, np.int8)
        d.seg_via = _ptr(self.keep["via"], ctypes.c_int8)
        self.desc = d
        self.n_samples = max(S, 1)


def rules_array(rules):
    """ems_chain_rule[] from a list of dicts (n_lo, n_hi, kind, M, CL)."""
    arr = (EmsChainRule * max(1, len(rules)))()
    for k, r in enumerate(rules):
        arr[k].n_lo, arr[k].n_hi = int(r["n_lo"]), int(r["n_hi"])
        arr[k].kind, arr[k].M, arr[k].CL = int(r["kind"]), int(r["M"]), int(r.get("CL", 1))
        arr[k].T = int(r.get("T", 0))
    return arr


def rule_dict(r):
    return {"n_lo": int(r.n_lo), "n_hi": int(r.n_hi), "kind": int(r.kind), "kernel": CHAIN_KINDS.get(r.kind, "?"),
            "M": int(r.M), "CL": int(r.CL), "T": int(r.T)}


def chain_candidates(n, precision):
    """Valid chain shapes for n nodes (ems_chain_candidates), built-in first."""
    L = lib()
    arr = (EmsChainRule * 32)()
    cnt = ctypes.c_int()
    st = L.ems_chain_candidates(int(n), int(precision), arr, 32, ctypes.byref(cnt))
    if st != 0:
        raise EmsError(st, "ems_chain_candidates")
    return [rule_dict(arr[k]) for k in range(cnt.value)]
