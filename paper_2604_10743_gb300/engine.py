"""Python face of the C ABI: one Engine per loaded grid.

PyTorch provides the device workspace (a uint8 tensor) and the CUDA stream;
every step of the EM/TM path runs inside libems.so.  Method names follow the
ABI calls (ems_ir_solve -> Engine.ir_solve, ...).
"""
import ctypes

import numpy as np

from . import _abi as A


class Engine:
    def __init__(self, params, grid, precision=A.EMS_F64, method=A.EMS_BE, ir_rtol=1e-13,
                 ir_max_iter=20000, max_voids=16, workspace="torch", stream=None, thermal=True,
                 ir_precond=A.EMS_PC_AUTO, window=0, chain_rules=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Engine needs a CUDA device")
        self.L = A.lib()
        self.p = dict(params)
        self.prm = A.make_params(params, precision, method, ir_rtol, ir_max_iter, max_voids, ir_precond, window)
        self.gd = A.GridDesc(grid)
        self.S = self.gd.n_samples
        self.chain_rules = list(chain_rules or [])
        self._rules = A.rules_array(self.chain_rules)
        nbytes = self.L.ems_workspace_bytes_rules(ctypes.byref(self.prm), ctypes.byref(self.gd.desc), self._rules,
                                                  len(self.chain_rules))
        if nbytes == 0:
            raise A.EmsError(A.EMS_E_INVAL, "invalid grid or parameters (ems_workspace_bytes returned 0)")
        self.ws_bytes = int(nbytes)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        if workspace == "torch":
            self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device="cuda")
            base = (self.ws.data_ptr() + 255) // 256 * 256
        else:
            self.ws = None
            base = None
        ctx = ctypes.c_void_p()
        self._check(self.L.ems_create(ctypes.byref(ctx), ctypes.byref(self.prm),
                                      ctypes.c_void_p(stream.cuda_stream), ctypes.c_void_p(base),
                                      ctypes.c_size_t(self.ws_bytes)), None)
        self.ctx = ctx
        if self.chain_rules:
            self._check(self.L.ems_set_chain_rules(self.ctx, self._rules, len(self.chain_rules)))
        self._check(self.L.ems_load_grid(self.ctx, ctypes.byref(self.gd.desc)))
        nt = ctypes.c_int(); nn = ctypes.c_int64(); ns = ctypes.c_int()
        self._check(self.L.ems_dims(self.ctx, ctypes.byref(nt), ctypes.byref(nn), ctypes.byref(ns)))
        self.n_trees, self.n_stress, self.S = nt.value, nn.value, ns.value
        self.n_nodes = self.gd.desc.n_nodes
        self.n_seg = self.gd.desc.n_seg
        th = grid.get("thermal") if thermal else None
        if th is not None:
            self.set_thermal_map(th)

    # -- plumbing -----------------------------------------------------------
    def _check(self, st, ctx="self"):
        if st != A.EMS_OK:
            msg = self.L.ems_last_error(self.ctx if ctx == "self" else None)
            raise A.EmsError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "ctx", None):
            self.L.ems_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- ABI calls ----------------------------------------------------------
    def set_thermal_map(self, th):
        if th is None:
            return self._check(self.L.ems_set_thermal_map(self.ctx, None, 0, 0, 0.0, 0.0, 0.0, 0.0))
        T = np.ascontiguousarray(th["T"], np.float64)
        ny, nx = T.shape
        self._check(self.L.ems_set_thermal_map(self.ctx, T.ctypes.data_as(A.c_double_p), nx, ny,
                                               th["x0"], th["y0"], th["x1"], th["y1"]))

    def set_thermal_perturbation(self, dT):
        """Per-sample temperature perturbation rasters [S, ny, nx] over the
        map's extent (ems_set_thermal_perturbation); None removes them."""
        if dT is None:
            return self._check(self.L.ems_set_thermal_perturbation(self.ctx, None, 0, 0))
        dT = np.ascontiguousarray(dT, np.float64)
        S, ny, nx = dT.shape
        if S != self.S:
            raise ValueError("one perturbation raster per sample")
        self._check(self.L.ems_set_thermal_perturbation(self.ctx, dT.ctypes.data_as(A.c_double_p), nx, ny))

    def joule_profile(self, k_cu=400.0, k_ild=1.4, t_ild=0.2e-6):
        """Joule-heating temperature profile along every branch (ems_joule_profile)."""
        self._check(self.L.ems_joule_profile(self.ctx, float(k_cu), float(k_ild), float(t_ild)))

    def node_temperature(self):
        T = np.empty(self.n_stress)
        self._check(self.L.ems_get_node_temperature(self.ctx, T.ctypes.data_as(A.c_double_p)))
        return T

    def ir_solve(self):
        u = np.empty((self.S, self.n_nodes)); d = np.empty(self.S)
        self._check(self.L.ems_ir_solve(self.ctx, u.ctypes.data_as(A.c_double_p), d.ctypes.data_as(A.c_double_p)))
        return u, d

    def immortality_check(self, want_sigma=False):
        m = np.empty((self.S, self.n_trees), np.uint8); mx = np.empty((self.S, self.n_trees))
        ss = np.empty((self.S, self.n_stress)) if want_sigma else None
        self._check(self.L.ems_immortality_check(self.ctx, m.ctypes.data_as(A.c_uint8_p),
                                                 mx.ctypes.data_as(A.c_double_p),
                                                 None if ss is None else ss.ctypes.data_as(A.c_double_p)))
        return m.astype(bool), mx, ss

    def stress_advance(self, dt, n_steps, method=A.EMS_BE):
        nv = ctypes.c_int()
        self._check(self.L.ems_stress_advance(self.ctx, float(dt), int(n_steps), int(method), ctypes.byref(nv)))
        return nv.value

    def autotune(self, n_steps=32, max_samples=2):
        """Time every valid chain shape of each launch group on scratch copies
        (ems_autotune); the context is unchanged.  Returns one rule per group
        with its time (ms) and the current shape's (ms_default)."""
        cap = 256
        arr = (A.EmsChainRule * cap)()
        ms = np.zeros(cap); md = np.zeros(cap)
        k = ctypes.c_int()
        self._check(self.L.ems_autotune(self.ctx, int(n_steps), int(max_samples), arr,
                                        ms.ctypes.data_as(A.c_double_p), md.ctypes.data_as(A.c_double_p), cap,
                                        ctypes.byref(k)))
        out = []
        for i in range(k.value):
            r = A.rule_dict(arr[i])
            r["ms"], r["ms_default"] = float(ms[i]), float(md[i])
            out.append(r)
        return out

    def autotune_log(self):
        """Every shape the last autotune timed: dicts with ms (-1: not
        launchable) and the group index."""
        n = ctypes.c_int()
        self._check(self.L.ems_autotune_log(self.ctx, 0, None, None, None, ctypes.byref(n)))
        cap = max(1, n.value)
        arr = (A.EmsChainRule * cap)()
        ms = np.zeros(cap); grp = np.zeros(cap, np.int32)
        self._check(self.L.ems_autotune_log(self.ctx, cap, arr, ms.ctypes.data_as(A.c_double_p),
                                            grp.ctypes.data_as(A.c_int32_p), ctypes.byref(n)))
        out = []
        for i in range(n.value):
            r = A.rule_dict(arr[i])
            r["ms"], r["group"] = float(ms[i]), int(grp[i])
            out.append(r)
        return out

    def krylov_reduce(self, q, eta=1.0):
        nr = ctypes.c_int(); nf = ctypes.c_int()
        self._check(self.L.ems_krylov_reduce(self.ctx, int(q), float(eta), ctypes.byref(nr), ctypes.byref(nf)))
        return nr.value, nf.value

    def void_update(self):
        n = ctypes.c_int()
        self._check(self.L.ems_void_update(self.ctx, ctypes.byref(n)))
        return n.value

    def ttf(self, screen=False, n_outer=0, graph=True):
        S = self.S
        nout = n_outer if n_outer > 0 else int(self.p["n_outer"])
        ttf = np.empty(S); d0 = np.empty(S); fd = np.empty(S)
        nv = np.empty(S, np.int32); nm = np.zeros(S, np.int32); drops = np.empty((S, nout + 1))
        r = A.EmsTtfResult()
        r.ttf = ttf.ctypes.data_as(A.c_double_p); r.drop0 = d0.ctypes.data_as(A.c_double_p)
        r.final_drop = fd.ctypes.data_as(A.c_double_p); r.n_voids = nv.ctypes.data_as(A.c_int32_p)
        r.n_mortal = nm.ctypes.data_as(A.c_int32_p); r.drops = drops.ctypes.data_as(A.c_double_p)
        o = A.EmsTtfOpts(); o.screen = 1 if screen else 0; o.n_outer = int(n_outer)
        o.no_graph = 0 if graph else 1
        self._check(self.L.ems_ttf(self.ctx, ctypes.byref(o), ctypes.byref(r)))
        return dict(ttf=ttf, drop0=d0, final_drop=fd, n_voids=nv, n_mortal=nm, drops=drops,
                    node_steps=r.node_steps, stress_ms=r.stress_ms, ir_ms=r.ir_ms,
                    ir_iterations=r.ir_iterations, ttf_mean=r.ttf_mean, ttf_std=r.ttf_std,
                    ttf_cov=r.ttf_cov, n_censored=int(r.n_censored), graph=bool(r.graph_launch),
                    node_steps_executed=r.node_steps_executed)

    def sigma(self):
        s = np.empty((self.S, self.n_stress))
        self._check(self.L.ems_get_sigma(self.ctx, s.ctypes.data_as(A.c_double_p)))
        return s

    def currents(self):
        j = np.empty((self.S, self.n_seg))
        self._check(self.L.ems_get_currents(self.ctx, j.ctypes.data_as(A.c_double_p)))
        return j

    def resistance(self):
        R = np.empty((self.S, self.n_seg))
        self._check(self.L.ems_get_resistance(self.ctx, R.ctypes.data_as(A.c_double_p)))
        return R

    def voids(self):
        n = ctypes.c_int()
        self._check(self.L.ems_get_voids(self.ctx, 0, None, None, None, None, None, ctypes.byref(n)))
        k = n.value
        smp = np.empty(k, np.int32); node = np.empty(k, np.int32); seg = np.empty(k, np.int32)
        vol = np.empty(k); tn = np.empty(k)
        self._check(self.L.ems_get_voids(self.ctx, k, smp.ctypes.data_as(A.c_int32_p),
                                         node.ctypes.data_as(A.c_int32_p), seg.ctypes.data_as(A.c_int32_p),
                                         vol.ctypes.data_as(A.c_double_p), tn.ctypes.data_as(A.c_double_p),
                                         ctypes.byref(n)))
        return dict(sample=smp, node=node, seg=seg, volume=vol, t_nuc=tn)

    def set_wait_limit(self, polls):
        self._check(self.L.ems_set_wait_limit(self.ctx, int(polls)))

    def ir_iterations(self):
        it = np.empty(self.S, np.int32)
        self._check(self.L.ems_ir_iterations(self.ctx, it.ctypes.data_as(A.c_int32_p)))
        return it

    def launch_count(self):
        n = ctypes.c_int64()
        self._check(self.L.ems_launch_count(self.ctx, ctypes.byref(n)))
        return n.value

    def state_export(self):
        nb = ctypes.c_size_t()
        self._check(self.L.ems_state_export(self.ctx, None, ctypes.byref(nb)))
        buf = np.empty(nb.value, np.uint8)
        self._check(self.L.ems_state_export(self.ctx, buf.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nb)))
        return buf

    def state_import(self, buf):
        buf = np.ascontiguousarray(buf, np.uint8)
        self._check(self.L.ems_state_import(self.ctx, buf.ctypes.data_as(ctypes.c_void_p), buf.size))

    # -- learned surrogate (include/ems_surrogate.h) ------------------------
    def features(self):
        """[S * n_trees, 24] float32 device tensor of the current features."""
        import torch
        x = torch.empty((self.S * self.n_trees, 24), dtype=torch.float32, device="cuda")
        self._check(self.L.ems_surrogate_features(self.ctx, ctypes.c_void_p(x.data_ptr())))
        return x

    def targets(self, t_cap, freeze=False):
        """[S * n_trees, 2] float32 device tensor (log10 t_nuc, node position)."""
        import torch
        t = torch.empty((self.S * self.n_trees, 2), dtype=torch.float32, device="cuda")
        self._check(self.L.ems_surrogate_targets(self.ctx, float(t_cap), 1 if freeze else 0,
                                                 ctypes.c_void_p(t.data_ptr())))
        return t

    def schedule(self, mlp, bound, coarsen=16, guard=0.8):
        """Per-tree step schedule from the network; returns (coarse trees per
        sample, predictions)."""
        import torch
        n = np.zeros(self.S, np.int32)
        pred = torch.empty((self.S * self.n_trees, 2), dtype=torch.float32, device="cuda")
        self._check(self.L.ems_surrogate_schedule(self.ctx, mlp.h, float(bound), int(coarsen), float(guard),
                                                  A._ptr(n, ctypes.c_int32), ctypes.c_void_p(pred.data_ptr())))
        return n, pred

    def clear_schedule(self):
        self._check(self.L.ems_surrogate_clear(self.ctx))
