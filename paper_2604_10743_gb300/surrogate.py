"""Python face of include/ems_surrogate.h (argument marshalling only).

Mlp wraps one ems_mlp network; gemm_bf16 the tensor-core dense-layer
primitive.  The pipeline functions string C-ABI calls together:

  generate_records   per (tree, sample): features at t = 0 and the first
                     nucleation time / node of the plain solver run with the
                     t = 0 currents, stepped to t_cap
  Mlp.fit_norm       standardisation statistics of a record set (device)
  validate_bound     the skip bound, validated end to end on held-out grids
                     (ems_surrogate_validate): the most aggressive candidate
                     whose scheduled TTF runs reproduce the plain solver's TTF
                     and final IR drop within the tolerance, plus a margin
  Engine.schedule    (engine.py) skip flags for one context

Every computation runs in libems.so; torch holds the device tensors.
"""
import ctypes
import numpy as np

from . import _abi as A
from .engine import Engine

N_FEATURES, N_OUTPUTS, WIDTH = 24, 2, 256


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class Mlp:
    """The surrogate network: 24 -> n_hidden x 256 (ReLU) -> 2, BF16 tensor-core
    kernels with FP32 master weights and accumulation."""

    def __init__(self, n_hidden=4, seed=0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Mlp needs a CUDA device")
        self.L = A.lib()
        self.stream = torch.cuda.current_stream() if stream is None else stream
        h = ctypes.c_void_p()
        st = self.L.ems_mlp_create(int(n_hidden), int(seed), ctypes.c_void_p(self.stream.cuda_stream),
                                   ctypes.byref(h))
        if st != A.EMS_OK:
            raise A.EmsError(st, "ems_mlp_create")
        self.h = h
        self.n_hidden = n_hidden
        self.n_params = int(self.L.ems_mlp_param_count(h))

    def _check(self, st):
        if st != A.EMS_OK:
            msg = self.L.ems_mlp_last_error(self.h)
            raise A.EmsError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            self.L.ems_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        out = np.empty(self.n_params, np.float32)
        self._check(self.L.ems_mlp_get_params(self.h, _fptr(out)))
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, np.float32)
        if flat.size != self.n_params:
            raise ValueError("expected %d parameters" % self.n_params)
        self._check(self.L.ems_mlp_set_params(self.h, _fptr(flat)))

    def set_norm(self, x_mean, x_std, t_mean, t_std):
        a = [np.ascontiguousarray(v, np.float32) for v in (x_mean, x_std, t_mean, t_std)]
        self.norm = a
        self._check(self.L.ems_mlp_set_norm(self.h, *[_fptr(v) for v in a]))

    def fit_norm(self, x, t):
        """Fit the standardisation to a record set on the device and install
        it (ems_mlp_fit_norm); returns (x_mean, x_std, t_mean, t_std)."""
        st = np.empty(2 * N_FEATURES + 2 * N_OUTPUTS)
        self._check(self.L.ems_mlp_fit_norm(self.h, _vp(x), _vp(t), int(x.shape[0]),
                                            st.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        nf = N_FEATURES
        self.norm = [st[:nf], st[nf:2 * nf], st[2 * nf:2 * nf + N_OUTPUTS], st[2 * nf + N_OUTPUTS:]]
        return tuple(self.norm)

    def gradients(self, x, t):
        g = np.empty(self.n_params, np.float32)
        loss = ctypes.c_float()
        self._check(self.L.ems_mlp_gradients(self.h, _vp(x), _vp(t), int(x.shape[0]), _fptr(g),
                                             ctypes.byref(loss)))
        return g, loss.value

    def train_step(self, x, t, lr):
        loss = ctypes.c_float()
        self._check(self.L.ems_mlp_train_step(self.h, _vp(x), _vp(t), int(x.shape[0]), float(lr),
                                              ctypes.byref(loss)))
        return loss.value

    def train(self, x, t, batch=512, epochs=20, lr=1e-3, seed=0):
        losses = np.empty(epochs, np.float32)
        self._check(self.L.ems_mlp_train(self.h, _vp(x), _vp(t), int(x.shape[0]), int(batch), int(epochs),
                                         float(lr), int(seed), _fptr(losses)))
        return losses

    def predict(self, x):
        import torch
        y = torch.empty((x.shape[0], N_OUTPUTS), dtype=torch.float32, device="cuda")
        self._check(self.L.ems_mlp_predict(self.h, _vp(x), int(x.shape[0]), _vp(y)))
        return y

    @staticmethod
    def unflatten(flat, n_hidden):
        """Flat parameter vector -> [(W [out, in], b [out])] per layer."""
        sizes = [N_FEATURES] + [WIDTH] * n_hidden + [N_OUTPUTS]
        out, o = [], 0
        for fi, fo in zip(sizes[:-1], sizes[1:]):
            W = flat[o:o + fo * fi].reshape(fo, fi); o += fo * fi
            b = flat[o:o + fo]; o += fo
            out.append((W, b))
        return out

    @staticmethod
    def flatten(layers):
        return np.concatenate([np.concatenate([W.reshape(-1), b.reshape(-1)]) for W, b in layers])


def gemm_bf16(a, b, bias=None, relu=False, scale=1.0, out_bf16=False):
    """D = scale * a @ b.T (+ bias, ReLU) on the tensor cores; a [M, K] and b
    [N, K] contiguous BF16 CUDA tensors.  Returns the FP32 result (and the BF16
    one when out_bf16)."""
    import torch
    L = A.lib()
    M, K = a.shape
    N = b.shape[0]
    d = torch.empty((M, N), dtype=torch.float32, device="cuda")
    d16 = torch.empty((M, N), dtype=torch.bfloat16, device="cuda") if out_bf16 else None
    st = L.ems_gemm_bf16(_vp(a), _vp(b), M, N, K, None if bias is None else _vp(bias), 1 if relu else 0,
                         float(scale), _vp(d), None if d16 is None else _vp(d16),
                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != A.EMS_OK:
        raise A.EmsError(st, "ems_gemm_bf16")
    return (d, d16) if out_bf16 else d


def generate_records(grid, params, t_cap_factor=10.0, precision=A.EMS_F32, ext_outer=None):
    """(features, targets) device tensors, one row per (sample, tree), from a
    plain-solver run of `grid` with its t = 0 currents: the horizon in the
    TTF run's own steps, then on to t_cap = t_cap_factor * horizon in
    ext_outer coarser aging steps.  A (tree, sample) stops stepping at its
    first nucleation, which is all its record needs."""
    H = float(params["horizon"])
    n_out, n_in = int(params["n_outer"]), int(params["n_inner"])
    t_cap = t_cap_factor * H
    eng = Engine(params, grid, precision=precision, max_voids=32)
    try:
        eng.ir_solve()
        x = eng.features()
        dti = H / n_out / n_in
        for _ in range(n_out):
            eng.stress_advance(dti, n_in)
            eng.targets(t_cap, freeze=True)
        ext = ext_outer if ext_outer is not None else max(1, n_out // 2)
        if t_cap > H and ext > 0:
            dt2 = (t_cap - H) / ext / n_in
            for _ in range(ext):
                eng.stress_advance(dt2, n_in)
                eng.targets(t_cap, freeze=True)
        t = eng.targets(t_cap)
    finally:
        eng.close()
    return x, t




def scale_to_drop(grid, params, target, precision=A.EMS_F32):
    """Scale the grid's sink currents so that the initial max IR drop of its
    first sample is `target` (the drop is linear in the currents).  Returns
    the scaled grid dict (a shallow copy)."""
    eng = Engine(params, grid, precision=precision)
    try:
        _, d = eng.ir_solve()
    finally:
        eng.close()
    g = dict(grid)
    g["sink_I"] = np.asarray(grid["sink_I"], np.float64) * (target / float(d[0]))
    return g


def validate_bound(mlp, grids, params, coarsen=16, guard=0.8, candidates=(-1.0, -0.6, -0.3, 0.0, 0.3, 0.6, 1.0, 1.5),
                   tol=5e-4, margin=0.1, precision=A.EMS_F32, max_voids=32):
    """Schedule bound validated end to end against the plain solver
    (ems_surrogate_validate on one context per held-out grid).  Returns
    (first passing candidate + margin, or inf when none passes;
    per-candidate log of dicts bound / coarse_frac / max_rel_err)."""
    engs = [Engine(params, g, precision=precision, max_voids=max_voids) for g in grids]
    try:
        ctxs = (ctypes.c_void_p * len(engs))(*[e.ctx.value for e in engs])
        cand = np.ascontiguousarray(candidates, np.float64)
        log = np.full((cand.size, 3), np.nan)
        bound = ctypes.c_double()
        dp = ctypes.POINTER(ctypes.c_double)
        st = engs[0].L.ems_surrogate_validate(ctxs, len(engs), mlp.h, cand.ctypes.data_as(dp), int(cand.size),
                                              int(coarsen), float(guard), float(tol), float(margin),
                                              ctypes.byref(bound), log.ctypes.data_as(dp))
        engs[0]._check(st)
    finally:
        for e in engs:
            e.close()
    rows = [dict(bound=float(r[0]), coarse_frac=float(r[1]), max_rel_err=float(r[2]))
            for r in log if not np.isnan(r[0])]
    return bound.value, rows
