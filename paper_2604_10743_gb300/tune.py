"""Chain-shape autotuning with a cache.

The per-tree eliminations of every size group run with the shape (kernel,
nodes per thread, CTAs per chain) measured fastest on this GPU for this grid:
ems_autotune times every valid shape on scratch copies of a loaded context,
the table is kept in a JSON cache keyed by the grid's connectivity and
discretisation, the sample counts and the precision, and the grid is loaded
again with ems_set_chain_rules so that the packed layout follows the table.
"""
import hashlib
import json
import os

import numpy as np

from . import _abi as A
from .engine import Engine


def grid_key(grid, precision, window=0, max_samples=2, n_steps=32):
    """Cache key: what the chain lengths and the launch sizes depend on."""
    h = hashlib.sha1()
    for name in ("seg_a", "seg_b", "seg_layer", "seg_cells", "seg_via", "pad_node"):
        v = grid.get(name)
        if v is not None:
            h.update(name.encode())
            h.update(np.ascontiguousarray(v).tobytes())
    kf = grid.get("kappa_factor")
    S = 1 if kf is None else int(np.asarray(kf).shape[0])
    h.update(("S%d W%d P%d m%d k%d" % (S, window, precision, max_samples, n_steps)).encode())
    return h.hexdigest()


def _load(cache):
    if cache and os.path.exists(cache):
        with open(cache) as f:
            return json.load(f)
    return {}


def tuned_engine(params, grid, cache=None, n_steps=32, max_samples=2, **kw):
    """An Engine whose chain shapes follow the autotuner's table for this grid
    (read from `cache` when it holds one, else measured on a first context
    after one IR solve and stored).  The table is on the engine as
    `tune_table`, each rule with its time and the built-in shape's."""
    precision = kw.get("precision", A.EMS_F64)
    key = grid_key(grid, precision, kw.get("window", 0), max_samples, n_steps)
    db = _load(cache)
    table = db.get(key)
    measured = table is None
    if measured:
        eng = Engine(params, grid, **kw)
        try:
            eng.ir_solve()
            table = eng.autotune(n_steps, max_samples)
        finally:
            eng.close()
        if cache:
            db = _load(cache)
            db[key] = table
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(db, f, indent=1)
            os.replace(tmp, cache)
    eng = Engine(params, grid, chain_rules=table, **kw)
    eng.tune_table = table
    eng.tune_measured = measured
    return eng
