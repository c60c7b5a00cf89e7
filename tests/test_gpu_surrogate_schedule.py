"""The surrogate's features against an independent restatement from the FP64
oracle's quantities, and the trained surrogate's step schedule against the
plain solver: same TTF and final IR drop within 0.05 % on a grid the network
and the bound never saw, with fewer stress node-steps executed."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ems_synth as es
    from paper_2604_10743_gb300 import _abi as A
    from paper_2604_10743_gb300 import surrogate as sg
    from paper_2604_10743_gb300.engine import Engine
    return es, A, sg, Engine


def test_features_match_oracle_quantities(mods):
    from oracle import flow as F
    es, A, sg, Engine = mods
    p = es.default_params()
    g = es.tiny_grid()
    eng = Engine(p, g, precision=A.EMS_F64)
    eng.ir_solve()
    x = eng.features().cpu().numpy().astype(np.float64)
    eng.close()
    tr = F.build_trees(g)
    phys = F.tree_physics(tr, p, F.node_temperature(tr, None, p["T0"]))
    R = np.asarray(g["seg_R0"], np.float64)
    j = F.current_density(g, F.ir_solve(g, R), R)
    G = F.face_G(tr, p, phys, j)
    mortal, smax, ss = F.screen(tr, p, phys, G)
    f = F.forcing(tr, phys, G)
    # local early-time estimate t_i = pi (sigma_crit,i S_i / (2 F_i))^2 with
    # S_i = sum over the faces at i of a_e sqrt(kappa_e)
    kap = np.where(tr["face_a"] > 0, phys["kap_a"] / np.where(tr["face_a"] > 0, tr["face_a"], 1.0), 0.0)
    w = np.where(tr["gpar"] >= 0, tr["face_a"] * np.sqrt(np.maximum(kap, 0.0)), 0.0)
    S = w.copy()
    has = tr["gpar"] >= 0
    np.add.at(S, tr["gpar"][has], w[has])
    with np.errstate(divide="ignore"):
        tl = np.where(f > 0, math.pi * (phys["sig_crit"] * S / (2.0 * f)) ** 2, np.inf)
    for t in range(tr["n_trees"]):
        o, e = tr["off"][t], tr["off"][t + 1]
        n = e - o
        assert x[t, 0] == pytest.approx(math.log10(n), abs=1e-6)
        assert x[t, 12] == pytest.approx(phys["sig_crit"][o:e].min() * 1e-8, rel=1e-6)
        assert x[t, 14] == pytest.approx(smax[t] * 1e-8, rel=1e-5, abs=1e-6)
        assert bool(x[t, 17]) == bool(mortal[t])
        m = ss[o:e] - phys["sig_crit"][o:e]
        assert x[t, 18] == pytest.approx(int(np.argmax(m)) / (n - 1), abs=1e-6)
        assert x[t, 5] == pytest.approx(math.log10(min(tl[o:e].min(), 1e13)), abs=1e-5)


def _result_error(ref, run):
    """Largest relative difference of TTF (where the reference's is finite)
    and final IR drop between two TTF results; inf when the sets of failed
    samples differ."""
    fr, fx = np.isfinite(ref["ttf"]), np.isfinite(run["ttf"])
    if np.any(fr != fx):
        return math.inf
    e = float(np.max(np.abs(run["final_drop"] - ref["final_drop"]) / ref["final_drop"]))
    if fr.any():
        t = ref["ttf"][fr]
        e = max(e, float(np.max(np.abs(run["ttf"][fr] - t) / np.maximum(t, 1e-30))))
    return e


def _grid(es, sg, p, seed, N=64, S=32):
    g = es.grid.surrogate_grid(seed=seed, N=N, n_samples=S)
    return sg.scale_to_drop(g, p, np.random.default_rng(seed + 7).uniform(0.07, 0.095))


def test_schedule_matches_plain_solver_with_fewer_steps(mods):
    es, A, sg, Engine = mods
    p = es.default_params()
    xs, ts = [], []
    for seed in range(1000, 1024):                 # ~98k (tree, sample) records
        x, t = sg.generate_records(_grid(es, sg, p, seed), p)
        xs.append(x); ts.append(t)
    X, T = torch.cat(xs), torch.cat(ts)
    m = sg.Mlp(n_hidden=4, seed=0)
    m.fit_norm(X, T)
    losses = m.train(X, T, batch=1024, epochs=30, lr=1e-3, seed=1)
    assert losses[-1] < 0.5 * losses[0]
    bound, log = sg.validate_bound(m, [_grid(es, sg, p, 2000 + k) for k in range(3)], p, coarsen=16, guard=0.8,
                                   candidates=(-0.3, 0.0, 0.3, 0.6, 1.0))
    assert math.isfinite(bound), log
    g = _grid(es, sg, p, 3000)
    e1 = Engine(p, g, precision=A.EMS_F32, max_voids=32)
    r1 = e1.ttf()
    e1.close()
    e2 = Engine(p, g, precision=A.EMS_F32, max_voids=32)
    e2.ir_solve()
    n_coarse, _ = e2.schedule(m, bound, 16, 0.8)
    r2 = e2.ttf()
    e2.close()
    assert n_coarse.sum() > 0
    assert _result_error(r1, r2) <= 5e-4
    assert r1["node_steps_executed"] == pytest.approx(r1["node_steps"])
    assert r2["node_steps_executed"] <= 0.9 * r1["node_steps_executed"]
