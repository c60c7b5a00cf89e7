"""Pins of the Krylov oracle (Sec. IV-E, Alg. 1) against mathematics:
a basis that spans the whole space reproduces backward Euler exactly; the
projection matches the shifted moments of Eq. rak_moment_recurrence; a zero
initial stress deflates the starting block; nucleation times approach the
full-order ones as q grows."""
import math

import numpy as np
import scipy.sparse.linalg as spla

import ems_synth as es
from oracle import flow as F
from oracle import krylov as K

P = es.default_params()


def _chain(cells, I_sink=2e-3, seed=0):
    g = es.tree_grid("chain", cells=cells, seed=seed, I_sink=I_sink)
    tr = F.build_trees(g)
    phys = F.tree_physics(tr, P, np.full(tr["n_nodes"], 378.0))
    u = F.ir_solve(g, g["seg_R0"])
    j = F.current_density(g, u, g["seg_R0"])
    f = F.forcing(tr, phys, F.face_G(tr, P, phys, j))
    return g, tr, phys, f


def test_full_span_basis_equals_backward_euler():
    g, tr, phys, f = _chain(cells=2)                  # 9 stress nodes
    n = tr["n_nodes"]
    ph = dict(phys, sig_crit=np.full(n, np.inf))
    dt = 2e4
    a = F.StressState(tr, P)
    b = F.StressState(tr, P)
    F.advance(tr, P, ph, f, a, 0.0, dt, 40)
    ks = K.KrylovStepper(q=n + 3)
    ks.use_krylov = lambda nn: True
    ks(tr, P, ph, f, b, 0.0, dt, 40)
    assert ks.n_reduced == 1 and ks.n_fallback == 0
    assert np.abs(a.sigma - b.sigma).max() < 1e-9 * np.abs(a.sigma).max()


def test_moment_matching_and_deflation():
    g, tr, phys, f = _chain(cells=25)                 # 101 nodes
    C, A, ft = K.tree_system(tr, phys, f, np.zeros(tr["n_nodes"], np.int32), 0)
    s0 = 1.0 / K.shift_time(tr, phys, 0, 1.0)
    q = 4
    sigma0 = np.zeros(tr["n_nodes"])
    V, Ah, Ch, fh, st = K.krylov_basis(C, A, ft, sigma0, s0, q)
    assert st == "ok"
    assert V.shape[1] == q                         # zero sigma0: one column per block
    assert np.abs(V.T @ V - np.eye(q)).max() < 1e-12
    # shifted moments (sigma0 = 0): m0 = R f, m_k = -R C m_{k-1}
    Kf = spla.splu((s0 * C - A).tocsc())
    Kh = s0 * Ch - Ah
    m = Kf.solve(ft)
    mh = np.linalg.solve(Kh, fh)
    for k in range(q):
        assert np.abs(V @ mh - m).max() < 1e-8 * np.abs(m).max(), k
        m = -Kf.solve(C @ m)
        mh = -np.linalg.solve(Kh, Ch @ mh)


def test_shift_time_closed_form():
    g, tr, phys, f = _chain(cells=10)
    dx = tr["face_dx"][1]
    L = (tr["n_nodes"] - 1) * dx
    kap = phys["kap_a"][1] / tr["face_a"][1]
    assert abs(K.shift_time(tr, phys, 0, 1.0) - L * L / (math.pi ** 2 * kap)) < 1e-12 * L * L / kap
    t = F.build_trees(es.tree_grid("T", cells=4))
    ph = F.tree_physics(t, P, np.full(t["n_nodes"], 378.0))
    # T tree: longest path joins two arm ends through the junction (2 segments)
    Lt = 2 * 10e-6
    kap = ph["kap_a"][1] / t["face_a"][1]
    assert abs(K.shift_time(t, ph, 0, 2.0) - 2.0 * Lt * Lt / (math.pi ** 2 * kap)) < 1e-12 * Lt * Lt / kap


def test_nucleation_time_converges_with_order():
    g, tr, phys, f = _chain(cells=40, I_sink=6e-3)    # 161 nodes
    n = tr["n_nodes"]
    sc = np.full(n, 150e6)
    ph = dict(phys, sig_crit=sc)
    dt = 2e3
    ref = F.StressState(tr, P)
    F.advance(tr, P, ph, f, ref, 0.0, dt, 3000)
    voids = np.nonzero(ref.void)[0]
    errs = []
    for q in (4, 8, 12):
        st = F.StressState(tr, P)
        K.KrylovStepper(q=q)(tr, P, ph, f, st, 0.0, dt, 3000)
        assert np.array_equal(np.nonzero(st.void)[0], voids)
        errs.append(np.max(np.abs(st.t_nuc[voids] - ref.t_nuc[voids]) / ref.t_nuc[voids]))
    # the cited accuracy (about 1 % at q = 4-6) tightens with the order
    assert errs[0] < 0.2 and errs[1] < 0.02 and errs[2] < 1e-3
    assert errs[2] < errs[1] < errs[0]


def test_augmented_basis_matches_the_new_input():
    """A basis cached for one forcing and stress, extended by the current
    starting block [R C s, R f] (the cache policy of Sec. IV-E.4): the
    columns stay orthonormal, R C s and R f lie in the span, so the reduced
    model reproduces the new input's zeroth shifted moment exactly."""
    g, tr, phys, f_old = _chain(cells=25, I_sink=2e-3)
    _, _, _, f_new = _chain(cells=25, I_sink=3e-3, seed=1)
    n = tr["n_nodes"]
    void = np.zeros(n, np.int32)
    C, A, fo = K.tree_system(tr, phys, f_old, void, 0)
    _, _, fn = K.tree_system(tr, phys, f_new, void, 0)
    s0 = 1.0 / K.shift_time(tr, phys, 0, 1.0)
    V, _, _, _, st = K.krylov_basis(C, A, fo, np.zeros(n), s0, 4)
    assert st == "ok" and V.shape[1] == 4
    a = F.StressState(tr, P)
    F.advance(tr, P, dict(phys, sig_crit=np.full(n, np.inf)), f_new, a, 0.0, 2e4, 30)
    lu = spla.splu((s0 * C - A).tocsc())
    Va = K.augment(V, lu, C, a.sigma, fn)
    assert Va.shape[1] == 6
    assert np.abs(Va.T @ Va - np.eye(6)).max() < 1e-12
    for x in (lu.solve(C @ a.sigma), lu.solve(fn)):
        assert np.linalg.norm(x - Va @ (Va.T @ x)) < 1e-10 * np.linalg.norm(x)
    Kh = Va.T @ ((s0 * C - A) @ Va)
    m = lu.solve(fn)
    assert np.abs(Va @ np.linalg.solve(Kh, Va.T @ fn) - m).max() < 1e-9 * np.abs(m).max()
    # a block already in the span adds nothing
    assert K.augment(Va, lu, C, a.sigma, fn).shape[1] == 6


def test_augmented_cache_tracks_backward_euler_stale_cache_does_not():
    """Two aging steps with different forcings on a 161-node chain: the cached
    basis augmented by the current block follows full BE closely, the same
    basis reused as it stands (keyed on C, A and s0 alone) does not."""
    g, tr, phys, f1 = _chain(cells=40, I_sink=2e-3)
    _, _, _, f2 = _chain(cells=40, I_sink=4e-3, seed=3)
    n = tr["n_nodes"]
    ph = dict(phys, sig_crit=np.full(n, np.inf))
    dt, ns = 2e4, 100
    ref = F.StressState(tr, P)
    F.advance(tr, P, ph, f1, ref, 0.0, dt, ns)
    F.advance(tr, P, ph, f2, ref, ns * dt, dt, ns)
    err = {}
    for policy in ("augment", "stale"):
        ks = K.KrylovStepper(q=6, policy=policy)
        ks.use_krylov = lambda nn: True
        st = F.StressState(tr, P)
        ks(tr, P, ph, f1, st, 0.0, dt, ns)
        ks(tr, P, ph, f2, st, ns * dt, dt, ns)
        assert ks.n_built == 1
        err[policy] = np.abs(st.sigma - ref.sigma).max() / np.abs(ref.sigma).max()
    assert err["augment"] < 3e-4
    assert err["stale"] > 30 * err["augment"]


def test_uniform_initial_stress_makes_the_second_block_rank_deficient():
    """Before any void the Neumann operator has A 1 = 0, so (s0 C - A)^-1 C 1
    = 1 / s0: the constant column of the starting block is mapped onto itself.
    The next block then holds that repeated direction (nothing left after
    orthogonalisation) beside a new one, which is the rank-deficient case of
    Sec. IV-E.5 under both orthogonalisation orders; with a zero initial
    stress the same tree reduces."""
    g, tr, phys, f = _chain(cells=25)
    n = tr["n_nodes"]
    C, A, ft = K.tree_system(tr, phys, f, np.zeros(n, np.int32), 0)
    s0 = 1.0 / K.shift_time(tr, phys, 0, 1.0)
    ones = np.ones(n)
    assert np.abs(A @ ones).max() < 1e-12 * abs(A).max() * n      # rows of A sum to zero
    lu = spla.splu((s0 * C - A).tocsc())
    assert np.abs(lu.solve(C @ ones) * s0 - 1.0).max() < 1e-12
    for ortho in ("mgs", "cgs2"):
        assert K.krylov_basis(C, A, ft, np.full(n, 50e6), s0, 6, ortho=ortho)[4] == "rank"
        assert K.krylov_basis(C, A, ft, np.zeros(n), s0, 6, ortho=ortho)[4] == "ok"
