"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: an exact
discrete eigen-solution, Korhonen's continuum series, atom conservation, a
dense library solve, brute-force steady states, hand-computed literals.
"""
import math

import numpy as np
import pytest

import ems_synth as es
from oracle import flow as F

P = es.default_params()


def _chain(cells=40, seg_len=10e-6, nseg=4):
    g = es.tree_grid("chain", cells=cells, seg_len=seg_len)
    assert g["seg_a"].size == nseg
    return g


def _uniform_chain_setup(cells=10, G_target=None, T=378.0):
    """One straight chain (4 segments), uniform T, uniform current density."""
    g = _chain(cells=cells)
    tr = F.build_trees(g)
    p = dict(P, T0=T)
    phys = F.tree_physics(tr, p, np.full(tr["n_nodes"], T))
    j = np.full(g["seg_a"].size, 2.0e10)
    G = F.face_G(tr, p, phys, j)
    return g, tr, p, phys, j, G


# ---------------------------------------------------------------------------
# T2: exact discrete solution of the node-centred FV + BE on a uniform chain
# ---------------------------------------------------------------------------

def test_be_matches_exact_discrete_modes():
    g, tr, p, phys, j, G = _uniform_chain_setup(cells=10)
    n = tr["n_nodes"]; N = n - 1
    x = np.arange(n) * tr["face_dx"][1]
    Gs = G[1]
    assert np.allclose(G[1:], Gs)
    kap = phys["g"][1] * tr["face_dx"][1] / tr["face_a"][1]
    dx = tr["face_dx"][1]
    # generalized eigenpairs: v_k(i) = cos(k pi i / N), lam_k = 4 kap/dx^2 sin^2(k pi / 2N)
    k = np.arange(n)
    Vk = np.cos(np.outer(np.arange(n), k) * math.pi / N)            # [node, mode]
    lam = 4.0 * kap / dx ** 2 * np.sin(k * math.pi / (2 * N)) ** 2
    Cw = np.full(n, 1.0); Cw[0] = Cw[-1] = 0.5                     # C / (a dx)
    L = N * dx
    sstar = Gs * (x - L / 2)                                         # exact discrete steady state
    e0 = -sstar
    ck = (Vk * (Cw * e0)[:, None]).sum(0) / (Vk * Vk * Cw[:, None]).sum(0)
    dt = 0.05 * L * L / (math.pi ** 2 * kap)
    nsteps = 37
    exact = sstar + Vk @ (ck * (1.0 + dt * lam) ** (-nsteps))
    f = F.forcing(tr, phys, G)
    st = F.StressState(tr, p)
    ph = dict(phys, sig_crit=np.full(n, np.inf))
    F.advance(tr, p, ph, f, st, 0.0, dt, nsteps)
    scale = np.abs(exact).max()
    assert np.abs(st.sigma - exact).max() / scale < 1e-12


# ---------------------------------------------------------------------------
# T1: Korhonen's series (blocking ends, constant G, uniform kappa, sigma0 = 0)
# ---------------------------------------------------------------------------

def _korhonen_series(x, t, L, G, kap, nterms=2001):
    s = G * (x - L / 2)
    for m in range(1, nterms, 2):
        s = s + 4 * G * L / (m * m * math.pi ** 2) * np.cos(m * math.pi * x / L) \
            * math.exp(-kap * m * m * math.pi ** 2 * t / (L * L))
    return s


@pytest.mark.parametrize("t_frac", [0.05, 0.3])
def test_be_converges_to_korhonen_series(t_frac):
    errs = []
    for cells, nsteps in ((5, 50), (10, 200), (20, 800)):
        g, tr, p, phys, j, G = _uniform_chain_setup(cells=cells)
        n = tr["n_nodes"]; dx = tr["face_dx"][1]; L = (n - 1) * dx
        kap = phys["g"][1] * dx / tr["face_a"][1]
        tau = L * L / (math.pi ** 2 * kap)
        t = t_frac * tau
        f = F.forcing(tr, phys, G)
        st = F.StressState(tr, p)
        F.advance(tr, p, dict(phys, sig_crit=np.full(n, np.inf)), f, st, 0.0, t / nsteps, nsteps)
        ref = _korhonen_series(np.arange(n) * dx, t, L, G[1], kap)
        errs.append(np.abs(st.sigma - ref).max() / np.abs(ref).max())
    # first order in time (dt quartered per halving of dx) and second order in space
    assert errs[2] < 0.02
    assert errs[1] / errs[2] > 3.0 and errs[0] / errs[1] > 3.0


# ---------------------------------------------------------------------------
# T3: atom conservation (Eq. void_volume_equation)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["T", "comb", "star"])
def test_atom_conservation_branched_with_tm(kind):
    g = es.tree_grid(kind, cells=6, seed=3)
    tr = F.build_trees(g)
    rng = np.random.default_rng(7)
    Tn = 360 + 30 * rng.random(tr["n_nodes"])           # rough temperature field (TM on)
    phys = F.tree_physics(tr, P, Tn)
    j = rng.normal(0, 3e10, size=g["seg_a"].size)
    G = F.face_G(tr, P, phys, j)
    f = F.forcing(tr, phys, G)
    assert abs(f.sum()) < 1e-12 * np.abs(f).sum()
    st = F.StressState(tr, P)
    st.sigma[:] = rng.normal(0, 1e7, tr["n_nodes"])
    m0 = (phys["V"] * st.sigma).sum()
    kap = phys["g"][1] * tr["face_dx"][1] / tr["face_a"][1]
    dt = 0.01 * (10e-6) ** 2 / kap
    F.advance(tr, P, dict(phys, sig_crit=np.full(tr["n_nodes"], np.inf)), f, st, 0.0, dt, 50)
    m1 = (phys["V"] * st.sigma).sum()
    assert abs(m1 - m0) < 1e-12 * (phys["V"] * np.abs(st.sigma)).sum()


def test_atom_conservation_with_voids():
    g, tr, p, phys, j, G = _uniform_chain_setup(cells=10)
    n = tr["n_nodes"]
    f = F.forcing(tr, phys, G)
    st = F.StressState(tr, p)
    kap = phys["g"][1] * tr["face_dx"][1] / tr["face_a"][1]
    L = (n - 1) * tr["face_dx"][1]
    dt = 0.002 * L * L / kap
    sc = np.full(n, 0.4 * G[1] * L / 2)              # reachable: steady max is G L / 2
    nv = F.advance(tr, p, dict(phys, sig_crit=sc), f, st, 0.0, dt, 400)
    assert nv >= 1
    total = (phys["V"] * st.sigma).sum() + p["B_modulus"] * st.vol.sum()
    assert abs(total) < 1e-11 * (phys["V"] * np.abs(st.sigma)).sum()


# ---------------------------------------------------------------------------
# T4 / T5: steady state and the immortality screen (Sec. III-B)
# ---------------------------------------------------------------------------

def _dense_M(tr, phys, dt, void):
    n = tr["n_nodes"]
    M = np.diag(phys["V"] + dt * phys["leak"] * void)
    for i in range(1, n):
        q = tr["par"][i]
        gi = phys["g"][i]
        M[i, i] += dt * gi; M[q, q] += dt * gi
        M[i, q] -= dt * gi; M[q, i] -= dt * gi
    return M


def _dense_A(tr, phys):
    n = tr["n_nodes"]
    A = np.zeros((n, n))
    for i in range(1, n):
        q = tr["par"][i]; gi = phys["g"][i]
        A[i, i] -= gi; A[q, q] -= gi; A[i, q] += gi; A[q, i] += gi
    return A


@pytest.mark.parametrize("kind", ["T", "comb", "star", "chain"])
def test_steady_state_brute_force(kind):
    g = es.tree_grid(kind, cells=5, seed=11)
    tr = F.build_trees(g)
    rng = np.random.default_rng(5)
    Tn = 350 + 40 * rng.random(tr["n_nodes"])
    phys = F.tree_physics(tr, P, Tn)
    j = rng.normal(0, 3e10, size=g["seg_a"].size)
    G = F.face_G(tr, P, phys, j)
    f = F.forcing(tr, phys, G)
    A = _dense_A(tr, phys)
    n = tr["n_nodes"]
    # A s = -f with sum V s = 0 (sigma_T = 0): bordered system
    K = np.zeros((n + 1, n + 1)); K[:n, :n] = A; K[:n, n] = phys["V"]; K[n, :n] = phys["V"]
    rhs = np.concatenate([-f, [0.0]])
    ref = np.linalg.solve(K, rhs)[:n]
    ss = F.steady_stress(tr, P, phys, G)
    assert np.abs(ss - ref).max() < 1e-9 * np.abs(ref).max()
    # T5: mortal iff the brute-force steady maximum exceeds sigma_crit
    for sc in (0.5 * ref.max(), 1.5 * ref.max()):
        ph = dict(phys, sig_crit=np.full(n, sc))
        mortal, smax, _ = F.screen(tr, P, ph, G)
        assert bool(mortal[0]) == bool(ref.max() > sc)
        assert abs(smax[0] - ref.max()) < 1e-9 * abs(ref).max()


def test_long_time_be_reaches_steady():
    g = es.tree_grid("comb", cells=5, seed=2)
    tr = F.build_trees(g)
    phys = F.tree_physics(tr, P, np.full(tr["n_nodes"], 378.0))
    j = np.random.default_rng(1).normal(0, 3e10, size=g["seg_a"].size)
    G = F.face_G(tr, P, phys, j)
    f = F.forcing(tr, phys, G)
    st = F.StressState(tr, P)
    kap = phys["g"][1] * tr["face_dx"][1] / tr["face_a"][1]
    F.advance(tr, P, dict(phys, sig_crit=np.full(tr["n_nodes"], np.inf)), f, st, 0.0,
              1e3 * (60e-6) ** 2 / kap, 40)
    ss = F.steady_stress(tr, P, phys, G)
    assert np.abs(st.sigma - ss).max() < 1e-9 * np.abs(ss).max()


# ---------------------------------------------------------------------------
# T6: one BE step against a dense LAPACK solve, with Robin void rows
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["T", "comb", "star", "chain"])
def test_be_step_dense_solve(kind):
    g = es.tree_grid(kind, cells=4, seed=4)
    tr = F.build_trees(g)
    rng = np.random.default_rng(9)
    n = tr["n_nodes"]
    phys = F.tree_physics(tr, P, 360 + 20 * rng.random(n))
    j = rng.normal(0, 3e10, size=g["seg_a"].size)
    f = F.forcing(tr, phys, F.face_G(tr, P, phys, j))
    st = F.StressState(tr, P)
    st.sigma[:] = rng.normal(0, 1e8, n)
    st.void[[1, n // 2]] = 1                         # a terminal-side and a mid-tree void
    dt = 3e4
    M = _dense_M(tr, phys, dt, st.void)
    ref = np.linalg.solve(M, phys["V"] * st.sigma + dt * f)
    F.advance(tr, P, dict(phys, sig_crit=np.full(n, np.inf)), f, st, 0.0, dt, 1)
    assert np.abs(st.sigma - ref).max() < 1e-12 * np.abs(ref).max()


# ---------------------------------------------------------------------------
# T8: Robin void limit and the saturated void volume
# ---------------------------------------------------------------------------

def test_void_saturates_to_closed_form():
    g, tr, p, phys, j, G = _uniform_chain_setup(cells=10)
    n = tr["n_nodes"]
    f = F.forcing(tr, phys, G)
    ss = F.steady_stress(tr, p, phys, G)
    v = int(np.argmax(ss))
    st = F.StressState(tr, p)
    st.sigma[:] = ss                                 # start at the void-free steady state
    st.void[v] = 1                                   # void at the steady maximum
    kap = phys["g"][1] * tr["face_dx"][1] / tr["face_a"][1]
    L = (n - 1) * tr["face_dx"][1]
    F.advance(tr, p, dict(phys, sig_crit=np.full(n, np.inf)), f, st, 0.0,
              0.02 * L * L / kap, 3000)
    Vtree = phys["V"].sum()
    vsat = ss.max() * Vtree / p["B_modulus"]
    assert abs(st.vol[v] - vsat) < 1e-6 * vsat
    assert abs(st.sigma[v]) < 1e-6 * ss.max()
    # stress is the path integral of G measured from the void: all <= 0 here
    assert st.sigma.max() < 1e-6 * ss.max()


def test_mid_tree_void_decouples_branches():
    """A void at the T junction: the stress there relaxes to ~0 and the
    branches stop exchanging atoms (Sec. IV-D)."""
    g = es.tree_grid("T", cells=8, seed=1)
    tr = F.build_trees(g)
    n = tr["n_nodes"]
    phys = F.tree_physics(tr, P, np.full(n, 378.0))
    j = np.zeros(g["seg_a"].size); j[0] = 4e10; j[1] = -4e10; j[2] = 4e10
    G = F.face_G(tr, P, phys, j)
    f = F.forcing(tr, phys, G)
    jn = int(np.nonzero(tr["ir"] == 1)[0][0])      # junction stress node
    st = F.StressState(tr, P)
    st.void[jn] = 1
    kap = phys["g"][1] * tr["face_dx"][1] / tr["face_a"][1]
    F.advance(tr, P, dict(phys, sig_crit=np.full(n, np.inf)), f, st, 0.0,
              1.0 * (10e-6) ** 2 / kap, 4000)
    assert abs(st.sigma[jn]) < 1e-4 * np.abs(st.sigma).max()
    # each branch is now at its own zero-flux state anchored at the junction:
    # sigma_child - sigma_parent = dx G on every face
    child = np.arange(1, n)
    dif = st.sigma[child] - st.sigma[tr["par"][child]]
    assert np.abs(dif - tr["face_dx"][child] * G[child]).max() < 1e-4 * np.abs(G).max() * 1.25e-6


# ---------------------------------------------------------------------------
# Nucleation time (Sec. III-D.2) from the exact discrete solution
# ---------------------------------------------------------------------------

def test_nucleation_time_interpolation():
    g, tr, p, phys, j, G = _uniform_chain_setup(cells=10)
    n = tr["n_nodes"]; N = n - 1; dx = tr["face_dx"][1]; L = N * dx
    kap = phys["g"][1] * dx / tr["face_a"][1]
    f = F.forcing(tr, phys, G)
    dt = 0.003 * L * L / kap
    sc_val = 0.6 * G[1] * L / 2
    st = F.StressState(tr, p)
    F.advance(tr, p, dict(phys, sig_crit=np.full(n, sc_val)), f, st, 100.0, dt, 300)
    assert st.void.sum() == 1
    v = int(np.nonzero(st.void)[0][0])
    # independent trajectory from the discrete modes (T2) at node v
    k = np.arange(n)
    Vk = np.cos(np.outer(np.arange(n), k) * math.pi / N)
    lam = 4.0 * kap / dx ** 2 * np.sin(k * math.pi / (2 * N)) ** 2
    Cw = np.full(n, 1.0); Cw[0] = Cw[-1] = 0.5
    sstar = G[1] * (np.arange(n) * dx - L / 2)
    ck = (Vk * (Cw * -sstar)[:, None]).sum(0) / (Vk * Vk * Cw[:, None]).sum(0)
    traj = [sstar + Vk @ (ck * (1.0 + dt * lam) ** (-m)) for m in range(301)]
    m1 = next(m for m in range(1, 301) if traj[m].max() >= sc_val)
    assert v == int(np.argmax(traj[m1])) == n - 1  # cathode end (current leaves there)
    s0, s1 = traj[m1 - 1][v], traj[m1][v]
    t_ref = 100.0 + (m1 - 1) * dt + (sc_val - s0) / (s1 - s0) * dt
    assert abs(st.t_nuc[v] - t_ref) < 1e-9 * dt


# ---------------------------------------------------------------------------
# T9: void resistance and IR solves on tiny networks
# ---------------------------------------------------------------------------

def test_delta_R_literal():
    g = es.tree_grid("chain", cells=4)
    tr = F.build_trees(g)
    st = F.StressState(tr, P)
    v = 2
    st.void[v] = 1; st.vseg[v] = 0
    W, H = 0.5e-6, 0.2e-6
    st.vol[v] = W * W * H + W * H * 1.0e-6          # void 1 um longer than critical
    R = F.void_resistance(g, P, st)
    # rho_Ta/(h_Ta (2H+W)) = 1.8e-6/(5e-9*0.9e-6) = 4.0e8 Ohm/m;
    # rho_Cu/(H W) = 2.25e-8/1e-13 = 2.25e5 Ohm/m  ->  dR = 1e-6 * (4e8 - 2.25e5)
    assert abs((R[0] - g["seg_R0"][0]) - 399.775) < 1e-9
    assert np.array_equal(R[1:], g["seg_R0"][1:])
    st.vol[v] = 0.5 * W * W * H                      # below critical: no change
    assert np.array_equal(F.void_resistance(g, P, st), g["seg_R0"])


def test_ir_series_chain():
    g = es.tree_grid("chain", cells=4)
    g["sink_node"] = np.array([4], np.int32); g["sink_I"] = np.array([1e-3])
    R = np.array([1.0, 2.0, 3.0, 4.0])
    u = F.ir_solve(g, R)
    assert np.allclose(u, [1.0, 1 - 1e-3, 1 - 3e-3, 1 - 6e-3, 1 - 10e-3], rtol=0, atol=1e-15)
    jd = F.current_density(g, u, R)
    assert np.allclose(jd, 1e-3 / (0.5e-6 * 0.2e-6), rtol=1e-12)


def test_ir_2x2_grid():
    g = es.stripe_mesh(2, 10e-6)
    g["pad_node"] = np.array([0], np.int32); g["pad_V"] = np.array([1.0])
    g["sink_node"] = np.array([3], np.int32); g["sink_I"] = np.array([2e-3])
    R = np.full(g["seg_a"].size, 5.0)
    u = F.ir_solve(g, R)
    # two parallel 10-Ohm paths from node 0 to node 3: 5 Ohm effective
    assert abs(u[3] - (1.0 - 2e-3 * 5.0)) < 1e-15
    assert abs(u[1] - (1.0 - 1e-3 * 5.0)) < 1e-15 and abs(u[2] - u[1]) < 1e-15
    assert abs(F.max_drop(u, 1.0) - 0.01) < 1e-15


def test_ir_3x3_against_dense():
    g = es.stripe_mesh(3, 10e-6)
    rng = np.random.default_rng(0)
    g["pad_node"] = np.array([0, 8], np.int32); g["pad_V"] = np.array([1.0, 0.99])
    g["sink_node"] = np.arange(9, dtype=np.int32); g["sink_I"] = rng.uniform(1e-4, 1e-3, 9)
    R = rng.uniform(1, 5, g["seg_a"].size)
    u = F.ir_solve(g, R)
    # KCL residual at every free node, and pads held
    n = 9
    res = np.zeros(n)
    for s in range(R.size):
        a, b = g["seg_a"][s], g["seg_b"][s]
        i = (u[a] - u[b]) / R[s]
        res[a] -= i; res[b] += i
    np.add.at(res, g["sink_node"], -g["sink_I"])
    free = np.setdiff1d(np.arange(n), g["pad_node"])
    assert np.abs(res[free]).max() < 1e-15
    assert u[0] == 1.0 and u[8] == 0.99


# ---------------------------------------------------------------------------
# Thermal sampling, kappa, tree extraction
# ---------------------------------------------------------------------------

def test_bilinear_reproduces_affine_field():
    xs = np.linspace(0, 1e-3, 33); ys = np.linspace(0, 2e-3, 17)
    X, Y = np.meshgrid(xs, ys)
    th = dict(T=300 + 1e4 * X + 3e4 * Y, x0=0.0, y0=0.0, x1=1e-3, y1=2e-3)
    rng = np.random.default_rng(3)
    px = rng.uniform(0, 1e-3, 100); py = rng.uniform(0, 2e-3, 100)
    assert np.allclose(F.bilinear(th, px, py), 300 + 1e4 * px + 3e4 * py, rtol=0, atol=1e-10)
    # clamped outside
    assert abs(F.bilinear(th, np.array([-1.0]), np.array([0.0]))[0] - 300.0) < 1e-12


def test_kappa_literal():
    # kappa(378 K) with D0 = 1e-8, Ea = 0.8 eV, B = 1e11, Omega = 1.18e-29:
    # Ea/(kB T) = 0.8*1.602176634e-19/(1.380649e-23*378) = 24.5598267122753...
    # kappa = 1e-8 * exp(-24.5598267...) * 1e11 * 1.18e-29 / (1.380649e-23*378)
    #       = 4.8765166025446264e-17 m^2/s (40-digit decimal arithmetic)
    k = F.kappa_of_T(np.array([378.0]), P)[0]
    assert abs(k - 4.8765166025446264e-17) / 4.8765166025446264e-17 < 1e-13


def test_tree_counts_and_structure():
    tr = F.build_trees(es.tiny_grid())
    assert tr["n_trees"] == 16 and tr["n_nodes"] == 16 * 281
    assert np.array_equal(np.diff(tr["off"]), np.full(16, 281))
    # a stripe is a chain rooted at its lowest-id end
    assert np.array_equal(tr["par"][1:281], np.arange(280))
    assert tr["ir"][0] == 0 and tr["ir"][280] == 7 and tr["ir"][281] == 8
    t = F.build_trees(es.tree_grid("T", cells=8))
    # junction IR node 1 at local 8; arms to IR 2 then IR 3 follow depth-first
    assert t["ir"][8] == 1 and t["ir"][16] == 2 and t["par"][17] == 8 and t["ir"][24] == 3
    mc = es.mc_grid(n_samples=0)
    tm = F.build_trees(mc)
    assert tm["n_nodes"] == int(sum(7 * c + 1 for c in mc["seg_cells"][::7][:16]))


def test_cycle_rejected():
    g = es.stripe_mesh(2, 10e-6)
    g["seg_layer"][:] = 0                         # one layer: the 2x2 ring is a cycle
    with pytest.raises(ValueError):
        F.build_trees(g)


def test_ttf_crossing_interpolation():
    assert F.crossing_time(10.0, 0.08, 0.12, 4.0, 0.10) == 12.0


def test_face_conductance_and_driving_force_literals():
    """g = a kappa / dx with the pinned kappa; S = e Z rho j / Omega;
    M = Q / (Omega T_e) dT/dx (Sec. III-D.1)."""
    g, tr, p, phys, j, G = _uniform_chain_setup(cells=10)
    dx = tr["face_dx"][1]; a = tr["face_a"][1]
    assert abs(phys["g"][1] - a * 4.8765166025446264e-17 / dx) < 1e-13 * phys["g"][1]
    # S(j = 2e10 A/m^2, Z = 5) = 1.602176634e-19*5*2.25e-8*2e10/1.18e-29
    #                          = 3.0549978190677966e13 Pa/m (40-digit decimal)
    assert abs(G[1] - 3.0549978190677966e13) < 1e-13 * G[1]
    # a linear temperature rise of 1 K per um along the face: T_e = 378 K at mid-face
    Tn = 378.0 + (np.arange(tr["n_nodes"]) - 0.5) * dx * 1e6
    ph = F.tree_physics(tr, p, Tn)
    # M = 0.09 eV / (1.18e-29 m^3 * 378 K) * 1e6 K/m = 3.2328019249394673e12 Pa/m
    assert abs(ph["M"][1] - 3.2328019249394673e12) < 1e-9 * ph["M"][1]
