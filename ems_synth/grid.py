"""Seeded synthetic power-grid netlists, thermal rasters and Monte Carlo factors.

These stand in for the paper's SAED32 power-grid netlists, YAML files and
measured thermal maps (Sec. V), which are not available.  The generator only
draws inputs; it holds none of the EM/TM method's arithmetic.  Both the CPU
oracle and the CUDA library consume the same arrays.

A grid is a dict of NumPy arrays (the content of an extracted netlist):

  node_x, node_y        float64 [n_nodes]   IR node coordinates (m)
  seg_a, seg_b          int32   [n_seg]     segment end nodes (a -> b is +x)
  seg_layer             int32   [n_seg]     metal layer; trees never cross layers
  seg_R0                float64 [n_seg]     resistance (Ohm), rho_Cu L/(W H)
  seg_W, seg_H, seg_L   float64 [n_seg]     width, thickness, length (m)
  seg_cells             int32   [n_seg]     finite-difference cells per segment
  pad_node, pad_V       int32/float64       supply pads (Dirichlet)
  sink_node, sink_I     int32/float64       current sinks (A drawn from node)
  thermal               None or dict(T=[ny,nx] K, x0, y0, x1, y1)
  kappa_factor          None or float64 [S, n_seg]  MC multiplier on kappa
  sigc_factor           None or float64 [S, n_seg]  MC multiplier on sigma_crit

Seeds follow NumPy Generator(PCG64(seed)).
"""
import math

import numpy as np

from .params import default_params


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def stripe_mesh(N, pitch, W=0.5e-6, H=0.2e-6, dx=0.5e-6, rho_Cu=None,
                tree_cells=None):
    """Two-layer mesh of N horizontal (layer 0) x N vertical (layer 1) stripes.

    Crossing (row i, column j) is IR node i*N + j at (j*pitch, i*pitch); the
    two layers are merged at each crossing (no via resistors).  Each stripe
    ends at its outermost crossings and carries N-1 segments of length pitch.
    Horizontal segments come first (row-major), then vertical ones.
    tree_cells: optional int array [2N] of FD cells per segment for each
    stripe (uneven trees); default is round(pitch / dx).
    """
    if rho_Cu is None:
        rho_Cu = default_params()["rho_Cu"]
    n = N * N
    jj, ii = np.meshgrid(np.arange(N), np.arange(N))
    node_x = (jj.ravel() * pitch).astype(np.float64)
    node_y = (ii.ravel() * pitch).astype(np.float64)
    a, b, layer, stripe = [], [], [], []
    for i in range(N):
        for j in range(N - 1):
            a.append(i * N + j); b.append(i * N + j + 1); layer.append(0); stripe.append(i)
    for j in range(N):
        for i in range(N - 1):
            a.append(i * N + j); b.append((i + 1) * N + j); layer.append(1); stripe.append(N + j)
    a = np.array(a, np.int32); b = np.array(b, np.int32)
    ns = a.size
    L = np.full(ns, pitch, np.float64)
    Wa = np.full(ns, W, np.float64)
    Ha = np.full(ns, H, np.float64)
    if tree_cells is None:
        cells = np.full(ns, int(round(pitch / dx)), np.int32)
    else:
        cells = np.asarray(tree_cells, np.int32)[np.array(stripe)]
    return dict(
        N=N, pitch=pitch,
        node_x=node_x, node_y=node_y,
        seg_a=a, seg_b=b, seg_layer=np.array(layer, np.int32),
        seg_R0=rho_Cu * L / (Wa * Ha), seg_W=Wa, seg_H=Ha, seg_L=L,
        seg_cells=cells,
        pad_node=np.zeros(0, np.int32), pad_V=np.zeros(0),
        sink_node=np.zeros(0, np.int32), sink_I=np.zeros(0),
        thermal=None, kappa_factor=None, sigc_factor=None,
    )


def hotspot_raster(rng, die, n_spots, base, amp_lo, amp_hi, s_frac, nx=512, ny=512):
    """Raster T(x, y) = base + sum_k A_k exp(-r_k^2 / (2 s^2)) over [0, die]^2.

    Vertex-centred: sample (ix, iy) sits at (ix*die/(nx-1), iy*die/(ny-1)).
    A_k ~ U(amp_lo, amp_hi); centres ~ U(die); s = s_frac * die (scalar or
    (lo, hi) range drawn per spot).
    """
    xs = np.linspace(0.0, die, nx)
    ys = np.linspace(0.0, die, ny)
    X, Y = np.meshgrid(xs, ys)
    T = np.full((ny, nx), float(base))
    for _ in range(n_spots):
        cx, cy = rng.uniform(0.0, die, size=2)
        A = rng.uniform(amp_lo, amp_hi) if amp_hi > amp_lo else amp_lo
        if isinstance(s_frac, tuple):
            s = rng.uniform(*s_frac) * die
        else:
            s = s_frac * die
        T += A * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * s * s))
    return dict(T=T, x0=0.0, y0=0.0, x1=die, y1=die)


def mc_factors(rng, n_samples, n_seg, cov=0.2):
    """Lognormal multipliers with mean 1 and the given CoV, independent per
    (sample, segment, parameter): returns (kappa_factor, sigc_factor)."""
    s_ln = math.sqrt(math.log(1.0 + cov * cov))
    mu = -0.5 * s_ln * s_ln
    kf = np.exp(rng.normal(mu, s_ln, size=(n_samples, n_seg)))
    sf = np.exp(rng.normal(mu, s_ln, size=(n_samples, n_seg)))
    return kf, sf


def _lognormal_currents(rng, k, median=0.707e-3, s_ln=0.98, lo=0.1e-3, hi=5e-3):
    return np.clip(rng.lognormal(math.log(median), s_ln, size=k), lo, hi)


def _pad_array(N, every):
    idx = np.arange(every // 2, N, every)
    return np.array([i * N + j for i in idx for j in idx], np.int32)


def via_mesh(seed=6, N=8, pitch=20e-6, R_via=2.0, W_via=0.2e-6, H_via=0.2e-6, I_lo=0.4e-3, I_hi=1.6e-3,
             cells=None):
    """Two-layer mesh with explicit via resistors: every crossing (i, j) has a
    lower-layer node i*N + j (horizontal stripes, layer 0) and an upper-layer
    node N*N + i*N + j (vertical stripes, layer 1) joined by a via resistor
    (seg_via = 1, resistance R_via).  Four corner pads on the upper layer, a
    U(I_lo, I_hi) sink on every lower-layer crossing."""
    rng = _rng(seed)
    rho = default_params()["rho_Cu"]
    g = stripe_mesh(N, pitch)
    nh = N * (N - 1)
    a = g["seg_a"].copy(); b = g["seg_b"].copy()
    a[nh:] += N * N; b[nh:] += N * N                     # vertical stripes on the upper nodes
    va = np.arange(N * N, dtype=np.int32); vb = va + N * N
    ns = a.size
    g["node_x"] = np.concatenate([g["node_x"], g["node_x"]])
    g["node_y"] = np.concatenate([g["node_y"], g["node_y"]])
    g["seg_a"] = np.concatenate([a, va]).astype(np.int32)
    g["seg_b"] = np.concatenate([b, vb]).astype(np.int32)
    g["seg_layer"] = np.concatenate([g["seg_layer"], np.zeros(N * N, np.int32)]).astype(np.int32)
    c = g["seg_cells"] if cells is None else np.full(ns, cells, np.int32)
    g["seg_cells"] = np.concatenate([c, np.ones(N * N, np.int32)]).astype(np.int32)
    g["seg_W"] = np.concatenate([g["seg_W"], np.full(N * N, W_via)])
    g["seg_H"] = np.concatenate([g["seg_H"], np.full(N * N, H_via)])
    g["seg_L"] = np.concatenate([g["seg_L"], np.full(N * N, H_via)])
    g["seg_R0"] = np.concatenate([rho * g["seg_L"][:ns] / (g["seg_W"][:ns] * g["seg_H"][:ns]), np.full(N * N, R_via)])
    g["seg_via"] = np.concatenate([np.zeros(ns, np.int8), np.ones(N * N, np.int8)])
    up = N * N
    g["pad_node"] = np.array([up, up + N - 1, up + N * (N - 1), up + N * N - 1], np.int32)
    g["pad_V"] = np.ones(4)
    g["sink_node"] = np.arange(N * N, dtype=np.int32)
    g["sink_I"] = rng.uniform(I_lo, I_hi, size=N * N)
    return g


def tiny_grid(seed=1, N=8, pitch=20e-6):
    """8x8 stripes of 7 x 20 um segments, 4 corner pads at 1 V, a sink on
    every crossing drawing U(0.5, 2) mA; uniform temperature (no map)."""
    rng = _rng(seed)
    g = stripe_mesh(N, pitch)
    g["pad_node"] = np.array([0, N - 1, N * (N - 1), N * N - 1], np.int32)
    g["pad_V"] = np.ones(4)
    g["sink_node"] = np.arange(N * N, dtype=np.int32)
    g["sink_I"] = rng.uniform(0.5e-3, 2e-3, size=N * N)
    return g


def mid_grid(seed=2, N=256, pitch=10e-6, n_spots=3, with_map=True, raster=512):
    """N x N stripes at 10 um, a pad every 32 crossings, 2 % of crossings as
    lognormal sinks (median 0.707 mA, s_ln 0.98, clipped to 0.1-5 mA), and a
    340 K map with 3 Gaussian +40 K hotspots of s = 15 % of the die width."""
    rng = _rng(seed)
    g = stripe_mesh(N, pitch)
    pads = _pad_array(N, 32 if N >= 64 else max(2, N // 2))
    g["pad_node"] = pads
    g["pad_V"] = np.ones(pads.size)
    free = np.setdiff1d(np.arange(N * N, dtype=np.int32), pads)
    k = max(1, int(round(0.02 * N * N)))
    g["sink_node"] = np.sort(rng.choice(free, size=k, replace=False)).astype(np.int32)
    g["sink_I"] = _lognormal_currents(rng, k)
    if with_map:
        die = (N - 1) * pitch
        g["thermal"] = hotspot_raster(rng, die, n_spots, 340.0, 40.0, 40.0, 0.15,
                                      nx=raster, ny=raster)
    return g


def mc_grid(seed=3, n_samples=1024, N=8, pitch=20e-6, cells_lo=32, cells_hi=1024):
    """The tiny grid with uneven trees: each stripe's total FD cell count is
    drawn log-uniform in [cells_lo, cells_hi] and split evenly over its N-1
    segments; n_samples sets of lognormal (CoV 20 %) kappa and sigma_crit
    factors per segment."""
    rng = _rng(seed)
    g = tiny_grid(seed=seed, N=N, pitch=pitch)
    tot = np.exp(rng.uniform(math.log(cells_lo), math.log(cells_hi), size=2 * N))
    per_seg = np.maximum(1, np.round(tot / (N - 1))).astype(np.int32)
    stripe = np.concatenate([np.repeat(np.arange(N), N - 1),
                             np.repeat(np.arange(N, 2 * N), N - 1)])
    g["seg_cells"] = per_seg[stripe].astype(np.int32)
    if n_samples > 0:
        g["kappa_factor"], g["sigc_factor"] = mc_factors(rng, n_samples, g["seg_a"].size)
    return g


def surrogate_grid(seed=11, N=128, pitch=10e-6, n_samples=32, raster=256):
    """Training / validation meshes of the learned surrogate: N x N stripes at
    10 um with a pad every 32 crossings, a seeded fraction (1-4 %) of the
    crossings as lognormal sinks whose median is scaled by U(0.6, 1.6), a
    random map of 1-8 hotspots (base U(330, 350) K, +U(20, 80) K, s = 8-20 %
    of the die) and n_samples sets of lognormal (CoV 20 %) kappa and
    sigma_crit factors per segment."""
    rng = _rng(seed)
    g = stripe_mesh(N, pitch)
    pads = _pad_array(N, 32 if N >= 64 else max(2, N // 2))
    g["pad_node"] = pads
    g["pad_V"] = np.ones(pads.size)
    free = np.setdiff1d(np.arange(N * N, dtype=np.int32), pads)
    k = max(1, int(round(rng.uniform(0.01, 0.04) * N * N)))
    g["sink_node"] = np.sort(rng.choice(free, size=k, replace=False)).astype(np.int32)
    g["sink_I"] = _lognormal_currents(rng, k, median=0.707e-3 * rng.uniform(0.6, 1.6))
    die = (N - 1) * pitch
    g["thermal"] = hotspot_raster(rng, die, int(rng.integers(1, 9)), rng.uniform(330.0, 350.0), 20.0, 80.0,
                                  (0.08, 0.20), nx=raster, ny=raster)
    if n_samples > 0:
        g["kappa_factor"], g["sigc_factor"] = mc_factors(rng, n_samples, g["seg_a"].size)
    return g


def large_grid(seed=5, N=2048, pitch=5e-6, n_samples=256, raster=512):
    """2048 x 2048 stripes at 5 um (10 cells per segment), a pad every 32
    crossings, 5 % lognormal sinks, 8 hotspots on 330 K with amplitudes
    U(0, 90) K, and n_samples MC factor sets."""
    rng = _rng(seed)
    g = stripe_mesh(N, pitch)
    pads = _pad_array(N, 32)
    g["pad_node"] = pads
    g["pad_V"] = np.ones(pads.size)
    free = np.setdiff1d(np.arange(N * N, dtype=np.int32), pads)
    k = int(round(0.05 * N * N))
    g["sink_node"] = np.sort(rng.choice(free, size=k, replace=False)).astype(np.int32)
    g["sink_I"] = _lognormal_currents(rng, k)
    die = (N - 1) * pitch
    g["thermal"] = hotspot_raster(rng, die, 8, 330.0, 0.0, 90.0, 0.15, nx=raster, ny=raster)
    if n_samples > 0:
        g["kappa_factor"], g["sigc_factor"] = mc_factors(rng, n_samples, g["seg_a"].size)
    return g


def tree_grid(kind, seed=0, seg_len=10e-6, cells=8, W=0.5e-6, H=0.2e-6, I_sink=2e-3,
              rho_Cu=None):
    """Single-layer branched test trees (one tree each) with one pad and sinks:
    'T' (3 arms from a junction), 'comb' (spine with 3 teeth), 'star'
    (5 arms), 'chain' (4 segments).  The pad sits at node 0; every other IR
    node draws a seeded U(0.5, 1.5) x I_sink."""
    if rho_Cu is None:
        rho_Cu = default_params()["rho_Cu"]
    rng = _rng(seed)
    if kind == "chain":
        xy = [(0, 0), (1, 0), (2, 0), (3, 0), (4, 0)]
        edges = [(0, 1), (1, 2), (2, 3), (3, 4)]
    elif kind == "T":
        xy = [(0, 0), (1, 0), (2, 0), (1, 1)]
        edges = [(0, 1), (1, 2), (1, 3)]
    elif kind == "comb":
        xy = [(0, 0), (1, 0), (2, 0), (3, 0), (1, 1), (2, 1), (3, 1)]
        edges = [(0, 1), (1, 2), (2, 3), (1, 4), (2, 5), (3, 6)]
    elif kind == "star":
        xy = [(0, 0), (1, 0), (2, 0), (1, 1), (1, -1), (0, 1)]
        edges = [(0, 1), (1, 2), (1, 3), (1, 4), (1, 5)]
    else:
        raise ValueError(kind)
    xy = np.array(xy, np.float64) * seg_len
    a = np.array([e[0] for e in edges], np.int32)
    b = np.array([e[1] for e in edges], np.int32)
    L = np.hypot(*(xy[b] - xy[a]).T)
    ns = a.size
    Wa = np.full(ns, W); Ha = np.full(ns, H)
    nn = xy.shape[0]
    return dict(
        N=0, pitch=seg_len,
        node_x=xy[:, 0].copy(), node_y=xy[:, 1].copy(),
        seg_a=a, seg_b=b, seg_layer=np.zeros(ns, np.int32),
        seg_R0=rho_Cu * L / (Wa * Ha), seg_W=Wa, seg_H=Ha, seg_L=L,
        seg_cells=np.full(ns, cells, np.int32),
        pad_node=np.array([0], np.int32), pad_V=np.ones(1),
        sink_node=np.arange(1, nn, dtype=np.int32),
        sink_I=I_sink * rng.uniform(0.5, 1.5, size=nn - 1),
        thermal=None, kappa_factor=None, sigc_factor=None,
    )


def config(name, **kw):
    """The five workloads by name: 'tiny' (8x8, 4,496 stress nodes), 'mid'
    (256x256 with map, 2,611,712 nodes), 'mc' (uneven 8x8 trees, 1,024
    samples), 'large' (2048x2048, 256 samples)."""
    if name == "tiny":
        return tiny_grid(**kw)
    if name == "mid":
        return mid_grid(**kw)
    if name == "mc":
        return mc_grid(**kw)
    if name == "large":
        return large_grid(**kw)
    raise ValueError(name)


def spice_netlist(seed=7, n_trees=4, n_seg=24, pitch_nm=10000, W=(0.5e-6, 0.8e-6), H=(0.2e-6, 0.3e-6),
                  R_via=1.0, n_vias=4, I_lo=0.2e-3, I_hi=0.7e-3, dx=0.5e-6):
    """A synthetic power-grid netlist in SPICE form with junction-heavy trees.

    Layer 1 holds n_trees random Manhattan trees (n_seg segments of 1-3
    lattice steps each, grown from random existing nodes, so many nodes are
    junctions); n_vias of each tree's nodes have a via (resistor R_via) up to
    layer 2, where one strap per tree links the via landings in order and
    carries a supply pad at each end.  Every layer-1 node other than the via
    ones draws a U(I_lo, I_hi) sink.  Node names n<layer>_<x>_<y> in nm.

    Returns (text, grid): the netlist text and the same grid as a dict, nodes
    numbered by first appearance in the text, segments and sources in text
    order (what a SPICE reader produces).
    """
    rng = _rng(seed)
    rho = default_params()["rho_Cu"]
    names, xs, ys, layers = [], [], [], []
    index = {}

    def node(layer, x, y):
        nm = "n%d_%d_%d" % (layer, x, y)
        if nm not in index:
            index[nm] = len(names)
            names.append(nm); xs.append(x * 1e-9); ys.append(y * 1e-9); layers.append(layer)
        return nm

    lines = ["* synthetic junction-heavy power grid (seed %d)" % seed]
    seg = dict(a=[], b=[], layer=[], cells=[], R=[], W=[], H=[], L=[], via=[])
    pads, sinks = [], []

    def wire(layer, n1, n2):
        # length = distance of the node coordinates in metres (as a reader computes it)
        i1, i2 = index[n1], index[n2]
        L = float(np.hypot(xs[i2] - xs[i1], ys[i2] - ys[i1]))
        R = rho * L / (W[layer - 1] * H[layer - 1])
        lines.append("R%d %s %s %.17g" % (len(seg["a"]) + 1, n1, n2, R))
        seg["a"].append(index[n1]); seg["b"].append(index[n2]); seg["layer"].append(layer)
        seg["cells"].append(max(1, int(math.floor(L / dx + 0.5)))); seg["R"].append(R)
        seg["W"].append(W[layer - 1]); seg["H"].append(H[layer - 1]); seg["L"].append(L); seg["via"].append(0)

    occupied = set()
    for t in range(n_trees):
        ox = t * 40 * pitch_nm
        pts = [(ox, 0)]
        occupied.add((ox, 0))
        tree_nodes = [node(1, ox, 0)]
        while len(tree_nodes) - 1 < n_seg:
            k = int(rng.integers(len(pts)))
            x0, y0 = pts[k]
            dxs, dys = [(1, 0), (-1, 0), (0, 1), (0, -1)][int(rng.integers(4))]
            steps = int(rng.integers(1, 4))
            path = [(x0 + dxs * pitch_nm * q, y0 + dys * pitch_nm * q) for q in range(1, steps + 1)]
            if any(pp in occupied for pp in path) or not (ox - 15 * pitch_nm <= path[-1][0] <= ox + 15 * pitch_nm):
                continue
            occupied.update(path)
            x1, y1 = path[-1]
            n1 = tree_nodes[k]
            n2 = node(1, x1, y1)
            wire(1, n1, n2)
            pts.append((x1, y1))
            tree_nodes.append(n2)
        vias = sorted(rng.choice(np.arange(1, len(tree_nodes)), size=n_vias, replace=False).tolist())
        landing = []
        for v in vias:
            x, y = pts[v]
            up = node(2, x, y)
            lines.append("R%d %s %s %.17g" % (len(seg["a"]) + 1, tree_nodes[v], up, R_via))
            seg["a"].append(index[tree_nodes[v]]); seg["b"].append(index[up]); seg["layer"].append(1)
            seg["cells"].append(1); seg["R"].append(R_via); seg["W"].append(0.2e-6); seg["H"].append(0.2e-6)
            seg["L"].append(0.2e-6); seg["via"].append(1)
            landing.append((x, y, up))
        landing.sort()
        for (xa, ya, na), (xb, yb, nb) in zip(landing[:-1], landing[1:]):
            wire(2, na, nb)
        for end in (landing[0][2], landing[-1][2]):
            lines.append("V%d %s 0 1.0" % (len(pads) + 1, end))
            pads.append(index[end])
        via_nodes = {tree_nodes[v] for v in vias}
        for nm in tree_nodes:
            if nm not in via_nodes:
                I = float(rng.uniform(I_lo, I_hi))
                lines.append("I%d %s 0 %.17g" % (len(sinks) + 1, nm, I))
                sinks.append((index[nm], I))
    lines.append(".end")
    g = dict(
        N=0, pitch=pitch_nm * 1e-9,
        node_x=np.array(xs), node_y=np.array(ys),
        seg_a=np.array(seg["a"], np.int32), seg_b=np.array(seg["b"], np.int32),
        seg_layer=np.array(seg["layer"], np.int32), seg_cells=np.array(seg["cells"], np.int32),
        seg_R0=np.array(seg["R"]), seg_W=np.array(seg["W"]), seg_H=np.array(seg["H"]), seg_L=np.array(seg["L"]),
        seg_via=np.array(seg["via"], np.int8),
        pad_node=np.array(pads, np.int32), pad_V=np.ones(len(pads)),
        sink_node=np.array([q[0] for q in sinks], np.int32), sink_I=np.array([q[1] for q in sinks]),
        thermal=None, kappa_factor=None, sigc_factor=None,
    )
    return "\n".join(lines) + "\n", g
