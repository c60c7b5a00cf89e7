"""Oracle for the coupled EM/TM stress, void and IR-drop flow (plain FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings of points the paper leaves open are stated where they are used; the
discretisation is a node-centred finite volume on each tree (Sec. III-D.4:
"finite-difference transient formulation ... similar to SunYu"):

  * a tree is a connected set of same-layer segments (vias separate trees);
    its stress nodes are the IR nodes it touches plus seg_cells-1 interior
    nodes per segment; node order is depth-first from the root (the
    lowest-id IR node of degree one), child segments in increasing id, a
    segment's interior nodes listed from the parent end;
  * face e joins node i to its parent; its direction is parent -> child;
    dx_e = L/cells, a_e = W H; V_i = sum over faces at i of a_e dx_e / 2;
  * Korhonen's PDE (Eq. tm_aware_korhonen_pde) integrated over node i's
    control volume gives C dsigma/dt = A sigma + f (Eq. em_tm_ode) with
    A_ij = g_e = a_e kappa_e / dx_e and f_parent -= a kappa G, f_child +=
    a kappa G, G = S + M along the face direction;
  * S = e Z rho j / Omega with j the current density along the face
    direction; M = Q / (Omega T_e) dT/dx; T_e = (T_i + T_parent)/2;
    kappa_e = D0 exp(-Ea/(k_B T_e)) B Omega / (k_B T_e) (Sec. III-D.1).
"""
import ctypes
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import build as _build

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(ctypes.c_long)
        L.orc_advance.restype = ctypes.c_int
        L.orc_advance.argtypes = [ctypes.c_int, lp, ip, dp, dp, dp, dp, dp, dp, ip, dp, dp,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_double, dp, dp, ctypes.c_int]
        L.orc_steady.restype = None
        L.orc_steady.argtypes = [ctypes.c_int, lp, ip, dp, dp, ctypes.c_double, dp]
        _LIB = L
    return _LIB


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


# ---------------------------------------------------------------------------
# Tree extraction (Sec. III-B "extracts the trees"; Sec. IV-A partition)
# ---------------------------------------------------------------------------

def build_trees(grid):
    """Partition the netlist into stress trees and lay out their FD nodes.

    Returns a dict of flat arrays over all stress nodes (see module doc) plus
    tree offsets.  Raises ValueError if a same-layer component has a cycle.
    """
    a = np.asarray(grid["seg_a"]); b = np.asarray(grid["seg_b"])
    layer = np.asarray(grid["seg_layer"]); cells = np.asarray(grid["seg_cells"])
    L = np.asarray(grid["seg_L"]); W = np.asarray(grid["seg_W"]); H = np.asarray(grid["seg_H"])
    x = np.asarray(grid["node_x"]); y = np.asarray(grid["node_y"])
    nseg = a.size
    via = np.asarray(grid["seg_via"], bool) if grid.get("seg_via") is not None else np.zeros(nseg, bool)
    # adjacency (node, layer) -> sorted list of wire segments (via resistors
    # join layers; they carry current but belong to no stress tree)
    adj = {}
    for s in range(nseg):
        if via[s]:
            continue
        adj.setdefault((int(a[s]), int(layer[s])), []).append(s)
        adj.setdefault((int(b[s]), int(layer[s])), []).append(s)
    seen = np.zeros(nseg, bool)
    seen[via] = True
    trees = []
    for s0 in range(nseg):            # trees ordered by their smallest segment id
        if seen[s0]:
            continue
        lay = int(layer[s0])
        comp, stack = [], [s0]
        seen[s0] = True
        while stack:
            s = stack.pop()
            comp.append(s)
            for nd in (int(a[s]), int(b[s])):
                for s2 in adj[(nd, lay)]:
                    if not seen[s2]:
                        seen[s2] = True
                        stack.append(s2)
        trees.append((lay, sorted(comp)))

    par, fseg, fdx, fa, fsign, px, py, ir, owner = [], [], [], [], [], [], [], [], []
    incident = []                     # per stress node: tree segments at an IR node
    off = [0]
    for lay, segs in trees:
        nodes = {}
        for s in segs:
            for nd in (int(a[s]), int(b[s])):
                nodes.setdefault(nd, []).append(s)
        if len(nodes) != len(segs) + 1:
            raise ValueError("same-layer component with a cycle: not a tree")
        leaves = [nd for nd, ss in nodes.items() if len(ss) == 1]
        root = min(leaves) if leaves else min(nodes)
        base = off[-1]
        cnt = 0

        def emit(parent, seg, dx, area, sign, xx, yy, irn, own, inc):
            nonlocal cnt
            par.append(parent); fseg.append(seg); fdx.append(dx); fa.append(area)
            fsign.append(sign); px.append(xx); py.append(yy); ir.append(irn)
            owner.append(own); incident.append(inc)
            cnt += 1
            return cnt - 1

        emit(-1, -1, 0.0, 0.0, 0, x[root], y[root], root, min(nodes[root]), sorted(nodes[root]))
        # iterative depth-first preorder; records are ("node", ir, local, came_by)
        # or ("seg", parent_ir, parent_local, seg, child_ir)
        stack = [("node", root, 0, -1)]
        visited = {root}
        while stack:
            rec = stack.pop()
            if rec[0] == "node":
                _, u, lu, came = rec
                kids = [s for s in sorted(nodes[u]) if s != came]
                for s in reversed(kids):     # reverse so the lowest id pops first
                    w = int(b[s]) if int(a[s]) == u else int(a[s])
                    if w in visited:
                        raise ValueError("cycle in tree")
                    visited.add(w)
                    stack.append(("seg", u, lu, s, w))
            else:
                _, uu, luu, s, w = rec
                c = int(cells[s]); dx = L[s] / c; area = W[s] * H[s]
                sign = 1 if int(a[s]) == uu else -1
                prev = luu
                for k in range(1, c):
                    t = k / c
                    prev = emit(prev, s, dx, area, sign,
                                x[uu] + t * (x[w] - x[uu]), y[uu] + t * (y[w] - y[uu]),
                                -1, s, [s])
                lw = emit(prev, s, dx, area, sign, x[w], y[w], w, min(nodes[w]),
                          sorted(nodes[w]))
                stack.append(("node", w, lw, s))
        off.append(base + cnt)
    tr = dict(
        n_trees=len(trees), off=np.array(off, np.int64),
        layer=np.array([t[0] for t in trees], np.int32),
        tree_segs=[t[1] for t in trees],
        par=np.array(par, np.int32), face_seg=np.array(fseg, np.int32),
        face_dx=np.array(fdx), face_a=np.array(fa), face_sign=np.array(fsign, np.int32),
        x=np.array(px), y=np.array(py), ir=np.array(ir, np.int32),
        owner_seg=np.array(owner, np.int32), incident=incident,
    )
    tr["n_nodes"] = int(tr["off"][-1])
    # global parent index (for vectorised face maths)
    gp = tr["par"].astype(np.int64).copy()
    for t in range(tr["n_trees"]):
        o = tr["off"][t]; e = tr["off"][t + 1]
        gp[o + 1:e] += o
    gp[tr["off"][:-1]] = -1
    tr["gpar"] = gp
    return tr


# ---------------------------------------------------------------------------
# Temperature, diffusivity and forcing (Sec. III-A, III-D.1)
# ---------------------------------------------------------------------------

def bilinear(thermal, xs, ys):
    """Bilinear interpolation of a vertex-centred raster T[iy, ix] covering
    [x0, x1] x [y0, y1]; points outside are clamped to the border."""
    T = np.asarray(thermal["T"], np.float64)
    ny, nx = T.shape
    fx = (np.asarray(xs) - thermal["x0"]) / (thermal["x1"] - thermal["x0"]) * (nx - 1)
    fy = (np.asarray(ys) - thermal["y0"]) / (thermal["y1"] - thermal["y0"]) * (ny - 1)
    fx = np.clip(fx, 0.0, nx - 1); fy = np.clip(fy, 0.0, ny - 1)
    ix = np.minimum(np.floor(fx).astype(np.int64), nx - 2)
    iy = np.minimum(np.floor(fy).astype(np.int64), ny - 2)
    tx = fx - ix; ty = fy - iy
    return ((1 - tx) * (1 - ty) * T[iy, ix] + tx * (1 - ty) * T[iy, ix + 1]
            + (1 - tx) * ty * T[iy + 1, ix] + tx * ty * T[iy + 1, ix + 1])


def node_temperature(tr, thermal, T0):
    if thermal is None:
        return np.full(tr["n_nodes"], float(T0))
    return bilinear(thermal, tr["x"], tr["y"])


def kappa_of_T(T, p):
    """kappa = D_a B Omega / (k_B T), D_a = D0 exp(-Ea / (k_B T))."""
    return p["D0"] * np.exp(-p["Ea"] / (p["k_B"] * T)) * p["B_modulus"] * p["Omega"] / (p["k_B"] * T)


def tree_physics(tr, p, Tn, kappa_factor=None, sigc_factor=None):
    """Static per-node / per-face arrays for one sample.

    Returns dict with V, g (face conductance at the child node), leak (Robin
    coefficient per node), kap_a (a kappa per face), M (TM gradient term per
    face), sig_crit (per node).  Face arrays are indexed by the child node;
    roots hold 0.
    """
    n = tr["n_nodes"]
    gp = tr["gpar"]
    child = np.nonzero(gp >= 0)[0]
    parent = gp[child]
    seg = tr["face_seg"][child]
    dx = tr["face_dx"][child]; area = tr["face_a"][child]
    Te = 0.5 * (Tn[child] + Tn[parent])
    kap = kappa_of_T(Te, p)
    if kappa_factor is not None:
        kap = kap * kappa_factor[seg]
    kap_a = np.zeros(n); kap_a[child] = area * kap
    g = np.zeros(n); g[child] = area * kap / dx
    M = np.zeros(n); M[child] = p["Q_star"] / (p["Omega"] * Te) * (Tn[child] - Tn[parent]) / dx
    V = np.zeros(n)
    np.add.at(V, child, 0.5 * area * dx)
    np.add.at(V, parent, 0.5 * area * dx)
    leak = np.zeros(n)
    np.add.at(leak, child, area * kap / p["delta"])
    np.add.at(leak, parent, area * kap / p["delta"])
    sc = np.full(n, float(p["sigma_crit"]))
    if sigc_factor is not None:
        sc = sc * sigc_factor[tr["owner_seg"]]
    return dict(V=V, g=g, leak=leak, kap_a=kap_a, M=M, sig_crit=sc, Te=np.r_[Te], child=child)


def face_G(tr, p, phys, j_seg):
    """G = S + M per face (child-indexed), S = e Z rho j_face / Omega."""
    n = tr["n_nodes"]
    child = phys["child"]
    jf = tr["face_sign"][child] * j_seg[tr["face_seg"][child]]
    G = np.zeros(n)
    G[child] = p["e_charge"] * p["Z_star"] * p["rho_Cu"] * jf / p["Omega"] + phys["M"][child]
    return G


def forcing(tr, phys, G):
    """f_i = -sum over faces at i of s_{i,e} a_e kappa_e G_e (s = +1 at the tail)."""
    n = tr["n_nodes"]
    child = phys["child"]
    q = phys["kap_a"][child] * G[child]
    f = np.zeros(n)
    np.add.at(f, tr["gpar"][child], -q)
    np.add.at(f, child, q)
    return f


# ---------------------------------------------------------------------------
# IR drop (Sec. III-C, Eq. ir_drop_mna)
# ---------------------------------------------------------------------------

def ir_solve(grid, R):
    """Nodal analysis: G u = -I_sink on non-pad nodes, pads held at pad_V.
    Returns node voltages u (all nodes).  Direct sparse solve."""
    n = len(grid["node_x"])
    a = np.asarray(grid["seg_a"]); b = np.asarray(grid["seg_b"])
    g = 1.0 / np.asarray(R, np.float64)
    fixed = np.zeros(n, bool); fixed[grid["pad_node"]] = True
    u = np.zeros(n); u[grid["pad_node"]] = grid["pad_V"]
    free = np.nonzero(~fixed)[0]
    idx = -np.ones(n, np.int64); idx[free] = np.arange(free.size)
    rows, cols, vals = [], [], []
    rhs = np.zeros(free.size)
    np.add.at(rhs, idx[grid["sink_node"]][~fixed[grid["sink_node"]]],
              -np.asarray(grid["sink_I"])[~fixed[grid["sink_node"]]])
    for (p_, q_) in ((a, b), (b, a)):
        fp = ~fixed[p_]
        rows.append(idx[p_[fp]]); cols.append(idx[p_[fp]]); vals.append(g[fp])
        both = fp & ~fixed[q_]
        rows.append(idx[p_[both]]); cols.append(idx[q_[both]]); vals.append(-g[both])
        pad_nb = fp & fixed[q_]
        np.add.at(rhs, idx[p_[pad_nb]], g[pad_nb] * u[q_[pad_nb]])
    Gm = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(free.size, free.size))
    u[free] = spla.spsolve(Gm, rhs)
    return u


def current_density(grid, u, R):
    """j_s = (u_a - u_b) / (R_s W_s H_s): positive when current flows a -> b."""
    a = np.asarray(grid["seg_a"]); b = np.asarray(grid["seg_b"])
    return (u[a] - u[b]) / (np.asarray(R) * grid["seg_W"] * grid["seg_H"])


def max_drop(u, Vdd):
    return float(np.max((Vdd - u) / Vdd))


# ---------------------------------------------------------------------------
# Screen (Sec. III-B)
# ---------------------------------------------------------------------------

def steady_stress(tr, p, phys, G):
    """Closed-form steady state per tree (no voids): sigma_child -
    sigma_parent = dx G on every face, constant from atom conservation."""
    dxG = tr["face_dx"] * G
    out = np.zeros(tr["n_nodes"])
    lib().orc_steady(tr["n_trees"], _p(tr["off"], ctypes.c_long),
                     _p(np.ascontiguousarray(tr["par"]), ctypes.c_int),
                     _p(np.ascontiguousarray(phys["V"]), ctypes.c_double),
                     _p(np.ascontiguousarray(dxG), ctypes.c_double),
                     float(p["sigma_T"]), _p(out, ctypes.c_double))
    return out


def screen(tr, p, phys, G):
    """Mortal iff some node's steady stress exceeds its critical stress.
    Returns (mortal[n_trees] bool, sigma_ss_max[n_trees], sigma_ss)."""
    ss = steady_stress(tr, p, phys, G)
    mortal = np.zeros(tr["n_trees"], bool); smax = np.zeros(tr["n_trees"])
    for t in range(tr["n_trees"]):
        o, e = tr["off"][t], tr["off"][t + 1]
        mortal[t] = bool(np.any(ss[o:e] > phys["sig_crit"][o:e]))
        smax[t] = ss[o:e].max()
    return mortal, smax, ss


# ---------------------------------------------------------------------------
# Stress advance (Sec. III-D.4, IV-B) -- C core
# ---------------------------------------------------------------------------

class StressState:
    """sigma, void flags / volumes / segments / nucleation times per node."""

    def __init__(self, tr, p):
        n = tr["n_nodes"]
        self.sigma = np.full(n, float(p["sigma_T"]))
        self.void = np.zeros(n, np.int32)
        self.vol = np.zeros(n)
        self.t_nuc = np.full(n, np.nan)
        self.vseg = -np.ones(n, np.int32)

    def copy(self):
        c = object.__new__(StressState)
        for k, v in self.__dict__.items():
            setattr(c, k, v.copy())
        return c


def advance(tr, p, phys, f, st, t0, dt, n_steps, margin=None, n_threads=0, gap=None):
    """n_steps backward-Euler steps of every tree; returns new void count."""
    L = lib()
    return L.orc_advance(
        tr["n_trees"], _p(tr["off"], ctypes.c_long),
        _p(np.ascontiguousarray(tr["par"]), ctypes.c_int),
        _p(np.ascontiguousarray(phys["V"]), ctypes.c_double),
        _p(np.ascontiguousarray(phys["g"]), ctypes.c_double),
        _p(np.ascontiguousarray(f), ctypes.c_double),
        _p(np.ascontiguousarray(phys["leak"]), ctypes.c_double),
        _p(np.ascontiguousarray(phys["sig_crit"]), ctypes.c_double),
        _p(st.sigma, ctypes.c_double), _p(st.void, ctypes.c_int),
        _p(st.vol, ctypes.c_double), _p(st.t_nuc, ctypes.c_double),
        float(t0), float(dt), int(n_steps), float(p["B_modulus"]),
        None if margin is None else _p(margin, ctypes.c_double),
        None if gap is None else _p(gap, ctypes.c_double), int(n_threads))


def assign_void_segments(tr, st, j_seg, new_nodes):
    """Segment that a new void degrades: an interior node's own segment; at
    an IR node, the incident tree segment with the larger |j| (lower id on
    ties), chosen with the currents of the step in which it nucleated."""
    for v in new_nodes:
        inc = tr["incident"][v]
        best = inc[0]
        for s in inc[1:]:
            if abs(j_seg[s]) > abs(j_seg[best]):
                best = s
        st.vseg[v] = best


# ---------------------------------------------------------------------------
# Void growth resistance (Sec. III-D.3) and TTF (Eq. ttf_calculation, Sec. V)
# ---------------------------------------------------------------------------

R_OPEN = 1.0e9   # Ohm: open-circuit sentinel of a severed via (early failure)


def up_vias(grid):
    """Per IR node: the via resistor to a node of a strictly higher metal
    layer (lowest segment id when several), -1 if none.  A node's layer is
    the layer of its wire segments."""
    n = len(grid["node_x"])
    a = np.asarray(grid["seg_a"]); b = np.asarray(grid["seg_b"]); layer = np.asarray(grid["seg_layer"])
    via = np.asarray(grid["seg_via"], bool) if grid.get("seg_via") is not None else np.zeros(a.size, bool)
    nl = np.full(n, -1)
    for s in np.nonzero(~via)[0]:
        nl[a[s]] = layer[s]; nl[b[s]] = layer[s]
    up = np.full(n, -1)
    for s in np.nonzero(via)[0]:
        for u, w in ((a[s], b[s]), (b[s], a[s])):
            if nl[u] >= 0 and nl[w] > nl[u] and up[u] < 0:
                up[u] = s
    return up


def void_resistance(grid, p, st, tr=None):
    """Late failure (Sec. III-D.3): R_s = R0_s + sum over voids on s of
    max(0, dR), dR = (V_v - V_crit)/(W H) [rho_Ta/(h_Ta(2H+W)) - rho_Cu/(H W)],
    V_crit = W * W * H (void length W: width is the critical dimension).
    Early failure (Sec. IV-C, explicit via resistors only): a void at an IR
    node that connects upward through a via to a strictly higher layer severs
    that via once its volume exceeds V_crit: the via's resistance becomes the
    open-circuit sentinel R_OPEN.  Without via resistors only late failure
    applies."""
    R = np.array(grid["seg_R0"], np.float64, copy=True)
    vn = np.nonzero(st.void)[0]
    up = up_vias(grid) if grid.get("seg_via") is not None and tr is not None else None
    for v in vn:
        s = st.vseg[v]
        W = grid["seg_W"][s]; H = grid["seg_H"][s]
        Vc = W * W * H
        coef = p["rho_Ta"] / (p["h_Ta"] * (2 * H + W)) - p["rho_Cu"] / (H * W)
        dR = (st.vol[v] - Vc) / (W * H) * coef
        if dR > 0.0:
            R[s] += dR
        if up is not None and tr["ir"][v] >= 0 and up[tr["ir"][v]] >= 0 and st.vol[v] > Vc:
            R[up[tr["ir"][v]]] = R_OPEN
    return R


def crossing_time(t_prev, d_prev, d_now, dt, thr):
    return t_prev + (thr - d_prev) / (d_now - d_prev) * dt


def run_ttf(grid, p, sample=None, screen_first=False, record=False, n_threads=0,
            n_outer=None, stepper=None, keep_state=False, Tn=None):
    """Coupled EM/TM/IR aging loop (Sec. IV-A) for one sample.

    Each outer step: G and f from the current j -> n_inner BE steps with
    nucleation -> resistance from void volumes -> IR re-solve -> max drop.
    TTF is the linear-interpolated first crossing of ir_fail_frac (0 if the
    initial drop already exceeds it, inf if never crossed).  `stepper`
    replaces the BE advance (Krylov path): stepper(tr, p, phys, f, st, t0,
    dt, n) -> new void count.  Tn replaces the node temperatures sampled
    from the map (e.g. a Joule-heating profile).
    """
    tr = build_trees(grid) if "trees" not in grid else grid["trees"]
    kf = None if sample is None or grid.get("kappa_factor") is None else grid["kappa_factor"][sample]
    sf = None if sample is None or grid.get("sigc_factor") is None else grid["sigc_factor"][sample]
    if Tn is None:
        Tn = node_temperature(tr, grid.get("thermal"), p["T0"])
    phys = tree_physics(tr, p, Tn, kf, sf)
    n_out = p["n_outer"] if n_outer is None else n_outer
    dto = p["horizon"] / p["n_outer"]
    dti = dto / p["n_inner"]
    thr = p["ir_fail_frac"]
    R = np.array(grid["seg_R0"], np.float64, copy=True)
    u = ir_solve(grid, R)
    j = current_density(grid, u, R)
    drops = [max_drop(u, p["Vdd"])]
    ttf = 0.0 if drops[0] >= thr else math.inf
    st = StressState(tr, p)
    mortal = None
    if screen_first:
        mortal, _, _ = screen(tr, p, phys, face_G(tr, p, phys, j))
    margin = np.full(tr["n_trees"], np.inf)
    gap = np.full(tr["n_trees"], np.inf)
    node_steps = 0
    for k in range(n_out):
        G = face_G(tr, p, phys, j)
        f = forcing(tr, phys, G)
        before = st.void.copy()
        mk = np.zeros(tr["n_trees"])
        gk = np.full(tr["n_trees"], np.inf)
        if stepper is None:
            advance(tr, p, phys, f, st, k * dto, dti, p["n_inner"], margin=mk, n_threads=n_threads, gap=gk)
        else:
            stepper(tr, p, phys, f, st, k * dto, dti, p["n_inner"], margin=mk)
        margin = np.minimum(margin, mk)
        gap = np.minimum(gap, gk)
        node_steps += tr["n_nodes"] * p["n_inner"]
        new = np.nonzero(st.void & ~before)[0]
        assign_void_segments(tr, st, j, new)
        R_new = void_resistance(grid, p, st, tr)
        if not np.array_equal(R_new, R):
            R = R_new
            u = ir_solve(grid, R)
            j = current_density(grid, u, R)
        drops.append(max_drop(u, p["Vdd"]))
        if math.isinf(ttf) and drops[-2] < thr <= drops[-1]:
            ttf = crossing_time(k * dto, drops[-2], drops[-1], dto, thr)
    res = dict(ttf=ttf, drop0=drops[0], final_drop=drops[-1], drops=np.array(drops),
               n_voids=int(st.void.sum()), margin=margin, gap=gap, node_steps=node_steps,
               mortal=mortal)
    tn = np.full(tr["n_trees"], np.inf)
    for t in range(tr["n_trees"]):
        o, e = tr["off"][t], tr["off"][t + 1]
        w = st.t_nuc[o:e]
        if np.any(np.isfinite(w)):
            tn[t] = np.nanmin(w)
    res["t_nuc_tree"] = tn
    res["void_nodes"] = np.nonzero(st.void)[0]
    res["void_seg"] = st.vseg[res["void_nodes"]]
    if keep_state or record:
        res["state"] = st; res["R"] = R; res["u"] = u; res["j"] = j
        res["trees"] = tr; res["phys"] = phys
    return res
