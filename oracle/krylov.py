"""Oracle for the constant-input block rational Krylov reduced model (Sec. IV-E).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Per tree, the BE descriptor system C s' = A s + f (Eq. rak_lti) is projected on
the block rational Krylov space of R C with R = (s0 C - A)^-1 built from the
starting block [R C s0, R f] (Eq. rak_start_block, Alg. 1), integrated in the
reduced space by backward Euler (Eq. rak_reduced) and lifted back.

Readings (where the paper is silent):
  * shift time t_s = eta L_max^2 / (pi^2 kappa_bar) (Eq. rak_shift_time) with
    L_max the longest path in the tree (its diameter, in metres) and kappa_bar
    the face-volume-weighted mean of kappa;
  * breakdown is measured against each block's own size, since the
    propagation operator R C has norm ~ t_s and a threshold tied to ||F0||
    would not be scale free: a starting-block column whose norm after
    orthogonalisation falls under 1e-10 of the largest starting column is
    dropped (at t = 0 the stress is zero, so the first column drops); a later
    block W ends the iteration when ||H_{j+1,j}||_F < 1e-10 ||W||_F (the
    paper's ||H|| < eps test), and sends the tree back to full backward Euler
    when only some of its columns fall under that bound (rank deficiency);
  * Krylov is used for trees with n >= max(3q, 30) (Eq. krylov_threshold);
  * bases are cached per tree (Sec. IV-E.4) under the key the paper gives:
    the descriptor matrices and s0.  Within a run C and s0 are fixed and A
    changes only when a void nucleates, so the key is (tree, void set).  A
    cached basis was built from an earlier stress and forcing, and reusing
    it as it stands loses the new input (on the 8 x 8 grid that moves the TTF
    by 21 %), so every hit is augmented by the current starting block
    [R C s0, R f], orthogonalised twice against the cached columns (a
    column whose norm falls under 1e-10 of its own is dropped).  The step
    that (re)builds the basis from the current stress and forcing uses it
    without augmentation, since that block is already its first block.
    (policy="forcing" keys on the forcing as well and rebuilds whenever it
    changes: the same accuracy, far more builds; policy="stale" reuses the
    cached basis as it stands.);
  * nucleation is checked on the lifted stress after every reduced step, as
    in the full-order path.
"""
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import flow as F


def tree_system(tr, phys, f, void, t):
    """Sparse C (diagonal), A and f of tree t (local indices)."""
    o, e = int(tr["off"][t]), int(tr["off"][t + 1])
    n = e - o
    par = tr["par"][o:e]
    g = phys["g"][o:e]
    rows, cols, vals = [], [], []
    diag = np.zeros(n)
    for i in range(1, n):
        q = par[i]
        rows += [i, q]; cols += [q, i]; vals += [g[i], g[i]]
        diag[i] -= g[i]; diag[q] -= g[i]
    diag -= phys["leak"][o:e] * (void[o:e] != 0)
    A = sp.csc_matrix((np.concatenate([vals, diag]), (np.concatenate([rows, np.arange(n)]),
                                                      np.concatenate([cols, np.arange(n)]))), shape=(n, n))
    C = sp.diags(phys["V"][o:e]).tocsc()
    return C, A, f[o:e].copy()


def shift_time(tr, phys, t, eta):
    """t_s = eta L_max^2 / (pi^2 kappa_bar)."""
    o, e = int(tr["off"][t]), int(tr["off"][t + 1])
    par = tr["par"][o:e]; dx = tr["face_dx"][o:e]; a = tr["face_a"][o:e]
    kap = np.where(a > 0, phys["kap_a"][o:e] / np.where(a > 0, a, 1.0), 0.0)
    w = a * dx
    kbar = float((w[1:] * kap[1:]).sum() / w[1:].sum())
    n = e - o
    # tree diameter: farthest node from the root, then farthest from that node
    nbr = [[] for _ in range(n)]
    for i in range(1, n):
        nbr[i].append((par[i], dx[i])); nbr[par[i]].append((i, dx[i]))

    def far(src):
        dist = np.full(n, -1.0); dist[src] = 0.0; stack = [src]
        while stack:
            u = stack.pop()
            for v, d in nbr[u]:
                if dist[v] < 0:
                    dist[v] = dist[u] + d; stack.append(v)
        return int(np.argmax(dist)), float(dist.max())

    u, _ = far(0)
    _, L = far(u)
    return eta * L * L / (math.pi ** 2 * kbar)


def krylov_basis(C, A, f, sigma0, s0, q, eps_rel=1e-10, ortho="mgs"):
    """Alg. 1.  Returns (V, A_h, C_h, f_h, status) with status 'ok',
    'empty' (nothing to reduce) or 'rank' (rank-deficient later block).
    ortho: "mgs" orthogonalises each new block against the earlier blocks
    block by block (twice) and then within itself by a QR; "cgs2" takes the
    block's columns one at a time, each orthogonalised against every earlier
    column by classical Gram-Schmidt applied twice.  The two span the same
    space in exact arithmetic; comparing them measures how far rounding
    alone moves the reduced model."""
    K = (s0 * C - A).tocsc()
    lu = spla.splu(K)

    def Mop(X):
        return lu.solve(np.asarray(C @ X))

    F0 = np.column_stack([lu.solve(C @ sigma0), lu.solve(f)])
    eps = eps_rel * np.linalg.norm(F0, axis=0).max()
    if eps == 0.0:
        return None, None, None, None, "empty"
    # thin QR of the starting block, dropping columns under eps
    cols = []
    for k in range(F0.shape[1]):
        w = F0[:, k].copy()
        for _ in range(2):
            for v in cols:
                w -= v * (v @ w)
        nw = np.linalg.norm(w)
        if nw >= eps_rel * np.linalg.norm(F0[:, k]) and nw >= eps:
            cols.append(w / nw)
    if not cols:
        return None, None, None, None, "empty"
    blocks = [np.column_stack(cols)]
    for j in range(1, q):
        W = Mop(blocks[-1])
        epsj = eps_rel * np.linalg.norm(W)
        if ortho == "cgs2":
            prev = np.column_stack(blocks)
            qs, norms = [], []
            for k in range(W.shape[1]):
                w = W[:, k].copy()
                for _ in range(2):
                    B = np.column_stack([prev] + qs) if qs else prev
                    w = w - B @ (B.T @ w)
                nw = np.linalg.norm(w)
                norms.append(nw)
                qs.append(w / nw if nw > 0 else w)
            if math.sqrt(sum(v * v for v in norms)) < epsj:
                break
            if min(norms) < epsj:
                return None, None, None, None, "rank"
            blocks.append(np.column_stack(qs))
            continue
        for _ in range(2):                      # block modified Gram-Schmidt, applied twice
            for Vi in blocks:                   # (the second pass restores orthogonality
                H = Vi.T @ W                    # lost to rounding; it leaves the span as is)
                W = W - Vi @ H
        Q, Rr = np.linalg.qr(W)
        d = np.abs(np.diag(Rr))
        if np.linalg.norm(Rr) < epsj:
            break
        if np.any(d < epsj):
            return None, None, None, None, "rank"
        blocks.append(Q)
    V = np.column_stack(blocks)
    Ah = V.T @ (A @ V)
    Ch = V.T @ (C @ V)
    fh = V.T @ f
    return V, Ah, Ch, fh, "ok"


def augment(V, lu, C, sigma0, f, eps_rel=1e-10):
    """A cached basis V extended by the current starting block
    [R C s0, R f] (R = (s0 C - A)^-1 through the cached factors `lu`), each
    column orthogonalised twice (classical Gram-Schmidt) against V and the
    columns already added; a column under eps_rel of its own norm after
    that is dropped."""
    cols = [V[:, i] for i in range(V.shape[1])]
    for x in (lu.solve(C @ sigma0), lu.solve(f)):
        nx = np.linalg.norm(x)
        if not nx > 0.0:
            continue
        w = x.copy()
        for _ in range(2):
            B = np.column_stack(cols)
            w = w - B @ (B.T @ w)
        nw = np.linalg.norm(w)
        if nw >= eps_rel * nx:
            cols.append(w / nw)
    return np.column_stack(cols)


class KrylovStepper:
    """Drop-in replacement for flow.advance inside flow.run_ttf."""

    def __init__(self, q=10, eta=1.0, n_threads=0, cache=True, policy="augment", ortho="mgs"):
        if policy not in ("augment", "forcing", "stale"):
            raise ValueError("policy must be 'augment', 'forcing' or 'stale'")
        self.ortho = ortho
        self.q = q
        self.eta = eta
        self.n_threads = n_threads
        self.n_reduced = 0
        self.n_fallback = 0
        self.n_built = 0
        self.policy = policy
        self.cache = {} if cache else None

    def use_krylov(self, n):
        return n >= max(3 * self.q, 30)

    def __call__(self, tr, p, phys, f, st, t0, dt, n_steps, margin=None):
        total = 0
        Binv = 1.0 / p["B_modulus"]
        for t in range(tr["n_trees"]):
            o, e = int(tr["off"][t]), int(tr["off"][t + 1])
            n = e - o
            if not self.use_krylov(n):
                total += self._be(tr, p, phys, f, st, t0, dt, n_steps, t, margin)
                continue
            sc = phys["sig_crit"][o:e]
            s0 = 1.0 / shift_time(tr, phys, t, self.eta)
            k = 0
            mmin = math.inf
            while k < n_steps:
                C, A, ft = tree_system(tr, phys, f, st.void, t)
                sig = st.sigma[o:e]
                key = (t, tuple(np.nonzero(st.void[o:e])[0]), s0)
                if self.policy == "forcing":
                    key = key + (ft.tobytes(),)
                if self.cache is not None and key in self.cache:
                    V, lu = self.cache[key]
                    if self.policy == "augment":
                        V = augment(V, lu, C, sig, ft)
                    Ah, Ch, fh, status = V.T @ (A @ V), V.T @ (C @ V), V.T @ ft, "ok"
                else:
                    V, Ah, Ch, fh, status = krylov_basis(C, A, ft, sig, s0, self.q, ortho=self.ortho)
                    self.n_built += 1
                    if status == "ok" and self.cache is not None:
                        self.cache[key] = (V, spla.splu((s0 * C - A).tocsc()))
                if status != "ok":
                    self.n_fallback += 1
                    total += self._be(tr, p, phys, f, st, t0 + k * dt, dt, n_steps - k, t, margin)
                    break
                self.n_reduced += 1
                Mh = Ch - dt * Ah
                sh = V.T @ st.sigma[o:e]
                nucleated = False
                while k < n_steps:
                    sh = np.linalg.solve(Mh, Ch @ sh + dt * fh)
                    prev = st.sigma[o:e].copy()
                    st.sigma[o:e] = V @ sh
                    s = st.sigma[o:e]
                    vn = np.nonzero(st.void[o:e])[0]
                    st.vol[o + vn] += dt * Binv * phys["leak"][o + vn] * s[vn]
                    m = np.where(st.void[o:e] != 0, -np.inf, s - sc)
                    arg = int(np.argmax(m))
                    best = m[arg]
                    if np.isfinite(best):
                        mmin = min(mmin, abs(best) / sc[arg])
                    k += 1
                    if best >= 0.0:
                        m0 = prev[arg] - sc[arg]
                        frac = -m0 / (best - m0) if m0 < 0.0 else 0.0
                        st.void[o + arg] = 1
                        st.vol[o + arg] = 0.0
                        st.t_nuc[o + arg] = t0 + (k - 1 + frac) * dt
                        total += 1
                        nucleated = True
                        break
                if not nucleated:
                    break
            if margin is not None:
                margin[t] = min(margin[t], mmin) if margin[t] > 0 else mmin
        return total

    def _be(self, tr, p, phys, f, st, t0, dt, n_steps, t, margin):
        off = np.array([tr["off"][t], tr["off"][t + 1]], np.int64)
        mk = np.zeros(1)
        sub = dict(tr, n_trees=1, off=off)
        nv = F.advance(sub, p, phys, f, st, t0, dt, n_steps, margin=mk, n_threads=self.n_threads)
        if margin is not None:
            margin[t] = mk[0]
        return nv
