"""FP64 reference for the learned surrogate's MLP (forward, backward, Adam).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The surrogate is not part of the paper; its network is a plain multilayer
perceptron: standardised inputs x (24 tree features), hidden layers
h_l = relu(W_l h_{l-1} + b_l) of width 256, and a linear head y = W h + b
with 2 outputs (log10 nucleation time, critical-node position along the
tree).  Loss: half the mean over the batch of the squared error summed over
outputs.  Optimiser: Adam with bias correction.
"""
import numpy as np


def init(sizes, seed=0):
    """He-normal weights (fan-in), zero biases; sizes = [24, 256, ..., 2]."""
    rng = np.random.default_rng(seed)
    params = []
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        params.append((rng.normal(0.0, np.sqrt(2.0 / fi), size=(fo, fi)), np.zeros(fo)))
    return params


def forward(params, x):
    """Returns (y, cache) for inputs x [B, fin]."""
    acts = [x]
    pre = []
    h = x
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        pre.append(z)
        h = np.maximum(z, 0.0) if li + 1 < len(params) else z
        acts.append(h)
    return h, (acts, pre)


def loss(y, t):
    d = y - t
    return 0.5 * float(np.mean(np.sum(d * d, axis=1)))


def backward(params, cache, y, t):
    """Gradients of loss() with respect to every (W, b)."""
    acts, pre = cache
    B = y.shape[0]
    g = (y - t) / B                                   # dL/dy
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        if li + 1 < len(params):
            g = g * (pre[li] > 0.0)                   # relu'
        grads[li] = (g.T @ acts[li], g.sum(axis=0))
        g = g @ W
    return grads


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        out = []
        for k, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
            new = []
            for j, (p, gp) in enumerate(((W, gW), (b, gb))):
                m = self.b1 * self.m[k][j] + (1.0 - self.b1) * gp
                v = self.b2 * self.v[k][j] + (1.0 - self.b2) * gp * gp
                self.m[k] = tuple(m if q == j else self.m[k][q] for q in range(2))
                self.v[k] = tuple(v if q == j else self.v[k][q] for q in range(2))
                new.append(p - self.lr * (m / c1) / (np.sqrt(v / c2) + self.eps))
            out.append(tuple(new))
        return out
