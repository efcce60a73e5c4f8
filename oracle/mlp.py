"""FP64 oracle of the density-reconstruction MLP (test infrastructure only).

The network maps a feature vector (noisy low-order Chebyshev moments and
degree statistics of a graph) to a B-bin spectral histogram.  This part has
no counterpart in the paper; it is checked here against its own definition:

    a_0 = x
    z_l = a_{l-1} W_l^T + b_l            (W_l: out_l x in_l)
    a_l = relu(z_l)          for hidden layers, a_L = z_L (logits)
    p   = softmax(a_L)                  (row-wise)
    loss = -(1/B_rows) sum_rows sum_bins t * log p       (cross-entropy
           against a target histogram t, rows of t sum to 1)

Backward: d a_L = (p - t) / B_rows; d z_l = d a_l * relu'(z_l) (hidden);
d W_l = d z_l^T a_{l-1}; d b_l = column sums of d z_l; d a_{l-1} = d z_l W_l.
Adam (Kingma & Ba 2015, Algorithm 1) with bias correction.

Pinned by central finite differences (tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np

__all__ = ["mlp_init", "mlp_forward", "mlp_loss_grad", "adam_step", "graph_stats", "mlp_features",
           "normalize_hist"]


def mlp_init(sizes, rng: np.random.Generator):
    """He-uniform weights, zero biases: list of (W, b) in float64."""
    params = []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / fan_in)
        params.append((rng.uniform(-lim, lim, (fan_out, fan_in)), np.zeros(fan_out)))
    return params


def mlp_forward(params, x):
    """Softmax probabilities and the cached pre-activations."""
    a = np.asarray(x, np.float64)
    zs, acts = [], [a]
    for l, (w, b) in enumerate(params):
        z = a @ w.T + b
        zs.append(z)
        a = np.maximum(z, 0.0) if l + 1 < len(params) else z
        acts.append(a)
    logits = acts[-1]
    e = np.exp(logits - logits.max(axis=1, keepdims=True))
    p = e / e.sum(axis=1, keepdims=True)
    return p, zs, acts


def mlp_loss_grad(params, x, t):
    """Cross-entropy loss and its gradient [(dW, db), ...]."""
    t = np.asarray(t, np.float64)
    p, zs, acts = mlp_forward(params, x)
    rows = p.shape[0]
    loss = -np.sum(t * np.log(np.maximum(p, 1e-300))) / rows
    grads = [None] * len(params)
    da = (p - t) / rows
    for l in range(len(params) - 1, -1, -1):
        w, _ = params[l]
        dz = da if l + 1 == len(params) else da * (zs[l] > 0.0)
        grads[l] = (dz.T @ acts[l], dz.sum(axis=0))
        da = dz @ w
    return loss, grads


def adam_step(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (in place on copies); returns new params, m, v."""
    out_p, out_m, out_v = [], [], []
    c1 = 1.0 - beta1 ** step
    c2 = 1.0 - beta2 ** step
    for (w, b), (gw, gb), (mw, mb), (vw, vb) in zip(params, grads, m, v):
        new = []
        for x, g, mm, vv in ((w, gw, mw, vw), (b, gb, mb, vb)):
            mm = beta1 * mm + (1.0 - beta1) * g
            vv = beta2 * vv + (1.0 - beta2) * g * g
            x = x - lr * (mm / c1) / (np.sqrt(vv / c2) + eps)
            new.append((x, mm, vv))
        out_p.append((new[0][0], new[1][0]))
        out_m.append((new[0][1], new[1][1]))
        out_v.append((new[0][2], new[1][2]))
    return out_p, out_m, out_v


def graph_stats(deg, nz: int):
    """Degree statistics of a graph's non-isolated nodes and its noise level:
    (mean degree, mean squared degree, largest degree, N * Nz)."""
    deg = np.asarray(deg, np.float64)
    return np.array([deg.mean(), np.mean(deg * deg), deg.max(), deg.size * float(nz)])


def mlp_features(hist, d, k, stats=None):
    """Feature row per graph: [B * bin masses of the histogram, d_1 .. d_{k-1}]
    and, with stats (rows of graph_stats), four more entries

        log(mean d) / 10,  (log(mean d^2) / 2 - log(mean d)) / 10,
        log(max d) / 10,   log(N Nz) / 10

    (the typical degree, its spread, the hub size and the number of probe
    entries that set the moments' noise; the / 10 keeps them O(1)).

    B * mass is the mean density over a bin scaled to [-1, 1] (O(1) values);
    d_0 = 1 after normalisation carries no information and is left out.
    """
    hist = np.asarray(hist, np.float64)
    d = np.asarray(d, np.float64)
    parts = [hist.shape[1] * hist, d[:, 1:k]]
    if stats is not None:
        st = np.asarray(stats, np.float64).reshape(-1, 4)
        mean, sq, mx, nnz = st[:, 0], st[:, 1], st[:, 2], st[:, 3]
        parts.append(np.stack([np.log(mean), 0.5 * np.log(sq) - np.log(mean), np.log(mx), np.log(nnz)], axis=1) / 10.0)
    return np.concatenate(parts, axis=1)


def normalize_hist(hist):
    """Target distribution: negative bins clipped to 0, rows scaled to sum 1
    (uniform where nothing is left)."""
    h = np.maximum(np.asarray(hist, np.float64), 0.0)
    s = h.sum(axis=1, keepdims=True)
    uni = np.full_like(h, 1.0 / h.shape[1])
    return np.where(s > 0.0, h / np.where(s > 0.0, s, 1.0), uni)
