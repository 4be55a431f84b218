"""Oracle for the learned vertex ordering -- TEST INFRASTRUCTURE ONLY.

Plain numpy in float64: the per-vertex features, the 6 -> 64 -> 64 -> 1 ReLU
network's forward pass, its weighted binary cross-entropy loss, the
analytic gradient and one Adam step.  The network's weights are rounded to bfloat16 (round to
nearest even) before use, as the CUDA kernels store them; biases stay at
float32 precision.  Nothing here is shared with the CUDA library.
"""
from __future__ import annotations

import numpy as np

F, H = 6, 64
OFF_W1 = 0
OFF_B1 = OFF_W1 + H * F
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H
NPARAMS = OFF_B3 + 1


def bf16_round(x):
    """float32 values rounded to the nearest bfloat16 (ties to even)."""
    a = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    finite = (a & 0x7F800000) != 0x7F800000
    r = np.where(finite, (a + 0x7FFF + ((a >> 16) & 1)) >> 16, a >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


T = 8  # neighbours that the triangle and colouring features look at


def features(g, core):
    """The six features of every vertex, by their definitions.  With d the
    degree, K = K(v), Kmax = K(G), Dmax the largest degree, c the number of
    neighbours whose core number is at least K(v), and Q(v) the first
    min(T, c) of those neighbours in increasing vertex id:
      f0 = log(1+d)/log(1+Dmax)           degree
      f1 = K/Kmax                         core number
      f2 = t/(T(T-1)/2)                   triangle count: t = edges among Q(v)
      f3 = (chi+1)/(T+1)                  neighbourhood colouring bound: chi =
                                          colours of the greedy colouring of
                                          G[Q(v)] in increasing id (0 if Q is
                                          empty), so chi+1 bounds a clique
                                          containing v inside Q(v) + v
      f4 = c/max(d,1),  f5 = log(1+c)/log(1+Dmax)."""
    n = g.n
    deg = np.diff(g.row_ptr).astype(np.float64)
    kmax = float(max(int(core.max()) if n else 0, 1))
    ldmax = np.log1p(float(max(int(deg.max()) if n else 0, 1)))
    nbsets = [set(g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(n)]
    out = np.zeros((n, F), np.float64)
    for v in range(n):
        nb = g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]
        qual = nb[core[nb] >= core[v]]
        c = float(len(qual))
        d = deg[v]
        Q = qual[:T].tolist()
        q = len(Q)
        adj = [[Q[j] in nbsets[Q[i]] for j in range(q)] for i in range(q)]
        t = sum(1 for i in range(q) for j in range(i + 1, q) if adj[i][j])
        col = [0] * q
        for i in range(q):
            used = {col[j] for j in range(i) if adj[i][j]}
            k = 1
            while k in used:
                k += 1
            col[i] = k
        chi = max(col) if q else 0
        out[v, 0] = np.log1p(d) / ldmax
        out[v, 1] = core[v] / kmax
        out[v, 2] = t / (T * (T - 1) / 2)
        out[v, 3] = (chi + 1) / (T + 1)
        out[v, 4] = c / max(d, 1.0)
        out[v, 5] = np.log1p(c) / ldmax
    return out


def unpack(p, bf16=True):
    """Split the flat parameters.  bf16=True: weights as bfloat16 values of
    their float32 master copy, biases as float32 (the kernels' storage);
    bf16=False: everything at the given precision (float64 for derivative
    checks)."""
    if bf16:
        p32 = np.asarray(p, dtype=np.float32)
        w = bf16_round(p32).astype(np.float64)
        p = p32.astype(np.float64)
    else:
        p = np.asarray(p, dtype=np.float64)
        w = p
    W1 = w[OFF_W1:OFF_B1].reshape(H, F)
    b1 = p[OFF_B1:OFF_W2]
    W2 = w[OFF_W2:OFF_B2].reshape(H, H)
    b2 = p[OFF_B2:OFF_W3]
    w3 = w[OFF_W3:OFF_B3]
    b3 = float(p[OFF_B3])
    return W1, b1, W2, b2, w3, b3


def forward(params, x, bf16=True):
    """Logits s = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 for every row."""
    W1, b1, W2, b2, w3, b3 = unpack(params, bf16)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.maximum(x @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ w3 + b3


def loss(params, x, y, pos_weight, bf16=True):
    """Mean over rows of w_y (log(1 + e^s) - y s), w_y = pos_weight if y = 1."""
    s = forward(params, x, bf16)
    y = np.asarray(y, dtype=np.float64)
    w = np.where(y > 0.5, pos_weight, 1.0)
    return float(np.mean(w * (np.logaddexp(0.0, s) - y * s)))


def gradient(params, x, y, pos_weight, bf16=True):
    """Analytic gradient of loss() with respect to the flat parameters (the
    weights enter through their bfloat16 values; the gradient is taken with
    respect to those values, as the kernels do)."""
    W1, b1, W2, b2, w3, b3 = unpack(params, bf16)
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = x.shape[0]
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    s = h2 @ w3 + b3
    w = np.where(y > 0.5, pos_weight, 1.0)
    gs = w * (1.0 / (1.0 + np.exp(-s)) - y) / n
    g = np.zeros(NPARAMS, np.float64)
    g[OFF_B3] = gs.sum()
    g[OFF_W3:OFF_B3] = h2.T @ gs
    d2 = np.outer(gs, w3) * (z2 > 0)
    g[OFF_W2:OFF_B2] = (d2.T @ h1).ravel()
    g[OFF_B2:OFF_W3] = d2.sum(axis=0)
    d1 = (d2 @ W2) * (z1 > 0)
    g[OFF_W1:OFF_B1] = (d1.T @ x).ravel()
    g[OFF_B1:OFF_W2] = d1.sum(axis=0)
    return g


def adam_step(params, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) in float64, the optimiser the
    training kernels use on the float32 master parameters.  t is the step
    number counted from 1; m and v are the first and second moment estimates
    before the step.  Returns (params, m, v) after it:
        m <- beta1 m + (1 - beta1) g,   v <- beta2 v + (1 - beta2) g^2,
        params <- params - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps)."""
    p = np.asarray(params, dtype=np.float64)
    g = np.asarray(grad, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
