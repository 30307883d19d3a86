"""FP64 CPU oracle of the learned proposal network (test infrastructure).

Only ``tests/`` (and ``bench.py``'s CPU legs) use this module; the product path
never does.  It restates, in plain numpy, what the network of the learned
proposal computes.  The paper has no network: the proposal only reorders the
candidate tests of the bisector search (Sec. 3.2, Sec. 5.1), and every clip is
still decided by the point-in-cell test of Sec. 3.1.

Definitions (written from the mathematics, no blocking or fusion):

* input of site i: the offsets (v_k - v_i) / d_1 of its 32 nearest sites in
  ascending distance (``features``), d_1 = distance to the nearest one;
  96 values, row-major [slot][xyz];
* label of site i: bit s set when slot s's site is a bisector neighbour of v_i,
  i.e. the two cells share a face of positive measure (Sec. 2.2) (``labels``);
* network: h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), z = h2 W3 + b3 with
  W1 [96, 64], W2 [64, 64], W3 [64, 32]; parameters flat in the order
  W1, b1, W2, b2, W3, b3 (weights row-major, input index first);
* loss: mean over rows and the 32 slots of the binary cross-entropy
  softplus(z) - y z of the logit z against the label bit y;
* Adam (Kingma and Ba): bias-corrected first and second moments.

``rounded=True`` rounds to bfloat16 where the GPU kernels do (inputs, weights,
h1 and h2 after ReLU; in the backward pass dZ, dH2 and dH1 where they enter a
product) and otherwise keeps FP64; the backward pass then treats each rounding
as the identity (the derivative the GPU kernels compute).  ``rounded=False`` is
the plain network, whose gradient is the exact derivative of ``loss``.

Pins (tests/test_mlp_oracle.py): central finite differences of ``loss`` against
``grad`` (``rounded=False``), closed forms of the forward pass and of the loss
at z = 0, bfloat16 rounding against torch's conversion, closed forms of the
first Adam steps, a planted transposition that the finite-difference check
catches, and brute-force nearest sites / neighbour sets for the features and
labels.
"""
from __future__ import annotations

import numpy as np

NIN, NH, NOUT = 96, 64, 32
SHAPES = (("W1", (NIN, NH)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH, NOUT)),
          ("b3", (NOUT,)))
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)  # 12448


def unflatten(p):
    p = np.asarray(p, dtype=np.float64)
    assert p.shape == (NPARAM,)
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def flatten(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def bf16_round(a):
    """Nearest bfloat16 (8 significant bits, ties to even) of float32(a), as float64."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    b = a32.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def label_bits(y):
    """[rows] bit masks -> [rows, 32] array of 0/1."""
    y = np.asarray(y).astype(np.int64) & 0xFFFFFFFF
    return ((y[:, None] >> np.arange(NOUT)[None, :]) & 1).astype(np.float64)


def _ident(a):
    return np.asarray(a, dtype=np.float64)


def forward(params, x, rounded=True):
    """Activations of every layer; x: [rows, 96]."""
    r = bf16_round if rounded else _ident
    w = unflatten(params)
    W1, W2, W3 = r(w["W1"]), r(w["W2"]), r(w["W3"])
    X = r(x)
    h1 = r(np.maximum(X @ W1 + w["b1"], 0.0))
    h2 = r(np.maximum(h1 @ W2 + w["b2"], 0.0))
    z = h2 @ W3 + w["b3"]
    return {"x": X, "h1": h1, "h2": h2, "z": z, "W1": W1, "W2": W2, "W3": W3}


def loss(params, x, y, rounded=True):
    z = forward(params, x, rounded)["z"]
    Y = label_bits(y)
    return float(np.mean(np.logaddexp(0.0, z) - Y * z))


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def grad(params, x, y, rounded=True):
    """(flat gradient of ``loss``, loss) by back-propagation."""
    r = bf16_round if rounded else _ident
    f = forward(params, x, rounded)
    Y = label_bits(y)
    z = f["z"]
    rows = z.shape[0]
    dz = (sigmoid(z) - Y) / (rows * NOUT)
    g = {"b3": dz.sum(axis=0)}
    dz_r = r(dz)
    g["W3"] = f["h2"].T @ dz_r
    dh2 = (dz_r @ f["W3"].T) * (f["h2"] > 0)
    g["b2"] = dh2.sum(axis=0)
    dh2_r = r(dh2)
    g["W2"] = f["h1"].T @ dh2_r
    dh1 = (dh2_r @ f["W2"].T) * (f["h1"] > 0)
    g["b1"] = dh1.sum(axis=0)
    dh1_r = r(dh1)
    g["W1"] = f["x"].T @ dh1_r
    L = float(np.mean(np.logaddexp(0.0, z) - Y * z))
    return flatten(g), L


def adam_step(p, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update; step = the 1-based index of this update.  Returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def knn32(sites):
    """The 32 nearest other sites of every site, ascending distance (brute force)."""
    s = np.asarray(sites, dtype=np.float64)
    n = s.shape[0]
    out = np.full((n, 32), -1, dtype=np.int64)
    for i in range(n):
        d2 = ((s - s[i]) ** 2).sum(axis=1)
        d2[i] = np.inf
        order = np.lexsort((np.arange(n), d2))[:min(32, n - 1)]
        out[i, :len(order)] = order
    return out


def features(sites, knn):
    """Network input of every site, FP64 [n, 96] (unrounded)."""
    s = np.asarray(sites, dtype=np.float64)
    n = s.shape[0]
    x = np.zeros((n, 32, 3))
    for i in range(n):
        ok = knn[i] >= 0
        d1 = np.sqrt(((s[knn[i, 0]] - s[i]) ** 2).sum())
        x[i, ok] = (s[knn[i, ok]] - s[i]) / d1
    return x.reshape(n, NIN)


def labels(knn, nbrs):
    """Bit s of site i set when knn[i, s] is in nbrs[i] (the neighbours of site i)."""
    n = knn.shape[0]
    y = np.zeros(n, dtype=np.int64)
    for i in range(n):
        nb = set(int(j) for j in nbrs[i])
        for s in range(32):
            if knn[i, s] >= 0 and int(knn[i, s]) in nb:
                y[i] |= 1 << s
    return y


def recall_at_k(scores, y, k):
    """Fraction of the neighbour bits captured by the k highest scores of each row
    (equal scores: the lower slot first)."""
    Y = label_bits(y)
    order = np.argsort(-np.asarray(scores, dtype=np.float64), axis=1, kind="stable")[:, :k]
    hit = np.take_along_axis(Y, order, axis=1).sum()
    return float(hit / max(Y.sum(), 1.0))
