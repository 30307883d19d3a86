"""Pins of the learned-proposal network oracle (CPU, no GPU).

The oracle's backward pass is checked against central finite differences of its
own loss, its forward pass and loss against closed forms, its bfloat16 rounding
against torch's conversion, its Adam step against the closed form of the first
updates, and its feature / label construction against brute force over all
sites and the Voronoi oracle's neighbour sets.
"""
import numpy as np
import pytest
import torch

from oracle import mlp

RNG = np.random.default_rng(0xB3000200)


def random_params(rng, scale=1.0):
    p = {}
    for name, shape in mlp.SHAPES:
        fan = shape[0] if len(shape) == 2 else 1
        p[name] = rng.standard_normal(shape) * (scale * np.sqrt(2.0 / fan) if len(shape) == 2 else 0.1)
    return mlp.flatten(p)


def random_batch(rng, rows):
    x = rng.standard_normal((rows, mlp.NIN)) * 1.5
    y = rng.integers(0, 2 ** 32, size=rows, dtype=np.int64)
    return x, y


def fd_check(grad_fn, loss_fn, p, idx, h=1e-6):
    g, _ = grad_fn(p)
    worst = 0.0
    for t in idx:
        e = np.zeros_like(p)
        e[t] = h
        fd = (loss_fn(p + e) - loss_fn(p - e)) / (2 * h)
        worst = max(worst, abs(fd - g[t]) / (abs(g[t]) + 1e-7))
    return worst


def param_sample(rng, per_block=60):
    idx, o = [], 0
    for _, shape in mlp.SHAPES:
        k = int(np.prod(shape))
        idx.extend((o + rng.choice(k, size=min(per_block, k), replace=False)).tolist())
        o += k
    return idx


def test_nparam_layout():
    assert mlp.NPARAM == 12448
    p = np.arange(mlp.NPARAM, dtype=np.float64)
    assert np.array_equal(mlp.flatten(mlp.unflatten(p)), p)
    w = mlp.unflatten(p)
    assert w["W1"][0, 1] == 1 and w["W1"][1, 0] == 64  # row-major, input index first
    assert w["b3"][-1] == mlp.NPARAM - 1


def test_backward_matches_central_differences():
    rng = np.random.default_rng(1)
    p = random_params(rng)
    x, y = random_batch(rng, 37)
    worst = fd_check(lambda q: mlp.grad(q, x, y, rounded=False),
                     lambda q: mlp.loss(q, x, y, rounded=False), p, param_sample(rng))
    assert worst < 1e-5, worst


def test_planted_transposition_is_caught():
    # a backward pass with W2 (not W2^T) in dH1 must fail the same check
    def bad_grad(q, x, y):
        f = mlp.forward(q, x, rounded=False)
        Y = mlp.label_bits(y)
        dz = (mlp.sigmoid(f["z"]) - Y) / (f["z"].shape[0] * mlp.NOUT)
        g = {"b3": dz.sum(0), "W3": f["h2"].T @ dz}
        dh2 = (dz @ f["W3"].T) * (f["h2"] > 0)
        g["b2"], g["W2"] = dh2.sum(0), f["h1"].T @ dh2
        dh1 = (dh2 @ f["W2"]) * (f["h1"] > 0)  # planted: missing transpose
        g["b1"], g["W1"] = dh1.sum(0), f["x"].T @ dh1
        return mlp.flatten(g), 0.0

    rng = np.random.default_rng(2)
    p = random_params(rng)
    x, y = random_batch(rng, 23)
    worst = fd_check(lambda q: bad_grad(q, x, y), lambda q: mlp.loss(q, x, y, rounded=False), p,
                     param_sample(rng, 30))
    assert worst > 1e-2


def test_forward_closed_form():
    # W1 = W2 = 0: h1 = relu(b1), h2 = relu(b2), z = relu(b2) W3 + b3 for every row
    rng = np.random.default_rng(3)
    w = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    w["b1"] = rng.integers(-4, 5, mlp.NH).astype(float)
    w["b2"] = rng.integers(-4, 5, mlp.NH).astype(float)
    w["W3"] = rng.integers(-3, 4, (mlp.NH, mlp.NOUT)).astype(float) / 4
    w["b3"] = rng.integers(-8, 9, mlp.NOUT).astype(float) / 8
    x, _ = random_batch(rng, 5)
    want = np.maximum(w["b2"], 0) @ w["W3"] + w["b3"]
    for rounded in (False, True):  # every value is exact in bfloat16
        z = mlp.forward(mlp.flatten(w), x, rounded)["z"]
        assert np.array_equal(z, np.broadcast_to(want, z.shape))
    # identity-like first layer: h1 = relu(x[:, :64]) for x exact in bfloat16
    w = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    w["W1"][:64, :] = np.eye(64)
    xi = rng.integers(-8, 9, (4, mlp.NIN)).astype(float)
    assert np.array_equal(mlp.forward(mlp.flatten(w), xi, True)["h1"], np.maximum(xi[:, :64], 0))


def test_loss_and_gradient_at_zero_logits():
    # all parameters 0: z = 0, loss = log 2, dL/db3_s = (1/2 - mean_r y_rs) / 32
    p = np.zeros(mlp.NPARAM)
    rng = np.random.default_rng(4)
    x, y = random_batch(rng, 9)
    for rounded in (False, True):
        g, L = mlp.grad(p, x, y, rounded)
        assert abs(L - np.log(2.0)) < 1e-15
        want = (0.5 - mlp.label_bits(y).mean(axis=0)) / mlp.NOUT
        assert np.allclose(mlp.unflatten(g)["b3"], want, rtol=0, atol=1e-15)
        assert not np.any(mlp.unflatten(g)["W3"])  # h2 = 0


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(5)
    a = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -(1.0 + 2 ** -8), 65504.0]])
    a32 = a.astype(np.float32)
    want = torch.from_numpy(a32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(a32), want)


def test_adam_first_steps_closed_form():
    # from zero moments with a constant gradient g, every step moves by -lr g / (|g| + eps)
    rng = np.random.default_rng(6)
    g = rng.standard_normal(100) * 10.0 ** rng.integers(-6, 0, 100)
    p0 = rng.standard_normal(100)
    m = v = np.zeros(100)
    p = p0
    for step in (1, 2, 3):
        p, m, v = mlp.adam_step(p, g, m, v, step, lr=1e-3)
        assert np.allclose(p - p0, -step * 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-18)


def test_rounded_gradient_close_to_exact():
    # bfloat16 rounding perturbs the gradient by a few 2^-8 relative, not more
    rng = np.random.default_rng(7)
    p = random_params(rng)
    x, y = random_batch(rng, 200)
    g0, _ = mlp.grad(p, x, y, rounded=False)
    g1, _ = mlp.grad(p, x, y, rounded=True)
    assert np.linalg.norm(g1 - g0) / np.linalg.norm(g0) < 0.05


def test_features_and_labels_against_brute_force():
    # 300 uniform sites in the unit square: nearest sites by brute force over all
    # pairs, neighbour sets from the Voronoi oracle
    import oracle as O
    from paper_2509_07175_b300 import inputs
    w = inputs.workload("square", 300, seed=11)
    n = len(w["sites"])
    pieces = O.Oracle(w["mode"], w["sites"], w["verts"], w["simp"]).enumerate()
    _, _, nbrs = O.per_site(n, w["sites"], pieces)
    s = w["sites"][:, :2]
    knn = mlp.knn32(s)
    d = np.sqrt(((s[knn] - s[:, None, :]) ** 2).sum(-1))
    assert np.all(np.diff(d, axis=1) >= 0)  # ascending distance
    full = np.sqrt(((s[:, None, :] - s[None, :, :]) ** 2).sum(-1))
    np.fill_diagonal(full, np.inf)
    assert np.allclose(np.sort(full, axis=1)[:, :32], d)
    y = mlp.labels(knn, nbrs)
    # the nearest site is always a Voronoi neighbour (the midpoint lies on both cells)
    assert np.all(y & 1)
    for i in range(0, n, 17):
        bits = {int(knn[i, k]) for k in range(32) if (y[i] >> k) & 1}
        assert bits == set(nbrs[i]) & set(knn[i].tolist())
    x = mlp.features(np.c_[s, np.zeros(n)], knn).reshape(-1, 32, 3)
    assert np.allclose(np.linalg.norm(x[:, 0], axis=1), 1.0)
    assert np.all(x[:, :, 2] == 0)


def test_recall_at_k_hand_example():
    y = np.array([0b1010])          # slots 1 and 3 are neighbours
    scores = np.zeros((1, 32))
    scores[0, 1], scores[0, 0], scores[0, 3] = 3.0, 2.0, 1.0
    assert mlp.recall_at_k(scores, y, 1) == 0.5
    assert mlp.recall_at_k(scores, y, 2) == 0.5
    assert mlp.recall_at_k(scores, y, 3) == 1.0
    # equal scores: the lower slot first
    assert mlp.recall_at_k(np.zeros((1, 32)), y, 2) == 0.5
