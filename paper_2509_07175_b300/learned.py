"""Training driver of the learned proposal (host orchestration only).

The training data and every training step come from libvd's kernels
(``vd_mlp_features``, ``vd_mlp_train``); this module only chooses the
instances and moves the state between contexts.  Labels are produced by the
method itself: a plain vd_compute of each training instance gives every site's
neighbour set, and label bit s of site i says whether slot s of its 32-NN list
is in it.
"""
from __future__ import annotations

import time

import torch

from . import binding, inputs

TRAIN_SEED0 = inputs.SEED_BASE + 0x100   # training instance s: seed TRAIN_SEED0 + s
HELDOUT_SEED = inputs.SEED_BASE + 0x1FF  # validation instance
INIT_SEED = 0x5EED
# training recipe: 8 instances x 100,000 uniform sites in the unit cube (800,000
# rows), 30 epochs of Adam, batch 1024, learning rate 1e-3
N_INSTANCES, N_SITES, EPOCHS, BATCH, LR = 8, 100_000, 30, 1024, 1e-3
# the headline's distribution beside the uniform cube: 4 cube and 4 clustered
# shell instances (16 Gaussians, sigma 0.02, + 10 % uniform; 100,000 sites each,
# so the clusters are sparser than at 1M -- the network's inputs are offsets
# scaled by the nearest distance, which removes the density)
MIX = (("cube", 4), ("shell", 4))


def instance(n_sites: int, seed: int, name: str = "cube"):
    return inputs.workload(name, n_sites, seed=seed)


def data_of(w: dict, options: dict | None = None):
    """(features bf16 [n, 96], labels int32 [n]) of one workload, from a plain compute."""
    d = binding.diagram_from_workload(w, options=dict(options or {}, learned=0))
    d.compute()
    x, y = d.mlp_features()
    d.close()
    return x, y


def training_set(n_instances: int = N_INSTANCES, n_sites: int = N_SITES, name: str = "cube", mix=None):
    """Features and labels of seeded instances: n_instances of `name`, or the
    (name, count) pairs of `mix` (instance s of the whole set: seed TRAIN_SEED0 + s)."""
    plan = list(mix) if mix else [(name, n_instances)]
    xs, ys = [], []
    s = 0
    for nm, count in plan:
        for _ in range(count):
            x, y = data_of(instance(n_sites, TRAIN_SEED0 + s, nm))
            xs.append(x)
            ys.append(y)
            s += 1
    return torch.cat(xs), torch.cat(ys)


def train(x, y, epochs: int = EPOCHS, batch: int = BATCH, lr: float = LR, seed: int = 1,
          init_seed: int = INIT_SEED, trainer=None):
    """Train a fresh network on (x, y) on the GPU; returns the state and the losses."""
    own = trainer is None
    if own:
        w = inputs.workload("cube", 64, seed=inputs.SEED_BASE + 0x1FE)
        trainer = binding.diagram_from_workload(w)
    trainer.mlp_init(init_seed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = trainer.mlp_train(x, y, batch=batch, epochs=epochs, lr=lr, seed=seed)
    seconds = time.perf_counter() - t0
    state = trainer.mlp_get_state()
    if own:
        trainer.close()
    return {"state": state, "epoch_loss": losses, "train_s": seconds, "rows": int(x.shape[0]),
            "epochs": epochs, "batch": batch, "lr": lr}


def trained_state(mix=None):
    """Train the network with the default recipe (or on the instances of `mix`);
    returns the training record."""
    t0 = time.perf_counter()
    x, y = training_set(mix=mix)
    torch.cuda.synchronize()
    data_s = time.perf_counter() - t0
    tr = train(x, y)
    tr["data_s"] = data_s
    del x, y
    return tr


def random_init_state(init_seed: int = INIT_SEED):
    """State of an untrained network (the control)."""
    w = inputs.workload("cube", 64, seed=inputs.SEED_BASE + 0x1FE)
    d = binding.diagram_from_workload(w)
    d.mlp_init(init_seed)
    st = d.mlp_get_state()
    d.close()
    return st


def load_state(diagram, state: dict):
    diagram.mlp_set_state(state["params"], state.get("adam_m"), state.get("adam_v"), state.get("step", 0))


def logits_of(state: dict, x):
    """Logits of rows x under a state (through a scratch context)."""
    w = inputs.workload("cube", 64, seed=inputs.SEED_BASE + 0x1FE)
    d = binding.diagram_from_workload(w)
    load_state(d, state)
    z = d.mlp_forward(x)
    torch.cuda.synchronize()
    d.close()
    return z


def recall_at_k(scores, y, k: int) -> float:
    """Fraction of neighbour label bits captured by the k best-scored slots (ties: lower slot)."""
    slots = torch.arange(32, device=scores.device)
    bits = ((y.to(torch.int64)[:, None] >> slots[None, :]) & 1).to(torch.float64)
    # stable order: score descending, then slot ascending
    order = torch.sort(-scores.to(torch.float64), dim=1, stable=True).indices[:, :k]
    hit = torch.gather(bits, 1, order).sum()
    return float(hit / bits.sum().clamp(min=1.0))
