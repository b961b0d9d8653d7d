"""Learned corrector: training data and training.

The corrector maps the state after a step with fewer acoustic substeps (the
"reduced" step) to the increments that bring it to the plain step taken from
the same input (interior w, exner and theta_v per cell column; vn per edge
column); rho is never corrected.  Everything numerical runs in the library:
features and targets (``Dycore.corrector_features/corrector_targets``), the
networks' forward/backward/Adam (``MLP.train_step``), the per-feature
normalisation statistics and the random training batches
(``MLP.fit_normalization``, ``MLP.train_step_sampled``) and the corrected
step itself (``step_learned``).  This module only drives them: it keeps the
training rows in device tensors and computes each step's learning rate.
"""
import numpy as np

from . import _binding as B


def col_dims(nlev):
    return 5 * nlev, 3 * nlev - 1


def edge_dims(nlev):
    return 11 * nlev, nlev


def init_params(n_in, n_hidden, n_out, rng):
    """Fan-in scaled Gaussian weights, zero biases; the last layer starts small so
    that an untrained network proposes increments near the target mean."""
    parts = [rng.standard_normal((n_hidden, n_in)) * np.sqrt(2.0 / n_in), np.zeros(n_hidden),
             rng.standard_normal((n_hidden, n_hidden)) * np.sqrt(2.0 / n_hidden), np.zeros(n_hidden),
             rng.standard_normal((n_out, n_hidden)) * (0.1 / np.sqrt(n_hidden)), np.zeros(n_out)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def make_nets(nlev, hidden=512, max_batch=16384, seed=0):
    """Column network (5 nlev -> 3 nlev - 1) and edge network (11 nlev -> nlev)."""
    rng = np.random.default_rng(seed)
    nets = []
    for n_in, n_out in (col_dims(nlev), edge_dims(nlev)):
        net = B.MLP(n_in, hidden, n_out, max_batch)
        net.set_params(init_params(n_in, hidden, n_out, rng))
        nets.append(net)
    return nets[0], nets[1]


def clone_state(st):
    return {k: v.clone() for k, v in st.items()}


class Dataset:
    """Training rows (device float32): column features/targets and edge features/targets."""

    def __init__(self):
        self.col_x, self.col_y, self.edge_x, self.edge_y = [], [], [], []

    def cat(self):
        import torch
        return (torch.cat(self.col_x), torch.cat(self.col_y), torch.cat(self.edge_x), torch.cat(self.edge_y))


def add_pair(reduced, plain, st, data, rows=None, gen=None):
    """Branch a reduced and a plain step from the state `st` (left unchanged), add
    the reduced state's features and the targets plain - reduced to `data`
    (all cells/edges, or `rows` sampled of each), and return the plain result."""
    import torch
    nlev = reduced.nlev
    nc, ne = reduced.grid.n_cells, reduced.grid.n_edges
    dev = st["vn"].device
    sr, sp = clone_state(st), clone_state(st)
    reduced.step(sr)
    plain.step(sp)
    cx = torch.empty((nc, col_dims(nlev)[0]), dtype=torch.float32, device=dev)
    ex = torch.empty((ne, edge_dims(nlev)[0]), dtype=torch.float32, device=dev)
    cy = torch.empty((nc, col_dims(nlev)[1]), dtype=torch.float32, device=dev)
    ey = torch.empty((ne, edge_dims(nlev)[1]), dtype=torch.float32, device=dev)
    reduced.corrector_features(sr, cx, ex)
    reduced.corrector_targets(sr, sp, cy, ey)
    reduced.synchronize()
    if rows is not None:
        ic = torch.randperm(nc, generator=gen, device="cpu")[:rows].to(dev)
        ie = torch.randperm(ne, generator=gen, device="cpu")[:rows].to(dev)
        cx, cy, ex, ey = cx[ic], cy[ic], ex[ie], ey[ie]
    data.col_x.append(cx)
    data.col_y.append(cy)
    data.edge_x.append(ex)
    data.edge_y.append(ey)
    return sp


def feature_groups(n, nlev):
    """First feature of every group of features (or outputs) that share a
    physical field: runs of nlev (the column's w interior outputs: nlev - 1)."""
    starts, start = [], 0
    while start < n:
        starts.append(start)
        start += nlev - 1 if (n == 3 * nlev - 1 and start == 0) else nlev
    return starts


def fit(net, x, y, nlev, steps, batch=4096, lr=1e-3, lr_final=1e-5, seed=0, rel_floor=1e-3, log_every=0):
    """Set the network's normalisation from the training rows (x, y) and train it
    for `steps` Adam steps on random batches of `batch` normalised rows, with a
    cosine learning-rate decay from lr to lr_final.  The statistics, the
    normalisation, the batches and the steps run in the library
    (icon_mlp_fit_normalization, icon_mlp_train_step_sampled); only the
    learning rate of each step is computed here.  Returns the loss history."""
    import torch
    xn, yn = torch.empty_like(x), torch.empty_like(y)
    net.fit_normalization(x, y, feature_groups(x.shape[1], nlev), feature_groups(y.shape[1], nlev), rel_floor,
                          xn, yn)
    batch = min(batch, net.max_batch, (x.shape[0] // 64) * 64)
    losses = []
    for t in range(steps):
        a = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * t / max(steps - 1, 1)))
        losses.append(net.train_step_sampled(xn, yn, batch, seed, t, float(a)))
        if log_every and t % log_every == 0:
            print("step %5d loss %.4e" % (t, losses[-1]), flush=True)
    return losses


def field_errors(a, b):
    """RMS differences of the corrected fields between two device states (host floats)."""
    out = {}
    for k in ("vn", "w", "exner", "theta_v"):
        out[k] = float(((a[k] - b[k]) ** 2).mean().sqrt())
    return out
