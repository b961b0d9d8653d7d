"""Learned corrector: training data and training.

The corrector maps the state after a step with fewer acoustic substeps (the
"reduced" step) to the increments that bring it to the plain step taken from
the same input (interior w, exner and theta_v per cell column; vn per edge
column); rho is never corrected.  Everything numerical runs in the library:
features and targets (``Dycore.corrector_features/corrector_targets``), the
networks' forward/backward/Adam (``MLP.train_step``) and the corrected step
itself (``step_learned``).  This module only drives them: it keeps the
training rows in device tensors, draws batches, and computes the per-feature
normalisation statistics that the networks are given.
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
    """Index groups of features (or outputs) that share a physical field: runs of
    nlev (the column's w interior outputs: nlev - 1)."""
    groups, start = [], 0
    while start < n:
        size = nlev - 1 if (n == 3 * nlev - 1 and start == 0) else nlev
        groups.append((start, start + size))
        start += size
    return groups


def statistics(x, nlev, rel_floor=1e-3):
    """Per-feature mean and standard deviation (float64 accumulation); a standard
    deviation below rel_floor times its field's largest is raised to that floor,
    so near-constant features (e.g. w at the lowest level) are not amplified."""
    xd = x.double()
    mean = xd.mean(0)
    std = xd.std(0)
    for a, b in feature_groups(x.shape[1], nlev):
        top = float(std[a:b].max())
        std[a:b] = std[a:b].clamp(min=max(top * rel_floor, 1e-30))
    return mean.float().cpu().numpy(), std.float().cpu().numpy()


def fit(net, x, y, nlev, steps, batch=4096, lr=1e-3, lr_final=1e-5, seed=0, log_every=0):
    """Set the network's normalisation from (x, y) and train it on the normalised
    rows for `steps` Adam steps of `batch` random rows (cosine learning-rate
    decay from lr to lr_final).  Returns the loss history."""
    import torch
    xm, xs = statistics(x, nlev)
    ym, ys = statistics(y, nlev)
    net.set_normalization(xm, xs, ym, ys)
    dev = x.device
    xn = ((x - torch.from_numpy(xm).to(dev)) / torch.from_numpy(xs).to(dev)).contiguous()
    yn = ((y - torch.from_numpy(ym).to(dev)) / torch.from_numpy(ys).to(dev)).contiguous()
    batch = min(batch, net.max_batch, (x.shape[0] // 64) * 64)
    gen = torch.Generator(device="cpu")
    gen.manual_seed(seed)
    losses = []
    for t in range(steps):
        idx = torch.randint(0, x.shape[0], (batch,), generator=gen).to(dev)
        xb, yb = xn.index_select(0, idx), yn.index_select(0, idx)
        a = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * t / max(steps - 1, 1)))
        losses.append(net.train_step(xb, yb, float(a)))
        if log_every and t % log_every == 0:
            print("step %5d loss %.4e" % (t, losses[-1]), flush=True)
    return losses


def field_errors(a, b):
    """RMS differences of the corrected fields between two device states (host floats)."""
    out = {}
    for k in ("vn", "w", "exner", "theta_v"):
        out[k] = float(((a[k] - b[k]) ** 2).mean().sqrt())
    return out
