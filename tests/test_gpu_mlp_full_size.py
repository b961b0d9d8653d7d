"""The tensor-core MLP at the benchmark's chunk of 65 536 rows, element by
element against the FP64 oracle (oracle/mlp.py).

At 65 536 rows every persistent CTA walks several 128 x 128 output tiles, so
the TMA ring continues across tiles and the two TMEM accumulators alternate;
the weight-gradient GEMMs reduce over K = 65 536.

Bounds:
* forward: the GPU stores the network input and both hidden activations in
  BF16 (relative rounding error at most 2^-9) and accumulates in FP32; the
  oracle computes in FP64 on the BF16-rounded weights and input.  Each
  output may differ by C = 12 times the root-sum-square propagation of those
  roundings through the oracle's layers (tests/mlp_bounds.py);
* gradients: the oracle's backward chain evaluated on the GPU's storage
  precision (BF16 operands of every GEMM, FP32 bias sums), checked first to
  equal oracle/mlp.backward without the rounding.  What remains is the FP32
  accumulation over K (bounded statistically, 16 2^-24 sqrt(sum of squared
  terms)) and rare BF16 rounding flips where the GPU's FP32 operand and the
  FP64 one straddle a rounding boundary (each flip moves one term by at most
  2^-8 of it; allowance 64 flips of the largest term)."""
import numpy as np
import pytest

from mlp_bounds import C, U32, bf16, forward_bound, init_params, rounded
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

B_FULL = 65536


@pytest.mark.parametrize("dims", [(450, 512, 269, B_FULL), (990, 512, 90, B_FULL), (450, 512, 269, B_FULL - 37)],
                         ids=["column-65536", "edge-65536", "column-ragged"])
def test_forward_elementwise_at_the_benchmark_chunk(built_lib, cuda, dims):
    import torch
    import paper_2608_21150_gb300 as P
    I, H, O, B = dims
    rng = np.random.default_rng(I + O + B)
    p = init_params(rng, I, H, O)
    x = rng.standard_normal((B, I)).astype(np.float32)
    net = P.MLP(I, H, O, max_batch=B_FULL)
    net.set_params(p)
    yd = torch.full((B, O), np.nan, dtype=torch.float32, device=cuda)
    net.forward(torch.from_numpy(x).to(cuda), yd)
    y = yd.cpu().numpy().astype(np.float64)
    y_ref, e_y = forward_bound(rounded(p, I, H, O), bf16(x), I, H, O)
    excess = np.abs(y - y_ref) - C * e_y
    assert np.all(np.isfinite(y))
    assert excess.max() <= 0.0, (float(excess.max()), np.unravel_index(int(np.argmax(excess)), excess.shape))
    # the bound is not vacuous: it is a small fraction of the output's size
    assert np.median(C * e_y / (np.abs(y_ref) + np.std(y_ref))) < 0.1
    net.close()


def _backward_on_storage(pr, x16, dy, I, H, O, q):
    """oracle/mlp.backward's chain with the GPU's storage rounding q (BF16 or
    the identity) applied where the GPU stores a GEMM operand; also returns
    the operands of each weight gradient."""
    W1, b1, W2, b2, W3, b3 = omlp.unpack(pr, I, H, O)
    z1 = x16 @ W1.T + b1
    h1 = q(omlp.gelu(z1))
    z2 = h1 @ W2.T + b2
    h2 = q(omlp.gelu(z2))
    d3 = q(dy)
    gW3, gb3 = d3.T @ h2, dy.sum(0)
    dz2 = (d3 @ W3) * omlp.gelu_grad(z2)
    d2 = q(dz2)
    gW2, gb2 = d2.T @ h1, dz2.sum(0)
    dz1 = (d2 @ W2) * omlp.gelu_grad(z1)
    d1 = q(dz1)
    gW1, gb1 = d1.T @ x16, dz1.sum(0)
    grads = [gW1, gb1, gW2, gb2, gW3, gb3]
    return grads, [(d1, x16, dz1), (d2, h1, dz2), (d3, h2, dy)]


def test_gradients_elementwise_at_the_benchmark_chunk(built_lib, cuda):
    import torch
    import paper_2608_21150_gb300 as P
    I, H, O, B = 450, 512, 269, B_FULL
    rng = np.random.default_rng(2024)
    p = init_params(rng, I, H, O)
    x = rng.standard_normal((B, I)).astype(np.float32)
    t = rng.standard_normal((B, O)).astype(np.float32)
    pr = rounded(p, I, H, O)
    x16 = bf16(x)
    y_ref, cache = omlp.forward(pr, x16, I, H, O)
    _, dy = omlp.mse(y_ref, t)
    dy = dy.astype(np.float32).astype(np.float64)
    # the chain without rounding is the oracle's backward
    g_plain, _ = _backward_on_storage(pr, x16, dy, I, H, O, lambda a: a)
    g_oracle = omlp.backward(pr, cache, dy, I, H, O)
    flat = np.concatenate([a.ravel() for a in g_plain])
    assert np.max(np.abs(flat - g_oracle)) <= 1e-12 * np.max(np.abs(g_oracle))
    g_ref, ops = _backward_on_storage(pr, x16, dy, I, H, O, bf16)

    net = P.MLP(I, H, O, max_batch=B_FULL)
    net.set_params(p)
    yd = torch.empty((B, O), dtype=torch.float32, device=cuda)
    net.forward(torch.from_numpy(x).to(cuda), yd)
    net.backward(torch.from_numpy(dy.astype(np.float32)).to(cuda))
    g = net.grads().astype(np.float64)
    off = 0
    names = ["W1", "b1", "W2", "b2", "W3", "b3"]
    for li, (name, ref) in enumerate(zip(names, g_ref)):
        n = ref.size
        got = g[off:off + n].reshape(ref.shape)
        off += n
        d16, h16, d32 = ops[li // 2]
        if name.startswith("W"):
            acc = 16.0 * U32 * np.sqrt(B) * np.sqrt((d16 * d16).T @ (h16 * h16))
            flips = 64.0 * 2.0 ** -8 * np.outer(np.abs(d16).max(0), np.abs(h16).max(0))
            drift = 4e-6 * (np.abs(d32).T @ np.abs(h16))
            tol = 2.0 * (acc + flips + drift)
        else:
            tol = 2.0 * (16.0 * U32 * np.sqrt(B) * np.sqrt((d32 * d32).sum(0)) + 4e-6 * np.abs(d32).sum(0))
        excess = np.abs(got - ref) - tol
        assert excess.max() <= 0.0, (name, float(excess.max()))
        # a misplaced tile or a stale accumulator changes entries by about their own size
        assert np.median(tol / (np.abs(ref) + 1e-30)) < 0.5, name
    net.close()
