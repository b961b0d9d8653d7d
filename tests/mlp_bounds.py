"""Error estimates of the GPU's BF16 tensor-core MLP against the FP64 oracle
(oracle/mlp.py), shared by the MLP and learned-corrector tests.

The GPU rounds the network input and both hidden activations to BF16
(relative error at most R = 2^-9, round to nearest) and accumulates in FP32
(unit roundoff U32 = 2^-24); its GELU uses an erf approximation with absolute
error at most 1.5e-7.  forward_bound propagates these errors to first order
through the layers of the oracle's own forward pass.  The roundings of
different elements are independent, so their effects on a sum add in
quadrature: the estimate is the root-sum-square of every rounding's bound
times its weight, e.g. for z = W h the variance (W*W) @ (e_h*e_h).  A test
allows a multiple c of it; an element of a sum of many independent
roundings stays within a few root-sum-squares of its bounds (each rounding's
standard deviation is at most its bound / sqrt 3), while a misplaced tile or
a stale accumulator is off by about the value itself, hundreds of times more."""
import numpy as np

from oracle import mlp as omlp

R = 2.0 ** -9        # BF16 round-to-nearest, relative
U32 = 2.0 ** -24     # FP32 unit roundoff


def bf16(a):
    """Round to the nearest BF16 value (ties to even), as the GPU stores weights and activations."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(rng, I, H, O):
    parts = [rng.standard_normal((H, I)) / np.sqrt(I), 0.1 * rng.standard_normal(H),
             rng.standard_normal((H, H)) / np.sqrt(H), 0.1 * rng.standard_normal(H),
             rng.standard_normal((O, H)) / np.sqrt(H), 0.1 * rng.standard_normal(O)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def rounded(p, I, H, O):
    W1, b1, W2, b2, W3, b3 = omlp.unpack(p, I, H, O)
    return np.concatenate([bf16(W1).ravel(), b1, bf16(W2).ravel(), b2, bf16(W3).ravel(), b3])


C = 12.0            # allowed multiple of the root-sum-square estimate


def forward_bound(pr, x, I, H, O, ex=None):
    """Oracle output y and the root-sum-square estimate e_y of |y_gpu - y| per
    element; ex: the input's own error bound (none: x is already BF16)."""
    W1, b1, W2, b2, W3, b3 = omlp.unpack(pr, I, H, O)
    y, (x_, z1, h1, z2, h2) = omlp.forward(pr, x, I, H, O)
    q1, q2, q3 = W1 * W1, W2 * W2, W3 * W3
    v_z1 = (0.0 if ex is None else (ex * ex) @ q1.T) + I * U32 ** 2 * ((x * x) @ q1.T + b1 * b1)
    v_h1 = omlp.gelu_grad(z1) ** 2 * v_z1 + (R * h1) ** 2 + (1e-7 * z1) ** 2
    v_z2 = v_h1 @ q2.T + H * U32 ** 2 * ((h1 * h1) @ q2.T + b2 * b2)
    v_h2 = omlp.gelu_grad(z2) ** 2 * v_z2 + (R * h2) ** 2 + (1e-7 * z2) ** 2
    v_y = v_h2 @ q3.T + H * U32 ** 2 * ((h2 * h2) @ q3.T + b3 * b3)
    return y, np.sqrt(v_y)
