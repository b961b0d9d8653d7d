"""FP64 CPU oracle of the learned corrector's MLP (test infrastructure only).

Row A13, an extension beyond the paper.  GELU in the erf form (Hendrycks and
Gimpel 2016), Adam (Kingma and Ba 2015).

y = W3 GELU(W2 GELU(W1 x + b1) + b2) + b3 with GELU(u) = u Phi(u) =
u (1 + erf(u / sqrt 2)) / 2, its exact gradients by the chain rule, the mean
squared error and one Adam step (Kingma & Ba, bias-corrected moments).
Parameters use the library's flat layout: W1 [H][I], b1 [H], W2 [H][H], b2,
W3 [O][H], b3.
"""
import numpy as np
from scipy.special import erf


def gelu(u):
    """GELU(u) = u Phi(u), Phi the standard normal CDF."""
    return 0.5 * u * (1.0 + erf(u / np.sqrt(2.0)))


def gelu_grad(u):
    """GELU'(u) = Phi(u) + u phi(u)."""
    return 0.5 * (1.0 + erf(u / np.sqrt(2.0))) + u * np.exp(-0.5 * u * u) / np.sqrt(2.0 * np.pi)


def unpack(params, n_in, n_hid, n_out):
    """The six parameter arrays W1, b1, W2, b2, W3, b3 from the flat vector."""
    shapes = [(n_hid, n_in), (n_hid,), (n_hid, n_hid), (n_hid,), (n_out, n_hid), (n_out,)]
    out, off = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(np.asarray(params[off:off + n], dtype=np.float64).reshape(s))
        off += n
    return out


def forward(params, x, n_in, n_hid, n_out):
    """Outputs y [rows, n_out] and the activations the backward pass needs."""
    W1, b1, W2, b2, W3, b3 = unpack(params, n_in, n_hid, n_out)
    z1 = x @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    y = h2 @ W3.T + b3
    return y, (x, z1, h1, z2, h2)


def backward(params, cache, dy, n_in, n_hid, n_out):
    """Gradients of all parameters (flat, library layout) for dL/dy."""
    W1, b1, W2, b2, W3, b3 = unpack(params, n_in, n_hid, n_out)
    x, z1, h1, z2, h2 = cache
    gW3 = dy.T @ h2
    gb3 = dy.sum(axis=0)
    dz2 = (dy @ W3) * gelu_grad(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * gelu_grad(z1)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(axis=0)
    return np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3)])


def mse(y, t):
    """Mean squared error and its gradient with respect to y."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam_step(params, grads, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns new params, m, v."""
    m = b1 * m + (1 - b1) * grads
    v = b2 * v + (1 - b2) * grads * grads
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
