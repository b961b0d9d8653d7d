"""The learned corrector's tensor-core MLP (BF16 weights/activations, FP32
accumulate) against the FP64 CPU oracle: forward pass, parameter gradients,
the first Adam step, and training on a fixed regression problem."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def bf16(a):
    """Round to the nearest BF16 value (ties to even), as the GPU stores weights and inputs."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(rng, I, H, O):
    parts = [rng.standard_normal((H, I)) / np.sqrt(I), 0.1 * rng.standard_normal(H),
             rng.standard_normal((H, H)) / np.sqrt(H), 0.1 * rng.standard_normal(H),
             rng.standard_normal((O, H)) / np.sqrt(H), 0.1 * rng.standard_normal(O)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def weights_rounded(p, I, H, O):
    """The oracle sees the BF16-rounded weight matrices and the FP32 biases."""
    W1, b1, W2, b2, W3, b3 = omlp.unpack(p, I, H, O)
    return np.concatenate([bf16(W1).ravel(), b1, bf16(W2).ravel(), b2, bf16(W3).ravel(), b3])


@pytest.mark.parametrize("dims", [(450, 512, 269, 256), (37, 64, 5, 128), (990, 512, 90, 192)])
def test_mlp_forward_and_gradients_match_oracle(built_lib, cuda, dims):
    import torch
    import paper_2608_21150_gb300 as P
    I, H, O, B = dims
    rng = np.random.default_rng(I + H + O)
    p = init_params(rng, I, H, O)
    x = rng.standard_normal((B, I)).astype(np.float32)
    t = rng.standard_normal((B, O)).astype(np.float32)
    net = P.MLP(I, H, O, max_batch=256)
    net.set_params(p)
    assert net.n_params == p.size
    xd = torch.from_numpy(x).to(cuda)
    yd = torch.empty((B, O), dtype=torch.float32, device=cuda)
    net.forward(xd, yd)
    pr = weights_rounded(p, I, H, O)
    y_ref, cache = omlp.forward(pr, bf16(x), I, H, O)
    y = yd.cpu().numpy()
    assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref) < 1e-2
    _, dy = omlp.mse(y_ref, t)
    g_ref = omlp.backward(pr, cache, dy, I, H, O)
    net.backward(torch.from_numpy(dy.astype(np.float32)).to(cuda))
    g = net.grads().astype(np.float64)
    off = 0
    for shape in [(H, I), (H,), (H, H), (H,), (O, H), (O,)]:
        n = int(np.prod(shape))
        a, b = g[off:off + n], g_ref[off:off + n]
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 3e-2, (shape, np.linalg.norm(a - b) / np.linalg.norm(b))
        off += n
    # the first Adam step moves every parameter with a clear gradient by lr * sign(g)
    lr = 1e-3
    net.adam(lr)
    q = net.params().astype(np.float64)
    big = np.abs(g) > 1e-4
    assert np.allclose((q - p)[big], -lr * np.sign(g[big]), rtol=0, atol=2e-5)


def test_mlp_training_reduces_the_loss(built_lib, cuda):
    import torch
    import paper_2608_21150_gb300 as P
    I, H, O, B = 32, 128, 8, 256
    rng = np.random.default_rng(5)
    x = rng.standard_normal((4 * B, I)).astype(np.float32)
    A = rng.standard_normal((I, O)) / np.sqrt(I)
    t = (np.tanh(x @ A) + 0.1 * x[:, :O] ** 2).astype(np.float32)
    net = P.MLP(I, H, O, max_batch=B)
    net.set_params(init_params(rng, I, H, O))
    xd, td = torch.from_numpy(x).to(cuda), torch.from_numpy(t).to(cuda)
    losses = []
    for it in range(300):
        s = (it % 4) * B
        losses.append(net.train_step(xd[s:s + B], td[s:s + B], 3e-3))
    assert losses[-1] < 0.1 * losses[0], (losses[0], losses[-1])
