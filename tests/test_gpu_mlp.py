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


def _splitmix64(z):
    """SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) on Python integers."""
    m = (1 << 64) - 1
    z = (z + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def test_training_statistics_and_batches_on_the_gpu(built_lib, cuda):
    """icon_mlp_fit_normalization: per-feature mean and sample standard
    deviation (numpy, FP64) with the group floor, set as the network's
    statistics and applied to the rows; icon_mlp_train_step_sampled trains on
    the rows SplitMix64 picks (a step on exactly those rows, given explicitly,
    gives the same loss and parameters)."""
    import torch
    import paper_2608_21150_gb300 as P
    I, H, O, rows = 40, 64, 9, 5000
    rng = np.random.default_rng(3)
    x = (rng.standard_normal((rows, I)) * np.linspace(0.5, 4.0, I) + np.linspace(-3, 3, I)).astype(np.float32)
    x[:, 7] = 2.0 + 1e-9 * rng.standard_normal(rows)         # near-constant feature: floored
    y = (rng.standard_normal((rows, O)) * 3.0 + 1.0).astype(np.float32)
    xg, yg = [0, 10, 20, 30], [0, 4]
    net = P.MLP(I, H, O, max_batch=256)
    net.set_params(init_params(rng, I, H, O))
    xd, yd = torch.from_numpy(x).to(cuda), torch.from_numpy(y).to(cuda)
    xn, yn = torch.empty_like(xd), torch.empty_like(yd)
    net.fit_normalization(xd, yd, xg, yg, 1e-3, xn, yn)
    xm, xs, ym, ys = net.normalization

    def ref_stats(a, groups):
        mean, sd = a.astype(np.float64).mean(0), a.astype(np.float64).std(0, ddof=1)
        bounds = list(groups) + [a.shape[1]]
        for g0, g1 in zip(bounds[:-1], bounds[1:]):
            sd[g0:g1] = np.maximum(sd[g0:g1], max(sd[g0:g1].max() * 1e-3, 1e-30))
        return mean, sd
    rm, rs = ref_stats(x, xg)
    assert np.allclose(xm, rm, rtol=1e-6, atol=1e-6) and np.allclose(xs, rs, rtol=1e-6)
    assert np.isclose(xs[7], rs[7], rtol=1e-6) and rs[7] > 1e-3     # the floor: a thousandth of the group largest
    rm, rs = ref_stats(y, yg)
    assert np.allclose(ym, rm, rtol=1e-6, atol=1e-6) and np.allclose(ys, rs, rtol=1e-6)
    assert np.allclose(xn.cpu().numpy(), (x - xm) / xs, rtol=1e-6, atol=1e-6)
    # a sampled step is the explicit step on the rows SplitMix64 picks
    seed, step, batch = 12345, 7, 128
    idx = np.array([_splitmix64(seed + (step << 32) + i) % rows for i in range(batch)])
    twin = P.MLP(I, H, O, max_batch=256)
    twin.set_params(net.params())
    la = net.train_step_sampled(xn, yn, batch, seed, step, 1e-3)
    lb = twin.train_step(xn[torch.from_numpy(idx).to(cuda)].contiguous(), yn[torch.from_numpy(idx).to(cuda)].contiguous(),
                         1e-3)
    assert la == lb
    assert np.array_equal(net.params(), twin.params())
