"""Pins of the CPU U-Net reference (oracle.unet): its convolution agrees with
a direct loop written from the definition, its gradient agrees with central
finite differences, pooling and nearest upsampling are adjoint up to the
factor 2^dim, and the parameter count is the planned ~91k in 3D."""
import numpy as np
import pytest
import torch

from oracle import unet as U


def _direct_conv(x, W, b):
    """Zero-padded cross-correlation, written as loops over the definition."""
    B, Ci = x.shape[:2]
    Co = W.shape[0]
    k = W.shape[2]
    p = k // 2
    sp = x.shape[2:]
    xp = np.pad(x, [(0, 0), (0, 0)] + [(p, p)] * len(sp))
    out = np.zeros((B, Co) + sp)
    for idx in np.ndindex(*sp):
        for off in np.ndindex(*([k] * len(sp))):
            sl = tuple(slice(i + o, i + o + 1) for i, o in zip(idx, off))
            patch = xp[(slice(None), slice(None)) + sl].reshape(B, Ci)
            out[(slice(None), slice(None)) + idx] += patch @ W[(slice(None), slice(None)) + off].T
    return out + b.reshape((1, Co) + (1,) * len(sp))


@pytest.mark.parametrize("dim", [2, 3])
def test_conv_matches_definition(dim):
    rng = np.random.default_rng(dim)
    sp = (5, 4) if dim == 2 else (4, 3, 5)
    x = rng.normal(size=(2, 3) + sp)
    W = rng.normal(size=(4, 3) + (3,) * dim)
    b = rng.normal(size=4)
    got = U._conv(torch.tensor(x), (torch.tensor(W), torch.tensor(b)), dim).numpy()
    assert np.allclose(got, _direct_conv(x, W, b), atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_pool_and_upsample_are_adjoint(dim):
    rng = np.random.default_rng(5)
    sp = (8, 4) if dim == 2 else (4, 8, 4)
    x = torch.tensor(rng.normal(size=(1, 2) + sp))
    y = torch.tensor(rng.normal(size=(1, 2) + tuple(s // 2 for s in sp)))
    lhs = (U._pool(x, dim) * y).sum()
    rhs = (x * U._up(y)).sum() / 2 ** dim
    assert abs(float(lhs - rhs)) < 1e-12


def test_parameter_count():
    assert 85_000 < U.n_params(3, 12, 6) < 100_000


@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_matches_finite_differences(dim):
    rng = np.random.default_rng(7)
    cin, cout = 4, 3
    sp = (8, 8) if dim == 2 else (4, 8, 4)
    th = U.init_params(dim, cin, cout, seed=1) + rng.normal(scale=0.01, size=U.n_params(dim, cin, cout))
    x = rng.normal(size=(2, cin) + sp)
    y = rng.normal(size=(2, cout) + sp)
    L, g = U.loss_and_grad(th, x, y, dim, cin, cout)
    for i in rng.choice(th.size, 25, replace=False):
        e = np.zeros_like(th)
        h = 1e-6 * max(1.0, abs(th[i]))
        e[i] = h
        fd = (U.loss_and_grad(th + e, x, y, dim, cin, cout)[0] - U.loss_and_grad(th - e, x, y, dim, cin, cout)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8, (i, fd, g[i])


def test_bf16_store_rounds_to_nearest_even_and_passes_gradients():
    # bfloat16 keeps 8 significant bits: the spacing just above 1 is 2^-7
    vals = torch.tensor([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -8 + 2.0 ** -20, -(1 + 2.0 ** -8 + 2.0 ** -20),
                         3.0, 0.0], dtype=torch.float64, requires_grad=True)
    want = [1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, -(1 + 2.0 ** -7), 3.0, 0.0]
    got = U.bf16_store(vals)
    assert got.detach().tolist() == want
    w = torch.arange(6, dtype=torch.float64)
    (got * w).sum().backward()
    assert vals.grad.tolist() == w.tolist()


def test_store_hook_is_neutral_when_it_is_the_identity():
    rng = np.random.default_rng(11)
    th = U.init_params(2, 4, 3, seed=2)
    x = rng.normal(size=(1, 4, 8, 8))
    y = rng.normal(size=(1, 3, 8, 8))
    L0, g0 = U.loss_and_grad(th, x, y, 2, 4, 3)
    L1, g1 = U.loss_and_grad(th, x, y, 2, 4, 3, store=lambda t: t)
    assert L0 == L1 and np.array_equal(g0, g1)
    # BF16 storage changes the output by about the BF16 precision, no more
    a = U.predict(th, x, 2, 4, 3)
    b = U.predict(th, x, 2, 4, 3, store=U.bf16_store)
    assert 0 < np.abs(a - b).max() <= 3e-2 * np.abs(a).max()
