"""FP64 CPU reference of the learned preconditioner's network (test
infrastructure only).

The network maps a Jacobi-scaled residual to a Jacobi-scaled error estimate
on the slot lattice (one channel per unknown field).  It is a three-level
U-Net (two 3x3(x3) convolutions with ReLU per level, 2x average-pool down,
nearest-neighbour up, skip concatenation, 1x1 output convolution).  Channel
widths 8/16/32.  Parameters are one flat vector in this order, each conv as
weight (Cout, Cin, k...) then bias (Cout):

  enc0a (cin->8)  enc0b (8->8)  enc1a (8->16) enc1b (16->16)
  enc2a (16->32)  enc2b (32->32)
  dec1a (32+16->16) dec1b (16->16)  dec0a (16+8->8) dec0b (8->8)
  out (8->cout, 1x1)

Concatenation order is [upsampled, skip].  Spatial sizes must be multiples
of 4.  Convolutions use zero padding 1.  Everything is FP64 torch CPU math;
torch's convolution routine is the library primitive, gradients come from
autograd.

``store`` optionally models a network that keeps its activations in a
narrower type: it is applied to every hidden activation after its ReLU and
to every pooled map (the values a kernel writes to memory and reads back),
with the gradient passed straight through, so the result is the FP64
network evaluated at the stored values.  ``bf16_store`` rounds to bfloat16
(round to nearest, ties to even).  ReLU masks and weight gradients then see
the same stored values as a kernel that stores BF16, which is how two
implementations can take the same ReLU decisions.
"""
import numpy as np
import torch
import torch.nn.functional as Fn

WIDTHS = (8, 16, 32)


def layer_shapes(dim, cin, cout):
    k = (3,) * dim
    w0, w1, w2 = WIDTHS
    convs = [("enc0a", w0, cin, k), ("enc0b", w0, w0, k), ("enc1a", w1, w0, k), ("enc1b", w1, w1, k),
             ("enc2a", w2, w1, k), ("enc2b", w2, w2, k), ("dec1a", w1, w2 + w1, k), ("dec1b", w1, w1, k),
             ("dec0a", w0, w1 + w0, k), ("dec0b", w0, w0, k), ("out", cout, w0, (1,) * dim)]
    return convs


def n_params(dim, cin, cout):
    return sum(co * ci * int(np.prod(k)) + co for _, co, ci, k in layer_shapes(dim, cin, cout))


def unpack(theta, dim, cin, cout):
    """Flat parameter vector -> dict name -> (W, b) torch tensors (views)."""
    out, o = {}, 0
    for name, co, ci, k in layer_shapes(dim, cin, cout):
        nw = co * ci * int(np.prod(k))
        W = theta[o:o + nw].reshape((co, ci) + k)
        o += nw
        b = theta[o:o + co]
        o += co
        out[name] = (W, b)
    assert o == theta.numel()
    return out


def init_params(dim, cin, cout, seed=0):
    """He-uniform weights, zero biases (float64 numpy)."""
    rng = np.random.default_rng(seed)
    parts = []
    for _, co, ci, k in layer_shapes(dim, cin, cout):
        fan_in = ci * int(np.prod(k))
        lim = np.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-lim, lim, co * ci * int(np.prod(k))))
        parts.append(np.zeros(co))
    return np.concatenate(parts)


def _conv(x, Wb, dim):
    W, b = Wb
    f = Fn.conv2d if dim == 2 else Fn.conv3d
    pad = W.shape[-1] // 2
    return f(x, W, b, padding=pad)


def _pool(x, dim):
    return Fn.avg_pool2d(x, 2) if dim == 2 else Fn.avg_pool3d(x, 2)


def _up(x):
    return Fn.interpolate(x, scale_factor=2, mode="nearest")


def bf16_store(t):
    """Values rounded to bfloat16, gradient passed through unchanged."""
    return t + (t.detach().to(torch.bfloat16).to(torch.float64) - t.detach())


def forward(theta, x, dim, cin, cout, store=None):
    """x: (B, cin, [Z,] Y, X) float64 tensor -> (B, cout, ...)."""
    P = unpack(theta, dim, cin, cout)
    s = store or (lambda t: t)
    r = lambda t: s(torch.relu(t))
    pool = lambda t: s(_pool(t, dim))
    e0 = r(_conv(r(_conv(x, P["enc0a"], dim)), P["enc0b"], dim))
    e1 = r(_conv(r(_conv(pool(e0), P["enc1a"], dim)), P["enc1b"], dim))
    e2 = r(_conv(r(_conv(pool(e1), P["enc2a"], dim)), P["enc2b"], dim))
    d1 = r(_conv(r(_conv(torch.cat([_up(e2), e1], 1), P["dec1a"], dim)), P["dec1b"], dim))
    d0 = r(_conv(r(_conv(torch.cat([_up(d1), e0], 1), P["dec0a"], dim)), P["dec0b"], dim))
    return _conv(d0, P["out"], dim)


def loss_and_grad(theta_np, x_np, y_np, dim, cin, cout, store=None):
    """Mean over samples of ||N(x) - y||^2 / ||y||^2 and its gradient."""
    theta = torch.tensor(theta_np, dtype=torch.float64, requires_grad=True)
    x = torch.as_tensor(x_np, dtype=torch.float64)
    y = torch.as_tensor(y_np, dtype=torch.float64)
    out = forward(theta, x, dim, cin, cout, store)
    num = ((out - y) ** 2).flatten(1).sum(1)
    den = (y ** 2).flatten(1).sum(1).clamp_min(1e-300)
    loss = (num / den).mean()
    loss.backward()
    return float(loss), theta.grad.numpy().copy()


def predict(theta_np, x_np, dim, cin, cout, store=None):
    with torch.no_grad():
        return forward(torch.as_tensor(theta_np), torch.as_tensor(x_np, dtype=torch.float64), dim, cin,
                       cout, store).numpy()
