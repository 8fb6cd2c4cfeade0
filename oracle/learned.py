"""FP64 reference of the learned Poisson initial guess (plain numpy).

TEST INFRASTRUCTURE ONLY: the definition the CUDA network kernels are checked against.

Network: three 3x3x3 "same" convolutions with zero padding on a channel-last grid [nz, ny, nx, C],
8 -> 8 (ReLU) -> 8 (ReLU) -> 1.  The input has 8 channels of which the first three carry features (the
others are zero).  Weights are W[l][co, tap, ci] with tap = (dz+1)*9 + (dy+1)*3 + (dx+1) and bias
B[l][co].  Loss: mean over cells of (out - target)^2.
"""
import numpy as np

C = 8
TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shift(x, dz, dy, dx):
    """y[z, y, x] = x[z + dz, y + dy, x + dx], zero outside the grid."""
    out = np.zeros_like(x)
    nz, ny, nx = x.shape[:3]
    zs, ze = max(0, -dz), min(nz, nz - dz)
    ys, ye = max(0, -dy), min(ny, ny - dy)
    xs, xe = max(0, -dx), min(nx, nx - dx)
    out[zs:ze, ys:ye, xs:xe] = x[zs + dz:ze + dz, ys + dy:ye + dy, xs + dx:xe + dx]
    return out


def conv(x, W, b):
    """z[c, co] = b[co] + sum_tap sum_ci W[co, tap, ci] x[c + off(tap), ci]."""
    z = np.zeros(x.shape[:3] + (W.shape[0],)) + b
    for t, (dz, dy, dx) in enumerate(TAPS):
        z += shift(x, dz, dy, dx) @ W[:, t, :].T
    return z


def conv_input_grad(dz_, W):
    """Gradient w.r.t. the input of conv: dx[c, ci] = sum_tap sum_co W[co, tap, ci] dz[c - off(tap), co]."""
    dx_ = np.zeros(dz_.shape[:3] + (W.shape[2],))
    for t, (dz, dy, dx) in enumerate(TAPS):
        dx_ += shift(dz_, -dz, -dy, -dx) @ W[:, t, :]
    return dx_


def conv_weight_grad(dz_, x):
    """dW[co, tap, ci] = sum_c dz[c, co] x[c + off(tap), ci];  db[co] = sum_c dz[c, co]."""
    co, ci = dz_.shape[-1], x.shape[-1]
    dW = np.zeros((co, 27, ci))
    D = dz_.reshape(-1, co)
    for t, (dz, dy, dx) in enumerate(TAPS):
        dW[:, t, :] = D.T @ shift(x, dz, dy, dx).reshape(-1, ci)
    return dW, D.sum(0)


def init_params(seed=0, scale=0.1):
    rng = np.random.default_rng(seed)
    W = [rng.standard_normal((C, 27, C)) * scale, rng.standard_normal((C, 27, C)) * scale,
         rng.standard_normal((1, 27, C)) * scale]
    B = [np.zeros(C), np.zeros(C), np.zeros(1)]
    return W, B


def forward(x, W, B):
    """Returns the output [.., 1] and the activations needed by backward."""
    z1 = conv(x, W[0], B[0])
    y1 = np.maximum(z1, 0.0)
    z2 = conv(y1, W[1], B[1])
    y2 = np.maximum(z2, 0.0)
    out = conv(y2, W[2], B[2])
    return out, (x, y1, y2)


def loss_and_grads(x, target, W, B):
    out, (x0, y1, y2) = forward(x, W, B)
    n = out[..., 0].size
    diff = out[..., 0] - target
    loss = np.mean(diff ** 2)
    d3 = (2.0 / n) * diff[..., None]
    dW3, dB3 = conv_weight_grad(d3, y2)
    dy2 = conv_input_grad(d3, W[2])
    d2 = dy2 * (y2 > 0)
    dW2, dB2 = conv_weight_grad(d2, y1)
    dy1 = conv_input_grad(d2, W[1])
    d1 = dy1 * (y1 > 0)
    dW1, dB1 = conv_weight_grad(d1, x0)
    return loss, [dW1, dW2, dW3], [dB1, dB2, dB3], out
