"""FP64 oracle of the learned 4x upsampler: forward, loss, backward and Adam.

TEST INFRASTRUCTURE ONLY. Only tests/, the package's smoke entry and the bench's
CPU-baseline leg import this module; the library never does. It shares no code
with the CUDA kernels.

The paper (Sec. 3.2) renders every robot camera at 640x480; the upsampler turns
a 160x120 render of the same pose into 640x480. The network is a plain residual
CNN, written here from the textbook definitions (numpy, float64, NHWC images):

    x0  = [rgb_lr - 1/2, S (rgb_lr - box3(rgb_lr))]  (6 channels)
    h_l = relu(conv3x3(h_{l-1}; W_l, b_l))           l = 1..5, 32 channels
    z6  = conv3x3(h_5; W_6, b_6)                     48 = 3 * 4 * 4 channels
    out = bilinear4(rgb_lr) + pixel_shuffle4(z6) / S  (3 channels at 4x)

with S = 32. The detail channels and the 1/S output scale keep the small
differences the network reads and writes (renders of dense scenes differ from
their bilinear upsampling by ~1e-3) far above the relative precision of BF16
storage (2^-9 of the value stored); in float64 they are only a change of units.
box3: mean of the 3x3 neighbourhood, indices clamped to the image.

conv3x3: cross-correlation with zero padding 1, weights [c_out][c_in][3][3]
    y[i, j, o] = b[o] + sum_{c, u, v} W[o, c, u, v] x[i + u - 1, j + v - 1, c]
pixel_shuffle4: out[4 i + dy, 4 j + dx, c] = z[i, j, 16 c + 4 dy + dx]
bilinear4: half-pixel centres (an HR pixel centre (i + 1/2) lies at LR
    coordinate (i + 1/2) / 4); source s = (i + 1/2) / 4 - 1/2, clamped to
    [0, n - 1]; i0 = floor(s), i1 = min(i0 + 1, n - 1), weight s - i0.
loss: mean over all HR pixels and channels of (out - target)^2.
Adam: Kingma & Ba (2015), bias-corrected moments.

Pins (tests/test_oracle_upsampler.py): conv against scipy.signal.correlate2d,
pixel shuffle against a brute-force index loop and torch.pixel_shuffle,
bilinear against torch.nn.functional.interpolate and on linear ramps (exact in
the interior), every gradient against central finite differences, Adam against
its closed-form first step.
"""
from __future__ import annotations

import numpy as np

C_MID = 32
N_LAYERS = 6
SCALE = 4
C_IN = 6
DETAIL_SCALE = 32.0


def layer_shapes(c_in: int = C_IN, c_mid: int = C_MID, scale: int = SCALE):
    """(c_out, c_in) of the six 3x3 convolutions."""
    c_out_last = 3 * scale * scale
    return [(c_mid, c_in)] + [(c_mid, c_mid)] * (N_LAYERS - 2) + [(c_out_last, c_mid)]


def init_params(seed: int, c_mid: int = C_MID, zero_last: bool = True) -> list:
    """He-normal weights, zero biases; the last layer zero so the network starts
    as plain bilinear upsampling."""
    rng = np.random.default_rng([seed, 7])
    params = []
    for li, (co, ci) in enumerate(layer_shapes(C_IN, c_mid)):
        std = np.sqrt(2.0 / (9 * ci))
        W = rng.normal(0.0, std, size=(co, ci, 3, 3))
        if zero_last and li == N_LAYERS - 1:
            W[:] = 0.0
        params.append((W, np.zeros(co)))
    return params


def conv3x3(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x [n][h][w][c_in], W [c_out][c_in][3][3], b [c_out] -> [n][h][w][c_out]."""
    n, h, w, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.broadcast_to(b, (n, h, w, W.shape[0])).astype(np.float64).copy()
    for u in range(3):
        for v in range(3):
            y += xp[:, u:u + h, v:v + w, :] @ W[:, :, u, v].T
    return y


def conv3x3_backward(x: np.ndarray, W: np.ndarray, dy: np.ndarray):
    """Gradients of conv3x3 given dL/dy: (dL/dx, dL/dW, dL/db)."""
    n, h, w, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for u in range(3):
        for v in range(3):
            win = xp[:, u:u + h, v:v + w, :]
            dW[:, :, u, v] = np.einsum("nijo,nijc->oc", dy, win)
            dxp[:, u:u + h, v:v + w, :] += dy @ W[:, :, u, v]
    return dxp[:, 1:h + 1, 1:w + 1, :], dW, dy.sum(axis=(0, 1, 2))


def pixel_shuffle(z: np.ndarray, r: int = SCALE) -> np.ndarray:
    """[n][h][w][c r^2] -> [n][h r][w r][c]; channel c r^2 + r dy + dx goes to
    (r i + dy, r j + dx)."""
    n, h, w, crr = z.shape
    c = crr // (r * r)
    t = z.reshape(n, h, w, c, r, r)            # [..., c, dy, dx]
    return t.transpose(0, 1, 4, 2, 5, 3).reshape(n, h * r, w * r, c)


def pixel_unshuffle(o: np.ndarray, r: int = SCALE) -> np.ndarray:
    """Inverse of pixel_shuffle (also its adjoint: a permutation)."""
    n, H, W, c = o.shape
    t = o.reshape(n, H // r, r, W // r, r, c)  # [n, i, dy, j, dx, c]
    return t.transpose(0, 1, 3, 5, 2, 4).reshape(n, H // r, W // r, c * r * r)


def _bilinear_axis(n_src: int, r: int):
    i = np.arange(n_src * r)
    s = np.clip((i + 0.5) / r - 0.5, 0.0, n_src - 1)
    i0 = np.floor(s).astype(np.int64)
    i1 = np.minimum(i0 + 1, n_src - 1)
    return i0, i1, s - i0


def bilinear(x: np.ndarray, r: int = SCALE) -> np.ndarray:
    """[n][h][w][c] -> [n][h r][w r][c], half-pixel centres, edge clamp."""
    _, h, w, _ = x.shape
    y0, y1, fy = _bilinear_axis(h, r)
    x0, x1, fx = _bilinear_axis(w, r)
    top = x[:, y0] * (1 - fy)[None, :, None, None] + x[:, y1] * fy[None, :, None, None]
    return top[:, :, x0] * (1 - fx)[None, None, :, None] + top[:, :, x1] * fx[None, None, :, None]


def box3(x: np.ndarray) -> np.ndarray:
    """Mean of the 3x3 neighbourhood of every pixel, indices clamped."""
    _, h, w, _ = x.shape
    acc = np.zeros_like(x, dtype=np.float64)
    for du in (-1, 0, 1):
        rows = np.clip(np.arange(h) + du, 0, h - 1)
        for dv in (-1, 0, 1):
            cols = np.clip(np.arange(w) + dv, 0, w - 1)
            acc += x[:, rows][:, :, cols]
    return acc / 9.0


def network_input(rgb: np.ndarray) -> np.ndarray:
    """x0 = [rgb - 1/2, S (rgb - box3(rgb))]."""
    x = np.asarray(rgb, np.float64)
    return np.concatenate([x - 0.5, DETAIL_SCALE * (x - box3(x))], axis=-1)


def forward(params: list, rgb: np.ndarray, keep: bool = False):
    """rgb [n][h][w][3] -> out [n][4h][4w][3]; with keep, also every layer's
    input and the last layer's output, as backward needs them."""
    x = np.asarray(rgb, np.float64)
    h = network_input(x)
    acts = [h]
    for li, (W, b) in enumerate(params):
        z = conv3x3(h, W, b)
        h = np.maximum(z, 0.0) if li < N_LAYERS - 1 else z
        acts.append(h)
    out = bilinear(x) + pixel_shuffle(acts[-1]) / DETAIL_SCALE
    return (out, acts) if keep else out


def loss_and_grads(params: list, rgb: np.ndarray, target: np.ndarray):
    """Mean squared error and its gradient for every (W, b)."""
    out, acts = forward(params, rgb, keep=True)
    diff = out - np.asarray(target, np.float64)
    loss = float(np.mean(diff * diff))
    d = pixel_unshuffle(2.0 * diff / diff.size) / DETAIL_SCALE
    grads = [None] * N_LAYERS
    for li in range(N_LAYERS - 1, -1, -1):
        W, _ = params[li]
        dx, dW, db = conv3x3_backward(acts[li], W, d)
        grads[li] = (dW, db)
        if li > 0:
            d = dx * (acts[li] > 0.0)   # relu'(z) of the layer below, from its output
    return loss, grads


def psnr(a: np.ndarray, b: np.ndarray) -> float:
    """10 log10(1 / MSE) on images clamped to [0, 1]."""
    mse = np.mean((np.clip(a, 0, 1) - np.clip(b, 0, 1)) ** 2)
    return float(10.0 * np.log10(1.0 / mse)) if mse > 0 else float("inf")


class Adam:
    """Adam with bias correction; state per parameter array."""

    def __init__(self, params: list, lr: float = 1e-3, beta1: float = 0.9,
                 beta2: float = 0.999, eps: float = 1e-8):
        self.lr, self.b1, self.b2, self.eps, self.t = lr, beta1, beta2, eps, 0
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]

    def step(self, params: list, grads: list) -> list:
        self.t += 1
        c1, c2 = 1 - self.b1 ** self.t, 1 - self.b2 ** self.t
        new = []
        for i, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
            pair = []
            for k, (p, g) in enumerate(((W, gW), (b, gb))):
                m = self.b1 * self.m[i][k] + (1 - self.b1) * g
                v = self.b2 * self.v[i][k] + (1 - self.b2) * g * g
                pair.append(p - self.lr * (m / c1) / (np.sqrt(v / c2) + self.eps))
                if k == 0:
                    mW, vW = m, v
                else:
                    self.m[i], self.v[i] = (mW, m), (vW, v)
            new.append(tuple(pair))
        return new
