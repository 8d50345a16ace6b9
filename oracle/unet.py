"""CPU oracle of the learned initialiser (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may import
this module; the library never does. It restates, in plain numpy (float64), what the
network computes: 3x3 convolutions with zero padding written as a sum over the nine
taps, ReLU, 2x2 average pooling, nearest-neighbour x2 upsampling, channel
concatenation, the mean-squared loss over the interior sites, the exact backward
pass of all of it, and the Adam update that trains it (Kingma & Ba 2015,
Algorithm 1). Nothing here is blocked, fused or reordered.

The paper has no learned component (it starts every relaxation from a
model-specific ansatz, Sec. 4.1); the architecture is the 4-level U-Net with
widths 16, 32, 48, 96 that the library implements, so this file follows that
definition, not a passage of the paper.

With ``bf16=True`` every value is rounded to bfloat16 where the GPU stores it
(inputs, weights, hidden activations, pooled and upsampled maps, and the output
gradient of each convolution before it enters a contraction); everything else is
float64. Rounding is round-to-nearest-even on the float32 value (the bfloat16
format keeps the upper 16 bits of an IEEE float32).

Pins: tests/test_unet_oracle.py (direct-sum definition, scipy correlation,
adjointness of every linear layer, central-difference gradients, torch's bfloat16
conversion, Adam's closed-form first steps).
"""
from __future__ import annotations

import numpy as np

WIDTHS = (16, 32, 48, 96)
CIN = 16
COUT = 16


def round_bf16(x) -> np.ndarray:
    """Nearest bfloat16 value (ties to even) of float32(x), as float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


# ---------------------------------------------------------------- layers
def shift(x: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """s[n, y, x] = x[n, y + dy, x + dx], zero outside the image."""
    N, H, W, C = x.shape
    s = np.zeros_like(x)
    ys, ye = max(0, -dy), min(H, H - dy)
    xs, xe = max(0, -dx), min(W, W - dx)
    s[:, ys:ye, xs:xe] = x[:, ys + dy:ye + dy, xs + dx:xe + dx]
    return s


TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]  # tap index 3 (dy + 1) + (dx + 1)


def conv3x3(x: np.ndarray, w: np.ndarray, b=None) -> np.ndarray:
    """out[n, y, x, co] = sum_{tap, ci} x[n, y + dy, x + dx, ci] w[co, tap, ci] (+ b[co])."""
    out = np.zeros(x.shape[:3] + (w.shape[0],))
    for t, (dy, dx) in enumerate(TAPS):
        out += shift(x, dy, dx) @ w[:, t, :].T
    if b is not None:
        out += b
    return out


def conv3x3_direct(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """The same sum with explicit loops (small inputs only)."""
    N, H, W, C = x.shape
    out = np.zeros((N, H, W, w.shape[0]))
    for n in range(N):
        for y in range(H):
            for xx in range(W):
                for co in range(w.shape[0]):
                    acc = 0.0
                    for t, (dy, dx) in enumerate(TAPS):
                        yy, xs = y + dy, xx + dx
                        if 0 <= yy < H and 0 <= xs < W:
                            for ci in range(C):
                                acc += x[n, yy, xs, ci] * w[co, t, ci]
                    out[n, y, xx, co] = acc
    return out


def conv3x3_grad_input(gy: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Adjoint of conv3x3 in x: gx[n, y, x, ci] = sum_{tap, co} gy[n, y - dy, x - dx, co] w[co, tap, ci]."""
    gx = np.zeros(gy.shape[:3] + (w.shape[2],))
    for t, (dy, dx) in enumerate(TAPS):
        gx += shift(gy, -dy, -dx) @ w[:, t, :]
    return gx


def conv3x3_grad_weight(x: np.ndarray, gy: np.ndarray) -> np.ndarray:
    """gw[co, tap, ci] = sum_{n, y, x} gy[n, y, x, co] x[n, y + dy, x + dx, ci]."""
    Co, Ci = gy.shape[3], x.shape[3]
    gw = np.zeros((Co, 9, Ci))
    g2 = gy.reshape(-1, Co)
    for t, (dy, dx) in enumerate(TAPS):
        gw[:, t, :] = g2.T @ shift(x, dy, dx).reshape(-1, Ci)
    return gw


def avgpool2(x: np.ndarray) -> np.ndarray:
    N, H, W, C = x.shape
    return x.reshape(N, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def avgpool2_backward(g: np.ndarray) -> np.ndarray:
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) / 4.0


def upsample2(x: np.ndarray) -> np.ndarray:
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_backward(g: np.ndarray) -> np.ndarray:
    N, H, W, C = g.shape
    return g.reshape(N, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


# ---------------------------------------------------------------- network
def layer_shapes(widths=WIDTHS, cin=CIN, cout=COUT):
    """(input channels, output channels) of the 15 convolutions, in execution order."""
    c1, c2, c3, c4 = widths
    return [(cin, c1), (c1, c1), (c1, c2), (c2, c2), (c2, c3), (c3, c3), (c3, c4), (c4, c4),
            (c4 + c3, c3), (c3, c3), (c3 + c2, c2), (c2, c2), (c2 + c1, c1), (c1, c1), (c1, cout)]


def unflatten(theta: np.ndarray, widths=WIDTHS, cin=CIN, cout=COUT):
    """Split the flat parameter vector (per layer W[cout][9][cin], then b[cout])."""
    out, k = [], 0
    for ci, co in layer_shapes(widths, cin, cout):
        w = theta[k:k + 9 * ci * co].reshape(co, 9, ci)
        k += 9 * ci * co
        b = theta[k:k + co]
        k += co
        out.append((w, b))
    assert k == theta.size
    return out


def num_params(widths=WIDTHS, cin=CIN, cout=COUT) -> int:
    return sum(9 * ci * co + co for ci, co in layer_shapes(widths, cin, cout))


def forward(theta: np.ndarray, x: np.ndarray, widths=WIDTHS, bf16: bool = True):
    """Returns (output, cache). x: [N, S, S, cin] input; output float64 [N, S, S, cout]."""
    r = round_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    P = [(r(w), np.asarray(b, dtype=np.float64)) for w, b in unflatten(theta, widths, x.shape[3])]
    relu = lambda a: np.maximum(a, 0.0)
    c = {}
    c["in"] = r(x)

    def cv(i, a):
        return r(relu(conv3x3(a, P[i][0], P[i][1])))

    c["e1a"] = cv(0, c["in"]); c["e1"] = cv(1, c["e1a"]); c["p1"] = r(avgpool2(c["e1"]))
    c["e2a"] = cv(2, c["p1"]); c["e2"] = cv(3, c["e2a"]); c["p2"] = r(avgpool2(c["e2"]))
    c["e3a"] = cv(4, c["p2"]); c["e3"] = cv(5, c["e3a"]); c["p3"] = r(avgpool2(c["e3"]))
    c["b1"] = cv(6, c["p3"]); c["b"] = cv(7, c["b1"])
    c["cat3"] = np.concatenate([upsample2(c["b"]), c["e3"]], axis=3)
    c["d3a"] = cv(8, c["cat3"]); c["d3"] = cv(9, c["d3a"])
    c["cat2"] = np.concatenate([upsample2(c["d3"]), c["e2"]], axis=3)
    c["d2a"] = cv(10, c["cat2"]); c["d2"] = cv(11, c["d2a"])
    c["cat1"] = np.concatenate([upsample2(c["d2"]), c["e1"]], axis=3)
    c["d1a"] = cv(12, c["cat1"]); c["d1"] = cv(13, c["d1a"])
    out = conv3x3(c["d1"], P[14][0], P[14][1])
    c["P"] = P
    return out, c


def mse(out: np.ndarray, target: np.ndarray, C: int):
    """Loss over the interior sites (halo of width 2 excluded) and the first C output
    channels; target [N, C, S, S] (SoA). Returns (loss, d loss / d out)."""
    N, S = out.shape[0], out.shape[1]
    t = np.transpose(np.asarray(target, dtype=np.float64), (0, 2, 3, 1))
    d = np.zeros_like(out)
    inner = (slice(None), slice(2, S - 2), slice(2, S - 2))
    diff = out[inner + (slice(0, C),)] - t[inner]
    count = N * (S - 4) ** 2 * C
    d[inner + (slice(0, C),)] = 2.0 * diff / count
    return float(np.sum(diff * diff) / count), d


def backward(theta: np.ndarray, cache: dict, gout: np.ndarray, widths=WIDTHS, bf16: bool = True,
             magnitudes: bool = False):
    """Gradient of the loss with respect to the flat parameter vector, given d loss / d output.
    With magnitudes=True, also the flat vector of the sums of the absolute values of
    the terms that make up each gradient entry (the same contractions on |x| and |g|):
    the scale against which an accumulation in another order or precision is judged."""
    r = round_bf16 if bf16 else (lambda a: a)
    c, P = cache, cache["P"]
    c1, c2, c3, c4 = widths
    grads = [None] * 15
    mags = [None] * 15

    def back(i, x, y, gy, need_gx=True):
        g = gy * (y > 0) if y is not None else gy
        grads[i] = (conv3x3_grad_weight(x, r(g)), g.sum(axis=(0, 1, 2)))
        if magnitudes:
            mags[i] = (conv3x3_grad_weight(np.abs(x), np.abs(r(g))), np.abs(g).sum(axis=(0, 1, 2)))
        return conv3x3_grad_input(r(g), P[i][0]) if need_gx else None

    g = back(14, c["d1"], None, gout)
    g = back(13, c["d1a"], c["d1"], g)
    gcat1 = back(12, c["cat1"], c["d1a"], g)
    g = back(11, c["d2a"], c["d2"], upsample2_backward(gcat1[..., :c2]))
    gcat2 = back(10, c["cat2"], c["d2a"], g)
    g = back(9, c["d3a"], c["d3"], upsample2_backward(gcat2[..., :c3]))
    gcat3 = back(8, c["cat3"], c["d3a"], g)
    g = back(7, c["b1"], c["b"], upsample2_backward(gcat3[..., :c4]))
    gp3 = back(6, c["p3"], c["b1"], g)
    g = back(5, c["e3a"], c["e3"], gcat3[..., c4:] + avgpool2_backward(gp3))
    gp2 = back(4, c["p2"], c["e3a"], g)
    g = back(3, c["e2a"], c["e2"], gcat2[..., c3:] + avgpool2_backward(gp2))
    gp1 = back(2, c["p1"], c["e2a"], g)
    g = back(1, c["e1a"], c["e1"], gcat1[..., c2:] + avgpool2_backward(gp1))
    back(0, c["in"], c["e1a"], g, need_gx=False)
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    if magnitudes:
        return flat, np.concatenate([np.concatenate([mw.ravel(), mb]) for mw, mb in mags])
    return flat


def loss_and_grad(theta, x, target, C, widths=WIDTHS, bf16=True):
    out, cache = forward(theta, x, widths, bf16)
    loss, gout = mse(out, target, C)
    return loss, backward(theta, cache, gout, widths, bf16), out


def pack_input(fields: np.ndarray, couplings, cin=CIN) -> np.ndarray:
    """NHWC input from SoA fields [N, C, S, S] and per-problem coupling values."""
    N, C, S, _ = fields.shape
    x = np.zeros((N, S, S, cin))
    x[..., :C] = np.transpose(fields, (0, 2, 3, 1))
    if couplings is not None:
        cp = np.asarray(couplings, dtype=np.float64).reshape(N, -1)
        for k in range(cp.shape[1]):
            x[..., C + k] = cp[:, k][:, None, None]
    return x


# ---------------------------------------------------------------- optimiser
def adam_step(theta, m, v, g, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """Update t (counted from 1) of Adam (Kingma & Ba 2015, Algorithm 1), in float64:
    the first and second moment estimates, their bias corrections 1 - beta^t, and the
    parameter step lr * m_hat / (sqrt(v_hat) + eps). Returns new (theta, m, v)."""
    theta, m, v, g = (np.asarray(a, dtype=np.float64) for a in (theta, m, v, g))
    m_new = beta1 * m + (1.0 - beta1) * g
    v_new = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m_new / (1.0 - beta1 ** t)
    v_hat = v_new / (1.0 - beta2 ** t)
    return theta - lr * m_hat / (np.sqrt(v_hat) + eps), m_new, v_new
