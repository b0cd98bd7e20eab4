"""FP64 reference of the learned initial-guess network: a small 3-D U-Net that maps the
Poisson right-hand side and the two previous pressures to a guess for the next pressure.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's method has no learned component; the network is an addition on top of its
Poisson solve (the projection step of Sec. 3 / Sec. 4), built from textbook pieces:
  * 3x3x3 cross-correlation with bias, ReLU (Goodfellow, Bengio & Courville, Deep Learning,
    Ch. 9.1-9.3), padded circularly along periodic axes and with zeros along walled axes;
  * 2x2x2 average pooling with stride 2 and the 2x2x2 stride-2 transposed convolution
    (ibid. Ch. 9.3 and 20.10.6), a 1x1x1 head;
  * the U-Net encoder/decoder with skip concatenation (Ronneberger, Fischer & Brox, 2015);
  * mean-squared-error loss and Adam with bias correction (Kingma & Ba, 2015, Algorithm 1).

Arrays are channel-first ``[C, Z, Y, X]`` with x fastest, the ordering of the grid's cells
(id = i + nx (j + ny k)).  ``bf16=True`` rounds (to nearest even) the operands the GPU
stores in BF16: the network input, every activation entering a convolution, pooling or
the up-sampling, the weights of the 3x3x3 and transposed convolutions, and the activation
gradients entering a backward convolution; sums stay in FP64 here (FP32 on the GPU).

Parity status: the forward and backward passes are pinned by central finite differences,
by adjoint identities, by a delta kernel (identity) and by brute-force loops on tiny grids
(tests/test_oracle_unet.py).  The *trained* network's predictions are a learned heuristic:
parity unpinned; what is pinned is that CG from its guess reaches the same tolerance.
"""
from __future__ import annotations

import dataclasses

import numpy as np

# ----------------------------------------------------------------------------- BF16


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64.

    The value is first rounded to FP32 (as the GPU holds it), then its low 16 bits are
    rounded away: add 0x7FFF plus the lowest kept bit, truncate.
    """
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _r(x, on):
    return bf16(x) if on else x


# ----------------------------------------------------------------------------- shifts

def shift(x: np.ndarray, dz: int, dy: int, dx: int, periodic=(False, True, True)) -> np.ndarray:
    """out[:, z, y, x] = x[:, z + dz, y + dy, x + dx]; wraps along periodic axes (z, y, x order),
    zero where a walled axis leaves the domain."""
    out = x
    for axis, d, per in ((1, dz, periodic[0]), (2, dy, periodic[1]), (3, dx, periodic[2])):
        if d == 0:
            continue
        out = np.roll(out, -d, axis=axis)
        if not per:
            idx = [slice(None)] * 4
            idx[axis] = slice(out.shape[axis] - d, None) if d > 0 else slice(0, -d)
            out = out.copy()
            out[tuple(idx)] = 0.0
    return out


TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


# ----------------------------------------------------------------------------- layers

def conv3_forward(x, W, b, periodic=(False, True, True)):
    """y[o] = b[o] + sum_{c, taps} W[o, c, dz+1, dy+1, dx+1] x[c](z+dz, y+dy, x+dx)."""
    y = np.zeros((W.shape[0],) + x.shape[1:])
    for dz, dy, dx in TAPS:
        y += np.einsum("oc,czyx->ozyx", W[:, :, dz + 1, dy + 1, dx + 1], shift(x, dz, dy, dx, periodic))
    return y + b[:, None, None, None]


def conv3_backward(x, W, gy, periodic=(False, True, True)):
    """Adjoint of conv3_forward: (gx, gW, gb) for the output gradient gy."""
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for dz, dy, dx in TAPS:
        w = W[:, :, dz + 1, dy + 1, dx + 1]
        gx += shift(np.einsum("oc,ozyx->czyx", w, gy), -dz, -dy, -dx, periodic)
        gW[:, :, dz + 1, dy + 1, dx + 1] = np.einsum("ozyx,czyx->oc", gy, shift(x, dz, dy, dx, periodic))
    return gx, gW, gy.sum(axis=(1, 2, 3))


def pool_forward(x):
    """2x2x2 average pooling, stride 2."""
    C, Z, Y, X = x.shape
    return x.reshape(C, Z // 2, 2, Y // 2, 2, X // 2, 2).mean(axis=(2, 4, 6))


def pool_backward(gy):
    return np.repeat(np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up_forward(x, W, b):
    """2x2x2 stride-2 transposed convolution:
    y[o](2z+a, 2y+c, 2x+e) = b[o] + sum_i W[i, o, a, c, e] x[i](z, y, x)."""
    Ci, Z, Y, X = x.shape
    Co = W.shape[1]
    y = np.einsum("ioace,izyx->ozaycxe", W, x)
    return y.reshape(Co, 2 * Z, 2 * Y, 2 * X) + b[:, None, None, None]


def up_backward(x, W, gy):
    Ci, Z, Y, X = x.shape
    Co = W.shape[1]
    g = gy.reshape(Co, Z, 2, Y, 2, X, 2)
    gx = np.einsum("ioace,ozaycxe->izyx", W, g)
    gW = np.einsum("izyx,ozaycxe->ioace", x, g)
    return gx, gW, gy.sum(axis=(1, 2, 3))


def relu(x):
    return np.maximum(x, 0.0)


# ----------------------------------------------------------------------------- network

@dataclasses.dataclass(frozen=True)
class Spec:
    """U-Net with len(channels) levels; level l works on the grid coarsened 2^l times."""

    channels: tuple = (8, 16, 32, 48)
    in_channels: int = 3
    periodic: tuple = (False, True, True)  # (z, y, x): walls in z, periodic in x and y

    @property
    def levels(self) -> int:
        return len(self.channels)


def layers(spec: Spec) -> list:
    """(name, kind, c_in, c_out) in the order of the flat parameter vector."""
    ch = spec.channels
    out = []
    cin = spec.in_channels
    for l, c in enumerate(ch):
        out.append((f"enc{l}a", "conv3", cin, c))
        out.append((f"enc{l}b", "conv3", c, c))
        cin = c
    for l in range(spec.levels - 2, -1, -1):
        out.append((f"up{l}", "up", ch[l + 1], ch[l]))
        out.append((f"dec{l}a", "conv3", 2 * ch[l], ch[l]))
        out.append((f"dec{l}b", "conv3", ch[l], ch[l]))
    out.append(("head", "head", ch[0], 1))
    return out


def param_count(spec: Spec) -> int:
    n = 0
    for _, kind, ci, co in layers(spec):
        n += {"conv3": 27 * ci * co, "up": 8 * ci * co, "head": ci}[kind] + co
    return n


def init_params(spec: Spec, normals: np.ndarray, head_scale: float = 1.0) -> dict:
    """He-scaled weights from given N(0,1) draws (``normals``, one per parameter, in the flat
    order), zero biases; the head's weights are further multiplied by ``head_scale``
    (He, Zhang, Ren & Sun 2015: variance 2 / fan_in)."""
    p = {}
    i = 0
    for name, kind, ci, co in layers(spec):
        if kind == "conv3":
            shape, fan = (co, ci, 3, 3, 3), 27 * ci
        elif kind == "up":
            shape, fan = (ci, co, 2, 2, 2), ci
        else:
            shape, fan = (ci,), ci
        n = int(np.prod(shape))
        scale = np.sqrt(2.0 / fan) * (head_scale if kind == "head" else 1.0)
        # the draws are consumed in the flat layout's order ([co][taps][ci] for conv3,
        # [co][offsets][ci] for the transposed convolution)
        flat = normals[i:i + n]
        if kind == "conv3":
            p[name + ".W"] = np.ascontiguousarray(np.transpose(flat.reshape(co, 3, 3, 3, ci), (0, 4, 1, 2, 3))) * scale
        elif kind == "up":
            p[name + ".W"] = np.ascontiguousarray(np.transpose(flat.reshape(co, 2, 2, 2, ci), (4, 0, 1, 2, 3))) * scale
        else:
            p[name + ".W"] = flat.copy() * scale
        i += n
        p[name + ".b"] = np.zeros(co)
        i += co
    return p


def to_flat(spec: Spec, p: dict) -> np.ndarray:
    """Flat vector in the library's layout: per layer W then b; conv3 W as [co][dz][dy][dx][ci],
    transposed-conv W as [co][a][c][e][ci] (a, c, e the z, y, x offsets), head W as [ci]."""
    parts = []
    for name, kind, ci, co in layers(spec):
        W = p[name + ".W"]
        if kind == "conv3":
            parts.append(np.transpose(W, (0, 2, 3, 4, 1)).ravel())
        elif kind == "up":
            parts.append(np.transpose(W, (1, 2, 3, 4, 0)).ravel())
        else:
            parts.append(W.ravel())
        parts.append(p[name + ".b"].ravel())
    return np.concatenate(parts)


def from_flat(spec: Spec, v: np.ndarray) -> dict:
    p = {}
    i = 0
    for name, kind, ci, co in layers(spec):
        if kind == "conv3":
            n = 27 * ci * co
            p[name + ".W"] = np.transpose(v[i:i + n].reshape(co, 3, 3, 3, ci), (0, 4, 1, 2, 3)).copy()
        elif kind == "up":
            n = 8 * ci * co
            p[name + ".W"] = np.transpose(v[i:i + n].reshape(co, 2, 2, 2, ci), (4, 0, 1, 2, 3)).copy()
        else:
            n = ci
            p[name + ".W"] = v[i:i + n].copy()
        i += n
        p[name + ".b"] = v[i:i + co].copy()
        i += co
    return p


def forward(spec: Spec, p: dict, x0: np.ndarray, bf=False):
    """Network output y[Z, Y, X] for input x0[C_in, Z, Y, X]; returns (y, cache)."""
    per = spec.periodic
    L = spec.levels
    cache = {"x0": _r(x0, bf)}
    x = cache["x0"]
    skips = []
    for l in range(L):
        for s in "ab":
            name = f"enc{l}{s}"
            cache[name + ".in"] = x
            x = _r(relu(conv3_forward(x, _r(p[name + ".W"], bf), p[name + ".b"], per)), bf)
            cache[name + ".out"] = x
        skips.append(x)
        if l < L - 1:
            x = _r(pool_forward(x), bf)
    for l in range(L - 2, -1, -1):
        name = f"up{l}"
        cache[name + ".in"] = x
        u = _r(up_forward(x, _r(p[name + ".W"], bf), p[name + ".b"]), bf)
        x = np.concatenate([u, skips[l]], axis=0)
        for s in "ab":
            name = f"dec{l}{s}"
            cache[name + ".in"] = x
            x = _r(relu(conv3_forward(x, _r(p[name + ".W"], bf), p[name + ".b"], per)), bf)
            cache[name + ".out"] = x
    cache["head.in"] = x
    y = np.einsum("c,czyx->zyx", p["head.W"], x) + p["head.b"][0]
    return y, cache


def backward(spec: Spec, p: dict, cache: dict, gy: np.ndarray, bf=False) -> dict:
    """Gradients of a scalar loss with respect to every parameter, given gy = dloss/dy.

    Walks the forward pass in reverse: the head, the decoder from the finest level to the
    coarsest (each level's up-sampling hands the gradient to the level below), then the
    encoder from the bottom up, where each level adds its skip gradient to the gradient that
    comes back through pooling.  With ``bf`` the stored activation gradients are rounded to
    BF16 where the GPU stores them: every ReLU-masked gradient entering a convolution and
    every gradient a backward convolution or up-sampling writes.
    """
    per = spec.periodic
    L = spec.levels
    g = {}
    g["head.W"] = np.einsum("zyx,czyx->c", gy, cache["head.in"])
    g["head.b"] = np.array([gy.sum()])
    grad = p["head.W"][:, None, None, None] * gy[None]  # gradient of dec0b's output (or of the bottom)
    gskip = [None] * L
    for l in range(L - 1):  # decoder levels, finest first
        for s in "ba":
            name = f"dec{l}{s}"
            gpre = _r(grad * (cache[name + ".out"] > 0), bf)
            grad, g[name + ".W"], g[name + ".b"] = conv3_backward(cache[name + ".in"], _r(p[name + ".W"], bf),
                                                                  gpre, per)
            grad = _r(grad, bf)
        cu = spec.channels[l]
        gskip[l] = grad[cu:]
        name = f"up{l}"
        grad, g[name + ".W"], g[name + ".b"] = up_backward(cache[name + ".in"], _r(p[name + ".W"], bf), grad[:cu])
        grad = _r(grad, bf)  # gradient of the output of level l + 1 (dec{l+1}b, or the bottom encoder)
    for l in range(L - 1, -1, -1):  # encoder levels, bottom first
        if l < L - 1:
            grad = gskip[l] + pool_backward(grad)
        for s in "ba":
            name = f"enc{l}{s}"
            gpre = _r(grad * (cache[name + ".out"] > 0), bf)
            grad, g[name + ".W"], g[name + ".b"] = conv3_backward(cache[name + ".in"], _r(p[name + ".W"], bf),
                                                                  gpre, per)
            grad = _r(grad, bf)
    return g


# ----------------------------------------------------------------------------- guess, loss, Adam

def rms(v: np.ndarray) -> float:
    return float(np.sqrt(np.mean(np.square(v))))


def scales(b: np.ndarray, p1: np.ndarray):
    """Input scales: s_b = rms(b), s_p = rms(p_{t-1}); 1 where a field is zero (the map b -> p is
    linear, so the network sees scale-free inputs)."""
    sb, sp = rms(b), rms(p1)
    return (sb if sb > 0 else 1.0), (sp if sp > 0 else 1.0)


def net_input(b, p1, p2, shape, bf=False):
    """x0 = (b / s_b, p_{t-1} / s_p, p_{t-2} / s_p) on the [Z, Y, X] grid."""
    sb, sp = scales(b, p1)
    x0 = np.stack([b / sb, p1 / sp, p2 / sp]).reshape((3,) + tuple(shape))
    return _r(x0, bf), sb, sp


def predict(spec: Spec, p: dict, b, p1, p2, shape, bf=False) -> np.ndarray:
    """Guess p_hat = p_{t-1} + s_p (y - mean y), then made zero-mean: the network predicts the
    scaled change of the pressure (a zero output returns the previous pressure)."""
    x0, sb, sp = net_input(b, p1, p2, shape, bf)
    y, _ = forward(spec, p, x0, bf)
    y = y.ravel()
    ph = p1 + sp * (y - y.mean())
    return ph - ph.mean()


def loss_and_grad(spec: Spec, p: dict, b, p1, p2, target, shape, bf=False):
    """MSE between the centred output and the centred scaled change (target - p_{t-1}) / s_p,
    and its parameter gradients."""
    x0, sb, sp = net_input(b, p1, p2, shape, bf)
    y, cache = forward(spec, p, x0, bf)
    ys = ((target - p1) / sp).reshape(y.shape)
    d = (y - y.mean()) - (ys - ys.mean())
    n = d.size
    loss = float(np.mean(d * d))
    gy = 2.0 * d / n  # already zero-mean, so the centring passes it through unchanged
    return loss, backward(spec, p, cache, gy, bf)


@dataclasses.dataclass
class Adam:
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8


def adam_step(theta, grad, m, v, t, h: Adam):
    """One Adam update (Kingma & Ba, Algorithm 1) at step t >= 1; returns (theta, m, v)."""
    m = h.beta1 * m + (1.0 - h.beta1) * grad
    v = h.beta2 * v + (1.0 - h.beta2) * grad * grad
    mhat = m / (1.0 - h.beta1**t)
    vhat = v / (1.0 - h.beta2**t)
    return theta - h.lr * mhat / (np.sqrt(vhat) + h.eps), m, v
