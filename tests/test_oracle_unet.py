"""Pins of the FP64 U-Net oracle (learned initial guess): brute-force loops, adjoint identities,
a delta kernel, central finite differences, the first Adam step in closed form and BF16
rounding against torch's own cast."""
import numpy as np
import pytest
import torch

from oracle import unet as U

PER = (False, True, True)


def _loops_conv3(x, W, b):
    """Brute-force 3x3x3 correlation: zero outside z, wrap in y and x."""
    C, Z, Y, X = x.shape
    O = W.shape[0]
    y = np.zeros((O, Z, Y, X))
    for o in range(O):
        for z in range(Z):
            for yy in range(Y):
                for xx in range(X):
                    s = b[o]
                    for c in range(C):
                        for a in range(3):
                            zz = z + a - 1
                            if zz < 0 or zz >= Z:
                                continue
                            for d in range(3):
                                for e in range(3):
                                    s += W[o, c, a, d, e] * x[c, zz, (yy + d - 1) % Y, (xx + e - 1) % X]
                    y[o, z, yy, xx] = s
    return y


def test_conv3_matches_loops():
    g = np.random.default_rng(1)
    x = g.standard_normal((2, 3, 4, 5))
    W = g.standard_normal((3, 2, 3, 3, 3))
    b = g.standard_normal(3)
    assert np.allclose(U.conv3_forward(x, W, b, PER), _loops_conv3(x, W, b), rtol=0, atol=1e-12)


def test_conv3_delta_kernel_is_identity_and_commutes_with_periodic_shifts():
    g = np.random.default_rng(2)
    x = g.standard_normal((4, 4, 6, 8))
    W = np.zeros((4, 4, 3, 3, 3))
    for c in range(4):
        W[c, c, 1, 1, 1] = 1.0
    assert np.array_equal(U.conv3_forward(x, W, np.zeros(4), PER), x)
    W = g.standard_normal((3, 4, 3, 3, 3))
    y = U.conv3_forward(x, W, np.zeros(3), PER)
    ys = U.conv3_forward(np.roll(x, (2, 3), axis=(2, 3)), W, np.zeros(3), PER)
    assert np.allclose(np.roll(y, (2, 3), axis=(2, 3)), ys, atol=1e-12)


def test_conv3_backward_is_the_adjoint():
    g = np.random.default_rng(3)
    x = g.standard_normal((3, 4, 5, 6))
    W = g.standard_normal((2, 3, 3, 3, 3))
    gy = g.standard_normal((2, 4, 5, 6))
    y0 = U.conv3_forward(x, W, np.zeros(2), PER)
    gx, gW, gb = U.conv3_backward(x, W, gy, PER)
    assert abs(np.vdot(y0, gy) - np.vdot(x, gx)) < 1e-10 * abs(np.vdot(y0, gy))
    assert abs(np.vdot(y0, gy) - np.vdot(W, gW)) < 1e-10 * abs(np.vdot(y0, gy))  # y is linear in W too
    assert np.allclose(gb, gy.sum(axis=(1, 2, 3)))


def test_pool_and_up_against_loops_and_adjoints():
    g = np.random.default_rng(4)
    x = g.standard_normal((2, 4, 6, 8))
    p = U.pool_forward(x)
    assert np.isclose(p[1, 1, 2, 3], x[1, 2:4, 4:6, 6:8].mean())
    gy = g.standard_normal(p.shape)
    assert np.isclose(np.vdot(p, gy), np.vdot(x, U.pool_backward(gy)))
    xc = g.standard_normal((3, 2, 3, 4))
    W = g.standard_normal((3, 2, 2, 2, 2))
    b = g.standard_normal(2)
    y = U.up_forward(xc, W, b)
    for (o, z, yy, xx) in [(0, 0, 0, 0), (1, 3, 5, 7), (0, 2, 1, 6), (1, 1, 4, 3)]:
        ref = b[o] + sum(W[i, o, z % 2, yy % 2, xx % 2] * xc[i, z // 2, yy // 2, xx // 2] for i in range(3))
        assert np.isclose(y[o, z, yy, xx], ref)
    gy = g.standard_normal(y.shape)
    gx, gW, gb = U.up_backward(xc, W, gy)
    y0 = U.up_forward(xc, W, np.zeros(2))
    assert np.isclose(np.vdot(y0, gy), np.vdot(xc, gx))
    assert np.isclose(np.vdot(y0, gy), np.vdot(W, gW))


def test_param_count_and_flat_layout():
    # (8,16,32,48): encoder 3->8, 8->8, 8->16, 16->16, 16->32, 32->32, 32->48, 48->48;
    # decoder up 48->32, 64->32, 32->32, up 32->16, 32->16, 16->16, up 16->8, 16->8, 8->8; head 8->1
    conv = [(3, 8), (8, 8), (8, 16), (16, 16), (16, 32), (32, 32), (32, 48), (48, 48), (64, 32), (32, 32),
            (32, 16), (16, 16), (16, 8), (8, 8)]
    ups = [(48, 32), (32, 16), (16, 8)]
    n = sum(27 * a * b + b for a, b in conv) + sum(8 * a * b + b for a, b in ups) + 8 + 1
    assert n == U.param_count(U.Spec()) == 284_553
    spec = U.Spec(channels=(4, 8))
    v = np.arange(U.param_count(spec), dtype=np.float64)
    p = U.from_flat(spec, v)
    assert np.array_equal(U.to_flat(spec, p), v)
    # conv3 weights are stored [co][dz][dy][dx][ci]: element (co=1, ci=2, dz=0, dy=2, dx=1) of enc0a
    assert p["enc0a.W"][1, 2, 0, 2, 1] == ((1 * 27 + (0 * 9 + 2 * 3 + 1)) * 3 + 2)


def _tiny(spec, seed, shape=(4, 4, 4)):
    g = np.random.default_rng(seed)
    p = U.init_params(spec, g.standard_normal(U.param_count(spec)))
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.1 * g.standard_normal(p[k].shape)
    n = int(np.prod(shape))
    b = g.standard_normal(n)
    p1 = g.standard_normal(n)
    p2 = g.standard_normal(n)
    t = p1 + 0.3 * g.standard_normal(n)
    return p, b, p1, p2, t


@pytest.mark.parametrize("channels,shape", [((4, 8), (4, 4, 4)), ((2, 4, 6), (4, 8, 8))])
def test_network_gradient_matches_central_differences(channels, shape):
    spec = U.Spec(channels=channels)
    p, b, p1, p2, t = _tiny(spec, 7 + len(channels), shape)
    loss, grads = U.loss_and_grad(spec, p, b, p1, p2, t, shape)
    g = np.random.default_rng(11)
    h = 1e-6
    checked = 0
    for name in p:
        flat = p[name].reshape(-1)
        for idx in g.choice(flat.size, size=min(3, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = U.loss_and_grad(spec, p, b, p1, p2, t, shape)
            flat[idx] = old - h
            lm, _ = U.loss_and_grad(spec, p, b, p1, p2, t, shape)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = grads[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(an)) + 1e-9, (name, idx, fd, an)
            checked += 1
    assert checked > 20


def test_zero_network_returns_the_previous_pressure():
    spec = U.Spec(channels=(4, 8))
    p = U.init_params(spec, np.zeros(U.param_count(spec)))
    g = np.random.default_rng(5)
    b, p1, p2 = (g.standard_normal(64) for _ in range(3))
    ph = U.predict(spec, p, b, p1, p2, (4, 4, 4))
    assert np.allclose(ph, p1 - p1.mean(), atol=1e-14)


def test_adam_first_step_closed_form():
    h = U.Adam(lr=1e-3)
    g = np.array([0.5, -2.0, 1e-3, -7.0])
    th, m, v = U.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, h)
    # bias correction gives m_hat = g, v_hat = g^2 at t = 1: a step of lr * g / (|g| + eps)
    assert np.allclose(th, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding_matches_torch_cast():
    g = np.random.default_rng(6)
    x = np.concatenate([g.standard_normal(4000) * 10.0 ** g.integers(-6, 6, 4000),
                        [1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-8, -1.0 - 2**-8, 0.0, 65504.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.bf16(x), ref)
    assert U.bf16(np.array([1.0 + 2**-8]))[0] == 1.0  # a tie goes to the even neighbour
