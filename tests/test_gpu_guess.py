"""The learned initial guess on the GPU (tcgen05 convolutions, streaming kernels, Adam) against
the FP64 U-Net oracle with BF16 rounding emulated at the same points."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import unet as U
from oracle import fvm
from tests.conftest import to_dev

pytestmark = pytest.mark.gpu


def _setup(rb, shape_xyz, channels, seed, periodic=(1, 1, 0)):
    nx, ny, nz = shape_xyz
    cfg = rb.guess_cfg(nx, ny, nz, channels, periodic)
    spec = U.Spec(channels=tuple(channels), periodic=(bool(periodic[2]), bool(periodic[1]), bool(periodic[0])))
    n_par = U.param_count(spec)
    assert rb.guess_param_count(cfg) == n_par
    p = U.init_params(spec, W.normal(n_par, seed))
    for k in p:  # non-zero biases so that they are exercised
        if k.endswith(".b"):
            p[k] = 0.05 * W.normal(p[k].shape, seed + 1 + len(k))
    theta = U.to_flat(spec, p).astype(np.float32)
    pref = U.from_flat(spec, theta.astype(np.float64))
    g = rb.Guess(cfg)
    g.set_params(to_dev(theta))
    n = nx * ny * nz
    b, p1, p2 = (W.normal(n, seed + 10 + i) for i in range(3))
    target = p1 + 0.3 * W.normal(n, seed + 20)
    return g, spec, pref, theta, (b, p1, p2, target), (nz, ny, nx)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _layer_out(g, i, level_shape, c):
    a = g.activation(i).cpu().numpy().astype(np.float64)
    return a.reshape(level_shape + (c,)).transpose(3, 0, 1, 2)


# grids of 128-cell rows run the level-0 convolutions on the row kernel (x wrapped or walled);
# levels whose rows are 16 or 32 cells (a multiple of 128 / W rows per plane) run the slab
# kernel: 16x16x8 (level 0, W = 16), 128x16x8 (level 2, W = 32, walled x), 128x64x8 (levels
# 2 and 3, W = 32 and 16, with the level-2 decoder and its input gradient at N = 192; x
# wrapped and walled)
CASES = [((16, 16, 8), (8, 16, 32, 48), (1, 1, 0)), ((10, 6, 6), (8, 16), (1, 1, 0)),
         ((8, 8, 8), (8, 16, 24), (1, 1, 0)), ((128, 4, 4), (8, 16), (1, 1, 0)),
         ((128, 8, 4), (8, 16, 32), (0, 1, 1)), ((128, 40, 16), (8, 16, 32, 48), (1, 1, 0)),
         ((64, 8, 4), (8, 16), (1, 1, 0)), ((128, 16, 8), (8, 16, 32), (0, 1, 1)),
         ((128, 64, 8), (8, 16, 32, 48), (1, 1, 0)), ((128, 64, 8), (8, 16, 32, 48), (0, 1, 1))]
IDS = ["16x16x8-4lvl", "ragged-10x6x6", "8cube-3lvl", "rows128-periodic-x", "rows128-walled-x",
       "rows128-40x16-4lvl", "rows64-level0", "rows128-then-64-walled-x", "slabs32-16-4lvl",
       "slabs32-16-4lvl-walled-x"]


@pytest.mark.parametrize("shape,channels,periodic", CASES, ids=IDS)
def test_forward_matches_oracle(rb, shape, channels, periodic):
    g, spec, pref, _, (b, p1, p2, _), zyx = _setup(rb, shape, channels, 1100, periodic)
    out = g.predict(to_dev(b), to_dev(p1), to_dev(p2)).cpu().numpy()
    x0, sb, sp = U.net_input(b, p1, p2, zyx, bf=True)
    y, cache = U.forward(spec, pref, x0, bf=True)
    L = spec.levels
    # every layer's BF16 output against the emulated oracle (differences: FP32 vs FP64 sums
    # and the occasional BF16 rounding flip they cause)
    names = [n for n, *_ in U.layers(spec)]
    errs = {}
    for i, name in enumerate(names[:-1]):
        kind = U.layers(spec)[i][1]
        lvl = int(name[3]) if name[:3] in ("enc", "dec") else int(name[2])
        ls = tuple(s >> lvl for s in zyx)
        c = U.layers(spec)[i][3]
        got = _layer_out(g, i, ls, c)
        if kind == "up":
            ref = cache[f"dec{lvl}a.in"][:c]
        else:
            ref = cache[name + ".out"]
        errs[name] = _rel(got, ref)
        assert errs[name] < 2e-2, (name, errs[name])
    yg = g.activation(len(names) - 1).cpu().numpy().astype(np.float64)
    errs["head"] = _rel(yg, y.ravel())
    print("relative activation errors:", {k: round(v, 5) for k, v in errs.items()})
    assert errs["head"] < 2e-2
    ref = U.predict(spec, pref, b, p1, p2, zyx, bf=True)
    contribution = ref - (p1 - p1.mean())  # s_p (y - mean y)
    assert np.linalg.norm(out - ref) < 2e-2 * np.linalg.norm(contribution)
    assert abs(out.mean()) < 1e-9 * np.abs(out).max()


@pytest.mark.parametrize("shape,channels,periodic", CASES, ids=IDS)
def test_gradient_matches_oracle(rb, shape, channels, periodic):
    g, spec, pref, _, (b, p1, p2, t), zyx = _setup(rb, shape, channels, 1200, periodic)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.loss_grad(to_dev(b), to_dev(p1), to_dev(p2), to_dev(t), accumulate=False, loss=loss)
    lref, gref = U.loss_and_grad(spec, pref, b, p1, p2, t, zyx, bf=True)
    assert abs(loss.item() - lref) <= 1e-2 * lref
    grad = g.grad().cpu().numpy().astype(np.float64)
    gg = U.from_flat(spec, grad)
    worst = {}
    for name, *_ in U.layers(spec):
        for part in ("W", "b"):
            key = f"{name}.{part}"
            if key == "head.b":  # sum of a zero-mean output gradient: zero up to rounding
                assert abs(gg[key][0]) <= 1e-5 * np.linalg.norm(gref["head.W"])
                continue
            worst[key] = _rel(gg[key], gref[key])
    print("relative gradient errors:", {k: round(v, 5) for k, v in worst.items()})
    assert max(worst.values()) < 5e-2, worst
    # accumulation: a second call with accumulate adds the same gradient again
    g.loss_grad(to_dev(b), to_dev(p1), to_dev(p2), to_dev(t), accumulate=True)
    assert _rel(g.grad().cpu().numpy().astype(np.float64), 2 * grad) < 1e-5


def test_adam_step_matches_oracle(rb):
    g, spec, pref, theta, (b, p1, p2, t), zyx = _setup(rb, (8, 8, 8), (8, 16), 1300)
    g.loss_grad(to_dev(b), to_dev(p1), to_dev(p2), to_dev(t))
    grad = g.grad().cpu().numpy().astype(np.float64)
    g.adam_step(lr=1e-3, grad_scale=0.5)
    new = g.params().cpu().numpy().astype(np.float64)
    ref, _, _ = U.adam_step(theta.astype(np.float64), 0.5 * grad, 0.0, 0.0, 1, U.Adam(lr=1e-3))
    assert np.allclose(new, ref, rtol=1e-6, atol=1e-7)
    assert np.count_nonzero(g.grad().cpu().numpy()) == 0  # the step consumes the gradient


def test_training_reduces_the_loss(rb):
    """A few dozen Adam steps on one pair: the kernels' gradients point downhill."""
    g, spec, pref, _, (b, p1, p2, t), zyx = _setup(rb, (16, 16, 8), (8, 16, 32), 1400)
    bd, p1d, p2d, td = (to_dev(v) for v in (b, p1, p2, t))
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.loss_grad(bd, p1d, p2d, td, loss=loss)
    first = loss.item()
    for _ in range(60):
        loss.zero_()
        g.loss_grad(bd, p1d, p2d, td, loss=loss)
        g.adam_step(lr=3e-3)
    assert loss.item() < 0.5 * first, (first, loss.item())


def test_select_takes_the_better_candidate(rb):
    grid = W.rbc_grid(8, 1.4)
    A = -fvm.laplacian(grid)
    n = A.shape[0]
    x = W.zero_mean(W.normal((n, 1), 1500))[:, 0]
    b = A @ x
    good, bad = x + 1e-6 * W.normal(n, 1501), x + 1e-2 * W.normal(n, 1502)
    g = rb.Guess(rb.guess_cfg(8, 8, 8, (8, 16), (1, 1, 0)))
    op = rb.Operator.from_scipy(A.tocsr())
    x0 = torch.empty(n, dtype=torch.float64, device="cuda")
    for c0, c1, want in ((bad, good, 1), (good, bad, 0)):
        res, choice = g.select(op, to_dev(b), to_dev(c0), to_dev(c1), x0)
        assert choice.item() == want
        ref = [np.linalg.norm(b - A @ c) / np.linalg.norm(b) for c in (c0, c1)]
        assert np.allclose(res.cpu().numpy(), ref, rtol=1e-10)
        assert np.array_equal(x0.cpu().numpy(), (c1 if want else c0))


def test_invalid_configurations(rb):
    lib = rb.lib()
    import ctypes as C
    h = C.c_void_p()
    for cfg in (rb.guess_cfg(8, 8, 8, (8, 16, 32, 48, 64)[:4], (1, 1, 0)),):
        cfg.levels = 5
        assert lib.rb_guess_create(C.byref(cfg), C.byref(h)) == rb.RB_EINVAL
    cfg = rb.guess_cfg(8, 8, 8, (12, 16), (1, 1, 0))
    assert lib.rb_guess_create(C.byref(cfg), C.byref(h)) == rb.RB_EINVAL
    cfg = rb.guess_cfg(10, 8, 8, (8, 16, 32), (1, 1, 0))  # 10 not divisible by 4
    assert lib.rb_guess_create(C.byref(cfg), C.byref(h)) == rb.RB_EINVAL


def test_init_params_matches_oracle(rb):
    spec = U.Spec(channels=(8, 16, 24))
    cfg = rb.guess_cfg(8, 8, 8, (8, 16, 24), (1, 1, 0))
    g = rb.Guess(cfg)
    nrm = W.normal(g.n_params, 1600).astype(np.float32)
    g.init_params(to_dev(nrm), head_scale=0.1)
    ref = U.to_flat(spec, U.init_params(spec, nrm.astype(np.float64), head_scale=0.1))
    got = g.params().cpu().numpy().astype(np.float64)
    assert np.allclose(got, ref, rtol=1e-6, atol=0)


def test_select_smoothing_matches_a_restatement(rb):
    """Damped Jacobi sweeps on both candidates before the judge, against scipy on the host."""
    grid = W.rbc_grid(8, 1.4)
    A = (-fvm.laplacian(grid)).tocsr()
    n = A.shape[0]
    b = W.zero_mean(W.normal((n, 1), 1700))[:, 0]
    c0, c1 = W.normal(n, 1701), W.normal(n, 1702)
    g = rb.Guess(rb.guess_cfg(8, 8, 8, (8, 16), (1, 1, 0)))
    op = rb.Operator.from_scipy(A)
    x0 = torch.empty(n, dtype=torch.float64, device="cuda")
    res, choice = g.select(op, to_dev(b), to_dev(c0), to_dev(c1), x0, sweeps=3, omega=0.7)
    dinv = 1.0 / A.diagonal()
    xs = []
    for c in (c0, c1):
        x = c.copy()
        for _ in range(3):
            x = x + 0.7 * dinv * (b - A @ x)
        xs.append(x)
    ref = [np.linalg.norm(b - A @ x) / np.linalg.norm(b) for x in xs]
    assert np.allclose(res.cpu().numpy(), ref, rtol=1e-9)
    want = int(ref[1] < ref[0])
    assert choice.item() == want
    assert np.allclose(x0.cpu().numpy(), xs[want], rtol=1e-12, atol=1e-12)


def test_full_size_shift_equivariance_and_zero_network(rb):
    """The 128^3 network of the bench (channels 8, 16, 32, 48; periodic x, y, walls in z), in
    the bench's launch configuration, checked through properties that hold at any size: a
    periodic shift of the inputs by 8 cells in x (a multiple of the three poolings) shifts the
    prediction by 8 cells (up to the rounding of the global input and output scalings), and
    the zero network returns the previous pressure."""
    from paper_2508_06710_gb300 import guess_pipeline as gp

    grid = W.rbc_grid(W.GUESS_N, 1.4)
    net = gp.network(grid)
    net.init_params(torch.as_tensor(W.normal(net.n_params, 1800).astype(np.float32), device="cuda"), head_scale=1.0)
    n = net.n
    N = W.GUESS_N
    b, p1, p2 = (torch.as_tensor(W.normal(n, 1801 + i), device="cuda") for i in range(3))
    out = net.predict(b, p1, p2).clone()

    def roll(v):
        return torch.roll(v.view(N, N, N), shifts=8, dims=2).reshape(-1).contiguous()

    out_s = net.predict(roll(b), roll(p1), roll(p2))
    contribution = (out - (p1 - p1.mean())).norm()
    assert float((out_s - roll(out)).norm()) <= 1e-3 * float(contribution)
    assert float(contribution) > 1e-3 * float(p1.norm())  # the network does contribute
    net.set_params(torch.zeros(net.n_params, dtype=torch.float32, device="cuda"))
    out0 = net.predict(b, p1, p2)
    assert torch.allclose(out0, p1 - p1.mean(), rtol=0, atol=1e-12 * float(p1.abs().max()))

