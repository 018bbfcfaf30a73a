"""Tensor-core U-Net (the learned warm start) against the FP64 oracle.

The GPU stores inputs, weights, activations and the gradients entering each convolution's backward
in BF16 and accumulates in FP32; the oracle rounds the same values to BF16 (oracle.unet.bf16) and
computes in FP64.  What remains is FP32 accumulation order (and, rarely, a BF16 rounding that an
FP32 intermediate pushes across a tie), so the bounds are relative to the largest magnitude.
"""
import numpy as np
import pytest

from oracle import unet as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2605_28800_b300 import tdgl
    c = tdgl.Context(0)
    yield c
    c.close()


def rel_err(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / max(np.max(np.abs(b)), 1e-30))


CONV_CASES = [
    # (ci, co, k, (nx, ny, nz), batch)
    (8, 16, 3, (8, 4, 3), 2),
    (16, 32, 3, (16, 8, 4), 1),
    (48, 16, 3, (8, 8, 2), 2),
    (192, 64, 3, (8, 4, 4), 1),
    (96, 32, 3, (8, 2, 2), 3),
    (32, 128, 3, (8, 8, 2), 1),
    (16, 8, 1, (24, 5, 3), 2),
    (16, 3, 1, (8, 8, 2), 1),
    (64, 64, 3, (16, 16, 8), 1),     # 2048 voxels: 16 tiles of 128
    # brick path (3x3x3, 16-channel chunks, y a multiple of 16): staged input, taps as offsets
    (16, 16, 3, (8, 16, 3), 2),
    (48, 16, 3, (16, 32, 2), 1),
    (32, 48, 3, (8, 16, 2), 1),      # three output tiles of 16
    (96, 32, 3, (8, 16, 4), 1),
    (192, 64, 3, (8, 16, 2), 1),     # twelve input chunks
    (16, 32, 3, (24, 48, 1), 1),     # one z plane: every tap off the grid in z
]


@pytest.mark.parametrize("ci,co,k,shape,B", CONV_CASES)
def test_conv3d_forward_matches_oracle(ctx, ci, co, k, shape, B):
    from paper_2605_28800_b300 import tdgl
    nx, ny, nz = shape
    g = np.random.default_rng(ci * 1000 + co)
    x = U.bf16(g.normal(size=(B, ci, nz, ny, nx)))
    w = U.bf16(g.normal(scale=(ci * k ** 3) ** -0.5, size=(co, ci, k, k, k)))
    b = g.normal(scale=0.1, size=co).astype(np.float32).astype(np.float64)
    y = tdgl.conv3d(ctx, x, w, b)
    ref = U.conv3d(x, w, b)
    assert rel_err(y, ref) < 1e-5
    yr = tdgl.conv3d(ctx, x, w, b, relu=True)
    assert rel_err(yr, np.maximum(ref, 0)) < 1e-5


@pytest.mark.parametrize("ci,co,k,shape,B", [c for c in CONV_CASES if c[1] % 8 == 0])
def test_conv3d_backward_matches_oracle(ctx, ci, co, k, shape, B):
    from paper_2605_28800_b300 import tdgl
    nx, ny, nz = shape
    g = np.random.default_rng(ci * 7 + co)
    x = U.bf16(g.normal(size=(B, ci, nz, ny, nx)))
    w = U.bf16(g.normal(scale=(ci * k ** 3) ** -0.5, size=(co, ci, k, k, k)))
    dy = U.bf16(g.normal(size=(B, co, nz, ny, nx)))
    dx, dw, db = tdgl.conv3d_backward(ctx, x, w, dy)
    rdx, rdw, rdb = U.conv3d_backward(x, w, dy)
    assert rel_err(dx, rdx) < 1e-5
    assert rel_err(dw, rdw) < 1e-5
    assert rel_err(db, rdb) < 1e-5


def small_net(ctx, seed=3, levels=3, chans=(16, 32, 32), shape=(32, 8, 4), B=2):
    from paper_2605_28800_b300 import tdgl
    net = tdgl.UNet(ctx, shape, cin=4, cout=3, chans=chans, max_batch=B, seed=seed)
    p = U.init(4, 3, chans, seed=seed)
    g = np.random.default_rng(seed)
    for n in p:
        if n.endswith(".b"):
            p[n] = g.normal(scale=0.05, size=p[n].shape)
    v = U.flat(p, levels).astype(np.float32)
    net.set_params(v)
    p = U.unflat(v, 4, 3, chans)        # the float32 values the GPU holds
    nx, ny, nz = shape
    x = g.normal(size=(B, 4, nz, ny, nx)).astype(np.float32)
    t = (0.3 * g.normal(size=(B, 3, nz, ny, nx))).astype(np.float32)
    return net, p, x, t, levels


@pytest.mark.parametrize("shape", [(32, 8, 4), (32, 32, 4)])
def test_unet_forward_matches_oracle(ctx, shape):
    net, p, x, t, levels = small_net(ctx, shape=shape)
    y = net.forward(x)
    ref, _ = U.forward(p, x.astype(np.float64), levels, q=U.bf16)
    assert y.shape == ref.shape
    assert rel_err(y, ref) < 2e-2          # BF16 ties flipped by FP32 sums move single activations
    assert np.sqrt(np.mean((y - ref) ** 2)) / np.sqrt(np.mean(ref ** 2)) < 3e-3


@pytest.mark.parametrize("shape", [(32, 8, 4), (32, 32, 4)])
def test_unet_gradients_match_oracle(ctx, shape):
    net, p, x, t, levels = small_net(ctx, seed=5, shape=shape)
    loss, gv = net.loss_grad(x, t)
    y, cache = U.forward(p, x.astype(np.float64), levels, q=U.bf16)
    rl, dy = U.mse(y, t.astype(np.float64))
    rg = U.flat(U.backward(p, cache, dy, levels), levels)
    assert loss == pytest.approx(rl, rel=5e-3)
    # per layer: direction and size of the gradient
    s = U.shapes(4, 3, (16, 32, 32))
    o = 0
    for name in U.layer_names(levels):
        co, ci, k = s[name]
        for part, size in (("w", co * ci * k ** 3), ("b", co)):
            a, b = gv[o:o + size].astype(np.float64), rg[o:o + size]
            o += size
            cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30)
            assert cos > 0.999, (name, part, cos)
            assert np.linalg.norm(a - b) < 0.03 * np.linalg.norm(b), (name, part)
    assert o == net.param_count()


def test_unet_params_roundtrip_and_init(ctx):
    from paper_2605_28800_b300 import tdgl
    net = tdgl.UNet(ctx, (64, 16, 8), cin=4, cout=3, chans=(16, 32, 64, 128), max_batch=1, seed=11)
    v = net.get_params()
    s = U.shapes(4, 3, (16, 32, 64, 128))
    assert v.size == sum(co * ci * k ** 3 + co for co, ci, k in s.values())
    o = 0
    for name in U.layer_names(4):          # He-normal: sample std close to sqrt(2 / fan_in)
        co, ci, k = s[name]
        w = v[o:o + co * ci * k ** 3]
        o += co * ci * k ** 3
        assert np.all(v[o:o + co] == 0.0)
        o += co
        sd = np.sqrt(2.0 / (ci * k ** 3))
        assert abs(w.std() / sd - 1.0) < (0.35 if w.size < 100 else 0.1), name
    net.set_params(v * 0.5)
    assert np.array_equal(net.get_params(), (v * 0.5).astype(np.float32))


def test_unet_train_step_matches_oracle_adam(ctx):
    net, p, x, t, levels = small_net(ctx, seed=7)
    lr = 1e-3
    l0 = net.train_step(x, t, lr)
    v1 = net.get_params().astype(np.float64)
    v0 = U.flat(p, levels)
    y, cache = U.forward(p, x.astype(np.float64), levels, q=U.bf16)
    rl, dy = U.mse(y, t.astype(np.float64))
    g = U.flat(U.backward(p, cache, dy, levels), levels)
    assert l0 == pytest.approx(rl, rel=5e-3)
    # first Adam step: each parameter moves by lr * g / (|g| + eps), i.e. lr * sign(g) wherever
    # |g| >> eps; compare where the gradient is clearly nonzero
    big = np.abs(g) > 1e-3 * np.max(np.abs(g))
    step = v1 - v0
    assert np.mean(np.sign(step[big]) == -np.sign(g[big])) > 0.995
    assert np.allclose(np.abs(step[big]), lr, rtol=1e-3)


def test_unet_adam_three_steps_match_oracle_adam(ctx):
    # Adam beyond the first step (bias corrections 1 - b^k at k = 2, 3): each GPU train step is
    # compared with the oracle's Adam applied to the GPU's own previous parameters and gradient
    # (the gradient is read with loss_grad first; training is bit-reproducible, so train_step
    # recomputes the same one), with the oracle's moments accumulated in float64
    net, p, x, t, levels = small_net(ctx, seed=23)
    lr = 2e-3
    prev = net.get_params().astype(np.float64)
    om = {"w": np.zeros_like(prev)}
    ov = {"w": np.zeros_like(prev)}
    for k in (1, 2, 3):
        _, g = net.loss_grad(x, t)
        g = g.astype(np.float64)
        net.train_step(x, t, lr)
        got = net.get_params().astype(np.float64)
        want = {"w": prev.copy()}
        U.adam(want, {"w": g}, om, ov, k, lr)
        # float32 moments and update: a relative 1e-6 of a step (|step| is of order lr) plus the
        # rounding of the parameter itself
        assert np.max(np.abs(got - want["w"])) <= 1e-4 * lr + 1e-6 * np.max(np.abs(prev)), k
        assert np.max(np.abs(got - prev)) > 0.5 * lr, k
        prev = got


def test_unet_training_reduces_loss(ctx):
    net, p, x, t, levels = small_net(ctx, seed=9)
    t = (0.2 * np.tanh(x[:, :3])).astype(np.float32)
    losses = [net.train_step(x, t, 3e-3) for _ in range(40)]
    assert losses[-1] < 0.5 * losses[0]


def test_unet_training_is_reproducible(ctx):
    # the gradient reductions add partial sums in a fixed order (no FP32 atomics): the same seed,
    # data and steps give bit-identical losses, gradients and parameters
    runs = []
    for _ in range(2):
        net, p, x, t, levels = small_net(ctx, seed=17, shape=(32, 32, 4))
        losses = [net.train_step(x, t, 2e-3) for _ in range(3)]
        loss, g = net.loss_grad(x, t)
        runs.append((losses + [loss], g, net.get_params()))
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1])
    assert np.array_equal(runs[0][2], runs[1][2])


def test_unet_device_tensors_match_host(ctx):
    import torch
    net, p, x, t, levels = small_net(ctx, seed=13)
    yh = net.forward(x)
    yd = net.forward(torch.from_numpy(x).cuda())
    assert isinstance(yd, torch.Tensor) and yd.is_cuda
    assert np.array_equal(yd.cpu().numpy(), yh)


def test_unet_rejects_bad_shapes(ctx):
    from paper_2605_28800_b300 import tdgl
    with pytest.raises(tdgl.TdglError):
        tdgl.UNet(ctx, (20, 8, 4), cin=4, cout=3, chans=(16, 32, 32))      # nx not a multiple of 32
    with pytest.raises(tdgl.TdglError):
        tdgl.UNet(ctx, (32, 8, 4), cin=4, cout=3, chans=(16, 24, 32))      # channels not multiples of 16
    net = tdgl.UNet(ctx, (32, 8, 4), cin=4, cout=3, chans=(16, 32, 32), max_batch=1)
    with pytest.raises(tdgl.TdglError):
        net.forward(np.zeros((2, 4, 4, 8, 32), np.float32))                # batch above max_batch
