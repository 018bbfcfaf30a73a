"""Pins of the U-Net oracle (oracle/unet.py) against definitions it does not share code with:
brute-force loops, scipy's correlate, adjoint identities, central finite differences and the
closed form of the first Adam step."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import unet as U


def brute_conv(x, w, b):
    B, Ci, Z, Y, X = x.shape
    Co, _, k, _, _ = w.shape
    h = k // 2
    y = np.zeros((B, Co, Z, Y, X))
    for bb in range(B):
        for o in range(Co):
            for z in range(Z):
                for yy in range(Y):
                    for xx in range(X):
                        s = b[o]
                        for i in range(Ci):
                            for a in range(k):
                                for c in range(k):
                                    for e in range(k):
                                        zz, y2, x2 = z + a - h, yy + c - h, xx + e - h
                                        if 0 <= zz < Z and 0 <= y2 < Y and 0 <= x2 < X:
                                            s += w[o, i, a, c, e] * x[bb, i, zz, y2, x2]
                        y[bb, o, z, yy, xx] = s
    return y


@pytest.mark.parametrize("k", [3, 1])
def test_conv3d_matches_brute_force(k):
    g = np.random.default_rng(0)
    x = g.normal(size=(2, 3, 3, 4, 5))
    w = g.normal(size=(2, 3, k, k, k))
    b = g.normal(size=2)
    assert np.allclose(U.conv3d(x, w, b), brute_conv(x, w, b), rtol=0, atol=1e-12)


def test_conv3d_matches_scipy_correlate():
    g = np.random.default_rng(1)
    x = g.normal(size=(1, 2, 6, 5, 7))
    w = g.normal(size=(3, 2, 3, 3, 3))
    b = np.zeros(3)
    ref = np.zeros((1, 3, 6, 5, 7))
    for o in range(3):
        for i in range(2):
            ref[0, o] += ndimage.correlate(x[0, i], w[o, i], mode="constant", cval=0.0)
    assert np.allclose(U.conv3d(x, w, b), ref, rtol=0, atol=1e-12)


def fd_check(f, arr, grad, n=12, h=1e-6, seed=0):
    g = np.random.default_rng(seed)
    flat = arr.reshape(-1)
    for idx in g.choice(flat.size, size=min(n, flat.size), replace=False):
        old = flat[idx]
        flat[idx] = old + h
        fp = f()
        flat[idx] = old - h
        fm = f()
        flat[idx] = old
        num = (fp - fm) / (2 * h)
        assert abs(num - grad.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(num)), (idx, num, grad.reshape(-1)[idx])


@pytest.mark.parametrize("k", [3, 1])
def test_conv3d_backward_matches_finite_differences(k):
    g = np.random.default_rng(2)
    x = g.normal(size=(2, 3, 3, 4, 4))
    w = g.normal(size=(4, 3, k, k, k))
    b = g.normal(size=4)
    r = g.normal(size=(2, 4, 3, 4, 4))          # loss = sum(r * conv(x))
    dx, dw, db = U.conv3d_backward(x, w, r)
    f = lambda: float((r * U.conv3d(x, w, b)).sum())
    fd_check(f, x, dx)
    fd_check(f, w, dw)
    fd_check(f, b, db)


def test_pool_and_up_adjoints():
    g = np.random.default_rng(3)
    x = g.normal(size=(2, 3, 4, 6, 8))
    yp = g.normal(size=(2, 3, 2, 3, 4))
    # <pool x, y> = <x, pool^T y>;  <up y, x> = <y, up^T x>
    assert np.isclose((U.pool(x) * yp).sum(), (x * U.pool_backward(yp)).sum(), rtol=1e-13)
    assert np.isclose((U.up(yp) * x).sum(), (yp * U.up_backward(x)).sum(), rtol=1e-13)
    # values: pooling a constant block returns it, upsampling repeats it
    c = np.full((1, 1, 2, 2, 2), 3.5)
    assert np.allclose(U.pool(c), 3.5) and U.up(U.pool(c)).shape == c.shape
    assert U.pool(np.arange(8.0).reshape(1, 1, 2, 2, 2))[0, 0, 0, 0, 0] == pytest.approx(3.5)


def test_unet_gradients_match_finite_differences():
    levels, chans = 3, (4, 8, 8)
    p = U.init(2, 3, chans, seed=4)
    g = np.random.default_rng(5)
    for n in p:                       # nonzero biases so every ReLU region is exercised
        if n.endswith(".b"):
            p[n] = g.normal(scale=0.1, size=p[n].shape)
    x = g.normal(size=(2, 2, 4, 8, 8))
    t = g.normal(size=(2, 3, 4, 8, 8))
    y, cache = U.forward(p, x, levels)
    assert y.shape == t.shape
    loss, dy = U.mse(y, t)
    grads = U.backward(p, cache, dy, levels)
    assert set(grads) == set(p)
    f = lambda: U.mse(U.forward(p, x, levels)[0], t)[0]
    for n in ["enc0a.w", "enc2b.w", "dec1a.w", "dec0b.b", "head.w", "head.b", "enc1a.b"]:
        fd_check(f, p[n], grads[n], n=6, h=1e-6)


def test_unet_shapes_and_parameter_count():
    s = U.shapes(8, 3, (16, 32, 64, 128))
    n = sum(co * ci * k ** 3 + co for co, ci, k in s.values())
    assert 1.0e6 < n < 2.0e6          # "~1 M parameters, 4 levels, 16-128 channels"
    assert s["dec2a"] == (64, 192, 3) and s["dec0a"] == (16, 48, 3) and s["head"] == (3, 16, 1)
    assert U.layer_names(4)[-1] == "head" and len(U.layer_names(4)) == 15


def test_adam_first_step_closed_form():
    # after one step, m_hat = g and v_hat = g^2, so the update is lr * g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p = {"w": np.zeros(4)}
    m = {"w": np.zeros(4)}
    v = {"w": np.zeros(4)}
    U.adam(p, {"w": g}, m, v, 1, lr=0.01)
    assert np.allclose(p["w"], -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_adam_constant_gradient_moves_lr_every_step():
    # Bias correction makes both moment estimates exact for a stationary gradient (Kingma & Ba,
    # Sec. 3): with g fixed, m_k = (1 - b1^k) g and v_k = (1 - b2^k) g^2, so m_hat = g, v_hat = g^2
    # and every step k moves each parameter by lr * g / (|g| + eps).  A wrong exponent in either
    # correction (k - 1, k + 1, or b^k in place of 1 - b^k) breaks this from step 2 on.
    g = np.array([0.5, -2.0, 1e-3, 3e-6])
    p = {"w": np.zeros(4)}
    m = {"w": np.zeros(4)}
    v = {"w": np.zeros(4)}
    lr = 0.01
    for k in range(1, 8):
        before = p["w"].copy()
        U.adam(p, {"w": g}, m, v, k, lr=lr)
        assert np.allclose(p["w"] - before, -lr * g / (np.abs(g) + 1e-8), rtol=1e-10, atol=0), k


def test_adam_is_invariant_to_gradient_scale_without_eps():
    # with eps = 0 the update m_hat / sqrt(v_hat) is homogeneous of degree 0 in g: scaling every
    # gradient of a changing sequence by c > 0 leaves the trajectory unchanged
    rng = np.random.default_rng(3)
    seq = [rng.normal(size=5) for _ in range(4)]
    traj = []
    for c in (1.0, 37.0):
        p, m, v = {"w": np.ones(5)}, {"w": np.zeros(5)}, {"w": np.zeros(5)}
        for k, g in enumerate(seq, 1):
            U.adam(p, {"w": c * g}, m, v, k, lr=0.05, eps=0.0)
        traj.append(p["w"])
    assert np.allclose(traj[0], traj[1], rtol=1e-12, atol=1e-14)


def test_adam_second_step_sign_reversal_bound():
    # two steps with g1 = +g then g2 = -g: m_2 = (1 - b1) g (b1 - 1), so m_hat_2 = -(1 - b1) g / (1 + b1)
    # (since 1 - b1^2 = (1 - b1)(1 + b1)), and v_hat_2 = g^2 (stationary magnitude): the second step
    # moves by +lr (1 - b1)/(1 + b1) * sign(g), a value fixed by the moment algebra, not by the code
    g = np.array([0.7, -1.3])
    b1 = 0.9
    p, m, v = {"w": np.zeros(2)}, {"w": np.zeros(2)}, {"w": np.zeros(2)}
    U.adam(p, {"w": g}, m, v, 1, lr=0.1, eps=0.0)
    before = p["w"].copy()
    U.adam(p, {"w": -g}, m, v, 2, lr=0.1, eps=0.0)
    assert np.allclose(p["w"] - before, 0.1 * (1 - b1) / (1 + b1) * np.sign(g), rtol=1e-12, atol=0)


def test_training_reduces_loss_on_a_fixed_batch():
    levels, chans = 2, (4, 8)
    p = U.init(2, 3, chans, seed=6)
    m = {n: np.zeros_like(a) for n, a in p.items()}
    v = {n: np.zeros_like(a) for n, a in p.items()}
    g = np.random.default_rng(7)
    x = g.normal(size=(2, 2, 4, 4, 4))
    t = 0.1 * np.tanh(x[:, :1]).repeat(3, axis=1)
    losses = [U.train_step(p, m, v, k, x, t, levels, lr=3e-3) for k in range(1, 31)]
    assert losses[-1] < 0.5 * losses[0]


def test_bf16_rounding_matches_definition():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa wins (1); 1 + 3*2^-9 rounds up
    assert U.bf16(1.0 + 2.0 ** -8) == 1.0
    assert U.bf16(1.0 + 3 * 2.0 ** -9) == 1.0 + 2.0 ** -7
    assert U.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6          # tie between odd 1+2^-7 and even 1+2^-6
    assert U.bf16(-3.0) == -3.0 and U.bf16(0.0) == 0.0
    x = np.random.default_rng(8).normal(size=1000)
    r = U.bf16(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x) * (1 + 1e-12))   # half an ulp: 2^-8 of the binade floor
    assert np.array_equal(U.bf16(r), r)                                  # idempotent


def test_flat_roundtrip_and_order():
    p = U.init(4, 3, (16, 32), seed=9)
    v = U.flat(p, 2)
    q = U.unflat(v, 4, 3, (16, 32))
    assert all(np.array_equal(p[n], q[n]) for n in p)
    assert v[:16 * 4 * 27].reshape(16, 4, 3, 3, 3)[2, 1, 0, 2, 1] == p["enc0a.w"][2, 1, 0, 2, 1]
