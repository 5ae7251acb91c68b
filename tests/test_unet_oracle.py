"""Pins of the FP64 denoiser oracle (oracle/unet_ref.py) against things other
than itself: brute-force loops, scipy's correlation, central finite
differences, Adam's closed form and torch's bfloat16 conversion."""
import numpy as np
import pytest
from scipy import signal

from oracle import unet_ref as U


def _rng(s=0):
    return np.random.default_rng(s)


def test_bf16_round_matches_torch_and_known_values():
    torch = pytest.importorskip("torch")
    r = _rng(1)
    a = np.concatenate([r.normal(size=20000) * 10.0 ** r.integers(-30, 30, 20000),
                        [0.0, -0.0, 1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, 65504.0, 1e-40]])
    want = torch.tensor(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.bf16_round(a), want)
    assert U.bf16_round(1.0 + 2.0 ** -8) == 1.0                 # tie -> even
    assert U.bf16_round(1.0 + 3 * 2.0 ** -9) == 1.0 + 2.0 ** -7  # above the tie -> up


def test_conv2d_against_loops_and_scipy():
    r = _rng(2)
    N, H, W, Ci, Co = 2, 5, 7, 3, 4
    x = r.normal(size=(N, H, W, Ci))
    for k in (1, 3):
        w = r.normal(size=(Co, k, k, Ci))
        b = r.normal(size=Co)
        y = U.conv2d(x, w, b)
        p = k // 2
        # brute force
        yb = np.zeros((N, H, W, Co))
        for n in range(N):
            for i in range(H):
                for j in range(W):
                    for o in range(Co):
                        s = b[o]
                        for dy in range(k):
                            for dx in range(k):
                                ii, jj = i + dy - p, j + dx - p
                                if 0 <= ii < H and 0 <= jj < W:
                                    s += np.dot(x[n, ii, jj, :], w[o, dy, dx, :])
                        yb[n, i, j, o] = s
        assert np.allclose(y, yb, rtol=1e-12, atol=1e-12)
        # scipy: 'same' correlation per channel pair
        ys = np.zeros_like(yb)
        for n in range(N):
            for o in range(Co):
                acc = np.full((H, W), b[o])
                for c in range(Ci):
                    acc += signal.correlate2d(x[n, :, :, c], w[o, :, :, c], mode="same", boundary="fill")
                ys[n, :, :, o] = acc
        assert np.allclose(y, ys, rtol=1e-12, atol=1e-12)


def _fd_check(f, arrays, grads, n_probe=25, h=1e-6, seed=0, rtol=1e-6):
    r = _rng(seed)
    for a, g in zip(arrays, grads):
        flat = a.reshape(-1)
        gf = g.reshape(-1)
        for idx in r.choice(flat.size, size=min(n_probe, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            fp = f()
            flat[idx] = old - h
            fm = f()
            flat[idx] = old
            num = (fp - fm) / (2 * h)
            assert num == pytest.approx(gf[idx], rel=rtol, abs=1e-8), (idx, num, gf[idx])


def test_conv2d_backward_finite_differences():
    r = _rng(3)
    for k in (1, 3):
        x = r.normal(size=(2, 4, 6, 3))
        w = r.normal(size=(5, k, k, 3))
        b = r.normal(size=5)
        c = r.normal(size=(2, 4, 6, 5))              # L = sum(c * y)
        dx, dw, db = U.conv2d_backward(x, w, c)
        _fd_check(lambda: float(np.sum(c * U.conv2d(x, w, b))), [x, w, b], [dx, dw, db])


def test_pool_upsample_relu_against_loops_and_fd():
    r = _rng(4)
    x = r.normal(size=(1, 4, 6, 2))
    y = U.maxpool2(x)
    for i in range(2):
        for j in range(3):
            for c in range(2):
                assert y[0, i, j, c] == max(x[0, 2 * i + a, 2 * j + b, c] for a in (0, 1) for b in (0, 1))
    c = r.normal(size=y.shape)
    _fd_check(lambda: float(np.sum(c * U.maxpool2(x))), [x], [U.maxpool2_backward(x, c)])
    # ties go to the first maximum in (0,0), (0,1), (1,0), (1,1) order
    t = np.zeros((1, 2, 2, 1))
    t[0, 0, 1, 0] = t[0, 1, 0, 0] = 5.0
    g = U.maxpool2_backward(t, np.ones((1, 1, 1, 1)))
    assert g[0, 0, 1, 0] == 1.0 and g.sum() == 1.0
    u = U.upsample2(y)
    assert u.shape == (1, 4, 6, 2) and u[0, 3, 5, 1] == y[0, 1, 2, 1] and u[0, 2, 4, 0] == y[0, 1, 2, 0]
    cu = r.normal(size=u.shape)
    _fd_check(lambda: float(np.sum(cu * U.upsample2(y))), [y], [U.upsample2_backward(cu)])
    z = r.normal(size=(3, 3))
    assert np.array_equal(U.relu_backward(U.relu(z), np.ones_like(z)), (z > 0).astype(float))


def test_mse_gradient():
    r = _rng(5)
    y, t = r.normal(size=(2, 3, 3, 1)), r.normal(size=(2, 3, 3, 1))
    loss, g = U.mse(y, t)
    assert loss == pytest.approx(np.sum((y - t) ** 2) / y.size, rel=1e-14)
    _fd_check(lambda: U.mse(y, t)[0], [y], [g])


def test_unet_layers_and_gradient_finite_differences():
    spec = U.UNetSpec(levels=3, c0=2, cin=1)
    names = [n for n, *_ in U.layers(spec)]
    assert names == ["enc0a", "enc0b", "enc1a", "enc1b", "enc2a", "enc2b", "dec1a", "dec1b", "dec0a", "dec0b", "out"]
    assert U.layers(spec)[6] == ("dec1a", 4, 3, 8 + 4)
    r = _rng(6)
    flat = r.normal(size=U.param_count(spec)) * 0.4
    flat[-1] = 0.1
    x = np.abs(r.normal(size=(1, 8, 8, 1)))
    t = r.normal(size=(1, 8, 8, 1))
    y, cache = U.forward(spec, flat, x)
    loss, dy = U.mse(y, t)
    g = U.backward(spec, cache, dy)
    assert g.shape == flat.shape

    def f():
        return U.mse(U.forward(spec, flat, x)[0], t)[0]

    _fd_check(f, [flat], [g], n_probe=80, rtol=2e-5)


def test_unet_default_spec_shapes():
    spec = U.UNetSpec()
    L = U.layers(spec)
    assert [c for _, c, _, _ in L[:8]] == [32, 32, 64, 64, 128, 128, 256, 256]
    assert L[8] == ("dec2a", 128, 3, 384) and L[-1] == ("out", 1, 1, 32)
    flat = np.arange(U.param_count(spec), dtype=np.float64)
    assert np.array_equal(U.pack(spec, U.unpack(spec, flat)), flat)


def test_adam_first_step_closed_form():
    r = _rng(7)
    p, g = r.normal(size=100), r.normal(size=100)
    p1, m, v = U.adam_step(p, g, np.zeros(100), np.zeros(100), 1, lr=1e-3)
    # after one step the bias-corrected moments are g and g^2: update = lr g / (|g| + eps)
    assert np.allclose(p1, p - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    p2, _, _ = U.adam_step(p1, g, m, v, 2, lr=1e-3)
    # a constant gradient keeps mhat = g, vhat = g^2
    assert np.allclose(p2, p1 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


def test_training_reduces_loss_on_a_tiny_problem():
    spec = U.UNetSpec(levels=2, c0=4, cin=1)
    r = _rng(8)
    L = U.layers(spec)
    parts = []
    for _, co, k, ci in L:
        parts += [r.normal(size=co * k * k * ci) * np.sqrt(2.0 / (k * k * ci)), np.zeros(co)]
    flat = np.concatenate(parts)
    yy, xx = np.mgrid[0:8, 0:8]
    clean = np.exp(-((yy - 3.5) ** 2 + (xx - 3.5) ** 2) / 8.0)[None, :, :, None]
    noisy = clean + 0.2 * r.normal(size=clean.shape)
    state = (np.zeros_like(flat), np.zeros_like(flat), 0)
    losses = []
    for _ in range(60):
        flat, state, loss, _ = U.train_step(spec, flat, noisy, clean, state, lr=3e-3)
        losses.append(loss)
    assert losses[-1] < 0.3 * losses[0]
