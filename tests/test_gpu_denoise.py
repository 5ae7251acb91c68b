"""GPU parity of the denoiser's tensor-core kernels and of the whole U-Net
against the FP64 oracle (oracle/unet_ref.py) on the same seeded inputs.

Tolerances follow from the arithmetic.  Operands are bfloat16 (exact
products in float32), accumulation is float32 over K terms (error below
K 2^-24 sum|terms|), and a stored result is rounded to bfloat16 (half an
ulp: 2^-9 relative, bounded here by 2^-8).  Hence, per element,
|gpu - ref| <= 2^-8 |ref| + 2e-5 sum|terms|, with sum|terms| the same
convolution taken over absolute values.  Weight gradients are float32 sums
over all pixels (atomics in any order): |gpu - ref| <= 1e-4 sum|terms|.
The whole network is compared with the oracle rounding to bfloat16 at the
same points; accumulation order still flips an occasional rounding, and
such flips propagate through 11-15 layers, so the network-level bounds are
on normalised errors (see each test).
"""
import numpy as np
import pytest

from oracle import unet_ref as U
from paper_2510_24154_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_24154_b300 import denoise as D  # noqa: E402

DEV = "cuda:0"


def _bf(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), dtype=torch.bfloat16, device=DEV)


def _np(t):
    return t.float().cpu().numpy().astype(np.float64)


def _f32(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device=DEV)


def _within(gpu, ref, bound):
    err = np.abs(gpu - ref)
    bad = err > bound
    return int(bad.sum()), float((err / np.maximum(bound, 1e-30)).max())


@pytest.mark.parametrize("case", [
    dict(N=2, H=5, W=130, c0=32, c1=0, co=64, k=3, relu=1),      # two x tiles, ragged tail
    dict(N=1, H=4, W=256, c0=64, c1=32, co=128, k=3, relu=1),    # concatenated input
    dict(N=1, H=3, W=40, c0=8, c1=0, co=32, k=3, relu=0),        # narrow input, W < 128
    dict(N=1, H=2, W=136, c0=32, c1=0, co=1, k=1, relu=0),       # 1x1 to one channel
    dict(N=1, H=2, W=128, c0=128, c1=256, co=320, k=3, relu=1),  # two N tiles, 384 input channels
    dict(N=1, H=3, W=260, c0=64, c1=32, co=32, k=3, relu=1),     # column taps in N, two sources, 3 tiles
    dict(N=2, H=4, W=126, c0=64, c1=0, co=64, k=3, relu=0),      # column taps in N, one exact tile
])
def test_conv_forward_parity(case):
    r = np.random.default_rng(1)
    N, H, Wd, c0, c1, co, k = (case[n] for n in ("N", "H", "W", "c0", "c1", "co", "k"))
    x0 = W.bf16_values(r, (N, H, Wd, c0))
    x1 = W.bf16_values(r, (N, H, Wd, c1)) if c1 else None
    w = (r.normal(size=(co, k, k, c0 + c1)) * np.sqrt(2.0 / (k * k * (c0 + c1)))).astype(np.float32)
    b = (r.normal(size=co) * 0.1).astype(np.float32)
    ys = max(co, 1)
    y = torch.zeros((N, H, Wd, ys), dtype=torch.bfloat16, device=DEV)
    D.conv2d_forward(_bf(x0), _f32(w), _f32(b), k, co, case["relu"], y, x1=_bf(x1) if c1 else None)
    xc = np.concatenate([x0, x1], axis=3) if c1 else x0.astype(np.float64)
    wq = U.bf16_round(w)
    ref = U.conv2d(xc.astype(np.float64), wq, b.astype(np.float64))
    mag = U.conv2d(np.abs(xc).astype(np.float64), np.abs(wq), np.abs(b).astype(np.float64))
    if case["relu"]:
        ref = np.maximum(ref, 0.0)
    bad, worst = _within(_np(y), ref, 2.0 ** -8 * np.abs(ref) + 2e-5 * mag + 1e-30)
    assert bad == 0, (bad, worst)


@pytest.mark.parametrize("case", [
    dict(N=2, H=5, W=130, c0=32, c1=0, co=64, k=3),
    dict(N=1, H=4, W=256, c0=64, c1=32, co=32, k=3),
    dict(N=1, H=3, W=64, c0=32, c1=0, co=1, k=1),
    dict(N=1, H=2, W=128, c0=256, c1=128, co=128, k=3),
    dict(N=1, H=3, W=300, c0=64, c1=0, co=64, k=3),              # column taps in N (N = 64)
])
def test_conv_backward_data_parity(case):
    r = np.random.default_rng(2)
    N, H, Wd, c0, c1, co, k = (case[n] for n in ("N", "H", "W", "c0", "c1", "co", "k"))
    zs = max(8, co)
    dz = np.zeros((N, H, Wd, zs), dtype=np.float32)
    dz[..., :co] = W.bf16_values(r, (N, H, Wd, co))
    w = (r.normal(size=(co, k, k, c0 + c1)) * 0.1).astype(np.float32)
    m0 = W.bf16_values(r, (N, H, Wd, c0))
    m1 = W.bf16_values(r, (N, H, Wd, c1)) if c1 else None
    dx0 = torch.zeros((N, H, Wd, c0), dtype=torch.bfloat16, device=DEV)
    dx1 = torch.zeros((N, H, Wd, c1), dtype=torch.bfloat16, device=DEV) if c1 else None
    D.conv2d_backward_data(_bf(dz), co, _f32(w), k, dx0, mask0=_bf(m0), dx1=dx1, mask1=_bf(m1) if c1 else None)
    wq = U.bf16_round(w)
    xc = np.zeros((N, H, Wd, c0 + c1))
    dx_ref, _, _ = U.conv2d_backward(xc, wq, dz[..., :co].astype(np.float64))
    dx_mag, _, _ = U.conv2d_backward(xc, np.abs(wq), np.abs(dz[..., :co]).astype(np.float64))
    mask = np.concatenate([m0, m1], axis=3) if c1 else m0
    dx_ref = np.where(mask > 0, dx_ref, 0.0)
    got = np.concatenate([_np(dx0), _np(dx1)], axis=3) if c1 else _np(dx0)
    bad, worst = _within(got, dx_ref, 2.0 ** -8 * np.abs(dx_ref) + 2e-5 * dx_mag + 1e-30)
    assert bad == 0, (bad, worst)


@pytest.mark.parametrize("case", [
    dict(N=2, H=5, W=130, c0=32, c1=0, co=64, k=3),
    dict(N=1, H=4, W=256, c0=64, c1=32, co=32, k=3),
    dict(N=1, H=3, W=64, c0=32, c1=0, co=1, k=1),
    dict(N=1, H=6, W=128, c0=128, c1=0, co=256, k=3),
    dict(N=1, H=3, W=136, c0=8, c1=0, co=32, k=3),
    dict(N=2, H=3, W=70, c0=64, c1=0, co=128, k=3),
])
def test_conv_backward_weights_parity(case):
    r = np.random.default_rng(3)
    N, H, Wd, c0, c1, co, k = (case[n] for n in ("N", "H", "W", "c0", "c1", "co", "k"))
    zs = max(8, co)
    dz = np.zeros((N, H, Wd, zs), dtype=np.float32)
    dz[..., :co] = W.bf16_values(r, (N, H, Wd, co))
    x0 = W.bf16_values(r, (N, H, Wd, c0))
    x1 = W.bf16_values(r, (N, H, Wd, c1)) if c1 else None
    dw = torch.zeros((co, k, k, c0 + c1), dtype=torch.float32, device=DEV)
    db = torch.zeros(co, dtype=torch.float32, device=DEV)
    D.conv2d_backward_weights(_bf(dz), co, _bf(x0), k, dw, db=db, x1=_bf(x1) if c1 else None)
    xc = (np.concatenate([x0, x1], axis=3) if c1 else x0).astype(np.float64)
    _, dw_ref, db_ref = U.conv2d_backward(xc, np.zeros((co, k, k, c0 + c1)), dz[..., :co].astype(np.float64))
    _, dw_mag, db_mag = U.conv2d_backward(np.abs(xc), np.zeros((co, k, k, c0 + c1)),
                                          np.abs(dz[..., :co]).astype(np.float64))
    bad, worst = _within(dw.cpu().numpy().astype(np.float64), dw_ref, 1e-4 * dw_mag + 1e-30)
    assert bad == 0, (bad, worst)
    bad, worst = _within(db.cpu().numpy().astype(np.float64), db_ref, 1e-4 * db_mag + 1e-30)
    assert bad == 0, (bad, worst)


def test_pool_and_upsample_parity():
    r = np.random.default_rng(4)
    x = W.bf16_values(r, (2, 6, 10, 32))
    x[0, 0, 0, :] = x[0, 0, 1, :]                         # ties: first maximum wins
    y = torch.zeros((2, 3, 5, 32), dtype=torch.bfloat16, device=DEV)
    D.maxpool2(_bf(x), y)
    assert np.array_equal(_np(y), U.maxpool2(x.astype(np.float64)))
    dy = W.bf16_values(r, (2, 3, 5, 32))
    add = W.bf16_values(r, (2, 6, 10, 32))
    dx = torch.zeros((2, 6, 10, 32), dtype=torch.bfloat16, device=DEV)
    D.maxpool2_backward(_bf(x), _bf(dy), dx, add=_bf(add))
    ref = U.bf16_round(U.maxpool2_backward(x.astype(np.float64), dy.astype(np.float64)) + add)
    assert np.array_equal(_np(dx), ref)
    u = torch.zeros((2, 6, 10, 32), dtype=torch.bfloat16, device=DEV)
    D.upsample2(_bf(dy), u)
    assert np.array_equal(_np(u), U.upsample2(dy.astype(np.float64)))
    du = torch.zeros((2, 3, 5, 32), dtype=torch.bfloat16, device=DEV)
    D.upsample2_backward(_bf(add), du)
    ref = U.upsample2_backward(add.astype(np.float64))
    assert np.allclose(_np(du), ref, rtol=2.0 ** -8, atol=0)


def _small_net(levels=3, H=32, Wd=256, batch=2, seed=5, cin=1):
    """A seeded network and batch.  With cin > 1 the input is planar
    [batch][cin][H][W]: the noisy image, a smooth map and a binary mask,
    the kinds of auxiliary planes the denoiser is given."""
    spec = U.UNetSpec(levels=levels, c0=32, cin=cin)
    params = W.unet_params(U.layers(spec), seed=seed)
    net = D.UNet(height=H, width=Wd, batch=batch, levels=levels, base_channels=32, seed=seed, in_channels=cin)
    net.set_params(params)
    r = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:Wd]
    clean = np.exp(-((yy - H / 2) ** 2 / (H * H / 8) + (xx - Wd / 2) ** 2 / (Wd * Wd / 8)))
    x = np.stack([U.bf16_round(np.abs(clean + 0.3 * r.normal(size=clean.shape))) for _ in range(batch)])
    if cin > 1:
        aux = [clean * (1 + 0.5 * np.sin(xx / 7.0)), ((np.abs(yy - H / 2) < H / 4) & (np.abs(xx - Wd / 2) < Wd / 3))]
        planes = [x] + [np.broadcast_to(U.bf16_round(a.astype(np.float64)), x.shape) for a in aux]
        planes += [U.bf16_round(r.uniform(-1, 1, size=x.shape)) for _ in range(cin - len(planes))]
        x = np.stack(planes[:cin], axis=1)
    t = U.bf16_round(np.stack([clean] * batch))
    return spec, params, net, x.astype(np.float32), t.astype(np.float32)


def _nhwc(x):
    return x[..., None] if x.ndim == 3 else np.moveaxis(x, 1, 3)


@pytest.mark.parametrize("levels,H,Wd,cin", [(3, 32, 256, 1), (4, 128, 256, 1), (3, 32, 256, 3), (4, 64, 128, 8)])
def test_unet_forward_and_gradient_parity(levels, H, Wd, cin):
    spec, params, net, x, t = _small_net(levels=levels, H=H, Wd=Wd, cin=cin)
    assert net.n_params == U.param_count(spec)
    xd, td = _f32(x), _f32(t)
    loss = net.train_step(xd, td, lr=0.0)
    out = torch.zeros_like(td)
    net.output(out)
    g = net.grads()
    y_ref, cache = U.forward(spec, params.astype(np.float64), _nhwc(x), emulate_bf16=True)
    loss_ref, dy = U.mse(y_ref, t[..., None])
    g_ref = U.backward(spec, cache, dy, emulate_bf16=True)
    # output: every element within 2 % of the output's range
    yo = out.cpu().numpy()[..., None].astype(np.float64)
    scale = np.abs(y_ref).max()
    assert np.abs(yo - y_ref).max() <= 0.02 * scale
    assert loss == pytest.approx(loss_ref, rel=0.02)
    # gradients, per layer: relative L2 error <= 5 % and cosine >= 0.998
    o = 0
    for name, co, k, ci in U.layers(spec):
        n = co * k * k * ci + co
        a, b = g[o:o + n].astype(np.float64), g_ref[o:o + n]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        cos = float(a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))
        assert rel <= 0.05 and cos >= 0.998, (name, rel, cos)
        o += n
    net.close()


def test_unet_in_scale_multiplies_only_the_image_plane():
    """in_scale applies to plane 0; auxiliary planes are taken as given."""
    spec, params, net, x, t = _small_net(cin=3, seed=9)
    out_a, out_b = torch.zeros_like(_f32(t)), torch.zeros_like(_f32(t))
    net.forward(_f32(x), out_a, in_scale=1.0)
    x2 = x.copy()
    x2[:, 0] *= 0.25
    net.forward(_f32(x2), out_b, in_scale=4.0)
    torch.cuda.synchronize()
    assert torch.equal(out_a, out_b)
    net.close()


def test_unet_adam_step_closed_form():
    spec, params, net, x, t = _small_net(seed=6)
    lr = 1e-3
    net.train_step(_f32(x), _f32(t), lr=lr)
    g = net.grads().astype(np.float64)
    p1 = net.params().astype(np.float64)
    # first Adam step: bias-corrected moments equal g and g^2
    want = params.astype(np.float64) - lr * g / (np.abs(g) + 1e-8)
    assert np.allclose(p1, want, rtol=0, atol=2e-6 + 1e-6 * np.abs(want).max())
    net.close()


def test_unet_training_reduces_loss():
    spec, params, net, x, t = _small_net(seed=7)
    xd, td = _f32(x), _f32(t)
    losses = [net.train_step(xd, td, lr=2e-3) for _ in range(150)]
    assert np.isfinite(losses).all()
    assert np.mean(losses[-10:]) < 0.2 * losses[0], (losses[0], losses[-10:])
    net.close()


def test_unet_full_size_forward_runs():
    """The 768 x 1024, 4-level, 32-256 channel network: one forward pass
    on a seeded image gives a finite output, and a training step a finite loss."""
    net = D.UNet(height=768, width=1024, batch=1, levels=4, base_channels=32, seed=3)
    r = np.random.default_rng(8)
    x = _f32(np.abs(r.normal(size=(1, 768, 1024))))
    out = torch.zeros_like(x)
    net.forward(x, out)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    loss = net.train_step(x, x, lr=1e-4)
    assert np.isfinite(loss)
    net.close()


def test_gamma_kernel_matches_oracle():
    """mc_gamma (GPU, FP64) against the oracle's gamma on the same images."""
    import oracle
    from paper_2510_24154_b300.binding import gamma
    r = np.random.default_rng(9)
    yy, xx = np.mgrid[0:60, 0:80]
    ref = np.exp(-((yy - 30) ** 2 + (xx - 40) ** 2) / 300.0) + 0.05
    for sig, shift in ((0.01, 0.0), (0.03, 0.7), (0.0, 1.6)):
        ev = np.exp(-((yy - 30 - shift) ** 2 + (xx - 40) ** 2) / 300.0) + 0.05 + sig * r.normal(size=ref.shape)
        for dd, dta, pix in ((0.02, 2.0, 2.5), (0.01, 1.0, 0.39 * 8)):
            rate_o, g_o = oracle.gamma(ref, ev, pix, dd=dd, dta_mm=dta, threshold=0.10)
            out = torch.empty((60, 80), dtype=torch.float64, device=DEV)
            rate_g = gamma(torch.tensor(ref, device=DEV), torch.tensor(ev, device=DEV), pix, dd, dta, 0.10, out=out)
            g_g = out.cpu().numpy()
            assert np.array_equal(np.isnan(g_g), np.isnan(g_o))
            ok = ~np.isnan(g_o)
            assert np.allclose(g_g[ok], g_o[ok], rtol=1e-9, atol=1e-12)
            near = np.abs(g_o[ok] - 1.0) < 1e-9          # decisions only differ within rounding of 1
            assert abs(rate_g - rate_o) <= near.sum() / ok.sum() + 1e-15


def test_denoiser_pipeline_on_mc_pairs_small():
    """Pairs from the transport, a few training steps, gamma evaluation: the
    pipeline runs end to end and the training loss falls."""
    from paper_2510_24154_b300.denoise_data import DoseSource, evaluate, make_pairs, train
    src = DoseSource()
    X, T, s = make_pairs(src, range(4), 100_000, 10_000_000, seed=3)
    assert X.shape == (4, 768, 1024) and torch.isfinite(X).all() and torch.isfinite(T).all()
    assert abs(float(X.mean()) - 1.0) < 1e-3
    net = D.UNet(768, 1024, batch=2, levels=4, base_channels=32, seed=3)
    losses = train(net, X, T, 60, 1e-3, 2, log_every=10)
    assert losses[-1][1] < losses[0][1]
    ev = D.UNet(768, 1024, batch=1, levels=4, base_channels=32)
    ev.set_params(net.params())
    res = evaluate(ev, src, [1000], 100_000, 30_000_000, seed=3)
    assert 0.0 <= res[0]["gamma_raw"] <= 1.0 and 0.0 <= res[0]["gamma_denoised"] <= 1.0
    net.close(); ev.close(); src.close()


def test_denoise_experiment_beats_raw_on_held_out_cases():
    """The evaluation driver on a small case (32 training pairs of 1e6 / 1e9
    histories, 1500 steps, the aperture, t-map and primary planes as extra
    input; 2 held-out cases against 1e9-history references): on the held-out
    cases the denoised image passes the 2 %/2 mm gamma more often than the raw
    input and has a smaller RMS error, and it matches plain Monte Carlo of
    more histories than its input.  Measured: gamma 0.70 raw, 0.82 denoised;
    RMS error 0.57 raw, 0.037 denoised (plain 1e8 histories: 0.058)."""
    import json
    import subprocess
    import sys
    cmd = [sys.executable, "-m", "paper_2510_24154_b300.denoise_experiment", "--pairs", "32", "--n-input", "1e6",
           "--n-target", "1e9", "--eval", "2", "--n-ref", "1e9", "--steps", "1500", "--aux", "--ladder",
           "1e6,1e7,1e8"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, check=True).stdout
    r = json.loads(out.strip().splitlines()[-1])
    assert r["in_channels"] == 4 and r["eval_cases"] == 2
    assert r["gamma_denoised_mean"] > r["gamma_raw_mean"] + 0.05, (r["gamma_raw_mean"], r["gamma_denoised_mean"])
    assert r["rms_denoised_mean"] < r["rms_raw_mean"], (r["rms_raw_mean"], r["rms_denoised_mean"])
    n_rms = r["matched"]["plain_histories_at_denoised_rms"]
    assert n_rms is None or n_rms > 3e7
