"""Denoiser data from the Monte Carlo path: training pairs, training loop and
gamma evaluation (the pipeline the paper proposes as future work, Sec. 5).

A case is a thorax phantom whose sizes and positions are jittered by up to
20 % (one phantom per `per_phantom` cases) with one IMRT field of 5-40
segments at a random gantry angle on the 1024 x 768, 0.39 mm EPID.  Its pair
is the sensitive-layer dose image of n_input histories (network input) and of
n_target independent histories (target; history ids from 2^40 on).  Both
images are divided by the input's mean over the image, so the network works
on O(1) values and the scale is known at inference.

Evaluation: the denoised low-count image and the raw one are compared with a
high-count reference by the global gamma index (2 %, 2 mm, 10 % threshold) on
the image binned b x b (b = 8 gives 3.1 mm pixels, near the paper's 2.5 mm).
Everything runs on the GPU through the library: transport, dose statistics,
the network and gamma; numpy only bins the three evaluation images.
"""
from __future__ import annotations

import time

import numpy as np

from . import workloads as W
from .binding import Simulator, gamma
from .denoise import UNet

TARGET_BASE = 1 << 40


def case_problem(case: int, seed: int = 3, per_phantom: int = 8, phantom_cache: dict | None = None):
    """Problem of case `case` of the data set with generator seed `seed`."""
    pid = case // per_phantom
    if phantom_cache is not None and pid in phantom_cache:
        ph = phantom_cache[pid]
    else:
        ph = W.thorax_ct(np.random.default_rng([seed, 7919, pid]), jitter=0.2)
        if phantom_cache is not None:
            phantom_cache.clear()
            phantom_cache[pid] = ph
    rng = np.random.default_rng([seed, case])
    fld = W.imrt_field(rng, int(rng.integers(5, 41)), float(rng.uniform(0.0, 360.0)))
    return W.Problem(name=f"denoise_case_{case}", phantom=ph, epid=W.epid_default(1024, 768, 0.039), field=fld,
                     lut=W.lut_bilinear(), physics=W.Physics(coupled=True), n_histories=0, seed=seed)


class DoseSource:
    """Dose images of cases on one Simulator (geometry reloaded per phantom)."""

    def __init__(self, device=0, bank_capacity=1 << 24):
        import torch
        self.torch = torch
        self.sim = Simulator(W.Physics(coupled=True), device=device, bank_capacity=bank_capacity)
        self.device = device
        self._phantom = None
        self.histories = 0
        self.seconds = 0.0

    def image(self, prob, n, hist_base, seed):
        """Per-history dose [768][1024] (float64 CUDA tensor) of n histories."""
        torch = self.torch
        if self._phantom is not prob.phantom:
            self.sim.init_geometry(prob.phantom, prob.epid)
            self._phantom = prob.phantom
        self.sim.set_field(prob.field, prob.lut)
        self.sim.set_history_base(hist_base)
        t0 = time.perf_counter()
        done = 0
        while done < n:                      # at most 2^32 - 1 histories per call
            k = min(n - done, 1 << 31)
            self.sim.run(k, seed)
            done += k
        self.seconds += time.perf_counter() - t0
        self.histories += n
        # dose statistics count histories from 0: rebase so the normalisation is per history
        self.sim.set_history_base(n)
        d = torch.empty((prob.epid.npy, prob.epid.npx), dtype=torch.float64, device=f"cuda:{self.device}")
        self.sim.dose_device(d)
        return d

    def close(self):
        self.sim.close()


def make_pairs(src: DoseSource, cases, n_input, n_target, seed=3):
    """Stacked float32 CUDA tensors X, T [len(cases)][768][1024] and the
    per-case scales (dose = image / scale)."""
    torch = src.torch
    xs, ts, scales = [], [], []
    cache = {}
    for c in cases:
        prob = case_problem(c, seed, phantom_cache=cache)
        d_in = src.image(prob, n_input, 0, seed)
        d_tg = src.image(prob, n_target, TARGET_BASE, seed)
        s = 1.0 / max(float(d_in.mean()), 1e-300)
        xs.append((d_in * s).float())
        ts.append((d_tg * s).float())
        scales.append(s)
    return torch.stack(xs), torch.stack(ts), np.array(scales)


def train(net: UNet, X, T, steps, lr, batch, seed=0, log_every=0, lr_final=None, augment=False):
    """Adam on random mini-batches of the pairs, the learning rate decaying
    from lr to lr_final on a half cosine; returns the loss history.  With
    augment, each mini-batch is mirrored along rows and/or columns at random
    (input and target alike: the noise has no preferred orientation)."""
    import math
    import torch
    lr_final = lr if lr_final is None else lr_final
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    losses = []
    for it in range(steps):
        idx = torch.as_tensor(rng.choice(n, size=batch, replace=n < batch), device=X.device)
        xb = X.index_select(0, idx)
        tb = T.index_select(0, idx)
        if augment:
            dims = [d for d, f in ((1, rng.random() < 0.5), (2, rng.random() < 0.5)) if f]
            if dims:
                xb, tb = torch.flip(xb, dims), torch.flip(tb, dims)
        xb, tb = xb.contiguous(), tb.contiguous()
        want = log_every and (it % log_every == 0 or it == steps - 1)
        lr_t = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * it / max(steps - 1, 1)))
        loss = net.train_step(xb, tb, lr_t, want_loss=bool(want))
        if want:
            losses.append((it, loss))
    return losses


def bin_image(a, b):
    ny, nx = a.shape
    return a[: ny - ny % b, : nx - nx % b].reshape(ny // b, b, nx // b, b).mean(axis=(1, 3))


def evaluate(net: UNet, src: DoseSource, cases, n_input, n_ref, seed=3, b=8, pixel_mm=0.39, dd=0.02,
             dta_mm=2.0, threshold=0.10, ladder=()):
    """Gamma pass rates of raw and denoised n_input-history images against
    n_ref-history references, per case (binned b x b); with a ladder of
    history counts, also the raw images' gamma and RMS error at each count
    (plain Monte Carlo at matched quality)."""
    torch = src.torch
    out = []
    cache = {}
    for c in cases:
        prob = case_problem(c, seed, phantom_cache=cache)
        d_in = src.image(prob, n_input, 0, seed + 1000)
        d_ref = src.image(prob, n_ref, TARGET_BASE, seed + 1000)
        s = 1.0 / max(float(d_in.mean()), 1e-300)
        x = (d_in * s).float()[None]
        y = torch.empty_like(x)
        net.forward(x, y, 1.0, 1.0 / s)
        torch.cuda.synchronize()
        ref = bin_image(d_ref.cpu().numpy(), b)
        raw = bin_image(d_in.cpu().numpy(), b)
        den = bin_image(y[0].double().cpu().numpy(), b)
        dev = f"cuda:{src.device}"
        R = torch.tensor(ref, device=dev)
        g_raw = gamma(R, torch.tensor(raw, device=dev), pixel_mm * b, dd, dta_mm, threshold)
        g_den = gamma(R, torch.tensor(den, device=dev), pixel_mm * b, dd, dta_mm, threshold)
        # the network need not conserve the image's integral, which the raw
        # image estimates without bias: the same output rescaled to it
        den_c = den * (raw.sum() / max(den.sum(), 1e-300))
        g_den_c = gamma(R, torch.tensor(den_c, device=dev), pixel_mm * b, dd, dta_mm, threshold)
        mask = ref >= threshold * ref.max()
        rel = lambda e: float(np.sqrt(np.mean(((e - ref) / ref.max())[mask] ** 2)))
        bias = lambda e: float(e[mask].sum() / ref[mask].sum() - 1.0)
        row = {"case": int(c), "gamma_raw": g_raw, "gamma_denoised": g_den, "rms_raw": rel(raw),
               "rms_denoised": rel(den), "gamma_denoised_rescaled": g_den_c, "rms_denoised_rescaled": rel(den_c),
               "bias_raw": bias(raw), "bias_denoised": bias(den), "ladder": []}
        for n in ladder:
            d_n = bin_image(src.image(prob, int(n), 0, seed + 1000).cpu().numpy(), b)
            row["ladder"].append({"n": float(n), "rms": rel(d_n),
                                  "gamma": gamma(R, torch.tensor(d_n, device=dev), pixel_mm * b, dd, dta_mm,
                                                 threshold)})
        out.append(row)
    return out


def matched_histories(ladder_means, target):
    """Histories at which the mean of a quality measure over the ladder reaches
    `target`, interpolated in log N; None when the ladder never reaches it.
    ladder_means: [(n, value)] with value increasing in n (gamma) -- pass
    negated values for a measure that falls (RMS error)."""
    pts = sorted(ladder_means)
    if pts and pts[0][1] >= target:
        return pts[0][0]
    for (n0, v0), (n1, v1) in zip(pts, pts[1:]):
        if v0 < target <= v1:
            f = (target - v0) / (v1 - v0)
            return float(np.exp(np.log(n0) + f * (np.log(n1) - np.log(n0))))
    return None
