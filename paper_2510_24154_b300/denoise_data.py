"""Denoiser data from the Monte Carlo path: training pairs, training loop and
gamma evaluation (the pipeline the paper proposes as future work, Sec. 5).

A case is a thorax phantom whose sizes and positions are jittered by up to
20 % (one phantom per `per_phantom` cases) with one IMRT field of 5-40
segments at a random gantry angle on the 1024 x 768, 0.39 mm EPID.  Its pair
is the sensitive-layer dose image of n_input histories (network input) and of
n_target independent histories (target; history ids from 2^40 on).  Both
images are divided by the input's mean over the image, so the network works
on O(1) values and the scale is known at inference.

With aux planes the network is also given what the noisy image cannot tell
it: the field's source fluence F on the EPID grid (where the MLC and jaw
edges are; the library's mc_get_field_fluence), the radiological thickness t
of the CT along each pixel's ray (the t-map of Sec. 3.1) and their product,
the uncollided primary estimate F exp(-mu t).  F and the primary estimate
are divided by their image means, t by 40 g/cm^2.  All three are computed
on the device.

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
AUX_PLANES = 3            # aperture fluence, t-map, primary estimate
MU_PRIMARY = 0.05         # cm^2/g: water near the 6 MV spectrum's mean energy


FAMILIES = ("thorax", "anthropomorphic")
CONFIG5_CASE = -1         # the anthropomorphic workload itself: phantom seed 4, one 40-segment field


def family_epid(family: str):
    """The EPID grid of a case family."""
    return W.epid_default(1024, 768, 0.039) if family == "thorax" else W.epid_default(1190, 1190, 0.0336)


def case_problem(case: int, seed: int = 3, per_phantom: int = 8, phantom_cache: dict | None = None,
                 family: str = "thorax"):
    """Problem of case `case` of the data set with generator seed `seed`.

    thorax: the 256x256x128 thorax CT at 2 mm with sizes and positions
    jittered by up to 20 %, one IMRT field of 5-40 segments at a random gantry
    angle, EPID 1024 x 768 at 0.39 mm.  anthropomorphic: the 512x512x200 CT at
    1 mm jittered the same way, EPID 1190 x 1190 at 0.336 mm; case
    CONFIG5_CASE is the unjittered phantom with its 40-segment field."""
    if family not in FAMILIES:
        raise ValueError(f"family must be one of {FAMILIES}")
    if family == "anthropomorphic" and case == CONFIG5_CASE:
        prob = W.config_anthropomorphic(n_histories=0, seed=4)
        prob.seed = seed
        return prob
    pid = case // per_phantom
    if phantom_cache is not None and pid in phantom_cache:
        ph = phantom_cache[pid]
    else:
        prng = np.random.default_rng([seed, 7919, pid])
        ph = W.thorax_ct(prng, jitter=0.2) if family == "thorax" else W.anthropomorphic_ct(prng, jitter=0.2)
        if phantom_cache is not None:
            phantom_cache.clear()
            phantom_cache[pid] = ph
    rng = np.random.default_rng([seed, case])
    fld = W.imrt_field(rng, int(rng.integers(5, 41)), float(rng.uniform(0.0, 360.0)))
    return W.Problem(name=f"denoise_{family}_{case}", phantom=ph, epid=family_epid(family), field=fld,
                     lut=W.lut_bilinear(), physics=W.Physics(coupled=True), n_histories=0, seed=seed)


def net_shape(epid, levels=4):
    """Network image size: the EPID grid rounded up to a multiple of
    2^(levels - 1) (the pooling steps); the margin is zero padding."""
    m = 1 << (levels - 1)
    return -(-epid.npy // m) * m, -(-epid.npx // m) * m


def _pad(a, shape):
    """Zero-pads the last two dimensions of a CUDA tensor at the high end."""
    import torch.nn.functional as Fn
    return Fn.pad(a, (0, shape[1] - a.shape[-1], 0, shape[0] - a.shape[-2]))


def aux_planes(F, t):
    """The auxiliary input planes [AUX_PLANES][npy][npx] from the source
    fluence F and the t-map t (g/cm^2), torch tensors [npy][npx] on one
    device: F / mean(F), t / 40 and F exp(-MU_PRIMARY t) / its mean."""
    import torch
    P = F * torch.exp(-MU_PRIMARY * t)
    nz = lambda a: a / torch.clamp(a.mean(), min=1e-300)
    return torch.stack([nz(F), t / 40.0, nz(P)])


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

    def aux(self, prob):
        """Auxiliary planes (float64 CUDA) of the field last set (call after image())."""
        torch = self.torch
        F = torch.empty((prob.epid.npy, prob.epid.npx), dtype=torch.float64, device=f"cuda:{self.device}")
        t = torch.empty_like(F)
        self.sim.fluence_device(F)
        self.sim.tmap_device(t)
        return aux_planes(F, t)

    def close(self):
        self.sim.close()


def input_planes(src: DoseSource, prob, d_in, aux: bool, shape=None):
    """Network input of one case: the normalised noisy image [H][W], with aux
    the planes [1 + AUX_PLANES][H][W] (float32 CUDA, zero-padded to `shape`),
    and the scale s (dose = image / s)."""
    torch = src.torch
    s = 1.0 / max(float(d_in.mean()), 1e-300)
    x = (d_in * s).float()
    if aux:
        x = torch.cat([x[None], src.aux(prob).float()])
    if shape is not None:
        x = _pad(x, shape)
    return x.contiguous(), s


def make_pairs(src: DoseSource, cases, n_input, n_target, seed=3, aux=False, family="thorax"):
    """Stacked float32 CUDA tensors X [len(cases)][H][W] (with aux
    [len(cases)][1 + AUX_PLANES][H][W]) and T [len(cases)][H][W] at the
    network size of the family's EPID (768 x 1024 for the thorax), and the
    per-case scales (dose = image / scale)."""
    torch = src.torch
    xs, ts, scales = [], [], []
    cache = {}
    for c in cases:
        prob = case_problem(c, seed, phantom_cache=cache, family=family)
        shape = net_shape(prob.epid)
        d_in = src.image(prob, n_input, 0, seed)
        x, s = input_planes(src, prob, d_in, aux, shape)
        d_tg = src.image(prob, n_target, TARGET_BASE, seed)
        xs.append(x)
        ts.append(_pad((d_tg * s).float(), shape))
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
            dims = [d for d, f in ((-2, rng.random() < 0.5), (-1, rng.random() < 0.5)) if f]
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


def evaluate(net: UNet, src: DoseSource, cases, n_input, n_ref, seed=3, b=8, pixel_mm=None, dd=0.02,
             dta_mm=2.0, threshold=0.10, ladder=(), aux=False, family="thorax"):
    """Gamma pass rates of raw and denoised n_input-history images against
    n_ref-history references, per case (binned b x b); with a ladder of
    history counts, also the raw images' gamma and RMS error at each count
    (plain Monte Carlo at matched quality)."""
    torch = src.torch
    out = []
    cache = {}
    for c in cases:
        prob = case_problem(c, seed, phantom_cache=cache, family=family)
        pixel_mm = 10.0 * prob.epid.pitch if pixel_mm is None else pixel_mm
        shape = net_shape(prob.epid)
        d_in = src.image(prob, n_input, 0, seed + 1000)
        x, s = input_planes(src, prob, d_in, aux, shape)
        x = x[None].contiguous()
        d_ref = src.image(prob, n_ref, TARGET_BASE, seed + 1000)
        y = torch.empty((1,) + shape, dtype=torch.float32, device=x.device)
        net.forward(x, y, 1.0, 1.0 / s)
        torch.cuda.synchronize()
        ny, nx = d_in.shape
        ref = bin_image(d_ref.cpu().numpy(), b)
        raw = bin_image(d_in.cpu().numpy(), b)
        den = bin_image(y[0, :ny, :nx].double().cpu().numpy(), b)
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
        # the denoised route of this field end to end on the device: field
        # set-up (t-map), n_input histories, dose, fluence, input planes, inference
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d_r = src.image(prob, n_input, 0, seed + 1000)
        x_r, s_r = input_planes(src, prob, d_r, aux, shape)
        net.forward(x_r[None].contiguous(), y, 1.0, 1.0 / s_r)
        torch.cuda.synchronize()
        row["route_s"] = time.perf_counter() - t0
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
