#!/usr/bin/env python
"""Throughput of the EPID transit Monte Carlo hot path on one or more B300s.

One step = the whole path over one field of the coupled thorax workload
(256x256x128 HU CT at 2 mm, one 9-segment IMRT field, EPID 1024x768 at
0.39 mm, 64x32 k-table): HU -> density, field set-up (source table,
radiological thickness map, Eq. 1), transport of the histories, dose
statistics and the k(t, s) corrected image.  Inputs are resident in HBM when
the timed region starts; the `e2e` leg repeats the step through the C-ABI
with host buffers (HU volume in, corrected image out) inside the timed region.

`--impl reference` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the only other place this script runs it is the
`cpu_baseline` leg).  Multi-GPU runs shard history ids across ranks (weak
scaling, no data-path collective); the timing takes the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HIST_PER_STEP = 100_000_000
SEED = 1
WORKLOAD = "thorax_imrt_9seg: CT 256x256x128 int16 HU @2mm, 9 MLC segments x 60 pairs, " \
           "EPID 1024x768 @0.39mm (Cu/Gd2O2S/a-Si), k-table 64x32, coupled photon/electron"
# Per CT electron step, counted by ncu over the CT-electron launch of the
# timed step of the 2e6-history thorax case (one wave, 36.2 M steps;
# profiles/electron_ct_small_case.md): executed thread instructions, executed
# warp instructions, single-precision operations (FADD + FMUL + 2 FFMA; no
# packed forms issued) and DRAM bytes read + written.
INST_PER_ESTEP_CT = 532.4
WARP_INST_PER_ESTEP_CT = 28.90
FLOPS_PER_ESTEP_CT = 155.7
DRAM_BYTES_PER_ESTEP_CT = 3.09
# The same launch under ncu --set full (profiles/electron_ct_small_case.md):
# fraction of scheduler cycles that issued a warp instruction, and the
# fraction of the SM's 64 warp slots occupied (at most 0.5 here: 4 CTAs of
# 256 threads, register-limited).
NCU_ISSUE_ACTIVE_ECT = 0.652
NCU_WARPS_ACTIVE_ECT = 0.456
# instruction issue: 148 SMs x 4 schedulers x 32 lanes x 2.032 GHz
ISSUE_PEAK_TINST = 148 * 4 * 32 * 2.032e9 / 1e12
# run-control block read back after every wave of a host-driven run
CTL_BYTES = 104
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12   # 148 SMs x 128 FP32 lanes x FMA x 2.032 GHz


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--histories", type=int, default=HIST_PER_STEP)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--bank-capacity", type=int, default=1 << 26,
                    help="particles per bank (0: library default); 2^26 = 25.8 GB of banks, 9 waves per step")
    ap.add_argument("--regs-variant", default="", help="CTAs/SM build per transport kernel, e.g. 3,3,3,3")
    ap.add_argument("--primaries-per-wave", type=int, default=0, help="new histories per wave (0: a quarter bank)")
    ap.add_argument("--no-batched", action="store_true", help="skip the 25-field batched-plan leg")
    ap.add_argument("--batched-scale", type=float, default=1.0, help="scale of the batched plan's history counts")
    ap.add_argument("--no-denoiser", action="store_true", help="skip the U-Net denoiser leg")
    ap.add_argument("--no-anthro", action="store_true", help="skip the anthropomorphic-phantom leg")
    ap.add_argument("--no-one-pct", action="store_true", help="skip the measured time-to-1 % leg")
    ap.add_argument("--anthro-histories", type=int, default=1_000_000_000)
    ap.add_argument("--dn-batch", type=int, default=4, help="images per denoiser training step")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for n, v in zip(names, r[4:8]):
                    if v.lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_model():
    """The host CPU's model name (first processor in /proc/cpuinfo), or None."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_sample(problem, n, threads):
    import oracle
    t0 = time.perf_counter()
    r = oracle.run(problem, n_histories=n, threads=threads)
    dt = time.perf_counter() - t0
    return n / dt, r["threads"], dt


def run_reference(args):
    """The FP64 oracle on the host cores, same workload, bounded samples."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2510_24154_b300 import workloads as W
    oracle.build()
    p = W.config_thorax_imrt(n_histories=args.histories, seed=SEED)
    threads = os.cpu_count() or 1
    sample = 2_000_000                 # about 3 s per step on 16 threads
    for _ in range(args.warmup):
        oracle.run(p, n_histories=200_000, threads=threads)
    t0 = time.perf_counter()
    done = 0
    for k in range(args.steps):
        oracle.run(p, n_histories=sample, hist_begin=k * sample, threads=threads)
        done += sample
    dt = time.perf_counter() - t0
    v = done / dt
    line = {
        "impl": "reference", "metric": "histories/s", "value": v, "unit": "histories/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "histories_per_step": sample, "seed": SEED},
        "cpu_baseline": {"value": v, "unit": "histories/s", "cores": min(threads, p.physics.n_batches),
                         "kind": "oracle", "sample": f"{sample} histories of the workload per step",
                         "host": {"cpu_model": cpu_model(), "logical_cpus": threads}},
        "e2e": {"value": v, "unit": "histories/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def unet_flops(H=768, W=1024, levels=4, c0=32):
    """Algorithmic FLOPs of one image: forward, and forward + input gradients
    + weight gradients (a training step), from the layer shapes (2 per MAC)."""
    layers = []
    ci = 1
    for l in range(levels):
        c = c0 << l
        layers += [(l, c, 3, ci, l > 0), (l, c, 3, c, True)]
        ci = c
    for l in range(levels - 2, -1, -1):
        c = c0 << l
        layers += [(l, c, 3, (c0 << (l + 1)) + c, True), (l, c, 3, c, True)]
    layers.append((0, 1, 1, c0, True))
    fwd = dgrad = 0.0
    for l, co, k, ci, has_dgrad in layers:
        f = 2.0 * (H >> l) * (W >> l) * co * k * k * ci
        fwd += f
        dgrad += f if has_dgrad else 0.0
    return fwd, 2.0 * fwd + dgrad


def denoised_route_leg(sim, p, stream, local, n_input=10_000_000, reps=5):
    """One field by the denoised route, end to end on the device and timed on
    the host clock with the device synchronized on both sides: field set-up
    (t-map, Eq. 1), n_input histories, dose, source fluence, the four input
    planes and one inference of the 768 x 1024 network (4 input planes;
    random weights: the time does not depend on them).  Median of reps."""
    import numpy as np
    import torch
    from paper_2510_24154_b300.denoise import UNet
    from paper_2510_24154_b300.denoise_data import AUX_PLANES, aux_planes
    ny, nx = p.epid.npy, p.epid.npx
    dev = f"cuda:{local}"
    net = UNet(ny, nx, batch=1, levels=4, base_channels=32, seed=1, device=local, in_channels=1 + AUX_PLANES)
    d = torch.empty((ny, nx), dtype=torch.float64, device=dev)
    F, t = torch.empty_like(d), torch.empty_like(d)
    y = torch.empty((1, ny, nx), dtype=torch.float32, device=dev)
    times = []
    for r in range(reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.set_field(p.field, p.lut, stream=stream)
        sim.set_history_base(0)
        sim.run(n_input, SEED + 17, stream=stream)
        sim.dose_device(d, stream=stream)
        sim.fluence_device(F, stream=stream)
        sim.tmap_device(t, stream=stream)
        s = 1.0 / torch.clamp(d.mean(), min=1e-300)
        x = torch.cat([(d * s)[None], aux_planes(F, t)]).float()[None].contiguous()
        net.forward(x, y, 1.0, float(1.0 / s), stream=stream)
        torch.cuda.synchronize()
        if r:                                   # the first pass warms up
            times.append(time.perf_counter() - t0)
    net.close()
    return {"route_s_median": float(np.median(times)), "input_histories": n_input, "reps": reps,
            "input_planes": 1 + AUX_PLANES,
            "steps": "set_field, mc_run, mc_get_dose, mc_get_field_fluence, mc_get_tmap, planes, dn_forward"}


def denoiser_leg(args, local, barrier):
    """U-Net (768 x 1024, 4 levels, 32-256 channels) training and inference
    throughput on the tensor-core kernels, against the measured bf16 peak."""
    import torch
    from paper_2510_24154_b300.denoise import UNet
    B = args.dn_batch
    net = UNet(768, 1024, batch=B, levels=4, base_channels=32, seed=1, device=local)
    g = torch.Generator(device=f"cuda:{local}").manual_seed(5)
    x = torch.rand((B, 768, 1024), device=f"cuda:{local}", generator=g)
    t = torch.rand((B, 768, 1024), device=f"cuda:{local}", generator=g)
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        net.train_step(x, t, 1e-4, stream=stream, want_loss=False)
    barrier()
    steps = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        net.train_step(x, t, 1e-4, stream=stream, want_loss=False)
    e1.record(stream)
    barrier()
    train_ms = e0.elapsed_time(e1) / steps
    for _ in range(3):
        net.forward(x, out, stream=stream)
    barrier()
    e0.record(stream)
    for _ in range(steps):
        net.forward(x, out, stream=stream)
    e1.record(stream)
    barrier()
    fwd_ms = e0.elapsed_time(e1) / steps
    net.close()
    f_fwd, f_train = unet_flops()
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak, kind = float(json.load(f)["bf16_tflops_sustained"]), "measured (sustained bf16)"
    except Exception:
        peak, kind = 1400.0, "fallback (sustained bf16)"
    ach = B * f_train / (train_ms / 1e3) / 1e12
    return {"workload": f"U-Net 768x1024, 4 levels 32-256 channels, bf16 operands / f32 accumulate, batch {B}",
            "train_step_ms": train_ms, "train_images_per_s": B * 1e3 / train_ms,
            "forward_ms": fwd_ms, "infer_images_per_s": B * 1e3 / fwd_ms,
            "flops_per_image": {"forward": f_fwd, "train": f_train},
            "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "peak_kind": kind, "scope": "whole training step (all kernels)"},
            "forward_tflops": B * f_fwd / (fwd_ms / 1e3) / 1e12}


def batched_plan(args, Simulator, W, p, extra, stream, local, rank, dist, barrier):
    """The 25-field plan (gantry U[0,360), 5-40 segments, N_f log-uniform in
    [1e7, 2e8]) on the same CT and EPID, all fields in one graph-driven run:
    one launch whose waves loop on the device.  Reports whole-plan histories/s
    and each field's time to 1 % uncertainty at that rate."""
    import statistics
    import torch
    ph, ep, fields, hist = W.config_batched_plan(seed=2)
    hist = [max(int(h * args.batched_scale), 1000) for h in hist]
    sim = Simulator(p.physics, device=local, use_graph=1, **extra)
    sim.init_geometry(ph, ep, stream=stream)
    sim.set_fields(fields, p.lut, stream=stream)
    base = rank * max(hist)
    sim.set_history_base(base)
    sim.run_batch([max(h // 100, 1000) for h in hist], SEED, stream=stream)         # warm-up
    sim.reset_tally(stream=stream)
    sim.set_history_base(base)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    st = sim.run_batch(hist, SEED, stream=stream)
    ev1.record(stream)
    barrier()
    t = ev0.elapsed_time(ev1) / 1e3
    if dist is not None:
        tt = torch.tensor([t], device=f"cuda:{local}")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    ws = 1 if dist is None else dist.get_world_size()
    rate = sum(hist) / t
    s_1pct = []
    for f in range(len(fields)):
        _, _, u = sim.dose(field=f, stream=stream)
        s_1pct.append(hist[f] * (u / 0.01) ** 2 / rate)
    # what batching buys: field set-up (t-maps) plus transport of the whole
    # plan as one batch, against the same fields set up and run one by one
    # (one run per field, each field's histories from its own stream base)
    def timed(fn):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    def batched():
        sim.set_fields(fields, p.lut, stream=stream)
        sim.set_history_base(base)
        sim.run_batch(hist, SEED, stream=stream)

    def one_by_one():
        for f, fld in enumerate(fields):
            sim.set_field(fld, p.lut, stream=stream)
            sim.set_history_base((f << 40) + base)
            sim.run(hist[f], SEED, stream=stream)

    t_batch = timed(batched)
    t_seq = timed(one_by_one)
    sim.close()
    return {"workload": f"{len(fields)}-field IMRT plan on the thorax CT, 5-40 segments, gantry U[0,360), "
                        f"N_f log-uniform [1e7,2e8] x {args.batched_scale:g}, one graph-driven run",
            "fields": len(fields), "histories": int(sum(hist)) * ws, "seconds": t,
            "histories_per_s": ws * sum(hist) / t, "waves": st["waves"], "kernel_launches_in_graph": st["launches"],
            "host_launches": 1, "s_per_field_1pct_median": statistics.median(s_1pct),
            "s_per_field_1pct_max": max(s_1pct), "s_plan_1pct_all_fields": sum(s_1pct),
            "setup_and_run_s": {"batched": t_batch, "one_field_at_a_time": t_seq,
                                "speedup": t_seq / t_batch}}


def anthropomorphic_leg(args, Simulator, W, extra, stream, local, rank, dist, barrier):
    """The 512 x 512 x 200 phantom at 1 mm, one 40-segment field, the
    1190 x 1190 EPID at 0.336 mm: one graph-driven run of the full history
    count, its rate and the time to 1 % at that rate."""
    import torch
    N = args.anthro_histories
    p = W.config_anthropomorphic(n_histories=N)
    sim = Simulator(p.physics, device=local, use_graph=1, **extra)
    sim.init_geometry(p.phantom, p.epid, stream=stream)
    sim.set_field(p.field, p.lut, stream=stream)
    sim.set_history_base(rank * N)
    sim.run(max(N // 100, 1000), SEED, stream=stream)                              # warm-up
    sim.reset_tally(stream=stream)
    sim.set_history_base(rank * N)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    st = sim.run(N, SEED, stream=stream)
    ev1.record(stream)
    barrier()
    t = ev0.elapsed_time(ev1) / 1e3
    if dist is not None:
        tt = torch.tensor([t], device=f"cuda:{local}")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    ws = 1 if dist is None else dist.get_world_size()
    _, _, u = sim.dose(stream=stream)
    sim.close()
    rate = N / t
    return {"workload": "anthropomorphic_40seg: CT 512x512x200 int16 HU @1mm (body, lungs, spine, ribs, organs), "
                        "one 40-segment IMRT field, EPID 1190x1190 @0.336mm, coupled",
            "histories": N * ws, "seconds": t, "histories_per_s": ws * rate, "waves": st["waves"],
            "u_at_run": u, "histories_for_1pct": N * (u / 0.01) ** 2,
            "s_per_field_1pct": N * (u / 0.01) ** 2 / rate,
            "energy_closure": abs(st["e_ct"] + sum(st["e_epid"]) + st["e_esc"] + st["e_lost"] - st["e_src"])
            / st["e_src"]}


def to_one_percent(args, Simulator, W, stream, local, barrier):
    """Seconds per field at <= 1 % statistical uncertainty, measured: the
    workload runs in chunks until the batch uncertainty u (mean relative sigma
    over pixels above half the maximum, B = 16) of the accumulated image is at
    most 1 %, on the EPID grid of the paper's comparisons (160 x 160 at
    2.5 mm).  Two fields: the small water workload coupled (open 10 x 10) and
    the thorax IMRT field.  The time includes the statistics of every chunk."""
    import torch
    out = {}
    thorax = W.config_thorax_imrt(n_histories=1, seed=SEED)
    thorax.epid = W.epid_default(160, 160, 0.25)
    cases = (("paper_grid_water_open", W.config_paper_grid(), 2 * 10 ** 8),
             ("paper_grid_thorax_imrt_9seg", thorax, 5 * 10 ** 8))
    for name, prob, chunk in cases:
        sim = Simulator(prob.physics, device=local, use_graph=1,
                        **({"bank_capacity": args.bank_capacity} if args.bank_capacity else {}))
        sim.init_geometry(prob.phantom, prob.epid, stream=stream)
        sim.set_field(prob.field, prob.lut, stream=stream)
        sim.run(chunk // 100, prob.seed, stream=stream)                          # warm-up
        sim.reset_tally(stream=stream)
        barrier()
        t0 = time.perf_counter()
        done, u, chunks = 0, float("inf"), 0
        while u > 0.01 and done < 2 * 10 ** 10:
            sim.run(chunk, prob.seed, stream=stream)
            done += chunk
            chunks += 1
            _, _, u = sim.dose(stream=stream)                                    # synchronizes
        t = time.perf_counter() - t0
        st = sim.stats()
        sim.close()
        out[name] = {"histories": done, "chunks": chunks, "u": u, "seconds": t, "histories_per_s": done / t,
                     "epid": "160x160 @ 2.5 mm", "energy_closure":
                     abs(st["e_ct"] + sum(st["e_epid"]) + st["e_esc"] + st["e_lost"] - st["e_src"]) / st["e_src"]}
    out["paper_context"] = "about 90 s per IMRT field at 1e9 histories to < 1 % on an RTX 3090, 2.5 mm pixels " \
                           "(paper Sec. 2.3, 4.1); a clinical plan, not these synthetic fields"
    return out


def fp64_agreement(Simulator, oracle, problem, n, local, stream, field=None):
    """The same histories (ids 0..n-1) through the GPU (FP32 transport) and
    the FP64 oracle: sensitive-layer energy ratio, largest relative difference
    of the event counters, and the 1 %/1 mm global gamma pass rate of the GPU
    image on the full pixel grid with the oracle's as reference."""
    import numpy as np
    fld = field if field is not None else problem.field
    sim = Simulator(problem.physics, device=local)
    sim.init_geometry(problem.phantom, problem.epid, stream=stream)
    sim.set_field(fld, problem.lut, stream=stream)
    st = sim.run(n, problem.seed, stream=stream)
    gd, _, _ = sim.dose(stream=stream)
    gt = sim.tally().astype(np.float64) / 2.56e8
    sim.close()
    t0 = time.perf_counter()
    orc = oracle.run(problem, n_histories=n, field=fld)
    t_orc = time.perf_counter() - t0
    od, _, _ = oracle.dose_stats(orc["tally"], n, problem.epid)
    rate, _ = oracle.gamma(od, gd, pixel_mm=problem.epid.pitch * 10.0, dd=0.01, dta_mm=1.0, threshold=0.10)
    keys = [k for k in oracle.COUNTER_NAMES if orc["counters"][k] > 0]
    cdev = max(abs(st["counters"][k] / orc["counters"][k] - 1.0) for k in keys)
    return {"histories": n, "sensitive_energy_ratio": float(gt.sum() / orc["tally"].sum()),
            "counters_max_rel_diff": cdev, "gamma_1pct_1mm_full_grid": rate,
            "pixels": f"{problem.epid.npx}x{problem.epid.npy} @ {problem.epid.pitch * 10:g} mm",
            "oracle_seconds": t_orc}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch
    from paper_2510_24154_b300 import workloads as W
    from paper_2510_24154_b300.binding import Simulator

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    p = W.config_thorax_imrt(n_histories=args.histories, seed=SEED)
    N = args.histories
    extra = {"bank_capacity": args.bank_capacity} if args.bank_capacity else {}
    if args.primaries_per_wave:
        extra["primaries_per_wave"] = args.primaries_per_wave
    if args.regs_variant:
        extra["regs_variant"] = [int(v) for v in args.regs_variant.split(",")]
    sim = Simulator(p.physics, device=local, time_kernels=1, **extra)
    stream = torch.cuda.current_stream()
    hu_dev = torch.from_numpy(p.phantom.hu).to(f"cuda:{local}")
    ny, nx = p.epid.npy, p.epid.npx
    dose = torch.empty((ny, nx), dtype=torch.float64, device=f"cuda:{local}")
    sigma = torch.empty_like(dose)
    signal = torch.empty((ny, nx), dtype=torch.float32, device=f"cuda:{local}")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=f"cuda:{local}")   # > 126 MB L2

    agg = {"kernel_ms": np.zeros(4), "kernel_launches": np.zeros(4), "esteps_ct": 0, "launches": 0}

    def step(record):
        sim.init_geometry(p.phantom, p.epid, stream=stream, hu_device=hu_dev)     # CT set-up
        sim.set_field(p.field, p.lut, stream=stream)                              # source, t-map, Eq. 1
        sim.set_history_base(rank * N)
        st = sim.run(N, SEED, stream=stream)                                      # transport
        sim.dose_device(dose, sigma, stream=stream)                               # statistics
        sim.epid_image_device(signal, stream=stream)                              # k(t, s) image
        flush.zero_()
        if record:
            agg["kernel_ms"] += np.array(st["kernel_ms"])
            agg["kernel_launches"] += np.array(st["kernel_launches"])
            agg["esteps_ct"] += st["counters"]["esteps_ct"]
            agg["launches"] += st["launches"] + 2 + 1 + 2
        return st

    for _ in range(max(args.warmup, 3)):
        step(False)
    barrier()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            last = step(True)
        ev1.record(stream)
        barrier()
        wall = time.perf_counter() - t0
    gpu_ms = ev0.elapsed_time(ev1)
    t_local = gpu_ms / 1e3
    t_all = t_local
    if dist is not None:
        t = torch.tensor([t_local], device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_all = float(t.item())
    total_hist = ws * N * args.steps
    value = total_hist / t_all

    # statistical uncertainty of one field -> seconds per field at <= 1 %
    _, _, u = sim.dose(stream=stream)
    n_1pct = N * (u / 0.01) ** 2
    per_gpu_rate = N * args.steps / t_local

    # live roofline of the dominant kernel (CT electrons)
    launches_e = max(agg["kernel_launches"][1], 1)
    avg_ms = agg["kernel_ms"][1] / launches_e
    steps_per_launch = agg["esteps_ct"] / launches_e
    insts = INST_PER_ESTEP_CT * steps_per_launch
    flops = FLOPS_PER_ESTEP_CT * steps_per_launch
    hbm_peak, peak_kind = peaks()
    # algorithmic bytes of a CT electron launch: one 4-byte density gather per
    # step plus the bank records read and written (48 bytes each)
    st_counts = last["counters"]
    bank_bytes = 48.0 * 2 * st_counts["electrons"] / max(last["kernel_launches"][1], 1)
    alg_bytes = 4.0 * steps_per_launch + bank_bytes
    mem_achieved = alg_bytes / (avg_ms / 1e3) / 1e9 if avg_ms > 0 else 0.0
    roofline = {
        "bound": "alu", "kernel": "k_transport<electrons in CT>",
        "achieved": insts / (avg_ms / 1e3) / 1e12 if avg_ms > 0 else 0.0,
        "peak": ISSUE_PEAK_TINST, "unit": "T thread-instructions/s",
        "peak_kind": "derived: 148 SMs x 4 schedulers x 32 lanes x 2.032 GHz (one warp instruction per "
                     "scheduler per clock)",
        "traffic": DRAM_BYTES_PER_ESTEP_CT * steps_per_launch,
        "traffic_note": "ncu DRAM read+write per CT electron step on the 2e6-history case, scaled by the "
                        "steps of one launch here",
        "inst_per_unit": INST_PER_ESTEP_CT, "unit_of_work": "CT electron step",
        "lanes_per_warp_inst": INST_PER_ESTEP_CT / WARP_INST_PER_ESTEP_CT,
        "ncu_issue_active": NCU_ISSUE_ACTIVE_ECT, "ncu_warps_active": NCU_WARPS_ACTIVE_ECT,
        "ncu_note": "ncu --set full of this kernel on the 2e6-history case: scheduler cycles that issued, "
                    "occupied warp slots of the SM's 64 (at most 0.5: 4 CTAs of 256 threads, register-limited)",
        "units_per_launch": steps_per_launch, "avg_launch_ms": avg_ms,
        "fp32": {"flops_per_unit": FLOPS_PER_ESTEP_CT,
                 "achieved_tflops": flops / (avg_ms / 1e3) / 1e12 if avg_ms > 0 else 0.0,
                 "peak_tflops": FP32_PEAK_TFLOPS},
        "kernel_share_of_transport": float(agg["kernel_ms"][1] / max(agg["kernel_ms"].sum(), 1e-12)),
        "lane_utilisation": {
            "photons_ct": last["counters"]["live_lanes_photon_ct"] / max(32 * last["counters"]["warp_iters_photon_ct"], 1),
            "electrons_ct": last["counters"]["live_lanes_electron_ct"] / max(32 * last["counters"]["warp_iters_electron_ct"], 1)},
        "transport_ms_per_step": {k: float(v / args.steps) for k, v in
                                  zip(("photons_ct", "electrons_ct", "photons_epid", "electrons_epid"),
                                      agg["kernel_ms"])},
    }
    roofline["frac"] = roofline["achieved"] / roofline["peak"]
    # measured arithmetic peaks of this GPU (outside the timed region): the
    # best issue rate any probe reached, and the FP32 FMA rate
    from paper_2510_24154_b300.binding import probe_alu_peaks
    probe = probe_alu_peaks(local)
    issue_meas = max(probe["ffma_tflops"] / 2.0, probe["int_tinst"], probe["mix_tinst"])
    roofline["probe"] = dict(probe, issue_tinst_measured=issue_meas)
    roofline["frac_of_probe_issue"] = roofline["achieved"] / issue_meas
    roofline["fp32"]["peak_tflops_measured"] = max(probe["ffma_tflops"], probe["ffma2_tflops"])
    roofline["fp32"]["frac_of_measured"] = roofline["fp32"]["achieved_tflops"] / roofline["fp32"]["peak_tflops_measured"]
    memory_roofline = {"bound": "hbm", "achieved": mem_achieved, "peak": hbm_peak, "unit": "GB/s",
                       "frac": mem_achieved / hbm_peak, "peak_kind": peak_kind,
                       "algorithmic_bytes_per_launch": alg_bytes}

    # end to end through the C-ABI with host buffers
    e2e = None
    if not args.no_e2e:
        hu_pinned = torch.from_numpy(p.phantom.hu).pin_memory()
        phantom_host = W.Phantom(hu_pinned.numpy(), p.phantom.vox, p.phantom.origin)
        fld = p.field
        h2d = (hu_pinned.numel() * 2 + fld.pair_edges.nbytes + fld.leaves.nbytes + fld.jaws.nbytes + fld.mu.nbytes
               + p.lut.t_nodes.nbytes + p.lut.s_nodes.nbytes + p.lut.k.nbytes)
        barrier()
        t0 = time.perf_counter()
        waves = 0
        for _ in range(args.steps):
            sim.init_geometry(phantom_host, p.epid, stream=stream)
            sim.set_field(p.field, p.lut, stream=stream)
            sim.set_history_base(rank * N)
            st = sim.run(N, SEED, stream=stream)
            img = sim.epid_image(stream=stream)
            waves += st["waves"]
        barrier()
        te = time.perf_counter() - t0
        if dist is not None:
            t = torch.tensor([te], device=f"cuda:{local}")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            te = float(t.item())
        d2h = img.nbytes + CTL_BYTES * waves // args.steps
        e2e = {"value": total_hist / te, "unit": "histories/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    batched = None
    if not args.no_batched:
        batched = batched_plan(args, Simulator, W, p, extra, stream, local, rank, dist, barrier)
    denoiser = None
    if not args.no_denoiser:
        denoiser = denoiser_leg(args, local, barrier)
    # the metric's two routes per field on this workload: plain Monte Carlo to
    # 1 % per pixel, and the denoised route measured end to end (set-up, 1e7
    # histories, dose, fluence and t-map planes, inference).  The second
    # route's image quality needs a trained network: the evaluation driver
    # measures it and a GPU test asserts it; it is not a number of this run.
    denoised_vs_plain = None
    if denoiser is not None:
        route = denoised_route_leg(sim, p, stream, local)
        denoised_vs_plain = {
            "plain_s_per_field_1pct": n_1pct / per_gpu_rate,
            "denoised_s_per_field": route["route_s_median"],
            "denoised_route": route,
        }
    one_pct = None
    if ws == 1 and not args.no_one_pct:
        one_pct = to_one_percent(args, Simulator, W, stream, local, barrier)
    anthro = None
    if not args.no_anthro:
        anthro = anthropomorphic_leg(args, Simulator, W, extra, stream, local, rank, dist, barrier)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        threads = os.cpu_count() or 1
        sample = 12_000_000           # about 11 s on 16 threads
        v, used, dt = cpu_sample(p, sample, threads)
        sample1 = 400_000             # about 6 s on one thread
        v1, _, dt1 = cpu_sample(p, sample1, 1)
        cpu = {"value": v, "unit": "histories/s", "cores": used, "kind": "oracle",
               "sample": f"{sample} histories of the same workload ({dt:.1f} s wall on {used} threads)",
               "threads_cap": f"the oracle's threads own sub-tallies: at most B = {p.physics.n_batches} threads",
               "host": {"cpu_model": cpu_model(), "logical_cpus": threads},
               "single_core": {"value": v1, "unit": "histories/s",
                               "sample": f"{sample1} histories on 1 thread ({dt1:.1f} s wall)"}}
        # FP32 transport against the FP64 oracle on the same histories, per
        # headline result (replay: same keys, same draw order)
        agree = {"thorax_imrt_9seg": fp64_agreement(Simulator, oracle, p, 2_000_000, local, stream)}
        if one_pct is not None:
            agree["paper_grid_water_open"] = fp64_agreement(Simulator, oracle, W.config_paper_grid(), 2_000_000,
                                                            local, stream)
        if batched is not None:
            ph, ep, fields, _ = W.config_batched_plan(seed=2)
            bp = W.config_thorax_imrt(n_histories=1, seed=SEED)
            bp.phantom, bp.epid = ph, ep
            agree["batched_plan_field0"] = fp64_agreement(Simulator, oracle, bp, 1_000_000, local, stream,
                                                          field=fields[0])
        if anthro is not None:
            agree["anthropomorphic_40seg"] = fp64_agreement(Simulator, oracle, W.config_anthropomorphic(),
                                                            200_000, local, stream)
        cpu["fp64_agreement"] = agree

    if rank == 0:
        line = {
            "metric": "histories/s", "value": value, "unit": "histories/s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "histories_per_step_per_gpu": N, "seed": SEED,
                       "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"history shards x{ws}, no collective"},
            "s_per_field_1pct": n_1pct / per_gpu_rate, "u_at_step": u, "histories_for_1pct": n_1pct,
            "roofline": roofline, "memory_roofline": memory_roofline, "cpu_baseline": cpu, "e2e": e2e,
            "batched_plan": batched, "denoiser": denoiser, "denoised_vs_plain": denoised_vs_plain,
            "to_1pct_measured": one_pct,
            "anthropomorphic": anthro,
            "events_per_history": {k: last["counters"][k] / N for k in
                                   ("flights_ct", "real_ct", "compton", "photo", "pair", "esteps_ct", "esteps_epid",
                                    "moller", "brem", "electrons", "primaries_at_epid")},
            "gpu_launches": int(agg["launches"]), "clocks": clk.summary(), "wall_s_timed": wall,
            "paper_context": "about 90 s per IMRT field at 1e9 histories on an RTX 3090 (paper Sec. 4.1)",
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    sim.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
