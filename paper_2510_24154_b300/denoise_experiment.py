"""Train and evaluate the denoiser on Monte Carlo pairs; prints one JSON line.

    python -m paper_2510_24154_b300.denoise_experiment --pairs 128 --n-input 1e6 \
        --n-target 1e9 --eval 8 --n-ref 1e10 --steps 3000

The default sizes are the reduced data set (128 training pairs instead of
2000, 8 held-out cases instead of 100) that one GPU session affords: the
targets alone are 1.3e11 histories.

With --family anthropomorphic the cases are the 512x512x200 phantom at 1 mm
(jittered) on the 1190 x 1190, 0.336 mm EPID, and the first held-out case is
the unjittered anthropomorphic workload with its 40-segment field: run with
--n-input 1e7 and a ladder reaching 1e9, it compares 1e7 histories plus the
denoiser with 1e9 plain histories on that workload.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=128)
    ap.add_argument("--n-input", type=float, default=1e6)
    ap.add_argument("--n-target", type=float, default=1e9)
    ap.add_argument("--eval", type=int, default=8)
    ap.add_argument("--n-ref", type=float, default=1e10)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-final", type=float, default=5e-5)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--bin", type=int, default=8)
    ap.add_argument("--augment", action="store_true", help="random row/column mirroring of the training pairs")
    ap.add_argument("--family", default="thorax", choices=("thorax", "anthropomorphic"))
    ap.add_argument("--aux", action="store_true",
                    help="give the network the aperture fluence, t-map and primary estimate as extra planes")
    ap.add_argument("--ladder", type=str, default="1e7,3e7,1e8,3e8,1e9,3e9",
                    help="history counts of plain Monte Carlo images evaluated beside the denoised ones")
    args = ap.parse_args()
    import torch
    from .denoise import UNet
    from .denoise_data import (AUX_PLANES, CONFIG5_CASE, DoseSource, evaluate, family_epid, make_pairs,
                               matched_histories, net_shape, train)

    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    src = DoseSource()
    X, T, _ = make_pairs(src, range(args.pairs), int(args.n_input), int(args.n_target), args.seed, aux=args.aux,
                         family=args.family)
    t_pairs = time.perf_counter() - t0
    mc_hist, mc_s = src.histories, src.seconds
    cin = 1 + AUX_PLANES if args.aux else 1
    H, Wd = net_shape(family_epid(args.family))
    net = UNet(H, Wd, batch=args.batch, levels=4, base_channels=32, seed=args.seed, in_channels=cin)
    t1 = time.perf_counter()
    losses = train(net, X, T, args.steps, args.lr, args.batch, seed=args.seed, log_every=max(args.steps // 20, 1),
                   lr_final=args.lr_final, augment=args.augment)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    del X, T
    # evaluation network: batch 1
    params = net.params()
    net.close()
    ev_net = UNet(H, Wd, batch=1, levels=4, base_channels=32, seed=args.seed, in_channels=cin)
    ev_net.set_params(params)
    cases = list(range(100000, 100000 + args.eval))
    if args.family == "anthropomorphic":
        cases = [CONFIG5_CASE] + cases[:-1]
    t2 = time.perf_counter()
    ladder = [float(v) for v in args.ladder.split(",")] if args.ladder else []
    res = evaluate(ev_net, src, cases, int(args.n_input), int(args.n_ref), seed=args.seed, b=args.bin,
                   ladder=ladder, aux=args.aux, family=args.family)
    t_eval = time.perf_counter() - t2
    # plain Monte Carlo at the denoised image's quality, and the time of each
    # route per field at the measured transport rate and inference time
    g_den = float(np.mean([r["gamma_denoised"] for r in res]))
    e_den = float(np.mean([r["rms_denoised"] for r in res]))
    lad_g = [(n, float(np.mean([r["ladder"][i]["gamma"] for r in res]))) for i, n in enumerate(ladder)]
    lad_e = [(n, -float(np.mean([r["ladder"][i]["rms"] for r in res]))) for i, n in enumerate(ladder)]
    rate = src.histories / max(src.seconds, 1e-9)
    x = torch.zeros((1, cin, H, Wd), dtype=torch.float32, device="cuda:0")
    y = torch.empty((1, H, Wd), dtype=torch.float32, device="cuda:0")
    ev_net.forward(x, y)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    for _ in range(10):
        ev_net.forward(x, y)
    torch.cuda.synchronize()
    t_inf = (time.perf_counter() - t3) / 10
    n_g, n_e = matched_histories(lad_g, g_den), matched_histories(lad_e, -e_den)
    matched = {
        "mc_histories_per_s": rate, "inference_s": t_inf,
        "denoised_s_per_field": args.n_input / rate + t_inf,
        # measured per held-out field: set-up, transport, dose, planes and inference
        "denoised_route_s_measured_median": float(np.median([r["route_s"] for r in res])),
        "plain_histories_at_denoised_gamma": n_g,
        "plain_s_per_field_at_denoised_gamma": None if n_g is None else n_g / rate,
        "plain_histories_at_denoised_rms": n_e,
        "plain_s_per_field_at_denoised_rms": None if n_e is None else n_e / rate,
        "ladder_gamma_mean": lad_g, "ladder_rms_mean": [(n, -v) for n, v in lad_e],
        # each plain history count against the denoised input, per field
        "vs_plain": [{"n": n, "s_per_field": n / rate, "gamma": g, "rms": -e,
                      "denoised_gamma_minus_plain": g_den - g, "denoised_rms_over_plain": e_den / -e}
                     for (n, g), (_, e) in zip(lad_g, lad_e)],
    }
    line = {
        "pairs": args.pairs, "n_input": args.n_input, "n_target": args.n_target, "eval_cases": args.eval,
        "n_ref": args.n_ref, "steps": args.steps, "augment": args.augment, "in_channels": cin,
        "family": args.family, "image": [H, Wd],
        "n_params": ev_net.n_params, "batch": args.batch, "lr": args.lr, "lr_final": args.lr_final, "bin": args.bin,
        "gamma": "2 %/2 mm global, 10 % threshold, binned {0}x{0} ({1:.2f} mm)".format(
            args.bin, 10 * family_epid(args.family).pitch * args.bin),
        "loss_first": losses[0][1], "loss_last": losses[-1][1], "losses": losses,
        "gamma_raw_mean": float(np.mean([r["gamma_raw"] for r in res])),
        "gamma_denoised_mean": float(np.mean([r["gamma_denoised"] for r in res])),
        "rms_raw_mean": float(np.mean([r["rms_raw"] for r in res])),
        "rms_denoised_mean": float(np.mean([r["rms_denoised"] for r in res])),
        "gamma_denoised_rescaled_mean": float(np.mean([r["gamma_denoised_rescaled"] for r in res])),
        "rms_denoised_rescaled_mean": float(np.mean([r["rms_denoised_rescaled"] for r in res])),
        "bias_raw_mean": float(np.mean([r["bias_raw"] for r in res])),
        "bias_denoised_mean": float(np.mean([r["bias_denoised"] for r in res])),
        "matched": matched,
        "cases": res, "seconds": {"pairs": t_pairs, "train": t_train, "eval": t_eval},
        "mc_histories_for_pairs": mc_hist, "mc_seconds_for_pairs": mc_s,
    }
    print(json.dumps(line), flush=True)
    ev_net.close()
    src.close()


if __name__ == "__main__":
    main()
