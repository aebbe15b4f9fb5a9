"""Single-workload drivers for profiling one kernel of the library in
isolation (for example under ncu): each runs a fixed, seeded workload through
the public API and exits.

    python -m paper_2108_12430_gb300.drivers bbhnet --precision fp8 --batch 256 --forwards 2
    python -m paper_2108_12430_gb300.drivers train --precision bf16 --batch 8 --length 8192

bbhnet: BBHnet (synth.bbhnet_params(3)) on random whitened strain of batch x 2 x
2048, `forwards` calls of gw_bbhnet_score (FP8: after gw_model_calibrate on the
same batch, which runs the FP32 path).  Each forward launches 13 tensor-core
conv kernels in the order stem, then per block shortcut, first conv, second conv.

train: one DeepClean training step (forward with tape, band loss with 2049
taps, its backward, the network backward) on batch x 21 x length seeded
windows; the backward's weight gradients run from the output layer down.
"""
from __future__ import annotations

import argparse

import numpy as np

from . import gwstream as G, synth

PRECISIONS = {"fp32": G.GW_FP32, "bf16": G.GW_BF16, "fp8": G.GW_FP8}


def bbhnet(precision, batch, forwards):
    import torch
    ctx = G.gw_ctx_create(0, 0)
    try:
        layers, head = synth.bbhnet_params(3)
        m = G.gw_model_create(ctx, G.GW_MODEL_BBHNET, precision, 2, synth.flatten_params(layers, head))
        gen = torch.Generator(device="cuda").manual_seed(3)
        x = torch.randn(batch, 2, 2048, device="cuda", generator=gen)
        lg = torch.empty(batch, device="cuda")
        if precision == G.GW_FP8:
            G.gw_model_calibrate(m, x.data_ptr(), batch, 2048)
        for _ in range(forwards):
            G.gw_bbhnet_score(m, x.data_ptr(), batch, 2048, lg.data_ptr())
        torch.cuda.synchronize()
        G.gw_model_status(m)
        G.gw_model_destroy(m)
    finally:
        G.gw_ctx_destroy(ctx)


def train(precision, batch, length):
    import torch
    C = 21
    ctx = G.gw_ctx_create(0, 0)
    try:
        t = G.gw_trainer_create(ctx, C, batch, length, 0, precision=precision)
        _, psd = synth.psd_grid(4096.0, 8192)
        g = G.gw_fir_create_band_loss(ctx, psd, 4096.0, 2049)
        x = torch.from_numpy(np.stack([synth.witness_channels(6 + b, C, length) for b in range(batch)])
                             .astype(np.float32)).cuda()
        s = torch.from_numpy((np.random.default_rng(5).standard_normal((batch, length)) * 0.3)
                             .astype(np.float32)).cuda()
        p = torch.from_numpy(synth.flatten_params(synth.deepclean_params(5))).cuda()
        y, dy, dp = torch.empty(batch, length, device="cuda"), torch.empty(batch, length, device="cuda"), \
            torch.empty_like(p)
        r = torch.empty(batch, length - 2048, device="cuda")
        loss = torch.empty(1, device="cuda")
        G.gw_trainer_forward(t, p.data_ptr(), x.data_ptr(), batch, y.data_ptr())
        G.gw_band_loss(g, s.data_ptr(), y.data_ptr(), batch, length, loss.data_ptr(), r.data_ptr())
        G.gw_band_loss_backward(g, r.data_ptr(), batch, length, 0, dy.data_ptr())
        G.gw_trainer_backward(t, dy.data_ptr(), dp.data_ptr())
        torch.cuda.synchronize()
        G.gw_trainer_status(t)
        G.gw_fir_destroy(g)
        G.gw_trainer_destroy(t)
    finally:
        G.gw_ctx_destroy(ctx)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    sub = ap.add_subparsers(dest="what", required=True)
    b = sub.add_parser("bbhnet")
    b.add_argument("--precision", choices=["fp32", "bf16", "fp8"], default="bf16")
    b.add_argument("--batch", type=int, default=256)
    b.add_argument("--forwards", type=int, default=2)
    t = sub.add_parser("train")
    t.add_argument("--precision", choices=["fp32", "bf16"], default="bf16")
    t.add_argument("--batch", type=int, default=8)
    t.add_argument("--length", type=int, default=8192)
    a = ap.parse_args()
    if a.what == "bbhnet":
        bbhnet(PRECISIONS[a.precision], a.batch, a.forwards)
    else:
        train(PRECISIONS[a.precision], a.batch, a.length)
    print("ok")


if __name__ == "__main__":
    main()
