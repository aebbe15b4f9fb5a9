"""One scored stream, the problem statement's call shape (create a stream
with its window and stride, push a snapshot, get back the cleaned strain and
the detection score), against the FP64 end-to-end oracle of one stream
(oracle/pipeline.py).  Snapshots are pushed one at a time through
gw_scored_stream_push and each ticket is waited for; the tolerances are the
serving tests' (FP32: relative L2 <= 1e-5 on the predicted noise and the
logits; BF16: <= 2e-2 on the noise, logits within 0.05)."""
import numpy as np
import pytest

from paper_2108_12430_gb300 import gwstream as G, synth
from tests.gpu_util import Ctx, rel_l2
from tests.test_gpu_serve import (BBH_SEED, C, FC, FS, FS2, KF, dc_params, oracle_stream, standardisation,
                                  strain_emitted, stream_inputs)

pytestmark = pytest.mark.gpu

W, S, N, DELTA, LB, KH, NFFT = 2048, 256, 20, 512, 512, 257, 512


@pytest.mark.parametrize("prec,out_scale", [(G.GW_FP32, 1.0), (G.GW_BF16, 1e-2)])
def test_scored_stream_push_matches_oracle(gpu_lib, prec, out_scale):
    ctx = Ctx()
    try:
        dcs = []
        for d in range(2):
            mean, std = standardisation(d)
            m = G.gw_model_create(ctx.h, G.GW_MODEL_DEEPCLEAN, prec, C, synth.flatten_params(dc_params(d, out_scale)),
                                  mean, std)
            ctx.objs.append((G.gw_model_destroy, m))
            dcs.append(m)
        bbh = ctx.bbhnet(BBH_SEED, prec)
        fdec = G.gw_fir_create_lowpass(ctx.h, FC, FS, KF)
        ctx.objs.append((G.gw_fir_destroy, fdec))
        _, psd = synth.psd_grid(FS2, NFFT)
        fw = G.gw_fir_create_whitening(ctx.h, psd, FS2, KH)
        ctx.objs.append((G.gw_fir_destroy, fw))
        s = G.gw_scored_stream_create(ctx.h, dcs, bbh, fdec, fw, C, W, S, G.GW_AGG_AVERAGE, DELTA, LB)
        wit, strn = stream_inputs(700, S, N)
        clean = np.zeros((N, 2, S), np.float32)
        score = np.zeros((N, 1), np.float32)
        for k in range(N):
            w = np.ascontiguousarray(wit[:, :, k * S:(k + 1) * S])
            x = np.ascontiguousarray(strn[:, k * S:(k + 1) * S])
            t = G.gw_scored_stream_push(s, w, x, clean[k], score[k])
            G.gw_scored_stream_wait(s, t, 60_000_000)
        G.gw_scored_stream_destroy(s)
        ref_cl, ref_lg = oracle_stream(700, S, N, G.GW_AGG_AVERAGE, DELTA, W, LB, KH, NFFT, out_scale)
        st = strain_emitted(700, S, N, DELTA)
        got_cl = clean.transpose(1, 0, 2)
        err = rel_l2(got_cl - st, ref_cl - st)
        lg = score[:, 0]
        print(f"prec {prec}: noise rel-L2 {err:.2e}, logit max abs err {np.abs(lg - ref_lg).max():.2e}")
        if prec == G.GW_FP32:
            assert err <= 1e-5 and rel_l2(lg, ref_lg) <= 1e-5
        else:
            assert err <= 2e-2 and np.abs(lg - ref_lg).max() <= 0.05
    finally:
        ctx.close()
