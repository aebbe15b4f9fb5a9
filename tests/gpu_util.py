"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch

from paper_2108_12430_gb300 import gwstream as G, synth


def rel_l2(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


class Ctx:
    def __init__(self, budget=0):
        self.h = G.gw_ctx_create(0, budget)
        self.objs = []

    def deepclean(self, seed, precision=G.GW_FP32, mean=None, std=None):
        p = synth.flatten_params(synth.deepclean_params(seed))
        m = G.gw_model_create(self.h, G.GW_MODEL_DEEPCLEAN, precision, 21, p, mean, std)
        self.objs.append((G.gw_model_destroy, m))
        return m

    def bbhnet(self, seed, precision=G.GW_FP32, act_scales=None):
        layers, head = synth.bbhnet_params(seed)
        p = synth.flatten_params(layers, head)
        m = G.gw_model_create(self.h, G.GW_MODEL_BBHNET, precision, 2, p, act_scales=act_scales)
        self.objs.append((G.gw_model_destroy, m))
        return m

    def close(self):
        torch.cuda.synchronize()
        for fn, o in reversed(self.objs):
            fn(o)
        G.gw_ctx_destroy(self.h)
