"""The oracle's DeepClean forward over many snapshot windows, spread over
the host's cores (test infrastructure; see the package header).

Nothing here computes anything of the method: every window is cut by
``stream.window`` and passed unchanged through ``nets.deepclean_forward``.
Long streams (a thousand 21 x 32768 windows) take minutes on one core, so
the windows are split over worker processes.  The workers are started with
the "spawn" method (a process forked from one that has used the GPU can
hang), read the stream from shared memory and hold their numerical
libraries to one thread each.
"""
from __future__ import annotations

import os

import numpy as np

_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
_state = None


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _init(shm_name, shape, W, S, params, layers, mean, std):
    global _state
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=shm_name)
    x = np.ndarray(shape, np.float64, buffer=shm.buf)
    _state = (shm, x, W, S, params, layers, mean, std)


def _forward(ks):
    from oracle import nets, stream
    _, x, W, S, params, layers, mean, std = _state
    wins = np.stack([stream.window(x, W, S, k) for k in ks])
    return nets.deepclean_forward(wins, params, layers, mean, std)


class DeepCleanPool:
    """Worker processes holding one stream x_total (C, N); forward(ks) returns
    the oracle's predictions (len(ks), W) of the snapshot windows ks."""

    def __init__(self, x_total, W, S, params, layers, mean=None, std=None, workers=None, chunk=4):
        self.x = np.ascontiguousarray(x_total, np.float64)
        self.args = (W, S, params, layers, mean, std)
        self.workers = max(1, workers or host_cores())
        self.chunk = chunk
        self.ex = None
        self.shm = None

    def __enter__(self):
        if self.workers > 1:
            import multiprocessing as mp
            from concurrent.futures import ProcessPoolExecutor
            from multiprocessing import shared_memory
            self.shm = shared_memory.SharedMemory(create=True, size=self.x.nbytes)
            np.ndarray(self.x.shape, np.float64, buffer=self.shm.buf)[...] = self.x
            saved = {v: os.environ.get(v) for v in _THREAD_VARS}
            try:
                for v in _THREAD_VARS:
                    os.environ[v] = "1"
                # a worker that dies makes map() raise (BrokenProcessPool)
                # instead of being replaced forever
                self.ex = ProcessPoolExecutor(self.workers, mp_context=mp.get_context("spawn"), initializer=_init,
                                              initargs=(self.shm.name, self.x.shape) + self.args)
                # one single-window task per worker: the executor starts a
                # process per task while none is idle, so every worker starts
                # now, under the one-thread settings, and runs once
                list(self.ex.map(_forward, [[k] for k in range(self.workers)]))
            finally:
                for v, val in saved.items():
                    if val is None:
                        os.environ.pop(v, None)
                    else:
                        os.environ[v] = val
        return self

    def forward(self, ks):
        from oracle import nets, stream
        ks = list(ks)
        parts = [ks[i:i + self.chunk] for i in range(0, len(ks), self.chunk)]
        if self.ex is None:
            W, S, params, layers, mean, std = self.args
            return np.concatenate([nets.deepclean_forward(np.stack([stream.window(self.x, W, S, k) for k in p]),
                                                          params, layers, mean, std) for p in parts])
        return np.concatenate(list(self.ex.map(_forward, parts)))

    def __exit__(self, *exc):
        if self.ex is not None:
            self.ex.shutdown()
        if self.shm is not None:
            self.shm.close()
            self.shm.unlink()


def deepclean_stream_windows(x_total, W, S, ks, params, layers, mean=None, std=None, workers=None, chunk=4):
    """Predictions (len(ks), W) of the snapshot windows ks of the stream
    x_total (C, N): the oracle's forward of stream.window(x_total, W, S, k)."""
    ks = list(ks)
    workers = min(workers or host_cores(), 16, max(1, len(ks) // chunk))
    with DeepCleanPool(x_total, W, S, params, layers, mean, std, workers, chunk) as p:
        return p.forward(ks)
