"""Run the FP64 oracle over several channels in parallel (spawned processes,
one channel each) -- a test helper for integrations too long for one core.

Each worker calls ``oracle.moff_image`` on its own channel's voltages exactly as
a single call would; only the channels are spread over processes.
"""
import multiprocessing as mp
import os

import numpy as np


def _one(args):
    codes, gains, pos, taps, N, P, jones = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import oracle
    return oracle.moff_image(codes, gains, pos, taps, N, P, jones=jones, time_chunk=64)[0]


def moff_image_channels(codes, gains, pos, taps, N, P, jones=False, workers=None):
    """[C, n_prod, N, N] oracle images of every channel of ``codes`` [T, C, A, P]."""
    C = codes.shape[1]
    items = [(np.ascontiguousarray(codes[:, c:c + 1]), np.asarray(gains)[c:c + 1], pos, taps, N, P, jones)
             for c in range(C)]
    n = min(C, workers or max(1, (os.cpu_count() or 1)))
    with mp.get_context("spawn").Pool(n) as pool:
        return np.stack(pool.map(_one, items))
