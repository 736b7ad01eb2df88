"""Run the CPU oracle on many shots at once in worker processes.

The workers are started with the "spawn" method, so they are fresh
interpreters that never touch the parent's CUDA context; they load only the
oracle.  Used by the GPU tests whose oracle side takes tens of seconds on one
core (large lattices, near-threshold shots).
"""
import os
from multiprocessing import get_context

import numpy as np

_POOL = None


def _decode_one(args):
    import oracle
    n, kw = args
    return oracle.decode_shot(n, **kw)


def _pool():
    global _POOL
    if _POOL is None:
        _POOL = get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1)))
    return _POOL


def decode_many(N_np, shot0=0, **kw):
    """oracle.decode_shot over the shots of N_np (uint8 [shots][2][L][L]) in
    parallel, shot i with index shot0 + i (the key of the random rules);
    returns (C, steps int32, flags uint8) stacked like decode_batch."""
    out = _pool().map(_decode_one, [(np.ascontiguousarray(n), dict(kw, shot=shot0 + i))
                                     for i, n in enumerate(N_np)])
    return (np.stack([o[0] for o in out]), np.array([o[1] for o in out], np.int32),
            np.array([o[2] for o in out], np.uint8))


def _run_one(args):
    import oracle
    fn, n, kw = args
    return getattr(oracle, fn)(n, **kw)


def run_many(fn, jobs):
    """oracle.<fn>(n, **kw) for each (n, kw) of jobs, in parallel; shots of
    different sizes and options may be mixed."""
    return _pool().map(_run_one, [(fn, np.ascontiguousarray(n), kw) for n, kw in jobs],
                       chunksize=1)


def close():
    global _POOL
    if _POOL is not None:
        _POOL.close()
        _POOL.join()
        _POOL = None
