"""Runs the FP64 oracle on large bandwidths across the host cores.

Test infrastructure like the rest of this package (the tests and the
benchmark's CPU-baseline leg use it).  The oracle's row-restricted routines (``forward_rows``, ``synthesis_rows``)
evaluate the same definitions as ``forward_separable`` / ``inverse_separable``
/ ``adjoint_separable`` for a subset of n; this module splits the n values of
both sectors into chunks and runs them in a pool of spawned processes (spawn,
not fork: the parent may already hold a CUDA context).  Inputs go to the
workers through a temporary .npy file that they map read-only.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import tempfile

import numpy as np

_THREAD_VARS = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")


def _n_values(N):
    return list(range(-(N - 1), N))          # doubled n of both sectors (|n| <= (N-1)/2)


def _chunks(vals, parts):
    # interleaved, so every chunk gets rows of every length of l
    return [vals[i::parts] for i in range(parts) if vals[i::parts]]


def _fwd_worker(args):
    path, ns, weights = args
    from . import transform as T
    fs = np.load(path, mmap_mode="r")
    return T.forward_rows(fs, ns, weights)


def _syn_worker(args):
    path, N, ns, ks, modes, weights = args
    from . import transform as T
    cs = np.load(path, mmap_mode="r")
    return T.synthesis_rows(cs, N, ns, ks, modes, weights)


def _stash(arr):
    fd, path = tempfile.mkstemp(suffix=".npy")
    os.close(fd)
    np.save(path, np.ascontiguousarray(arr))
    return path


class Runner:
    """A pool of spawned worker processes (one BLAS thread each) that stays up
    across calls: ``with Runner() as r: r.forward_all(fs)``."""

    def __init__(self, workers=None):
        self.workers = workers or os.cpu_count() or 1
        self.pool = None

    def __enter__(self):
        saved = {v: os.environ.get(v) for v in _THREAD_VARS}
        for v in _THREAD_VARS:
            os.environ[v] = "1"                   # one BLAS thread per worker
        try:
            self.pool = mp.get_context("spawn").Pool(self.workers)
        finally:
            for v, x in saved.items():
                if x is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = x
        return self

    def __exit__(self, *exc):
        self.pool.close()
        self.pool.join()

    def forward_all(self, fs, weights="cc", row_stride=1):
        """Every coefficient of each grid in fs [B, N, N, N]: [B, C] complex128.

        row_stride > 1 computes only the pairs whose n lies in every
        row_stride-th row of each sector, stage 1 included (a bounded sample;
        the other coefficients stay zero)."""
        fs = np.asarray(fs, dtype=np.complex128)
        B, N = fs.shape[0], fs.shape[1]
        ns = [n2 for n2 in _n_values(N) if ((n2 + N - 1) // 2) % row_stride == 0]
        path = _stash(fs)
        try:
            jobs = [(path, ch, weights) for ch in _chunks(ns, 4 * self.workers)]
            res = self.pool.map(_fwd_worker, jobs, chunksize=1)
        finally:
            os.remove(path)
        out = np.zeros((B, N * (N + 1) * (2 * N + 1) // 6), dtype=np.complex128)
        for idx, vals in res:
            out[:, idx] = vals
        return out

    def synthesis_planes(self, cs, N, ks, modes=("synthesis",), weights="cc"):
        """Synthesis and/or adjoint of packed coefficients cs [B, C] at the beta
        nodes ks: {mode: grid values f[B, N (alpha), len(ks), N (gamma)]}."""
        from . import transform as T
        cs = np.asarray(cs, dtype=np.complex128)
        path = _stash(cs)
        try:
            jobs = [(path, N, ch, list(ks), tuple(modes), weights) for ch in _chunks(_n_values(N), 4 * self.workers)]
            parts = self.pool.map(_syn_worker, jobs, chunksize=1)
        finally:
            os.remove(path)
        return {mode: T.planes_from_rows([pt[mode] for pt in parts], N) for mode in modes}


def forward_all(fs, weights="cc", workers=None, row_stride=1):
    """``Runner.forward_all`` with a pool for this call only."""
    with Runner(workers) as r:
        return r.forward_all(fs, weights, row_stride)


def synthesis_planes(cs, N, ks, modes=("synthesis",), weights="cc", workers=None):
    """``Runner.synthesis_planes`` with a pool for this call only."""
    with Runner(workers) as r:
        return r.synthesis_planes(cs, N, ks, modes, weights)
