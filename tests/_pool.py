"""Process pool for running many oracle trajectories in parallel (test helper).

BLAS threads are pinned to one per worker before numpy is imported in the
children, and workers are started with 'spawn' so that no CUDA context is ever
forked.
"""
import multiprocessing as mp
import os


def oracle_pool(n_workers=None):
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    n = n_workers or max(1, min(os.cpu_count() or 1, 16))
    return mp.get_context("spawn").Pool(n)
