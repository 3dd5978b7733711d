"""Autotuner for the batched solve: the number of concurrent streams.

Small active spaces leave most of the GPU idle, so several are solved at
once; too many in flight contend for memory and launch bandwidth.  The tuner
times hci_solve_batch on the given instances for each candidate stream
count and returns the fastest (timings included)."""
from __future__ import annotations

import time

import torch

from . import _abi


def tune_nstreams(instances, eps1, candidates=(1, 2, 4, 8, 16, 32), dav_tol=1e-9, want_rdm=False):
    times = {}
    for ns in candidates:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _abi.hci_solve_batch(instances, eps1, dav_tol=dav_tol, nstreams=ns, want_rdm=want_rdm)
        torch.cuda.synchronize()
        times[ns] = time.perf_counter() - t0
    best = min(times, key=times.get)
    return best, times
