"""Concurrent multishift solves of several systems (e.g. the k-points of one workload).

Each job runs on its own CUDA stream from its own host thread (the library call releases the
Python interpreter lock), so the persistent solver kernels of different systems share the
GPU: the CTAs of one kernel take over the SMs that another kernel's last right-hand sides
leave idle.  Every system handle is used by exactly one thread, as the C ABI requires.
"""
from __future__ import annotations

import threading


def solve_concurrent(jobs, omega, eta, tol=1e-10, omegas=None, **kwargs):
    """jobs: list of dicts with keys sys, rhs, e_ref, out (CUDA tensors, or pinned host tensors
    that the library stages on each job's stream); every job solves at `omega`, or job i at
    omegas[i].  Returns [(report, converged)] in job order.  (sgw_solve_batched packs several
    systems into one persistent launch instead.)"""
    import torch
    results = [None] * len(jobs)
    errors = []
    device = torch.device("cuda", torch.cuda.current_device())
    streams = [torch.cuda.Stream(device=device) for _ in jobs]
    current = torch.cuda.current_stream(device)
    for s in streams:
        s.wait_stream(current)

    def run(i):
        try:
            with torch.cuda.stream(streams[i]):
                j = jobs[i]
                om = omegas[i] if omegas is not None else omega
                _, rep, ok = j["sys"].solve_shifted(j["rhs"], j["e_ref"], om, eta, tol=tol, out=j["out"],
                                                    stream=streams[i].cuda_stream, **kwargs)
                results[i] = (rep, ok)
        except Exception as e:  # re-raised in the caller's thread
            errors.append(e)

    threads = [threading.Thread(target=run, args=(i,)) for i in range(len(jobs))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for s in streams:
        current.wait_stream(s)
    if errors:
        raise errors[0]
    return results
