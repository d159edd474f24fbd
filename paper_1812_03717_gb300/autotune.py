"""Autotuner of the multishift kernel's launch shape, per size bucket.

A size bucket is the FFT box, the plane-wave count (rounded), the occupied states, the
projectors, the number of shifts and the precision.  For a bucket the tuner times short probe
solves of the multishift kernel -- a fixed number of Lanczos steps for as many right-hand sides
as the kernel holds at once, no corrections -- over the candidate CTA sizes (256, 384, 512
threads) and the cluster sizes whose split fits (one CTA per vector whenever the box fits it;
for boxes that need a cluster, the library's choice and the next larger sizes), and keeps the
shape with the least time per Lanczos step.  Choices are cached in a JSON file
($SGW_TUNE_CACHE, default <tmp>/sgw_tune.json) keyed by the bucket and the GPU's name, so a
bucket is timed once per machine.  The radix schedule of each FFT axis (prime-factor stages
where the axis factors into 2, 3, 4, 5, 8, 9, else radix-4/2/3/5 stages) and the planes per
pass (the most that fit next to the kernel's shared memory) are set by the library; the tuner
picks what only timing can: CTA and cluster size.
"""
from __future__ import annotations

import json
import os
import tempfile

import numpy as np


def _cache_path():
    return os.environ.get("SGW_TUNE_CACHE") or os.path.join(tempfile.gettempdir(), "sgw_tune.json")


def _load():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d):
    path = _cache_path()
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def bucket_key(system, dims, nocc, nproj, nomega, precision):
    import torch
    npw_bucket = int(round(system.n_pw / 256.0)) * 256
    gpu = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return f"{gpu}|box{dims[0]}x{dims[1]}x{dims[2]}|npw~{npw_bucket}|occ{nocc}|proj{nproj}|w{nomega}|{precision}"


def tune(system, rhs, e_ref, omega, eta, dims, nocc, nproj, precision="df32", probe_steps=40,
         threads=(256, 384, 512), refresh=False):
    """Best (threads, cluster size) for this system's bucket; times probes on `rhs` (a device
    tensor of right-hand sides of the system, at least as many as the kernel holds at once)
    unless the cache has the bucket.  Leaves the system on the chosen cluster size and returns
    {"threads", "csize", "ms_per_step", "timed": [...]}."""
    key = bucket_key(system, dims, nocc, nproj, len(omega), precision)
    cache = _load()
    if key in cache and not refresh:
        choice = cache[key]
        system.set_split(choice["csize"] if choice["csize"] != system.split()[0] else 0)
        return choice
    auto_c = system.split()[0 if precision != "fp32" else 1]
    csizes = [1] if auto_c == 1 else sorted({auto_c, min(16, auto_c + 1), min(16, auto_c + 3)})
    timed = []
    for c in csizes:
        try:
            system.set_split(c if c != auto_c else 0)
        except Exception:
            continue
        for nt in threads:
            try:
                owners = system.lanczos_owners(len(omega), precision, nt)
                n = min(rhs.shape[0], owners)
                _, rep, _ = system.solve_shifted(rhs[:n].contiguous(), e_ref[:n], omega, eta, tol=1e-30,
                                                 precision=precision, threads=nt, max_matvec=probe_steps,
                                                 max_refine=-1, cert_tol=-1)
                steps = float(rep["matvecs"].max(axis=1).mean())
                # time per step of the whole GPU: per owner-step, scaled by the owners in flight
                ms = float(rep["kernel_ms"][0]) / max(steps, 1.0) / n
                timed.append({"threads": nt, "csize": c, "ms_per_step": ms})
            except Exception:
                continue
    if not timed:
        system.set_split(0)
        return {"threads": 0, "csize": auto_c, "ms_per_step": None, "timed": []}
    best = min(timed, key=lambda t: t["ms_per_step"])
    system.set_split(best["csize"] if best["csize"] != auto_c else 0)
    choice = dict(best, timed=timed)
    cache[key] = choice
    _store(cache)
    return choice
