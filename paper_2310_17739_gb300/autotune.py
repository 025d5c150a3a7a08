"""Autotuner for the compile configuration (fusion level, fused block width
k_max, tile size, threads per block).

Times each candidate configuration on a prefix of the caller's own gate stream
through the C ABI (compile once, run twice, CUDA-event timed on the context's
stream) and keeps the fastest.  Candidates: the paper's fusion (fusion 1) with
dense blocks of up to k_max = 2..5 qubits (5 is the compiler's largest block),
and Pauli-gadget rotations (fusion 2), at the three largest tile sizes.
Results are cached in a JSON file keyed by (GPU name, n, dtype, fusion family,
prefix size), so a later run with the same key reuses the choice without
timing.  tune_batch tunes a batch per width group and applies each group's
choice to its instances.
"""
from __future__ import annotations

import json
import os
import time

from . import qsim as qs

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")


def candidates(n: int, dtype: str, allow_rotations: bool = True):
    """Configurations worth timing for an n-qubit state."""
    mx = 14 if dtype == "c64" else 13
    if n <= mx:  # the whole state in one block: the tile size is n
        out = [dict(fusion=1, k_max=k, tile_bits=n) for k in (2, 3, 4, 5)]
        if allow_rotations:
            out.append(dict(fusion=2, k_max=2, tile_bits=n))
        return out
    tiles = sorted({min(n, t) for t in (mx - 2, mx - 1, mx)})
    out = []
    for t in tiles:
        for k in (2, 3, 4, 5):
            out.append(dict(fusion=1, k_max=k, tile_bits=t))
        if dtype == "c64":  # twice the warps per block (a 14-dimensional tile fills an SM's shared memory)
            out.append(dict(fusion=1, k_max=2, tile_bits=t, threads=512))
        if allow_rotations:
            out.append(dict(fusion=2, k_max=2, tile_bits=t))
            if dtype == "c64":
                out.append(dict(fusion=2, k_max=2, tile_bits=t, threads=512))
    return out


def _key(gpu: str, n: int, dtype: str, family: str, prefix: int) -> str:
    return f"{gpu}|n={n}|{dtype}|{family}|prefix={prefix}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _save(d):
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def tune(n: int, gates, dtype: str = "c64", prefix: int = 1_000_000, allow_rotations: bool = True,
         use_cache: bool = True, verbose: bool = False):
    """Return (best_config, report) for running `gates` on an n-qubit state."""
    import torch
    gpu = torch.cuda.get_device_name()
    family = "rotations+paper" if allow_rotations else "paper"
    g = gates[: min(len(gates), prefix)]
    key = _key(gpu, n, dtype, family, len(g))
    cache = _load() if use_cache else {}
    if key in cache:
        return cache[key]["best"], cache[key]
    report = []
    stream = torch.cuda.current_stream()
    for cfg in candidates(n, dtype, allow_rotations):
        sim = qs.Sim(n, dtype, stream=stream, config=cfg)
        t0 = time.perf_counter()
        prog = sim.compile(g)
        t_compile = time.perf_counter() - t0
        sim.run(prog)
        sim.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.run(prog)
        sim.run(prog)
        e1.record(stream)
        sim.sync()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 2
        info = prog.info()
        report.append(dict(config=cfg, ms=ms, gates_per_s=len(g) / (ms / 1e3), passes=info["passes"],
                           fused_ops=info["fused_ops"], compile_s=t_compile))
        if verbose:
            print(report[-1], flush=True)
        prog.free()
        sim.close()
    best = min(report, key=lambda r: r["ms"])["config"]
    entry = dict(best=best, report=report, gpu=gpu, when=time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()))
    cache = _load()
    cache[key] = entry
    try:
        _save(cache)
    except OSError:
        pass
    return best, entry


def tune_batch(batch, circuits, dtype: str = "c64", allow_rotations: bool = True, prefix: int = 200_000,
               use_cache: bool = True):
    """Tune once per distinct width of a batch (on the first instance of that
    width, through a single-state context) and set that configuration on every
    instance of the width (qsim_batch_set_instance_config); compile afterwards.
    Returns {n: best_config}."""
    first = {}
    for i, c in enumerate(circuits):
        first.setdefault(batch.n[i], c)
    best = {}
    for n, c in sorted(first.items()):
        best[n], _ = tune(n, c.gates, dtype, prefix=prefix, allow_rotations=allow_rotations, use_cache=use_cache)
    for i in range(len(batch)):
        batch.set_instance_config(i, **best[batch.n[i]])
    return best
