"""Autotuner of the step kernels' launch schedule.

The schedule -- CTAs of the step kernel, delivery warps per CTA, steps per captured
graph (pipelined engine), or CTAs of the delivery kernel (graph engine), and for a
batch the circuits per group -- changes only speed, never results.  ``autotune`` times candidate schedules on the live
network between a checkpoint and its restore (so the dynamics are untouched, but the
host spike history restarts: read spikes before tuning), keeps the fastest, and
remembers it in a JSON cache keyed by GPU, network shape, record format and engine.
"""

from __future__ import annotations

import json
import os
from typing import Dict, Iterable, List, Optional

import numpy as np

from . import ENGINE_GRAPH, ENGINE_PIPELINED, Network

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "snn_gb300_schedules.json")


def candidates(net: Network, num_sms: int) -> List[Dict[str, int]]:
    info = net.info()
    groups = [0] + [g for g in (4, 8, 16) if g < info.n_circuits]
    if info.engine == ENGINE_PIPELINED:
        return [dict(grid_ctas=g, delivery_warps=w, steps_per_graph=s, circuits_per_group=c)
                for g in (num_sms, 2 * num_sms, 3 * num_sms) for w in (4, 8) for s in (1024,) for c in groups]
    if info.engine == ENGINE_GRAPH:
        return [dict(grid_ctas=g, delivery_warps=0, steps_per_graph=s, circuits_per_group=c)
                for g in (num_sms, 2 * num_sms, 4 * num_sms) for s in (1024,) for c in groups]
    return []


def _apply(net: Network, cand: Dict[str, int]) -> None:
    sched = {k: v for k, v in cand.items() if k != "circuits_per_group"}
    net.set_schedule(**sched)
    if "circuits_per_group" in cand:
        net.set_circuit_groups(cand["circuits_per_group"])


def _key(net: Network) -> str:
    import torch

    info = net.info()
    return "|".join(str(x) for x in (torch.cuda.get_device_name(net.device), info.n_neurons, info.n_synapses,
                                     info.record_format, info.engine, info.n_circuits))


def autotune(net: Network, trials: Optional[Iterable[Dict[str, int]]] = None, steps: int = 2048,
             cache_path: Optional[str] = DEFAULT_CACHE, use_cache: bool = True) -> Dict:
    """Pick the fastest schedule for `net` and apply it.  Returns the choice and the
    measured microseconds per step of every candidate."""
    import torch

    key = _key(net)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        _apply(net, cache[key]["schedule"])
        return cache[key]
    num_sms = torch.cuda.get_device_properties(net.device).multi_processor_count
    trials = list(trials) if trials is not None else candidates(net, num_sms)
    if not trials:
        return {"schedule": {}, "timings": []}
    blob = net.save_state()
    stream = torch.cuda.current_stream(net.device)
    timings = []
    for cand in trials:
        _apply(net, cand)
        net.step(steps)  # warm-up
        torch.cuda.synchronize(net.device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        net.step(steps)
        e1.record(stream)
        torch.cuda.synchronize(net.device)
        timings.append({"schedule": cand, "us_per_step": e0.elapsed_time(e1) * 1e3 / steps})
        net.read_spikes(allow_overflow=True)
    best = min(timings, key=lambda r: r["us_per_step"])
    net.load_state(blob)
    _apply(net, best["schedule"])
    result = {"schedule": best["schedule"], "us_per_step": best["us_per_step"], "timings": timings}
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        cache[key] = result
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return result
