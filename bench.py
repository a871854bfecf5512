"""Benchmark of the full-scale Potjans-Diesmann microcircuit step loop on GB300.

One bench step = 1,024 simulation steps of 0.1 ms (102.4 ms of biological time: one
launch of the resident engine, by default, or one CUDA-graph replay) of the full microcircuit (77,169 neurons, 284,811,022 synapses,
seed 1 + rank), so the default --steps 100 covers the paper's 10 s runs (§4).  Prints
one JSON line.

  value     recurrent synaptic events/s (sum of the spikers' out-degrees / seconds),
            device-timed with CUDA events around the snn_step_n calls
  rtf       real-time factor = wall time / biological time (§4.2)
  events_incl_thalamic  value plus the thalamic drive's expected input events
            (N_b K_ext,b nu_th per biological second, over the same wall time)
  e2e       the same metric through the public API with the raster read back to
            host memory every bench step (snn_step_n + snn_collect_spikes, which
            reads the previous bench step's spikes while the GPU runs this one)
  roofline  the dominant kernel's algorithmic bytes per launch / its average
            CUDA-event duration, against the measured HBM copy bandwidth
  cpu_baseline  the CPU oracle (single thread) on a bounded sample of the workload,
            and in its `multithreaded` entry the same step on every host core
  energy    the GPU board's energy counter over the timed region / recurrent events
Further objects: delivery_saturating (phase 2 alone over 2,048-20,480 random senders,
plain and target-blocked records), compressed_records (int8, bf16, blocked forms) and
workloads (32 uneven circuits in autotuned circuit groups; the 4x-scale circuit in
plain and int8 records).

--impl reference times the CPU oracle itself on the same workload (rank 0 only).
Under torchrun with N > 1, every rank simulates its own circuit (replicas: the
method has no data-path exchange on one circuit); value sums events over ranks and
divides by the slowest rank's time.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workload  # noqa: E402

TICKS_PER_STEP = 1024
UPDATE_BYTES_PER_NEURON = 26   # U r/w 8 + I r/w 8 + R r/w 2 + ring slot read + clear 8
EVENT_BYTES = 13               # tgt 4 + w 4 + delay 1 read + 4-byte ring reduction
SPIKE_BYTES = 20               # row_ptr pair 16 + queue entry 4
WORKLOAD = "pd_full"
METRIC = "synaptic events/s and real-time factor (full microcircuit, 1 GB300), % HBM roofline"


def _kernel_sources_hash(files=("kernels.cu", "internal.hpp")) -> str:
    """Hash of the code lines (comment-only and blank lines ignored) of kernel sources."""
    import hashlib

    csrc = os.path.join(ROOT, "paper_2405_02019_gb300", "csrc")
    lines = []
    for f in files:
        for line in open(os.path.join(csrc, f), encoding="utf-8"):
            code = line.strip()
            if code and not code.startswith("//"):
                lines.append(code)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()[:16]


# the sources each recorded kernel is built from
_RESIDENT_KERNELS = ("k_resident", "k_deliver_regions")


def _recorded_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu record, only if the kernel's sources
    are unchanged since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if kernel in _RESIDENT_KERNELS:
        valid = d.get("resident_sha256_16") == _kernel_sources_hash(("resident.cu", "internal.hpp"))
    else:
        valid = d.get("kernels_sha256_16") == _kernel_sources_hash()
    if not valid or kernel not in d:
        return None
    return d[kernel].get("dram_bytes_per_launch")


def thalamic_events_per_bio_s(model, pop_offsets) -> float:
    """Expected thalamic input events per biological second: every neuron of population
    b receives K_ext,b independent Poisson inputs at nu_th (§2.2).  The step loop draws
    their per-step sums from counter-based Poisson streams, so they are not counted on
    the device; this is their expectation."""
    n = np.diff(np.asarray(list(pop_offsets)[: model.n_pops + 1], dtype=np.int64))
    return float((n * np.asarray(model.k_ext[: model.n_pops], dtype=np.float64) * model.nu_th_hz).sum())


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.proc is None:
            return
        time.sleep(0.2)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in self.rows for j in range(4) if r[3 + j].lower() == "active"})
        pw = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows),
                "power_w_mean": float(np.mean(pw)) if pw else None}


class EnergyCounter:
    """The GPU's cumulative energy counter (NVML, millijoules since the driver loaded),
    read before and after the timed region through ctypes; None where NVML or the
    counter is unavailable.  Reads only."""

    def __init__(self, gpu_index: int):
        import ctypes as C

        self.mj = None
        try:
            self.lib = C.CDLL("libnvidia-ml.so.1")
            if self.lib.nvmlInit_v2() != 0:
                raise OSError("nvmlInit")
            self.dev = C.c_void_p()
            if self.lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(gpu_index), C.byref(self.dev)) != 0:
                raise OSError("handle")
        except (OSError, AttributeError):
            self.lib = None

    def read(self):
        import ctypes as C

        if self.lib is None:
            return None
        v = C.c_ulonglong()
        return int(v.value) if self.lib.nvmlDeviceGetTotalEnergyConsumption(self.dev, C.byref(v)) == 0 else None


def _dist():
    import torch.distributed as dist

    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1 and not dist.is_initialized():
        import torch

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def _max_over_ranks(x: float, ws: int, device=None) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(x: float, ws: int, device=None) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def _barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def cpu_oracle_sample(model, wl, ticks: int):
    """Time the oracle (single thread) on the first `ticks` steps of the workload."""
    import oracle

    oracle.build()
    t0 = time.perf_counter()
    onet = oracle.build_network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed)
    build_s = time.perf_counter() - t0
    sim = oracle.Sim(model, onet, wl.seed)
    t0 = time.perf_counter()
    st, si = sim.run(ticks)
    secs = time.perf_counter() - t0
    outdeg = np.diff(onet.row_ptr)
    events = int(outdeg[si].sum())
    return {"value": events / secs, "unit": "synaptic events/s", "cores": 1, "kind": "oracle",
            "sample": f"first {ticks} steps ({ticks * 0.1:.0f} ms biological) of {wl.name}, seed {wl.seed}, "
                      f"network build excluded ({build_s:.1f} s)",
            "rtf": secs / (ticks * model.dt_ms * 1e-3), "seconds": secs, "events": events,
            "spikes": int(len(st))}, onet, sim


def cpu_mt_sample(model, wl, onet, ticks: int):
    """The oracle's step on every host core (oracle/cpu_mt.c: neurons and ring split by
    thread-owned target ranges, no atomics; same raster as the oracle), first `ticks`
    steps of the workload."""
    import oracle

    threads = os.cpu_count() or 1
    try:
        oracle.build_mt()
    except Exception as e:  # no OpenMP toolchain on this host
        return {"unavailable": f"could not build the multithreaded baseline: {e}"}
    t0 = time.perf_counter()
    sim = oracle.SimMT(model, onet, wl.seed, threads)
    prep = time.perf_counter() - t0
    t0 = time.perf_counter()
    st, si = sim.run(ticks)
    secs = time.perf_counter() - t0
    events = int(np.diff(onet.row_ptr)[si].sum())
    return {"value": events / secs, "unit": "synaptic events/s", "cores": threads, "kind": "oracle, thread-partitioned",
            "sample": f"first {ticks} steps of {wl.name}, seed {wl.seed}; partition by target range {prep:.1f} s, "
                      f"not timed", "rtf": secs / (ticks * model.dt_ms * 1e-3), "seconds": secs, "events": events}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    model = workload.microcircuit_model()
    wl = workload.WORKLOADS[WORKLOAD]
    import oracle

    oracle.build()
    onet = oracle.build_network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed)
    sim = oracle.Sim(model, onet, wl.seed)
    outdeg = np.diff(onet.row_ptr)
    ticks = args.reference_ticks
    for _ in range(args.warmup):
        sim.run(ticks)
    events = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, si = sim.run(ticks)
        events += int(outdeg[si].sum())
    secs = time.perf_counter() - t0
    value = events / secs
    bio = args.steps * ticks * model.dt_ms * 1e-3
    line = {
        "impl": "reference", "metric": METRIC,
        "value": value, "unit": "synaptic events/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/i32", "data": "synthetic (PD microcircuit sampled from the paper's tables)",
        "config": {"workload": f"{wl.name}: 77,169 neurons, 284,811,022 synapses, dt 0.1 ms, seed {wl.seed}",
                   "ticks_per_step": ticks},
        "rtf": secs / bio,
        "cpu_baseline": {"value": value, "unit": "synaptic events/s", "cores": 1, "kind": "oracle",
                         "sample": f"{ticks} steps per bench step after {args.warmup * ticks} warm-up steps"},
        "e2e": {"value": value, "unit": "synaptic events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2405_02019_gb300 as snn

    model = workload.microcircuit_model()
    wl = workload.WORKLOADS[WORKLOAD]
    seed = wl.seed + rank
    tps = args.ticks_per_step
    t0 = time.perf_counter()
    engine = {"default": snn.ENGINE_DEFAULT, "graph": snn.ENGINE_GRAPH, "persistent": snn.ENGINE_PERSISTENT,
              "pipelined": snn.ENGINE_PIPELINED, "resident": snn.ENGINE_RESIDENT}[args.engine]
    # the compressed forms, batches and the 4x circuit run where the resident engine does not
    others = snn.ENGINE_DEFAULT if engine == snn.ENGINE_RESIDENT else engine
    engine_name = {snn.ENGINE_GRAPH: "graph", snn.ENGINE_PERSISTENT: "persistent", snn.ENGINE_PIPELINED: "pipelined",
                   snn.ENGINE_RESIDENT: "resident"}
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, seed, steps_per_graph=tps,
                      raster_capacity=1 << 25, device=dev, engine=engine)
    build_s = time.perf_counter() - t0
    info = net.info()
    stream = torch.cuda.current_stream(dev)

    # warm-up
    net.step(args.warmup * tps)
    net.read_spikes()
    e0 = net.info().events_read
    s0 = net.info().spikes_read

    # device-timed region
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    _barrier(ws)
    torch.cuda.synchronize(dev)
    energy = EnergyCounter(local)
    with ClockSampler(local) as clk:
        mj0 = energy.read()
        if args.profile_region == "timed":
            torch.cuda.profiler.start()
        start.record(stream)
        for _ in range(args.steps):
            net.step(tps)
        end.record(stream)
        torch.cuda.synchronize(dev)
        if args.profile_region == "timed":
            torch.cuda.profiler.stop()
        mj1 = energy.read()
    _barrier(ws)
    ms = start.elapsed_time(end)
    net.read_spikes()
    inf = net.info()
    events = inf.events_read - e0
    spikes = inf.spikes_read - s0
    secs_max = _max_over_ranks(ms / 1e3, ws, dev)
    events_all = _sum_over_ranks(float(events), ws, dev)
    value = events_all / secs_max
    bio_s = args.steps * tps * model.dt_ms * 1e-3
    rtf = secs_max / bio_s
    thal_bio = thalamic_events_per_bio_s(model, inf.pop_offsets)

    # end to end through the public API: step + raster read into host memory per bench step
    _barrier(ws)
    torch.cuda.synchronize(dev)
    e_e0 = net.info().events_read
    d2h = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        net.step(tps)
        st, si = net.collect_spikes()  # the previous bench step's spikes, while this one runs
        d2h += 8 * len(st) + 4
    st, si = net.read_spikes()  # the last bench step's
    d2h += 8 * len(st) + 64
    e2e_s = time.perf_counter() - t0
    e2e_events = net.info().events_read - e_e0
    e2e_s = _max_over_ranks(e2e_s, ws, dev)
    e2e_value = _sum_over_ranks(float(e2e_events), ws, dev) / e2e_s

    # per-kernel durations (CUDA events on the launching stream) for the roofline
    prof_ticks = args.profile_ticks
    net.read_spikes()
    pe0, ps0 = net.info().events_read, net.info().spikes_read
    ms_u, ms_d = net.profile_steps(prof_ticks)
    net.read_spikes()
    pe = net.info().events_read - pe0
    pspk = net.info().spikes_read - ps0
    n = info.n_neurons
    upd_bytes = UPDATE_BYTES_PER_NEURON * n
    dlv_bytes = (EVENT_BYTES * pe + SPIKE_BYTES * pspk) / prof_ticks
    upd_gbs = upd_bytes / (ms_u / prof_ticks * 1e-3) / 1e9
    dlv_gbs = dlv_bytes / (ms_d / prof_ticks * 1e-3) / 1e9 if ms_d > 0 else 0.0  # resident: one launch, both phases
    peak, peak_kind = _peaks()
    kernels = {
        "k_update": {"avg_us": ms_u / prof_ticks * 1e3, "bytes_per_launch": upd_bytes, "gbs": upd_gbs,
                     "share": ms_u / (ms_u + ms_d)},
        "k_deliver": {"avg_us": ms_d / prof_ticks * 1e3, "bytes_per_launch": dlv_bytes, "gbs": dlv_gbs,
                      "share": ms_d / (ms_u + ms_d), "events_per_launch": pe / prof_ticks,
                      "spikes_per_launch": pspk / prof_ticks},
    }
    if info.engine == snn.ENGINE_PIPELINED:
        # the timed region is k_step launches only (plus one k_advance per graph): its
        # average launch duration there is the region's time per step
        step_bytes = UPDATE_BYTES_PER_NEURON * n + (EVENT_BYTES * events + SPIKE_BYTES * spikes) / (args.steps * tps)
        avg_s = secs_max / (args.steps * tps)
        kernels = {"k_step": {"avg_us": avg_s * 1e6, "bytes_per_launch": step_bytes,
                              "gbs": step_bytes / avg_s / 1e9, "share": 1.0,
                              "events_per_launch": events / (args.steps * tps),
                              "spikes_per_launch": spikes / (args.steps * tps),
                              "isolated_avg_us": ms_u / prof_ticks * 1e3,
                              "note": "avg_us over the timed graph replays; isolated_avg_us brackets single "
                                      "launches with CUDA events (launch latency included)"}}
        dom = "k_step"
    elif info.engine in (snn.ENGINE_PERSISTENT, snn.ENGINE_RESIDENT):
        # one cooperative launch per bench step: all of its steps' algorithmic bytes over its duration
        per_launch = tps * (upd_bytes + (EVENT_BYTES * events + SPIKE_BYTES * spikes) / (args.steps * tps))
        dom = "k_persistent" if info.engine == snn.ENGINE_PERSISTENT else "k_resident"
        kernels = {dom: {"avg_us": secs_max * 1e6 / args.steps, "bytes_per_launch": per_launch,
                         "gbs": per_launch / (secs_max / args.steps) / 1e9, "share": 1.0,
                         "steps_per_launch": tps, "us_per_step": secs_max * 1e6 / (args.steps * tps),
                         "events_per_launch": events / args.steps, "spikes_per_launch": spikes / args.steps}}
        if info.engine == snn.ENGINE_PERSISTENT:
            kernels[dom]["isolated_k_step_avg_us"] = ms_u / prof_ticks * 1e3
            kernels[dom]["note"] = ("isolated_k_step_avg_us: the same step as one k_step launch, bracketed with "
                                    "CUDA events (launch latency included)")
        else:
            kernels[dom]["note"] = ("one cooperative launch per bench step (1,024 steps); its algorithmic bytes "
                                    "count the ring row and neuron state per neuron-step although the kernel keeps "
                                    "both on chip; its DRAM traffic is the synapse segments it reads")
    else:
        dom = "k_update" if ms_u >= ms_d else "k_deliver"
    traffic = _recorded_traffic(dom)
    roofline = {"kernel": dom, "bound": "hbm", "achieved": kernels[dom]["gbs"], "peak": peak, "unit": "GB/s",
                "frac": kernels[dom]["gbs"] / peak, "traffic": traffic,
                "peak_source": f"{peak_kind} hbm_gbs (copy bandwidth, burst)"}

    # delivery alone at saturating load: random senders of the same network, fresh list
    # per launch (rows >> L2 for the larger lists); the ring is left modified, so this
    # runs after every other measurement
    sat = []
    outdeg = net.out_degrees()
    snet = net
    if info.engine == snn.ENGINE_RESIDENT:
        # the resident engine stores its records block-major (no sender rows): phase 2
        # alone runs on the row-major network of the same spec and seed
        net.close()
        snet = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, seed, steps_per_graph=tps,
                           raster_capacity=1 << 25, device=dev, engine=others)
    rng = np.random.default_rng(1234 + rank)
    for nsp in args.saturating:
        ms_list, ev_list = [], []
        for r in range(args.saturating_reps + 2):
            spk = rng.integers(0, n, nsp).astype(np.int32)
            dev_spk = torch.from_numpy(spk).to(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            if args.profile_region == "saturating":
                torch.cuda.profiler.start()
            e0.record(stream)
            snet.deliver_spikes(dev_spk, 0)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if args.profile_region == "saturating":
                torch.cuda.profiler.stop()
            if r >= 2:
                ms_list.append(e0.elapsed_time(e1))
                ev_list.append(int(outdeg[spk].sum()))
        ms_avg = float(np.median(ms_list))  # median over the repetitions: robust to a stray slow launch
        ev_avg = float(np.mean(ev_list))
        nbytes = EVENT_BYTES * ev_avg + SPIKE_BYTES * nsp
        sat.append({"spikers": nsp, "events": ev_avg, "ms": ms_avg, "bytes": nbytes,
                    "gbs": nbytes / (ms_avg * 1e-3) / 1e9, "frac": nbytes / (ms_avg * 1e-3) / 1e9 / peak,
                    "reductions_per_s": ev_avg / (ms_avg * 1e-3)})

    snet.close()

    # the paper's RTF is the mean over 10 random network instances (§4): the same step loop
    # on network seeds seed .. seed + n - 1, each after one warm-up bench step
    instances = []
    for k in range(args.seeds):
        sk = seed + k
        inet = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, sk, steps_per_graph=tps,
                           raster_capacity=1 << 25, device=dev, engine=engine)
        inet.step(tps)
        inet.read_spikes()
        ie0 = inet.info().events_read
        torch.cuda.synchronize(dev)
        i0 = torch.cuda.Event(enable_timing=True)
        i1 = torch.cuda.Event(enable_timing=True)
        i0.record(stream)
        for _ in range(args.seed_steps):
            inet.step(tps)
        i1.record(stream)
        torch.cuda.synchronize(dev)
        isecs = i0.elapsed_time(i1) * 1e-3
        inet.read_spikes()
        iev = inet.info().events_read - ie0
        instances.append({"seed": sk, "events_per_s": iev / isecs,
                          "rtf": isecs / (args.seed_steps * tps * model.dt_ms * 1e-3)})
        inet.close()
    seeds_summary = None
    if instances:
        ev = np.array([x["events_per_s"] for x in instances])
        rt = np.array([x["rtf"] for x in instances])
        seeds_summary = {"n": len(instances), "steps_each": args.seed_steps * tps,
                         "events_per_s_mean": float(ev.mean()), "events_per_s_sd": float(ev.std(ddof=1)) if len(ev) > 1 else 0.0,
                         "rtf_mean": float(rt.mean()), "rtf_sd": float(rt.std(ddof=1)) if len(rt) > 1 else 0.0,
                         "realtime_x_mean": float((1.0 / rt).mean()), "instances": instances,
                         "note": "network seeds seed .. seed + n - 1 (the paper's RTF is the mean over 10 instances, "
                                 "section 4); each timed over steps_each steps after one warm-up bench step"}
    torch.cuda.empty_cache()

    # compressed synapse records on the same workload: step time and saturating delivery
    forms = {}
    blocked_formats = (snn.RECORD_BLOCKED6, snn.RECORD_BLOCKED4, snn.RECORD_BLOCKED8)
    for fname, fmt in (("int8_pair", snn.RECORD_PACKED_I8), ("bf16", snn.RECORD_PACKED_BF16),
                       ("blocked6", snn.RECORD_BLOCKED6), ("blocked4", snn.RECORD_BLOCKED4),
                       ("blocked8", snn.RECORD_BLOCKED8)):
        if fname not in args.forms:
            continue
        feng = snn.ENGINE_DEFAULT if fmt in blocked_formats else others
        fnet = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, seed, steps_per_graph=tps,
                           raster_capacity=1 << 25, device=dev, engine=feng, record_format=fmt)
        fnet.step(args.warmup * tps)
        fnet.read_spikes()
        fe0 = fnet.info().events_read
        torch.cuda.synchronize(dev)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.form_steps):
            fnet.step(tps)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        fsecs = a0.elapsed_time(a1) * 1e-3
        fnet.read_spikes()
        fev = fnet.info().events_read - fe0
        fsat = []
        finfo = fnet.info()
        blocked = fmt in blocked_formats
        for nsp in (args.saturating if blocked else args.saturating[-1:]):
            ms_l, ev_l, nnz_l = [], [], []
            ring = fnet.device_view("ring", torch.int32, 64 * int(fnet.layout().n_neurons_padded)) if blocked else None
            for r in range(args.saturating_reps + 2):
                spk_np = rng.integers(0, n, nsp).astype(np.int32)
                spk = torch.from_numpy(spk_np).to(dev)
                if blocked:
                    ring.zero_()  # so that the entries this launch updates can be counted
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize(dev)
                if args.profile_region == "saturating":
                    torch.cuda.profiler.start()
                e0.record(stream)
                fnet.deliver_spikes(spk, 0)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                if args.profile_region == "saturating":
                    torch.cuda.profiler.stop()
                if r >= 2:
                    ms_l.append(e0.elapsed_time(e1))
                    ev_l.append(int(outdeg[spk_np].sum()))
                    if blocked:
                        nnz_l.append(int(torch.count_nonzero(ring).item()))
            ms_avg, ev_avg = float(np.median(ms_l)), float(np.mean(ev_l))
            plain_ms = [p_["ms"] for p_ in sat if p_["spikers"] == nsp]
            pt = {"spikers": nsp, "events": ev_avg, "ms": ms_avg, "events_per_s": ev_avg / (ms_avg * 1e-3),
                  "speedup_vs_plain": float(plain_ms[0] / ms_avg) if plain_ms else None}
            if blocked:
                # the blocked kernel's own algorithmic bytes: its record bytes per event; per
                # sender its list entry, row start and block-table row; 8 B (read + write)
                # per ring entry it updates
                nnz = float(np.mean(nnz_l))
                nb = finfo.target_blocks
                nbytes = finfo.bytes_per_synapse * ev_avg + (12 + 2 * (nb + 1)) * nsp + 8 * nnz
                pt.update({"ring_entries_updated": nnz, "bytes": nbytes, "gbs": nbytes / (ms_avg * 1e-3) / 1e9,
                           "frac": nbytes / (ms_avg * 1e-3) / 1e9 / peak,
                           "plain_equivalent_gbs": (EVENT_BYTES * ev_avg + SPIKE_BYTES * nsp) / (ms_avg * 1e-3) / 1e9})
            fsat.append(pt)
        forms[fname] = {"bytes_per_synapse": finfo.bytes_per_synapse, "value": fev / fsecs,
                        "engine": engine_name[finfo.engine],
                        "unit": "synaptic events/s", "rtf": fsecs / (args.form_steps * tps * model.dt_ms * 1e-3),
                        "steps": args.form_steps * tps, "delivery_saturating": fsat,
                        "note": "raster bit-exact with the oracle on the read-back weights; statistics vs FP64 "
                                "in tests/test_precision_accuracy.py"}
        fnet.close()

    torch.cuda.empty_cache()

    # phase 2 alone on block-major records (the resident engine's layout): one CTA per
    # target block reads only its region, where consecutive senders' segments are
    # adjacent; the same random senders, and the same list sorted by sender
    regions = []
    if args.regions and args.saturating:
        rnet = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, seed, steps_per_graph=tps,
                           raster_capacity=1 << 25, device=dev, engine=snn.ENGINE_RESIDENT)
        rinfo = rnet.info()
        rring = rnet.device_view("ring", torch.int32, 64 * int(rnet.layout().n_neurons_padded))
        nblk = int(rinfo.target_blocks)
        for nsp in args.saturating:
            for order in ("random", "sorted"):
                ms_l, ev_l, nnz_l = [], [], []
                for r in range(args.saturating_reps + 2):
                    spk_np = rng.integers(0, n, nsp).astype(np.int32)
                    if order == "sorted":
                        spk_np.sort()
                    spk = torch.from_numpy(spk_np).to(dev)
                    rring.zero_()  # so that the entries this launch updates can be counted
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize(dev)
                    if args.profile_region == "regions":
                        torch.cuda.profiler.start()
                    e0.record(stream)
                    rnet.deliver_spikes(spk, 0)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    if args.profile_region == "regions":
                        torch.cuda.profiler.stop()
                    if r >= 2:
                        ms_l.append(e0.elapsed_time(e1))
                        ev_l.append(int(outdeg[spk_np].sum()))
                        nnz_l.append(int(torch.count_nonzero(rring).item()))
                ms_avg, ev_avg, nnz = float(np.median(ms_l)), float(np.mean(ev_l)), float(np.mean(nnz_l))
                # own bytes: 9 B per record (target, weight, delay); per sender its list
                # entry and its two segment offsets in every block's table; 8 B (read +
                # write) per ring entry updated
                nbytes = 9 * ev_avg + (4 + 8 * nblk) * nsp + 8 * nnz
                plain_ms = [p_["ms"] for p_ in sat if p_["spikers"] == nsp]
                regions.append({"spikers": nsp, "order": order, "events": ev_avg, "ms": ms_avg,
                                "events_per_s": ev_avg / (ms_avg * 1e-3), "bytes": nbytes,
                                "gbs": nbytes / (ms_avg * 1e-3) / 1e9, "frac": nbytes / (ms_avg * 1e-3) / 1e9 / peak,
                                "ring_entries_updated": nnz,
                                "speedup_vs_plain": float(plain_ms[0] / ms_avg) if plain_ms else None})
        rnet.close()
        del rring
        torch.cuda.empty_cache()

    def run_workload(label, circuits=None, wlx=None, fmt=snn.RECORD_PLAIN9, n_steps=None, tune=False, weng=None,
                     region=None):
        """Build, optionally autotune, warm up and time a workload; returns a summary.  With
        --profile-region equal to `region`, the timed region is bracketed by
        cudaProfilerStart/Stop (for ncu --profile-from-start off)."""
        t0 = time.perf_counter()
        weng = others if weng is None else weng
        if circuits is not None:
            xnet = snn.Network(model, circuits=circuits, steps_per_graph=tps, raster_capacity=1 << 27, device=dev,
                               engine=weng, record_format=fmt)
        else:
            xnet = snn.Network(model, wlx.scale_n_permille, wlx.scale_k_permille, wlx.seed + rank,
                               steps_per_graph=tps, raster_capacity=1 << 27, device=dev, engine=weng,
                               record_format=fmt)
        build = time.perf_counter() - t0
        tuned = None
        if tune and args.batched_groups >= 0:
            xnet.set_circuit_groups(args.batched_groups)  # fixed grouping, default schedule
        elif tune:
            from paper_2405_02019_gb300 import autotune

            tuned = autotune.autotune(xnet, steps=tps, cache_path=None)
        xnet.step(tps)
        xnet.read_spikes()
        x0 = xnet.info().events_read
        s0 = xnet.info().spikes_read
        nsteps = n_steps // tps * tps
        torch.cuda.synchronize(dev)
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        prof = region is not None and args.profile_region == region
        if prof:
            torch.cuda.profiler.start()
        b0.record(stream)
        xnet.step(nsteps)
        b1.record(stream)
        if prof:
            torch.cuda.synchronize(dev)
            torch.cuda.profiler.stop()
        torch.cuda.synchronize(dev)
        xsecs = b0.elapsed_time(b1) * 1e-3
        xnet.read_spikes()
        xi = xnet.info()
        ev = xi.events_read - x0
        out = {"workload": label, "engine": engine_name[xi.engine],
               "circuits_per_group": int(xi.circuits_per_group),
               "neurons": int(xi.n_neurons), "synapses": int(xi.n_synapses),
               "circuits": int(xi.n_circuits), "bytes_per_synapse": int(xi.bytes_per_synapse),
               "steps": nsteps, "value": ev / xsecs, "unit": "synaptic events/s",
               "us_per_step": xsecs / nsteps * 1e6, "rtf": xsecs / (nsteps * model.dt_ms * 1e-3),
               "spikes_per_step": (xi.spikes_read - s0) / nsteps, "events_per_step": ev / nsteps,
               "build_s": build}
        if tuned is not None:
            out["autotuned_schedule"] = tuned["schedule"]
            out["autotune_timings"] = tuned["timings"]
        xnet.close()
        del xnet
        torch.cuda.empty_cache()
        return out

    extra = {}
    if "batched" in args.extra:
        bw = workload.batched_workloads(32, 2026, 20000)
        extra["batched"] = run_workload("32 PD circuits, neuron/in-degree scales U{100..1000} permille, seeds "
                                        "1000+c, 2 s each", circuits=[(w.scale_n_permille, w.scale_k_permille, w.seed)
                                                                      for w in bw],
                                        n_steps=args.batched_steps, tune=True, region="batched")
        extra["batched"]["speedup_vs_single_circuit"] = extra["batched"]["value"] / value
    if "x4" in args.extra:
        wx = workload.WORKLOADS["pd_x4"]
        extra["scaled_up_plain"] = run_workload("pd_x4 plain: 308,676 neurons, full in-degrees", wlx=wx,
                                                n_steps=args.x4_steps, region="x4")
        extra["scaled_up_int8"] = run_workload("pd_x4 packed int8 records", wlx=wx, fmt=snn.RECORD_PACKED_I8,
                                               n_steps=args.x4_steps)
        extra["scaled_up_int8"]["speedup_vs_plain"] = (extra["scaled_up_int8"]["value"] /
                                                       extra["scaled_up_plain"]["value"])

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, onet, _ = cpu_oracle_sample(model, wl, args.cpu_ticks)
        try:
            import multiprocessing

            cpu["host_cores_available"] = multiprocessing.cpu_count()
        except Exception:
            pass
        cpu["multithreaded"] = cpu_mt_sample(model, wl, onet, args.cpu_ticks)

    line = {
        "metric": METRIC,
        "value": value, "unit": "synaptic events/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs_max * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32/i32", "data": "synthetic (PD microcircuit sampled from the paper's tables)",
        "config": {"workload": f"{wl.name}: 77,169 neurons, 284,811,022 synapses, dt 0.1 ms, seed {wl.seed}+rank",
                   "ticks_per_step": tps, "bio_seconds": bio_s, "steps_per_graph": info.steps_per_graph,
                   "engine": engine_name[info.engine],
                   "deliver_blocks": info.deliver_blocks, "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 (2.56 GB synapse store); ring and neuron state are L2-resident by design"},
        "rtf": rtf, "realtime_x": 1.0 / rtf, "spikes_per_tick": spikes / (args.steps * tps),
        "instances": seeds_summary,
        "events_incl_thalamic": {
            "value": value + ws * thal_bio * bio_s / secs_max, "unit": "synaptic events/s",
            "thalamic_per_bio_second": thal_bio,
            "note": "recurrent events counted on the device plus the thalamic drive's expected events "
                    "(sum over populations of N_b K_ext,b nu_th per biological second)"},
        "events_per_tick": events / (args.steps * tps),
        "e2e": {"value": e2e_value, "unit": "synaptic events/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": d2h / args.steps,
                "note": "network uploaded once by snn_build_network (setup, untimed as in the paper's RTF); "
                        "every bench step enqueues 1,024 steps (snn_step_n) and moves the previous bench "
                        "step's raster to host memory while they run (snn_collect_spikes); a final "
                        "snn_read_spikes inside the timed region returns the last one"},
        "gpu_launches": args.steps * {snn.ENGINE_PERSISTENT: 1, snn.ENGINE_RESIDENT: 1, snn.ENGINE_PIPELINED: tps + 1,
                                      snn.ENGINE_GRAPH: 2 * tps + 1}[info.engine],
        "roofline": roofline, "kernels": kernels,
        "compressed_records": forms,
        "workloads": extra,
        "delivery_saturating": {"kernel": "k_deliver_list", "bound": "hbm", "peak": peak, "unit": "GB/s",
                                "traffic_20480": _recorded_traffic("k_deliver_list"),
                                "note": "phase 2 alone over random senders of the same network "
                                        "(13 B per event + 20 B per sender); int32 red.add into the ring",
                                "points": sat,
                                "blocked6": {"kernel": "k_deliver_blocked",
                                             "traffic_20480": _recorded_traffic("k_deliver_blocked"),
                                             "note": "one CTA per target block, sums in shared memory; frac on "
                                                     "its own bytes (6 B per event, sender index, 8 B per ring "
                                                     "entry updated)",
                                             "points": forms.get("blocked6", {}).get("delivery_saturating")},
                                "blocked4": {"kernel": "k_deliver_blocked",
                                             "traffic_20480": _recorded_traffic("k_deliver_blocked_bf16"),
                                             "note": "the same with bfloat16 weights (4 B per event)",
                                             "points": forms.get("blocked4", {}).get("delivery_saturating")},
                                "blocked8": {"kernel": "k_deliver_blocked",
                                             "traffic_20480": _recorded_traffic("k_deliver_blocked_8"),
                                             "note": "exact weights interleaved with the records (8 B per event): "
                                                     "one contiguous read per segment",
                                             "points": forms.get("blocked8", {}).get("delivery_saturating")},
                                "block_major": {"kernel": "k_deliver_regions",
                                                "note": "the resident engine's block-major records (9 B per event): "
                                                        "one CTA per target block reads its region's segments; frac "
                                                        "on its own bytes (records, per-sender offsets in every "
                                                        "block's table, 8 B per ring entry updated); random and "
                                                        "sorted sender lists",
                                                "points": regions}},
        "clocks": clk.summary(), "build_s": build_s,
        "paper_context": {"fpga_best_rtf": 0.79, "hardware": "Intel Agilex 7 FPGA (horiz/multi/s)"},
    }
    pw = line["clocks"].get("power_w_mean")
    if mj0 is not None and mj1 is not None and mj1 > mj0 and events > 0:
        # the energy-per-synaptic-event metric of Sec. 5 (whole board, as the paper's upper
        # bound): the GPU's energy counter over the timed region / recurrent events
        joules = (mj1 - mj0) * 1e-3
        line["energy"] = {"joules": joules, "power_w_mean": joules / (ms * 1e-3),
                          "nj_per_event": joules / events * 1e9,
                          "source": "NVML total energy counter, whole GPU board, over the timed region",
                          "power_w_sampled": pw,
                          "paper_context": "21 nJ (whole FPGA board, 44.9 W) / 9 nJ (fabric only)"}
    elif pw is not None and events > 0:
        # no energy counter: board power sampled over the timed region x its duration
        line["energy"] = {"power_w_mean": pw, "nj_per_event": pw * secs_max / events * 1e9,
                          "joules": pw * secs_max, "source": "nvidia-smi power.draw, whole GPU board",
                          "paper_context": "21 nJ (whole FPGA board, 44.9 W) / 9 nJ (fabric only)"}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--ticks-per-step", type=int, default=TICKS_PER_STEP)
    ap.add_argument("--profile-ticks", type=int, default=2000)
    ap.add_argument("--cpu-ticks", type=int, default=5000)
    ap.add_argument("--reference-ticks", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--saturating", type=int, nargs="*", default=[2048, 8192, 20480])
    ap.add_argument("--saturating-reps", type=int, default=5)
    ap.add_argument("--forms", nargs="*", default=["int8_pair", "bf16", "blocked6", "blocked4", "blocked8"])
    ap.add_argument("--extra", nargs="*", default=["batched", "x4"])
    ap.add_argument("--batched-steps", type=int, default=20480)
    ap.add_argument("--batched-groups", type=int, default=-1,
                    help="circuits per group for the batched workload instead of autotuning (-1: autotune)")
    ap.add_argument("--x4-steps", type=int, default=10240)
    ap.add_argument("--profile-region", choices=["none", "timed", "saturating", "regions", "batched", "x4"],
                    default="none",
                    help="bracket that region (the main timed region, the saturating delivery launches, or a "
                         "workload's timed region) with cudaProfilerStart/Stop")
    ap.add_argument("--form-steps", type=int, default=20)
    ap.add_argument("--regions", type=int, default=1, help="saturating delivery on block-major records (0: skip)")
    ap.add_argument("--seeds", type=int, default=10, help="network instances timed for the mean RTF (0: none)")
    ap.add_argument("--seed-steps", type=int, default=10, help="bench steps timed per instance")
    ap.add_argument("--engine", default="resident", choices=["default", "graph", "persistent", "pipelined", "resident"],
                    help="engine of the headline step loop (the resident engine: one launch per 1,024 steps)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
