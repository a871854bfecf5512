"""Long oracle runs that several GPU tests compare against.

Test infrastructure only.  Each run (network build plus the step loop, a few minutes
of one host core at full scale) starts in a background thread as soon as a test
session that needs it begins -- the oracle's C functions release the interpreter lock
-- so that the runs overlap each other and the GPU tests; a test then waits for the
result it needs.  Threads, not processes: nothing is forked after the first GPU call.
"""

from __future__ import annotations

import threading

import oracle
import workload

FULL_STEPS = 100_000  # 10 s of biological time, the paper's run length (§4)


class Run:
    def __init__(self, fn):
        self.result = None
        self.error = None
        self.thread = threading.Thread(target=self._go, args=(fn,), daemon=True)
        self.thread.start()

    def _go(self, fn):
        try:
            self.result = fn()
        except BaseException as e:  # re-raised by get()
            self.error = e

    def get(self):
        self.thread.join()
        if self.error is not None:
            raise self.error
        return self.result


def _full(seed: int, fp64: bool):
    def fn():
        m = workload.microcircuit_model()
        wl = workload.WORKLOADS["pd_full"]
        net = oracle.build_network(m, wl.scale_n_permille, wl.scale_k_permille, seed, with_pA=fp64)
        sim = oracle.Sim(m, net, seed, fp64=fp64)
        t, i = sim.run(FULL_STEPS, raster_cap=1 << 26)
        return {"net": net, "sim": sim, "t": t, "i": i}
    return fn


# name -> (test modules that use it, what it runs)
RUNS = {
    "full_fp32_seed1": (("test_long_parity_gpu",), _full(1, False)),
    "full_fp64_seed1": (("test_precision_accuracy",), _full(1, True)),
    "full_fp64_seed2": (("test_precision_accuracy",), _full(2, True)),
    "full_fp64_seed3": (("test_precision_accuracy",), _full(3, True)),
}
_started: dict[str, Run] = {}
_lock = threading.Lock()


def start(name: str) -> Run:
    with _lock:
        if name not in _started:
            oracle.build()
            _started[name] = Run(RUNS[name][1])
        return _started[name]


def get(name: str):
    return start(name).get()


def start_for_modules(modules) -> None:
    """Start every run that one of the given test modules uses."""
    for name, (users, _) in RUNS.items():
        if any(u in modules for u in users):
            start(name)
