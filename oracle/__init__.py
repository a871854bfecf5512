"""CPU oracle of the microcircuit step loop (ctypes wrapper around oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the CPU
baseline leg of bench.py, never by the simulator library.  All arithmetic is in
oracle.c; this module marshals arguments and owns the arrays.

Functions mirror the paper's steps:
  constants / step_constants  -- §2.2 equations for w_f, p11, p22, p21
  pop_sizes / pair_count      -- Table params2 sizes, the N_pre N_post p count (§2.2)
  build_network               -- synapse sampling with replacement, grouped by sender (§2.2, §3.5)
  initial_u                   -- u_init Gaussians (Table params2)
  poisson_table / poisson_count_at / draws -- thalamic Poisson drive (§2.2)
  lif_trace                   -- one neuron under a given input (Listing push, Eqs. mem/psc/ref)
  Sim.run                     -- the full deferred-push step loop (Listings push, push2; §3.2 ring)
  SimMT.run                   -- the same loop on host threads that own target ranges (cpu_mt.c),
                                 a CPU timing baseline with the oracle's raster
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MAX_POPS = 8
MAX_OVR = 4
D_MAX = 64
PKMAX = 24


def build(force: bool = False) -> str:
    """Compile oracle.c with FMA contraction and fast-math off."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-Wall", "-Wextra", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class OrModel(C.Structure):
    _fields_ = [
        ("n_pops", C.c_int32), ("n_ovr", C.c_int32),
        ("dt_ms", C.c_double), ("C_m_pF", C.c_double), ("tau_m_ms", C.c_double),
        ("tau_ref_ms", C.c_double), ("tau_syn_ms", C.c_double),
        ("u_rest_mV", C.c_double), ("u_reset_mV", C.c_double), ("u_thr_mV", C.c_double),
        ("nu_th_hz", C.c_double), ("w_ext_mV", C.c_double),
        ("n_full", C.c_int64 * MAX_POPS),
        ("k_ext", C.c_double * MAX_POPS),
        ("u0_mean", C.c_double * MAX_POPS), ("u0_sd", C.c_double * MAX_POPS),
        ("w_mean", C.c_double * MAX_POPS), ("w_sd", C.c_double * MAX_POPS),
        ("d_mean", C.c_double * MAX_POPS), ("d_sd", C.c_double * MAX_POPS),
        ("conn_p", (C.c_double * MAX_POPS) * MAX_POPS),
        ("ovr_src", C.c_int32 * MAX_OVR), ("ovr_tgt", C.c_int32 * MAX_OVR),
        ("ovr_mean", C.c_double * MAX_OVR), ("ovr_sd", C.c_double * MAX_OVR),
    ]


def _model(m) -> OrModel:
    s = OrModel()
    s.n_pops = m.n_pops
    s.n_ovr = len(m.overrides)
    for f in ("dt_ms", "C_m_pF", "tau_m_ms", "tau_ref_ms", "tau_syn_ms", "u_rest_mV",
              "u_reset_mV", "u_thr_mV", "nu_th_hz", "w_ext_mV"):
        setattr(s, f, float(getattr(m, f)))
    for b in range(m.n_pops):
        s.n_full[b] = int(m.n_full[b])
        s.k_ext[b] = float(m.k_ext[b])
        s.u0_mean[b] = float(m.u0_mean_mV[b])
        s.u0_sd[b] = float(m.u0_sd_mV[b])
        s.w_mean[b] = float(m.w_mean_mV[b])
        s.w_sd[b] = float(m.w_sd_mV[b])
        s.d_mean[b] = float(m.d_mean_ms[b])
        s.d_sd[b] = float(m.d_sd_ms[b])
        for a in range(m.n_pops):
            s.conn_p[b][a] = float(m.conn_p[b][a])
    for o, (src, tgt, mu, sd) in enumerate(m.overrides):
        s.ovr_src[o], s.ovr_tgt[o], s.ovr_mean[o], s.ovr_sd[o] = src, tgt, mu, sd
    return s


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        P = C.POINTER
        vp = C.c_void_p
        L.or_philox4x64_10.argtypes = [P(C.c_uint64), P(C.c_uint64), P(C.c_uint64)]
        L.or_constants.argtypes = [P(OrModel), P(C.c_double)]
        L.or_step_constants.argtypes = [P(OrModel), P(C.c_float), P(C.c_int32)]
        L.or_pop_sizes.argtypes = [P(OrModel), C.c_int32, P(C.c_int64)]
        L.or_pair_count.argtypes = [P(OrModel), C.c_int32, C.c_int32, C.c_int32, C.c_int32]
        L.or_pair_count.restype = C.c_int64
        L.or_total_synapses.argtypes = [P(OrModel), C.c_int32, C.c_int32]
        L.or_total_synapses.restype = C.c_int64
        L.or_build.argtypes = [P(OrModel), C.c_int32, C.c_int32, C.c_uint64, vp, vp, vp, vp, vp]
        L.or_build.restype = C.c_int
        L.or_initial_u.argtypes = [P(OrModel), C.c_int32, C.c_uint64, vp]
        L.or_poisson_table.argtypes = [P(OrModel), C.c_int32, vp]
        L.or_poisson_count_at.argtypes = [P(OrModel), C.c_int32, C.c_uint64]
        L.or_poisson_count_at.restype = C.c_int32
        L.or_poisson_draws.argtypes = [P(OrModel), C.c_uint64, C.c_int32, C.c_int64, C.c_int64,
                                       C.c_int64, vp]
        L.or_lif_trace.argtypes = [P(OrModel), C.c_float, C.c_float, C.c_int32, C.c_int64, vp, vp,
                                   vp, vp, vp]
        L.or_run.argtypes = [P(OrModel), C.c_uint64, C.c_int64, vp, vp, vp, vp, vp, vp, vp, vp,
                             vp, C.c_int64, C.c_int64, vp, vp, C.c_int64, P(C.c_int64)]
        L.or_run.restype = C.c_int
        L.or_quantize_i8.argtypes = [C.c_int32, vp, C.c_int64, vp, vp, vp, vp, vp, vp]
        L.or_quantize_bf16.argtypes = [C.c_int64, vp, vp]
        L.or_run_f64.argtypes = L.or_run.argtypes  # weights double[S] in pA, ring double[DMAX*N]
        L.or_run_f64.restype = C.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------- helpers


def philox(ctr, key) -> np.ndarray:
    c = (C.c_uint64 * 4)(*[int(x) & (2**64 - 1) for x in ctr])
    k = (C.c_uint64 * 2)(*[int(x) & (2**64 - 1) for x in key])
    o = (C.c_uint64 * 4)()
    lib().or_philox4x64_10(c, k, o)
    return np.array(list(o), dtype=np.uint64)


def constants(m) -> dict:
    o = (C.c_double * 6)()
    lib().or_constants(C.byref(_model(m)), o)
    return dict(zip(("w_f", "p11", "p22", "beta", "gamma", "p21"), list(o)))


def step_constants(m) -> dict:
    f = (C.c_float * 5)()
    i = (C.c_int32 * 2)()
    lib().or_step_constants(C.byref(_model(m)), f, i)
    d = dict(zip(("p11", "p21", "p22", "theta", "u_reset"), [np.float32(x) for x in f]))
    d["t_ref"], d["w_ext_fx"] = int(i[0]), int(i[1])
    return d


def pop_sizes(m, scale_n: int) -> np.ndarray:
    o = (C.c_int64 * MAX_POPS)()
    lib().or_pop_sizes(C.byref(_model(m)), scale_n, o)
    return np.array(list(o)[: m.n_pops], dtype=np.int64)


def pop_offsets(m, scale_n: int) -> np.ndarray:
    return np.concatenate([[0], np.cumsum(pop_sizes(m, scale_n))]).astype(np.int64)


def pair_count(m, scale_n: int, scale_k: int, target: int, source: int) -> int:
    return int(lib().or_pair_count(C.byref(_model(m)), scale_n, scale_k, target, source))


def total_synapses(m, scale_n: int, scale_k: int) -> int:
    return int(lib().or_total_synapses(C.byref(_model(m)), scale_n, scale_k))


def poisson_table(m, pop: int) -> np.ndarray:
    out = np.zeros(PKMAX, dtype=np.uint64)
    lib().or_poisson_table(C.byref(_model(m)), pop, _p(out))
    return out


def poisson_count_at(m, pop: int, v: int) -> int:
    """T = #{k : v >= C_k} for a chosen 63-bit v (the inversion step of the draws)."""
    return int(lib().or_poisson_count_at(C.byref(_model(m)), pop, v))


def poisson_draws(m, seed: int, pop: int, t: int, i0: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.int32)
    lib().or_poisson_draws(C.byref(_model(m)), seed, pop, t, i0, n, _p(out))
    return out


def initial_u(m, scale_n: int, seed: int) -> np.ndarray:
    n = int(pop_sizes(m, scale_n).sum())
    out = np.zeros(n, dtype=np.float32)
    lib().or_initial_u(C.byref(_model(m)), scale_n, seed, _p(out))
    return out


def lif_trace(m, in_fx, U0: float = 0.0, I0: float = 0.0, R0: int = 0) -> dict:
    in_fx = np.ascontiguousarray(in_fx, dtype=np.int32)
    n = len(in_fx)
    U = np.zeros(n, np.float32)
    I = np.zeros(n, np.float32)
    R = np.zeros(n, np.int32)
    S = np.zeros(n, np.int32)
    lib().or_lif_trace(C.byref(_model(m)), np.float32(U0), np.float32(I0), R0, n, _p(in_fx), _p(U),
                       _p(I), _p(R), _p(S))
    return {"U": U, "I": I, "R": R, "spike": S}


@dataclass
class Network:
    """A network grouped by sending neuron: row i is row_ptr[i]..row_ptr[i+1]."""

    n: int
    pop_off: np.ndarray
    row_ptr: np.ndarray
    post: np.ndarray
    w_fx: np.ndarray
    delay: np.ndarray
    u0: np.ndarray
    w_pA: Optional[np.ndarray] = None  # currents in pA before rounding to 2^-12 pA (FP64 loop)


def build_network(m, scale_n: int, scale_k: int, seed: int, with_pA: bool = False) -> Network:
    """with_pA also keeps every synapse's current in pA before its rounding to 2^-12 pA
    (the FP64 loop's weights)."""
    off = pop_offsets(m, scale_n)
    n = int(off[-1])
    s = total_synapses(m, scale_n, scale_k)
    row_ptr = np.zeros(n + 1, np.int64)
    post = np.zeros(max(s, 1), np.int32)
    w = np.zeros(max(s, 1), np.int32)
    d = np.zeros(max(s, 1), np.uint8)
    w_pA = np.zeros(max(s, 1), np.float64) if with_pA else None
    rc = lib().or_build(C.byref(_model(m)), scale_n, scale_k, seed, _p(row_ptr), _p(post), _p(w), _p(d),
                        _p(w_pA) if with_pA else None)
    if rc != 0:
        raise MemoryError("oracle network build failed")
    return Network(n, off, row_ptr, post[:s], w[:s], d[:s], initial_u(m, scale_n, seed),
                   w_pA[:s] if with_pA else None)


def network_from_edges(n: int, pre, post, w_fx, delay, u0, pop_off=None, w_pA=None) -> Network:
    """A hand-made network (tests): edges grouped by sender, order kept within a row;
    w_pA optionally gives the FP64 loop's weights in pA (else w_fx / 4096)."""
    pre = np.asarray(pre, np.int64)
    order = np.argsort(pre, kind="stable")
    counts = np.bincount(pre, minlength=n) if len(pre) else np.zeros(n, np.int64)
    row_ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    if pop_off is None:
        pop_off = np.array([0, n], np.int64)
    return Network(n, np.asarray(pop_off, np.int64), row_ptr,
                   np.ascontiguousarray(np.asarray(post, np.int32)[order]),
                   np.ascontiguousarray(np.asarray(w_fx, np.int32)[order]),
                   np.ascontiguousarray(np.asarray(delay, np.uint8)[order]),
                   np.ascontiguousarray(np.asarray(u0, np.float32)),
                   None if w_pA is None else np.ascontiguousarray(np.asarray(w_pA, np.float64)[order]))


def quantize_i8(net: "Network", n_pops: int = 8):
    """Read-back weights of the int8 per-population-pair store, plus its tables."""
    out = np.zeros(max(1, len(net.w_fx)), np.int32)
    base = np.zeros(64, np.int32)
    step = np.zeros(64, np.int32)
    post = net.post if len(net.post) else np.zeros(1, np.int32)
    w = net.w_fx if len(net.w_fx) else np.zeros(1, np.int32)
    lib().or_quantize_i8(n_pops, _p(net.pop_off), net.n, _p(net.row_ptr), _p(post), _p(w), _p(out), _p(base),
                         _p(step))
    return out[: len(net.w_fx)], base.reshape(8, 8), step.reshape(8, 8)


def quantize_bf16(w_fx: np.ndarray) -> np.ndarray:
    w_fx = np.ascontiguousarray(w_fx, np.int32)
    out = np.zeros(max(1, len(w_fx)), np.int32)
    lib().or_quantize_bf16(len(w_fx), _p(w_fx if len(w_fx) else np.zeros(1, np.int32)), _p(out))
    return out[: len(w_fx)]


def with_weights(net: "Network", w_fx: np.ndarray) -> "Network":
    return Network(net.n, net.pop_off, net.row_ptr, net.post, np.ascontiguousarray(w_fx, np.int32), net.delay,
                   net.u0, net.w_pA)


class Sim:
    """State of one circuit under the oracle: U, I (FP32), R (steps), exact ring."""

    def __init__(self, m, net: Network, seed: int, fp64: bool = False):
        """fp64=True runs the same loop in FP64: neuron state, propagators, the weights in
        pA before rounding (net.w_pA, else w_fx / 4096) and a double ring."""
        self.m, self.net, self.seed = m, net, int(seed)
        self._cm = _model(m)
        self.fp64 = fp64
        n = net.n
        dt = np.float64 if fp64 else np.float32
        self.U = net.u0.astype(dt)
        self.I = np.zeros(n, dt)
        self.R = np.zeros(n, np.int32)
        self.W = np.zeros(D_MAX * n, np.float64 if fp64 else np.int64)
        if fp64:
            self.w_pA = net.w_pA if net.w_pA is not None else net.w_fx.astype(np.float64) / 4096.0
        self.t = 0
        self.status = 0

    def run(self, n_steps: int, raster_cap: Optional[int] = None):
        """Advance n_steps; returns (steps, neurons) of the spikes, sorted by (t, i)."""
        cap = raster_cap if raster_cap is not None else max(1024, 64 * self.net.n + 1024)
        cap = min(cap, max(1, n_steps) * max(1, self.net.n))
        rt = np.zeros(cap, np.int32)
        ri = np.zeros(cap, np.int32)
        nr = C.c_int64(0)
        net = self.net
        post = net.post if len(net.post) else np.zeros(1, np.int32)
        w = net.w_fx if len(net.w_fx) else np.zeros(1, np.int32)
        if self.fp64:
            w = self.w_pA if len(self.w_pA) else np.zeros(1, np.float64)
        d = net.delay if len(net.delay) else np.zeros(1, np.uint8)
        run = lib().or_run_f64 if self.fp64 else lib().or_run
        rc = run(C.byref(self._cm), self.seed, net.n, _p(net.pop_off), _p(net.row_ptr),
                          _p(post), _p(w), _p(d), _p(self.U), _p(self.I), _p(self.R), _p(self.W),
                          self.t, n_steps, _p(rt), _p(ri), cap, C.byref(nr))
        if rc < 0:
            raise MemoryError("oracle run failed")
        self.status = max(self.status, rc)
        if rc == 2:
            raise OverflowError("synaptic input left the int32 range")
        if rc == 1:
            raise OverflowError("oracle raster capacity exceeded")
        self.t += n_steps
        k = nr.value
        return rt[:k].copy(), ri[:k].copy()


# --------------------------------------------------------------------------- multithreaded baseline

_MT_SRC = os.path.join(_HERE, "cpu_mt.c")
_MT_LIB = os.path.join(_HERE, "liboracle_mt.so")
_mt = None


def build_mt(force: bool = False) -> str:
    """Compile cpu_mt.c (the oracle's definitions, thread-partitioned; OpenMP)."""
    newest = max(os.path.getmtime(_MT_SRC), os.path.getmtime(_SRC))
    if force or not os.path.exists(_MT_LIB) or os.path.getmtime(_MT_LIB) < newest:
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-Wall", "-Wextra", "-Wno-unused-function", _MT_SRC, "-o", _MT_LIB + ".tmp", "-lm"]
        subprocess.run(cmd, check=True, cwd=_HERE)
        os.replace(_MT_LIB + ".tmp", _MT_LIB)
    return _MT_LIB


def lib_mt():
    global _mt
    if _mt is None:
        L = C.CDLL(build_mt())
        vp = C.c_void_p
        L.mt_build.argtypes = [C.c_int32, C.c_int64, vp, vp, vp, vp]
        L.mt_build.restype = vp
        L.mt_free.argtypes = [vp]
        L.mt_run.argtypes = [C.POINTER(OrModel), C.c_uint64, vp, vp, vp, vp, vp, vp, C.c_int64, C.c_int64, vp,
                             vp, C.c_int64, C.POINTER(C.c_int64)]
        L.mt_run.restype = C.c_int
        _mt = L
    return _mt


class SimMT:
    """The step loop of Sim on `threads` host threads (a CPU timing baseline): the same
    raster and state as Sim, with an int32 ring."""

    def __init__(self, m, net: Network, seed: int, threads: int):
        self.m, self.net, self.seed, self.threads = m, net, int(seed), int(threads)
        self._cm = _model(m)
        n = net.n
        post = net.post if len(net.post) else np.zeros(1, np.int32)
        w = net.w_fx if len(net.w_fx) else np.zeros(1, np.int32)
        d = net.delay if len(net.delay) else np.zeros(1, np.uint8)
        self._h = lib_mt().mt_build(self.threads, n, _p(net.row_ptr), _p(post), _p(w), _p(d))
        if not self._h:
            raise MemoryError("thread partition failed")
        self.U = net.u0.astype(np.float32)
        self.I = np.zeros(n, np.float32)
        self.R = np.zeros(n, np.int32)
        self.W = np.zeros(D_MAX * n, np.int32)
        self.t = 0

    def run(self, n_steps: int, raster_cap: Optional[int] = None):
        cap = raster_cap if raster_cap is not None else max(1024, 64 * self.net.n + 1024)
        cap = min(cap, max(1, n_steps) * max(1, self.net.n))
        rt = np.zeros(cap, np.int32)
        ri = np.zeros(cap, np.int32)
        nr = C.c_int64(0)
        rc = lib_mt().mt_run(C.byref(self._cm), self.seed, self._h, _p(self.net.pop_off), _p(self.U), _p(self.I),
                             _p(self.R), _p(self.W), self.t, n_steps, _p(rt), _p(ri), cap, C.byref(nr))
        if rc < 0:
            raise MemoryError("baseline run failed")
        if rc == 1:
            raise OverflowError("raster capacity exceeded")
        self.t += n_steps
        k = nr.value
        return rt[:k].copy(), ri[:k].copy()

    def __del__(self):
        try:
            if self._h:
                lib_mt().mt_free(self._h)
                self._h = None
        except Exception:
            pass
