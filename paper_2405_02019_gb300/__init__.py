"""Python binding of the GB300 microcircuit simulator (include/snn.h).

Argument marshalling only: every step of the simulation runs in libsnn.so's CUDA
kernels.  PyTorch provides the device arena (torch.empty on the GPU) and the stream.

Low-level functions carry the C names (snn_query_sizes, snn_build_network,
snn_step_n, snn_read_spikes, snn_read_rates, snn_get_info, snn_get_layout,
snn_profile_steps, snn_destroy); ``Network`` wraps them.
"""

from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import _abi
from ._abi import (ABI_VERSION, D_MAX, ENGINE_DEFAULT, ENGINE_GRAPH, ENGINE_PERSISTENT, ENGINE_PIPELINED,  # noqa: F401
                   ENGINE_RESIDENT,
                   RECORD_BLOCKED4, RECORD_BLOCKED6, RECORD_BLOCKED8, RECORD_PACKED_BF16, RECORD_PACKED_I8, RECORD_PLAIN9,
                   FX_SHIFT, MAX_POPS, POISSON_KMAX, SNN_EOVERFLOW, SNN_ETIMEOUT, load, snn_info, snn_layout,
                   snn_sizes, snn_spec)


class SnnError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        msg = lib.snn_last_error().decode(errors="replace")
        super().__init__(f"{where}: {_abi.STATUS.get(code, code)} ({msg})")
        self.code = code


def _check(code: int, where: str) -> int:
    if code != 0:
        raise SnnError(code, where)
    return code


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def model_struct(m) -> _abi.snn_model:
    """snn_model from a workload.Model-like object."""
    s = _abi.snn_model()
    s.n_pops = m.n_pops
    s.n_overrides = len(m.overrides)
    for f in ("dt_ms", "C_m_pF", "tau_m_ms", "tau_ref_ms", "tau_syn_ms", "u_rest_mV", "u_reset_mV",
              "u_thr_mV", "nu_th_hz", "w_ext_mV"):
        setattr(s, f, float(getattr(m, f)))
    for b in range(m.n_pops):
        s.n_full[b] = int(m.n_full[b])
        s.k_ext[b] = float(m.k_ext[b])
        s.u0_mean_mV[b] = float(m.u0_mean_mV[b])
        s.u0_sd_mV[b] = float(m.u0_sd_mV[b])
        s.w_mean_mV[b] = float(m.w_mean_mV[b])
        s.w_sd_mV[b] = float(m.w_sd_mV[b])
        s.d_mean_ms[b] = float(m.d_mean_ms[b])
        s.d_sd_ms[b] = float(m.d_sd_ms[b])
        for a in range(m.n_pops):
            s.conn_p[b][a] = float(m.conn_p[b][a])
    for o, (src, tgt, mu, sd) in enumerate(m.overrides):
        s.ovr_source[o], s.ovr_target[o] = int(src), int(tgt)
        s.ovr_w_mean_mV[o], s.ovr_w_sd_mV[o] = float(mu), float(sd)
    return s


class _Spec:
    """An snn_spec plus the host arrays it points to (kept alive together)."""

    def __init__(self, model, scale_n=1000, scale_k=1000, seed=1, custom=None, steps_per_graph=0,
                 raster_capacity=0, deliver_blocks=0, n_threads=0, engine=0, record_format=0, circuits=None,
                 smem_ring_rows=0):
        s = snn_spec()
        s.smem_ring_rows = int(smem_ring_rows)
        s.engine = int(engine)
        s.record_format = int(record_format)
        s.abi_version = ABI_VERSION
        s.scale_n_permille = int(scale_n)
        s.scale_k_permille = int(scale_k)
        s.steps_per_graph = int(steps_per_graph)
        s.seed = int(seed)
        s.raster_capacity = int(raster_capacity)
        s.deliver_blocks = int(deliver_blocks)
        s.n_threads = int(n_threads)
        s.model = model_struct(model)
        self._keep = []
        if custom is not None:
            cn = _abi.snn_custom_net()
            arrs = {
                "pre": np.ascontiguousarray(custom["pre"], dtype=np.int32),
                "post": np.ascontiguousarray(custom["post"], dtype=np.int32),
                "w_fx": np.ascontiguousarray(custom["w_fx"], dtype=np.int32),
                "delay": np.ascontiguousarray(custom["delay"], dtype=np.uint8),
                "u0": np.ascontiguousarray(custom["u0"], dtype=np.float32),
            }
            self._keep.append(arrs)
            cn.n_neurons = int(len(arrs["u0"]))
            cn.n_synapses = int(len(arrs["pre"]))
            for k in ("pre", "post", "w_fx", "delay", "u0"):
                setattr(cn, k, arrs[k].ctypes.data if arrs[k].size else None)
            po = custom.get("pop_offsets")
            if po is None:
                po = [0] + [cn.n_neurons] * model.n_pops
            for b in range(MAX_POPS + 1):
                cn.pop_offsets[b] = int(po[b]) if b < len(po) else cn.n_neurons
            self._keep.append(cn)
            s.custom = C.pointer(cn)
        if circuits:
            arr = (_abi.snn_circuit * len(circuits))()
            for c, (sn, sk, sd) in enumerate(circuits):
                arr[c].scale_n_permille, arr[c].scale_k_permille, arr[c].seed = int(sn), int(sk), int(sd)
            self._keep.append(arr)
            s.n_circuits = len(circuits)
            s.circuits = C.cast(arr, C.POINTER(_abi.snn_circuit))
        self.spec = s


def snn_query_sizes(spec: snn_spec) -> snn_sizes:
    out = snn_sizes()
    _check(load().snn_query_sizes(C.byref(spec), C.byref(out)), "snn_query_sizes")
    return out


def snn_export_network(spec: snn_spec) -> dict:
    """The network of `spec` built on the host, without a GPU (snn_export_network):
    row_ptr, post, w_fx, delay and u0 as numpy arrays, rows without their padding."""
    sz = snn_query_sizes(spec)
    n, S = int(sz.n_neurons), int(sz.n_synapses)
    out = {"row_ptr": np.zeros(n + 1, np.int64), "post": np.zeros(S, np.int32), "w_fx": np.zeros(S, np.int32),
           "delay": np.zeros(S, np.uint8), "u0": np.zeros(n, np.float32)}
    _check(load().snn_export_network(C.byref(spec), *(C.c_void_p(_ptr(out[k])) for k in
                                                      ("row_ptr", "post", "w_fx", "delay", "u0"))),
           "snn_export_network")
    return out


def export_network(model, scale_n: int = 1000, scale_k: int = 1000, seed: int = 1, circuits=None) -> dict:
    """Host-only build of a microcircuit (or a batch of circuits, as in Network) with the
    simulator's own builder; see snn_export_network."""
    return snn_export_network(_Spec(model, scale_n, scale_k, seed, circuits=circuits).spec)


def snn_build_network(spec: snn_spec, arena_ptr: int, arena_bytes: int, stream: int) -> int:
    h = C.c_void_p()
    _check(load().snn_build_network(C.byref(spec), C.c_void_p(arena_ptr), arena_bytes, C.c_void_p(stream),
                                    C.byref(h)), "snn_build_network")
    return h.value


def snn_step_n(handle: int, n_steps: int, stream: int) -> None:
    _check(load().snn_step_n(C.c_void_p(handle), int(n_steps), C.c_void_p(stream)), "snn_step_n")


def snn_read_spikes(handle: int, allow_overflow: bool = False, collect: bool = False):
    """All unread spikes as (steps int64[k], neurons int32[k]), ordered by (step, neuron);
    with collect=True only those of the calls before the latest snn_step_n
    (snn_collect_spikes, which does not wait for the latest call)."""
    lib = load()
    fn, name = (lib.snn_collect_spikes, "snn_collect_spikes") if collect else (lib.snn_read_spikes, "snn_read_spikes")
    n = C.c_int64()
    code = fn(C.c_void_p(handle), None, None, 0, C.byref(n))
    if code and not (allow_overflow and code == SNN_EOVERFLOW):
        _check(code, name)
    steps = np.empty(n.value, np.int64)
    neurons = np.empty(n.value, np.int32)
    got = C.c_int64()
    code = fn(C.c_void_p(handle), C.c_void_p(_ptr(steps) if n.value else 0),
              C.c_void_p(_ptr(neurons) if n.value else 0), n.value, C.byref(got))
    if code and not (allow_overflow and code == SNN_EOVERFLOW):
        _check(code, name)
    return steps[: got.value], neurons[: got.value]


def snn_read_rates(handle: int, t_begin: int, t_end: int, n_pops: int, n_neurons: int):
    rates = np.zeros(n_pops, np.float64)
    counts = np.zeros(n_neurons, np.int32)
    _check(load().snn_read_rates(C.c_void_p(handle), int(t_begin), int(t_end), C.c_void_p(_ptr(rates)),
                                 C.c_void_p(_ptr(counts))), "snn_read_rates")
    return rates, counts


def snn_get_info(handle: int) -> snn_info:
    out = snn_info()
    _check(load().snn_get_info(C.c_void_p(handle), C.byref(out)), "snn_get_info")
    return out


def snn_get_layout(handle: int) -> snn_layout:
    out = snn_layout()
    _check(load().snn_get_layout(C.c_void_p(handle), C.byref(out)), "snn_get_layout")
    return out


def snn_profile_steps(handle: int, n_steps: int, stream: int):
    a, b = C.c_double(), C.c_double()
    _check(load().snn_profile_steps(C.c_void_p(handle), int(n_steps), C.c_void_p(stream), C.byref(a),
                                    C.byref(b)), "snn_profile_steps")
    return a.value, b.value


def snn_deliver_spikes(handle: int, spikers_ptr: int, n: int, t: int, blocks: int, stream: int) -> None:
    _check(load().snn_deliver_spikes(C.c_void_p(handle), C.c_void_p(spikers_ptr), int(n), int(t), int(blocks),
                                     C.c_void_p(stream)), "snn_deliver_spikes")


def snn_destroy(handle: int) -> None:
    if handle:
        load().snn_destroy(C.c_void_p(handle))


class Network:
    """One simulated circuit on one GPU.

    ``model`` is a workload.Model (the paper's tables); the circuit is sampled at
    ``scale_n``/``scale_k`` permille with ``seed``, or given edge by edge via
    ``custom`` (dict with pre, post, w_fx, delay, u0 and optional pop_offsets).
    """

    def __init__(self, model, scale_n=1000, scale_k=1000, seed=1, custom=None, steps_per_graph=0,
                 raster_capacity=0, deliver_blocks=0, n_threads=0, device=None, engine=ENGINE_DEFAULT,
                 record_format=RECORD_PLAIN9, circuits=None, smem_ring_rows=0):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.device = torch.device(device if device is not None else "cuda")
        self._spec = _Spec(model, scale_n, scale_k, seed, custom, steps_per_graph, raster_capacity,
                           deliver_blocks, n_threads, engine, record_format, circuits, smem_ring_rows)
        self.sizes = snn_query_sizes(self._spec.spec)
        self.model = model
        with torch.cuda.device(self.device):
            nbytes = int(self.sizes.arena_bytes) + 256
            self._arena = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            base = self._arena.data_ptr()
            self._arena_ptr = (base + 255) // 256 * 256
            self._handle = 0
            stream = torch.cuda.current_stream(self.device).cuda_stream
            self._handle = snn_build_network(self._spec.spec, self._arena_ptr, int(self.sizes.arena_bytes), stream)
        self.n_neurons = int(self.sizes.n_neurons)
        self.n_pops = int(model.n_pops)

    def _stream(self, stream=None) -> int:
        import torch

        if stream is None:
            return torch.cuda.current_stream(self.device).cuda_stream
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)

    def step(self, n_steps: int, stream=None) -> None:
        snn_step_n(self._handle, n_steps, self._stream(stream))

    def read_spikes(self, allow_overflow: bool = False):
        return snn_read_spikes(self._handle, allow_overflow)

    def collect_spikes(self):
        """Spikes of the steps enqueued before the latest step() call, without waiting for
        that call (snn_collect_spikes): overlaps the host read with the GPU's next batch."""
        return snn_read_spikes(self._handle, False, collect=True)

    def read_rates(self, t_begin: int, t_end: int):
        return snn_read_rates(self._handle, t_begin, t_end, self.n_pops, self.n_neurons)

    def info(self) -> snn_info:
        return snn_get_info(self._handle)

    def save_state(self) -> bytes:
        """Checkpoint of the dynamic state (see snn_save_state)."""
        lib = load()
        n = C.c_uint64()
        _check(lib.snn_save_state(C.c_void_p(self._handle), None, 0, C.byref(n)), "snn_save_state")
        buf = np.zeros(n.value, np.uint8)
        _check(lib.snn_save_state(C.c_void_p(self._handle), C.c_void_p(_ptr(buf)), n.value, C.byref(n)),
               "snn_save_state")
        return buf.tobytes()

    def load_state(self, blob: bytes) -> None:
        buf = np.frombuffer(blob, np.uint8).copy()
        _check(load().snn_load_state(C.c_void_p(self._handle), C.c_void_p(_ptr(buf)), len(buf)), "snn_load_state")

    def set_schedule(self, grid_ctas: int = 0, delivery_warps: int = 0, steps_per_graph: int = 0) -> None:
        """Launch shape of the step kernels (results never depend on it)."""
        _check(load().snn_set_schedule(C.c_void_p(self._handle), int(grid_ctas), int(delivery_warps),
                                       int(steps_per_graph)), "snn_set_schedule")

    def set_circuit_groups(self, circuits_per_group: int) -> None:
        """Batches (graph or pipelined engine): run consecutive circuits in groups of this
        many, one group after another over each run of steps (0 = all at once); results
        never depend on it, and it may change between any two steps."""
        _check(load().snn_set_circuit_groups(C.c_void_p(self._handle), int(circuits_per_group)),
               "snn_set_circuit_groups")

    def circuits(self):
        """(base, n_neurons) arrays: where every circuit of a batch sits in the index space."""
        k = int(self.info().n_circuits)
        base = np.zeros(k, np.int64)
        n = np.zeros(k, np.int64)
        _check(load().snn_get_circuits(C.c_void_p(self._handle), C.c_void_p(_ptr(base)), C.c_void_p(_ptr(n))),
               "snn_get_circuits")
        return base, n

    def out_degrees(self) -> np.ndarray:
        out = np.zeros(self.n_neurons, np.int32)
        _check(load().snn_get_out_degrees(C.c_void_p(self._handle), C.c_void_p(_ptr(out))), "snn_get_out_degrees")
        return out

    def layout(self) -> snn_layout:
        return snn_get_layout(self._handle)

    def profile_steps(self, n_steps: int, stream=None):
        return snn_profile_steps(self._handle, n_steps, self._stream(stream))

    def deliver_spikes(self, spikers, t: int, blocks: int = 0, stream=None) -> None:
        """Phase 2 alone for a device int32 tensor of senders (see snn_deliver_spikes)."""
        import torch

        assert spikers.dtype == torch.int32 and spikers.is_cuda and spikers.is_contiguous()
        snn_deliver_spikes(self._handle, spikers.data_ptr(), spikers.numel(), t, blocks, self._stream(stream))

    def device_view(self, field: str, dtype, count: int, offset_elems: int = 0):
        """A torch view of one device buffer of the arena (inspection and tests)."""
        import torch

        off = getattr(self.layout(), field)
        item = torch.empty((), dtype=dtype).element_size()
        start = self._arena_ptr - self._arena.data_ptr() + int(off) + offset_elems * item
        return self._arena[start: start + count * item].view(dtype)

    def close(self) -> None:
        """Releases the handle and the device arena."""
        if getattr(self, "_handle", 0):
            snn_destroy(self._handle)
            self._handle = 0
        self._arena = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
