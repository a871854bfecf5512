"""ctypes mirror of include/snn.h (argument marshalling only)."""

from __future__ import annotations

import ctypes as C
import os

MAX_POPS = 8
MAX_OVERRIDES = 4
D_MAX = 64
FX_SHIFT = 12
POISSON_KMAX = 24
ABI_VERSION = 2
ENGINE_DEFAULT, ENGINE_GRAPH, ENGINE_PERSISTENT, ENGINE_PIPELINED, ENGINE_RESIDENT = 0, 1, 2, 3, 4
RECORD_PLAIN9, RECORD_PACKED_I8, RECORD_PACKED_BF16, RECORD_BLOCKED6, RECORD_BLOCKED4, RECORD_BLOCKED8 = 0, 1, 2, 3, 4, 5

STATUS = {0: "SNN_OK", 1: "SNN_EINVAL", 2: "SNN_ENOMEM", 3: "SNN_ECUDA", 4: "SNN_EOVERFLOW",
          5: "SNN_ETIMEOUT", 6: "SNN_ESTATE", 7: "SNN_ENOTSUP"}
SNN_OK, SNN_EINVAL, SNN_ENOMEM, SNN_ECUDA, SNN_EOVERFLOW, SNN_ETIMEOUT, SNN_ESTATE, SNN_ENOTSUP = range(8)


class snn_model(C.Structure):
    _fields_ = [
        ("n_pops", C.c_int32), ("n_overrides", C.c_int32),
        ("dt_ms", C.c_double), ("C_m_pF", C.c_double), ("tau_m_ms", C.c_double),
        ("tau_ref_ms", C.c_double), ("tau_syn_ms", C.c_double),
        ("u_rest_mV", C.c_double), ("u_reset_mV", C.c_double), ("u_thr_mV", C.c_double),
        ("nu_th_hz", C.c_double), ("w_ext_mV", C.c_double),
        ("n_full", C.c_int64 * MAX_POPS),
        ("k_ext", C.c_double * MAX_POPS),
        ("u0_mean_mV", C.c_double * MAX_POPS), ("u0_sd_mV", C.c_double * MAX_POPS),
        ("w_mean_mV", C.c_double * MAX_POPS), ("w_sd_mV", C.c_double * MAX_POPS),
        ("d_mean_ms", C.c_double * MAX_POPS), ("d_sd_ms", C.c_double * MAX_POPS),
        ("conn_p", (C.c_double * MAX_POPS) * MAX_POPS),
        ("ovr_source", C.c_int32 * MAX_OVERRIDES), ("ovr_target", C.c_int32 * MAX_OVERRIDES),
        ("ovr_w_mean_mV", C.c_double * MAX_OVERRIDES), ("ovr_w_sd_mV", C.c_double * MAX_OVERRIDES),
    ]


class snn_custom_net(C.Structure):
    _fields_ = [
        ("n_neurons", C.c_int64), ("n_synapses", C.c_int64),
        ("pre", C.c_void_p), ("post", C.c_void_p), ("w_fx", C.c_void_p), ("delay", C.c_void_p),
        ("u0", C.c_void_p),
        ("pop_offsets", C.c_int64 * (MAX_POPS + 1)),
    ]


class snn_circuit(C.Structure):
    _fields_ = [("scale_n_permille", C.c_int32), ("scale_k_permille", C.c_int32), ("seed", C.c_uint64)]


class snn_spec(C.Structure):
    _fields_ = [
        ("abi_version", C.c_uint32), ("scale_n_permille", C.c_int32), ("scale_k_permille", C.c_int32),
        ("steps_per_graph", C.c_int32), ("seed", C.c_uint64), ("raster_capacity", C.c_int64),
        ("deliver_blocks", C.c_int32), ("n_threads", C.c_int32),
        ("engine", C.c_int32), ("record_format", C.c_int32),
        ("model", snn_model),
        ("custom", C.POINTER(snn_custom_net)),
        ("n_circuits", C.c_int32), ("smem_ring_rows", C.c_int32),
        ("circuits", C.POINTER(snn_circuit)),
    ]


class snn_sizes(C.Structure):
    _fields_ = [
        ("arena_bytes", C.c_uint64), ("n_neurons", C.c_int64), ("n_neurons_padded", C.c_int64),
        ("n_synapses", C.c_int64), ("n_synapses_padded_max", C.c_int64), ("raster_capacity", C.c_int64),
    ]


class snn_layout(C.Structure):
    _fields_ = [(f, C.c_uint64) for f in ("ctl", "U", "I", "R", "ring", "row_ptr", "syn_tgt", "syn_w",
                                          "syn_delay", "rast_neuron", "rast_step", "params")] + [
        ("n_neurons_padded", C.c_int64), ("n_synapses_padded", C.c_int64), ("blocks", C.c_uint64),
        ("block_starts", C.c_uint64)]


class snn_info(C.Structure):
    _fields_ = [
        ("n_neurons", C.c_int64), ("n_synapses", C.c_int64), ("n_synapses_padded", C.c_int64),
        ("t", C.c_int64), ("spikes_read", C.c_int64), ("events_read", C.c_int64),
        ("n_pops", C.c_int32), ("t_ref_steps", C.c_int32),
        ("pop_offsets", C.c_int64 * (MAX_POPS + 1)),
        ("w_f", C.c_double), ("p11", C.c_double), ("p22", C.c_double), ("p21", C.c_double),
        ("p11_f32", C.c_float), ("p21_f32", C.c_float), ("p22_f32", C.c_float),
        ("theta_f32", C.c_float), ("u_reset_f32", C.c_float),
        ("w_ext_fx", C.c_int32),
        ("poisson_thresholds", (C.c_uint64 * POISSON_KMAX) * MAX_POPS),
        ("max_row_length", C.c_int32), ("chunks_per_row", C.c_int32),
        ("steps_per_graph", C.c_int32), ("deliver_blocks", C.c_int32),
        ("device_error", C.c_uint32), ("engine", C.c_int32),
        ("record_format", C.c_int32), ("bytes_per_synapse", C.c_int32),
        ("n_circuits", C.c_int32), ("schedule_ctas", C.c_int32), ("schedule_delivery_warps", C.c_int32),
        ("target_blocks", C.c_int32),
        ("i8_base", (C.c_int32 * MAX_POPS) * MAX_POPS), ("i8_step", (C.c_int32 * MAX_POPS) * MAX_POPS),
        ("circuits_per_group", C.c_int32), ("reserved3", C.c_int32), ("last_error", C.c_char * 256),
    ]


STATIC_MAX_NEURONS = 131072


class snn_static_io(C.Structure):
    _fields_ = [
        ("row_ptr", C.c_void_p), ("syn_tgt", C.c_void_p), ("syn_w", C.c_void_p), ("syn_delay", C.c_void_p),
        ("U", C.c_void_p), ("I", C.c_void_p), ("R", C.c_void_p), ("ring", C.c_void_p),
        ("ring_stride", C.c_int64), ("spikes", C.c_void_p), ("n_spikes", C.c_void_p),
    ]


LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsnn.so")

# name -> (restype, argtypes)
PROTOTYPES = {
    "snn_query_sizes": (C.c_int, [C.POINTER(snn_spec), C.POINTER(snn_sizes)]),
    "snn_build_network": (C.c_int, [C.POINTER(snn_spec), C.c_void_p, C.c_uint64, C.c_void_p,
                                    C.POINTER(C.c_void_p)]),
    "snn_export_network": (C.c_int, [C.POINTER(snn_spec), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p]),
    "snn_step_n": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p]),
    "snn_read_spikes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "snn_read_rates": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p]),
    "snn_get_info": (C.c_int, [C.c_void_p, C.POINTER(snn_info)]),
    "snn_get_layout": (C.c_int, [C.c_void_p, C.POINTER(snn_layout)]),
    "snn_profile_steps": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]),
    "snn_get_out_degrees": (C.c_int, [C.c_void_p, C.c_void_p]),
    "snn_get_circuits": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "snn_set_schedule": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32]),
    "snn_set_circuit_groups": (C.c_int, [C.c_void_p, C.c_int32]),
    "snn_collect_spikes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "snn_save_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.POINTER(C.c_uint64)]),
    "snn_load_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64]),
    "snn_deliver_spikes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_void_p]),
    "snn_destroy": (None, [C.c_void_p]),
    "snn_step_static": (C.c_int, [C.c_void_p, C.POINTER(snn_static_io), C.c_uint64, C.c_int64, C.c_void_p]),
    "snn_strerror": (C.c_char_p, [C.c_int]),
    "snn_last_error": (C.c_char_p, []),
}

_lib = None


def load():
    """Load libsnn.so.  Raises if it has not been built: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; g.build()\"`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib
