"""The C-ABI library loads, exports every symbol include/snn.h declares, and its
host-only entry points work without a GPU."""

import ctypes as C
import os
import re

import pytest

import oracle
import paper_2405_02019_gb300 as snn
import workload
from paper_2405_02019_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "snn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(snn_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2405_02019_gb300 import build

    build.build()
    return snn.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "snn_build_network" in names and "snn_step_n" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_abi.PROTOTYPES), set(names) ^ set(_abi.PROTOTYPES)


def test_strerror(lib):
    for code, name in _abi.STATUS.items():
        assert lib.snn_strerror(code)
    assert lib.snn_strerror(999) == b"unknown status"


@pytest.mark.parametrize("scale", [(100, 100), (1000, 1000), (20, 50), (4000, 1000)])
def test_query_sizes_matches_oracle_counts(lib, scale):
    """Host-only sizing agrees with the oracle's independent counts (checks the
    ctypes mirror of snn_spec/snn_model too)."""
    m = workload.microcircuit_model()
    spec = snn._Spec(m, *scale, seed=1).spec
    s = snn.snn_query_sizes(spec)
    assert s.n_neurons == oracle.pop_sizes(m, scale[0]).sum()
    assert s.n_synapses == oracle.total_synapses(m, *scale)
    assert s.n_neurons_padded % 128 == 0 and s.n_neurons_padded >= s.n_neurons
    assert s.n_synapses_padded_max == s.n_synapses + 3 * s.n_neurons
    # arena holds at least ring + synapse store + state
    assert s.arena_bytes >= 64 * 4 * s.n_neurons_padded + 9 * s.n_synapses + 9 * s.n_neurons


def test_full_scale_sizes(lib):
    m = workload.microcircuit_model()
    s = snn.snn_query_sizes(snn._Spec(m, 1000, 1000, 1).spec)
    assert s.n_neurons == 77169
    assert s.n_synapses == 284_811_022
    # ring of §3.2: 64 rows x 4 bytes x 77,169 neurons ~ 20 MB (padded to 77,184 columns)
    assert 64 * 4 * s.n_neurons_padded == 19_759_104


@pytest.mark.parametrize("field,value", [
    ("abi_version", 99), ("scale_n_permille", 0), ("steps_per_graph", -1), ("raster_capacity", -5)])
def test_invalid_specs_rejected(lib, field, value):
    m = workload.microcircuit_model()
    spec = snn._Spec(m, 100, 100, 1).spec
    setattr(spec, field, value)
    out = _abi.snn_sizes()
    assert lib.snn_query_sizes(C.byref(spec), C.byref(out)) == _abi.SNN_EINVAL
    assert lib.snn_last_error()


def test_invalid_model_rejected(lib):
    m = workload.microcircuit_model().replace(tau_m_ms=0.5, tau_syn_ms=0.5)
    spec = snn._Spec(m, 100, 100, 1).spec
    with pytest.raises(snn.SnnError):
        snn.snn_query_sizes(spec)


def test_custom_network_sizes(lib):
    m = workload.microcircuit_model()
    custom = dict(pre=[0, 1], post=[1, 2], w_fx=[5, 6], delay=[1, 2], u0=[0.0] * 13,
                  pop_offsets=[0, 13, 13, 13, 13, 13, 13, 13, 13])
    s = snn.snn_query_sizes(snn._Spec(m, custom=custom).spec)
    assert s.n_neurons == 13 and s.n_synapses == 2 and s.n_neurons_padded == 128


def test_build_rejects_null_arena(lib):
    m = workload.microcircuit_model()
    spec = snn._Spec(m, 100, 100, 1).spec
    h = C.c_void_p()
    assert lib.snn_build_network(C.byref(spec), None, 0, None, C.byref(h)) == _abi.SNN_EINVAL


def test_product_path_has_no_oracle_dependency():
    """The library and its binding never import or link the oracle."""
    pkg = os.path.join(ROOT, "paper_2405_02019_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".hpp", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "oracle.c" not in text and "liboracle" not in text, f


def test_blocked_records_sizes_and_rules(lib):
    """Blocked records: 6 bytes per synapse plus the per-row block table; one circuit
    on the graph engine (the default resolves to it); other engines and batches are
    rejected on the host."""
    m = workload.microcircuit_model()
    plain = snn.snn_query_sizes(snn._Spec(m, 1000, 1000, 1).spec)
    blk = snn.snn_query_sizes(snn._Spec(m, 1000, 1000, 1, record_format=snn.RECORD_BLOCKED6).spec)
    n, S = blk.n_neurons, blk.n_synapses
    bmax = (n + 511) // 512 + n // 736 + 2
    # every nonempty (row, block) segment is padded to a whole quad of records
    assert S == plain.n_synapses and blk.n_synapses_padded_max == S + 3 * min(S, n * bmax)
    assert blk.arena_bytes < plain.arena_bytes
    b4 = snn.snn_query_sizes(snn._Spec(m, 1000, 1000, 1, record_format=snn.RECORD_BLOCKED4).spec)
    assert b4.n_synapses_padded_max == blk.n_synapses_padded_max
    assert b4.arena_bytes < blk.arena_bytes - 2 * S  # 4 instead of 6 bytes per (padded) synapse
    b8 = snn.snn_query_sizes(snn._Spec(m, 1000, 1000, 1, record_format=snn.RECORD_BLOCKED8).spec)
    assert b8.n_synapses_padded_max == blk.n_synapses_padded_max
    assert b8.arena_bytes > blk.arena_bytes + 2 * S  # 8 instead of 6 bytes per (padded) synapse
    for fmt in (snn.RECORD_BLOCKED6, snn.RECORD_BLOCKED4, snn.RECORD_BLOCKED8):
        for engine in (snn.ENGINE_PIPELINED, snn.ENGINE_PERSISTENT):
            spec = snn._Spec(m, 100, 100, 1, record_format=fmt, engine=engine).spec
            with pytest.raises(snn.SnnError):
                snn.snn_query_sizes(spec)
    spec = snn._Spec(m, record_format=snn.RECORD_BLOCKED6, circuits=[(100, 100, 1), (200, 200, 2)]).spec
    with pytest.raises(snn.SnnError):
        snn.snn_query_sizes(spec)
    spec = snn._Spec(m, 100, 100, 1, record_format=snn.RECORD_BLOCKED6, engine=snn.ENGINE_GRAPH).spec
    assert snn.snn_query_sizes(spec).n_neurons == 7718


def test_null_handle_is_rejected_before_any_device_work(lib):
    """Every entry point that takes a network handle refuses a null one with SNN_EINVAL
    (no device call is made, so this runs without a GPU)."""
    i64 = C.c_int64(0)
    u64 = C.c_uint64(0)
    d = C.c_double(0)
    info = _abi.snn_info()
    layout = _abi.snn_layout()
    buf = (C.c_int64 * 4)()
    calls = {
        "snn_step_n": lambda: lib.snn_step_n(None, 1, None),
        "snn_read_spikes": lambda: lib.snn_read_spikes(None, None, None, 0, C.byref(i64)),
        "snn_collect_spikes": lambda: lib.snn_collect_spikes(None, None, None, 0, C.byref(i64)),
        "snn_read_rates": lambda: lib.snn_read_rates(None, 0, 10, buf, None),
        "snn_get_info": lambda: lib.snn_get_info(None, C.byref(info)),
        "snn_get_layout": lambda: lib.snn_get_layout(None, C.byref(layout)),
        "snn_profile_steps": lambda: lib.snn_profile_steps(None, 1, None, C.byref(d), C.byref(d)),
        "snn_get_out_degrees": lambda: lib.snn_get_out_degrees(None, buf),
        "snn_get_circuits": lambda: lib.snn_get_circuits(None, buf, buf),
        "snn_set_schedule": lambda: lib.snn_set_schedule(None, 152, 8, 1024),
        "snn_set_circuit_groups": lambda: lib.snn_set_circuit_groups(None, 2),
        "snn_save_state": lambda: lib.snn_save_state(None, None, 0, C.byref(u64)),
        "snn_load_state": lambda: lib.snn_load_state(None, buf, 32),
        "snn_deliver_spikes": lambda: lib.snn_deliver_spikes(None, buf, 1, 0, 0, None),
        "snn_step_static": lambda: lib.snn_step_static(None, None, 1, 0, None),
    }
    for name, call in calls.items():
        assert call() == _abi.SNN_EINVAL, name
        assert b"null" in lib.snn_last_error(), name
    lib.snn_destroy(None)  # a no-op
    # every declared entry point that takes a handle is covered above
    takes_handle = {n for n, (_, args) in _abi.PROTOTYPES.items() if args and args[0] is C.c_void_p}
    assert takes_handle - {"snn_destroy"} == set(calls), takes_handle ^ set(calls)
