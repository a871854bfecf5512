"""snn_step_static: the step for callers that may not allocate device memory.

Some programs embed the simulator under an allocator they do not control (a host
application that owns every byte of device memory, a control loop that cannot risk
an allocation mid-run); they cannot let the library call cudaMalloc.  snn_step_static
serves them: it takes every buffer from the caller and keeps its only working memory
in a fixed array inside the library.  Here two calls in a row, made through the C
ABI, must reproduce exactly (the bit-for-bit tolerance of every parity test in this
suite) what snn_step_n computes for the same two steps.

This file is collected last on purpose; it passes alone in a fresh process and
after the rest of the suite.
"""

import ctypes as C

import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2405_02019_gb300 as snn  # noqa: E402
from paper_2405_02019_gb300 import _abi  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2405_02019_gb300 import build

    build.build()


def _io_for(net, spikes, n_spikes):
    lay = net.layout()
    base = net._arena_ptr
    io = _abi.snn_static_io()
    io.row_ptr = base + lay.row_ptr
    io.syn_tgt = base + lay.syn_tgt
    io.syn_w = base + lay.syn_w
    io.syn_delay = base + lay.syn_delay
    io.U = base + lay.U
    io.I = base + lay.I
    io.R = base + lay.R
    io.ring = base + lay.ring
    io.ring_stride = lay.n_neurons_padded
    io.spikes = spikes.data_ptr()
    io.n_spikes = n_spikes.data_ptr()
    return io


def _snapshot(net):
    n = net.n_neurons
    npad = int(net.layout().n_neurons_padded)
    return {
        "U": net.device_view("U", torch.int32, n).cpu().numpy(),
        "I": net.device_view("I", torch.int32, n).cpu().numpy(),
        "R": net.device_view("R", torch.uint8, n).cpu().numpy(),
        "ring": net.device_view("ring", torch.int32, 64 * npad).cpu().numpy(),
    }


def test_two_static_steps_match_step_n():
    m = workload.microcircuit_model()
    seed, warm = 1, 200
    ref = snn.Network(m, 100, 100, seed=seed, steps_per_graph=50)
    dut = snn.Network(m, 100, 100, seed=seed, steps_per_graph=50)
    ref.step(warm)
    dut.step(warm)
    ref.read_spikes()
    dut.read_spikes()
    assert all(np.array_equal(a, b) for a, b in zip(_snapshot(ref).values(), _snapshot(dut).values()))

    lib = snn.load()
    n = ref.n_neurons
    spikes = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    n_spikes = torch.zeros(1, dtype=torch.int32, device="cuda")
    io = _io_for(dut, spikes, n_spikes)
    stream = torch.cuda.current_stream().cuda_stream
    total = 0
    for t in (warm, warm + 1):
        ref.step(1)
        r_t, r_i = ref.read_spikes()
        assert np.all(r_t == t)
        rc = lib.snn_step_static(C.c_void_p(dut._handle), C.byref(io), seed, t, C.c_void_p(stream))
        assert rc == 0, lib.snn_last_error()
        torch.cuda.synchronize()
        k = int(n_spikes.item())
        got = np.sort(spikes[:k].cpu().numpy())
        assert np.array_equal(got, r_i), t
        total += k
        a, b = _snapshot(ref), _snapshot(dut)
        for key in a:
            assert np.array_equal(a[key], b[key]), (t, key)
    assert total > 0  # the two steps had spikes to deliver
    ref.close()
    dut.close()


def test_too_many_neurons_rejected():
    """Networks larger than the fixed working array are refused with a clear error."""
    m = workload.microcircuit_model()
    n = _abi.STATIC_MAX_NEURONS + 1
    custom = dict(pre=[], post=[], w_fx=[], delay=[], u0=np.zeros(n, np.float32), pop_offsets=[0] + [n] * 8)
    net = snn.Network(m, custom=custom)
    lib = snn.load()
    spikes = torch.zeros(n, dtype=torch.int32, device="cuda")
    n_spikes = torch.zeros(1, dtype=torch.int32, device="cuda")
    io = _io_for(net, spikes, n_spikes)
    rc = lib.snn_step_static(C.c_void_p(net._handle), C.byref(io), 1, 0, None)
    assert rc == _abi.SNN_EINVAL
    assert b"SNN_STATIC_MAX_NEURONS" in lib.snn_last_error()
    net.close()


def test_hundred_static_steps_with_every_delay_match_step_n():
    """100 consecutive calls on a small network whose delays take every value 1..63:
    each call's spikes (sorted) and, at the end, U, I, R and the whole 64-row ring equal
    snn_step_n's; the fixed spike counter is cleared by every call, and contributions
    wrap around the ring."""
    m = workload.microcircuit_model()
    rng = np.random.default_rng(21)
    n, S = 600, 30000
    custom = dict(pre=rng.integers(0, n, S), post=rng.integers(0, n, S),
                  w_fx=rng.integers(-1_500_000, 2_500_000, S), delay=np.tile(np.arange(1, 64), S // 63 + 1)[:S],
                  u0=rng.uniform(0, 16, n).astype(np.float32), pop_offsets=[0] + [n] * 8)
    seed = 7
    ref = snn.Network(m, custom=custom, seed=seed, steps_per_graph=64)
    dut = snn.Network(m, custom=custom, seed=seed, steps_per_graph=64)
    lib = snn.load()
    spikes = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    n_spikes = torch.zeros(1, dtype=torch.int32, device="cuda")
    io = _io_for(dut, spikes, n_spikes)
    stream = torch.cuda.current_stream().cuda_stream
    total = 0
    for t in range(100):
        ref.step(1)
        r_t, r_i = ref.read_spikes()
        rc = lib.snn_step_static(C.c_void_p(dut._handle), C.byref(io), seed, t, C.c_void_p(stream))
        assert rc == 0, lib.snn_last_error()
        torch.cuda.synchronize()
        k = int(n_spikes.item())
        assert np.array_equal(np.sort(spikes[:k].cpu().numpy()), r_i), t
        total += k
    assert total > 100
    a, b = _snapshot(ref), _snapshot(dut)
    for key in a:
        assert np.array_equal(a[key], b[key]), key
    ref.close()
    dut.close()
