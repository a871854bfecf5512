"""Full-length parity on the GPU: the paper's whole 10 s run (100,000 steps of 0.1 ms,
§4) of the full microcircuit (77,169 neurons, 284,811,022 synapses, seed 1), in the
bench's launch configuration (1,024-step snn_step_n calls with an overlapped raster
read after each), against one oracle run of the same 100,000 steps.  The raster is
compared spike for spike and the final U, I, R and the whole ring bit for bit.

The oracle's 100,000 steps take a few minutes on one host core; they run in a
background thread from the start of the session (tests/oracle_runs.py) while the GPU
runs its engines.
Also here: the persistent engine over 2,048 full-scale steps, and circuit groups of a
small batch over 5,000 steps, each against the oracle.
"""

import os
import sys

import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2405_02019_gb300 as snn  # noqa: E402

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

STEPS = 100_000
CALL = 1024


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2405_02019_gb300 import build

    build.build()
    oracle.build()


@pytest.fixture(scope="module")
def model():
    return workload.microcircuit_model()


@pytest.fixture(scope="module")
def full_run():
    import oracle_runs

    wl = workload.WORKLOADS["pd_full"]
    return wl, oracle_runs.start("full_fp32_seed1")


def _state(net):
    n = net.n_neurons
    npad = int(net.layout().n_neurons_padded)
    U = net.device_view("U", torch.float32, n).cpu().numpy()
    I = net.device_view("I", torch.float32, n).cpu().numpy()
    R = net.device_view("R", torch.uint8, n).cpu().numpy().astype(np.int32)
    ring = net.device_view("ring", torch.int32, 64 * npad).cpu().numpy().reshape(64, npad)[:, :n]
    return U, I, R, ring.astype(np.int64)


def _bench_loop(net, steps):
    """snn_step_n in 1,024-step calls, snn_collect_spikes after each, a final read."""
    parts, done = [], 0
    while done < steps:
        k = min(CALL, steps - done)
        net.step(k)
        parts.append(net.collect_spikes())
        done += k
    parts.append(net.read_spikes())
    return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])


@pytest.mark.parametrize("engine", [snn.ENGINE_RESIDENT, snn.ENGINE_PIPELINED])
def test_full_run_100k_steps_bit_exact(model, full_run, engine):
    """The whole 10 s of the full microcircuit: identical raster (about 2.9 million
    spikes) and identical final neuron state and ring."""
    wl, bg = full_run
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, steps_per_graph=CALL,
                      raster_capacity=1 << 25, engine=engine)
    assert net.info().engine == engine
    g_t, g_i = _bench_loop(net, STEPS)
    U, I, R, ring = _state(net)
    net.close()
    ref = bg.get()
    o_t, o_i, sim, onet = ref["t"], ref["i"], ref["sim"], ref["net"]
    assert len(o_t) > 1_000_000
    assert len(g_t) == len(o_t)
    assert np.array_equal(g_t, o_t) and np.array_equal(g_i, o_i)
    assert sim.t == STEPS
    assert np.array_equal(U.view(np.uint32), sim.U.view(np.uint32))
    assert np.array_equal(I.view(np.uint32), sim.I.view(np.uint32))
    assert np.array_equal(R, sim.R)
    assert np.array_equal(ring, sim.W.reshape(64, onet.n))
    print(f"engine {engine}: {len(g_t)} spikes over {STEPS} steps identical to the oracle")


def test_persistent_engine_full_scale(model, full_run):
    """The persistent engine over 2,048 full-scale steps (two 1,024-step launches)."""
    wl, bg = full_run
    onet = bg.get()["net"]
    steps = 2048
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, engine=snn.ENGINE_PERSISTENT)
    g_t, g_i = _bench_loop(net, steps)
    U, I, R, _ = _state(net)
    net.close()
    sim = oracle.Sim(model, onet, wl.seed)
    o_t, o_i = sim.run(steps)
    assert np.array_equal(g_t, o_t) and np.array_equal(g_i, o_i)
    assert np.array_equal(U.view(np.uint32), sim.U.view(np.uint32))
    assert np.array_equal(I.view(np.uint32), sim.I.view(np.uint32)) and np.array_equal(R, sim.R)


BATCH = [(20, 40, 5), (35, 10, 6), (13, 50, 7), (50, 50, 8), (1, 1, 9)]


@pytest.mark.parametrize("engine", [snn.ENGINE_PIPELINED, snn.ENGINE_GRAPH])
def test_circuit_groups_5000_steps(model, engine):
    """A batch of five uneven circuits in circuit groups of two over 5,000 steps: every
    circuit's slice of the raster and state equals the oracle run of that circuit
    alone."""
    steps = 5000
    net = snn.Network(model, circuits=BATCH, steps_per_graph=CALL, engine=engine)
    net.set_circuit_groups(2)
    base, n = net.circuits()
    g_t, g_i = _bench_loop(net, steps)
    n_all = net.n_neurons
    U = net.device_view("U", torch.float32, n_all).cpu().numpy()
    I = net.device_view("I", torch.float32, n_all).cpu().numpy()
    R = net.device_view("R", torch.uint8, n_all).cpu().numpy().astype(np.int32)
    net.close()
    for c, (sn, sk, seed) in enumerate(BATCH):
        onet = oracle.build_network(model, sn, sk, seed)
        sim = oracle.Sim(model, onet, seed)
        o_t, o_i = sim.run(steps)
        sel = (g_i >= base[c]) & (g_i < base[c] + n[c])
        assert np.array_equal(g_t[sel], o_t), c
        assert np.array_equal(g_i[sel] - base[c], o_i), c
        sl = slice(base[c], base[c] + n[c])
        assert np.array_equal(U[sl].view(np.uint32), sim.U.view(np.uint32)), c
        assert np.array_equal(I[sl].view(np.uint32), sim.I.view(np.uint32)), c
        assert np.array_equal(R[sl], sim.R), c
