"""The multithreaded CPU baseline (oracle/cpu_mt.c) reproduces the oracle bit for bit:
it is the same step with the neurons and the ring partitioned over threads."""

import numpy as np
import pytest

import oracle
import workload


@pytest.fixture(scope="module")
def tiny():
    m = workload.microcircuit_model()
    wl = workload.WORKLOADS["pd_tiny"]
    onet = oracle.build_network(m, wl.scale_n_permille, wl.scale_k_permille, wl.seed)
    ref = oracle.Sim(m, onet, wl.seed)
    o = ref.run(400)
    return m, wl, onet, ref, o


@pytest.mark.parametrize("threads", [1, 2, 5, 16])
def test_threads_reproduce_the_oracle(tiny, threads):
    m, wl, onet, ref, (o_t, o_i) = tiny
    sim = oracle.SimMT(m, onet, wl.seed, threads)
    a = sim.run(150)
    b = sim.run(250)
    g_t = np.concatenate([a[0], b[0]])
    g_i = np.concatenate([a[1], b[1]])
    assert len(o_t) > 1000
    assert np.array_equal(g_t, o_t) and np.array_equal(g_i, o_i)
    assert np.array_equal(sim.U.view(np.uint32), ref.U.view(np.uint32))
    assert np.array_equal(sim.I.view(np.uint32), ref.I.view(np.uint32))
    assert np.array_equal(sim.R, ref.R) and np.array_equal(sim.W.astype(np.int64), ref.W)


def test_more_threads_than_neurons():
    m = workload.microcircuit_model()
    u0 = np.array([14.0, 3.0, 15.5], np.float32)
    onet = oracle.network_from_edges(3, [0, 1, 2], [1, 2, 0], [400_000, 500_000, -300_000], [1, 2, 63], u0)
    ref = oracle.Sim(m, onet, 3)
    sim = oracle.SimMT(m, onet, 3, 8)
    assert all(np.array_equal(x, y) for x, y in zip(ref.run(200), sim.run(200)))
