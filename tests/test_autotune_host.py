"""Host logic of the schedule autotuner: which candidates it tries for each engine and
batch size, and how it applies one (no GPU: a stand-in network records the calls)."""

from types import SimpleNamespace

import pytest

import paper_2405_02019_gb300 as snn
from paper_2405_02019_gb300 import autotune


class FakeNet:
    def __init__(self, engine, n_circuits):
        self._info = SimpleNamespace(engine=engine, n_circuits=n_circuits)
        self.calls = []

    def info(self):
        return self._info

    def set_schedule(self, **kw):
        self.calls.append(("set_schedule", kw))

    def set_circuit_groups(self, k):
        self.calls.append(("set_circuit_groups", k))


@pytest.mark.parametrize("engine", [snn.ENGINE_PIPELINED, snn.ENGINE_GRAPH])
def test_batch_candidates_include_circuit_groups(engine):
    cands = autotune.candidates(FakeNet(engine, 32), 152)
    groups = sorted({c["circuits_per_group"] for c in cands})
    assert groups == [0, 4, 8, 16]
    grids = sorted({c["grid_ctas"] for c in cands})
    if engine == snn.ENGINE_PIPELINED:
        assert grids == [152, 304, 456]
        assert sorted({c["delivery_warps"] for c in cands}) == [4, 8]
        assert len(cands) == 3 * 2 * 4
    else:
        assert grids == [152, 304, 608]
        assert len(cands) == 3 * 4
    # every candidate is a distinct schedule
    assert len({tuple(sorted(c.items())) for c in cands}) == len(cands)


@pytest.mark.parametrize("n_circuits,groups", [(1, [0]), (5, [0, 4]), (9, [0, 4, 8]), (16, [0, 4, 8])])
def test_group_sizes_stay_below_the_batch(n_circuits, groups):
    cands = autotune.candidates(FakeNet(snn.ENGINE_PIPELINED, n_circuits), 152)
    assert sorted({c["circuits_per_group"] for c in cands}) == groups


def test_persistent_engine_has_no_candidates():
    assert autotune.candidates(FakeNet(snn.ENGINE_PERSISTENT, 32), 152) == []


def test_apply_sets_schedule_then_groups():
    net = FakeNet(snn.ENGINE_PIPELINED, 32)
    autotune._apply(net, dict(grid_ctas=456, delivery_warps=4, steps_per_graph=1024, circuits_per_group=8))
    assert net.calls == [("set_schedule", dict(grid_ctas=456, delivery_warps=4, steps_per_graph=1024)),
                         ("set_circuit_groups", 8)]
    net = FakeNet(snn.ENGINE_PIPELINED, 1)
    autotune._apply(net, dict(grid_ctas=152, delivery_warps=8, steps_per_graph=1024))
    assert net.calls == [("set_schedule", dict(grid_ctas=152, delivery_warps=8, steps_per_graph=1024))]
