"""The simulator's network builder, run on the host through snn_export_network (no GPU),
against the oracle's independent build: the same rows (as multisets of target, delay and
weight), the indexed store's delay order inside each row (§3.5), the same initial
potentials bit for bit, and batches placed circuit by circuit."""

import ctypes as C

import numpy as np
import pytest

import oracle
import paper_2405_02019_gb300 as snn
from paper_2405_02019_gb300 import _abi


@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_2405_02019_gb300 import build

    build.build()


def _row_keys(row_ptr, post, delay, w, shift=0):
    """One sortable key per synapse: (row, target, delay, weight), rows as given."""
    lens = np.diff(row_ptr)
    row = np.repeat(np.arange(len(lens), dtype=np.int64), lens)
    k = np.lexsort((w, delay, post.astype(np.int64) - shift, row))
    return row[k], post[k].astype(np.int64) - shift, delay[k], w[k]


def _assert_same_network(g, onet, base=0):
    """g: the export restricted to one circuit's rows; onet: the oracle's network."""
    assert np.array_equal(g["row_ptr"] - g["row_ptr"][0], onet.row_ptr)
    a = _row_keys(g["row_ptr"] - g["row_ptr"][0], g["post"], g["delay"], g["w_fx"], shift=base)
    b = _row_keys(onet.row_ptr, onet.post, onet.delay, onet.w_fx)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.array_equal(g["u0"].view(np.uint32), onet.u0.view(np.uint32))


def _slice(net, lo, hi):
    rp = net["row_ptr"]
    a, b = rp[lo], rp[hi]
    return {"row_ptr": rp[lo: hi + 1], "post": net["post"][a:b], "delay": net["delay"][a:b],
            "w_fx": net["w_fx"][a:b], "u0": net["u0"][lo:hi]}


@pytest.mark.parametrize("scale", [(100, 100, 1), (20, 50, 7), (35, 10, 6)])
def test_export_equals_oracle_network(model, scale):
    net = snn.export_network(model, *scale)
    onet = oracle.build_network(model, *scale)
    _assert_same_network(net, onet)
    # the indexed store (§3.5): every row sorted by delay
    rp, d = net["row_ptr"], net["delay"].astype(np.int64)
    row = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    same_row = row[1:] == row[:-1]
    assert np.all(d[1:][same_row] >= d[:-1][same_row])


def test_export_equals_oracle_when_clipping_is_common(model):
    """The same comparison under a model whose draws often leave the clipping bounds:
    weight SD equal to the mean (about 16 % of weights clip at zero) and excitatory
    delays of 5.5 +- 1.5 ms (a fifth clip at 63 steps), inhibitory ones of 0.2 +- 0.2 ms
    (most clip at 1 step)."""
    m2 = model.replace(w_sd_mV=[abs(mu) for mu in model.w_mean_mV], overrides=[(2, 0, 0.3, 0.3)],
                       d_mean_ms=[5.5 if b % 2 == 0 else 0.2 for b in range(8)],
                       d_sd_ms=[1.5 if b % 2 == 0 else 0.2 for b in range(8)])
    net = snn.export_network(m2, 30, 30, 4)
    onet = oracle.build_network(m2, 30, 30, 4)
    _assert_same_network(net, onet)
    assert np.count_nonzero(net["delay"] == 63) > 0.1 * len(net["delay"]) * 0.5
    assert np.count_nonzero(net["w_fx"] == 0) > 0.1 * len(net["w_fx"])


def test_export_of_a_batch_places_each_circuit_alone(model):
    circuits = [(20, 40, 5), (35, 10, 6), (1, 1, 9)]
    net = snn.export_network(model, circuits=circuits)
    base = 0
    for c, (sn, sk, seed) in enumerate(circuits):
        onet = oracle.build_network(model, sn, sk, seed)
        _assert_same_network(_slice(net, base, base + onet.n), onet, base=base)
        nxt = (base + onet.n + 127) // 128 * 128
        if c + 1 < len(circuits):  # the neurons up to the next circuit are inert: no synapses
            assert net["row_ptr"][nxt] == net["row_ptr"][base + onet.n]
        base = nxt


@pytest.mark.parametrize("fmt", [snn.RECORD_PACKED_I8, snn.RECORD_PACKED_BF16])
def test_export_of_packed_records_reads_back_the_oracles_quantised_weights(model, fmt):
    """Packed records (Z18): targets and delays decode from the packed words unchanged, and
    the weight the kernels read back equals the oracle's quantiser applied to the oracle's
    network (int8: per population pair base + code * step; bf16: the round-to-nearest-even
    bfloat16 current read back as rint(f * 4096))."""
    onet = oracle.build_network(model, 100, 100, 1)
    if fmt == snn.RECORD_PACKED_I8:
        wq = oracle.quantize_i8(onet)[0]
    else:
        wq = oracle.quantize_bf16(onet.w_fx)
    net = snn.snn_export_network(snn._Spec(model, 100, 100, 1, record_format=fmt).spec)
    _assert_same_network(net, oracle.with_weights(onet, wq))


def test_export_refuses_other_formats_and_null(model):
    lib = snn.load()
    spec = snn._Spec(model, 20, 20, 1, record_format=snn.RECORD_BLOCKED6).spec
    assert lib.snn_export_network(C.byref(spec), None, None, None, None, None) == _abi.SNN_EINVAL
    assert lib.snn_export_network(None, None, None, None, None, None) == _abi.SNN_EINVAL
    # all outputs optional
    spec = snn._Spec(model, 20, 20, 1).spec
    assert lib.snn_export_network(C.byref(spec), None, None, None, None, None) == 0
