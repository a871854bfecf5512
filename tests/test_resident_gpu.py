"""GPU parity of the resident engine (one cooperative CTA per target block, neuron state
in registers, the block's ring columns and segment tables in shared memory, block-major
records, spikes exchanged through step-tagged inbox slots) against the CPU oracle,
through the C ABI.

The engine's arithmetic is the plain mode's (FP32 without FMA, int32 ring), so rasters
and states are compared element by element with no tolerance.  The cases reach the
engine's own mechanics: launch boundaries at every phase of the ring, the shared-memory
window with long delays in global memory, bursts larger than the per-pass gather list
and slots holding more spikes than one probe reads, the block-major tables and their
escaped lengths, a checkpoint loaded into a handle whose mailboxes hold later steps,
and the bounded mailbox wait.
"""

import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2405_02019_gb300 as snn  # noqa: E402

RES = snn.ENGINE_RESIDENT


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2405_02019_gb300 import build

    build.build()
    oracle.build()


@pytest.fixture(scope="module")
def model():
    return workload.microcircuit_model()


@pytest.fixture(scope="module")
def tiny(model):
    wl = workload.WORKLOADS["pd_tiny"]
    return wl, oracle.build_network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed)


def _state(net):
    n = net.n_neurons
    U = net.device_view("U", torch.float32, n).cpu().numpy()
    I = net.device_view("I", torch.float32, n).cpu().numpy()
    R = net.device_view("R", torch.uint8, n).cpu().numpy().astype(np.int32)
    return U, I, R


def _ring(net):
    npad = int(net.layout().n_neurons_padded)
    ring = net.device_view("ring", torch.int32, 64 * npad).cpu().numpy().reshape(64, npad)
    return ring[:, : net.n_neurons].astype(np.int64)


def _oracle_ring(sim):
    """The oracle's ring as [64][n] (slot-major, like the device's)."""
    return sim.W.reshape(64, sim.net.n)


def _assert_same(net, sim, ring=True):
    U, I, R = _state(net)
    assert np.array_equal(U.view(np.uint32), sim.U.view(np.uint32))
    assert np.array_equal(I.view(np.uint32), sim.I.view(np.uint32))
    assert np.array_equal(R, sim.R)
    if ring:
        assert np.array_equal(_ring(net), _oracle_ring(sim))


def _tables(net):
    """The block-major tables (rbase, offt, lens, coarse) read back from the arena."""
    n, B = net.n_neurons, int(net.info().target_blocks)
    up = lambda x: (x + 255) // 256 * 256  # noqa: E731
    coarse_stride, lens_stride = (n + 31) // 32 + 1, (n + 31) // 32 * 32
    o_coarse = up(8 * (B + 1))
    o_lens = up(o_coarse + 4 * B * coarse_stride)
    o_offt = up(o_lens + B * lens_stride)
    start = net._arena_ptr - net._arena.data_ptr() + int(net.layout().block_starts)
    raw = net._arena[start: start + o_offt + 4 * B * (n + 1)].cpu().numpy()
    rbase = raw[: 8 * (B + 1)].view(np.int64)
    coarse = raw[o_coarse: o_coarse + 4 * B * coarse_stride].view(np.uint32).reshape(B, coarse_stride)
    lens = raw[o_lens: o_lens + B * lens_stride].reshape(B, lens_stride)[:, :n]
    offt = raw[o_offt: o_offt + 4 * B * (n + 1)].view(np.uint32).reshape(B, n + 1).astype(np.int64)
    return rbase, offt, lens, coarse


def test_resident_structure_tiny(model, tiny):
    """Blocks of equal width (a multiple of 32) cover the neurons, one CTA each.  The
    records are block-major: block b's region holds, sender by sender, exactly the
    oracle's synapses of that sender into block b, in delay order; the tables give every
    segment's offset (exact), its length capped at 255 (with escapes flagged per group of
    32 senders) and each group's first offset."""
    wl, onet = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, engine=RES)
    info = net.info()
    assert info.engine == RES and info.record_format == snn.RECORD_PLAIN9
    B = int(info.target_blocks)
    assert B >= 1 and info.schedule_ctas == B and info.schedule_delivery_warps * 32 >= B
    n = onet.n
    bounds = net.device_view("blocks", torch.int32, B + 1).cpu().numpy().astype(np.int64)
    width = bounds[1] - bounds[0]
    assert bounds[0] == 0 and bounds[-1] == n and width % 32 == 0 and width <= 1024
    assert np.all(np.diff(bounds)[:-1] == width) and 0 < bounds[-1] - bounds[-2] <= width
    rbase, offt, lens, coarse = _tables(net)
    S = len(onet.post)
    assert rbase[0] == 0 and rbase[-1] == S and int(net.layout().n_synapses_padded) == S
    assert np.array_equal(np.diff(rbase), offt[:, n])
    seglen = np.diff(offt, axis=1)
    assert np.array_equal(lens, np.minimum(seglen, 255))
    assert np.array_equal(coarse[:, :-1] & 0x7FFFFFFF, offt[:, 0:n:32])
    flagged = (coarse[:, :-1] >> 31).astype(bool)
    groups = np.add.reduceat(seglen >= 255, np.arange(0, n, 32), axis=1) > 0
    assert np.array_equal(flagged, groups)
    tg = net.device_view("syn_tgt", torch.int32, S).cpu().numpy().astype(np.int64)
    w = net.device_view("syn_w", torch.int32, S).cpu().numpy()
    d = net.device_view("syn_delay", torch.uint8, S).cpu().numpy()
    blk_of = np.searchsorted(bounds, onet.post, side="right") - 1
    for i in range(0, n, 7):
        oa, ob = onet.row_ptr[i], onet.row_ptr[i + 1]
        for b in range(0, B, 5):
            a0, a1 = rbase[b] + offt[b, i], rbase[b] + offt[b, i + 1]
            sel = slice(oa, ob)
            mine = blk_of[sel] == b
            o = np.sort(onet.post[sel][mine].astype(np.int64) << 38 | onet.delay[sel][mine].astype(np.int64) << 32
                        | (onet.w_fx[sel][mine].astype(np.int64) + 2**31))
            g = np.sort(tg[a0:a1] << 38 | d[a0:a1].astype(np.int64) << 32 | (w[a0:a1].astype(np.int64) + 2**31))
            assert np.array_equal(o, g), (i, b)
            assert np.all(np.diff(d[a0:a1].astype(int)) >= 0)
            assert np.all((tg[a0:a1] >= bounds[b]) & (tg[a0:a1] < bounds[b + 1]))
    net.close()


@pytest.mark.parametrize("nspk", [1, 63, 64, 700, 2048, 2049, 9000])
def test_resident_deliver_spikes_matches_oracle_network(model, tiny, nspk):
    """Phase 2 alone on block-major records (one CTA per target block reading its
    region's segments), below and above the 64-sender switch to shared-memory sums and
    across 2,048-sender passes, repeats included: the ring equals the sums over the
    oracle's rows."""
    wl, onet = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, engine=RES)
    rng = np.random.default_rng(300 + nspk)
    spikers = rng.integers(0, onet.n, nspk).astype(np.int32)
    t = 61
    net.deliver_spikes(torch.from_numpy(spikers).cuda(), t)
    torch.cuda.synchronize()
    npad = int(net.layout().n_neurons_padded)
    ring = net.device_view("ring", torch.int32, 64 * npad).cpu().numpy().reshape(64, npad).astype(np.int64)
    lens = np.diff(onet.row_ptr)
    idx = np.concatenate([np.arange(onet.row_ptr[s], onet.row_ptr[s] + lens[s]) for s in spikers])
    flat = ((t + onet.delay[idx].astype(np.int64)) % 64) * npad + onet.post[idx]
    exp = np.bincount(flat, weights=onet.w_fx[idx].astype(np.float64), minlength=64 * npad)
    assert np.array_equal(ring, exp.astype(np.int64).reshape(64, npad))
    net.close()


def test_resident_escaped_segment_lengths(model):
    """Segments of 255 synapses or more (a sender with many synapses into one block) are
    escaped in the 8-bit length table; their group is flagged and their offsets come
    from the exact table.  Raster and state equal the oracle's."""
    n = 600
    rng = np.random.default_rng(17)
    pre = np.concatenate([np.full(700, 3), np.full(300, 40), rng.integers(0, n, 20000)])
    post = np.concatenate([rng.integers(0, 32, 700), rng.integers(64, 96, 300), rng.integers(0, n, 20000)])
    S = len(pre)
    c = dict(pre=pre, post=post, w_fx=rng.integers(-800_000, 1_600_000, S), delay=rng.integers(1, 64, S),
             u0=rng.uniform(5, 16, n).astype(np.float32), pop_offsets=[0] + [n] * 8)
    net = snn.Network(model, custom=c, seed=9, engine=RES)
    rbase, offt, lens, coarse = _tables(net)
    assert (np.diff(offt, axis=1) >= 255).any() and ((coarse[:, :-1] >> 31) == 1).any()
    onet = oracle.network_from_edges(n, c["pre"], c["post"], c["w_fx"], c["delay"], c["u0"], c["pop_offsets"])
    sim = oracle.Sim(model, onet, 9)
    net.step(300)
    g = net.read_spikes()
    o = sim.run(300)
    assert len(o[0]) > 100
    assert np.array_equal(g[0], o[0]) and np.array_equal(g[1], o[1])
    _assert_same(net, sim)
    net.close()


@pytest.mark.parametrize("rows", [0, 8, 16, 32, 64])
def test_resident_raster_state_and_ring(model, tiny, rows):
    """Tiny microcircuit, 1,000 steps in calls that start at many ring phases (each call
    is one launch): raster, U/I/R and the whole ring equal the oracle's, with the ring
    rows in shared memory capped at 8..64 (delays at or above the cap go through the
    ring in global memory)."""
    wl, onet = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, engine=RES, smem_ring_rows=rows)
    sim = oracle.Sim(model, onet, wl.seed)
    calls = [1, 2, 61, 63, 64, 65, 7, 137, 600]
    assert sum(calls) == 1000
    parts_g, parts_o = [], []
    for c in calls:
        net.step(c)
        parts_g.append(net.read_spikes())
        parts_o.append(sim.run(c))
        _assert_same(net, sim)
    g_t = np.concatenate([p[0] for p in parts_g])
    o_t = np.concatenate([p[0] for p in parts_o])
    assert np.array_equal(g_t, o_t) and len(o_t) > 1000
    assert np.array_equal(np.concatenate([p[1] for p in parts_g]), np.concatenate([p[1] for p in parts_o]))
    net.close()


def _burst_net(n, seed, syn_per_neuron=40):
    rng = np.random.default_rng(seed)
    S = n * syn_per_neuron
    pre = rng.integers(0, n, S)
    post = rng.integers(0, n, S)
    w = rng.integers(-2_000_000, 2_000_000, S)
    d = rng.integers(1, 64, S)
    u0 = np.full(n, 20.0, np.float32)  # above threshold: every neuron spikes at step 0
    u0[::3] = rng.uniform(0, 14, len(u0[::3])).astype(np.float32)
    po = [0] + [int(n * k / 8) for k in range(1, 8)] + [n]
    return dict(pre=pre, post=post, w_fx=w, delay=d, u0=u0, pop_offsets=po)


@pytest.mark.parametrize("rows", [0, 8])
def test_resident_bursts_beyond_gather_list(model, rows):
    """Two thirds of 7,000 neurons spike at step 0: a step's spike list exceeds the
    256-entry gather list (several passes) and every slot holds more spikes than its
    three entries (the rest come from the sender's outbox); 150 steps against the
    oracle."""
    m = model
    n = 7000
    c = _burst_net(n, 3)
    net = snn.Network(m, custom=c, seed=4, engine=RES, smem_ring_rows=rows)
    onet = oracle.network_from_edges(n, c["pre"], c["post"], c["w_fx"], c["delay"], c["u0"], c["pop_offsets"])
    sim = oracle.Sim(m, onet, 4)
    net.step(150)
    g = net.read_spikes()
    o = sim.run(150)
    assert (o[0] == 0).sum() > 4000
    assert np.array_equal(g[0], o[0]) and np.array_equal(g[1], o[1])
    _assert_same(net, sim)
    net.close()


@pytest.mark.parametrize("t1", [2, 63, 64])
@pytest.mark.parametrize("d", [1, 7, 8, 63])
def test_resident_hand_placed_arrival_short_window(t1, d):
    """With 8 ring rows in shared memory, delays 1 and 7 stay in shared memory and 8 and
    63 go through the global ring: a spike at t1 still reaches the target's current at
    the end of step t1 + d with the exact amplitude."""
    m = workload.microcircuit_model().replace(k_ext=[0.0] * 8)
    w2 = 12345 * 16
    c = dict(pre=[0, 1], post=[1, 2], w_fx=[200_000_000, w2], delay=[t1 - 1, d], u0=[20.0, 0.0, 0.0],
             pop_offsets=[0, 3, 3, 3, 3, 3, 3, 3, 3])
    net = snn.Network(m, custom=c, engine=RES, smem_ring_rows=8)
    onet = oracle.network_from_edges(3, c["pre"], c["post"], c["w_fx"], c["delay"], c["u0"], c["pop_offsets"])
    sim = oracle.Sim(m, onet, 1)
    t_arr = t1 + d
    for step in range(t_arr + 3):
        net.step(1)
        sim.run(1)
        _, I, _ = _state(net)
        assert I.view(np.uint32)[2] == sim.I.view(np.uint32)[2], step
        if step == t_arr:
            assert I[2] == np.float32(w2) * np.float32(2.0**-12)
    g_t, g_i = net.read_spikes()
    assert list(zip(g_t.tolist(), g_i.tolist()))[:2] == [(0, 0), (t1, 1)]
    net.close()


def test_resident_delivery_warps_do_not_change_results(model, tiny):
    wl, onet = tiny
    o = oracle.Sim(model, onet, wl.seed).run(400)
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, engine=RES)
    B = int(net.info().target_blocks)
    team = max(1, (B + 31) // 32)
    parts = []
    for k, dw in enumerate(range(2 * team, 2 * team + 6, 2)):
        net.set_schedule(delivery_warps=dw)
        assert net.info().schedule_delivery_warps == dw
        net.step(50)
        parts.append(net.read_spikes())
    net.step(400 - 50 * len(parts))
    parts.append(net.read_spikes())
    assert np.array_equal(np.concatenate([p[0] for p in parts]), o[0])
    assert np.array_equal(np.concatenate([p[1] for p in parts]), o[1])
    with pytest.raises(snn.SnnError):
        net.set_schedule(grid_ctas=10)
    with pytest.raises(snn.SnnError):
        net.set_schedule(delivery_warps=2 * team + 1)  # teams of equal size only
    net.close()


def test_resident_checkpoint_into_a_handle_that_ran_further(model, tiny):
    """A state saved at step 700 and loaded into a handle whose mailboxes already hold
    steps up to 1,500 (mailbox tags of later steps must not be taken for fresh ones)
    resumes the uninterrupted run bit for bit."""
    wl, onet = tiny
    a = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, engine=RES)
    a.step(700)
    first = a.read_spikes()
    blob = a.save_state()
    a.close()
    b = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, engine=RES)
    b.step(1500)
    b.read_spikes()
    b.load_state(blob)
    assert b.info().t == 700
    b.step(800)
    second = b.read_spikes()
    sim = oracle.Sim(model, onet, wl.seed)
    o = sim.run(1500)
    assert np.array_equal(np.concatenate([first[0], second[0]]), o[0])
    assert np.array_equal(np.concatenate([first[1], second[1]]), o[1])
    _assert_same(b, sim)
    b.close()


def test_resident_mailbox_wait_is_bounded_and_reported(model, monkeypatch):
    """Failure detection without a GPU fault: with SNN_FAULT=barrier_stall the first CTA
    waits for a mailbox tag no CTA writes; its wait gives up after 20 ms, the other
    CTAs see the recorded error and leave, the read reports SNN_ETIMEOUT, and the
    context stays usable for the next network."""
    monkeypatch.setenv("SNN_FAULT", "barrier_stall")
    net = snn.Network(model, 20, 20, seed=1, engine=RES)
    net.step(3)
    with pytest.raises(snn.SnnError) as e:
        net.read_spikes()
    assert e.value.code == snn.SNN_ETIMEOUT
    assert net.info().device_error & 2
    with pytest.raises(snn.SnnError):
        net.step(1)
    net.close()
    monkeypatch.delenv("SNN_FAULT")
    onet = oracle.build_network(model, 20, 20, 1)
    net = snn.Network(model, 20, 20, seed=1, engine=RES)
    net.step(50)
    g = net.read_spikes()
    o = oracle.Sim(model, onet, 1).run(50)
    assert np.array_equal(g[0], o[0]) and np.array_equal(g[1], o[1])
    net.close()


def test_resident_rejects_what_it_does_not_run(model):
    with pytest.raises(snn.SnnError):
        snn.Network(model, circuits=[(20, 20, 1), (30, 30, 2)], engine=RES)
    for fmt in (snn.RECORD_PACKED_I8, snn.RECORD_PACKED_BF16, snn.RECORD_BLOCKED6):
        with pytest.raises(snn.SnnError):
            snn.Network(model, 20, 20, seed=1, engine=RES, record_format=fmt)
    with pytest.raises(snn.SnnError):
        snn.Network(model, 20, 20, seed=1, engine=RES, smem_ring_rows=12)
