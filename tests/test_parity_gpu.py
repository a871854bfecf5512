"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Plain mode is bit-exact by construction (FP32 without FMA on both sides, int32
fixed-point input, the same Philox streams), so rasters, states and networks are
compared element by element with no tolerance.
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2405_02019_gb300 import build

    build.build()
    oracle.build()


def _state(net):
    n = net.n_neurons
    U = net.device_view("U", torch.float32, n).cpu().numpy()
    I = net.device_view("I", torch.float32, n).cpu().numpy()
    R = net.device_view("R", torch.uint8, n).cpu().numpy().astype(np.int32)
    return U, I, R


def _assert_same_state(net, sim):
    U, I, R = _state(net)
    assert np.array_equal(U.view(np.uint32), sim.U.view(np.uint32))
    assert np.array_equal(I.view(np.uint32), sim.I.view(np.uint32))
    assert np.array_equal(R, sim.R)


def _resident_tables(net):
    """The resident engine's block-major tables (rbase, offt) read back from the arena."""
    n, B = net.n_neurons, int(net.info().target_blocks)
    up = lambda x: (x + 255) // 256 * 256  # noqa: E731
    coarse_stride = (n + 31) // 32 + 1
    lens_stride = (n + 31) // 32 * 32
    o_coarse = up(8 * (B + 1))
    o_lens = up(o_coarse + 4 * B * coarse_stride)
    o_offt = up(o_lens + B * lens_stride)
    base = int(net.layout().block_starts)
    region = net._arena[net._arena_ptr - net._arena.data_ptr() + base:][: o_offt + 4 * B * (n + 1)]
    raw = region.cpu().numpy()
    rbase = raw[: 8 * (B + 1)].view(np.int64)
    coarse = raw[o_coarse: o_coarse + 4 * B * coarse_stride].view(np.uint32).reshape(B, coarse_stride)
    lens = raw[o_lens: o_lens + B * lens_stride].reshape(B, lens_stride)
    offt = raw[o_offt: o_offt + 4 * B * (n + 1)].view(np.uint32).reshape(B, n + 1).astype(np.int64)
    return rbase, offt, lens, coarse


def _device_network(net):
    """(row_ptr, post, w, delay) of the device network in row form: rows padded to
    multiples of 4 with entries that deliver nothing.  The resident engine stores its
    records block-major; its rows are reassembled here, each grouped by target block."""
    lay = net.layout()
    n = net.n_neurons
    sp = int(lay.n_synapses_padded)
    tg = net.device_view("syn_tgt", torch.int32, sp).cpu().numpy()
    w = net.device_view("syn_w", torch.int32, sp).cpu().numpy()
    d = net.device_view("syn_delay", torch.uint8, sp).cpu().numpy()
    if net.info().engine != RES:
        rp = net.device_view("row_ptr", torch.int64, n + 1).cpu().numpy()
        return rp, tg, w, d
    rbase, offt, _, _ = _resident_tables(net)
    lens = np.diff(offt, axis=1)                                  # [block][sender]
    sender = np.concatenate([np.repeat(np.arange(n), lens[b]) for b in range(len(lens))])
    order = np.argsort(sender, kind="stable")                     # by sender, blocks in order
    deg = lens.sum(axis=0)
    plen = (deg + 3) // 4 * 4
    rp = np.concatenate([[0], np.cumsum(plen)]).astype(np.int64)
    pos = np.arange(len(order)) - np.repeat(np.concatenate([[0], np.cumsum(deg)[:-1]]), deg) \
        + np.repeat(rp[:-1], deg)
    T = np.repeat(np.arange(n, dtype=np.int32), plen)             # padding: onto the sender, w = 0
    W = np.zeros(rp[-1], np.int32)
    D = np.ones(rp[-1], np.uint8)
    T[pos], W[pos], D[pos] = tg[order], w[order], d[order]
    return rp, T, W, D


def _resident_rows(net, rows):
    """The resident engine's rows `rows` reassembled from the block-major regions (sampled
    rows of a large network); returns {row: (post, w, delay)}."""
    rbase, offt, _, _ = _resident_tables(net)
    sp = int(net.layout().n_synapses_padded)
    tg = net.device_view("syn_tgt", torch.int32, sp).cpu().numpy()
    w = net.device_view("syn_w", torch.int32, sp).cpu().numpy()
    d = net.device_view("syn_delay", torch.uint8, sp).cpu().numpy()
    out = {}
    for i in rows:
        idx = np.concatenate([np.arange(rbase[b] + offt[b, i], rbase[b] + offt[b, i + 1]) for b in range(len(offt))])
        out[int(i)] = (tg[idx], w[idx], d[idx])
    return out


def _block_bounds(net):
    """Target-block boundaries of a resident-engine network (None for other engines)."""
    info = net.info()
    if info.engine != snn.ENGINE_RESIDENT:
        return None
    return net.device_view("blocks", torch.int32, int(info.target_blocks) + 1).cpu().numpy().astype(np.int64)


def _assert_row_order(bounds, tg, d, starts, lens):
    """Rows are delay-sorted (indexed store of §3.5); on the resident engine grouped by
    target block first, delay-sorted inside each block."""
    for a, L in zip(starts, lens):
        seg_d = d[a:a + L].astype(np.int64)
        key = seg_d if bounds is None else (np.searchsorted(bounds, tg[a:a + L], side="right") - 1) * 64 + seg_d
        assert np.all(np.diff(key) >= 0)


def _row_multisets_equal(onet, rp, tg, w, d, bounds=None):
    n = onet.n
    lens = np.diff(onet.row_ptr)
    plen = np.diff(rp)
    assert np.all(plen % 4 == 0) and np.all(plen >= lens) and np.all(plen - lens < 4)
    pos = np.arange(rp[-1]) - np.repeat(rp[:-1], plen)
    real = pos < np.repeat(lens, plen)
    assert np.all(w[: rp[-1]][~real] == 0)
    pre_l = np.repeat(np.arange(n), plen)[real]
    tl, wl, dl = tg[: rp[-1]][real], w[: rp[-1]][real], d[: rp[-1]][real]
    sample = np.arange(0, n, max(1, n // 200))
    _assert_row_order(bounds, tg, d, rp[sample], lens[sample])
    pre_o = np.repeat(np.arange(n), lens)
    ko = np.lexsort((onet.w_fx, onet.delay, onet.post, pre_o))
    kl = np.lexsort((wl, dl, tl, pre_l))
    assert np.array_equal(pre_o[ko], pre_l[kl])
    assert np.array_equal(onet.post[ko], tl[kl])
    assert np.array_equal(onet.delay[ko], dl[kl])
    assert np.array_equal(onet.w_fx[ko], wl[kl])


@pytest.fixture(scope="module")
def model():
    return workload.microcircuit_model()


@pytest.fixture(scope="module")
def tiny(model):
    wl = workload.WORKLOADS["pd_tiny"]
    onet = oracle.build_network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed)
    return wl, onet


def test_constants_bit_identical(model, tiny):
    wl, _ = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed)
    info = net.info()
    c = oracle.constants(model)
    s = oracle.step_constants(model)
    for k in ("w_f", "p11", "p22", "p21"):
        assert getattr(info, k) == c[k], k
    assert np.float32(info.p11_f32) == s["p11"] and np.float32(info.p21_f32) == s["p21"]
    assert np.float32(info.p22_f32) == s["p22"] and np.float32(info.theta_f32) == s["theta"]
    assert np.float32(info.u_reset_f32) == s["u_reset"]
    assert info.t_ref_steps == s["t_ref"] and info.w_ext_fx == s["w_ext_fx"]
    thr = np.ctypeslib.as_array(info.poisson_thresholds)
    for b in range(8):
        assert np.array_equal(thr[b], oracle.poisson_table(model, b))
    net.close()


def test_network_identical_tiny(model, tiny):
    wl, onet = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed)
    assert net.info().n_synapses == len(onet.post)
    _row_multisets_equal(onet, *_device_network(net))
    U, _, _ = _state(net)
    assert np.array_equal(U.view(np.uint32), onet.u0.view(np.uint32))
    net.close()


GRAPH, PERSIST, PIPE, RES = snn.ENGINE_GRAPH, snn.ENGINE_PERSISTENT, snn.ENGINE_PIPELINED, snn.ENGINE_RESIDENT
ENGINES = [GRAPH, PERSIST, PIPE, RES]


@pytest.mark.parametrize("engine,spg", [(GRAPH, 96), (GRAPH, 1000), (PERSIST, 0), (PIPE, 96), (PIPE, 1000),
                                        (RES, 0)])
def test_raster_bit_exact_tiny(model, tiny, engine, spg):
    """Tiny microcircuit (7,718 neurons, 2.85e6 synapses), 1,000 steps: identical raster
    and final state.  spg=96 mixes graph replays with directly launched remainders."""
    wl, onet = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, steps_per_graph=spg,
                      engine=engine)
    assert net.info().engine == engine
    net.step(wl.steps)
    g_t, g_i = net.read_spikes()
    sim = oracle.Sim(model, onet, wl.seed)
    o_t, o_i = sim.run(wl.steps)
    assert len(o_t) > 1000
    assert np.array_equal(g_t, o_t) and np.array_equal(g_i, o_i)
    _assert_same_state(net, sim)
    info = net.info()
    assert info.spikes_read == len(o_t)
    assert info.events_read == int(np.diff(onet.row_ptr)[o_i].sum())
    net.close()


@pytest.mark.parametrize("engine", ENGINES)
def test_incremental_reads_and_rates(model, tiny, engine):
    wl, onet = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, steps_per_graph=50,
                      engine=engine)
    parts = []
    for n in (1, 7, 120, 372):
        net.step(n)
        parts.append(net.read_spikes())
    g_t = np.concatenate([p[0] for p in parts])
    g_i = np.concatenate([p[1] for p in parts])
    sim = oracle.Sim(model, onet, wl.seed)
    o_t, o_i = sim.run(500)
    assert np.array_equal(g_t, o_t) and np.array_equal(g_i, o_i)
    rates, counts = net.read_rates(100, 500)
    sel = (o_t >= 100) & (o_t < 500)
    exp_counts = np.bincount(o_i[sel], minlength=onet.n)
    assert np.array_equal(counts, exp_counts)
    sizes = np.diff(onet.pop_off)
    pops = np.searchsorted(onet.pop_off, o_i[sel], side="right") - 1
    exp_rates = np.bincount(pops, minlength=8) / (sizes * 400 * 1e-4)
    np.testing.assert_allclose(rates, exp_rates, rtol=1e-12)
    net.close()


def _collect_run(net, calls, overlapped=True):
    """step(n); collect_spikes() for every n, then a blocking read; returns the raster.
    overlapped: no collect may fall back to waiting (the raster is large enough), so each
    returns steps of earlier calls only."""
    parts, t = [], 0
    for n in calls:
        net.step(n)
        st, si = net.collect_spikes()
        assert len(st) == 0 or st.max() < (t if overlapped else t + n)
        assert np.all(np.diff(st) >= 0)
        parts.append((st, si))
        t += n
    parts.append(net.read_spikes())
    g_t = np.concatenate([p[0] for p in parts])
    g_i = np.concatenate([p[1] for p in parts])
    order = np.lexsort((g_i, g_t))
    assert np.array_equal(order, np.arange(len(g_t)))  # ordered by (step, neuron) overall
    return g_t, g_i


@pytest.mark.parametrize("engine", ENGINES)
def test_collect_overlapped_reads(model, tiny, engine):
    """Overlapped reads (snn_collect_spikes after every step call, uneven call sizes,
    graph replays and remainders) return the oracle's raster, each spike once."""
    wl, onet = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, steps_per_graph=64,
                      engine=engine)
    calls = [1, 7, 120, 372, 64, 100, 136]
    g_t, g_i = _collect_run(net, calls)
    o_t, o_i = oracle.Sim(model, onet, wl.seed).run(sum(calls))
    assert np.array_equal(g_t, o_t) and np.array_equal(g_i, o_i)
    net.close()


def test_collect_small_raster_and_circuit_groups(model, tiny):
    """A raster that holds about four calls' spikes (collect falls back to waiting reads),
    and circuit groups (a call's raster is not in step order)."""
    wl, onet = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, steps_per_graph=64,
                      raster_capacity=10000)
    g_t, g_i = _collect_run(net, [100] * 8, overlapped=False)
    o_t, o_i = oracle.Sim(model, onet, wl.seed).run(800)
    assert np.array_equal(g_t, o_t) and np.array_equal(g_i, o_i)
    net.close()
    ref = snn.Network(model, circuits=BATCH, steps_per_graph=64, engine=GRAPH)
    ref.step(300)
    r_t, r_i = ref.read_spikes()
    ref.close()
    net = snn.Network(model, circuits=BATCH, steps_per_graph=64, engine=GRAPH)
    net.set_circuit_groups(2)
    g_t, g_i = _collect_run(net, [64, 100, 36, 100])
    assert np.array_equal(g_t, r_t) and np.array_equal(g_i, r_i)
    net.close()


@pytest.mark.parametrize("engine", ENGINES)
def test_profile_steps_same_dynamics(model, tiny, engine):
    """The kernel-by-kernel timing path computes the same steps as either engine, and
    can be interleaved with it."""
    wl, onet = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, steps_per_graph=64,
                      engine=engine)
    net.step(100)
    mu, md = net.profile_steps(300)
    assert mu > 0 and (md > 0 or engine == RES)  # the resident launch runs both phases
    net.step(100)
    g_t, g_i = net.read_spikes()
    o_t, o_i = oracle.Sim(model, onet, wl.seed).run(500)
    assert np.array_equal(g_t, o_t) and np.array_equal(g_i, o_i)
    net.close()


@pytest.mark.parametrize("nspk", [1, 37, 700])
def test_deliver_spikes_matches_oracle_network(model, tiny, nspk):
    """Phase 2 alone (snn_deliver_spikes) on a zero ring: every cell equals the sum of
    w over the senders' synapses with (t + d) mod 64 and that target (repeats kept)."""
    wl, onet = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed)
    assert np.array_equal(net.out_degrees(), np.diff(onet.row_ptr))
    rng = np.random.default_rng(nspk)
    spikers = rng.integers(0, onet.n, nspk).astype(np.int32)
    t = 61
    net.deliver_spikes(torch.from_numpy(spikers).cuda(), t)
    torch.cuda.synchronize()
    npad = int(net.layout().n_neurons_padded)
    ring = net.device_view("ring", torch.int32, 64 * npad).cpu().numpy().reshape(64, npad).astype(np.int64)
    exp = np.zeros((64, npad), np.int64)
    for s_ in spikers:
        a, b = onet.row_ptr[s_], onet.row_ptr[s_ + 1]
        np.add.at(exp, ((t + onet.delay[a:b].astype(np.int64)) % 64, onet.post[a:b]), onet.w_fx[a:b])
    assert np.array_equal(ring, exp)
    net.close()


# ------------------------------------------------------------ hand-placed spikes


def _chain(d_first, d_second, w2):
    big = 200_000_000
    return dict(pre=[0, 1], post=[1, 2], w_fx=[big, w2], delay=[d_first, d_second], u0=[20.0, 0.0, 0.0],
                pop_offsets=[0, 3, 3, 3, 3, 3, 3, 3, 3])


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("t1", [2, 62, 63, 64])
@pytest.mark.parametrize("d", [1, 15, 16, 63])
def test_hand_placed_spike_arrival(t1, d, engine):
    """A spike at step t1 with delay d reaches the target's current at the end of step
    t1 + d, with the exact amplitude, on the GPU as in the oracle (ring wrap included)."""
    m = workload.microcircuit_model().replace(k_ext=[0.0] * 8)
    w2 = 12345 * 16
    c = _chain(t1 - 1, d, w2)
    net = snn.Network(m, custom=c, steps_per_graph=7, engine=engine)
    onet = oracle.network_from_edges(3, c["pre"], c["post"], c["w_fx"], c["delay"], c["u0"], c["pop_offsets"])
    sim = oracle.Sim(m, onet, 1)
    t_arr = t1 + d
    for step in range(t_arr + 3):
        net.step(1)
        sim.run(1)
        _, I, _ = _state(net)
        assert I.view(np.uint32)[2] == sim.I.view(np.uint32)[2], step
        if step == t_arr - 1:
            assert I[2] == 0.0
        if step == t_arr:
            assert I[2] == np.float32(w2) * np.float32(2.0**-12)
    g_t, g_i = net.read_spikes()
    assert list(zip(g_t.tolist(), g_i.tolist()))[:2] == [(0, 0), (t1, 1)]
    net.close()


# ------------------------------------------------------------------ edge cases


def _custom_parity(m, custom, steps, spg=16, seed=5, engine=GRAPH, **kw):
    n = len(custom["u0"])
    net = snn.Network(m, custom=custom, steps_per_graph=spg, seed=seed, engine=engine, **kw)
    onet = oracle.network_from_edges(n, custom["pre"], custom["post"], custom["w_fx"], custom["delay"],
                                     custom["u0"], custom.get("pop_offsets"))
    sim = oracle.Sim(m, onet, seed)
    net.step(steps)
    g = net.read_spikes()
    o = sim.run(steps)
    assert np.array_equal(g[0], o[0]) and np.array_equal(g[1], o[1])
    _assert_same_state(net, sim)
    net.close()
    return o


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("n", [1, 3, 13, 129, 517])
def test_ragged_neuron_counts_no_synapses(n, engine):
    """Neuron counts that fill neither a quad nor a 128-wide ring row; no synapses;
    thalamic drive only (population 0 = L23E)."""
    m = workload.microcircuit_model()
    rng = np.random.default_rng(n)
    u0 = rng.uniform(0, 16, n).astype(np.float32)
    custom = dict(pre=[], post=[], w_fx=[], delay=[], u0=u0, pop_offsets=[0] + [n] * 8)
    o = _custom_parity(m, custom, 300, engine=engine)
    assert len(o[0]) > 0


@pytest.mark.parametrize("engine", ENGINES)
def test_long_rows_ragged_chunks_and_all_delays(engine):
    """Rows longer than one 256-synapse chunk with ragged tails, every delay 1..63,
    multapses and autapses, mixed signs, several populations."""
    m = workload.microcircuit_model()
    rng = np.random.default_rng(11)
    n = 301
    pre, post, w, d = [], [], [], []
    for s, L in ((0, 1), (5, 255), (6, 256), (7, 257), (8, 1000), (9, 3001), (300, 513)):
        pre += [s] * L
        post += list(rng.integers(0, n, L))
        w += list(rng.integers(-3_000_000, 3_000_000, L))
        d += list(rng.integers(1, 64, L))
    pre += [10] * 64
    post += [10] * 64          # autapses, each delay once
    w += [400_000] * 64
    d += list(range(1, 64)) + [63]
    u0 = rng.uniform(10, 16, n).astype(np.float32)
    po = [0, 40, 80, 120, 160, 200, 240, 280, n]
    custom = dict(pre=pre, post=post, w_fx=w, delay=d, u0=u0, pop_offsets=po)
    o = _custom_parity(m, custom, 400, spg=33, engine=engine)
    assert len(o[0]) > 50


@pytest.mark.parametrize("engine", ENGINES)
def test_raster_overflow_is_reported(model, engine):
    """A raster smaller than the spikes of the run fails loudly with SNN_EOVERFLOW."""
    net = snn.Network(model, 20, 20, seed=1, raster_capacity=64, engine=engine)
    net.step(300)
    with pytest.raises(snn.SnnError) as e:
        net.read_spikes()
    assert e.value.code == snn.SNN_EOVERFLOW
    assert b"raster" in net.info().last_error  # also kept on the handle
    with pytest.raises(snn.SnnError):
        net.step(1)
    assert b"device error" in net.info().last_error
    net.close()


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("scale", [(1, 1), (5, 300), (300, 5)])
def test_extreme_scales(model, scale, engine):
    sn, sk = scale
    onet = oracle.build_network(model, sn, sk, 9)
    net = snn.Network(model, sn, sk, seed=9, steps_per_graph=40, engine=engine)
    _row_multisets_equal(onet, *_device_network(net), bounds=_block_bounds(net))
    net.step(250)
    g = net.read_spikes()
    sim = oracle.Sim(model, onet, 9)
    o = sim.run(250)
    assert np.array_equal(g[0], o[0]) and np.array_equal(g[1], o[1])
    _assert_same_state(net, sim)
    net.close()


def test_zero_steps_and_empty_reads(model):
    net = snn.Network(model, 20, 20, seed=2)
    net.step(0)
    t, i = net.read_spikes()
    assert len(t) == 0
    net.close()


# ------------------------------------------------------- full-scale microcircuit


@pytest.fixture(scope="module")
def full(model):
    wl = workload.WORKLOADS["pd_full"]
    onet = oracle.build_network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed)
    return wl, onet


def _rows_equal_sampled(onet, rp, tg, w, d, rows, bounds=None):
    """Exact per-row multiset comparison for the given rows, plus global sums over all
    synapses (the full sort of 2.8e8 records is left to the smaller scales)."""
    lens = np.diff(onet.row_ptr)
    plen = np.diff(rp)
    assert np.all(plen % 4 == 0) and np.all(plen >= lens) and np.all(plen - lens < 4)
    for i in rows:
        a, L = onet.row_ptr[i], lens[i]
        b = rp[i]
        o = np.sort(onet.post[a:a + L].astype(np.int64) << 38 | onet.delay[a:a + L].astype(np.int64) << 32
                    | (onet.w_fx[a:a + L].astype(np.int64) + 2**31))
        g = np.sort(tg[b:b + L].astype(np.int64) << 38 | d[b:b + L].astype(np.int64) << 32
                    | (w[b:b + L].astype(np.int64) + 2**31))
        assert np.array_equal(o, g), i
        _assert_row_order(bounds, tg, d, [b], [L])
        assert np.all(w[b + L:rp[i + 1]] == 0)
    n_real = rp[-1]
    assert int(w[:n_real].astype(np.int64).sum()) == int(onet.w_fx.astype(np.int64).sum())
    assert int(tg[:n_real].astype(np.int64).sum()) - int(
        (np.repeat(np.arange(onet.n), plen - lens)).sum()) == int(onet.post.astype(np.int64).sum())
    assert int(d[:n_real].astype(np.int64).sum()) - int((plen - lens).sum()) == int(
        onet.delay.astype(np.int64).sum())


@pytest.mark.parametrize("engine", [snn.ENGINE_DEFAULT, GRAPH, RES])
def test_full_scale_parity(model, full, engine):
    """Full microcircuit (77,169 neurons, 284,811,022 synapses) in the bench's launch
    configuration (default engine) and with the graph engine: the network (every row
    that spikes in the window, 2,000 random rows, global sums), and an identical raster
    and state over the first 1,200 steps (120 ms of biological time)."""
    wl, onet = full
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, engine=engine)
    assert net.info().n_synapses == 284_811_022
    steps = 1200
    net.step(steps)
    g_t, g_i = net.read_spikes()
    sim = oracle.Sim(model, onet, wl.seed)
    o_t, o_i = sim.run(steps)
    assert len(o_t) > 0
    assert np.array_equal(g_t, o_t) and np.array_equal(g_i, o_i)
    _assert_same_state(net, sim)
    rng = np.random.default_rng(0)
    if engine == RES:
        # block-major records: sampled rows reassembled from the 151 block regions
        rows = np.unique(np.concatenate([rng.choice(o_i, 300), rng.integers(0, onet.n, 700)]))
        got = _resident_rows(net, rows)
        bounds = _block_bounds(net)
        for i in rows:
            a, L = onet.row_ptr[i], onet.row_ptr[i + 1] - onet.row_ptr[i]
            o = np.sort(onet.post[a:a + L].astype(np.int64) << 38 | onet.delay[a:a + L].astype(np.int64) << 32
                        | (onet.w_fx[a:a + L].astype(np.int64) + 2**31))
            tg, w, d = got[int(i)]
            g = np.sort(tg.astype(np.int64) << 38 | d.astype(np.int64) << 32 | (w.astype(np.int64) + 2**31))
            assert np.array_equal(o, g), i
            _assert_row_order(bounds, tg, d, [0], [L])
        sp = int(net.layout().n_synapses_padded)
        assert sp == len(onet.post)
        assert int(net.device_view("syn_w", torch.int32, sp).cpu().numpy().astype(np.int64).sum()) == \
            int(onet.w_fx.astype(np.int64).sum())
    else:
        rows = np.unique(np.concatenate([o_i, rng.integers(0, onet.n, 2000)]))
        _rows_equal_sampled(onet, *_device_network(net), rows, bounds=_block_bounds(net))
    net.close()


def test_full_scale_activity_band(model, full):
    """The paper reports ~23 spiking neurons per step on average at full scale (a weak
    band: flagged, not failed, outside 5..100 per step); the GPU run must stay free
    of raster overflow over 1 s of biological time."""
    wl, _ = full
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed)
    net.step(10000)
    t, i = net.read_spikes()
    per_step = len(t) / 10000.0
    assert per_step > 0.5
    if not (5 <= per_step <= 100):
        import warnings

        warnings.warn(f"full-scale activity {per_step:.1f} spikes/step is outside the paper's band")
    net.close()


def test_barrier_wait_is_bounded_and_reported(model, monkeypatch):
    """Failure detection without a GPU fault: with SNN_FAULT=barrier_stall every grid
    barrier of the persistent engine waits for an arrival that never comes; the wait
    gives up after its 20 ms bound, the run reports SNN_ETIMEOUT, and the context stays
    usable for the next network."""
    monkeypatch.setenv("SNN_FAULT", "barrier_stall")
    net = snn.Network(model, 20, 20, seed=1, engine=PERSIST)
    net.step(3)
    with pytest.raises(snn.SnnError) as e:
        net.read_spikes()
    assert e.value.code == snn.SNN_ETIMEOUT
    assert net.info().device_error & 2
    net.close()
    monkeypatch.delenv("SNN_FAULT")
    onet = oracle.build_network(model, 20, 20, 1)
    net = snn.Network(model, 20, 20, seed=1, engine=PERSIST)
    net.step(50)
    g = net.read_spikes()
    o = oracle.Sim(model, onet, 1).run(50)
    assert np.array_equal(g[0], o[0]) and np.array_equal(g[1], o[1])
    net.close()


@pytest.mark.parametrize("engine", ENGINES)
def test_checkpoint_resume_is_bit_exact(model, tiny, engine):
    """2,000 steps straight equal 1,000 steps, save, restore into a fresh handle, 1,000
    more steps (counter-based random numbers make the resumed run identical)."""
    wl, onet = tiny
    a = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, steps_per_graph=128, engine=engine)
    a.step(2000)
    full_t, full_i = a.read_spikes()
    U_a, I_a, R_a = _state(a)
    b = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, steps_per_graph=128, engine=engine)
    b.step(1000)
    first = b.read_spikes()
    blob = b.save_state()
    b.close()
    c = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, steps_per_graph=128, engine=engine)
    c.load_state(blob)
    assert c.info().t == 1000
    c.step(1000)
    second = c.read_spikes()
    assert np.array_equal(np.concatenate([first[0], second[0]]), full_t)
    assert np.array_equal(np.concatenate([first[1], second[1]]), full_i)
    U_c, I_c, R_c = _state(c)
    assert np.array_equal(U_a.view(np.uint32), U_c.view(np.uint32))
    assert np.array_equal(I_a.view(np.uint32), I_c.view(np.uint32)) and np.array_equal(R_a, R_c)
    o = oracle.Sim(model, onet, wl.seed).run(2000)
    assert np.array_equal(o[0], full_t) and np.array_equal(o[1], full_i)
    a.close()
    c.close()


def test_load_state_rejects_other_shapes(model):
    a = snn.Network(model, 20, 20, seed=1)
    blob = a.save_state()
    b = snn.Network(model, 30, 20, seed=1)
    with pytest.raises(snn.SnnError):
        b.load_state(blob)
    with pytest.raises(snn.SnnError):
        a.load_state(b"not a state")
    a.close()
    b.close()


# ------------------------------------------------------- compressed synapse records

FORMATS = [snn.RECORD_PACKED_I8, snn.RECORD_PACKED_BF16]


def _oracle_weights(onet, fmt):
    if fmt == snn.RECORD_PACKED_I8:
        return oracle.quantize_i8(onet)[0]
    return oracle.quantize_bf16(onet.w_fx)


def _decode_device_records(net, fmt):
    """(row_ptr, target, delay, target population, pad flag, read-back weight) from the
    device arena, decoded in numpy from the format's definition."""
    lay = net.layout()
    n = net.n_neurons
    sp = int(lay.n_synapses_padded)
    rp = net.device_view("row_ptr", torch.int64, n + 1).cpu().numpy()
    word = net.device_view("syn_tgt", torch.int32, sp).cpu().numpy().view(np.uint32)
    tgt = (word & 0xFFFFF).astype(np.int32)
    d = ((word >> 20) & 63).astype(np.uint8)
    pop = ((word >> 26) & 7).astype(np.int64)
    pad = (word >> 31).astype(bool)
    info = net.info()
    if fmt == snn.RECORD_PACKED_I8:
        code = net.device_view("syn_w", torch.int8, sp).cpu().numpy().astype(np.int64)
        base = np.ctypeslib.as_array(info.i8_base).astype(np.int64)
        step = np.ctypeslib.as_array(info.i8_step).astype(np.int64)
        src = np.repeat(np.searchsorted(np.ctypeslib.as_array(info.pop_offsets)[1:8], np.arange(n), side="right"),
                        np.diff(rp))
        w = base[src, pop] + code * step[src, pop]
    else:
        h = net.device_view("syn_w", torch.int16, sp).cpu().numpy().view(np.uint16).astype(np.uint32) << 16
        w = (h.view(np.float32) * np.float32(4096.0)).astype(np.int64)
    return rp, tgt, d, pop, pad, w


@pytest.mark.parametrize("fmt", FORMATS)
def test_packed_records_decode_to_oracle_quantization(model, tiny, fmt):
    wl, onet = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, record_format=fmt)
    info = net.info()
    assert info.record_format == fmt and info.bytes_per_synapse == (5 if fmt == snn.RECORD_PACKED_I8 else 6)
    if fmt == snn.RECORD_PACKED_I8:
        _, base, step = oracle.quantize_i8(onet)
        assert np.array_equal(np.ctypeslib.as_array(info.i8_base), base)
        assert np.array_equal(np.ctypeslib.as_array(info.i8_step), step)
    rp, tgt, d, pop, pad, w = _decode_device_records(net, fmt)
    lens = np.diff(onet.row_ptr)
    plen = np.diff(rp)
    pos = np.arange(rp[-1]) - np.repeat(rp[:-1], plen)
    real = pos < np.repeat(lens, plen)
    assert np.array_equal(pad[: rp[-1]], ~real)
    assert np.array_equal(pop[: rp[-1]][real], np.searchsorted(onet.pop_off[1:8], tgt[: rp[-1]][real], side="right"))
    qw = _oracle_weights(onet, fmt)
    ow = oracle.with_weights(onet, qw)
    _row_multisets_equal(ow, rp, tgt, np.where(real, w[: rp[-1]], 0).astype(np.int32), d)
    net.close()


@pytest.mark.parametrize("engine", [PIPE, GRAPH])
@pytest.mark.parametrize("fmt", FORMATS)
def test_packed_raster_bit_exact_tiny(model, tiny, fmt, engine):
    """The compressed forms are bit-exact against the oracle run on the same read-back
    weights (integer dequantisation), which pins the kernels apart from the precision
    loss."""
    wl, onet = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, record_format=fmt,
                      engine=engine, steps_per_graph=128)
    net.step(wl.steps)
    g_t, g_i = net.read_spikes()
    sim = oracle.Sim(model, oracle.with_weights(onet, _oracle_weights(onet, fmt)), wl.seed)
    o_t, o_i = sim.run(wl.steps)
    assert np.array_equal(g_t, o_t) and np.array_equal(g_i, o_i)
    _assert_same_state(net, sim)
    net.close()


@pytest.mark.parametrize("fmt", FORMATS)
def test_packed_deliver_spikes_match(model, tiny, fmt):
    wl, onet = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, record_format=fmt)
    qw = _oracle_weights(onet, fmt)
    spikers = np.random.default_rng(5).integers(0, onet.n, 300).astype(np.int32)
    net.deliver_spikes(torch.from_numpy(spikers).cuda(), 9)
    torch.cuda.synchronize()
    npad = int(net.layout().n_neurons_padded)
    ring = net.device_view("ring", torch.int32, 64 * npad).cpu().numpy().reshape(64, npad).astype(np.int64)
    exp = np.zeros((64, npad), np.int64)
    for s_ in spikers:
        a, b = onet.row_ptr[s_], onet.row_ptr[s_ + 1]
        np.add.at(exp, ((9 + onet.delay[a:b].astype(np.int64)) % 64, onet.post[a:b]), qw[a:b])
    assert np.array_equal(ring, exp)
    net.close()


@pytest.mark.parametrize("fmt", FORMATS)
def test_packed_full_scale_parity(model, full, fmt):
    """Full microcircuit with compressed records, default engine: raster and state
    identical to the oracle on the read-back weights over 600 steps."""
    wl, onet = full
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, record_format=fmt)
    net.step(600)
    g_t, g_i = net.read_spikes()
    sim = oracle.Sim(model, oracle.with_weights(onet, _oracle_weights(onet, fmt)), wl.seed)
    o_t, o_i = sim.run(600)
    assert len(o_t) > 0
    assert np.array_equal(g_t, o_t) and np.array_equal(g_i, o_i)
    _assert_same_state(net, sim)
    net.close()


def test_static_step_rejects_packed(model):
    import ctypes as C
    from paper_2405_02019_gb300 import _abi

    net = snn.Network(model, 20, 20, seed=1, record_format=snn.RECORD_PACKED_I8)
    io = _abi.snn_static_io()
    rc = snn.load().snn_step_static(C.c_void_p(net._handle), C.byref(io), 1, 0, None)
    assert rc == _abi.SNN_ENOTSUP
    net.close()



# ------------------------------------------------------------ batched circuits

BATCH = [(20, 40, 5), (35, 10, 6), (13, 50, 7), (50, 50, 8), (1, 1, 9)]


# ------------------------------------------------------------ blocked records

BLK = snn.RECORD_BLOCKED6


def _bf16_fx(h):
    """bfloat16 currents (uint16) read back as 2^-12 pA, as the device does."""
    f = (h.astype(np.uint32) << 16).view(np.float32)
    return np.rint(f * np.float32(4096.0)).astype(np.int32)


def _check_blocked_structure(net, onet, rows=None):
    """Decodes the blocked records in the arena and compares them with the oracle's
    network: every synapse (rows=None) or the given rows exactly plus global sums.
    Zero weights mark the padding that ends every (row, block) segment on a quad.
    For BLOCKED4 `onet` must carry the read-back (bfloat16) weights."""
    info = net.info()
    n, B, S = net.n_neurons, info.target_blocks, info.n_synapses
    SP = int(net.layout().n_synapses_padded)
    blk = net.device_view("blocks", torch.int32, B + 1).cpu().numpy().astype(np.int64)
    rp = net.device_view("row_ptr", torch.int64, n + 1).cpu().numpy()
    seg = net.device_view("syn_delay", torch.int16, n * (B + 1)).cpu().numpy().view(np.uint16)
    seg = seg.reshape(n, B + 1).astype(np.int64)
    q = 4  # records per padding unit (a quad)
    LM, DS = 1023, 10  # record = local target | delay << DS
    if info.record_format == snn.RECORD_BLOCKED8:
        pairs = net.device_view("syn_tgt", torch.int32, 2 * SP).cpu().numpy().reshape(-1, 2)
        w = np.ascontiguousarray(pairs[:, 0])
        rec = pairs[:, 1].astype(np.int64)  # local target (16 bits) | delay << 16
        LM, DS = 0xFFFF, 16
    elif info.record_format == snn.RECORD_BLOCKED4:
        quads = net.device_view("syn_tgt", torch.int16, 2 * SP).cpu().numpy().view(np.uint16).reshape(-1, 8)
        rec = np.ascontiguousarray(quads[:, :4]).reshape(-1)
        w = _bf16_fx(np.ascontiguousarray(quads[:, 4:]).reshape(-1))
    else:
        rec = net.device_view("syn_tgt", torch.int16, SP).cpu().numpy().view(np.uint16)
        w = net.device_view("syn_w", torch.int32, SP).cpu().numpy()
    assert blk[0] == 0 and blk[-1] == n and np.all(np.diff(blk) > 0)
    assert np.all(blk[1:-1] % 32 == 0) and np.all(np.diff(blk) <= 768)
    lens = np.diff(onet.row_ptr)
    plen = np.diff(rp)
    assert rp[0] == 0 and rp[-1] == SP and np.all(plen >= lens) and np.all(rp % q == 0)
    assert np.all(seg[:, 0] == 0) and np.array_equal(seg[:, -1], plen) and np.all(np.diff(seg, axis=1) >= 0)
    assert np.all(seg % q == 0)
    real = w != 0
    assert int(real.sum()) == S and np.all(rec[~real] == 1 << DS)  # padding: local 0, delay 1
    # block of every entry, segment starts, then chunked decode
    bid = np.repeat(np.tile(np.arange(B, dtype=np.int16), n), np.diff(seg, axis=1).ravel())
    start = np.zeros(SP + 1, bool)
    start[(rp[:-1, None] + seg[:, :-1]).ravel()] = True
    width = np.diff(blk)
    sums = np.zeros(3, np.int64)
    for c0 in range(0, SP, 1 << 24):
        c1 = min(SP, c0 + (1 << 24))
        r = rec[c0:c1].astype(np.int64)
        b = bid[c0:c1].astype(np.int64)
        rl = real[c0:c1]
        local, d = r & LM, r >> DS
        assert np.all(local < width[b])
        # padding only after the real entries of a segment; delay order among them
        assert not np.any(~rl[:-1] & rl[1:] & ~start[c0 + 1:c1])
        dd = np.diff(d)
        assert np.all(dd[~start[c0 + 1:c1] & rl[1:] & rl[:-1]] >= 0)
        sums += [int((blk[b] + local)[rl].sum()), int(d[rl].sum()), int(w[c0:c1].astype(np.int64).sum())]
    assert sums[0] == int(onet.post.astype(np.int64).sum())
    assert sums[1] == int(onet.delay.astype(np.int64).sum())
    assert sums[2] == int(onet.w_fx.astype(np.int64).sum())
    if rows is None:
        rows = np.arange(n)
        # fewer than q padding entries per segment
        segid = np.repeat(np.arange(n * B), np.diff(seg, axis=1).ravel())
        pads = np.bincount(segid[~real], minlength=n * B)
        assert pads.max() < q
    for i in rows:
        a, L = onet.row_ptr[i], lens[i]
        sl = slice(rp[i], rp[i + 1])
        keep = real[sl]
        r = rec[sl].astype(np.int64)[keep]
        tg = blk[bid[sl].astype(np.int64)[keep]] + (r & LM)
        o = np.sort(onet.post[a:a + L].astype(np.int64) << 38 | onet.delay[a:a + L].astype(np.int64) << 32
                    | (onet.w_fx[a:a + L].astype(np.int64) + 2**31))
        g = np.sort(tg << 38 | (r >> DS) << 32 | (w[sl][keep].astype(np.int64) + 2**31))
        assert np.array_equal(o, g), i
    # blocks balanced by in-degree (the heaviest within 30 % of the mean, up to one
    # 32-neuron group), and no more than whole waves of one CTA per SM
    indeg = np.bincount(onet.post, minlength=n)
    grp = np.add.reduceat(indeg, np.arange(0, n, 32))
    loads = np.add.reduceat(indeg, blk[:-1])
    assert loads.max() <= 1.3 * loads.mean() + grp.max()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    waves = -(-(n // 736 + 1) // sms)
    assert B <= waves * sms
    return B


def test_blocked_structure_and_raster_tiny(model, tiny):
    """Blocked records of the tiny circuit: block boundaries, per-row block table and
    decoded synapses equal the oracle's network; 1,000 steps give the oracle's raster
    and state bit for bit."""
    wl, onet = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, record_format=BLK,
                      steps_per_graph=96)
    info = net.info()
    assert info.record_format == BLK and info.bytes_per_synapse == 6 and info.engine == GRAPH
    assert _check_blocked_structure(net, onet) == info.target_blocks
    net.step(1000)
    g_t, g_i = net.read_spikes()
    sim = oracle.Sim(model, onet, wl.seed)
    o_t, o_i = sim.run(1000)
    assert len(o_t) > 0 and np.array_equal(g_t, o_t) and np.array_equal(g_i, o_i)
    _assert_same_state(net, sim)
    net.close()


def _expected_ring(onet, spikers, t, npad):
    lens = np.diff(onet.row_ptr)
    starts = onet.row_ptr[spikers]
    cnt = lens[spikers]
    idx = np.repeat(starts - np.concatenate([[0], np.cumsum(cnt)[:-1]]), cnt) + np.arange(cnt.sum())
    flat = ((t + onet.delay[idx].astype(np.int64)) % 64) * npad + onet.post[idx]
    exp = np.bincount(flat, weights=onet.w_fx[idx].astype(np.float64), minlength=64 * npad)
    assert np.abs(exp).max() < 2**31
    return exp.astype(np.int64).reshape(64, npad)


@pytest.mark.parametrize("fmt", [BLK, snn.RECORD_BLOCKED4, snn.RECORD_BLOCKED8])
@pytest.mark.parametrize("nspk", [1, 63, 64, 700, 1024, 1025, 2048, 2049, 3000, 9000])
def test_blocked_deliver_spikes_matches_oracle_network(model, tiny, nspk, fmt):
    """Phase 2 alone with blocked records, below (reductions straight into the ring) and
    above (shared-memory sums) the 64-sender switch and across the 2,048-sender staging
    passes, repeats included: the ring equals the sums over the oracle's rows (bfloat16 read-back
    weights for BLOCKED4)."""
    wl, onet = tiny
    if fmt == snn.RECORD_BLOCKED4:
        onet = oracle.with_weights(onet, oracle.quantize_bf16(onet.w_fx))
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, record_format=fmt)
    rng = np.random.default_rng(100 + nspk)
    spikers = rng.integers(0, onet.n, nspk).astype(np.int32)
    t = 61
    net.deliver_spikes(torch.from_numpy(spikers).cuda(), t)
    torch.cuda.synchronize()
    npad = int(net.layout().n_neurons_padded)
    ring = net.device_view("ring", torch.int32, 64 * npad).cpu().numpy().reshape(64, npad).astype(np.int64)
    assert np.array_equal(ring, _expected_ring(onet, spikers, t, npad))
    net.close()


@pytest.mark.parametrize("fmt", [BLK, snn.RECORD_BLOCKED4, snn.RECORD_BLOCKED8])
def test_blocked_deliver_spikes_beyond_one_map_window(model, fmt):
    """A target block whose segments in one 2,048-sender pass hold more quads than the
    kernel maps at once (32,768): every sender has 80 synapses into targets 0..31 (one
    block that the cut cannot narrow), every other sender a few more elsewhere, so that
    other blocks see empty segments between nonempty ones; repeated senders, two passes."""
    m = model
    rng = np.random.default_rng(77)
    n = 2600
    pre, post, w, d = [], [], [], []
    for s in range(n):
        L = 80 + (s % 7)
        pre += [s] * L
        post += list(rng.integers(0, 32, L))
        if s % 2 == 0:
            pre += [s] * 5
            post += list(rng.integers(1000, n, 5))
    k = len(pre)
    w = list(rng.integers(-200_000, 300_000, k))
    d = list(rng.integers(1, 64, k))
    u0 = rng.uniform(0, 10, n).astype(np.float32)
    custom = dict(pre=pre, post=post, w_fx=w, delay=d, u0=u0, pop_offsets=[0, 325, 650, 975, 1300, 1625, 1950, 2275, n])
    onet = oracle.network_from_edges(n, pre, post, w, d, u0, custom["pop_offsets"])
    if fmt == snn.RECORD_BLOCKED4:
        onet = oracle.with_weights(onet, oracle.quantize_bf16(onet.w_fx))
    net = snn.Network(m, custom=custom, record_format=fmt)
    spikers = rng.integers(0, n, 3000).astype(np.int32)
    t = 5
    net.deliver_spikes(torch.from_numpy(spikers).cuda(), t)
    torch.cuda.synchronize()
    npad = int(net.layout().n_neurons_padded)
    ring = net.device_view("ring", torch.int32, 64 * npad).cpu().numpy().reshape(64, npad).astype(np.int64)
    assert np.array_equal(ring, _expected_ring(onet, spikers, t, npad))
    net.close()


@pytest.mark.parametrize("n", [1, 13, 517, 2000])
def test_blocked_ragged_counts_no_synapses(n):
    """No synapses (blocks cut by width alone: 768, 768, 464 for 2,000 neurons)."""
    m = workload.microcircuit_model()
    rng = np.random.default_rng(n)
    u0 = rng.uniform(0, 16, n).astype(np.float32)
    custom = dict(pre=[], post=[], w_fx=[], delay=[], u0=u0, pop_offsets=[0] + [n] * 8)
    o = _custom_parity(m, custom, 300, record_format=BLK)
    assert len(o[0]) > 0


def test_blocked_long_rows_all_delays():
    """Rows longer than a 32-lane pass, every delay, autapses, multapses, mixed signs,
    targets in several blocks (n = 2,301), with many senders per step."""
    m = workload.microcircuit_model()
    rng = np.random.default_rng(12)
    n = 2301
    pre, post, w, d = [], [], [], []
    for s, L in ((0, 1), (5, 255), (6, 256), (7, 257), (8, 1000), (9, 3001), (2300, 513)):
        pre += [s] * L
        post += list(rng.integers(0, n, L))
        w += list(rng.integers(-3_000_000, 3_000_000, L))
        d += list(rng.integers(1, 64, L))
    pre += [10] * 64
    post += [10] * 64
    w += [400_000] * 64
    d += list(range(1, 64)) + [63]
    # a dense random block so that some steps have more than 64 senders
    k = 40000
    pre += list(rng.integers(100, 2300, k))
    post += list(rng.integers(0, n, k))
    w += list(rng.integers(-600_000, 900_000, k))
    d += list(rng.integers(1, 64, k))
    u0 = rng.uniform(10, 16, n).astype(np.float32)
    po = [0, 300, 600, 900, 1200, 1500, 1800, 2100, n]
    custom = dict(pre=pre, post=post, w_fx=w, delay=d, u0=u0, pop_offsets=po)
    o = _custom_parity(m, custom, 400, spg=33, record_format=BLK)
    assert np.bincount(o[0]).max() >= 64


@pytest.mark.parametrize("t1", [2, 63, 64])
@pytest.mark.parametrize("d", [1, 16, 63])
def test_blocked_hand_placed_spike_arrival(t1, d):
    m = workload.microcircuit_model().replace(k_ext=[0.0] * 8)
    w2 = 12345 * 16
    c = _chain(t1 - 1, d, w2)
    net = snn.Network(m, custom=c, steps_per_graph=7, record_format=BLK)
    t_arr = t1 + d
    net.step(t_arr)
    _, I, _ = _state(net)
    assert I[2] == 0.0
    net.step(1)
    _, I, _ = _state(net)
    assert I[2] == np.float32(w2) * np.float32(2.0**-12)
    net.close()


BLK4 = snn.RECORD_BLOCKED4


def test_blocked4_structure_and_raster_tiny(model, tiny):
    """Blocked records with bfloat16 weights (4 bytes per synapse): the decoded network
    equals the oracle's with its bfloat16 read-back weights, and 1,000 steps give the
    raster of the oracle run on those weights and of the packed bf16 form, bit for bit."""
    wl, onet = tiny
    qnet = oracle.with_weights(onet, oracle.quantize_bf16(onet.w_fx))
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, record_format=BLK4,
                      steps_per_graph=96)
    info = net.info()
    assert info.record_format == BLK4 and info.bytes_per_synapse == 4 and info.engine == GRAPH
    _check_blocked_structure(net, qnet)
    net.step(1000)
    g_t, g_i = net.read_spikes()
    sim = oracle.Sim(model, qnet, wl.seed)
    o_t, o_i = sim.run(1000)
    assert len(o_t) > 0 and np.array_equal(g_t, o_t) and np.array_equal(g_i, o_i)
    _assert_same_state(net, sim)
    net.close()
    pk = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, record_format=snn.RECORD_PACKED_BF16)
    pk.step(1000)
    p_t, p_i = pk.read_spikes()
    assert np.array_equal(p_t, g_t) and np.array_equal(p_i, g_i)
    pk.close()


def test_blocked8_structure_and_raster_tiny(model, tiny):
    """Blocked records with interleaved (int32 weight, record) pairs, 8 bytes per synapse:
    the decoded network equals the oracle's exactly, and 1,000 steps give the oracle's
    raster and state bit for bit."""
    wl, onet = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, record_format=snn.RECORD_BLOCKED8,
                      steps_per_graph=96)
    info = net.info()
    assert info.record_format == snn.RECORD_BLOCKED8 and info.bytes_per_synapse == 8 and info.engine == GRAPH
    _check_blocked_structure(net, onet)
    net.step(1000)
    g_t, g_i = net.read_spikes()
    sim = oracle.Sim(model, onet, wl.seed)
    o_t, o_i = sim.run(1000)
    assert len(o_t) > 0 and np.array_equal(g_t, o_t) and np.array_equal(g_i, o_i)
    _assert_same_state(net, sim)
    net.close()


@pytest.mark.parametrize("nspk", [37, 700, 3000])
def test_blocked4_deliver_spikes_matches_oracle_network(model, tiny, nspk):
    wl, onet = tiny
    qnet = oracle.with_weights(onet, oracle.quantize_bf16(onet.w_fx))
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, record_format=BLK4)
    spikers = np.random.default_rng(200 + nspk).integers(0, onet.n, nspk).astype(np.int32)
    net.deliver_spikes(torch.from_numpy(spikers).cuda(), 61)
    torch.cuda.synchronize()
    npad = int(net.layout().n_neurons_padded)
    ring = net.device_view("ring", torch.int32, 64 * npad).cpu().numpy().reshape(64, npad).astype(np.int64)
    assert np.array_equal(ring, _expected_ring(qnet, spikers, 61, npad))
    net.close()


def test_blocked4_long_rows_all_delays():
    m = workload.microcircuit_model()
    rng = np.random.default_rng(13)
    n = 1501
    pre = list(rng.integers(0, 1500, 30000)) + [7] * 3001
    post = list(rng.integers(0, n, 30000)) + list(rng.integers(0, n, 3001))
    w = list(rng.integers(-2_000_000, 2_000_000, 33001))
    d = list(rng.integers(1, 64, 33001))
    u0 = rng.uniform(10, 16, n).astype(np.float32)
    custom = dict(pre=pre, post=post, w_fx=w, delay=d, u0=u0, pop_offsets=[0, 200, 400, 600, 800, 1000, 1200, 1400, n])
    net = snn.Network(m, custom=custom, steps_per_graph=33, seed=5, record_format=BLK4)
    onet = oracle.network_from_edges(n, pre, post, w, d, u0, custom["pop_offsets"])
    qnet = oracle.with_weights(onet, oracle.quantize_bf16(onet.w_fx))
    sim = oracle.Sim(m, qnet, 5)
    net.step(300)
    g = net.read_spikes()
    o = sim.run(300)
    assert len(o[0]) > 50 and np.array_equal(g[0], o[0]) and np.array_equal(g[1], o[1])
    _assert_same_state(net, sim)
    net.close()


def test_blocked_checkpoint_and_profiling_path(model, tiny):
    """Blocked records through a checkpoint, a resume after diverging steps and the
    kernel-by-kernel profiling path: the oracle's raster and state."""
    wl, onet = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, record_format=BLK,
                      steps_per_graph=64)
    net.step(150)
    blob = net.save_state()
    first = net.read_spikes()
    net.step(77)
    net.load_state(blob)
    net.profile_steps(50)
    net.step(100)
    g_t, g_i = net.read_spikes()
    g_t = np.concatenate([first[0], g_t])
    g_i = np.concatenate([first[1], g_i])
    sim = oracle.Sim(model, onet, wl.seed)
    o_t, o_i = sim.run(300)
    assert np.array_equal(g_t, o_t) and np.array_equal(g_i, o_i)
    _assert_same_state(net, sim)
    net.close()


def test_blocked_rejects_rows_beyond_16_bit_offsets():
    """Segment offsets are 16-bit: a row of more than 65,535 (padded) synapses is refused."""
    m = workload.microcircuit_model()
    n = 40
    L = 70000
    custom = dict(pre=[0] * L, post=list(np.arange(L) % n), w_fx=[1000] * L, delay=[1] * L,
                  u0=np.zeros(n, np.float32), pop_offsets=[0] + [n] * 8)
    with pytest.raises(snn.SnnError):
        snn.Network(m, custom=custom, record_format=BLK)
    net = snn.Network(m, custom=custom)  # plain records take it
    net.close()


def test_blocked_rejects_other_engines_and_batches(model):
    for eng in (PIPE, PERSIST):
        with pytest.raises(snn.SnnError):
            snn.Network(model, 20, 20, seed=1, record_format=BLK, engine=eng)
    with pytest.raises(snn.SnnError):
        snn.Network(model, circuits=[(20, 20, 1), (30, 30, 2)], record_format=BLK)


def test_blocked_full_scale_parity(model, full):
    """Full microcircuit with blocked records: the structure (boundaries, quotas, every
    synapse), 1,200 steps of raster and state equal to the oracle, and a saturating
    delivery of 4,096 random senders equal to the ring sums over the oracle's rows (also
    with bfloat16 weights: the oracle's read-back weights and a sample of decoded rows)."""
    wl, onet = full
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, record_format=BLK)
    assert net.info().n_synapses == 284_811_022
    _check_blocked_structure(net, onet, rows=np.random.default_rng(3).integers(0, onet.n, 2000))
    steps = 1200
    net.step(steps)
    g_t, g_i = net.read_spikes()
    sim = oracle.Sim(model, onet, wl.seed)
    o_t, o_i = sim.run(steps)
    assert len(o_t) > 0 and np.array_equal(g_t, o_t) and np.array_equal(g_i, o_i)
    _assert_same_state(net, sim)
    net.close()
    spikers = np.random.default_rng(7).integers(0, onet.n, 4096).astype(np.int32)
    qnet = oracle.with_weights(onet, oracle.quantize_bf16(onet.w_fx))
    for fmt, ref in ((BLK, onet), (snn.RECORD_BLOCKED4, qnet), (snn.RECORD_BLOCKED8, onet)):
        net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, record_format=fmt)
        net.deliver_spikes(torch.from_numpy(spikers).cuda(), 40)
        torch.cuda.synchronize()
        npad = int(net.layout().n_neurons_padded)
        ring = net.device_view("ring", torch.int32, 64 * npad).cpu().numpy().reshape(64, npad).astype(np.int64)
        assert np.array_equal(ring, _expected_ring(ref, spikers, 40, npad))
        if fmt != BLK:
            _check_blocked_structure(net, ref, rows=np.random.default_rng(4).integers(0, onet.n, 500))
        net.close()


@pytest.mark.parametrize("fmt", [snn.RECORD_PLAIN9, snn.RECORD_PACKED_BF16])
@pytest.mark.parametrize("engine", [GRAPH, PERSIST, PIPE])  # the resident engine takes one circuit
def test_batched_circuits_equal_standalone_runs(model, engine, fmt):
    """Circuits of uneven scale and seed stepped together: every circuit's slice of the
    batched raster and state equals the oracle run of that circuit alone."""
    net = snn.Network(model, circuits=BATCH, steps_per_graph=128, engine=engine, record_format=fmt)
    base, n = net.circuits()
    assert np.all(base % 128 == 0) and np.all(base[1:] >= base[:-1] + n[:-1])
    steps = 400
    net.step(steps)
    g_t, g_i = net.read_spikes()
    U, I, R = _state(net)
    for c, (sn, sk, seed) in enumerate(BATCH):
        onet = oracle.build_network(model, sn, sk, seed)
        if fmt == snn.RECORD_PACKED_BF16:
            onet = oracle.with_weights(onet, oracle.quantize_bf16(onet.w_fx))
        assert n[c] == onet.n
        sim = oracle.Sim(model, onet, seed)
        o_t, o_i = sim.run(steps)
        sel = (g_i >= base[c]) & (g_i < base[c] + n[c])
        assert np.array_equal(g_t[sel], o_t), c
        assert np.array_equal(g_i[sel] - base[c], o_i), c
        sl = slice(base[c], base[c] + n[c])
        assert np.array_equal(U[sl].view(np.uint32), sim.U.view(np.uint32)), c
        assert np.array_equal(I[sl].view(np.uint32), sim.I.view(np.uint32)), c
        assert np.array_equal(R[sl], sim.R), c
    # inert neurons between circuits never spike
    inside = np.zeros(len(U), bool)
    for c in range(len(BATCH)):
        inside[base[c]: base[c] + n[c]] = True
    assert inside[g_i].all()
    net.close()


@pytest.mark.parametrize("engine", [GRAPH, PIPE])
@pytest.mark.parametrize("cpg", [1, 2, 3])
def test_circuit_groups_equal_one_launch(model, engine, cpg):
    """Circuits taken in groups (each group through a whole run of steps before the next)
    give the raster and state of the ungrouped batch, across graph replays, directly
    launched remainders, the profiling path, changes of grouping between steps and a
    checkpoint loaded under another grouping than it was saved with (on the pipelined
    engine the spikes pending for the next step move between the groups' queues)."""
    ref = snn.Network(model, circuits=BATCH, steps_per_graph=64, engine=engine)
    ref.step(300)
    r_t, r_i = ref.read_spikes()
    rU, rI, rR = _state(ref)
    ref.close()
    other = 0 if cpg > 1 else 2
    net = snn.Network(model, circuits=BATCH, steps_per_graph=64, engine=engine)
    net.set_circuit_groups(cpg)
    assert net.info().circuits_per_group == (cpg if cpg < len(BATCH) else 0)
    net.step(100)   # one replay and 36 direct steps
    blob = net.save_state()
    part = net.read_spikes()
    net.step(77)
    net.set_circuit_groups(other)
    net.load_state(blob)  # back to step 100 under the other grouping; the host history restarts there
    net.step(50)
    net.set_circuit_groups(cpg)
    net.step(20)
    net.set_circuit_groups(other)
    net.step(86)    # 22 direct steps, then one replay from step 192
    net.set_circuit_groups(cpg)
    net.profile_steps(44)  # the kernel-by-kernel path takes the groups too
    g_t, g_i = net.read_spikes()
    g_t = np.concatenate([part[0], g_t])
    g_i = np.concatenate([part[1], g_i])
    assert np.array_equal(g_t, r_t) and np.array_equal(g_i, r_i)
    U, I, R = _state(net)
    assert np.array_equal(U.view(np.uint32), rU.view(np.uint32)) and np.array_equal(I.view(np.uint32),
                                                                                      rI.view(np.uint32))
    assert np.array_equal(R, rR)
    net.close()


def test_pipelined_circuit_groups_equal_standalone_runs(model):
    """Pipelined engine in circuit groups of two: every circuit's slice of the raster
    equals the oracle run of that circuit alone."""
    net = snn.Network(model, circuits=BATCH, steps_per_graph=64, engine=PIPE)
    net.set_circuit_groups(2)
    base, n = net.circuits()
    steps = 200
    net.step(steps)
    g_t, g_i = net.read_spikes()
    for c, (sn, sk, seed) in enumerate(BATCH):
        onet = oracle.build_network(model, sn, sk, seed)
        o_t, o_i = oracle.Sim(model, onet, seed).run(steps)
        sel = (g_i >= base[c]) & (g_i < base[c] + n[c])
        assert np.array_equal(g_t[sel], o_t), c
        assert np.array_equal(g_i[sel] - base[c], o_i), c
    net.close()


def test_circuit_groups_not_on_the_persistent_engine(model):
    net = snn.Network(model, circuits=BATCH, engine=PERSIST)
    with pytest.raises(snn.SnnError):
        net.set_circuit_groups(2)
    net.close()


# ------------------------------------------------------------ schedules, autotuner


@pytest.mark.parametrize("engine,sched", [(PIPE, dict(grid_ctas=304, delivery_warps=4, steps_per_graph=256)),
                                          (PIPE, dict(grid_ctas=37, delivery_warps=2)),
                                          (GRAPH, dict(grid_ctas=17, steps_per_graph=100))])
def test_schedule_does_not_change_results(model, tiny, engine, sched):
    wl, onet = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, steps_per_graph=128, engine=engine)
    net.step(300)
    net.set_schedule(**sched)
    info = net.info()
    assert info.schedule_ctas == sched["grid_ctas"]
    net.step(700)
    g = net.read_spikes()
    o = oracle.Sim(model, onet, wl.seed).run(1000)
    assert np.array_equal(g[0], o[0]) and np.array_equal(g[1], o[1])
    net.close()


def test_autotune_keeps_dynamics(model, tiny, tmp_path):
    from paper_2405_02019_gb300 import autotune

    wl, onet = tiny
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed)
    net.step(200)
    first = net.read_spikes()
    res = autotune.autotune(net, steps=256, cache_path=str(tmp_path / "sched.json"))
    assert res["schedule"] and len(res["timings"]) >= 2
    net.step(300)
    second = net.read_spikes()
    o = oracle.Sim(model, onet, wl.seed).run(500)
    assert np.array_equal(np.concatenate([first[0], second[0]]), o[0])
    assert np.array_equal(np.concatenate([first[1], second[1]]), o[1])
    res2 = autotune.autotune(net, steps=256, cache_path=str(tmp_path / "sched.json"))
    assert res2["schedule"] == res["schedule"]
    net.close()


def test_autotune_on_a_batch_keeps_dynamics(model):
    """Pipelined batch: the autotuner tries circuit groupings between a checkpoint and its
    restore (which moves the pending spikes between queue layouts); every circuit's raster
    still equals its standalone oracle run."""
    from paper_2405_02019_gb300 import autotune

    net = snn.Network(model, circuits=BATCH, steps_per_graph=64, engine=PIPE)
    net.step(100)
    first = net.read_spikes()
    res = autotune.autotune(net, steps=64, cache_path=None)
    assert {c["schedule"]["circuits_per_group"] for c in res["timings"]} == {0, 4}
    assert net.info().circuits_per_group == res["schedule"]["circuits_per_group"]
    net.step(150)
    second = net.read_spikes()
    g_t = np.concatenate([first[0], second[0]])
    g_i = np.concatenate([first[1], second[1]])
    base, n = net.circuits()
    for c, (sn, sk, seed) in enumerate(BATCH):
        o_t, o_i = oracle.Sim(model, oracle.build_network(model, sn, sk, seed), seed).run(250)
        sel = (g_i >= base[c]) & (g_i < base[c] + n[c])
        assert np.array_equal(g_t[sel], o_t), c
        assert np.array_equal(g_i[sel] - base[c], o_i), c
    net.close()
