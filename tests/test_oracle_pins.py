"""Pins of the CPU oracle to what the paper and mathematics fix (no GPU needed).

Each test checks an oracle function against something independent of the oracle:
values the paper prints (tests/golden/paper_values.json), closed forms derived by
hand, scipy/numpy library routines, or hand-written expectations of the paper's
stated rules.  A plausible slip in the oracle (a dropped term, a transposed table,
a wrong index or sign) fails at least one of them.
"""

import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

import oracle
import workload
from workload import POP_NAMES

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
P = {n: i for i, n in enumerate(POP_NAMES)}


# ----------------------------------------------------------------------------- RNG


@pytest.mark.parametrize("ctr,key", [
    ((1, 0, 0, 0), (1, 2)),
    ((12345, 678, 9, 10), (0xDEADBEEF, 0x7A)),
    ((2**64 - 1, 5, 2**63, 7), (2**64 - 1, 0)),
    ((0, 2**64 - 1, 0, 0), (42, 0xC0)),
])
def test_philox_matches_numpy(ctr, key):
    """Philox4x64-10 equals numpy's implementation (numpy bumps the counter before
    each block, so its state is set one below the counter we evaluate)."""
    c = np.array(ctr, dtype=object)
    # numpy state = ctr - 1 as a 256-bit little-endian integer
    v = sum(int(x) << (64 * j) for j, x in enumerate(c)) - 1
    v %= 2**256
    prev = np.array([(v >> (64 * j)) & (2**64 - 1) for j in range(4)], dtype=np.uint64)
    bg = np.random.Philox(counter=prev, key=np.array(key, dtype=np.uint64))
    ref = bg.random_raw(4).astype(np.uint64)
    got = oracle.philox(ctr, key)
    assert np.array_equal(got, ref)


# ----------------------------------------------------------------------- constants


def test_constants_match_printed_values(model):
    c = oracle.constants(model)
    for k in ("w_f", "p11", "p22", "p21"):
        g = GOLDEN[k]
        assert abs(c[k] - g["printed"]) <= g["tol"], (k, c[k], g)


def test_propagators_are_the_exact_flow_of_the_lif_ode(model):
    """Over one step, the linear system dU/dt = -U/tau_m + I/C, dI/dt = -I/tau_syn is
    advanced exactly by expm(A dt) = [[p22, p21], [0, p11]] (exact integration)."""
    c = oracle.constants(model)
    A = np.array([[-1.0 / model.tau_m_ms, 1.0 / model.C_m_pF], [0.0, -1.0 / model.tau_syn_ms]])
    E = scipy.linalg.expm(A * model.dt_ms)
    assert E[0, 0] == pytest.approx(c["p22"], rel=1e-13)
    assert E[1, 1] == pytest.approx(c["p11"], rel=1e-13)
    assert E[0, 1] == pytest.approx(c["p21"], rel=1e-11)
    assert E[1, 0] == 0.0


def test_w_f_maps_psc_amplitude_to_psp_peak(model):
    """w_f is the current amplitude whose PSP peaks at 1 mV: the continuous PSP of a
    current step w decaying with tau_syn is (w/C) beta (e^{-t/tau_m} - e^{-t/tau_syn}),
    which peaks at t* = beta ln(tau_m/tau_syn)."""
    c = oracle.constants(model)
    tm, ts, C = model.tau_m_ms, model.tau_syn_ms, model.C_m_pF
    beta = ts * tm / (tm - ts)
    tpk = beta * math.log(tm / ts)
    peak = (c["w_f"] / C) * beta * (math.exp(-tpk / tm) - math.exp(-tpk / ts))
    assert peak == pytest.approx(1.0, rel=1e-12)


def test_step_constants(model):
    s = oracle.step_constants(model)
    c = oracle.constants(model)
    assert s["theta"] == np.float32(15.0)          # u_thr - u_rest
    assert s["u_reset"] == np.float32(0.0)         # reset at rest
    assert s["t_ref"] == 20                         # 2 ms / 0.1 ms
    assert s["p11"] == np.float32(c["p11"]) and s["p22"] == np.float32(c["p22"])
    assert s["p21"] == np.float32(c["p21"])
    # thalamic PSC = w_f * 0.15 mV = 87.81 pA, in 2^-12 pA units
    assert abs(s["w_ext_fx"] / 4096.0 - 87.8085) < 1e-3


# ---------------------------------------------------------------- neuron dynamics


def _closed_form_crossing(model, x_fx):
    """First step n (0-based, the step during which U reaches theta) for a neuron at
    rest with constant per-step input x: I_n = I*(1 - p11^n), U_n = U* + a p22^n + b p11^n
    solving U_{n+1} = p22 U_n + p21 I_n (derived by hand; FP64)."""
    c = oracle.constants(model)
    p11, p22, p21 = c["p11"], c["p22"], c["p21"]
    x = x_fx / 4096.0
    Istar = x / (1 - p11)
    Ustar = p21 * Istar / (1 - p22)
    b = p21 * Istar / (p22 - p11)
    a = -Ustar - b
    n = 0
    while True:
        n += 1
        U = Ustar + a * p22**n + b * p11**n
        if U >= 15.0:
            return n - 1, U  # U after step n-1 is U_n
        if n > 100000:
            return None, U


@pytest.mark.parametrize("x_pA", [80.0, 95.5, 150.0, 400.0])
def test_time_to_threshold_closed_form(model, x_pA):
    x_fx = int(round(x_pA * 4096))
    n_star, U_at = _closed_form_crossing(model, x_fx)
    assert n_star is not None
    assert U_at - 15.0 > 1e-3  # not a near-tie
    tr = oracle.lif_trace(model, np.full(n_star + 50, x_fx, np.int32))
    first = int(np.argmax(tr["spike"]))
    assert tr["spike"][first] == 1
    assert first == n_star


def test_refractory_clamp_and_isi_closed_form(model):
    """After a spike U sits at reset for exactly t_ref = 20 steps, then integrates
    the (converged) current again: U = U*(1 - p22^j), so ISI = 20 + j*."""
    c = oracle.constants(model)
    x_fx = int(round(110.0 * 4096))
    n = 3000
    tr = oracle.lif_trace(model, np.full(n, x_fx, np.int32))
    spk = np.flatnonzero(tr["spike"])
    assert len(spk) > 5
    for s in spk[:-1]:
        assert tr["U"][s] == 0.0  # reset on the spike step itself
        assert np.all(tr["U"][s + 1: s + 21] == 0.0)
        assert tr["R"][s] == 20 and tr["R"][s + 20] == 0
        assert tr["U"][s + 21] > 0.0
    I_star = (x_fx / 4096.0) / (1 - c["p11"])
    U_star = c["p21"] * I_star / (1 - c["p22"])
    j_star = math.ceil(math.log(1 - 15.0 / U_star) / math.log(c["p22"]))
    isi = np.diff(spk)
    assert np.all(isi[2:] == 20 + j_star)
    assert np.all(isi >= 21)


def test_refractory_clamp_holds_the_reset_value(model):
    """Eq. ref holds U at u_reset, which need not be the rest potential: with u_reset
    5 mV below rest, U is -5 mV (relative to rest) from the spike step through the 20
    refractory steps, and integrates again from there."""
    m2 = model.replace(u_reset_mV=model.u_rest_mV - 5.0)
    assert oracle.step_constants(m2)["u_reset"] == np.float32(-5.0)
    tr = oracle.lif_trace(m2, np.full(3000, int(round(110.0 * 4096)), np.int32))
    spk = np.flatnonzero(tr["spike"])
    assert len(spk) > 5
    for s in spk[:-1]:
        assert np.all(tr["U"][s: s + 21] == np.float32(-5.0))
        assert tr["U"][s + 21] > -5.0


def _float_with_product(p, target, below=False):
    """A float32 u with fl(p*u) == target (or the float just below target)."""
    want = np.float32(target)
    if below:
        want = np.nextafter(want, np.float32(0))
    u = np.float32(float(want) / float(p))
    for _ in range(1000):
        prod = np.float32(p) * u
        if prod == want:
            return u
        u = np.nextafter(u, np.float32(np.inf) if prod < want else np.float32(-np.inf))
    raise AssertionError("no float found")


def test_threshold_is_inclusive(model):
    """Eq. ref spikes when u >= u_thr: an update landing exactly on theta spikes,
    one ulp below does not."""
    s = oracle.step_constants(model)
    u_eq = _float_with_product(s["p22"], 15.0)
    u_lo = _float_with_product(s["p22"], 15.0, below=True)
    assert oracle.lif_trace(model, [0], U0=u_eq)["spike"][0] == 1
    assert oracle.lif_trace(model, [0], U0=u_lo)["spike"][0] == 0


def test_psc_jump_and_psp_shape(model):
    """One input w at step 0: I jumps to exactly w after the step, U then follows the
    sampled exact PSP gamma w (p22^n - p11^n), peaking near omega = 0.15 mV when
    w = w_f * 0.15 mV."""
    c = oracle.constants(model)
    w_fx = int(round(c["w_f"] * 0.15 * 4096))
    n = 200
    inp = np.zeros(n, np.int32)
    inp[0] = w_fx
    tr = oracle.lif_trace(model, inp)
    assert tr["I"][0] == np.float32(w_fx) * np.float32(2.0**-12)
    assert tr["U"][0] == 0.0
    w = float(tr["I"][0])
    k = np.arange(1, n)
    analytic = c["gamma"] * w * (c["p22"] ** k - c["p11"] ** k)
    np.testing.assert_allclose(tr["U"][1:], analytic, rtol=2e-5, atol=1e-9)
    assert abs(tr["U"].max() - 0.15) < 0.15 * 0.005
    # the grid maximum sits at the continuous peak time t* = 1.577 ms
    assert int(np.argmax(tr["U"])) in (15, 16)


# ------------------------------------------------------------ ring buffer / delays


def _chain_net(d_first, d_second, w2_fx):
    """Neuron 0 starts above threshold (spikes at step 0); it drives neuron 1 through a
    synapse strong enough to make it spike one step after arrival; neuron 1 drives
    neuron 2 with delay d_second."""
    big = 200_000_000  # 48,828 pA: p21 * I > theta on the next step
    return oracle.network_from_edges(3, pre=[0, 1], post=[1, 2], w_fx=[big, w2_fx],
                                     delay=[d_first, d_second], u0=[20.0, 0.0, 0.0])


@pytest.mark.parametrize("t1", [2, 62, 63, 64])
@pytest.mark.parametrize("d", [1, 15, 16, 63])
def test_spike_arrives_exactly_d_steps_later(t1, d):
    """Listing push: a spike at step t adds w to W[(t+d) mod 64] which the target reads
    (and clears) at step t+d, so its current jumps by exactly w at the end of step t+d
    and is untouched before (with 64 ring rows, §3.2)."""
    m = workload.microcircuit_model().replace(k_ext=[0.0] * 8)
    w2 = 12345 * 16
    net = _chain_net(t1 - 1, d, w2)
    sim = oracle.Sim(m, net, seed=7)
    t_arr = t1 + d
    I2 = []
    spikes = []
    for _ in range(t_arr + 2):
        st, si = sim.run(1)
        spikes += list(zip(st.tolist(), si.tolist()))
        I2.append(float(sim.I[2]))
    assert (0, 0) in spikes and (t1, 1) in spikes
    assert all(v == 0.0 for v in I2[:t_arr])
    assert I2[t_arr] == float(np.float32(w2) * np.float32(2.0**-12))
    # the ring row was cleared after the read: no second delivery 64 steps later
    sim.run(64)
    assert float(sim.I[2]) < I2[t_arr] * 1e-5


def test_simultaneous_arrivals_sum_exactly():
    """Two senders spiking at step 0 with equal delay deliver w1 + w2 in one step."""
    m = workload.microcircuit_model().replace(k_ext=[0.0] * 8)
    net = oracle.network_from_edges(3, pre=[0, 1, 0], post=[2, 2, 2], w_fx=[1000, -300, 7],
                                    delay=[5, 5, 6], u0=[20.0, 20.0, 0.0])
    sim = oracle.Sim(m, net, seed=1)
    sim.run(6)
    assert float(sim.I[2]) == float(np.float32(700) * np.float32(2.0**-12))
    sim.run(1)
    p11 = oracle.step_constants(m)["p11"]
    expect = np.float32(p11 * np.float32(700 / 4096.0)) + np.float32(7 / 4096.0)
    assert np.float32(sim.I[2]) == expect


def test_ring_sizing_value_from_paper():
    g = GOLDEN["ring_tail_prob"]
    assert scipy.stats.norm(1.5, 0.75).cdf(6.4) == pytest.approx(g["printed"], abs=g["tol"])


# ----------------------------------------------------------------- Poisson drive


def test_poisson_tables_match_scipy(model):
    for b in range(8):
        lam = model.k_ext[b] * model.nu_th_hz * model.dt_ms * 1e-3
        tab = oracle.poisson_table(model, b)
        F = tab.astype(np.float64) / 2.0**63
        ref = scipy.stats.poisson.cdf(np.arange(24), lam)
        np.testing.assert_allclose(F[:-1], ref[:-1], rtol=0, atol=4e-16)
        assert tab[-1] == 2**63
        assert np.all(np.diff(tab.astype(object)) >= 0)


def test_thalamic_rate_example(model):
    g = GOLDEN["thalamic_rate_example"]
    assert model.k_ext[P[g["pop"]]] * model.nu_th_hz == g["printed"]


@pytest.mark.parametrize("pop", range(8))
def test_poisson_inversion_boundaries(model, pop):
    """T = #{k : v >= C_k}: a uniform exactly on threshold C_k already counts it (T =
    k + 1), one below does not (T = k); v = 0 gives 0 and the largest 63-bit value the
    last count whose threshold is below 2^63."""
    C = oracle.poisson_table(model, pop)
    assert oracle.poisson_count_at(model, pop, 0) == 0
    for k in range(6):
        assert C[k] < C[k + 1]
        assert oracle.poisson_count_at(model, pop, int(C[k])) == k + 1
        assert oracle.poisson_count_at(model, pop, int(C[k]) - 1) == k
    top = 2**63 - 1
    assert oracle.poisson_count_at(model, pop, top) == int(np.count_nonzero(C <= top))


@pytest.mark.parametrize("pop", range(8))
def test_poisson_draw_statistics(model, pop):
    n = 400_000
    T = oracle.poisson_draws(model, seed=3, pop=pop, t=11, i0=0, n=n).astype(np.float64)
    lam = model.k_ext[pop] * model.nu_th_hz * model.dt_ms * 1e-3
    se = math.sqrt(lam / n)
    assert abs(T.mean() - lam) < 4.5 * se
    assert abs(T.var() - lam) < 4.5 * lam * math.sqrt(2.0 / n) * 2
    kmax = 9
    obs = np.bincount(np.minimum(T.astype(int), kmax), minlength=kmax + 1)
    pmf = scipy.stats.poisson.pmf(np.arange(kmax), lam)
    exp = np.concatenate([pmf, [1 - pmf.sum()]]) * n
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert scipy.stats.chi2.sf(chi2, kmax) > 1e-4


def test_poisson_draws_independent_across_neurons_and_steps(model):
    """Neighbouring neurons share one Philox block but use different words; the same
    neuron at consecutive steps uses different counters: no correlation."""
    n = 200_000
    a = oracle.poisson_draws(model, 5, 0, 100, 0, n).astype(float)
    b = oracle.poisson_draws(model, 5, 0, 101, 0, n).astype(float)
    assert abs(np.corrcoef(a[:-1], a[1:])[0, 1]) < 0.015
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.015
    c = oracle.poisson_draws(model, 6, 0, 100, 0, n).astype(float)
    assert abs(np.corrcoef(a, c)[0, 1]) < 0.015


# ------------------------------------------------------------------- network


def test_population_sizes_and_totals(model):
    g = GOLDEN
    assert oracle.pop_sizes(model, 1000).sum() == g["n_neurons"]["printed"]
    assert list(oracle.pop_sizes(model, 1000)) == list(model.n_full)
    assert list(oracle.pop_sizes(model, 100)) == [2068, 583, 2192, 548, 485, 107, 1440, 295]
    tot = oracle.total_synapses(model, 1000, 1000)
    assert abs(tot - g["total_synapses"]["printed"]) <= g["total_synapses"]["tol_rel"] * 3e8
    ex = g["pair_example"]
    k = oracle.pair_count(model, 1000, 1000, target=P[ex["target"]], source=P[ex["source"]])
    assert abs(k - ex["printed"]) <= ex["tol_rel"] * ex["printed"]
    assert abs(k - 5834 * 4850 * 0.0755) <= 1.0


@pytest.fixture(scope="module")
def tiny_net(model):
    return oracle.build_network(model, 100, 100, seed=1)


def _pre_post_pops(net):
    pre = np.repeat(np.arange(net.n), np.diff(net.row_ptr))
    pp = np.searchsorted(net.pop_off, pre, side="right") - 1
    qp = np.searchsorted(net.pop_off, net.post, side="right") - 1
    return pre, pp, qp


def test_pair_counts_realised(model, tiny_net):
    pre, pp, qp = _pre_post_pops(tiny_net)
    for a in range(8):
        for b in range(8):
            assert np.count_nonzero((pp == a) & (qp == b)) == oracle.pair_count(model, 100, 100, b, a)


def test_in_and_out_degrees_are_binomial(model, tiny_net):
    """Drawing with replacement makes a target's in-degree from one source population
    Binomial(K_ab, 1/N_b) and a source's out-degree Binomial(K_ab, 1/N_a): test the
    mean exactly and the variance by the chi-square dispersion statistic."""
    net = tiny_net
    pre, pp, qp = _pre_post_pops(net)
    sizes = np.diff(net.pop_off)
    for a in range(8):
        for b in range(8):
            K = oracle.pair_count(model, 100, 100, b, a)
            if K < 2000:
                continue
            sel = (pp == a) & (qp == b)
            indeg = np.bincount(net.post[sel] - net.pop_off[b], minlength=sizes[b])
            outdeg = np.bincount(pre[sel] - net.pop_off[a], minlength=sizes[a])
            for deg, n in ((indeg, sizes[b]), (outdeg, sizes[a])):
                assert deg.sum() == K
                mu = K / n
                var_b = K * (1 / n) * (1 - 1 / n)
                stat = ((deg - mu) ** 2).sum() / var_b
                p = scipy.stats.chi2.sf(stat, n - 1)
                assert 1e-4 < p < 1 - 1e-4, (a, b, p)


def test_connection_table_orientation(model, tiny_net):
    """Reading: rows of Table params3 are targets.  L6I receives from L6E with p=0.0658
    (row L6I) rather than 0.2252 (column L6I)."""
    pre, pp, qp = _pre_post_pops(tiny_net)
    n_l6i = np.diff(tiny_net.pop_off)[P["L6I"]]
    mean_in = np.count_nonzero((pp == P["L6E"]) & (qp == P["L6I"])) / n_l6i
    assert mean_in == pytest.approx(0.0658 * 14395 * 0.1, rel=0.01)


def test_weight_distributions(model, tiny_net):
    c = oracle.constants(model)
    pre, pp, qp = _pre_post_pops(tiny_net)
    w_mV = tiny_net.w_fx / 4096.0 / c["w_f"]
    for name, sel, mu, sd in (
        ("exc", (pp % 2 == 0) & ~((pp == P["L4E"]) & (qp == P["L23E"])), 0.15, 0.015),
        ("inh", pp % 2 == 1, -0.6, 0.06),
        ("L4E->L23E", (pp == P["L4E"]) & (qp == P["L23E"]), 0.3, 0.03),
    ):
        x = w_mV[sel]
        n = len(x)
        assert abs(x.mean() - mu) < 4 * sd / math.sqrt(n), name
        assert abs(x.std() - sd) < 4 * sd / math.sqrt(2 * n) + sd * 1e-3, name
        ks = scipy.stats.kstest(x, scipy.stats.norm(mu, sd).cdf)
        # the fixed-point quantum (1/4096 pA / w_f ~ 4e-7 mV) is far below sd
        assert ks.pvalue > 1e-4, name


def test_weights_clip_at_zero_on_their_own_side(model):
    """A weight drawn past zero is clipped to zero, never flipped in sign: with the SD
    raised to the full mean (so that clipping is common), excitatory weights stay >= 0,
    inhibitory ones <= 0, and each side's share of zeros is Phi(-1) within 4 standard
    errors."""
    m2 = model.replace(w_sd_mV=[abs(mu) for mu in model.w_mean_mV], overrides=[(2, 0, 0.3, 0.3)])
    net = oracle.build_network(m2, 50, 50, 3)
    pre, pp, qp = _pre_post_pops(net)
    p0 = scipy.stats.norm.cdf(-1.0)
    for name, sel, sign in (("exc", pp % 2 == 0, 1), ("inh", pp % 2 == 1, -1)):
        w = net.w_fx[sel]
        assert np.all(sign * w >= 0), name
        n = len(w)
        frac = np.count_nonzero(w == 0) / n
        assert abs(frac - p0) < 4 * math.sqrt(p0 * (1 - p0) / n), (name, frac, p0)


def _discretised_clipped_normal(mu, sd, dt=0.1, dmax=63):
    """P(d = k) for d = clip(round(N(mu, sd)/dt), 1, dmax), by scipy's normal CDF."""
    edges = (np.arange(1, dmax) + 0.5) * dt
    cdf = scipy.stats.norm(mu, sd).cdf(edges)
    p = np.diff(np.concatenate([[0.0], cdf, [1.0]]))
    return p  # index 0 <-> k=1 ... index dmax-1 <-> k=dmax


def test_delay_distributions(model, tiny_net):
    pre, pp, qp = _pre_post_pops(tiny_net)
    d = tiny_net.delay.astype(int)
    assert d.min() >= 1 and d.max() <= 63
    for exc, mu, sd in ((True, 1.5, 0.75), (False, 0.75, 0.375)):
        x = d[(pp % 2 == 0) == exc]
        p = _discretised_clipped_normal(mu, sd)
        obs = np.bincount(x - 1, minlength=63)
        expct = p * len(x)
        keep = expct > 20
        o = np.concatenate([obs[keep], [obs[~keep].sum()]])
        e = np.concatenate([expct[keep], [expct[~keep].sum()]])
        chi2 = ((o - e) ** 2 / e).sum()
        assert scipy.stats.chi2.sf(chi2, len(o) - 1) > 1e-4, exc


def test_initial_potentials(model):
    """Table params2, column u_init: per-population Gaussian, stored relative to rest."""
    U = oracle.initial_u(model, 1000, seed=2)
    off = oracle.pop_offsets(model, 1000)
    for b in range(8):
        u = U[off[b]:off[b + 1]].astype(np.float64) + model.u_rest_mV
        mu, sd = model.u0_mean_mV[b], model.u0_sd_mV[b]
        ks = scipy.stats.kstest(u, scipy.stats.norm(mu, sd).cdf)
        assert ks.pvalue > 1e-4, b


# --------------------------------------------------------------- whole network


def test_tiny_network_runs_and_is_deterministic(model, tiny_net):
    s1 = oracle.Sim(model, tiny_net, seed=1)
    a = s1.run(300)
    s2 = oracle.Sim(model, tiny_net, seed=1)
    b1 = s2.run(120)
    b2 = s2.run(180)
    assert np.array_equal(a[0], np.concatenate([b1[0], b2[0]]))
    assert np.array_equal(a[1], np.concatenate([b1[1], b2[1]]))
    assert len(a[0]) > 0
    # no neuron fires twice within its refractory period (min ISI 21 steps)
    for i in np.unique(a[1]):
        ts = a[0][a[1] == i]
        assert np.all(np.diff(ts) >= 21)


def test_sender_order_is_irrelevant(model, tiny_net):
    """Integer accumulation makes delivery order-independent: permuting the synapses
    within every row leaves the raster unchanged."""
    rng = np.random.default_rng(0)
    net = tiny_net
    perm = np.arange(len(net.post))
    for i in range(net.n):
        a, b = net.row_ptr[i], net.row_ptr[i + 1]
        perm[a:b] = a + rng.permutation(b - a)
    net2 = oracle.Network(net.n, net.pop_off, net.row_ptr, net.post[perm].copy(),
                          net.w_fx[perm].copy(), net.delay[perm].copy(), net.u0)
    r1 = oracle.Sim(model, net, 1).run(200)
    r2 = oracle.Sim(model, net2, 1).run(200)
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1])


# ------------------------------------------------ compressed records and FP64 loop


def test_int8_pair_quantizer_bounds(model, tiny_net):
    """Per (source, target) population pair: the read-back weight is within half a step
    of the true weight, every code fits int8, and the pair's extremes set base/step."""
    q, base, step = oracle.quantize_i8(tiny_net)
    pre, pp, qp = _pre_post_pops(tiny_net)
    w = tiny_net.w_fx.astype(np.int64)
    for a in range(8):
        for b in range(8):
            sel = (pp == a) & (qp == b)
            if not sel.any():
                assert base[a, b] == 0 and step[a, b] == 1
                continue
            lo, hi = w[sel].min(), w[sel].max()
            assert base[a, b] == lo + (hi - lo) // 2
            assert step[a, b] == max(1, -(-(hi - lo) // 254))
            code = (q[sel].astype(np.int64) - base[a, b]) / step[a, b]
            assert np.all(code == np.round(code)) and np.all(np.abs(code) <= 127)
            assert np.all(np.abs(q[sel] - w[sel]) <= step[a, b] / 2 + 0.5)


def test_bf16_quantizer_matches_torch():
    """The bf16 read-back equals torch's float32 -> bfloat16 conversion (ties to even)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    w = np.concatenate([rng.integers(-6_000_000, 6_000_000, 20000), [0, 1, -1, 255, 256, 257, 4095, 2**24 - 1],
                        [0x7F8080, 0x7F8180]]).astype(np.int32)
    got = oracle.quantize_bf16(w)
    f = torch.from_numpy((w.astype(np.float32) / np.float32(4096.0)))
    ref = (f.to(torch.bfloat16).to(torch.float32) * 4096.0).numpy().astype(np.int64)
    assert np.array_equal(got.astype(np.int64), ref)
    nz = w != 0
    assert np.all(np.abs(got[nz] - w[nz]) / np.abs(w[nz]) <= 2.0**-8 + 1e-12)


def test_fp64_loop_psc_and_psp():
    """FP64 loop: one spike of weight w arrives after its delay as exactly w * 2^-12 pA,
    and the target's potential then follows the exact PSP gamma I (p22^n - p11^n) to
    FP64 rounding."""
    m = workload.microcircuit_model().replace(k_ext=[0.0] * 8)
    c = oracle.constants(m)
    w = 359_664
    net = oracle.network_from_edges(2, pre=[0], post=[1], w_fx=[w], delay=[3], u0=[20.0, 0.0])
    sim = oracle.Sim(m, net, seed=1, fp64=True)
    sim.run(3)
    assert sim.I[1] == 0.0
    sim.run(1)
    assert sim.I[1] == w / 4096.0
    U = []
    for _ in range(60):
        sim.run(1)
        U.append(sim.U[1])
    k = np.arange(1, 61)
    np.testing.assert_allclose(U, c["gamma"] * (w / 4096.0) * (c["p22"] ** k - c["p11"] ** k), rtol=1e-12)


def test_fp64_loop_uses_unrounded_weights_and_currents():
    """FP64 loop: a weight given in pA that 2^-12 pA cannot represent arrives unrounded,
    simultaneous arrivals add in pA, and the thalamic input of a step is T w_f w_ext in
    pA with T the Poisson count of that neuron and step."""
    m0 = workload.microcircuit_model().replace(k_ext=[0.0] * 8)
    w_pA = [87.808521234567, -351.23399991]
    net = oracle.network_from_edges(3, pre=[0, 1], post=[2, 2], w_fx=[359_664, -1_438_654], delay=[2, 2],
                                    u0=[20.0, 20.0, 0.0], w_pA=w_pA)
    sim = oracle.Sim(m0, net, seed=1, fp64=True)
    sim.run(2)
    assert sim.I[2] == 0.0
    sim.run(1)
    assert sim.I[2] == w_pA[0] + w_pA[1]
    assert sim.I[2] != (359_664 - 1_438_654) / 4096.0
    m = workload.microcircuit_model()
    c = oracle.constants(m)
    one = oracle.network_from_edges(1, pre=[], post=[], w_fx=[], delay=[], u0=[0.0],
                                    pop_off=[0, 1, 1, 1, 1, 1, 1, 1, 1])
    sim = oracle.Sim(m, one, seed=5, fp64=True)
    Is = []
    for _ in range(40):
        sim.run(1)
        Is.append(sim.I[0])
    T = [int(oracle.poisson_draws(m, 5, 0, t, 0, 1)[0]) for t in range(40)]
    w_ext = c["w_f"] * m.w_ext_mV
    exp, cur = [], 0.0
    for t in range(40):
        cur = c["p11"] * cur + (0.0 + T[t] * w_ext)
        exp.append(cur)
    assert sum(T) > 10
    assert Is == exp


def test_build_keeps_unrounded_currents():
    """The FP64 loop's weights are the drawn currents before rounding: rounding them to
    2^-12 pA gives the integer weights bit for bit, excitatory currents are >= 0 and
    inhibitory ones <= 0, and their scale is pA (the mean excitatory current is
    w_f * 0.15 mV, about 87.8 pA)."""
    m = workload.microcircuit_model()
    net = oracle.build_network(m, 50, 50, 3, with_pA=True)
    assert np.array_equal(np.rint(net.w_pA * 4096.0).astype(np.int64), net.w_fx.astype(np.int64))
    pre = np.repeat(np.arange(net.n), np.diff(net.row_ptr))
    pops = np.searchsorted(net.pop_off, pre, side="right") - 1
    exc = pops % 2 == 0
    assert np.all(net.w_pA[exc] >= 0) and np.all(net.w_pA[~exc] <= 0)
    c = oracle.constants(m)
    plain = exc & ~((pops == 2) & (np.searchsorted(net.pop_off, net.post, side="right") - 1 == 0))
    assert abs(net.w_pA[plain].mean() / (c["w_f"] * 0.15) - 1.0) < 0.01
