// Host side of network construction (setup; not part of the timed step loop, as in
// the paper's RTF definition of §4.2).
//
//  - model constants of §2.2 (w_f, p11, p22, beta, gamma, p21) in FP64, rounded once
//    to FP32 for the device;
//  - thalamic Poisson thresholds: the CDF of Poisson(nu_th K dt) scaled to 63 bits;
//  - population sizes and the expected pair counts N_pre N_post p of §2.2;
//  - every synapse drawn with replacement from counter-based Philox streams, so the
//    result does not depend on the thread count;
//  - the indexed synapse store of §3.5: rows grouped by sender and sorted by delay,
//    each padded to a multiple of four entries with zero-weight synapses so that
//    every row starts on a 16-byte boundary for vector loads.
//
// Built with -ffp-contract=off: every FP64 product and sum is rounded on its own.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <thread>

#include "internal.hpp"
#include "philox.cuh"

namespace snn {

namespace {

constexpr double kTwoPi = 6.283185307179586;
constexpr double kInv2Pow53 = 1.0 / 9007199254740992.0;
constexpr double kTwoPow63 = 9223372036854775808.0;

inline double unit_open(uint64_t x) { return (static_cast<double>(x >> 11) + 0.5) * kInv2Pow53; }

// Uniform integer in [0, n): the high word of x * n.
inline int64_t scale_below(uint64_t x, int64_t n)
{
    uint64_t hi, lo;
    mul_wide(x, static_cast<uint64_t>(n), hi, lo);
    return static_cast<int64_t>(hi);
}

// Box-Muller transform of two uniforms: (r cos th, r sin th), r = sqrt(-2 ln u), th = 2 pi v.
inline void gauss_pair(uint64_t u, uint64_t v, double &zc, double &zs)
{
    const double r = std::sqrt(-2.0 * std::log(unit_open(u)));
    const double th = kTwoPi * unit_open(v);
    zc = r * std::cos(th);
    zs = r * std::sin(th);
}

void parallel_for(int nthreads, int64_t n, const std::function<void(int, int64_t, int64_t)> &body)
{
    if (n <= 0) return;
    nthreads = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(nthreads, n)));
    if (nthreads == 1) {
        body(0, 0, n);
        return;
    }
    std::vector<std::thread> pool;
    pool.reserve(nthreads);
    for (int t = 0; t < nthreads; ++t) {
        const int64_t lo = n * t / nthreads, hi = n * (t + 1) / nthreads;
        pool.emplace_back(body, t, lo, hi);
    }
    for (auto &th : pool) th.join();
}

}  // namespace

int resolve_threads(int32_t requested)
{
    if (requested > 0) return requested;
    const unsigned hc = std::thread::hardware_concurrency();
    return hc ? static_cast<int>(std::min(hc, 64u)) : 4;
}

void compute_constants(const snn_model &m, Constants &c)
{
    const double ts = m.tau_syn_ms, tm = m.tau_m_ms, C = m.C_m_pF, dt = m.dt_ms;
    // PSC amplitude that gives a 1 mV PSP peak (§2.2)
    const double d = ts - tm;
    const double p = ts * tm;
    const double q = tm / ts;
    c.w_f = C * d / (p * (std::pow(q, tm / d) - std::pow(q, ts / d)));
    // one-step propagators (§2.2)
    c.p11 = std::exp(-dt / ts);
    c.p22 = std::exp(-dt / tm);
    c.beta = ts * tm / (tm - ts);
    c.gamma = c.beta / C;
    c.p21 = c.p11 * c.gamma * (std::exp(dt / c.beta) - 1.0);
    c.p11f = static_cast<float>(c.p11);
    c.p21f = static_cast<float>(c.p21);
    c.p22f = static_cast<float>(c.p22);
    c.theta = static_cast<float>(m.u_thr_mV - m.u_rest_mV);
    c.u_reset = static_cast<float>(m.u_reset_mV - m.u_rest_mV);
    c.t_ref = static_cast<int32_t>(std::llround(m.tau_ref_ms / dt));
    c.w_ext_fx = static_cast<int32_t>(std::llround(c.w_f * m.w_ext_mV * 4096.0));
    // Poisson(lambda) CDF thresholds, lambda = nu_th K dt
    std::memset(c.thresholds, 0, sizeof(c.thresholds));
    for (int b = 0; b < m.n_pops; ++b) {
        const double lam = m.k_ext[b] * m.nu_th_hz * dt * 1e-3;
        double pk = std::exp(-lam);
        double cdf = pk;
        for (int k = 0; k < kPK; ++k) {
            if (k > 0) {
                pk = pk * lam / static_cast<double>(k);
                cdf = cdf + pk;
            }
            const bool saturated = (k == kPK - 1) || cdf >= 1.0;
            c.thresholds[b][k] = saturated ? (1ull << 63) : static_cast<uint64_t>(cdf * kTwoPow63);
        }
    }
}

void population_sizes(const snn_model &m, int32_t scale_n, int64_t out[SNN_MAX_POPS])
{
    for (int b = 0; b < SNN_MAX_POPS; ++b)
        out[b] = b < m.n_pops ? (m.n_full[b] * static_cast<int64_t>(scale_n) + 500) / 1000 : 0;
}

int64_t pair_count(const snn_model &m, int32_t scale_n, int32_t scale_k, int target, int source)
{
    int64_t nb[SNN_MAX_POPS];
    population_sizes(m, scale_n, nb);
    const double src = static_cast<double>(m.n_full[source] * static_cast<int64_t>(scale_k)) / 1000.0;
    return static_cast<int64_t>(std::llround(m.conn_p[target][source] * src * static_cast<double>(nb[target])));
}

namespace {

int64_t circuit_neurons(const snn_model &m, int32_t scale_n)
{
    int64_t nb[SNN_MAX_POPS];
    population_sizes(m, scale_n, nb);
    int64_t n = 0;
    for (int b = 0; b < m.n_pops; ++b) n += nb[b];
    return n;
}

int64_t circuit_synapses(const snn_model &m, int32_t scale_n, int32_t scale_k)
{
    int64_t s = 0;
    for (int a = 0; a < m.n_pops; ++a)
        for (int b = 0; b < m.n_pops; ++b) s += pair_count(m, scale_n, scale_k, b, a);
    return s;
}

// A single circuit described by the batch entry c (or the spec itself).
snn_spec circuit_spec(const snn_spec &spec, int c)
{
    snn_spec one = spec;
    one.n_circuits = 0;
    one.circuits = nullptr;
    if (spec.n_circuits > 0) {
        one.scale_n_permille = spec.circuits[c].scale_n_permille;
        one.scale_k_permille = spec.circuits[c].scale_k_permille;
        one.seed = spec.circuits[c].seed;
    }
    return one;
}

}  // namespace

int64_t count_neurons(const snn_spec &spec)
{
    if (spec.custom) return spec.custom->n_neurons;
    if (spec.n_circuits <= 0) return circuit_neurons(spec.model, spec.scale_n_permille);
    int64_t base = 0, last = 0;
    for (int c = 0; c < spec.n_circuits; ++c) {
        base = (base + last + 127) / 128 * 128;
        last = circuit_neurons(spec.model, spec.circuits[c].scale_n_permille);
        if (c == 0) base = 0;
    }
    return base + last;
}

int64_t count_synapses(const snn_spec &spec)
{
    if (spec.custom) return spec.custom->n_synapses;
    if (spec.n_circuits <= 0) return circuit_synapses(spec.model, spec.scale_n_permille, spec.scale_k_permille);
    int64_t s = 0;
    for (int c = 0; c < spec.n_circuits; ++c)
        s += circuit_synapses(spec.model, spec.circuits[c].scale_n_permille, spec.circuits[c].scale_k_permille);
    return s;
}

bool validate_spec(const snn_spec &spec, std::string &why)
{
    const snn_model &m = spec.model;
    auto fail = [&](const char *msg) {
        why = msg;
        return false;
    };
    if (spec.abi_version != SNN_ABI_VERSION) return fail("abi_version mismatch");
    if (m.n_pops < 1 || m.n_pops > SNN_MAX_POPS) return fail("n_pops out of [1, SNN_MAX_POPS]");
    if (m.n_overrides < 0 || m.n_overrides > SNN_MAX_OVERRIDES) return fail("n_overrides out of range");
    if (!(m.dt_ms > 0) || !(m.C_m_pF > 0) || !(m.tau_m_ms > 0) || !(m.tau_syn_ms > 0) || !(m.tau_ref_ms >= 0))
        return fail("time constants, dt and C_m must be positive");
    if (m.tau_m_ms == m.tau_syn_ms) return fail("tau_m == tau_syn is not supported (w_f and p21 are singular)");
    if (!(m.nu_th_hz >= 0)) return fail("nu_th must be >= 0");
    const double tref_steps = m.tau_ref_ms / m.dt_ms;
    if (tref_steps > 255.0) return fail("tau_ref / dt must be <= 255 steps");
    for (int b = 0; b < m.n_pops; ++b) {
        if (!(m.k_ext[b] >= 0)) return fail("k_ext must be >= 0");
        const double lam = m.k_ext[b] * m.nu_th_hz * m.dt_ms * 1e-3;
        if (lam > 4.0) return fail("thalamic mean per step above 4 exceeds the Poisson table's accuracy");
        if (m.n_full[b] < 0) return fail("n_full must be >= 0");
    }
    for (int o = 0; o < m.n_overrides; ++o)
        if (m.ovr_source[o] < 0 || m.ovr_source[o] >= m.n_pops || m.ovr_target[o] < 0 || m.ovr_target[o] >= m.n_pops)
            return fail("override population out of range");
    if (spec.raster_capacity < 0 || spec.raster_capacity > (int64_t{1} << 31) - 1)
        return fail("raster_capacity out of [0, 2^31-1]");
    if (spec.steps_per_graph < 0 || spec.steps_per_graph > 100000) return fail("steps_per_graph out of [0, 100000]");
    if (spec.deliver_blocks < 0 || spec.deliver_blocks > 65535) return fail("deliver_blocks out of range");
    if (spec.engine < SNN_ENGINE_DEFAULT || spec.engine > SNN_ENGINE_RESIDENT) return fail("unknown engine");
    if (spec.smem_ring_rows != 0 && spec.smem_ring_rows != 8 && spec.smem_ring_rows != 16 &&
        spec.smem_ring_rows != 32 && spec.smem_ring_rows != 64)
        return fail("smem_ring_rows must be 0, 8, 16, 32 or 64");
    if (spec.engine == SNN_ENGINE_RESIDENT) {
        if (spec.n_circuits > 0) return fail("the resident engine takes one circuit");
        if (spec.record_format != SNN_RECORD_PLAIN9) return fail("the resident engine reads plain records");
        if (count_neurons(spec) > kResidentMaxNeurons) return fail("more neurons than the resident engine holds");
    }
    if (spec.record_format < SNN_RECORD_PLAIN9 || spec.record_format > SNN_RECORD_BLOCKED8)
        return fail("unknown record_format");
    if ((spec.record_format == SNN_RECORD_PACKED_I8 || spec.record_format == SNN_RECORD_PACKED_BF16) &&
        count_neurons(spec) > kPackedMaxNeurons)
        return fail("packed records hold at most 2^20 neurons");
    if (is_blocked(spec.record_format)) {
        if (spec.n_circuits > 0) return fail("blocked records take one circuit");
        if (spec.engine == SNN_ENGINE_PERSISTENT || spec.engine == SNN_ENGINE_PIPELINED)
            return fail("blocked records run on the graph engine");
    }
    if (spec.n_circuits < 0 || spec.n_circuits > SNN_MAX_CIRCUITS) return fail("n_circuits out of [0, SNN_MAX_CIRCUITS]");
    if (spec.n_circuits > 0 && !spec.circuits) return fail("circuits missing");
    if (spec.n_circuits > 0 && spec.custom) return fail("a custom network cannot be batched");
    for (int c = 0; c < spec.n_circuits; ++c) {
        snn_spec one = spec;
        one.n_circuits = 0;
        one.circuits = nullptr;
        one.scale_n_permille = spec.circuits[c].scale_n_permille;
        one.scale_k_permille = spec.circuits[c].scale_k_permille;
        if (!validate_spec(one, why)) {
            why = "circuit " + std::to_string(c) + ": " + why;
            return false;
        }
    }
    if (spec.n_circuits > 0) {
        if (count_neurons(spec) > (int64_t{1} << 30)) return fail("batched neuron count above 2^30");
        if (count_synapses(spec) > (int64_t{1} << 35)) return fail("batched synapse count above 2^35");
        return true;
    }
    if (spec.custom) {
        const snn_custom_net &c = *spec.custom;
        if (c.n_neurons < 1 || c.n_neurons > (int64_t{1} << 30)) return fail("custom n_neurons out of [1, 2^30]");
        if (c.n_synapses < 0) return fail("custom n_synapses < 0");
        if (c.n_synapses > 0 && (!c.pre || !c.post || !c.w_fx || !c.delay))
            return fail("custom synapse arrays missing");
        if (!c.u0) return fail("custom u0 missing");
        if (c.pop_offsets[0] != 0 || c.pop_offsets[m.n_pops] != c.n_neurons)
            return fail("custom pop_offsets must run from 0 to n_neurons");
        for (int b = 0; b < m.n_pops; ++b)
            if (c.pop_offsets[b + 1] < c.pop_offsets[b]) return fail("custom pop_offsets must be nondecreasing");
    } else {
        if (spec.scale_n_permille < 1 || spec.scale_k_permille < 0 || spec.scale_n_permille > 100000 ||
            spec.scale_k_permille > 100000)
            return fail("scales out of range");
        int64_t nb[SNN_MAX_POPS];
        population_sizes(m, spec.scale_n_permille, nb);
        int64_t n = 0;
        for (int b = 0; b < m.n_pops; ++b) n += nb[b];
        if (n < 1 || n > (int64_t{1} << 30)) return fail("neuron count out of [1, 2^30]");
        for (int a = 0; a < m.n_pops; ++a)
            for (int b = 0; b < m.n_pops; ++b) {
                if (!(m.conn_p[b][a] >= 0)) return fail("connection probability < 0");
                const int64_t k = pair_count(m, spec.scale_n_permille, spec.scale_k_permille, b, a);
                if (k > 0 && (nb[a] == 0 || nb[b] == 0)) return fail("synapses requested for an empty population");
                if (!(m.d_sd_ms[a] >= 0) || !(m.w_sd_mV[a] >= 0)) return fail("negative SD");
            }
        if (count_synapses(spec) > (int64_t{1} << 34)) return fail("more than 2^34 synapses");
    }
    return true;
}

Layout make_layout(const snn_spec &spec)
{
    auto up = [](uint64_t x) { return (x + 255) & ~uint64_t{255}; };
    Layout L{};
    const int64_t n = count_neurons(spec);
    const int64_t s = count_synapses(spec);
    L.npad = (n + kNeuronAlign - 1) / kNeuronAlign * kNeuronAlign;
    L.syn_padded_max = s + int64_t{kRowAlign - 1} * n;
    L.rast_cap = spec.raster_capacity > 0 ? spec.raster_capacity : (int64_t{1} << 24);
    uint64_t o = 0;
    L.ctl = o; o = up(o + sizeof(Ctl));
    L.tables = o; o = up(o + sizeof(StaticTables));
    L.U = o; o = up(o + 4 * L.npad);
    L.I = o; o = up(o + 4 * L.npad);
    L.R = o; o = up(o + L.npad);
    L.ring = o; o = up(o + uint64_t{4} * kDMax * L.npad);
    L.row_ptr = o; o = up(o + 8 * (n + 5));  // 4 spare entries: quads read row_ptr[i0 .. i0+4]
    const int fmt = spec.record_format;
    const uint64_t wbytes = fmt == SNN_RECORD_PACKED_I8 ? 1 : fmt == SNN_RECORD_PACKED_BF16 ? 2 : 4;
    if (is_blocked(fmt)) {
        // rows of quad-padded block segments (a nonempty segment gains at most
        // kBlockQuad - 1 pad entries): BLOCKED6 keeps uint16 records and int32 weights,
        // BLOCKED4 16-byte quads of records and bfloat16 weights, BLOCKED8 interleaved
        // (weight, record) pairs; then the per-row block table
        L.syn_padded_max = s + (kBlockQuad - 1) * std::min<int64_t>(s, n * int64_t{max_target_blocks(n)});
        if (fmt == SNN_RECORD_BLOCKED6) {
            L.syn_tgt = o; o = up(o + 2 * L.syn_padded_max + 16);
            L.syn_w = o; o = up(o + 4 * L.syn_padded_max + 16);
        } else if (fmt == SNN_RECORD_BLOCKED8) {
            L.syn_tgt = o; o = up(o + 8 * L.syn_padded_max + 16);
            L.syn_w = o; o = up(o + 16);
        } else {
            L.syn_tgt = o; o = up(o + 4 * L.syn_padded_max + 16);
            L.syn_w = o; o = up(o + 16);
        }
        L.syn_d = o; o = up(o + 2 * uint64_t(n) * (max_target_blocks(n) + 1) + 16);
    } else {
        L.syn_tgt = o; o = up(o + 4 * L.syn_padded_max);
        L.syn_w = o; o = up(o + wbytes * L.syn_padded_max + 16);
        L.syn_d = o; o = up(o + (fmt == SNN_RECORD_PLAIN9 ? L.syn_padded_max : 0) + 16);
    }
    const bool resident = spec.engine == SNN_ENGINE_RESIDENT;
    const int64_t res_blocks = resident ? resident_max_blocks(n) : 0;
    L.blocks = o; o = up(o + 4 * std::max<int64_t>(is_blocked(fmt) ? max_target_blocks(n) + 1 : 1, res_blocks + 1));
    // resident engine: the block tables, the outboxes and the inbox slots
    L.seg = o; o = up(o + (resident ? resident_tables(n, res_blocks).total : 0));
    L.mbox = o; o = up(o + (resident ? 4 * uint64_t{4} * res_blocks * kResidentMboxWords : 0));
    L.inbox = o; o = up(o + (resident ? 4 * uint64_t{4} * res_blocks * res_blocks * kResidentSlotWords : 0));
    L.res_rec = o; o = up(o + (resident ? 8 * uint64_t(L.syn_padded_max) + 16 : 0));
    L.rast_nrn = o; o = up(o + 4 * L.rast_cap);
    L.rast_t = o; o = up(o + 4 * L.rast_cap);
    L.U2 = o; o = up(o + 4 * L.npad);
    L.R2 = o; o = up(o + L.npad);
    L.queue = o; o = up(o + uint64_t{4} * sizeof(QueueEntry) * L.npad);
    L.qcount = o; o = up(o + uint64_t{4} * 4 * (L.npad / 128 + 1));
    L.pop_id = o; o = up(o + L.npad);
    L.group_circuit = o; o = up(o + 4 * (L.npad / 128 + 1));
    L.circuits = o; o = up(o + sizeof(CircuitInfo) * std::max(1, spec.n_circuits));
    L.total = o;
    return L;
}

namespace {

// Amplitude law of a synapse from population a to population b.
void amplitude_law(const snn_model &m, int a, int b, double &mu, double &sd)
{
    mu = m.w_mean_mV[a];
    sd = m.w_sd_mV[a];
    for (int o = 0; o < m.n_overrides; ++o)
        if (m.ovr_source[o] == a && m.ovr_target[o] == b) {
            mu = m.ovr_w_mean_mV[o];
            sd = m.ovr_w_sd_mV[o];
        }
}

struct EdgeList {
    std::vector<int32_t> pre, post, w;
    std::vector<uint8_t> d;
};

// Sample every synapse of the microcircuit.  Synapse k of pair (a -> b) uses Philox
// counter (k, a, b, 0) under key (seed, kStreamConnect); the list is in (a, b, k) order.
void sample_edges(const snn_spec &spec, const Constants &c, EdgeList &e, int nthreads)
{
    const snn_model &m = spec.model;
    const int P = m.n_pops;
    int64_t nb[SNN_MAX_POPS], off[SNN_MAX_POPS + 1];
    population_sizes(m, spec.scale_n_permille, nb);
    off[0] = 0;
    for (int b = 0; b < P; ++b) off[b + 1] = off[b] + nb[b];
    // pair bases in (a, b) order
    std::vector<int64_t> base(P * P + 1, 0);
    for (int a = 0; a < P; ++a)
        for (int b = 0; b < P; ++b)
            base[a * P + b + 1] = base[a * P + b] + pair_count(m, spec.scale_n_permille, spec.scale_k_permille, b, a);
    const int64_t S = base[P * P];
    e.pre.resize(S);
    e.post.resize(S);
    e.w.resize(S);
    e.d.resize(S);
    const uint64_t seed = spec.seed;
    const double w_f = c.w_f, dt = m.dt_ms;
    parallel_for(nthreads, S, [&](int, int64_t lo, int64_t hi) {
        int pair = static_cast<int>(std::upper_bound(base.begin(), base.end(), lo) - base.begin()) - 1;
        for (int64_t s = lo; s < hi; ++s) {
            while (s >= base[pair + 1]) ++pair;
            const int a = pair / P, b = pair % P;
            const int64_t k = s - base[pair];
            const Block4 r = philox4x64_10(static_cast<uint64_t>(k), static_cast<uint64_t>(a),
                                           static_cast<uint64_t>(b), 0, seed, kStreamConnect);
            e.pre[s] = static_cast<int32_t>(off[a] + scale_below(r.w[0], nb[a]));
            e.post[s] = static_cast<int32_t>(off[b] + scale_below(r.w[1], nb[b]));
            double zc, zs;
            gauss_pair(r.w[2], r.w[3], zc, zs);
            double mu, sd;
            amplitude_law(m, a, b, mu, sd);
            double amp = mu + sd * zc;
            if (mu >= 0.0) amp = amp < 0.0 ? 0.0 : amp;  // excitatory stays >= 0
            else amp = amp > 0.0 ? 0.0 : amp;            // inhibitory stays <= 0
            e.w[s] = static_cast<int32_t>(std::llround(amp * w_f * 4096.0));
            const double delay_ms = m.d_mean_ms[a] + m.d_sd_ms[a] * zs;
            long long steps = std::llround(delay_ms / dt);
            steps = std::min<long long>(std::max<long long>(steps, 1), kDMax - 1);
            e.d[s] = static_cast<uint8_t>(steps);
        }
    });
}

uint16_t to_bf16_even(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return static_cast<uint16_t>(u >> 16);
}

// Compressed records (§5.3): packed words, and int8 codes fitted per population pair or
// bfloat16 currents; the plain arrays are released afterwards.
void pack_records(HostNetwork &net, int /*n_pops*/, int nthreads)
{
    const int64_t n = net.n;
    const int64_t S = net.n_syn_padded;
    net.word.assign(S, 0);
    std::vector<uint8_t> tpop(S, 0);
    // extremes of each (source, target) pair, per thread then merged
    const int T = std::max(1, nthreads);
    std::vector<std::vector<int64_t>> lo(T, std::vector<int64_t>(64, INT64_MAX)), hi(T, std::vector<int64_t>(64, INT64_MIN));
    parallel_for(T, n, [&](int th, int64_t r0, int64_t r1) {
        for (int64_t i = r0; i < r1; ++i) {
            const int a = net.pop_id[i];
            const int64_t real_end = net.row_ptr[i] + net.out_degree[i];
            for (int64_t s = net.row_ptr[i]; s < net.row_ptr[i + 1]; ++s) {
                const int b = net.pop_id[net.tgt[s]];
                tpop[s] = static_cast<uint8_t>(b);
                uint32_t w = static_cast<uint32_t>(net.tgt[s]) | (static_cast<uint32_t>(net.d[s]) << kWordDelayShift) |
                             (static_cast<uint32_t>(b) << kWordPopShift);
                if (s >= real_end) {
                    w |= kWordPad;
                } else {
                    lo[th][a * 8 + b] = std::min<int64_t>(lo[th][a * 8 + b], net.w[s]);
                    hi[th][a * 8 + b] = std::max<int64_t>(hi[th][a * 8 + b], net.w[s]);
                }
                net.word[s] = w;
            }
        }
    });
    for (int a = 0; a < SNN_MAX_POPS; ++a)
        for (int b = 0; b < SNN_MAX_POPS; ++b) {
            int64_t l = INT64_MAX, h = INT64_MIN;
            for (int th = 0; th < T; ++th) {
                l = std::min(l, lo[th][a * 8 + b]);
                h = std::max(h, hi[th][a * 8 + b]);
            }
            int64_t base = 0, step = 1;
            if (l <= h) {
                base = l + (h - l) / 2;
                step = std::max<int64_t>(1, (h - l + 253) / 254);
            }
            net.i8_base[a][b] = static_cast<int32_t>(base);
            net.i8_step[a][b] = static_cast<int32_t>(step);
        }
    if (net.format == SNN_RECORD_PACKED_I8) {
        net.wbytes.assign(S, 0);
        parallel_for(T, n, [&](int, int64_t r0, int64_t r1) {
            for (int64_t i = r0; i < r1; ++i) {
                const int a = net.pop_id[i];
                const int64_t real_end = net.row_ptr[i] + net.out_degree[i];
                for (int64_t s = net.row_ptr[i]; s < real_end; ++s) {
                    const int b = tpop[s];
                    const int64_t base = net.i8_base[a][b], step = net.i8_step[a][b];
                    long long q = std::llround(static_cast<double>(net.w[s] - base) / static_cast<double>(step));
                    q = std::min<long long>(127, std::max<long long>(-127, q));
                    net.wbytes[s] = static_cast<uint8_t>(static_cast<int8_t>(q));
                }
            }
        });
    } else {
        net.wbytes.assign(2 * S, 0);
        parallel_for(T, S, [&](int, int64_t s0, int64_t s1) {
            for (int64_t s = s0; s < s1; ++s) {
                const uint16_t h = to_bf16_even(static_cast<float>(net.w[s]) * (1.0f / 4096.0f));
                std::memcpy(&net.wbytes[2 * s], &h, 2);
            }
        });
    }
    std::vector<int32_t>().swap(net.tgt);
    std::vector<int32_t>().swap(net.w);
    std::vector<uint8_t>().swap(net.d);
}

}  // namespace

namespace {

// Target blocks of the blocked format: boundaries at multiples of kBlockAlign, no block
// wider than kBlockMaxWidth.  One CTA per SM delivers into a block, so the launch takes
// as long as its heaviest block: the cut minimises the largest in-degree sum of a block
// (the events a block receives from uniformly drawn senders) for a block count of at
// most `budget`.  For a bound L, cutting greedily wherever the next group of kBlockAlign
// targets would pass L or the width limit gives the fewest blocks; the smallest L whose
// greedy cut fits the budget is found by bisection.
std::vector<int32_t> cut_blocks(const std::vector<int64_t> &grp, int64_t n, int64_t L, int64_t maxw)
{
    std::vector<int32_t> blk{0};
    int64_t load = 0;
    for (size_t g = 0; g < grp.size(); ++g) {
        const int64_t j = static_cast<int64_t>(g) * kBlockAlign;
        if (j > blk.back() && (j - blk.back() + kBlockAlign > maxw || load + grp[g] > L)) {
            blk.push_back(static_cast<int32_t>(j));
            load = 0;
        }
        load += grp[g];
    }
    blk.push_back(static_cast<int32_t>(n));
    return blk;
}

// Budget: the fewest whole waves of `num_sms` CTAs that the width limit allows, but no
// more blocks than leave segments of ~16 synapses on average (shorter ones are mostly
// quad padding) and no more than the layout holds; num_sms = 0 asks for n / 512 blocks.
std::vector<int32_t> target_blocks(const std::vector<int64_t> &indeg, int64_t n, int num_sms)
{
    std::vector<int64_t> grp((n + kBlockAlign - 1) / kBlockAlign, 0);
    int64_t total = 0, gmax = 0;
    for (int64_t j = 0; j < n; ++j) grp[j / kBlockAlign] += indeg[j];
    for (int64_t g : grp) {
        total += g;
        gmax = std::max(gmax, g);
    }
    auto bisect = [&](int64_t budget, int64_t maxw) {
        int64_t lo = gmax, hi = std::max(gmax, total);
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (static_cast<int64_t>(cut_blocks(grp, n, mid, maxw).size()) - 1 <= budget) hi = mid;
            else lo = mid + 1;
        }
        return cut_blocks(grp, n, lo, maxw);
    };
    const int64_t seg_cap = total / (16 * std::max<int64_t>(n, 1));  // ~16 synapses per (row, block) segment
    const int64_t min_blocks = n / (kBlockMaxWidth - kBlockAlign) + 1;
    int64_t budget;
    if (num_sms > 0) {
        budget = (min_blocks + num_sms - 1) / num_sms * num_sms;
        budget = std::min(budget, std::max(min_blocks, seg_cap));
    } else {
        budget = std::max(min_blocks, (n + kBlockAvgWidth - 1) / kBlockAvgWidth);
    }
    budget = std::min<int64_t>(budget, max_target_blocks(n));
    return bisect(budget, kBlockMaxWidth);
}

// Regroups the delay-sorted rows into block-grouped rows (delay order kept inside a
// block) and encodes each synapse as (local target | delay << 10).  Every (row, block)
// segment is padded to a multiple of kBlockQuad records with zero-weight entries
// (local target 0, delay 1), so that a segment is a whole number of aligned quads.
bool pack_blocked(HostNetwork &net, int nthreads, int num_sms, std::string &why)
{
    const int64_t n = net.n;
    std::vector<int64_t> indeg(n, 0);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t s = net.row_ptr[i], e = net.row_ptr[i] + net.out_degree[i]; s < e; ++s) ++indeg[net.tgt[s]];
    net.blk = target_blocks(indeg, n, num_sms);
    const int B = static_cast<int>(net.blk.size()) - 1;
    if (B > max_target_blocks(n)) {
        why = "internal: more target blocks than the layout bound";
        return false;
    }
    std::vector<int32_t> block_of(n);
    for (int b = 0; b < B; ++b)
        for (int64_t j = net.blk[b]; j < net.blk[b + 1]; ++j) block_of[j] = b;
    // padded segment lengths give the row lengths
    net.seg.assign(static_cast<size_t>(n) * (B + 1), 0);
    std::vector<int64_t> rp(n + 1, 0);
    std::atomic<bool> too_long{false};
    parallel_for(nthreads, n, [&](int, int64_t lo, int64_t hi) {
        std::vector<int64_t> cnt(B);
        for (int64_t i = lo; i < hi; ++i) {
            std::fill(cnt.begin(), cnt.end(), 0);
            for (int64_t s = net.row_ptr[i], e = s + net.out_degree[i]; s < e; ++s) ++cnt[block_of[net.tgt[s]]];
            uint16_t *sg = &net.seg[static_cast<size_t>(i) * (B + 1)];
            int64_t run = 0;
            for (int b = 0; b < B; ++b) {
                sg[b] = static_cast<uint16_t>(run);
                run += (cnt[b] + kBlockQuad - 1) / kBlockQuad * kBlockQuad;
                if (run > 65535) too_long.store(true, std::memory_order_relaxed);
            }
            sg[B] = static_cast<uint16_t>(run);
            rp[i + 1] = run;
        }
    });
    if (too_long) {
        why = "blocked records hold rows of at most 65535 padded synapses";
        return false;
    }
    for (int64_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
    const int64_t S = rp[n];
    // BLOCKED8 keeps the local target and the delay in separate 16-bit fields of its
    // 32-bit record; the other formats pack both in 16 bits
    const bool wide = net.format == SNN_RECORD_BLOCKED8;
    if (wide) net.word.assign(2 * S, 0);
    else net.rec16.assign(S, static_cast<uint16_t>(1u << kBlockLocalBits));
    std::vector<int32_t> w(S, 0);
    parallel_for(nthreads, n, [&](int, int64_t lo, int64_t hi) {
        std::vector<int64_t> pos(B);
        for (int64_t i = lo; i < hi; ++i) {
            const uint16_t *sg = &net.seg[static_cast<size_t>(i) * (B + 1)];
            for (int b = 0; b < B; ++b) pos[b] = rp[i] + sg[b];
            for (int64_t s = net.row_ptr[i], e = s + net.out_degree[i]; s < e; ++s) {
                const int b = block_of[net.tgt[s]];
                const int64_t dst = pos[b]++;
                const uint32_t local = static_cast<uint32_t>(net.tgt[s] - net.blk[b]);
                if (wide) net.word[2 * dst + 1] = local | (uint32_t{net.d[s]} << 16);
                else net.rec16[dst] = static_cast<uint16_t>(local | (uint32_t{net.d[s]} << kBlockLocalBits));
                w[dst] = net.w[s];
            }
        }
    });
    net.row_ptr = std::move(rp);
    net.n_syn_padded = S;
    std::vector<int32_t>().swap(net.tgt);
    std::vector<uint8_t>().swap(net.d);
    if (net.format == SNN_RECORD_BLOCKED4) {
        // quad q: words 4q, 4q+1 hold records 4q..4q+3, words 4q+2, 4q+3 their bfloat16
        // currents (round to nearest even, the SNN_RECORD_PACKED_BF16 weights)
        net.word.assign(S, 0);
        parallel_for(nthreads, S / kBlockQuad, [&](int, int64_t q0, int64_t q1) {
            for (int64_t q = q0; q < q1; ++q) {
                const int64_t e = q * kBlockQuad;
                uint16_t h[4];
                for (int k = 0; k < 4; ++k) h[k] = to_bf16_even(static_cast<float>(w[e + k]) * (1.0f / 4096.0f));
                net.word[e] = uint32_t{net.rec16[e]} | uint32_t{net.rec16[e + 1]} << 16;
                net.word[e + 1] = uint32_t{net.rec16[e + 2]} | uint32_t{net.rec16[e + 3]} << 16;
                net.word[e + 2] = uint32_t{h[0]} | uint32_t{h[1]} << 16;
                net.word[e + 3] = uint32_t{h[2]} | uint32_t{h[3]} << 16;
            }
        });
        std::vector<uint16_t>().swap(net.rec16);
        std::vector<int32_t>().swap(net.w);
    } else if (net.format == SNN_RECORD_BLOCKED8) {
        // synapse e: word 2e its int32 weight, word 2e+1 its record (local target | delay
        // << 16; padding: local 0, delay 1, weight 0), so a quad is 32 contiguous bytes
        parallel_for(nthreads, S, [&](int, int64_t e0, int64_t e1) {
            for (int64_t e = e0; e < e1; ++e) {
                net.word[2 * e] = static_cast<uint32_t>(w[e]);
                if (w[e] == 0) net.word[2 * e + 1] = 1u << 16;
            }
        });
        std::vector<int32_t>().swap(net.w);
    } else {
        net.w = std::move(w);
    }
    return true;
}

// Resident engine: targets cut into blocks of `width` consecutive neurons (one CTA each),
// and the records rearranged block-major: block p's region holds every synapse into the
// block, sender by sender, each sender's segment in the delay order of its row (a stable
// pass over the delay-sorted rows).  The plain record arrays keep their types; row_ptr
// then only gives row lengths (prefix sums of the out-degrees).  The tables of
// resident_tables() locate every (block, sender) segment.
bool block_major_records(HostNetwork &net, int64_t width, int nthreads, std::string &why)
{
    const int64_t n = net.n;
    const int B = static_cast<int>((n + width - 1) / width);
    net.blk.resize(B + 1);
    for (int b = 0; b <= B; ++b) net.blk[b] = static_cast<int32_t>(std::min<int64_t>(n, int64_t{b} * width));
    // segment lengths, [block][sender]
    std::vector<uint32_t> len(static_cast<size_t>(B) * n, 0);
    parallel_for(nthreads, n, [&](int, int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i)
            for (int64_t s = net.row_ptr[i], e = s + net.out_degree[i]; s < e; ++s)
                ++len[static_cast<size_t>(net.tgt[s] / width) * n + i];
    });
    const ResTables T = resident_tables(n, B);
    net.restab.assign(T.total, 0);
    int64_t *rbase = reinterpret_cast<int64_t *>(net.restab.data() + T.rbase);
    uint32_t *coarse = reinterpret_cast<uint32_t *>(net.restab.data() + T.coarse);
    uint8_t *lens = net.restab.data() + T.lens;
    uint32_t *offt = reinterpret_cast<uint32_t *>(net.restab.data() + T.offt);
    rbase[0] = 0;
    for (int b = 0; b < B; ++b) {
        uint64_t run = 0;
        const uint32_t *lb = &len[static_cast<size_t>(b) * n];
        uint32_t *ob = offt + static_cast<size_t>(b) * (n + 1);
        uint32_t *cb = coarse + static_cast<size_t>(b) * T.coarse_stride;
        uint8_t *lnb = lens + static_cast<size_t>(b) * T.lens_stride;
        for (int64_t i = 0; i < n; ++i) {
            if (i % 32 == 0) cb[i / 32] = static_cast<uint32_t>(run);
            ob[i] = static_cast<uint32_t>(run);
            lnb[i] = static_cast<uint8_t>(std::min<uint32_t>(lb[i], kResidentEscape));
            if (lb[i] >= kResidentEscape) cb[i / 32] |= kResidentGroupFlag;
            run += lb[i];
        }
        if (run >= kResidentGroupFlag) {
            why = "a target block receives more than 2^31 synapses";
            return false;
        }
        ob[n] = static_cast<uint32_t>(run);
        cb[(n + 31) / 32] = static_cast<uint32_t>(run);
        rbase[b + 1] = rbase[b] + static_cast<int64_t>(run);
    }
    const int64_t S = rbase[B];
    std::vector<int32_t> t2(S), w2(S);
    std::vector<uint8_t> d2(S);
    parallel_for(nthreads, n, [&](int, int64_t lo, int64_t hi) {
        std::vector<int64_t> pos(B);
        for (int64_t i = lo; i < hi; ++i) {
            for (int b = 0; b < B; ++b) pos[b] = rbase[b] + offt[static_cast<size_t>(b) * (n + 1) + i];
            for (int64_t s = net.row_ptr[i], e = s + net.out_degree[i]; s < e; ++s) {
                const int64_t dst = pos[net.tgt[s] / width]++;
                t2[dst] = net.tgt[s];
                w2[dst] = net.w[s];
                d2[dst] = net.d[s];
            }
        }
    });
    // the step kernel's 8-byte records: the weight in the low word, the target's index in
    // its block and the delay (above bit 16) in the high word: one contiguous read per
    // segment (the three arrays stay for phase 2 alone and the tests)
    net.rec8.resize(S);
    parallel_for(nthreads, B, [&](int, int64_t lo, int64_t hi) {
        for (int64_t b = lo; b < hi; ++b)
            for (int64_t k = rbase[b]; k < rbase[b + 1]; ++k) {
                const uint32_t local = static_cast<uint32_t>(t2[k] - net.blk[b]);
                net.rec8[k] = static_cast<uint64_t>(static_cast<uint32_t>(w2[k])) |
                              (static_cast<uint64_t>(local | (static_cast<uint32_t>(d2[k]) << 16)) << 32);
            }
    });
    net.tgt = std::move(t2);
    net.w = std::move(w2);
    net.d = std::move(d2);
    for (int64_t i = 0; i < n; ++i) net.row_ptr[i + 1] = net.row_ptr[i] + net.out_degree[i];
    net.n_syn_padded = S;
    return true;
}

bool build_one(const snn_spec &spec, const Constants &c, HostNetwork &net, std::string &why, int num_sms);
}

bool build_host_network(const snn_spec &spec, const Constants &c, HostNetwork &net, std::string &why, int num_sms)
{
    if (spec.n_circuits <= 0) {
        if (!build_one(spec, c, net, why, num_sms)) return false;
        net.circuits = {CircuitInfo{0, net.n, spec.seed, 0}};
        if (spec.engine == SNN_ENGINE_RESIDENT && num_sms > 0) {
            const int64_t width = resident_width(net.n, num_sms);
            if (width == 0) {
                why = "more neurons than the resident engine holds on this GPU (1024 per SM)";
                return false;
            }
            if (!block_major_records(net, width, resolve_threads(spec.n_threads), why)) return false;
        }
        return true;
    }
    // a batch: every circuit built alone (in plain records), placed at a 128-aligned base
    const int fmt = spec.record_format;
    HostNetwork all;
    all.format = SNN_RECORD_PLAIN9;
    {
        const int64_t n_all = count_neurons(spec);
        const int64_t s_all = count_synapses(spec) + int64_t{kRowAlign - 1} * n_all;
        all.row_ptr.reserve(n_all + 1);
        all.out_degree.reserve(n_all);
        all.u0.reserve(n_all);
        all.pop_id.reserve(n_all);
        all.tgt.reserve(s_all);
        all.w.reserve(s_all);
        all.d.reserve(s_all);
    }
    int64_t base = 0;
    for (int ci = 0; ci < spec.n_circuits; ++ci) {
        snn_spec one = circuit_spec(spec, ci);
        one.record_format = SNN_RECORD_PLAIN9;
        HostNetwork h;
        if (!build_one(one, c, h, why, 0)) return false;
        if (ci > 0) base = (all.n + 127) / 128 * 128;
        // neurons: gap (inert) then the circuit
        const int64_t syn_base = all.row_ptr.empty() ? 0 : all.row_ptr.back();
        if (all.row_ptr.empty()) all.row_ptr.push_back(0);
        while (all.n < base) {
            all.row_ptr.push_back(syn_base);
            all.out_degree.push_back(0);
            all.u0.push_back(0.0f);
            all.pop_id.push_back(0);
            ++all.n;
        }
        for (int64_t i = 0; i < h.n; ++i) {
            all.row_ptr.push_back(syn_base + h.row_ptr[i + 1]);
            all.out_degree.push_back(h.out_degree[i]);
            all.u0.push_back(h.u0[i]);
            all.pop_id.push_back(h.pop_id[i]);
        }
        all.n += h.n;
        for (size_t s2 = 0; s2 < h.tgt.size(); ++s2) all.tgt.push_back(h.tgt[s2] + static_cast<int32_t>(base));
        all.w.insert(all.w.end(), h.w.begin(), h.w.end());
        all.d.insert(all.d.end(), h.d.begin(), h.d.end());
        all.n_syn += h.n_syn;
        all.max_row = std::max(all.max_row, h.max_row);
        all.circuits.push_back(CircuitInfo{base, h.n, one.seed, 0});
    }
    all.npad = (all.n + kNeuronAlign - 1) / kNeuronAlign * kNeuronAlign;
    all.n_syn_padded = all.row_ptr.back();
    all.pop_off.assign(SNN_MAX_POPS + 1, all.n);
    all.pop_off[0] = 0;
    all.format = fmt;
    if (fmt != SNN_RECORD_PLAIN9) pack_records(all, spec.model.n_pops, resolve_threads(spec.n_threads));
    net = std::move(all);
    return true;
}

namespace {

bool build_one(const snn_spec &spec, const Constants &c, HostNetwork &net, std::string &why, int num_sms)
{
    const int nthreads = resolve_threads(spec.n_threads);
    const snn_model &m = spec.model;
    const int64_t n = count_neurons(spec);
    net.n = n;
    net.npad = (n + kNeuronAlign - 1) / kNeuronAlign * kNeuronAlign;
    net.pop_off.assign(SNN_MAX_POPS + 1, n);
    EdgeList e;
    if (spec.custom) {
        const snn_custom_net &cn = *spec.custom;
        for (int b = 0; b <= m.n_pops; ++b) net.pop_off[b] = cn.pop_offsets[b];
        const int64_t S = cn.n_synapses;
        e.pre.assign(cn.pre, cn.pre + S);
        e.post.assign(cn.post, cn.post + S);
        e.w.assign(cn.w_fx, cn.w_fx + S);
        e.d.assign(cn.delay, cn.delay + S);
        for (int64_t s = 0; s < S; ++s) {
            if (e.pre[s] < 0 || e.pre[s] >= n || e.post[s] < 0 || e.post[s] >= n) {
                why = "custom synapse endpoint out of [0, n_neurons)";
                return false;
            }
            if (e.d[s] < 1 || e.d[s] > kDMax - 1) {
                why = "custom delay out of [1, 63]";
                return false;
            }
        }
        net.u0.assign(cn.u0, cn.u0 + n);
    } else {
        int64_t nb[SNN_MAX_POPS];
        population_sizes(m, spec.scale_n_permille, nb);
        net.pop_off[0] = 0;
        for (int b = 0; b < m.n_pops; ++b) net.pop_off[b + 1] = net.pop_off[b] + nb[b];
        sample_edges(spec, c, e, nthreads);
        // initial potentials: Philox counter (i, 0, 0, 0) under key (seed, kStreamInitial)
        net.u0.resize(n);
        for (int b = 0; b < m.n_pops; ++b) {
            const int64_t lo = net.pop_off[b], hi = net.pop_off[b + 1];
            const double mu = m.u0_mean_mV[b], sd = m.u0_sd_mV[b], rest = m.u_rest_mV;
            parallel_for(nthreads, hi - lo, [&](int, int64_t a0, int64_t a1) {
                for (int64_t i = lo + a0; i < lo + a1; ++i) {
                    const Block4 r = philox4x64_10(static_cast<uint64_t>(i), 0, 0, 0, spec.seed, kStreamInitial);
                    double zc, zs;
                    gauss_pair(r.w[0], r.w[1], zc, zs);
                    net.u0[i] = static_cast<float>(mu + sd * zc - rest);
                }
            });
        }
    }
    const int64_t S = static_cast<int64_t>(e.pre.size());
    net.n_syn = S;

    // Pass 1: stable counting sort by sender (per-thread histograms keep it deterministic).
    const int T = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(nthreads, S / 65536 + 1)));
    std::vector<std::vector<int64_t>> hist(T, std::vector<int64_t>(n + 1, 0));
    parallel_for(T, S, [&](int t, int64_t lo, int64_t hi) {
        auto &h = hist[t];
        for (int64_t s = lo; s < hi; ++s) ++h[e.pre[s]];
    });
    std::vector<int64_t> row_len(n, 0);
    {
        int64_t run = 0;
        for (int64_t i = 0; i < n; ++i) {
            for (int t = 0; t < T; ++t) {
                const int64_t cnt = hist[t][i];
                hist[t][i] = run;
                run += cnt;
                row_len[i] += cnt;
            }
        }
    }
    std::vector<int32_t> s_post(S), s_w(S);
    std::vector<uint8_t> s_d(S);
    parallel_for(T, S, [&](int t, int64_t lo, int64_t hi) {
        auto &h = hist[t];
        for (int64_t s = lo; s < hi; ++s) {
            const int64_t dst = h[e.pre[s]]++;
            s_post[dst] = e.post[s];
            s_w[dst] = e.w[s];
            s_d[dst] = e.d[s];
        }
    });
    hist.clear();
    hist.shrink_to_fit();
    EdgeList().pre.swap(e.pre);
    EdgeList().post.swap(e.post);
    EdgeList().w.swap(e.w);
    EdgeList().d.swap(e.d);

    // Pass 2: within each row, stable counting sort by delay into the padded layout.
    net.row_ptr.assign(n + 1, 0);
    net.out_degree.resize(n);
    std::vector<int64_t> src_ptr(n + 1, 0);
    int64_t maxrow = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t padded = (row_len[i] + kRowAlign - 1) / kRowAlign * kRowAlign;
        net.row_ptr[i + 1] = net.row_ptr[i] + padded;
        src_ptr[i + 1] = src_ptr[i] + row_len[i];
        net.out_degree[i] = static_cast<int32_t>(row_len[i]);
        maxrow = std::max(maxrow, padded);
    }
    net.max_row = static_cast<int32_t>(maxrow);
    net.n_syn_padded = net.row_ptr[n];
    net.tgt.assign(net.n_syn_padded, 0);
    net.w.assign(net.n_syn_padded, 0);
    net.d.assign(net.n_syn_padded, 1);
    parallel_for(nthreads, n, [&](int, int64_t lo, int64_t hi) {
        int64_t cnt[kDMax];
        for (int64_t i = lo; i < hi; ++i) {
            std::fill(cnt, cnt + kDMax, 0);
            for (int64_t s = src_ptr[i]; s < src_ptr[i + 1]; ++s) ++cnt[s_d[s]];
            int64_t pos = net.row_ptr[i];
            for (int k = 0; k < kDMax; ++k) {
                const int64_t c0 = cnt[k];
                cnt[k] = pos;
                pos += c0;
            }
            for (int64_t s = src_ptr[i]; s < src_ptr[i + 1]; ++s) {
                const int64_t dst = cnt[s_d[s]]++;
                net.tgt[dst] = s_post[s];
                net.w[dst] = s_w[s];
                net.d[dst] = s_d[s];
            }
            // padding entries: zero weight onto the sender itself, delay 1
            for (int64_t s = pos; s < net.row_ptr[i + 1]; ++s) {
                net.tgt[s] = static_cast<int32_t>(i);
                net.w[s] = 0;
                net.d[s] = 1;
            }
        }
    });
    net.pop_id.assign(n, 0);
    for (int b = 0; b < m.n_pops; ++b)
        for (int64_t i = net.pop_off[b]; i < net.pop_off[b + 1]; ++i) net.pop_id[i] = static_cast<uint8_t>(b);
    net.format = spec.record_format;
    if (is_blocked(net.format)) return pack_blocked(net, nthreads, num_sms, why);
    if (net.format != SNN_RECORD_PLAIN9) pack_records(net, spec.model.n_pops, nthreads);
    return true;
}

}  // namespace

}  // namespace snn
