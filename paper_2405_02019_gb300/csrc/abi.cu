// C ABI of the simulator: network setup, the CUDA-graph step engine and raster readout.
//
// The step engine captures `steps_per_graph` steps (each: k_update then k_deliver,
// the two phases of Listing push2, §3.1) plus one counter advance into a CUDA graph
// at build time and replays it; remainders are launched directly.  The step index
// lives on the device (Ctl::t_base), so a replay needs no host-side parameter update
// and no host round trip happens between steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.hpp"

namespace {

thread_local std::string g_last_error;
// The handle whose entry point this thread is running (a HandleScope sets it): its
// failures are also recorded on the handle, where snn_get_info reports them.
thread_local snn_net *g_current = nullptr;
void record_on_handle(const std::string &msg);

int fail(int code, const std::string &msg)
{
    g_last_error = msg;
    record_on_handle(msg);
    return code;
}

#define SNN_CUDA_TRY(expr)                                                                     \
    do {                                                                                       \
        cudaError_t err_ = (expr);                                                             \
        if (err_ != cudaSuccess)                                                               \
            return fail(SNN_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(err_));      \
    } while (0)

}  // namespace

namespace snn {
// Lets other translation units report through snn_last_error.
void set_last_error(const char *msg) { g_last_error = msg; }
}  // namespace snn

struct snn_net {
    snn_spec spec{};
    snn::Constants c{};
    snn::Layout L{};
    snn::StepArgs args{};
    int64_t n = 0, npad = 0, n_syn = 0, n_syn_padded = 0;
    int32_t max_row = 0, chunks_per_row = 1;
    std::vector<int64_t> pop_off;
    std::vector<int32_t> out_degree;
    int format = SNN_RECORD_PLAIN9;
    std::vector<uint8_t> pop_id;
    std::vector<snn::CircuitInfo> circuits;
    int32_t i8_base[SNN_MAX_POPS][SNN_MAX_POPS] = {};
    int32_t i8_step[SNN_MAX_POPS][SNN_MAX_POPS] = {};
    uint8_t *arena = nullptr;
    int device = 0;
    int num_sms = 0;
    int update_grid = 0;
    int deliver_grid = 0;
    int steps_per_graph = 0;
    int engine = SNN_ENGINE_GRAPH;
    int persistent_grid = 0;
    int step_grid = 0;
    cudaStream_t capture_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaEvent_t ev_done = nullptr;
    bool ev_recorded = false;
    int64_t t = 0;
    uint32_t device_error = 0;
    // drained raster, ordered by (step, neuron)
    std::vector<int32_t> hist_t, hist_i;
    int64_t read_pos = 0;
    int64_t events_read = 0;
    int32_t *pin_nrn = nullptr, *pin_t = nullptr;
    int64_t pin_cap = 0;
    // overlapped reads: every snn_step_n ends by copying the device raster cursor into
    // snap_cursor[call mod kSnaps] (pinned) and recording snap_ev there; raster_read is
    // the device raster index up to which spikes are already in the host history
    static constexpr int kSnaps = 4;
    uint32_t *snap_cursor = nullptr;
    cudaEvent_t snap_ev[kSnaps] = {};
    int64_t snap_t[kSnaps] = {};   // steps enqueued at each snapshot
    int64_t n_snaps = 0;           // snapshots recorded
    int64_t snaps_valid_from = 0;  // earlier snapshots predate the last cursor reset
    int64_t raster_read = 0;
    int64_t collected_t = 0;       // spikes of steps below this are in the host history
    cudaStream_t copy_stream = nullptr;
    // batches: circuits per group (0 = one group) and each group's update (graph engine)
    // or step (pipelined engine) arguments and grid; empty when the whole index space
    // runs in one launch
    int32_t circuits_per_group = 0;
    std::vector<snn::StepArgs> group_args;
    std::vector<int> group_grid;
    // pipelined engine: the step grid / delivery warps were set by snn_set_schedule (else
    // each circuit group takes the default for its size)
    bool step_grid_set = false;
    bool delivery_warps_set = false;
    std::string last_error;  // message of this handle's last failed call
};

namespace {

void record_on_handle(const std::string &msg)
{
    if (g_current) g_current->last_error = msg;
}

// Marks the handle an entry point works on, for the length of the call.
struct HandleScope {
    snn_net *prev;
    explicit HandleScope(const snn_net *net) : prev(g_current) { g_current = const_cast<snn_net *>(net); }
    ~HandleScope() { g_current = prev; }
};

}  // namespace

namespace {

// Phase 2 of graph-engine step t_base + k: blocked records have their own kernel.
void launch_phase2(const snn_net *net, int k, cudaStream_t st)
{
    if (snn::is_blocked(net->format)) snn::launch_deliver_blocked(net->args, nullptr, 0, 0, k, st);
    else snn::launch_deliver(net->args, k, net->deliver_grid, st);
}

// Pipelined engine: neuron warps per CTA so that `grid` CTAs cover `quad_warps` groups
// of 128 neurons in as few passes as the CTA allows.
int32_t step_neuron_warps(int64_t quad_warps, int grid)
{
    return static_cast<int32_t>(
        std::min<int64_t>(snn::kStepMaxNeuronWarps, std::max<int64_t>(1, (quad_warps + grid - 1) / grid)));
}

// Neuron range [lo, hi) of every circuit group under `cpg` circuits per group (one
// group, the whole index space, when cpg is 0 or covers every circuit).
std::vector<std::pair<int64_t, int64_t>> group_ranges(const snn_net *net, int cpg)
{
    const int C = static_cast<int>(net->circuits.size());
    if (cpg <= 0 || cpg >= C) return {{0, net->n}};
    std::vector<std::pair<int64_t, int64_t>> r;
    for (int c0 = 0; c0 < C; c0 += cpg) {
        const int c1 = std::min(C, c0 + cpg);
        r.push_back({net->circuits[c0].base, net->circuits[c1 - 1].base + net->circuits[c1 - 1].n});
    }
    return r;
}

// Pipelined engine: arena offset of the four queue counts of group g of `n_groups`
// (the control block's for a single group, else the group's slot of the count array).
uint64_t queue_count_offset(const snn_net *net, size_t g, size_t n_groups)
{
    return n_groups <= 1 ? net->L.ctl + offsetof(snn::Ctl, qcnt) : net->L.qcount + 16 * g;
}

// Batches: consecutive circuits in groups of circuits_per_group, each group updating
// (graph engine) or stepping (pipelined engine) only its own neuron range.  The groups
// are independent, so a run of steps may take them one after another: each group's
// ring and state then stay in L2 for the whole run instead of the whole batch's
// competing for it every step.  Circuits start on multiples of 128 neurons, so a group
// is a whole number of 128-neuron groups.
void build_groups(snn_net *net)
{
    net->group_args.clear();
    net->group_grid.clear();
    const auto ranges = group_ranges(net, net->circuits_per_group);
    if (ranges.size() <= 1) return;
    if (net->engine != SNN_ENGINE_GRAPH && net->engine != SNN_ENGINE_PIPELINED) return;
    for (size_t g = 0; g < ranges.size(); ++g) {
        const int64_t lo = ranges[g].first, hi = ranges[g].second;
        snn::StepArgs a = net->args;
        a.quad_base = lo / 4;
        a.n = hi;
        int grid = snn::update_grid(hi - lo);
        if (net->engine == SNN_ENGINE_PIPELINED) {
            const int64_t qw_end = ((hi + 3) / 4 + 31) / 32;
            const int64_t qw = qw_end - lo / 128;
            grid = net->step_grid_set ? net->step_grid : snn::step_grid(net->num_sms, qw);
            if (!net->delivery_warps_set)
                a.delivery_warps = grid > net->num_sms ? snn::kStepDeliverWarps / 2 : snn::kStepDeliverWarps;
            a.neuron_warps = step_neuron_warps(qw, grid);
            a.quad_warps = static_cast<int32_t>(qw_end);
            a.queue = net->args.queue + lo;
            a.queue_cap = hi - lo;
            a.qcount = reinterpret_cast<uint32_t *>(net->arena + queue_count_offset(net, g, ranges.size()));
            a.group_launch = 1;
        }
        net->group_args.push_back(a);
        net->group_grid.push_back(grid);
    }
}

// Pipelined engine: moves the spikes pending at a step boundary (queue t mod 4) from the
// queue layout of `old_cpg` circuits per group to the current one.  Entries keep their
// content; within a queue their order carries no meaning (a step's raster is ordered on
// the host, ring sums are integer).
int regroup_queue(snn_net *net, int old_cpg)
{
    const auto from = group_ranges(net, old_cpg);
    const auto to = group_ranges(net, net->circuits_per_group);
    const int s = static_cast<int>(net->t & 3);
    const uint64_t qbase = net->L.queue + sizeof(snn::QueueEntry) * (static_cast<uint64_t>(s) * net->npad);
    std::vector<snn::QueueEntry> pending;
    for (size_t g = 0; g < from.size(); ++g) {
        uint32_t cnt = 0;
        SNN_CUDA_TRY(cudaMemcpy(&cnt, net->arena + queue_count_offset(net, g, from.size()) + 4 * s, 4,
                                cudaMemcpyDeviceToHost));
        if (cnt > static_cast<uint64_t>(from[g].second - from[g].first))
            return fail(SNN_ESTATE, "pending spike queue is corrupt");
        const size_t at = pending.size();
        pending.resize(at + cnt);
        if (cnt)
            SNN_CUDA_TRY(cudaMemcpy(pending.data() + at, net->arena + qbase + sizeof(snn::QueueEntry) * from[g].first,
                                    sizeof(snn::QueueEntry) * cnt, cudaMemcpyDeviceToHost));
    }
    for (size_t g = 0; g < to.size(); ++g) {
        std::vector<snn::QueueEntry> mine;
        for (const auto &e : pending)
            if (e.neuron >= to[g].first && e.neuron < to[g].second) mine.push_back(e);
        if (mine.size() > static_cast<uint64_t>(to[g].second - to[g].first))
            return fail(SNN_ESTATE, "pending spike queue is corrupt");
        if (!mine.empty())
            SNN_CUDA_TRY(cudaMemcpy(net->arena + qbase + sizeof(snn::QueueEntry) * to[g].first, mine.data(),
                                    sizeof(snn::QueueEntry) * mine.size(), cudaMemcpyHostToDevice));
        const uint32_t cnt[2] = {static_cast<uint32_t>(mine.size()), 0u};  // queue t mod 4, and the next one
        const uint64_t off = queue_count_offset(net, g, to.size());
        SNN_CUDA_TRY(cudaMemcpy(net->arena + off + 4 * s, &cnt[0], 4, cudaMemcpyHostToDevice));
        SNN_CUDA_TRY(cudaMemcpy(net->arena + off + 4 * ((s + 1) & 3), &cnt[1], 4, cudaMemcpyHostToDevice));
    }
    return SNN_OK;
}

// Graph engine: m steps from the device's t_base, every group in turn, then t_base += m.
void enqueue_graph_steps(snn_net *net, int64_t m, cudaStream_t st)
{
    const size_t G = net->group_args.size();
    for (size_t g = 0; g < std::max<size_t>(G, 1); ++g) {
        const snn::StepArgs &a = G ? net->group_args[g] : net->args;
        const int grid = G ? net->group_grid[g] : net->update_grid;
        for (int64_t k = 0; k < m; ++k) {
            snn::launch_update(a, static_cast<int>(k), grid, st);
            launch_phase2(net, static_cast<int>(k), st);
        }
        if (g + 1 < G) snn::launch_resync(net->args.ctl, st);
    }
    snn::launch_advance(net->args.ctl, m, st);
}

// Pipelined engine: m step kernels from step t0 (the device's t_base), every circuit
// group in turn, then t_base += m.  Consecutive kernels of a group may overlap their
// launch with the previous one (programmatic edges, inside a captured graph); a group's
// first kernel follows the previous group's resync in plain stream order.
int enqueue_pipelined_steps(snn_net *net, int64_t m, cudaStream_t st, int64_t t0, bool programmatic)
{
    const size_t G = net->group_args.size();
    for (size_t g = 0; g < std::max<size_t>(G, 1); ++g) {
        const snn::StepArgs &a = G ? net->group_args[g] : net->args;
        const int grid = G ? net->group_grid[g] : net->step_grid;
        for (int64_t k = 0; k < m; ++k) {
            const int ph = static_cast<int>((t0 + k) % snn::kPhasePeriod);
            const int e = snn::launch_step(a, static_cast<int>(k), ph, grid, st, programmatic && k > 0);
            if (e != 0) return fail(SNN_ECUDA, std::string("step launch: ") + cudaGetErrorString(static_cast<cudaError_t>(e)));
        }
        if (g + 1 < G) snn::launch_resync(net->args.ctl, st);
    }
    snn::launch_advance(net->args.ctl, m, st);
    return SNN_OK;
}

// m steps launched one by one, starting at step t0 (the device counter t_base equals t0).
int launch_steps_direct(snn_net *net, int64_t m, cudaStream_t st, int64_t t0)
{
    if (net->engine == SNN_ENGINE_PIPELINED) {
        const int rc = enqueue_pipelined_steps(net, m, st, t0, false);
        if (rc) return rc;
    } else {
        enqueue_graph_steps(net, m, st);
    }
    SNN_CUDA_TRY(cudaGetLastError());
    return SNN_OK;
}

int launch_steps_persistent(snn_net *net, int64_t n, cudaStream_t st)
{
    while (n > 0) {
        const int64_t m = std::min<int64_t>(n, snn::kMaxPersistentSteps);
        SNN_CUDA_TRY(cudaMemsetAsync(net->arena + net->L.ctl + offsetof(snn::Ctl, bar), 0, sizeof(uint32_t), st));
        const int e = snn::launch_persistent(net->args, m, net->persistent_grid, st);
        if (e != 0)
            return fail(SNN_ECUDA, std::string("cooperative launch: ") + cudaGetErrorString(static_cast<cudaError_t>(e)));
        n -= m;
    }
    return SNN_OK;
}

// Resident engine: every call's steps in cooperative launches of at most
// kResidentMaxSteps steps; each launch reads the step counter and the raster cursor
// from the control block at its start and writes them back at its end.  Mailbox words
// are tagged with the step's rank in its launch, so the mailboxes are zeroed first.
int launch_steps_resident(snn_net *net, int64_t n, cudaStream_t st)
{
    const uint64_t B = net->args.n_blocks;
    const uint64_t mbox_bytes = 4 * 4 * B * snn::kResidentMboxWords;
    const uint64_t inbox_bytes = 4 * 4 * B * B * snn::kResidentSlotWords;
    while (n > 0) {
        const int64_t m = std::min<int64_t>(n, snn::kResidentMaxSteps);
        SNN_CUDA_TRY(cudaMemsetAsync(net->arena + net->L.mbox, 0, mbox_bytes, st));
        SNN_CUDA_TRY(cudaMemsetAsync(net->arena + net->L.inbox, 0, inbox_bytes, st));
        const int e = snn::launch_resident(net->args, m, st);
        if (e != 0)
            return fail(SNN_ECUDA, std::string("cooperative launch: ") + cudaGetErrorString(static_cast<cudaError_t>(e)));
        n -= m;
    }
    return SNN_OK;
}

int capture_graph(snn_net *net)
{
    SNN_CUDA_TRY(cudaStreamCreateWithFlags(&net->capture_stream, cudaStreamNonBlocking));
    SNN_CUDA_TRY(cudaStreamBeginCapture(net->capture_stream, cudaStreamCaptureModeThreadLocal));
    if (net->engine == SNN_ENGINE_PIPELINED) {
        // replays start on a multiple of the phase period (see snn_step_n)
        const int rc = enqueue_pipelined_steps(net, net->steps_per_graph, net->capture_stream, 0, true);
        if (rc != SNN_OK) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(net->capture_stream, &g);
            if (g) cudaGraphDestroy(g);
            return rc;
        }
    } else {
        enqueue_graph_steps(net, net->steps_per_graph, net->capture_stream);
    }
    cudaError_t launch_err = cudaGetLastError();
    cudaGraph_t g = nullptr;
    cudaError_t end_err = cudaStreamEndCapture(net->capture_stream, &g);
    if (launch_err != cudaSuccess) return fail(SNN_ECUDA, std::string("capture: ") + cudaGetErrorString(launch_err));
    if (end_err != cudaSuccess) return fail(SNN_ECUDA, std::string("end capture: ") + cudaGetErrorString(end_err));
    net->graph = g;
    SNN_CUDA_TRY(cudaGraphInstantiate(&net->graph_exec, net->graph, 0));
    return SNN_OK;
}

// Replaces the captured step graph after a schedule change.
int recapture(snn_net *net)
{
    if (net->graph_exec) cudaGraphExecDestroy(net->graph_exec);
    if (net->graph) cudaGraphDestroy(net->graph);
    if (net->capture_stream) cudaStreamDestroy(net->capture_stream);
    net->graph_exec = nullptr;
    net->graph = nullptr;
    net->capture_stream = nullptr;
    return capture_graph(net);
}

int wait_done(snn_net *net)
{
    if (net->ev_recorded) SNN_CUDA_TRY(cudaEventSynchronize(net->ev_done));
    return SNN_OK;
}

// Raster entries [lo, hi) of the device raster into the host history, ordered by
// (step, neuron), through the handle's copy stream (the steps that wrote them are done).
int append_raster(snn_net *net, int64_t lo, int64_t hi)
{
    const int64_t cnt = hi - lo;
    if (cnt <= 0) return SNN_OK;
    if (cnt > net->pin_cap) {
        if (net->pin_nrn) cudaFreeHost(net->pin_nrn);
        if (net->pin_t) cudaFreeHost(net->pin_t);
        net->pin_nrn = net->pin_t = nullptr;
        net->pin_cap = 0;
        const int64_t want = std::max<int64_t>(cnt, 1 << 16);
        SNN_CUDA_TRY(cudaMallocHost(&net->pin_nrn, sizeof(int32_t) * want));
        SNN_CUDA_TRY(cudaMallocHost(&net->pin_t, sizeof(int32_t) * want));
        net->pin_cap = want;
    }
    const int32_t *dn = reinterpret_cast<const int32_t *>(net->arena + net->L.rast_nrn) + lo;
    const int32_t *dt = reinterpret_cast<const int32_t *>(net->arena + net->L.rast_t) + lo;
    SNN_CUDA_TRY(cudaMemcpyAsync(net->pin_nrn, dn, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost, net->copy_stream));
    SNN_CUDA_TRY(cudaMemcpyAsync(net->pin_t, dt, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost, net->copy_stream));
    SNN_CUDA_TRY(cudaStreamSynchronize(net->copy_stream));
    std::vector<int64_t> key(cnt);
    bool steps_in_order = true;
    for (int64_t j = 0; j < cnt; ++j) {
        key[j] = (static_cast<int64_t>(net->pin_t[j]) << 32) | static_cast<uint32_t>(net->pin_nrn[j]);
        if (j > 0 && net->pin_t[j] < net->pin_t[j - 1]) steps_in_order = false;
    }
    if (steps_in_order) {
        // one step's spikes are contiguous (a few dozen at full scale): order each run
        for (int64_t r0 = 0; r0 < cnt;) {
            int64_t r1 = r0 + 1;
            while (r1 < cnt && net->pin_t[r1] == net->pin_t[r0]) ++r1;
            if (r1 - r0 > 64) {
                std::sort(key.begin() + r0, key.begin() + r1);
            } else {
                for (int64_t j = r0 + 1; j < r1; ++j) {
                    const int64_t v = key[j];
                    int64_t m = j;
                    while (m > r0 && key[m - 1] > v) {
                        key[m] = key[m - 1];
                        --m;
                    }
                    key[m] = v;
                }
            }
            r0 = r1;
        }
    } else {
        std::sort(key.begin(), key.end());  // circuit groups write runs of steps group by group
    }
    // the range covers whole steps after every step already in the history (a snapshot
    // ends an snn_step_n call), so appending keeps the history ordered
    const size_t base = net->hist_t.size();
    net->hist_t.resize(base + cnt);
    net->hist_i.resize(base + cnt);
    for (int64_t j = 0; j < cnt; ++j) {
        net->hist_t[base + j] = static_cast<int32_t>(key[j] >> 32);
        const int32_t i = static_cast<int32_t>(key[j] & 0xFFFFFFFFll);
        net->hist_i[base + j] = i;
        net->events_read += net->out_degree[i];
    }
    return SNN_OK;
}

// Waits for every enqueued step, moves the rest of the device raster to the host
// history and resets the device cursor.
int drain(snn_net *net)
{
    int rc = wait_done(net);
    if (rc) return rc;
    snn::Ctl ctl;
    SNN_CUDA_TRY(cudaMemcpy(&ctl, net->arena + net->L.ctl, sizeof(ctl), cudaMemcpyDeviceToHost));
    net->device_error |= ctl.err;
    const int64_t cnt = std::min<int64_t>(ctl.cursor, net->L.rast_cap);
    rc = append_raster(net, std::min(net->raster_read, cnt), cnt);
    if (rc) return rc;
    if (ctl.cursor != 0) {
        uint32_t zero[3] = {0, 0, 0};  // cursor, step_begin[0], step_begin[1]
        SNN_CUDA_TRY(cudaMemcpy(net->arena + net->L.ctl + offsetof(snn::Ctl, cursor), zero, sizeof(zero),
                                cudaMemcpyHostToDevice));
    }
    net->raster_read = 0;
    net->snaps_valid_from = net->n_snaps;  // their cursors refer to the raster before the reset
    net->collected_t = net->t;
    if (net->device_error & snn::kErrTimeout)
        return fail(SNN_ETIMEOUT, "a bounded device wait (persistent barrier or resident mailbox) timed out");
    if (net->device_error & snn::kErrRaster)
        return fail(SNN_EOVERFLOW, "device raster filled before it was read; raise raster_capacity");
    return SNN_OK;
}

// Moves the spikes of the calls before the latest snn_step_n into the host history
// without waiting for the latest call.  Falls back to drain() when the device raster is
// more than a quarter full: the cursor is only reset while the device is idle, and up to
// two more calls' spikes are written before the next chance.
int collect(snn_net *net)
{
    const int64_t j = net->n_snaps - 2;
    if (j < 0 || j < net->snaps_valid_from) return SNN_OK;
    const int slot = static_cast<int>(j % snn_net::kSnaps);
    SNN_CUDA_TRY(cudaEventSynchronize(net->snap_ev[slot]));
    const int64_t cur = net->snap_cursor[slot];
    if (cur > net->L.rast_cap / 4) return drain(net);
    const int rc = append_raster(net, net->raster_read, std::max(net->raster_read, cur));
    if (rc) return rc;
    net->raster_read = std::max(net->raster_read, cur);
    net->collected_t = std::max(net->collected_t, net->snap_t[slot]);
    return SNN_OK;
}

}  // namespace

extern "C" {

const char *snn_strerror(int code)
{
    switch (code) {
    case SNN_OK: return "ok";
    case SNN_EINVAL: return "invalid argument";
    case SNN_ENOMEM: return "out of memory";
    case SNN_ECUDA: return "CUDA error";
    case SNN_EOVERFLOW: return "raster overflow";
    case SNN_ETIMEOUT: return "device wait timed out";
    case SNN_ESTATE: return "invalid state";
    case SNN_ENOTSUP: return "not supported";
    default: return "unknown status";
    }
}

const char *snn_last_error(void) { return g_last_error.c_str(); }

int snn_query_sizes(const snn_spec *spec, snn_sizes *out)
{
    if (!spec || !out) return fail(SNN_EINVAL, "null argument");
    try {
        std::string why;
        if (!snn::validate_spec(*spec, why)) return fail(SNN_EINVAL, why);
        const snn::Layout L = snn::make_layout(*spec);
        out->arena_bytes = L.total;
        out->n_neurons = snn::count_neurons(*spec);
        out->n_neurons_padded = L.npad;
        out->n_synapses = snn::count_synapses(*spec);
        out->n_synapses_padded_max = L.syn_padded_max;
        out->raster_capacity = L.rast_cap;
    } catch (const std::bad_alloc &) {
        return fail(SNN_ENOMEM, "host allocation failed");
    }
    return SNN_OK;
}

int snn_export_network(const snn_spec *spec, int64_t *row_ptr, int32_t *post, int32_t *w_fx, uint8_t *delay,
                       float *u0)
{
    if (!spec) return fail(SNN_EINVAL, "null argument");
    std::string why;
    if (!snn::validate_spec(*spec, why)) return fail(SNN_EINVAL, why);
    const int fmt = spec->record_format;
    if (fmt != SNN_RECORD_PLAIN9 && fmt != SNN_RECORD_PACKED_I8 && fmt != SNN_RECORD_PACKED_BF16)
        return fail(SNN_EINVAL, "export takes plain or packed records");
    try {
        snn::Constants c;
        snn::compute_constants(spec->model, c);
        snn::HostNetwork hn;
        if (!snn::build_host_network(*spec, c, hn, why)) return fail(SNN_EINVAL, why);
        // the caller sized the arrays by snn_query_sizes
        int64_t real = 0;
        for (int64_t i = 0; i < hn.n; ++i) real += hn.out_degree[i];
        if (hn.n != snn::count_neurons(*spec) || hn.n_syn != snn::count_synapses(*spec) || real != hn.n_syn)
            return fail(SNN_EINVAL, "built network disagrees with snn_query_sizes");
        // the padded rows of the indexed store keep their real synapses first
        int64_t k = 0;
        if (row_ptr) row_ptr[0] = 0;
        for (int64_t i = 0; i < hn.n; ++i) {
            const int64_t a = hn.row_ptr[i];
            const int64_t len = hn.out_degree[i];
            if (fmt == SNN_RECORD_PLAIN9) {
                if (post) std::memcpy(post + k, hn.tgt.data() + a, sizeof(int32_t) * len);
                if (w_fx) std::memcpy(w_fx + k, hn.w.data() + a, sizeof(int32_t) * len);
                if (delay) std::memcpy(delay + k, hn.d.data() + a, len);
            } else {
                // packed records: the fields of each word and the weight the kernels read back
                const int src = hn.pop_id[i];
                for (int64_t j = 0; j < len; ++j) {
                    const uint32_t word = hn.word[a + j];
                    if (post) post[k + j] = static_cast<int32_t>(word & snn::kWordTargetMask);
                    if (delay) delay[k + j] = static_cast<uint8_t>((word >> snn::kWordDelayShift) & 63u);
                    if (!w_fx) continue;
                    if (fmt == SNN_RECORD_PACKED_I8) {
                        const int tgt = static_cast<int>((word >> snn::kWordPopShift) & 7u);
                        const int8_t code = static_cast<int8_t>(hn.wbytes[a + j]);
                        w_fx[k + j] = hn.i8_base[src][tgt] + static_cast<int32_t>(code) * hn.i8_step[src][tgt];
                    } else {
                        uint16_t h;
                        std::memcpy(&h, &hn.wbytes[2 * (a + j)], 2);
                        const uint32_t bits = static_cast<uint32_t>(h) << 16;
                        float f;
                        std::memcpy(&f, &bits, 4);
                        w_fx[k + j] = static_cast<int32_t>(std::lrintf(f * 4096.0f));  // nearest, ties to even
                    }
                }
            }
            k += len;
            if (row_ptr) row_ptr[i + 1] = k;
        }
        if (u0) std::memcpy(u0, hn.u0.data(), sizeof(float) * hn.n);
    } catch (const std::bad_alloc &) {
        return fail(SNN_ENOMEM, "host allocation failed while building the network");
    }
    return SNN_OK;
}

int snn_build_network(const snn_spec *spec, void *dev_arena, uint64_t arena_bytes, void *cuda_stream,
                      snn_net **out)
{
    if (!spec || !out || !dev_arena) return fail(SNN_EINVAL, "null argument");
    *out = nullptr;
    if (reinterpret_cast<uintptr_t>(dev_arena) % 256 != 0) return fail(SNN_EINVAL, "arena not 256-byte aligned");
    std::string why;
    if (!snn::validate_spec(*spec, why)) return fail(SNN_EINVAL, why);
    cudaPointerAttributes attr;
    SNN_CUDA_TRY(cudaPointerGetAttributes(&attr, dev_arena));
    if (attr.type != cudaMemoryTypeDevice) return fail(SNN_EINVAL, "arena is not device memory");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    snn_net *net = nullptr;
    try {
        net = new snn_net();
        net->spec = *spec;
        net->spec.custom = nullptr;
        net->spec.circuits = nullptr;
        net->L = snn::make_layout(*spec);
        if (arena_bytes < net->L.total) {
            delete net;
            return fail(SNN_ENOMEM, "arena smaller than snn_query_sizes().arena_bytes");
        }
        snn::compute_constants(spec->model, net->c);
        snn::HostNetwork hn;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, attr.device) != cudaSuccess) sms = 0;
        if (!snn::build_host_network(*spec, net->c, hn, why, sms)) {
            delete net;
            return fail(SNN_EINVAL, why);
        }
        net->arena = static_cast<uint8_t *>(dev_arena);
        net->device = attr.device;
        net->n = hn.n;
        net->npad = hn.npad;
        net->n_syn = hn.n_syn;
        net->n_syn_padded = hn.n_syn_padded;
        net->max_row = hn.max_row;
        net->chunks_per_row = std::max(1, (hn.max_row + snn::kChunk - 1) / snn::kChunk);
        net->pop_off = hn.pop_off;
        net->out_degree = std::move(hn.out_degree);
        net->format = hn.format;
        net->circuits = hn.circuits;
        std::memcpy(net->i8_base, hn.i8_base, sizeof(net->i8_base));
        std::memcpy(net->i8_step, hn.i8_step, sizeof(net->i8_step));

        int rc = SNN_OK;
        auto cuda_ok = [&](cudaError_t e, const char *what) {
            if (e != cudaSuccess && rc == SNN_OK) rc = fail(SNN_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
            return e == cudaSuccess;
        };
        cuda_ok(cudaSetDevice(net->device), "cudaSetDevice");
        cuda_ok(cudaDeviceGetAttribute(&net->num_sms, cudaDevAttrMultiProcessorCount, net->device), "attr");
        uint8_t *A = net->arena;
        const snn::Layout &L = net->L;
        snn::StaticTables tabs{};
        std::memcpy(tabs.thresholds, net->c.thresholds, sizeof(tabs.thresholds));
        for (int b = 0; b <= SNN_MAX_POPS; ++b) tabs.pop_off[b] = b < (int)hn.pop_off.size() ? hn.pop_off[b] : hn.n;
        tabs.n_pops = spec->model.n_pops;
        for (int sa = 0; sa < SNN_MAX_POPS; ++sa)
            for (int tb = 0; tb < SNN_MAX_POPS; ++tb) tabs.i8_pair[sa][tb] = {hn.i8_base[sa][tb], hn.i8_step[sa][tb]};
        std::vector<float> u0(net->npad, 0.0f);
        std::copy(hn.u0.begin(), hn.u0.end(), u0.begin());
        std::vector<uint8_t> pop_dev(net->npad, 0);
        std::copy(hn.pop_id.begin(), hn.pop_id.end(), pop_dev.begin());
        std::vector<int32_t> group_circuit(net->npad / 128 + 1, 0);
        for (size_t g = 0, ci = 0; g < group_circuit.size(); ++g) {
            while (ci + 1 < hn.circuits.size() && static_cast<int64_t>(g) * 128 >= hn.circuits[ci + 1].base) ++ci;
            group_circuit[g] = static_cast<int32_t>(ci);
        }
        cuda_ok(cudaMemcpyAsync(A + L.pop_id, pop_dev.data(), net->npad, cudaMemcpyHostToDevice, st), "pop_id");
        cuda_ok(cudaMemcpyAsync(A + L.group_circuit, group_circuit.data(), 4 * group_circuit.size(),
                                cudaMemcpyHostToDevice, st), "group_circuit");
        cuda_ok(cudaMemcpyAsync(A + L.circuits, hn.circuits.data(), sizeof(snn::CircuitInfo) * hn.circuits.size(),
                                cudaMemcpyHostToDevice, st), "circuits");
        net->pop_id = std::move(pop_dev);
        cuda_ok(cudaMemsetAsync(A + L.ctl, 0, sizeof(snn::Ctl), st), "memset ctl");
        cuda_ok(cudaMemcpyAsync(A + L.tables, &tabs, sizeof(tabs), cudaMemcpyHostToDevice, st), "tables");
        cuda_ok(cudaMemcpyAsync(A + L.U, u0.data(), 4 * net->npad, cudaMemcpyHostToDevice, st), "U");
        cuda_ok(cudaMemsetAsync(A + L.I, 0, 4 * net->npad, st), "I");
        cuda_ok(cudaMemsetAsync(A + L.R, 0, net->npad, st), "R");
        cuda_ok(cudaMemsetAsync(A + L.ring, 0, uint64_t{4} * snn::kDMax * net->npad, st), "ring");
        cuda_ok(cudaMemcpyAsync(A + L.row_ptr, hn.row_ptr.data(), 8 * (net->n + 1), cudaMemcpyHostToDevice, st),
                "row_ptr");
        if (net->n_syn_padded > 0 && hn.format == SNN_RECORD_PLAIN9) {
            cuda_ok(cudaMemcpyAsync(A + L.syn_tgt, hn.tgt.data(), 4 * net->n_syn_padded, cudaMemcpyHostToDevice, st),
                    "tgt");
            cuda_ok(cudaMemcpyAsync(A + L.syn_w, hn.w.data(), 4 * net->n_syn_padded, cudaMemcpyHostToDevice, st), "w");
            cuda_ok(cudaMemcpyAsync(A + L.syn_d, hn.d.data(), net->n_syn_padded, cudaMemcpyHostToDevice, st), "d");
        } else if (hn.format == SNN_RECORD_BLOCKED4 || hn.format == SNN_RECORD_BLOCKED8) {
            if (net->n_syn_padded > 0)
                cuda_ok(cudaMemcpyAsync(A + L.syn_tgt, hn.word.data(), 4 * hn.word.size(), cudaMemcpyHostToDevice, st),
                        "record quads");
            cuda_ok(cudaMemcpyAsync(A + L.syn_d, hn.seg.data(), 2 * hn.seg.size(), cudaMemcpyHostToDevice, st),
                    "block table");
            cuda_ok(cudaMemcpyAsync(A + L.blocks, hn.blk.data(), 4 * hn.blk.size(), cudaMemcpyHostToDevice, st),
                    "blocks");
        } else if (hn.format == SNN_RECORD_BLOCKED6) {
            if (net->n_syn_padded > 0) {
                cuda_ok(cudaMemcpyAsync(A + L.syn_tgt, hn.rec16.data(), 2 * net->n_syn_padded, cudaMemcpyHostToDevice,
                                        st),
                        "records");
                cuda_ok(cudaMemcpyAsync(A + L.syn_w, hn.w.data(), 4 * net->n_syn_padded, cudaMemcpyHostToDevice, st),
                        "w");
            }
            cuda_ok(cudaMemcpyAsync(A + L.syn_d, hn.seg.data(), 2 * hn.seg.size(), cudaMemcpyHostToDevice, st),
                    "block table");
            cuda_ok(cudaMemcpyAsync(A + L.blocks, hn.blk.data(), 4 * hn.blk.size(), cudaMemcpyHostToDevice, st),
                    "blocks");
        } else if (net->n_syn_padded > 0) {
            cuda_ok(cudaMemcpyAsync(A + L.syn_tgt, hn.word.data(), 4 * net->n_syn_padded, cudaMemcpyHostToDevice, st),
                    "words");
            cuda_ok(cudaMemcpyAsync(A + L.syn_w, hn.wbytes.data(), hn.wbytes.size(), cudaMemcpyHostToDevice, st),
                    "weights");
        }
        cuda_ok(cudaStreamSynchronize(st), "upload sync");
        if (rc != SNN_OK) {
            delete net;
            return rc;
        }

        snn::StepArgs &a = net->args;
        a.ctl = reinterpret_cast<snn::Ctl *>(A + L.ctl);
        a.tables = reinterpret_cast<const snn::StaticTables *>(A + L.tables);
        a.U = reinterpret_cast<float *>(A + L.U);
        a.I = reinterpret_cast<float *>(A + L.I);
        a.R = A + L.R;
        a.ring = reinterpret_cast<int32_t *>(A + L.ring);
        a.row_ptr = reinterpret_cast<const int64_t *>(A + L.row_ptr);
        a.syn_tgt = reinterpret_cast<const int32_t *>(A + L.syn_tgt);
        a.syn_w = reinterpret_cast<const int32_t *>(A + L.syn_w);
        a.syn_d = A + L.syn_d;
        a.rast_nrn = reinterpret_cast<int32_t *>(A + L.rast_nrn);
        a.rast_t = reinterpret_cast<int32_t *>(A + L.rast_t);
        a.n = net->n;
        a.npad = net->npad;
        a.seed = spec->seed;
        a.rast_cap = static_cast<uint32_t>(L.rast_cap);
        a.chunks_per_row = net->chunks_per_row;
        a.format = net->format;
        a.n_circuits = static_cast<int32_t>(net->circuits.size());
        a.pop_id = A + L.pop_id;
        a.group_circuit = reinterpret_cast<const int32_t *>(A + L.group_circuit);
        a.circuits = reinterpret_cast<const snn::CircuitInfo *>(A + L.circuits);
        a.blk_rec = reinterpret_cast<const uint16_t *>(A + L.syn_tgt);
        a.blk_seg = reinterpret_cast<const uint16_t *>(A + L.syn_d);
        a.blk_off = reinterpret_cast<const int32_t *>(A + L.blocks);
        a.n_blocks = snn::is_blocked(hn.format) ? static_cast<int32_t>(hn.blk.size()) - 1 : 0;
        a.p11 = net->c.p11f;
        a.p21 = net->c.p21f;
        a.p22 = net->c.p22f;
        a.theta = net->c.theta;
        a.u_reset = net->c.u_reset;
        a.t_ref = net->c.t_ref;
        a.w_ext_fx = net->c.w_ext_fx;
        for (int b = 0; b <= SNN_MAX_POPS; ++b) a.pop_off[b] = tabs.pop_off[b];
        a.n_pops = spec->model.n_pops;
        a.barrier_timeout_ns = snn::kBarrierTimeoutNs;
        a.barrier_extra = 0;
        // Fault injection for tests of the bounded barrier wait: with SNN_FAULT=barrier_stall
        // in the environment at build time, every barrier expects one arrival that never
        // comes and gives up after 20 ms, so the run must end with SNN_ETIMEOUT.
        if (const char *f = std::getenv("SNN_FAULT")) {
            if (std::string(f) == "barrier_stall") {
                a.barrier_extra = 1;
                a.barrier_timeout_ns = 20000000ull;
            }
        }
        net->update_grid = snn::update_grid(net->n);
        net->deliver_grid = spec->deliver_blocks > 0 ? spec->deliver_blocks : 2 * net->num_sms;
        net->steps_per_graph = spec->steps_per_graph > 0 ? spec->steps_per_graph : 1000;
        net->engine = spec->engine != SNN_ENGINE_DEFAULT     ? spec->engine
                      : snn::is_blocked(net->format)       ? SNN_ENGINE_GRAPH
                                                           : SNN_ENGINE_PIPELINED;
        if (snn::is_blocked(net->format) && snn::prepare_blocked_kernel() != 0) {
            snn_destroy(net);
            return fail(SNN_ECUDA, "shared memory opt-in of the blocked delivery kernel failed");
        }
        if (net->engine == SNN_ENGINE_PIPELINED || net->engine == SNN_ENGINE_PERSISTENT) {
            // the persistent engine runs the pipelined schedule on the same state
            // state "after 0 steps" is buffer 1; the first kernel decides step 0's spikes
            const int64_t quad_warps = ((net->n + 3) / 4 + 31) / 32;
            net->step_grid = snn::step_grid(net->num_sms, quad_warps);
            a.neuron_warps = step_neuron_warps(quad_warps, net->step_grid);
            // a larger grid brings more delivery warps already: fewer per CTA
            a.delivery_warps = net->step_grid > net->num_sms ? snn::kStepDeliverWarps / 2 : snn::kStepDeliverWarps;
            a.U2 = reinterpret_cast<float *>(A + L.U2);
            a.R2 = A + L.R2;
            a.queue = reinterpret_cast<snn::QueueEntry *>(A + L.queue);
            a.quad_warps = static_cast<int32_t>(quad_warps);
            a.qcount = reinterpret_cast<uint32_t *>(A + L.ctl + offsetof(snn::Ctl, qcnt));
            a.queue_cap = net->npad;
            if (snn::prepare_step_kernel(a) != 0) {
                snn_destroy(net);
                return fail(SNN_ENOTSUP, "network too large for the pipelined engine's shared memory");
            }
            cuda_ok(cudaMemsetAsync(A + L.qcount, 0, 4 * 4 * (net->npad / 128 + 1), st), "qcount");
            cuda_ok(cudaMemcpyAsync(A + L.U2, u0.data(), 4 * net->npad, cudaMemcpyHostToDevice, st), "U2");
            cuda_ok(cudaMemsetAsync(A + L.R2, 0, net->npad, st), "R2");
            cuda_ok(cudaMemsetAsync(A + L.queue, 0xFF, 4 * sizeof(snn::QueueEntry) * net->npad, st), "queue");
            // a graph holds a whole number of phase periods
            net->steps_per_graph = std::max(snn::kPhasePeriod,
                                            (spec->steps_per_graph > 0 ? spec->steps_per_graph : 1024) /
                                                snn::kPhasePeriod * snn::kPhasePeriod);
            snn::launch_prime(a, net->step_grid, st);
            cuda_ok(cudaGetLastError(), "prime launch");
            cuda_ok(cudaStreamSynchronize(st), "prime");
            if (rc != SNN_OK) {
                snn_destroy(net);
                return rc;
            }
        }
        if (net->engine == SNN_ENGINE_RESIDENT) {
            const int64_t width = snn::resident_width(net->n, net->num_sms);
            const int B = static_cast<int>(hn.blk.size()) - 1;
            int coop = 0;
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, net->device);
            if (width == 0 || B < 1 || B > net->num_sms) {
                snn_destroy(net);
                return fail(SNN_ENOTSUP, "network too large for the resident engine (1024 neurons per SM)");
            }
            a.n_blocks = B;
            a.blk_off = reinterpret_cast<const int32_t *>(A + L.blocks);
            const snn::ResTables T = snn::resident_tables(net->n, B);
            a.res_rbase = reinterpret_cast<const int64_t *>(A + L.seg + T.rbase);
            a.res_coarse = reinterpret_cast<const uint32_t *>(A + L.seg + T.coarse);
            a.res_lens = A + L.seg + T.lens;
            a.res_offt = reinterpret_cast<const uint32_t *>(A + L.seg + T.offt);
            a.res_lens_stride = static_cast<int32_t>(T.lens_stride);
            a.res_coarse_stride = static_cast<int32_t>(T.coarse_stride);
            a.mbox = reinterpret_cast<uint32_t *>(A + L.mbox);
            a.inbox = reinterpret_cast<uint32_t *>(A + L.inbox);
            a.res_stride = static_cast<int32_t>(width);
            a.res_rows = snn::resident_rows(static_cast<int>(width), spec->smem_ring_rows, net->n);
            a.neuron_warps = static_cast<int32_t>((width + 127) / 128);
            // two delivery teams, each with a lane per mailbox, and up to kResidentTeamWarps
            // warps each where the CTA has room (more warps share a step's synapse loads)
            const int need = 2 * ((B + 31) / 32);
            a.delivery_warps = std::max(need, std::min(2 * snn::kResidentTeamWarps,
                                                       (snn::kResidentMaxWarps - a.neuron_warps) & ~1));
            if (a.neuron_warps + a.delivery_warps > snn::kResidentMaxWarps) {
                snn_destroy(net);
                return fail(SNN_ENOTSUP, "the resident engine's CTA would exceed its warp limit for this network");
            }
            cuda_ok(cudaMemcpyAsync(A + L.seg, hn.restab.data(), hn.restab.size(), cudaMemcpyHostToDevice, st),
                    "block tables");
            if (!hn.rec8.empty())
                cuda_ok(cudaMemcpyAsync(A + L.res_rec, hn.rec8.data(), 8 * hn.rec8.size(), cudaMemcpyHostToDevice, st),
                        "block-major records");
            a.res_rec = A + L.res_rec;
            cuda_ok(cudaMemcpyAsync(A + L.blocks, hn.blk.data(), 4 * hn.blk.size(), cudaMemcpyHostToDevice, st),
                    "blocks");
            cuda_ok(cudaStreamSynchronize(st), "resident upload");
            if (rc != SNN_OK) {
                snn_destroy(net);
                return rc;
            }
            if (a.res_rows == 0 || !coop || snn::prepare_resident_kernel(a) != 0 ||
                snn::resident_blocks_per_sm(a) < 1) {
                snn_destroy(net);
                return fail(SNN_ENOTSUP, "the resident engine's cooperative launch does not fit this GPU");
            }
            net->steps_per_graph = spec->steps_per_graph > 0 ? spec->steps_per_graph : 1024;
        }
        if (net->engine == SNN_ENGINE_PERSISTENT) {
            // every CTA of the cooperative launch must be resident at once
            int coop = 0;
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, net->device);
            const int per_sm = coop ? snn::persistent_blocks_per_sm(a) : 0;
            if (per_sm < 1) {
                snn_destroy(net);
                return fail(SNN_ENOTSUP, "cooperative launch of the persistent engine is not available");
            }
            net->persistent_grid = std::min(net->step_grid, per_sm * net->num_sms);
            net->step_grid = net->persistent_grid;
            a.neuron_warps = step_neuron_warps(a.quad_warps, net->persistent_grid);
            if (snn::persistent_blocks_per_sm(a) * net->num_sms < net->persistent_grid) {
                snn_destroy(net);
                return fail(SNN_ENOTSUP, "the persistent engine's grid does not fit on the GPU at once");
            }
        }
        rc = (net->engine == SNN_ENGINE_GRAPH || net->engine == SNN_ENGINE_PIPELINED) ? capture_graph(net) : SNN_OK;
        if (rc == SNN_OK && cudaEventCreateWithFlags(&net->ev_done, cudaEventDisableTiming) != cudaSuccess)
            rc = fail(SNN_ECUDA, "event create");
        for (int k = 0; k < snn_net::kSnaps && rc == SNN_OK; ++k)
            if (cudaEventCreateWithFlags(&net->snap_ev[k], cudaEventDisableTiming) != cudaSuccess)
                rc = fail(SNN_ECUDA, "event create");
        if (rc == SNN_OK && cudaMallocHost(&net->snap_cursor, sizeof(uint32_t) * snn_net::kSnaps) != cudaSuccess)
            rc = fail(SNN_ECUDA, "pinned snapshot slots");
        if (rc == SNN_OK && cudaStreamCreateWithFlags(&net->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
            rc = fail(SNN_ECUDA, "copy stream");
        if (rc != SNN_OK) {
            snn_destroy(net);
            return rc;
        }
    } catch (const std::bad_alloc &) {
        delete net;
        return fail(SNN_ENOMEM, "host allocation failed while building the network");
    }
    *out = net;
    return SNN_OK;
}

int snn_step_n(snn_net *net, int64_t n_steps, void *cuda_stream)
{
    HandleScope scope(net);
    if (!net) return fail(SNN_EINVAL, "null network");
    if (n_steps < 0) return fail(SNN_EINVAL, "n_steps < 0");
    if (net->device_error) return fail(SNN_ESTATE, "a previous device error is pending");
    if (n_steps == 0) return SNN_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (net->engine == SNN_ENGINE_PERSISTENT || net->engine == SNN_ENGINE_RESIDENT) {
        const int rc = net->engine == SNN_ENGINE_RESIDENT ? launch_steps_resident(net, n_steps, st)
                                                          : launch_steps_persistent(net, n_steps, st);
        if (rc) return rc;
    } else {
        int64_t t = net->t, n = n_steps;
        if (net->engine == SNN_ENGINE_PIPELINED) {
            // single steps up to the next multiple of the phase period, where graphs start
            const int64_t head = std::min<int64_t>(n, (snn::kPhasePeriod - t % snn::kPhasePeriod) % snn::kPhasePeriod);
            if (head > 0) {
                const int rc = launch_steps_direct(net, head, st, t);
                if (rc) return rc;
                t += head;
                n -= head;
            }
        }
        for (; n >= net->steps_per_graph; n -= net->steps_per_graph, t += net->steps_per_graph)
            SNN_CUDA_TRY(cudaGraphLaunch(net->graph_exec, st));
        if (n > 0) {
            const int rc = launch_steps_direct(net, n, st, t);
            if (rc) return rc;
        }
    }
    SNN_CUDA_TRY(cudaEventRecord(net->ev_done, st));
    net->ev_recorded = true;
    net->t += n_steps;
    // where the raster ends after these steps, for snn_collect_spikes
    const int slot = static_cast<int>(net->n_snaps % snn_net::kSnaps);
    SNN_CUDA_TRY(cudaMemcpyAsync(net->snap_cursor + slot, net->arena + net->L.ctl + offsetof(snn::Ctl, cursor),
                                 sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    SNN_CUDA_TRY(cudaEventRecord(net->snap_ev[slot], st));
    net->snap_t[slot] = net->t;
    net->n_snaps += 1;
    return SNN_OK;
}

int snn_profile_steps(snn_net *net, int64_t n_steps, void *cuda_stream, double *ms_update, double *ms_deliver)
{
    HandleScope scope(net);
    if (!net) return fail(SNN_EINVAL, "null network");
    if (n_steps < 0) return fail(SNN_EINVAL, "n_steps < 0");
    if (net->device_error) return fail(SNN_ESTATE, "a previous device error is pending");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (net->engine == SNN_ENGINE_RESIDENT) {
        // one cooperative launch runs both phases of every step: its time goes to ms_update
        cudaEvent_t e0, e1;
        SNN_CUDA_TRY(cudaEventCreate(&e0));
        SNN_CUDA_TRY(cudaEventCreate(&e1));
        cudaEventRecord(e0, st);
        int rc = launch_steps_resident(net, n_steps, st);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (rc == SNN_OK) {
            const cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) rc = fail(SNN_ECUDA, std::string("profile: ") + cudaGetErrorString(e));
            else cudaEventElapsedTime(&ms, e0, e1);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc != SNN_OK) return rc;
        net->t += n_steps;
        if (ms_update) *ms_update = ms;
        if (ms_deliver) *ms_deliver = 0.0;
        return SNN_OK;
    }
    double su = 0.0, sd = 0.0;
    const int64_t batch = 256;
    const size_t G = std::max<size_t>(net->group_args.size(), 1);
    const bool grouped = !net->group_args.empty();
    std::vector<cudaEvent_t> ev(3 * batch * G);
    for (auto &e : ev) SNN_CUDA_TRY(cudaEventCreate(&e));
    int rc = SNN_OK;
    for (int64_t done = 0; done < n_steps && rc == SNN_OK; done += batch) {
        const int64_t m = std::min(batch, n_steps - done);
        int64_t used = 0;  // event triples recorded in this batch
        for (size_t g = 0; g < G; ++g) {
            for (int64_t k = 0; k < m; ++k, ++used) {
                cudaEventRecord(ev[3 * used], st);
                if (net->engine == SNN_ENGINE_PIPELINED || net->engine == SNN_ENGINE_PERSISTENT) {
                    const int ph = static_cast<int>((net->t + done + k) % snn::kPhasePeriod);
                    snn::launch_step(grouped ? net->group_args[g] : net->args, static_cast<int>(k), ph,
                                     grouped ? net->group_grid[g] : net->step_grid, st);
                    cudaEventRecord(ev[3 * used + 1], st);
                } else {
                    snn::launch_update(grouped ? net->group_args[g] : net->args, static_cast<int>(k),
                                       grouped ? net->group_grid[g] : net->update_grid, st);
                    cudaEventRecord(ev[3 * used + 1], st);
                    launch_phase2(net, static_cast<int>(k), st);
                }
                cudaEventRecord(ev[3 * used + 2], st);
            }
            if (g + 1 < G) snn::launch_resync(net->args.ctl, st);
        }
        snn::launch_advance(net->args.ctl, m, st);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[3 * used - 1]);
        if (e != cudaSuccess) {
            rc = fail(SNN_ECUDA, std::string("profile: ") + cudaGetErrorString(e));
            break;
        }
        for (int64_t k = 0; k < used; ++k) {
            float a = 0.f, b = 0.f;
            cudaEventElapsedTime(&a, ev[3 * k], ev[3 * k + 1]);
            cudaEventElapsedTime(&b, ev[3 * k + 1], ev[3 * k + 2]);
            su += a;
            sd += b;
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (rc != SNN_OK) return rc;
    SNN_CUDA_TRY(cudaStreamSynchronize(st));
    net->t += n_steps;
    if (ms_update) *ms_update = su;
    if (ms_deliver) *ms_deliver = sd;
    return SNN_OK;
}

namespace {

// Copies history entries of steps below t_done, from the read position on.
int read_history(snn_net *net, int64_t t_done, int64_t *steps, int32_t *neurons, int64_t capacity,
                 int64_t *n_written, int rc)
{
    const int64_t done_end =
        std::lower_bound(net->hist_t.begin(), net->hist_t.end(), static_cast<int32_t>(std::min<int64_t>(t_done, INT32_MAX))) -
        net->hist_t.begin();
    const int64_t avail = std::max<int64_t>(0, done_end - net->read_pos);
    if (!steps && !neurons) {
        *n_written = avail;
        return rc;
    }
    if (!steps || !neurons || capacity < 0) return fail(SNN_EINVAL, "bad output arrays");
    const int64_t m = std::min(avail, capacity);
    for (int64_t j = 0; j < m; ++j) {
        steps[j] = net->hist_t[net->read_pos + j];
        neurons[j] = net->hist_i[net->read_pos + j];
    }
    net->read_pos += m;
    *n_written = m;
    return rc;
}

}  // namespace

int snn_read_spikes(snn_net *net, int64_t *steps, int32_t *neurons, int64_t capacity, int64_t *n_written)
{
    HandleScope scope(net);
    if (!net || !n_written) return fail(SNN_EINVAL, "null argument");
    *n_written = 0;
    const int rc = drain(net);
    // only spikes of completed steps (the pipelined engine has already decided the next
    // step's spikes, but keeps them in its queue)
    return read_history(net, net->t, steps, neurons, capacity, n_written, rc);
}

int snn_collect_spikes(snn_net *net, int64_t *steps, int32_t *neurons, int64_t capacity, int64_t *n_written)
{
    HandleScope scope(net);
    if (!net || !n_written) return fail(SNN_EINVAL, "null argument");
    *n_written = 0;
    if (net->device_error) return drain(net);  // report it now
    const int rc = collect(net);
    return read_history(net, net->collected_t, steps, neurons, capacity, n_written, rc);
}

int snn_read_rates(snn_net *net, int64_t t_begin, int64_t t_end, double *pop_rates_hz, int32_t *neuron_counts)
{
    HandleScope scope(net);
    if (!net || !pop_rates_hz) return fail(SNN_EINVAL, "null argument");
    if (t_begin < 0 || t_end <= t_begin) return fail(SNN_EINVAL, "empty or negative window");
    if (t_end > net->t) return fail(SNN_EINVAL, "window ends after the steps enqueued so far");
    int rc = drain(net);
    const int P = net->spec.model.n_pops;
    std::vector<int64_t> pop_cnt(P, 0);
    if (neuron_counts) std::fill(neuron_counts, neuron_counts + net->n, 0);
    const auto lo = std::lower_bound(net->hist_t.begin(), net->hist_t.end(), t_begin) - net->hist_t.begin();
    const auto hi = std::lower_bound(net->hist_t.begin(), net->hist_t.end(), t_end) - net->hist_t.begin();
    for (auto j = lo; j < hi; ++j) {
        const int32_t i = net->hist_i[j];
        ++pop_cnt[net->pop_id[i]];
        if (neuron_counts) ++neuron_counts[i];
    }
    // population sizes over every circuit (inert neurons between circuits excluded)
    std::vector<int64_t> pop_n(P, 0);
    for (const auto &ci : net->circuits)
        for (int64_t i = ci.base; i < ci.base + ci.n; ++i) ++pop_n[net->pop_id[i]];
    const double secs = static_cast<double>(t_end - t_begin) * net->spec.model.dt_ms * 1e-3;
    for (int b = 0; b < P; ++b)
        pop_rates_hz[b] = pop_n[b] > 0 ? static_cast<double>(pop_cnt[b]) / (static_cast<double>(pop_n[b]) * secs) : 0.0;
    return rc;
}

int snn_get_info(const snn_net *net, snn_info *out)
{
    if (!net || !out) return fail(SNN_EINVAL, "null argument");
    std::memset(out, 0, sizeof(*out));
    out->n_neurons = net->n;
    out->n_synapses = net->n_syn;
    out->n_synapses_padded = net->n_syn_padded;
    out->t = net->t;
    // count spikes of completed steps only (the pipelined engine records the next
    // step's spikes one launch early)
    const int64_t done_end =
        std::lower_bound(net->hist_t.begin(), net->hist_t.end(), static_cast<int32_t>(std::min<int64_t>(net->t, INT32_MAX))) -
        net->hist_t.begin();
    int64_t pending_events = 0;
    for (size_t j = static_cast<size_t>(done_end); j < net->hist_t.size(); ++j) pending_events += net->out_degree[net->hist_i[j]];
    out->spikes_read = done_end;
    out->events_read = net->events_read - pending_events;
    out->n_pops = net->spec.model.n_pops;
    out->t_ref_steps = net->c.t_ref;
    for (int b = 0; b <= SNN_MAX_POPS; ++b)
        out->pop_offsets[b] = b < (int)net->pop_off.size() ? net->pop_off[b] : net->n;
    out->w_f = net->c.w_f;
    out->p11 = net->c.p11;
    out->p22 = net->c.p22;
    out->p21 = net->c.p21;
    out->p11_f32 = net->c.p11f;
    out->p21_f32 = net->c.p21f;
    out->p22_f32 = net->c.p22f;
    out->theta_f32 = net->c.theta;
    out->u_reset_f32 = net->c.u_reset;
    out->w_ext_fx = net->c.w_ext_fx;
    std::memcpy(out->poisson_thresholds, net->c.thresholds, sizeof(out->poisson_thresholds));
    out->max_row_length = net->max_row;
    out->chunks_per_row = net->chunks_per_row;
    out->steps_per_graph = net->steps_per_graph;
    out->deliver_blocks = net->deliver_grid;
    out->device_error = net->device_error;
    out->engine = net->engine;
    out->record_format = net->format;
    out->bytes_per_synapse = snn::record_bytes(net->format);
    out->n_circuits = static_cast<int32_t>(net->circuits.size());
    const bool step_kernel = net->engine == SNN_ENGINE_PIPELINED || net->engine == SNN_ENGINE_PERSISTENT;
    const bool resident = net->engine == SNN_ENGINE_RESIDENT;
    out->schedule_ctas = resident ? net->args.n_blocks : step_kernel ? net->step_grid : net->deliver_grid;
    out->schedule_delivery_warps = step_kernel || resident ? net->args.delivery_warps : 0;
    out->target_blocks = net->args.n_blocks;
    out->circuits_per_group = net->circuits_per_group;
    std::strncpy(out->last_error, net->last_error.c_str(), sizeof(out->last_error) - 1);
    std::memcpy(out->i8_base, net->i8_base, sizeof(out->i8_base));
    std::memcpy(out->i8_step, net->i8_step, sizeof(out->i8_step));
    return SNN_OK;
}

int snn_get_layout(const snn_net *net, snn_layout *out)
{
    if (!net || !out) return fail(SNN_EINVAL, "null argument");
    const snn::Layout &L = net->L;
    out->ctl = L.ctl;
    out->params = L.tables;
    const bool second = (net->engine == SNN_ENGINE_PIPELINED || net->engine == SNN_ENGINE_PERSISTENT) &&
                        ((net->t - 1) & 1);
    out->U = second ? L.U2 : L.U;
    out->I = L.I;
    out->R = second ? L.R2 : L.R;
    out->ring = L.ring;
    out->row_ptr = L.row_ptr;
    out->syn_tgt = L.syn_tgt;
    out->syn_w = L.syn_w;
    out->syn_delay = L.syn_d;
    out->rast_neuron = L.rast_nrn;
    out->rast_step = L.rast_t;
    out->n_neurons_padded = net->npad;
    out->n_synapses_padded = net->n_syn_padded;
    out->blocks = L.blocks;
    out->block_starts = net->engine == SNN_ENGINE_RESIDENT ? L.seg : 0;
    return SNN_OK;
}

namespace {

constexpr uint64_t kStateMagic = 0x534E4E5354415432ull;  // "SNNSTAT2"

struct StateHeader {
    uint64_t magic;
    uint64_t bytes;
    int64_t n, npad, t;
    int32_t engine, n_segments;
    int32_t circuits_per_group;  // the pending spike queue's layout (pipelined engine)
    int32_t reserved;
};

// Device segments that make up the dynamic state, as (arena offset, bytes).
std::vector<std::pair<uint64_t, uint64_t>> state_segments(const snn_net *net)
{
    const snn::Layout &L = net->L;
    std::vector<std::pair<uint64_t, uint64_t>> seg = {
        {L.ctl, sizeof(snn::Ctl)}, {L.U, 4 * uint64_t(net->npad)}, {L.I, 4 * uint64_t(net->npad)},
        {L.R, uint64_t(net->npad)}, {L.ring, 4 * uint64_t(snn::kDMax) * net->npad}};
    if (net->engine == SNN_ENGINE_PIPELINED || net->engine == SNN_ENGINE_PERSISTENT) {
        seg.push_back({L.U2, 4 * uint64_t(net->npad)});
        seg.push_back({L.R2, uint64_t(net->npad)});
        seg.push_back({L.queue, 4 * sizeof(snn::QueueEntry) * net->npad});
        seg.push_back({L.qcount, 16 * uint64_t(net->npad / 128 + 1)});
    }
    return seg;
}

}  // namespace

int snn_save_state(snn_net *net, void *host_buf, uint64_t capacity, uint64_t *written)
{
    HandleScope scope(net);
    if (!net || !written) return fail(SNN_EINVAL, "null argument");
    const auto seg = state_segments(net);
    uint64_t total = sizeof(StateHeader);
    for (const auto &sg : seg) total += sg.second;
    *written = total;
    if (!host_buf) return SNN_OK;
    if (capacity < total) return fail(SNN_ENOMEM, "state buffer too small");
    int rc = drain(net);  // spikes so far go to the host history; the device raster restarts at 0
    if (rc) return rc;
    StateHeader h{kStateMagic, total, net->n, net->npad, net->t, net->engine, static_cast<int32_t>(seg.size()),
                  net->circuits_per_group, 0};
    uint8_t *out = static_cast<uint8_t *>(host_buf);
    std::memcpy(out, &h, sizeof(h));
    uint64_t off = sizeof(h);
    for (const auto &sg : seg) {
        SNN_CUDA_TRY(cudaMemcpy(out + off, net->arena + sg.first, sg.second, cudaMemcpyDeviceToHost));
        off += sg.second;
    }
    return SNN_OK;
}

int snn_load_state(snn_net *net, const void *host_buf, uint64_t bytes)
{
    HandleScope scope(net);
    if (!net || !host_buf) return fail(SNN_EINVAL, "null argument");
    if (bytes < sizeof(StateHeader)) return fail(SNN_EINVAL, "state buffer too small");
    StateHeader h;
    std::memcpy(&h, host_buf, sizeof(h));
    const auto seg = state_segments(net);
    uint64_t total = sizeof(StateHeader);
    for (const auto &sg : seg) total += sg.second;
    if (h.magic != kStateMagic || h.bytes != total || bytes < total)
        return fail(SNN_EINVAL, "not a state saved by snn_save_state");
    if (h.n != net->n || h.npad != net->npad || h.engine != net->engine || h.n_segments != static_cast<int32_t>(seg.size()))
        return fail(SNN_EINVAL, "state was saved from a network of another shape or engine");
    int rc = wait_done(net);
    if (rc) return rc;
    const uint8_t *in = static_cast<const uint8_t *>(host_buf);
    uint64_t off = sizeof(h);
    for (const auto &sg : seg) {
        SNN_CUDA_TRY(cudaMemcpy(net->arena + sg.first, in + off, sg.second, cudaMemcpyHostToDevice));
        off += sg.second;
    }
    net->t = h.t;
    if (net->engine == SNN_ENGINE_PIPELINED && h.circuits_per_group != net->circuits_per_group) {
        // saved under another circuit grouping: move the pending spikes to this one's queues
        rc = regroup_queue(net, h.circuits_per_group);
        if (rc) return rc;
    }
    net->hist_t.clear();
    net->hist_i.clear();
    net->read_pos = 0;
    net->raster_read = 0;
    net->snaps_valid_from = net->n_snaps;
    net->collected_t = h.t;
    net->events_read = 0;
    net->device_error = 0;
    return SNN_OK;
}

int snn_set_schedule(snn_net *net, int32_t grid_ctas, int32_t delivery_warps, int32_t steps_per_graph)
{
    HandleScope scope(net);
    if (!net) return fail(SNN_EINVAL, "null network");
    if (grid_ctas < 0 || grid_ctas > 65535 || delivery_warps < 0 || steps_per_graph < 0 || steps_per_graph > 100000)
        return fail(SNN_EINVAL, "schedule out of range");
    int rc = wait_done(net);
    if (rc) return rc;
    snn::StepArgs &a = net->args;
    if (net->engine == SNN_ENGINE_PIPELINED) {
        if (delivery_warps > 0 && delivery_warps + snn::kStepMaxNeuronWarps > snn::kStepMaxThreads / 32)
            return fail(SNN_EINVAL, "too many delivery warps per CTA");
        if (grid_ctas > 0) {
            net->step_grid = grid_ctas;
            net->step_grid_set = true;
        }
        if (delivery_warps > 0) {
            a.delivery_warps = delivery_warps;
            net->delivery_warps_set = true;
        }
        a.neuron_warps = step_neuron_warps(((net->n + 3) / 4 + 31) / 32, net->step_grid);
        if (steps_per_graph > 0)
            net->steps_per_graph = std::max(snn::kPhasePeriod, steps_per_graph / snn::kPhasePeriod * snn::kPhasePeriod);
    } else if (net->engine == SNN_ENGINE_GRAPH) {
        if (grid_ctas > 0) net->deliver_grid = grid_ctas;
        if (steps_per_graph > 0) net->steps_per_graph = steps_per_graph;
    } else if (net->engine == SNN_ENGINE_RESIDENT) {
        // one CTA per target block; the delivery warps must cover one mailbox per lane
        if (grid_ctas > 0) return fail(SNN_ENOTSUP, "the resident engine runs one CTA per target block");
        if (delivery_warps > 0) {
            // two teams of delivery_warps / 2 warps, each with a lane per mailbox
            if (delivery_warps % 2 != 0 || (delivery_warps / 2) * 32 < a.n_blocks ||
                a.neuron_warps + delivery_warps > snn::kResidentMaxWarps)
                return fail(SNN_EINVAL, "resident engine: delivery warps must be even, give each of the two teams "
                                        "a lane per target block and fit the CTA");
            a.delivery_warps = delivery_warps;
        }
        if (steps_per_graph > 0) net->steps_per_graph = steps_per_graph;
        return SNN_OK;
    } else {
        if (grid_ctas > 0 || delivery_warps > 0 || steps_per_graph > 0)
            return fail(SNN_ENOTSUP, "the persistent engine has a fixed schedule");
        return SNN_OK;
    }
    build_groups(net);  // the group arguments copy the schedule
    return recapture(net);
}

int snn_set_circuit_groups(snn_net *net, int32_t circuits_per_group)
{
    HandleScope scope(net);
    if (!net) return fail(SNN_EINVAL, "null network");
    if (circuits_per_group < 0) return fail(SNN_EINVAL, "circuits_per_group < 0");
    if (net->engine != SNN_ENGINE_GRAPH && net->engine != SNN_ENGINE_PIPELINED)
        return fail(SNN_ENOTSUP, "circuit groups run on the graph and pipelined engines");
    if (net->device_error) return fail(SNN_ESTATE, "a previous device error is pending");
    int rc = wait_done(net);
    if (rc) return rc;
    const int32_t old = net->circuits_per_group;
    net->circuits_per_group = circuits_per_group >= static_cast<int32_t>(net->circuits.size()) ? 0 : circuits_per_group;
    if (net->engine == SNN_ENGINE_PIPELINED && net->circuits_per_group != old) {
        rc = regroup_queue(net, old);
        if (rc) {
            net->circuits_per_group = old;
            return rc;
        }
    }
    build_groups(net);
    return recapture(net);
}

int snn_get_circuits(const snn_net *net, int64_t *base, int64_t *n_neurons)
{
    if (!net || !base || !n_neurons) return fail(SNN_EINVAL, "null argument");
    for (size_t c = 0; c < net->circuits.size(); ++c) {
        base[c] = net->circuits[c].base;
        n_neurons[c] = net->circuits[c].n;
    }
    return SNN_OK;
}

int snn_get_out_degrees(const snn_net *net, int32_t *out)
{
    if (!net || !out) return fail(SNN_EINVAL, "null argument");
    std::copy(net->out_degree.begin(), net->out_degree.end(), out);
    return SNN_OK;
}

int snn_deliver_spikes(snn_net *net, const int32_t *spikers, int64_t n_spikers, int64_t t, int32_t blocks,
                       void *cuda_stream)
{
    HandleScope scope(net);
    if (!net || (n_spikers > 0 && !spikers)) return fail(SNN_EINVAL, "null argument");
    if (n_spikers < 0 || t < 0 || blocks < 0) return fail(SNN_EINVAL, "negative argument");
    if (n_spikers == 0) return SNN_OK;
    if (net->engine == SNN_ENGINE_RESIDENT) {
        // block-major records: each target block's CTA reads its region's segments
        const int e = snn::launch_deliver_regions(net->args, spikers, n_spikers, t, cuda_stream);
        if (e != 0) return fail(SNN_ECUDA, std::string("deliver: ") + cudaGetErrorString(static_cast<cudaError_t>(e)));
        return SNN_OK;
    }
    if (snn::is_blocked(net->format)) {
        snn::launch_deliver_blocked(net->args, spikers, n_spikers, t, 0, cuda_stream);
        SNN_CUDA_TRY(cudaGetLastError());
        return SNN_OK;
    }
    const int grid = blocks > 0 ? blocks : net->num_sms * snn::deliver_list_blocks_per_sm();
    snn::launch_deliver_list(net->args, spikers, n_spikers, t, grid, cuda_stream);
    SNN_CUDA_TRY(cudaGetLastError());
    return SNN_OK;
}

void snn_destroy(snn_net *net)
{
    if (!net) return;
    if (net->ev_recorded) cudaEventSynchronize(net->ev_done);
    if (net->graph_exec) cudaGraphExecDestroy(net->graph_exec);
    if (net->graph) cudaGraphDestroy(net->graph);
    if (net->capture_stream) cudaStreamDestroy(net->capture_stream);
    if (net->ev_done) cudaEventDestroy(net->ev_done);
    for (int k = 0; k < snn_net::kSnaps; ++k)
        if (net->snap_ev[k]) cudaEventDestroy(net->snap_ev[k]);
    if (net->snap_cursor) cudaFreeHost(net->snap_cursor);
    if (net->copy_stream) cudaStreamDestroy(net->copy_stream);
    if (net->pin_nrn) cudaFreeHost(net->pin_nrn);
    if (net->pin_t) cudaFreeHost(net->pin_t);
    delete net;
}

}  // extern "C"
