// Internal declarations shared by the host builder, the kernels and the ABI layer.
#pragma once

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/snn.h"

namespace snn {

constexpr int kDMax = SNN_D_MAX;             // ring rows (§3.2)
constexpr int kDMask = SNN_D_MAX - 1;
constexpr int kPK = SNN_POISSON_KMAX;
constexpr int64_t kNeuronAlign = 128;        // ring row stride granularity
constexpr int kRowAlign = 4;                 // synapse rows padded to whole int4 quads
constexpr int kChunk = 256;                  // synapses per delivery work item (32 lanes x 2 quads)
constexpr int kUpdateThreads = 128;          // 4 neurons per thread
constexpr int kDeliverThreads = 256;
constexpr int kStepDeliverWarps = 8;         // delivery warps per CTA of the pipelined step kernel
constexpr int kStepMaxThreads = 384;            // neuron warps (<= 4) + delivery warps per CTA
constexpr int kStepMaxNeuronWarps = 4;
constexpr int kPhasePeriod = 64;             // pipelined engine: buffers repeat with t mod 64
constexpr uint32_t kErrRaster = 1u;
constexpr uint32_t kErrTimeout = 2u;
constexpr uint64_t kBarrierTimeoutNs = 2000000000ull;  // default bound of every grid-barrier wait
constexpr int64_t kMaxPersistentSteps = 1 << 20;        // steps per cooperative launch

// Device control block (first bytes of the arena).
struct alignas(64) Ctl {
    int64_t t_base;          // first step of the next graph replay / launch batch
    uint32_t cursor;         // spikes appended to the raster since the last drain
    uint32_t step_begin[2];  // raster index where step t's spikes start, by t mod 2
    uint32_t err;            // sticky error bits
    uint32_t bar;            // grid-barrier arrivals of the running persistent launch
    uint32_t qcnt[4];        // pipelined engine: spikes queued for step s in queue s mod 4
    uint32_t pad[5];
};

// Pipelined engine: one queue entry per spike of a step, written by the thread that
// decided the spike, consumed by the next kernel's delivery warps.
struct alignas(16) QueueEntry {
    uint32_t row_quad;   // first synapse of the row / 4
    uint32_t len_quads;  // padded row length / 4
    int32_t neuron;
    int32_t step;        // low 32 bits of the step index (tells fresh entries from stale ones)
};

// int8 read-back of one (source, target) population pair: w = base + code * step.
struct alignas(8) PairQ {
    int32_t base;
    int32_t step;
};

// One circuit of the neuron index space (a single network is circuit 0).
struct alignas(16) CircuitInfo {
    int64_t base;    // first neuron (a multiple of 128)
    int64_t n;       // neurons
    uint64_t seed;   // seed of its random streams
    int64_t pad;
};

// Read-only tables in the arena.
struct alignas(16) StaticTables {
    uint64_t thresholds[SNN_MAX_POPS][kPK];  // 63-bit Poisson CDF thresholds
    int64_t pop_off[SNN_MAX_POPS + 1];
    int32_t n_pops;
    int32_t pad;
    PairQ i8_pair[SNN_MAX_POPS][SNN_MAX_POPS];  // packed int8 records: read-back per [source][target]
};

// Packed synapse word: target (20 bits), delay (6), target population (3), padding flag.
constexpr int kWordTargetBits = 20;
constexpr uint32_t kWordTargetMask = (1u << kWordTargetBits) - 1;
constexpr int kWordDelayShift = 20;
constexpr int kWordPopShift = 26;
constexpr uint32_t kWordPad = 1u << 31;
constexpr int64_t kPackedMaxNeurons = int64_t{1} << kWordTargetBits;
inline int record_bytes(int format)
{
    return format == SNN_RECORD_PACKED_I8                                         ? 5
           : format == SNN_RECORD_PACKED_BF16 || format == SNN_RECORD_BLOCKED6 ? 6
           : format == SNN_RECORD_BLOCKED4                                      ? 4
           : format == SNN_RECORD_BLOCKED8                                      ? 8
                                                                                : 9;
}
inline bool is_blocked(int format)
{
    return format == SNN_RECORD_BLOCKED6 || format == SNN_RECORD_BLOCKED4 || format == SNN_RECORD_BLOCKED8;
}

// Blocked records: target blocks and the delivery kernel that owns one block per CTA.
constexpr int kBlockLocalBits = 10;          // record = local target | delay << 10
constexpr int kBlockMaxWidth = 768;          // targets per block (shared-memory bins [64][768])
constexpr int kBlockAvgWidth = 512;          // sets the number of in-degree quotas
constexpr int kBlockAlign = 32;              // block boundaries are multiples of 32
constexpr int kBlockQuad = 4;                // (row, block) segments are whole quads of records
constexpr int kBlockedThreads = 1024;
constexpr int kBlockedBatch = 2048;          // senders staged per pass
constexpr int kBlockedWindow = 8192;         // quads of a pass whose record-array index is tabled at once
constexpr int kBlockedBinDelays = 32;        // delays summed in shared memory (longer: ring reductions)
constexpr int kBlockedRounds = 4;            // quads in flight per lane (32 per round and warp)
constexpr int64_t kBlockedAggregateMin = 64; // fewer senders: reduce straight into the ring
inline int max_target_blocks(int64_t n)
{
    return static_cast<int>((n + kBlockAvgWidth - 1) / kBlockAvgWidth + n / (kBlockMaxWidth - kBlockAlign) + 2);
}

// Resident engine: one cooperative CTA per target block of consecutive neurons, which
// keeps its neurons' state in registers and its columns of the ring in shared memory
// for a whole launch; spikes cross between CTAs through inbox slots (one per reader and
// sender) and, beyond three spikes of a block in one step, the sender's outbox.
constexpr int kResidentMaxWidth = 1024;      // neurons per block (8 neuron warps x 128)
constexpr int kResidentMaxBlocks = 256;      // blocks (CTAs, at most one per SM)
constexpr int kResidentAlign = 32;           // block boundaries are multiples of 32
constexpr int kResidentMaxWarps = 20;        // neuron warps + delivery warps per CTA
constexpr int kResidentTeamWarps = 8;        // delivery warps per team where the CTA has room (two teams)
constexpr int kResidentMboxWords = kResidentMaxWidth + 4;  // u32 words of one outbox (entries of a step)
constexpr int kResidentSlotWords = 4;        // u32 words of one inbox slot: header and three entries
constexpr int64_t kResidentMaxSteps = int64_t{1} << 19;     // steps per launch (mailbox tags count them)
constexpr int kResidentGather = 256;         // spikes of a step staged in shared memory per pass
constexpr int64_t kResidentMaxNeurons = int64_t{kResidentMaxBlocks} * kResidentMaxWidth;
constexpr uint32_t kResidentEscape = 255;    // segment length code: 255 or more, read the exact offsets
constexpr uint32_t kResidentGroupFlag = 1u << 31;  // a group of 32 senders holds an escaped length
inline int resident_max_blocks(int64_t n)
{
    return static_cast<int>(std::min<int64_t>(kResidentMaxBlocks, (n + kResidentAlign - 1) / kResidentAlign));
}

// Resident engine: the records are stored block-major -- every synapse into target block
// p, by sender and then delay, forms block p's region starting at record rbase[p] -- and
// each block has its segment tables: offt[p][s] (uint32, offset of sender s's segment in
// the region, offt[p][n] the region's length), lens[p][s] = min(length, 255) (uint8) and
// coarse[p][g] = offt[p][32 g] with kResidentGroupFlag set if one of the group's lengths
// is escaped.  A CTA keeps its lens and coarse rows in shared memory.  This gives the
// tables' byte offsets within their arena region.
struct ResTables {
    uint64_t rbase, coarse, lens, offt, total;
    int64_t lens_stride, coarse_stride;
};
inline ResTables resident_tables(int64_t n, int64_t blocks)
{
    auto up = [](uint64_t x) { return (x + 255) & ~uint64_t{255}; };
    ResTables t{};
    t.lens_stride = (n + 31) / 32 * 32;
    t.coarse_stride = (n + 31) / 32 + 1;
    uint64_t o = 0;
    t.rbase = o; o = up(o + 8 * uint64_t(blocks + 1));
    t.coarse = o; o = up(o + 4 * uint64_t(blocks) * t.coarse_stride);
    t.lens = o; o = up(o + uint64_t(blocks) * t.lens_stride);
    t.offt = o; o = up(o + 4 * uint64_t(blocks) * (n + 1));
    t.total = o;
    return t;
}

// Kernel arguments (by value; small).
struct StepArgs {
    Ctl *ctl;
    const StaticTables *tables;
    float *U;
    float *I;
    uint8_t *R;
    int32_t *ring;
    const int64_t *row_ptr;
    const int32_t *syn_tgt;
    const int32_t *syn_w;
    const uint8_t *syn_d;
    int32_t *rast_nrn;
    int32_t *rast_t;
    int64_t n;        // neurons
    int64_t npad;     // ring row stride
    uint64_t seed;
    uint32_t rast_cap;
    int32_t chunks_per_row;
    float p11, p21, p22, theta, u_reset;
    int32_t t_ref;
    int32_t w_ext_fx;
    uint64_t barrier_timeout_ns;  // bound of each grid-barrier wait (persistent engine)
    uint32_t barrier_extra;       // arrivals expected beyond the grid (0; 1 only for the stall test)
    int32_t neuron_warps;         // pipelined engine: neuron warps per CTA
    float *U2;                    // pipelined engine: second U / R buffers (state after A(s) in buffer s mod 2)
    uint8_t *R2;
    QueueEntry *queue;            // pipelined engine: 4 queues, entry j of queue s at queue[s * npad + j]
    int64_t pop_off[SNN_MAX_POPS + 1];  // population offsets (read from the launch arguments)
    int32_t n_pops;
    int32_t quad_warps;           // pipelined engine: end of the launch's groups of 128 neurons
    uint32_t *qcount;             // pipelined engine: spikes in each of the 4 queues (Ctl::qcnt, or a circuit group's)
    int32_t format;               // SNN_RECORD_*
    int32_t n_circuits;
    int32_t delivery_warps;       // pipelined engine: delivery warps per CTA
    int32_t group_launch;         // pipelined engine: 1 for a circuit group's launch (its own queues and range)
    const uint8_t *pop_id;        // population of every neuron [npad]
    const int32_t *group_circuit; // circuit of every group of 128 neurons [npad / 128]
    const CircuitInfo *circuits;  // [n_circuits]
    const uint16_t *blk_rec;      // blocked records: local target | delay << 10
    const uint16_t *blk_seg;      // blocked records: [n][n_blocks + 1] block starts within each row
    const int32_t *blk_off;       // blocked records: block boundaries [n_blocks + 1]
    int32_t n_blocks;
    int32_t pad4;
    int64_t quad_base;            // first quad the update (or step) launch covers, n its end neuron
    int64_t queue_cap;            // pipelined engine: entries of each queue (a circuit group's neurons)
    uint32_t *mbox;               // resident engine: outboxes [4][n_blocks][kResidentMboxWords]
    uint32_t *inbox;              // resident engine: inbox slots [4][n_blocks (reader)][n_blocks (sender)][4]
    const int64_t *res_rbase;     // resident engine: first record of every block's region [n_blocks + 1]
    const uint32_t *res_coarse;   // resident engine: [n_blocks][coarse_stride] (see resident_tables)
    const uint8_t *res_lens;      // resident engine: [n_blocks][lens_stride]
    const uint32_t *res_offt;     // resident engine: [n_blocks][n + 1]
    const void *res_rec;          // resident engine: block-major int2 records {weight, local target | delay << 16}
    int32_t res_lens_stride;
    int32_t res_coarse_stride;
    int32_t res_rows;             // resident engine: ring rows kept in shared memory (power of two, 8..64)
    int32_t res_stride;           // resident engine: shared ring row stride (widest block, multiple of 32)
};

// Host constants of one model (§2.2).
struct Constants {
    double w_f, p11, p22, beta, gamma, p21;
    float p11f, p21f, p22f, theta, u_reset;
    int32_t t_ref;
    int32_t w_ext_fx;
    uint64_t thresholds[SNN_MAX_POPS][kPK];
};

// Network in host memory, in the device layout.
struct HostNetwork {
    int format = SNN_RECORD_PLAIN9;
    std::vector<uint8_t> pop_id;         // population of every neuron
    std::vector<CircuitInfo> circuits;   // circuit table (one entry for a single network)
    std::vector<uint32_t> word;    // packed records: words
    std::vector<uint8_t> wbytes;   // packed records: int8 codes or bfloat16 currents
    int32_t i8_base[SNN_MAX_POPS][SNN_MAX_POPS] = {};
    int32_t i8_step[SNN_MAX_POPS][SNN_MAX_POPS] = {};
    int64_t n = 0;
    int64_t npad = 0;
    int64_t n_syn = 0;         // true synapses
    int64_t n_syn_padded = 0;  // including row padding
    int32_t max_row = 0;
    std::vector<int64_t> pop_off;
    std::vector<int64_t> row_ptr;   // padded offsets, n+1
    std::vector<int32_t> out_degree;  // true row lengths
    std::vector<int32_t> tgt;
    std::vector<int32_t> w;
    std::vector<uint8_t> d;
    std::vector<float> u0;
    std::vector<int32_t> blk;      // blocked records: block boundaries
    std::vector<uint16_t> rec16;   // blocked records: local target | delay << 10
    std::vector<uint16_t> seg;     // blocked records: [n][blocks + 1] block starts per row
    std::vector<uint8_t> restab;   // resident engine: the tables of resident_tables(n, blocks), as bytes
    std::vector<uint64_t> rec8;    // resident engine: weight (low word), local target | delay << 16 (high word)
};

// Arena layout for a spec.
struct Layout {
    uint64_t ctl, tables, U, I, R, ring, row_ptr, syn_tgt, syn_w, syn_d, rast_nrn, rast_t, U2, R2, queue, qcount, pop_id,
        group_circuit, circuits, blocks, seg, mbox, inbox, res_rec, total;
    int64_t npad, syn_padded_max, rast_cap;
};

// builder.cpp
bool validate_spec(const snn_spec &spec, std::string &why);
void compute_constants(const snn_model &m, Constants &c);
void population_sizes(const snn_model &m, int32_t scale_n, int64_t out[SNN_MAX_POPS]);
int64_t pair_count(const snn_model &m, int32_t scale_n, int32_t scale_k, int target, int source);
int64_t count_neurons(const snn_spec &spec);
int64_t count_synapses(const snn_spec &spec);
Layout make_layout(const snn_spec &spec);
// num_sms: SMs of the device (blocked records size their target blocks to it; 0 = no limit)
bool build_host_network(const snn_spec &spec, const Constants &c, HostNetwork &net, std::string &why,
                        int num_sms = 0);
int resolve_threads(int32_t requested);

// kernels.cu
void launch_update(const StepArgs &a, int k, int grid, void *stream);
void launch_deliver(const StepArgs &a, int k, int grid, void *stream);
void launch_advance(Ctl *ctl, int64_t m, void *stream);
// circuit groups: the next group starts the same steps where the raster now ends
void launch_resync(Ctl *ctl, void *stream);
void launch_deliver_list(const StepArgs &a, const int32_t *list, int64_t n, int64_t t, int grid, void *stream);
// blocked records: one CTA per target block; list == nullptr delivers step t_base + k's
// spikes from the raster (graph engine), else list[0 .. n) as spikes of step t
int prepare_blocked_kernel();
void launch_deliver_blocked(const StepArgs &a, const int32_t *list, int64_t n, int64_t t, int k, void *stream);
int deliver_list_blocks_per_sm();
int update_grid(int64_t n);  // CTAs of k_update for n neurons
int persistent_blocks_per_sm(const StepArgs &a);
int launch_persistent(const StepArgs &a, int64_t n_steps, int grid, void *stream);
// pipelined: B(t), A(t+1), D(t); ph = t mod 64.  With `programmatic`, the launch may
// begin while the previous kernel in the stream still runs (it waits inside).
int launch_step(const StepArgs &a, int k, int ph, int grid, void *stream, bool programmatic = false);
void launch_prime(const StepArgs &a, int grid, void *stream);         // pipelined: A(0)
int prepare_step_kernel(const StepArgs &a);                           // dynamic shared memory opt-in
int step_grid(int num_sms, int64_t quad_warps);  // default CTAs of the step kernel
int step_threads(const StepArgs &a);

// resident.cu
// Block width of the resident engine for n neurons on num_sms SMs (a multiple of
// kResidentAlign; 0 if n does not fit kResidentMaxWidth per SM).
int64_t resident_width(int64_t n, int num_sms);
size_t resident_smem_bytes(int rows, int stride, int64_t n);
// Ring rows in shared memory: the largest power of two in [8, 64] (at most `cap` when
// cap > 0) whose shared memory fits one CTA; 0 if none fits.
int resident_rows(int stride, int cap, int64_t n);
int prepare_resident_kernel(const StepArgs &a);
int resident_blocks_per_sm(const StepArgs &a);
// n_steps steps from the device's t_base in one cooperative launch of a.n_blocks CTAs
int launch_resident(const StepArgs &a, int64_t n_steps, void *stream);
// phase 2 alone for list[0 .. n) as spikes of step t on block-major records: one CTA per
// target block, reads confined to the block's region
int launch_deliver_regions(const StepArgs &a, const int32_t *list, int64_t n, int64_t t, void *stream);

}  // namespace snn
