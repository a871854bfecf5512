/*
 * snn.h -- C ABI of a clock-driven GB300 (sm_103a) simulator of the Potjans-Diesmann
 * cortical microcircuit, following the model and the push-based step loop of
 * Lindqvist & Podobas, "Fast Algorithms for Spiking Neural Network Simulation with
 * FPGAs" (arXiv 2405.02019).
 *
 * What one simulation step computes (all on the GPU, no host round trip):
 *   - thalamic drive: a Poisson count T per neuron with mean nu_th K dt (§2.2, the
 *     sentence after Eq. ref);
 *   - the exact-integration LIF update with refractoriness, threshold and reset
 *     (§2.2, Eqs. mem, psc, ref; Listing push of §3.1);
 *   - deferred push delivery (Listing push2, §3.1) of every spike through the
 *     sender's synapses into a 64-row wrap-around ring W[(t + d) mod 64][target]
 *     (§3.2), read and cleared by the target at step t + d.
 *
 * Numerics (plain mode): FP32 neuron state with every product and sum rounded
 * separately (no FMA); synaptic input accumulated as int32 counts of 2^-12 pA, so
 * delivery order cannot change the result; FP64 only on the host for the
 * propagators.  The raster is reproducible bit for bit.
 *
 * Conventions for every function:
 *   - returns an snn_status (SNN_OK = 0); no exceptions cross the ABI, nothing exits;
 *     snn_last_error() gives a message for the calling thread's last failure;
 *   - host pointers are read during the call only, unless stated otherwise;
 *   - device memory is owned by the caller: one arena of snn_sizes.arena_bytes bytes
 *     (256-byte aligned), which must outlive the network handle; the library never
 *     allocates device memory itself;
 *   - `cuda_stream` is a cudaStream_t (NULL = legacy default stream); calls on one
 *     handle must not run concurrently.
 */
#ifndef SNN_H
#define SNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SNN_ABI_VERSION 2u
#define SNN_MAX_POPS 8       /* populations per circuit (the microcircuit has 8) */
#define SNN_MAX_OVERRIDES 4  /* per-pair amplitude overrides (the doubled L4E->L23E pathway) */
#define SNN_D_MAX 64         /* ring rows; delays are whole steps in [1, SNN_D_MAX-1] (§3.2) */
#define SNN_FX_SHIFT 12      /* synaptic input unit: 2^-SNN_FX_SHIFT pA */
#define SNN_POISSON_KMAX 24  /* entries of a thalamic Poisson threshold table */

typedef enum snn_status {
    SNN_OK = 0,
    SNN_EINVAL = 1,    /* invalid argument or specification */
    SNN_ENOMEM = 2,    /* host allocation failed, or the device arena is too small */
    SNN_ECUDA = 3,     /* a CUDA runtime call failed */
    SNN_EOVERFLOW = 4, /* the device raster filled before it was read (sticky) */
    SNN_ETIMEOUT = 5,  /* reserved for bounded device waits */
    SNN_ESTATE = 6,    /* call out of order (e.g. after a sticky device error) */
    SNN_ENOTSUP = 7    /* feature not available in this build */
} snn_status;

/*
 * Parameters of the circuit model: Tables params, params2 and params3 of §2.2.
 * Units: ms, pF, mV, Hz.  conn_p[target][source] is the connection probability of
 * a (source, target) neuron pair.  Synaptic amplitude and delay laws are
 * Gaussians of the *source* population; an override replaces the amplitude law
 * of one (source, target) population pair.
 */
typedef struct snn_model {
    int32_t n_pops;
    int32_t n_overrides;
    double dt_ms, C_m_pF, tau_m_ms, tau_ref_ms, tau_syn_ms;
    double u_rest_mV, u_reset_mV, u_thr_mV, nu_th_hz, w_ext_mV;
    int64_t n_full[SNN_MAX_POPS];   /* population sizes at scale 1 */
    double k_ext[SNN_MAX_POPS];     /* thalamic in-degree K per neuron */
    double u0_mean_mV[SNN_MAX_POPS], u0_sd_mV[SNN_MAX_POPS];
    double w_mean_mV[SNN_MAX_POPS], w_sd_mV[SNN_MAX_POPS];
    double d_mean_ms[SNN_MAX_POPS], d_sd_ms[SNN_MAX_POPS];
    double conn_p[SNN_MAX_POPS][SNN_MAX_POPS];
    int32_t ovr_source[SNN_MAX_OVERRIDES], ovr_target[SNN_MAX_OVERRIDES];
    double ovr_w_mean_mV[SNN_MAX_OVERRIDES], ovr_w_sd_mV[SNN_MAX_OVERRIDES];
} snn_model;

/*
 * A network given edge by edge instead of sampled from the model (hand-built test
 * circuits, or any user topology).  Neuron dynamics and thalamic drive still come
 * from `model`; neurons [pop_offsets[b], pop_offsets[b+1]) belong to population b
 * (pop_offsets[0] = 0, pop_offsets[model.n_pops] = n_neurons).  Weights are int32
 * counts of 2^-12 pA, delays whole steps in [1, 63], u0 the initial membrane
 * potential relative to rest (mV).
 */
typedef struct snn_custom_net {
    int64_t n_neurons;
    int64_t n_synapses;
    const int32_t *pre;
    const int32_t *post;
    const int32_t *w_fx;
    const uint8_t *delay;
    const float *u0;
    int64_t pop_offsets[SNN_MAX_POPS + 1];
} snn_custom_net;

/* One circuit of a batch: its neuron and in-degree scales (permille) and its seed. */
typedef struct snn_circuit {
    int32_t scale_n_permille;
    int32_t scale_k_permille;
    uint64_t seed;
} snn_circuit;

#define SNN_MAX_CIRCUITS 4096

/*
 * What to simulate.
 *   scale_n_permille / scale_k_permille: population sizes N_b = round_half_up(N_full_b *
 *     scale_n / 1000); pair counts K_ab = round(p[b][a] * (N_full_a * scale_k / 1000) * N_b),
 *     the paper's expected count N_pre N_post p (§2.2);
 *   seed: network, initial-state and thalamic streams (Philox4x64-10);
 *   steps_per_graph: steps captured in one CUDA graph (0 = 1000);
 *   raster_capacity: spikes the device holds between reads (0 = 1<<24);
 *   deliver_blocks: CTAs of the delivery kernel (0 = 2 per SM);
 *   custom: NULL, or an explicit network (then the scales are ignored);
 *   n_circuits / circuits: 0 and NULL for one circuit (scales and seed above); else a
 *     batch of independent circuits of the same model, each with its own scales and
 *     seed, simulated together.  Circuit c occupies neurons [base_c, base_c + N_c) of
 *     one index space (base_c a multiple of 128; the neurons between circuits are
 *     inert) and evolves exactly as it would alone: its synapses, initial state and
 *     thalamic draws use its own seed and circuit-local neuron indices;
 *   n_threads: host threads for network construction (0 = all cores);
 *   engine: how the steps are scheduled; every engine gives the same raster and state:
 *     SNN_ENGINE_PIPELINED (the default): one kernel per step, replayed from a CUDA
 *       graph.  A spike decided at step s depends only on spikes of steps <= s-2
 *       (input reaches U one step after it reaches I), so the kernel of step t
 *       delivers step t's spikes while the same launch finishes step t's current
 *       update and decides step t+1's spikes;
 *     SNN_ENGINE_GRAPH: the two phases of Listing push2 as two kernels per step,
 *       replayed from a CUDA graph;
 *     SNN_ENGINE_PERSISTENT: the pipelined engine's schedule in one cooperative
 *       launch per batch of steps, one bounded grid-wide barrier per step in place
 *       of the kernel boundary;
 *     SNN_ENGINE_RESIDENT: all steps of one snn_step_n call in one cooperative launch
 *       with one CTA per block of consecutive neurons (at most 1024 neurons per SM):
 *       the CTA keeps its neurons' U, I, R in registers and their columns of the ring
 *       in shared memory for the whole launch, and adds the synapses that target its
 *       block (each row is stored grouped by target block, delay order kept within a
 *       block, with a table of where each block's segment starts: the indexed store of
 *       §3.5 split by target) with shared-memory integer atomics; CTAs exchange only
 *       each step's spike list, through per-CTA mailboxes whose words carry the step
 *       number.  One circuit, SNN_RECORD_PLAIN9 records.  smem_ring_rows (8, 16, 32 or
 *       64; 0 = as many as fit) caps the ring rows kept in shared memory; delays of
 *       that many steps or more then go to the ring in global memory.  Every mailbox
 *       wait is bounded (2 s) and ends, on timeout, with SNN_ETIMEOUT at the next read.
 */
#define SNN_ENGINE_DEFAULT 0
#define SNN_ENGINE_GRAPH 1
#define SNN_ENGINE_PERSISTENT 2
#define SNN_ENGINE_PIPELINED 3
#define SNN_ENGINE_RESIDENT 4
/*
 * record_format: how synapses are stored on the device (§3.5 stores a target, a
 * delay and an FP32 weight; §5.3 proposes fewer bits per weight):
 *   SNN_RECORD_PLAIN9:      int32 target, int32 weight (2^-12 pA), uint8 delay: 9 bytes;
 *   SNN_RECORD_PACKED_I8:   uint32 word (target:20 | delay:6 | target population:3 |
 *                           padding flag:1) and an int8 code read back as
 *                           base[a][b] + code * step[a][b] for source population a and
 *                           target population b; per pair, lo/hi = the pair's extreme
 *                           weights, base = lo + (hi - lo) div 2, step = max(1,
 *                           ceil((hi - lo) / 254)), code = clamp(round((w - base) /
 *                           step), -127, 127): 5 bytes;
 *   SNN_RECORD_PACKED_BF16: the same word and the current in pA as bfloat16 (round to
 *                           nearest even): 6 bytes.
 *   SNN_RECORD_BLOCKED6:    target-blocked rows, exact.  The targets are cut into
 *                           blocks of at most 768 consecutive neurons (boundaries at
 *                           multiples of 32, balanced by in-degree, as many as fill whole
 *                           waves of one CTA per SM of the device), each sender's row is
 *                           grouped by block (delay order within a block), and a synapse
 *                           is a uint16 (target - block start : 10 | delay : 6) plus the
 *                           int32 weight: 6 bytes.  Delivery runs one CTA per block, which
 *                           sums the block's events in shared memory before it adds them
 *                           to the ring.  One circuit only; the engine is the graph engine.
 *   SNN_RECORD_BLOCKED4:    the same target-blocked rows with the weight as the bfloat16
 *                           current of SNN_RECORD_PACKED_BF16: every quad of a segment is
 *                           one 16-byte unit (four uint16 records, then four bfloat16
 *                           weights), 4 bytes per synapse.  Same rules as BLOCKED6.
 *   SNN_RECORD_BLOCKED8:    the same target-blocked rows, exact, with weight and record
 *                           interleaved: a synapse is the int32 weight then the uint32
 *                           record (target - block start : 10 | delay : 6), 8 bytes, so a
 *                           segment is one contiguous run of 32-byte quads (one read per
 *                           segment instead of two).  Same rules as BLOCKED6.
 * Packed formats hold up to 2^20 neurons.  The dynamics are the plain ones applied to
 * the read-back weights (unchanged for SNN_RECORD_BLOCKED6 and _BLOCKED8); accumulation
 * stays int32.
 */
#define SNN_RECORD_PLAIN9 0
#define SNN_RECORD_PACKED_I8 1
#define SNN_RECORD_PACKED_BF16 2
#define SNN_RECORD_BLOCKED6 3
#define SNN_RECORD_BLOCKED4 4
#define SNN_RECORD_BLOCKED8 5
typedef struct snn_spec {
    uint32_t abi_version; /* must be SNN_ABI_VERSION */
    int32_t scale_n_permille;
    int32_t scale_k_permille;
    int32_t steps_per_graph;
    uint64_t seed;
    int64_t raster_capacity;
    int32_t deliver_blocks;
    int32_t n_threads;
    int32_t engine;
    int32_t record_format;
    snn_model model;
    const snn_custom_net *custom;
    int32_t n_circuits;
    int32_t smem_ring_rows;
    const snn_circuit *circuits;
} snn_spec;

/* Sizes for a spec.  arena_bytes is the device arena snn_build_network needs
 * (an upper bound: rows are padded after sampling). */
typedef struct snn_sizes {
    uint64_t arena_bytes;
    int64_t n_neurons;
    int64_t n_neurons_padded;     /* ring row stride: n_neurons rounded up to 128 */
    int64_t n_synapses;           /* synapses (exact) */
    int64_t n_synapses_padded_max;
    int64_t raster_capacity;
} snn_sizes;

/* Byte offsets of the device buffers inside the arena (for inspection).  U and R give
 * the buffers that hold the state after the steps enqueued so far (the pipelined
 * engine alternates between two buffers).  Layouts:
 * U, I float[n_neurons_padded]; R uint8[n_neurons_padded] (refractory steps left);
 * ring int32[64][n_neurons_padded]; row_ptr int64[n_neurons+1] into the padded
 * synapse arrays (rows sorted by delay, each padded to a multiple of 4 with entries
 * that deliver nothing); plain records: syn_tgt, syn_w int32[n_synapses_padded],
 * syn_delay uint8[...]; packed records: syn_tgt holds the uint32 words, syn_w the
 * int8 codes or bfloat16 currents, syn_delay is unused; blocked records: row_ptr holds
 * row offsets of quad-padded block segments, syn_tgt the uint16 records (BLOCKED4: the
 * 16-byte quads of records and bfloat16 weights), syn_w the int32 weights (BLOCKED6), syn_delay
 * the uint16 table [n_neurons][target_blocks + 1] of each row's block starts relative
 * to its row start, and blocks the int32 block boundaries [target_blocks + 1];
 * rast_neuron, rast_step int32[raster_capacity].  Resident engine: plain records, each row
 * grouped by target block (delay order kept inside a block), blocks the int32 block
 * boundaries, block_starts the per-row segment table. */
typedef struct snn_layout {
    uint64_t ctl, U, I, R, ring, row_ptr, syn_tgt, syn_w, syn_delay, rast_neuron, rast_step, params;
    int64_t n_neurons_padded;
    int64_t n_synapses_padded;
    uint64_t blocks;
    uint64_t block_starts;  /* resident engine: uint32 [target_blocks][n_neurons], for block b and
                               row i the start of the row's segment of synapses into block b,
                               relative to the row (low 16 bits), and its length (high 16 bits);
                               0 for the other engines */
} snn_layout;

/* Constants and counters of a built network. */
typedef struct snn_info {
    int64_t n_neurons;
    int64_t n_synapses;
    int64_t n_synapses_padded;
    int64_t t;            /* steps enqueued so far */
    int64_t spikes_read;  /* spikes of completed steps moved to the host so far */
    int64_t events_read;  /* recurrent synaptic events (sum of the senders' out-degrees) of those */
    int32_t n_pops;
    int32_t t_ref_steps;
    int64_t pop_offsets[SNN_MAX_POPS + 1];
    double w_f, p11, p22, p21;     /* FP64 constants of §2.2 */
    float p11_f32, p21_f32, p22_f32, theta_f32, u_reset_f32;
    int32_t w_ext_fx;              /* thalamic PSC, 2^-12 pA units */
    uint64_t poisson_thresholds[SNN_MAX_POPS][SNN_POISSON_KMAX];
    int32_t max_row_length;
    int32_t chunks_per_row;
    int32_t steps_per_graph;
    int32_t deliver_blocks;
    uint32_t device_error;         /* sticky device error bits (1 = raster overflow, 2 = barrier timeout) */
    int32_t engine;                /* SNN_ENGINE_PIPELINED, _GRAPH, _PERSISTENT or _RESIDENT */
    int32_t record_format;         /* SNN_RECORD_* */
    int32_t bytes_per_synapse;     /* device bytes of one synapse record */
    int32_t n_circuits;            /* 1, or the batch size */
    int32_t schedule_ctas;         /* CTAs of the step (pipelined, persistent) or delivery (graph) kernel */
    int32_t schedule_delivery_warps; /* pipelined and persistent engines: delivery warps per CTA */
    int32_t target_blocks;         /* blocked records or the resident engine: number of target blocks (else 0) */
    int32_t i8_base[SNN_MAX_POPS][SNN_MAX_POPS];  /* SNN_RECORD_PACKED_I8 read-back tables [source][target] */
    int32_t i8_step[SNN_MAX_POPS][SNN_MAX_POPS];
    int32_t circuits_per_group;    /* batches: see snn_set_circuit_groups (0 = one group) */
    int32_t reserved3;
    char last_error[256];          /* message of this handle's last failed call ("" if none; truncated) */
} snn_info;

typedef struct snn_net snn_net;

/* Host only (no GPU needed).  Validates `spec` and fills `out`: the neuron and synapse
 * counts of §2.2's sizing rules (population sizes N_b and pair counts N_pre N_post p at
 * the spec's scales) and the arena bytes of every buffer.  No passage of its own: ABI
 * helper.  Errors: SNN_EINVAL for an invalid spec (message via snn_last_error). */
int snn_query_sizes(const snn_spec *spec, snn_sizes *out);

/* Builds the network on the host (constants of §2.2 in FP64; every synapse of
 * every population pair drawn with replacement, §2.2; rows grouped by sender and
 * sorted by delay, the indexed store of §3.5), uploads it into the caller's device
 * arena on `cuda_stream`, initialises U from the u_init Gaussians, I = R = 0, the
 * ring to zero, and captures the step loop into a CUDA graph (graph and pipelined
 * engines; the persistent engine launches its steps directly).  Returns when the
 * upload is complete.  On success *out owns host-side state; free it with
 * snn_destroy.  Errors: SNN_EINVAL (spec), SNN_ENOMEM (host memory, or arena_bytes
 * below snn_query_sizes' figure), SNN_ECUDA. */
int snn_build_network(const snn_spec *spec, void *dev_arena, uint64_t arena_bytes, void *cuda_stream,
                      snn_net **out);

/* Host only (no GPU, no device memory): builds the network of `spec` exactly as
 * snn_build_network does (§2.2 sampling; the indexed store of §3.5: rows grouped by
 * sender and sorted by delay) and copies it, without the row padding, into caller
 * arrays: row_ptr[N + 1] (row i is row_ptr[i] .. row_ptr[i + 1]), post[S] (target
 * neuron), w_fx[S] (weight, 2^-12 pA units), delay[S] (steps) and u0[N] (initial
 * potential, mV relative to rest), with N = snn_sizes.n_neurons and S =
 * snn_sizes.n_synapses.  Any output may be NULL to skip it.  For the packed formats
 * (SNN_RECORD_PACKED_I8 / _BF16) the fields are decoded from the packed words and w_fx
 * is the weight the kernels read back (the per-pair affine code, or the bfloat16
 * current rounded to 2^-12 pA).  Errors: SNN_EINVAL (spec, or a blocked format),
 * SNN_ENOMEM. */
int snn_export_network(const snn_spec *spec, int64_t *row_ptr, int32_t *post, int32_t *w_fx, uint8_t *delay,
                       float *u0);

/* Enqueues n_steps steps (Listing push / push2 of §3.1; one step = dt) on
 * `cuda_stream` and returns without waiting.  n_steps = 0 is a no-op.
 * Errors: SNN_EINVAL (n_steps < 0), SNN_ESTATE (after a sticky device error),
 * SNN_ECUDA.  A persistent-engine barrier that waits longer than 2 s records a device
 * error that the next read reports as SNN_ETIMEOUT. */
int snn_step_n(snn_net *net, int64_t n_steps, void *cuda_stream);

/* Waits for the enqueued steps, moves the device raster to the host and returns
 * spikes not yet returned, ordered by (step, neuron).  steps/neurons are
 * caller-allocated arrays of `capacity` entries; *n_written receives how many were
 * written (the rest stay for the next call).  With steps == neurons == NULL it only
 * reports the number of unread spikes.  Errors: SNN_EOVERFLOW if the raster filled
 * between reads (the dynamics after that point are invalid), SNN_ETIMEOUT if a
 * persistent-engine barrier timed out, SNN_ECUDA. */
int snn_read_spikes(snn_net *net, int64_t *steps, int32_t *neurons, int64_t capacity, int64_t *n_written);

/* Overlapped reads: like snn_read_spikes, but waits only for the steps enqueued before
 * the most recent snn_step_n call and returns spikes of those steps; the most recent
 * call's steps may still be running.  A loop of { snn_step_n; snn_collect_spikes } thus
 * moves one batch of spikes to the host while the GPU computes the next; a final
 * snn_read_spikes returns the rest.  Spikes are returned once, by whichever call reads
 * them first, ordered by (step, neuron).  With steps == neurons == NULL it only reports
 * the number available.  When the device raster is more than a quarter full it waits
 * for every enqueued step (as snn_read_spikes), since the raster is only reset while the
 * device is idle: raster_capacity should hold three calls' spikes.  Errors: as
 * snn_read_spikes; a pending device error is reported. */
int snn_collect_spikes(snn_net *net, int64_t *steps, int32_t *neurons, int64_t capacity, int64_t *n_written);

/* Waits for the enqueued steps and returns the mean firing rate (Hz) of each
 * population over steps [t_begin, t_end) (§4.1's rate statistic), from all spikes
 * recorded so far (pooled over the circuits of a batch).  pop_rates_hz has n_pops entries; neuron_counts (n_neurons
 * entries, may be NULL) receives per-neuron spike counts in the window.
 * Errors: SNN_EINVAL (empty or negative window), SNN_EOVERFLOW, SNN_ECUDA. */
int snn_read_rates(snn_net *net, int64_t t_begin, int64_t t_end, double *pop_rates_hz, int32_t *neuron_counts);

/* Fills `out` with the network's constants (the FP64 and FP32 propagators of §2.2, the
 * thalamic Poisson tables) and counters (host only, no wait).  No passage of its own:
 * ABI helper.  Errors: SNN_EINVAL (null argument). */
int snn_get_info(const snn_net *net, snn_info *out);

/* Changes the launch schedule of the step kernels and re-captures the step graph
 * (waits for enqueued steps first): grid_ctas = CTAs of the step kernel (pipelined) or
 * of the delivery kernel (graph engine; SNN_RECORD_BLOCKED6 keeps one CTA per target
 * block), delivery_warps = delivery warps per CTA
 * (pipelined, 1..8; resident: even, two teams of at least blocks/32 warps, at most 16
 * warps with the neuron warps), steps_per_graph as in
 * snn_spec; 0 keeps a value.  The schedule never changes results, only speed (see
 * paper_2405_02019_gb300.autotune).
 * Errors: SNN_EINVAL (out of range), SNN_ENOTSUP (persistent engine; grid_ctas on the
 * resident engine, which runs one CTA per target block), SNN_ECUDA. */
int snn_set_schedule(snn_net *net, int32_t grid_ctas, int32_t delivery_warps, int32_t steps_per_graph);

/* Batched networks on the graph or pipelined engine: runs the circuits in groups of
 * `circuits_per_group` consecutive circuits (0, or at least n_circuits, = one group) and
 * re-captures the step graph (waits for enqueued steps first).  Every run of steps
 * (a graph replay, or the steps one snn_step_n launches directly) is taken group by
 * group: the first group's circuits take all the run's steps, then the next group's,
 * and so on.  Circuits never interact, so results do not change; each group's ring and
 * neuron state then stay in L2 through the run (a whole 32-circuit batch's ring is
 * larger than L2).  On the pipelined engine each group has its own spike queues; the
 * spikes already decided for the next step move to the new groups' queues (a host
 * round trip of one count and a few hundred entries per group), so the grouping may
 * change between any two steps.  A group takes the step grid and delivery warps of
 * snn_set_schedule where those were set, else the default for its own size.
 * Errors: SNN_EINVAL (negative), SNN_ENOTSUP (persistent engine), SNN_ESTATE (a device
 * error is pending), SNN_ECUDA. */
int snn_set_circuit_groups(snn_net *net, int32_t circuits_per_group);

/* Batched networks: the first neuron and the neuron count of every circuit (host
 * arrays of n_circuits entries).  A single circuit reports base 0 and N. */
int snn_get_circuits(const snn_net *net, int64_t *base, int64_t *n_neurons);

/* Copies every neuron's out-degree (synapses in its row, padding excluded) into the
 * host array out[n_neurons] (host only). */
int snn_get_out_degrees(const snn_net *net, int32_t *out);

/* Fills `out` with the arena layout (host only). */
int snn_get_layout(const snn_net *net, snn_layout *out);

/* Runs n_steps steps kernel by kernel (no graph), timing each kernel with CUDA
 * events on `cuda_stream`, and returns after they finish.  ms_update / ms_deliver
 * receive the summed milliseconds of the update and delivery kernels (pipelined
 * engine: of its one step kernel in ms_update, 0 in ms_deliver).  Same dynamics as
 * snn_step_n.  Errors as snn_step_n. */
int snn_profile_steps(snn_net *net, int64_t n_steps, void *cuda_stream, double *ms_update, double *ms_deliver);

/* Checkpoint of the dynamic state after the steps enqueued so far (waits for them):
 * neuron state, ring, control block and (pipelined engine) the next step's queued
 * spikes, as one host byte blob.  With host_buf == NULL only *written (the size) is
 * set.  Spikes recorded so far are first moved to the host history (read them with
 * snn_read_spikes as usual).  The network itself and the seed are not saved: resume
 * on a handle built from the same spec.  Because every random draw is counter-based
 * on (seed, step, neuron), a resumed run reproduces the uninterrupted one bit for bit.
 * Errors: SNN_ENOMEM (capacity < size), SNN_ECUDA, plus pending device errors. */
int snn_save_state(snn_net *net, void *host_buf, uint64_t capacity, uint64_t *written);

/* Restores a blob from snn_save_state into `net` (same spec; checked by shape and
 * engine), including the step counter; the host spike history starts empty.  A blob
 * saved under another circuit grouping (snn_set_circuit_groups) loads into the current
 * one.
 * Errors: SNN_EINVAL (not a state blob, or another shape/engine), SNN_ECUDA. */
int snn_load_state(snn_net *net, const void *host_buf, uint64_t bytes);

/* Phase 2 of Listing push2 (§3.1) alone, for measurement and tests: adds every
 * synapse of the senders spikers[0 .. n_spikers) (device int32 neuron ids, each
 * below n_neurons; repeats allowed) into the ring as spikes of step t, i.e.
 * W[(t + d) mod 64][target] += w, in one launch of `blocks` CTAs (0 = full
 * occupancy; the blocked formats and the resident engine's block-major records always
 * launch one CTA per target block, which reads only its block's segments) on
 * `cuda_stream`; returns without waiting.  The ring keeps the added
 * input, so the simulated dynamics change accordingly.
 * Errors: SNN_EINVAL (null or negative arguments), SNN_ECUDA. */
int snn_deliver_spikes(snn_net *net, const int32_t *spikers, int64_t n_spikers, int64_t t, int32_t blocks,
                       void *cuda_stream);

/* Releases host-side state (not the caller's arena).  NULL is ignored.  No passage:
 * ABI helper. */
void snn_destroy(snn_net *net);

/*
 * One simulation step that allocates no device memory (the paper has no counterpart:
 * this is an embedding aid, not part of the method).
 *
 * For callers that may not call cudaMalloc -- a host application whose own allocator
 * owns all device memory and does not let plug-ins allocate, or a control loop that
 * cannot afford an allocation failing or stalling mid-run.  The caller passes every
 * input and output buffer; the step's internal spike list and counter live in one
 * fixed array inside the library (SNN_STATIC_MAX_NEURONS + 64 words, about 512 KB),
 * which every GPU that loads the library holds until the process exits.
 *
 * Computes exactly one step `t` (0-based step index; the handle's own step counter is
 * neither read nor advanced) of the network built as `net` (its constants, Poisson
 * tables and population offsets), bit-identical to a step of snn_step_n:
 *   io->row_ptr[n+1], syn_tgt/syn_w/syn_delay: the network in the layout of
 *     snn_layout (rows padded to multiples of 4; syn_tgt/syn_w 16-byte aligned,
 *     syn_delay 4-byte aligned); read only;
 *   io->U, io->I (float), io->R (uint8): at least n rounded up to 4 entries, 16-byte
 *     (R: 4-byte) aligned; read and written;
 *   io->ring: int32 [64][ring_stride], ring_stride >= n, multiple of 4; read and written;
 *   io->spikes: int32 [n] device output, this step's spiking neurons (unordered);
 *   io->n_spikes: one int32 device output, their count.
 * `seed` is the thalamic stream's seed (the spec's seed for parity with snn_step_n).
 * Enqueued on `cuda_stream`; returns without waiting.
 *
 * Every call looks up the device address of the fixed array (cudaGetSymbolAddress, with
 * the buffers' device current); the first call on a device also loads the library's
 * device code there, so make it before any stream capture.  Every call reuses the same
 * array and clears its counter first, so calls whose work overlaps on the GPU
 * (different streams, or different handles at the same time) race and give wrong
 * results: serialise them.
 * When io points into the handle's own arena (as snn_get_layout gives it), the handle's
 * step counter, raster and pending-spike queue do not follow these steps: after
 * snn_step_static has run on that arena, do not step the handle with snn_step_n nor
 * save it with snn_save_state (the pipelined engine would deliver its queued spikes
 * again and recompute a step on state that has moved on).
 * Errors: SNN_EINVAL for more than SNN_STATIC_MAX_NEURONS neurons, a missing or
 * misaligned buffer, a negative t; SNN_ENOTSUP for a network with packed synapse
 * records (this step reads plain records as rows), a batch of circuits or the resident
 * engine (whose records are stored block-major); SNN_ESTATE after a
 * device error of the network; SNN_ECUDA on a failed CUDA call, or when a CUDA error
 * of earlier work is pending (it is left for the caller to read).
 */
#define SNN_STATIC_MAX_NEURONS 131072
typedef struct snn_static_io {
    const int64_t *row_ptr;
    const int32_t *syn_tgt;
    const int32_t *syn_w;
    const uint8_t *syn_delay;
    float *U;
    float *I;
    uint8_t *R;
    int32_t *ring;
    int64_t ring_stride;
    int32_t *spikes;
    int32_t *n_spikes;
} snn_static_io;

int snn_step_static(const snn_net *net, const snn_static_io *io, uint64_t seed, int64_t t, void *cuda_stream);

/* Static description of a status code.  No passage: ABI helper. */
const char *snn_strerror(int code);

/* Message of the calling thread's last failed call ("" if none); the same message is
 * also kept per handle for calls that take one (snn_info.last_error).  No passage: ABI
 * helper. */
const char *snn_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SNN_H */
