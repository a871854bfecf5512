// Device side of the simulation step (sm_103a).
//
// Phase 1 (Listing push of §3.1, fused with the ring read of §3.2 and the spike queue
// of Listing push2), for every neuron:
//     in   = W[t mod 64][i] + T(t, i) * w_ext      (int32, 2^-12 pA units)
//     W[t mod 64][i] = 0
//     if R == 0: x = p22 U + p21 I; spike if x >= theta (then x = reset, R = t_ref); U = x
//     else:      U = reset; R -= 1
//     I = p11 I + in * 2^-12
// T is Poisson(nu_th K dt) by CDF inversion of one Philox word (§2.2).  Spikers are
// compacted warp by warp (one atomic per warp with spikes) into the raster, which is
// also the step's spike queue.
// Phase 2 (Listing push2 of §3.1): every queued spiker's row (sorted by delay, §3.5)
// is cut into runs of 256-synapse chunks; a warp streams a chunk with 16-byte loads and
// adds each weight into W[(t + d) mod 64][target] with a fire-and-forget int32
// reduction, so the order of delivery cannot change the result.
//
// Three engines run these phases (every one gives the same raster):
//   k_step               -- pipelined (default): one kernel per step delivers step t's
//                           spikes while it finishes step t's update and decides step
//                           t+1's spikes (a spike at s depends only on spikes <= s-2);
//                           replayed from a CUDA graph with programmatic launch
//                           (batches may run in circuit groups);
//   k_update + k_deliver -- one kernel per phase, replayed from a CUDA graph (batches
//                           may run in circuit groups: k_update takes a neuron range);
//   k_persistent         -- the pipelined schedule in one cooperative launch for a
//                           batch of steps, one grid-wide barrier per step whose
//                           spin-wait is bounded (on timeout the kernel records an
//                           error and exits).
// k_deliver_list delivers a given sender list (measurement and tests); blocked records
// (target-blocked rows) have their own phase 2, k_deliver_blocked, at the end of this
// file.
//
// No FMA in the neuron arithmetic: __fmul_rn / __fadd_rn round every product and sum
// on its own, which is what makes the raster reproducible bit for bit.
#include <cuda_runtime.h>

#include "internal.hpp"
#include "philox.cuh"

namespace snn {

namespace {

__device__ __forceinline__ void red_add_s32(int32_t *addr, int32_t v)
{
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t v;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
    return v;
}

// Streaming 16-byte load of read-once data (evict-first in L1/L2).
__device__ __forceinline__ int4 ld_stream4(const int32_t *p) { return __ldcs(reinterpret_cast<const int4 *>(p)); }
__device__ __forceinline__ uint32_t ld_stream_u32(const uint8_t *p)
{
    return __ldcs(reinterpret_cast<const unsigned int *>(p));
}

// Global warp number with consecutive numbers on consecutive CTAs, so that a short
// list of work items spreads over all SMs instead of filling the first CTAs.
__device__ __forceinline__ int64_t spread_warp()
{
    return static_cast<int64_t>(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
}

__device__ __forceinline__ void red_release_add_u32(uint32_t *addr, uint32_t v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(addr), "r"(v) : "memory");
}

struct SharedTables {
    uint64_t thr[SNN_MAX_POPS * kPK];
};

__device__ __forceinline__ void stage_tables(const StepArgs &a, SharedTables &s)
{
    for (int j = threadIdx.x; j < SNN_MAX_POPS * kPK; j += blockDim.x) s.thr[j] = (&a.tables->thresholds[0][0])[j];
    __syncthreads();
}

__device__ __forceinline__ int32_t neuron_step(const StepArgs &a, float &u, float &cur, uint32_t &r, int32_t in)
{
    int32_t spike = 0;
    if (r == 0u) {
        float x = __fadd_rn(__fmul_rn(a.p22, u), __fmul_rn(a.p21, cur));
        if (x >= a.theta) {
            spike = 1;
            x = a.u_reset;
            r = static_cast<uint32_t>(a.t_ref);
        }
        u = x;
    } else {
        u = a.u_reset;
        r -= 1u;
    }
    cur = __fadd_rn(__fmul_rn(a.p11, cur), __fmul_rn(__int2float_rn(in), 0x1p-12f));
    return spike;
}

// Phase 1 for neurons 4q .. 4q+3 (those below n).  The ring row is read through L2
// (other SMs add into it between steps).
__device__ __forceinline__ void update_quad(const StepArgs &a, const SharedTables &s, int64_t t, int64_t q,
                                            int32_t spk[4])
{
    const int64_t i0 = q * 4;
    const int64_t slot = t & kDMask;
    float4 u4 = *reinterpret_cast<const float4 *>(a.U + i0);
    float4 c4 = *reinterpret_cast<const float4 *>(a.I + i0);
    const uint32_t r4 = *reinterpret_cast<const uint32_t *>(a.R + i0);
    int32_t *wrow = a.ring + slot * a.npad + i0;
    const int4 w4 = __ldcg(reinterpret_cast<const int4 *>(wrow));
    *reinterpret_cast<int4 *>(wrow) = make_int4(0, 0, 0, 0);
    const CircuitInfo ci = a.circuits[a.group_circuit[i0 >> 7]];
    const uint32_t pops = *reinterpret_cast<const uint32_t *>(a.pop_id + i0);
    const Block4 rnd = philox4x64_10(static_cast<uint64_t>(t), static_cast<uint64_t>((i0 - ci.base) >> 2), 0, 0,
                                     ci.seed, kStreamThalamic);
    float uu[4] = {u4.x, u4.y, u4.z, u4.w};
    float cc[4] = {c4.x, c4.y, c4.z, c4.w};
    const int32_t ww[4] = {w4.x, w4.y, w4.z, w4.w};
    uint32_t rr[4] = {r4 & 0xFFu, (r4 >> 8) & 0xFFu, (r4 >> 16) & 0xFFu, r4 >> 24};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t i = i0 + j;
        if (i < ci.base + ci.n) {
            const int b = (pops >> (8 * j)) & 0xFF;
            const uint64_t v = rnd.w[j] >> 1;
            const uint64_t *thr = s.thr + b * kPK;
            uint32_t T = 0;
            while (T < static_cast<uint32_t>(kPK) && v >= thr[T]) ++T;
            const int32_t in =
                static_cast<int32_t>(static_cast<uint32_t>(ww[j]) + T * static_cast<uint32_t>(a.w_ext_fx));
            spk[j] = neuron_step(a, uu[j], cc[j], rr[j], in);
        }
    }
    *reinterpret_cast<float4 *>(a.U + i0) = make_float4(uu[0], uu[1], uu[2], uu[3]);
    *reinterpret_cast<float4 *>(a.I + i0) = make_float4(cc[0], cc[1], cc[2], cc[3]);
    *reinterpret_cast<uint32_t *>(a.R + i0) = rr[0] | (rr[1] << 8) | (rr[2] << 16) | (rr[3] << 24);
}

// Warp-collective (every lane must call): append the warp's spikers to the raster.
__device__ __forceinline__ void append_spikes(const StepArgs &a, int64_t t, int64_t i0, const int32_t spk[4])
{
    const int lane = threadIdx.x & 31;
    const int cnt = spk[0] + spk[1] + spk[2] + spk[3];
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (total == 0) return;
    uint32_t base = 0;
    if (lane == 31) base = atomicAdd(&a.ctl->cursor, static_cast<uint32_t>(total));
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    uint32_t pos = base + static_cast<uint32_t>(incl - cnt);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (spk[j]) {
            if (pos < a.rast_cap) {
                a.rast_nrn[pos] = static_cast<int32_t>(i0 + j);
                a.rast_t[pos] = static_cast<int32_t>(t);
            } else {
                atomicOr(&a.ctl->err, kErrRaster);
            }
            ++pos;
        }
    }
}

// One 256-synapse chunk [off, min(off + 256, re)) of a row whose sender belongs to
// population src_pop: each lane takes two quads, loads them with 16-byte streaming
// loads and adds every weight into W[(slot + d) mod 64][target].  FMT selects the
// record format; the padding entries of a row deliver nothing.
template <int FMT>
__device__ __forceinline__ void deliver_chunk(const StepArgs &a, int64_t slot, int64_t off, int64_t re, int src_pop)
{
    const int lane = threadIdx.x & 31;
    int32_t *const ring = a.ring;
    const int64_t npad = a.npad;
    int4 tg[2];
    int4 wv[2];
    uint32_t dv[2];
    uint2 hv[2];
    bool ok[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int64_t o = off + u * 128 + lane * 4;
        ok[u] = o < re;
        if (ok[u]) {
            tg[u] = ld_stream4(a.syn_tgt + o);
            if (FMT == SNN_RECORD_PLAIN9) {
                wv[u] = ld_stream4(a.syn_w + o);
                dv[u] = ld_stream_u32(a.syn_d + o);
            } else if (FMT == SNN_RECORD_PACKED_I8) {
                dv[u] = ld_stream_u32(reinterpret_cast<const uint8_t *>(a.syn_w) + o);
            } else {
                hv[u] = __ldcs(reinterpret_cast<const uint2 *>(reinterpret_cast<const uint16_t *>(a.syn_w) + o));
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        if (!ok[u]) continue;
        const int32_t tt[4] = {tg[u].x, tg[u].y, tg[u].z, tg[u].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            int32_t w, target;
            int64_t d;
            if (FMT == SNN_RECORD_PLAIN9) {
                const int32_t wq[4] = {wv[u].x, wv[u].y, wv[u].z, wv[u].w};
                w = wq[e];
                target = tt[e];
                d = (dv[u] >> (8 * e)) & 0xFFu;
            } else {
                const uint32_t word = static_cast<uint32_t>(tt[e]);
                if (word & kWordPad) continue;
                target = static_cast<int32_t>(word & kWordTargetMask);
                d = (word >> kWordDelayShift) & 63u;
                const int b = static_cast<int>((word >> kWordPopShift) & 7u);
                if (FMT == SNN_RECORD_PACKED_I8) {
                    const int2 pq = __ldg(reinterpret_cast<const int2 *>(&a.tables->i8_pair[src_pop][b]));
                    const int32_t code = static_cast<int8_t>((dv[u] >> (8 * e)) & 0xFFu);
                    w = pq.x + code * pq.y;
                } else {
                    const uint32_t h = e < 2 ? (hv[u].x >> (16 * e)) : (hv[u].y >> (16 * (e - 2)));
                    w = __float2int_rn(__fmul_rn(__uint_as_float((h & 0xFFFFu) << 16), 4096.0f));
                }
            }
            if (w != 0) red_add_s32(ring + ((slot + d) & kDMask) * npad + target, w);
        }
    }
}

// Phase 2 for the spikers list[0 .. nspk), work items grid-strided over warps:
// item = (spiker, 256-synapse chunk of its row).
// Items per spike when nspk spikes share nwarps warps: enough to keep every warp busy
// while there are few spikes (one 256-synapse chunk per item), fewer and longer items
// (consecutive chunks of one row) when spikes outnumber warps.
__device__ __forceinline__ int64_t items_per_spike(int64_t cpr, int64_t nspk, int64_t nwarps)
{
    const int64_t ipj = nspk > 0 ? nwarps / nspk : cpr;
    return ipj < 1 ? 1 : (ipj > cpr ? cpr : ipj);
}

template <int FMT>
__device__ __forceinline__ void deliver_list_fmt(const StepArgs &a, int64_t t, const int32_t *list, int64_t nspk,
                                                 int64_t warp, int64_t nwarps)
{
    const int64_t cpr = a.chunks_per_row;
    const int64_t ipj = items_per_spike(cpr, nspk, nwarps);
    const int64_t per = (cpr + ipj - 1) / ipj;  // chunks per item
    const int64_t items = nspk * ipj;
    for (int64_t it = warp; it < items; it += nwarps) {
        const int64_t j = it / ipj;
        const int64_t part = it - j * ipj;
        const int32_t s = __ldcg(list + j);
        const int64_t rs = a.row_ptr[s];
        const int64_t re = a.row_ptr[s + 1];
        const int src = FMT == SNN_RECORD_PACKED_I8 ? __ldg(a.pop_id + s) : 0;
        for (int64_t c = part * per, off = rs + c * kChunk; c < (part + 1) * per && off < re; ++c, off += kChunk)
            deliver_chunk<FMT>(a, t, off, re, src);
    }
}

__device__ __forceinline__ void deliver_list(const StepArgs &a, int64_t t, const int32_t *list, int64_t nspk,
                                             int64_t warp, int64_t nwarps)
{
    if (a.format == SNN_RECORD_PACKED_I8) deliver_list_fmt<SNN_RECORD_PACKED_I8>(a, t, list, nspk, warp, nwarps);
    else if (a.format == SNN_RECORD_PACKED_BF16) deliver_list_fmt<SNN_RECORD_PACKED_BF16>(a, t, list, nspk, warp, nwarps);
    else deliver_list_fmt<SNN_RECORD_PLAIN9>(a, t, list, nspk, warp, nwarps);
}

__global__ void __launch_bounds__(kUpdateThreads) k_update(const StepArgs a, const int k)
{
    __shared__ SharedTables s;
    stage_tables(a, s);
    const int64_t t = a.ctl->t_base + k;
    const int64_t q = a.quad_base + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    int32_t spk[4] = {0, 0, 0, 0};
    if (q * 4 < a.n) update_quad(a, s, t, q, spk);
    append_spikes(a, t, q * 4, spk);
}

__global__ void __launch_bounds__(kDeliverThreads) k_deliver(const StepArgs a, const int k)
{
    const int64_t t = a.ctl->t_base + k;
    const uint32_t cur = a.ctl->cursor;
    const uint32_t begin = a.ctl->step_begin[t & 1];
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->step_begin[(t + 1) & 1] = cur;
    const uint32_t end = cur < a.rast_cap ? cur : a.rast_cap;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const int64_t nspk = end > begin ? static_cast<int64_t>(end - begin) : 0;
    deliver_list(a, t, a.rast_nrn + begin, nspk, spread_warp(), nwarps);
}

// Phase 2 alone for a caller-given list of senders (measurement and tests).
__global__ void __launch_bounds__(kDeliverThreads) k_deliver_list(const StepArgs a, const int32_t *list,
                                                                  const int64_t n, const int64_t t)
{
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    deliver_list(a, t, list, n, spread_warp(), nwarps);
}

__global__ void k_advance(Ctl *ctl, int64_t m) { ctl->t_base += m; }

// Circuit groups run the same steps one group after another: the next group's first
// step appends its spikes from where the raster ends now.
__global__ void k_resync(Ctl *ctl) { ctl->step_begin[ctl->t_base & 1] = ctl->cursor; }

// Grid-wide barrier of a cooperative launch: the `index`-th barrier of the launch
// waits until all gridDim.x blocks have arrived index times.  The wait is bounded by
// a.barrier_timeout_ns; on timeout the error bit is set (which releases every other
// waiting block too) and false returned.
__device__ __forceinline__ bool grid_barrier(const StepArgs &a, Ctl *ctl, uint32_t index)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        // the CTA barrier above orders the block's writes before this release
        red_release_add_u32(&ctl->bar, 1u);
        const uint32_t target = index * gridDim.x + a.barrier_extra;
        if (ld_acquire_u32(&ctl->bar) < target) {
            const uint64_t t0 = global_ns();
            uint32_t spins = 0;
            while (ld_acquire_u32(&ctl->bar) < target) {
                if ((++spins & 255u) == 0 && global_ns() - t0 > a.barrier_timeout_ns) {
                    atomicOr(&ctl->err, kErrTimeout);
                    ok = 0;
                    break;
                }
                if ((spins & 63u) == 0 && (ld_acquire_u32(&ctl->err) & kErrTimeout)) {
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------------------
// Pipelined engine: one kernel per step.
//
// In the recurrence a spike decided at step s uses I after step s-1, which already
// holds W[s-1]; W[s-1] only receives spikes of steps <= s-2.  So the spike decision
// of step t+1 (A(t+1)) needs the current update of step t (B(t): I <- p11 I + W[t] +
// T w_ext) but not the delivery of step t's spikes (D(t), which writes slots t+1 ..
// t+63 and is read from step t+1 on).  Kernel K_t therefore runs, concurrently:
//   neuron warps:   B(t) then A(t+1) for their neurons (same thread, program order);
//   delivery warps: D(t) for the spikes of step t decided by K_{t-1}.
// Each neuron still sees A(0), B(0), A(1), B(1), ... in order, so the arithmetic is
// the same as the two-phase engines.  U and R after A(s) live in buffer s mod 2 (the
// state after s steps is in buffer (s-1) mod 2).
//
// Spike queue of step s (buffer s mod 4, count qcount[s mod 4]): a warp with
// spikers reserves room with one atomic and writes their entries (row bounds were
// loaded with the neuron state).  A batch in circuit groups runs one launch per group
// and step; the group's launch covers only its own groups of 128 neurons, and its
// queues and counts are its own (queue region from the group's first neuron, counts
// in the group's slot of the count array), so the groups' kernels are independent.  The rows are prefetched into L2 for the next
// kernel.  A delivery warp loads the step's spike count and the entry of its first
// item in the same round trip, then the synapses; the warp delivering chunk 0 of spike
// j records it at raster position base + j, the raster base advancing once per step
// (Ctl::step_begin[t mod 2]).  Every buffer choice depends on t mod 64 only, which the
// launch passes in (`ph`).
// ---------------------------------------------------------------------------

__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Poisson count T = #{k : v >= thr[k]} (thresholds nondecreasing): the first eight
// thresholds of the quad's population come in registers, the rest from memory.
__device__ __forceinline__ uint32_t poisson_count(uint64_t v, const uint64_t (&r)[8], const uint64_t *thr_row)
{
    uint32_t T = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) T += (v >= r[k]) ? 1u : 0u;
    if (T == 8u)
        while (T < static_cast<uint32_t>(kPK) && v >= __ldg(thr_row + T)) ++T;
    return T;
}

// Waits until the previous kernel of the stream has completed and its writes are
// visible (a no-op unless this launch was made programmatic).
__device__ __forceinline__ void wait_previous_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_next_grid() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Neuron part for quad q = 32 g + lane: B(t) (unless do_b is false: the first kernel,
// t = -1) then A(t+1).  Warp-collective: every lane of group g must call it (lanes
// without a quad pass valid = false).  Everything that does not depend on the
// previous step (row bounds, Poisson thresholds, the Philox block) is done before
// `wait_first` (if set) waits for the previous kernel.
// A launch of one circuit group (kGroup) takes its queue counts, queue size and first
// group of 128 neurons from the arguments; a launch over the whole index space uses the
// control block's counts, npad entries per queue and group 0.  The two are separate
// instantiations, so that the whole-network kernel carries none of the group indirection.
template <bool kGroup>
__device__ __forceinline__ uint32_t *queue_counts(const StepArgs &a)
{
    return kGroup ? a.qcount : a.ctl->qcnt;
}
template <bool kGroup>
__device__ __forceinline__ int64_t queue_entries(const StepArgs &a)
{
    return kGroup ? a.queue_cap : a.npad;
}
template <bool kGroup>
__device__ __forceinline__ int64_t first_quad_warp(const StepArgs &a)
{
    return kGroup ? (a.quad_base >> 5) : 0;
}

template <bool kGroup>
__device__ __forceinline__ void pipe_quad(const StepArgs &a, const int64_t &t, int ph, int64_t g, bool valid,
                                          bool do_b, bool wait_first)
{
    const int lane = threadIdx.x & 31;
    const int64_t q = g * 32 + lane;
    const int64_t i0 = q * 4;
    const int phn = ph + 1;  // phase of the step whose spikes are decided here
    int32_t spk[4] = {0, 0, 0, 0};
    int64_t rp[5] = {0, 0, 0, 0, 0};
    // independent of the previous step: network, tables, circuit, random numbers
    uint64_t tr[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    Block4 rnd = {{0, 0, 0, 0}};
    int b0 = 0;
    uint32_t pops = 0;
    int64_t end_valid = 0;  // neurons of the quad's circuit end here
    const uint64_t *thr0 = a.tables->thresholds[0];
    if (valid) {
        const longlong2 rpa = __ldg(reinterpret_cast<const longlong2 *>(a.row_ptr + i0));
        const longlong2 rpb = __ldg(reinterpret_cast<const longlong2 *>(a.row_ptr + i0 + 2));
        const int64_t rpc = __ldg(a.row_ptr + i0 + 4);
        rp[0] = rpa.x; rp[1] = rpa.y; rp[2] = rpb.x; rp[3] = rpb.y; rp[4] = rpc;
        const CircuitInfo ci = a.circuits[__ldg(a.group_circuit + g)];
        end_valid = ci.base + ci.n;
        pops = __ldg(reinterpret_cast<const unsigned int *>(a.pop_id + i0));
        b0 = pops & 0xFF;
        thr0 = &a.tables->thresholds[b0][0];
        if (do_b) {
#pragma unroll
            for (int k = 0; k < 8; k += 2) {
                const ulonglong2 v2 = __ldg(reinterpret_cast<const ulonglong2 *>(thr0 + k));
                tr[k] = v2.x;
                tr[k + 1] = v2.y;
            }
            rnd = philox4x64_10(static_cast<uint64_t>(t), static_cast<uint64_t>((i0 - ci.base) >> 2), 0, 0, ci.seed,
                                kStreamThalamic);
        }
    }
    if (wait_first) wait_previous_grid();
    if (valid) {
        const float *Uin = (ph & 1) ? a.U2 : a.U;
        const uint8_t *Rin = (ph & 1) ? a.R2 : a.R;
        float *Uout = (phn & 1) ? a.U2 : a.U;
        uint8_t *Rout = (phn & 1) ? a.R2 : a.R;
        // the state of the quad, in one round trip
        const float4 u4 = *reinterpret_cast<const float4 *>(Uin + i0);
        const float4 c4 = *reinterpret_cast<const float4 *>(a.I + i0);
        const uint32_t r4 = *reinterpret_cast<const uint32_t *>(Rin + i0);
        int32_t *wrow = a.ring + (ph & kDMask) * a.npad + i0;
        int4 w4 = make_int4(0, 0, 0, 0);
        if (do_b) w4 = __ldcg(reinterpret_cast<const int4 *>(wrow));
        float uu[4] = {u4.x, u4.y, u4.z, u4.w};
        float cc[4] = {c4.x, c4.y, c4.z, c4.w};
        uint32_t rr[4] = {r4 & 0xFFu, (r4 >> 8) & 0xFFu, (r4 >> 16) & 0xFFu, r4 >> 24};
        if (do_b) {
            *reinterpret_cast<int4 *>(wrow) = make_int4(0, 0, 0, 0);
            const int32_t ww[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t i = i0 + j;
                if (i < end_valid) {
                    const int b = (pops >> (8 * j)) & 0xFF;
                    const uint64_t v = rnd.w[j] >> 1;
                    uint32_t T;
                    if (b == b0) {
                        T = poisson_count(v, tr, thr0);
                    } else {  // a population boundary inside the quad: read that row from memory
                        const uint64_t *thr = &a.tables->thresholds[b][0];
                        T = 0;
                        while (T < static_cast<uint32_t>(kPK) && v >= __ldg(thr + T)) ++T;
                    }
                    const int32_t in =
                        static_cast<int32_t>(static_cast<uint32_t>(ww[j]) + T * static_cast<uint32_t>(a.w_ext_fx));
                    cc[j] = __fadd_rn(__fmul_rn(a.p11, cc[j]), __fmul_rn(__int2float_rn(in), 0x1p-12f));
                }
            }
            *reinterpret_cast<float4 *>(a.I + i0) = make_float4(cc[0], cc[1], cc[2], cc[3]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (i0 + j >= end_valid) continue;
            if (rr[j] == 0u) {
                float x = __fadd_rn(__fmul_rn(a.p22, uu[j]), __fmul_rn(a.p21, cc[j]));
                if (x >= a.theta) {
                    spk[j] = 1;
                    x = a.u_reset;
                    rr[j] = static_cast<uint32_t>(a.t_ref);
                }
                uu[j] = x;
            } else {
                uu[j] = a.u_reset;
                rr[j] -= 1u;
            }
        }
        *reinterpret_cast<float4 *>(Uout + i0) = make_float4(uu[0], uu[1], uu[2], uu[3]);
        *reinterpret_cast<uint32_t *>(Rout + i0) = rr[0] | (rr[1] << 8) | (rr[2] << 16) | (rr[3] << 24);
    }
    // the group's spikes of step t+1: count and entries, plain stores in its own region
    const int cnt = spk[0] + spk[1] + spk[2] + spk[3];
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (total == 0) return;
    uint32_t base = 0;
    if (lane == 31) base = atomicAdd(&queue_counts<kGroup>(a)[phn & 3], static_cast<uint32_t>(total));
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    if (cnt == 0) return;
    QueueEntry *region = a.queue + (phn & 3) * a.npad + base;
    int k = incl - cnt;
    const int64_t sn = t + 1;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (!spk[j]) continue;
        const int64_t rs = rp[j];
        const int64_t re = rp[j + 1];
        if (re > rs) {
            prefetch_l2(a.syn_tgt + rs, static_cast<uint32_t>(4 * (re - rs)));
            if (a.format == SNN_RECORD_PLAIN9) {
                prefetch_l2(a.syn_w + rs, static_cast<uint32_t>(4 * (re - rs)));
                const int64_t d0 = rs & ~int64_t{15}, d1 = (re + 15) & ~int64_t{15};
                prefetch_l2(a.syn_d + d0, static_cast<uint32_t>(d1 - d0));
            } else {
                const int64_t bp = a.format == SNN_RECORD_PACKED_I8 ? 1 : 2;
                const int64_t w0 = (rs * bp) & ~int64_t{15}, w1 = (re * bp + 15) & ~int64_t{15};
                prefetch_l2(reinterpret_cast<const uint8_t *>(a.syn_w) + w0, static_cast<uint32_t>(w1 - w0));
            }
        }
        QueueEntry e;
        e.row_quad = static_cast<uint32_t>(rs >> 2);
        e.len_quads = static_cast<uint32_t>((re - rs) >> 2);
        e.neuron = static_cast<int32_t>(i0 + j);
        e.step = static_cast<int32_t>(sn);
        *reinterpret_cast<int4 *>(region + k) = *reinterpret_cast<const int4 *>(&e);
        ++k;
    }
}

// D(t), run by the delivery warps: grid-stride over (spike, 256-synapse chunk) items
// of queue t mod 4.  The count, the raster base and the first item's entry are loaded
// in one round trip.  The warp taking chunk 0 of spike j records it in the raster.
template <int FMT, bool kGroup>
__device__ __forceinline__ void pipe_deliver_fmt(const StepArgs &a, const int64_t &t, int ph, int64_t dw, int64_t ndw,
                                                 uint32_t n, uint32_t rbase, int4 first)
{
    const int lane = threadIdx.x & 31;
    const QueueEntry *qbuf = a.queue + (ph & 3) * a.npad;
    const int64_t cpr = a.chunks_per_row;
    const int64_t cap = queue_entries<kGroup>(a);
    // items are (spike, run of `per` chunks); when every item is one chunk (few spikes) the
    // entry `first` loaded before n arrived belongs to this warp's first item
    const int64_t ipj = items_per_spike(cpr, n, ndw);
    const int64_t per = (cpr + ipj - 1) / ipj;
    for (int64_t it = dw;; it += ndw) {
        const int64_t j = it / ipj;
        if (j >= cap || j >= n) break;
        const int4 raw = (it == dw && ipj == cpr) ? first : __ldcg(reinterpret_cast<const int4 *>(qbuf + j));
        const int64_t part = it - j * ipj;
        if (part == 0 && lane == 0) {
            const uint64_t pos = static_cast<uint64_t>(rbase) + static_cast<uint64_t>(j);
            if (pos < a.rast_cap) {
                a.rast_nrn[pos] = raw.z;
                a.rast_t[pos] = static_cast<int32_t>(t);
            }
        }
        const int64_t rs = static_cast<int64_t>(static_cast<uint32_t>(raw.x)) * 4;
        const int64_t re = rs + static_cast<int64_t>(static_cast<uint32_t>(raw.y)) * 4;
        const int src = FMT == SNN_RECORD_PACKED_I8 ? __ldg(a.pop_id + raw.z) : 0;
        for (int64_t c = part * per, off = rs + c * kChunk; c < (part + 1) * per && off < re; ++c, off += kChunk)
            deliver_chunk<FMT>(a, ph, off, re, src);
    }
}

template <bool kGroup>
__device__ __forceinline__ void pipe_deliver(const StepArgs &a, const int64_t &t, int ph, bool leader, int64_t dw,
                                             int64_t ndw, bool wait_first)
{
    if (wait_first) wait_previous_grid();
    const uint32_t n = __ldcg(&queue_counts<kGroup>(a)[ph & 3]);
    const uint32_t rbase = __ldcg(&a.ctl->step_begin[t & 1]);
    // speculative: the entry of this warp's first item under one chunk per item, issued
    // alongside the count so both arrive in one round trip
    const int64_t j0 = dw / a.chunks_per_row;
    const int4 first = j0 < queue_entries<kGroup>(a) ? __ldcg(reinterpret_cast<const int4 *>(a.queue + (ph & 3) * a.npad + j0))
                                   : make_int4(0, 0, 0, 0);
    if (leader) {
        a.ctl->step_begin[(t + 1) & 1] = rbase + n;
        a.ctl->cursor = rbase + n;
        queue_counts<kGroup>(a)[(ph + 2) & 3] = 0;  // the queue the next kernel fills after this one
        if (static_cast<uint64_t>(rbase) + n > a.rast_cap) atomicOr(&a.ctl->err, kErrRaster);
    }
    if (a.format == SNN_RECORD_PACKED_I8)
        pipe_deliver_fmt<SNN_RECORD_PACKED_I8, kGroup>(a, t, ph, dw, ndw, n, rbase, first);
    else if (a.format == SNN_RECORD_PACKED_BF16)
        pipe_deliver_fmt<SNN_RECORD_PACKED_BF16, kGroup>(a, t, ph, dw, ndw, n, rbase, first);
    else
        pipe_deliver_fmt<SNN_RECORD_PLAIN9, kGroup>(a, t, ph, dw, ndw, n, rbase, first);
}

// t_base is read before waiting on the previous kernel: within a graph replay it only
// changes in the replay's last node, and direct launches are not programmatic.
template <bool kGroup>
__global__ void __launch_bounds__(kStepMaxThreads, 2) k_step(const StepArgs a, const int k, const int ph)
{
    allow_next_grid();
    const int64_t t = a.ctl->t_base + k;  // used for Philox counters and step tags only
    const int wib = threadIdx.x >> 5;
    if (wib < a.neuron_warps) {
        const int64_t nquads = (a.n + 3) / 4;
        const int64_t nw = static_cast<int64_t>(a.neuron_warps) * gridDim.x;
        bool first = true;
        for (int64_t g = first_quad_warp<kGroup>(a) + static_cast<int64_t>(wib) * gridDim.x + blockIdx.x;
             g < a.quad_warps; g += nw) {
            pipe_quad<kGroup>(a, t, ph, g, g * 32 + (threadIdx.x & 31) < nquads, true, first);
            first = false;
        }
        if (first) wait_previous_grid();
    } else {
        const int dwarps = static_cast<int>(blockDim.x >> 5) - a.neuron_warps;
        const bool leader = blockIdx.x == 0 && threadIdx.x == 32 * a.neuron_warps;
        const int64_t dw = static_cast<int64_t>(wib - a.neuron_warps) * gridDim.x + blockIdx.x;
        pipe_deliver<kGroup>(a, t, ph, leader, dw, static_cast<int64_t>(dwarps) * gridDim.x, true);
    }
}

__global__ void __launch_bounds__(kStepMaxThreads, 2) k_prime(const StepArgs a)
{
    const int wib = threadIdx.x >> 5;
    if (wib >= a.neuron_warps) return;
    const int64_t nquads = (a.n + 3) / 4;
    const int64_t nw = static_cast<int64_t>(a.neuron_warps) * gridDim.x;
    const int64_t t = -1;
    for (int64_t g = (a.quad_base >> 5) + static_cast<int64_t>(wib) * gridDim.x + blockIdx.x; g < a.quad_warps; g += nw)
        pipe_quad<true>(a, t, -1, g, g * 32 + (threadIdx.x & 31) < nquads, false, false);
}

// Persistent engine: the pipelined schedule in one cooperative launch for a run of
// steps.  Iteration t does what the step kernel K_t does (neuron warps: B(t) then
// A(t+1); delivery warps: D(t)); one bounded grid barrier between iterations stands in
// for the kernel boundary, which orders D(t)'s ring sums and A(t+1)'s queue before
// iteration t+1 reads them.  Every warp keeps its neuron groups for the whole launch.
__global__ void __launch_bounds__(kStepMaxThreads, 1) k_persistent(const StepArgs a, const int64_t n_steps)
{
    Ctl *ctl = a.ctl;
    const int64_t t0 = ctl->t_base;
    const int wib = threadIdx.x >> 5;
    const int64_t nquads = (a.n + 3) / 4;
    const int64_t nw = static_cast<int64_t>(a.neuron_warps) * gridDim.x;
    const int dwarps = static_cast<int>(blockDim.x >> 5) - a.neuron_warps;
    const bool leader = blockIdx.x == 0 && threadIdx.x == 32 * a.neuron_warps;
    const int64_t dw = static_cast<int64_t>(wib - a.neuron_warps) * gridDim.x + blockIdx.x;
    uint32_t nbar = 0;
    for (int64_t st = 0; st < n_steps; ++st) {
        const int64_t t = t0 + st;
        const int ph = static_cast<int>(t & (kPhasePeriod - 1));
        if (wib < a.neuron_warps) {
            for (int64_t g = static_cast<int64_t>(wib) * gridDim.x + blockIdx.x; g < a.quad_warps; g += nw)
                pipe_quad<false>(a, t, ph, g, g * 32 + (threadIdx.x & 31) < nquads, true, false);
        } else {
            pipe_deliver<false>(a, t, ph, leader, dw, static_cast<int64_t>(dwarps) * gridDim.x, false);
        }
        if (!grid_barrier(a, ctl, ++nbar)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->t_base = t0 + n_steps;
}


// ---------------------------------------------------------------------------------
// Blocked records: phase 2 with one CTA per block of consecutive targets.
//
// Each sender's row is grouped by target block, so CTA p reads, for every sender, only
// the segment that lands in its block (row_ptr[s] + seg[s][p] .. + seg[s][p + 1]); a
// segment is a whole number of aligned quads of records (zero-weight padding).  Per
// pass the CTA stages up to kBlockedBatch senders' nonempty segments (first quad and
// the exclusive prefix of the quad counts, compacted) in shared memory, which makes the
// pass one stream of quads.  The stream is taken in windows of kBlockedMapWindow quads
// (one per pass at the microcircuit's sizes); a map gives the segment holding every
// 16th quad of the window, from which a quad's segment is a short forward walk.  The
// quads are then independent work: warp w takes rounds w, w + 32, ... of 32 consecutive
// quads, in sets of kBlockedRounds / 2 rounds whose loads (per quad 8 bytes of records
// and 16 of int32 weights, one 16-byte unit of records and bfloat16 weights, or 32
// bytes of (weight, record) pairs) are issued while the previous set's weights are
// added.
// With many senders the weights of delays up to kBlockedBinDelays are summed per (delay,
// local target) in shared memory and each nonzero sum is added to its ring entry once at
// the end; only this CTA writes these ring columns during the launch, so that final add
// is a plain read-modify-write.  Longer delays (about 1 % of the microcircuit's events)
// and, with few senders, all weights go straight to the ring as reductions; they land
// in other ring rows than the plain adds.  Integer addition makes every order give the
// same ring.
// ---------------------------------------------------------------------------------

constexpr int kBlockedWarps = kBlockedThreads / 32;
// dynamic shared memory of k_deliver_blocked, in bytes from its start
// kW: width of the bins (kBlockMaxWidth)
constexpr int kBlockedMapWindow = 32768;     // quads of a pass mapped to their segments at once
constexpr int kBlockedChunkShift = 5;        // the map gives the segment of every 32nd quad (a round's first)
constexpr int kBlockedChunks = kBlockedMapWindow >> kBlockedChunkShift;  // map entries per window
// How a format locates a window's quads: BLOCKED8 (two 16-byte loads per quad, on
// consecutive lanes) through a table of every quad's record-array index, the others
// through the map of segments per round (measured faster for each).
template <int FMT>
struct BlockedCfg {
    static constexpr bool table = FMT == SNN_RECORD_BLOCKED8;
    static constexpr size_t index_bytes = table ? sizeof(uint32_t) * kBlockedWindow
                                                : sizeof(uint16_t) * kBlockedChunks;
};
// Table formats stage every sender (empty segments too) with its quad count; map formats
// only the nonempty segments, followed by 32 INT32_MAX starts.
template <int kW, int FMT>
struct BlockedSmem {
    static constexpr bool table = BlockedCfg<FMT>::table;
    static constexpr size_t seg_q = sizeof(int32_t) * (kBlockedBinDelays + 1) * kW;    // after the bins
    static constexpr size_t pfx = seg_q + sizeof(uint32_t) * kBlockedBatch;          // first quad per segment
    static constexpr size_t nq = pfx + sizeof(int32_t) * (kBlockedBatch + (table ? 0 : 32));  // quad prefix
    static constexpr size_t warp = nq + (table ? sizeof(int32_t) * kBlockedBatch : 0);  // quads per sender
    static constexpr size_t index = warp + (table ? sizeof(int32_t) : sizeof(int2)) * kBlockedWarps;  // scan scratch
    static constexpr size_t total = index + BlockedCfg<FMT>::index_bytes;             // table or map
};
template <int FMT>
constexpr size_t blocked_smem_bytes() { return BlockedSmem<kBlockMaxWidth, FMT>::total; }
static_assert(blocked_smem_bytes<SNN_RECORD_BLOCKED8>() <= 232448 && blocked_smem_bytes<SNN_RECORD_BLOCKED6>() <= 232448,
              "blocked delivery: shared memory above the 227 KB opt-in limit");
static_assert(kBlockedBatch <= 65536, "segment numbers are 16-bit in the map");
static_assert(kBlockedBatch % kBlockedThreads == 0, "staged senders per thread");
static_assert(kBlockedBinDelays >= 1 && kBlockedBinDelays < kDMax && kBlockMaxWidth % 4 == 0, "bins");

template <bool kAggregate, int kW>
__device__ __forceinline__ void blocked_apply(const StepArgs &a, int32_t *bins, int64_t t, int32_t base, uint32_t rec,
                                              int32_t w)
{
    if (w == 0) return;  // padding (adding zero changes nothing)
    const int d = static_cast<int>(rec >> kBlockLocalBits);
    const int lt = static_cast<int>(rec & ((1u << kBlockLocalBits) - 1));
    if (kAggregate && d <= kBlockedBinDelays) atomicAdd(bins + d * kW + lt, w);
    else red_add_s32(a.ring + ((t + d) & kDMask) * a.npad + base + lt, w);
}

// The same for a BLOCKED8 record: local target in the low 16 bits, delay above.
template <bool kAggregate, int kW>
__device__ __forceinline__ void blocked_apply_wide(const StepArgs &a, int32_t *bins, int64_t t, int32_t base,
                                                   uint32_t rec, int32_t w)
{
    if (w == 0) return;
    const int d = static_cast<int>(rec >> 16);
    const int lt = static_cast<int>(rec & 0xFFFFu);
    if (kAggregate && d <= kBlockedBinDelays) atomicAdd(bins + d * kW + lt, w);
    else red_add_s32(a.ring + ((t + d) & kDMask) * a.npad + base + lt, w);
}

// Exclusive prefix sum of one value per thread over the CTA into out[threadIdx.x];
// returns the total.
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t *out, int32_t *warp_sums)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < kBlockedWarps ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kBlockedWarps) warp_sums[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    out[threadIdx.x] = (warp > 0 ? warp_sums[warp - 1] : 0) + x - v;
    return warp_sums[kBlockedWarps - 1];
}

// Exclusive prefix sums of two values per thread over the CTA; returns this thread's
// prefixes and sets `total` to the sums over the CTA.
__device__ __forceinline__ int2 block_exclusive_scan2(int2 v, int2 *warp_sums, int2 &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int2 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t yx = __shfl_up_sync(0xffffffffu, x.x, o);
        const int32_t yy = __shfl_up_sync(0xffffffffu, x.y, o);
        if (lane >= o) {
            x.x += yx;
            x.y += yy;
        }
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int2 w = lane < kBlockedWarps ? warp_sums[lane] : make_int2(0, 0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t yx = __shfl_up_sync(0xffffffffu, w.x, o);
            const int32_t yy = __shfl_up_sync(0xffffffffu, w.y, o);
            if (lane >= o) {
                w.x += yx;
                w.y += yy;
            }
        }
        if (lane < kBlockedWarps) warp_sums[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const int2 before = warp > 0 ? warp_sums[warp - 1] : make_int2(0, 0);
    total = warp_sums[kBlockedWarps - 1];
    return make_int2(before.x + x.x - v.x, before.y + x.y - v.y);
}

// A pass's compacted segments in shared memory: segment k's first quad in the record
// arrays and its first quad in the pass's stream (32 entries past the last segment hold
// INT32_MAX); jmap[c]: the segment holding the window's quad w0 + 32 c, where w0 is a
// multiple of kBlockedMapWindow; or qidx[e - w0]: quad e's record-array index.
struct BlockedPass {
    const uint32_t *seg_q;
    const int32_t *pfx;
    const uint16_t *jmap;
    const uint32_t *qidx;
};

// Record-array quad of stream quad eb + lane, for a round of 32 quads starting at eb, a
// multiple of 32 inside the current window (every lane of the warp calls it).  The map
// gives the segment k0 holding eb; the next 32 segments' starts, one per lane, mark the
// quads of the round where a segment begins, and a lane's segment is k0 plus the marks at
// or below it.
__device__ __forceinline__ uint32_t blocked_round_quad(const BlockedPass &ps, int32_t eb, int lane)
{
    const int k0 = ps.jmap[(eb >> kBlockedChunkShift) & (kBlockedChunks - 1)];
    const int32_t st = ps.pfx[k0 + 1 + lane] - eb;  // >= 1: segment k0 holds eb
    const uint32_t marks = __reduce_or_sync(0xffffffffu, st < 32 ? 1u << st : 0u);
    const int k = k0 + __popc(marks & ((2u << lane) - 1u));
    return ps.seg_q[k] + static_cast<uint32_t>(eb + lane - ps.pfx[k]);
}

// bfloat16 current (pA) -> 2^-12 pA, as the SNN_RECORD_PACKED_BF16 read-back
__device__ __forceinline__ int32_t bf16_fx(uint32_t h)
{
    return __float2int_rn(__fmul_rn(__uint_as_float((h & 0xFFFFu) << 16), 4096.0f));
}

// Quads [w0, w1) of the staged stream, located through the pass's map: BLOCKED6 reads 8
// bytes of records and 16 of int32 weights per quad, BLOCKED4 one 16-byte unit of
// records and bfloat16 weights, BLOCKED8 32 bytes of (weight, record) pairs.  The window is taken in sets of
// kBlockedRounds / 2 rounds, software-pipelined: the loads of the next set are in flight
// while the current set's weights are added, so the record stream never drains inside
// a window.
constexpr int kBlockedSet = kBlockedRounds / 2;  // rounds per pipelined set

// A set's loads are kept raw (decoded only when added, so that issuing the next set
// never waits for this one): per round two 16-byte values, used per format as
//   BLOCKED6: va.xy = the quad's four uint16 records, vb = its four int32 weights;
//   BLOCKED4: va = the 16-byte unit (records, then bfloat16 currents);
//   BLOCKED8: va, vb = the 32-byte quad of (int32 weight, uint32 record) pairs.
template <int FMT>
__device__ __forceinline__ void blocked_load_set(const StepArgs &a, const BlockedPass &ps, int32_t w0, int32_t w1,
                                                 int32_t e0, uint4 (&va)[kBlockedSet], uint4 (&vb)[kBlockedSet])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint2 *recq = reinterpret_cast<const uint2 *>(a.blk_rec);
    const uint4 *wq = reinterpret_cast<const uint4 *>(a.syn_w);
    const uint4 *q16 = reinterpret_cast<const uint4 *>(a.blk_rec);
#pragma unroll
    for (int k = 0; k < kBlockedSet; ++k) {
        // round k of a set is quads eb .. eb + 32, eb = e0 + 32 * (warp + kBlockedWarps * k):
        // the warps of the CTA interleave, so that a window's rounds spread evenly over them
        const int32_t eb = e0 + 32 * (warp + kBlockedWarps * k);
        const int32_t e = eb + lane;
        va[k] = make_uint4(0, 0, 0, 0);
        vb[k] = make_uint4(0, 0, 0, 0);
        if (BlockedCfg<FMT>::table) {
            // BLOCKED8: the round's 32 quads as 64 16-byte halves, consecutive halves on
            // consecutive lanes (so one load instruction reads whole lines of a segment):
            // lane l takes halves l and 32 + l, of quads l / 2 and 16 + l / 2
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int32_t eq = eb + 16 * j + (lane >> 1);
                if (eq < w1) {
                    const uint4 v = __ldcs(q16 + 2 * uint64_t(ps.qidx[eq - w0]) + (lane & 1));
                    if (j == 0) va[k] = v;
                    else vb[k] = v;
                }
            }
            continue;
        }
        if (eb >= w1) continue;  // the whole warp
        const uint32_t qe = blocked_round_quad(ps, eb, lane);
        if (e < w1) {
            const uint32_t q = qe;
            if (FMT == SNN_RECORD_BLOCKED4) {
                va[k] = __ldcs(q16 + q);
            } else if (FMT == SNN_RECORD_BLOCKED8) {
                // loaded below, by half-quads
            } else {
                const uint2 r = __ldcs(recq + q);
                va[k] = make_uint4(r.x, r.y, 0, 0);
                vb[k] = __ldcs(wq + q);
            }
        }
    }
}

template <bool kAggregate, int FMT, int kW>
__device__ __forceinline__ void blocked_apply_set(const StepArgs &a, int32_t *bins, int64_t t, int32_t base,
                                                  const uint4 (&va)[kBlockedSet], const uint4 (&vb)[kBlockedSet])
{
#pragma unroll
    for (int k = 0; k < kBlockedSet; ++k) {
        uint32_t r01, r23;
        int32_t w0v, w1v, w2v, w3v;
        if (FMT == SNN_RECORD_BLOCKED4) {
            r01 = va[k].x;
            r23 = va[k].y;
            w0v = bf16_fx(va[k].z);
            w1v = bf16_fx(va[k].z >> 16);
            w2v = bf16_fx(va[k].w);
            w3v = bf16_fx(va[k].w >> 16);
        } else if (FMT == SNN_RECORD_BLOCKED8) {
            // two (weight, record) pairs per 16-byte half
            blocked_apply_wide<kAggregate, kW>(a, bins, t, base, va[k].y, static_cast<int32_t>(va[k].x));
            blocked_apply_wide<kAggregate, kW>(a, bins, t, base, va[k].w, static_cast<int32_t>(va[k].z));
            blocked_apply_wide<kAggregate, kW>(a, bins, t, base, vb[k].y, static_cast<int32_t>(vb[k].x));
            blocked_apply_wide<kAggregate, kW>(a, bins, t, base, vb[k].w, static_cast<int32_t>(vb[k].z));
            continue;
        } else {
            r01 = va[k].x;
            r23 = va[k].y;
            w0v = static_cast<int32_t>(vb[k].x);
            w1v = static_cast<int32_t>(vb[k].y);
            w2v = static_cast<int32_t>(vb[k].z);
            w3v = static_cast<int32_t>(vb[k].w);
        }
        // quads past the window end were left zero: zero weights add nothing
        blocked_apply<kAggregate, kW>(a, bins, t, base, r01 & 0xffffu, w0v);
        blocked_apply<kAggregate, kW>(a, bins, t, base, r01 >> 16, w1v);
        blocked_apply<kAggregate, kW>(a, bins, t, base, r23 & 0xffffu, w2v);
        blocked_apply<kAggregate, kW>(a, bins, t, base, r23 >> 16, w3v);
    }
}

template <bool kAggregate, int FMT, int kW>
__device__ __forceinline__ void blocked_window(const StepArgs &a, int32_t *bins, const BlockedPass &ps, int32_t w0,
                                               int32_t w1, int64_t t, int32_t base)
{
    constexpr int32_t kStep = kBlockedThreads * kBlockedSet;
    uint4 aA[kBlockedSet], bA[kBlockedSet], aB[kBlockedSet], bB[kBlockedSet];
    int32_t e0 = w0;
    blocked_load_set<FMT>(a, ps, w0, w1, e0, aA, bA);
    for (;;) {
        if (e0 + kStep < w1) blocked_load_set<FMT>(a, ps, w0, w1, e0 + kStep, aB, bB);
        blocked_apply_set<kAggregate, FMT, kW>(a, bins, t, base, aA, bA);
        e0 += kStep;
        if (e0 >= w1) break;
        if (e0 + kStep < w1) blocked_load_set<FMT>(a, ps, w0, w1, e0 + kStep, aA, bA);
        blocked_apply_set<kAggregate, FMT, kW>(a, bins, t, base, aB, bB);
        e0 += kStep;
        if (e0 >= w1) break;
    }
}

// One pass of the table formats over senders spk[0 .. nb): every sender's segment (first
// quad, quad count, prefix of the counts) in the staging tables, then per window of
// kBlockedWindow quads the record-array index of every quad.
template <int FMT, int kW>
__device__ __forceinline__ void blocked_pass_table(const StepArgs &a, uint8_t *sm, int32_t *bins, const int32_t *spk,
                                                   int nb, int p, bool aggregate, int64_t t, int32_t base)
{
    using SL = BlockedSmem<kW, FMT>;
    constexpr int kPer = kBlockedBatch / kBlockedThreads;  // senders staged per thread
    uint32_t *seg_q = reinterpret_cast<uint32_t *>(sm + SL::seg_q);   // [kBlockedBatch]
    int32_t *pfx = reinterpret_cast<int32_t *>(sm + SL::pfx);         // [kBlockedBatch]
    int32_t *seg_nq = reinterpret_cast<int32_t *>(sm + SL::nq);       // [kBlockedBatch]
    int32_t *warp_sums = reinterpret_cast<int32_t *>(sm + SL::warp);  // [kBlockedWarps]
    uint32_t *qidx = reinterpret_cast<uint32_t *>(sm + SL::index);    // [kBlockedWindow]
    const int tid = threadIdx.x;
    const int64_t stride = a.n_blocks + 1;
    // thread tid stages senders tid * kPer .. + kPer (consecutive, for the scan)
    int32_t mine = 0;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int j = tid * kPer + i;
        int32_t nq = 0;
        if (j < nb) {
            const int32_t s = __ldcg(spk + j);
            const uint16_t *sg = a.blk_seg + static_cast<int64_t>(s) * stride + p;
            const int32_t o0 = __ldg(sg), o1 = __ldg(sg + 1);
            seg_q[j] = static_cast<uint32_t>((__ldg(a.row_ptr + s) + o0) / kBlockQuad);
            nq = (o1 - o0) / kBlockQuad;
        }
        seg_nq[j] = nq;
        mine += nq;
    }
    // the window table is idle here: it holds the scan's per-thread output
    int32_t *scan_out = reinterpret_cast<int32_t *>(qidx);
    const int32_t total = block_exclusive_scan(mine, scan_out, warp_sums);
    {
        int32_t run = scan_out[tid];
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            pfx[tid * kPer + i] = run;
            run += seg_nq[tid * kPer + i];
        }
    }
    __syncthreads();
    for (int32_t w0 = 0; w0 < total; w0 += kBlockedWindow) {
        const int32_t w1 = total - w0 < kBlockedWindow ? total : w0 + kBlockedWindow;
        // record-array index of every quad of the window
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int j = tid * kPer + i;
            if (j >= nb) break;
            const int32_t lo = max(pfx[j], w0), hi = min(pfx[j] + seg_nq[j], w1);
            const uint32_t q0 = seg_q[j] - static_cast<uint32_t>(pfx[j]);
            for (int32_t e = lo; e < hi; ++e) qidx[e - w0] = q0 + static_cast<uint32_t>(e);
        }
        __syncthreads();
        const BlockedPass ps{seg_q, pfx, nullptr, qidx};
        if (aggregate) blocked_window<true, FMT, kW>(a, bins, ps, w0, w1, t, base);
        else blocked_window<false, FMT, kW>(a, bins, ps, w0, w1, t, base);
        __syncthreads();  // the table is rebuilt for the next window
    }
}

// One pass of the map formats over senders spk[0 .. nb): the nonempty segments, compacted
// in sender order, then per window of kBlockedMapWindow quads the segment holding every
// 32nd quad.
template <int FMT, int kW>
__device__ __forceinline__ void blocked_pass_map(const StepArgs &a, uint8_t *sm, int32_t *bins, const int32_t *spk,
                                                 int nb, int p, bool aggregate, int64_t t, int32_t base)
{
    using SL = BlockedSmem<kW, FMT>;
    constexpr int kPer = kBlockedBatch / kBlockedThreads;  // senders staged per thread
    uint32_t *seg_q = reinterpret_cast<uint32_t *>(sm + SL::seg_q);  // [kBlockedBatch]
    int32_t *pfx = reinterpret_cast<int32_t *>(sm + SL::pfx);        // [kBlockedBatch + 32]
    int2 *warp_sums = reinterpret_cast<int2 *>(sm + SL::warp);       // [kBlockedWarps]
    uint16_t *jmap = reinterpret_cast<uint16_t *>(sm + SL::index);   // [kBlockedChunks]
    const int tid = threadIdx.x;
    const int64_t stride = a.n_blocks + 1;
    // thread tid stages senders tid * kPer .. + kPer (consecutive, for the scan)
    uint32_t sq[kPer];
    int32_t nq[kPer];
    int2 mine = make_int2(0, 0);  // (quads, nonempty segments)
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int j = tid * kPer + i;
        sq[i] = 0;
        nq[i] = 0;
        if (j < nb) {
            const int32_t s = __ldcg(spk + j);
            const uint16_t *sg = a.blk_seg + static_cast<int64_t>(s) * stride + p;
            const int32_t o0 = __ldg(sg), o1 = __ldg(sg + 1);
            sq[i] = static_cast<uint32_t>((__ldg(a.row_ptr + s) + o0) / kBlockQuad);
            nq[i] = (o1 - o0) / kBlockQuad;
        }
        mine.x += nq[i];
        mine.y += nq[i] > 0 ? 1 : 0;
    }
    int2 total;
    const int2 at = block_exclusive_scan2(mine, warp_sums, total);
    // the nonempty segments, in sender order (the scan's scratch is read by now)
    {
        int32_t run = at.x, k = at.y;
#pragma unroll
        for (int i = 0; i < kPer; ++i)
            if (nq[i] > 0) {
                seg_q[k] = sq[i];
                pfx[k] = run;
                run += nq[i];
                ++k;
            }
        if (tid < 32) pfx[total.y + tid] = INT32_MAX;  // past the last segment
    }
    for (int32_t w0 = 0; w0 < total.x; w0 += kBlockedMapWindow) {
        const int32_t w1 = total.x - w0 < kBlockedMapWindow ? total.x : w0 + kBlockedMapWindow;
        __syncthreads();  // the segments are written; the previous window's map is free
        // the segment holding every 32nd quad of the window
        for (int k = tid; k < total.y; k += kBlockedThreads) {
            const int32_t lo = max(pfx[k], w0), hi = min(pfx[k + 1], w1);
            constexpr int32_t kC = 1 << kBlockedChunkShift;
            for (int32_t c = (lo - w0 + kC - 1) >> kBlockedChunkShift; w0 + (c << kBlockedChunkShift) < hi; ++c)
                jmap[c] = static_cast<uint16_t>(k);
        }
        __syncthreads();
        const BlockedPass ps{seg_q, pfx, jmap, nullptr};
        if (aggregate) blocked_window<true, FMT, kW>(a, bins, ps, w0, w1, t, base);
        else blocked_window<false, FMT, kW>(a, bins, ps, w0, w1, t, base);
    }
    __syncthreads();  // the segment tables are rewritten by the next pass
}

template <int FMT>
__global__ void __launch_bounds__(kBlockedThreads, 1)
    k_deliver_blocked(const StepArgs a, const int32_t *list, int64_t n_list, int64_t t_list, int k)
{
    constexpr int kW = kBlockMaxWidth;
    using CF = BlockedCfg<FMT>;
    extern __shared__ int4 smem4[];
    uint8_t *sm = reinterpret_cast<uint8_t *>(smem4);
    int32_t *bins = reinterpret_cast<int32_t *>(sm);  // [kBlockedBinDelays + 1][kW]

    int64_t t;
    const int32_t *spk;
    int64_t nspk;
    if (list != nullptr) {
        t = t_list;
        spk = list;
        nspk = n_list;
    } else {
        // graph engine: the spikes step t appended to the raster
        t = a.ctl->t_base + k;
        const uint32_t cur = a.ctl->cursor;
        const uint32_t begin = a.ctl->step_begin[t & 1];
        if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->step_begin[(t + 1) & 1] = cur;
        const uint32_t end = cur < a.rast_cap ? cur : a.rast_cap;
        spk = a.rast_nrn + begin;
        nspk = end > begin ? static_cast<int64_t>(end - begin) : 0;
    }
    if (nspk == 0) return;

    const int p = blockIdx.x;
    const int32_t base = a.blk_off[p];
    const int32_t width = a.blk_off[p + 1] - base;
    const bool aggregate = nspk >= kBlockedAggregateMin;
    const int tid = threadIdx.x;

    if (aggregate)
        for (int j = tid; j < (kBlockedBinDelays + 1) * kW / 4; j += kBlockedThreads) smem4[j] = make_int4(0, 0, 0, 0);

    for (int64_t b0 = 0; b0 < nspk; b0 += kBlockedBatch) {
        const int nb = static_cast<int>(nspk - b0 < kBlockedBatch ? nspk - b0 : kBlockedBatch);
        if (CF::table) blocked_pass_table<FMT, kW>(a, sm, bins, spk + b0, nb, p, aggregate, t, base);
        else blocked_pass_map<FMT, kW>(a, sm, bins, spk + b0, nb, p, aggregate, t, base);
    }
    if (!aggregate) return;
    // add the sums of delays 1..kBlockedBinDelays to their ring rows; width is a multiple
    // of 4 except for the last block, whose extra columns lie inside the padded ring row
    const int w4 = (width + 3) >> 2;
    for (int q = tid; q < kBlockedBinDelays * w4; q += kBlockedThreads) {
        const int d = 1 + q / w4;
        const int c4 = q - (d - 1) * w4;
        const int4 v = smem4[(d * kW) / 4 + c4];
        if ((v.x | v.y | v.z | v.w) == 0) continue;
        int4 *dst = reinterpret_cast<int4 *>(a.ring + ((t + d) & kDMask) * a.npad + base) + c4;
        int4 o = __ldcg(dst);
        o.x = static_cast<int32_t>(static_cast<uint32_t>(o.x) + static_cast<uint32_t>(v.x));
        o.y = static_cast<int32_t>(static_cast<uint32_t>(o.y) + static_cast<uint32_t>(v.y));
        o.z = static_cast<int32_t>(static_cast<uint32_t>(o.z) + static_cast<uint32_t>(v.z));
        o.w = static_cast<int32_t>(static_cast<uint32_t>(o.w) + static_cast<uint32_t>(v.w));
        __stcg(dst, o);
    }
}

}  // namespace

// One CTA per SM while its kStepMaxNeuronWarps neuron warps cover the network's groups of
// 128 neurons in one pass; larger networks get up to three CTAs per SM, so that a neuron
// warp walks fewer groups one after another (each group is a chain of dependent loads).
int step_grid(int num_sms, int64_t quad_warps)
{
    const int64_t per_pass = static_cast<int64_t>(kStepMaxNeuronWarps) * num_sms;
    const int64_t mult = std::min<int64_t>(3, std::max<int64_t>(1, (quad_warps + per_pass - 1) / per_pass));
    return static_cast<int>(mult * num_sms);
}

int step_threads(const StepArgs &a) { return 32 * (a.neuron_warps + a.delivery_warps); }

static size_t step_smem(const StepArgs &) { return 0; }

int prepare_step_kernel(const StepArgs &) { return 0; }

int launch_step(const StepArgs &a, int k, int ph, int grid, void *stream, bool programmatic)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(step_threads(a));
    cfg.dynamicSmemBytes = step_smem(a);
    cfg.stream = static_cast<cudaStream_t>(stream);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = programmatic ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (a.group_launch) return static_cast<int>(cudaLaunchKernelEx(&cfg, k_step<true>, a, k, ph));
    return static_cast<int>(cudaLaunchKernelEx(&cfg, k_step<false>, a, k, ph));
}

void launch_prime(const StepArgs &a, int grid, void *stream)
{
    k_prime<<<grid, step_threads(a), 0, static_cast<cudaStream_t>(stream)>>>(a);
}

int update_grid(int64_t n)
{
    const int64_t quads = (n + 3) / 4;
    return static_cast<int>((quads + kUpdateThreads - 1) / kUpdateThreads);
}

void launch_update(const StepArgs &a, int k, int grid, void *stream)
{
    k_update<<<grid, kUpdateThreads, 0, static_cast<cudaStream_t>(stream)>>>(a, k);
}

void launch_deliver(const StepArgs &a, int k, int grid, void *stream)
{
    k_deliver<<<grid, kDeliverThreads, 0, static_cast<cudaStream_t>(stream)>>>(a, k);
}

void launch_deliver_list(const StepArgs &a, const int32_t *list, int64_t n, int64_t t, int grid, void *stream)
{
    k_deliver_list<<<grid, kDeliverThreads, 0, static_cast<cudaStream_t>(stream)>>>(a, list, n, t);
}

int prepare_blocked_kernel()
{
    cudaError_t e = cudaFuncSetAttribute(k_deliver_blocked<SNN_RECORD_BLOCKED6>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(blocked_smem_bytes<SNN_RECORD_BLOCKED6>()));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_deliver_blocked<SNN_RECORD_BLOCKED4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(blocked_smem_bytes<SNN_RECORD_BLOCKED4>()));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_deliver_blocked<SNN_RECORD_BLOCKED8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(blocked_smem_bytes<SNN_RECORD_BLOCKED8>()));
    return static_cast<int>(e);
}

void launch_deliver_blocked(const StepArgs &a, const int32_t *list, int64_t n, int64_t t, int k, void *stream)
{
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (a.format == SNN_RECORD_BLOCKED4)
        k_deliver_blocked<SNN_RECORD_BLOCKED4><<<a.n_blocks, kBlockedThreads, blocked_smem_bytes<SNN_RECORD_BLOCKED4>(), st>>>(a, list, n, t, k);
    else if (a.format == SNN_RECORD_BLOCKED8)
        k_deliver_blocked<SNN_RECORD_BLOCKED8><<<a.n_blocks, kBlockedThreads, blocked_smem_bytes<SNN_RECORD_BLOCKED8>(), st>>>(a, list, n, t, k);
    else
        k_deliver_blocked<SNN_RECORD_BLOCKED6><<<a.n_blocks, kBlockedThreads, blocked_smem_bytes<SNN_RECORD_BLOCKED6>(), st>>>(a, list, n, t, k);
}

int deliver_list_blocks_per_sm()
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_deliver_list, kDeliverThreads, 0) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

void launch_advance(Ctl *ctl, int64_t m, void *stream)
{
    k_advance<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(ctl, m);
}

void launch_resync(Ctl *ctl, void *stream) { k_resync<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(ctl); }

int persistent_blocks_per_sm(const StepArgs &a)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_persistent, step_threads(a), 0) != cudaSuccess) return 0;
    return nb;
}

int launch_persistent(const StepArgs &a, int64_t n_steps, int grid, void *stream)
{
    StepArgs args = a;
    int64_t n = n_steps;
    void *params[] = {&args, &n};
    const cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_persistent), dim3(grid),
                                                      dim3(step_threads(a)), params, 0,
                                                      static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? 0 : static_cast<int>(e);
}

}  // namespace snn
