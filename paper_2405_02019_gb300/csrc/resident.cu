// Resident engine (sm_103a): the step loop of Listing push / push2 (§3.1) for a whole run
// of steps in one cooperative launch, one CTA per block of consecutive neurons.
//
// CTA p owns neurons [blk_off[p], blk_off[p+1]) both as senders and as targets:
//   - their U, I and R stay in the registers of its neuron warps for the whole launch
//     (four neurons per lane);
//   - their columns of the 64-row ring W[(t + d) mod 64][i] (§3.2) stay in its shared
//     memory (all 64 rows when they fit; otherwise the rows of delays below `rows` sit in
//     shared memory and longer delays go to the ring in global memory, which only this
//     CTA reads or writes for these columns);
//   - the records are stored block-major: every synapse into the block, sender by
//     sender and each sender's segment in delay order, forms one region (the indexed
//     store of §3.5 split by target), and the CTA keeps the block's segment lengths
//     (8 bits) and one offset per 32 senders in shared memory, so it finds a spike's
//     segment without touching global memory.
// The only traffic between CTAs is the spike list of every step.  After deciding its
// spikes, a CTA writes, into one 16-byte inbox slot per reading CTA, the step's spike
// count and up to three spikes (their index in the block); further spikes go once into
// its outbox.  Each CTA thus polls only lines that it alone reads.
// Once a step's slots are all in, the lanes that received spikes locate their segments in
// the block's tables, and the team adds them into its shared ring with shared-memory
// integer atomics (order-independent, so the raster stays bit-exact).  Every mailbox word
// carries the step's rank in the launch, so a reader tells a fresh word from an old one
// without any other handshake (the host zeroes the mailboxes before each launch).  A CTA
// appends its own spikes to the raster with one atomic on the raster cursor per step
// that has any.
//
// The two warp groups of a CTA run their own loops:
//   neuron warps:   for each t: wait until D(t-1) is complete in this CTA, then B(t)
//                   (I <- p11 I + (W[t] + T w_ext) 2^-12, W[t] <- 0), A(t+1) (the U update
//                   and threshold of step t+1), the mailboxes of step t+1, and the thalamic
//                   draws of step t+1;
//   delivery warps: for each t: D(t), step t's spikes from the inbox into the shared ring,
//                   as soon as every CTA's slot of step t is written; then a release of the
//                   count of delivered steps.
// A(t+1) needs only B(t); B(t+1) needs D(t) (delay 1), which the count orders; D(t) writes
// rows t+1 .. t+63, never row t, and D(t+1) cannot start before this CTA's own slot of step
// t+1, written after its B(t).  A mailbox buffer is reused every four steps: no CTA can be
// more than two steps ahead of a reader.  Every wait is bounded (`barrier_timeout_ns`); on
// timeout the CTA records SNN_ETIMEOUT in the control block and every CTA leaves its loops.
//
// No FMA in the neuron arithmetic (__fmul_rn / __fadd_rn), as in the other engines.
#include <cuda_runtime.h>

#include "internal.hpp"
#include "philox.cuh"

namespace snn {

namespace {

constexpr int kResidentMaxThreads = 32 * kResidentMaxWarps;  // neuron warps + two delivery teams
constexpr int kResU = 8;  // synapses in flight per lane of a delivery warp
constexpr int kJmapShift = 5;  // the flattened synapse list in chunks of 32 ...
constexpr int kJmap = 256;     // ... the first kJmap of which map to the spike holding their first synapse

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t v;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
    return v;
}

__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed_v4u32(uint32_t *p, uint32_t x, uint32_t y, uint32_t z, uint32_t w)
{
    asm volatile("st.relaxed.gpu.global.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(x), "r"(y), "r"(z), "r"(w)
                 : "memory");
}

__device__ __forceinline__ uint4 ld_relaxed_v4u32(const uint32_t *p)
{
    uint4 v;
    asm volatile("ld.relaxed.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p)
                 : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Shared-memory flag between the CTA's warp groups: release after the adds it covers,
// acquire before the reads that need them.
__device__ __forceinline__ void st_release_shared(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.cta.shared.u32 [%0], %1;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(p))),
                 "r"(v)
                 : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire_shared(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.cta.shared.u32 %0, [%1];"
                 : "=r"(v)
                 : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(p)))
                 : "memory");
    return v;
}

__device__ __forceinline__ void st_volatile_shared(uint32_t *p, uint32_t v) { *reinterpret_cast<volatile uint32_t *>(p) = v; }
__device__ __forceinline__ uint32_t ld_volatile_shared(const uint32_t *p) { return *reinterpret_cast<const volatile uint32_t *>(p); }

__device__ __forceinline__ void red_add_s32(int32_t *addr, int32_t v)
{
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(addr), "r"(v) : "memory");
}

// Barrier among the `n` threads of one warp group (ids 1 and 2; 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// The same barrier, returning to every participant whether any of them passed v = true.
__device__ __forceinline__ bool group_sync_or(int id, int n, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pin, pout;\n\tsetp.ne.u32 pin, %1, 0;\n\t"
        "bar.red.or.pred pout, %2, %3, pin;\n\tselp.u32 %0, 1, 0, pout;\n\t}"
        : "=r"(r)
        : "r"(static_cast<uint32_t>(v)), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}

// Shared memory of one CTA, in bytes from the start of the dynamic allocation.
struct ResLayout {
    size_t ring, lens, coarse, thr, base, wsum, own, glist, sstart, soff, jmap, misc, total;
};

__host__ __device__ constexpr size_t res_up16(size_t x) { return (x + 15) & ~size_t{15}; }

__host__ __device__ inline ResLayout res_layout(int rows, int stride, int lens_stride, int coarse_stride)
{
    ResLayout L{};
    L.ring = 0;                                                                   // int32 [rows][stride]
    L.lens = res_up16(L.ring + sizeof(int32_t) * size_t(rows) * stride);          // u8 [lens_stride]
    L.coarse = res_up16(L.lens + size_t(lens_stride));                            // u32 [coarse_stride]
    L.thr = res_up16(L.coarse + sizeof(uint32_t) * size_t(coarse_stride));        // u64 [8][24]
    L.base = res_up16(L.thr + sizeof(uint64_t) * SNN_MAX_POPS * kPK);             // int32 [blocks + 1]
    L.wsum = res_up16(L.base + sizeof(int32_t) * (kResidentMaxBlocks + 1));       // int32 [2 teams][32] warp sums
    L.own = res_up16(L.wsum + sizeof(int32_t) * 2 * 32);                          // u16 [2][stride]
    L.glist = res_up16(L.own + sizeof(uint16_t) * 2 * stride);                    // int32 [2 teams][gather]
    L.sstart = res_up16(L.glist + sizeof(int32_t) * 2 * kResidentGather);         // u32 [2][gather] segment starts
    L.soff = res_up16(L.sstart + sizeof(uint32_t) * 2 * kResidentGather);         // u32 [2][gather] flattened offsets
    L.jmap = res_up16(L.soff + sizeof(uint32_t) * 2 * kResidentGather);           // u16 [2][kJmap] chunk -> spike
    L.misc = res_up16(L.jmap + sizeof(uint16_t) * 2 * kJmap);                     // counters and flags
    L.total = res_up16(L.misc + 64);
    return L;
}

struct ResMisc {
    uint32_t own_cnt[2];  // neuron warps: own spikes of the step with parity s, in own[s & 1]
    uint32_t d_done[2];   // per delivery team: rank in the launch of its last step delivered into the ring
    uint32_t abort;       // a bounded wait timed out: every warp group leaves its loop
};

// Mailbox words carry the step's rank in the launch: a header its low 20 bits above the
// 12-bit spike count, an entry its low 22 bits above the sender's 10-bit index in its
// block.  Every word is read whole, so each one tells by itself whether it is fresh.
constexpr uint32_t kHeaderTagMask = (1u << 20) - 1;
constexpr uint32_t kEntryTagMask = (1u << 22) - 1;

__device__ __forceinline__ bool entry_ok(uint32_t v, uint32_t etag) { return (v >> 10) == etag; }

__device__ __forceinline__ uint32_t poisson_count_s(uint64_t v, const uint64_t (&r)[8], const uint64_t *thr_row)
{
    uint32_t T = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) T += (v >= r[k]) ? 1u : 0u;
    if (T == 8u)
        while (T < static_cast<uint32_t>(kPK) && v >= thr_row[T]) ++T;
    return T;
}

// Waits until mailbox entry `word` carries tag `etag`; false if the wait ran past the
// bound or another CTA recorded a timeout.
__device__ __forceinline__ bool wait_entry(const uint32_t *word, uint32_t etag, uint32_t &v, const StepArgs &a)
{
    v = ld_relaxed_u32(word);
    if (entry_ok(v, etag)) return true;
    const uint64_t t_start = global_ns();
    for (uint32_t spins = 1;; ++spins) {
        v = ld_relaxed_u32(word);
        if (entry_ok(v, etag)) return true;
        if ((spins & 31u) == 0) {
            if (global_ns() - t_start > a.barrier_timeout_ns) return false;
            if (ld_relaxed_u32(&a.ctl->err) & kErrTimeout) return false;
        }
    }
}

// Segment of sender s in block p's region: first record (relative to the region) and
// length, from the CTA's shared tables (8-bit lengths and one offset per 32 senders);
// a group of 32 senders with an escaped length reads its exact offsets from global memory.
__device__ __forceinline__ void res_segment(const StepArgs &a, const uint32_t *s_coarse, const uint8_t *s_lens, int p,
                                            int32_t s, uint32_t &st, uint32_t &ln)
{
    st = 0;
    ln = 0;
    if (static_cast<uint32_t>(s) >= static_cast<uint64_t>(a.n)) return;
    const uint32_t c = s_coarse[s >> 5];
    if (c & kResidentGroupFlag) {  // an escaped length in the group: exact offsets
        const uint32_t *o = a.res_offt + static_cast<int64_t>(p) * (a.n + 1) + s;
        st = __ldcg(o);
        ln = __ldcg(o + 1) - st;
        return;
    }
    const uint4 *gl = reinterpret_cast<const uint4 *>(s_lens + (s & ~31));
    const uint4 lo4 = gl[0], hi4 = gl[1];
    const uint32_t wv8[8] = {lo4.x, lo4.y, lo4.z, lo4.w, hi4.x, hi4.y, hi4.z, hi4.w};
    const int before_s = s & 31;
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int nb = min(max(before_s - 4 * k, 0), 4);
        const uint32_t mask = nb == 4 ? 0xFFFFFFFFu : ((1u << (8 * nb)) - 1u);
        acc = __dp4a(wv8[k] & mask, 0x01010101u, acc);
    }
    st = c + acc;
    ln = s_lens[s];
}

// The m spikes' segments (t_sstart: first record, t_soff: offset in their concatenation,
// Tt records in all; t_jmap: the spike holding each chunk of 32 records' first record)
// added into the block's ring columns: thread gt of the G takes records gt, gt + G, ...,
// kResU at a time, each one 8-byte record (weight, local target | delay << 16).
__device__ __forceinline__ void res_adds(const StepArgs &a, int32_t *s_ring, const uint32_t *t_sstart,
                                         const uint32_t *t_soff, const uint16_t *t_jmap, int m, uint32_t Tt, int gt,
                                         int G, int64_t rbase, int32_t base, int32_t width, int64_t t, int rows,
                                         int stride, bool full_ring)
{
    const int rmask = rows - 1;
    const int2 *rec8 = reinterpret_cast<const int2 *>(a.res_rec);
    for (uint32_t e0 = 0; e0 < Tt; e0 += static_cast<uint32_t>(G) * kResU) {
        int2 rv[kResU];
#pragma unroll
        for (int u = 0; u < kResU; ++u) {
            const uint32_t e = e0 + static_cast<uint32_t>(gt + G * u);
            rv[u] = make_int2(0, 0);
            if (e < Tt) {
                // the last spike whose segment starts at or before e: from the spike
                // holding e's chunk start, a short walk forward (segments of empty spikes
                // share their offset)
                int lo_j;
                if ((e >> kJmapShift) < static_cast<uint32_t>(kJmap)) {
                    lo_j = t_jmap[e >> kJmapShift];
                } else {
                    int lo = 0, hi = m - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (t_soff[mid] <= e) lo = mid;
                        else hi = mid - 1;
                    }
                    lo_j = lo;
                }
                while (lo_j + 1 < m && t_soff[lo_j + 1] <= e) ++lo_j;
                const int64_t idx = rbase + t_sstart[lo_j] + (e - t_soff[lo_j]);
                rv[u] = __ldcg(rec8 + idx);
            }
        }
#pragma unroll
        for (int u = 0; u < kResU; ++u) {
            const int lt = rv[u].y & 0xFFFF;
            if (rv[u].x == 0 || lt >= width) continue;
            const int d = static_cast<int>(static_cast<uint32_t>(rv[u].y) >> 16);
            if (full_ring || d < rows)
                atomicAdd(s_ring + ((t + d) & rmask) * stride + lt, rv[u].x);
            else
                red_add_s32(a.ring + ((t + d) & kDMask) * a.npad + base + lt, rv[u].x);
        }
    }
}

__global__ void __launch_bounds__(kResidentMaxThreads, 1) k_resident(const StepArgs a, const int64_t n_steps)
{
    extern __shared__ int4 res_smem4[];
    uint8_t *sm = reinterpret_cast<uint8_t *>(res_smem4);
    const int rows = a.res_rows, stride = a.res_stride;
    const ResLayout SL = res_layout(rows, stride, a.res_lens_stride, a.res_coarse_stride);
    int32_t *s_ring = reinterpret_cast<int32_t *>(sm + SL.ring);
    uint8_t *s_lens = sm + SL.lens;
    uint32_t *s_coarse = reinterpret_cast<uint32_t *>(sm + SL.coarse);
    uint64_t *s_thr = reinterpret_cast<uint64_t *>(sm + SL.thr);
    int32_t *s_base = reinterpret_cast<int32_t *>(sm + SL.base);
    int32_t *s_wsum = reinterpret_cast<int32_t *>(sm + SL.wsum);
    uint16_t *s_own = reinterpret_cast<uint16_t *>(sm + SL.own);
    int32_t *s_glist = reinterpret_cast<int32_t *>(sm + SL.glist);
    uint32_t *s_sstart = reinterpret_cast<uint32_t *>(sm + SL.sstart);
    uint32_t *s_soff = reinterpret_cast<uint32_t *>(sm + SL.soff);
    uint16_t *s_jmap = reinterpret_cast<uint16_t *>(sm + SL.jmap);
    ResMisc *s_misc = reinterpret_cast<ResMisc *>(sm + SL.misc);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NW = a.neuron_warps, DW = a.delivery_warps;
    const int B = a.n_blocks;
    const int p = blockIdx.x;
    const int rmask = rows - 1;
    const bool full_ring = rows == kDMax;
    Ctl *ctl = a.ctl;
    const int64_t t0 = ctl->t_base;
    const int64_t tend = t0 + n_steps;
    const int32_t base = __ldg(a.blk_off + p);
    const int32_t width = __ldg(a.blk_off + p + 1) - base;
    const int32_t wpad = (width + 3) & ~3;
    const int64_t npad = a.npad;

    // ---- set-up: tables, block bounds, the block's segment tables and ring columns ----
    for (int j = threadIdx.x; j < SNN_MAX_POPS * kPK; j += blockDim.x) s_thr[j] = (&a.tables->thresholds[0][0])[j];
    {
        const int4 *src = reinterpret_cast<const int4 *>(a.res_lens + static_cast<int64_t>(p) * a.res_lens_stride);
        for (int j = threadIdx.x; j < a.res_lens_stride / 16; j += blockDim.x)
            reinterpret_cast<int4 *>(s_lens)[j] = __ldcg(src + j);
        const uint32_t *cs = a.res_coarse + static_cast<int64_t>(p) * a.res_coarse_stride;
        for (int j = threadIdx.x; j < a.res_coarse_stride; j += blockDim.x) s_coarse[j] = __ldcg(cs + j);
    }
    const int64_t rbase = __ldg(a.res_rbase + p);  // first record of this block's region
    for (int j = threadIdx.x; j <= B; j += blockDim.x) s_base[j] = __ldg(a.blk_off + j);
    if (threadIdx.x == 0) {
        s_misc->own_cnt[0] = 0;
        s_misc->own_cnt[1] = 0;
        s_misc->d_done[0] = 0;
        s_misc->d_done[1] = 0;
        s_misc->abort = 0;
    }
    // shared row r holds the ring row of the step in [t0, t0 + rows) congruent to r
    for (int idx = threadIdx.x; idx < rows * (stride >> 2); idx += blockDim.x) {
        const int r = idx / (stride >> 2);
        const int c = (idx - r * (stride >> 2)) * 4;
        int4 v = make_int4(0, 0, 0, 0);
        if (c < wpad) {
            const int64_t slot = (t0 + ((r - t0) & rmask)) & kDMask;
            int4 *g = reinterpret_cast<int4 *>(a.ring + slot * npad + base + c);
            v = __ldcg(g);
            if (!full_ring) __stcg(g, make_int4(0, 0, 0, 0));
        }
        *reinterpret_cast<int4 *>(s_ring + r * stride + c) = v;
    }
    __syncthreads();

    const bool is_neuron = warp < NW;
    const int q = warp * 32 + lane;
    const int i0 = 4 * q;  // local index of the lane's first neuron
    const bool active = is_neuron && i0 < width;
    const int64_t g0 = static_cast<int64_t>(base) + i0;
    float uu[4] = {0.f, 0.f, 0.f, 0.f}, cc[4] = {0.f, 0.f, 0.f, 0.f};
    uint32_t rr[4] = {0, 0, 0, 0};

    if (is_neuron) {
        // ====== neuron warps: B(t), then A(t+1), the mailboxes of step t+1 and its draws ======
        uint32_t pops = 0;
        int b0 = 0;
        uint64_t tr[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int32_t thal[4] = {0, 0, 0, 0};    // thalamic input T w_ext of the next B, drawn ahead of time
        int4 gw4 = make_int4(0, 0, 0, 0);  // global ring row of the next B (rows < 64 only)
        if (active) {
            const float4 u4 = *reinterpret_cast<const float4 *>(a.U + g0);
            const float4 c4 = *reinterpret_cast<const float4 *>(a.I + g0);
            const uint32_t r4 = *reinterpret_cast<const uint32_t *>(a.R + g0);
            uu[0] = u4.x; uu[1] = u4.y; uu[2] = u4.z; uu[3] = u4.w;
            cc[0] = c4.x; cc[1] = c4.y; cc[2] = c4.z; cc[3] = c4.w;
            rr[0] = r4 & 0xFFu; rr[1] = (r4 >> 8) & 0xFFu; rr[2] = (r4 >> 16) & 0xFFu; rr[3] = r4 >> 24;
            pops = __ldg(reinterpret_cast<const unsigned int *>(a.pop_id + g0));
            b0 = pops & 0xFF;
#pragma unroll
            for (int k = 0; k < 8; ++k) tr[k] = s_thr[b0 * kPK + k];
        }
        for (int64_t t = t0 - 1; t < tend; ++t) {
            if (t >= t0) {
                // D(t-1) must be complete in this CTA before row t is read (delay 1 adds to it)
                bool stop = false;
                if (warp == 0 && lane == 0) {
                    // the list of step t+1 starts empty (its last reader, the mailbox of step
                    // t-1, was written by this thread's own warp)
                    s_misc->own_cnt[(t + 1) & 1] = 0;
                    // D(t-1) and D(t-2) come from different teams; each team delivers its
                    // steps in order, so these two bound every earlier step as well
                    const uint32_t r1 = static_cast<uint32_t>(t - t0);  // rank of step t-1 (0: none)
                    const uint32_t need_a = r1, need_b = r1 > 1 ? r1 - 1 : 0;
                    uint32_t *done_a = &s_misc->d_done[(r1 + 1) & 1], *done_b = &s_misc->d_done[r1 & 1];
                    if (ld_acquire_shared(done_a) < need_a || ld_acquire_shared(done_b) < need_b) {
                        const uint64_t t_start = global_ns();
                        for (uint32_t spins = 1;; ++spins) {
                            if (ld_acquire_shared(done_a) >= need_a && ld_acquire_shared(done_b) >= need_b) break;
                            if (ld_volatile_shared(&s_misc->abort)) {
                                stop = true;
                                break;
                            }
                            if ((spins & 255u) == 0 && global_ns() - t_start > 2 * a.barrier_timeout_ns) {
                                stop = true;
                                atomicOr(&ctl->err, kErrTimeout);
                                break;
                            }
                        }
                    }
                }
                if (group_sync_or(1, NW * 32, stop)) break;
                if (active) {
                    // B(t): input of step t from the ring row, then cleared (§3.2)
                    int4 *srow = reinterpret_cast<int4 *>(s_ring + (t & rmask) * stride + i0);
                    int4 w4 = *srow;
                    *srow = make_int4(0, 0, 0, 0);
                    if (!full_ring) {
                        w4.x = static_cast<int32_t>(static_cast<uint32_t>(w4.x) + static_cast<uint32_t>(gw4.x));
                        w4.y = static_cast<int32_t>(static_cast<uint32_t>(w4.y) + static_cast<uint32_t>(gw4.y));
                        w4.z = static_cast<int32_t>(static_cast<uint32_t>(w4.z) + static_cast<uint32_t>(gw4.z));
                        w4.w = static_cast<int32_t>(static_cast<uint32_t>(w4.w) + static_cast<uint32_t>(gw4.w));
                    }
                    const int32_t ww[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int32_t in = static_cast<int32_t>(static_cast<uint32_t>(ww[j]) + static_cast<uint32_t>(thal[j]));
                        cc[j] = __fadd_rn(__fmul_rn(a.p11, cc[j]), __fmul_rn(__int2float_rn(in), 0x1p-12f));
                    }
                }
            }
            if (t + 1 >= tend) continue;
            // A(t+1): membrane update, threshold, reset and refractoriness (Eqs. mem, ref)
            int32_t spk[4] = {0, 0, 0, 0};
            if (active) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (i0 + j >= width) continue;
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
            }
            // the block's spikes of step t+1 (index in the block)
            const int par = static_cast<int>((t + 1) & 1);
            const int cnt = spk[0] + spk[1] + spk[2] + spk[3];
            if (__ballot_sync(0xFFFFFFFFu, cnt != 0)) {
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                    if (lane >= o) incl += v;
                }
                const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
                uint32_t wbase = 0;
                if (lane == 31) wbase = atomicAdd(&s_misc->own_cnt[par], static_cast<uint32_t>(total));
                wbase = __shfl_sync(0xFFFFFFFFu, wbase, 31);
                int k = static_cast<int>(wbase) + incl - cnt;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (spk[j]) s_own[par * stride + k++] = static_cast<uint16_t>(i0 + j);
            }
            group_sync(1, NW * 32);
            uint32_t n_raster = 0, rpos = 0;  // warp 0: own spikes of step t+1 and their raster position
            if (warp == 0) {
                // mailboxes of step t+1: one slot in every CTA's inbox (header and the first
                // three spikes), the other spikes once in this CTA's outbox
                const uint32_t rel = static_cast<uint32_t>(t + 1 - t0 + 1);
                const uint32_t n_own = s_misc->own_cnt[par];
                const uint32_t etag = (rel & kEntryTagMask) << 10;
                const uint16_t *own = s_own + par * stride;
                const size_t buf = static_cast<size_t>((t + 1) & 3);
                uint32_t *ob = a.mbox + (buf * B + p) * kResidentMboxWords;
                for (uint32_t j = 3 + lane; j < n_own; j += 32) st_relaxed_u32(ob + j, etag | own[j]);
                const uint32_t h = ((rel & kHeaderTagMask) << 12) | n_own;
                const uint32_t e0 = n_own > 0 ? (etag | own[0]) : 0u, e1 = n_own > 1 ? (etag | own[1]) : 0u;
                const uint32_t e2 = n_own > 2 ? (etag | own[2]) : 0u;
                // B(t) of every neuron warp (ordered by the group barrier) before the slots:
                // this CTA's own delivery of step t+1 adds into ring row t with d = 63
                __threadfence_block();
                uint32_t *slots = a.inbox + (buf * B * B + p) * kResidentSlotWords;  // reader c's slot: + c * B * 4
                for (int c = lane; c < B; c += 32)
                    st_relaxed_v4u32(slots + static_cast<size_t>(c) * B * kResidentSlotWords, h, e0, e1, e2);
                // raster space for the own spikes; the position is used after the draws, so
                // the atomic's round trip overlaps them
                n_raster = n_own;
                if (n_own > 0 && lane == 0) rpos = atomicAdd(&ctl->cursor, n_own);
            }
            if (active) {
                // thalamic input of step t+1 (counter-based: independent of the dynamics)
                const Block4 r4 = philox4x64_10(static_cast<uint64_t>(t + 1), static_cast<uint64_t>(g0 >> 2), 0, 0,
                                                a.seed, kStreamThalamic);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int b = (pops >> (8 * j)) & 0xFF;
                    const uint64_t v = r4.w[j] >> 1;
                    uint32_t T;
                    if (b == b0) {
                        T = poisson_count_s(v, tr, s_thr + b0 * kPK);
                    } else {
                        const uint64_t *thr = s_thr + b * kPK;
                        T = 0;
                        while (T < static_cast<uint32_t>(kPK) && v >= thr[T]) ++T;
                    }
                    thal[j] = static_cast<int32_t>(T * static_cast<uint32_t>(a.w_ext_fx));
                }
                if (!full_ring) {
                    // delays >= rows reached global row t+1 at least rows - 1 steps ago, and a
                    // fence in the delivery warps at least every rows / 2 steps has made them
                    // visible; read and clear each entry in one atomic
                    int32_t *g = a.ring + ((t + 1) & kDMask) * npad + g0;
                    gw4.x = atomicExch(g, 0);
                    gw4.y = atomicExch(g + 1, 0);
                    gw4.z = atomicExch(g + 2, 0);
                    gw4.w = atomicExch(g + 3, 0);
                }
            }
            if (warp == 0 && n_raster > 0) {
                // the own spikes of step t+1 into the raster (the reader orders entries by
                // step and neuron); own[(t + 1) & 1] is rewritten only by A(t+3)
                rpos = __shfl_sync(0xFFFFFFFFu, rpos, 0);
                const uint16_t *own = s_own + par * stride;
                for (uint32_t j = lane; j < n_raster; j += 32) {
                    const uint64_t pos = static_cast<uint64_t>(rpos) + j;
                    if (pos < a.rast_cap) {
                        a.rast_nrn[pos] = base + own[j];
                        a.rast_t[pos] = static_cast<int32_t>(t + 1);
                    }
                }
                if (lane == 0 && static_cast<uint64_t>(rpos) + n_raster > a.rast_cap) atomicOr(&ctl->err, kErrRaster);
            }
        }
    } else {
        // ====== delivery warps: two teams, each delivering every other step as soon as
        // every slot of that step is written, so that consecutive steps overlap ======
        const int dw = warp - NW;
        const int TW = DW >> 1;         // warps per team
        const int team = dw / TW;       // team k delivers the steps of rank k+1, k+3, ...
        const int tw = dw - team * TW;  // warp within the team
        const int ql = tw * 32 + lane;  // the sender whose slot this lane polls
        const int bar = 2 + team, nbar = TW * 32;
        int32_t *t_wsum = s_wsum + team * 32;  // [0, 16): counts, [16, 32): segment lengths
        int32_t *t_glist = s_glist + team * kResidentGather;
        uint32_t *t_sstart = s_sstart + team * kResidentGather;
        uint32_t *t_soff = s_soff + team * kResidentGather;
        uint16_t *t_jmap = s_jmap + team * kJmap;
        const bool stall_test = a.barrier_extra != 0 && p == 0;  // waits for a tag nobody writes
        for (int64_t t = t0 + team; t < tend; t += 2) {
            const uint32_t rel = static_cast<uint32_t>(t - t0 + 1);
            const uint32_t htag = stall_test ? kHeaderTagMask : (rel & kHeaderTagMask);
            const uint32_t etag = rel & kEntryTagMask;
            if (!full_ring) __threadfence();  // this lane's earlier long-delay adds are visible
            const size_t buf = static_cast<size_t>(t & 3);
            uint32_t cnt = 0;
            uint4 h = make_uint4(0, 0, 0, 0);
            bool ok = true;
            if (ql < B) {
                const uint32_t *sl = a.inbox + ((buf * B + p) * B + ql) * kResidentSlotWords;
                h = ld_relaxed_v4u32(sl);
                if ((h.x >> 12) != htag) {
                    const uint64_t t_start = global_ns();
                    for (uint32_t spins = 1;; ++spins) {
                        h = ld_relaxed_v4u32(sl);
                        if ((h.x >> 12) == htag) break;
                        if ((spins & 31u) == 0 && (global_ns() - t_start > a.barrier_timeout_ns ||
                                                   (ld_relaxed_u32(&ctl->err) & kErrTimeout) ||
                                                   ld_volatile_shared(&s_misc->abort))) {
                            ok = false;
                            break;
                        }
                    }
                }
                if (ok) cnt = h.x & 0xFFFu;
                if (ql == p) __threadfence_block();  // pairs with the fence before this CTA's own slots
            }
            if (!ok) atomicOr(&ctl->err, kErrTimeout);
            // exclusive prefix of the counts over the senders
            int incl = static_cast<int>(cnt);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) t_wsum[tw] = incl;
            if (group_sync_or(bar, nbar, !ok)) {
                if (tw == 0 && lane == 0) st_volatile_shared(&s_misc->abort, 1u);
                break;
            }
            int before = 0, total = 0;
            for (int w = 0; w < TW; ++w) {
                const int v = t_wsum[w];
                before += w < tw ? v : 0;
                total += v;
            }
            const int off = before + incl - static_cast<int>(cnt);
            bool late = false;  // a wait for a spike entry gave up
            const int G = nbar, gt = ql;
            // passes of kResidentGather spikes through the gather list (one at the usual load)
            for (int lo = 0; lo < total; lo += kResidentGather) {
                const int m = total - lo < kResidentGather ? total - lo : kResidentGather;
                // spikes lo .. lo + m of the step into the gather list; a slot's entries
                // may predate its header, so each is checked
                if (cnt > 0) {
                    const int j0 = lo > off ? lo - off : 0;
                    const int j1 = min(static_cast<int>(cnt), lo + m - off);
                    const uint32_t *sl = a.inbox + ((buf * B + p) * B + ql) * kResidentSlotWords;
                    const uint32_t *ob = a.mbox + (buf * B + ql) * kResidentMboxWords;
                    const int32_t src_base = s_base[ql];
                    for (int j = j0; j < j1; ++j) {
                        uint32_t v = j == 0 ? h.y : j == 1 ? h.z : h.w;
                        int32_t s_id = -1;  // no segment if the wait gives up
                        if ((j >= 3 || !entry_ok(v, etag)) && !wait_entry(j < 3 ? sl + 1 + j : ob + j, etag, v, a)) {
                            atomicOr(&ctl->err, kErrTimeout);
                            late = true;
                        } else {
                            s_id = src_base + static_cast<int32_t>(v & 0x3FFu);
                        }
                        t_glist[off + j - lo] = s_id;
                    }
                }
                group_sync(bar, nbar);
                // every spike's segment, thread gt taking spikes gt * kper .. + kper, so
                // that a prefix over threads orders them
                const int kper = (m + G - 1) / G;
                uint32_t mine = 0;
                for (int q = 0; q < kper; ++q) {
                    const int j = gt * kper + q;
                    if (j >= m) break;
                    uint32_t st = 0, ln = 0;
                    res_segment(a, s_coarse, s_lens, p, t_glist[j], st, ln);
                    t_sstart[j] = st;
                    t_soff[j] = ln;
                    mine += ln;
                }
                uint32_t sincl = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, sincl, o);
                    if (lane >= o) sincl += v;
                }
                if (lane == 31) t_wsum[16 + tw] = static_cast<int32_t>(sincl);
                group_sync(bar, nbar);
                uint32_t run = 0, Tt = 0;
                for (int w = 0; w < TW; ++w) {
                    const uint32_t v = static_cast<uint32_t>(t_wsum[16 + w]);
                    run += w < tw ? v : 0u;
                    Tt += v;
                }
                run += sincl - mine;
                for (int q = 0; q < kper; ++q) {
                    const int j = gt * kper + q;
                    if (j >= m) break;
                    const uint32_t ln = t_soff[j];
                    t_soff[j] = run;
                    for (uint32_t k = (run + 31u) >> kJmapShift; k < static_cast<uint32_t>(kJmap) &&
                                                                 (k << kJmapShift) < run + ln; ++k)
                        t_jmap[k] = static_cast<uint16_t>(j);
                    run += ln;
                }
                group_sync(bar, nbar);
                res_adds(a, s_ring, t_sstart, t_soff, t_jmap, m, Tt, gt, G, rbase, base, width, t, rows, stride,
                         full_ring);
                group_sync(bar, nbar);  // every add of this pass is done; the list may be rewritten
            }
            if (group_sync_or(bar, nbar, late)) {
                if (tw == 0 && lane == 0) st_volatile_shared(&s_misc->abort, 1u);
                break;
            }
            if (tw == 0 && lane == 0) st_release_shared(&s_misc->d_done[team], rel);
        }
    }
    if (!full_ring) __threadfence();  // the long-delay adds before the ring write-back reads them
    __syncthreads();
    if (ld_volatile_shared(&s_misc->abort)) return;  // a wait timed out: the error is recorded, the state is void
    if (p == 0 && threadIdx.x == 0) ctl->t_base = tend;  // the raster cursor advanced atomically

    // ---- write the state after tend steps back to the arena ----
    if (active) {
        *reinterpret_cast<float4 *>(a.U + g0) = make_float4(uu[0], uu[1], uu[2], uu[3]);
        *reinterpret_cast<float4 *>(a.I + g0) = make_float4(cc[0], cc[1], cc[2], cc[3]);
        *reinterpret_cast<uint32_t *>(a.R + g0) = rr[0] | (rr[1] << 8) | (rr[2] << 16) | (rr[3] << 24);
    }
    for (int idx = threadIdx.x; idx < rows * (stride >> 2); idx += blockDim.x) {
        const int r = idx / (stride >> 2);
        const int c = (idx - r * (stride >> 2)) * 4;
        if (c >= wpad) continue;
        const int64_t slot = (tend + ((r - tend) & rmask)) & kDMask;
        int4 *g = reinterpret_cast<int4 *>(a.ring + slot * npad + base + c);
        int4 v = *reinterpret_cast<const int4 *>(s_ring + r * stride + c);
        if (!full_ring) {
            const int4 o = __ldcg(g);
            v.x = static_cast<int32_t>(static_cast<uint32_t>(v.x) + static_cast<uint32_t>(o.x));
            v.y = static_cast<int32_t>(static_cast<uint32_t>(v.y) + static_cast<uint32_t>(o.y));
            v.z = static_cast<int32_t>(static_cast<uint32_t>(v.z) + static_cast<uint32_t>(o.z));
            v.w = static_cast<int32_t>(static_cast<uint32_t>(v.w) + static_cast<uint32_t>(o.w));
        }
        __stcg(g, v);
    }
}


// ---------------------------------------------------------------------------------
// Phase 2 alone on block-major records (snn_deliver_spikes of a resident-engine
// network): one CTA per target block p reads, for every sender of the list, that
// sender's segment of block p's region (offsets from the block's exact segment table),
// so all of its reads stay inside its own region, where consecutive senders' segments
// are adjacent.  Per pass of kRegBatch senders the segments are concatenated; the
// stream is taken in windows of kRegWindow records whose region index is tabled, and
// each window in pipelined sets of kRegSet rounds (lane l of warp w: records
// 32 (w + 32 k) + l), the next set's loads in flight while the current one is added.
// With at least kBlockedAggregateMin senders the weights of delays up to
// kBlockedBinDelays are summed per (delay, local target) in shared memory and added
// to the ring once at the end (only this CTA writes these ring columns); longer delays,
// and all of them for short lists, are reductions into the ring.
// ---------------------------------------------------------------------------------
constexpr int kRegThreads = 1024;
constexpr int kRegWarps = kRegThreads / 32;
constexpr int kRegBatch = 2048;   // senders per pass
constexpr int kRegWindow = 8192;  // records whose region index is tabled at once
constexpr int kRegSet = 2;        // rounds per pipelined set

__host__ __device__ inline size_t regions_smem_bytes(int stride)
{
    return sizeof(int32_t) * (size_t(kBlockedBinDelays + 1) * stride + 3 * kRegBatch + kRegWarps + kRegWindow);
}

struct RegSet {
    int32_t tg[kRegSet], w[kRegSet];
    uint32_t d[kRegSet];
};

__device__ __forceinline__ void regions_load(const StepArgs &a, int64_t rbase, const uint32_t *ridx, int32_t w0,
                                             int32_t w1, int32_t e0, int warp, int lane, RegSet &r)
{
#pragma unroll
    for (int k = 0; k < kRegSet; ++k) {
        const int32_t e = e0 + 32 * (warp + kRegWarps * k) + lane;
        r.tg[k] = 0;
        r.w[k] = 0;
        r.d[k] = 1;
        if (e < w1) {
            const int64_t idx = rbase + ridx[e - w0];
            r.tg[k] = __ldcs(a.syn_tgt + idx);
            r.w[k] = __ldcs(a.syn_w + idx);
            r.d[k] = __ldcs(a.syn_d + idx);
        }
    }
}

template <bool kAggregate>
__device__ __forceinline__ void regions_apply(const StepArgs &a, int32_t *bins, int stride, int64_t t, int32_t base,
                                              int32_t width, const RegSet &r)
{
#pragma unroll
    for (int k = 0; k < kRegSet; ++k) {
        const int lt = r.tg[k] - base;
        if (r.w[k] == 0 || static_cast<uint32_t>(lt) >= static_cast<uint32_t>(width)) continue;
        const int d = static_cast<int>(r.d[k]);
        if (kAggregate && d <= kBlockedBinDelays) atomicAdd(bins + d * stride + lt, r.w[k]);
        else red_add_s32(a.ring + ((t + d) & kDMask) * a.npad + base + lt, r.w[k]);
    }
}

template <bool kAggregate>
__device__ __forceinline__ void regions_window(const StepArgs &a, int32_t *bins, int stride, const uint32_t *ridx,
                                               int32_t w0, int32_t w1, int64_t t, int32_t base, int32_t width,
                                               int64_t rbase)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int32_t kStep = kRegThreads * kRegSet;
    RegSet A, Bs;
    int32_t e0 = w0;
    regions_load(a, rbase, ridx, w0, w1, e0, warp, lane, A);
    for (;;) {
        if (e0 + kStep < w1) regions_load(a, rbase, ridx, w0, w1, e0 + kStep, warp, lane, Bs);
        regions_apply<kAggregate>(a, bins, stride, t, base, width, A);
        e0 += kStep;
        if (e0 >= w1) break;
        if (e0 + kStep < w1) regions_load(a, rbase, ridx, w0, w1, e0 + kStep, warp, lane, A);
        regions_apply<kAggregate>(a, bins, stride, t, base, width, Bs);
        e0 += kStep;
        if (e0 >= w1) break;
    }
}

// Exclusive prefix over the CTA of one value per thread into out[threadIdx.x]; returns
// the total.
__device__ __forceinline__ int32_t regions_scan(int32_t v, int32_t *out, int32_t *warp_sums)
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
        int32_t w = lane < kRegWarps ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kRegWarps) warp_sums[lane] = w;
    }
    __syncthreads();
    out[threadIdx.x] = (warp > 0 ? warp_sums[warp - 1] : 0) + x - v;
    return warp_sums[kRegWarps - 1];
}

__global__ void __launch_bounds__(kRegThreads, 1)
    k_deliver_regions(const StepArgs a, const int32_t *list, int64_t nspk, int64_t t)
{
    extern __shared__ int4 reg_smem4[];
    const int stride = a.res_stride;
    int32_t *bins = reinterpret_cast<int32_t *>(reg_smem4);                            // [33][stride]
    uint32_t *seg_st = reinterpret_cast<uint32_t *>(bins + (kBlockedBinDelays + 1) * stride);  // [kRegBatch]
    int32_t *pfx = reinterpret_cast<int32_t *>(seg_st + kRegBatch);                    // [kRegBatch]
    int32_t *seg_n = pfx + kRegBatch;                                                  // [kRegBatch]
    int32_t *warp_sums = seg_n + kRegBatch;                                            // [kRegWarps]
    uint32_t *ridx = reinterpret_cast<uint32_t *>(warp_sums + kRegWarps);              // [kRegWindow]

    const int p = blockIdx.x, tid = threadIdx.x;
    const int32_t base = __ldg(a.blk_off + p);
    const int32_t width = __ldg(a.blk_off + p + 1) - base;
    const int64_t rbase = __ldg(a.res_rbase + p);
    const uint32_t *offt = a.res_offt + static_cast<int64_t>(p) * (a.n + 1);
    const bool aggregate = nspk >= kBlockedAggregateMin;
    constexpr int kPer = kRegBatch / kRegThreads;
    if (aggregate)
        for (int j = tid; j < (kBlockedBinDelays + 1) * stride; j += kRegThreads) bins[j] = 0;
    for (int64_t b0 = 0; b0 < nspk; b0 += kRegBatch) {
        const int nb = static_cast<int>(nspk - b0 < kRegBatch ? nspk - b0 : kRegBatch);
        int32_t mine = 0;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int j = tid * kPer + i;
            int32_t len = 0;
            if (j < nb) {
                const int32_t s = __ldcg(list + b0 + j);
                if (static_cast<uint32_t>(s) < static_cast<uint64_t>(a.n)) {
                    const uint32_t st = __ldg(offt + s);
                    seg_st[j] = st;
                    len = static_cast<int32_t>(__ldg(offt + s + 1) - st);
                }
            }
            seg_n[j] = len;
            mine += len;
        }
        int32_t *scan_out = reinterpret_cast<int32_t *>(ridx);  // the window table is idle here
        const int32_t total = regions_scan(mine, scan_out, warp_sums);
        {
            int32_t run = scan_out[tid];
#pragma unroll
            for (int i = 0; i < kPer; ++i) {
                pfx[tid * kPer + i] = run;
                run += seg_n[tid * kPer + i];
            }
        }
        __syncthreads();
        for (int32_t w0 = 0; w0 < total; w0 += kRegWindow) {
            const int32_t w1 = total - w0 < kRegWindow ? total : w0 + kRegWindow;
#pragma unroll
            for (int i = 0; i < kPer; ++i) {
                const int j = tid * kPer + i;
                if (j >= nb) break;
                const int32_t lo = max(pfx[j], w0), hi = min(pfx[j] + seg_n[j], w1);
                const uint32_t r0 = seg_st[j] - static_cast<uint32_t>(pfx[j]);
                for (int32_t e = lo; e < hi; ++e) ridx[e - w0] = r0 + static_cast<uint32_t>(e);
            }
            __syncthreads();
            if (aggregate) regions_window<true>(a, bins, stride, ridx, w0, w1, t, base, width, rbase);
            else regions_window<false>(a, bins, stride, ridx, w0, w1, t, base, width, rbase);
            __syncthreads();  // the table is rebuilt for the next window
        }
    }
    if (!aggregate) return;
    // the sums of delays 1..kBlockedBinDelays into their ring rows (plain read-modify-
    // writes: only this CTA writes these columns during the launch); stride and the ring
    // row are multiples of 4, and the last block's extra columns lie inside the padded row
    const int w4 = (width + 3) >> 2, s4 = stride >> 2;
    for (int q = tid; q < kBlockedBinDelays * w4; q += kRegThreads) {
        const int d = 1 + q / w4;
        const int c4 = q - (d - 1) * w4;
        const int4 v = reinterpret_cast<const int4 *>(bins)[d * s4 + c4];
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

int64_t resident_width(int64_t n, int num_sms)
{
    const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(num_sms, kResidentMaxBlocks));
    int64_t w = (n + ctas - 1) / ctas;
    w = (w + kResidentAlign - 1) / kResidentAlign * kResidentAlign;
    w = std::max<int64_t>(w, kResidentAlign);
    return w > kResidentMaxWidth ? 0 : w;
}

size_t resident_smem_bytes(int rows, int stride, int64_t n)
{
    const ResTables T = resident_tables(n, 1);
    return res_layout(rows, stride, static_cast<int>(T.lens_stride), static_cast<int>(T.coarse_stride)).total;
}

int resident_rows(int stride, int cap, int64_t n)
{
    for (int rows = kDMax; rows >= 8; rows >>= 1)
        if ((cap <= 0 || rows <= cap) && resident_smem_bytes(rows, stride, n) <= 232448) return rows;
    return 0;
}

int prepare_resident_kernel(const StepArgs &a)
{
    cudaError_t e = cudaFuncSetAttribute(k_resident, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(resident_smem_bytes(a.res_rows, a.res_stride, a.n)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_deliver_regions, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(regions_smem_bytes(a.res_stride)));
    return static_cast<int>(e);
}

int launch_deliver_regions(const StepArgs &a, const int32_t *list, int64_t n, int64_t t, void *stream)
{
    k_deliver_regions<<<a.n_blocks, kRegThreads, regions_smem_bytes(a.res_stride), static_cast<cudaStream_t>(stream)>>>(
        a, list, n, t);
    return static_cast<int>(cudaGetLastError());
}

int resident_blocks_per_sm(const StepArgs &a)
{
    int nb = 0;
    const int threads = 32 * (a.neuron_warps + a.delivery_warps);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_resident, threads,
                                                      resident_smem_bytes(a.res_rows, a.res_stride, a.n)) != cudaSuccess)
        return 0;
    return nb;
}

int launch_resident(const StepArgs &a, int64_t n_steps, void *stream)
{
    StepArgs args = a;
    int64_t n = n_steps;
    void *params[] = {&args, &n};
    const cudaError_t e = cudaLaunchCooperativeKernel(
        reinterpret_cast<const void *>(k_resident), dim3(a.n_blocks), dim3(32 * (a.neuron_warps + a.delivery_warps)),
        params, resident_smem_bytes(a.res_rows, a.res_stride, a.n), static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? 0 : static_cast<int>(e);
}

}  // namespace snn
