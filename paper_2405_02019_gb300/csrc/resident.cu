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
//   - each sender's row is stored grouped by target block (delay order kept inside a
//     block), and the CTA's own row of a segment table says where each row's segment into
//     its block starts and how long it is, so the CTA reads only the synapses that land
//     in its block (the indexed store of §3.5 split by target).
// The only traffic between CTAs is the spike list of every step.  After deciding its
// spikes, a CTA writes, into one 32-byte inbox slot per reading CTA, the step's spike
// count and up to three spikes (its index in the block and the row's offset); further
// spikes go once into its outbox.  Each CTA thus polls only lines that it alone reads.
// It then adds its segments of those rows into its shared ring with shared-memory integer
// atomics (order-independent, so the raster stays bit-exact).  Every mailbox word carries
// the step's rank in the launch, so a reader tells a fresh word from an old one without
// any other handshake (the host zeroes the mailboxes before each launch).
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

constexpr int kResidentMaxThreads = 32 * (kResidentMaxWidth / 128 + 8);  // neuron + delivery warps
constexpr int kResU = 4;  // synapses in flight per lane of a delivery warp

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t v;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed_v2u64(uint64_t *p, uint64_t x, uint64_t y)
{
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(x), "l"(y) : "memory");
}

__device__ __forceinline__ ulonglong2 ld_relaxed_v2u64(const uint64_t *p)
{
    ulonglong2 v;
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
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

__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
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
    size_t ring, thr, base, wsum, own, glist, misc, total;
};

__host__ __device__ constexpr size_t res_up16(size_t x) { return (x + 15) & ~size_t{15}; }

__host__ __device__ inline ResLayout res_layout(int rows, int stride)
{
    ResLayout L{};
    L.ring = 0;                                                                   // int32 [rows][stride]
    L.thr = res_up16(L.ring + sizeof(int32_t) * size_t(rows) * stride);           // u64 [8][24]
    L.base = res_up16(L.thr + sizeof(uint64_t) * SNN_MAX_POPS * kPK);             // int32 [blocks + 1]
    L.wsum = res_up16(L.base + sizeof(int32_t) * (kResidentMaxBlocks + 1));       // int32 [16] warp sums
    L.own = res_up16(L.wsum + sizeof(int32_t) * 16);                              // u64 [2][stride]
    L.glist = res_up16(L.own + sizeof(uint64_t) * 2 * stride);                    // u64 [gather]
    L.misc = res_up16(L.glist + sizeof(uint64_t) * kResidentGather);              // counters and flags
    L.total = res_up16(L.misc + 64);
    return L;
}

struct ResMisc {
    uint32_t own_cnt[2];  // neuron warps: own spikes of the step with parity s, in own[s & 1]
    uint32_t d_done;      // steps of this launch whose delivery into the shared ring is complete
    uint32_t abort;       // a bounded wait timed out: both warp groups leave their loops
};

// Mailbox words (64-bit, so that a word is read whole) carry the step's rank in the
// launch in their low half: a header its low 20 bits above the 12-bit spike count, an
// entry its low 22 bits above the sender's 10-bit index in its block, with the first quad
// of the sender's row (row offset / 4) in the high half.
constexpr uint32_t kHeaderTagMask = (1u << 20) - 1;
constexpr uint32_t kEntryTagMask = (1u << 22) - 1;

__device__ __forceinline__ bool entry_ok(uint64_t v, uint32_t etag) { return (static_cast<uint32_t>(v) >> 10) == etag; }

// Largest k in [0, 32) with off_k <= e, for off nondecreasing over the lanes (off_0 = 0).
__device__ __forceinline__ int lane_of(int off, int e)
{
    int k = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int ov = __shfl_sync(0xFFFFFFFFu, off, k + step);
        if (ov <= e) k += step;
    }
    return k;
}

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
__device__ __forceinline__ bool wait_entry(const uint64_t *word, uint32_t etag, uint64_t &v, const StepArgs &a)
{
    v = ld_relaxed_u64(word);
    if (entry_ok(v, etag)) return true;
    const uint64_t t_start = global_ns();
    for (uint32_t spins = 1;; ++spins) {
        v = ld_relaxed_u64(word);
        if (entry_ok(v, etag)) return true;
        if ((spins & 31u) == 0) {
            if (global_ns() - t_start > a.barrier_timeout_ns) return false;
            if (ld_relaxed_u32(&a.ctl->err) & kErrTimeout) return false;
        }
    }
}

__global__ void __launch_bounds__(kResidentMaxThreads, 1) k_resident(const StepArgs a, const int64_t n_steps)
{
    extern __shared__ int4 res_smem4[];
    uint8_t *sm = reinterpret_cast<uint8_t *>(res_smem4);
    const int rows = a.res_rows, stride = a.res_stride;
    const ResLayout SL = res_layout(rows, stride);
    int32_t *s_ring = reinterpret_cast<int32_t *>(sm + SL.ring);
    uint64_t *s_thr = reinterpret_cast<uint64_t *>(sm + SL.thr);
    int32_t *s_base = reinterpret_cast<int32_t *>(sm + SL.base);
    int32_t *s_wsum = reinterpret_cast<int32_t *>(sm + SL.wsum);
    uint64_t *s_own = reinterpret_cast<uint64_t *>(sm + SL.own);
    uint64_t *s_glist = reinterpret_cast<uint64_t *>(sm + SL.glist);
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

    // ---- set-up: tables, block bounds, the block's ring columns ----
    for (int j = threadIdx.x; j < SNN_MAX_POPS * kPK; j += blockDim.x) s_thr[j] = (&a.tables->thresholds[0][0])[j];
    for (int j = threadIdx.x; j <= B; j += blockDim.x) s_base[j] = __ldg(a.blk_off + j);
    if (threadIdx.x == 0) {
        s_misc->own_cnt[0] = 0;
        s_misc->own_cnt[1] = 0;
        s_misc->d_done = 0;
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
        int64_t rp[5] = {0, 0, 0, 0, 0};
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
            for (int j = 0; j < 5; ++j) rp[j] = __ldg(a.row_ptr + g0 + j);
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
                    const uint32_t need = static_cast<uint32_t>(t - t0);
                    if (ld_acquire_shared(&s_misc->d_done) < need) {
                        const uint64_t t_start = global_ns();
                        for (uint32_t spins = 1;; ++spins) {
                            if (ld_acquire_shared(&s_misc->d_done) >= need) break;
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
            // the block's spikes of step t+1 (index in the block | first row quad << 32)
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
                for (int j = 0; j < 4; ++j) {
                    if (!spk[j]) continue;
                    const int64_t rs = rp[j], re = rp[j + 1];
                    s_own[par * stride + k++] = static_cast<uint64_t>(i0 + j) | static_cast<uint64_t>(rs >> 2) << 32;
                    // every CTA reads its segment of the row soon: bring the row into L2 now
                    if (re > rs) {
                        prefetch_l2(a.syn_tgt + rs, static_cast<uint32_t>(4 * (re - rs)));
                        prefetch_l2(a.syn_w + rs, static_cast<uint32_t>(4 * (re - rs)));
                        const int64_t d0 = rs & ~int64_t{15}, d1 = (re + 15) & ~int64_t{15};
                        prefetch_l2(a.syn_d + d0, static_cast<uint32_t>(d1 - d0));
                    }
                }
            }
            group_sync(1, NW * 32);
            if (warp == 0) {
                // mailboxes of step t+1: one slot in every CTA's inbox (header and the first
                // three spikes), the other spikes once in this CTA's outbox
                const uint32_t rel = static_cast<uint32_t>(t + 1 - t0 + 1);
                const uint32_t n_own = s_misc->own_cnt[par];
                const uint64_t etag = static_cast<uint64_t>((rel & kEntryTagMask) << 10);
                const uint64_t *own = s_own + par * stride;
                const size_t buf = static_cast<size_t>((t + 1) & 3);
                uint64_t *ob = a.mbox + (buf * B + p) * kResidentMboxWords;
                for (uint32_t j = 3 + lane; j < n_own; j += 32) st_relaxed_u64(ob + j, etag | own[j]);
                const uint64_t h = ((rel & kHeaderTagMask) << 12) | n_own;
                const uint64_t e0 = n_own > 0 ? (etag | own[0]) : 0, e1 = n_own > 1 ? (etag | own[1]) : 0;
                const uint64_t e2 = n_own > 2 ? (etag | own[2]) : 0;
                // B(t) of every neuron warp (ordered by the group barrier) before the slots:
                // this CTA's own delivery of step t+1 adds into ring row t with d = 63
                __threadfence_block();
                uint64_t *slots = a.inbox + (buf * B * B + p) * kResidentSlotWords;  // reader c's slot: + c * B * 4
                for (int c = lane; c < B; c += 32) {
                    uint64_t *sl = slots + static_cast<size_t>(c) * B * kResidentSlotWords;
                    st_relaxed_v2u64(sl, h, e0);
                    if (n_own > 1) st_relaxed_v2u64(sl + 2, e1, e2);
                }
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
        }
    } else {
        // ====== delivery warps: D(t) for every step, as soon as every slot of step t is written ======
        const int dw = warp - NW;
        const int ql = dw * 32 + lane;  // the sender whose slot this lane polls
        uint32_t cursor = ctl->cursor;
        const bool stall_test = a.barrier_extra != 0 && p == 0;  // waits for a tag nobody writes
        for (int64_t t = t0; t < tend; ++t) {
            const uint32_t rel = static_cast<uint32_t>(t - t0 + 1);
            const uint32_t htag = stall_test ? kHeaderTagMask : (rel & kHeaderTagMask);
            const uint32_t etag = rel & kEntryTagMask;
            if (!full_ring && (t & ((rows >> 1) - 1)) == 0) __threadfence();  // earlier long-delay adds visible
            const size_t buf = static_cast<size_t>(t & 3);
            uint32_t cnt = 0;
            ulonglong2 h = make_ulonglong2(0, 0), e = make_ulonglong2(0, 0);
            bool ok = true;
            if (ql < B) {
                const uint64_t *sl = a.inbox + ((buf * B + p) * B + ql) * kResidentSlotWords;
                h = ld_relaxed_v2u64(sl);
                e = ld_relaxed_v2u64(sl + 2);
                if ((static_cast<uint32_t>(h.x) >> 12) != htag) {
                    const uint64_t t_start = global_ns();
                    for (uint32_t spins = 1;; ++spins) {
                        h = ld_relaxed_v2u64(sl);
                        e = ld_relaxed_v2u64(sl + 2);
                        if ((static_cast<uint32_t>(h.x) >> 12) == htag) break;
                        if ((spins & 31u) == 0 && (global_ns() - t_start > a.barrier_timeout_ns ||
                                                   (ld_relaxed_u32(&ctl->err) & kErrTimeout))) {
                            ok = false;
                            break;
                        }
                    }
                }
                if (ok) cnt = static_cast<uint32_t>(h.x) & 0xFFFu;
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
            if (lane == 31) s_wsum[dw] = incl;
            if (group_sync_or(2, DW * 32, !ok)) {
                if (dw == 0 && lane == 0) st_volatile_shared(&s_misc->abort, 1u);
                break;
            }
            int before = 0, total = 0;
            for (int w = 0; w < DW; ++w) {
                const int v = s_wsum[w];
                before += w < dw ? v : 0;
                total += v;
            }
            const int off = before + incl - static_cast<int>(cnt);
            bool late = false;  // a spike entry never arrived
            for (int lo = 0; lo < total; lo += kResidentGather) {
                const int m = total - lo < kResidentGather ? total - lo : kResidentGather;
                // spikes lo .. lo + m of the step into the gather list (global index | row quad
                // << 32); a slot's entries may predate its header, so each is checked
                if (cnt > 0) {
                    const int j0 = lo > off ? lo - off : 0;
                    const int j1 = min(static_cast<int>(cnt), lo + m - off);
                    const uint64_t *sl = a.inbox + ((buf * B + p) * B + ql) * kResidentSlotWords;
                    const uint64_t *ob = a.mbox + (buf * B + ql) * kResidentMboxWords;
                    const int32_t src_base = s_base[ql];
                    for (int j = j0; j < j1; ++j) {
                        uint64_t v = j == 0 ? h.y : j == 1 ? e.x : e.y;
                        if (j >= 3 || !entry_ok(v, etag)) {
                            if (!wait_entry(j < 3 ? sl + 1 + j : ob + j, etag, v, a)) {
                                atomicOr(&ctl->err, kErrTimeout);
                                late = true;
                                v = 0;
                            }
                        }
                        const int32_t s_id = src_base + static_cast<int32_t>(v & 0x3FFu);
                        s_glist[off + j - lo] = static_cast<uint32_t>(s_id) | (v & 0xFFFFFFFF00000000ull);
                        if (ql == p) {
                            // this CTA's own spikes of step t go into the raster, in slot order
                            const uint64_t pos = static_cast<uint64_t>(cursor) + static_cast<uint64_t>(off + j);
                            if (pos < a.rast_cap) {
                                a.rast_nrn[pos] = s_id;
                                a.rast_t[pos] = static_cast<int32_t>(t);
                            }
                        }
                    }
                }
                group_sync(2, DW * 32);
                // warp dw takes spikes dw, dw + DW, ...; lane k of a round the (k+1)-th of them
                for (int jb = dw; jb < m; jb += DW * 32) {
                    const int j = jb + DW * lane;
                    int64_t start = 0;
                    int len = 0;
                    if (j < m) {
                        const uint64_t g = s_glist[j];
                        const uint32_t s = static_cast<uint32_t>(g);
                        if (s < static_cast<uint64_t>(a.n)) {
                            const uint32_t sg = __ldcg(a.res_segt + static_cast<int64_t>(p) * a.n + s);
                            start = static_cast<int64_t>(g >> 32) * 4 + (sg & 0xFFFFu);
                            len = static_cast<int>(sg >> 16);
                        }
                    }
                    int sincl = len;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int v = __shfl_up_sync(0xFFFFFFFFu, sincl, o);
                        if (lane >= o) sincl += v;
                    }
                    const int T = __shfl_sync(0xFFFFFFFFu, sincl, 31);
                    const int soff = sincl - len;
                    for (int e0 = 0; e0 < T; e0 += 32 * kResU) {
                        int32_t tg[kResU], wv[kResU];
                        uint32_t dv[kResU];
#pragma unroll
                        for (int u = 0; u < kResU; ++u) {
                            const int ei = e0 + 32 * u + lane;
                            const int k = lane_of(soff, ei < T ? ei : T - 1);
                            const int64_t st = __shfl_sync(0xFFFFFFFFu, start, k);
                            const int so = __shfl_sync(0xFFFFFFFFu, soff, k);
                            wv[u] = 0;
                            tg[u] = base;
                            dv[u] = 1;
                            if (ei < T) {
                                const int64_t idx = st + (ei - so);
                                tg[u] = __ldcg(a.syn_tgt + idx);
                                wv[u] = __ldcg(a.syn_w + idx);
                                dv[u] = __ldcg(a.syn_d + idx);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < kResU; ++u) {
                            const int lt = tg[u] - base;
                            if (wv[u] == 0 || static_cast<uint32_t>(lt) >= static_cast<uint32_t>(width)) continue;
                            const int d = static_cast<int>(dv[u]);
                            if (full_ring || d < rows)
                                atomicAdd(s_ring + ((t + d) & rmask) * stride + lt, wv[u]);
                            else
                                red_add_s32(a.ring + ((t + d) & kDMask) * npad + base + lt, wv[u]);
                        }
                    }
                }
                group_sync(2, DW * 32);  // every add of this pass is done; the list may be rewritten
            }
            cursor += static_cast<uint32_t>(total);
            if (group_sync_or(2, DW * 32, late)) {
                if (dw == 0 && lane == 0) st_volatile_shared(&s_misc->abort, 1u);
                break;
            }
            if (dw == 0 && lane == 0) st_release_shared(&s_misc->d_done, static_cast<uint32_t>(t - t0 + 1));
        }
        if (p == 0 && dw == 0 && lane == 0 && !ld_volatile_shared(&s_misc->abort)) {
            ctl->cursor = cursor;
            if (cursor > a.rast_cap) atomicOr(&ctl->err, kErrRaster);
            ctl->t_base = tend;
        }
    }
    if (!full_ring) __threadfence();  // the long-delay adds before the ring write-back reads them
    __syncthreads();
    if (ld_volatile_shared(&s_misc->abort)) return;  // a wait timed out: the error is recorded, the state is void

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

}  // namespace

int64_t resident_width(int64_t n, int num_sms)
{
    const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(num_sms, kResidentMaxBlocks));
    int64_t w = (n + ctas - 1) / ctas;
    w = (w + kResidentAlign - 1) / kResidentAlign * kResidentAlign;
    w = std::max<int64_t>(w, kResidentAlign);
    return w > kResidentMaxWidth ? 0 : w;
}

size_t resident_smem_bytes(int rows, int stride) { return res_layout(rows, stride).total; }

int resident_rows(int stride, int cap)
{
    for (int rows = kDMax; rows >= 8; rows >>= 1)
        if ((cap <= 0 || rows <= cap) && resident_smem_bytes(rows, stride) <= 232448) return rows;
    return 0;
}

int prepare_resident_kernel(const StepArgs &a)
{
    return static_cast<int>(cudaFuncSetAttribute(k_resident, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(resident_smem_bytes(a.res_rows, a.res_stride))));
}

int resident_blocks_per_sm(const StepArgs &a)
{
    int nb = 0;
    const int threads = 32 * (a.neuron_warps + a.delivery_warps);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_resident, threads,
                                                      resident_smem_bytes(a.res_rows, a.res_stride)) != cudaSuccess)
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
        params, resident_smem_bytes(a.res_rows, a.res_stride), static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? 0 : static_cast<int>(e);
}

}  // namespace snn
