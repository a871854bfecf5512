// Device side of one simulation step (sm_103a).
//
// k_update  -- Listing push of §3.1, phase 1, for every neuron, fused with the
//              ring read of §3.2 and the spike queue of Listing push2:
//                in   = W[t mod 64][i] + T(t, i) * w_ext      (int32, 2^-12 pA units)
//                W[t mod 64][i] = 0
//                if R == 0: x = p22 U + p21 I; spike if x >= theta (then x = reset, R = t_ref); U = x
//                else:      U = reset; R -= 1
//                I = p11 I + in * 2^-12
//              T is Poisson(nu_th K dt) by CDF inversion of one Philox word (§2.2).
//              Spikers are compacted warp by warp (one atomic per warp with spikes)
//              into the raster, which doubles as the step's spike queue.
// k_deliver -- Listing push2 of §3.1, phase 2: every queued spiker's row (sorted by
//              delay, §3.5) is cut into 256-synapse chunks; a warp streams a chunk
//              with 16-byte loads and adds each weight into W[(t + d) mod 64][target]
//              with a fire-and-forget int32 reduction (order-independent).
// k_advance -- moves the step counter after a batch of steps.
//
// No FMA anywhere in the neuron arithmetic: __fmul_rn / __fadd_rn round every
// product and sum on its own, matching the host reference bit for bit.
#include <cuda_runtime.h>

#include "internal.hpp"
#include "philox.cuh"

namespace snn {

namespace {

__device__ __forceinline__ void red_add_s32(int32_t *addr, int32_t v)
{
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(addr), "r"(v) : "memory");
}

// Streaming 16-byte load of read-once data (evict-first in L1/L2).
__device__ __forceinline__ int4 ld_stream4(const int32_t *p) { return __ldcs(reinterpret_cast<const int4 *>(p)); }
__device__ __forceinline__ uint32_t ld_stream_u32(const uint8_t *p)
{
    return __ldcs(reinterpret_cast<const unsigned int *>(p));
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

__global__ void __launch_bounds__(kUpdateThreads) k_update(const StepArgs a, const int k)
{
    __shared__ uint64_t s_thr[SNN_MAX_POPS * kPK];
    __shared__ int64_t s_off[SNN_MAX_POPS + 1];
    __shared__ int s_npops;
    for (int j = threadIdx.x; j < SNN_MAX_POPS * kPK; j += blockDim.x)
        s_thr[j] = (&a.tables->thresholds[0][0])[j];
    if (threadIdx.x <= SNN_MAX_POPS) s_off[threadIdx.x] = a.tables->pop_off[threadIdx.x];
    if (threadIdx.x == 0) s_npops = a.tables->n_pops;
    __syncthreads();

    const int64_t t = a.ctl->t_base + k;
    const int64_t slot = t & kDMask;
    const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;  // neuron quad
    const int64_t i0 = q * 4;
    int32_t spk[4] = {0, 0, 0, 0};

    if (i0 < a.n) {
        float4 u4 = *reinterpret_cast<const float4 *>(a.U + i0);
        float4 c4 = *reinterpret_cast<const float4 *>(a.I + i0);
        uint32_t r4 = *reinterpret_cast<const uint32_t *>(a.R + i0);
        int32_t *wrow = a.ring + slot * a.npad + i0;
        const int4 w4 = *reinterpret_cast<const int4 *>(wrow);
        *reinterpret_cast<int4 *>(wrow) = make_int4(0, 0, 0, 0);
        const Block4 rnd = philox4x64_10(static_cast<uint64_t>(t), static_cast<uint64_t>(q), 0, 0, a.seed,
                                         kStreamThalamic);
        float uu[4] = {u4.x, u4.y, u4.z, u4.w};
        float cc[4] = {c4.x, c4.y, c4.z, c4.w};
        const int32_t ww[4] = {w4.x, w4.y, w4.z, w4.w};
        uint32_t rr[4] = {r4 & 0xFFu, (r4 >> 8) & 0xFFu, (r4 >> 16) & 0xFFu, r4 >> 24};
        int b = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t i = i0 + j;
            if (i < a.n) {
                while (b + 1 < s_npops && i >= s_off[b + 1]) ++b;
                const uint64_t v = rnd.w[j] >> 1;
                const uint64_t *thr = s_thr + b * kPK;
                uint32_t T = 0;
                while (T < static_cast<uint32_t>(kPK) && v >= thr[T]) ++T;
                const int32_t in = static_cast<int32_t>(static_cast<uint32_t>(ww[j]) +
                                                        T * static_cast<uint32_t>(a.w_ext_fx));
                spk[j] = neuron_step(a, uu[j], cc[j], rr[j], in);
            }
        }
        *reinterpret_cast<float4 *>(a.U + i0) = make_float4(uu[0], uu[1], uu[2], uu[3]);
        *reinterpret_cast<float4 *>(a.I + i0) = make_float4(cc[0], cc[1], cc[2], cc[3]);
        *reinterpret_cast<uint32_t *>(a.R + i0) = rr[0] | (rr[1] << 8) | (rr[2] << 16) | (rr[3] << 24);
    }

    // warp-aggregated append of this step's spikers to the raster / spike queue
    const int lane = threadIdx.x & 31;
    const int cnt = spk[0] + spk[1] + spk[2] + spk[3];
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (total > 0) {
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
}

__global__ void __launch_bounds__(kDeliverThreads) k_deliver(const StepArgs a, const int k)
{
    const int64_t t = a.ctl->t_base + k;
    const uint32_t cur = a.ctl->cursor;
    const uint32_t begin = a.ctl->step_begin[t & 1];
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->step_begin[(t + 1) & 1] = cur;
    const uint32_t end = cur < a.rast_cap ? cur : a.rast_cap;
    const int64_t nspk = end > begin ? static_cast<int64_t>(end - begin) : 0;
    const int64_t items = nspk * a.chunks_per_row;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    int32_t *const ring = a.ring;
    const int64_t npad = a.npad;

    for (int64_t it = warp; it < items; it += nwarps) {
        const int64_t j = it / a.chunks_per_row;
        const int64_t c = it - j * a.chunks_per_row;
        const int32_t s = a.rast_nrn[begin + j];
        const int64_t rs = a.row_ptr[s];
        const int64_t re = a.row_ptr[s + 1];
        const int64_t off = rs + c * kChunk;
        if (off >= re) continue;
        int4 tg[2], wv[2];
        uint32_t dv[2];
        bool ok[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t o = off + u * 128 + lane * 4;
            ok[u] = o < re;
            if (ok[u]) {
                tg[u] = ld_stream4(a.syn_tgt + o);
                wv[u] = ld_stream4(a.syn_w + o);
                dv[u] = ld_stream_u32(a.syn_d + o);
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (!ok[u]) continue;
            const int32_t tt[4] = {tg[u].x, tg[u].y, tg[u].z, tg[u].w};
            const int32_t wq[4] = {wv[u].x, wv[u].y, wv[u].z, wv[u].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int64_t d = (dv[u] >> (8 * e)) & 0xFFu;
                if (wq[e] != 0) red_add_s32(ring + ((t + d) & kDMask) * npad + tt[e], wq[e]);
            }
        }
    }
}

__global__ void k_advance(Ctl *ctl, int64_t m) { ctl->t_base += m; }

}  // namespace

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

void launch_advance(Ctl *ctl, int64_t m, void *stream)
{
    k_advance<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(ctl, m);
}

}  // namespace snn
