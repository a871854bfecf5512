// snn_step_static: one simulation step that allocates no device memory at all.
//
// Who needs this: programs that embed the simulator but may not call cudaMalloc
// themselves -- for example a host application whose own allocator owns every byte
// of device memory and forbids plug-ins from allocating, or a closed-loop control
// loop that cannot risk an allocation failing or stalling in the middle of a run.
// They pass every input and output buffer in; the only working memory the step
// needs beyond those -- the list of this step's spiking neurons that the delivery
// phase walks, and its counter -- lives in one fixed array compiled into this
// library (g_static_scratch below).  Every GPU that loads the library holds that
// array (about 512 KB) until the process exits.
//
// The step computed is the same as one step of snn_step_n (Poisson drive, LIF update,
// ring read/clear, push delivery into the 64-row ring), bit for bit; the spikes of the
// step are written to the caller's array in unspecified order.
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/snn.h"
#include "philox.cuh"

namespace snn {
void set_last_error(const char *msg);  // defined with snn_last_error in abi.cu
}

namespace {

constexpr int kStaticCtlWords = 64;  // word 0: spike counter of the current call
constexpr int kRingMask = SNN_D_MAX - 1;
constexpr int kQuadThreads = 128;
constexpr int kDeliverWarpsThreads = 256;
constexpr int kSynChunk = 256;

// The fixed working memory: kStaticCtlWords control words, then one queue entry per
// neuron (every neuron spikes at most once per step).
__device__ __align__(256) uint32_t g_static_scratch[kStaticCtlWords + SNN_STATIC_MAX_NEURONS];

struct StaticArgs {
    const int64_t *row_ptr;
    const int32_t *syn_tgt;
    const int32_t *syn_w;
    const uint8_t *syn_d;
    float *U;
    float *I;
    uint8_t *R;
    int32_t *ring;
    int64_t stride;
    int64_t n;
    int32_t *spikes_out;
    int32_t *n_spikes_out;
    uint32_t *scratch;  // device address of g_static_scratch
    uint64_t seed;
    int64_t t;
    float p11, p21, p22, theta, u_reset;
    int32_t t_ref, w_ext_fx, chunks_per_row, n_pops;
    int64_t pop_off[SNN_MAX_POPS + 1];
    uint64_t thr[SNN_MAX_POPS][SNN_POISSON_KMAX];
};

__global__ void __launch_bounds__(kQuadThreads) k_static_update(const StaticArgs a)
{
    __shared__ uint64_t s_thr[SNN_MAX_POPS * SNN_POISSON_KMAX];
    for (int j = threadIdx.x; j < SNN_MAX_POPS * SNN_POISSON_KMAX; j += blockDim.x)
        s_thr[j] = (&a.thr[0][0])[j];
    __syncthreads();

    const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t i0 = q * 4;
    const int64_t slot = a.t & kRingMask;
    int32_t spk[4] = {0, 0, 0, 0};
    if (i0 < a.n) {
        const float4 u4 = *reinterpret_cast<const float4 *>(a.U + i0);
        const float4 c4 = *reinterpret_cast<const float4 *>(a.I + i0);
        const uint32_t r4 = *reinterpret_cast<const uint32_t *>(a.R + i0);
        int32_t *wrow = a.ring + slot * a.stride + i0;
        const int4 w4 = *reinterpret_cast<const int4 *>(wrow);
        *reinterpret_cast<int4 *>(wrow) = make_int4(0, 0, 0, 0);
        const snn::Block4 rnd =
            snn::philox4x64_10(static_cast<uint64_t>(a.t), static_cast<uint64_t>(q), 0, 0, a.seed, snn::kStreamThalamic);
        float uu[4] = {u4.x, u4.y, u4.z, u4.w};
        float cc[4] = {c4.x, c4.y, c4.z, c4.w};
        const int32_t ww[4] = {w4.x, w4.y, w4.z, w4.w};
        uint32_t rr[4] = {r4 & 0xFFu, (r4 >> 8) & 0xFFu, (r4 >> 16) & 0xFFu, r4 >> 24};
        int b = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t i = i0 + j;
            if (i >= a.n) continue;
            while (b + 1 < a.n_pops && i >= a.pop_off[b + 1]) ++b;
            const uint64_t v = rnd.w[j] >> 1;
            uint32_t T = 0;
            while (T < static_cast<uint32_t>(SNN_POISSON_KMAX) && v >= s_thr[b * SNN_POISSON_KMAX + T]) ++T;
            const int32_t in =
                static_cast<int32_t>(static_cast<uint32_t>(ww[j]) + T * static_cast<uint32_t>(a.w_ext_fx));
            float u = uu[j], cur = cc[j];
            uint32_t r = rr[j];
            if (r == 0u) {
                float x = __fadd_rn(__fmul_rn(a.p22, u), __fmul_rn(a.p21, cur));
                if (x >= a.theta) {
                    spk[j] = 1;
                    x = a.u_reset;
                    r = static_cast<uint32_t>(a.t_ref);
                }
                u = x;
            } else {
                u = a.u_reset;
                r -= 1u;
            }
            cur = __fadd_rn(__fmul_rn(a.p11, cur), __fmul_rn(__int2float_rn(in), 0x1p-12f));
            uu[j] = u;
            cc[j] = cur;
            rr[j] = r;
        }
        *reinterpret_cast<float4 *>(a.U + i0) = make_float4(uu[0], uu[1], uu[2], uu[3]);
        *reinterpret_cast<float4 *>(a.I + i0) = make_float4(cc[0], cc[1], cc[2], cc[3]);
        *reinterpret_cast<uint32_t *>(a.R + i0) = rr[0] | (rr[1] << 8) | (rr[2] << 16) | (rr[3] << 24);
    }
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
        if (lane == 31) base = atomicAdd(&a.scratch[0], static_cast<uint32_t>(total));
        base = __shfl_sync(0xFFFFFFFFu, base, 31);
        uint32_t pos = base + static_cast<uint32_t>(incl - cnt);
        uint32_t *queue = a.scratch + kStaticCtlWords;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (spk[j]) {
                queue[pos] = static_cast<uint32_t>(i0 + j);  // pos < n <= SNN_STATIC_MAX_NEURONS
                a.spikes_out[pos] = static_cast<int32_t>(i0 + j);
                ++pos;
            }
        }
    }
}

__global__ void __launch_bounds__(kDeliverWarpsThreads) k_static_deliver(const StaticArgs a)
{
    const uint32_t nspk = a.scratch[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.n_spikes_out = static_cast<int32_t>(nspk);
    const uint32_t *queue = a.scratch + kStaticCtlWords;
    const int64_t items = static_cast<int64_t>(nspk) * a.chunks_per_row;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t it = warp; it < items; it += nwarps) {
        const int64_t j = it / a.chunks_per_row;
        const int64_t c = it - j * a.chunks_per_row;
        const uint32_t s = queue[j];
        const int64_t rs = a.row_ptr[s];
        const int64_t re = a.row_ptr[s + 1];
        const int64_t off = rs + c * kSynChunk;
        if (off >= re) continue;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t o = off + u * 128 + lane * 4;
            if (o >= re) continue;
            const int4 tg = __ldcs(reinterpret_cast<const int4 *>(a.syn_tgt + o));
            const int4 wv = __ldcs(reinterpret_cast<const int4 *>(a.syn_w + o));
            const uint32_t dv = __ldcs(reinterpret_cast<const unsigned int *>(a.syn_d + o));
            const int32_t tt[4] = {tg.x, tg.y, tg.z, tg.w};
            const int32_t wq[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int64_t d = (dv >> (8 * e)) & 0xFFu;
                if (wq[e] != 0) atomicAdd(a.ring + ((a.t + d) & kRingMask) * a.stride + tt[e], wq[e]);
            }
        }
    }
}

int static_fail(int code, const char *msg)
{
    snn::set_last_error(msg);
    return code;
}

// Device address of g_static_scratch on the current device.  In host code the array's
// name stands for a host-side shadow, not a device address, so the address is looked up
// here, with the device current, on every call: the lookup is cheap once the library's
// device code is loaded, and a fresh address cannot go stale when the caller resets the
// device between calls.
int scratch_address(uint32_t **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return static_fail(SNN_ECUDA, "cudaGetSymbolAddress(g_static_scratch) failed");
    *out = static_cast<uint32_t *>(p);
    return SNN_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" int snn_step_static(const snn_net *net, const snn_static_io *io, uint64_t seed, int64_t t,
                               void *cuda_stream)
{
    if (!net || !io) return static_fail(SNN_EINVAL, "snn_step_static: null argument");
    if (t < 0) return static_fail(SNN_EINVAL, "snn_step_static: negative step index");
    snn_info info;
    if (snn_get_info(net, &info) != SNN_OK) return static_fail(SNN_EINVAL, "snn_step_static: bad network handle");
    if (info.device_error != 0)
        return static_fail(SNN_ESTATE, "snn_step_static: a device error of this network is pending");
    if (info.n_neurons < 1) return static_fail(SNN_EINVAL, "snn_step_static: network without neurons");
    if (info.record_format != SNN_RECORD_PLAIN9)
        return static_fail(SNN_ENOTSUP, "snn_step_static: only plain synapse records are supported");
    if (info.n_circuits != 1) return static_fail(SNN_ENOTSUP, "snn_step_static: batched networks are not supported");
    if (info.engine == SNN_ENGINE_RESIDENT)
        return static_fail(SNN_ENOTSUP, "snn_step_static: the resident engine's records are block-major, not rows");
    if (info.n_neurons > SNN_STATIC_MAX_NEURONS)
        return static_fail(SNN_EINVAL,
                           "snn_step_static: network has more neurons than the static scratch holds "
                           "(SNN_STATIC_MAX_NEURONS = 131072)");
    if (!io->row_ptr || !io->U || !io->I || !io->R || !io->ring || !io->spikes || !io->n_spikes ||
        (info.n_synapses_padded > 0 && (!io->syn_tgt || !io->syn_w || !io->syn_delay)))
        return static_fail(SNN_EINVAL, "snn_step_static: missing buffer");
    if (!aligned16(io->U) || !aligned16(io->I) || !aligned16(io->ring) || (reinterpret_cast<uintptr_t>(io->R) & 3u) ||
        (info.n_synapses_padded > 0 && (!aligned16(io->syn_tgt) || !aligned16(io->syn_w) ||
                                         (reinterpret_cast<uintptr_t>(io->syn_delay) & 3u))))
        return static_fail(SNN_EINVAL, "snn_step_static: buffers must be 16-byte aligned (R and syn_delay 4-byte)");
    if (io->ring_stride < ((info.n_neurons + 3) / 4) * 4 || io->ring_stride % 4 != 0)
        return static_fail(SNN_EINVAL, "snn_step_static: ring_stride must be a multiple of 4 and cover every neuron");

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return static_fail(SNN_ECUDA, "cudaGetDevice failed");
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, io->U) != cudaSuccess || attr.type != cudaMemoryTypeDevice)
        return static_fail(SNN_EINVAL, "snn_step_static: U is not device memory");
    const int dev = attr.device;
    if (dev != prev && cudaSetDevice(dev) != cudaSuccess) return static_fail(SNN_ECUDA, "cudaSetDevice failed");

    StaticArgs a;
    std::memset(&a, 0, sizeof(a));
    uint32_t *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc == SNN_OK && cudaPeekAtLastError() != cudaSuccess)
        rc = static_fail(SNN_ECUDA, "snn_step_static: a CUDA error from earlier work is pending (not cleared)");
    if (rc == SNN_OK) {
        a.row_ptr = io->row_ptr;
        a.syn_tgt = io->syn_tgt;
        a.syn_w = io->syn_w;
        a.syn_d = io->syn_delay;
        a.U = io->U;
        a.I = io->I;
        a.R = io->R;
        a.ring = io->ring;
        a.stride = io->ring_stride;
        a.n = info.n_neurons;
        a.spikes_out = io->spikes;
        a.n_spikes_out = io->n_spikes;
        a.scratch = scratch;
        a.seed = seed;
        a.t = t;
        a.p11 = info.p11_f32;
        a.p21 = info.p21_f32;
        a.p22 = info.p22_f32;
        a.theta = info.theta_f32;
        a.u_reset = info.u_reset_f32;
        a.t_ref = info.t_ref_steps;
        a.w_ext_fx = info.w_ext_fx;
        a.chunks_per_row = info.chunks_per_row;
        a.n_pops = info.n_pops;
        std::memcpy(a.pop_off, info.pop_offsets, sizeof(a.pop_off));
        std::memcpy(a.thr, info.poisson_thresholds, sizeof(a.thr));
        cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        // the counter keeps the previous call's value: clear it first
        cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(uint32_t) * kStaticCtlWords, st);
        const int64_t quads = (info.n_neurons + 3) / 4;
        const int ugrid = static_cast<int>((quads + kQuadThreads - 1) / kQuadThreads);
        if (e != cudaSuccess) {
            rc = static_fail(SNN_ECUDA, "snn_step_static: clearing the spike counter failed");
        } else {
            k_static_update<<<ugrid, kQuadThreads, 0, st>>>(a);
            e = cudaGetLastError();
            if (e == cudaSuccess) {
                k_static_deliver<<<info.deliver_blocks > 0 ? info.deliver_blocks : 1, kDeliverWarpsThreads, 0, st>>>(a);
                e = cudaGetLastError();
            }
            if (e != cudaSuccess) rc = static_fail(SNN_ECUDA, "snn_step_static: launch failed");
        }
    }
    if (dev != prev) cudaSetDevice(prev);
    return rc;
}
