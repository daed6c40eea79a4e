// Plain FP32 SPIIR filter kernel for sm_103a.
//
// Computes, for every (detector, template) work item, the summed single-pole
// IIR bank of the SPIIR method (section "GPU accelerated SPIIR method",
// subsection "SPIIR method"):
//     y_l[k] = a_l y_l[k-1] + b_l x[k-d_l],   z[k] = sum_l y_l[k]
// stores z (optional) and keeps the running peak max |z|^2 with its first
// index.
//
// Mapping (subsection "Optimized GPU implementation of SPIIR" describes the
// prior-art Maxwell version; this is its sm_103a redesign):
//  * strain: one shared-memory ring per CTA holds the last Dh samples (>= the
//    largest delay) plus the current and the next block of Tb samples; blocks
//    arrive by 1-D TMA bulk copies (cp.async.bulk) signalled on mbarriers,
//    double buffered.  This replaces the read-only-cache reuse of the paper.
//    The ring exists in C copies whose bank offsets differ, and the layout
//    places filters so the 32 lanes of a round read 32 different banks;
//  * state in registers: lane i of warp w keeps the complex outputs of its F
//    filters across the whole call, as the paper keeps each filter's output
//    in a register.  F is capped (the kernel is compiled per cap, with launch
//    bounds that follow its register need); a template with more filters
//    than 32*cap spans several warps of the CTA (the paper maps such a
//    template to a block);
//  * the recurrence runs two filters per packed FP32x2 instruction
//    (fma/mul/add .f32x2), 8 packed operations per filter pair and sample;
//  * the sum over filters: each lane first adds its own filters, then the
//    warp sums across lanes with a transpose-reduce over 8 samples (the
//    paper's shuffle sum, with explicit __shfl_*_sync since sm_70 warps are
//    not implicitly synchronous).  Odd lanes hold their filters in (im, re)
//    order, so the first exchange level needs no lane-dependent select;
//  * no atomics: each warp writes its per-sample sums for the block into
//    shared memory; after the block barrier the template's first warp adds
//    its warps' sums in a fixed order, stores z with coalesced 8-byte stores
//    and keeps the running peak (the paper sums across warps with atomics,
//    which would make the peak's argmax depend on timing).
#include "spiir_k1_body.h"

namespace spiir {

namespace {

__global__ void peak_out_kernel(const float *best, const int64_t *idx, int64_t count,
                                float *out_abs, int64_t *out_idx)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float b = best[i];
    out_abs[i] = b < 0.f ? 0.f : sqrtf(b);
    out_idx[i] = idx[i];
}

// The same, for a call whose error word may be set: if a bounded wait of
// the call gave up, every entry reads (NaN, -1), so the caller sees the
// failure in its outputs without a status read-back.
__global__ void peak_out_checked_kernel(const float *best, const int64_t *idx, int64_t count,
                                        const int32_t *err, float *out_abs, int64_t *out_idx)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    if (*err != 0) {
        out_abs[i] = __int_as_float(0x7fc00000);
        out_idx[i] = -1;
        return;
    }
    const float b = best[i];
    out_abs[i] = b < 0.f ? 0.f : sqrtf(b);
    out_idx[i] = idx[i];
}

__global__ void segment_carry_kernel(const float4 *params, const float2 *state,
                                     const float2 *seg_end, float2 *seg_init, int64_t n_slots,
                                     int D, int P, int n_seg)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // det * n_slots + slot
    if (i >= (int64_t)D * n_slots) return;
    const int64_t s = i % n_slots;
    const float4 p = params[s];   // kernel form: the pole matches the stored state's form
    // a^n_seg by repeated squaring in FP64
    double br = p.x, bi = p.y, rr = 1.0, ri = 0.0;
    for (int e = n_seg; e > 0; e >>= 1) {
        if (e & 1) {
            const double nr = rr * br - ri * bi, ni = rr * bi + ri * br;
            rr = nr;
            ri = ni;
        }
        const double nr = br * br - bi * bi, ni = 2.0 * br * bi;
        br = nr;
        bi = ni;
    }
    const float2 y0 = state[i];
    seg_init[i] = y0;
    double yr = y0.x, yi = y0.y;
    for (int q = 0; q + 1 < P; ++q) {
        const float2 e = __ldg(&seg_end[(int64_t)q * D * n_slots + i]);
        const double nr = rr * yr - ri * yi + (double)e.x;
        const double ni = rr * yi + ri * yr + (double)e.y;
        yr = nr;
        yi = ni;
        seg_init[(int64_t)(q + 1) * D * n_slots + i] = make_float2((float)yr, (float)yi);
    }
}

// One warp per (detector, template) entry: lanes read segments q = lane,
// lane + 32, ..., keep their largest (earliest segment on ties), then a
// butterfly keeps the largest with the smallest segment; the plan's running
// peak wins ties (earlier samples).
__global__ void peak_merge_kernel(const float *seg_best, const int64_t *seg_idx, int P,
                                  int64_t count, float *best, int64_t *idx, int64_t *t0,
                                  int64_t advance)
{
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gt == 0 && t0 != nullptr) *t0 += advance;   // nothing here reads the counter
    const int64_t i = gt >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= count) return;                          // whole warps leave together
    float b = -2.0f;
    int q_b = P;
    for (int q = lane; q < P; q += 32) {
        const float v = seg_best[(int64_t)q * count + i];
        if (v > b) {
            b = v;
            q_b = q;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, b, o);
        const int oq = __shfl_xor_sync(0xffffffffu, q_b, o);
        if (ob > b || (ob == b && oq < q_b)) {
            b = ob;
            q_b = oq;
        }
    }
    if (lane == 0 && q_b < P && b > best[i]) {
        best[i] = b;
        idx[i] = seg_idx[(int64_t)q_b * count + i];
    }
}

__global__ void advance_kernel(int64_t *t0, int64_t n)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *t0 += n;
}

__global__ void peak_reset_kernel(float *best, int64_t *idx, int64_t count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    best[i] = -1.0f;
    idx[i] = -1;
}

__global__ void decimate_kernel(const float *x, int64_t n, int R, int64_t nb, float *xe,
                                int64_t xe_stride, int64_t Dh)
{
    const int d = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb;
         i += (int64_t)gridDim.x * blockDim.x)
        xe[(int64_t)d * xe_stride + Dh + i] = x[(int64_t)d * n + (int64_t)R * i];
}

// Front end of a band: x_b[k] = sum_{i < L} h[i] x[R k - i] for this call's
// band samples, from xt = [H samples of history | the call's x] per
// detector (xr[j] = x[t0 + j] for j >= -H, L - 1 <= H).  FP32 accumulation
// in tap order; the taps sit in shared memory.
__global__ void fir_decimate_kernel(const float *xt, int64_t xt_stride, int H, int R, int64_t nb,
                                    const float *taps, int L, float *xe, int64_t xe_stride,
                                    int64_t Dh)
{
    extern __shared__ float th[];
    for (int i = threadIdx.x; i < L; i += blockDim.x) th[i] = taps[i];
    __syncthreads();
    const int d = blockIdx.y;
    const float *xr = xt + (int64_t)d * xt_stride + H;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nb;
         k += (int64_t)gridDim.x * blockDim.x) {
        const float *c = xr + (int64_t)R * k;
        float acc = 0.f;
        for (int i = 0; i < L; ++i) acc = __fmaf_rn(th[i], c[-i], acc);
        xe[(int64_t)d * xe_stride + Dh + k] = acc;
    }
}

__global__ void bounded_wait_probe(int32_t *err, uint64_t limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_addr(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // nothing arrives on this barrier: the wait must give up by itself
    const bool ok = mbar_wait(b, 0, limit_ns);
    if (!ok && threadIdx.x == 0) atomicOr(err, 2);
}

}  // namespace

// CTAs of `k` resident on the device at once (occupancy x SMs), computed
// once per (kernel, device, shared-memory size).
cudaError_t resident_ctas(const void *k, int threads, int smem_bytes, int *out)
{
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, int, int>, int> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(k, dev, threads, smem_bytes);
    auto it = done.find(key);
    if (it != done.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    int per_sm = 0, n_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem_bytes)) !=
            cudaSuccess ||
        (e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    *out = done[key] = std::max(1, per_sm) * std::max(1, n_sm);
    return cudaSuccess;
}

cudaError_t launch_k1(const K1Args &a, int64_t n_units, int smem_bytes, cudaStream_t s)
{
    if (n_units <= 0 || a.n <= 0) return cudaSuccess;
    if (a.anchors != nullptr || a.mode == kModeCompensated || a.mode == kModeChunked)
        return launch_k1_precise(a, n_units, smem_bytes, s);
    // the smallest compiled cap that holds the layout's cap
    if (a.fcap <= 2) return launch_k1_cap_2(a, n_units, smem_bytes, s);
    if (a.fcap <= 4) return launch_k1_cap_4(a, n_units, smem_bytes, s);
    if (a.fcap <= 6) return launch_k1_cap_6(a, n_units, smem_bytes, s);
    if (a.fcap <= 8) return launch_k1_cap_8(a, n_units, smem_bytes, s);
    if (a.fcap <= 10) return launch_k1_cap_10(a, n_units, smem_bytes, s);
    return cudaErrorInvalidValue;
}

int k1_plain_regs(int fcap)
{
    const void *k = fcap <= 2   ? k1_plain_kernel_2()
                    : fcap <= 4 ? k1_plain_kernel_4()
                    : fcap <= 6 ? k1_plain_kernel_6()
                    : fcap <= 8 ? k1_plain_kernel_8()
                                : k1_plain_kernel_10();
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return fa.numRegs;
}

cudaError_t ensure_smem_limit(const void *kernel, int smem_bytes)
{
    // the attribute is set once per (kernel, device, size): later launches,
    // including those recorded during stream capture, make no attribute call
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> done;
    if (smem_bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    int &have = done[std::make_pair(kernel, dev)];
    if (have >= smem_bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e == cudaSuccess) have = smem_bytes;
    return e;
}

cudaError_t launch_peak_out(const float *best, const int64_t *idx, int64_t count,
                            float *out_abs, int64_t *out_idx, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    peak_out_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(best, idx, count, out_abs,
                                                                    out_idx);
    return cudaGetLastError();
}

cudaError_t launch_peak_out_checked(const float *best, const int64_t *idx, int64_t count,
                                   const int32_t *err, float *out_abs, int64_t *out_idx,
                                   cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    peak_out_checked_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(best, idx, count, err,
                                                                            out_abs, out_idx);
    return cudaGetLastError();
}

cudaError_t launch_segment_carry(const float4 *params, const float2 *state,
                                 const float2 *seg_end, float2 *seg_init, int64_t n_slots, int D,
                                 int P, int n_seg, cudaStream_t s)
{
    const int64_t count = (int64_t)D * n_slots;
    if (count <= 0 || P < 2) return cudaSuccess;
    // FP64 is a narrow pipe: 32-thread blocks spread the work over the SMs
    segment_carry_kernel<<<(unsigned)((count + 31) / 32), 32, 0, s>>>(
        params, state, seg_end, seg_init, n_slots, D, P, n_seg);
    return cudaGetLastError();
}

cudaError_t launch_peak_merge(const float *seg_best, const int64_t *seg_idx, int P,
                              int64_t count, float *best, int64_t *idx, int64_t *t0,
                              int64_t advance, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const int64_t threads = count * 32;
    peak_merge_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        seg_best, seg_idx, P, count, best, idx, t0, advance);
    return cudaGetLastError();
}

cudaError_t launch_advance(int64_t *t0, int64_t n, cudaStream_t s)
{
    advance_kernel<<<1, 32, 0, s>>>(t0, n);
    return cudaGetLastError();
}

cudaError_t launch_peak_reset(float *best, int64_t *idx, int64_t count, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    peak_reset_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(best, idx, count);
    return cudaGetLastError();
}

cudaError_t launch_fir_decimate(const float *xt, int64_t xt_stride, int H, int D, int R,
                               int64_t nb, const float *taps, int L, float *xe,
                               int64_t xe_stride, int64_t Dh, cudaStream_t s)
{
    if (nb <= 0 || D <= 0) return cudaSuccess;
    if (L < 1 || L - 1 > H) return cudaErrorInvalidValue;
    const int64_t blocks = std::min<int64_t>((nb + 255) / 256, 4096);
    fir_decimate_kernel<<<dim3((unsigned)blocks, (unsigned)D), 256, L * sizeof(float), s>>>(
        xt, xt_stride, H, R, nb, taps, L, xe, xe_stride, Dh);
    return cudaGetLastError();
}

cudaError_t launch_decimate(const float *x, int64_t n, int D, int R, int64_t nb, float *xe,
                            int64_t xe_stride, int64_t Dh, cudaStream_t s)
{
    if (nb <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((nb + 255) / 256, 4096);
    decimate_kernel<<<dim3((unsigned)blocks, (unsigned)D), 256, 0, s>>>(x, n, R, nb, xe,
                                                                       xe_stride, Dh);
    return cudaGetLastError();
}

cudaError_t launch_bounded_wait_probe(int32_t *err, uint64_t limit_ns, cudaStream_t s)
{
    bounded_wait_probe<<<1, 32, 0, s>>>(err, limit_ns);
    return cudaGetLastError();
}

}  // namespace spiir
