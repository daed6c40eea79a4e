// Measurement probe (not part of the filter path): the FP32 rate the filter
// kernel's inner step reaches in isolation, on data that stays in registers
// and a conflict-free shared-memory window.
//
// The step is the one the filter kernel runs per lane and 8-sample batch:
// F single-pole filters, y <- a y + b x (two filters per packed FP32x2
// instruction, an odd one in scalar FP32), summed over the lane's filters,
// then over G lanes by the 8-sample transpose-reduce with shuffles (G = 32,
// 16 or 8; G = 0: a stand-in of two adds per sample instead of the
// cross-lane sum).  No ring, no TMA, no barriers, no combine and no stores
// of z: the figure is a ceiling for the instruction mix, against which the
// filter kernel's own rate is read.
//
// extern "C" spiir_probe_step(F, G, ctas_per_sm, iters, &ms, &frac):
// F in 2..10, G in {0, 16, 32} (and G = 8 with F = 8),
// ctas_per_sm in {4, 6} (128 threads each: 16 or 24 warps per SM), iters >= 1
// batches per thread.  Returns 0,
// or -1 for an unsupported combination, or the CUDA error code.  ms is the
// CUDA-event time of the timed launch, frac the achieved 8 lane-ops per
// filter-update over 128 FP32 lanes x SMs x the device's clock rate.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr unsigned kAll = 0xffffffffu;
constexpr int kSteps = 8;

__device__ __forceinline__ uint64_t pack2(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(uint64_t v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t fmul2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t fadd2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ float ld_shared(uint32_t addr)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

// sum of 8 samples (re, im per lane; odd lanes hold (im, re)) over groups of
// G lanes; the group's 16 sums go to out[(lane / G) * 16 + ...]
template <int G>
__device__ __forceinline__ void group_sum(const float (&zr)[kSteps], const float (&zi)[kSteps],
                                          int lane, float *out)
{
    float v[kSteps];
#pragma unroll
    for (int j = 0; j < kSteps; ++j) v[j] = zr[j] + __shfl_xor_sync(kAll, zi[j], 1);
    const bool b1 = (lane & 2) != 0, b2 = (lane & 4) != 0, b3 = (lane & 8) != 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float give = b1 ? v[i] : v[i + 4], keep = b1 ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(kAll, give, 2);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float give = b2 ? v[i] : v[i + 2], keep = b2 ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(kAll, give, 4);
    }
    if (G == 8) {   // two samples per lane are left
        const int s = (b1 ? 4 : 0) + (b2 ? 2 : 0);
        out[(lane >> 3) * 16 + 2 * s + (lane & 1)] = v[0];
        out[(lane >> 3) * 16 + 2 * s + 2 + (lane & 1)] = v[1];
        return;
    }
    {
        const float give = b3 ? v[0] : v[1], keep = b3 ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(kAll, give, 8);
    }
    const int s = (b1 ? 4 : 0) + (b2 ? 2 : 0) + (b3 ? 1 : 0);
    if (G == 16) {
        out[(lane >> 4) * 16 + 2 * s + (lane & 1)] = v[0];
        return;
    }
    v[0] += __shfl_xor_sync(kAll, v[0], 16);
    if (lane < 16) out[2 * s + (lane & 1)] = v[0];
}

constexpr int kWin = 32 * 4 * 12 + 64;   // shared window (floats)

template <int F, int G, int MINB>
__global__ void __launch_bounds__(128, MINB) probe_kernel(float *out, int iters, float seed)
{
    constexpr int NP = F / 2;
    constexpr bool ODD = (F & 1) != 0;
    constexpr int NPA = NP > 0 ? NP : 1;
    __shared__ float win[kWin];
    __shared__ float sums[4][64];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < kWin; i += 128) win[i] = 0.001f * (float)(i % 97) - 0.05f;
    __syncthreads();
    uint64_t AR[NPA], AI[NPA], NAI[NPA], BR[NPA], BI[NPA], YR[NPA], YI[NPA];
    float ar1 = 0.9f, ai1 = 0.1f, br1 = 0.01f, bi1 = 0.02f, yr1 = 0.f, yi1 = 0.f;
    uint32_t ad[F];
#pragma unroll
    for (int r = 0; r < F; ++r)   // lane-consecutive words: one wavefront per load
        ad[r] = (uint32_t)__cvta_generic_to_shared(&win[lane + 32 * (r % 12)]);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const float ar = 0.95f * __cosf(0.1f * q + seed), ai = 0.95f * __sinf(0.1f * q + seed);
        AR[q] = pack2(ar, ar * 0.999f);
        AI[q] = pack2(ai, ai * 0.998f);
        NAI[q] = pack2(-ai, -ai * 0.998f);
        BR[q] = pack2(0.01f, 0.02f);
        BI[q] = pack2(0.03f, -0.01f);
        YR[q] = 0;
        YI[q] = 0;
    }
    float acc = 0.f;
    for (int it = 0; it < iters; ++it) {
        float zr[kSteps], zi[kSteps];
#pragma unroll
        for (int t = 0; t < kSteps; ++t) {
            uint64_t ZR = 0, ZI = 0;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const uint64_t X = pack2(ld_shared(ad[2 * q] + 4u * (t & 3)),
                                         ld_shared(ad[2 * q + 1] + 4u * (t & 3)));
                uint64_t TR = fmul2(BR[q], X), TI = fmul2(BI[q], X);
                TR = ffma2(AR[q], YR[q], TR);
                TI = ffma2(AI[q], YR[q], TI);
                TI = ffma2(AR[q], YI[q], TI);
                TR = ffma2(NAI[q], YI[q], TR);
                YR[q] = TR;
                YI[q] = TI;
                ZR = q == 0 ? YR[0] : fadd2(ZR, YR[q]);
                ZI = q == 0 ? YI[0] : fadd2(ZI, YI[q]);
            }
            float sr = 0.f, si = 0.f;
            if (NP > 0) {
                float lo, hi;
                unpack2(ZR, lo, hi);
                sr = lo + hi;
                unpack2(ZI, lo, hi);
                si = lo + hi;
            }
            if (ODD) {
                const float x1 = ld_shared(ad[F - 1] + 4u * (t & 3));
                const float nr = fmaf(ar1, yr1, fmaf(-ai1, yi1, br1 * x1));
                const float ni = fmaf(ar1, yi1, fmaf(ai1, yr1, bi1 * x1));
                yr1 = nr;
                yi1 = ni;
                sr = NP > 0 ? sr + yr1 : yr1;
                si = NP > 0 ? si + yi1 : yi1;
            }
            zr[t] = sr;
            zi[t] = si;
        }
        if (G > 0) {
            group_sum<(G > 0 ? G : 32)>(zr, zi, lane, sums[warp]);
        } else {
#pragma unroll
            for (int t = 0; t < kSteps; ++t) acc += zr[t] + zi[t];
        }
    }
    __syncwarp();
    if (G > 0) acc += sums[warp][lane];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        float lo, hi;
        unpack2(YR[q], lo, hi);
        acc += lo + hi;
    }
    out[blockIdx.x * 128 + tid] = acc + yr1;   // keeps the work observable
}

template <int F, int G, int MINB> int run(int iters, double *ms_out, double *frac_out)
{
    int dev = 0, n_sm = 0, clk_khz = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev)) != cudaSuccess)
        return (int)e;
    const int grid = n_sm * MINB;
    float *out = nullptr;
    if ((e = cudaMalloc(&out, sizeof(float) * (size_t)grid * 128)) != cudaSuccess) return (int)e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    if ((e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess) {
        probe_kernel<F, G, MINB><<<grid, 128>>>(out, 16, 0.001f);   // warm-up
        cudaEventRecord(e0);
        probe_kernel<F, G, MINB><<<grid, 128>>>(out, iters, 0.001f);
        cudaEventRecord(e1);
        if ((e = cudaEventSynchronize(e1)) == cudaSuccess &&
            (e = cudaGetLastError()) == cudaSuccess)
            e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return (int)e;
    const double lane_ops = 8.0 * F * kSteps * (double)iters * grid * 128.0;
    const double peak = 128.0 * n_sm * clk_khz * 1e3;
    *ms_out = ms;
    *frac_out = lane_ops / (ms * 1e-3) / peak;
    return 0;
}

template <int F, int G> int run_b(int ctas, int iters, double *ms, double *frac)
{
    if (ctas == 4) return run<F, G, 4>(iters, ms, frac);
    if (ctas == 6) return run<F, G, 6>(iters, ms, frac);
    return -1;
}

template <int F> int run_f(int G, int ctas, int iters, double *ms, double *frac)
{
    if (G == 0) return run_b<F, 0>(ctas, iters, ms, frac);
    if (G == 16) return run_b<F, 16>(ctas, iters, ms, frac);
    if (G == 32) return run_b<F, 32>(ctas, iters, ms, frac);
    return -1;
}

}  // namespace

extern "C" int spiir_probe_step(int F, int G, int ctas_per_sm, int iters, double *ms, double *frac)
{
    if (iters < 1 || ms == nullptr || frac == nullptr) return -1;
    if (G == 8) return F == 8 ? run_b<8, 8>(ctas_per_sm, iters, ms, frac) : -1;
    switch (F) {
    case 2: return run_f<2>(G, ctas_per_sm, iters, ms, frac);
    case 3: return run_f<3>(G, ctas_per_sm, iters, ms, frac);
    case 4: return run_f<4>(G, ctas_per_sm, iters, ms, frac);
    case 5: return run_f<5>(G, ctas_per_sm, iters, ms, frac);
    case 6: return run_f<6>(G, ctas_per_sm, iters, ms, frac);
    case 7: return run_f<7>(G, ctas_per_sm, iters, ms, frac);
    case 8: return run_f<8>(G, ctas_per_sm, iters, ms, frac);
    case 9: return run_f<9>(G, ctas_per_sm, iters, ms, frac);
    case 10: return run_f<10>(G, ctas_per_sm, iters, ms, frac);
    default: return -1;
    }
}
