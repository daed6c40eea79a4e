// Chi^2 signal-based veto at each template's peak.
//
// Allen's discriminator splits a template into p bins of equal expected SNR
// and compares each bin's SNR with its share of the total,
//     chi^2 = p sum_i |z_i - z / p|^2,   z = sum_i z_i,
// small for a signal that matches the template and large for a glitch that
// loads a few bins.  For a bank of single-pole filters the bins are groups
// of a template's filters (contiguous in frequency, equal impulse-response
// energy); filtering each group as its own template gives the partial
// series z_i, laid out [D][T][p][n] by spiir_filter on the regrouped bank.
// This pass takes, per (detector, template), z = sum_i z_i (float32, group
// order), the first t maximising |z|^2 (re*re + im*im, separately rounded)
// and chi^2 there.  One CTA per (detector, template) streams its p rows
// once: bound by HBM bandwidth.
#include "spiir_kernels.h"

#include <climits>
#include <cmath>
#include <cstdint>

namespace spiir {

namespace {

constexpr int kVetoThreads = 256;

__device__ __forceinline__ bool vbetter(float v, int64_t i, float bv, int64_t bi)
{
    return v > bv || (v == bv && i < bi);
}

__global__ void __launch_bounds__(kVetoThreads) chi2_peak_kernel(const float2 *zg, int64_t T,
                                                                 int p, int64_t n, float *peak,
                                                                 int64_t *tout, float *chi2)
{
    __shared__ float sv[kVetoThreads / 32];
    __shared__ int64_t si[kVetoThreads / 32];
    const int64_t row = blockIdx.x;                 // detector * T + template
    const float2 *base = zg + row * p * n;          // p consecutive rows of n samples
    float best = -INFINITY;
    int64_t best_t = 0;
    for (int64_t t = threadIdx.x; t < n; t += kVetoThreads) {
        float zr = 0.f, zi = 0.f;
        for (int i = 0; i < p; ++i) {
            const float2 v = base[(int64_t)i * n + t];
            zr = __fadd_rn(zr, v.x);
            zi = __fadd_rn(zi, v.y);
        }
        const float m2 = __fadd_rn(__fmul_rn(zr, zr), __fmul_rn(zi, zi));
        if (m2 > best) {   // a thread's t increase
            best = m2;
            best_t = t;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_down_sync(0xffffffffu, best, o);
        const int64_t oi = __shfl_down_sync(0xffffffffu, best_t, o);
        if (vbetter(ov, oi, best, best_t)) {
            best = ov;
            best_t = oi;
        }
    }
    if (lane == 0) {
        sv[warp] = best;
        si[warp] = best_t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kVetoThreads / 32; ++w)
            if (vbetter(sv[w], si[w], sv[0], si[0])) {
                sv[0] = sv[w];
                si[0] = si[w];
            }
        const int64_t ts = si[0];
        float zr = 0.f, zi = 0.f;
        for (int i = 0; i < p; ++i) {
            const float2 v = base[(int64_t)i * n + ts];
            zr = __fadd_rn(zr, v.x);
            zi = __fadd_rn(zi, v.y);
        }
        const float sr = zr / (float)p, sI = zi / (float)p;
        float c = 0.f;
        for (int i = 0; i < p; ++i) {
            const float2 v = base[(int64_t)i * n + ts];
            const float dr = v.x - sr, di = v.y - sI;
            c += dr * dr + di * di;
        }
        peak[row] = __fsqrt_rn(sv[0]);
        tout[row] = ts;
        chi2[row] = (float)p * c;
    }
}

}  // namespace

cudaError_t launch_chi2_peak(const float2 *zg, int D, int64_t T, int p, int64_t n, float *peak,
                             int64_t *t, float *chi2, cudaStream_t s)
{
    if (D <= 0 || T <= 0 || n <= 0) return cudaSuccess;
    if (p < 1 || (int64_t)D * T > INT32_MAX) return cudaErrorInvalidValue;
    chi2_peak_kernel<<<(unsigned)((int64_t)D * T), kVetoThreads, 0, s>>>(zg, T, p, n, peak, t,
                                                                        chi2);
    return cudaGetLastError();
}

}  // namespace spiir
